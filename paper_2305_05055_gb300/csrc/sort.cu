// Batch sort (Sec. 4: "an unsorted batch can be converted into a sorted batch
// in O(k log k) work") as an LSD radix sort over 8-bit digits, plus the
// adjacent-repeat compaction used by the constructor.
//
// Digit passes whose 8 bits are equal across the whole batch are skipped: an
// OR/AND reduction of the keys gives the varying bits first (40-bit uniform
// keys need 5 passes, not 8).  Each pass is histogram -> scan of the
// digit-major histogram -> scatter.  The scatter ranks a 4096-key tile
// stably in shared memory (warp match_any per digit, then per-warp prefixes)
// and writes every digit's run of the tile contiguously, so global stores are
// coalesced.  Batches of at most one tile are sorted by a single block with no
// host round trip.
#include <algorithm>

#include "dev_common.cuh"
#include "internal.h"

using namespace cpmadev;

namespace cpmaimpl {
namespace {

constexpr int kT = 256;
constexpr int kWarps = kT / 32;
constexpr int kItems = 16;
constexpr int kTile = kT * kItems;  // 4096 keys

template <bool VALS>
struct TileSmemT {
  uint64_t keys[kTile];
  uint32_t vals[VALS ? kTile : 1];  // optional 32-bit payload moved with the keys
  uint32_t wcnt[kWarps][256];
  uint32_t dstart[256];
  uint64_t goff[256];
  uint32_t scan_tmp[kWarps];
};

// Stable partition of the tile by digit (key >> shift) & 255.  Item j of lane
// l in warp w is tile element w*32*kItems + j*32 + l; the first `nvalid`
// elements are real.  On return sm.keys[0..nvalid) holds the tile sorted by
// digit (stable) and sm.dstart[d] is where digit d starts.
template <bool VALS>
__device__ __forceinline__ void tile_rank(const uint64_t (&key)[kItems], const uint32_t (&val)[kItems],
                                          uint32_t nvalid, int shift, TileSmemT<VALS>& sm) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * 256; i += kT) (&sm.wcnt[0][0])[i] = 0;
  __syncthreads();
  uint32_t rank[kItems];
#pragma unroll
  for (int j = 0; j < kItems; j++) {
    const uint32_t li = warp * 32 * kItems + j * 32 + lane;
    const bool valid = li < nvalid;
    const uint32_t d = (uint32_t)(key[j] >> shift) & 255u;
    const unsigned vm = __ballot_sync(FULL, valid);
    unsigned peers = 0, before = 0;
    if (valid) {
      peers = __match_any_sync(vm, d);
      before = __popc(peers & lanemask_lt());
      rank[j] = sm.wcnt[warp][d] + before;
    }
    __syncwarp();
    if (valid && before == 0) sm.wcnt[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, then over digits
  {
    const int d = threadIdx.x;  // kT == 256 digits
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; w++) {
      uint32_t c = sm.wcnt[w][d];
      sm.wcnt[w][d] = run;
      run += c;
    }
    uint32_t inc = warp_incl_scan(run);
    if (lane == 31) sm.scan_tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      uint32_t v = lane < kWarps ? sm.scan_tmp[lane] : 0;
      uint32_t vi = warp_incl_scan(v);
      if (lane < kWarps) sm.scan_tmp[lane] = vi - v;
    }
    __syncthreads();
    sm.dstart[d] = sm.scan_tmp[warp] + inc - run;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kItems; j++) {
    const uint32_t li = warp * 32 * kItems + j * 32 + lane;
    if (li < nvalid) {
      const uint32_t d = (uint32_t)(key[j] >> shift) & 255u;
      const uint32_t pos = sm.dstart[d] + sm.wcnt[warp][d] + rank[j];
      sm.keys[pos] = key[j];
      if constexpr (VALS) sm.vals[pos] = val[j];
    }
  }
  __syncthreads();
}

__global__ void k_mask_init(Status* st) {
  st->mask_or = 0;
  st->mask_and = ~0ull;
}

__global__ void __launch_bounds__(kT) k_mask(const uint64_t* __restrict__ in, uint64_t k,
                                             Status* st) {
  ull o = 0, a = ~0ull;
  for (uint64_t i = (uint64_t)blockIdx.x * kT + threadIdx.x; i < k; i += (uint64_t)gridDim.x * kT) {
    const uint64_t x = in[i];
    o |= x;
    a &= x;
  }
#pragma unroll
  for (int s = 16; s; s >>= 1) {
    o |= __shfl_xor_sync(FULL, o, s);
    a &= __shfl_xor_sync(FULL, a, s);
  }
  if (lane_id() == 0) {
    atomicOr(&st->mask_or, o);
    atomicAnd(&st->mask_and, a);
  }
}

__global__ void __launch_bounds__(kT) k_hist(const uint64_t* __restrict__ in, uint64_t k,
                                             int shift, uint32_t* __restrict__ hist,
                                             uint32_t ntiles) {
  __shared__ uint32_t hs[256];
  hs[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kTile;
  for (int i = threadIdx.x; i < kTile; i += kT) {
    const uint64_t g = base + i;
    if (g < k) atomicAdd(&hs[(uint32_t)(in[g] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = hs[threadIdx.x];
}

template <bool VALS>
__global__ void __launch_bounds__(kT) k_scatter(const uint64_t* __restrict__ in,
                                                uint64_t* __restrict__ out,
                                                const uint32_t* __restrict__ vin,
                                                uint32_t* __restrict__ vout, uint64_t k, int shift,
                                                const uint64_t* __restrict__ hoff,
                                                uint32_t ntiles) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  TileSmemT<VALS>& sm = *reinterpret_cast<TileSmemT<VALS>*>(smem_raw);
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const uint64_t base = (uint64_t)blockIdx.x * kTile;
  const uint32_t nvalid = (uint32_t)min((uint64_t)kTile, k - base);
  sm.goff[threadIdx.x] = hoff[(uint64_t)threadIdx.x * ntiles + blockIdx.x];
  uint64_t key[kItems];
  uint32_t val[kItems];
#pragma unroll
  for (int j = 0; j < kItems; j++) {
    const uint32_t li = warp * 32 * kItems + j * 32 + lane;
    key[j] = li < nvalid ? in[base + li] : 0ull;
    if constexpr (VALS) val[j] = li < nvalid ? vin[base + li] : 0u;
    else val[j] = 0u;
  }
  tile_rank<VALS>(key, val, nvalid, shift, sm);
  for (uint32_t i = threadIdx.x; i < nvalid; i += kT) {
    const uint64_t x = sm.keys[i];
    const uint32_t d = (uint32_t)(x >> shift) & 255u;
    const uint64_t o = sm.goff[d] + i - sm.dstart[d];
    out[o] = x;
    if constexpr (VALS) vout[o] = sm.vals[i];
  }
}

// Whole batch in one tile: all varying digits in one block.
template <bool VALS>
__global__ void __launch_bounds__(kT) k_sort_small(const uint64_t* __restrict__ in,
                                                   uint64_t* __restrict__ out,
                                                   const uint32_t* __restrict__ vin,
                                                   uint32_t* __restrict__ vout, uint32_t k) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  TileSmemT<VALS>& sm = *reinterpret_cast<TileSmemT<VALS>*>(smem_raw);
  __shared__ ull s_or, s_and;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) { s_or = 0; s_and = ~0ull; }
  __syncthreads();
  uint64_t key[kItems];
  uint32_t val[kItems];
  ull o = 0, a = ~0ull;
#pragma unroll
  for (int j = 0; j < kItems; j++) {
    const uint32_t li = warp * 32 * kItems + j * 32 + lane;
    key[j] = li < k ? in[li] : 0ull;
    if constexpr (VALS) val[j] = li < k ? vin[li] : 0u;
    else val[j] = 0u;
    if (li < k) { o |= key[j]; a &= key[j]; }
  }
  atomicOr(&s_or, o);
  atomicAnd(&s_and, a);
  __syncthreads();
  const ull vary = s_or ^ s_and;
  for (int p = 0; p < 8; p++) {
    if (((vary >> (8 * p)) & 255u) == 0) continue;
    tile_rank<VALS>(key, val, k, 8 * p, sm);
#pragma unroll
    for (int j = 0; j < kItems; j++) {
      const uint32_t li = warp * 32 * kItems + j * 32 + lane;
      if (li < k) {
        key[j] = sm.keys[li];
        if constexpr (VALS) val[j] = sm.vals[li];
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < kItems; j++) {
    const uint32_t li = warp * 32 * kItems + j * 32 + lane;
    if (li < k) {
      out[li] = key[j];
      if constexpr (VALS) vout[li] = val[j];
    }
  }
}

__global__ void k_unique_flags(const uint64_t* __restrict__ in, uint64_t k,
                               uint32_t* __restrict__ flags) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
       i += (uint64_t)gridDim.x * blockDim.x)
    flags[i] = (i == 0 || in[i] != in[i - 1]) ? 1u : 0u;
}

__global__ void k_unique_scatter(const uint64_t* __restrict__ in, uint64_t k,
                                 const uint32_t* __restrict__ flags,
                                 const uint64_t* __restrict__ pos, uint64_t* __restrict__ out,
                                 Status* st) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
       i += (uint64_t)gridDim.x * blockDim.x) {
    if (flags[i]) out[pos[i]] = in[i];
    if (i == k - 1) st->nunique = pos[k];
  }
}

}  // namespace

template <bool VALS>
int sort_impl(cpma* h, const uint64_t* d_in, const uint32_t* v_in, uint64_t k, const uint64_t** out,
              const uint32_t** vout, cudaStream_t st) {
  *out = d_in;
  if (vout) *vout = v_in;
  if (k <= 1) return CPMA_OK;
  CPMA_TRY(ensure(h->s.keysA, k * 8));
  uint64_t* A = (uint64_t*)h->s.keysA.p;
  uint32_t* VA = nullptr;
  if (VALS) {
    CPMA_TRY(ensure(h->s.valsA, k * 4));
    VA = (uint32_t*)h->s.valsA.p;
  }
  const size_t smem = sizeof(TileSmemT<VALS>);
  static bool attr_done = false;  // one per instantiation
  if (!attr_done) {
    CPMA_CUDA(cudaFuncSetAttribute(k_scatter<VALS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CPMA_CUDA(cudaFuncSetAttribute(k_sort_small<VALS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_done = true;
  }
  if (k <= (uint64_t)kTile) {
    prof_add_bytes(h, PH_SORT, (VALS ? 24ull : 16ull) * k);
    k_sort_small<VALS><<<1, kT, smem, st>>>(d_in, A, v_in, VA, (uint32_t)k);
    h->launches++;
    *out = A;
    if (vout) *vout = VA;
    return check_cuda(cudaGetLastError());
  }
  CPMA_TRY(ensure(h->s.keysB, k * 8));
  uint64_t* B = (uint64_t*)h->s.keysB.p;
  uint32_t* VB = nullptr;
  if (VALS) {
    CPMA_TRY(ensure(h->s.valsB, k * 4));
    VB = (uint32_t*)h->s.valsB.p;
  }
  k_mask_init<<<1, 1, 0, st>>>(h->d_status);
  const int grid = (int)std::min<uint64_t>((uint64_t)h->num_sms * 4, (k + kT - 1) / kT);
  k_mask<<<grid, kT, 0, st>>>(d_in, k, h->d_status);
  h->launches += 2;
  CPMA_CUDA(cudaGetLastError());
  CPMA_TRY(sync_status(h, st));
  const ull vary = h->h_status->mask_or ^ h->h_status->mask_and;
  const uint32_t ntiles = (uint32_t)((k + kTile - 1) / kTile);
  CPMA_TRY(ensure(h->s.hist, (size_t)256 * ntiles * 4));
  CPMA_TRY(ensure(h->s.hoff, ((size_t)256 * ntiles + 1) * 8));
  uint32_t* hist = (uint32_t*)h->s.hist.p;
  uint64_t* hoff = (uint64_t*)h->s.hoff.p;
  const uint64_t* src = d_in;
  const uint32_t* vsrc = v_in;
  uint64_t* dst = A;
  uint32_t* vdst = VA;
  prof_add_bytes(h, PH_SORT, 8ull * k);  // the OR/AND pass
  for (int p = 0; p < 8; p++) {
    if (((vary >> (8 * p)) & 255u) == 0) continue;
    // histogram reads the keys; the scatter reads and writes keys (and tags)
    prof_add_bytes(h, PH_SORT, (VALS ? 32ull : 24ull) * k);
    k_hist<<<ntiles, kT, 0, st>>>(src, k, 8 * p, hist, ntiles);
    h->launches++;
    CPMA_TRY(scan_u32_to_u64(h, hist, hoff, (uint64_t)256 * ntiles, nullptr, st));
    k_scatter<VALS><<<ntiles, kT, smem, st>>>(src, dst, vsrc, vdst, k, 8 * p, hoff, ntiles);
    h->launches++;
    CPMA_CUDA(cudaGetLastError());
    src = dst;
    vsrc = vdst;
    dst = (dst == A) ? B : A;
    vdst = (vdst == VA) ? VB : VA;
  }
  if (src == d_in) {  // every key equal
    CPMA_CUDA(cudaMemcpyAsync(A, d_in, k * 8, cudaMemcpyDeviceToDevice, st));
    if (VALS) CPMA_CUDA(cudaMemcpyAsync(VA, v_in, k * 4, cudaMemcpyDeviceToDevice, st));
    src = A;
    vsrc = VA;
  }
  *out = src;
  if (vout) *vout = vsrc;
  return CPMA_OK;
}

int sort_keys(cpma* h, const uint64_t* d_in, uint64_t k, const uint64_t** out,
              cudaStream_t st) {
  return sort_impl<false>(h, d_in, nullptr, k, out, nullptr, st);
}

int sort_pairs(cpma* h, const uint64_t* d_in, const uint32_t* v_in, uint64_t k,
               const uint64_t** out, const uint32_t** vout, cudaStream_t st) {
  return sort_impl<true>(h, d_in, v_in, k, out, vout, st);
}

int unique_keys(cpma* h, const uint64_t* in, uint64_t k, uint64_t* out, cudaStream_t st) {
  if (k == 0) {
    CPMA_CUDA(cudaMemsetAsync(&h->d_status->nunique, 0, 8, st));
    return CPMA_OK;
  }
  CPMA_TRY(ensure(h->s.leaf_of, k * 4));
  CPMA_TRY(ensure(h->s.flags_scan, (k + 1) * 8));
  uint32_t* flags = (uint32_t*)h->s.leaf_of.p;
  uint64_t* pos = (uint64_t*)h->s.flags_scan.p;
  const int grid = (int)std::min<uint64_t>((uint64_t)h->num_sms * 8, (k + 255) / 256);
  k_unique_flags<<<grid, 256, 0, st>>>(in, k, flags);
  h->launches++;
  CPMA_TRY(scan_u32_to_u64(h, flags, pos, k, nullptr, st));
  k_unique_scatter<<<grid, 256, 0, st>>>(in, k, flags, pos, out, h->d_status);
  h->launches++;
  return check_cuda(cudaGetLastError());
}

}  // namespace cpmaimpl
