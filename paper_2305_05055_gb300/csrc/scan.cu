// Exclusive prefix sums over device arrays (reduce, scan of block partials,
// rescan).  A fixed grid of 2 blocks per SM splits the input into equal
// ranges, so the element count may live in device memory: the launch is sized
// by a host upper bound and every block reads the true count.  Tiles of 2048
// elements are staged through shared memory so global loads and stores stay
// coalesced.
#include <algorithm>

#include "dev_common.cuh"
#include "internal.h"

using namespace cpmadev;

namespace cpmaimpl {
namespace {

constexpr int kT = 256;
constexpr int kItems = 8;
constexpr int kTile = kT * kItems;
constexpr uint64_t kSingleTiles = 4;  // up to 8192 elements: one block, one launch

__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t* warp_tot,
                                                    uint64_t* total) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  uint64_t inc = warp_incl_scan(v);
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < (kT / 32) ? warp_tot[lane] : 0;
    uint64_t wi = warp_incl_scan(w);
    if (lane < (kT / 32)) warp_tot[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  uint64_t r = warp_tot[warp] + inc - v;
  __syncthreads();
  return r;
}

// The kItems consecutive elements of one thread in a full tile, by vector
// loads (p is 16-byte aligned for 32- and 64-bit input, 8-byte for bytes).
__device__ __forceinline__ void load_items(const uint8_t* p, uint64_t v[kItems]) {
  const uint2 x = *reinterpret_cast<const uint2*>(p);
#pragma unroll
  for (int q = 0; q < 4; q++) {
    v[q] = (x.x >> (8 * q)) & 0xFFu;
    v[q + 4] = (x.y >> (8 * q)) & 0xFFu;
  }
}
__device__ __forceinline__ void load_items(const uint32_t* p, uint64_t v[kItems]) {
  const uint4 a = reinterpret_cast<const uint4*>(p)[0], b = reinterpret_cast<const uint4*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void load_items(const uint64_t* p, uint64_t v[kItems]) {
#pragma unroll
  for (int q = 0; q < kItems; q += 2) {
    const ulonglong2 x = reinterpret_cast<const ulonglong2*>(p)[q / 2];
    v[q] = x.x;
    v[q + 1] = x.y;
  }
}

// Blocks own whole tiles: block b scans tiles [T b / G, T (b+1) / G).
__device__ __forceinline__ void block_tiles(uint64_t n, uint64_t& t0, uint64_t& t1) {
  const uint64_t T = (n + kTile - 1) / kTile, G = gridDim.x;
  t0 = T * blockIdx.x / G;
  t1 = T * (blockIdx.x + 1) / G;
}

template <typename Tin>
__global__ void __launch_bounds__(kT) k_reduce(const Tin* __restrict__ in, uint64_t n_host,
                                               const ull* n_dev, uint64_t* partials) {
  pdl_wait();
  pdl_launch();
  const uint64_t n = n_dev ? *n_dev : n_host;
  uint64_t tb0, tb1;
  block_tiles(n, tb0, tb1);
  const bool vec = (reinterpret_cast<uintptr_t>(in) & 15) == 0;
  uint64_t s = 0;
  for (uint64_t t = tb0; t < tb1; t++) {
    const uint64_t base = t * kTile, cnt = min((uint64_t)kTile, n - base);
    if (vec && cnt == kTile) {
      uint64_t v[kItems];
      load_items(in + base + threadIdx.x * kItems, v);
#pragma unroll
      for (int q = 0; q < kItems; q++) s += v[q];
    } else {
      for (uint64_t i = threadIdx.x; i < cnt; i += kT) s += (uint64_t)in[base + i];
    }
  }
  s = warp_sum(s);
  __shared__ uint64_t ws[kT / 32];
  if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint64_t v = threadIdx.x < kT / 32 ? ws[threadIdx.x] : 0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
}

// One block: exclusive scan of G partials in place, partials[G] = total.
__global__ void __launch_bounds__(1024) k_partials(uint64_t* partials, int G) {
  pdl_wait();
  pdl_launch();
  __shared__ uint64_t wt[32];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < G; base += 1024) {
    const int i = base + threadIdx.x;
    uint64_t v = i < G ? partials[i] : 0;
    uint64_t inc = warp_incl_scan(v);
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    if (lane == 31) wt[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = wt[lane];
      uint64_t wi = warp_incl_scan(w);
      wt[lane] = wi - w;
    }
    __syncthreads();
    uint64_t ex = carry + wt[warp] + inc - v;
    if (i < G) partials[i] = ex;
    __syncthreads();
    if (threadIdx.x == 1023) carry = ex + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[G] = carry;
}

// SINGLE: the whole scan in one block (small inputs; no partials pass).
template <typename Tin, bool SINGLE = false>
__global__ void __launch_bounds__(kT) k_down(const Tin* __restrict__ in, uint64_t* __restrict__ out,
                                             uint64_t n_host, const ull* n_dev,
                                             const uint64_t* __restrict__ partials) {
  pdl_wait();
  pdl_launch();
  __shared__ uint64_t tile[kTile];
  __shared__ uint64_t warp_tot[kT / 32];
  __shared__ uint64_t tile_total;
  const uint64_t n = n_dev ? *n_dev : n_host;
  const uint64_t G = gridDim.x;
  uint64_t tb0, tb1;
  block_tiles(n, tb0, tb1);
  const bool vec = (reinterpret_cast<uintptr_t>(in) & 15) == 0;
  uint64_t carry = SINGLE ? 0 : partials[blockIdx.x];
  for (uint64_t t = tb0; t < tb1; t++) {
    const uint64_t t0 = t * kTile, cnt = min((uint64_t)kTile, n - t0);
    uint64_t v[kItems];
    if (vec && cnt == kTile) {
      load_items(in + t0 + threadIdx.x * kItems, v);
    } else {
      for (uint32_t i = threadIdx.x; i < kTile; i += kT)
        tile[i] = i < cnt ? (uint64_t)in[t0 + i] : 0;
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kItems; q++) v[q] = tile[threadIdx.x * kItems + q];
    }
    uint64_t s = 0;
#pragma unroll
    for (int q = 0; q < kItems; q++) s += v[q];
    uint64_t ex = block_excl_scan(s, warp_tot, &tile_total);
    uint64_t run = carry + ex;
#pragma unroll
    for (int q = 0; q < kItems; q++) { tile[threadIdx.x * kItems + q] = run; run += v[q]; }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < cnt; i += kT) out[t0 + i] = tile[i];
    carry += tile_total;
    __syncthreads();
  }
  if (blockIdx.x == G - 1 && threadIdx.x == 0) out[n] = SINGLE ? carry : partials[G];
}

template <typename Tin>
int scan_impl(cpma* h, const Tin* in, uint64_t* out, uint64_t n_host, const ull* n_dev,
              cudaStream_t st, Buf* partials = nullptr) {
  uint64_t tiles = (n_host + kTile - 1) / kTile;
  if (tiles <= kSingleTiles) {
    CPMA_CUDA(launch_pdl(k_down<Tin, true>, 1, kT, 0, st, in, out, n_host, n_dev, nullptr));
    h->launches++;
    return check_cuda(cudaGetLastError());
  }
  int G = (int)std::min<uint64_t>((uint64_t)2 * h->num_sms, std::max<uint64_t>(tiles, 1));
  Buf& pb = partials ? *partials : h->s.partials;
  CPMA_TRY(ensure(h, pb, (size_t)(G + 1) * 8));
  uint64_t* part = (uint64_t*)pb.p;
  // each kernel may be scheduled while the one before it finishes
  CPMA_CUDA(launch_pdl(k_reduce<Tin>, (unsigned)G, kT, 0, st, in, n_host, n_dev, part));
  CPMA_CUDA(launch_pdl(k_partials, 1, 1024, 0, st, part, G));
  CPMA_CUDA(launch_pdl(k_down<Tin>, (unsigned)G, kT, 0, st, in, out, n_host, n_dev, part));
  h->launches += 3;
  return check_cuda(cudaGetLastError());
}

}  // namespace

int scan_u32_to_u64(cpma* h, const uint32_t* in, uint64_t* out, uint64_t n_host,
                    const ull* n_dev, cudaStream_t st) {
  return scan_impl<uint32_t>(h, in, out, n_host, n_dev, st);
}
int scan_u8_to_u64(cpma* h, const uint8_t* in, uint64_t* out, uint64_t n_host,
                   const ull* n_dev, cudaStream_t st) {
  return scan_impl<uint8_t>(h, in, out, n_host, n_dev, st);
}
int scan_u64(cpma* h, const uint64_t* in, uint64_t* out, uint64_t n_host, const ull* n_dev,
             cudaStream_t st) {
  return scan_impl<uint64_t>(h, in, out, n_host, n_dev, st);
}

int scan_u64_query(cpma* h, const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t st) {
  return scan_impl<uint64_t>(h, in, out, n, nullptr, st, &h->s.partials_q);
}
int scan_u32_query(cpma* h, const uint32_t* in, uint64_t* out, uint64_t n, cudaStream_t st) {
  return scan_impl<uint32_t>(h, in, out, n, nullptr, st, &h->s.partials_q);
}

int scan_u64_given_partials(cpma* h, const uint64_t* in, uint64_t* out, uint64_t n_host,
                            uint64_t* partials, uint64_t partials_cap, cudaStream_t st) {
  uint64_t tiles = (n_host + kTile - 1) / kTile;
  if (tiles <= kSingleTiles) {
    CPMA_CUDA(launch_pdl(k_down<uint64_t, true>, 1, kT, 0, st, in, out, n_host, nullptr, nullptr));
    h->launches++;
    return check_cuda(cudaGetLastError());
  }
  int G = (int)std::min<uint64_t>((uint64_t)2 * h->num_sms, std::max<uint64_t>(tiles, 1));
  if ((uint64_t)G + 1 > partials_cap) return CPMA_EINVAL;
  CPMA_CUDA(launch_pdl(k_reduce<uint64_t>, (unsigned)G, kT, 0, st, in, n_host, nullptr, partials));
  CPMA_CUDA(launch_pdl(k_partials, 1, 1024, 0, st, partials, G));
  CPMA_CUDA(launch_pdl(k_down<uint64_t>, (unsigned)G, kT, 0, st, in, out, n_host, nullptr,
                       partials));
  h->launches += 3;
  return check_cuda(cudaGetLastError());
}

}  // namespace cpmaimpl
