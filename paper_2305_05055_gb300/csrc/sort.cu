// Batch sort (Sec. 4: "an unsorted batch can be converted into a sorted batch
// in O(k log k) work") as an LSD radix sort over 8-bit digits, plus the
// adjacent-repeat compaction used by the constructor.
//
// One sweep per digit: a first kernel builds the histograms of all eight
// digits in one read of the batch; its last block scans them and marks the
// digits that vary (40-bit uniform keys need 5 passes, not 8).  Each varying
// digit is then one scatter launch: a tile of 4096 keys is ranked stably in
// shared memory (the lanes of a warp sharing a digit found by eight ballots,
// then per-warp prefixes), its
// global offsets come from the tiles before it by decoupled look-back (each
// tile publishes its per-digit count, then its inclusive prefix), and every
// digit's run of the tile is written contiguously.  Digits that do not vary
// return at once; the passes alternate buffers so that the last one lands in
// the first scratch buffer.  No host round trip.  Batches of at most one tile
// are sorted by a single block.
//
// Batches of up to 1.25M keys go most significant bits first instead: one
// pass takes the OR and AND of the keys, which give the 8 highest bits that
// vary; one pass counts them (256 buckets); one scatter pass (the same tile
// ranking and look-back) moves the keys to their buckets, and each bucket is
// then sorted by the bits below them in one block: in shared memory when it
// holds at most 6144 keys (k / 256 on average), else (heavy repeats or skew)
// by a block-level LSD radix sort through global memory.  Three reads and
// two writes of the batch instead of six and five, with no pass that
// depends on how the keys fall.
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
// Bucket sort: one block of kBT threads, kBItems keys each, sorts a bucket of
// up to kBTile keys (spread evenly over its warps).
constexpr int kBT = 512;
constexpr int kBItems = 12;
constexpr int kBTile = kBT * kBItems;  // 6144 keys
// Batches of more than one tile and at most this many keys take the
// top-digit buckets (k / 256 keys per bucket on average, far below kBTile).
constexpr uint64_t kBucketMax = 1280ull * 1024;

template <bool VALS, int KT = kT, int ITEMS = kItems>
struct TileSmemT {
  uint64_t keys[KT * ITEMS];
  uint32_t vals[VALS ? KT * ITEMS : 1];  // optional 32-bit payload moved with the keys
  uint32_t wcnt[KT / 32][256];
  uint32_t dstart[256];
  uint32_t scan_tmp[8];
};

// Stable partition of the tile by digit (key >> shift) & 255.  Item j of lane
// l in warp w (j < ipw <= ITEMS) is tile element w*32*ipw + j*32 + l; the first `nvalid`
// elements are real.  On return sm.keys[0..nvalid) holds the tile sorted by
// digit (stable) and sm.dstart[d] is where digit d starts.
template <bool VALS, int KT = kT, int ITEMS = kItems>
__device__ __forceinline__ void tile_rank(const uint64_t (&key)[ITEMS], const uint32_t (&val)[ITEMS],
                                          uint32_t nvalid, int shift, TileSmemT<VALS, KT, ITEMS>& sm,
                                          uint32_t ipw = ITEMS) {
  constexpr int W = KT / 32;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < W * 256; i += KT) (&sm.wcnt[0][0])[i] = 0;
  __syncthreads();
  uint32_t rank[ITEMS];
#pragma unroll
  for (int j = 0; j < ITEMS; j++) {
    if ((uint32_t)j >= ipw) break;
    const uint32_t li = warp * 32 * ipw + j * 32 + lane;
    const bool valid = li < nvalid;
    const uint32_t d = (uint32_t)(key[j] >> shift) & 255u;
    const unsigned vm = __ballot_sync(FULL, valid);
    // lanes holding the same digit: one ballot per digit bit
    unsigned peers = vm, before = 0;
#pragma unroll
    for (int b = 0; b < 8; b++) {
      const bool bit = (d >> b) & 1u;
      const unsigned bb = __ballot_sync(FULL, bit);
      peers &= bit ? bb : ~bb;
    }
    if (valid) {
      before = __popc(peers & lanemask_lt());
      rank[j] = sm.wcnt[warp][d] + before;
    }
    __syncwarp();
    if (valid && before == 0) sm.wcnt[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit (threads 0..255): exclusive prefix over warps, then over digits
  {
    const int d = threadIdx.x;
    uint32_t run = 0, inc = 0;
    if (d < 256) {
#pragma unroll
      for (int w = 0; w < W; w++) {
        uint32_t c = sm.wcnt[w][d];
        sm.wcnt[w][d] = run;
        run += c;
      }
      inc = warp_incl_scan(run);
      if (lane == 31) sm.scan_tmp[warp] = inc;
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t v = lane < 8 ? sm.scan_tmp[lane] : 0;
      uint32_t vi = warp_incl_scan(v);
      if (lane < 8) sm.scan_tmp[lane] = vi - v;
    }
    __syncthreads();
    if (d < 256) sm.dstart[d] = sm.scan_tmp[warp] + inc - run;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < ITEMS; j++) {
    if ((uint32_t)j >= ipw) break;
    const uint32_t li = warp * 32 * ipw + j * 32 + lane;
    if (li < nvalid) {
      const uint32_t d = (uint32_t)(key[j] >> shift) & 255u;
      const uint32_t pos = sm.dstart[d] + sm.wcnt[warp][d] + rank[j];
      sm.keys[pos] = key[j];
      if constexpr (VALS) sm.vals[pos] = val[j];
    }
  }
  __syncthreads();
}

constexpr uint32_t kFlagA = 1u << 30;  // tile count published
constexpr uint32_t kFlagP = 2u << 30;  // inclusive prefix published
constexpr uint32_t kCountMask = (1u << 30) - 1u;
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr int kLook = 8;  // predecessors read per look-back step

// Control block of one sort, zeroed before the first kernel.
struct SortCtl {
  uint32_t hist[8][256];   // digit histograms
  uint32_t off[8][256];    // exclusive digit offsets
  uint32_t varying[8];     // digit p varies across the batch
  uint32_t rank[8];        // position of digit p among the varying ones
  uint32_t npass;          // number of varying digits
  uint32_t done_blocks;    // histogram blocks finished
  uint32_t tile_ctr[9];    // next tile id per pass (8: the top-digit scatter)
  uint32_t top;            // highest varying digit
  // bucket path: OR / AND of every key, and the bucket field they give: the
  // top 8 varying bits, bits [fshift, fshift + 8)
  ull or_all, and_all;
  uint32_t fshift;
  uint32_t done_or;        // OR/AND blocks finished
};

__device__ __forceinline__ uint32_t bucket_of(uint64_t x, uint32_t fshift) {
  return (uint32_t)(x >> fshift) & 255u;
}

// Bucket path, pass 1: OR and AND of the keys; the last block turns them into
// the bucket field (the 8 highest bits that vary; fewer when fewer vary) and
// npass (0 when every key is equal).
__global__ void __launch_bounds__(kT) k_orand(const uint64_t* __restrict__ in, uint64_t k,
                                              SortCtl* ctl) {
  __shared__ ull s_or[kWarps], s_and[kWarps];
  __shared__ bool last;
  pdl_wait();
  pdl_launch();
  ull o = 0, a = ~0ull;
  // eight keys per thread and step, loaded together
  const uint64_t stride = (uint64_t)gridDim.x * kT;
  uint64_t i = (uint64_t)blockIdx.x * kT + threadIdx.x;
  for (; i + 7 * stride < k; i += 8 * stride) {
    uint64_t x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = in[i + j * stride];
#pragma unroll
    for (int j = 0; j < 8; j++) { o |= x[j]; a &= x[j]; }
  }
  for (; i < k; i += stride) {
    const uint64_t x = in[i];
    o |= x;
    a &= x;
  }
  const uint32_t olo = __reduce_or_sync(FULL, (uint32_t)o), ohi = __reduce_or_sync(FULL, (uint32_t)(o >> 32));
  const uint32_t alo = __reduce_and_sync(FULL, (uint32_t)a), ahi = __reduce_and_sync(FULL, (uint32_t)(a >> 32));
  if (lane_id() == 0) {
    s_or[threadIdx.x >> 5] = ((ull)ohi << 32) | olo;
    s_and[threadIdx.x >> 5] = ((ull)ahi << 32) | alo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ull bo = 0, ba = ~0ull;
    for (int w = 0; w < kWarps; w++) { bo |= s_or[w]; ba &= s_and[w]; }
    atomicOr(&ctl->or_all, bo);
    atomicAnd(&ctl->and_all, ba);
    __threadfence();
    last = atomicAdd(&ctl->done_or, 1u) == gridDim.x - 1;
    if (last) {
      __threadfence();
      const ull vary = *((volatile ull*)&ctl->or_all) ^ *((volatile ull*)&ctl->and_all);
      const uint32_t hb = vary ? 64u - (uint32_t)__clzll((long long)vary) : 0u;
      ctl->fshift = hb > 8u ? hb - 8u : 0u;
      ctl->npass = vary ? 1u : 0u;
    }
  }
}

// Bucket path, pass 2: histogram of the bucket field; the last block writes
// the buckets' exclusive offsets (hist[0], off[0]).
__global__ void __launch_bounds__(kT) k_hist_field(const uint64_t* __restrict__ in, uint64_t k,
                                                   SortCtl* ctl) {
  __shared__ uint32_t hs[256];
  __shared__ bool last;
  __shared__ uint32_t wt[kWarps];
  pdl_wait();
  pdl_launch();
  hs[threadIdx.x] = 0;  // kT == 256
  __syncthreads();
  const uint32_t fs = ctl->fshift;
  const uint64_t stride = (uint64_t)gridDim.x * kT;
  uint64_t i = (uint64_t)blockIdx.x * kT + threadIdx.x;
  for (; i + 7 * stride < k; i += 8 * stride) {  // eight keys per thread and step
    uint64_t x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = in[i + j * stride];
#pragma unroll
    for (int j = 0; j < 8; j++) atomicAdd(&hs[bucket_of(x[j], fs)], 1u);
  }
  for (; i < k; i += stride) atomicAdd(&hs[bucket_of(in[i], fs)], 1u);
  __syncthreads();
  if (hs[threadIdx.x]) atomicAdd(&ctl->hist[0][threadIdx.x], hs[threadIdx.x]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&ctl->done_blocks, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const uint32_t d = threadIdx.x;
  const uint32_t v = *((volatile uint32_t*)&ctl->hist[0][d]);
  const uint32_t inc = warp_incl_scan(v);
  if (lane_id() == 31) wt[d >> 5] = inc;
  __syncthreads();
  uint32_t wbase = 0;
  for (unsigned q = 0; q < (d >> 5); q++) wbase += wt[q];
  ctl->off[0][d] = wbase + inc - v;
}

__global__ void __launch_bounds__(kT) k_hist_all(const uint64_t* __restrict__ in, uint64_t k,
                                                 SortCtl* ctl) {
  __shared__ uint32_t hs[8][256];
  __shared__ bool last;
  pdl_wait();
  pdl_launch();
  for (int i = threadIdx.x; i < 8 * 256; i += kT) (&hs[0][0])[i] = 0;
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * kT + threadIdx.x; i < k; i += (uint64_t)gridDim.x * kT) {
    const uint64_t x = in[i];
#pragma unroll
    for (int p = 0; p < 8; p++) atomicAdd(&hs[p][(uint32_t)(x >> (8 * p)) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 8 * 256; i += kT) {
    const uint32_t v = (&hs[0][0])[i];
    if (v) atomicAdd(&(&ctl->hist[0][0])[i], v);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&ctl->done_blocks, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // last block: exclusive scans, varying digits, pass ranks
  const int d = threadIdx.x;  // kT == 256
  __shared__ uint32_t wt[kWarps];
  for (int p = 0; p < 8; p++) {
    const uint32_t v = *((volatile uint32_t*)&ctl->hist[p][d]);
    const uint32_t inc = warp_incl_scan(v);
    if (lane_id() == 31) wt[threadIdx.x >> 5] = inc;
    __syncthreads();
    uint32_t wbase = 0;
    for (unsigned q = 0; q < (threadIdx.x >> 5); q++) wbase += wt[q];
    ctl->off[p][d] = wbase + inc - v;
    const int full = __syncthreads_or(v == (uint32_t)k);
    if (d == 0) ctl->varying[p] = full ? 0u : 1u;
    __syncthreads();
  }
  if (d == 0) {
    uint32_t r = 0, top = 0;
    for (int p = 0; p < 8; p++) {
      ctl->rank[p] = r;
      r += ctl->varying[p];
      if (ctl->varying[p]) top = (uint32_t)p;
    }
    ctl->npass = r;
    ctl->top = top;
  }
}

// Every key equal: no pass runs, the batch is copied to the result buffer.
__global__ void k_copy_if_no_pass(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                  const uint32_t* __restrict__ vin, uint32_t* __restrict__ vout,
                                  uint64_t k, const SortCtl* ctl) {
  pdl_wait();
  pdl_launch();
  if (ctl->npass != 0) return;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
       i += (uint64_t)gridDim.x * blockDim.x) {
    out[i] = in[i];
    if (vin) vout[i] = vin[i];
  }
}

// One digit pass.  Buffers: the input, then A and B alternately, arranged so
// that the last varying pass writes A.  With top != 0 it is instead the
// stable scatter of the input by the bucket field (the 8 highest varying
// bits) into B, the buckets k_bucket_sort finishes.  Blocks take tiles in
// order from a counter until none is left, so the grid can be smaller than
// the tile count (a pass over a digit that does not vary costs one short
// launch).
template <bool VALS>
__global__ void __launch_bounds__(kT, 3) k_onesweep(const uint64_t* __restrict__ in,
                                                 const uint32_t* __restrict__ vin,
                                                 uint64_t* __restrict__ A, uint64_t* __restrict__ B,
                                                 uint32_t* __restrict__ VA, uint32_t* __restrict__ VB,
                                                 uint64_t k, int p, int top, SortCtl* ctl,
                                                 uint32_t* __restrict__ look, Status* st,
                                                 uint32_t spin_limit, uint32_t silent) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  TileSmemT<VALS>& sm = *reinterpret_cast<TileSmemT<VALS>*>(smem_raw);
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_excl[256];
  pdl_wait();
  pdl_launch();
  const uint64_t* src;
  uint64_t* dst;
  const uint32_t* vsrc;
  uint32_t* vdst;
  uint32_t* ctr;
  int shift;
  if (top) {
    if (ctl->npass == 0) return;
    p = 0;  // the bucket field's histogram and offsets are row 0
    shift = (int)ctl->fshift;
    src = in;
    dst = B;
    vsrc = vin;
    vdst = VB;
    ctr = &ctl->tile_ctr[8];
  } else {
    if (!ctl->varying[p]) return;
    const uint32_t r = ctl->rank[p], P = ctl->npass;
    // pass r writes B when P-1-r is odd, else A (so pass P-1 writes A) and
    // reads what pass r-1 wrote
    src = (r == 0) ? in : (((P - r) & 1u) ? B : A);
    dst = ((P - 1u - r) & 1u) ? B : A;
    vsrc = (r == 0) ? vin : (((P - r) & 1u) ? VB : VA);
    vdst = ((P - 1u - r) & 1u) ? VB : VA;
    ctr = &ctl->tile_ctr[p];
    shift = 8 * p;
  }
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t ntiles = (uint32_t)((k + kTile - 1) / kTile);
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= ntiles) return;
    const uint64_t base = (uint64_t)tile * kTile;
    const uint32_t nvalid = (uint32_t)min((uint64_t)kTile, k - base);
    uint64_t key[kItems];
    uint32_t val[kItems];
#pragma unroll
    for (int j = 0; j < kItems; j++) {
      const uint32_t li = warp * 32 * kItems + j * 32 + lane;
      key[j] = li < nvalid ? src[base + li] : 0ull;
      if constexpr (VALS) val[j] = li < nvalid ? vsrc[base + li] : 0u;
      else val[j] = 0u;
    }
    tile_rank<VALS>(key, val, nvalid, shift, sm);
    // publish this tile's count per digit, then look back for the tiles before
    const int d = threadIdx.x;
    const uint32_t cnt = (d < 255 ? sm.dstart[d + 1] : nvalid) - sm.dstart[d];
    volatile uint32_t* lk = look + (size_t)tile * 256;
    const bool publish = tile != silent;  // a silent tile (tests only) never publishes
    if (tile == 0) {
      if (publish) lk[d] = kFlagP | cnt;
      s_excl[d] = 0;
    } else {
      if (publish) lk[d] = kFlagA | cnt;
      uint32_t excl = 0;
      bool done = false;
      const volatile uint32_t* lv = look;
      // kLook predecessors are read at once (their loads in flight together),
      // then taken in order until one with an inclusive prefix
      for (int64_t tp = (int64_t)tile - 1; tp >= 0 && !done; tp -= kLook) {
        uint32_t v[kLook];
#pragma unroll
        for (int i = 0; i < kLook; i++) v[i] = tp >= i ? lv[(size_t)(tp - i) * 256 + d] : 0u;
#pragma unroll
        for (int i = 0; i < kLook; i++) {
          if (done || tp < i) break;
          uint32_t spins = 0;
          while (!(v[i] & (kFlagA | kFlagP)) && spins < spin_limit) {
            v[i] = lv[(size_t)(tp - i) * 256 + d];
            spins++;
          }
          if (spins >= spin_limit) {  // a predecessor never published: give up
            atomicOr(&st->err, kErrSort);
            done = true;
            break;
          }
          excl += v[i] & kCountMask;
          if (v[i] & kFlagP) done = true;
        }
      }
      __threadfence();
      if (publish) lk[d] = kFlagP | (excl + cnt);
      s_excl[d] = excl;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nvalid; i += kT) {
      const uint64_t x = sm.keys[i];
      const uint32_t dd = (uint32_t)(x >> shift) & 255u;
      const uint64_t o = (uint64_t)ctl->off[p][dd] + s_excl[dd] + (i - sm.dstart[dd]);
      dst[o] = x;
      if constexpr (VALS) vdst[o] = sm.vals[i];
    }
    __syncthreads();  // the next tile reuses the shared arrays
  }
}

// Bucket b of the field scatter (B[off .. off + n)), sorted stably by the
// bits below the field, into the same positions of A.  A bucket of at most
// kBTile keys is sorted in shared memory, digit by digit over the digits
// that vary inside it.  A larger one (heavy repeats or skew) is sorted by a
// block-level LSD radix sort through global memory: per varying digit, one
// counting pass over the bucket, then its tiles in order, each ranked stably
// in shared memory and scattered to the running digit offsets, alternating
// between B and A (and copied to A if it ends in B).
template <bool VALS>
__global__ void __launch_bounds__(kBT, 2) k_bucket_sort(uint64_t* __restrict__ B,
                                                     uint32_t* __restrict__ VB,
                                                     uint64_t* __restrict__ A,
                                                     uint32_t* __restrict__ VA, SortCtl* ctl,
                                                     const uint64_t* __restrict__ in,
                                                     const uint32_t* __restrict__ vin,
                                                     uint64_t k) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  TileSmemT<VALS, kBT, kBItems>& sm = *reinterpret_cast<TileSmemT<VALS, kBT, kBItems>*>(smem_raw);
  __shared__ ull s_or, s_and;
  __shared__ uint32_t s_run[256];
  __shared__ uint32_t s_wt[8];
  pdl_wait();
  pdl_launch();
  if (ctl->npass == 0) {
    // every key equal: the batch as given is the result
    for (uint64_t i = (uint64_t)blockIdx.x * kBT + threadIdx.x; i < k;
         i += (uint64_t)gridDim.x * kBT) {
      A[i] = in[i];
      if constexpr (VALS) VA[i] = vin[i];
    }
    return;
  }
  const uint32_t b = blockIdx.x;
  const uint32_t n = ctl->hist[0][b];
  if (n == 0) return;
  const uint64_t base = ctl->off[0][b];
  const uint32_t npd = (ctl->fshift + 7u) / 8u;  // digits below the field
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) { s_or = 0; s_and = ~0ull; }
  __syncthreads();
  if (n <= (uint32_t)kBTile) {
    // items per warp: the bucket spread over every warp, in element order
    const uint32_t ipw = (n + 32u * (kBT / 32) - 1u) / (32u * (kBT / 32));
    uint64_t key[kBItems];
    uint32_t val[kBItems];
    ull o = 0, a = ~0ull;
#pragma unroll
    for (int j = 0; j < kBItems; j++) {
      const uint32_t li = warp * 32 * ipw + j * 32 + lane;
      const bool ok = (uint32_t)j < ipw && li < n;
      key[j] = ok ? B[base + li] : 0ull;
      if constexpr (VALS) val[j] = ok ? VB[base + li] : 0u;
      else val[j] = 0u;
      if (ok) { o |= key[j]; a &= key[j]; }
    }
    atomicOr(&s_or, o);
    atomicAnd(&s_and, a);
    __syncthreads();
    const ull vary = s_or ^ s_and;
    for (uint32_t p = 0; p < npd; p++) {
      if (((vary >> (8 * p)) & 255u) == 0) continue;
      tile_rank<VALS, kBT, kBItems>(key, val, n, 8 * (int)p, sm, ipw);
#pragma unroll
      for (int j = 0; j < kBItems; j++) {
        const uint32_t li = warp * 32 * ipw + j * 32 + lane;
        if ((uint32_t)j < ipw && li < n) {
          key[j] = sm.keys[li];
          if constexpr (VALS) val[j] = sm.vals[li];
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < kBItems; j++) {
      const uint32_t li = warp * 32 * ipw + j * 32 + lane;
      if ((uint32_t)j < ipw && li < n) {
        A[base + li] = key[j];
        if constexpr (VALS) VA[base + li] = val[j];
      }
    }
    return;
  }
  // ---- oversized bucket: block-level LSD through global memory ----
  {
    ull o = 0, a = ~0ull;
    for (uint32_t i = threadIdx.x; i < n; i += kBT) {
      const uint64_t x = B[base + i];
      o |= x;
      a &= x;
    }
    atomicOr(&s_or, o);
    atomicAnd(&s_and, a);
  }
  __syncthreads();
  const ull vary = s_or ^ s_and;
  uint64_t* src = B + base;
  uint64_t* dst = A + base;
  uint32_t* vsrc = VALS ? VB + base : nullptr;
  uint32_t* vdst = VALS ? VA + base : nullptr;
  bool in_a = false;
  for (uint32_t p = 0; p < npd; p++) {
    if (((vary >> (8 * p)) & 255u) == 0) continue;
    const int shift = 8 * (int)p;
    // counting pass, then exclusive offsets of the digits
    if (threadIdx.x < 256) s_run[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += kBT)
      atomicAdd(&s_run[(uint32_t)(src[i] >> shift) & 255u], 1u);
    __syncthreads();
    uint32_t v = 0, inc = 0;
    if (threadIdx.x < 256) {
      v = s_run[threadIdx.x];
      inc = warp_incl_scan(v);
      if (lane == 31) s_wt[warp] = inc;
    }
    __syncthreads();
    if (threadIdx.x < 256) {
      uint32_t wbase = 0;
      for (unsigned q = 0; q < warp; q++) wbase += s_wt[q];
      s_run[threadIdx.x] = wbase + inc - v;
    }
    __syncthreads();
    // the tiles in order: stable rank, scatter to the running offsets
    for (uint32_t t0 = 0; t0 < n; t0 += (uint32_t)kBTile) {
      const uint32_t nv = min((uint32_t)kBTile, n - t0);
      const uint32_t ipw = (nv + 32u * (kBT / 32) - 1u) / (32u * (kBT / 32));
      uint64_t key[kBItems];
      uint32_t val[kBItems];
#pragma unroll
      for (int j = 0; j < kBItems; j++) {
        const uint32_t li = warp * 32 * ipw + j * 32 + lane;
        const bool ok = (uint32_t)j < ipw && li < nv;
        key[j] = ok ? src[t0 + li] : 0ull;
        if constexpr (VALS) val[j] = ok ? vsrc[t0 + li] : 0u;
        else val[j] = 0u;
      }
      tile_rank<VALS, kBT, kBItems>(key, val, nv, shift, sm, ipw);
      for (uint32_t i = threadIdx.x; i < nv; i += kBT) {
        const uint64_t x = sm.keys[i];
        const uint32_t d = (uint32_t)(x >> shift) & 255u;
        const uint32_t o = s_run[d] + (i - sm.dstart[d]);
        dst[o] = x;
        if constexpr (VALS) vdst[o] = sm.vals[i];
      }
      __syncthreads();
      if (threadIdx.x < 256) {
        const uint32_t d = threadIdx.x;
        s_run[d] += (d < 255 ? sm.dstart[d + 1] : nv) - sm.dstart[d];
      }
      __syncthreads();
    }
    uint64_t* t = src; src = dst; dst = t;
    uint32_t* tv = vsrc; vsrc = vdst; vdst = tv;
    in_a = !in_a;
    __syncthreads();
  }
  if (!in_a) {
    for (uint32_t i = threadIdx.x; i < n; i += kBT) {
      A[base + i] = B[base + i];
      if constexpr (VALS) VA[base + i] = VB[base + i];
    }
  }
}

// Untagged batches of at most kTile keys: one block, a bitonic sorting
// network over the batch padded with 2^64-1 to n (a power of two) in shared
// memory, one compare-exchange of each pair per stage (equal keys are equal
// values, so order among them does not matter).
constexpr int kBitT = 1024;
__global__ void __launch_bounds__(kBitT) k_sort_bitonic(const uint64_t* __restrict__ in,
                                                        uint64_t* __restrict__ out, uint32_t k,
                                                        uint32_t n) {
  __shared__ uint64_t s[kTile];
  for (uint32_t i = threadIdx.x; i < n; i += kBitT) s[i] = i < k ? in[i] : ~0ull;
  __syncthreads();
  for (uint32_t size = 2; size <= n; size <<= 1) {
    for (uint32_t stride = size >> 1; stride; stride >>= 1) {
      for (uint32_t t = threadIdx.x; t < n / 2; t += kBitT) {
        const uint32_t i = 2 * t - (t & (stride - 1)), j = i + stride;  // pair t of this stage
        const uint64_t a = s[i], b = s[j];
        if ((a > b) == ((i & size) == 0)) {  // ascending runs where bit `size` of i is 0
          s[i] = b;
          s[j] = a;
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < k; i += kBitT) out[i] = s[i];
}

// Tagged batches of at most kTile keys: a stable rank sort spread over many
// blocks.  Every block holds the whole batch in shared memory; P consecutive
// threads share one key, each counting over a P-th of the batch the keys
// below it and the equal keys before it, and the sum of their counts (a
// shuffle reduction) is where the key (and its tag) goes.
constexpr int kRankT = 256;
template <bool VALS>
__global__ void __launch_bounds__(kRankT) k_sort_rank(const uint64_t* __restrict__ in,
                                                      uint64_t* __restrict__ out,
                                                      const uint32_t* __restrict__ vin,
                                                      uint32_t* __restrict__ vout, uint32_t k,
                                                      uint32_t P) {
  extern __shared__ __align__(16) uint64_t s_keys[];
  for (uint32_t i = threadIdx.x; i < k; i += kRankT) s_keys[i] = in[i];
  __syncthreads();
  const uint32_t g = blockIdx.x * kRankT + threadIdx.x;
  const uint32_t i = g / P, part = g % P;
  const bool valid = i < k;
  const uint64_t x = valid ? s_keys[i] : 0ull;
  const uint32_t per = (k + P - 1) / P;
  const uint32_t j0 = min(k, part * per), j1 = min(k, j0 + per);
  uint32_t r = 0;
  if (valid) {
    // equal keys count only before i: two ranges with a fixed test
    const uint32_t jm = min(max(i, j0), j1);
#pragma unroll 8
    for (uint32_t j = j0; j < jm; j++) r += s_keys[j] <= x;
#pragma unroll 8
    for (uint32_t j = jm; j < j1; j++) r += s_keys[j] < x;
  }
  for (uint32_t o = 1; o < P; o <<= 1) r += __shfl_xor_sync(FULL, r, o);
  if (valid && part == 0) {
    out[r] = x;
    if constexpr (VALS) vout[r] = vin[i];
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

namespace {
size_t ctl_bytes() { return (sizeof(SortCtl) + 255) & ~(size_t)255; }
size_t look_bytes(uint64_t k) {  // one array per digit pass (the bucket path uses one)
  const uint64_t ntiles = (k + kTile - 1) / kTile;
  return (size_t)8 * ntiles * 256 * 4;
}
template <bool VALS>
int& sweep_blocks_per_sm() {
  static int n = 1;
  return n;
}
template <bool VALS>
void sort_attrs() {
  static bool done = false;  // one per instantiation
  if (done) return;
  const int smem = (int)sizeof(TileSmemT<VALS>);
  cudaFuncSetAttribute(k_onesweep<VALS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_bucket_sort<VALS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(TileSmemT<VALS, kBT, kBItems>));
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_onesweep<VALS>, kT, smem) ==
          cudaSuccess &&
      bps > 0)
    sweep_blocks_per_sm<VALS>() = bps;
  cudaGetLastError();
  done = true;
}
}  // namespace

int sort_scratch(cpma* h, uint64_t k, bool vals) {
  sort_attrs<false>();
  if (vals) sort_attrs<true>();
  if (k <= 1) return CPMA_OK;
  CPMA_TRY(ensure(h, h->s.keysA, k * 8));
  if (vals) CPMA_TRY(ensure(h, h->s.valsA, k * 4));
  if (k <= (uint64_t)kTile) return CPMA_OK;
  CPMA_TRY(ensure(h, h->s.keysB, k * 8));
  if (vals) CPMA_TRY(ensure(h, h->s.valsB, k * 4));
  return ensure(h, h->s.hist, ctl_bytes() + look_bytes(k));
}

template <bool VALS>
int sort_impl(cpma* h, const uint64_t* d_in, const uint32_t* v_in, uint64_t k, const uint64_t** out,
              const uint32_t** vout, cudaStream_t st) {
  *out = d_in;
  if (vout) *vout = v_in;
  if (k <= 1) return CPMA_OK;
  CPMA_TRY(sort_scratch(h, k, VALS));
  uint64_t* A = (uint64_t*)h->s.keysA.p;
  uint32_t* VA = VALS ? (uint32_t*)h->s.valsA.p : nullptr;
  const size_t smem = sizeof(TileSmemT<VALS>);
  if (!VALS && k <= (uint64_t)kTile) {
    prof_add_bytes(h, PH_SORT, 16ull * k);
    uint32_t n = 2;
    while (n < k) n <<= 1;
    k_sort_bitonic<<<1, kBitT, 0, st>>>(d_in, A, (uint32_t)k, n);
    h->launches++;
    *out = A;
    return check_cuda(cudaGetLastError());
  }
  if (k <= (uint64_t)kTile) {
    prof_add_bytes(h, PH_SORT, (VALS ? 24ull : 16ull) * k);
    // threads per key: a power of two keeping each thread's share at 256 keys
    uint32_t P = 1;
    while (P < 32 && k > 256ull * P) P <<= 1;
    const uint32_t nb = (uint32_t)((k * P + kRankT - 1) / kRankT);
    k_sort_rank<VALS><<<nb, kRankT, k * 8, st>>>(d_in, A, v_in, VA, (uint32_t)k, P);
    h->launches++;
    *out = A;
    if (vout) *vout = VA;
    return check_cuda(cudaGetLastError());
  }
  uint64_t* B = (uint64_t*)h->s.keysB.p;
  uint32_t* VB = VALS ? (uint32_t*)h->s.valsB.p : nullptr;
  const uint32_t ntiles = (uint32_t)((k + kTile - 1) / kTile);
  // the look-back wait's poll limit and a tile that never publishes (tests)
  const uint32_t spin = h->sort_poll_limit ? h->sort_poll_limit : kSpinLimit;
  const uint32_t silent = h->sort_silent_tile >= 0 && h->sort_silent_tile < (int64_t)ntiles
                              ? (uint32_t)h->sort_silent_tile : 0xFFFFFFFFu;
  SortCtl* ctl = reinterpret_cast<SortCtl*>(h->s.hist.p);
  uint32_t* look = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(h->s.hist.p) + ctl_bytes());
  const int hgrid = (int)std::min<uint64_t>((uint64_t)h->num_sms * 2, (k + kT - 1) / kT);
  const unsigned sgrid = (unsigned)std::min<uint64_t>(
      ntiles, (uint64_t)h->num_sms * (uint64_t)sweep_blocks_per_sm<VALS>());
  if (k <= kBucketMax) {
    // most significant bits first: OR / AND of the keys give the 8 highest
    // bits that vary, their histogram, one scatter into 256 buckets by them,
    // then every bucket sorted by the bits below in one block.  The control
    // block and one look-back array are zeroed first (and_all starts at ~0).
    CPMA_CUDA(cudaMemsetAsync(h->s.hist.p, 0, ctl_bytes() + (size_t)ntiles * 256 * 4, st));
    CPMA_CUDA(cudaMemsetAsync(&ctl->and_all, 0xFF, sizeof(ull), st));
    // about eight keys per thread: one step of the unrolled loops
    const int ogrid = (int)std::max<uint64_t>(
        1, std::min<uint64_t>((uint64_t)h->num_sms * 8, (k + 8 * kT - 1) / (8 * kT)));
    // each kernel after the first may be scheduled while the one before it
    // finishes (programmatic dependent launch; each waits for it first)
    k_orand<<<ogrid, kT, 0, st>>>(d_in, k, ctl);
    CPMA_CUDA(launch_pdl(k_hist_field, ogrid, kT, 0, st, d_in, k, ctl));
    CPMA_CUDA(launch_pdl(k_onesweep<VALS>, sgrid, kT, smem, st, d_in, v_in, A, B, VA, VB, k, 0, 1,
                         ctl, look, h->d_status, spin, silent));
    CPMA_CUDA(launch_pdl(k_bucket_sort<VALS>, 256, kBT, sizeof(TileSmemT<VALS, kBT, kBItems>), st,
                         B, VB, A, VA, ctl, d_in, v_in, k));
    h->launches += 4;
    // OR/AND and histogram reads, scatter and bucket read + write
    prof_add_bytes(h, PH_SORT, 16ull * k + (VALS ? 24ull : 16ull) * k * 2);
  } else {
    // least significant digit first over the digits that vary
    CPMA_CUDA(cudaMemsetAsync(h->s.hist.p, 0, ctl_bytes() + look_bytes(k), st));
    k_hist_all<<<hgrid, kT, 0, st>>>(d_in, k, ctl);
    h->launches++;
    prof_add_bytes(h, PH_SORT, 8ull * k);  // the histogram read
    for (int p = 0; p < 8; p++) {
      // digits that vary: the scatter reads and writes keys (and tags)
      CPMA_CUDA(launch_pdl(k_onesweep<VALS>, sgrid, kT, smem, st, d_in, v_in, A, B, VA, VB, k, p,
                           0, ctl, look + (size_t)p * ntiles * 256, h->d_status, spin, silent));
      h->launches++;
    }
    prof_add_bytes(h, PH_SORT, (VALS ? 24ull : 16ull) * k * 5);  // typical: 5 varying digits
    CPMA_CUDA(launch_pdl(k_copy_if_no_pass,
                         (unsigned)std::min<uint64_t>((uint64_t)h->num_sms * 4, (k + kT - 1) / kT),
                         kT, 0, st, d_in, A, v_in, VA, k, ctl));
    h->launches++;
  }
  CPMA_CUDA(cudaGetLastError());
  const uint64_t* src = A;
  const uint32_t* vsrc = VA;
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
  CPMA_TRY(ensure(h, h->s.leaf_of, k * 4));
  CPMA_TRY(ensure(h, h->s.flags_scan, (k + 1) * 8));
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
