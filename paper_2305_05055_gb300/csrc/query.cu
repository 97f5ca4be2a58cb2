// Queries over the compressed leaves.
//  has (Sec. 5 "Point queries"): binary search on the uncompressed heads, then
//    one warp-cooperative pass over the leaf.
//  range_map (Sec. 3: a search for the first element, then a scan to the end
//    of the range) with f = (sum mod 2^64, count): every query is routed to
//    its first and last leaf; the (query, leaf) pairs of all queries are
//    numbered by a prefix sum and split into equal contiguous shares, one per
//    warp of a persistent grid, so long and short ranges balance.  Leaves
//    strictly inside a range need no filter.  A warp keeps per-lane partial
//    sums while it stays on one query and adds them atomically when it
//    leaves it (addition mod 2^64 is associative, so the order is free).
//  sum (App. A sum()): every leaf once.
#include <algorithm>
#include <mutex>

#include "dev_common.cuh"
#include "internal.h"

using namespace cpmadev;

namespace cpmaimpl {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ uint64_t gtid() {
  return (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ uint64_t gstride() { return (uint64_t)gridDim.x * blockDim.x; }

__global__ void __launch_bounds__(kT) k_has(const uint64_t* __restrict__ keys, uint64_t q,
                                            const uint8_t* __restrict__ data,
                                            const uint32_t* __restrict__ used,
                                            const uint64_t* __restrict__ heads, uint64_t L,
                                            uint32_t LB, uint8_t* __restrict__ out,
                                            ull* prof) {
  const unsigned lane = lane_id();
  const uint64_t gw = gtid() >> 5, nw = gstride() >> 5;
  ull nbytes = 0;
  for (uint64_t i = gw; i < q; i += nw) {
    const uint64_t x = keys[i];
    const uint64_t j = route_leaf(heads, L, x);
    bool found = false;
    const uint32_t u = min(used[j], LB);
    warp_decode(data + j * LB, u, [&](uint32_t, uint64_t v) { found |= (v == x); });
    found = __any_sync(FULL, found);
    if (lane == 0) out[i] = found ? 1 : 0;
    nbytes += u + 9;  // leaf bytes, key in, answer out
  }
  if (prof && lane == 0 && nbytes) atomicAdd(prof, nbytes);
}

__global__ void __launch_bounds__(kT) k_range_prep(const uint64_t* __restrict__ lo,
                                                   const uint64_t* __restrict__ hi, uint64_t q,
                                                   const uint64_t* __restrict__ heads, uint64_t L,
                                                   uint64_t* __restrict__ first,
                                                   uint64_t* __restrict__ items,
                                                   uint64_t* __restrict__ sum,
                                                   uint64_t* __restrict__ count) {
  for (uint64_t i = gtid(); i < q; i += gstride()) {
    const uint64_t a = lo[i], b = hi[i];
    uint64_t fl = 0, n = 0;
    if (a < b) {
      fl = route_leaf(heads, L, a);
      n = route_leaf(heads, L, b - 1) - fl + 1;
    }
    first[i] = fl;
    items[i] = n;
    sum[i] = 0;
    count[i] = 0;
  }
}

struct RangeArgs {
  const uint64_t* lo;
  const uint64_t* hi;
  uint64_t q;
  const uint64_t* first;
  const uint64_t* off;  // q + 1 entries
  const uint8_t* data;
  const uint32_t* used;
  const uint32_t* cnt;
  uint32_t LB;
  uint64_t* sum;
  uint64_t* count;
  ull* prof;  // profiling: leaf bytes scanned (nullable)
};

__global__ void __launch_bounds__(kT) k_range(RangeArgs a) {
  const unsigned lane = lane_id();
  const uint64_t gw = gtid() >> 5, nw = gstride() >> 5;
  const uint64_t N = a.off[a.q];
  const uint64_t g0 = N * gw / nw, g1 = N * (gw + 1) / nw;
  if (g0 >= g1) return;
  uint64_t qi = upper_count(a.off, a.q + 1, g0) - 1;
  uint64_t s = 0, c = 0;
  ull nbytes = 0;
  uint64_t qend = a.off[qi + 1];
  uint64_t lo = a.lo[qi], hi = a.hi[qi], fl = a.first[qi], qoff = a.off[qi];
  uint64_t g = g0;
  while (g < g1) {
    while (g >= qend) {
      s = warp_sum(s);
      c = warp_sum(c);
      if (lane == 0 && (s | c)) {
        atomicAdd((ull*)&a.sum[qi], (ull)s);
        atomicAdd((ull*)&a.count[qi], (ull)c);
      }
      s = 0;
      c = 0;
      qi++;
      qend = a.off[qi + 1];
      lo = a.lo[qi]; hi = a.hi[qi]; fl = a.first[qi]; qoff = a.off[qi];
    }
    const uint64_t li = g - qoff, n = qend - qoff;
    if (li > 0 && li + 1 < n) {
      // leaves strictly inside the range: no filter, chunked span sum
      const uint64_t stop = min(g1, qend - 1);  // exclusive, global item index
      uint64_t cc = 0;
      warp_span_sum(a.data, a.used, a.cnt, a.LB, fl + li, fl + (stop - qoff), s, cc, nbytes);
      if (lane == 0) c += warp_sum(cc); else warp_sum(cc);
      g = stop;
      continue;
    }
    const uint64_t j = fl + li;
    const uint32_t u = min(a.used[j], a.LB);
    nbytes += u;
    warp_decode(a.data + j * a.LB, u, [&](uint32_t, uint64_t v) {
      if (v >= lo && v < hi) { s += v; c++; }
    });
    g++;
  }
  s = warp_sum(s);
  c = warp_sum(c);
  if (lane == 0 && (s | c)) {
    atomicAdd((ull*)&a.sum[qi], (ull)s);
    atomicAdd((ull*)&a.count[qi], (ull)c);
  }
  nbytes = warp_sum(nbytes);
  if (a.prof && lane == 0 && nbytes) atomicAdd(a.prof, nbytes);
}

__global__ void __launch_bounds__(kT) k_sum(const uint8_t* __restrict__ data,
                                            const uint32_t* __restrict__ used,
                                            const uint32_t* __restrict__ cnt, uint64_t L,
                                            uint32_t LB, uint64_t* sum, uint64_t* count,
                                            ull* prof) {
  const unsigned lane = lane_id();
  const uint64_t gw = gtid() >> 5, nw = gstride() >> 5;
  const uint64_t j0 = L * gw / nw, j1 = L * (gw + 1) / nw;
  uint64_t s = 0, c = 0;
  ull nbytes = 0;
  warp_span_sum(data, used, cnt, LB, j0, j1, s, c, nbytes);
  s = warp_sum(s);
  c = warp_sum(c);
  nbytes = warp_sum(nbytes);
  if (lane == 0 && (s | c)) {
    atomicAdd((ull*)sum, (ull)s);
    if (count) atomicAdd((ull*)count, (ull)c);
  }
  if (prof && lane == 0 && nbytes) atomicAdd(prof, nbytes + 8ull * (j1 - j0));
}

int persistent_grid(const cpma* h) { return h->num_sms * 8; }

// Scratch of the allocation-free range_map: per-query first leaf, item count
// and item offsets, plus the partial sums of the offset scan.  It lives in the
// library's own device image, so every GPU that loads the library holds these
// 2 MiB until the process exits, and every call shares them.
constexpr uint64_t kNoAllocMaxQueries = 1ull << 16;
constexpr uint64_t kNoAllocPartials = 1024;
constexpr size_t kNoAllocBytes = 2u << 20;
static_assert((3 * kNoAllocMaxQueries + 1 + kNoAllocPartials) * 8 <= kNoAllocBytes,
              "range scratch too small");
static __device__ __align__(256) uint8_t g_range_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_range_scratch on device `dev` (which must be current).
// The host-side name of the array is only a stand-in, so the address is
// looked up once per device with cudaGetSymbolAddress and cached.
int scratch_address(int dev, uint8_t** out) {
  if (dev < 0 || dev >= kMaxDevices) return CPMA_EINVAL;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_range_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return CPMA_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<uint8_t*>(g_scratch_addr[dev]);
  return CPMA_OK;
}

}  // namespace

int run_has(const cpma* h, const uint64_t* d_keys, uint64_t q, uint8_t* d_out, cudaStream_t st) {
  if (q == 0) return CPMA_OK;
  const int grid = (int)std::max<uint64_t>(
      1, std::min<uint64_t>((q * 32 + kT - 1) / kT, (uint64_t)persistent_grid(h)));
  prof_begin(h, PH_HAS, st);
  k_has<<<grid, kT, 0, st>>>(d_keys, q, h->data, h->used, h->heads, h->L, h->cfg.leaf_bytes,
                             d_out, prof_bytes(h, PH_HAS));
  CPMA_LAUNCHED(h);
  prof_end(h, st);
  return check_cuda(cudaGetLastError());
}

int run_range(const cpma* h, const uint64_t* lo, const uint64_t* hi, uint64_t q, uint64_t* sum,
              uint64_t* count, cudaStream_t st) {
  if (q == 0) return CPMA_OK;
  cpma* hm = const_cast<cpma*>(h);
  CPMA_TRY(ensure(hm->s.q_first, q * 8));
  CPMA_TRY(ensure(hm->s.q_items, q * 8));
  CPMA_TRY(ensure(hm->s.q_off, (q + 1) * 8));
  uint64_t* first = (uint64_t*)hm->s.q_first.p;
  uint64_t* items = (uint64_t*)hm->s.q_items.p;
  uint64_t* off = (uint64_t*)hm->s.q_off.p;
  const int g1 = (int)std::max<uint64_t>(
      1, std::min<uint64_t>((q + kT - 1) / kT, (uint64_t)h->num_sms * 8));
  prof_begin(h, PH_RANGE_PREP, st);
  prof_add_bytes(h, PH_RANGE_PREP, 72ull * q);  // lo, hi in; first, items, sums out; scan
  k_range_prep<<<g1, kT, 0, st>>>(lo, hi, q, h->heads, h->L, first, items, sum, count);
  CPMA_LAUNCHED(h);
  CPMA_TRY(scan_u64_query(hm, items, off, q, st));
  prof_end(h, st);
  RangeArgs a;
  a.lo = lo;
  a.hi = hi;
  a.q = q;
  a.first = first;
  a.off = off;
  a.data = h->data;
  a.used = h->used;
  a.cnt = h->cnt;
  a.LB = h->cfg.leaf_bytes;
  a.sum = sum;
  a.count = count;
  a.prof = prof_bytes(h, PH_RANGE);
  prof_begin(h, PH_RANGE, st);
  k_range<<<persistent_grid(h), kT, 0, st>>>(a);
  CPMA_LAUNCHED(h);
  prof_end(h, st);
  return check_cuda(cudaGetLastError());
}

int run_range_noalloc(const cpma* h, const uint64_t* lo, const uint64_t* hi, uint64_t q,
                      uint64_t* sum, uint64_t* count, cudaStream_t st) {
  if (q > kNoAllocMaxQueries) return CPMA_EINVAL;
  if (q == 0) return CPMA_OK;
  int dev = -1;
  CPMA_CUDA(cudaGetDevice(&dev));
  if (dev != h->device) return CPMA_EINVAL;
  uint8_t* base = nullptr;
  CPMA_TRY(scratch_address(dev, &base));
  uint64_t* first = reinterpret_cast<uint64_t*>(base);
  uint64_t* items = first + kNoAllocMaxQueries;
  uint64_t* off = items + kNoAllocMaxQueries;            // q + 1 entries
  uint64_t* partials = off + kNoAllocMaxQueries + 1;     // kNoAllocPartials entries
  const int g1 = (int)std::max<uint64_t>(
      1, std::min<uint64_t>((q + kT - 1) / kT, (uint64_t)h->num_sms * 8));
  // every scratch entry read below is written first on this stream: nothing
  // carries over from an earlier call
  k_range_prep<<<g1, kT, 0, st>>>(lo, hi, q, h->heads, h->L, first, items, sum, count);
  CPMA_LAUNCHED(h);
  CPMA_CUDA(cudaGetLastError());
  CPMA_TRY(scan_u64_given_partials(const_cast<cpma*>(h), items, off, q, partials,
                                   kNoAllocPartials, st));
  RangeArgs a;
  a.lo = lo;
  a.hi = hi;
  a.q = q;
  a.first = first;
  a.off = off;
  a.data = h->data;
  a.used = h->used;
  a.cnt = h->cnt;
  a.LB = h->cfg.leaf_bytes;
  a.sum = sum;
  a.count = count;
  a.prof = nullptr;
  k_range<<<persistent_grid(h), kT, 0, st>>>(a);
  CPMA_LAUNCHED(h);
  return check_cuda(cudaGetLastError());
}

int run_sum(const cpma* h, uint64_t* sum, uint64_t* count, cudaStream_t st) {
  CPMA_CUDA(cudaMemsetAsync(sum, 0, 8, st));
  if (count) CPMA_CUDA(cudaMemsetAsync(count, 0, 8, st));
  prof_begin(h, PH_SUM, st);
  k_sum<<<persistent_grid(h), kT, 0, st>>>(h->data, h->used, h->cnt, h->L, h->cfg.leaf_bytes, sum,
                                           count, prof_bytes(h, PH_SUM));
  CPMA_LAUNCHED(h);
  prof_end(h, st);
  return check_cuda(cudaGetLastError());
}

}  // namespace cpmaimpl
