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
//  map_range_length (App. A: f on at most `length` elements from the first
//    key >= start): a prefix sum of the leaves' element counts turns each
//    query into a range of global ranks [r0, r1); the same load-balanced
//    walk then sums whole leaves inside it and filters the two end leaves by
//    rank instead of by key.
//  range_reduce (Sec. 3 range_map with other functions): min, max, xor or
//    sum of the keys of [lo, hi) whose masked bits match a value, with the
//    count of those keys; every covered leaf is decoded.
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

// Warp per query key, 32 keys routed per step.  A key equal to its leaf's
// head, below it or above the leaf's last element needs no decode beyond the
// lane summaries; otherwise only the lane whose value interval holds the key
// is decoded (one byte position per lane).  Leaves with codes longer than 4
// bytes or more than 512 used bytes go through the general decoder.
__global__ void __launch_bounds__(kT) k_has(const uint64_t* __restrict__ keys, uint64_t q,
                                            const uint8_t* __restrict__ data,
                                            const uint32_t* __restrict__ used,
                                            const uint64_t* __restrict__ heads, uint64_t L,
                                            uint32_t LB, uint8_t* __restrict__ out,
                                            ull* prof, int raw) {
  const unsigned lane = lane_id();
  const uint64_t gw = gtid() >> 5, nw = gstride() >> 5;
  ull nbytes = 0;
  uint64_t r0, r1;
  warp_share(q, gw, nw, r0, r1);
  if (!raw) {
    // byte codes: one key per thread, its leaf decoded up to the key
    for (uint64_t qi = r0 + lane; qi < r1; qi += 32) {
      const uint64_t x = keys[qi];
      const uint64_t j = route_leaf(heads, L, x);
      const uint32_t u = min(used[j], LB);
      nbytes += u + 9;
      out[qi] = thread_leaf_has(data + j * LB, u, x) ? 1u : 0u;
    }
    nbytes = warp_sum(nbytes);
    if (prof && lane == 0 && nbytes) atomicAdd(prof, nbytes);
    return;
  }
  for (uint64_t base = r0; base < r1; base += 32) {
    const uint64_t qi = base + lane;
    uint64_t xi = 0, ji = 0;
    uint32_t ui = 0;
    if (qi < r1) {
      xi = keys[qi];
      ji = route_leaf(heads, L, xi);
      ui = min(used[ji], LB);
    }
    const uint32_t nk = (uint32_t)min((uint64_t)32, r1 - base);
    uint32_t found_bits = 0;
    for (uint32_t k = 0; k < nk; k++) {
      const uint64_t x = __shfl_sync(FULL, xi, k);
      const uint64_t j = __shfl_sync(FULL, ji, k);
      const uint32_t u = __shfl_sync(FULL, ui, k);
      const uint8_t* leaf = data + j * LB;
      nbytes += u + 9;
      bool found = false;
      if (raw) {  // codec 1: compare the cells
        bool f = false;
        warp_decode(leaf, u, [&](uint32_t, uint64_t val) { f |= (val == x); }, true);
        found = __any_sync(FULL, f);
      } else if (u > 0) {
        const uint32_t p0 = lane * 16u;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (p0 < u) v = __ldg(reinterpret_cast<const uint4*>(leaf + p0));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        const int b_lo = lane == 0 ? 8 : 0;
        const int b_hi = (u > p0) ? (int)min(16u, u - p0) : 0;
        LaneCodes lc;
        lane_codes<false>(w, b_lo, b_hi, lc);
        bool bad = lc.bad || u > 512;  // one 16-byte chunk per lane covers 512 bytes
        uint32_t pv = __shfl_up_sync(FULL, lc.tail, 1);
        uint32_t ps = __shfl_up_sync(FULL, lc.tail_sh, 1);
        if (lane == 0) { pv = 0; ps = 0; }
        uint32_t D = 0;
        if (lc.term) {
          if (ps / 7u + lc.first_len > 4u) bad = true;
          D = lc.D - lc.first_own + pv + (lc.first_own << ps);
        }
        if (__any_sync(FULL, bad)) {
          bool f = false;
          warp_decode(leaf, u, [&](uint32_t, uint64_t val) { f |= (val == x); });
          found = __any_sync(FULL, f);
        } else {
          const uint64_t head = __shfl_sync(FULL, (uint64_t)w[0] | ((uint64_t)w[1] << 32), 0);
          const uint64_t Dinc = warp_incl_scan((uint64_t)D);
          const uint64_t V = head + (Dinc - D);
          const uint64_t lastv = head + __shfl_sync(FULL, Dinc, 31);
          if (x == head) {
            found = true;
          } else if (x > head && x <= lastv) {
            const unsigned own = __ballot_sync(FULL, lc.term != 0 && V < x && x <= V + D);
            const unsigned o = __ffs(own) - 1;
            uint32_t xo[4];
#pragma unroll
            for (int t = 0; t < 4; t++) xo[t] = __shfl_sync(FULL, lc.x[t], o);
            const uint32_t term_o = __shfl_sync(FULL, lc.term, o);
            const uint32_t pv_o = __shfl_sync(FULL, pv, o), ps_o = __shfl_sync(FULL, ps, o);
            const uint64_t V_o = __shfl_sync(FULL, V, o);
            const bool is_t = lane < 16 && ((term_o >> lane) & 1u);
            const uint32_t before = lane < 16 ? (term_o & ((1u << lane) - 1u)) : 0u;
            const bool firstc = before == 0;
            const uint32_t st0 = firstc ? (o == 0 ? 8u : 0u) : (32u - (uint32_t)__clz(before));
            uint32_t code = 0;
            if (is_t) {
              const uint32_t own_bits = compact7(window32(xo, st0)) & mask7(lane + 1u - st0);
              code = firstc ? pv_o + (own_bits << ps_o) : own_bits;
            }
            const uint64_t val = V_o + warp_incl_scan(code);
            found = __any_sync(FULL, is_t && val == x);
          }
        }
      }
      if (found) found_bits |= 1u << k;
    }
    if (qi < r1) out[qi] = (found_bits >> lane) & 1u;
  }
  if (prof && lane == 0 && nbytes) atomicAdd(prof, nbytes);
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
  const uint64_t* P = nullptr;  // rank mode: elements before each leaf (L + 1)
  int raw = 0;                  // leaves hold 8-byte cells (codec 1)
};

__global__ void __launch_bounds__(kT) k_range_prep(const uint64_t* __restrict__ lo,
                                                   const uint64_t* __restrict__ hi, uint64_t q,
                                                   const uint64_t* __restrict__ heads, uint64_t L,
                                                   uint64_t* __restrict__ first,
                                                   uint64_t* __restrict__ items,
                                                   uint64_t* __restrict__ sum,
                                                   uint64_t* __restrict__ count,
                                                   uint64_t init = 0) {
  for (uint64_t i = gtid(); i < q; i += gstride()) {
    const uint64_t a = lo[i], b = hi[i];
    uint64_t fl = 0, n = 0;
    if (a < b) {
      fl = route_leaf(heads, L, a);
      n = route_leaf(heads, L, b - 1) - fl + 1;
    }
    first[i] = fl;
    items[i] = n;
    sum[i] = init;
    count[i] = 0;
  }
}

// Rank of the first key >= x: elements before its leaf plus the leaf's
// elements below x (the whole warp decodes the leaf).
__device__ __forceinline__ uint64_t rank_of(uint64_t x, const uint64_t* __restrict__ heads,
                                            const uint8_t* __restrict__ data,
                                            const uint32_t* __restrict__ used, uint64_t L,
                                            uint32_t LB, const uint64_t* __restrict__ P, int raw) {
  const uint64_t j = route_leaf(heads, L, x);
  uint32_t below = 0;
  warp_decode(data + j * LB, min(used[j], LB), [&](uint32_t, uint64_t v) { below += v < x; },
              raw);
  return P[j] + warp_sum(below);
}

// Step 1 of the rank-space queries (warp per query): the rank range
// [r0, r1) and the leaves holding it.  KEYS: [a, b) is a key range, r0 =
// rank(a), r1 = rank(b) (r1 = r0 when a >= b).  Otherwise (map_range_length)
// a is the start key and b the length: r1 = min(r0 + b, n).
template <bool KEYS>
__global__ void __launch_bounds__(kT) k_rank_prep(const uint64_t* __restrict__ A,
                                                  const uint64_t* __restrict__ B, uint64_t q,
                                                  const uint64_t* __restrict__ heads,
                                                  const uint8_t* __restrict__ data,
                                                  const uint32_t* __restrict__ used, uint64_t L,
                                                  uint32_t LB, const uint64_t* __restrict__ P,
                                                  uint64_t* __restrict__ r0o,
                                                  uint64_t* __restrict__ r1o,
                                                  uint64_t* __restrict__ first,
                                                  uint64_t* __restrict__ items,
                                                  uint64_t* __restrict__ sum,
                                                  uint64_t* __restrict__ count, int raw) {
  const unsigned lane = lane_id();
  const uint64_t gw = gtid() >> 5, nw = gstride() >> 5;
  const uint64_t n = P[L];
  for (uint64_t i = gw; i < q; i += nw) {
    const uint64_t a = A[i], b = B[i];
    const uint64_t r0 = rank_of(a, heads, data, used, L, LB, P, raw);
    uint64_t r1;
    if constexpr (KEYS) r1 = a < b ? rank_of(b, heads, data, used, L, LB, P, raw) : r0;
    else r1 = (b >= n - r0) ? n : r0 + b;
    uint64_t f = 0, it = 0;
    if (r1 > r0) {
      f = upper_count(P, L + 1, r0) - 1;
      it = upper_count(P, L + 1, r1 - 1) - f;
    }
    if (lane == 0) {
      r0o[i] = r0;
      r1o[i] = r1;
      first[i] = f;
      items[i] = it;
      if (sum) sum[i] = 0;
      if (count) count[i] = KEYS ? r1 - r0 : 0;
    }
  }
}

// range_extract: the keys of ranks [r0, r1) of every query, written from
// out[off[i]] on (entries at or past cap are dropped).  Same load-balanced
// (query, leaf) walk as k_range.
struct ExtractArgs {
  const uint64_t* r0;
  const uint64_t* r1;
  uint64_t q;
  const uint64_t* first;
  const uint64_t* item_off;  // q + 1
  const uint64_t* out_off;   // q + 1
  const uint64_t* P;
  const uint8_t* data;
  const uint32_t* used;
  uint32_t LB;
  uint64_t* out;
  uint64_t cap;
  int raw;
};

__global__ void __launch_bounds__(kT) k_extract(ExtractArgs a) {
  const uint64_t gw = gtid() >> 5, nw = gstride() >> 5;
  const uint64_t N = a.item_off[a.q];
  const uint64_t g0 = N * gw / nw, g1 = N * (gw + 1) / nw;
  if (g0 >= g1) return;
  uint64_t qi = upper_count(a.item_off, a.q + 1, g0) - 1;
  for (uint64_t g = g0; g < g1; g++) {
    while (g >= a.item_off[qi + 1]) qi++;
    const uint64_t j = a.first[qi] + (g - a.item_off[qi]);
    const uint64_t r0 = a.r0[qi], r1 = a.r1[qi], base = a.P[j], o = a.out_off[qi];
    warp_decode(a.data + j * a.LB, min(a.used[j], a.LB), [&](uint32_t idx, uint64_t v) {
      const uint64_t r = base + idx;
      if (r >= r0 && r < r1 && o + (r - r0) < a.cap) a.out[o + (r - r0)] = v;
    }, a.raw);
  }
}

// range_reduce: the functions, their identities and their atomics
template <int OP>
__device__ __forceinline__ uint64_t op_apply(uint64_t a, uint64_t b) {
  if constexpr (OP == CPMA_OP_SUM) return a + b;
  else if constexpr (OP == CPMA_OP_MIN) return a < b ? a : b;
  else if constexpr (OP == CPMA_OP_MAX) return a > b ? a : b;
  else return a ^ b;
}
template <int OP>
__host__ __device__ __forceinline__ uint64_t op_identity() {
  return OP == CPMA_OP_MIN ? ~0ull : 0ull;
}
template <int OP>
__device__ __forceinline__ void op_atomic(uint64_t* p, uint64_t v) {
  if constexpr (OP == CPMA_OP_SUM) atomicAdd((ull*)p, (ull)v);
  else if constexpr (OP == CPMA_OP_MIN) atomicMin((ull*)p, (ull)v);
  else if constexpr (OP == CPMA_OP_MAX) atomicMax((ull*)p, (ull)v);
  else atomicXor((ull*)p, (ull)v);
}

// Thread-per-leaf reduction of a byte-code leaf: every element v with
// (v & mask) == value is reduced into (r, c), the running value kept as in
// thread_leaf_sum; bytes past u are no terminators here (a repeated value
// would count twice), and a leaf with a code over 4 bytes is reduced again
// exactly.
template <int OP, bool FIRST>
__device__ __forceinline__ void leaf_reduce_chunk(const uint32_t (&w)[4], uint32_t valid,
                                                  uint64_t mask, uint64_t value, uint64_t& val,
                                                  uint64_t& r, uint64_t& c, uint32_t& acc,
                                                  uint32_t& pw, uint32_t& pwmax) {
#pragma unroll
  for (int b = FIRST ? 8 : 0; b < 16; b++) {
    const uint32_t wb = w[b >> 2];
    const bool in = (valid >> b) & 1u;  // bytes past u: neither codes nor terminators
    acc += (__byte_perm(wb, 0u, 0x4440u + (uint32_t)(b & 3)) & 0x7Fu) * pw;
    const bool term = in && (wb & (0x80u << (8 * (b & 3)))) == 0u;
    pwmax = (in && pw > pwmax) ? pw : pwmax;
    val += term ? (uint64_t)acc : 0ull;
    const bool hit = term && (val & mask) == value;
    r = hit ? op_apply<OP>(r, val) : r;
    c += hit ? 1u : 0u;
    acc = (term || !in) ? 0u : acc;
    pw = (term || !in) ? 1u : pw << 7;
  }
}

template <int OP>
__device__ __forceinline__ void thread_leaf_reduce(const uint8_t* __restrict__ leafp, uint32_t u,
                                                   uint64_t mask, uint64_t value, uint64_t& r,
                                                   uint64_t& c) {
  uint4 v = *reinterpret_cast<const uint4*>(leafp);
  uint4 v2 = u > 16u ? *reinterpret_cast<const uint4*>(leafp + 16) : make_uint4(0u, 0u, 0u, 0u);
  uint64_t val = (uint64_t)v.x | ((uint64_t)v.y << 32);
  uint64_t lr = op_identity<OP>(), lc = 0;
  if ((val & mask) == value) { lr = op_apply<OP>(lr, val); lc++; }
  uint32_t acc = 0, pw = 1, pwmax = 0;
  for (uint32_t p0 = 0; p0 < u; p0 += 32) {
    if (p0) {
      v = *reinterpret_cast<const uint4*>(leafp + p0);
      v2 = p0 + 16u < u ? *reinterpret_cast<const uint4*>(leafp + p0 + 16) : make_uint4(0u, 0u, 0u, 0u);
    }
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    const uint32_t va = p0 + 16u <= u ? 0xFFFFu : (1u << (u - p0)) - 1u;
    if (p0) leaf_reduce_chunk<OP, false>(w, va, mask, value, val, lr, lc, acc, pw, pwmax);
    else leaf_reduce_chunk<OP, true>(w, va, mask, value, val, lr, lc, acc, pw, pwmax);
    if (p0 + 16u < u) {
      const uint32_t w2[4] = {v2.x, v2.y, v2.z, v2.w};
      const uint32_t vb = p0 + 32u <= u ? 0xFFFFu : (1u << (u - p0 - 16u)) - 1u;
      leaf_reduce_chunk<OP, false>(w2, vb, mask, value, val, lr, lc, acc, pw, pwmax);
    }
  }
  if (pwmax >= (1u << 28)) {  // a long code: exact 64-bit decode
    val = *reinterpret_cast<const uint64_t*>(leafp);
    lr = op_identity<OP>();
    lc = 0;
    if ((val & mask) == value) { lr = op_apply<OP>(lr, val); lc++; }
    uint64_t a64 = 0;
    uint32_t sh = 0;
    for (uint32_t p = 8; p < u; p++) {
      const uint32_t b = leafp[p];
      if (sh < 64) a64 |= (uint64_t)(b & 0x7Fu) << sh;
      if (b & 0x80u) {
        sh += 7;
      } else {
        val += a64;
        if ((val & mask) == value) { lr = op_apply<OP>(lr, val); lc++; }
        a64 = 0;
        sh = 0;
      }
    }
  }
  r = op_apply<OP>(r, lr);
  c += lc;
}

// Same load-balanced (query, leaf) walk as k_range: the end leaves of a
// query are decoded by the warp and filtered by range and mask, the leaves
// strictly inside are reduced one per thread (byte codes).
template <int OP>
__global__ void __launch_bounds__(kT) k_range_reduce(RangeArgs a, uint64_t mask,
                                                     uint64_t value) {
  const unsigned lane = lane_id();
  const uint64_t gw = gtid() >> 5, nw = gstride() >> 5;
  const uint64_t N = a.off[a.q];
  const uint64_t g0 = N * gw / nw, g1 = N * (gw + 1) / nw;
  if (g0 >= g1) return;
  uint64_t qi = upper_count(a.off, a.q + 1, g0) - 1;
  uint64_t r = op_identity<OP>(), c = 0;
  uint64_t qend = a.off[qi + 1];
  uint64_t lo = a.lo[qi], hi = a.hi[qi], fl = a.first[qi], qoff = a.off[qi];
  for (uint64_t g = g0; g < g1;) {
    while (g >= qend) {
#pragma unroll
      for (int o = 16; o; o >>= 1) r = op_apply<OP>(r, __shfl_xor_sync(FULL, r, o));
      c = warp_sum(c);
      if (lane == 0 && c) {
        op_atomic<OP>(&a.sum[qi], r);
        atomicAdd((ull*)&a.count[qi], (ull)c);
      }
      r = op_identity<OP>();
      c = 0;
      qi++;
      qend = a.off[qi + 1];
      lo = a.lo[qi]; hi = a.hi[qi]; fl = a.first[qi]; qoff = a.off[qi];
    }
    const uint64_t li = g - qoff, n = qend - qoff;
    if (!a.raw && li > 0 && li + 1 < n) {
      // leaves strictly inside the range (byte codes): one leaf per lane
      const uint64_t stop = min(g1, qend - 1);
      for (uint64_t j = fl + li + lane; j < fl + (stop - qoff); j += 32) {
        const uint32_t u = min(a.used[j], a.LB);
        if (u) thread_leaf_reduce<OP>(a.data + j * a.LB, u, mask, value, r, c);
      }
      g = stop;
      continue;
    }
    const uint64_t j = fl + li;
    warp_decode(a.data + j * a.LB, min(a.used[j], a.LB), [&](uint32_t, uint64_t v) {
      if (v >= lo && v < hi && (v & mask) == value) { r = op_apply<OP>(r, v); c++; }
    }, a.raw);
    g++;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) r = op_apply<OP>(r, __shfl_xor_sync(FULL, r, o));
  c = warp_sum(c);
  if (lane == 0 && c) {
    op_atomic<OP>(&a.sum[qi], r);
    atomicAdd((ull*)&a.count[qi], (ull)c);
  }
}


// RANK: lo/hi of a query are global element ranks [r0, r1) and the end
// leaves filter by rank P[j] + index; otherwise they are keys.
template <bool RANK>
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
      if (a.raw)
        warp_span_sum(a.data, a.used, a.cnt, a.LB, fl + li, fl + (stop - qoff), s, cc, nbytes,
                      a.raw);
      else  // byte codes: one leaf per lane
        thread_span_sum(a.data, a.used, a.cnt, a.LB, fl + li, fl + (stop - qoff), s, cc, nbytes);
      if (lane == 0) c += warp_sum(cc); else warp_sum(cc);
      g = stop;
      continue;
    }
    const uint64_t j = fl + li;
    const uint32_t u = min(a.used[j], a.LB);
    nbytes += u;
    if constexpr (RANK) {
      const uint64_t r = a.P[j];
      warp_decode(a.data + j * a.LB, u, [&](uint32_t idx, uint64_t v) {
        if (r + idx >= lo && r + idx < hi) { s += v; c++; }
      }, a.raw);
    } else {
      warp_decode(a.data + j * a.LB, u, [&](uint32_t, uint64_t v) {
        if (v >= lo && v < hi) { s += v; c++; }
      }, a.raw);
    }
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

constexpr uint32_t kSumShift = 4;      // sort key of a leaf: used bytes / 16
constexpr uint32_t kSumBuckets = 128;  // enough for 2048-byte leaves (a multiple of 32)

__global__ void __launch_bounds__(kT) k_sum(const uint8_t* __restrict__ data,
                                            const uint32_t* __restrict__ used,
                                            const uint32_t* __restrict__ cnt, uint64_t L,
                                            uint32_t LB, uint64_t* sum, uint64_t* count,
                                            ull* prof, int raw) {
  const unsigned lane = lane_id();
  const uint64_t gw = gtid() >> 5, nw = gstride() >> 5;
  const uint64_t j0 = L * gw / nw, j1 = L * (gw + 1) / nw;
  uint64_t s = 0, c = 0;
  ull nbytes = 0;
  if (raw) {
    warp_span_sum(data, used, cnt, LB, j0, j1, s, c, nbytes, raw);
  } else {
    // The block's leaves in tiles of kT, each ordered by used bytes (a
    // counting sort in shared memory), so the 32 leaves a warp decodes side
    // by side take about the same number of steps.
    __shared__ uint32_t s_hist[kSumBuckets];
    __shared__ uint32_t s_order[kT];
    const uint64_t b0 = L * blockIdx.x / gridDim.x, b1 = L * (blockIdx.x + 1) / gridDim.x;
    for (uint64_t t0 = b0; t0 < b1; t0 += kT) {
      for (uint32_t i = threadIdx.x; i < kSumBuckets; i += kT) s_hist[i] = 0;
      __syncthreads();
      const uint64_t j = t0 + threadIdx.x;
      const uint32_t u = j < b1 ? min(used[j], LB) : 0u;
      const uint32_t bkt = min(u >> kSumShift, kSumBuckets - 1);
      const uint32_t slot = j < b1 ? atomicAdd(&s_hist[bkt], 1u) : 0u;
      __syncthreads();
      if (threadIdx.x < 32) {  // exclusive scan of the bucket counts
        uint32_t run = 0;
        for (uint32_t b = 0; b < kSumBuckets; b += 32) {
          const uint32_t v = s_hist[b + lane];
          const uint32_t inc = warp_incl_scan(v);
          s_hist[b + lane] = run + inc - v;
          run += __shfl_sync(FULL, inc, 31);
        }
      }
      __syncthreads();
      if (j < b1) s_order[s_hist[bkt] + slot] = threadIdx.x;
      __syncthreads();
      const uint32_t nt = (uint32_t)min((uint64_t)kT, b1 - t0);
      if (threadIdx.x < nt) {
        const uint64_t jj = t0 + s_order[threadIdx.x];
        const uint32_t uu = min(used[jj], LB);
        nbytes += 8;  // its used and element counts
        if (uu) {
          s += thread_leaf_sum(data + jj * LB, uu);
          c += cnt[jj];
          nbytes += uu;
        }
      }
      __syncthreads();  // s_hist and s_order are reused
    }
  }
  s = warp_sum(s);
  c = warp_sum(c);
  nbytes = warp_sum(nbytes);
  if (lane == 0 && (s | c)) {
    atomicAdd((ull*)sum, (ull)s);
    if (count) atomicAdd((ull*)count, (ull)c);
  }
  if (prof && lane == 0 && nbytes) atomicAdd(prof, nbytes + (raw ? 8ull * (j1 - j0) : 0ull));
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
      1, std::min<uint64_t>((q + kT - 1) / kT, (uint64_t)persistent_grid(h)));
  prof_begin(h, PH_HAS, st);
  k_has<<<grid, kT, 0, st>>>(d_keys, q, h->data, h->used, h->heads, h->L, h->cfg.leaf_bytes,
                             d_out, prof_bytes(h, PH_HAS), (int)h->cfg.codec);
  CPMA_LAUNCHED(h);
  prof_end(h, st);
  return check_cuda(cudaGetLastError());
}

int run_range(const cpma* h, const uint64_t* lo, const uint64_t* hi, uint64_t q, uint64_t* sum,
              uint64_t* count, cudaStream_t st) {
  if (q == 0) return CPMA_OK;
  cpma* hm = const_cast<cpma*>(h);
  CPMA_TRY(ensure(hm, hm->s.q_first, q * 8));
  CPMA_TRY(ensure(hm, hm->s.q_items, q * 8));
  CPMA_TRY(ensure(hm, hm->s.q_off, (q + 1) * 8));
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
  a.raw = (int)h->cfg.codec;
  prof_begin(h, PH_RANGE, st);
  k_range<false><<<persistent_grid(h), kT, 0, st>>>(a);
  CPMA_LAUNCHED(h);
  prof_end(h, st);
  return check_cuda(cudaGetLastError());
}

int run_range_length(const cpma* h, const uint64_t* start, const uint64_t* length, uint64_t q,
                     uint64_t* sum, uint64_t* count, cudaStream_t st) {
  if (q == 0) return CPMA_OK;
  cpma* hm = const_cast<cpma*>(h);
  Scratch& s = hm->s;
  CPMA_TRY(ensure(hm, s.q_first, q * 8));
  CPMA_TRY(ensure(hm, s.q_items, q * 8));
  CPMA_TRY(ensure(hm, s.q_off, (q + 1) * 8));
  CPMA_TRY(ensure(hm, s.q_lo, q * 8));
  CPMA_TRY(ensure(hm, s.q_hi, q * 8));
  CPMA_TRY(ensure(hm, s.q_rank, (h->L + 1) * 8));
  uint64_t* P = (uint64_t*)s.q_rank.p;
  uint64_t* r0 = (uint64_t*)s.q_lo.p;
  uint64_t* r1 = (uint64_t*)s.q_hi.p;
  uint64_t* first = (uint64_t*)s.q_first.p;
  uint64_t* items = (uint64_t*)s.q_items.p;
  uint64_t* off = (uint64_t*)s.q_off.p;
  prof_begin(h, PH_RANGE_PREP, st);
  prof_add_bytes(h, PH_RANGE_PREP, 12ull * h->L + 88ull * q);
  CPMA_TRY(scan_u32_query(hm, h->cnt, P, h->L, st));
  const int g1 = (int)std::max<uint64_t>(
      1, std::min<uint64_t>((q * 32 + kT - 1) / kT, (uint64_t)h->num_sms * 16));
  k_rank_prep<false><<<g1, kT, 0, st>>>(start, length, q, h->heads, h->data, h->used, h->L,
                                        h->cfg.leaf_bytes, P, r0, r1, first, items, sum, count,
                                        (int)h->cfg.codec);
  CPMA_LAUNCHED(h);
  CPMA_TRY(scan_u64_query(hm, items, off, q, st));
  prof_end(h, st);
  RangeArgs a;
  a.lo = r0;
  a.hi = r1;
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
  a.P = P;
  a.raw = (int)h->cfg.codec;
  prof_begin(h, PH_RANGE, st);
  k_range<true><<<persistent_grid(h), kT, 0, st>>>(a);
  CPMA_LAUNCHED(h);
  prof_end(h, st);
  return check_cuda(cudaGetLastError());
}

int run_range_extract(const cpma* h, const uint64_t* lo, const uint64_t* hi, uint64_t q,
                      uint64_t* offsets, uint64_t* out, uint64_t cap, cudaStream_t st) {
  if (q == 0) return check_cuda(cudaMemsetAsync(offsets, 0, 8, st));
  cpma* hm = const_cast<cpma*>(h);
  Scratch& s = hm->s;
  CPMA_TRY(ensure(hm, s.q_first, q * 8));
  CPMA_TRY(ensure(hm, s.q_items, (q + 1) * 8));
  CPMA_TRY(ensure(hm, s.q_off, (q + 1) * 8));
  CPMA_TRY(ensure(hm, s.q_lo, q * 8));
  CPMA_TRY(ensure(hm, s.q_hi, q * 8));
  CPMA_TRY(ensure(hm, s.q_rank, (h->L + 1) * 8));
  uint64_t* P = (uint64_t*)s.q_rank.p;
  uint64_t* r0 = (uint64_t*)s.q_lo.p;
  uint64_t* r1 = (uint64_t*)s.q_hi.p;
  uint64_t* first = (uint64_t*)s.q_first.p;
  uint64_t* items = (uint64_t*)s.q_items.p;
  uint64_t* off = (uint64_t*)s.q_off.p;
  prof_begin(h, PH_RANGE_PREP, st);
  CPMA_TRY(scan_u32_query(hm, h->cnt, P, h->L, st));
  const int g1 = (int)std::max<uint64_t>(
      1, std::min<uint64_t>((q * 32 + kT - 1) / kT, (uint64_t)h->num_sms * 16));
  // counts (r1 - r0) go into `items` of a second pass: first the ranks
  k_rank_prep<true><<<g1, kT, 0, st>>>(lo, hi, q, h->heads, h->data, h->used, h->L,
                                       h->cfg.leaf_bytes, P, r0, r1, first, items, nullptr,
                                       offsets, (int)h->cfg.codec);
  CPMA_LAUNCHED(h);
  CPMA_TRY(scan_u64_query(hm, offsets, offsets, q, st));
  CPMA_TRY(scan_u64_query(hm, items, off, q, st));
  prof_end(h, st);
  if (!out || cap == 0) return check_cuda(cudaGetLastError());
  ExtractArgs a;
  a.r0 = r0;
  a.r1 = r1;
  a.q = q;
  a.first = first;
  a.item_off = off;
  a.out_off = offsets;
  a.P = P;
  a.data = h->data;
  a.used = h->used;
  a.LB = h->cfg.leaf_bytes;
  a.out = out;
  a.cap = cap;
  a.raw = (int)h->cfg.codec;
  prof_begin(h, PH_RANGE, st);
  k_extract<<<persistent_grid(h), kT, 0, st>>>(a);
  CPMA_LAUNCHED(h);
  prof_end(h, st);
  return check_cuda(cudaGetLastError());
}

int run_range_reduce(const cpma* h, const uint64_t* lo, const uint64_t* hi, uint64_t q, int op,
                     uint64_t mask, uint64_t value, uint64_t* out, uint64_t* count,
                     cudaStream_t st) {
  if (op == CPMA_OP_SUM && mask == 0 && value == 0)
    return run_range(h, lo, hi, q, out, count, st);
  if (q == 0) return CPMA_OK;
  cpma* hm = const_cast<cpma*>(h);
  CPMA_TRY(ensure(hm, hm->s.q_first, q * 8));
  CPMA_TRY(ensure(hm, hm->s.q_items, q * 8));
  CPMA_TRY(ensure(hm, hm->s.q_off, (q + 1) * 8));
  uint64_t* first = (uint64_t*)hm->s.q_first.p;
  uint64_t* items = (uint64_t*)hm->s.q_items.p;
  uint64_t* off = (uint64_t*)hm->s.q_off.p;
  const int g1 = (int)std::max<uint64_t>(
      1, std::min<uint64_t>((q + kT - 1) / kT, (uint64_t)h->num_sms * 8));
  uint64_t init = 0;
  switch (op) {
    case CPMA_OP_SUM: init = op_identity<CPMA_OP_SUM>(); break;
    case CPMA_OP_MIN: init = op_identity<CPMA_OP_MIN>(); break;
    case CPMA_OP_MAX: init = op_identity<CPMA_OP_MAX>(); break;
    case CPMA_OP_XOR: init = op_identity<CPMA_OP_XOR>(); break;
    default: return CPMA_EINVAL;
  }
  prof_begin(h, PH_RANGE_PREP, st);
  k_range_prep<<<g1, kT, 0, st>>>(lo, hi, q, h->heads, h->L, first, items, out, count, init);
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
  a.sum = out;
  a.count = count;
  a.prof = nullptr;
  a.raw = (int)h->cfg.codec;
  prof_begin(h, PH_RANGE, st);
  const int G = persistent_grid(h);
  switch (op) {
    case CPMA_OP_SUM: k_range_reduce<CPMA_OP_SUM><<<G, kT, 0, st>>>(a, mask, value); break;
    case CPMA_OP_MIN: k_range_reduce<CPMA_OP_MIN><<<G, kT, 0, st>>>(a, mask, value); break;
    case CPMA_OP_MAX: k_range_reduce<CPMA_OP_MAX><<<G, kT, 0, st>>>(a, mask, value); break;
    default: k_range_reduce<CPMA_OP_XOR><<<G, kT, 0, st>>>(a, mask, value); break;
  }
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
  // the offset scan needs at most 2 * SMs + 1 partials: checked before any
  // launch, so a rejected call leaves the outputs untouched
  if ((uint64_t)2 * h->num_sms + 1 > kNoAllocPartials) return CPMA_EINVAL;
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
  a.raw = (int)h->cfg.codec;
  k_range<false><<<persistent_grid(h), kT, 0, st>>>(a);
  CPMA_LAUNCHED(h);
  return check_cuda(cudaGetLastError());
}

int run_sum(const cpma* h, uint64_t* sum, uint64_t* count, cudaStream_t st) {
  CPMA_CUDA(cudaMemsetAsync(sum, 0, 8, st));
  if (count) CPMA_CUDA(cudaMemsetAsync(count, 0, 8, st));
  prof_begin(h, PH_SUM, st);
  k_sum<<<persistent_grid(h), kT, 0, st>>>(h->data, h->used, h->cnt, h->L, h->cfg.leaf_bytes, sum,
                                           count, prof_bytes(h, PH_SUM), (int)h->cfg.codec);
  CPMA_LAUNCHED(h);
  prof_end(h, st);
  return check_cuda(cudaGetLastError());
}

}  // namespace cpmaimpl
