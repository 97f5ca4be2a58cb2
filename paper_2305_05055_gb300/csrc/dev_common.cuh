// Device helpers shared by the CPMA kernels: the byte codec, warp scans, the
// warp-cooperative leaf decoder/encoder and the exact density-bound test.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cpmadev {

typedef unsigned long long ull;
constexpr uint64_t KEY_MAX = ~0ull;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

// Sec. 5 byte codes read as unsigned LEB128: max(1, ceil(bitlen(d) / 7)).
__device__ __forceinline__ unsigned leb_len(uint64_t d) {
  unsigned bl = 64u - (unsigned)__clzll((long long)(d | 1ull));
  return (bl + 6u) / 7u;
}

// Writes the code of d at p (7-bit groups, least significant first, high bit
// set on every byte but the last).  Returns the length.
__device__ __forceinline__ unsigned leb_put(uint8_t* p, uint64_t d) {
  unsigned n = 0;
  while (d >= 128u) { p[n++] = (uint8_t)(d | 0x80u); d >>= 7; }
  p[n++] = (uint8_t)d;
  return n;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(FULL, v, o);
    if ((int)lane_id() >= o) v += n;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// First index i in [0, n) with a[i] >= x (n if none).
template <typename P>
__device__ __forceinline__ uint64_t lower_bound(P a, uint64_t n, uint64_t x) {
  uint64_t lo = 0;
  while (n > 0) {
    uint64_t half = n >> 1;
    if (a[lo + half] < x) { lo += half + 1; n -= half + 1; }
    else n = half;
  }
  return lo;
}

// Number of entries <= x in the sorted array a[0..n), n >= 1 (branch-free).
__device__ __forceinline__ uint64_t upper_count(const uint64_t* __restrict__ a, uint64_t n,
                                                uint64_t x) {
  const uint64_t* base = a;
  while (n > 1) {
    uint64_t half = n >> 1;
    base = (__ldg(base + half) <= x) ? base + half : base;
    n -= half;
  }
  return (uint64_t)(base - a) + (__ldg(base) <= x ? 1u : 0u);
}

// Routing (Sec. 4 batch merge search, Sec. 5 point queries): the last leaf
// whose head-index entry is <= x, else leaf 0.
__device__ __forceinline__ uint64_t route_leaf(const uint64_t* __restrict__ heads, uint64_t L,
                                               uint64_t x) {
  uint64_t c = upper_count(heads, L, x);
  return c ? c - 1 : 0;
}

// Density bound test of Sec. 3 with byte density (Sec. 5): does a node at
// height h of a tree of height H, holding `b` bytes over `leaves` leaves of
// LB bytes, violate its upper or lower bound?  Exact 128-bit integers.
struct Bounds {
  uint32_t LB, tau_leaf, tau_root, rho_leaf, rho_root;
};

__device__ __host__ __forceinline__ bool node_violates(const Bounds& B, unsigned H, unsigned h,
                                                       uint64_t leaves, uint64_t b) {
  typedef unsigned __int128 u128;
  u128 cap = (u128)leaves * B.LB;
  if (H == 0) return (u128)b * 1000u > cap * B.tau_root;
  u128 lhs = (u128)b * 1000u * H;
  u128 up = cap * ((u128)B.tau_leaf * H - (u128)(B.tau_leaf - B.tau_root) * h);
  if (lhs > up) return true;
  u128 lo = cap * ((u128)B.rho_leaf * H + (u128)(B.rho_root - B.rho_leaf) * h);
  return lhs < lo;
}

// ---------------------------------------------------------------------------
// Warp-cooperative leaf decoder.
//
// A leaf is an 8-byte little-endian head followed by LEB128 deltas in bytes
// [8, used).  Each lane takes 16 bytes per 512-byte round (one coalesced
// 16-byte load).  A byte whose high bit is clear ends a code; a code spans at
// most two neighbouring lanes (it is at most 10 bytes long, and 16 bytes
// always contain a code end except in lane 0's 8 bytes after the head), so
// each lane first decodes the codes that end in its bytes, taking the partial
// code left by the previous lane through one shuffle.  Warp scans of the code
// counts and delta sums then give every element's index and value, and
// f(index, value) is called once per element by the lane that owns it.
// Returns the element count (warp-uniform).
// ---------------------------------------------------------------------------
template <class F>
__device__ __forceinline__ uint32_t warp_decode(const uint8_t* __restrict__ leaf, uint32_t used,
                                                F&& f) {
  if (used == 0) return 0;
  const unsigned lane = lane_id();
  const uint64_t head = *reinterpret_cast<const uint64_t*>(leaf);
  if (lane == 0) f(0u, head);
  uint32_t base_idx = 1;
  uint64_t base_val = head;
  uint64_t carry_val = 0;
  uint32_t carry_sh = 0;
  for (uint32_t r0 = 0; r0 < used; r0 += 512) {
    const uint32_t p0 = r0 + lane * 16u;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (p0 < used) v = __ldg(reinterpret_cast<const uint4*>(leaf + p0));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    const int b_lo = (p0 < 8u) ? (int)(8u - p0) : 0;
    const int b_hi = (used > p0) ? (int)min(16u, used - p0) : 0;
    uint32_t range = 0;
    if (b_hi > b_lo) range = ((b_hi == 16) ? 0xFFFFu : ((1u << b_hi) - 1u)) & ~((1u << b_lo) - 1u);
    // pass 1: codes that end in this lane, without the previous lane's part
    uint64_t d[16];
    uint32_t term = 0;
    uint64_t cur = 0;
    uint32_t sh = 0;
#pragma unroll
    for (int b = 0; b < 16; b++) {
      const uint32_t byte = (w[b >> 2] >> (8 * (b & 3))) & 0xFFu;
      const bool inr = (range >> b) & 1u;
      const bool t = inr && !(byte & 0x80u);
      if (inr) { cur |= (uint64_t)(byte & 0x7Fu) << sh; sh += 7; }
      d[b] = t ? cur : 0ull;
      if (t) { term |= 1u << b; cur = 0; sh = 0; }
    }
    // the partial code this lane leaves for the next one
    uint64_t prev_val = __shfl_up_sync(FULL, cur, 1);
    uint32_t prev_sh = __shfl_up_sync(FULL, sh, 1);
    if (lane == 0) { prev_val = carry_val; prev_sh = carry_sh; }
    // prepend the previous lane's partial code to this lane's first code
    if (term) {
      const int fb = __ffs(term) - 1;
#pragma unroll
      for (int b = 0; b < 16; b++)
        if (b == fb) d[b] = prev_val | (d[b] << prev_sh);
    } else {
      cur = prev_val | (cur << prev_sh);
      sh += prev_sh;
    }
    const uint32_t c = __popc(term);
    uint64_t s = 0;
#pragma unroll
    for (int b = 0; b < 16; b++) s += d[b];
    const uint32_t ci = warp_incl_scan(c);
    const uint64_t si = warp_incl_scan(s);
    uint32_t idx = base_idx + ci - c;
    uint64_t val = base_val + si - s;
#pragma unroll
    for (int b = 0; b < 16; b++) {
      if ((term >> b) & 1u) {
        val += d[b];
        f(idx, val);
        idx++;
      }
    }
    base_idx += __shfl_sync(FULL, ci, 31);
    base_val += __shfl_sync(FULL, si, 31);
    carry_val = __shfl_sync(FULL, cur, 31);
    carry_sh = __shfl_sync(FULL, sh, 31);
  }
  return base_idx;
}

// Encodes z[0..r) (shared memory) into buf (shared, zeroed, 8-byte aligned):
// head as 8 little-endian bytes, then one code per following delta.  Returns
// the used byte count (0 when r == 0).  The caller guarantees it fits.
__device__ __forceinline__ uint32_t warp_encode(const uint64_t* z, uint32_t r, uint8_t* buf) {
  if (r == 0) return 0;
  const unsigned lane = lane_id();
  if (lane == 0) *reinterpret_cast<uint64_t*>(buf) = z[0];
  uint32_t pos = 8;
  for (uint32_t c0 = 1; c0 < r; c0 += 32) {
    const uint32_t i = c0 + lane;
    uint64_t dd = 0;
    uint32_t len = 0;
    if (i < r) { dd = z[i] - z[i - 1]; len = leb_len(dd); }
    const uint32_t incl = warp_incl_scan(len);
    if (i < r) leb_put(buf + pos + incl - len, dd);
    pos += __shfl_sync(FULL, incl, 31);
  }
  __syncwarp();
  return pos;
}

// Byte cost of z[i] in a stream: 8 for the first element, else its code.
__device__ __forceinline__ uint32_t elem_cost(const uint64_t* z, uint32_t i) {
  return i == 0 ? 8u : leb_len(z[i] - z[i - 1]);
}

}  // namespace cpmadev
