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

// Warp wid of nw takes the contiguous share [r0, r1) of n work items, shares
// differing by at most one: a short list spreads over all warps instead of
// filling a few warps 32 items at a time.
__device__ __forceinline__ void warp_share(uint64_t n, uint64_t wid, uint64_t nw, uint64_t& r0,
                                           uint64_t& r1) {
  const uint64_t per = n / nw, extra = n % nw;
  r0 = wid * per + (wid < extra ? wid : extra);
  r1 = r0 + per + (wid < extra ? 1 : 0);
}

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
// whose head-index entry is <= x, else leaf 0.  Every entry is <= 2^64-1, so
// that key instead goes to the last non-empty leaf, whose index the head
// array keeps in its extra entry heads[L] (empty leaves after it must not
// take the key).
__device__ __forceinline__ uint64_t route_leaf(const uint64_t* __restrict__ heads, uint64_t L,
                                               uint64_t x) {
  if (x == KEY_MAX) return heads[L];
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
// WITH_POS: f(index, value, byte position of the last byte of the element's
// code) -- 7 for the head.
template <bool WITH_POS, class F>
__device__ __forceinline__ uint32_t warp_decode_impl(const uint8_t* __restrict__ leaf,
                                                     uint32_t used, F&& f) {
  if (used == 0) return 0;
  const unsigned lane = lane_id();
  const uint64_t head = *reinterpret_cast<const uint64_t*>(leaf);
  if (lane == 0) {
    if constexpr (WITH_POS) f(0u, head, 7u);
    else f(0u, head);
  }
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
        if constexpr (WITH_POS) f(idx, val, p0 + (uint32_t)b);
        else f(idx, val);
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

// The uncompressed format (8-byte cells, codec 1): lane l reads two cells of
// every 512-byte step; f sees the same (index, value[, last byte]) calls.
template <bool WITH_POS, class F>
__device__ __forceinline__ uint32_t warp_decode_cells(const uint8_t* __restrict__ leaf,
                                                      uint32_t used, F&& f) {
  const unsigned lane = lane_id();
  for (uint32_t p0 = lane * 16u; p0 < used; p0 += 512) {
    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(leaf + p0));
    const uint32_t i = p0 >> 3;
    if constexpr (WITH_POS) f(i, (uint64_t)v.x, p0 + 7u);
    else f(i, (uint64_t)v.x);
    if (p0 + 8 < used) {
      if constexpr (WITH_POS) f(i + 1, (uint64_t)v.y, p0 + 15u);
      else f(i + 1, (uint64_t)v.y);
    }
  }
  return used >> 3;
}

// raw: the leaf holds 8-byte cells (codec 1) instead of byte codes.
template <class F>
__device__ __forceinline__ uint32_t warp_decode(const uint8_t* __restrict__ leaf, uint32_t used,
                                                F&& f, bool raw = false) {
  return raw ? warp_decode_cells<false>(leaf, used, f) : warp_decode_impl<false>(leaf, used, f);
}

template <class F>
__device__ __forceinline__ uint32_t warp_decode_pos(const uint8_t* __restrict__ leaf,
                                                    uint32_t used, F&& f, bool raw = false) {
  return raw ? warp_decode_cells<true>(leaf, used, f) : warp_decode_impl<true>(leaf, used, f);
}

// Encodes z[0..r) (shared memory) into buf (shared, zeroed, 8-byte aligned):
// head as 8 little-endian bytes, then one code per following delta.  Returns
// the used byte count (0 when r == 0).  The caller guarantees it fits.
__device__ __forceinline__ uint32_t warp_encode(const uint64_t* z, uint32_t r, uint8_t* buf,
                                               bool raw = false) {
  if (r == 0) return 0;
  const unsigned lane = lane_id();
  if (raw) {  // codec 1: one 8-byte cell per element
    for (uint32_t i = lane; i < r; i += 32) reinterpret_cast<uint64_t*>(buf)[i] = z[i];
    __syncwarp();
    return 8 * r;
  }
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

// Byte cost of z[i] in a stream: 8 for the first element, else its code
// (8 for every element of the uncompressed format).
__device__ __forceinline__ uint32_t elem_cost(const uint64_t* z, uint32_t i, bool raw = false) {
  return (i == 0 || raw) ? 8u : leb_len(z[i] - z[i - 1]);
}

// ---------------------------------------------------------------------------
// Bit-parallel summary of the codes in one lane's 16 bytes of a leaf, for
// leaves whose codes are at most 4 bytes long (deltas < 2^28).
//
// Bytes outside [b_lo, b_hi) are zeroed; they then read as one-byte codes of
// value 0 and are dropped from the terminator mask.  For every byte the group
// index g (its position inside its code, counted within this lane) follows
// from the continuation flags of the 1, 2 and 3 bytes before it (funnel
// shifts across words); the sum of the codes' own bits is then
// sum_g 2^(7g) * (sum of the 7-bit values of the bytes with that g), four
// byte-class dot products per word (__vcmpeq4, __dp4a).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t bytemask4(uint32_t b4) {  // 4 bits -> 0x00/0xFF bytes
  return ((b4 * 0x00204081u) & 0x01010101u) * 0xFFu;
}
__device__ __forceinline__ uint32_t gather4(uint32_t x01) {  // bit 0 of each byte -> 4 bits
  return ((x01 * 0x01020408u) >> 24) & 0xFu;
}
__device__ __forceinline__ uint32_t compact7(uint32_t y) {  // 4 bytes' 7-bit groups, LSB first
  y &= 0x7F7F7F7Fu;
  return (y & 0x7Fu) | ((y >> 1) & 0x3F80u) | ((y >> 2) & 0x1FC000u) | ((y >> 3) & 0xFE00000u);
}
__device__ __forceinline__ uint32_t mask7(uint32_t groups) {  // low 7*groups bits, groups <= 4
  return groups >= 4 ? 0x0FFFFFFFu : ((1u << (7u * groups)) - 1u);
}
// 32-bit window of the 4*NW bytes x[] starting at byte s <= 4*NW (zeros past
// the end)
template <int NW = 4>
__device__ __forceinline__ uint32_t window32(const uint32_t (&x)[NW], uint32_t s) {
  static_assert(NW == 4 || NW == 8, "4 or 8 words per lane");
  const uint32_t i = s >> 2, sh = 8u * (s & 3u);
  uint32_t lo, hi;
  // explicit selects: an indexed form would put x[] in local memory
  if constexpr (NW == 4) {
    lo = i == 0 ? x[0] : i == 1 ? x[1] : i == 2 ? x[2] : i == 3 ? x[3] : 0u;
    hi = i == 0 ? x[1] : i == 1 ? x[2] : i == 2 ? x[3] : 0u;
  } else {
    lo = i == 0 ? x[0] : i == 1 ? x[1] : i == 2 ? x[2] : i == 3 ? x[3] : i == 4 ? x[4]
       : i == 5 ? x[5] : i == 6 ? x[6] : i == 7 ? x[7] : 0u;
    hi = i == 0 ? x[1] : i == 1 ? x[2] : i == 2 ? x[3] : i == 3 ? x[4] : i == 4 ? x[5]
       : i == 5 ? x[6] : i == 6 ? x[7] : 0u;
  }
  return __funnelshift_r(lo, hi, sh);
}

template <int NW>
struct LaneCodesN {
  uint32_t x[NW];     // the lane's bytes, zero outside [b_lo, b_hi)
  uint32_t term;      // bit b: byte b ends a code
  uint32_t D;         // own bits of the codes ending here (first one without carry)
  uint32_t W;         // sum over those codes of (index among them) * own bits
  uint32_t first_own; // own bits of the first code ending here
  uint32_t first_len; // its own byte count
  uint32_t tail;      // bits of the partial code after the last terminator
  uint32_t tail_sh;   // 7 * its byte count
  bool bad;           // a code longer than 4 bytes, or no terminator
};

using LaneCodes = LaneCodesN<4>;

// NW words (4*NW <= 32 bytes) per lane; b_lo, b_hi in bytes of the lane.
template <bool WANT_W, int NW = 4>
__device__ __forceinline__ void lane_codes(const uint32_t (&w)[NW], int b_lo, int b_hi,
                                           LaneCodesN<NW>& L) {
  uint32_t range = 0;
  if (b_hi > b_lo)
    range = ((b_hi >= 32) ? 0xFFFFFFFFu : ((1u << b_hi) - 1u)) & ~((1u << b_lo) - 1u);
  uint32_t cb[NW], tb[NW];
#pragma unroll
  for (int q = 0; q < NW; q++) {
    const uint32_t rm = bytemask4((range >> (4 * q)) & 0xFu);
    L.x[q] = w[q] & rm;
    cb[q] = (L.x[q] >> 7) & 0x01010101u;
    tb[q] = (rm & 0x01010101u) & ~cb[q];
  }
  L.term = 0;
#pragma unroll
  for (int q = 0; q < NW; q++) L.term |= gather4(tb[q]) << (4 * q);
  // Byte b's 7 payload bits sit at group g_b = (continuation bytes right
  // before it, at most 3) of its code.  With 0/1 byte masks m_i of g_b == i,
  // dp4a with multipliers m0 + 128 m1 and m2 + 128 m3 gives S0 + (S1 << 7)
  // and S2 + (S3 << 7) directly, S_i the sum of the group-i payloads.
  uint32_t S01 = 0, S23 = 0, W0 = 0, W1 = 0, W2 = 0, W3 = 0;
  uint32_t badm = 0, base = 0;
#pragma unroll
  for (int q = 0; q < NW; q++) {
    const uint32_t prev = q ? cb[q - 1] : 0u;
    const uint32_t p1 = __funnelshift_l(prev, cb[q], 8);
    const uint32_t p2 = __funnelshift_l(prev, cb[q], 16);
    const uint32_t p3 = __funnelshift_l(prev, cb[q], 24);
    const uint32_t a12 = p1 & p2, a123 = a12 & p3;
    badm |= a123 & cb[q];
    const uint32_t v = L.x[q] & 0x7F7F7F7Fu;
    const uint32_t m0 = ~p1 & 0x01010101u, m1 = p1 ^ a12, m2 = a12 ^ a123, m3 = a123;
    S01 = __dp4a(v, m0 | (m1 << 7), S01);
    S23 = __dp4a(v, m2 | (m3 << 7), S23);
    if constexpr (WANT_W) {
      // terminators before each byte of the word (bytes), plus the earlier words'
      const uint32_t lidx = tb[q] * 0x01010100u + base * 0x01010101u;
      W0 = __dp4a(v & (m0 * 0x7Fu), lidx, W0);
      W1 = __dp4a(v & (m1 * 0x7Fu), lidx, W1);
      W2 = __dp4a(v & (m2 * 0x7Fu), lidx, W2);
      W3 = __dp4a(v & (m3 * 0x7Fu), lidx, W3);
      base += __popc(tb[q]);
    }
  }
  const uint32_t Dall = S01 + (S23 << 14);
  L.bad = badm != 0 || (range != 0 && L.term == 0);
  L.tail = 0;
  L.tail_sh = 0;
  L.first_own = 0;
  L.first_len = 0;
  L.D = 0;
  L.W = 0;
  if (L.term) {
    const uint32_t lt = 31u - (uint32_t)__clz(L.term);
    const uint32_t tl = (uint32_t)b_hi - 1u - lt;
    L.tail = compact7(window32<NW>(L.x, lt + 1u));
    L.tail_sh = 7u * tl;
    const uint32_t ft = (uint32_t)__ffs(L.term) - 1u;
    L.first_len = ft + 1u - (uint32_t)b_lo;
    L.first_own = compact7(b_lo == 0 ? L.x[0] : L.x[2]) & mask7(L.first_len);
    L.D = Dall - L.tail;
    if constexpr (WANT_W) {
      const uint32_t c = __popc(L.term);
      L.W = (W0 + (W1 << 7) + (W2 << 14) + (W3 << 21)) - c * L.tail;
    }
  }
}

// ---------------------------------------------------------------------------
// Thread-per-leaf sum of byte-code leaves (codec 0): the sum (mod 2^64) of
// the elements of the leaf at leafp with u >= 8 used bytes.  One thread walks
// the leaf eight bytes at a time keeping the running element value val and
// the running sum s.  Inside the eight bytes everything is 32-bit: each byte
// adds its payload times 128^(bytes before it in its code) to acc, and acc is
// not cleared at a terminator, so at the k-th terminator of the group acc_k
// holds the bits of every code closed so far in the group (plus the open code
// carried in): the element closed there is val + acc_k.  The group adds T *
// val + sum_k acc_k to s (T terminators), val moves on by the acc of its last
// terminator and acc keeps only the open code's bits.  With codes of at most 4
// bytes at most 11 bytes of payload feed one group and sum_k acc_k < 9 * 2^28
// fits in 32 bits.  Bytes after u are read as zero: each of them acts as a
// terminator adding the last value again, which is taken off at the end.  A
// code of more than 4 bytes overflows the 32-bit code accumulator; such a
// leaf is summed again exactly, byte by byte.
__device__ __forceinline__ void leaf_sum_group(uint32_t wa, uint32_t wb, uint64_t& val,
                                               uint64_t& s, uint32_t& acc, uint32_t& pw,
                                               uint32_t& pwor) {
  const uint32_t pa = wa & 0x7F7F7F7Fu, pb = wb & 0x7F7F7F7Fu;
  uint32_t ss = 0, r = 0;
#pragma unroll
  for (int b = 0; b < 8; b++) {
    const uint32_t wv = b < 4 ? wa : wb, pv = b < 4 ? pa : pb;
    acc += __byte_perm(pv, 0u, 0x4440u + (uint32_t)(b & 3)) * pw;
    const bool term = (wv & (0x80u << (8 * (b & 3)))) == 0u;
    pwor |= pw;
    ss += term ? acc : 0u;
    r = term ? acc : r;
    pw = term ? 1u : pw << 7;
  }
  const uint32_t T = __popc(~wa & 0x80808080u) + __popc(~wb & 0x80808080u);
  s += (uint64_t)T * val + ss;
  val += r;
  acc -= r;
}

// Bytes of w past u - p0 cleared (the leaf's zero padding, read as such).
__device__ __forceinline__ void mask_past(uint32_t (&w)[4], uint32_t p0, uint32_t u) {
  if (p0 + 16u > u) {
    const uint32_t keep = u > p0 ? (1u << (u - p0)) - 1u : 0u;
#pragma unroll
    for (int i = 0; i < 4; i++) w[i] &= bytemask4((keep >> (4 * i)) & 0xFu);
  }
}

__device__ __forceinline__ uint64_t thread_leaf_sum(const uint8_t* __restrict__ leafp, uint32_t u) {
  // 32 bytes (one sector) per step: both halves are loaded before either is
  // decoded, so each sector is requested once
  uint4 v = *reinterpret_cast<const uint4*>(leafp);
  uint4 v2 = u > 16u ? *reinterpret_cast<const uint4*>(leafp + 16) : make_uint4(0u, 0u, 0u, 0u);
  uint32_t w[4] = {v.x, v.y, v.z, v.w};
  uint64_t val = (uint64_t)w[0] | ((uint64_t)w[1] << 32), s = val;
  uint32_t acc = 0, pw = 1, pwor = 0;
  for (uint32_t p0 = 0; p0 < u; p0 += 32) {
    if (p0) {
      v = *reinterpret_cast<const uint4*>(leafp + p0);
      v2 = p0 + 16u < u ? *reinterpret_cast<const uint4*>(leafp + p0 + 16) : make_uint4(0u, 0u, 0u, 0u);
      w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    }
    mask_past(w, p0, u);
    if (p0) leaf_sum_group(w[0], w[1], val, s, acc, pw, pwor);  // bytes 0-7 are the head
    leaf_sum_group(w[2], w[3], val, s, acc, pw, pwor);
    if (p0 + 16u < u) {
      uint32_t w2[4] = {v2.x, v2.y, v2.z, v2.w};
      mask_past(w2, p0 + 16u, u);
      leaf_sum_group(w2[0], w2[1], val, s, acc, pw, pwor);
      leaf_sum_group(w2[2], w2[3], val, s, acc, pw, pwor);
    }
  }
  s -= (uint64_t)(((u + 15u) & ~15u) - u) * val;
  if (pwor >= (1u << 28)) {  // a long code: exact 64-bit decode
    val = *reinterpret_cast<const uint64_t*>(leafp);
    s = val;
    uint64_t a64 = 0;
    uint32_t sh = 0;
    for (uint32_t p = 8; p < u; p++) {
      const uint32_t c = leafp[p];
      if (sh < 64) a64 |= (uint64_t)(c & 0x7Fu) << sh;
      if (c & 0x80u) {
        sh += 7;
      } else {
        val += a64;
        s += val;
        a64 = 0;
        sh = 0;
      }
    }
  }
  return s;
}

// Is x an element of the byte-code leaf at leafp (u used bytes)?  One
// thread decodes the leaf from its head, 16 bytes at a time, until the
// running value passes x.  The bytes are taken eight at a time as in
// thread_leaf_sum: the element closed at a terminator is val + acc with a
// 32-bit acc, so it equals x exactly when acc equals x - val (no element of
// the group can when x - val >= 2^32, since acc stays below 9 * 2^28).
// Zero bytes after u repeat the last value, which is an element.  A leaf
// with a code over 4 bytes is decoded again exactly, byte by byte.
__device__ __forceinline__ void leaf_has_group(uint32_t wa, uint32_t wb, uint64_t x,
                                               uint64_t& val, bool& found, uint32_t& acc,
                                               uint32_t& pw, uint32_t& pwor) {
  const uint64_t dx = x - val;  // wraps past 2^32 once val > x: no match then
  const uint32_t d32 = dx > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)dx;
  const uint32_t pa = wa & 0x7F7F7F7Fu, pb = wb & 0x7F7F7F7Fu;
  uint32_t r = 0;
#pragma unroll
  for (int b = 0; b < 8; b++) {
    const uint32_t wv = b < 4 ? wa : wb, pv = b < 4 ? pa : pb;
    acc += __byte_perm(pv, 0u, 0x4440u + (uint32_t)(b & 3)) * pw;
    const bool term = (wv & (0x80u << (8 * (b & 3)))) == 0u;
    pwor |= pw;
    found |= term && acc == d32;
    r = term ? acc : r;
    pw = term ? 1u : pw << 7;
  }
  val += r;
  acc -= r;
}

__device__ __forceinline__ bool thread_leaf_has(const uint8_t* __restrict__ leafp, uint32_t u,
                                                uint64_t x) {
  if (u == 0) return false;
  uint4 v = *reinterpret_cast<const uint4*>(leafp);
  uint32_t w[4] = {v.x, v.y, v.z, v.w};
  uint64_t val = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
  if (x <= val) return x == val;
  bool found = false;
  uint32_t acc = 0, pw = 1, pwor = 0;
  for (uint32_t p0 = 0; p0 < u && val < x; p0 += 16) {
    if (p0) {
      v = *reinterpret_cast<const uint4*>(leafp + p0);
      w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    }
    mask_past(w, p0, u);
    if (p0) leaf_has_group(w[0], w[1], x, val, found, acc, pw, pwor);  // bytes 0-7: the head
    leaf_has_group(w[2], w[3], x, val, found, acc, pw, pwor);
  }
  if (pwor >= (1u << 28)) {  // a long code: exact 64-bit decode
    val = *reinterpret_cast<const uint64_t*>(leafp);
    found = false;
    uint64_t a64 = 0;
    uint32_t sh = 0;
    for (uint32_t p = 8; p < u && val < x; p++) {
      const uint32_t c = leafp[p];
      if (sh < 64) a64 |= (uint64_t)(c & 0x7Fu) << sh;
      if (c & 0x80u) {
        sh += 7;
      } else {
        val += a64;
        found |= val == x;
        a64 = 0;
        sh = 0;
      }
    }
  }
  return found;
}

// Sum (mod 2^64), count and used bytes of the byte-code leaves [j0, j1), one
// leaf per lane at a time, added to the calling lane's partials.
__device__ __forceinline__ void thread_span_sum(const uint8_t* __restrict__ data,
                                                const uint32_t* __restrict__ used,
                                                const uint32_t* __restrict__ cnt, uint32_t LB,
                                                uint64_t j0, uint64_t j1, uint64_t& s,
                                                uint64_t& c, unsigned long long& nbytes) {
  for (uint64_t j = j0 + lane_id(); j < j1; j += 32) {
    const uint32_t u = min(used[j], LB);
    if (u == 0) continue;
    s += thread_leaf_sum(data + j * LB, u);
    c += cnt[j];
    nbytes += u;
  }
}

// ---------------------------------------------------------------------------
// Sum (mod 2^64) and count of every element of the leaves [j0, j1), added to
// the calling lane's partials (the caller reduces them over the warp).
//
// Leaves are taken 32 at a time.  Their used bytes are cut into 16-byte
// chunks and the warp takes 32 chunks per step, so no lane idles on the zero
// padding of a leaf.  The sum of a leaf with m elements, head h and deltas
// d_1..d_{m-1} is m*h + sum_c (m - c) d_c; a chunk holding the codes c =
// 1+B .. B+n (B = codes earlier in its leaf, a segmented warp scan) adds
// (m - 1 - B) * D - W with D = sum of its deltas and W = sum of lidx * delta
// (lidx = position among the chunk's codes).  The code a chunk starts in the
// middle of is completed with the previous chunk's partial bits (one
// shuffle).  Chunks are summarised bit-parallel (lane_codes), valid while
// every code is at most 4 bytes (deltas < 2^28); a window of leaves with a
// longer code is summed again by the general decoder instead.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_span_sum(const uint8_t* __restrict__ data,
                                              const uint32_t* __restrict__ used,
                                              const uint32_t* __restrict__ cnt, uint32_t LB,
                                              uint64_t j0, uint64_t j1, uint64_t& acc,
                                              uint64_t& cacc, ull& nbytes, bool raw = false) {
  const unsigned lane = lane_id();
  if (raw) {
    // codec 1: add the cells.  The used 16-byte chunks of 32 leaves are
    // numbered by a prefix sum and spread over the lanes, four loads in
    // flight per lane.
    for (uint64_t w0 = j0; w0 < j1; w0 += 32) {
      const uint64_t jj = w0 + lane;
      const uint32_t u_i = jj < j1 ? min(__ldg(used + jj), LB) : 0u;
      cacc += jj < j1 ? __ldg(cnt + jj) : 0u;
      nbytes += u_i;
      const uint32_t nc_i = (u_i + 15u) >> 4;
      const uint32_t cinc = warp_incl_scan(nc_i);
      const uint32_t NC = __shfl_sync(FULL, cinc, 31);
      for (uint32_t g0 = 0; g0 < NC; g0 += 128) {
        ulonglong2 v[4];
        uint32_t lim[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const uint32_t ci = g0 + 32u * q + lane;
          uint32_t li = 0;
#pragma unroll
          for (int stp = 16; stp >= 1; stp >>= 1) {
            const uint32_t cv = __shfl_sync(FULL, cinc, li + stp - 1);
            if (cv <= ci) li += stp;
          }
          const uint32_t lis = min(li, 31u);
          const uint32_t cstart = __shfl_sync(FULL, cinc, lis) - __shfl_sync(FULL, nc_i, lis);
          const uint32_t u = __shfl_sync(FULL, u_i, lis);
          const uint32_t p0 = (ci - cstart) * 16u;
          v[q] = make_ulonglong2(0ull, 0ull);
          lim[q] = 0;
          if (ci < NC) {
            v[q] = __ldg(reinterpret_cast<const ulonglong2*>(data + (w0 + lis) * LB + p0));
            lim[q] = u - p0;  // used bytes from this chunk on: 8 or at least 16
          }
        }
#pragma unroll
        for (int q = 0; q < 4; q++) acc += v[q].x * (lim[q] >= 8) + v[q].y * (lim[q] >= 16);
      }
    }
    return;
  }
  for (uint64_t w0 = j0; w0 < j1; w0 += 32) {
    const uint64_t jj = w0 + lane;
    const bool lv = jj < j1;
    const uint32_t u_i = lv ? min(__ldg(used + jj), LB) : 0u;
    const uint32_t m_i = lv ? __ldg(cnt + jj) : 0u;
    cacc += m_i;
    nbytes += u_i;
    const uint32_t nc_i = (u_i + 15u) >> 4;
    const uint32_t cinc = warp_incl_scan(nc_i);
    const uint32_t NC = __shfl_sync(FULL, cinc, 31);
    uint64_t wacc = 0;
    bool bad = false;
    uint32_t cont_li = 0xFFFFFFFFu, cont_cnt = 0, cont_val = 0, cont_sh = 0;
    // Chunk ci of the 32 leaves: its leaf slot (the number of leaves whose
    // chunks end at or before ci), that leaf's first chunk, used bytes and
    // count; the 16 bytes are loaded one step ahead of their use so the load
    // of the next step overlaps the decode of this one.
    struct Chunk { uint32_t li, lis, cstart, u, m; uint4 v; };
    auto locate = [&](uint32_t g0, Chunk& k) {
      const uint32_t ci = g0 + lane;
      uint32_t li = 0;
#pragma unroll
      for (int stp = 16; stp >= 1; stp >>= 1) {
        const uint32_t v = __shfl_sync(FULL, cinc, li + stp - 1);
        if (v <= ci) li += stp;
      }
      k.li = li;
      k.lis = min(li, 31u);
      k.cstart = __shfl_sync(FULL, cinc, k.lis) - __shfl_sync(FULL, nc_i, k.lis);
      k.u = __shfl_sync(FULL, u_i, k.lis);
      k.m = __shfl_sync(FULL, m_i, k.lis);
      k.v = make_uint4(0u, 0u, 0u, 0u);
      if (ci < NC)
        k.v = __ldg(reinterpret_cast<const uint4*>(data + (w0 + k.lis) * LB +
                                                    (ci - k.cstart) * 16u));
    };
    Chunk cur, nxt;
    if (NC) locate(0, cur);
    for (uint32_t g0 = 0; g0 < NC; g0 += 32) {
      if (g0 + 32 < NC) locate(g0 + 32, nxt);
      const uint32_t ci = g0 + lane;
      const bool act = ci < NC;
      const uint32_t li = cur.li, cstart = cur.cstart, u = cur.u, m = cur.m;
      const uint32_t cw = ci - cstart;
      const uint32_t p0 = cw * 16u;
      const uint32_t w[4] = {cur.v.x, cur.v.y, cur.v.z, cur.v.w};
      const int b_lo = (cw == 0) ? 8 : 0;
      const int b_hi = act ? (int)min(16u, u - p0) : 0;
      LaneCodes lc;
      lane_codes<true>(w, b_lo, b_hi, lc);
      bad |= lc.bad;
      // the partial code left by the previous chunk of the same leaf
      const uint32_t prev_li = __shfl_up_sync(FULL, li, 1);
      uint32_t pv = __shfl_up_sync(FULL, lc.tail, 1);
      uint32_t ps = __shfl_up_sync(FULL, lc.tail_sh, 1);
      if (lane == 0 || prev_li != li) {
        if (lane == 0 && cont_li == li && cw > 0) { pv = cont_val; ps = cont_sh; }
        else { pv = 0; ps = 0; }
      }
      const uint32_t term = lc.term;
      uint32_t D = 0;
      const uint32_t W = lc.W;
      if (term) {
        if (ps / 7u + lc.first_len > 4u) bad = true;
        D = lc.D - lc.first_own + pv + (lc.first_own << ps);
      }
      // codes of this leaf in earlier chunks (segmented scan)
      const uint32_t c = __popc(term);
      const uint32_t incl = warp_incl_scan(c);
      const uint32_t excl = incl - c;
      const bool started_before = cstart < g0;
      const uint32_t seg_lane = started_before ? 0u : cstart - g0;
      const uint32_t B = excl - __shfl_sync(FULL, excl, seg_lane & 31u) +
                         (started_before ? cont_cnt : 0u);
      if (act) {
        uint64_t contrib = (uint64_t)(m - 1u - B) * D - W;
        if (cw == 0) contrib += (uint64_t)m * ((uint64_t)w[0] | ((uint64_t)w[1] << 32));
        wacc += contrib;
      }
      cont_li = __shfl_sync(FULL, li, 31);
      cont_cnt = __shfl_sync(FULL, B + c, 31);
      cont_val = __shfl_sync(FULL, lc.tail, 31);
      cont_sh = __shfl_sync(FULL, lc.tail_sh, 31);
      cur = nxt;
    }
    if (__any_sync(FULL, bad)) {
      const uint64_t je = min(w0 + 32, j1);
      for (uint64_t q = w0; q < je; q++)
        warp_decode(data + q * LB, min(__ldg(used + q), LB), [&](uint32_t, uint64_t val) { acc += val; });
    } else {
      acc += wacc;
    }
  }
}

}  // namespace cpmadev
