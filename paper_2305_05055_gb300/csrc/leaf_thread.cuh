// Thread-granular insert of a few keys into one leaf of byte codes (Sec. 4
// batch merge, Sec. 5 leaf format: an 8-byte little-endian head, then the
// deltas to the following keys as unsigned LEB128 codes, packed left, zero
// bytes after the used ones).
//
// One thread owns one leaf.  Pass A sums the leaf 16 bytes at a time with
// word-parallel arithmetic (each byte's position inside its code from the
// continuation flags of the bytes before it, then two dot products per word
// with byte weights 1 / 128 and 2^14 / 2^21), recording for every key of
// the slice the chunk it lands in; those chunks are then decoded byte by
// byte to place each key: before the head (a new head), inside the gap that one code spans
// (the code is split), or after the last element (appended); a key equal to
// an element or to the slice key before it is skipped.  Keys sharing a gap
// form one edit: old bytes [os, oe) replaced by nl new bytes.  Every edit of
// an insert grows or keeps the size (a split code never needs more bytes
// than its two parts), so pass B rewrites the leaf in place from the end
// backwards, 16 bytes at a time: each destination chunk gathers the old
// bytes that land in it (one shift per segment between edits; a chunk wholly
// inside the segment after the last edit is one shifted 16-byte read) and is
// stored whole, before the edits' own bytes are written.  Every read of pass
// B is of a chunk at or below the one being written, so it sees old bytes
// (a delete shrinks: forward, reads at or above).
//
// The functions are __host__ __device__ so that the same code can be run on
// the host.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define LT_HD __host__ __device__ __forceinline__
#else
#define LT_HD inline
#endif

namespace leafthr {

constexpr uint32_t kKeys = 4;  // slice keys per leaf on this path

// key record kinds
constexpr uint32_t kGap = 0;    // inside the gap of the code [cs, ce)
constexpr uint32_t kHead = 1;   // before the head
constexpr uint32_t kAfter = 2;  // after the last element
constexpr uint32_t kSkip = 3;   // a repeat of the slice key before it
constexpr uint32_t kChunk = 4;  // (pass A, step 1) in a code ending in the chunk at cs
constexpr uint32_t kHit = 5;    // equal to an element: the code [cs, ce) is its own

// kinds an insert leaves alone
LT_HD bool no_insert(uint32_t kind) { return kind == kSkip || kind == kHit; }

// results
constexpr uint32_t kUnchanged = 0;  // every key present: nothing written
constexpr uint32_t kWritten = 1;    // leaf rewritten in place
constexpr uint32_t kTooBig = 2;     // result exceeds the leaf: nothing written
constexpr uint32_t kLongCode = 3;   // a code of more than 4 bytes: nothing written

struct Result {
  uint32_t nb;       // new used bytes
  uint32_t newc;     // new element count
  uint32_t added;    // bit q: slice key q was added
  uint32_t wlo, whi; // byte range rewritten (kWritten)
  uint32_t E;        // edits
  uint32_t maxcode;  // longest code the edits write (bytes)
  uint64_t newhead;
};

LT_HD uint32_t fshr(uint32_t lo, uint32_t hi, uint32_t sh) {  // low word of (hi:lo) >> sh, sh < 32
#if defined(__CUDA_ARCH__)
  return __funnelshift_r(lo, hi, sh);
#else
  return sh ? (lo >> sh) | (hi << (32u - sh)) : lo;
#endif
}

LT_HD uint32_t fshl(uint32_t lo, uint32_t hi, uint32_t sh) {  // high word of (hi:lo) << sh, 0 < sh < 32
#if defined(__CUDA_ARCH__)
  return __funnelshift_l(lo, hi, sh);
#else
  return (hi << sh) | (lo >> (32u - sh));
#endif
}

LT_HD uint32_t dp4a(uint32_t a, uint32_t b, uint32_t c) {  // c + sum of the four byte products
#if defined(__CUDA_ARCH__)
  return __dp4a(a, b, c);
#else
  for (int i = 0; i < 4; i++) c += ((a >> (8 * i)) & 0xFFu) * ((b >> (8 * i)) & 0xFFu);
  return c;
#endif
}

LT_HD uint32_t clz32(uint32_t x) {  // leading zeros, 32 for x == 0
#if defined(__CUDA_ARCH__)
  return (uint32_t)__clz((int)x);
#else
  return x ? (uint32_t)__builtin_clz(x) : 32u;
#endif
}

LT_HD void ld16(const uint8_t* p, uint32_t (&w)[4]) {
#if defined(__CUDA_ARCH__)
  const uint4 v = *reinterpret_cast<const uint4*>(p);
  w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
#else
  memcpy(w, p, 16);
#endif
}

LT_HD void st16(uint8_t* p, const uint32_t (&w)[4]) {
#if defined(__CUDA_ARCH__)
  *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
#else
  memcpy(p, w, 16);
#endif
}

LT_HD uint32_t popc(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return (uint32_t)__popc(x);
#else
  return (uint32_t)__builtin_popcount(x);
#endif
}

LT_HD uint32_t bmask4(uint32_t b4) {  // 4 bits -> 0x00 / 0xFF bytes
  return ((b4 * 0x00204081u) & 0x01010101u) * 0xFFu;
}

LT_HD uint32_t leb_bytes(uint64_t d) {  // unsigned LEB128 length of d
#if defined(__CUDA_ARCH__)
  const uint32_t bl = 64u - (uint32_t)__clzll((long long)(d | 1ull));
#else
  const uint32_t bl = 64u - (uint32_t)__builtin_clzll(d | 1ull);
#endif
  return (bl + 6u) / 7u;
}

LT_HD uint32_t leb_write(uint8_t* p, uint64_t d) {
  uint32_t n = 0;
  while (d >= 128u) { p[n++] = (uint8_t)(d | 0x80u); d >>= 7; }
  p[n++] = (uint8_t)d;
  return n;
}

LT_HD uint64_t pick(const uint64_t (&y)[kKeys], uint32_t q) {
  static_assert(kKeys == 4, "four slice keys");
  return q == 0 ? y[0] : q == 1 ? y[1] : q == 2 ? y[2] : y[3];
}

// Per-thread scratch: arrays of kKeys entries at stride `rs` (key records and
// edits), so that a block's threads index shared memory without conflicts.
struct Scratch {
  uint32_t* rpos;   // key q: cs | ce << 12 | kind << 24
  uint64_t* rval;   // key q: successor value (kGap), the head (kHead), the last value (kAfter)
  uint32_t* rcode;  // key q: value of the code [cs, ce) (kGap)
  uint32_t* epos;   // edit e: os | oe << 12 | kind << 24
  int32_t* esa;     // edit e: total size change of edits 0..e
  uint32_t* ekey;   // edit e: first key | end key << 8 | nl << 16
  uint32_t rs;
};

LT_HD uint32_t byte_of(uint32_t v, int i) {  // byte i of v, zero-extended
#if defined(__CUDA_ARCH__)
  return __byte_perm(v, 0u, 0x4440u + (uint32_t)i);
#else
  return (v >> (8 * i)) & 0xFFu;
#endif
}

// Pass A, step 1: the byte weights of one 4-byte word of codes.  cb, p1, p2
// carry the flags of the word before (bit 7 of each byte): cb = the byte is
// a continuation byte, p1 = the byte before it is one (its position g in its
// code is >= 1), p2 = g >= 2.  A byte at position g weighs 128^g in the
// value of its code, so the sum of the (partial) codes in the word is
// dp4a(pay, w01) + 2^14 dp4a(pay, w23) with w01 = 1 / 128 for g = 0 / 1 and
// w23 = 1 / 128 for g = 2 / 3 (0 elsewhere).  lc collects continuation
// bytes at position >= 3: a code of more than 4 bytes, which the 32-bit
// arithmetic does not cover.
LT_HD uint32_t word_sum(uint32_t w, uint32_t& cb, uint32_t& p1, uint32_t& p2, uint32_t& lc,
                        uint32_t& pay, uint32_t& w01, uint32_t& w23) {
  const uint32_t c = w & 0x80808080u;
  const uint32_t q1 = fshl(cb, c, 8);
  const uint32_t q2 = q1 & fshl(p1, q1, 8);
  const uint32_t q3 = q2 & fshl(p2, q2, 8);
  lc |= q3 & c;
  pay = w & 0x7F7F7F7Fu;
  w01 = ((q1 ^ 0x80808080u) >> 7) | (q1 ^ q2);
  w23 = ((q2 ^ q3) >> 7) | q3;
  cb = c;
  p1 = q1;
  p2 = q2;
  return dp4a(pay, w01, 0u) + (dp4a(pay, w23, 0u) << 14);
}

// Pass A, step 2: the codes of the chunk at p0 take keys q..q1-1 (all of
// them: their values lie between the element before the chunk and the last
// element completed in it).  Decode the chunk byte by byte from the state it
// was entered with (val0: the element before it; carry0, g0: the bits and
// byte count of the code open at p0) and give each key its gap.
LT_HD void place_in_chunk(const uint8_t* leafp, uint32_t uold, uint32_t p0, uint64_t val0,
                          uint32_t carry0, uint32_t g0, const uint64_t (&y)[kKeys], uint32_t q,
                          uint32_t q1, const Scratch& S) {
  uint32_t w[4];
  ld16(leafp + p0, w);
  if (p0 + 16u > uold) {
    const uint32_t keep = (1u << (uold - p0)) - 1u;
#pragma unroll
    for (int i = 0; i < 4; i++) w[i] &= bmask4((keep >> (4 * i)) & 0xFu);
  }
  uint64_t val = val0;
  uint32_t acc = carry0, sh = 7u * g0, cs = p0 == 0 ? 8u : p0 - g0;
  uint64_t ycur = pick(y, q);
  const int b0 = p0 == 0 ? 8 : 0;
#pragma unroll
  for (int b = 0; b < 16; b++) {  // unrolled: w[] stays in registers
    if (b < b0) continue;
    const uint32_t c = byte_of(w[b >> 2], b & 3);
    acc |= (c & 0x7Fu) << sh;
    if (c & 0x80u) {
      sh += 7u;
      continue;
    }
    val += acc;
    const uint32_t ce = p0 + (uint32_t)b + 1u;
    while (ycur <= val) {  // this code's gap (val - acc, val] takes the keys up to val
      const bool rep = q > 0 && pick(y, q - 1) == ycur;
      const uint32_t kind = rep ? kSkip : ycur == val ? kHit : kGap;
      S.rpos[q * S.rs] = cs | (ce << 12) | (kind << 24);
      S.rval[q * S.rs] = val;
      S.rcode[q * S.rs] = acc;
      if (++q >= q1) return;
      ycur = pick(y, q);
    }
    acc = 0u;
    sh = 0u;
    cs = ce;
  }
}

// The 16 bytes at byte offset `src` (which may be negative: missing bytes
// read as zero) of the old leaf, masked to chunk bytes [a, b), OR-ed into r.
LT_HD void gather(const uint8_t* leafp, uint32_t LB, int32_t src, uint32_t a, uint32_t b,
                  uint32_t (&r)[4]) {
  const int32_t A = (src >> 4) * 16;  // floor to 16
  const uint32_t d = (uint32_t)(src - A);
  uint32_t W[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  if (A >= 0) {
    uint32_t t[4];
    ld16(leafp + A, t);
    W[0] = t[0]; W[1] = t[1]; W[2] = t[2]; W[3] = t[3];
  }
  if (d != 0u && A + 16 >= 0 && (uint32_t)(A + 16) < LB) {
    uint32_t t[4];
    ld16(leafp + A + 16, t);
    W[4] = t[0]; W[5] = t[1]; W[6] = t[2]; W[7] = t[3];
  }
  const uint32_t q = d >> 2, s8 = 8u * (d & 3u);
  uint32_t V[5];
#pragma unroll
  for (int i = 0; i < 5; i++)
    V[i] = q == 0 ? W[i] : q == 1 ? W[i + 1] : q == 2 ? W[i + 2] : W[i + 3];
  const uint32_t m16 = ((b >= 16u ? 0xFFFFu : ((1u << b) - 1u)) & ~((1u << a) - 1u));
#pragma unroll
  for (int i = 0; i < 4; i++) r[i] |= fshr(V[i], V[i + 1], s8) & bmask4((m16 >> (4 * i)) & 0xFu);
}

// Pass B: destination bounds [dlo, dhi) and shift sa of segment e (-1 .. E-1):
// the old bytes [oe_e, os_{e+1}) moved by sa_e (oe_{-1} = 0, os_E = uold,
// sa_{-1} = 0).
LT_HD void seg_bounds(const Scratch& S, uint32_t E, uint32_t uold, uint32_t os0, int e,
                      int32_t& dlo, int32_t& dhi, int32_t& sa) {
  uint32_t lo = 0u, hi = os0;
  sa = 0;
  if (e >= 0) {
    lo = (S.epos[e * S.rs] >> 12) & 0xFFFu;
    hi = (e + 1 < (int)E) ? (S.epos[(e + 1) * S.rs] & 0xFFFu) : uold;
    sa = S.esa[e * S.rs];
  }
  dlo = (int32_t)lo + sa;
  dhi = (int32_t)hi + sa;
}

// Pass A: a record for every slice key (kind, code bytes, values; see
// Scratch).  Returns kWritten when every key is placed (nothing is written),
// else kLongCode (the leaf holds a code of more than 4 bytes).  head
// receives the leaf's first element.
constexpr uint32_t kPlaced = kWritten;
LT_HD uint32_t pass_a(const uint8_t* leafp, uint32_t uold, uint32_t m, const uint64_t (&y)[kKeys],
                      uint32_t s, const Scratch& S, uint64_t& head) {
  uint32_t w[4];
  ld16(leafp, w);
  head = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
  uint32_t k = 0;
  while (k < s && pick(y, k) <= head) {
    const uint64_t x = pick(y, k);
    const bool rep = k > 0 && pick(y, k - 1) == x;
    const uint32_t kind = rep ? kSkip : x == head ? kHit : kHead;
    S.rpos[k * S.rs] = 0u | (8u << 12) | (kind << 24);
    S.rval[k * S.rs] = head;
    S.rcode[k * S.rs] = 0u;
    k++;
  }
  // step 1: chunk sums over the whole leaf (a warp's threads then take the
  // same number of steps); every key gets the chunk (p0, entry state) of
  // the code it falls in, or stays for the end
  uint64_t ycur = k < s ? pick(y, k) : ~0ull;
  uint64_t val = head;
  uint32_t carry = 0, lc = 0, cb = 0, p1 = 0, p2 = 0;
  for (uint32_t p0 = 0; p0 < uold; p0 += 16) {
    if (p0) ld16(leafp + p0, w);  // bytes past the used ones are zero (packed left)
    const uint32_t cb_in = cb;    // flags of the last word before p0
    uint32_t tsum = 0, pay = 0, w01 = 0, w23 = 0;
    if (p0) {
      tsum += word_sum(w[0], cb, p1, p2, lc, pay, w01, w23);
      tsum += word_sum(w[1], cb, p1, p2, lc, pay, w01, w23);
    }
    tsum += word_sum(w[2], cb, p1, p2, lc, pay, w01, w23);
    tsum += word_sum(w[3], cb, p1, p2, lc, pay, w01, w23);
    // the code still open at the chunk end: the bytes of the last word after
    // its last terminator (a code of at most 4 bytes has one there)
    const uint32_t tw = ~cb & 0x80808080u;
    const uint32_t ps = pay & (tw ? ~(0xFFFFFFFFu >> clz32(tw)) : 0xFFFFFFFFu);
    const uint32_t cnew = dp4a(ps, w01, 0u) + (dp4a(ps, w23, 0u) << 14);
    lc |= tw ? 0u : 1u;
    const uint64_t vend = val + (uint32_t)(carry + tsum - cnew);
    if (vend >= ycur) {
      // bytes of the code open at p0 (trailing continuation bytes before it)
      const uint32_t g0 = clz32(~cb_in & 0x80808080u) >> 3;
      while (k < s && ycur <= vend) {
        S.rpos[k * S.rs] = p0 | (g0 << 12) | (kChunk << 24);
        S.rval[k * S.rs] = val;
        S.rcode[k * S.rs] = carry;
        k++;
        ycur = k < s ? pick(y, k) : ~0ull;
      }
    }
    val = vend;
    carry = cnew;
  }
  if (lc) return kLongCode;
  // step 2: exact gaps inside the recorded chunks
  for (uint32_t q = 0; q < k; q++) {
    const uint32_t rp = S.rpos[q * S.rs];
    if ((rp >> 24) != kChunk) continue;  // placed (head keys, or by an earlier chunk)
    const uint32_t p0 = rp & 0xFFFu;
    uint32_t q1 = q + 1;
    while (q1 < k && S.rpos[q1 * S.rs] == rp) q1++;
    place_in_chunk(leafp, uold, p0, S.rval[q * S.rs], S.rcode[q * S.rs], (rp >> 12) & 0xFFFu, y,
                   q, q1, S);
    q = q1 - 1;
  }
  const uint64_t lastv = val;
  for (; k < s; k++) {
    const uint64_t x = pick(y, k);
    const bool rep = k > 0 && pick(y, k - 1) == x;
    S.rpos[k * S.rs] = uold | (uold << 12) | ((rep ? kSkip : kAfter) << 24);
    S.rval[k * S.rs] = lastv;
    S.rcode[k * S.rs] = 0u;
  }
  return kPlaced;
}

// Pass A and the edits of inserting the sorted slice y[0..s) (1 <= s <=
// kKeys, repeats allowed) into the leaf at leafp (uold >= 8 used bytes, m
// elements, LB bytes, 16-byte aligned).  Returns one of the results above
// and writes nothing; kWritten means the leaf is to be rewritten (R.wlo ..
// R.whi, the R.E edits in S).
LT_HD uint32_t plan_leaf(uint8_t* leafp, uint32_t LB, uint32_t uold, uint32_t m,
                           const uint64_t (&y)[kKeys], uint32_t s, const Scratch& S,
                           Result& R) {
  uint64_t head;
  const uint32_t pa = pass_a(leafp, uold, m, y, s, S, head);
  if (pa != kPlaced) return pa;
  // ---- edits: new keys grouped by the gap they fall in ----
  uint32_t E = 0, nn = 0, added = 0, mc = 0;
  int32_t tot = 0;
  uint64_t newhead = head;
  for (uint32_t q = 0; q < s;) {
    const uint32_t rp = S.rpos[q * S.rs];
    const uint32_t kind = rp >> 24;
    if (no_insert(kind)) { q++; continue; }
    // keys q..q1 (kSkip ones among them are repeats) share this gap
    const uint32_t os = rp & 0xFFFu, oe = (rp >> 12) & 0xFFFu;
    const uint64_t rv = S.rval[q * S.rs];
    uint64_t prev = pick(y, q);
    uint32_t nl, cl = 0;
    if (kind == kHead) { nl = 8u; newhead = prev; }
    else if (kind == kGap) nl = cl = leb_bytes(prev - (rv - S.rcode[q * S.rs]));
    else nl = cl = leb_bytes(prev - rv);
    mc = mc > cl ? mc : cl;
    added |= 1u << q;
    nn++;
    uint32_t q1 = q + 1;
    for (; q1 < s; q1++) {
      const uint32_t rp1 = S.rpos[q1 * S.rs];
      if ((rp1 & 0xFFFu) != os) break;
      if (no_insert(rp1 >> 24)) continue;
      const uint64_t x = pick(y, q1);
      cl = leb_bytes(x - prev);
      mc = mc > cl ? mc : cl;
      nl += cl;
      prev = x;
      added |= 1u << q1;
      nn++;
    }
    if (kind != kAfter) {  // the old successor (head or code end)
      cl = leb_bytes(rv - prev);
      mc = mc > cl ? mc : cl;
      nl += cl;
    }
    tot += (int32_t)nl - (int32_t)(oe - os);
    S.epos[E * S.rs] = os | (oe << 12) | (kind << 24);
    S.esa[E * S.rs] = tot;
    S.ekey[E * S.rs] = q | (q1 << 8) | (nl << 16);
    E++;
    q = q1;
  }
  R.added = added;
  R.maxcode = mc;
  R.newc = m + nn;
  R.nb = (uint32_t)((int32_t)uold + tot);
  R.newhead = newhead;
  R.E = E;
  if (nn == 0) return kUnchanged;
  if (R.nb > LB) return kTooBig;
  R.wlo = (S.epos[0] & 0xFFFu) & ~15u;
  R.whi = (R.nb + 15u) & ~15u;
  return kWritten;
}

// The segment after the last edit: old bytes [oe, uold) land at [dlo, nb)
// shifted by sa (nb = the new used bytes).
LT_HD void tail_segment(const Scratch& S, uint32_t E, uint32_t uold, int32_t& dlo, int32_t& nb,
                        int32_t& sa) {
  seg_bounds(S, E, uold, S.epos[0] & 0xFFFu, (int)E - 1, dlo, nb, sa);
}

// The 16 bytes at leaf[src, src + 16) (0 <= src, src + 16 <= the old used
// bytes): the aligned chunk below src and, unless src is aligned, the one
// after it, shifted together.  A destination chunk wholly inside the
// segment after the last edit is exactly this, with src = o - sa.
LT_HD void chunk_tail(const uint8_t* leafp, int32_t src, uint32_t (&r)[4]) {
#if defined(__CUDA_ARCH__)
  // five 4-byte words from the 4-byte boundary at or below src, then the
  // byte shift inside a word (no word selects).  The fifth word is needed
  // only for an unaligned src; its bytes past src + 16 (the leaf's zero
  // bytes, the next leaf, or the padding after the last leaf) are shifted
  // out.
  const uint32_t* w = reinterpret_cast<const uint32_t*>(leafp + (src & ~3));
  const uint32_t s8 = 8u * (uint32_t)(src & 3);
  uint32_t W[5];
#pragma unroll
  for (int i = 0; i < 4; i++) W[i] = w[i];
  W[4] = s8 ? w[4] : 0u;
#pragma unroll
  for (int i = 0; i < 4; i++) r[i] = fshr(W[i], W[i + 1], s8);
#else
  const int32_t A = src & ~15;
  const uint32_t d = (uint32_t)(src - A);
  uint32_t W[8];
  uint32_t t[4];
  ld16(leafp + A, t);
  W[0] = t[0]; W[1] = t[1]; W[2] = t[2]; W[3] = t[3];
  W[4] = W[5] = W[6] = W[7] = 0u;
  if (d) {
    ld16(leafp + A + 16, t);
    W[4] = t[0]; W[5] = t[1]; W[6] = t[2]; W[7] = t[3];
  }
  // words q .. q + 4 of the 32 bytes (two selects per word), then the byte
  // shift inside a word
  const uint32_t q = d >> 2, s8 = 8u * (d & 3u);
  uint32_t X[7];
#pragma unroll
  for (int i = 0; i < 7; i++) X[i] = (q & 1u) ? W[i + 1] : W[i];
  uint32_t V[5];
#pragma unroll
  for (int i = 0; i < 5; i++) V[i] = (q & 2u) ? X[i + 2] : X[i];
#pragma unroll
  for (int i = 0; i < 4; i++) r[i] = fshr(V[i], V[i + 1], s8);
#endif
}

// Pass B by one thread: the chunks R.wlo .. R.whi of the leaf from the end
// backwards, each gathered from the segments that land in it and stored
// whole (the edits' own bytes are left zero: write_edits fills them).
LT_HD void rewrite_leaf(uint8_t* leafp, uint32_t LB, uint32_t uold, const Scratch& S,
                        const Result& R) {
  const uint32_t E = R.E;
  const uint32_t os0 = S.epos[0] & 0xFFFu;
  const uint32_t olo = R.wlo, ohi = R.whi;
  int32_t tlo, tnb, tsa;
  tail_segment(S, E, uold, tlo, tnb, tsa);
  int cur = (int)E - 1;
  for (int32_t o = (int32_t)ohi - 16; o >= (int32_t)olo; o -= 16) {
    if (o >= tlo && o + 16 <= tnb) {  // wholly inside the last segment
      uint32_t r[4];
      chunk_tail(leafp, o - tsa, r);
      st16(leafp + o, r);
      continue;
    }
    for (;;) {  // the highest segment not wholly above chunk o
      int32_t dlo, dhi, sa;
      seg_bounds(S, E, uold, os0, cur, dlo, dhi, sa);
      if (cur < 0 || dlo < o + 16) break;
      cur--;
    }
    uint32_t r[4] = {0u, 0u, 0u, 0u};
    for (int e = cur; e >= -1; e--) {
      int32_t dlo, dhi, sa;
      seg_bounds(S, E, uold, os0, e, dlo, dhi, sa);
      if (dhi <= o) break;  // wholly below this chunk: so are the earlier ones
      if (dhi > dlo) {
        const uint32_t a = (uint32_t)((dlo > o ? dlo : o) - o);
        const uint32_t b = (uint32_t)((dhi < o + 16 ? dhi : o + 16) - o);
        gather(leafp, LB, o - sa, a, b, r);
      }
    }
    st16(leafp + o, r);
  }
}

// The edits' own bytes (new head, split codes), after the chunks are stored.
LT_HD void write_edits(uint8_t* leafp, const uint64_t (&y)[kKeys], const Scratch& S,
                       const Result& R) {
  for (uint32_t e = 0; e < R.E; e++) {
    const uint32_t ep = S.epos[e * S.rs], ek = S.ekey[e * S.rs];
    const uint32_t kind = ep >> 24, os = ep & 0xFFFu;
    const uint32_t q0 = ek & 0xFFu, q1 = (ek >> 8) & 0xFFu;
    const int32_t sb = e ? S.esa[(e - 1) * S.rs] : 0;
    uint8_t* p = leafp + (int32_t)os + sb;
    const uint64_t rv = S.rval[q0 * S.rs];
    uint64_t prev = pick(y, q0);
    if (kind == kHead) {
#pragma unroll
      for (int i = 0; i < 8; i++) p[i] = (uint8_t)(prev >> (8 * i));
      p += 8;
    } else if (kind == kGap) {
      p += leb_write(p, prev - (rv - S.rcode[q0 * S.rs]));
    } else {
      p += leb_write(p, prev - rv);
    }
    for (uint32_t q = q0 + 1; q < q1; q++) {
      if (no_insert(S.rpos[q * S.rs] >> 24)) continue;
      const uint64_t x = pick(y, q);
      p += leb_write(p, x - prev);
      prev = x;
    }
    if (kind != kAfter) leb_write(p, rv - prev);
  }
}

// ---------------------------------------------------------------------------
// Delete.  Keys equal to elements (kHit) whose codes are adjacent form a run;
// a run's edit replaces the codes of its elements and of the element after
// it (the successor) by one code: successor minus the element before the run
// (Sec. 3: the neighbours of a removed key become neighbours), or, for a run
// that starts at the head, the successor as the new 8-byte head; a run that
// reaches the last element just goes.  Such an edit never grows the leaf
// (the merged delta needs no more bytes than the two it replaces), so the
// rewrite runs forward.
// ---------------------------------------------------------------------------

// Unsigned LEB128 code at p (at most 10 bytes): value, and its length in len.
LT_HD uint64_t leb_read(const uint8_t* p, uint32_t& len) {
  uint64_t v = 0;
  uint32_t n = 0;
  for (;;) {
    const uint32_t c = p[n];
    v |= (uint64_t)(c & 0x7Fu) << (7u * n);
    n++;
    if (!(c & 0x80u) || n == 10u) break;
  }
  len = n;
  return v;
}

// Pass A and the edits of deleting the sorted slice y[0..s) (1 <= s <=
// kKeys, repeats allowed) from the leaf (as plan_leaf).  R.added: bit q =
// slice key q was removed; R.wlo .. R.whi covers the old used bytes from the
// first edit on, so the bytes freed at the end are cleared.
LT_HD uint32_t plan_delete(uint8_t* leafp, uint32_t LB, uint32_t uold, uint32_t m,
                           const uint64_t (&y)[kKeys], uint32_t s, const Scratch& S,
                           Result& R) {
  uint64_t head;
  const uint32_t pa = pass_a(leafp, uold, m, y, s, S, head);
  if (pa != kPlaced) return pa;
  uint32_t E = 0, nn = 0, removed = 0;
  int32_t tot = 0;
  uint64_t newhead = head;
  for (uint32_t q = 0; q < s;) {
    const uint32_t rp = S.rpos[q * S.rs];
    if ((rp >> 24) != kHit) { q++; continue; }
    const uint32_t os = rp & 0xFFFu;
    uint32_t ce = (rp >> 12) & 0xFFFu;
    const uint64_t pred = S.rval[q * S.rs] - S.rcode[q * S.rs];  // unused when os == 0
    uint64_t lastv = S.rval[q * S.rs];
    removed |= 1u << q;
    nn++;
    uint32_t q1 = q + 1;
    for (; q1 < s; q1++) {
      const uint32_t r1 = S.rpos[q1 * S.rs], k1 = r1 >> 24;
      if (k1 == kSkip) continue;          // a repeat
      if ((r1 & 0xFFFu) != ce) break;     // beyond the successor's code
      if (k1 != kHit) continue;           // absent, in the gap before the successor
      ce = (r1 >> 12) & 0xFFFu;           // the successor itself goes: the run grows
      lastv = S.rval[q1 * S.rs];
      removed |= 1u << q1;
      nn++;
    }
    uint32_t oe = uold, nl = 0;
    uint64_t nv = 0;
    if (ce < uold) {  // the successor's code: right after the run
      uint32_t dl;
      const uint64_t succ = lastv + leb_read(leafp + ce, dl);
      oe = ce + dl;
      if (os == 0) {
        nl = 8u;
        nv = succ;
        newhead = succ;
      } else {
        nv = succ - pred;
        nl = leb_bytes(nv);
      }
    }
    tot += (int32_t)nl - (int32_t)(oe - os);
    S.epos[E * S.rs] = os | (oe << 12) | ((os == 0 ? kHead : kGap) << 24);
    S.esa[E * S.rs] = tot;
    S.ekey[E * S.rs] = q | (q1 << 8) | (nl << 16);
    S.rval[q * S.rs] = nv;  // what the edit writes (the record is used up)
    E++;
    q = q1;
  }
  R.added = removed;
  R.maxcode = 0;
  R.newc = m - nn;
  R.nb = (uint32_t)((int32_t)uold + tot);
  R.newhead = R.newc ? newhead : ~0ull;
  R.E = E;
  if (nn == 0) return kUnchanged;
  R.wlo = (S.epos[0] & 0xFFFu) & ~15u;
  R.whi = (uold + 15u) & ~15u;
  return kWritten;
}

// Pass B of a delete by one thread: the chunks R.wlo .. R.whi from the front,
// each gathered from the segments that land in it (every shift is <= 0, so a
// chunk's sources lie at or above it: not yet written).
LT_HD void rewrite_forward(uint8_t* leafp, uint32_t LB, uint32_t uold, const Scratch& S,
                           const Result& R) {
  const uint32_t E = R.E;
  const uint32_t os0 = S.epos[0] & 0xFFFu;
  int32_t tlo, tnb, tsa;
  tail_segment(S, E, uold, tlo, tnb, tsa);
  int cur = -1;
  for (int32_t o = (int32_t)R.wlo; o < (int32_t)R.whi; o += 16) {
    if (o >= tlo && o + 16 <= tnb) {  // wholly inside the last segment
      uint32_t r[4];
      chunk_tail(leafp, o - tsa, r);
      st16(leafp + o, r);
      continue;
    }
    for (;;) {  // the lowest segment not wholly below chunk o
      int32_t dlo, dhi, sa;
      seg_bounds(S, E, uold, os0, cur, dlo, dhi, sa);
      if (cur + 1 >= (int)E || dhi > o) break;
      cur++;
    }
    uint32_t r[4] = {0u, 0u, 0u, 0u};
    for (int e = cur; e < (int)E; e++) {
      int32_t dlo, dhi, sa;
      seg_bounds(S, E, uold, os0, e, dlo, dhi, sa);
      if (dlo >= o + 16) break;  // wholly above this chunk: so are the later ones
      if (dhi > dlo && dhi > o) {
        const uint32_t a = (uint32_t)((dlo > o ? dlo : o) - o);
        const uint32_t b = (uint32_t)((dhi < o + 16 ? dhi : o + 16) - o);
        gather(leafp, LB, o - sa, a, b, r);
      }
    }
    st16(leafp + o, r);
  }
}

// The delete edits' own bytes: a new head, or the merged code.
LT_HD void write_delete_edits(uint8_t* leafp, const Scratch& S, const Result& R) {
  for (uint32_t e = 0; e < R.E; e++) {
    const uint32_t ep = S.epos[e * S.rs], ek = S.ekey[e * S.rs];
    const uint32_t nl = ek >> 16;
    if (!nl) continue;
    const uint32_t q0 = ek & 0xFFu, os = ep & 0xFFFu;
    const int32_t sb = e ? S.esa[(e - 1) * S.rs] : 0;
    uint8_t* p = leafp + (int32_t)os + sb;
    const uint64_t nv = S.rval[q0 * S.rs];
    if ((ep >> 24) == kHead) {
#pragma unroll
      for (int i = 0; i < 8; i++) p[i] = (uint8_t)(nv >> (8 * i));
    } else {
      leb_write(p, nv);
    }
  }
}

LT_HD uint32_t delete_leaf(uint8_t* leafp, uint32_t LB, uint32_t uold, uint32_t m,
                           const uint64_t (&y)[kKeys], uint32_t s, const Scratch& S,
                           Result& R) {
  const uint32_t res = plan_delete(leafp, LB, uold, m, y, s, S, R);
  if (res == kWritten) {
    rewrite_forward(leafp, LB, uold, S, R);
    write_delete_edits(leafp, S, R);
  }
  return res;
}

// All of it by one thread: returns one of the results above; the leaf is
// written only for kWritten.
LT_HD uint32_t insert_leaf(uint8_t* leafp, uint32_t LB, uint32_t uold, uint32_t m,
                           const uint64_t (&y)[kKeys], uint32_t s, const Scratch& S,
                           Result& R) {
  const uint32_t res = plan_leaf(leafp, LB, uold, m, y, s, S, R);
  if (res == kWritten) {
    rewrite_leaf(leafp, LB, uold, S, R);
    write_edits(leafp, y, S, R);
  }
  return res;
}

}  // namespace leafthr
