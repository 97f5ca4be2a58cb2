/*
 * CPU oracle for the CPMA hot path (Wheatman, Burns, Bulu\c{c}, Xu,
 * "CPMA: An Efficient Batch-Parallel Compressed Set Without Pointers").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or helper with the
 * CUDA library; the two meet only through seeded inputs.
 *
 * Two independent oracles live here, both single-threaded and deliberately
 * slow and plain:
 *
 *  1. The plain definition of the set (Sec. 3, "Design and operations":
 *     insert, delete-if-present, search, half-open range_map; App. A API:
 *     insert_batch returns the number added, remove_batch the number
 *     removed, sum, size).  A sorted array of distinct uint64 keys, updated
 *     with a textbook merge.  Every set-level answer of the GPU path (set
 *     contents, has, range sums mod 2^64, counts, sizes) is compared with it.
 *
 *  2. A sequential CPMA that follows the paper's steps one batch at a time,
 *     so that the GPU layout (leaf bytes, used bytes, heads, leaf count and
 *     therefore get_size) can be compared byte for byte.  Each step names the
 *     passage it follows; where the paper is silent or garbled the reading
 *     taken is stated at the step.  The layout is "parity unpinned" against
 *     the paper itself: none of the paper's worked examples survive (its
 *     figures are images), so the layout is pinned only by invariants, by
 *     hand-computed small cases and by the plain definition above.
 *
 * Readings (also listed in the design notes):
 *   R1 codec (Sec. 5 "Data compression techniques", Fig. cpma-update shown
 *      only as an image): delta d_i = e_i - e_{i-1} >= 1 stored as unsigned
 *      LEB128: 7-bit groups, least significant first, high bit set on every
 *      byte but the last.  len(d) = max(1, ceil(bitlen(d)/7)) <= 10.
 *   R2 leaf (Sec. 5 "CPMA structure"): 8-byte little-endian head, then the
 *      codes of the following elements, packed left; bytes past the used
 *      count are zero.  used == 0 marks an empty leaf.
 *   R3 tree (Sec. 3): L leaves of LB bytes, H = ceil(log2 L); node (h, j)
 *      covers leaves [j*2^h, min((j+1)*2^h, L)), capacity = leaves*LB.
 *   R4 bounds (Sec. 3 "depends on its height"; leaf bound 0.9 in the figure
 *      captions; Sec. 5 byte density): upper tau_h = tau_leaf -
 *      (tau_leaf - tau_root) h/H, lower rho_h = rho_leaf + (rho_root -
 *      rho_leaf) h/H, in permille, tested in exact 128-bit integers; with
 *      L == 1 only the upper root bound applies.
 *   R16 uncompressed PMA (Sec. 3 PMA; the compression ablation of Sec. 6):
 *      codec 1 stores every element in an 8-byte little-endian cell, packed
 *      left; costs are 8 per element, so byte-balanced cut points are
 *      element-balanced; everything else (bounds, routing, counting,
 *      resizing) is the same batch algorithm.
 *   R5 routing (Sec. 4 batch merge search, Sec. 5 point queries): a key goes
 *      to the last leaf whose head-index entry is <= key, else leaf 0; an
 *      empty leaf's head-index entry is the head of the next non-empty leaf,
 *      or 2^64-1 if there is none.  The key 2^64-1 goes to the last
 *      non-empty leaf (else leaf 0): every entry is <= it, and empty leaves
 *      after the last non-empty one must not take it.
 *   R6 merge (Sec. 4 batch-merge phase): each routed leaf becomes content
 *      union slice (insert) or content minus slice (delete); a leaf is
 *      "touched" when its content changed.
 *   R7 counting (Sec. 4 counting phase): from every touched leaf walk up to
 *      the first node that violates neither bound; that node is the leaf's
 *      window (a touched leaf within its own bounds is rewritten in place);
 *      only maximal windows are redistributed; a walk that passes the root
 *      resizes.
 *   R8 redistribute (Sec. 4 redistribution phase, "equalizing the
 *      densities"; byte density Sec. 5): byte-balanced cut points: with
 *      costs c_0 = 8, c_i = len(e_i - e_{i-1}), prefix C_i, total S over W
 *      leaves, leaf w starts at min{i : C_i >= floor(w S / W)}.
 *   R9 resize (Sec. 3 "Resizing a PMA"; growing factor 1.2 in App. B; the
 *      shrink rule is not given): grow L' = ceil(L' * 6/5) while the root
 *      upper bound fails, shrink L' = max(1, floor(L' * 5/6)) while L' > 1
 *      and the root lower bound fails; then redistribute over L' leaves.
 *   R10 build (App. A constructor; target density not given):
 *      L = max(1, ceil(1000 S / (build_pm LB - 8000))), then R8 over L.
 *   R11 get_size (App. A): L * (LB + 16): the leaf array plus, per leaf, an
 *      8-byte head-index entry, a 4-byte used count and a 4-byte element
 *      count.
 *   R13 leaf size (Sec. 5 "CPMA structure": leaves of Theta(log n) so that
 *      the bounds hold; Sec. 6 space usage: the leaf size grows with the
 *      number of elements; no formula is given): with leaf_growth = 0 the
 *      leaf size is fixed; with leaf_growth = g > 0 every build (R10, R14)
 *      and every resize (R9) first sets LB = min(2048, max(LB_min,
 *      16 ceil(g bitlen(n) / 16))) for the n keys the array will hold
 *      (bitlen(0) = 0); a resize then starts from the leaf count of equal
 *      capacity, ceil(L * LB_old / LB), before growing or shrinking.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define OK 0
#define E_INVAL 1
#define E_NOMEM 2
#define E_FIT 3   /* a redistributed leaf did not fit: a broken invariant */

/* ------------------------------------------------------------------------ */
/* 1. Plain definition: sorted array of distinct keys                       */
/* ------------------------------------------------------------------------ */

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

/* Sort a[0..k) ascending and drop repeats in place; returns the new length. */
size_t oset_sort_unique(uint64_t* a, size_t k) {
  if (k == 0) return 0;
  qsort(a, k, sizeof(uint64_t), cmp_u64);
  size_t w = 1;
  for (size_t i = 1; i < k; i++)
    if (a[i] != a[w - 1]) a[w++] = a[i];
  return w;
}

/* out = S union U (both sorted, distinct).  Returns |out|. */
size_t oset_union(const uint64_t* S, size_t n, const uint64_t* U, size_t k,
                  uint64_t* out) {
  size_t i = 0, j = 0, w = 0;
  while (i < n && j < k) {
    if (S[i] < U[j]) out[w++] = S[i++];
    else if (U[j] < S[i]) out[w++] = U[j++];
    else { out[w++] = S[i++]; j++; }
  }
  while (i < n) out[w++] = S[i++];
  while (j < k) out[w++] = U[j++];
  return w;
}

/* out = S minus U (both sorted, distinct).  Returns |out|. */
size_t oset_difference(const uint64_t* S, size_t n, const uint64_t* U,
                       size_t k, uint64_t* out) {
  size_t i = 0, j = 0, w = 0;
  while (i < n) {
    while (j < k && U[j] < S[i]) j++;
    if (j < k && U[j] == S[i]) { i++; continue; }
    out[w++] = S[i++];
  }
  return w;
}

/* First index i with S[i] >= x (n if none). */
static size_t lower_bound_u64(const uint64_t* S, size_t n, uint64_t x) {
  size_t lo = 0, hi = n;
  while (lo < hi) {
    size_t mid = lo + (hi - lo) / 2;
    if (S[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

int oset_has(const uint64_t* S, size_t n, uint64_t x) {
  size_t i = lower_bound_u64(S, n, x);
  return i < n && S[i] == x;
}

/* Sum (mod 2^64) and count of the keys in [lo, hi). */
void oset_range(const uint64_t* S, size_t n, uint64_t lo, uint64_t hi,
                uint64_t* sum, uint64_t* count) {
  uint64_t s = 0, c = 0;
  if (lo < hi) {
    size_t i = lower_bound_u64(S, n, lo), j = lower_bound_u64(S, n, hi);
    for (size_t t = i; t < j; t++) s += S[t];
    c = j - i;
  }
  *sum = s;
  *count = c;
}

/* App. A map_range_length: the function runs on at most `length` elements,
 * starting from the first key >= start.  Here the function is the sum
 * (mod 2^64); count = how many elements it ran on. */
void oset_range_length(const uint64_t* S, size_t n, uint64_t start, uint64_t length,
                       uint64_t* sum, uint64_t* count) {
  size_t i = lower_bound_u64(S, n, start);
  size_t j = (length >= n - i) ? n : i + (size_t)length;
  uint64_t s = 0;
  for (size_t t = i; t < j; t++) s += S[t];
  *sum = s;
  *count = j - i;
}

/* Sec. 3 range_map with other functions: over the keys x in [lo, hi) with
 * (x & mask) == value, op 0 = sum mod 2^64, 1 = minimum (2^64-1 if none),
 * 2 = maximum (0 if none), 3 = exclusive or (0 if none); count = how many
 * keys passed the filter. */
void oset_range_reduce(const uint64_t* S, size_t n, uint64_t lo, uint64_t hi, int op,
                       uint64_t mask, uint64_t value, uint64_t* out, uint64_t* count) {
  uint64_t r = (op == 1) ? ~0ull : 0, c = 0;
  if (lo < hi) {
    size_t i = lower_bound_u64(S, n, lo), j = lower_bound_u64(S, n, hi);
    for (size_t t = i; t < j; t++) {
      const uint64_t x = S[t];
      if ((x & mask) != value) continue;
      c++;
      if (op == 0) r += x;
      else if (op == 1) r = x < r ? x : r;
      else if (op == 2) r = x > r ? x : r;
      else r ^= x;
    }
  }
  *out = r;
  *count = c;
}

/* ------------------------------------------------------------------------ */
/* 2. Codec (R1, R2)                                                        */
/* ------------------------------------------------------------------------ */

unsigned o_leb_len(uint64_t d) {
  unsigned n = 1;
  while (d >= 128) { d >>= 7; n++; }
  return n;
}

unsigned o_leb_put(uint8_t* p, uint64_t d) {
  unsigned n = 0;
  for (;;) {
    uint8_t b = (uint8_t)(d & 0x7F);
    d >>= 7;
    if (d) { p[n++] = (uint8_t)(b | 0x80); }
    else { p[n++] = b; return n; }
  }
}

/* Decode one code starting at p; stores the value and returns its length. */
unsigned o_leb_get(const uint8_t* p, uint64_t* d) {
  uint64_t v = 0;
  unsigned n = 0, shift = 0;
  for (;;) {
    uint8_t b = p[n++];
    v |= (uint64_t)(b & 0x7F) << shift;
    if (!(b & 0x80)) break;
    shift += 7;
  }
  *d = v;
  return n;
}

/* Bytes a leaf holding e[0..m) needs: 8 for the head plus one code per
 * following element (0 when m == 0). */
uint64_t o_leaf_bytes(const uint64_t* e, size_t m) {
  if (m == 0) return 0;
  uint64_t b = 8;
  for (size_t i = 1; i < m; i++) b += o_leb_len(e[i] - e[i - 1]);
  return b;
}

/* Write e[0..m) into a zeroed leaf buffer of LB bytes; returns used bytes. */
uint64_t o_leaf_encode(uint8_t* leaf, uint32_t LB, const uint64_t* e,
                       size_t m) {
  memset(leaf, 0, LB);
  if (m == 0) return 0;
  uint64_t h = e[0];
  for (int t = 0; t < 8; t++) leaf[t] = (uint8_t)(h >> (8 * t));
  uint64_t pos = 8;
  for (size_t i = 1; i < m; i++) pos += o_leb_put(leaf + pos, e[i] - e[i - 1]);
  return pos;
}

/* Decode a leaf with `used` bytes into out; returns the element count. */
size_t o_leaf_decode(const uint8_t* leaf, uint64_t used, uint64_t* out) {
  if (used == 0) return 0;
  uint64_t v = 0;
  for (int t = 0; t < 8; t++) v |= (uint64_t)leaf[t] << (8 * t);
  size_t m = 0;
  out[m++] = v;
  uint64_t pos = 8;
  while (pos < used) {
    uint64_t d;
    pos += o_leb_get(leaf + pos, &d);
    v += d;
    out[m++] = v;
  }
  return m;
}

/* R16, the uncompressed PMA of Sec. 3 as a leaf format: every element in an
 * 8-byte little-endian cell, packed left (the head is cell 0). */
uint64_t o_raw_leaf_bytes(size_t m) { return 8 * (uint64_t)m; }

uint64_t o_raw_leaf_encode(uint8_t* leaf, uint32_t LB, const uint64_t* e, size_t m) {
  memset(leaf, 0, LB);
  for (size_t i = 0; i < m; i++)
    for (int t = 0; t < 8; t++) leaf[8 * i + t] = (uint8_t)(e[i] >> (8 * t));
  return 8 * (uint64_t)m;
}

size_t o_raw_leaf_decode(const uint8_t* leaf, uint64_t used, uint64_t* out) {
  size_t m = (size_t)(used / 8);
  for (size_t i = 0; i < m; i++) {
    uint64_t v = 0;
    for (int t = 0; t < 8; t++) v |= (uint64_t)leaf[8 * i + t] << (8 * t);
    out[i] = v;
  }
  return m;
}

/* ------------------------------------------------------------------------ */
/* 3. Sequential CPMA                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint32_t LB;     /* leaf size in use */
  uint32_t lb_min, leaf_growth; /* R13 */
  uint32_t tau_leaf, tau_root, rho_leaf, rho_root; /* permille */
  uint32_t grow_num, grow_den;
  uint32_t build_pm;
  uint64_t L;
  uint8_t* data;   /* L * LB */
  uint32_t* used;  /* L */
  uint64_t* head;  /* L: head-index entry (R5) */
  uint64_t n;
  uint32_t rebuild_pm; /* R14: 0 = never */
  uint32_t codec;      /* R16: 0 = byte codes (CPMA), 1 = 8-byte cells (PMA) */
  /* diagnostics of the last batch, for invariant tests */
  uint64_t last_resized, last_nwindows, last_touched;
  uint64_t* last_win;   /* pairs (first leaf, leaf count) */
  uint64_t last_win_cap;
} ocpma;

static unsigned ceil_log2(uint64_t L) {
  unsigned H = 0;
  while (((uint64_t)1 << H) < L) H++;
  return H;
}

/* R3/R4: does node (h) with `leaves` leaves and `b` bytes violate a bound
 * in a tree of height H? */
int o_violates(uint32_t LB, uint32_t tau_leaf, uint32_t tau_root,
               uint32_t rho_leaf, uint32_t rho_root, unsigned H, unsigned h,
               uint64_t leaves, uint64_t b) {
  u128 cap = (u128)leaves * LB;
  if (H == 0) return (u128)b * 1000 > cap * tau_root;
  u128 lhs = (u128)b * 1000 * H;
  u128 up = cap * ((u128)tau_leaf * H - (u128)(tau_leaf - tau_root) * h);
  if (lhs > up) return 1;
  u128 lo = cap * ((u128)rho_leaf * H + (u128)(rho_root - rho_leaf) * h);
  return lhs < lo;
}

static int violates(const ocpma* o, unsigned H, unsigned h, uint64_t leaves,
                    uint64_t b) {
  return o_violates(o->LB, o->tau_leaf, o->tau_root, o->rho_leaf,
                    o->rho_root, H, h, leaves, b);
}

/* R10: leaf count of a freshly built CPMA whose stream needs S bytes. */
uint64_t o_build_leaves(uint64_t S, uint32_t LB, uint32_t build_pm) {
  u128 num = (u128)S * 1000, den = (u128)build_pm * LB - 8000;
  uint64_t L = (uint64_t)((num + den - 1) / den);
  return L < 1 ? 1 : L;
}

/* R13: leaf size for an array that will hold n keys. */
uint32_t o_leaf_size(uint64_t n, uint32_t lb_min, uint32_t leaf_growth) {
  if (leaf_growth == 0) return lb_min;
  uint32_t bl = 0;
  while (bl < 64 && (n >> bl) != 0) bl++;
  uint64_t want = ((uint64_t)leaf_growth * bl + 15) / 16 * 16;
  if (want < lb_min) want = lb_min;
  if (want > 2048) want = 2048;
  return (uint32_t)want;
}

/* R9: leaf count after a resize of a CPMA holding T bytes over L leaves. */
uint64_t o_resize_leaves(uint64_t T, uint64_t L, uint32_t LB,
                         uint32_t tau_root, uint32_t rho_root,
                         uint32_t grow_num, uint32_t grow_den) {
  uint64_t Lp = L;
  if ((u128)T * 1000 > (u128)tau_root * Lp * LB) {
    while ((u128)T * 1000 > (u128)tau_root * Lp * LB)
      Lp = (uint64_t)(((u128)Lp * grow_num + grow_den - 1) / grow_den);
  } else {
    while (Lp > 1 && (u128)T * 1000 < (u128)rho_root * Lp * LB) {
      uint64_t nx = (uint64_t)((u128)Lp * grow_den / grow_num);
      Lp = nx < 1 ? 1 : nx;
    }
  }
  return Lp;
}

/* Leaf format of this instance (R1/R2 byte codes, or R16 cells). */
static uint64_t leaf_bytes(const ocpma* o, const uint64_t* e, size_t m) {
  return o->codec ? o_raw_leaf_bytes(m) : o_leaf_bytes(e, m);
}
static uint64_t leaf_encode(const ocpma* o, uint8_t* leaf, const uint64_t* e, size_t m) {
  return o->codec ? o_raw_leaf_encode(leaf, o->LB, e, m) : o_leaf_encode(leaf, o->LB, e, m);
}
static size_t leaf_decode(const ocpma* o, const uint8_t* leaf, uint64_t used, uint64_t* out) {
  return o->codec ? o_raw_leaf_decode(leaf, used, out) : o_leaf_decode(leaf, used, out);
}

/* R8: cut points.  starts[w] for w in [0, W], starts[W] = m. */
static void cut_points(uint32_t codec, const uint64_t* e, size_t m, uint64_t W,
                       uint64_t* starts) {
  uint64_t* C = (uint64_t*)malloc((m + 1) * sizeof(uint64_t));
  C[0] = 0;
  for (size_t i = 0; i < m; i++)  /* cost of e[i] in a leaf: head or code (R8), cell (R16) */
    C[i + 1] = C[i] + ((i == 0 || codec) ? 8 : o_leb_len(e[i] - e[i - 1]));
  uint64_t S = C[m];
  for (uint64_t w = 0; w < W; w++) {
    uint64_t theta = (uint64_t)((u128)w * S / W);
    starts[w] = lower_bound_u64(C, m + 1, theta);
  }
  starts[W] = m;
  free(C);
}

void o_cut_points(const uint64_t* e, size_t m, uint64_t W, uint64_t* starts) {
  cut_points(0, e, m, W, starts);
}

/* Redistribute e[0..m) over leaves [first, first+W) of the arrays given.
 * Returns OK or E_FIT. */
static int spread(uint32_t codec, uint8_t* data, uint32_t* used, uint64_t* head, uint32_t LB,
                  uint64_t first, uint64_t W, const uint64_t* e, size_t m) {
  uint64_t* s = (uint64_t*)malloc((W + 1) * sizeof(uint64_t));
  cut_points(codec, e, m, W, s);
  int rc = OK;
  for (uint64_t w = 0; w < W; w++) {
    uint64_t j = first + w;
    size_t a = s[w], b = s[w + 1];
    const uint64_t nb = codec ? o_raw_leaf_bytes(b - a) : o_leaf_bytes(e + a, b - a);
    if (nb > LB) { rc = E_FIT; break; }
    used[j] = (uint32_t)(codec ? o_raw_leaf_encode(data + j * LB, LB, e + a, b - a)
                               : o_leaf_encode(data + j * LB, LB, e + a, b - a));
    head[j] = (b > a) ? e[a] : UINT64_MAX;
  }
  free(s);
  return rc;
}

/* R5: the head index keeps empty leaves pointing at the next non-empty head. */
static void fix_empty_heads(ocpma* o) {
  uint64_t next = UINT64_MAX;
  for (uint64_t j = o->L; j-- > 0;) {
    if (o->used[j] == 0) o->head[j] = next;
    else next = o->head[j];
  }
}

static uint64_t route(const ocpma* o, uint64_t x) {
  if (x == UINT64_MAX) {
    for (uint64_t j = o->L; j-- > 0;)
      if (o->used[j]) return j;
    return 0;
  }
  /* number of entries <= x, minus one, floored at 0 */
  uint64_t lo = 0, hi = o->L;
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (o->head[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo == 0 ? 0 : lo - 1;
}

static int alloc_arrays(uint64_t L, uint32_t LB, uint8_t** d, uint32_t** u,
                        uint64_t** h) {
  *d = (uint8_t*)calloc(L, LB);
  *u = (uint32_t*)calloc(L, sizeof(uint32_t));
  *h = (uint64_t*)malloc(L * sizeof(uint64_t));
  if (!*d || !*u || !*h) { free(*d); free(*u); free(*h); return E_NOMEM; }
  for (uint64_t j = 0; j < L; j++) (*h)[j] = UINT64_MAX;
  return OK;
}

void ocpma_destroy(ocpma* o) {
  if (!o) return;
  free(o->data); free(o->used); free(o->head); free(o->last_win);
  free(o);
}

/* App. A constructor: build from keys (any order, repeats allowed). */
int ocpma_create(ocpma** out, uint32_t LB, uint32_t tau_leaf,
                 uint32_t tau_root, uint32_t rho_leaf, uint32_t rho_root,
                 uint32_t grow_num, uint32_t grow_den, uint32_t build_pm,
                 uint32_t codec, uint32_t leaf_growth, const uint64_t* keys,
                 uint64_t k) {
  *out = NULL;
  if (codec > 1 || leaf_growth > 2048) return E_INVAL;
  if (LB < 64 || LB % 16 || !(rho_leaf <= rho_root && rho_root < tau_root &&
                               tau_root <= tau_leaf && tau_leaf < 1000) ||
      grow_num <= grow_den || grow_den == 0 ||
      (uint64_t)build_pm * LB <= 8000 || build_pm > tau_root ||
      (uint64_t)(1000 - tau_leaf) * LB < 20000)
    return E_INVAL;
  ocpma* o = (ocpma*)calloc(1, sizeof(ocpma));
  o->lb_min = LB; o->leaf_growth = leaf_growth;
  o->LB = LB; o->tau_leaf = tau_leaf; o->tau_root = tau_root;
  o->rho_leaf = rho_leaf; o->rho_root = rho_root;
  o->grow_num = grow_num; o->grow_den = grow_den; o->build_pm = build_pm;
  o->codec = codec;
  uint64_t* e = (uint64_t*)malloc((k ? k : 1) * sizeof(uint64_t));
  memcpy(e, keys, k * sizeof(uint64_t));
  size_t m = oset_sort_unique(e, k);
  LB = o->LB = o_leaf_size(m, o->lb_min, o->leaf_growth); /* R13 */
  uint64_t L = o_build_leaves(leaf_bytes(o, e, m), LB, build_pm);
  int rc = alloc_arrays(L, LB, &o->data, &o->used, &o->head);
  if (rc == OK) {
    o->L = L;
    rc = spread(o->codec, o->data, o->used, o->head, LB, 0, L, e, m);
    fix_empty_heads(o);
    o->n = m;
  }
  free(e);
  if (rc != OK) { ocpma_destroy(o); return rc; }
  *out = o;
  return OK;
}

typedef struct {
  uint64_t leaf;
  uint64_t* e;   /* merged content (owned) */
  size_t m;
  uint64_t bytes;
} touched_t;

/* Elements of leaf j as they stand after the merge phase. */
static size_t leaf_content(const ocpma* o, const touched_t* T, size_t nT,
                           const int64_t* tidx, uint64_t j, uint64_t* out) {
  if (tidx[j] >= 0) {
    const touched_t* t = &T[tidx[j]];
    memcpy(out, t->e, t->m * sizeof(uint64_t));
    return t->m;
  }
  (void)nT;
  return leaf_decode(o, o->data + j * o->LB, o->used[j], out);
}

/* R14 (Sec. 4: for a batch of k >= n/10 keys the best strategy is to rebuild
 * the whole structure by one merge): when rebuild_pm > 0 and
 * 1000 k >= rebuild_pm n (k = the batch's length as given, n = keys before
 * it), the new set S' = S union U (or S minus U) is built like the App. A
 * constructor (R10, then R8 over all leaves). */
void ocpma_set_rebuild(ocpma* o, uint32_t rebuild_pm) { o->rebuild_pm = rebuild_pm; }

static int rebuild(ocpma* o, const uint64_t* keys, uint64_t k, int is_delete, uint64_t* delta) {
  const uint32_t LBold = o->LB;
  uint64_t* S = (uint64_t*)malloc((o->n + 1) * sizeof(uint64_t));
  size_t m = 0;
  for (uint64_t j = 0; j < o->L; j++)
    m += leaf_decode(o, o->data + j * LBold, o->used[j], S + m);
  uint64_t* U = (uint64_t*)malloc((k ? k : 1) * sizeof(uint64_t));
  memcpy(U, keys, k * sizeof(uint64_t));
  size_t ku = oset_sort_unique(U, k);
  uint64_t* e = (uint64_t*)malloc((m + ku + 1) * sizeof(uint64_t));
  size_t mn = is_delete ? oset_difference(S, m, U, ku, e) : oset_union(S, m, U, ku, e);
  *delta = is_delete ? (uint64_t)(m - mn) : (uint64_t)(mn - m);
  free(S);
  free(U);
  const uint32_t LB = o_leaf_size(mn, o->lb_min, o->leaf_growth); /* R13 */
  uint64_t L = o_build_leaves(leaf_bytes(o, e, mn), LB, o->build_pm);
  uint8_t* d;
  uint32_t* u;
  uint64_t* h;
  int rc = alloc_arrays(L, LB, &d, &u, &h);
  if (rc == OK) rc = spread(o->codec, d, u, h, LB, 0, L, e, mn);
  free(e);
  if (rc != OK) return rc;
  free(o->data); free(o->used); free(o->head);
  o->data = d; o->used = u; o->head = h; o->L = L; o->n = mn; o->LB = LB;
  fix_empty_heads(o);
  o->last_resized = 1; o->last_nwindows = 0; o->last_touched = 0;
  return OK;
}

/* Sec. 4: one batch (insert when is_delete == 0).  Returns the number of keys
 * added or removed through *delta; the return value is OK or an error. */
static int update(ocpma* o, const uint64_t* keys, uint64_t k, int is_delete,
                  uint64_t* delta) {
  if (o->rebuild_pm && k && (u128)1000 * k >= (u128)o->rebuild_pm * o->n)
    return rebuild(o, keys, k, is_delete, delta);
  const uint32_t LB = o->LB;
  const uint64_t L = o->L;
  const unsigned H = ceil_log2(L);
  *delta = 0;
  o->last_resized = 0; o->last_nwindows = 0; o->last_touched = 0;

  /* Sec. 4: sort the batch (and drop repeats, App. A: repeats are not
   * counted). */
  uint64_t* U = (uint64_t*)malloc((k ? k : 1) * sizeof(uint64_t));
  memcpy(U, keys, k * sizeof(uint64_t));
  size_t ku = oset_sort_unique(U, k);

  /* Batch merge (R5, R6): slice of U per leaf, new content per leaf. */
  touched_t* T = (touched_t*)calloc(ku ? ku : 1, sizeof(touched_t));
  size_t nT = 0;
  int64_t* tidx = (int64_t*)malloc(L * sizeof(int64_t));
  for (uint64_t j = 0; j < L; j++) tidx[j] = -1;
  uint64_t* old = (uint64_t*)malloc((LB + 1) * sizeof(uint64_t));
  size_t i = 0;
  while (i < ku) {
    uint64_t j = route(o, U[i]);
    size_t b = i;
    while (i < ku && route(o, U[i]) == j) i++;
    size_t s = i - b;
    size_t m = leaf_decode(o, o->data + j * LB, o->used[j], old);
    uint64_t* e = (uint64_t*)malloc((m + s + 1) * sizeof(uint64_t));
    size_t mn = is_delete ? oset_difference(old, m, U + b, s, e)
                          : oset_union(old, m, U + b, s, e);
    if (mn == m) { free(e); continue; }   /* content unchanged: untouched */
    T[nT].leaf = j; T[nT].e = e; T[nT].m = mn;
    T[nT].bytes = leaf_bytes(o, e, mn);
    tidx[j] = (int64_t)nT;
    *delta += is_delete ? (uint64_t)(m - mn) : (uint64_t)(mn - m);
    nT++;
  }
  o->last_touched = nT;
  free(old);

  /* Byte count of every leaf after the merge. */
  uint64_t* bytes = (uint64_t*)malloc(L * sizeof(uint64_t));
  for (uint64_t j = 0; j < L; j++) bytes[j] = o->used[j];
  for (size_t t = 0; t < nT; t++) bytes[T[t].leaf] = T[t].bytes;

  /* Counting phase (R7): walk up from every touched leaf. */
  uint64_t* win = (uint64_t*)malloc((2 * nT + 2) * sizeof(uint64_t));
  size_t nw = 0;
  int resize = 0;
  for (size_t t = 0; t < nT; t++) {
    uint64_t j = T[t].leaf;
    if (!violates(o, H, 0, 1, bytes[j])) {
      /* within its own bounds: rewrite the leaf in place */
      o->used[j] = (uint32_t)leaf_encode(o, o->data + j * LB, T[t].e,
                                           T[t].m);
      o->head[j] = T[t].m ? T[t].e[0] : UINT64_MAX;
      continue;
    }
    unsigned h;
    for (h = 1; h <= H; h++) {
      uint64_t a = (j >> h) << h;
      uint64_t z = a + ((uint64_t)1 << h);
      if (z > L) z = L;
      uint64_t sum = 0;
      for (uint64_t q = a; q < z; q++) sum += bytes[q];
      if (!violates(o, H, h, z - a, sum)) {
        win[2 * nw] = a; win[2 * nw + 1] = z - a; nw++;
        break;
      }
    }
    if (h > H) resize = 1;
  }

  int rc = OK;
  uint64_t* buf = NULL;
  if (resize) {
    /* R9: whole-array resize. */
    uint64_t Ttot = 0;
    for (uint64_t j = 0; j < L; j++) Ttot += bytes[j];
    uint64_t ntot = o->n + (is_delete ? -(int64_t)*delta : (int64_t)*delta);
    /* R13: the leaf size for the new key count, from equal capacity */
    const uint32_t LBp = o_leaf_size(ntot, o->lb_min, o->leaf_growth);
    const uint64_t L0 = LBp == LB ? L : (L * LB + LBp - 1) / LBp;
    uint64_t Lp = o_resize_leaves(Ttot, L0 ? L0 : 1, LBp, o->tau_root, o->rho_root,
                                  o->grow_num, o->grow_den);
    buf = (uint64_t*)malloc((ntot + 1) * sizeof(uint64_t));
    size_t m = 0;
    for (uint64_t j = 0; j < L; j++) m += leaf_content(o, T, nT, tidx, j, buf + m);
    uint8_t* nd; uint32_t* nu; uint64_t* nh;
    rc = alloc_arrays(Lp, LBp, &nd, &nu, &nh);
    if (rc == OK) {
      rc = spread(o->codec, nd, nu, nh, LBp, 0, Lp, buf, m);
      free(o->data); free(o->used); free(o->head);
      o->data = nd; o->used = nu; o->head = nh; o->L = Lp; o->LB = LBp;
    }
    o->last_resized = 1;
    nw = 0;
  } else {
    /* Keep maximal windows only (dyadic nodes nest or are disjoint). */
    size_t keep = 0;
    for (size_t a = 0; a < nw; a++) {
      int inside = 0, dup = 0;
      for (size_t b = 0; b < nw; b++) {
        if (b == a) continue;
        uint64_t a0 = win[2 * a], a1 = a0 + win[2 * a + 1];
        uint64_t b0 = win[2 * b], b1 = b0 + win[2 * b + 1];
        if (b0 <= a0 && a1 <= b1) {
          if (b0 == a0 && b1 == a1) { if (b < a) dup = 1; }
          else inside = 1;
        }
      }
      if (!inside && !dup) {
        win[2 * keep] = win[2 * a]; win[2 * keep + 1] = win[2 * a + 1];
        keep++;
      }
    }
    nw = keep;
    for (size_t w = 0; w < nw && rc == OK; w++) {
      uint64_t a = win[2 * w], W = win[2 * w + 1];
      size_t cap = 0;
      for (uint64_t j = a; j < a + W; j++)
        cap += tidx[j] >= 0 ? T[tidx[j]].m : LB;
      uint64_t* e = (uint64_t*)malloc((cap + 1) * sizeof(uint64_t));
      size_t m = 0;
      for (uint64_t j = a; j < a + W; j++) m += leaf_content(o, T, nT, tidx, j, e + m);
      rc = spread(o->codec, o->data, o->used, o->head, LB, a, W, e, m);
      free(e);
    }
  }
  if (rc == OK) {
    fix_empty_heads(o);
    o->n = is_delete ? o->n - *delta : o->n + *delta;
    free(o->last_win);
    o->last_win = win; o->last_nwindows = nw;
    win = NULL;
  }
  free(win); free(buf); free(bytes); free(tidx);
  for (size_t t = 0; t < nT; t++) free(T[t].e);
  free(T); free(U);
  return rc;
}

int ocpma_insert(ocpma* o, const uint64_t* keys, uint64_t k, uint64_t* added) {
  return update(o, keys, k, 0, added);
}

int ocpma_delete(ocpma* o, const uint64_t* keys, uint64_t k,
                 uint64_t* removed) {
  return update(o, keys, k, 1, removed);
}

/* Sec. 5 point query: binary search over heads, then a pass over the leaf. */
int ocpma_has(const ocpma* o, uint64_t x) {
  uint64_t j = route(o, x);
  uint64_t* e = (uint64_t*)malloc((o->LB + 1) * sizeof(uint64_t));
  size_t m = leaf_decode(o, o->data + j * o->LB, o->used[j], e);
  int r = oset_has(e, m, x);
  free(e);
  return r;
}

/* Sec. 3 range_map with f = (sum, count) over [lo, hi): search, then scan. */
void ocpma_range(const ocpma* o, uint64_t lo, uint64_t hi, uint64_t* sum,
                 uint64_t* count) {
  uint64_t s = 0, c = 0;
  if (lo < hi) {
    uint64_t* e = (uint64_t*)malloc((o->LB + 1) * sizeof(uint64_t));
    for (uint64_t j = route(o, lo); j < o->L; j++) {
      if (o->used[j] && o->head[j] >= hi) break;
      size_t m = leaf_decode(o, o->data + j * o->LB, o->used[j], e);
      for (size_t t = 0; t < m; t++)
        if (e[t] >= lo && e[t] < hi) { s += e[t]; c++; }
    }
    free(e);
  }
  *sum = s;
  *count = c;
}

/* App. A sum(): every element, mod 2^64. */
uint64_t ocpma_sum(const ocpma* o) {
  uint64_t s = 0;
  uint64_t* e = (uint64_t*)malloc((o->LB + 1) * sizeof(uint64_t));
  for (uint64_t j = 0; j < o->L; j++) {
    size_t m = leaf_decode(o, o->data + j * o->LB, o->used[j], e);
    for (size_t t = 0; t < m; t++) s += e[t];
  }
  free(e);
  return s;
}

uint64_t ocpma_size(const ocpma* o) { return o->n; }
uint64_t ocpma_leaves(const ocpma* o) { return o->L; }
uint32_t ocpma_leaf_bytes(const ocpma* o) { return o->LB; }
uint64_t ocpma_bytes(const ocpma* o) { return o->L * ((uint64_t)o->LB + 16); }

/* All elements in order; returns the count. */
uint64_t ocpma_elements(const ocpma* o, uint64_t* out) {
  uint64_t m = 0;
  for (uint64_t j = 0; j < o->L; j++)
    m += leaf_decode(o, o->data + j * o->LB, o->used[j], out + m);
  return m;
}

/* Copy of the layout, for byte-for-byte comparison. */
void ocpma_layout(const ocpma* o, uint8_t* data, uint32_t* used,
                  uint64_t* head) {
  memcpy(data, o->data, o->L * o->LB);
  memcpy(used, o->used, o->L * sizeof(uint32_t));
  memcpy(head, o->head, o->L * sizeof(uint64_t));
}

void ocpma_last_batch(const ocpma* o, uint64_t* resized, uint64_t* nwindows,
                      uint64_t* touched) {
  *resized = o->last_resized;
  *nwindows = o->last_nwindows;
  *touched = o->last_touched;
}

void ocpma_last_windows(const ocpma* o, uint64_t* out) {
  memcpy(out, o->last_win, 2 * o->last_nwindows * sizeof(uint64_t));
}

/* Structural invariants (Sec. 3, Sec. 5).  Returns 0 when all hold, else the
 * number of the first failed check. */
int ocpma_check(const ocpma* o) {
  uint64_t* e = (uint64_t*)malloc((o->LB + 1) * sizeof(uint64_t));
  uint64_t total = 0, prev = 0, next_head = UINT64_MAX;
  int have_prev = 0, rc = 0;
  for (uint64_t j = 0; j < o->L && !rc; j++) {
    const uint8_t* leaf = o->data + j * o->LB;
    uint64_t u = o->used[j];
    if (u > o->LB) { rc = 1; break; }                 /* fits in its leaf */
    if (u > 0 && u < 8) { rc = 2; break; }            /* a head is 8 bytes */
    for (uint64_t t = u; t < o->LB; t++)
      if (leaf[t]) { rc = 3; break; }                 /* packed left */
    if (rc) break;
    size_t m = leaf_decode(o, leaf, u, e);
    /* the decode consumed exactly `used` bytes: re-encoding gives u back */
    if (leaf_bytes(o, e, m) != u) { rc = 4; break; }
    for (size_t t = 0; t < m; t++) {
      if (have_prev && e[t] <= prev) { rc = 5; break; } /* strictly sorted */
      prev = e[t]; have_prev = 1;
    }
    if (u > 0 && o->head[j] != e[0]) { rc = 6; break; } /* head = first */
    total += m;
  }
  /* empty leaves point at the next non-empty head (R5) */
  for (uint64_t j = o->L; j-- > 0 && !rc;) {
    if (o->used[j] == 0 && o->head[j] != next_head) rc = 7;
    if (o->used[j]) next_head = o->head[j];
  }
  if (!rc && total != o->n) rc = 8;
  free(e);
  return rc;
}
