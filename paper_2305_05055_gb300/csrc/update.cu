// Batch updates of the CPMA (Sec. 4 "Parallel Batch Updates in a PMA",
// applied to compressed leaves as Sec. 5 prescribes), resize (Sec. 3
// "Resizing a PMA") and the constructor (App. A).
//
// Phases of one batch, all on the caller's stream:
//  1. sort the batch (sort.cu);
//  2. route (one kernel): every sorted key goes to the last leaf whose
//     head-index entry is <= key; runs of equal leaf ids are the touched
//     leaves, further split every kChunk keys into merge work items (their
//     counts scanned across tiles by decoupled look-back);
//  3. merge: decode the leaf, merge (insert: union with the repeat-free
//     slice; delete: difference), count the new bytes -- one thread per leaf
//     for slices of at most four keys, a warp per leaf or per work item
//     otherwise.  A leaf whose result fits is rewritten in place; otherwise
//     the leaf is "pending" and its merged elements go to an overflow buffer
//     (Sec. 4: "copies all elements into separate memory");
//  4. counting (Sec. 4 "Counting phase"): every changed leaf that violates
//     its own bound walks up the implicit tree over a prefix sum of the byte
//     counts to the first node within bounds; distinct nodes are recorded in
//     per-level bitsets and only nodes without a recorded ancestor are kept
//     (maximal windows); a walk past the root requests a resize;
//  5. redistribute (Sec. 4 "Redistribution phase"): pack the windows'
//     elements into a buffer, compute byte costs and their prefix, place the
//     byte-balanced cut points and re-encode every destination leaf.
//     A resize is the same with the whole array as one window and L' leaves.
#include <algorithm>
#include <vector>

#include "dev_common.cuh"
#include "internal.h"
#include "leaf_thread.cuh"

using namespace cpmadev;

namespace cpmaimpl {
namespace {

constexpr int kT = 256;

struct Levels {
  uint64_t off[kMaxLevels + 1];  // word offset of each level's bitset
};

__host__ __device__ __forceinline__ size_t merge_warp_bytes(uint32_t LB) {
  // old[LB] + z[LB + kChunk] + sl[kChunk] + nk[kChunk] (u64) + buf[LB] bytes
  return (size_t)8 * (2 * LB + 3 * kChunk) + LB;
}

__device__ __forceinline__ uint64_t gtid() {
  return (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ uint64_t gstride() { return (uint64_t)gridDim.x * blockDim.x; }

__device__ __forceinline__ bool bsearch_sm(const uint64_t* a, uint32_t n, uint64_t x) {
  uint32_t i = (uint32_t)lower_bound(a, n, x);
  return i < n && a[i] == x;
}

// ---------------------------------------------------------------------------
// 2. routing
// ---------------------------------------------------------------------------
struct RouteOut {
  uint32_t *chunk_begin, *chunk_leaf, *chunk_tid;
  uint32_t *T_leaf, *T_begin, *T_first_chunk, *T_oldcnt, *T_oldused, *T_newcnt, *T_state;
  ull* T_newbytes;
};

// One-pass routing: the search, the run and chunk flags, their scan and the
// touched-leaf and work-item entries in one kernel.  Blocks take tiles of
// KPT * 256 consecutive sorted keys in order from a counter; thread t holds
// keys [t KPT, (t + 1) KPT) of its tile.  The heads a tile can reach lie
// between the sampled heads around the key before the tile and around its
// last key (kRSamples evenly spaced heads, one load each, bisected in shared
// memory); they are copied to shared memory when there are at most kRHeads
// of them (else every step-th of them, and the last candidates are searched
// in the global array, seven probes per round trip).  A thread bisects for
// its first key and gallops from there for the next ones.  The tile's run and chunk counts are scanned in the block
// and joined to the tiles before it by decoupled look-back: the whole block
// reads 256 predecessors per step; each published value packs runs << 31 |
// chunks with an aggregate / inclusive flag.  A predecessor that has not
// published after spin_limit polls sets kErrRoute instead of waiting longer;
// `silent` names a tile that never publishes (tests of that bound only).
// The tile's entries are gathered in shared memory and written out
// coalesced; every run starts a work item, so a touched leaf's key index
// and leaf come from its first item.
constexpr int kRT = 256;
constexpr uint32_t kRHeads = 4096;             // staged heads per tile (32 KB)
constexpr uint64_t kRSamples = 1024;           // heads sampled to bound a tile's range
constexpr uint64_t kRFlagA = 1ull << 62;       // tile aggregate published
constexpr uint64_t kRFlagP = 1ull << 63;       // inclusive prefix published
constexpr uint64_t kRValue = kRFlagA - 1;      // runs << 31 | chunks

// First index in [a, b) whose entry is > x (b if none), given that the
// entries before a are <= x and those from b on are > x.
__device__ __forceinline__ uint32_t bisect_upper(const uint64_t* h, uint32_t a, uint32_t b,
                                                 uint64_t x) {
  while (a < b) {
    const uint32_t mid = (a + b) >> 1;
    if (h[mid] <= x) a = mid + 1;
    else b = mid;
  }
  return a;
}

// The same in global memory with seven probes per round, loaded together
// (one round trip narrows the range eightfold), then the last few entries.
__device__ __forceinline__ uint32_t kary_upper(const uint64_t* __restrict__ g, uint32_t a,
                                               uint32_t b, uint64_t x) {
  while (b - a > 8) {
    const uint64_t w = b - a;
    uint64_t v[7];
#pragma unroll
    for (int i = 0; i < 7; i++) v[i] = __ldg(g + a + (uint64_t)(i + 1) * w / 8);
    uint32_t c = 0;  // probes <= x (a prefix of them)
#pragma unroll
    for (int i = 0; i < 7; i++) c += v[i] <= x ? 1u : 0u;
    const uint32_t na = c ? a + (uint32_t)((uint64_t)c * w / 8) + 1 : a;
    const uint32_t nb = c < 7 ? a + (uint32_t)((uint64_t)(c + 1) * w / 8) : b;
    a = na;
    b = nb;
  }
  uint64_t v[8];
#pragma unroll
  for (int i = 0; i < 8; i++) v[i] = a + i < b ? __ldg(g + a + i) : ~0ull;
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) c += (a + i < b && v[i] <= x) ? 1u : 0u;
  return a + c;
}

// The same over [a, n), probing a, a + 1, a + 3, ... first (the answer is
// usually close to a).
__device__ __forceinline__ uint32_t gallop_upper(const uint64_t* h, uint32_t a, uint32_t n,
                                                 uint64_t x) {
  uint32_t d = 1, b = n;
  while (a < n) {
    const uint32_t probe = a + d - 1;
    if (probe >= n) break;
    if (h[probe] > x) { b = probe; break; }
    a = probe + 1;
    d <<= 1;
  }
  return bisect_upper(h, a, b, x);
}

// Shared memory of a routing tile: the staged heads, then (once every key
// has its leaf) the tile's work items -- first key, leaf, touched-leaf entry
// -- and each touched leaf's first work item.
template <int KPT>
union RouteSmem {
  uint64_t heads[kRHeads];
  struct {
    uint32_t c_begin[kRT * KPT], c_leaf[kRT * KPT], c_t[kRT * KPT], t_fc[kRT * KPT];
  } e;
};

template <int KPT>
__global__ void __launch_bounds__(kRT, 4) k_route(const uint64_t* __restrict__ u, uint64_t k,
                                                  const uint64_t* __restrict__ heads, uint64_t L,
                                                  const uint32_t* __restrict__ cnt,
                                                  const uint32_t* __restrict__ used, RouteOut o,
                                                  uint64_t* look_raw, Status* st,
                                                  uint32_t spin_limit, uint32_t silent) {
  constexpr uint32_t kTileKeys = (uint32_t)kRT * KPT;
  constexpr int kW = kRT / 32;
  static_assert(sizeof(RouteSmem<KPT>) <= 32 * 1024, "routing tile smem");
  __shared__ RouteSmem<KPT> sm;
  __shared__ uint64_t s_c[2];
  __shared__ uint64_t s_wsum[kW];
  __shared__ uint64_t s_lsum[kW];
  __shared__ uint32_t s_wlast[kW];
  __shared__ uint32_t s_tile, s_pmin, s_tmo;
  pdl_wait();
  pdl_launch();
  uint32_t* ctr = reinterpret_cast<uint32_t*>(look_raw);
  volatile uint64_t* look = look_raw + 1;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t ntiles = (uint32_t)((k + kTileKeys - 1) / kTileKeys);
  const bool vec = (reinterpret_cast<uintptr_t>(u) & 15u) == 0;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= ntiles) return;
    const uint64_t base = (uint64_t)tile * kTileKeys;
    const uint32_t nvalid = (uint32_t)min((uint64_t)kTileKeys, k - base);
    const uint32_t i0 = threadIdx.x * KPT;
    uint64_t x[KPT];
    bool loaded = false;
    if constexpr (KPT % 2 == 0) {
      if (vec && i0 + KPT <= nvalid) {
#pragma unroll
        for (int j = 0; j < KPT; j += 2) {
          const uint4 v = *reinterpret_cast<const uint4*>(u + base + i0 + j);
          x[j] = (uint64_t)v.x | ((uint64_t)v.y << 32);
          x[j + 1] = (uint64_t)v.z | ((uint64_t)v.w << 32);
        }
        loaded = true;
      }
    }
    if (!loaded) {
#pragma unroll
      for (int j = 0; j < KPT; j++) x[j] = i0 + j < nvalid ? u[base + i0 + j] : KEY_MAX;
    }
    // the heads the tile can reach: kRSamples evenly spaced heads put the
    // counts of the key before the tile and of its last key in two
    // intervals, and the heads [c_lo, c_hi) from the start of the first to
    // the end of the second are the only ones its keys can need
    const uint64_t S1 = (L + kRSamples - 1) / kRSamples;
    const uint32_t ns1 = (uint32_t)(L / S1);
    for (uint32_t j = threadIdx.x; j < ns1; j += kRT)
      sm.heads[j] = __ldg(heads + (uint64_t)(j + 1) * S1 - 1);
    __syncthreads();
    if (threadIdx.x < 2) {
      const uint64_t y = threadIdx.x == 0 ? u[base ? base - 1 : 0] : u[base + nvalid - 1];
      const uint64_t m = bisect_upper(sm.heads, 0, ns1, y);
      s_c[threadIdx.x] = threadIdx.x == 0 ? m * S1 : min((m + 1) * S1 - 1, L);
    }
    __syncthreads();
    const uint64_t c_lo = s_c[0];
    const uint32_t nh = (uint32_t)(s_c[1] > c_lo ? s_c[1] - c_lo : 0);  // unsorted: empty
    // every step-th of those heads in shared memory (all of them when they fit)
    const uint32_t step = nh <= kRHeads ? 1u : (nh + kRHeads - 1) / kRHeads;
    const uint32_t ns = nh / step;
    for (uint32_t j = threadIdx.x; j < ns; j += kRT)
      sm.heads[j] = __ldg(heads + c_lo + (uint64_t)(j + 1) * step - 1);
    __syncthreads();
    // leaf of x: m staged heads <= x put the count of heads <= x in
    // c_lo + [m step, min(m step + step - 1, nh)], searched in the global
    // array (nothing left to search when every head is staged)
    auto leaf_of = [&](uint64_t y, uint32_t m) -> uint32_t {
      const uint32_t a = m * step, b = min(a + step - 1u, nh);
      const uint64_t c = c_lo + (a < b ? kary_upper(heads + c_lo, a, b, y) : a);
      return (uint32_t)(c ? c - 1 : 0);
    };
    uint32_t leaf[KPT];
    uint32_t m = 0;
    bool unsorted = false;
#pragma unroll
    for (int j = 0; j < KPT; j++) {
      if (j && x[j - 1] > x[j]) unsorted = true;
      if (x[j] == KEY_MAX) {
        leaf[j] = (uint32_t)__ldg(heads + L);
        continue;
      }
      m = j == 0 ? bisect_upper(sm.heads, 0, ns, x[j]) : gallop_upper(sm.heads, m, ns, x[j]);
      leaf[j] = leaf_of(x[j], m);
    }
    // predecessor of the thread's first key: the thread before it, the warp
    // before it, or the key before the tile
    uint32_t prev = __shfl_up_sync(FULL, leaf[KPT - 1], 1);
    uint64_t px = __shfl_up_sync(FULL, x[KPT - 1], 1);
    if (threadIdx.x == 0 && base) {
      px = u[base - 1];
      prev = px == KEY_MAX ? (uint32_t)__ldg(heads + L)
                           : leaf_of(px, bisect_upper(sm.heads, 0, ns, px));
    }
    if (lane == 31) s_wlast[warp] = leaf[KPT - 1];
    __syncthreads();  // also: every key has left the staged heads
    if (lane == 0 && warp && i0 < nvalid) {
      prev = s_wlast[warp - 1];
      px = u[base + i0 - 1];
    }
    uint32_t runs = 0, chunks = 0;
    uint32_t rflags = 0, cflags = 0;
#pragma unroll
    for (int j = 0; j < KPT; j++) {
      const uint64_t i = base + i0 + j;
      if (i0 + j >= nvalid) break;
      const uint32_t pl = j ? leaf[j - 1] : prev;
      if (j == 0 && i > 0 && px > x[0]) unsorted = true;
      const bool run = i == 0 || leaf[j] != pl;
      const bool ch = run || (i % kChunk) == 0;
      rflags |= (uint32_t)run << j;
      cflags |= (uint32_t)ch << j;
      runs += run;
      chunks += ch;
    }
    if (unsorted) atomicOr(&st->err, kErrUnsorted);
    // block exclusive scan of (runs, chunks) packed as runs << 32 | chunks
    const uint64_t mine = ((uint64_t)runs << 32) | chunks;
    const uint64_t incl = warp_incl_scan(mine);
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = lane < kW ? s_wsum[lane] : 0ull;
      w = warp_incl_scan(w);
      if (lane < kW) s_wsum[lane] = w;
    }
    __syncthreads();
    const uint64_t tot = s_wsum[kW - 1];
    const uint32_t runs_tile = (uint32_t)(tot >> 32), chunks_tile = (uint32_t)tot;
    const uint64_t agg = ((uint64_t)runs_tile << 31) | chunks_tile;
    const bool publish = tile != silent;
    // look-back: thread i polls tile tp - i
    uint64_t excl = 0;
    if (threadIdx.x == 0 && publish) look[tile] = (tile ? kRFlagA : kRFlagP) | agg;
    if (tile > 0) {
      int64_t tp = (int64_t)tile - 1;
      for (;;) {
        const int64_t q = tp - (int64_t)threadIdx.x;
        uint64_t v = kRFlagA;  // past tile 0: counts nothing
        if (q >= 0) {
          uint32_t spins = 0;
          v = look[q];
          while (!(v & (kRFlagA | kRFlagP)) && spins < spin_limit) {
            v = look[q];
            spins++;
          }
        }
        if (threadIdx.x == 0) { s_pmin = kRT; s_tmo = 0; }
        __syncthreads();
        if (!(v & (kRFlagA | kRFlagP))) s_tmo = 1;
        if (q >= 0 && (v & kRFlagP)) atomicMin(&s_pmin, threadIdx.x);
        __syncthreads();
        const uint32_t stop = s_pmin;  // nearest predecessor with its inclusive prefix
        const uint64_t add = warp_sum(q >= 0 && threadIdx.x <= stop ? (v & kRValue) : 0ull);
        if (lane == 0) s_lsum[warp] = add;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kW; w++) excl += s_lsum[w];
        const bool gave_up = s_tmo != 0;
        if (gave_up || stop < (uint32_t)kRT || tp < kRT) {
          if (gave_up && threadIdx.x == 0) atomicOr(&st->err, kErrRoute);
          break;
        }
        tp -= kRT;
        __syncthreads();  // s_pmin, s_tmo and s_lsum are reused
      }
      if (threadIdx.x == 0 && publish) {
        __threadfence();
        look[tile] = kRFlagP | (excl + agg);
      }
    }
    const uint32_t g_runs = (uint32_t)(excl >> 31), g_chunks = (uint32_t)(excl & 0x7FFFFFFFull);
    // this tile's work items and touched-leaf starts, in shared memory
    const uint64_t before = (warp ? s_wsum[warp - 1] : 0ull) + incl - mine;
    uint32_t r = (uint32_t)(before >> 32), c = (uint32_t)before;  // local indices
#pragma unroll
    for (int j = 0; j < KPT; j++) {
      if (i0 + j >= nvalid) break;
      const bool run = (rflags >> j) & 1u, ch = (cflags >> j) & 1u;
      r += run;  // r - 1: the key's touched leaf, local
      if (run) sm.e.t_fc[r - 1] = c;
      if (ch) {
        sm.e.c_begin[c] = (uint32_t)(base + i0 + j);
        sm.e.c_leaf[c] = leaf[j];
        sm.e.c_t[c] = g_runs + r - 1;
        c++;
      }
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < chunks_tile; q += kRT) {
      o.chunk_begin[g_chunks + q] = sm.e.c_begin[q];
      o.chunk_leaf[g_chunks + q] = sm.e.c_leaf[q];
      o.chunk_tid[g_chunks + q] = sm.e.c_t[q];
    }
    // touched leaves: every thread's (at most KPT) old counts are loaded
    // together before any entry is stored
    {
      uint32_t lf[KPT], oc[KPT], ou[KPT];
#pragma unroll
      for (int j = 0; j < KPT; j++) {
        const uint32_t q = threadIdx.x + (uint32_t)j * kRT;
        lf[j] = q < runs_tile ? sm.e.c_leaf[sm.e.t_fc[q]] : 0u;
        oc[j] = q < runs_tile ? cnt[lf[j]] : 0u;
        ou[j] = q < runs_tile ? used[lf[j]] : 0u;
      }
#pragma unroll
      for (int j = 0; j < KPT; j++) {
        const uint32_t q = threadIdx.x + (uint32_t)j * kRT;
        if (q >= runs_tile) break;
        const uint32_t fc = sm.e.t_fc[q], t = g_runs + q;
        o.T_leaf[t] = lf[j];
        o.T_begin[t] = sm.e.c_begin[fc];
        o.T_first_chunk[t] = g_chunks + fc;
        o.T_oldcnt[t] = oc[j];
        o.T_oldused[t] = ou[j];
        o.T_newcnt[t] = 0;
        o.T_newbytes[t] = 0;
        o.T_state[t] = kUnchanged;
      }
    }
    if (threadIdx.x == 0 && base + nvalid == k) {
      const uint32_t nT = g_runs + runs_tile, nC = g_chunks + chunks_tile;
      st->nT = nT;
      st->nchunks = nC;
      o.T_begin[nT] = (uint32_t)k;
      o.T_first_chunk[nT] = nC;
      o.chunk_begin[nC] = (uint32_t)k;
    }
    __syncthreads();  // the next tile reuses the shared arrays
  }
}

// ---------------------------------------------------------------------------
// 3. merge
// ---------------------------------------------------------------------------
struct MergeArgs {
  const uint64_t* u;
  uint8_t* data;
  uint32_t* used;
  uint32_t* cnt;
  uint64_t* heads;
  uint32_t LB;
  const uint32_t *chunk_begin, *chunk_leaf, *chunk_tid;
  uint32_t* chunk_cnt;
  const uint64_t* chunk_off;
  const uint32_t *T_begin, *T_oldcnt, *T_oldused, *T_leaf, *T_first_chunk;
  uint32_t *T_newcnt, *T_state;
  ull* T_newbytes;
  uint64_t* ovf;
  int is_delete;
  Status* st;
  ull* prof;  // profiling: algorithmic bytes of this kernel (nullable)
  const uint32_t* tags;  // per sorted key: request tag (nullable)
  ull* tag_counts;       // per tag: keys added / removed (nullable)
  uint32_t* list_lane;   // touched leaves for k_insert_lane (count st->n_lane)
  uint32_t* list_v1;     // touched leaves for k_merge_small (count st->n_v1)
  uint32_t* list_gen;    // work items for k_merge in count mode (st->n_gen)
  uint32_t* list_pend;   // pending leaves of k_insert_thread / k_insert_lane (st->n_pendl)
  int raw;               // leaves hold 8-byte cells (codec 1), not byte codes
  int small;             // a small batch: every slice goes to a warp per leaf
  Bounds B;              // density bounds and tree height, for the leaves the
  unsigned H;            // thread-granular merge finalises itself
  uint32_t* viol;        // touched leaves over their own bound (count st->nviol)
  uint8_t* pstage;       // point path: 512-byte staging slot per key (first key of a leaf)
  struct PointRec* prec; // point path: the staged result per key (first key of a leaf)
};

// A touched leaf's result staged by the point path's plan pass: the new
// head, used bytes and count, the rewritten byte range [lo, wend) held in
// the staging slot, and the keys added and byte change.
struct PointRec {
  uint64_t head;
  uint32_t leaf, nb, newc, lo, wend, added;
  int32_t dbytes;
  uint32_t pad;
};

// Append to a work list, one atomic per warp (all lanes must call).
__device__ __forceinline__ void warp_append(bool pred, uint32_t value, uint32_t* list, ull* ctr) {
  const unsigned m = __ballot_sync(FULL, pred);
  if (!m) return;
  const unsigned leader = __ffs(m) - 1;
  ull base = 0;
  if (lane_id() == leader) base = atomicAdd(ctr, (ull)__popc(m));
  base = __shfl_sync(FULL, base, leader);
  if (pred) list[base + __popc(m & lanemask_lt())] = value;
}

// Credit one added / removed key to the request that owns its first
// occurrence in the sorted batch.
__device__ __forceinline__ void credit(const MergeArgs& a, uint64_t key_index) {
  if (a.tag_counts) atomicAdd(a.tag_counts + a.tags[key_index], 1ull);
}

// Slices of at most kSmall keys into a non-empty leaf take the splice path.
constexpr uint32_t kSmall = 32;
// T-entry state set by the lane-granular insert when a leaf holds a code of
// more than 4 bytes: the element-array splice takes it instead.
constexpr uint32_t kFallback = 3;
// T-entry state of a leaf the thread-granular merge rewrote in place and
// also counted (batch totals, own-bound test): the finalize pass skips it.
constexpr uint32_t kDone = 4;

// Copy the bytes of the old leaf (global, uold bytes) that lie outside the E
// edits into out[] (shared, zeroed), each shifted by the size change of the
// edits before it.  Edit e replaces old bytes [es[e], ee[e]); shc[e] is the
// total size change of edits 0..e.  A lane whose 16 bytes hold no edit
// boundary copies them as words (funnel shifts; the two partial words are
// OR-ed in, the buffer being zeroed and every byte having one writer).  The
// word copy writes up to 20 bytes from a lane's start, past the used bytes
// (zeros there, packed left): out[] needs 32 bytes of slack after LB.
__device__ __forceinline__ void splice_copy(const uint8_t* __restrict__ leafp, uint32_t uold,
                                            uint8_t* out, uint32_t E, const uint32_t* es,
                                            const uint32_t* ee, const int32_t* shc) {
  const unsigned lane = lane_id();
  for (uint32_t p0 = lane * 16; p0 < uold; p0 += 512) {
    const uint4 v = *reinterpret_cast<const uint4*>(leafp + p0);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t q = 0;
    while (q < E && ee[q] <= p0) q++;
    int32_t shift = q ? shc[q - 1] : 0;
    const uint32_t lim = min(16u, uold - p0);
    if (q == E || es[q] >= p0 + 16) {
      // bytes past uold are zero (packed left), so the whole 16 can go
      const uint32_t d0 = (uint32_t)((int32_t)p0 + shift);
      uint32_t* ow = reinterpret_cast<uint32_t*>(out);
      const uint32_t k0 = d0 >> 2, sb = d0 & 3u;
      if (sb == 0) {
        ow[k0] = w[0]; ow[k0 + 1] = w[1]; ow[k0 + 2] = w[2]; ow[k0 + 3] = w[3];
      } else {
        const uint32_t sh8 = 8u * sb;
        atomicOr(ow + k0, w[0] << sh8);
        ow[k0 + 1] = __funnelshift_l(w[0], w[1], sh8);
        ow[k0 + 2] = __funnelshift_l(w[1], w[2], sh8);
        ow[k0 + 3] = __funnelshift_l(w[2], w[3], sh8);
        atomicOr(ow + k0 + 4, w[3] >> (32u - sh8));
      }
    } else {
#pragma unroll
      for (int b = 0; b < 16; b++) {
        const uint32_t tt = p0 + b;
        if ((uint32_t)b >= lim) continue;
        while (q < E && ee[q] <= tt) { shift = shc[q]; q++; }
        if (q < E && es[q] <= tt) continue;
        out[(int32_t)tt + shift] = (uint8_t)(w[b >> 2] >> (8 * (b & 3)));
      }
    }
  }
}

__host__ __device__ __forceinline__ size_t small_warp_bytes(uint32_t LB) {
  // old[LB] u64, pos[LB] u16, out[LB + 32] bytes (the word copy may spill
  // up to 20 zero bytes past LB), keys[kSmall] u64, ranks[kSmall] u32, edits:
  // old start, old end, new start, cumulative shift (u32 each)
  return (size_t)8 * LB + 2 * LB + LB + 32 + 8 * kSmall + 4 * kSmall + 16 * kSmall;
}

__device__ __forceinline__ bool small_slice(uint32_t tb, uint32_t te, uint32_t uold) {
  return te - tb <= kSmall && uold > 0;
}

// Lane-granular insert: lanes per leaf (a segment), and per segment
// out[512 + 32] (slack for the word copy), 3 u64 and 8 u32 arrays of SEG keys.
// A whole warp per leaf (16 bytes per lane) measured slightly faster than a
// half warp per leaf (32 bytes per lane, two leaves per warp step): the
// per-lane summary and splice work dominates, not the per-leaf bookkeeping.
constexpr int kLaneSeg = 32;
constexpr size_t kLaneOut = 512 + 32;
__host__ __device__ constexpr size_t lane_seg_bytes(int seg) {
  return kLaneOut + (size_t)seg * (3 * 8 + 8 * 4);
}
__host__ __device__ constexpr size_t lane_warp_bytes(int seg) {
  return (size_t)(32 / seg) * lane_seg_bytes(seg);
}

// Inserts into byte-code leaves are split by slice size: up to kThrKeys keys
// -> k_insert_thread (which walks the touched leaves itself), then up to
// kLaneSeg keys into leaves of at most 512 used bytes -> k_insert_lane (from
// the list k_classify builds).
constexpr uint32_t kThrKeys = leafthr::kKeys;
// A small batch touches few leaves, so its merge time is latency rather than
// throughput: every slice then goes to a warp per leaf (one coalesced load of
// the leaf instead of a thread's chain of dependent 16-byte loads).
constexpr uint64_t kSmallBatch = 8192;
__device__ __forceinline__ bool thread_class(uint32_t s, uint32_t uold, int small = 0) {
  return !small && s >= 1 && s <= kThrKeys && uold > 0;
}
__device__ __forceinline__ bool lane_class(uint32_t s, uint32_t uold, int small = 0) {
  return s > (small ? 0u : kThrKeys) && s <= (uint32_t)kLaneSeg && uold > 0 && uold <= 512;
}

// Copy of the kept old bytes for the lane-granular insert: the lane's 4*NW
// bytes are cut into the segments that no edit removes, and each segment is
// OR-ed into out[] as NW + 1 shifted words (out[] zeroed, one writer per byte,
// 32 bytes of slack after the leaf).
template <int NW = 4>
__device__ __forceinline__ void splice_copy_words(const uint32_t (&w)[NW], uint32_t p0,
                                                  uint32_t uold, uint8_t* out, uint32_t E,
                                                  const uint32_t* es, const uint32_t* ee,
                                                  const int32_t* shc) {
  constexpr uint32_t kB = 4 * NW;  // bytes per lane
  if (p0 >= uold) return;
  uint32_t q = 0;
  while (q < E && ee[q] <= p0) q++;
  int32_t shift = q ? shc[q - 1] : 0;
  uint32_t cur = p0;
  const uint32_t lim = min(p0 + kB, uold);
  uint32_t* ow = reinterpret_cast<uint32_t*>(out);
  while (cur < lim) {
    const uint32_t send = (q < E) ? min(es[q], lim) : lim;
    if (send > cur) {
      // bytes [cur, send) of the lane, shifted by `shift`
      const uint32_t a = cur - p0, b = send - p0;
      const uint32_t segm = ((b >= 32) ? 0xFFFFFFFFu : ((1u << b) - 1u)) & ~((1u << a) - 1u);
      uint32_t m[NW];
#pragma unroll
      for (int k = 0; k < NW; k++) m[k] = w[k] & bytemask4((segm >> (4 * k)) & 0xFu);
      const uint32_t d0 = (uint32_t)((int32_t)p0 + shift);
      const uint32_t k0 = d0 >> 2, sh8 = 8u * (d0 & 3u);
      if (sh8 == 0) {
#pragma unroll
        for (int k = 0; k < NW; k++)
          if (m[k]) atomicOr(ow + k0 + k, m[k]);
      } else {
        if (m[0] << sh8) atomicOr(ow + k0, m[0] << sh8);
#pragma unroll
        for (int k = 1; k < NW; k++) {
          const uint32_t y = __funnelshift_l(m[k - 1], m[k], sh8);
          if (y) atomicOr(ow + k0 + k, y);
        }
        const uint32_t yl = m[NW - 1] >> (32u - sh8);
        if (yl) atomicOr(ow + k0 + NW, yl);
      }
    }
    if (q < E && es[q] < lim) {
      cur = max(cur, ee[q]);
      shift = shc[q];
      q++;
    } else {
      break;
    }
  }
}

// Segment (SEG consecutive lanes, mask `seg`, segment index sg, lane sl in
// it) ballot as SEG bits, and inclusive scan.
template <int SEG>
__device__ __forceinline__ unsigned seg_ballot(unsigned seg, unsigned sg, bool p) {
  const unsigned b = __ballot_sync(seg, p);
  return SEG == 32 ? b : (b >> (sg * SEG)) & ((1u << SEG) - 1u);
}
template <int SEG, typename T>
__device__ __forceinline__ T seg_scan(unsigned seg, unsigned sl, T v) {
#pragma unroll
  for (int o = 1; o < SEG; o <<= 1) {
    const T n = __shfl_up_sync(seg, v, o, SEG);
    if ((int)sl >= o) v += n;
  }
  return v;
}

// What the per-leaf body of the lane-granular insert does with a leaf:
// kLaneBatch -- the batch merge (work-list bookkeeping, pending and fallback
// leaves handed on); kLaneStage -- the point path's plan: the leaf is left
// as it is, and a result that can go in place is written to the leaf's
// staging slot instead (the rewritten 16-byte chunks at their leaf offsets)
// with a PointRec, for k_point_commit.  kLaneStage returns kLeafInPlace,
// kLeafSame (every key already present) or kLeafBatch (the leaf needs the
// batch algorithm: a slice over SEG keys, an empty leaf or one over 512 used
// bytes, a code over 4 bytes, a result over the leaf or over 512 bytes, or
// one that violates the leaf's own density bound).
constexpr int kLaneBatch = 0, kLaneStage = 1;
constexpr uint32_t kLeafInPlace = 0, kLeafSame = 1, kLeafBatch = 2;

// One leaf of the lane-granular insert, taken by the segment sg of SEG lanes
// (lane sl in it, mask seg); wbase is the segment's shared scratch.  The
// leaf's keys are u[tb, te); nbytes, dl and db accumulate the algorithmic
// bytes, keys added and byte total change (lane 0 of the segment).
template <int SEG, int MODE>
__device__ __forceinline__ uint32_t lane_leaf(const MergeArgs& a, uint8_t* wbase, unsigned sg,
                                              unsigned sl, unsigned seg, uint32_t t, uint32_t tb,
                                              uint32_t te, uint32_t uold, uint32_t j, uint32_t m,
                                              uint32_t fc0, uint32_t fc1, ull& nbytes, ull& dl,
                                              ull& db) {
  constexpr int NW = 512 / (4 * SEG);        // words per lane
  constexpr uint32_t kLB = 4u * NW;          // bytes per lane
  constexpr uint32_t KS = SEG;               // keys per slice
  constexpr bool BATCH = MODE == kLaneBatch;
  const unsigned lt_mask = (1u << sl) - 1u;
  uint8_t* out = wbase;
  uint64_t* kx = reinterpret_cast<uint64_t*>(wbase + kLaneOut);  // key
  uint64_t* kp = kx + KS;                                         // predecessor value
  uint64_t* ks = kp + KS;                                         // successor value
  uint32_t* kr = reinterpret_cast<uint32_t*>(ks + KS);  // rank; bit 31 = present
  uint32_t* kcs = kr + KS;                              // successor code start
  uint32_t* kce = kcs + KS;                             // successor code end (excl.)
  uint32_t* ktl = kce + KS;                             // owning lane
  uint32_t* es = ktl + KS;
  uint32_t* ee = es + KS;
  uint32_t* en = ee + KS;
  int32_t* shc = reinterpret_cast<int32_t*>(en + KS);
  const uint32_t s = te - tb;
  if (!BATCH && (s > KS || uold == 0 || uold > 512)) return kLeafBatch;
  uint8_t* leafp = a.data + (size_t)j * a.LB;
  // the old leaf, the slice and ~28 bytes of per-leaf metadata
  if (BATCH) nbytes += uold + 8u * s + 28u;
  // ---- bit-parallel summary of each lane's bytes ----
  const uint32_t p0 = sl * kLB;
  uint32_t w[NW];
#pragma unroll
  for (int q = 0; q < NW; q += 4) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (p0 + 4u * q < uold) v = *reinterpret_cast<const uint4*>(leafp + p0 + 4u * q);
    w[q] = v.x; w[q + 1] = v.y; w[q + 2] = v.z; w[q + 3] = v.w;
  }
  // the slice's keys, loaded now so their latency overlaps the summary
  uint64_t x = 0, xprev = 0;
  if (sl < s) {
    x = a.u[tb + sl];
    if (sl > 0) xprev = a.u[tb + sl - 1];
  }
  const int b_lo = sl == 0 ? 8 : 0;
  const int b_hi = (uold > p0) ? (int)min(kLB, uold - p0) : 0;
  LaneCodesN<NW> lc;
  lane_codes<false, NW>(w, b_lo, b_hi, lc);
  bool bad = lc.bad;
  uint32_t pv = __shfl_up_sync(seg, lc.tail, 1, SEG);
  uint32_t ps = __shfl_up_sync(seg, lc.tail_sh, 1, SEG);
  if (sl == 0) { pv = 0; ps = 0; }
  uint32_t D = 0;
  if (lc.term) {
    if (ps / 7u + lc.first_len > 4u) bad = true;
    D = lc.D - lc.first_own + pv + (lc.first_own << ps);
  }
  if (__any_sync(seg, bad)) {
    if (BATCH && sl == 0) {
      a.T_state[t] = kFallback;
      a.list_v1[atomicAdd(&a.st->n_v1, 1ull)] = t;
    }
    return kLeafBatch;
  }
  const uint32_t c = __popc(lc.term);
  const uint32_t B = seg_scan<SEG, uint32_t>(seg, sl, c) - c;                       // codes in earlier lanes
  if (__shfl_sync(seg, B + c, SEG - 1, SEG) + 1u != m) {   // must match the stored count
    if (sl == 0) atomicOr(&a.st->err, kErrState);
    return kLeafBatch;
  }
  const uint64_t Dinc = seg_scan<SEG, uint64_t>(seg, sl, (uint64_t)D);
  const uint64_t head = __shfl_sync(seg, (uint64_t)w[0] | ((uint64_t)w[1] << 32), 0, SEG);
  const uint64_t V = head + (Dinc - D);                             // element before my codes
  const uint64_t lastv = head + __shfl_sync(seg, Dinc, SEG - 1, SEG);  // the last element
  // ---- keys: owning lane, or before the head / after the last element ----
  const bool valid = sl < s && !(sl > 0 && xprev == x);
  unsigned owners = 0;
  for (uint32_t k = 0; k < s; k++) {
    const uint64_t xk = __shfl_sync(seg, x, k, SEG);
    const unsigned own = seg_ballot<SEG>(seg, sg, c > 0 && V < xk && xk <= V + D);
    if (sl == k) ktl[k] = own ? (uint32_t)(__ffs(own) - 1) : 0xFFFFFFFFu;
    owners |= own;
  }
  if (sl < s) {
    kx[sl] = x;
    if (x <= head) {            // before the head, or the head itself
      kr[sl] = (x == head) ? 0x80000000u : 0u;
      kp[sl] = 0; ks[sl] = head; kcs[sl] = 0; kce[sl] = 8;
    } else if (x > lastv) {     // after the last element
      kr[sl] = m;
      kp[sl] = lastv; ks[sl] = 0; kcs[sl] = uold; kce[sl] = uold;
    }
  }
  __syncwarp(seg);
  // ---- each owning lane decodes its own codes (all owners at once) ----
  // Walking its codes in order, the lane keeps the running value; a key
  // takes the first code whose value reaches it: that code's element is
  // its successor (rank 1 + codes before it), the value before is its
  // predecessor, and the code's bytes are the ones an insert replaces.
  if ((owners >> sl) & 1u) {
    uint32_t kq = 0;
    while (ktl[kq] != sl) kq++;  // this lane's keys are consecutive
    uint32_t tm2 = lc.term, st = (sl == 0) ? 8u : 0u, rank = 1u + B;
    uint64_t val = V;
    bool firstc = true;
    while (tm2 && kq < s && ktl[kq] == sl) {
      const uint32_t tb8 = (uint32_t)__ffs(tm2) - 1u;
      tm2 &= tm2 - 1u;
      const uint32_t own = compact7(window32<NW>(lc.x, st)) & mask7(tb8 + 1u - st);
      const uint32_t code = firstc ? pv + (own << ps) : own;
      const uint32_t cs = kLB * sl + st - (firstc ? ps / 7u : 0u);
      const uint64_t prev = val;
      val += code;
      while (kq < s && ktl[kq] == sl && kx[kq] <= val) {
        kr[kq] = rank | (kx[kq] == val ? 0x80000000u : 0u);
        kp[kq] = prev;
        ks[kq] = val;
        kcs[kq] = cs;
        kce[kq] = kLB * sl + tb8 + 1u;
        kq++;
      }
      rank++;
      st = tb8 + 1u;
      firstc = false;
    }
  }
  __syncwarp(seg);
  // ---- kept keys and their gaps ----
  uint32_t r = 0;
  bool keep = false;
  if (sl < s) {
    r = kr[sl];
    keep = valid && !(r & 0x80000000u);
  }
  const unsigned kb = seg_ballot<SEG>(seg, sg, keep);
  const uint32_t nn = __popc(kb);
  uint64_t mx = 0, mp = 0, ms = 0;
  uint32_t mcs = 0, mce = 0;
  if (keep) { mx = kx[sl]; mp = kp[sl]; ms = ks[sl]; mcs = kcs[sl]; mce = kce[sl]; }
  __syncwarp(seg);
  if (keep) {
    const uint32_t q = __popc(kb & lt_mask);
    kx[q] = mx; kp[q] = mp; ks[q] = ms; kcs[q] = mcs; kce[q] = mce; kr[q] = r;
  }
  __syncwarp(seg);
  if (nn == 0) {
    if (BATCH) {
      if (sl == 0) {
        a.T_state[t] = kUnchanged;
        a.T_newcnt[t] = m;
        a.T_newbytes[t] = uold;
      }
      for (uint32_t cq = fc0 + sl; cq < fc1; cq += SEG) a.chunk_cnt[cq] = 0;
      __syncwarp(seg);
    }
    return kLeafSame;
  }
  bool lead = false;
  if (sl < nn) lead = sl == 0 || kr[sl - 1] != kr[sl];
  const unsigned lb = seg_ballot<SEG>(seg, sg, lead);
  const uint32_t E = __popc(lb);
  uint32_t e_os = 0, e_oe = 0, e_nl = 0, gend = 0, g0 = 0;
  if (lead) {
    const unsigned after = lb & ~((2u << sl) - 1u);
    gend = after ? (uint32_t)(__ffs(after) - 1) : nn;
    g0 = kr[sl];
    e_os = kcs[sl];
    e_oe = kce[sl];
    uint64_t prev = kx[sl];
    uint32_t len = (g0 == 0) ? 8u : leb_len(kx[sl] - kp[sl]);
    for (uint32_t q = sl + 1; q < gend; q++) { len += leb_len(kx[q] - prev); prev = kx[q]; }
    if (g0 < m) len += leb_len(ks[sl] - prev);
    e_nl = len;
  }
  const uint32_t eidx = __popc(lb & lt_mask);
  const int32_t delta = lead ? (int32_t)e_nl - (int32_t)(e_oe - e_os) : 0;
  const int32_t dinc = (int32_t)seg_scan<SEG, uint32_t>(seg, sl, (uint32_t)delta);
  const int32_t total = (int32_t)__shfl_sync(seg, (uint32_t)dinc, SEG - 1, SEG);
  if (lead) {
    es[eidx] = e_os;
    ee[eidx] = e_oe;
    en[eidx] = (uint32_t)((int32_t)e_os + dinc - delta);
    shc[eidx] = dinc;
  }
  const uint32_t nb = (uint32_t)((int32_t)uold + total);
  const uint32_t newc = m + nn;
  const uint64_t newhead = (kr[0] == 0) ? kx[0] : head;
  __syncwarp(seg);
  if (nb > a.LB) {
    if (BATCH) {
      if (sl == 0) {
        a.T_state[t] = kPending;
        a.T_newcnt[t] = newc;
        a.T_newbytes[t] = nb;
        a.list_pend[atomicAdd(&a.st->n_pendl, 1ull)] = t;
      }
      for (uint32_t cq = fc0 + sl; cq < fc1; cq += SEG) a.chunk_cnt[cq] = (cq == fc0) ? newc : 0u;
      if (keep) credit(a, tb + sl);
      __syncwarp(seg);
    }
    return kLeafBatch;
  }
  if (nb > 512) {  // fits the leaf but not this kernel's 512-byte buffer
    if (BATCH && sl == 0) {
      a.T_state[t] = kFallback;
      a.list_v1[atomicAdd(&a.st->n_v1, 1ull)] = t;
    }
    __syncwarp(seg);
    return kLeafBatch;
  }
  // outside the batch merge a leaf is only rewritten when it stays within its
  // own bound (the batch merge writes it either way and starts a walk)
  const bool viol = node_violates(a.B, a.H, 0, 1, nb);
  if (!BATCH && viol) return kLeafBatch;
  const uint32_t wend = (max(uold, nb) + 15u) & ~15u;
  // lanes whose bytes lie wholly before the first edit keep them: they
  // neither rebuild nor rewrite them
  const bool touched = p0 + kLB > es[0];
  if (touched)
#pragma unroll
    for (uint32_t q = 0; q < kLB; q += 16)
      if (p0 + q < wend) *reinterpret_cast<uint4*>(out + p0 + q) = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp(seg);
  if (touched) splice_copy_words<NW>(w, p0, uold, out, E, es, ee, shc);
  __syncwarp(seg);
  if (lead) {
    uint8_t* o = out + en[eidx];
    uint64_t prev = kx[sl];
    if (g0 == 0) {
#pragma unroll
      for (int b = 0; b < 8; b++) o[b] = (uint8_t)(prev >> (8 * b));
      o += 8;
    } else {
      o += leb_put(o, prev - kp[sl]);
    }
    for (uint32_t q = sl + 1; q < gend; q++) { o += leb_put(o, kx[q] - prev); prev = kx[q]; }
    if (g0 < m) leb_put(o, ks[sl] - prev);
  }
  __syncwarp(seg);
  uint8_t* dst = BATCH ? leafp : a.pstage + (size_t)tb * 512;
  if (touched)
#pragma unroll
    for (uint32_t q = 0; q < kLB; q += 16)
      if (p0 + q < wend)
        *reinterpret_cast<uint4*>(dst + p0 + q) = *reinterpret_cast<const uint4*>(out + p0 + q);
  if (!BATCH) {
    if (sl == 0) {
      PointRec R;
      R.head = newhead;
      R.leaf = j;
      R.nb = nb;
      R.newc = newc;
      R.lo = es[0] & ~15u;
      R.wend = wend;
      R.added = nn;
      R.dbytes = total;
      a.prec[tb] = R;
    }
    __syncwarp(seg);
    return kLeafInPlace;
  }
  if (sl == 0) nbytes += wend - min(wend, es[0] & ~15u);
  if (keep) credit(a, tb + sl);
  if (sl == 0) {
    a.used[j] = nb;
    a.cnt[j] = newc;
    a.heads[j] = newhead;
    // the finalize pass's work for this leaf, done here
    dl += newc - m;
    db += (ull)nb - (ull)uold;
    a.T_newcnt[t] = newc;
    a.T_newbytes[t] = nb;
    if (viol) a.viol[atomicAdd(&a.st->nviol, 1ull)] = j;
    a.T_state[t] = kDone;
  }
  for (uint32_t cq = fc0 + sl; cq < fc1; cq += SEG) a.chunk_cnt[cq] = 0;
  __syncwarp(seg);
  return kLeafInPlace;
}

// Insert of a small slice (at most SEG keys) into a leaf of at most 512 used
// bytes, without decoding the whole leaf into an element array.  A segment
// of SEG lanes takes one leaf (32 / SEG leaves per warp step), each lane
// 512 / SEG bytes of it.  Each lane summarises its bytes bit-parallel
// (lane_codes: how many codes end there and the sum of their deltas);
// segment scans then give every lane the value of the element before its
// first code.  A key x belongs to the lane whose value interval holds it;
// every owning lane walks its own codes to the first value >= x: x's rank,
// its neighbours and the byte span of the code x splits.  Edits are as in
// the element-array splice below, which also takes any leaf this kernel
// cannot (a code longer than 4 bytes, or a result over 512 bytes that still
// fits a larger leaf: state kFallback).  Per-leaf metadata is loaded for 32
// leaves at once; segments of a warp run independently (segment-masked
// shuffles and ballots) between those loads.
template <int SEG>
__global__ void __launch_bounds__(kT, SEG == 32 ? 4 : 3) k_insert_lane(MergeArgs a) {
  constexpr int SPW = 32 / SEG;              // segments (leaves) per warp step
  constexpr unsigned SEGBITS = SEG == 32 ? 0xFFFFFFFFu : ((1u << SEG) - 1u);
  extern __shared__ __align__(16) uint8_t smem[];
  if (a.st->err) return;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const unsigned sg = lane / SEG, sl = lane % SEG;
  const unsigned seg = SEGBITS << (sg * SEG);
  const unsigned wpb = blockDim.x >> 5;
  uint8_t* wbase = smem + (size_t)warp * lane_warp_bytes(SEG) + (size_t)sg * lane_seg_bytes(SEG);
  const uint64_t nL = a.st->n_lane;
  ull nbytes = 0;  // algorithmic bytes (lane 0 of each segment)
  ull dl = 0, db = 0;  // keys added, byte total change (lane 0 of each segment)
  uint64_t r0, r1;
  warp_share(nL, (uint64_t)blockIdx.x * wpb + warp, (uint64_t)gridDim.x * wpb, r0, r1);
  for (uint64_t tbase = r0; tbase < r1; tbase += 32) {
    // metadata of up to 32 touched leaves of the work list, one per lane
    const bool have = tbase + lane < r1;
    const uint32_t ti = have ? a.list_lane[tbase + lane] : 0u;
    uint32_t i_tb = 0, i_te = 0, i_uold = 0, i_j = 0, i_m = 0, i_fc0 = 0, i_fc1 = 0;
    if (have) {
      i_tb = a.T_begin[ti]; i_te = a.T_begin[ti + 1]; i_uold = a.T_oldused[ti];
      i_j = a.T_leaf[ti]; i_m = a.T_oldcnt[ti];
      i_fc0 = a.T_first_chunk[ti]; i_fc1 = a.T_first_chunk[ti + 1];
    }
    unsigned todo = __ballot_sync(FULL, have);
    while (todo) {
      // segment sg takes the sg-th remaining leaf of this step
      unsigned tm = todo;
      for (unsigned q = 0; q < sg; q++) tm &= tm - 1u;
      const bool mine = tm != 0;
      const unsigned src = mine ? (unsigned)(__ffs(tm) - 1) : 0u;
      const uint32_t t = __shfl_sync(FULL, ti, src);
      const uint32_t tb = __shfl_sync(FULL, i_tb, src), te = __shfl_sync(FULL, i_te, src);
      const uint32_t uold = __shfl_sync(FULL, i_uold, src), j = __shfl_sync(FULL, i_j, src);
      const uint32_t m = __shfl_sync(FULL, i_m, src);
      const uint32_t fc0 = __shfl_sync(FULL, i_fc0, src), fc1 = __shfl_sync(FULL, i_fc1, src);
#pragma unroll
      for (int q = 0; q < SPW; q++) todo &= todo - 1u;
      if (!mine) continue;
      lane_leaf<SEG, kLaneBatch>(a, wbase, sg, sl, seg, t, tb, te, uold, j, m, fc0, fc1, nbytes,
                                 dl, db);
    }
  }
  nbytes = warp_sum(sl == 0 ? nbytes : 0ull);
  dl = warp_sum(sl == 0 ? dl : 0ull);
  db = warp_sum(sl == 0 ? db : 0ull);
  if (lane == 0) {
    if (a.prof && nbytes) atomicAdd(a.prof, nbytes);
    if (dl) atomicAdd(&a.st->delta, dl);
    if (db) atomicAdd(&a.st->bytes_total, db);
  }
}

// ---------------------------------------------------------------------------
// Point path (Sec. 4: a batch much smaller than the set is applied as point
// updates instead of by the batch algorithm).  An untagged insert of at most
// kPointMax keys is sorted and routed (k_point_sort_route; the batch sort
// first above kPointRankMax keys); a
// plan pass then takes each touched leaf with a warp and decides whether the
// leaf's keys go in place: the lane-granular insert's conditions (at most 32
// keys, a non-empty leaf of at most 512 used bytes, codes of at most four
// bytes, a result of at most 512 bytes) and, in addition, that the leaf stays
// within its own density bound.  When every touched leaf does, an apply pass
// rewrites them (the same bytes the batch merge writes); otherwise nothing is
// written and the update runs the batch algorithm.  With no pending leaf and
// no leaf over its bound the batch algorithm's counting phase starts no walk,
// so both give the same structure.
constexpr uint32_t kPointMax = 16384;     // keys of an insert
constexpr uint32_t kPointDelMax = 4096;   // keys of a delete (its leaves are planned by one
                                          // lane each: larger deletes are faster batched)
constexpr uint32_t kPointRankMax = 4096;  // ranked in k_point_sort_route (the batch in one
                                          // block's shared memory); larger batches are
                                          // sorted first by the batch sort

constexpr int kPRT = 256;

// A warp per key: its stable rank (the lanes count over the batch, held in
// shared memory by every block, the keys below it and the equal keys before
// it) -- or, for a batch given sorted, rank = index (the plan pass checks the
// order) -- and its leaf by route_leaf's rule (the last leaf whose head is <= x,
// else leaf 0; 2^64-1 to the leaf heads[L] names), searched 32-ary in the
// head array: 31 probes per round trip, loaded together, narrow the range
// 32-fold, so 10^6 leaves take four.  Writes the key to u[rank] and its
// leaf to leaf_of[rank].  Clears the status words the point path uses.
__global__ void __launch_bounds__(kPRT) k_point_sort_route(const uint64_t* __restrict__ in,
                                                          uint32_t k, int sorted,
                                                          uint64_t* __restrict__ u,
                                                          uint32_t* __restrict__ leaf_of,
                                                          const uint64_t* __restrict__ heads,
                                                          uint64_t L, Status* st) {
  extern __shared__ __align__(16) uint64_t s_keys[];
  pdl_launch();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->err = 0;
    st->point_fb = 0;
    st->point_done = 0;
    st->delta = 0;
  }
  if (!sorted) {  // (a sorted batch is only read at each warp's own key)
    for (uint32_t i = threadIdx.x; i < k; i += kPRT) s_keys[i] = in[i];
    __syncthreads();
  }
  const unsigned lane = lane_id();
  const uint32_t i = blockIdx.x * (kPRT / 32) + (threadIdx.x >> 5);
  if (i >= k) return;
  const uint64_t x = sorted ? in[i] : s_keys[i];
  uint32_t r = i;
  if (!sorted) {
    uint32_t c = 0;
    for (uint32_t j = lane; j < k; j += 32) {
      const uint64_t y = s_keys[j];
      c += (y < x || (y == x && j < i)) ? 1u : 0u;
    }
    r = warp_sum(c);
  }
  uint64_t a = 0;  // heads before a are <= x; from b on they are > x
  if (x == KEY_MAX) {
    a = __ldg(heads + L) + 1;
  } else {
    uint64_t b = L;
    while (b - a > 32) {
      const uint64_t w = b - a;
      const uint64_t p = a + (uint64_t)(lane + 1) * w / 32;  // lanes 0..30
      const unsigned le = __ballot_sync(FULL, lane < 31 && __ldg(heads + p) <= x);
      const uint32_t c = (uint32_t)__popc(le);  // the probes <= x are a prefix
      const uint64_t na = c ? a + (uint64_t)c * w / 32 + 1 : a;
      const uint64_t nb = c < 31 ? a + (uint64_t)(c + 1) * w / 32 : b;
      a = na;
      b = nb;
    }
    a += (uint32_t)__popc(__ballot_sync(FULL, a + lane < b && __ldg(heads + a + lane) <= x));
  }
  if (lane == 0) {
    u[r] = x;
    leaf_of[r] = (uint32_t)(a ? a - 1 : 0);
  }
}

// Commit the staged result of the leaf whose first key is i: the rewritten
// bytes, used bytes, count and head (a warp; lane 0 adds to dl and db).
__device__ __forceinline__ void point_commit(const MergeArgs& a, uint32_t i, ull& dl, ull& db) {
  const PointRec R = a.prec[i];
  uint8_t* leafp = a.data + (size_t)R.leaf * a.LB;
  const uint8_t* src = a.pstage + (size_t)i * 512;
  const uint32_t q = R.lo + 16u * lane_id();
  if (q < R.wend)
    *reinterpret_cast<uint4*>(leafp + q) = *reinterpret_cast<const uint4*>(src + q);
  if (lane_id() == 0) {
    a.used[R.leaf] = R.nb;
    a.cnt[R.leaf] = R.newc;
    a.heads[R.leaf] = R.head;
    dl += R.added;
    db += (ull)(long long)R.dbytes;
  }
}

// Is sorted key i the first of its leaf, and which leaf ([tb, te) its keys;
// te = tb when more than 32 of the keys share the leaf)?  A warp.
__device__ __forceinline__ bool point_first(const uint32_t* __restrict__ leaf_of, uint32_t k,
                                            uint32_t i, uint32_t& j, uint32_t& te) {
  j = leaf_of[i];
  if (i > 0 && leaf_of[i - 1] == j) return false;
  // the leaf's keys end at the first of the next 32 in another leaf
  const uint32_t q = i + 1 + lane_id();
  const unsigned other = __ballot_sync(FULL, q >= k || leaf_of[q] != j);
  te = other ? i + (uint32_t)__ffs(other) : i;
  return true;
}

// Delete of the slice u[i, i + s) (s <= leafthr::kKeys) from leaf j by the
// thread-granular delete, staged: the warp copies the leaf to the staging
// slot of key i, then lane 0 plans the delete and rewrites the slot in
// place.  The leaf goes in place unless it holds a code over 4 bytes, would
// be emptied (the head fix-up is the batch algorithm's) or would leave its
// own bound.  wbase holds lane 0's scratch.
__device__ __forceinline__ uint32_t point_stage_delete(const MergeArgs& a, uint8_t* wbase,
                                                       uint32_t i, uint32_t s, uint32_t j) {
  constexpr uint32_t K = leafthr::kKeys;
  const unsigned lane = lane_id();
  const uint32_t uold = a.used[j], m = a.cnt[j];
  if (s > K || uold == 0) return kLeafBatch;
  uint8_t* slot = a.pstage + (size_t)i * 512;
  const uint8_t* leafp = a.data + (size_t)j * a.LB;
  if (16u * lane < a.LB)
    *reinterpret_cast<uint4*>(slot + 16u * lane) =
        *reinterpret_cast<const uint4*>(leafp + 16u * lane);
  __syncwarp();
  uint32_t verdict = kLeafBatch;
  if (lane == 0) {
    uint64_t* rval = reinterpret_cast<uint64_t*>(wbase);
    uint32_t* w32 = reinterpret_cast<uint32_t*>(wbase + 8 * K);
    const leafthr::Scratch S{w32, rval, w32 + K, w32 + 2 * K,
                             reinterpret_cast<int32_t*>(w32 + 3 * K), w32 + 4 * K, 1u};
    uint64_t y[K];
#pragma unroll
    for (uint32_t q = 0; q < K; q++) y[q] = q < s ? a.u[i + q] : 0ull;
    leafthr::Result R;
    R.E = 0;
    const uint32_t res = leafthr::plan_delete(slot, a.LB, uold, m, y, s, S, R);
    if (res == leafthr::kUnchanged) {
      verdict = kLeafSame;
    } else if (res == leafthr::kWritten && R.newc > 0 &&
               !node_violates(a.B, a.H, 0, 1, R.nb)) {
      leafthr::rewrite_forward(slot, a.LB, uold, S, R);
      leafthr::write_delete_edits(slot, S, R);
      PointRec rec;
      rec.head = R.newhead;
      rec.leaf = j;
      rec.nb = R.nb;
      rec.newc = R.newc;
      rec.lo = R.wlo;
      rec.wend = R.whi;
      rec.added = m - R.newc;
      rec.dbytes = (int32_t)R.nb - (int32_t)uold;
      a.prec[i] = rec;
      verdict = kLeafInPlace;
    }
  }
  return __shfl_sync(FULL, verdict, 0);
}

// The point path's plan pass, a warp per sorted key: the order of the keys
// is checked, and the warp of the first key of each leaf stages the leaf's
// result (an insert by kLaneStage, a delete by point_stage_delete) or counts
// the leaf in st->point_fb.  With COMMIT (few
// keys) the block that finishes last -- every block's stagings and counts
// are then visible -- commits every staged leaf itself when there is no
// error and no leaf for the batch algorithm, and writes the keys added to
// d_delta.
template <bool COMMIT, bool DEL>
__global__ void __launch_bounds__(kT, 4) k_point_plan(MergeArgs a,
                                                      const uint32_t* __restrict__ leaf_of,
                                                      uint32_t k, uint64_t* d_delta) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ bool s_last;
  __shared__ ull s_dl[kT / 32], s_db[kT / 32];
  pdl_wait();
  pdl_launch();
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const unsigned wpb = blockDim.x >> 5;
  uint8_t* wbase = smem + (size_t)warp * lane_warp_bytes(kLaneSeg);
  ull nbytes = 0, dl = 0, db = 0;
  ull nfb = 0;
  for (uint32_t i = blockIdx.x * wpb + warp; i < k; i += gridDim.x * wpb) {
    if (lane == 0 && i > 0 && a.u[i - 1] > a.u[i]) atomicOr(&a.st->err, kErrUnsorted);
    uint32_t j, te;
    if (!point_first(leaf_of, k, i, j, te)) continue;
    // the slice must be in order before the leaf is planned
    const bool down = lane + 1 < te - i && a.u[i + lane] > a.u[i + lane + 1];
    if (te == i || __any_sync(FULL, down)) {
      nfb++;
      continue;
    }
    const uint32_t r =
        DEL ? point_stage_delete(a, wbase, i, te - i, j)
            : lane_leaf<kLaneSeg, kLaneStage>(a, wbase, 0u, lane, FULL, 0u, i, te, a.used[j], j,
                                              a.cnt[j], 0u, 0u, nbytes, dl, db);
    nfb += r == kLeafBatch ? 1u : 0u;
    if (lane == 0 && r == kLeafSame) a.prec[i].leaf = 0xFFFFFFFFu;  // nothing to commit
  }
  if (lane == 0 && nfb) atomicAdd(&a.st->point_fb, nfb);
  if (!COMMIT) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&a.st->point_done, 1ull) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const volatile Status* vs = a.st;
  if (vs->err || vs->point_fb) return;
  dl = db = 0;
  for (uint32_t i = warp; i < k; i += wpb) {
    uint32_t j, te;
    if (point_first(leaf_of, k, i, j, te) && a.prec[i].leaf != 0xFFFFFFFFu)
      point_commit(a, i, dl, db);
  }
  if (lane == 0) { s_dl[warp] = dl; s_db[warp] = db; }
  __syncthreads();
  if (threadIdx.x == 0) {
    ull tdl = 0, tdb = 0;
    for (unsigned w = 0; w < wpb; w++) { tdl += s_dl[w]; tdb += s_db[w]; }
    a.st->delta = tdl;
    if (tdb) atomicAdd(&a.st->bytes_total, tdb);
    if (d_delta) *d_delta = tdl;
  }
}

// The point path's commit pass for larger batches: when there is no error
// and no leaf for the batch algorithm, a warp per sorted key commits the
// leaf the key is the first of; the block that finishes last writes the
// keys added to d_delta.
__global__ void __launch_bounds__(kT) k_point_commit(MergeArgs a,
                                                     const uint32_t* __restrict__ leaf_of,
                                                     uint32_t k, uint64_t* d_delta) {
  __shared__ bool s_last;
  pdl_wait();
  if (a.st->err || a.st->point_fb) return;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const unsigned wpb = blockDim.x >> 5;
  ull dl = 0, db = 0;
  for (uint32_t i = blockIdx.x * wpb + warp; i < k; i += gridDim.x * wpb) {
    uint32_t j, te;
    if (point_first(leaf_of, k, i, j, te) && a.prec[i].leaf != 0xFFFFFFFFu)
      point_commit(a, i, dl, db);
  }
  dl = warp_sum(dl);
  db = warp_sum(db);
  if (lane == 0) {
    if (dl) atomicAdd(&a.st->delta, dl);
    if (db) atomicAdd(&a.st->bytes_total, db);
  }
  if (!d_delta) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&a.st->point_done, 1ull) == gridDim.x - 1;
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    *d_delta = *reinterpret_cast<const volatile ull*>(&a.st->delta);
  }
}

// Insert of a slice of at most leafthr::kKeys keys into one leaf of byte
// codes, one thread per leaf (leaf_thread.cuh): the thread sums its leaf
// chunk by chunk up to the chunks where its keys land, places them and
// rewrites the bytes from the first edit on in place, 16 bytes at a time.  Slices this small are the common case of a
// batch that is small against the set (about one key per touched leaf), where
// a warp per leaf leaves most lanes idle.  A leaf with a code of more than 4
// bytes goes to the element-array splice (state kFallback); a result over LB
// bytes is left pending for the general merge.
constexpr int kThrT = 256;
constexpr int kThrBuckets = 128;  // tile sort buckets: 16-byte chunks of the old leaf

// DEL: the same for deletes of at most kThrKeys keys from a byte-code leaf
// (plan_delete, forward rewrite; never over LB bytes).
template <bool DEL>
__global__ void __launch_bounds__(kThrT) k_insert_thread(MergeArgs a) {
  constexpr uint32_t K = leafthr::kKeys;
  __shared__ uint32_t s_rpos[K * kThrT], s_rcode[K * kThrT];
  __shared__ uint64_t s_rval[K * kThrT];
  __shared__ uint32_t s_epos[K * kThrT], s_ekey[K * kThrT];
  __shared__ int32_t s_esa[K * kThrT];
  __shared__ uint32_t s_tile[kThrT];
  __shared__ uint32_t s_hist[kThrBuckets + 1];
  if (a.st->err) return;
  const unsigned tid = threadIdx.x;
  const leafthr::Scratch S{s_rpos + tid, s_rval + tid, s_rcode + tid, s_epos + tid,
                           s_esa + tid,  s_ekey + tid, (uint32_t)kThrT};
  const uint64_t n = a.st->nT;
  ull nbytes = 0;
  // Tiles of kThrT touched leaves; those of this kernel's class are sorted by
  // the size of the old leaf (counting sort in shared memory), so that the 32
  // leaves of a warp take about the same number of decode steps.
  for (uint64_t base = (uint64_t)blockIdx.x * kThrT; base < n; base += (uint64_t)gridDim.x * kThrT) {
    for (uint32_t i = tid; i <= kThrBuckets; i += kThrT) s_hist[i] = 0u;
    __syncthreads();
    const uint64_t idx = base + tid;
    uint32_t bkt = 0, slot = 0;
    bool mine = false;
    if (idx < n) {
      const uint32_t uo = a.T_oldused[idx];
      mine = thread_class(a.T_begin[idx + 1] - a.T_begin[idx], uo, a.small);
      if (mine) {
        bkt = min((uint32_t)kThrBuckets - 1u, (uo + 15u) >> 4);
        slot = atomicAdd(&s_hist[bkt], 1u);
      }
    }
    __syncthreads();
    if (tid < 32) {  // exclusive scan of the bucket counts, total in s_hist[128]
      static_assert(kThrBuckets == 128, "4 buckets per lane");
      const uint32_t c0 = s_hist[4 * tid], c1 = s_hist[4 * tid + 1], c2 = s_hist[4 * tid + 2],
                     c3 = s_hist[4 * tid + 3];
      const uint32_t sum = c0 + c1 + c2 + c3;
      const uint32_t inc = warp_incl_scan(sum), ex = inc - sum;
      s_hist[4 * tid] = ex;
      s_hist[4 * tid + 1] = ex + c0;
      s_hist[4 * tid + 2] = ex + c0 + c1;
      s_hist[4 * tid + 3] = ex + c0 + c1 + c2;
      if (tid == 31) s_hist[kThrBuckets] = inc;
    }
    __syncthreads();
    if (mine) s_tile[s_hist[bkt] + slot] = (uint32_t)idx;
    __syncthreads();
    ull dl = 0, db = 0;  // db: change of the byte total, mod 2^64
    if (tid < s_hist[kThrBuckets]) {
      const uint32_t t = s_tile[tid];
      const uint32_t tb = a.T_begin[t], s = a.T_begin[t + 1] - tb;
      const uint32_t uold = a.T_oldused[t], j = a.T_leaf[t], m = a.T_oldcnt[t];
      const uint32_t fc0 = a.T_first_chunk[t], fc1 = a.T_first_chunk[t + 1];
      uint8_t* leafp = a.data + (size_t)j * a.LB;
      // algorithmic bytes of a touched leaf: the old leaf, the new one and
      // 24 bytes of metadata (the new leaf added below once it is known)
      nbytes += uold + 24u;
      uint64_t y[K];
#pragma unroll
      for (uint32_t q = 0; q < K; q++) y[q] = q < s ? a.u[tb + q] : 0ull;
      leafthr::Result R;
      R.E = 0;
      const uint32_t res = DEL ? leafthr::plan_delete(leafp, a.LB, uold, m, y, s, S, R)
                               : leafthr::plan_leaf(leafp, a.LB, uold, m, y, s, S, R);
      if (res == leafthr::kLongCode) {
        a.T_state[t] = kFallback;
        a.list_v1[atomicAdd(&a.st->n_v1, 1ull)] = t;
      } else {
        uint32_t c0 = 0;
        if (res == leafthr::kUnchanged) {
          nbytes += uold;
          a.T_state[t] = kUnchanged;
          a.T_newcnt[t] = m;
          a.T_newbytes[t] = uold;
        } else if (res == leafthr::kTooBig) {
          a.T_state[t] = kPending;
          a.T_newcnt[t] = R.newc;
          a.T_newbytes[t] = R.nb;
          a.list_pend[atomicAdd(&a.st->n_pendl, 1ull)] = t;
          c0 = R.newc;
        } else {
          if (DEL) {
            leafthr::rewrite_forward(leafp, a.LB, uold, S, R);
            leafthr::write_delete_edits(leafp, S, R);
            if (R.newc == 0) atomicAdd(&a.st->nempty, 1ull);
          } else {
            leafthr::rewrite_leaf(leafp, a.LB, uold, S, R);
            leafthr::write_edits(leafp, y, S, R);
          }
          nbytes += R.nb;
          a.used[j] = R.nb;
          a.cnt[j] = R.newc;
          a.heads[j] = R.newhead;
          a.T_newcnt[t] = R.newc;
          a.T_newbytes[t] = R.nb;
          // the finalize pass's work for this leaf, done here
          dl += DEL ? m - R.newc : R.newc - m;
          db += (ull)R.nb - (ull)uold;
          if (node_violates(a.B, a.H, 0, 1, R.nb)) a.viol[atomicAdd(&a.st->nviol, 1ull)] = j;
          a.T_state[t] = kDone;
        }
        for (uint32_t cq = fc0; cq < fc1; cq++) a.chunk_cnt[cq] = cq == fc0 ? c0 : 0u;
        if (a.tag_counts)
          for (uint32_t q = 0; q < s; q++)
            if ((R.added >> q) & 1u) credit(a, tb + q);
      }
    }
    dl = warp_sum(dl);
    db = warp_sum(db);
    if (lane_id() == 0) {
      if (dl) atomicAdd(&a.st->delta, dl);
      if (db) atomicAdd(&a.st->bytes_total, db);
    }
    __syncthreads();
  }
  nbytes = warp_sum(nbytes);
  if (a.prof && lane_id() == 0 && nbytes) atomicAdd(a.prof, nbytes);
}

// Sort the touched leaves into the merge kernels' work lists: inserts of at
// most kThrKeys keys go to k_insert_thread, which walks the touched leaves
// itself (no list); other small inserts into leaves of at most 512 used
// bytes -> k_insert_lane; other small slices into non-empty leaves ->
// k_merge_small; the rest -> k_merge, one entry per
// work item (a slice of at most kChunk keys is merged whole by its first item,
// the others get a zero overflow count here).
__global__ void __launch_bounds__(kT) k_classify(MergeArgs a) {
  if (a.st->err) return;
  const unsigned lane = lane_id();
  const uint64_t nT = a.st->nT;
  for (uint64_t base = gtid() - lane; base < nT; base += gstride()) {
    const uint64_t t = base + lane;
    uint32_t cls = 3;
    uint32_t tb = 0, te = 0, fc0 = 0, fc1 = 0;
    if (t < nT) {
      tb = a.T_begin[t];
      te = a.T_begin[t + 1];
      const uint32_t uold = a.T_oldused[t];
      if (small_slice(tb, te, uold)) {
        const bool ins = !a.is_delete && !a.raw;
        cls = (!a.raw && thread_class(te - tb, uold, a.small)) ? 4u
            : (ins && lane_class(te - tb, uold, a.small)) ? 0u : 1u;
      } else {
        cls = 2;
        fc0 = a.T_first_chunk[t];
        fc1 = a.T_first_chunk[t + 1];
      }
    }
    warp_append(cls == 0, (uint32_t)t, a.list_lane, &a.st->n_lane);
    warp_append(cls == 1, (uint32_t)t, a.list_v1, &a.st->n_v1);
    if (cls == 2) {
      if (te - tb <= kChunk) {
        const ull i = atomicAdd(&a.st->n_gen, 1ull);
        a.list_gen[i] = fc0;
        for (uint32_t c = fc0 + 1; c < fc1; c++) a.chunk_cnt[c] = 0;
      } else {
        const ull i = atomicAdd(&a.st->n_gen, (ull)(fc1 - fc0));
        for (uint32_t c = fc0; c < fc1; c++) a.list_gen[i + (c - fc0)] = c;
      }
    }
  }
}

// Splice merge of a small slice into one leaf (warp per touched leaf).  The
// leaf is decoded once into shared memory (values and the byte position where
// each code ends); every key finds its rank by binary search in its own lane.
// Keys that land in the same gap (insert) or delete a run of neighbours form
// one edit: a byte range of the old leaf replaced by new bytes (new head
// and/or codes).  The new leaf is then the old bytes outside the edits, each
// shifted by the size change of the edits before it, plus the edits' bytes --
// the same bytes as encoding the merged sequence from scratch, produced
// without re-encoding the untouched codes.  A result over LB bytes is left
// pending for the general merge.
__global__ void __launch_bounds__(kT, 3) k_merge_small(MergeArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  pdl_wait();
  pdl_launch();
  if (a.st->err) return;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const unsigned wpb = blockDim.x >> 5;
  const uint32_t LB = a.LB;
  uint8_t* wbase = smem + (size_t)warp * small_warp_bytes(LB);
  uint64_t* old = reinterpret_cast<uint64_t*>(wbase);
  uint16_t* pos = reinterpret_cast<uint16_t*>(wbase + 8 * (size_t)LB);
  uint8_t* out = wbase + 10 * (size_t)LB;
  uint64_t* nk = reinterpret_cast<uint64_t*>(wbase + 11 * (size_t)LB + 32);
  uint32_t* nr = reinterpret_cast<uint32_t*>(nk + kSmall);
  uint32_t* es = nr + kSmall;
  uint32_t* ee = es + kSmall;
  uint32_t* en = ee + kSmall;
  int32_t* shc = reinterpret_cast<int32_t*>(en + kSmall);
  const uint64_t nV = a.st->n_v1;
  ull nbytes = 0;
  for (uint64_t li = (uint64_t)blockIdx.x * wpb + warp; li < nV; li += (uint64_t)gridDim.x * wpb) {
    const uint32_t t = a.list_v1[li];
    const uint32_t tb = a.T_begin[t], te = a.T_begin[t + 1];
    const uint32_t uold = a.T_oldused[t];
    const uint32_t s = te - tb;
    const uint32_t j = a.T_leaf[t];
    const uint32_t m = a.T_oldcnt[t];
    const uint32_t fc0 = a.T_first_chunk[t], fc1 = a.T_first_chunk[t + 1];
    uint8_t* leafp = a.data + (size_t)j * LB;
    nbytes += uold + 8u * s + 24u;
    warp_decode_pos(leafp, min(uold, LB), [&](uint32_t idx, uint64_t v, uint32_t p) {
      old[idx] = v;
      pos[idx] = (uint16_t)p;
    }, a.raw);
    __syncwarp();
    // the keys that change the leaf, with their ranks among the old elements
    uint64_t x = 0;
    uint32_t r = 0;
    bool keep = false;
    if (lane < s) {
      x = a.u[tb + lane];
      const bool dup = lane > 0 && a.u[tb + lane - 1] == x;
      r = (uint32_t)lower_bound(old, m, x);
      const bool present = r < m && old[r] == x;
      keep = !dup && (a.is_delete ? present : !present);
    }
    const unsigned kb = __ballot_sync(FULL, keep);
    const uint32_t nn = __popc(kb);
    if (keep) {
      const uint32_t k = __popc(kb & lanemask_lt());
      nk[k] = x;
      nr[k] = r;
    }
    __syncwarp();
    if (nn == 0) {
      if (lane == 0) {
        a.T_state[t] = kUnchanged;
        a.T_newcnt[t] = m;
        a.T_newbytes[t] = uold;
      }
      for (uint32_t c = fc0 + lane; c < fc1; c += 32) a.chunk_cnt[c] = 0;
      __syncwarp();
      continue;
    }
    // one edit per group: insert = keys of equal rank, delete = a run of
    // consecutive ranks
    bool lead = false;
    if (lane < nn) {
      const uint32_t rk = nr[lane];
      lead = lane == 0 || (a.is_delete ? nr[lane - 1] + 1 != rk : nr[lane - 1] != rk);
    }
    const unsigned lb = __ballot_sync(FULL, lead);
    const uint32_t E = __popc(lb);
    uint32_t e_os = 0, e_oe = 0, e_nl = 0, gend = 0, r0 = 0;
    if (lead) {
      const unsigned after = lb & ~((2u << lane) - 1u);
      gend = after ? (uint32_t)(__ffs(after) - 1) : nn;
      r0 = nr[lane];
      if (a.raw) {
        // cells: an insert adds one cell per key before old cell r0, a delete
        // removes cells r0 .. r1-1; no neighbouring cell changes
        if (!a.is_delete) { e_os = e_oe = 8u * r0; e_nl = 8u * (gend - lane); }
        else { e_os = 8u * r0; e_oe = 8u * (r0 + (gend - lane)); e_nl = 0; }
      } else if (!a.is_delete) {
        if (r0 == 0) { e_os = 0; e_oe = 8; }
        else if (r0 < m) { e_os = pos[r0 - 1] + 1u; e_oe = pos[r0] + 1u; }
        else { e_os = uold; e_oe = uold; }
        uint32_t len;
        uint64_t prev = nk[lane];
        len = (r0 == 0) ? 8u : leb_len(nk[lane] - old[r0 - 1]);
        for (uint32_t q = lane + 1; q < gend; q++) { len += leb_len(nk[q] - prev); prev = nk[q]; }
        if (r0 < m) len += leb_len(old[r0] - prev);
        e_nl = len;
      } else {
        const uint32_t r1 = r0 + (gend - lane);
        e_os = (r0 == 0) ? 0u : pos[r0 - 1] + 1u;
        e_oe = (r1 < m) ? pos[r1] + 1u : uold;
        e_nl = (r1 >= m) ? 0u : (r0 == 0 ? 8u : leb_len(old[r1] - old[r0 - 1]));
      }
    }
    const uint32_t eidx = __popc(lb & lanemask_lt());
    const int32_t delta = lead ? (int32_t)e_nl - (int32_t)(e_oe - e_os) : 0;
    const int32_t dinc = warp_incl_scan(delta);
    const int32_t total = __shfl_sync(FULL, dinc, 31);
    if (lead) {
      es[eidx] = e_os;
      ee[eidx] = e_oe;
      en[eidx] = (uint32_t)((int32_t)e_os + dinc - delta);
      shc[eidx] = dinc;
    }
    const uint32_t nb = (uint32_t)((int32_t)uold + total);
    const uint32_t newc = a.is_delete ? m - nn : m + nn;
    // new head: the first key when it goes before the old head; the first
    // survivor when the old head is deleted
    const uint32_t g0end = __shfl_sync(FULL, gend, 0);
    uint64_t newhead = old[0];
    if (nr[0] == 0) newhead = a.is_delete ? (g0end < m ? old[g0end] : KEY_MAX) : nk[0];
    __syncwarp();
    if (nb > LB) {
      if (lane == 0) {
        a.T_state[t] = kPending;
        a.T_newcnt[t] = newc;
        a.T_newbytes[t] = nb;
      }
      for (uint32_t c = fc0 + lane; c < fc1; c += 32) a.chunk_cnt[c] = (c == fc0) ? newc : 0u;
      if (keep) credit(a, tb + lane);
      __syncwarp();
      continue;
    }
    const uint32_t wend = (max(uold, nb) + 15u) & ~15u;
    for (uint32_t p = lane * 16; p < wend; p += 512)
      *reinterpret_cast<uint4*>(out + p) = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    // old bytes outside the edits, shifted
    splice_copy(leafp, uold, out, E, es, ee, shc);
    __syncwarp();
    // the edits' new bytes
    if (lead && a.raw) {
      if (!a.is_delete)
        for (uint32_t q = lane; q < gend; q++)
          reinterpret_cast<uint64_t*>(out + en[eidx])[q - lane] = nk[q];
    } else if (lead) {
      uint8_t* o = out + en[eidx];
      if (!a.is_delete) {
        uint64_t prev = nk[lane];
        if (r0 == 0) {
#pragma unroll
          for (int b = 0; b < 8; b++) o[b] = (uint8_t)(prev >> (8 * b));
          o += 8;
        } else {
          o += leb_put(o, prev - old[r0 - 1]);
        }
        for (uint32_t q = lane + 1; q < gend; q++) { o += leb_put(o, nk[q] - prev); prev = nk[q]; }
        if (r0 < m) leb_put(o, old[r0] - prev);
      } else {
        const uint32_t r1 = r0 + (gend - lane);
        if (r1 < m) {
          if (r0 == 0) {
#pragma unroll
            for (int b = 0; b < 8; b++) o[b] = (uint8_t)(old[r1] >> (8 * b));
          } else {
            leb_put(o, old[r1] - old[r0 - 1]);
          }
        }
      }
    }
    __syncwarp();
    for (uint32_t p = lane * 16; p < wend; p += 512)
      *reinterpret_cast<uint4*>(leafp + p) = *reinterpret_cast<const uint4*>(out + p);
    nbytes += wend;
    if (keep) credit(a, tb + lane);
    if (lane == 0) {
      a.used[j] = nb;
      a.cnt[j] = newc;
      a.heads[j] = newc ? newhead : KEY_MAX;
      a.T_state[t] = kInPlace;
      a.T_newcnt[t] = newc;
      a.T_newbytes[t] = nb;
      if (newc == 0) atomicAdd(&a.st->nempty, 1ull);
    }
    for (uint32_t c = fc0 + lane; c < fc1; c += 32) a.chunk_cnt[c] = 0;
    __syncwarp();
  }
  if (a.prof && lane == 0 && nbytes) atomicAdd(a.prof, nbytes);
}

// WRITE == false: count every work item, rewrite single-item leaves in place
// when they fit.  WRITE == true: recompute the items of pending leaves and
// store their merged elements in the overflow buffer.
template <bool WRITE>
__global__ void __launch_bounds__(kT, 2) k_merge(MergeArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  pdl_wait();
  pdl_launch();
  if (a.st->err) return;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const unsigned wpb = blockDim.x >> 5;
  const uint32_t LB = a.LB;
  uint64_t* old = reinterpret_cast<uint64_t*>(smem + (size_t)warp * merge_warp_bytes(LB));
  uint64_t* z = old + LB;
  uint64_t* sl = z + LB + kChunk;
  uint64_t* nk = sl + kChunk;
  uint8_t* buf = reinterpret_cast<uint8_t*>(nk + kChunk);
  // count mode: the work items of the list; write mode: the items of pending
  // leaves, 32 screened per step (one per lane)
  const uint64_t nitems = WRITE ? a.st->nchunks : a.st->n_gen;
  uint64_t r0, r1;
  warp_share(nitems, (uint64_t)blockIdx.x * wpb + warp, (uint64_t)gridDim.x * wpb, r0, r1);
  for (uint64_t base = r0; base < r1; base += 32) {
   bool need = false;
   uint64_t myc = 0;
   {
    const uint64_t cc = base + lane;
    if (cc < r1) {
      if (WRITE) {
        myc = cc;
        need = a.T_state[a.chunk_tid[cc]] == kPending;
      } else {
        myc = a.list_gen[cc];
        need = true;
      }
    }
   }
   unsigned todo = __ballot_sync(FULL, need);
   while (todo) {
    const uint64_t c = __shfl_sync(FULL, myc, __ffs(todo) - 1);
    todo &= todo - 1;
    const uint32_t t = a.chunk_tid[c];
    const uint32_t j = a.chunk_leaf[c];
    uint32_t b = a.chunk_begin[c], e = a.chunk_begin[c + 1];
    const uint32_t tb = a.T_begin[t], te = a.T_begin[t + 1];
    // a slice of at most kChunk keys that the chunk grid happens to split is
    // merged whole by its first item (the others have nothing to do)
    if (te - tb <= kChunk) {
      if (b != tb) {
        if (!WRITE && lane == 0) a.chunk_cnt[c] = 0;
        continue;
      }
      e = te;
    }
    const bool first = (b == tb), last = (e == te);
    const uint32_t s = e - b;
    const uint32_t uold = a.T_oldused[t], m = a.T_oldcnt[t];
    uint8_t* leafp = a.data + (size_t)j * LB;
    warp_decode(leafp, min(uold, LB), [&](uint32_t idx, uint64_t v) { old[idx] = v; }, a.raw);
    for (uint32_t i = lane; i < s; i += 32) sl[i] = a.u[b + i];
    __syncwarp();
    const bool has_hi = !last;
    const uint64_t hiv = has_hi ? a.u[e] : 0;
    const uint64_t lov = sl[0];
    const uint32_t oa = first ? 0u : (uint32_t)lower_bound(old, m, lov);
    const uint32_t ob = has_hi ? (uint32_t)lower_bound(old, m, hiv) : m;
    uint32_t r = 0;
    if (!a.is_delete) {
      uint32_t nn = 0;
      for (uint32_t i0 = 0; i0 < s; i0 += 32) {
        const uint32_t i = i0 + lane;
        bool keep = false;
        uint64_t x = 0;
        if (i < s) {
          x = sl[i];
          keep = (!has_hi || x < hiv) && (i == 0 || x != sl[i - 1]) && !bsearch_sm(old, m, x);
        }
        const unsigned bal = __ballot_sync(FULL, keep);
        if (keep) nk[nn + __popc(bal & lanemask_lt())] = x;
        if (!WRITE && keep) credit(a, b + i);
        nn += __popc(bal);
      }
      __syncwarp();
      for (uint32_t q = oa + lane; q < ob; q += 32) {
        const uint64_t x = old[q];
        z[(q - oa) + (uint32_t)lower_bound(nk, nn, x)] = x;
      }
      for (uint32_t i = lane; i < nn; i += 32) {
        const uint64_t x = nk[i];
        z[i + (uint32_t)lower_bound(old + oa, ob - oa, x)] = x;
      }
      r = (ob - oa) + nn;
    } else {
      for (uint32_t q0 = oa; q0 < ob; q0 += 32) {
        const uint32_t q = q0 + lane;
        bool keep = false;
        uint64_t x = 0;
        if (q < ob) {
          x = old[q];
          const uint32_t p = (uint32_t)lower_bound(sl, s, x);
          keep = !(p < s && sl[p] == x);
          if (!WRITE && !keep) credit(a, b + p);
        }
        const unsigned bal = __ballot_sync(FULL, keep);
        if (keep) z[r + __popc(bal & lanemask_lt())] = x;
        r += __popc(bal);
      }
    }
    __syncwarp();
    // predecessor of z[0] in the whole merged leaf (items after the first)
    bool has_pred = false;
    uint64_t pred = 0;
    if (!first) {
      if (!a.is_delete) {
        if (oa > 0) { pred = old[oa - 1]; has_pred = true; }
        const uint64_t idx = lower_bound(a.u + tb, b - tb, lov);
        if (idx > 0) {
          const uint64_t x = a.u[tb + idx - 1];
          if (!has_pred || x > pred) pred = x;
          has_pred = true;
        }
      } else {
        for (int64_t q0 = (int64_t)oa - 1; q0 >= 0 && !has_pred; q0 -= 32) {
          const int64_t q = q0 - (int64_t)lane;
          bool alive = false;
          uint64_t x = 0;
          if (q >= 0) {
            x = old[q];
            const uint64_t p = lower_bound(a.u + tb, b - tb, x);
            alive = !(p < b - tb && a.u[tb + p] == x);
          }
          const unsigned bal = __ballot_sync(FULL, alive);
          if (bal) {
            pred = __shfl_sync(FULL, x, __ffs(bal) - 1);
            has_pred = true;
          }
        }
      }
    }
    uint32_t bsum = 0;
    for (uint32_t i = lane; i < r; i += 32)
      bsum += a.raw ? 8u
                    : (i == 0) ? (has_pred ? leb_len(z[0] - pred) : 8u) : leb_len(z[i] - z[i - 1]);
    bsum = warp_sum(bsum);
    if (WRITE) {
      const uint64_t off = a.chunk_off[c];
      for (uint32_t i = lane; i < r; i += 32) a.ovf[off + i] = z[i];
      __syncwarp();
      continue;
    }
    const bool single = first && last;
    if (single) {
      if (r == m) {
        if (lane == 0) {
          a.T_state[t] = kUnchanged;
          a.T_newcnt[t] = m;
          a.T_newbytes[t] = uold;
          a.chunk_cnt[c] = 0;
        }
      } else if (bsum <= LB) {
        for (uint32_t p = lane * 16; p < LB; p += 512)
          *reinterpret_cast<uint4*>(buf + p) = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();
        const uint32_t nb = warp_encode(z, r, buf, a.raw);
        const uint32_t wend = (max(uold, nb) + 15u) & ~15u;
        for (uint32_t p = lane * 16; p < wend; p += 512)
          *reinterpret_cast<uint4*>(leafp + p) = *reinterpret_cast<const uint4*>(buf + p);
        if (lane == 0) {
          a.used[j] = nb;
          a.cnt[j] = r;
          a.heads[j] = r ? z[0] : KEY_MAX;
          a.T_state[t] = kInPlace;
          a.T_newcnt[t] = r;
          a.T_newbytes[t] = nb;
          a.chunk_cnt[c] = 0;
          if (nb != bsum) atomicOr(&a.st->err, kErrState);
          if (r == 0) atomicAdd(&a.st->nempty, 1ull);
        }
      } else if (lane == 0) {
        a.T_state[t] = kPending;
        a.T_newcnt[t] = r;
        a.T_newbytes[t] = bsum;
        a.chunk_cnt[c] = r;
      }
    } else if (lane == 0) {
      atomicAdd(&a.T_newcnt[t], r);
      atomicAdd(&a.T_newbytes[t], (ull)bsum);
      a.T_state[t] = kPending;
      a.chunk_cnt[c] = r;
    }
    __syncwarp();
   }
  }
}

// ---------------------------------------------------------------------------
// 4. counting
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mark_node(uint32_t* bits, const Levels& lv, unsigned h, uint64_t a,
                                          uint64_t* cand, Status* st) {
  const uint64_t idx = a >> h;
  uint32_t* w = bits + lv.off[h] + (idx >> 5);
  const uint32_t bit = 1u << (idx & 31);
  const uint32_t old = atomicOr(w, bit);
  if (!(old & bit)) {
    const ull c = atomicAdd(&st->ncand, 1ull);
    cand[c] = ((uint64_t)h << 56) | a;
  }
}

struct FinArgs {
  uint32_t* used;
  uint32_t* cnt;
  const uint32_t *T_leaf, *T_first_chunk, *T_oldcnt, *T_newcnt, *T_begin, *T_oldused;
  ull* merge_bytes;  // profiling: algorithmic bytes of the merge (nullable)
  uint32_t* T_state;
  const ull* T_newbytes;
  uint32_t* chunk_cnt;
  const uint32_t* chunk_tid;
  const uint32_t *list_v1, *list_gen, *list_pend;
  uint32_t* viol;
  uint64_t* cand;
  uint32_t* bits;
  Levels lv;
  Bounds B;
  unsigned H;
  int is_delete;
  Status* st;
};

__global__ void __launch_bounds__(kT) k_finalize(FinArgs a) {
  pdl_wait();
  pdl_launch();
  if (a.st->err) return;
  ull mb = 0, dl = 0, np = 0, db = 0, ov = 0;  // db: change of the byte total, mod 2^64
  // the touched leaves the thread- and lane-granular inserts did not finish
  // themselves: the element-array splice's list, the general merge's leaves
  // (each once, by its first work item) and the pending leaves they left
  const uint64_t nv = a.st->n_v1, ng = a.st->n_gen, npl = a.st->n_pendl;
  for (uint64_t i = gtid(); i < nv + ng + npl; i += gstride()) {
    uint64_t t;
    if (i < nv) {
      t = a.list_v1[i];
    } else if (i < nv + ng) {
      const uint32_t c = a.list_gen[i - nv];
      t = a.chunk_tid[c];
      if (a.T_first_chunk[t] != c) continue;
    } else {
      t = a.list_pend[i - nv - ng];
    }
    const uint32_t state = a.T_state[t];
    const uint32_t oldc = a.T_oldcnt[t], newc = a.T_newcnt[t];
    const uint32_t j = a.T_leaf[t];
    if (a.merge_bytes && state != kUnchanged && a.T_begin[t + 1] - a.T_begin[t] > kSmall) {
      // leaves of the element-array / general merge: old leaf, slice,
      // metadata, and the rewrite when in place
      mb += a.T_oldused[t] + 8ull * (a.T_begin[t + 1] - a.T_begin[t]) + 24;
      if (state == kInPlace) mb += (max(a.T_oldused[t], (uint32_t)a.T_newbytes[t]) + 15u) & ~15u;
    }
    if (newc == oldc) {
      if (state == kPending) {
        a.T_state[t] = kUnchanged;
        for (uint32_t c = a.T_first_chunk[t]; c < a.T_first_chunk[t + 1]; c++) a.chunk_cnt[c] = 0;
      }
      continue;
    }
    dl += (ull)(a.is_delete ? oldc - newc : newc - oldc);
    const uint64_t nb = a.T_newbytes[t];
    db += nb - (ull)a.T_oldused[t];
    if (state == kPending) {
      a.used[j] = (uint32_t)nb;
      a.cnt[j] = newc;
      np++;
      // its merged elements, counted per work item (the overflow total)
      for (uint32_t c = a.T_first_chunk[t]; c < a.T_first_chunk[t + 1]; c++) ov += a.chunk_cnt[c];
    }
    if (node_violates(a.B, a.H, 0, 1, nb)) {
      const ull v = atomicAdd(&a.st->nviol, 1ull);
      a.viol[v] = j;
    } else if (state == kPending) {
      mark_node(a.bits, a.lv, 0, j, a.cand, a.st);
    }
  }
  // one atomic per warp for the batch totals
  dl = warp_sum(dl);
  np = warp_sum(np);
  db = warp_sum(db);
  ov = warp_sum(ov);
  if (lane_id() == 0) {
    if (dl) atomicAdd(&a.st->delta, dl);
    if (np) atomicAdd(&a.st->npend, np);
    if (db) atomicAdd(&a.st->bytes_total, db);
    if (ov) atomicAdd(&a.st->novf, ov);
  }
  if (a.merge_bytes) {
    mb = warp_sum(mb);
    if (lane_id() == 0 && mb) atomicAdd(a.merge_bytes, mb);
  }
}

__global__ void k_put_u64(uint64_t* dst, uint64_t v) { *dst = v; }

__global__ void __launch_bounds__(kT) k_check_tags(const uint32_t* __restrict__ tags, uint64_t k,
                                                   uint64_t ntags, Status* st) {
  bool bad = false;
  for (uint64_t i = gtid(); i < k; i += gstride()) bad |= tags[i] >= ntags;
  if (__any_sync(FULL, bad) && lane_id() == 0) atomicOr(&st->err, kErrUnsorted);
}

struct WalkArgs {
  const uint32_t* viol;
  const uint64_t* P;
  uint64_t L;
  uint32_t* bits;
  uint64_t* cand;
  Levels lv;
  Bounds B;
  unsigned H;
  Status* st;
};

__global__ void __launch_bounds__(kT) k_walk(WalkArgs a) {
  pdl_wait();
  pdl_launch();
  if (gtid() == 0) a.st->total_bytes = a.P[a.L];
  const uint64_t nv = a.st->nviol;
  for (uint64_t v = gtid(); v < nv; v += gstride()) {
    const uint64_t j = a.viol[v];
    bool done = false;
    for (unsigned h = 1; h <= a.H && !done; h++) {
      const uint64_t s = (j >> h) << h;
      const uint64_t e = min(s + ((uint64_t)1 << h), a.L);
      if (!node_violates(a.B, a.H, h, e - s, a.P[e] - a.P[s])) {
        mark_node(a.bits, a.lv, h, s, a.cand, a.st);
        done = true;
      }
    }
    if (!done) a.st->resize = 1;
  }
}

__global__ void __launch_bounds__(kT) k_maximal(const uint64_t* __restrict__ cand,
                                                const uint32_t* __restrict__ bits, Levels lv,
                                                unsigned H, uint64_t L, uint64_t* wins,
                                                Status* st) {
  pdl_wait();
  pdl_launch();
  if (st->resize) return;
  const uint64_t nc = st->ncand;
  for (uint64_t c = gtid(); c < nc; c += gstride()) {
    const uint64_t v = cand[c];
    const unsigned h = (unsigned)(v >> 56);
    const uint64_t a = v & ((1ull << 56) - 1);
    bool maximal = true;
    for (unsigned h2 = h + 1; h2 <= H && maximal; h2++) {
      const uint64_t idx = a >> h2;
      if (bits[lv.off[h2] + (idx >> 5)] & (1u << (idx & 31))) maximal = false;
    }
    if (maximal) {
      const uint64_t W = min((uint64_t)1 << h, L - a);
      const ull w = atomicAdd(&st->nwin, 1ull);
      wins[2 * w] = a;
      wins[2 * w + 1] = W;
      atomicAdd(&st->win_leaves, (ull)W);
    }
  }
}

__global__ void __launch_bounds__(kT) k_clear_bits(const uint64_t* __restrict__ cand,
                                                   uint32_t* bits, Levels lv, Status* st) {
  pdl_wait();
  pdl_launch();
  const uint64_t nc = st->ncand;
  for (uint64_t c = gtid(); c < nc; c += gstride()) {
    const uint64_t v = cand[c];
    const unsigned h = (unsigned)(v >> 56);
    const uint64_t idx = (v & ((1ull << 56) - 1)) >> h;
    atomicAnd(bits + lv.off[h] + (idx >> 5), ~(1u << (idx & 31)));
  }
}

// ---------------------------------------------------------------------------
// 5. redistribution
// ---------------------------------------------------------------------------
// Windows: src leaves [sa, sa + sW) of the source arrays, dst leaves
// [da, da + dW) of the destination arrays.  win_src holds (sa, sW) pairs,
// win_dst (da, dW) pairs; leaf_off / dst_off are their exclusive prefix sums
// of sW / dW; elem_off the element offsets (filled after the source counts).
struct WinArgs {
  const uint64_t* win_src;
  const uint64_t* win_dst;
  const uint64_t* leaf_off;
  const uint64_t* dst_off;
  uint64_t* elem_off;
  uint64_t nwin;
};

__device__ __forceinline__ uint64_t find_seg(const uint64_t* off, uint64_t nseg, uint64_t x) {
  // last s with off[s] <= x
  return upper_count(off, nseg + 1, x) - 1;
}

__global__ void __launch_bounds__(kT) k_win_sizes(const uint64_t* __restrict__ wins, uint64_t nwin,
                                                  uint64_t* __restrict__ sizes) {
  pdl_wait();
  pdl_launch();
  for (uint64_t w = gtid(); w < nwin; w += gstride()) sizes[w] = wins[2 * w + 1];
}

// Element count of every source leaf; the leaves' bytes leave the total
// (the encode adds the new ones).
__global__ void __launch_bounds__(kT) k_src_counts(WinArgs w, const uint32_t* __restrict__ cnt,
                                                   const uint32_t* __restrict__ used, uint64_t nsrc,
                                                   uint32_t* __restrict__ srccnt, Status* st) {
  pdl_wait();
  pdl_launch();
  ull gone = 0;
  for (uint64_t f = gtid(); f < nsrc; f += gstride()) {
    const uint64_t s = find_seg(w.leaf_off, w.nwin, f);
    const uint64_t j = w.win_src[2 * s] + (f - w.leaf_off[s]);
    srccnt[f] = cnt[j];
    gone += used[j];
  }
  gone = warp_sum(gone);
  if (lane_id() == 0 && gone) atomicAdd(&st->bytes_total, 0ull - gone);
}

__global__ void k_elem_offsets(WinArgs w, const uint64_t* __restrict__ srcoff, Status* st) {
  pdl_wait();
  pdl_launch();
  for (uint64_t s = gtid(); s <= w.nwin; s += gstride()) w.elem_off[s] = srcoff[w.leaf_off[s]];
  if (gtid() == 0) st->nelem = srcoff[w.leaf_off[w.nwin]];
}

struct UnpackArgs {
  WinArgs w;
  uint64_t nsrc;
  const uint8_t* data;
  const uint32_t* used;
  const uint32_t* cnt;
  uint32_t LB;
  const uint64_t* srcoff;
  // pending leaves of the current batch (sorted by leaf)
  const uint32_t* T_leaf;
  const uint32_t* T_state;
  const uint32_t* T_first_chunk;
  const uint64_t* chunk_off;
  uint64_t nT;
  const uint64_t* ovf;
  uint64_t* E;
  Status* st;
  int raw;
};

__global__ void __launch_bounds__(kT) k_unpack(UnpackArgs a) {
  pdl_wait();
  pdl_launch();
  const unsigned lane = lane_id();
  const uint64_t gw = gtid() >> 5, nw = gstride() >> 5;
  for (uint64_t f = gw; f < a.nsrc; f += nw) {
    const uint64_t s = find_seg(a.w.leaf_off, a.w.nwin, f);
    const uint64_t j = a.w.win_src[2 * s] + (f - a.w.leaf_off[s]);
    uint64_t* dst = a.E + a.srcoff[f];
    bool pend = false;
    uint64_t t = 0;
    if (a.nT) {
      t = lower_bound(a.T_leaf, a.nT, j);
      pend = t < a.nT && a.T_leaf[t] == j && a.T_state[t] == kPending;
    }
    if (pend) {
      const uint64_t off = a.chunk_off[a.T_first_chunk[t]];
      const uint32_t m = a.cnt[j];
      for (uint32_t i = lane; i < m; i += 32) dst[i] = a.ovf[off + i];
    } else {
      const uint32_t m = a.cnt[j];
      const uint32_t got = warp_decode(a.data + j * a.LB, min(a.used[j], a.LB),
                                       [&](uint32_t idx, uint64_t v) { if (idx < m) dst[idx] = v; },
                                       a.raw);
      if (lane == 0 && got != m) atomicOr(&a.st->err, kErrState);
    }
  }
}

__global__ void __launch_bounds__(kT) k_costs(WinArgs w, const uint64_t* __restrict__ E,
                                              const ull* nelem, uint8_t* __restrict__ cost,
                                              int raw) {
  pdl_wait();
  pdl_launch();
  const uint64_t n = *nelem;
  for (uint64_t i = gtid(); i < n; i += gstride()) {
    const uint64_t s = find_seg(w.elem_off, w.nwin, i);
    cost[i] = (raw || i == w.elem_off[s]) ? (uint8_t)8 : (uint8_t)leb_len(E[i] - E[i - 1]);
  }
}

__global__ void __launch_bounds__(kT) k_starts(WinArgs w, const uint64_t* __restrict__ C,
                                               uint64_t ndst, uint64_t* __restrict__ dstart) {
  pdl_wait();
  pdl_launch();
  typedef unsigned __int128 u128;
  for (uint64_t g = gtid(); g < ndst; g += gstride()) {
    const uint64_t s = find_seg(w.dst_off, w.nwin, g);
    const uint64_t wl = g - w.dst_off[s];
    const uint64_t Wd = w.win_dst[2 * s + 1];
    const uint64_t e0 = w.elem_off[s], e1 = w.elem_off[s + 1];
    const uint64_t B = C[e0], S = C[e1] - B;
    const uint64_t theta = (uint64_t)((u128)wl * S / Wd);
    dstart[g] = e0 + lower_bound(C + e0, e1 - e0 + 1, B + theta);
  }
}

struct EncodeArgs {
  WinArgs w;
  uint64_t ndst;
  const uint64_t* dstart;
  const uint64_t* E;
  const uint64_t* C;
  uint8_t* data;
  uint32_t* used;
  uint32_t* cnt;
  uint64_t* heads;
  uint32_t LB;
  Status* st;
  int raw;
};

__global__ void __launch_bounds__(kT) k_encode(EncodeArgs a) {
  pdl_wait();
  pdl_launch();
  extern __shared__ __align__(16) uint8_t smem[];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  uint8_t* buf = smem + (size_t)warp * a.LB;
  const uint64_t gw = gtid() >> 5, nw = gstride() >> 5;
  ull added = 0;  // lane 0: bytes of this warp's leaves
  for (uint64_t g = gw; g < a.ndst; g += nw) {
    const uint64_t s = find_seg(a.w.dst_off, a.w.nwin, g);
    const uint64_t wl = g - a.w.dst_off[s];
    const uint64_t Wd = a.w.win_dst[2 * s + 1];
    const uint64_t j = a.w.win_dst[2 * s] + wl;
    const uint64_t b = a.dstart[g];
    const uint64_t e = (wl + 1 < Wd) ? a.dstart[g + 1] : a.w.elem_off[s + 1];
    const uint32_t r = (uint32_t)(e - b);
    // bytes: the first element becomes an 8-byte head
    uint64_t nb = 0;
    if (r) nb = a.C[e] - a.C[b + 1] + 8;
    uint8_t* leafp = a.data + j * a.LB;
    if (nb > a.LB) {
      if (lane == 0) atomicOr(&a.st->err, kErrFit);
      continue;
    }
    for (uint32_t p = lane * 16; p < a.LB; p += 512)
      *reinterpret_cast<uint4*>(buf + p) = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    const uint32_t got = warp_encode(a.E + b, r, buf, a.raw);
    for (uint32_t p = lane * 16; p < a.LB; p += 512)
      *reinterpret_cast<uint4*>(leafp + p) = *reinterpret_cast<const uint4*>(buf + p);
    if (lane == 0) {
      a.used[j] = got;
      a.cnt[j] = r;
      a.heads[j] = r ? a.E[b] : KEY_MAX;
      added += got;
      if (got != nb) atomicOr(&a.st->err, kErrState);
      if (r == 0) atomicAdd(&a.st->nempty, 1ull);
    }
    __syncwarp();
  }
  if (lane == 0 && added) atomicAdd(&a.st->bytes_total, added);
}

// Head index of empty leaves: the head of the next non-empty leaf, or
// 2^64-1.  One block; each thread owns a contiguous segment.
// Head fix-up (R5): every empty leaf's head-index entry becomes the head of
// the next non-empty leaf (2^64-1 if none), heads[L] the index of the last
// non-empty leaf, status->empties the number of empty leaves.  Three passes
// over tiles of kFHTile leaves: per-tile first non-empty head and counts;
// one block turns those into each tile's carry (the first non-empty head
// after it); per-tile fill with a block-wide suffix scan.
constexpr int kFH = 1024, kFHItems = 4;
constexpr uint64_t kFHTile = (uint64_t)kFH * kFHItems;

struct FHTile {
  uint64_t first;     // head of the tile's first non-empty leaf
  uint64_t carry;     // first non-empty head after the tile (valid if carry_ok)
  uint64_t last1;     // 1 + index of the tile's last non-empty leaf (0: none)
  uint32_t has_first, carry_ok, empties, pad;
};

__global__ void __launch_bounds__(kFH) k_fh_tiles(const uint32_t* __restrict__ used,
                                                  const uint64_t* __restrict__ heads, uint64_t L,
                                                  FHTile* __restrict__ tiles) {
  pdl_wait();
  pdl_launch();
  __shared__ int first_t;
  __shared__ unsigned int ne_s;
  __shared__ ull last_s;
  if (threadIdx.x == 0) { first_t = kFH; ne_s = 0; last_s = 0; }
  __syncthreads();
  const uint64_t j0 = blockIdx.x * kFHTile + (uint64_t)threadIdx.x * kFHItems;
  unsigned int ne = 0;
  ull l1 = 0;
  uint64_t fj = KEY_MAX;
#pragma unroll
  for (int q = 0; q < kFHItems; q++) {
    const uint64_t j = j0 + q;
    if (j < L) {
      if (used[j]) { if (fj == KEY_MAX) fj = j; l1 = j + 1; }
      else ne++;
    }
  }
  if (fj != KEY_MAX) atomicMin(&first_t, (int)threadIdx.x);
  if (ne) atomicAdd(&ne_s, ne);
  if (l1) atomicMax(&last_s, l1);
  __syncthreads();
  FHTile& t = tiles[blockIdx.x];
  if ((int)threadIdx.x == first_t) t.first = heads[fj];
  if (threadIdx.x == 0) {
    t.has_first = first_t < kFH;
    t.empties = ne_s;
    t.last1 = last_s;
  }
}

// One block: carry of every tile (first non-empty head in later tiles), the
// empty-leaf count and heads[L].
__global__ void __launch_bounds__(kFH) k_fh_carry(FHTile* __restrict__ tiles, uint64_t nt,
                                                  uint64_t* __restrict__ heads, uint64_t L,
                                                  Status* st) {
  pdl_wait();
  pdl_launch();
  __shared__ uint64_t cv[kFH];
  __shared__ uint32_t cok[kFH];
  __shared__ ull ne_s, last_s;
  if (threadIdx.x == 0) { ne_s = 0; last_s = 0; }
  __syncthreads();
  const uint64_t per = (nt + kFH - 1) / kFH;
  const uint64_t c0 = min(nt, threadIdx.x * per), c1 = min(nt, c0 + per);
  // this thread's chunk of tiles: its first non-empty head, counts
  uint64_t fv = 0;
  bool fok = false;
  ull ne = 0, l1 = 0;
  for (uint64_t b = c0; b < c1; b++) {
    if (!fok && tiles[b].has_first) { fok = true; fv = tiles[b].first; }
    ne += tiles[b].empties;
    l1 = max(l1, (ull)tiles[b].last1);
  }
  cv[threadIdx.x] = fv;
  cok[threadIdx.x] = fok;
  atomicAdd(&ne_s, ne);
  if (l1) atomicMax(&last_s, l1);
  __syncthreads();
  if (threadIdx.x == 0) {
    // exclusive suffix over the chunks, in place
    uint64_t nv = 0;
    uint32_t nok = 0;
    for (int t = kFH - 1; t >= 0; t--) {
      const uint64_t v = cv[t];
      const uint32_t ok = cok[t];
      cv[t] = nv;
      cok[t] = nok;
      if (ok) { nv = v; nok = 1; }
    }
    st->empties = ne_s;
    heads[L] = last_s ? last_s - 1 : 0;  // routing of the key 2^64-1
  }
  __syncthreads();
  uint64_t nv = cv[threadIdx.x];
  uint32_t nok = cok[threadIdx.x];
  for (uint64_t b = c1; b-- > c0;) {
    tiles[b].carry = nv;
    tiles[b].carry_ok = nok;
    if (tiles[b].has_first) { nv = tiles[b].first; nok = 1; }
  }
}

__global__ void __launch_bounds__(kFH) k_fh_fill(const uint32_t* __restrict__ used,
                                                 uint64_t* __restrict__ heads, uint64_t L,
                                                 const FHTile* __restrict__ tiles) {
  pdl_wait();
  pdl_launch();
  __shared__ uint64_t wv[kFH / 32], wc[kFH / 32];
  __shared__ uint32_t wok[kFH / 32], wcok[kFH / 32];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const uint64_t j0 = blockIdx.x * kFHTile + (uint64_t)threadIdx.x * kFHItems;
  // first non-empty head of this thread's leaves
  bool ok = false;
  uint64_t v = 0;
#pragma unroll
  for (int q = 0; q < kFHItems; q++) {
    const uint64_t j = j0 + q;
    if (!ok && j < L && used[j]) { ok = true; v = heads[j]; }
  }
  // inclusive suffix "first valid at or after me" within the warp
  bool sok = ok;
  uint64_t sv = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const bool ok2 = __shfl_down_sync(FULL, sok, o);
    const uint64_t v2 = __shfl_down_sync(FULL, sv, o);
    if (!sok && lane + o < 32) { sok = ok2; sv = v2; }
  }
  if (lane == 0) { wv[warp] = sv; wok[warp] = sok; }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t nv = tiles[blockIdx.x].carry;
    uint32_t nok = tiles[blockIdx.x].carry_ok;
    for (int w = kFH / 32 - 1; w >= 0; w--) {
      wc[w] = nv;
      wcok[w] = nok;
      if (wok[w]) { nv = wv[w]; nok = 1; }
    }
  }
  __syncthreads();
  // exclusive: the next lane's inclusive value, else the warp's carry
  bool nok = __shfl_down_sync(FULL, sok, 1);
  uint64_t nv = __shfl_down_sync(FULL, sv, 1);
  if (lane == 31 || !nok) { nok = wcok[warp]; nv = wc[warp]; }
  if (!nok) nv = KEY_MAX;
  for (int q = kFHItems - 1; q >= 0; q--) {
    const uint64_t j = j0 + q;
    if (j >= L) continue;
    if (used[j]) nv = heads[j];
    else heads[j] = nv;
  }
}

__global__ void k_set_window(uint64_t* win_src, uint64_t* win_dst, uint64_t* leaf_off,
                             uint64_t* dst_off, uint64_t sa, uint64_t sW, uint64_t da,
                             uint64_t dW) {
  pdl_wait();
  pdl_launch();
  win_src[0] = sa; win_src[1] = sW;
  win_dst[0] = da; win_dst[1] = dW;
  leaf_off[0] = 0; leaf_off[1] = sW;
  dst_off[0] = 0; dst_off[1] = dW;
}

template <typename T>
T* P(Buf& b) { return reinterpret_cast<T*>(b.p); }

int grid_for(const cpma* h, uint64_t work, int per_block = kT) {
  uint64_t g = (work + per_block - 1) / per_block;
  g = std::max<uint64_t>(1, std::min<uint64_t>(g, (uint64_t)h->num_sms * 8));
  return (int)g;
}

Bounds bounds_of(const cpma* h) {
  Bounds B;
  B.LB = h->cfg.leaf_bytes;
  B.tau_leaf = h->cfg.tau_leaf;
  B.tau_root = h->cfg.tau_root;
  B.rho_leaf = h->cfg.rho_leaf;
  B.rho_root = h->cfg.rho_root;
  return B;
}

Levels levels_of(uint64_t L, unsigned H, uint64_t* words) {
  Levels lv;
  uint64_t off = 0;
  for (unsigned h = 0; h <= (unsigned)kMaxLevels; h++) {
    lv.off[h] = off;
    if (h <= H) {
      const uint64_t nodes = (L + (1ull << h) - 1) >> h;
      off += (nodes + 31) / 32;
    }
  }
  *words = off;
  return lv;
}

int ensure_bits(cpma* h, cudaStream_t st, Levels* lv) {
  const unsigned H = ceil_log2(h->L);
  uint64_t words = 0;
  *lv = levels_of(h->L, H, &words);
  if (words != h->bits_words) {
    CPMA_TRY(ensure(h, h->s.bits, words * 4));
    CPMA_CUDA(cudaMemsetAsync(h->s.bits.p, 0, words * 4, st));
    h->bits_words = words;
  }
  return CPMA_OK;
}

// The handle's live leaf arrays.
Arrays live_arrays(const cpma* h) {
  Arrays a;
  a.data = h->data;
  a.used = h->used;
  a.cnt = h->cnt;
  a.heads = h->heads;
  a.cap_leaves = h->cap_leaves;
  a.cap_bytes = h->cap_bytes;
  return a;
}

void set_live(cpma* h, const Arrays& a) {
  h->data = a.data;
  h->used = a.used;
  h->cnt = a.cnt;
  h->heads = a.heads;
  h->cap_leaves = a.cap_leaves;
  h->cap_bytes = a.cap_bytes;
}

// Shared tail of every redistribution: costs over E, their prefix, cut points
// and the encode into `dst`.  The window arrays and elem_off must be set;
// nelem_dev points at the element count.
int spread(cpma* h, cudaStream_t st, WinArgs w, uint64_t nelem_bound, const ull* nelem_dev,
           uint64_t ndst, Arrays dst, uint32_t LBdst) {
  CPMA_TRY(ensure(h, h->s.cost, nelem_bound + 1));
  CPMA_TRY(ensure(h, h->s.C, (nelem_bound + 2) * 8));
  CPMA_TRY(ensure(h, h->s.dstart, (ndst + 1) * 8));
  CPMA_CUDA(launch_pdl(k_costs, (unsigned)(grid_for(h, nelem_bound)), kT, 0, st, w,
                       P<uint64_t>(h->s.E), nelem_dev, P<uint8_t>(h->s.cost), (int)h->cfg.codec));
  h->launches++;
  CPMA_TRY(scan_u8_to_u64(h, P<uint8_t>(h->s.cost), P<uint64_t>(h->s.C), nelem_bound, nelem_dev,
                          st));
  CPMA_CUDA(launch_pdl(k_starts, (unsigned)(grid_for(h, ndst)), kT, 0, st, w, P<uint64_t>(h->s.C),
                       ndst, P<uint64_t>(h->s.dstart)));
  h->launches++;
  EncodeArgs ea;
  ea.w = w;
  ea.ndst = ndst;
  ea.dstart = P<uint64_t>(h->s.dstart);
  ea.E = P<uint64_t>(h->s.E);
  ea.C = P<uint64_t>(h->s.C);
  ea.data = dst.data;
  ea.used = dst.used;
  ea.cnt = dst.cnt;
  ea.heads = dst.heads;
  ea.LB = LBdst;
  ea.st = h->d_status;
  ea.raw = (int)h->cfg.codec;
  const size_t smem = (size_t)(kT / 32) * LBdst;
  CPMA_CUDA(launch_pdl(k_encode, (unsigned)(grid_for(h, ndst * 32)), kT, smem, st, ea));
  h->launches++;
  return check_cuda(cudaGetLastError());
}

WinArgs win_args(cpma* h, uint64_t nwin) {
  WinArgs w;
  w.win_src = P<uint64_t>(h->s.win_src);
  w.win_dst = P<uint64_t>(h->s.win_dst);
  w.leaf_off = P<uint64_t>(h->s.win_leaf_off);
  w.dst_off = P<uint64_t>(h->s.win_dst_off);
  w.elem_off = P<uint64_t>(h->s.win_elem_off);
  w.nwin = nwin;
  return w;
}

int ensure_win(cpma* h, uint64_t nwin) {
  CPMA_TRY(ensure(h, h->s.win_src, (nwin + 1) * 16));
  CPMA_TRY(ensure(h, h->s.win_dst, (nwin + 1) * 16));
  CPMA_TRY(ensure(h, h->s.win_leaf_off, (nwin + 2) * 8));
  CPMA_TRY(ensure(h, h->s.win_dst_off, (nwin + 2) * 8));
  CPMA_TRY(ensure(h, h->s.win_elem_off, (nwin + 2) * 8));
  return CPMA_OK;
}

// Pack the source windows into E (sources are the live arrays plus the
// pending leaves of the current batch), then spread into dst.
int pack(cpma* h, cudaStream_t st, uint64_t nwin, uint64_t nsrc, uint64_t nelem_bound,
         uint64_t nT) {
  WinArgs w = win_args(h, nwin);
  CPMA_TRY(ensure(h, h->s.srccnt, (nsrc + 1) * 4));
  CPMA_TRY(ensure(h, h->s.srcoff, (nsrc + 2) * 8));
  CPMA_TRY(ensure(h, h->s.E, (nelem_bound + 1) * 8));
  CPMA_CUDA(launch_pdl(k_src_counts, (unsigned)(grid_for(h, nsrc)), kT, 0, st, w, h->cnt, h->used,
                       nsrc, P<uint32_t>(h->s.srccnt), h->d_status));
  h->launches++;
  CPMA_TRY(scan_u32_to_u64(h, P<uint32_t>(h->s.srccnt), P<uint64_t>(h->s.srcoff), nsrc, nullptr,
                           st));
  CPMA_CUDA(launch_pdl(k_elem_offsets, (unsigned)(1), kT, 0, st, w, P<uint64_t>(h->s.srcoff),
                       h->d_status));
  h->launches++;
  UnpackArgs ua;
  ua.w = w;
  ua.nsrc = nsrc;
  ua.data = h->data;
  ua.used = h->used;
  ua.cnt = h->cnt;
  ua.LB = h->cfg.leaf_bytes;
  ua.srcoff = P<uint64_t>(h->s.srcoff);
  ua.T_leaf = P<uint32_t>(h->s.T_leaf);
  ua.T_state = P<uint32_t>(h->s.T_state);
  ua.T_first_chunk = P<uint32_t>(h->s.T_first_chunk);
  ua.chunk_off = P<uint64_t>(h->s.chunk_off);
  ua.nT = nT;
  ua.ovf = P<uint64_t>(h->s.C);  // the overflow elements (C is written only after the pack)
  ua.E = P<uint64_t>(h->s.E);
  ua.st = h->d_status;
  ua.raw = (int)h->cfg.codec;
  CPMA_CUDA(launch_pdl(k_unpack, (unsigned)(grid_for(h, nsrc * 32)), kT, 0, st, ua));
  h->launches++;
  return check_cuda(cudaGetLastError());
}

int redistribute(cpma* h, cudaStream_t st, uint64_t nwin, uint64_t nsrc, uint64_t ndst,
                 uint64_t nelem_bound, uint64_t nT, Arrays dst, uint32_t LBdst) {
  CPMA_TRY(pack(h, st, nwin, nsrc, nelem_bound, nT));
  return spread(h, st, win_args(h, nwin), nelem_bound, &h->d_status->nelem, ndst, dst, LBdst);
}

int fix_heads(cpma* h, cudaStream_t st) {
  const uint64_t nt = (h->L + kFHTile - 1) / kFHTile;
  CPMA_TRY(ensure(h, h->s.fh, nt * sizeof(FHTile)));
  FHTile* tiles = P<FHTile>(h->s.fh);
  CPMA_CUDA(launch_pdl(k_fh_tiles, (unsigned)((unsigned)nt), kFH, 0, st, h->used, h->heads, h->L,
                       tiles));
  CPMA_CUDA(launch_pdl(k_fh_carry, (unsigned)(1), kFH, 0, st, tiles, nt, h->heads, h->L,
                       h->d_status));
  CPMA_CUDA(launch_pdl(k_fh_fill, (unsigned)((unsigned)nt), kFH, 0, st, h->used, h->heads, h->L,
                       tiles));
  h->launches += 3;
  return check_cuda(cudaGetLastError());
}

// Leaf size for a structure of n keys (R13): the configured size, or with
// leaf_growth > 0 the size that grows with log n,
// min(2048, max(leaf_bytes, 16 ceil(leaf_growth bitlen(n) / 16))).
uint32_t leaf_size_for(const cpma* h, uint64_t n) {
  const uint32_t g = h->cfg.leaf_growth;
  if (!g) return h->lb_min;
  uint32_t bl = 0;
  while (bl < 64 && (n >> bl)) bl++;
  const uint64_t want = ((uint64_t)g * bl + 15) / 16 * 16;
  return (uint32_t)std::min<uint64_t>(2048, std::max<uint64_t>(h->lb_min, want));
}

// R9 of the readings: grow by grow_num/grow_den (rounded up) while the root
// upper bound fails, shrink by the inverse (rounded down) while the root
// lower bound fails and more than one leaf remains, for leaves of LB bytes.
uint64_t resize_target(const cpma_config& c, uint64_t T, uint64_t L, uint32_t LB) {
  typedef unsigned __int128 u128;
  uint64_t Lp = L;
  if ((u128)T * 1000 > (u128)c.tau_root * Lp * LB) {
    while ((u128)T * 1000 > (u128)c.tau_root * Lp * LB)
      Lp = (uint64_t)(((u128)Lp * c.grow_num + c.grow_den - 1) / c.grow_den);
  } else {
    while (Lp > 1 && (u128)T * 1000 < (u128)c.rho_root * Lp * LB) {
      uint64_t nx = (uint64_t)((u128)Lp * c.grow_den / c.grow_num);
      Lp = nx < 1 ? 1 : nx;
    }
  }
  return Lp;
}

// The leaf count and size a resize gives for T bytes and n_after keys: the
// leaf size for n_after, then R9 from the leaf count of the same capacity.
void resize_plan(const cpma* h, uint64_t T, uint64_t n_after, uint64_t* Lp, uint32_t* LBp) {
  const uint32_t LB = h->cfg.leaf_bytes, LB2 = leaf_size_for(h, n_after);
  const uint64_t L0 = LB2 == LB ? h->L : std::max<uint64_t>(1, (h->L * LB + LB2 - 1) / LB2);
  *LBp = LB2;
  *Lp = resize_target(h->cfg, T, L0, LB2);
}

// Whole-array redistribution into L' leaves of LB' bytes (R9, R13).  The
// destination is the live arrays when they have the capacity (the pack reads
// every element before the encode writes), else the spare arrays reserved
// before the update; nothing is allocated here.
int do_resize(cpma* h, cudaStream_t st, uint64_t T, uint64_t n_after, uint64_t nT) {
  uint64_t Lp = 0;
  uint32_t LBp = 0;
  resize_plan(h, T, n_after, &Lp, &LBp);
  const bool in_place = Lp <= h->cap_leaves && Lp * LBp <= h->cap_bytes;
  if (!in_place && (Lp > h->spare.cap_leaves || Lp * LBp > h->spare.cap_bytes))
    return CPMA_EINTERNAL;  // the reservation missed this case
  Arrays dst = in_place ? live_arrays(h) : h->spare;
  CPMA_CUDA(launch_pdl(k_set_window, (unsigned)(1), 1, 0, st, P<uint64_t>(h->s.win_src),
                       P<uint64_t>(h->s.win_dst), P<uint64_t>(h->s.win_leaf_off),
                       P<uint64_t>(h->s.win_dst_off), 0, h->L, 0, Lp));
  h->launches++;
  CPMA_TRY(redistribute(h, st, 1, h->L, Lp, n_after, nT, dst, LBp));
  CPMA_CUDA(cudaStreamSynchronize(st));
  if (!in_place) {
    Arrays old = live_arrays(h);
    free_arrays(h, &old);
    set_live(h, dst);
    h->spare = Arrays{};
  }
  h->cfg.leaf_bytes = LBp;
  h->L = Lp;
  return CPMA_OK;
}

// ---- rebuild of the whole set for a large batch (reading R14) ----
//
// All n elements are packed into E, merged with the sorted batch u into M
// (stable: an element of E precedes equal batch keys), compacted to the
// union or the difference, and built like the constructor.

__global__ void __launch_bounds__(kT) k_check_sorted(const uint64_t* __restrict__ u, uint64_t k,
                                                     Status* st) {
  bool bad = false;
  for (uint64_t i = gtid() + 1; i < k; i += gstride()) bad |= u[i - 1] > u[i];
  if (__any_sync(FULL, bad) && lane_id() == 0) atomicOr(&st->err, kErrUnsorted);
}

// Number of E elements among the first d outputs of the stable merge of
// A[0..na) and B[0..nb) (merge path: ties take A first).
template <typename PA, typename PB>
__device__ __forceinline__ uint64_t merge_split(PA A, uint64_t na, PB B, uint64_t nb, uint64_t d) {
  uint64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (A[mid] <= B[d - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

constexpr int kMergeItems = 8;
constexpr int kMergeTile = kT * kMergeItems;  // outputs per block step

// Stable merge of A (n) and B (k) into M with fromB[i] = 1 for batch keys.
// Each tile of kMergeTile outputs stages its A and B ranges in shared memory
// (found by two merge-path searches), every thread merges kMergeItems
// outputs from its own split, and the tile is written back coalesced.
__global__ void __launch_bounds__(kT) k_merge_path(const uint64_t* __restrict__ A, uint64_t n,
                                                   const uint64_t* __restrict__ B, uint64_t k,
                                                   uint64_t* __restrict__ M,
                                                   uint8_t* __restrict__ fromB) {
  pdl_wait();
  pdl_launch();
  __shared__ uint64_t sA[kMergeTile + 1], sB[kMergeTile + 1];
  __shared__ uint64_t split[2];
  const uint64_t N = n + k;
  for (uint64_t d0 = (uint64_t)blockIdx.x * kMergeTile; d0 < N;
       d0 += (uint64_t)gridDim.x * kMergeTile) {
    const uint64_t d1 = min(N, d0 + kMergeTile);
    if (threadIdx.x < 2) split[threadIdx.x] = merge_split(A, n, B, k, threadIdx.x ? d1 : d0);
    __syncthreads();
    const uint64_t a0 = split[0], a1 = split[1];
    const uint64_t b0 = d0 - a0, b1 = d1 - a1;
    const uint32_t na = (uint32_t)(a1 - a0), nb = (uint32_t)(b1 - b0);
    for (uint32_t i = threadIdx.x; i < na; i += kT) sA[i] = A[a0 + i];
    for (uint32_t i = threadIdx.x; i < nb; i += kT) sB[i] = B[b0 + i];
    __syncthreads();
    const uint32_t dd = threadIdx.x * kMergeItems, tot = na + nb;
    // outputs dd .. dd+cnt-1 of the tile (ia + ib = dd + q < tot keeps every
    // read below na or nb)
    const uint32_t cnt = dd < tot ? min((uint32_t)kMergeItems, tot - dd) : 0u;
    uint64_t v[kMergeItems];
    uint32_t fb = 0;
    if (cnt) {
      uint32_t ia = (uint32_t)merge_split(sA, na, sB, nb, dd), ib = dd - ia;
#pragma unroll
      for (int q = 0; q < kMergeItems; q++) {
        if ((uint32_t)q < cnt) {
          const bool takeA = ib >= nb || (ia < na && sA[ia] <= sB[ib]);
          v[q] = takeA ? sA[ia] : sB[ib];
          if (takeA) ia++; else { ib++; fb |= 1u << q; }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMergeItems; q++) {
      if ((uint32_t)q < cnt) {
        sA[dd + q] = v[q];
        reinterpret_cast<uint8_t*>(sB)[dd + q] = (uint8_t)((fb >> q) & 1u);
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tot; i += kT) {
      M[d0 + i] = sA[i];
      fromB[d0 + i] = reinterpret_cast<const uint8_t*>(sB)[i];
    }
    __syncthreads();
  }
}

// keep[i]: union keeps the first of every run of equal keys; difference keeps
// an element of E that no batch key equals (equal batch keys follow it).
__global__ void __launch_bounds__(kT) k_rebuild_flags(const uint64_t* __restrict__ M,
                                                      const uint8_t* __restrict__ fromB,
                                                      uint64_t N, int is_delete,
                                                      uint8_t* __restrict__ keep) {
  pdl_wait();
  pdl_launch();
  for (uint64_t i = gtid(); i < N; i += gstride()) {
    const uint64_t x = M[i];
    bool kp;
    if (is_delete) kp = !fromB[i] && (i + 1 == N || M[i + 1] != x);
    else kp = i == 0 || M[i - 1] != x;
    keep[i] = kp ? 1 : 0;
  }
}

__global__ void __launch_bounds__(kT) k_rebuild_scatter(const uint64_t* __restrict__ M,
                                                        const uint8_t* __restrict__ keep,
                                                        const uint64_t* __restrict__ pos,
                                                        uint64_t N, uint64_t n_old,
                                                        int is_delete,
                                                        uint64_t* __restrict__ E, Status* st) {
  pdl_wait();
  pdl_launch();
  for (uint64_t i = gtid(); i < N; i += gstride())
    if (keep[i]) E[pos[i]] = M[i];
  if (gtid() == 0) {
    const uint64_t m = pos[N];
    st->nelem = m;
    st->delta = is_delete ? n_old - m : m - n_old;
  }
}

// Host-side values the front segment of an update leaves for the rest of it.
struct Front {
  MergeArgs ma;
  FinArgs fa;
  Levels lv;
  unsigned H = 0;
  int mgrid = 0, mwarps = 0;
  size_t msmem = 0;
  uint64_t k = 0;  // keys the front segment ran over (the work items are fewer)
};

void merge_attrs() {
  static bool done = false;  // one process, one device
  if (done) return;
  cudaFuncSetAttribute(k_merge<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_merge<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_merge_small, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaGetLastError();
  done = true;
}

// The thread-granular insert (or delete) over the touched leaves of a batch
// of k keys (at most k of them).
template <bool DEL>
void launch_insert_thread(cpma* h, const MergeArgs& ma, uint64_t k, cudaStream_t st) {
  const int g = (int)std::max<uint64_t>(
      1, std::min<uint64_t>((k + kThrT - 1) / kThrT, (uint64_t)h->num_sms * 16));
  k_insert_thread<DEL><<<g, kThrT, 0, st>>>(ma);
  h->launches++;
}

// Every buffer the front segment of a batch of k keys touches, sized before
// it runs (a graph capture must not allocate), plus the window bitsets of the
// current tree.
int front_scratch(cpma* h, uint64_t k, bool tagged, cudaStream_t st) {
  Scratch& s = h->s;
  merge_attrs();
  if (!h->side) {
    // highest priority: the side kernels' few blocks go ahead of the thread
    // kernel's many
    int least = 0, greatest = 0;
    CPMA_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CPMA_CUDA(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, greatest));
  }
  if (!h->ev_fork) CPMA_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  if (!h->ev_join) CPMA_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  CPMA_TRY(sort_scratch(h, k, tagged));
  CPMA_TRY(ensure(h, s.partials, (size_t)(2 * h->num_sms + 2) * 8));
  // the routing's tile counter and look-back words (tiles of >= 256 keys)
  CPMA_TRY(ensure(h, s.flags, (k / 256 + 3) * 8));
  for (Buf* b : {&s.chunk_begin, &s.chunk_leaf, &s.chunk_tid, &s.chunk_cnt, &s.T_leaf, &s.T_begin,
                 &s.T_first_chunk, &s.T_oldcnt, &s.T_oldused, &s.T_newcnt, &s.T_state, &s.viol})
    CPMA_TRY(ensure(h, *b, (k + 2) * 4));
  CPMA_TRY(ensure(h, s.chunk_off, (k + 2) * 8));
  CPMA_TRY(ensure(h, s.T_newbytes, (k + 2) * 8));
  CPMA_TRY(ensure(h, s.list_lane, (k + 2) * 4));
  CPMA_TRY(ensure(h, s.list_v1, (k + 2) * 4));
  CPMA_TRY(ensure(h, s.list_gen, (k + 2) * 4));
  CPMA_TRY(ensure(h, s.list_pend, (k + 2) * 4));
  CPMA_TRY(ensure(h, s.cand, (2 * k + 2) * 8));
  CPMA_TRY(ensure(h, s.wins, (2 * k + 2) * 16));
  CPMA_TRY(ensure(h, s.prefix, (h->L + 2) * 8));
  Levels lv;
  return ensure_bits(h, st, &lv);
}

// The front segment of an update: status reset, tag check, sort, route,
// work lists, the in-place merges, finalize and the overflow-offset scan --
// everything before the first host read of the status block.  It reads the
// host state only through h's fields and its arguments, never allocates
// (front_scratch sized everything) and never waits, so it can be captured
// into a CUDA graph.  f receives the host-side values the rest of the update
// needs.
int run_front(cpma* h, const uint64_t* d_keys, uint64_t k, int sorted, int is_delete,
              cudaStream_t st, const uint32_t* tags, uint64_t* tag_counts, uint64_t ntags,
              Front* f) {
  Status* ds = h->d_status;
  CPMA_CUDA(cudaMemsetAsync(ds, 0, offsetof(Status, empties), st));
  // routing tiles: keys per thread, the most (8, 4, 2) that still gives two
  // tiles per SM when the batch is dense against the leaves (a tile then
  // reaches about as many heads as it has keys), one otherwise.  The tile
  // counter and look-back words are cleared now, so that the routing kernel
  // directly follows the sort's last kernel.
  int kpt = 1;
  if (2 * k >= h->L)
    for (int c = 8; c > 1 && kpt == 1; c >>= 1)
      if (k >= (uint64_t)h->num_sms * 2 * kRT * c) kpt = c;
  const uint64_t tile_keys = (uint64_t)kRT * kpt;
  const uint64_t ntiles = (k + tile_keys - 1) / tile_keys;
  uint64_t* look = P<uint64_t>(h->s.flags);
  CPMA_CUDA(cudaMemsetAsync(look, 0, (ntiles + 1) * 8, st));
  const uint64_t* u = d_keys;
  const uint32_t* ut = tags;
  if (tags) {
    k_check_tags<<<grid_for(h, k), kT, 0, st>>>(tags, k, ntags, ds);
    h->launches++;
  }
  if (!sorted) {
    prof_begin(h, PH_SORT, st);
    if (tags) CPMA_TRY(sort_pairs(h, d_keys, tags, k, &u, &ut, st));
    else CPMA_TRY(sort_keys(h, d_keys, k, &u, st));
    prof_end(h, st);
  }
  Scratch& s = h->s;
  Levels lv;
  CPMA_TRY(ensure_bits(h, st, &lv));  // sized by front_scratch: no memset here
  const unsigned H = ceil_log2(h->L);
  const Bounds B = bounds_of(h);
  const uint32_t LB = h->cfg.leaf_bytes;

  // ---- route ----
  prof_begin(h, PH_ROUTE, st);
  RouteOut ro;
  ro.chunk_begin = P<uint32_t>(s.chunk_begin);
  ro.chunk_leaf = P<uint32_t>(s.chunk_leaf);
  ro.chunk_tid = P<uint32_t>(s.chunk_tid);
  ro.T_leaf = P<uint32_t>(s.T_leaf);
  ro.T_begin = P<uint32_t>(s.T_begin);
  ro.T_first_chunk = P<uint32_t>(s.T_first_chunk);
  ro.T_oldcnt = P<uint32_t>(s.T_oldcnt);
  ro.T_oldused = P<uint32_t>(s.T_oldused);
  ro.T_newcnt = P<uint32_t>(s.T_newcnt);
  ro.T_state = P<uint32_t>(s.T_state);
  ro.T_newbytes = P<ull>(s.T_newbytes);
  {
    const unsigned grid = (unsigned)std::min<uint64_t>(ntiles, (uint64_t)h->num_sms * 4);
    const uint32_t spin = h->sort_poll_limit ? h->sort_poll_limit : (1u << 22);
    const uint32_t silent = h->sort_silent_tile >= 0 && h->sort_silent_tile < (int64_t)ntiles
                                ? (uint32_t)h->sort_silent_tile : 0xFFFFFFFFu;
    // keys, the heads searched, and per touched leaf its entries (36 bytes),
    // old counts (8) and work item (12)
    prof_add_bytes(h, PH_ROUTE, 8ull * k + 64ull * std::min<uint64_t>(k, h->L));
    const uint64_t* H = h->heads;
    // scheduled while the sort's last kernel finishes (it waits for it first)
    const uint64_t L = h->L;
    switch (kpt) {
      case 8:
        CPMA_CUDA(launch_pdl(k_route<8>, grid, kRT, 0, st, u, k, H, L, h->cnt, h->used, ro, look,
                             ds, spin, silent));
        break;
      case 4:
        CPMA_CUDA(launch_pdl(k_route<4>, grid, kRT, 0, st, u, k, H, L, h->cnt, h->used, ro, look,
                             ds, spin, silent));
        break;
      case 2:
        CPMA_CUDA(launch_pdl(k_route<2>, grid, kRT, 0, st, u, k, H, L, h->cnt, h->used, ro, look,
                             ds, spin, silent));
        break;
      default:
        CPMA_CUDA(launch_pdl(k_route<1>, grid, kRT, 0, st, u, k, H, L, h->cnt, h->used, ro, look,
                             ds, spin, silent));
    }
    h->launches++;
    CPMA_CUDA(cudaGetLastError());
  }

  // ---- merge (count; in-place rewrites) ----
  MergeArgs ma;
  ma.u = u;
  ma.data = h->data;
  ma.used = h->used;
  ma.cnt = h->cnt;
  ma.heads = h->heads;
  ma.LB = LB;
  ma.chunk_begin = ro.chunk_begin;
  ma.chunk_leaf = ro.chunk_leaf;
  ma.chunk_tid = ro.chunk_tid;
  ma.chunk_cnt = P<uint32_t>(s.chunk_cnt);
  ma.chunk_off = P<uint64_t>(s.chunk_off);
  ma.T_begin = ro.T_begin;
  ma.T_oldcnt = ro.T_oldcnt;
  ma.T_oldused = ro.T_oldused;
  ma.T_leaf = ro.T_leaf;
  ma.T_first_chunk = ro.T_first_chunk;
  ma.T_newcnt = ro.T_newcnt;
  ma.T_state = ro.T_state;
  ma.T_newbytes = ro.T_newbytes;
  ma.ovf = nullptr;
  ma.is_delete = is_delete;
  ma.st = ds;
  ma.prof = nullptr;
  ma.tags = ut;
  ma.tag_counts = tags ? reinterpret_cast<ull*>(tag_counts) : nullptr;
  ma.list_lane = P<uint32_t>(s.list_lane);
  ma.list_v1 = P<uint32_t>(s.list_v1);
  ma.list_gen = P<uint32_t>(s.list_gen);
  ma.list_pend = P<uint32_t>(s.list_pend);
  ma.raw = (int)h->cfg.codec;
  ma.small = k <= kSmallBatch ? 1 : 0;
  ma.B = B;
  ma.H = H;
  ma.viol = P<uint32_t>(s.viol);
  const size_t per = merge_warp_bytes(LB);
  const int mwarps = (int)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / per));
  const size_t msmem = per * mwarps;
  const int mgrid = (int)std::max<uint64_t>(
      1, std::min<uint64_t>((k + kChunk + mwarps - 1) / mwarps, (uint64_t)h->num_sms * 4));
  // inserts: k_classify runs on the side stream, ahead of the lane kernel
  // and beside the thread kernel (which walks the touched leaves itself)
  if (is_delete) {
    k_classify<<<grid_for(h, k), kT, 0, st>>>(ma);
    h->launches++;
  }
  prof_end(h, st);
  prof_begin(h, PH_MERGE, st);
  {
    const size_t sper = small_warp_bytes(LB);
    const int swarps = (int)std::max<size_t>(1, std::min<size_t>(8, (216 * 1024) / (4 * sper)));
    const int sgrid = (int)std::max<uint64_t>(
        1, std::min<uint64_t>((k + swarps - 1) / swarps, (uint64_t)h->num_sms * 8));
    if (!is_delete) {
      // the thread-granular insert on st and the work lists plus the
      // lane-granular insert on the side stream at the same time: disjoint
      // leaves and outputs (shared counters by atomics); the lane kernel's
      // few leaves are latency-bound
      CPMA_CUDA(cudaEventRecord(h->ev_fork, st));
      CPMA_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
      prof_begin_side(h, PH_MERGE_LANE, h->side);
      MergeArgs ml = ma;
      ml.prof = prof_bytes(h, PH_MERGE_LANE);
      k_classify<<<grid_for(h, k), kT, 0, h->side>>>(ma);
      k_insert_lane<kLaneSeg><<<sgrid, 256, lane_warp_bytes(kLaneSeg) * 8, h->side>>>(ml);
      h->launches += 2;
      prof_end_side(h, h->side);
      CPMA_CUDA(cudaEventRecord(h->ev_join, h->side));
      ma.prof = prof_bytes(h, PH_MERGE);
      if (!ma.raw && !ma.small) {
        launch_insert_thread<false>(h, ma, k, st);
      }
      ma.prof = nullptr;
      CPMA_CUDA(cudaStreamWaitEvent(st, h->ev_join, 0));
    }
    if (is_delete && !ma.raw && !ma.small) {
      ma.prof = prof_bytes(h, PH_MERGE);
      launch_insert_thread<true>(h, ma, k, st);
      ma.prof = nullptr;
    }
    prof_end(h, st);
    prof_begin(h, PH_MERGE2, st);
    ma.prof = prof_bytes(h, PH_MERGE2);
    k_merge_small<<<sgrid, swarps * 32, sper * swarps, st>>>(ma);
    h->launches++;
    ma.prof = nullptr;
  }
  CPMA_CUDA(launch_pdl(k_merge<false>, (unsigned)mgrid, (unsigned)(mwarps * 32), msmem, st, ma));
  h->launches++;
  CPMA_CUDA(cudaGetLastError());
  prof_end(h, st);
  prof_begin(h, PH_COUNT, st);

  FinArgs fa;
  fa.used = h->used;
  fa.cnt = h->cnt;
  fa.T_leaf = ro.T_leaf;
  fa.T_first_chunk = ro.T_first_chunk;
  fa.T_oldcnt = ro.T_oldcnt;
  fa.T_newcnt = ro.T_newcnt;
  fa.T_begin = ro.T_begin;
  fa.T_oldused = ro.T_oldused;
  fa.merge_bytes = prof_bytes(h, PH_MERGE2);
  fa.T_state = ro.T_state;
  fa.T_newbytes = ro.T_newbytes;
  fa.chunk_cnt = ma.chunk_cnt;
  fa.chunk_tid = ma.chunk_tid;
  fa.list_v1 = ma.list_v1;
  fa.list_gen = ma.list_gen;
  fa.list_pend = ma.list_pend;
  fa.viol = P<uint32_t>(s.viol);
  fa.cand = P<uint64_t>(s.cand);
  fa.bits = P<uint32_t>(s.bits);
  fa.lv = lv;
  fa.B = B;
  fa.H = H;
  fa.is_delete = is_delete;
  fa.st = ds;
  CPMA_CUDA(launch_pdl(k_finalize, (unsigned)grid_for(h, k), kT, 0, st, fa));
  h->launches++;
  CPMA_CUDA(cudaGetLastError());
  prof_end(h, st);
  f->ma = ma;
  f->fa = fa;
  f->lv = lv;
  f->H = H;
  f->mgrid = mgrid;
  f->mwarps = mwarps;
  f->msmem = msmem;
  f->k = k;
  return CPMA_OK;
}


// ---- CUDA graphs for the front segment ----
//
// A batch of k keys is staged into a library buffer of K = graph_bucket(k)
// keys (k rounded up to 5 significant bits: K <= 17k/16), staged[j] =
// batch[floor(j k / K)]: every key appears once or twice, in the batch's own
// order (a sorted batch stays sorted), so the repeats are spread evenly over
// the touched leaves instead of piling into one.  Repeats are dropped by the
// merge (first occurrence wins), so the padded batch changes the set exactly
// as the original does, and one graph serves every k of its bucket.  A graph
// bakes in the addresses of the structure's arrays, of the scratch buffers
// the segment touches and the leaf count, so it is keyed by (K, sorted,
// insert/delete, those addresses and L) and captured again when any of them
// changed (a resize, a scratch buffer that had to grow).

constexpr int kGraphSlots = 8;

constexpr int kSigPtrs = 34;

struct FrontSig {
  const void* p[kSigPtrs];
  uint64_t L, LB;
  uint32_t poll;    // sort look-back poll limit and silent tile (tests)
  int64_t silent;
  bool operator==(const FrontSig& o) const {
    if (L != o.L || LB != o.LB || poll != o.poll || silent != o.silent) return false;
    for (int i = 0; i < kSigPtrs; i++)
      if (p[i] != o.p[i]) return false;
    return true;
  }
};

FrontSig front_sig(const cpma* h) {
  const Scratch& s = h->s;
  return FrontSig{{s.stage.p,     s.keysA.p,      s.keysB.p,         s.hist.p,      s.partials.p,
                   s.leaf_of.p,   s.flags.p,      s.flags_scan.p,    s.chunk_begin.p,
                   s.chunk_leaf.p, s.chunk_tid.p, s.chunk_cnt.p,     s.chunk_off.p, s.T_leaf.p,
                   s.T_begin.p,   s.T_first_chunk.p, s.T_oldcnt.p,   s.T_oldused.p, s.T_newcnt.p,
                   s.T_newbytes.p, s.T_state.p,   s.viol.p,          s.list_lane.p, s.list_v1.p,
                   s.list_gen.p,  s.list_pend.p,  s.cand.p,          s.wins.p,      s.bits.p,  h->data,
                   h->used,       h->cnt,         h->heads,          h->d_status},
                  h->L, h->cfg.leaf_bytes, h->sort_poll_limit, h->sort_silent_tile};
}

struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  uint64_t K = 0, last_use = 0, launches = 0;
  int sorted = 0, is_delete = 0;
  bool prof = false;  // captured with per-phase profiling (event record nodes)
  uint32_t prof_mask = 0;  // the phases that got event nodes
  FrontSig sig{};
  Front f;
  std::vector<Prof::Rec> recs;        // the graph's event pairs
  unsigned long long host_bytes[PH_N] = {0};
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    for (Prof::Rec& r : recs) {
      if (r.a) cudaEventDestroy(r.a);
      if (r.b) cudaEventDestroy(r.b);
    }
    recs.clear();
  }
};

struct GraphCache {
  GraphSlot slot[kGraphSlots];
  uint64_t clock = 0;
};

// k rounded up to 4 significant bits (at most 1/8 extra keys), at least 16
uint64_t graph_bucket(uint64_t k) {  // k rounded up to 5 significant bits
  if (k <= 16) return 16;
  const unsigned e = 63u - (unsigned)__builtin_clzll(k);
  const uint64_t step = 1ull << (e - 4);
  return (k + step - 1) / step * step;
}

// staged[j] = batch[floor(j k / K)] with r = floor(2^32 k / K): (j r) >> 32 is
// floor(j k / K) or one less (j < 2^31, so the error j (2^32 k / K - r) is
// below 2^32), fixed by one comparison; no division on the device
__global__ void __launch_bounds__(kT) k_stage(const uint64_t* __restrict__ in, uint64_t k,
                                              uint64_t* __restrict__ out, uint64_t K, uint64_t r) {
  for (uint64_t j = gtid(); j < K; j += gstride()) {
    uint64_t i = (j * r) >> 32;
    if ((i + 1) * K <= j * k) i++;
    out[j] = in[i];
  }
}


int run_front_graph(cpma* h, const uint64_t* d_keys, uint64_t k, int sorted, int is_delete,
                    cudaStream_t st, Front* f) {
  const uint64_t K = graph_bucket(k);
  CPMA_TRY(ensure(h, h->s.stage, K * 8));
  CPMA_TRY(front_scratch(h, K, false, st));
  uint64_t* stage = P<uint64_t>(h->s.stage);
  const uint64_t r = (uint64_t)(((unsigned __int128)k << 32) / K);  // 2^32 when K == k
  k_stage<<<grid_for(h, K), kT, 0, st>>>(d_keys, k, stage, K, r);
  h->launches++;
  CPMA_CUDA(cudaGetLastError());
  if (!h->graphs) h->graphs = new GraphCache();
  GraphCache& c = *static_cast<GraphCache*>(h->graphs);
  const FrontSig sig = front_sig(h);
  GraphSlot* slot = nullptr;
  const bool prof = h->prof.on;
  for (GraphSlot& g : c.slot)
    if (g.exec && g.K == K && g.sorted == sorted && g.is_delete == is_delete && g.sig == sig &&
        g.prof == prof && (!prof || g.prof_mask == h->prof.mask))
      slot = &g;
  if (!slot) {
    slot = &c.slot[0];
    for (GraphSlot& g : c.slot)
      if (!g.exec || g.last_use < slot->last_use) slot = &g;
    if (slot->exec) {
      // the previous update on this handle has been waited for, so no
      // launch of this graph is still in flight; its event pairs were
      // resolved at that wait
      slot->release();
    }
    if (!h->cap_stream)
      CPMA_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const uint64_t l0 = h->launches;
    Prof& pr = h->prof;
    if (prof) {
      pr.capturing = true;
      pr.ncap = 0;
      for (int i = 0; i < PH_N; i++) pr.cap_host_bytes[i] = 0;
    }
    CPMA_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    int rc = run_front(h, stage, K, sorted, is_delete, h->cap_stream, nullptr, nullptr, 0,
                       &slot->f);
    set_capturing(false);
    if (prof) {
      pr.capturing = false;
      slot->recs.assign(pr.cap_recs, pr.cap_recs + pr.ncap);
      for (int i = 0; i < PH_N; i++) slot->host_bytes[i] = pr.cap_host_bytes[i];
      pr.ncap = 0;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc == CPMA_OK) rc = check_cuda(e);
    cudaGraphExec_t ex = nullptr;
    if (rc == CPMA_OK) rc = check_cuda(cudaGraphInstantiate(&ex, g, 0));
    if (g) cudaGraphDestroy(g);
    slot->launches = h->launches - l0;
    h->launches = l0;
    if (rc != CPMA_OK) {
      cudaGetLastError();
      slot->release();  // events created during the failed capture
      return rc;
    }
    slot->exec = ex;
    slot->prof = prof;
    slot->prof_mask = h->prof.mask;
    slot->K = K;
    slot->sorted = sorted;
    slot->is_delete = is_delete;
    slot->sig = sig;
    h->graph_captures++;
  }
  slot->last_use = ++c.clock;
  CPMA_CUDA(cudaGraphLaunch(slot->exec, st));
  if (slot->prof) prof_push(h, slot->recs.data(), (int)slot->recs.size(), slot->host_bytes);
  h->launches += slot->launches;
  h->graph_launches++;
  *f = slot->f;
  return CPMA_OK;
}

// May an update take the point path?  Untagged updates of 1 .. point_max
// keys on a non-empty set of byte-code leaves of at most 512 bytes (the
// lane-granular insert's buffer, the staging slot), unless a test of the
// bounded waits is set up (those waits are in the batch algorithm's sort and
// routing).
bool point_ok(const cpma* h, uint64_t k, int is_delete, const uint32_t* tags) {
  return !tags && k >= 1 &&
         k <= std::min<uint64_t>(h->point_max, is_delete ? kPointDelMax : kPointMax) &&
         h->cfg.codec == 0 && h->cfg.leaf_bytes <= 512 && h->n > 0 && h->L > 0 &&
         h->sort_poll_limit == 0 && h->sort_silent_tile < 0;
}

// Scratch of the point path for batches of up to k keys: the sort buffer,
// one leaf word, one 512-byte staging slot and one staged record per key.
int point_scratch(cpma* h, uint64_t k, cudaStream_t st) {
  k = std::min<uint64_t>(std::max<uint64_t>(k, 2), kPointMax);
  if (k > kPointRankMax) CPMA_TRY(sort_scratch(h, k, false));
  CPMA_TRY(ensure(h, h->s.keysA, k * 8, st));
  CPMA_TRY(ensure(h, h->s.T_leaf, (k + 2) * 4, st));
  CPMA_TRY(ensure(h, h->s.point_stage, k * 512, st));
  return ensure(h, h->s.point_rec, k * sizeof(PointRec), st);
}

// The point path: sort and route, stage a warp per touched leaf, commit when
// no leaf needs the batch algorithm (in the staging kernel's last block for
// up to kPointFew keys, else in a commit kernel), then read the status.  On
// return *fb tells whether some leaf needs the batch algorithm (nothing has
// been written then).  point_scratch sized the buffers it uses.
constexpr uint64_t kPointFew = 32;
int run_point(cpma* h, const uint64_t* d_keys, uint64_t k, int sorted, int is_delete,
              uint64_t* d_delta, cudaStream_t st, bool* fb) {
  Status* ds = h->d_status;
  Scratch& s = h->s;
  uint64_t* u = P<uint64_t>(s.keysA);
  uint32_t* leaf_of = P<uint32_t>(s.T_leaf);
  if (!sorted && k > kPointRankMax) {
    // the batch sort (into one of its scratch buffers); the routing kernel
    // then copies the keys to u (a no-op when they are already there)
    prof_begin(h, PH_SORT, st);
    const uint64_t* srt = nullptr;
    CPMA_TRY(sort_keys(h, d_keys, k, &srt, st));
    prof_end(h, st);
    d_keys = srt;
    sorted = 1;
  }
  const unsigned grid = (unsigned)((k + kPRT / 32 - 1) / (kPRT / 32));  // a warp per key
  prof_begin(h, PH_ROUTE, st);
  prof_add_bytes(h, PH_ROUTE, 20ull * k);
  k_point_sort_route<<<grid, kPRT, sorted ? 0 : k * 8, st>>>(d_keys, (uint32_t)k, sorted, u,
                                                             leaf_of, h->heads, h->L, ds);
  prof_end(h, st);
  MergeArgs ma;
  memset(&ma, 0, sizeof(ma));
  ma.u = u;
  ma.data = h->data;
  ma.used = h->used;
  ma.cnt = h->cnt;
  ma.heads = h->heads;
  ma.LB = h->cfg.leaf_bytes;
  ma.st = ds;
  ma.small = 1;
  ma.B = bounds_of(h);
  ma.H = ceil_log2(h->L);
  ma.pstage = P<uint8_t>(s.point_stage);
  ma.prec = P<PointRec>(s.point_rec);
  const size_t smem = lane_warp_bytes(kLaneSeg) * (kT / 32);
  prof_begin(h, PH_MERGE_LANE, st);
  const uint32_t k32 = (uint32_t)k;
  uint64_t* none = nullptr;
  if (k <= kPointFew) {
    CPMA_CUDA(is_delete ? launch_pdl(k_point_plan<true, true>, grid, kT, smem, st, ma, leaf_of,
                                     k32, d_delta)
                        : launch_pdl(k_point_plan<true, false>, grid, kT, smem, st, ma, leaf_of,
                                     k32, d_delta));
    h->launches += 2;
  } else {
    CPMA_CUDA(is_delete ? launch_pdl(k_point_plan<false, true>, grid, kT, smem, st, ma, leaf_of,
                                     k32, none)
                        : launch_pdl(k_point_plan<false, false>, grid, kT, smem, st, ma, leaf_of,
                                     k32, none));
    CPMA_CUDA(launch_pdl(k_point_commit, grid, kT, 0, st, ma, leaf_of, k32, d_delta));
    h->launches += 3;
  }
  prof_end(h, st);
  CPMA_CUDA(cudaGetLastError());
  CPMA_TRY(sync_status(h, st));
  const Status& hs = *h->h_status;
  if (hs.err & kErrUnsorted) return CPMA_EINVAL;
  if (hs.err) return CPMA_EINTERNAL;
  *fb = hs.point_fb != 0;
  if (!*fb) {
    h->n = is_delete ? h->n - hs.delta : h->n + hs.delta;
    h->t_known = hs.bytes_total;
  }
  return CPMA_OK;
}

}  // namespace

void graph_cache_free(cpma* h) {
  if (h->graphs) {
    GraphCache* c = static_cast<GraphCache*>(h->graphs);
    for (GraphSlot& g : c->slot) g.release();
    delete c;
    h->graphs = nullptr;
  }
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  h->cap_stream = nullptr;
  if (h->side) cudaStreamDestroy(h->side);
  h->side = nullptr;
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  h->ev_fork = h->ev_join = nullptr;
}

// R14: apply the batch by merging it with every element and building the
// result like the constructor.  Nothing is replaced before the new arrays
// are complete, so a rejected batch leaves the set unchanged.
int run_rebuild(cpma* h, const uint64_t* d_keys, uint64_t k, int sorted, int is_delete,
                uint64_t* d_delta, cudaStream_t st) {
  Status* ds = h->d_status;
  Scratch& s = h->s;
  const uint64_t n = h->n, N = n + k;
  CPMA_CUDA(cudaMemsetAsync(ds, 0, offsetof(Status, empties), st));
  const uint64_t* u = d_keys;
  prof_begin(h, PH_SORT, st);
  if (!sorted) {
    CPMA_TRY(sort_keys(h, d_keys, k, &u, st));
  } else {
    k_check_sorted<<<grid_for(h, k), kT, 0, st>>>(u, k, ds);
    h->launches++;
  }
  prof_end(h, st);
  prof_begin(h, PH_REDIST, st);
  // every element, in order, into E (one window over all leaves); E later
  // takes the merged set, up to n + k keys
  CPMA_TRY(ensure(h, s.E, (N + 1) * 8));
  CPMA_TRY(ensure_win(h, 1));
  k_set_window<<<1, 1, 0, st>>>(P<uint64_t>(s.win_src), P<uint64_t>(s.win_dst),
                                P<uint64_t>(s.win_leaf_off), P<uint64_t>(s.win_dst_off), 0, h->L,
                                0, h->L);
  h->launches++;
  CPMA_TRY(pack(h, st, 1, h->L, n, 0));
  CPMA_TRY(ensure(h, s.C, (N + 2) * 8));
  CPMA_TRY(ensure(h, s.cost, N + 1));
  CPMA_TRY(ensure(h, s.flags_scan, (N + 2) * 8));
  CPMA_TRY(ensure(h, s.srccnt, N + 1));
  uint64_t* M = P<uint64_t>(s.C);  // dead once the result is in E
  uint8_t* fromB = P<uint8_t>(s.srccnt);
  uint8_t* keep = P<uint8_t>(s.cost);
  uint64_t* pos = P<uint64_t>(s.flags_scan);
  // one block per tile of outputs: the scheduler overlaps the tiles' load,
  // merge and store phases across blocks
  const uint64_t mg = std::max<uint64_t>(1, (N + kMergeTile - 1) / kMergeTile);
  if (mg >= (1ull << 31)) return CPMA_EINVAL;
  CPMA_CUDA(launch_pdl(k_merge_path, (unsigned)((unsigned)mg), kT, 0, st, P<uint64_t>(s.E), n, u, k,
                       M, fromB));
  CPMA_CUDA(launch_pdl(k_rebuild_flags, (unsigned)(grid_for(h, N)), kT, 0, st, M, fromB, N,
                       is_delete, keep));
  h->launches += 2;
  CPMA_TRY(scan_u8_to_u64(h, keep, pos, N, nullptr, st));
  CPMA_CUDA(launch_pdl(k_rebuild_scatter, (unsigned)(grid_for(h, N)), kT, 0, st, M, keep, pos, N, n,
                       is_delete, P<uint64_t>(s.E), ds));
  h->launches++;
  CPMA_CUDA(cudaGetLastError());
  CPMA_TRY(sync_status(h, st));
  Status hs = *h->h_status;
  if (hs.err & (kErrSort | kErrRoute)) return CPMA_ETIMEOUT;
  if (hs.err & kErrUnsorted) return CPMA_EINVAL;
  if (hs.err) return CPMA_EINTERNAL;
  CPMA_TRY(build_from_sorted_unique(h, P<uint64_t>(s.E), hs.nelem, st));
  prof_end(h, st);
  if (d_delta) {
    // build_from_sorted_unique reset the status block; the count is on the host
    const uint64_t delta = is_delete ? n - hs.nelem : hs.nelem - n;
    k_put_u64<<<1, 1, 0, st>>>(d_delta, delta);
    h->launches++;
  }
  return check_cuda(cudaGetLastError());
}

int reserve_update(cpma* h, uint64_t k, int is_delete, cudaStream_t st, bool as_if_resizing);

int reserve(cpma* h, uint64_t max_batch, int tagged, cudaStream_t st) {
  if (max_batch >= (1ull << 31)) return CPMA_EINVAL;
  if (max_batch == 0) return CPMA_OK;
  // everything an insert of max_batch keys reserves, a growing resize included
  CPMA_TRY(reserve_update(h, max_batch, 0, st, true));
  CPMA_TRY(front_scratch(h, max_batch, tagged != 0, st));
  if (!tagged && h->point_max) CPMA_TRY(point_scratch(h, std::min(max_batch, h->point_max), st));
  if (h->graph_max_batch && !tagged) {
    const uint64_t K = graph_bucket(std::min(max_batch, h->graph_max_batch));
    if (K < (1ull << 31)) {
      CPMA_TRY(ensure(h, h->s.stage, K * 8));
      CPMA_TRY(front_scratch(h, K, false, st));
    }
  }
  return CPMA_OK;
}

// Everything an update of k keys can allocate once it starts changing the
// structure, reserved before it does, so that running out of memory (or out
// of budget) leaves the set unchanged: the redistribution buffers for the
// whole set (elements, costs, their prefix -- which also holds the overflow
// elements of pending leaves -- and the source counts and offsets), the
// window lists, the cut points, level bitsets and head fix-up tiles of the
// largest tree a resize can give, and spare leaf arrays when the batch can
// make the array outgrow the live ones.  A resize needs the root bound to
// fail; the used bytes after the merge lie within t_known -+ t_slack (the
// redistribution after the last merge) and 10 bytes per key (an inserted
// key adds at most a 10-byte code, a deleted one removes at most one).
int reserve_update(cpma* h, uint64_t k, int is_delete, cudaStream_t st, bool as_if_resizing) {
  Scratch& s = h->s;
  const uint64_t n = h->n, L = h->L;
  const uint64_t n_hi = is_delete ? n : n + k, n_lo = is_delete ? (n > k ? n - k : 0) : n;
  // grown with an eighth to spare, so that a set growing batch by batch
  // does not reallocate them at every step
  const uint64_t n_res = n_hi + n_hi / 8;
  if (s.E.cap < (n_hi + 1) * 8) CPMA_TRY(ensure(h, s.E, (n_res + 1) * 8, st));
  if (s.cost.cap < n_hi + 1) CPMA_TRY(ensure(h, s.cost, n_res + 1, st));
  if (s.C.cap < (n_hi + 2) * 8) CPMA_TRY(ensure(h, s.C, (n_res + 2) * 8, st));
  const uint64_t dk = 10 * k;
  const uint64_t t_hi = h->t_known + h->t_slack + (is_delete ? 0 : dk);
  const uint64_t sub = h->t_slack + (is_delete ? dk : 0);
  const uint64_t t_lo = h->t_known > sub ? h->t_known - sub : 0;
  const Bounds B = bounds_of(h);
  const unsigned H = ceil_log2(L);
  const bool may_resize = as_if_resizing || node_violates(B, H, H, L, t_hi) ||
                          node_violates(B, H, H, L, t_lo);
  uint64_t Lmax = L, bytes_max = L * h->cfg.leaf_bytes;
  if (may_resize) {
    // the most leaves and bytes over every key count the batch can leave
    // (each leaf size between theirs) at the most bytes
    uint32_t b_lo = 0, b_hi = 0;
    while (b_lo < 64 && (n_lo >> b_lo)) b_lo++;
    while (b_hi < 64 && (n_hi >> b_hi)) b_hi++;
    for (uint32_t b = b_lo; b <= b_hi; b++) {
      const uint64_t nn = b == b_lo ? n_lo : b == b_hi ? n_hi : (1ull << (b - 1));
      uint64_t Lp = 0;
      uint32_t LBp = 0;
      // (as_if_resizing: at least the bytes that would need one more grow)
      const uint64_t tt = as_if_resizing ? std::max<uint64_t>(
          t_hi, (uint64_t)((unsigned __int128)h->cfg.tau_root * L * h->cfg.leaf_bytes / 1000 + 1))
                                         : t_hi;
      resize_plan(h, tt, nn, &Lp, &LBp);
      Lmax = std::max(Lmax, Lp);
      bytes_max = std::max(bytes_max, Lp * LBp);
    }
  }
  if (Lmax > h->cap_leaves || bytes_max > h->cap_bytes) {
    h->spare_idle = 0;
    if (h->spare.cap_leaves < Lmax || h->spare.cap_bytes < bytes_max) {
      free_arrays(h, &h->spare);  // never in use between updates
      CPMA_TRY(alloc_arrays(h, Lmax, bytes_max, &h->spare, st));
    }
  } else if (h->spare.data && ++h->spare_idle > 64) {
    // kept while resizes stay likely; returned after 64 updates that could
    // not have resized
    free_arrays(h, &h->spare);
  }
  // leaf-count buffers for the larger of the two trees, so that the update
  // after a resize finds them sized too
  CPMA_TRY(ensure_win(h, std::min(k, Lmax) + 2));
  CPMA_TRY(ensure(h, s.srccnt, (Lmax + 1) * 4, st));
  CPMA_TRY(ensure(h, s.srcoff, (Lmax + 2) * 8, st));
  CPMA_TRY(ensure(h, s.prefix, (Lmax + 2) * 8, st));
  CPMA_TRY(ensure(h, s.dstart, (Lmax + 1) * 8, st));
  uint64_t words = 0;
  levels_of(Lmax, ceil_log2(Lmax), &words);
  const void* bits_before = s.bits.p;
  CPMA_TRY(ensure(h, s.bits, words * 4, st));
  if (s.bits.p != bits_before) h->bits_words = 0;  // a new buffer: ensure_bits zeroes it
  CPMA_TRY(ensure(h, s.fh, ((Lmax + kFHTile - 1) / kFHTile) * sizeof(FHTile), st));
  return CPMA_OK;
}

// Every scratch buffer of the update path and the spare leaf arrays freed
// (after the device is idle), and the graphs that bake their addresses in.
void trim_update_scratch(cpma* h) {
  cudaDeviceSynchronize();
  graph_cache_free(h);
  Scratch& s = h->s;
  for (Buf* b : {&s.keysA, &s.keysB, &s.valsA, &s.valsB, &s.hist, &s.flags, &s.flags_scan,
                 &s.leaf_of, &s.chunk_begin, &s.chunk_leaf, &s.chunk_tid, &s.chunk_cnt,
                 &s.chunk_off, &s.T_leaf, &s.T_begin, &s.T_first_chunk, &s.T_oldcnt, &s.T_oldused,
                 &s.T_newcnt, &s.T_newbytes, &s.T_state, &s.viol, &s.list_lane, &s.list_v1,
                 &s.list_gen, &s.list_pend, &s.point_stage, &s.point_rec, &s.cand, &s.wins,
                 &s.bits, &s.prefix, &s.E, &s.cost, &s.C,
                 &s.srccnt, &s.srcoff, &s.dstart, &s.win_src, &s.win_dst, &s.win_leaf_off,
                 &s.win_elem_off, &s.win_dst_off, &s.partials, &s.stage, &s.fh})
    release(h, *b);
  h->bits_words = 0;
  free_arrays(h, &h->spare);
}

// Set while an update changes the structure: every allocation then fails.
struct NoAlloc {
  cpma* h;
  explicit NoAlloc(cpma* hh) : h(hh) { h->no_alloc = true; }
  ~NoAlloc() { h->no_alloc = false; }
};

int run_update(cpma* h, const uint64_t* d_keys, uint64_t k, int sorted, int is_delete,
               uint64_t* d_delta, cudaStream_t st, const uint32_t* tags, uint64_t* tag_counts,
               uint64_t ntags) {
  Status* ds = h->d_status;
  if (tag_counts && ntags) CPMA_CUDA(cudaMemsetAsync(tag_counts, 0, ntags * 8, st));
  if (k == 0) {
    if (d_delta) CPMA_CUDA(cudaMemsetAsync(d_delta, 0, 8, st));
    return CPMA_OK;
  }
  if (k >= (1ull << 31)) return CPMA_EINVAL;
  if (h->cfg.rebuild_pm && !tags &&
      (unsigned __int128)1000 * k >= (unsigned __int128)h->cfg.rebuild_pm * h->n)
    return run_rebuild(h, d_keys, k, sorted, is_delete, d_delta, st);
  Scratch& s = h->s;
  const bool graph = k <= h->graph_max_batch && !tags && graph_bucket(k) < (1ull << 31);
  int rc = reserve_update(h, k, is_delete, st, false);
  if (rc == CPMA_OK && graph) {
    rc = ensure(h, s.stage, graph_bucket(k) * 8, st);
    if (rc == CPMA_OK) rc = front_scratch(h, graph_bucket(k), false, st);
  } else if (rc == CPMA_OK) {
    rc = front_scratch(h, k, tags != nullptr, st);
  }
  if (rc == CPMA_ENOMEM) {
    // refused before any change; give back the scratch grown so far, so
    // that a smaller batch after this one starts from the structure alone
    trim_update_scratch(h);
    return rc;
  }
  CPMA_TRY(rc);
  // the point path; the batch algorithm below when its scratch cannot be
  // had within the memory budget, or when some touched leaf cannot change
  // in place (nothing has been written then)
  const int prc = point_ok(h, k, is_delete, tags) ? point_scratch(h, k, st) : CPMA_ENOMEM;
  if (prc != CPMA_OK && prc != CPMA_ENOMEM) return prc;
  if (prc == CPMA_OK) {
    bool fb = false;
    CPMA_TRY(run_point(h, d_keys, k, sorted, is_delete, d_delta, st, &fb));
    h->point_calls++;
    if (!fb) return CPMA_OK;
    h->point_batch++;
  }
  Front f;
  if (graph) {
    CPMA_TRY(run_front_graph(h, d_keys, k, sorted, is_delete, st, &f));
  } else {
    CPMA_TRY(run_front(h, d_keys, k, sorted, is_delete, st, tags, tag_counts, ntags, &f));
  }
  const NoAlloc guard(h);  // from here on everything needed is reserved
  MergeArgs& ma = f.ma;
  FinArgs& fa = f.fa;
  const Levels& lv = f.lv;
  const unsigned H = f.H;
  const Bounds B = bounds_of(h);
  const int mgrid = f.mgrid, mwarps = f.mwarps;
  const size_t msmem = f.msmem;
  CPMA_TRY(sync_status(h, st));
  prof_begin(h, PH_COUNT, st);
  Status hs = *h->h_status;
  if (hs.err & (kErrSort | kErrRoute)) return CPMA_ETIMEOUT;
  if (hs.err & kErrUnsorted) return CPMA_EINVAL;
  if (hs.err) return CPMA_EINTERNAL;
  const uint64_t t_merged = hs.bytes_total;  // exact: every leaf changed by the merge counted
  uint64_t t_slack = 0;
  const uint64_t delta = hs.delta;
  const uint64_t n_after = is_delete ? h->n - delta : h->n + delta;
  // empty leaves: made by this batch's merges, or left when the last head
  // fix-up ran (a window redistribution never empties a leaf: each gets
  // about S/W >= rho_leaf LB > 10 bytes, more than one code)
  h->may_have_empty = hs.nempty || hs.empties;

  // ---- pending leaves: materialise their merged elements ----
  if (hs.npend) {
    if (s.C.cap < (hs.novf + 1) * 8) return CPMA_EINTERNAL;  // reserved: novf <= n + k
    // offsets of the work items' merged elements, only needed here
    CPMA_TRY(scan_u32_to_u64(h, ma.chunk_cnt, P<uint64_t>(s.chunk_off), f.k + 1, &ds->nchunks,
                             st));
    ma.ovf = P<uint64_t>(s.C);
    ma.tag_counts = nullptr;
    CPMA_CUDA(launch_pdl(k_merge<true>, (unsigned)(mgrid), mwarps * 32, msmem, st, ma));
    h->launches++;
    CPMA_CUDA(cudaGetLastError());
  }

  // ---- counting ----
  bool resized = false;
  if (hs.nviol || hs.npend) {
    if (hs.nviol) {
      CPMA_TRY(scan_u32_to_u64(h, h->used, P<uint64_t>(s.prefix), h->L, nullptr, st));
      WalkArgs wa;
      wa.viol = fa.viol;
      wa.P = P<uint64_t>(s.prefix);
      wa.L = h->L;
      wa.bits = fa.bits;
      wa.cand = fa.cand;
      wa.lv = lv;
      wa.B = B;
      wa.H = H;
      wa.st = ds;
      CPMA_CUDA(launch_pdl(k_walk, (unsigned)(grid_for(h, hs.nviol)), kT, 0, st, wa));
      h->launches++;
    }
    const uint64_t ncand_bound = hs.nviol + hs.npend + 1;
    CPMA_CUDA(launch_pdl(k_maximal, (unsigned)(grid_for(h, ncand_bound)), kT, 0, st, fa.cand,
                         fa.bits, lv, H, h->L, P<uint64_t>(s.wins), ds));
    CPMA_CUDA(launch_pdl(k_clear_bits, (unsigned)(grid_for(h, ncand_bound)), kT, 0, st, fa.cand,
                         fa.bits, lv, ds));
    h->launches += 2;
    CPMA_CUDA(cudaGetLastError());
    prof_end(h, st);
    CPMA_TRY(sync_status(h, st));
    hs = *h->h_status;
    if (hs.err) return CPMA_EINTERNAL;
    prof_begin(h, PH_REDIST, st);
    if (hs.resize) {
      const uint64_t L0 = h->L;
      CPMA_TRY(do_resize(h, st, hs.total_bytes, n_after, hs.nT));
      t_slack = 9 * std::max(L0, h->L);
      resized = true;
    } else if (hs.nwin) {
      const uint64_t nwin = hs.nwin;
      CPMA_TRY(ensure_win(h, nwin));
      // windows in place: destination = source
      CPMA_CUDA(cudaMemcpyAsync(s.win_src.p, s.wins.p, nwin * 16, cudaMemcpyDeviceToDevice, st));
      CPMA_CUDA(cudaMemcpyAsync(s.win_dst.p, s.wins.p, nwin * 16, cudaMemcpyDeviceToDevice, st));
      CPMA_CUDA(launch_pdl(k_win_sizes, (unsigned)(grid_for(h, nwin)), kT, 0, st,
                           P<uint64_t>(s.wins), nwin, P<uint64_t>(s.prefix)));
      h->launches++;
      CPMA_TRY(scan_u64(h, P<uint64_t>(s.prefix), P<uint64_t>(s.win_leaf_off), nwin, nullptr, st));
      CPMA_CUDA(cudaMemcpyAsync(s.win_dst_off.p, s.win_leaf_off.p, (nwin + 1) * 8,
                                cudaMemcpyDeviceToDevice, st));
      CPMA_TRY(redistribute(h, st, nwin, hs.win_leaves, hs.win_leaves, n_after, hs.nT,
                            live_arrays(h), h->cfg.leaf_bytes));
      t_slack = 9 * hs.win_leaves;
    }
  }
  prof_end(h, st);
  prof_begin(h, PH_FINISH, st);
  if (resized) {
    Levels lv2;
    CPMA_TRY(ensure_bits(h, st, &lv2));
    h->may_have_empty = true;
  }
  if (h->may_have_empty) CPMA_TRY(fix_heads(h, st));
  h->n = n_after;
  // the bytes a re-encode changes: a new head costs at most 7 more than the
  // code it replaces, a former head at most 2 more as a code (and the
  // reverse), per leaf of the larger side
  h->t_known = t_merged;
  h->t_slack = t_slack;
  if (d_delta)
    CPMA_CUDA(cudaMemcpyAsync(d_delta, &ds->delta, 8, cudaMemcpyDeviceToDevice, st));
  CPMA_CUDA(cudaGetLastError());
  prof_end(h, st);
  return CPMA_OK;
}

// App. A constructor over sorted distinct keys E[0..n) (already in the E
// scratch buffer): L = max(1, ceil(1000 S / (build_pm LB - 8000))) leaves for
// a stream of S bytes, then one byte-balanced spread.
int build_from_sorted_unique(cpma* h, const uint64_t* E, uint64_t n, cudaStream_t st) {
  typedef unsigned __int128 u128;
  const uint32_t LB = leaf_size_for(h, n);
  Scratch& s = h->s;
  CPMA_TRY(ensure_win(h, 1));
  CPMA_TRY(ensure(h, s.cost, n + 1));
  CPMA_TRY(ensure(h, s.C, (n + 2) * 8));
  if (E != P<uint64_t>(s.E)) return CPMA_EINTERNAL;
  // costs and stream bytes (one window, no source leaves)
  CPMA_CUDA(launch_pdl(k_set_window, (unsigned)(1), 1, 0, st, P<uint64_t>(s.win_src),
                       P<uint64_t>(s.win_dst), P<uint64_t>(s.win_leaf_off),
                       P<uint64_t>(s.win_dst_off), 0, 0, 0, 1));
  h->launches++;
  uint64_t eo[2] = {0, n};
  CPMA_CUDA(cudaMemcpyAsync(s.win_elem_off.p, eo, 16, cudaMemcpyHostToDevice, st));
  CPMA_CUDA(cudaMemcpyAsync(&h->d_status->nelem, &n, 8, cudaMemcpyHostToDevice, st));
  WinArgs w = win_args(h, 1);
  CPMA_CUDA(launch_pdl(k_costs, (unsigned)(grid_for(h, n)), kT, 0, st, w, E, &h->d_status->nelem,
                       P<uint8_t>(s.cost), (int)h->cfg.codec));
  h->launches++;
  CPMA_TRY(scan_u8_to_u64(h, P<uint8_t>(s.cost), P<uint64_t>(s.C), n, nullptr, st));
  CPMA_CUDA(cudaMemcpyAsync(&h->d_status->stream_bytes, P<uint64_t>(s.C) + n, 8,
                            cudaMemcpyDeviceToDevice, st));
  CPMA_TRY(sync_status(h, st));
  const uint64_t S = h->h_status->stream_bytes;
  const u128 num = (u128)S * 1000, den = (u128)h->cfg.build_pm * LB - 8000;
  uint64_t L = (uint64_t)((num + den - 1) / den);
  if (L < 1) L = 1;
  Arrays na;
  CPMA_TRY(alloc_arrays(h, L, L * LB, &na, st));
  CPMA_CUDA(launch_pdl(k_set_window, (unsigned)(1), 1, 0, st, P<uint64_t>(s.win_src),
                       P<uint64_t>(s.win_dst), P<uint64_t>(s.win_leaf_off),
                       P<uint64_t>(s.win_dst_off), 0, 0, 0, L));
  h->launches++;
  CPMA_TRY(ensure(h, s.dstart, (L + 1) * 8));
  CPMA_CUDA(launch_pdl(k_starts, (unsigned)(grid_for(h, L)), kT, 0, st, w, P<uint64_t>(s.C), L,
                       P<uint64_t>(s.dstart)));
  h->launches++;
  EncodeArgs ea;
  ea.w = w;
  ea.ndst = L;
  ea.dstart = P<uint64_t>(s.dstart);
  ea.E = E;
  ea.C = P<uint64_t>(s.C);
  ea.data = na.data;
  ea.used = na.used;
  ea.cnt = na.cnt;
  ea.heads = na.heads;
  ea.LB = LB;
  ea.st = h->d_status;
  ea.raw = (int)h->cfg.codec;
  // the byte total restarts with the new leaves (the encode adds them)
  int rc = check_cuda(cudaMemsetAsync(&h->d_status->bytes_total, 0, 8, st));
  if (rc == CPMA_OK) {
    CPMA_CUDA(launch_pdl(k_encode, (unsigned)(grid_for(h, L * 32)), kT, (size_t)(kT / 32) * LB, st,
                         ea));
    h->launches++;
    rc = check_cuda(cudaGetLastError());
  }
  if (rc == CPMA_OK) rc = check_cuda(cudaStreamSynchronize(st));
  if (rc != CPMA_OK) {
    free_arrays(h, &na);
    return rc;
  }
  Arrays old = live_arrays(h);
  free_arrays(h, &old);
  free_arrays(h, &h->spare);
  set_live(h, na);
  h->cfg.leaf_bytes = LB;
  h->L = L;
  h->n = n;
  Levels lv;
  CPMA_TRY(ensure_bits(h, st, &lv));
  h->may_have_empty = true;
  CPMA_TRY(fix_heads(h, st));
  CPMA_TRY(sync_status(h, st));
  if (h->h_status->err) return CPMA_EINTERNAL;
  h->may_have_empty = h->h_status->empties > 0;
  h->t_known = h->h_status->bytes_total;
  h->t_slack = 0;
  return CPMA_OK;
}

}  // namespace cpmaimpl
