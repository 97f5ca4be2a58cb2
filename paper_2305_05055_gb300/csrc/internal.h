// Host-side internals of the CPMA library: the handle, its scratch buffers and
// the kernel launchers of each translation unit.
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cpma.h"

namespace cpmaimpl {

typedef unsigned long long ull;

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation (launch_pdl) may be scheduled while the kernel before it in
// the stream still runs.  pdl_wait() returns once that kernel has completed
// and its memory operations are visible (at once when the launch carried no
// such dependency), so a kernel calls it before reading anything its
// predecessor wrote -- and every kernel so launched calls it, so that its
// own completion implies its predecessors'.  pdl_launch() lets the next
// kernel be scheduled.
#if defined(__CUDACC__)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kern)(Params...), unsigned grid, unsigned block, size_t smem,
                       cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Params>(args)...);
}
#endif

// Device-side control block of one batch.  The host reads it back once or
// twice per update to size the later phases.
struct Status {
  ull nT;          // routed leaves (runs of the sorted batch)
  ull nchunks;     // merge work items (runs split every kChunk keys)
  ull delta;       // keys added (insert) or removed (delete)
  ull npend;       // leaves whose merged content waits in the overflow buffer
  ull novf;        // overflow elements
  ull nviol;       // touched leaves that violate their own bound
  ull ncand;       // window candidates (distinct tree nodes)
  ull resize;      // some walk passed the root
  ull nwin;        // maximal windows
  ull win_leaves;  // leaves over all maximal windows
  ull total_bytes; // bytes over all leaves after the merge
  ull nempty;      // empty leaves written by this batch
  ull err;         // device-side error flags (kErr*)
  ull mask_or;     // OR / AND of the batch keys (radix pass selection)
  ull mask_and;
  ull nelem;       // elements moved by the current redistribution
  ull nunique;     // distinct keys after sort+dedup (create)
  ull stream_bytes;// bytes of the build stream (create)
  ull n_lane;      // touched leaves for the lane-granular insert
  ull n_v1;        // touched leaves for the element-array splice
  ull n_gen;       // work items for the general merge
  ull n_pendl;     // pending leaves left by the thread- and lane-granular inserts
  ull point_fb;    // point path: touched leaves that need the batch algorithm
  ull point_done;  // point path: blocks finished (the last one finishes the pass)
  ull pad[7];
  ull empties;     // empty leaves in the structure (written by the head
                   // fix-up; not cleared at the start of a batch)
  ull bytes_total; // used bytes over all leaves, kept exact by the merge,
                   // redistribution and build kernels (not cleared either)
};

constexpr ull kErrUnsorted = 1;   // a batch promised sorted was not
constexpr ull kErrFit = 2;        // a redistributed leaf did not fit
constexpr ull kErrState = 4;      // inconsistent leaf state
constexpr ull kErrSort = 8;       // a sort tile waited too long for its predecessor
constexpr ull kErrRoute = 16;     // a routing tile waited too long for its predecessor

constexpr uint32_t kChunk = 256;  // keys per merge work item
constexpr int kMaxLevels = 48;

// T-entry states after the merge
constexpr uint32_t kUnchanged = 0, kInPlace = 1, kPending = 2;

// A grow-only device buffer.
struct Buf {
  void* p = nullptr;
  size_t cap = 0;
};

// Leaf arrays: data (leaves x LB bytes), used, cnt, heads (leaves + 1), with
// the capacity they were allocated for.
struct Arrays {
  uint8_t* data = nullptr;
  uint32_t* used = nullptr;
  uint32_t* cnt = nullptr;
  uint64_t* heads = nullptr;
  uint64_t cap_leaves = 0;   // entries of used / cnt (heads: one more)
  uint64_t cap_bytes = 0;    // bytes of data
};

struct Scratch {
  Buf keysA, keysB;       // sort ping-pong (u64)
  Buf valsA, valsB;       // sort ping-pong of 32-bit tags
  Buf hist;               // sort control block and look-back arrays
  Buf flags;              // routing: tile counter and look-back words (u64)
  Buf flags_scan;         // build and rebuild: scanned flags (u64)
  Buf leaf_of;            // build: unique flags (u32)
  Buf chunk_begin, chunk_leaf, chunk_tid, chunk_cnt, chunk_off;
  Buf T_leaf, T_begin, T_first_chunk, T_oldcnt, T_oldused, T_newcnt, T_newbytes, T_state;
  Buf viol, cand, wins;   // violating leaves, window candidates, windows
  Buf list_lane, list_v1, list_gen;  // merge work lists
  Buf list_pend;          // pending leaves of the thread- and lane-granular inserts
  Buf point_stage;        // point path: 512-byte staging slot per key
  Buf point_rec;          // point path: staged result per key
  Buf bits;               // per-level window bitsets (u32 words)
  Buf prefix;             // prefix sums of used bytes (u64, L+1)
  Buf E, cost, C;         // redistribution: elements, costs, cost prefix; C also holds
                          // the overflow elements of pending leaves until the pack
  Buf srccnt, srcoff, dstart;
  Buf win_src, win_dst, win_leaf_off, win_elem_off, win_dst_off;
  Buf partials;           // scan partials (update path)
  Buf partials_q;         // scan partials of the query path, which may run
                          // on another stream while an update sorts
  Buf q_first, q_items, q_off; // range queries
  Buf q_lo, q_hi, q_rank;       // map_range_length: rank bounds, leaf-count prefix
  Buf stage;              // padded batch of a graph-launched update
  Buf fh;                 // head fix-up: per-tile summaries
};

// Profiling phases (cpma_profile_read order).
enum Phase {
  PH_SORT = 0, PH_ROUTE, PH_MERGE, PH_COUNT, PH_REDIST, PH_FINISH,
  PH_HAS, PH_RANGE_PREP, PH_RANGE, PH_SUM, PH_MERGE2, PH_MERGE_LANE, PH_N
};

// Optional per-phase device timing: event pairs recorded around each phase
// and resolved at the next host synchronisation, so profiling adds no waits.
struct Prof {
  bool on = false;
  uint32_t mask = ~0u;  // phases timed (bit per phase); the byte counts cover all
  // pooled: the events go back to the pool once resolved; a captured graph's
  // events belong to the graph and are recorded again by every replay
  struct Rec { int phase; cudaEvent_t a, b; bool pooled; };
  Rec open_rec{-1, nullptr, nullptr, true};
  Rec side_rec{-1, nullptr, nullptr, true};  // a phase running on the side stream meanwhile
  // while a graph is being captured: its event pairs and its host-side byte
  // counts, which each replay adds
  bool capturing = false;
  Rec* cap_recs = nullptr;
  int ncap = 0, cap_max = 0;
  unsigned long long cap_host_bytes[PH_N] = {0};
  Rec* pending = nullptr;
  int npending = 0, cap = 0;
  cudaEvent_t* pool = nullptr;
  int npool = 0, pool_cap = 0;
  double ms[PH_N] = {0};
  unsigned long long calls[PH_N] = {0};
  unsigned long long* d_bytes = nullptr;  // device: algorithmic bytes per phase
  unsigned long long host_bytes[PH_N] = {0};  // bytes known on the host
};

}  // namespace cpmaimpl

struct cpma {
  cpma_config cfg;       // cfg.leaf_bytes is the leaf size in use
  uint32_t lb_min = 0;   // the configured leaf size (smallest with leaf_growth)
  int device = 0;
  int num_sms = 0;
  uint64_t L = 0;        // leaves
  uint64_t n = 0;        // keys
  uint8_t* data = nullptr;
  uint32_t* used = nullptr;
  uint32_t* cnt = nullptr;
  uint64_t* heads = nullptr;       // L + 1 entries; heads[L] = last non-empty leaf
  uint64_t cap_leaves = 0, cap_bytes = 0;  // capacity of the arrays above
  cpmaimpl::Arrays spare;          // arrays kept for a resize the next update may need
  uint32_t spare_idle = 0;         // updates since a resize was last possible
  // memory: bytes held (structure, spare arrays, scratch, status), and a
  // flag that makes every allocation fail (set while an update is changing
  // the structure: everything it needs was reserved before)
  uint64_t mem_held = 0, mem_peak = 0;
  bool no_alloc = false;
  // used bytes over all leaves: exact after the last merge (t_known) and a
  // bound on how much the redistribution after it changed them (t_slack)
  uint64_t t_known = 0, t_slack = 0;
  // batch sort look-back (tests): poll limit (0 = default), silent tile (-1 = none)
  uint32_t sort_poll_limit = 0;
  int64_t sort_silent_tile = -1;
  uint64_t bits_words = 0;          // words of the window bitsets now zeroed
  bool may_have_empty = false;      // some leaf may be empty (head fix-up)
  cpmaimpl::Status* d_status = nullptr;
  cpmaimpl::Status* h_status = nullptr;  // pinned
  cpmaimpl::Scratch s;
  // kernels launched; atomic because const queries on one handle may be
  // issued from several host threads
  std::atomic<uint64_t> launches{0};
  cpmaimpl::Prof prof;
  uint64_t graph_max_batch = 0;     // batches up to this size run their front segment as a graph
  void* graphs = nullptr;           // graph cache (update.cu)
  cudaStream_t cap_stream = nullptr;  // private stream graphs are captured on
  // side stream of the merge fork (k_insert_lane next to k_insert_thread) and
  // its fork / join events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  uint64_t graph_captures = 0, graph_launches = 0;
  // untagged updates of up to this many keys try the point path first (at
  // most 16384; 0 = never); updates that took it, and those of them that the
  // batch algorithm finished instead
  uint64_t point_max = 16384;
  uint64_t point_calls = 0, point_batch = 0;
};

namespace cpmaimpl {

// memory.  Every device allocation goes through dev_alloc / dev_free: the
// configured allocator (or cudaMalloc / cudaFree), the memory budget, and the
// handle's count of bytes held.  ensure() grows a buffer (never shrinks).
// While a graph is being captured on this thread, or while h->no_alloc is
// set, it refuses to allocate (CPMA_EINTERNAL) instead.
int dev_alloc(cpma* h, void** p, size_t bytes, cudaStream_t st);
void dev_free(cpma* h, void* p, size_t bytes, cudaStream_t st);
int ensure(cpma* h, Buf& b, size_t bytes, cudaStream_t st = nullptr);
void release(cpma* h, Buf& b);
int alloc_arrays(cpma* h, uint64_t leaves, uint64_t data_bytes, Arrays* a, cudaStream_t st);
void free_arrays(cpma* h, Arrays* a);
void set_capturing(bool on);

// update.cu: graph cache and scratch reservation
void graph_cache_free(cpma* h);
int reserve(cpma* h, uint64_t max_batch, int tagged, cudaStream_t st);

// scan.cu: exclusive prefix sums.  out has n+1 entries (out[n] = total).
// The element count is n_host, or *n_dev when n_dev != nullptr (n_host is
// then an upper bound used to size the launch).
int scan_u32_to_u64(cpma* h, const uint32_t* in, uint64_t* out, uint64_t n_host,
                    const ull* n_dev, cudaStream_t st);
int scan_u8_to_u64(cpma* h, const uint8_t* in, uint64_t* out, uint64_t n_host,
                   const ull* n_dev, cudaStream_t st);
int scan_u64(cpma* h, const uint64_t* in, uint64_t* out, uint64_t n_host, const ull* n_dev,
             cudaStream_t st);
// scan_u64 with the query path's own partials buffer
int scan_u64_query(cpma* h, const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t st);
int scan_u32_query(cpma* h, const uint32_t* in, uint64_t* out, uint64_t n, cudaStream_t st);
// Same as scan_u64 for a host-known count, with caller-provided partials
// (partials_cap entries); it never allocates.
int scan_u64_given_partials(cpma* h, const uint64_t* in, uint64_t* out, uint64_t n_host,
                            uint64_t* partials, uint64_t partials_cap, cudaStream_t st);

// sort.cu: size the sort scratch for k keys (with 32-bit payloads if vals)
// and set the kernels' shared-memory attributes.
int sort_scratch(cpma* h, uint64_t k, bool vals);
// sort.cu: sort k keys ascending into *out (one of the scratch buffers).
int sort_keys(cpma* h, const uint64_t* d_in, uint64_t k, const uint64_t** out,
              cudaStream_t st);
// the same, moving a 32-bit payload with every key (stable)
int sort_pairs(cpma* h, const uint64_t* d_in, const uint32_t* v_in, uint64_t k,
               const uint64_t** out, const uint32_t** vout, cudaStream_t st);
// sort.cu: drop adjacent repeats of sorted keys; result count into status->nunique.
int unique_keys(cpma* h, const uint64_t* in, uint64_t k, uint64_t* out, cudaStream_t st);

// update.cu
// tags / tag_counts (nullable): per key a request tag; every key that the
// batch adds (insert) or removes (delete) adds 1 to tag_counts[tag of its
// first occurrence in the sorted batch]; tag_counts has ntags entries.
int run_update(cpma* h, const uint64_t* d_keys, uint64_t k, int sorted, int is_delete,
               uint64_t* d_delta, cudaStream_t st, const uint32_t* tags = nullptr,
               uint64_t* tag_counts = nullptr, uint64_t ntags = 0);
int build_from_sorted_unique(cpma* h, const uint64_t* E, uint64_t n, cudaStream_t st);

// query.cu
int run_has(const cpma* h, const uint64_t* d_keys, uint64_t q, uint8_t* d_out, cudaStream_t st);
int run_range(const cpma* h, const uint64_t* lo, const uint64_t* hi, uint64_t q, uint64_t* sum,
              uint64_t* count, cudaStream_t st);
int run_sum(const cpma* h, uint64_t* sum, uint64_t* count, cudaStream_t st);
int run_range_length(const cpma* h, const uint64_t* start, const uint64_t* length, uint64_t q,
                     uint64_t* sum, uint64_t* count, cudaStream_t st);
int run_range_extract(const cpma* h, const uint64_t* lo, const uint64_t* hi, uint64_t q,
                      uint64_t* offsets, uint64_t* out, uint64_t cap, cudaStream_t st);
int run_range_reduce(const cpma* h, const uint64_t* lo, const uint64_t* hi, uint64_t q, int op,
                     uint64_t mask, uint64_t value, uint64_t* out, uint64_t* count,
                     cudaStream_t st);
int run_range_noalloc(const cpma* h, const uint64_t* lo, const uint64_t* hi, uint64_t q,
                      uint64_t* sum, uint64_t* count, cudaStream_t st);

int check_cuda(cudaError_t e);
int sync_status(cpma* h, cudaStream_t st);

// profiling (no-ops unless enabled)
void prof_begin(const cpma* h, int phase, cudaStream_t st);
void prof_end(const cpma* h, cudaStream_t st);
// A second phase open at the same time, on another stream (the side stream
// of a fork).
void prof_begin_side(const cpma* h, int phase, cudaStream_t st);
void prof_end_side(const cpma* h, cudaStream_t st);
void prof_resolve(const cpma* h);  // call only after the stream is idle
// queue a replayed graph's event pairs for resolution and add its host bytes
void prof_push(const cpma* h, const Prof::Rec* recs, int n, const unsigned long long* host_bytes);
inline void prof_add_bytes(const cpma* h, int phase, unsigned long long b) {
  Prof& p = const_cast<cpma*>(h)->prof;
  if (!p.on) return;
  if (p.capturing) p.cap_host_bytes[phase] += b;
  else p.host_bytes[phase] += b;
}
inline unsigned long long* prof_bytes(const cpma* h, int phase) {
  return h->prof.on ? h->prof.d_bytes + phase : nullptr;
}

inline unsigned ceil_log2(uint64_t L) {
  unsigned H = 0;
  while ((1ull << H) < L) H++;
  return H;
}

}  // namespace cpmaimpl

#define CPMA_TRY(x)              \
  do {                           \
    int _rc = (x);               \
    if (_rc != CPMA_OK) return _rc; \
  } while (0)
#define CPMA_CUDA(x) CPMA_TRY(::cpmaimpl::check_cuda(x))
#define CPMA_LAUNCHED(h) (const_cast<cpma*>(h)->launches.fetch_add(1, std::memory_order_relaxed))
