/*
 * cpma.h -- C ABI of a GPU (sm_103a) batch-parallel compressed set: the
 * Compressed Packed Memory Array (CPMA) of Wheatman, Burns, Bulu\c{c} and Xu,
 * "CPMA: An Efficient Batch-Parallel Compressed Set Without Pointers"
 * (PPoPP '24).
 *
 * A CPMA stores a set of distinct 64-bit keys in one flat array of L leaves
 * of LB bytes.  Each non-empty leaf holds its first key (the head) as 8
 * little-endian bytes followed by the deltas to the following keys in
 * unsigned LEB128 byte codes, packed to the left (Sec. 5 "CPMA structure",
 * "Data compression techniques").  An implicit binary tree over the leaves
 * carries byte-density bounds per height (Sec. 3 "Design and operations",
 * Sec. 5 byte density); batch updates merge, count and redistribute
 * (Sec. 4); the array grows by 6/5 when the root bound fails (Sec. 3
 * "Resizing a PMA"; growing factor in App. B).
 *
 * Conventions shared by every call:
 *  - All key, query and result pointers are DEVICE pointers owned by the
 *    caller.  They must stay valid until the work queued on `stream`
 *    completes.  The library never keeps them and never writes to inputs.
 *  - Every uint64 value 0 .. 2^64-1 is a valid key.  Batches may be unsorted
 *    and may repeat keys; repeats are counted once.
 *  - Updates on one handle are single-writer: issue them on one stream (or
 *    order the streams).  cpma_has_batch and cpma_sum use no scratch and may
 *    run concurrently with each other and with the range calls; the range
 *    calls (cpma_range_map, _length, _extract, _reduce) share the handle's
 *    query scratch, so two of them on one handle must be ordered (one
 *    stream, or events).  No query may overlap an update unless the caller
 *    orders them.  A handle's host-side state is not locked: calls on one
 *    handle from several host threads must be serialised by the caller,
 *    except the const queries above, which only read it.
 *  - Every call returns CPMA_OK (0) or a negative error code (below).  An
 *    update is all or nothing with respect to memory: before it changes
 *    anything it reserves every byte of device memory it can need (scratch
 *    for the batch, overflow and redistribution buffers for the whole set,
 *    and new leaf arrays when the batch can make the array grow), so
 *    CPMA_ENOMEM -- from the allocator or the memory budget -- and
 *    CPMA_EINVAL, CPMA_ETIMEOUT and the rejection of an unsorted "sorted"
 *    batch all leave the set and the handle exactly as they were.  Only
 *    CPMA_ECUDA (a failed CUDA call) and CPMA_EINTERNAL (a device-side
 *    consistency check) can come after the structure has started to change;
 *    the handle is then unusable (destroy it).
 *  - Calls that take a stream enqueue device work on it; the update calls and
 *    cpma_create also wait on it once or twice for small control values
 *    (batch sizes, whether to resize), so they return with the update
 *    complete on the device.
 */
#ifndef CPMA_H
#define CPMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cpma_stream_t; /* a cudaStream_t; NULL = legacy default */
typedef struct cpma cpma_t;                /* opaque handle */

enum {
  CPMA_OK = 0,
  CPMA_EINVAL = -1,    /* bad argument or configuration */
  CPMA_ENOMEM = -2,    /* device or host allocation failed */
  CPMA_ECUDA = -3,     /* a CUDA call failed */
  CPMA_EINTERNAL = -4, /* a device-side consistency check failed */
  CPMA_ETIMEOUT = -5,  /* a bounded device-side wait gave up (the look-back
                          of the batch sort or of the routing: a tile whose
                          predecessor never published its counts); the set
                          is unchanged */
};

/* Device memory callbacks (cpma_config.alloc / .free).  alloc returns
 * `bytes` of device memory on the handle's device, aligned to at least 256
 * bytes, or NULL when it cannot (the call then fails with CPMA_ENOMEM and
 * leaves the set unchanged).  `stream` is the stream of the library call that
 * needs the memory (NULL when the call has none).  free(p, stream, ctx)
 * returns a block; the library frees a block only after the device has
 * finished all work that uses it (it synchronises first), so any allocator
 * -- stream-ordered or not -- may hand the block out again at once. */
typedef void* (*cpma_alloc_fn)(size_t bytes, cpma_stream_t stream, void* ctx);
typedef void (*cpma_free_fn)(void* p, cpma_stream_t stream, void* ctx);

/* Tunables.  The density bounds follow Sec. 3 ("the density bound of a node
 * depends on its height"; leaf bound 0.9 in the figure captions) read as a
 * linear interpolation from leaf to root:
 *   upper(h) = tau_leaf - (tau_leaf - tau_root) * h / H,
 *   lower(h) = rho_leaf + (rho_root - rho_leaf) * h / H   (permille),
 * H = ceil(log2 L).  With L == 1 only the upper root bound applies.
 * Requirements: 256 <= leaf_bytes <= 2048, leaf_bytes % 16 == 0,
 * rho_leaf <= rho_root < tau_root <= tau_leaf < 1000,
 * (1000 - tau_leaf) * leaf_bytes >= 20000 (a redistributed leaf then always
 * fits), grow_num > grow_den > 0, 8000 < build_pm * leaf_bytes,
 * build_pm <= tau_root.
 * rebuild_pm (Sec. 4: a batch of k >= n/10 keys is best applied by one merge
 * of everything): when it is > 0, an untagged batch of k keys (its length as
 * given) into a set of n keys with 1000 k >= rebuild_pm * n is applied by
 * merging it with all the keys and building the result like cpma_create
 * (layout included); other batches take the batch-merge path.  0 = never
 * (default).
 * codec 1 keeps every key in an 8-byte little-endian cell, packed left,
 * under the same batch algorithm (bounds, routing, counting, resizing): the
 * uncompressed PMA, for measuring what the compression buys.
 * leaf_growth > 0 makes the leaf size grow with the number of keys, as the
 * CPMA's Theta(log n) leaves do (Sec. 5 "CPMA structure"; Sec. 6 space
 * usage): whenever the leaf array is built (cpma_create, a rebuild) or
 * resized, the leaf size becomes
 *   LB(n) = min(2048, max(leaf_bytes, 16 * ceil(leaf_growth * bitlen(n) / 16)))
 * for the n keys it will hold (bitlen(n) = floor(log2 n) + 1, 0 for n = 0),
 * leaf_bytes being the smallest size.  A resize to size LB' starts from the
 * leaf count of equal capacity, ceil(L * LB / LB'), and then grows or
 * shrinks by the growing factor as with a fixed size.  cpma_leaf_bytes
 * returns the size in use. */
typedef struct {
  uint32_t leaf_bytes; /* LB; default 512 */
  uint32_t tau_leaf;   /* default 900 */
  uint32_t tau_root;   /* default 700 */
  uint32_t rho_leaf;   /* default 100 */
  uint32_t rho_root;   /* default 300 */
  uint32_t grow_num;   /* growing factor grow_num / grow_den; default 6/5 */
  uint32_t grow_den;
  uint32_t build_pm;   /* fill density of cpma_create; default 500 */
  uint32_t rebuild_pm; /* batch-to-set ratio that rebuilds; default 0 = never */
  uint32_t codec;      /* leaf format: 0 = byte codes (the CPMA, default),
                          1 = 8-byte cells (the uncompressed PMA of Sec. 3) */
  uint32_t leaf_growth; /* leaf size that grows with n: 0 = fixed leaf_bytes
                           (default); else bytes per bit of n (see below) */
  uint32_t reserved;    /* must be 0 */
  cpma_alloc_fn alloc;  /* device memory; NULL (default) = cudaMalloc */
  cpma_free_fn free;    /* NULL (default) = cudaFree; set both or neither */
  void* alloc_ctx;      /* passed to alloc and free */
  uint64_t mem_budget_bytes; /* cap on the device memory the handle holds
                                (structure and every scratch buffer); a call
                                that would exceed it fails with CPMA_ENOMEM
                                before it changes anything; 0 = no cap */
} cpma_config;

/* Fill *cfg with the defaults above. */
void cpma_default_config(cpma_config* cfg);

/* App. A constructor "CPMA(key_type *start, key_type *end)": build a CPMA
 * holding the distinct keys of d_keys[0..n).  d_keys: device, any order,
 * repeats allowed (n == 0 gives an empty set; d_keys may then be NULL).
 * cfg: NULL for defaults.  The new handle is written to *out and owns all the
 * device memory it allocates (cudaMalloc on the current device). */
int cpma_create(cpma_t** out, const cpma_config* cfg, const uint64_t* d_keys,
                uint64_t n, cpma_stream_t stream);

/* Free the handle and all its device memory (synchronises its last stream). */
int cpma_destroy(cpma_t* h);

/* A deep copy of src (device to device) on `stream`: *out gets a new handle. */
int cpma_clone(const cpma_t* src, cpma_t** out, cpma_stream_t stream);

/* App. A insert_batch: insert the keys d_keys[0..k) (Sec. 4 batch insert:
 * sort, batch merge, counting, redistribute, resize).  sorted != 0 promises
 * that the keys are non-decreasing (repeats still allowed) and skips the
 * sort; a batch that breaks the promise is rejected with CPMA_EINVAL and the
 * set is unchanged.  If d_added is not NULL, the number of keys that were not
 * already present is written to the device uint64 *d_added. */
int cpma_insert_batch(cpma_t* h, const uint64_t* d_keys, uint64_t k,
                      int sorted, uint64_t* d_added, cpma_stream_t stream);

/* App. A remove_batch: delete the keys of d_keys[0..k) that are present
 * (Sec. 3 "deletes x ... if it exists"; Sec. 4 "batch deletes are
 * symmetric").  d_removed (nullable, device) receives the number removed. */
int cpma_delete_batch(cpma_t* h, const uint64_t* d_keys, uint64_t k,
                      int sorted, uint64_t* d_removed, cpma_stream_t stream);

/* Tagged forms of the two updates, for callers that coalesce the batches of
 * several requests into one (Sec. 4 batch updates): d_tags[i] < ntags names
 * the request of d_keys[i].  The result is the set the untagged call gives;
 * in addition d_counts[t] (ntags device uint64, zeroed by the call) receives
 * how many keys request t added (insert) or removed (delete), every changed
 * key being credited to the request of its first occurrence in the batch
 * (the sort is stable, so with the keys laid out in request order the result
 * equals applying the requests one after another in that order).  With
 * sorted != 0 the keys must be non-decreasing and d_tags ordered with them.
 * A tag >= ntags is rejected with CPMA_EINVAL and the set is unchanged. */
int cpma_insert_batch_tagged(cpma_t* h, const uint64_t* d_keys,
                             const uint32_t* d_tags, uint64_t k, int sorted,
                             uint64_t ntags, uint64_t* d_counts,
                             cpma_stream_t stream);
int cpma_delete_batch_tagged(cpma_t* h, const uint64_t* d_keys,
                             const uint32_t* d_tags, uint64_t k, int sorted,
                             uint64_t ntags, uint64_t* d_counts,
                             cpma_stream_t stream);

/* The batch sort of the update path (Sec. 4: an unsorted batch is sorted
 * first) on its own: d_keys[0..k) ascending into d_keys_out, stable, moving
 * d_tags (nullable) along into d_tags_out.  Lets a caller sort the next batch
 * while queries still run on another stream; pass the result to an update
 * with sorted = 1.  Uses the handle's sort scratch: do not overlap it with an
 * update on the same handle. */
int cpma_sort_batch(cpma_t* h, const uint64_t* d_keys, const uint32_t* d_tags,
                    uint64_t k, uint64_t* d_keys_out, uint32_t* d_tags_out,
                    cpma_stream_t stream);

/* App. A has, batched: d_out[i] = 1 if d_keys[i] is in the set, else 0
 * (Sec. 5 "Point queries": binary search on the heads, then one pass over
 * the leaf).  d_keys: q device uint64 in any order; d_out: q device bytes. */
int cpma_has_batch(const cpma_t* h, const uint64_t* d_keys, uint64_t q,
                   uint8_t* d_out, cpma_stream_t stream);

/* Sec. 3 range_map(start, end, f) with f = (sum, count), batched: for every
 * i < q, d_sum[i] = sum of the keys x with d_lo[i] <= x < d_hi[i], modulo
 * 2^64, and d_count[i] = how many there are (both device uint64 arrays of q
 * entries).  lo >= hi gives 0 and 0.  All q queries run in one load-balanced
 * launch over (query, leaf) work items. */
int cpma_range_map(const cpma_t* h, const uint64_t* d_lo, const uint64_t* d_hi,
                   uint64_t q, uint64_t* d_sum, uint64_t* d_count,
                   cpma_stream_t stream);

/* App. A map_range_length(f, start, length) with f = (sum, count), batched:
 * for every i < q, the first min(d_length[i], #keys >= d_start[i]) keys that
 * are >= d_start[i]; d_sum[i] = their sum modulo 2^64, d_count[i] = how many
 * (all device uint64 arrays of q entries).  Length 1 gives the successor of
 * start (Sec. 3 search); start 0 and length 1 the minimum.  One prefix sum of
 * the leaves' element counts per call turns every query into a range of
 * global ranks; the ranks then run through the same load-balanced leaf walk
 * as cpma_range_map.  Errors: CPMA_EINVAL (null handle or array with q > 0),
 * CPMA_ENOMEM (scratch). */
int cpma_range_map_length(const cpma_t* h, const uint64_t* d_start,
                          const uint64_t* d_length, uint64_t q, uint64_t* d_sum,
                          uint64_t* d_count, cpma_stream_t stream);

/* Sec. 3 range_map with f = "emit the key", batched: the keys of [d_lo[i],
 * d_hi[i]) in order, all queries' keys packed into one device array.
 * d_offsets (q + 1 device uint64) receives the exclusive prefix sum of the
 * per-query counts: query i's keys go to d_out[d_offsets[i] ..
 * d_offsets[i+1]) and d_offsets[q] is the total.  Keys at positions >=
 * out_cap are not written; with d_out NULL or out_cap 0 only d_offsets is
 * computed, so a caller sizes d_out from d_offsets[q] and calls again.  Both
 * range ends are turned into global ranks (a prefix sum of the leaves'
 * element counts, then one leaf decode per end), and the leaves between them
 * are decoded by the load-balanced walk of cpma_range_map.  Errors:
 * CPMA_EINVAL (null handle, d_offsets NULL, or d_lo / d_hi NULL with q > 0),
 * CPMA_ENOMEM. */
int cpma_range_extract(const cpma_t* h, const uint64_t* d_lo, const uint64_t* d_hi,
                       uint64_t q, uint64_t* d_offsets, uint64_t* d_out, uint64_t out_cap,
                       cpma_stream_t stream);

/* Functions for cpma_range_reduce. */
#define CPMA_OP_SUM 0 /* sum modulo 2^64; 0 when no key passes */
#define CPMA_OP_MIN 1 /* smallest key; 2^64-1 when no key passes */
#define CPMA_OP_MAX 2 /* largest key; 0 when no key passes */
#define CPMA_OP_XOR 3 /* exclusive or; 0 when no key passes */

/* Sec. 3 range_map(start, end, f) with f one of the CPMA_OP_* reductions over
 * a filter, batched: for every i < q, over the keys x with d_lo[i] <= x <
 * d_hi[i] and (x & mask) == value, d_out[i] = the reduction and d_count[i] =
 * how many keys passed (so mask/value filters give filter-counts).  Every
 * covered leaf is decoded; with CPMA_OP_SUM and mask = value = 0 this is
 * cpma_range_map.  Errors: CPMA_EINVAL (null handle or array with q > 0, op
 * not a CPMA_OP_*), CPMA_ENOMEM. */
int cpma_range_reduce(const cpma_t* h, const uint64_t* d_lo, const uint64_t* d_hi,
                      uint64_t q, int op, uint64_t mask, uint64_t value,
                      uint64_t* d_out, uint64_t* d_count, cpma_stream_t stream);

/* cpma_range_map without any device allocation (the paper has no counterpart:
 * this is a deployment variant).  cpma_range_map grows private scratch with
 * cudaMalloc/cudaFree when a larger batch of queries arrives; some callers
 * cannot let that happen, e.g. a process whose device memory is all handed to
 * another allocator up front, or a latency-bound serving thread that must not
 * hit the device-wide synchronisation cudaFree implies.  This entry point
 * takes its scratch from a fixed 2 MiB array inside the library's device
 * image instead, so it allocates nothing.  Arguments and results are those of
 * cpma_range_map.
 *  - q <= CPMA_RANGE_NOALLOC_MAX_QUERIES (65536); larger q returns
 *    CPMA_EINVAL without doing anything.
 *  - The handle's device must be the current device (else CPMA_EINVAL).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and caches it for the life of the process; make
 *    that first call before any stream capture.  cudaDeviceReset destroys
 *    the array together with every handle on that device, and the cached
 *    address then points nowhere: do not use this entry point on a device
 *    after resetting it (reload the library in a new process).
 *  - Every call on a device shares the one array: calls whose work overlaps
 *    on the GPU (different streams, not ordered) race and give wrong results.
 *    Order them on one stream. */
#define CPMA_RANGE_NOALLOC_MAX_QUERIES 65536
int cpma_range_map_noalloc(const cpma_t* h, const uint64_t* d_lo,
                           const uint64_t* d_hi, uint64_t q, uint64_t* d_sum,
                           uint64_t* d_count, cpma_stream_t stream);

/* App. A sum(): sum of all keys modulo 2^64 into the device uint64 *d_sum
 * (and, if d_count is not NULL, the number of keys into *d_count). */
int cpma_sum(const cpma_t* h, uint64_t* d_sum, uint64_t* d_count,
             cpma_stream_t stream);

/* App. A size(): number of keys, as a host value.  Exact after every update
 * call has returned (the update calls keep a host copy). */
int cpma_size(const cpma_t* h, uint64_t* out);

/* App. A get_size(): bytes of the structure: L * (leaf_bytes + 16), i.e. the
 * leaf array plus an 8-byte head-index entry, a 4-byte used-byte count and a
 * 4-byte element count per leaf.  Per-batch scratch is not included. */
int cpma_bytes(const cpma_t* h, uint64_t* out);

/* Number of leaves L (host value). */
int cpma_leaves(const cpma_t* h, uint64_t* out);

/* Leaf size in bytes now in use (cfg.leaf_bytes unless leaf_growth > 0). */
int cpma_leaf_bytes(const cpma_t* h, uint64_t* out);

/* Device memory the handle holds now: structure, spare leaf arrays kept for
 * a possible resize, and every scratch buffer (what mem_budget_bytes caps). */
int cpma_mem_held(const cpma_t* h, uint64_t* out);

/* The most device memory the handle has held at any moment (within calls
 * too: an update holds its reservation and, during a resize, both leaf
 * arrays). */
int cpma_mem_peak(const cpma_t* h, uint64_t* out);

/* Change the memory budget of a live handle (0 = no cap).  Memory already
 * held is kept; the cap applies to the next allocations. */
int cpma_set_mem_budget(cpma_t* h, uint64_t bytes);

/* For tests of the bounded wait (no counterpart in the paper): poll_limit
 * replaces the number of polls after which a tile of the batch sort or of
 * the routing stops waiting for its predecessor (0 restores the default,
 * 2^22), and silent_tile >= 0 makes that tile of every sort pass and of the
 * routing skip publishing its counts, so the tiles after it wait until the
 * limit; the update then returns CPMA_ETIMEOUT with the set unchanged.
 * silent_tile < 0 turns it off. */
int cpma_test_sort_stall(cpma_t* h, uint32_t poll_limit, int64_t silent_tile);

/* Copy the layout into caller device buffers: d_data (L * leaf_bytes bytes),
 * d_used (L uint32), d_heads (L uint64; for an empty leaf the head of the next
 * non-empty leaf, or 2^64-1).  Any pointer may be NULL to skip it. */
int cpma_export_layout(const cpma_t* h, uint8_t* d_data, uint32_t* d_used,
                       uint64_t* d_heads, cpma_stream_t stream);

/* Pre-size the scratch that an update of up to max_batch keys (tagged != 0:
 * with request tags) and a range_map of up to max_queries queries use, so
 * that those calls do not allocate: the batch's sort, routing and merge
 * buffers, the redistribution buffers for the whole set plus the batch, and
 * spare leaf arrays for the resize the batch could cause (held until a
 * resize uses them, or until 64 updates in a row could not have resized).
 * Later updates that grow the set past these sizes reserve more before they
 * change anything.  With graphs on (cpma_use_graphs) it also sizes the
 * staging buffer of the padded batch.  Errors: CPMA_EINVAL (null handle,
 * max_batch >= 2^31), CPMA_ENOMEM.  Synchronises the device when an existing
 * buffer has to grow. */
int cpma_reserve(cpma_t* h, uint64_t max_batch, uint64_t max_queries, int tagged,
                 cpma_stream_t stream);

/* Run the front segment of untagged updates of at most max_batch keys --
 * sort, route, the in-place merges and the finalize pass, everything before
 * the update's first host read -- as a CUDA graph (max_batch = 0: never; the
 * default).  A batch of k keys is staged into a library buffer of K keys, K =
 * k rounded up to five significant bits (at least 16, at most k * 17/16 for
 * k >= 16), entry j being key floor(j k / K): each key appears once or twice,
 * in the batch's order.  Repeats of a key change nothing (Sec. 4 batches are
 * sets; App. A counts only keys actually added or removed), so one graph
 * serves every k of a bucket.  Graphs are captured on first use per (K,
 * sorted, insert or delete) and replayed afterwards; a graph is captured
 * again after the leaf arrays are replaced (resize) or a scratch buffer it
 * uses moved; the 8 most recently used are kept.  Sets, counts and layouts
 * are the same with and without graphs.  Per-phase profiling works with
 * graphs: a graph captured while profiling is on carries its phase
 * boundaries as event-record nodes, resolved after every replay.  Graphs pay
 * off for small batches,
 * whose time is launch latency; larger batches do up to 1/8 more sort and
 * route work.  Errors: CPMA_EINVAL (null handle). */
int cpma_use_graphs(cpma_t* h, uint64_t max_batch);

/* Point path (Sec. 4: a batch much smaller than the set is applied as point
 * updates rather than by the batch merge).  An untagged insert of 1 ..
 * max_keys keys (at most 16384; default 16384; 0 = never), or delete of at
 * most min(max_keys, 4096) keys, on a non-empty set of byte-code leaves of
 * at most 512 bytes is first sorted (up to 4096 keys by ranks in the
 * routing kernel, more by the batch sort) and routed (a warp per key), and
 * each touched leaf is checked by a warp: it changes in place when it
 * receives at most 32 keys (4 for a delete), holds codes of at most 4 bytes
 * and, for an insert, at most 512 used bytes before and after, is not
 * emptied by a delete, and stays within its own density bound (Sec. 3
 * bounds at height 0).  The results are staged; if every touched leaf
 * qualifies they are committed and the update is done (two or three kernels
 * after the sort, and one status read); otherwise nothing is written and
 * the update runs the batch algorithm.  Counts, sets and layouts are the
 * same either way: with no leaf pending, emptied or outside its bound the
 * batch algorithm rewrites exactly those leaves, with the same bytes, and
 * starts no redistribution.  The point path's scratch (about 550 bytes per
 * key, held like the rest) is reserved by cpma_reserve for max_batch keys;
 * when it cannot be had within the memory budget the update takes the
 * batch algorithm instead.  Errors: CPMA_EINVAL (null handle). */
int cpma_set_point_max(cpma_t* h, uint64_t max_keys);

/* Updates that took the point path (calls) and those of them that the batch
 * algorithm finished instead (batch) since the handle was created. */
int cpma_point_stats(const cpma_t* h, uint64_t* calls, uint64_t* batch);

/* Graph captures and graph launches of updates on this handle so far. */
int cpma_graph_stats(const cpma_t* h, uint64_t* captures, uint64_t* launches);

/* Device time and kernel-launch counters of the calls on this handle since the
 * last reset, for profiling: *launches = kernels launched by the library. */
int cpma_stats(const cpma_t* h, uint64_t* launches);
int cpma_reset_stats(cpma_t* h);

/* Optional per-phase device timing for profiling.  cpma_profile(h, 1) resets
 * and enables it (synchronising the device); the library then records CUDA
 * events around each phase on the caller's stream, resolved at the host
 * synchronisations the update calls already make, and counts each phase's
 * algorithmic bytes (what the method must read and write).  Phases, in
 * order: 0 sort, 1 route, 2 merge of inserts of a few keys per leaf (the
 * thread-granular kernel), 3 counting (incl. overflow write),
 * 4 redistribute/resize, 5 finish (head fix-up), 6 has, 7 range routing +
 * scan, 8 range scan of the leaves, 9 sum, 10 the other merges (deletes,
 * large slices, fallbacks), 11 merge of other small inserts (the
 * lane-granular kernel).
 * cpma_profile_read synchronises the device and copies up to nphases entries
 * (any pointer may be NULL). */
#define CPMA_NPHASES 12
int cpma_profile(cpma_t* h, int enable);
/* Time only the phases whose bit is set in mask (bit i = phase i; default
 * all): fewer event pairs on the stream and in captured graphs, so the timed
 * work is disturbed less.  Byte counts still cover every phase.  Synchronises
 * the device; graphs captured under another mask are captured again. */
int cpma_profile_mask(cpma_t* h, uint32_t mask);
int cpma_profile_read(cpma_t* h, double* ms, uint64_t* bytes, uint64_t* calls, int nphases);

/* Text for an error code. */
const char* cpma_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* CPMA_H */
