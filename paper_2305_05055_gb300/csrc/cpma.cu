// C ABI of the CPMA library (declared in include/cpma.h): handle lifecycle,
// argument checks and the dispatch to the update and query launchers.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"

using namespace cpmaimpl;

namespace cpmaimpl {

int check_cuda(cudaError_t e) {
  if (e == cudaSuccess) return CPMA_OK;
  if (e == cudaErrorMemoryAllocation) return CPMA_ENOMEM;
  return CPMA_ECUDA;
}

namespace {
thread_local bool g_capturing = false;
}  // namespace

void set_capturing(bool on) { g_capturing = on; }

int dev_alloc(cpma* h, void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (h->no_alloc || g_capturing) return CPMA_EINTERNAL;
  if (bytes == 0) bytes = 16;
  const uint64_t budget = h->cfg.mem_budget_bytes;
  if (budget && (h->mem_held > budget || bytes > budget - h->mem_held)) return CPMA_ENOMEM;
  if (h->cfg.alloc) {
    *p = h->cfg.alloc(bytes, (cpma_stream_t)st, h->cfg.alloc_ctx);
    if (!*p) return CPMA_ENOMEM;
    if (reinterpret_cast<uintptr_t>(*p) & 15u) {  // vector loads need 16-byte alignment
      h->cfg.free(*p, (cpma_stream_t)st, h->cfg.alloc_ctx);
      *p = nullptr;
      return CPMA_EINVAL;
    }
  } else if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return CPMA_ENOMEM;
  }
  h->mem_held += bytes;
  h->mem_peak = std::max(h->mem_peak, h->mem_held);
  return CPMA_OK;
}

void dev_free(cpma* h, void* p, size_t bytes, cudaStream_t st) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  if (h->cfg.free) h->cfg.free(p, (cpma_stream_t)st, h->cfg.alloc_ctx);
  else cudaFree(p);
  h->mem_held -= bytes;
}

int ensure(cpma* h, Buf& b, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return CPMA_OK;
  if (h->no_alloc || g_capturing) return CPMA_EINTERNAL;
  size_t want = std::max(bytes, b.cap + b.cap / 2);
  want = (want + 255) & ~(size_t)255;
  if (b.p) {
    // growth only: the old contents are dead, but queued kernels may still
    // read them
    if (cudaDeviceSynchronize() != cudaSuccess) return CPMA_ECUDA;
    dev_free(h, b.p, b.cap, st);
    b.p = nullptr;
    b.cap = 0;
  }
  int rc = dev_alloc(h, &b.p, want, st);
  if (rc == CPMA_ENOMEM && want > bytes) {  // without the growth slack
    want = (bytes + 255) & ~(size_t)255;
    rc = dev_alloc(h, &b.p, want, st);
  }
  if (rc != CPMA_OK) return rc;
  b.cap = want;
  return CPMA_OK;
}

void release(cpma* h, Buf& b) {
  dev_free(h, b.p, b.cap, nullptr);
  b.p = nullptr;
  b.cap = 0;
}

// The leaf bytes get kLeafPad bytes of padding: a thread rewriting a chunk
// reads whole 4-byte words, which may reach up to 3 bytes past the last leaf.
constexpr uint64_t kLeafPad = 16;

int alloc_arrays(cpma* h, uint64_t leaves, uint64_t data_bytes, Arrays* a, cudaStream_t st) {
  *a = Arrays{};
  int rc = dev_alloc(h, (void**)&a->data, data_bytes + kLeafPad, st);
  if (rc == CPMA_OK) rc = dev_alloc(h, (void**)&a->used, leaves * 4, st);
  if (rc == CPMA_OK) rc = dev_alloc(h, (void**)&a->cnt, leaves * 4, st);
  if (rc == CPMA_OK) rc = dev_alloc(h, (void**)&a->heads, (leaves + 1) * 8, st);
  a->cap_leaves = leaves;
  a->cap_bytes = data_bytes;
  if (rc != CPMA_OK) free_arrays(h, a);
  return rc;
}

void free_arrays(cpma* h, Arrays* a) {
  if (a->data) dev_free(h, a->data, a->cap_bytes + kLeafPad, nullptr);
  dev_free(h, a->used, a->cap_leaves * 4, nullptr);
  dev_free(h, a->cnt, a->cap_leaves * 4, nullptr);
  dev_free(h, a->heads, (a->cap_leaves + 1) * 8, nullptr);
  *a = Arrays{};
}

int sync_status(cpma* h, cudaStream_t st) {
  CPMA_CUDA(cudaMemcpyAsync(h->h_status, h->d_status, sizeof(Status), cudaMemcpyDeviceToHost, st));
  CPMA_CUDA(cudaStreamSynchronize(st));
  prof_resolve(h);
  return CPMA_OK;
}

namespace {
cudaEvent_t take_event(Prof& p) {
  if (p.npool > 0) return p.pool[--p.npool];
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return e;
}
void give_event(Prof& p, cudaEvent_t e) {
  if (!e) return;
  if (p.npool == p.pool_cap) {
    int nc = p.pool_cap ? 2 * p.pool_cap : 64;
    cudaEvent_t* np = new cudaEvent_t[nc];
    for (int i = 0; i < p.npool; i++) np[i] = p.pool[i];
    delete[] p.pool;
    p.pool = np;
    p.pool_cap = nc;
  }
  p.pool[p.npool++] = e;
}
}  // namespace

namespace {
void rec_begin(Prof& p, Prof::Rec& r, int phase, cudaStream_t st) {
  r.phase = phase;
  if (p.capturing) {
    // events of the graph being captured: recorded by every replay
    r.a = r.b = nullptr;
    r.pooled = false;
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaEventRecordWithFlags(r.a, st, cudaEventRecordExternal);
    return;
  }
  r.pooled = true;
  r.a = take_event(p);
  r.b = take_event(p);
  if (r.a) cudaEventRecord(r.a, st);
}

void rec_end(Prof& p, Prof::Rec& r, cudaStream_t st) {
  if (p.capturing) {
    if (r.b) cudaEventRecordWithFlags(r.b, st, cudaEventRecordExternal);
    if (p.ncap == p.cap_max) {
      int nc = p.cap_max ? 2 * p.cap_max : 16;
      Prof::Rec* np = new Prof::Rec[nc];
      for (int i = 0; i < p.ncap; i++) np[i] = p.cap_recs[i];
      delete[] p.cap_recs;
      p.cap_recs = np;
      p.cap_max = nc;
    }
    p.cap_recs[p.ncap++] = r;
    r.phase = -1;
    return;
  }
  if (r.b) cudaEventRecord(r.b, st);
  if (p.npending == p.cap) {
    int nc = p.cap ? 2 * p.cap : 64;
    Prof::Rec* np = new Prof::Rec[nc];
    for (int i = 0; i < p.npending; i++) np[i] = p.pending[i];
    delete[] p.pending;
    p.pending = np;
    p.cap = nc;
  }
  p.pending[p.npending++] = r;
  r.phase = -1;
}
}  // namespace

void prof_begin(const cpma* hc, int phase, cudaStream_t st) {
  cpma* h = const_cast<cpma*>(hc);
  Prof& p = h->prof;
  if (!p.on) return;
  if (p.open_rec.phase >= 0) prof_end(h, st);
  if (!((p.mask >> phase) & 1u)) return;
  rec_begin(p, p.open_rec, phase, st);
}

void prof_end(const cpma* hc, cudaStream_t st) {
  cpma* h = const_cast<cpma*>(hc);
  Prof& p = h->prof;
  if (!p.on || p.open_rec.phase < 0) return;
  rec_end(p, p.open_rec, st);
}

void prof_begin_side(const cpma* hc, int phase, cudaStream_t st) {
  cpma* h = const_cast<cpma*>(hc);
  Prof& p = h->prof;
  if (!p.on) return;
  if (p.side_rec.phase >= 0) rec_end(p, p.side_rec, st);
  if (!((p.mask >> phase) & 1u)) return;
  rec_begin(p, p.side_rec, phase, st);
}

void prof_end_side(const cpma* hc, cudaStream_t st) {
  cpma* h = const_cast<cpma*>(hc);
  Prof& p = h->prof;
  if (!p.on || p.side_rec.phase < 0) return;
  rec_end(p, p.side_rec, st);
}

void prof_resolve(const cpma* hc) {
  cpma* h = const_cast<cpma*>(hc);
  Prof& p = h->prof;
  for (int i = 0; i < p.npending; i++) {
    Prof::Rec& r = p.pending[i];
    float ms = 0.f;
    if (r.a && r.b && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      p.ms[r.phase] += ms;
      p.calls[r.phase]++;
    } else {
      cudaGetLastError();
    }
    if (r.pooled) {
      give_event(p, r.a);
      give_event(p, r.b);
    }
  }
  p.npending = 0;
}

void prof_push(const cpma* hc, const Prof::Rec* recs, int n, const unsigned long long* host_bytes) {
  cpma* h = const_cast<cpma*>(hc);
  Prof& p = h->prof;
  for (int i = 0; i < n; i++) {
    if (p.npending == p.cap) {
      int nc = p.cap ? 2 * p.cap : 64;
      Prof::Rec* np = new Prof::Rec[nc];
      for (int q = 0; q < p.npending; q++) np[q] = p.pending[q];
      delete[] p.pending;
      p.pending = np;
      p.cap = nc;
    }
    p.pending[p.npending++] = recs[i];
  }
  for (int i = 0; i < PH_N; i++) p.host_bytes[i] += host_bytes[i];
}

}  // namespace cpmaimpl

namespace {

int validate(const cpma_config& c) {
  if (c.leaf_bytes < 256 || c.leaf_bytes > 2048 || c.leaf_bytes % 16) return CPMA_EINVAL;
  if (!(c.rho_leaf <= c.rho_root && c.rho_root < c.tau_root && c.tau_root <= c.tau_leaf &&
        c.tau_leaf < 1000))
    return CPMA_EINVAL;
  if ((uint64_t)(1000 - c.tau_leaf) * c.leaf_bytes < 20000) return CPMA_EINVAL;
  if (c.grow_den == 0 || c.grow_num <= c.grow_den) return CPMA_EINVAL;
  if (c.codec > 1) return CPMA_EINVAL;
  if ((uint64_t)c.build_pm * c.leaf_bytes <= 8000 || c.build_pm > c.tau_root) return CPMA_EINVAL;
  if (c.leaf_growth > 2048 || c.reserved) return CPMA_EINVAL;
  if ((c.alloc == nullptr) != (c.free == nullptr)) return CPMA_EINVAL;
  return CPMA_OK;
}

void release_all(cpma* h) {
  Scratch& s = h->s;
  for (Buf* b : {&s.keysA, &s.keysB, &s.valsA, &s.valsB, &s.hist, &s.flags, &s.flags_scan, &s.leaf_of,
                 &s.chunk_begin, &s.chunk_leaf, &s.chunk_tid, &s.chunk_cnt, &s.chunk_off,
                 &s.T_leaf, &s.T_begin, &s.T_first_chunk, &s.T_oldcnt, &s.T_oldused, &s.T_newcnt,
                 &s.T_newbytes, &s.T_state, &s.viol, &s.list_lane, &s.list_v1, &s.list_gen, &s.list_pend, &s.point_stage, &s.point_rec, &s.cand,
                 &s.wins, &s.bits, &s.prefix, &s.E, &s.cost, &s.C, &s.srccnt, &s.srcoff, &s.dstart,
                 &s.win_src, &s.win_dst, &s.win_leaf_off, &s.win_elem_off, &s.win_dst_off,
                 &s.partials, &s.partials_q, &s.q_first, &s.q_items, &s.q_off, &s.stage, &s.q_lo,
                 &s.q_hi, &s.q_rank, &s.fh})
    release(h, *b);
  prof_resolve(h);  // before the graphs (and their events) go
  graph_cache_free(h);
  Arrays cur;
  cur.data = h->data;
  cur.used = h->used;
  cur.cnt = h->cnt;
  cur.heads = h->heads;
  cur.cap_leaves = h->cap_leaves;
  cur.cap_bytes = h->cap_bytes;
  free_arrays(h, &cur);
  free_arrays(h, &h->spare);
  dev_free(h, h->d_status, sizeof(Status), nullptr);
  if (h->h_status) cudaFreeHost(h->h_status);
  prof_resolve(h);
  for (int i = 0; i < h->prof.npool; i++) cudaEventDestroy(h->prof.pool[i]);
  delete[] h->prof.pool;
  delete[] h->prof.pending;
  delete[] h->prof.cap_recs;
  h->prof.cap_recs = nullptr;
  h->prof.ncap = h->prof.cap_max = 0;
  h->prof.pool = nullptr;
  h->prof.pending = nullptr;
  h->prof.npool = h->prof.pool_cap = h->prof.npending = h->prof.cap = 0;
  dev_free(h, h->prof.d_bytes, sizeof(unsigned long long) * PH_N, nullptr);
  h->prof.d_bytes = nullptr;
  h->data = nullptr;
  h->used = nullptr;
  h->cnt = nullptr;
  h->heads = nullptr;
  h->cap_leaves = h->cap_bytes = 0;
  h->d_status = nullptr;
  h->h_status = nullptr;
}

int new_handle(const cpma_config* cfg, cpma** out) {
  cpma_config c;
  cpma_default_config(&c);
  if (cfg) c = *cfg;
  CPMA_TRY(validate(c));
  cpma* h = new (std::nothrow) cpma();
  if (!h) return CPMA_ENOMEM;
  h->cfg = c;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { delete h; return CPMA_ECUDA; }
  h->device = dev;
  if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete h;
    return CPMA_ECUDA;
  }
  h->lb_min = c.leaf_bytes;
  int rc = dev_alloc(h, (void**)&h->d_status, sizeof(Status), nullptr);
  if (rc != CPMA_OK) {
    delete h;
    return rc;
  }
  if (cudaMallocHost(&h->h_status, sizeof(Status)) != cudaSuccess) {
    cudaGetLastError();
    release_all(h);
    delete h;
    return CPMA_ENOMEM;
  }
  if (cudaMemset(h->d_status, 0, sizeof(Status)) != cudaSuccess) {
    release_all(h);
    delete h;
    return CPMA_ECUDA;
  }
  *out = h;
  return CPMA_OK;
}

}  // namespace

extern "C" {

void cpma_default_config(cpma_config* c) {
  c->leaf_bytes = 512;
  c->tau_leaf = 900;
  c->tau_root = 700;
  c->rho_leaf = 100;
  c->rho_root = 300;
  c->grow_num = 6;
  c->grow_den = 5;
  c->build_pm = 500;
  c->rebuild_pm = 0;
  c->codec = 0;
  c->leaf_growth = 0;
  c->reserved = 0;
  c->alloc = nullptr;
  c->free = nullptr;
  c->alloc_ctx = nullptr;
  c->mem_budget_bytes = 0;
}

int cpma_create(cpma_t** out, const cpma_config* cfg, const uint64_t* d_keys, uint64_t n,
                cpma_stream_t stream) {
  if (!out || (n && !d_keys)) return CPMA_EINVAL;
  *out = nullptr;
  cpma* h = nullptr;
  CPMA_TRY(new_handle(cfg, &h));
  cudaStream_t st = (cudaStream_t)stream;
  int rc = CPMA_OK;
  do {
    rc = ensure(h, h->s.E, (n + 1) * 8);
    if (rc) break;
    uint64_t nu = 0;
    if (n) {
      const uint64_t* sorted = nullptr;
      rc = sort_keys(h, d_keys, n, &sorted, st);
      if (rc) break;
      rc = unique_keys(h, sorted, n, (uint64_t*)h->s.E.p, st);
      if (rc) break;
      rc = sync_status(h, st);
      if (rc) break;
      nu = h->h_status->nunique;
    }
    rc = build_from_sorted_unique(h, (const uint64_t*)h->s.E.p, nu, st);
  } while (0);
  if (rc != CPMA_OK) {
    cudaStreamSynchronize(st);
    release_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return CPMA_OK;
}

int cpma_destroy(cpma_t* h) {
  if (!h) return CPMA_EINVAL;
  cudaDeviceSynchronize();
  release_all(h);
  delete h;
  return CPMA_OK;
}

int cpma_clone(const cpma_t* src, cpma_t** out, cpma_stream_t stream) {
  if (!src || !out) return CPMA_EINVAL;
  *out = nullptr;
  cpma* h = nullptr;
  CPMA_TRY(new_handle(&src->cfg, &h));
  h->lb_min = src->lb_min;
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t L = src->L, LB = src->cfg.leaf_bytes;
  Arrays a;
  int rc = alloc_arrays(h, L, L * LB, &a, st);
  if (rc != CPMA_OK) {
    release_all(h);
    delete h;
    return rc;
  }
  h->data = a.data;
  h->used = a.used;
  h->cnt = a.cnt;
  h->heads = a.heads;
  h->cap_leaves = a.cap_leaves;
  h->cap_bytes = a.cap_bytes;
  rc |= check_cuda(cudaMemcpyAsync(h->data, src->data, L * LB, cudaMemcpyDeviceToDevice, st));
  rc |= check_cuda(cudaMemcpyAsync(h->used, src->used, L * 4, cudaMemcpyDeviceToDevice, st));
  rc |= check_cuda(cudaMemcpyAsync(h->cnt, src->cnt, L * 4, cudaMemcpyDeviceToDevice, st));
  rc |= check_cuda(cudaMemcpyAsync(h->heads, src->heads, (L + 1) * 8, cudaMemcpyDeviceToDevice,
                                   st));
  // the empty-leaf count and the byte total (the two fields after it)
  rc |= check_cuda(cudaMemcpyAsync(&h->d_status->empties, &src->d_status->empties, 16,
                                   cudaMemcpyDeviceToDevice, st));
  if (rc != CPMA_OK) {
    cudaStreamSynchronize(st);
    release_all(h);
    delete h;
    return CPMA_ECUDA;
  }
  h->L = L;
  h->n = src->n;
  h->may_have_empty = src->may_have_empty;
  h->t_known = src->t_known;
  h->t_slack = src->t_slack;
  *out = h;
  return CPMA_OK;
}

int cpma_insert_batch(cpma_t* h, const uint64_t* d_keys, uint64_t k, int sorted,
                      uint64_t* d_added, cpma_stream_t stream) {
  if (!h || (k && !d_keys)) return CPMA_EINVAL;
  return run_update(h, d_keys, k, sorted, 0, d_added, (cudaStream_t)stream);
}

int cpma_delete_batch(cpma_t* h, const uint64_t* d_keys, uint64_t k, int sorted,
                      uint64_t* d_removed, cpma_stream_t stream) {
  if (!h || (k && !d_keys)) return CPMA_EINVAL;
  return run_update(h, d_keys, k, sorted, 1, d_removed, (cudaStream_t)stream);
}

int cpma_insert_batch_tagged(cpma_t* h, const uint64_t* d_keys, const uint32_t* d_tags,
                             uint64_t k, int sorted, uint64_t ntags, uint64_t* d_counts,
                             cpma_stream_t stream) {
  if (!h || (k && (!d_keys || !d_tags)) || !d_counts || ntags == 0) return CPMA_EINVAL;
  return run_update(h, d_keys, k, sorted, 0, nullptr, (cudaStream_t)stream, d_tags, d_counts,
                    ntags);
}

int cpma_delete_batch_tagged(cpma_t* h, const uint64_t* d_keys, const uint32_t* d_tags,
                             uint64_t k, int sorted, uint64_t ntags, uint64_t* d_counts,
                             cpma_stream_t stream) {
  if (!h || (k && (!d_keys || !d_tags)) || !d_counts || ntags == 0) return CPMA_EINVAL;
  return run_update(h, d_keys, k, sorted, 1, nullptr, (cudaStream_t)stream, d_tags, d_counts,
                    ntags);
}

int cpma_sort_batch(cpma_t* h, const uint64_t* d_keys, const uint32_t* d_tags, uint64_t k,
                    uint64_t* d_keys_out, uint32_t* d_tags_out, cpma_stream_t stream) {
  if (!h || (k && (!d_keys || !d_keys_out)) || (d_tags && !d_tags_out)) return CPMA_EINVAL;
  if (k == 0) return CPMA_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t* u = nullptr;
  const uint32_t* ut = nullptr;
  if (d_tags) CPMA_TRY(sort_pairs(h, d_keys, d_tags, k, &u, &ut, st));
  else CPMA_TRY(sort_keys(h, d_keys, k, &u, st));
  CPMA_CUDA(cudaMemcpyAsync(d_keys_out, u, k * 8, cudaMemcpyDeviceToDevice, st));
  if (d_tags) CPMA_CUDA(cudaMemcpyAsync(d_tags_out, ut, k * 4, cudaMemcpyDeviceToDevice, st));
  return CPMA_OK;
}

int cpma_has_batch(const cpma_t* h, const uint64_t* d_keys, uint64_t q, uint8_t* d_out,
                   cpma_stream_t stream) {
  if (!h || (q && (!d_keys || !d_out))) return CPMA_EINVAL;
  return run_has(h, d_keys, q, d_out, (cudaStream_t)stream);
}

int cpma_range_map(const cpma_t* h, const uint64_t* d_lo, const uint64_t* d_hi, uint64_t q,
                   uint64_t* d_sum, uint64_t* d_count, cpma_stream_t stream) {
  if (!h || (q && (!d_lo || !d_hi || !d_sum || !d_count))) return CPMA_EINVAL;
  return run_range(h, d_lo, d_hi, q, d_sum, d_count, (cudaStream_t)stream);
}

int cpma_range_map_length(const cpma_t* h, const uint64_t* d_start, const uint64_t* d_length,
                          uint64_t q, uint64_t* d_sum, uint64_t* d_count, cpma_stream_t stream) {
  if (!h || (q && (!d_start || !d_length || !d_sum || !d_count))) return CPMA_EINVAL;
  return run_range_length(h, d_start, d_length, q, d_sum, d_count, (cudaStream_t)stream);
}

int cpma_range_extract(const cpma_t* h, const uint64_t* d_lo, const uint64_t* d_hi, uint64_t q,
                       uint64_t* d_offsets, uint64_t* d_out, uint64_t out_cap,
                       cpma_stream_t stream) {
  if (!h || !d_offsets || (q && (!d_lo || !d_hi))) return CPMA_EINVAL;
  return run_range_extract(h, d_lo, d_hi, q, d_offsets, d_out, out_cap, (cudaStream_t)stream);
}

int cpma_range_reduce(const cpma_t* h, const uint64_t* d_lo, const uint64_t* d_hi, uint64_t q,
                      int op, uint64_t mask, uint64_t value, uint64_t* d_out, uint64_t* d_count,
                      cpma_stream_t stream) {
  if (!h || (q && (!d_lo || !d_hi || !d_out || !d_count))) return CPMA_EINVAL;
  if (op < CPMA_OP_SUM || op > CPMA_OP_XOR) return CPMA_EINVAL;
  return run_range_reduce(h, d_lo, d_hi, q, op, mask, value, d_out, d_count,
                          (cudaStream_t)stream);
}

int cpma_range_map_noalloc(const cpma_t* h, const uint64_t* d_lo, const uint64_t* d_hi,
                           uint64_t q, uint64_t* d_sum, uint64_t* d_count, cpma_stream_t stream) {
  if (!h || (q && (!d_lo || !d_hi || !d_sum || !d_count))) return CPMA_EINVAL;
  return run_range_noalloc(h, d_lo, d_hi, q, d_sum, d_count, (cudaStream_t)stream);
}

int cpma_sum(const cpma_t* h, uint64_t* d_sum, uint64_t* d_count, cpma_stream_t stream) {
  if (!h || !d_sum) return CPMA_EINVAL;
  return run_sum(h, d_sum, d_count, (cudaStream_t)stream);
}

int cpma_size(const cpma_t* h, uint64_t* out) {
  if (!h || !out) return CPMA_EINVAL;
  *out = h->n;
  return CPMA_OK;
}

int cpma_bytes(const cpma_t* h, uint64_t* out) {
  if (!h || !out) return CPMA_EINVAL;
  *out = h->L * ((uint64_t)h->cfg.leaf_bytes + 16);
  return CPMA_OK;
}

int cpma_leaves(const cpma_t* h, uint64_t* out) {
  if (!h || !out) return CPMA_EINVAL;
  *out = h->L;
  return CPMA_OK;
}

int cpma_leaf_bytes(const cpma_t* h, uint64_t* out) {
  if (!h || !out) return CPMA_EINVAL;
  *out = h->cfg.leaf_bytes;
  return CPMA_OK;
}

int cpma_mem_held(const cpma_t* h, uint64_t* out) {
  if (!h || !out) return CPMA_EINVAL;
  *out = h->mem_held;
  return CPMA_OK;
}

int cpma_mem_peak(const cpma_t* h, uint64_t* out) {
  if (!h || !out) return CPMA_EINVAL;
  *out = h->mem_peak;
  return CPMA_OK;
}

int cpma_set_mem_budget(cpma_t* h, uint64_t bytes) {
  if (!h) return CPMA_EINVAL;
  h->cfg.mem_budget_bytes = bytes;
  return CPMA_OK;
}

int cpma_test_sort_stall(cpma_t* h, uint32_t poll_limit, int64_t silent_tile) {
  if (!h) return CPMA_EINVAL;
  h->sort_poll_limit = poll_limit;
  h->sort_silent_tile = silent_tile < 0 ? -1 : silent_tile;
  return CPMA_OK;
}

int cpma_export_layout(const cpma_t* h, uint8_t* d_data, uint32_t* d_used, uint64_t* d_heads,
                       cpma_stream_t stream) {
  if (!h) return CPMA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t L = h->L;
  if (d_data)
    CPMA_CUDA(cudaMemcpyAsync(d_data, h->data, L * h->cfg.leaf_bytes, cudaMemcpyDeviceToDevice, st));
  if (d_used) CPMA_CUDA(cudaMemcpyAsync(d_used, h->used, L * 4, cudaMemcpyDeviceToDevice, st));
  if (d_heads) CPMA_CUDA(cudaMemcpyAsync(d_heads, h->heads, L * 8, cudaMemcpyDeviceToDevice, st));
  return CPMA_OK;
}

int cpma_stats(const cpma_t* h, uint64_t* launches) {
  if (!h || !launches) return CPMA_EINVAL;
  *launches = h->launches;
  return CPMA_OK;
}

int cpma_reserve(cpma_t* h, uint64_t max_batch, uint64_t max_queries, int tagged,
                 cpma_stream_t stream) {
  if (!h) return CPMA_EINVAL;
  CPMA_TRY(reserve(h, max_batch, tagged, (cudaStream_t)stream));
  if (max_queries) {
    Scratch& s = h->s;
    CPMA_TRY(ensure(h, s.q_first, max_queries * 8));
    CPMA_TRY(ensure(h, s.q_items, max_queries * 8));
    CPMA_TRY(ensure(h, s.q_off, (max_queries + 1) * 8));
    CPMA_TRY(ensure(h, s.partials_q, (size_t)(2 * h->num_sms + 2) * 8));
  }
  return CPMA_OK;
}

int cpma_use_graphs(cpma_t* h, uint64_t max_batch) {
  if (!h) return CPMA_EINVAL;
  h->graph_max_batch = max_batch;
  return CPMA_OK;
}

int cpma_set_point_max(cpma_t* h, uint64_t max_keys) {
  if (!h) return CPMA_EINVAL;
  h->point_max = max_keys;
  return CPMA_OK;
}

int cpma_point_stats(const cpma_t* h, uint64_t* calls, uint64_t* batch) {
  if (!h) return CPMA_EINVAL;
  if (calls) *calls = h->point_calls;
  if (batch) *batch = h->point_batch;
  return CPMA_OK;
}

int cpma_graph_stats(const cpma_t* h, uint64_t* captures, uint64_t* launches) {
  if (!h) return CPMA_EINVAL;
  if (captures) *captures = h->graph_captures;
  if (launches) *launches = h->graph_launches;
  return CPMA_OK;
}

int cpma_reset_stats(cpma_t* h) {
  if (!h) return CPMA_EINVAL;
  h->launches = 0;
  return CPMA_OK;
}

int cpma_profile(cpma_t* h, int enable) {
  if (!h) return CPMA_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return CPMA_ECUDA;
  prof_resolve(h);
  Prof& p = h->prof;
  if (!p.d_bytes) CPMA_TRY(dev_alloc(h, (void**)&p.d_bytes, sizeof(unsigned long long) * PH_N, nullptr));
  CPMA_CUDA(cudaMemset(p.d_bytes, 0, sizeof(unsigned long long) * PH_N));
  for (int i = 0; i < PH_N; i++) { p.ms[i] = 0; p.calls[i] = 0; p.host_bytes[i] = 0; }
  p.on = enable != 0;
  return CPMA_OK;
}

int cpma_profile_mask(cpma_t* h, uint32_t mask) {
  if (!h) return CPMA_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return CPMA_ECUDA;
  prof_resolve(h);
  h->prof.mask = mask;
  return CPMA_OK;
}

int cpma_profile_read(cpma_t* h, double* ms, uint64_t* bytes, uint64_t* calls, int nphases) {
  if (!h || nphases < 0) return CPMA_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return CPMA_ECUDA;
  prof_resolve(h);
  unsigned long long db[PH_N] = {0};
  if (h->prof.d_bytes)
    CPMA_CUDA(cudaMemcpy(db, h->prof.d_bytes, sizeof(db), cudaMemcpyDeviceToHost));
  for (int i = 0; i < nphases && i < PH_N; i++) {
    if (ms) ms[i] = h->prof.ms[i];
    if (bytes) bytes[i] = db[i] + h->prof.host_bytes[i];
    if (calls) calls[i] = h->prof.calls[i];
  }
  return CPMA_OK;
}

const char* cpma_strerror(int code) {
  switch (code) {
    case CPMA_OK: return "ok";
    case CPMA_EINVAL: return "invalid argument or configuration";
    case CPMA_ENOMEM: return "out of device or host memory";
    case CPMA_ECUDA: return "CUDA error";
    case CPMA_EINTERNAL: return "device-side consistency check failed";
    case CPMA_ETIMEOUT: return "a bounded device-side wait gave up";
    default: return "unknown error";
  }
}

}  // extern "C"
