// Multi-table batches: one launch per phase services many independent tables.
//
// A batch is a list of segments, each an op range on one table.  The host
// (1) grows resizable tables for the inserts their segments may add, planning
// the split launches of all tables as waves (a table joins a wave with the
// splits of one linear-hashing round, so the jobs of a wave touch disjoint
// buckets), (2) writes segment descriptors, per-table views, the list of
// tables the batch touches and the split jobs into one pinned staging buffer
// that a single copy moves to the device, then (3) runs the fixed part --
// bulk kernel over all segments, eviction kernel, stash maintenance and size
// gather of the touched tables -- as direct launches or as one replay of a
// CUDA graph captured on the first call.
//
// Two growth modes:
//  - exact (default): the host waits for each batch, applies the contraction
//    policy to its resizable tables and knows every size exactly;
//  - asynchronous (HIVE_MULTI_ASYNC): the host never waits for a batch it just
//    queued.  Growth is planned from an upper bound of each size: the last
//    gathered size plus the inserts of the batches queued after it.  Tables
//    are not contracted in this mode.  Two batches may be in flight, so the
//    host builds batch k+1 while batch k runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hive.h"
#include "hive_internal.h"

using namespace hive;

namespace {

hive_status mfail(hive_status s, const std::string& msg) {
  set_last_error(msg);
  return s;
}

hive_status mcuda(cudaError_t e, const char* what) {
  set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? HIVE_ERR_OOM : HIVE_ERR_CUDA;
}

#define MCK(call)                                   \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return mcuda(e_, #call); \
  } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// One of the two staging slots: a batch in flight owns one.
struct Slot {
  uint8_t* h_stage = nullptr;
  cudaEvent_t done = nullptr;       // recorded after the batch
  uint64_t seq = 0;                 // batch number, 0 = never used
  bool applied = true;              // its gathered sizes have been taken
  std::vector<uint32_t> touched;    // tables of the batch
  std::vector<uint64_t> ins;        // inserts per touched table (same order)
};

}  // namespace

struct hive_multi {
  std::vector<hive_table*> tables;
  uint32_t max_segs = 0;
  uint64_t max_ops = 0;
  uint32_t max_jobs = 0;
  bool use_graph = false;
  bool async = false;
  bool any_resizable = false;
  Launch L{};
  // staging layout: header | segments | views | touched tables | jobs
  size_t off_segs = 0, off_views = 0, off_touched = 0, off_jobs = 0, stage_bytes = 0;
  uint8_t* d_stage = nullptr;
  Slot slot[2];
  uint64_t seq = 0;
  // overflow list of a batch (entries tagged with their segment)
  uint64_t* ovf_words = nullptr;
  uint32_t* ovf_idx = nullptr;
  uint32_t* ovf_seg = nullptr;
  unsigned* d_count = nullptr;
  // per-table size and stash fill after a batch (entries of touched tables)
  unsigned long long* d_gather = nullptr;
  unsigned long long* h_gather = nullptr;
  std::vector<uint64_t> ub;  // asynchronous mode: upper bound of each size
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::vector<MultiJob> jobs;
  std::vector<uint32_t> wave_begin;
};

namespace {

MultiHdr* hdr_of(uint8_t* base) { return reinterpret_cast<MultiHdr*>(base); }
MultiSeg* segs_of(hive_multi* m, uint8_t* base) {
  return reinterpret_cast<MultiSeg*>(base + m->off_segs);
}
View* views_of(hive_multi* m, uint8_t* base) { return reinterpret_cast<View*>(base + m->off_views); }
uint32_t* touched_of(hive_multi* m, uint8_t* base) {
  return reinterpret_cast<uint32_t*>(base + m->off_touched);
}
MultiJob* jobs_of(hive_multi* m, uint8_t* base) {
  return reinterpret_cast<MultiJob*>(base + m->off_jobs);
}

// HIVE_DEBUG tables: the batch contract holds per table, over all of its
// segments of the batch taken in order.  Copies those keys and op codes to
// the host (waiting on `s`) and checks them with hive_check_batch.
hive_status check_table_segments(const hive_segment* segs, uint32_t n_segs, uint32_t tb,
                                 cudaStream_t s) {
  uint64_t total = 0;
  for (uint32_t i = 0; i < n_segs; ++i)
    if (segs[i].table == tb) total += segs[i].n;
  if (total >= (1ull << 32))
    return mfail(HIVE_ERR_INVALID_ARG, "a table's segments hold 2^32 ops or more");
  std::vector<uint32_t> hk;
  std::vector<uint8_t> ho;
  try {
    hk.resize(total);
    ho.resize(total);
  } catch (const std::bad_alloc&) {
    return mfail(HIVE_ERR_OOM, "batch contract check: host allocation failed");
  }
  uint64_t at = 0;
  for (uint32_t i = 0; i < n_segs; ++i) {
    const hive_segment& g = segs[i];
    if (g.table != tb || !g.n) continue;
    MCK(cudaMemcpyAsync(hk.data() + at, g.keys, g.n * sizeof(uint32_t), cudaMemcpyDefault, s));
    MCK(cudaMemcpyAsync(ho.data() + at, g.ops, g.n, cudaMemcpyDefault, s));
    at += g.n;
  }
  MCK(cudaStreamSynchronize(s));
  uint64_t bad = 0;
  const hive_status st =
      hive_check_batch(ho.data(), HIVE_OP_FIND, hk.data(), total, kReservedKeyMin, &bad);
  if (st != HIVE_OK) set_last_error("table " + std::to_string(tb) + ": " + hive_last_error());
  return st;
}

// The fixed part of a batch; `s` is the caller's stream or the capture stream.
hive_status enqueue_fixed(hive_multi* m, cudaStream_t s) {
  const List ovf{m->ovf_words, m->ovf_idx, m->d_count, m->ovf_seg};
  const uint32_t nt = static_cast<uint32_t>(m->tables.size());
  const MultiHdr* hd = hdr_of(m->d_stage);
  const View* dv = views_of(m, m->d_stage);
  const uint32_t* tc = touched_of(m, m->d_stage);
  MCK(cudaMemsetAsync(m->d_count, 0, sizeof(unsigned), s));
  const int S = static_cast<int>(m->tables[0]->S);
  MCK(launch_multi_ops(S, hd, segs_of(m, m->d_stage), dv, ovf, m->L, s));
  MCK(launch_multi_overflow(S, segs_of(m, m->d_stage), dv, ovf, m->L, s));
  MCK(launch_multi_maint(S, hd, dv, tc, nt, s));
  MCK(launch_multi_gather(hd, dv, tc, nt, m->d_gather, s));
  MCK(cudaMemcpyAsync(m->h_gather, m->d_gather, 2 * sizeof(unsigned long long) * nt,
                      cudaMemcpyDeviceToHost, s));
  return HIVE_OK;
}

// Asynchronous mode: take the sizes gathered by the newest completed batch.
// h_gather holds them, or sizes of a later batch in flight that completed
// meanwhile; either way gathered size + inserts of later batches bounds the
// size from above.
void refresh_bounds(hive_multi* m) {
  Slot* newest = nullptr;
  for (auto& sl : m->slot)
    if (sl.seq && !sl.applied && cudaEventQuery(sl.done) == cudaSuccess)
      if (!newest || sl.seq > newest->seq) newest = &sl;
  cudaGetLastError();
  if (!newest) return;
  Slot* later = nullptr;
  for (auto& sl : m->slot)
    if (sl.seq > newest->seq && !sl.applied) later = &sl;
  for (uint32_t t : newest->touched) m->ub[t] = m->h_gather[2 * t];
  if (later)
    for (size_t j = 0; j < later->touched.size(); ++j) m->ub[later->touched[j]] += later->ins[j];
  for (auto& sl : m->slot)
    if (sl.seq && sl.seq <= newest->seq) sl.applied = true;
}

void release(hive_multi* m) {
  if (m->graph) cudaGraphExecDestroy(m->graph);
  if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
  cudaFree(m->d_stage);
  for (auto& sl : m->slot) {
    if (sl.h_stage) cudaFreeHost(sl.h_stage);
    if (sl.done) cudaEventDestroy(sl.done);
  }
  cudaFree(m->ovf_words);
  cudaFree(m->ovf_idx);
  cudaFree(m->ovf_seg);
  cudaFree(m->d_count);
  cudaFree(m->d_gather);
  if (m->h_gather) cudaFreeHost(m->h_gather);
  delete m;
}

}  // namespace

extern "C" {

hive_status hive_multi_create(hive_table* const* tables, uint32_t n_tables, uint32_t max_segments,
                              uint64_t max_ops, int flags, void* stream, hive_multi** out) {
  (void)stream;
  if (!out) return mfail(HIVE_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  if (!tables || n_tables == 0 || max_segments == 0 || max_ops == 0 || max_ops >= (1ull << 32))
    return mfail(HIVE_ERR_INVALID_ARG,
                 "need tables, n_tables > 0, max_segments > 0 and 0 < max_ops < 2^32");
  if (flags & ~(HIVE_MULTI_GRAPH | HIVE_MULTI_ASYNC))
    return mfail(HIVE_ERR_INVALID_ARG, "unknown flags");
  hive_multi* m = new (std::nothrow) hive_multi();
  if (!m) return mfail(HIVE_ERR_OOM, "host allocation failed");
  for (uint32_t i = 0; i < n_tables; ++i) {
    if (!tables[i]) {
      delete m;
      return mfail(HIVE_ERR_INVALID_ARG, "a table handle is NULL");
    }
    if (tables[i]->S != tables[0]->S) {
      delete m;
      return mfail(HIVE_ERR_INVALID_ARG, "all tables of a group need the same bucket_slots");
    }
    m->tables.push_back(tables[i]);
    m->any_resizable |= tables[i]->cfg.resizable != 0;
    m->ub.push_back(tables[i]->size_host);
  }
  m->max_segs = max_segments;
  m->max_ops = max_ops;
  m->max_jobs = 64u * n_tables;
  m->use_graph = (flags & HIVE_MULTI_GRAPH) != 0;
  m->async = (flags & HIVE_MULTI_ASYNC) != 0;
  m->L = tables[0]->L;
  m->off_segs = align_up(sizeof(MultiHdr), 64);
  m->off_views = align_up(m->off_segs + sizeof(MultiSeg) * max_segments, 64);
  m->off_touched = align_up(m->off_views + sizeof(View) * n_tables, 64);
  m->off_jobs = align_up(m->off_touched + sizeof(uint32_t) * n_tables, 64);
  m->stage_bytes = align_up(m->off_jobs + sizeof(MultiJob) * m->max_jobs, 256);
  cudaError_t e = cudaMalloc(&m->d_stage, m->stage_bytes);
  for (auto& sl : m->slot) {
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_stage, m->stage_bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMalloc(&m->ovf_words, max_ops * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&m->ovf_idx, max_ops * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&m->ovf_seg, max_ops * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_count, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_gather, 2 * sizeof(unsigned long long) * n_tables);
  if (e == cudaSuccess) e = cudaMallocHost(&m->h_gather, 2 * sizeof(unsigned long long) * n_tables);
  if (e == cudaSuccess && m->use_graph)
    e = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    hive_status st = mcuda(e, "hive_multi_create");
    release(m);
    return st;
  }
  *out = m;
  return HIVE_OK;
}

hive_status hive_multi_destroy(hive_multi* m) {
  if (!m) return HIVE_OK;
  cudaDeviceSynchronize();
  release(m);
  return HIVE_OK;
}

hive_status hive_multi_bounds(hive_multi* m, uint64_t* out, uint32_t n_tables) {
  if (!m || !out) return mfail(HIVE_ERR_INVALID_ARG, "group and out must not be NULL");
  if (n_tables > m->tables.size()) return mfail(HIVE_ERR_INVALID_ARG, "n_tables above the group's");
  if (m->async) refresh_bounds(m);
  for (uint32_t t = 0; t < n_tables; ++t) out[t] = m->async ? m->ub[t] : m->tables[t]->size_host;
  return HIVE_OK;
}

hive_status hive_multi_execute(hive_multi* m, const hive_segment* segs, uint32_t n_segs,
                               void* stream) {
  if (!m) return mfail(HIVE_ERR_INVALID_ARG, "multi is NULL");
  if (n_segs > m->max_segs) return mfail(HIVE_ERR_INVALID_ARG, "more segments than max_segments");
  if (n_segs && !segs) return mfail(HIVE_ERR_INVALID_ARG, "segs must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t nt = static_cast<uint32_t>(m->tables.size());
  uint64_t total_ops = 0;
  std::vector<uint64_t> ins(nt, 0);
  std::vector<char> is_touched(nt, 0);
  std::vector<uint32_t> touched;
  for (uint32_t i = 0; i < n_segs; ++i) {
    const hive_segment& g = segs[i];
    if (g.table >= nt) return mfail(HIVE_ERR_INVALID_ARG, "segment table index out of range");
    if (g.reserved0 != 0) return mfail(HIVE_ERR_INVALID_ARG, "segment reserved0 must be 0");
    if (g.n >= (1ull << 32)) return mfail(HIVE_ERR_INVALID_ARG, "segment n must be below 2^32");
    if (g.n && (!g.ops || !g.keys))
      return mfail(HIVE_ERR_INVALID_ARG, "segment ops and keys must not be NULL");
    total_ops += g.n;
    ins[g.table] += std::min<uint64_t>(g.n_insert, g.n);
    if (!is_touched[g.table]) {
      is_touched[g.table] = 1;
      touched.push_back(g.table);
    }
  }
  if (total_ops > m->max_ops) return mfail(HIVE_ERR_INVALID_ARG, "batch larger than max_ops");
  for (uint32_t tb : touched) {
    if (!m->tables[tb]->check_contract) continue;
    hive_status st = check_table_segments(segs, n_segs, tb, s);
    if (st != HIVE_OK) return st;
  }

  // The slot of this batch: wait until the batch that used it two calls ago
  // is done (its staging buffer is then free).
  Slot& sl = m->slot[m->seq & 1];
  MCK(cudaEventSynchronize(sl.done));
  if (m->async) refresh_bounds(m);

  // (1) growth, planned as waves of split jobs
  m->jobs.clear();
  m->wave_begin.clear();
  std::vector<std::vector<MultiJob>> waves;
  for (uint32_t t : touched) {
    hive_table* tb = m->tables[t];
    if (!tb->cfg.resizable || !ins[t]) continue;
    const uint64_t size_now = m->async ? m->ub[t] : tb->size_host;
    uint32_t wave = 0;
    bool any = false;
    while (over_grow(tb, size_now + ins[t], tb->nb) && tb->nb < tb->nb_max) {
      const uint32_t M_before = tb->M;
      SplitPlan pl{};
      if (!plan_split(tb, &pl)) break;
      any = true;
      if (waves.size() <= wave) waves.resize(wave + 1);
      waves[wave].push_back(MultiJob{t, pl.src0, pl.count, pl.half, 0, pl.M, pl.p, 0});
      if (pl.M != M_before) ++wave;  // the next split starts a new round
    }
    if (any && tb->host_ctrl->stash_n) {
      hive_status st = mark_stash_dirty(tb, s);
      if (st != HIVE_OK) return st;
    }
  }
  for (uint32_t t : touched) {  // back the buckets the split waves create
    hive_status st = ensure_committed(m->tables[t], s);
    if (st != HIVE_OK) return st;
  }
  for (auto& w : waves) {
    m->wave_begin.push_back(static_cast<uint32_t>(m->jobs.size()));
    uint32_t pair0 = 0;
    for (auto& j : w) {
      j.pair0 = pair0;
      pair0 += j.count;
      m->jobs.push_back(j);
    }
  }
  if (m->jobs.size() > m->max_jobs)
    return mfail(HIVE_ERR_INVALID_ARG, "batch needs more split launches than the staging holds");

  // (2) staging
  uint8_t* h = sl.h_stage;
  MultiHdr* hd = hdr_of(h);
  MultiSeg* sg = segs_of(m, h);
  uint32_t chunk = 0;
  for (uint32_t i = 0; i < n_segs; ++i) {
    const hive_segment& g = segs[i];
    MultiSeg& d = sg[i];
    std::memset(&d, 0, sizeof(d));
    d.table = g.table;
    d.n = static_cast<uint32_t>(g.n);
    d.chunk0 = chunk;
    d.ops = g.ops;
    d.keys = g.keys;
    d.vals = g.vals;
    d.vals_out = g.vals_out;
    d.status = g.status;
    chunk += static_cast<uint32_t>((g.n + 31) / 32);
  }
  hd->n_segs = n_segs;
  hd->total_chunks = chunk;
  hd->n_tables = nt;
  hd->n_touched = static_cast<uint32_t>(touched.size());
  View* vw = views_of(m, h);
  for (uint32_t t = 0; t < nt; ++t) vw[t] = make_view(m->tables[t]);
  if (!touched.empty())
    std::memcpy(touched_of(m, h), touched.data(), touched.size() * sizeof(uint32_t));
  if (!m->jobs.empty())
    std::memcpy(jobs_of(m, h), m->jobs.data(), m->jobs.size() * sizeof(MultiJob));
  const size_t bytes = m->off_jobs + m->jobs.size() * sizeof(MultiJob);
  MCK(cudaMemcpyAsync(m->d_stage, h, bytes, cudaMemcpyHostToDevice, s));

  // split waves, in order
  for (size_t w = 0; w < m->wave_begin.size(); ++w) {
    const uint32_t b = m->wave_begin[w];
    const uint32_t e = w + 1 < m->wave_begin.size() ? m->wave_begin[w + 1]
                                                    : static_cast<uint32_t>(m->jobs.size());
    const MultiJob& last = m->jobs[e - 1];
    MCK(launch_multi_split(static_cast<int>(m->tables[0]->S), jobs_of(m, m->d_stage) + b, e - b,
                           last.pair0 + last.count, views_of(m, m->d_stage), s));
  }

  // (3) the fixed part
  if (m->use_graph) {
    if (!m->graph) {
      MCK(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
      hive_status st = enqueue_fixed(m, m->cap_stream);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(m->cap_stream, &g);
      if (st != HIVE_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      MCK(e);
      e = cudaGraphInstantiate(&m->graph, g, 0);
      cudaGraphDestroy(g);
      MCK(e);
    }
    MCK(cudaGraphLaunch(m->graph, s));
  } else {
    hive_status st = enqueue_fixed(m, s);
    if (st != HIVE_OK) return st;
  }
  MCK(cudaEventRecord(sl.done, s));
  sl.seq = ++m->seq;
  sl.applied = false;
  sl.touched = touched;
  sl.ins.clear();
  for (uint32_t t : touched) {
    sl.ins.push_back(ins[t]);
    m->ub[t] += ins[t];
  }

  if (m->async) return HIVE_OK;

  // exact mode: take the sizes and contract (one synchronisation for all tables)
  MCK(cudaEventSynchronize(sl.done));
  sl.applied = true;
  for (uint32_t t : touched) {
    hive_table* tb = m->tables[t];
    tb->size_host = m->h_gather[2 * t];
    m->ub[t] = tb->size_host;
    if (tb->cfg.resizable && tb->nb > tb->nb_init && under_shrink(tb, tb->size_host, tb->nb)) {
      hive_status st = contract_table(tb, s);
      if (st != HIVE_OK) return st;
      m->ub[t] = tb->size_host;
    }
  }
  return HIVE_OK;
}

}  // extern "C"
