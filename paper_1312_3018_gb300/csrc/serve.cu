// Query server: continuous batching of BFS and SSSP queries on one resident graph.
//
// A worker thread owns all device work. Each pass of its loop:
//  - BFS lanes: when the lane search's superstep in flight has completed, the lanes whose
//    search ended have their levels written out (one kernel for all of them) and are freed;
//    queued BFS queries then take free lanes and the next superstep is issued for every
//    lane holding a search. Queries join and leave between supersteps while the others
//    keep running: the batch is never drained to admit new work.
//  - SSSP slots: every running job whose round has completed issues its next round (or its
//    result copy); a free slot takes the next queued SSSP query. Jobs run on their own
//    streams, so rounds of different queries overlap on the device. Batched jobs (when
//    enabled) take up to sb_job_lanes() queued SSSP queries at once as one multi-lane
//    search that reads each edge once for all of them; the worker starts one when no
//    single-query slot is free or when at least half a batch is waiting, so a lone query
//    keeps the lower latency of a single job.
//  - completions: a query is complete when the event recorded after its result writes has
//    completed; it is then handed to graph_server_poll with its timestamps.
// Nothing blocks on the device: the loop only queries events, and sleeps briefly (or until
// a submission) when nothing progressed.
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"
#include "jobs.cuh"

namespace gg {
namespace {

using Clock = std::chrono::steady_clock;

struct Query {
  uint64_t ticket = 0;
  int kind = 0;
  uint32_t source = 0;
  uint32_t* out = nullptr;
  double t_submit = 0, t_admit = 0;
  int supersteps = 0;
};

// Lanes whose results were issued after one superstep, complete when `ev` has.
struct LaneBatch {
  cudaEvent_t ev = nullptr;
  std::vector<Query> queries;
};

}  // namespace
}  // namespace gg

using namespace gg;

struct graph_server {
  graph* g = nullptr;
  int out_mem = GRAPH_MEM_HOST;
  uint32_t sssp_delta = 0;  // near-far bucket width of the SSSP jobs
  bool sssp_batch = false;  // batched SSSP jobs enabled
  Clock::time_point t0;
  BfsLanes* lanes = nullptr;
  uint32_t nlanes = 0;
  std::vector<SsspJob*> jobs;
  std::vector<SbJob*> bjobs;
  uint64_t bytes_lanes = 0, bytes_job = 0, bytes_bjob = 0, budget = 0;

  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::deque<Query> q_bfs, q_sssp;       // submitted, not yet admitted (under mu)
  std::deque<graph_completion> done;     // completed, not yet polled (under mu)
  uint64_t next_ticket = 1;
  uint64_t submitted = 0, completed = 0;

  // worker-only state
  Query lane_q[GRAPH_BATCH_MAX];
  std::vector<Query> job_q;
  std::vector<char> job_busy;
  std::vector<std::vector<Query>> bjob_q;
  std::vector<char> bjob_busy;
  std::vector<cudaEvent_t> ev_free;
  std::deque<LaneBatch> lane_batches;
  std::atomic<uint32_t> max_lanes_busy{0}, max_slots_busy{0}, max_batch_busy{0};
  std::atomic<uint64_t> sssp_batched{0};
  std::atomic<uint64_t> bfs_steps{0};
  graph_status lane_error = GRAPH_OK;

  double now() const {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  }
};

namespace {

void emit(graph_server* s, const Query& q, int status, double t_done) {
  graph_completion c;
  memset(&c, 0, sizeof(c));
  c.ticket = q.ticket;
  c.kind = q.kind;
  c.status = status;
  c.source = q.source;
  c.supersteps = q.supersteps;
  c.t_submit_ms = q.t_submit;
  c.t_admit_ms = q.t_admit;
  c.t_done_ms = t_done;
  std::lock_guard<std::mutex> lk(s->mu);
  s->done.push_back(c);
  s->completed++;
  s->cv_done.notify_all();
}

void bump(std::atomic<uint32_t>& peak, uint32_t v) {
  uint32_t p = peak.load();
  while (v > p && !peak.compare_exchange_weak(p, v)) {
  }
}

// One pass over the BFS lanes; returns true if anything progressed.
bool step_lanes(graph_server* s, std::deque<Query>& pend) {
  graph* g = s->g;
  bool prog = false;
  if (!s->lanes) {
    while (!pend.empty()) {  // no lanes fit the budget
      emit(s, pend.front(), GRAPH_EINVAL, s->now());
      pend.pop_front();
    }
    return false;
  }
  if (s->lane_error != GRAPH_OK) {
    while (!pend.empty()) {
      emit(s, pend.front(), s->lane_error, s->now());
      pend.pop_front();
    }
    return false;
  }
  if (bfs_lanes_busy(s->lanes)) {
    if (s->ev_free.empty()) return false;
    cudaEvent_t ev = s->ev_free.back();
    uint64_t fin = 0;
    int steps[GRAPH_BATCH_MAX] = {};
    const int r = bfs_lanes_poll(g, s->lanes, &fin, steps, ev);
    if (r < 0) {
      s->lane_error = r;
      for (uint32_t l = 0; l < s->nlanes; ++l)
        if (s->lane_q[l].ticket) {
          emit(s, s->lane_q[l], r, s->now());
          s->lane_q[l] = Query();
        }
      return true;
    }
    if (r == 0) return false;
    prog = true;
    s->bfs_steps++;
    if (fin) {
      s->ev_free.pop_back();
      LaneBatch b;
      b.ev = ev;
      for (uint64_t f = fin; f; f &= f - 1) {
        const int l = __builtin_ctzll(f);
        Query q = s->lane_q[l];
        q.supersteps = steps[l];
        b.queries.push_back(q);
        s->lane_q[l] = Query();
      }
      s->lane_batches.push_back(std::move(b));
    }
  }
  // Between supersteps: admit queued queries on free lanes, then issue the next superstep.
  uint64_t fr = bfs_lanes_free(s->lanes);
  while (fr && !pend.empty()) {
    const int l = __builtin_ctzll(fr);
    fr &= fr - 1;
    Query q = pend.front();
    pend.pop_front();
    const graph_status st = bfs_lanes_admit(s->lanes, l, q.source, q.out, s->out_mem);
    q.t_admit = s->now();
    if (st != GRAPH_OK) {
      emit(s, q, st, s->now());
      continue;
    }
    s->lane_q[l] = q;
    prog = true;
  }
  const uint64_t busy = ~bfs_lanes_free(s->lanes) & (s->nlanes >= 64 ? ~0ull
                                                                      : ((1ull << s->nlanes) - 1));
  bump(s->max_lanes_busy, (uint32_t)__builtin_popcountll(busy));
  if (busy) {
    const graph_status st = bfs_lanes_launch(g, s->lanes);
    if (st != GRAPH_OK) {
      s->lane_error = st;
      for (uint32_t l = 0; l < s->nlanes; ++l)
        if (s->lane_q[l].ticket) {
          emit(s, s->lane_q[l], st, s->now());
          s->lane_q[l] = Query();
        }
    }
  }
  return prog;
}

bool finish_lane_batches(graph_server* s) {
  bool prog = false;
  while (!s->lane_batches.empty()) {
    LaneBatch& b = s->lane_batches.front();
    const cudaError_t q = cudaEventQuery(b.ev);
    if (q == cudaErrorNotReady) break;
    const double t = s->now();
    for (const Query& x : b.queries) emit(s, x, q == cudaSuccess ? GRAPH_OK : GRAPH_ECUDA, t);
    s->ev_free.push_back(b.ev);
    s->lane_batches.pop_front();
    prog = true;
  }
  return prog;
}

bool step_jobs(graph_server* s, std::deque<Query>& pend) {
  graph* g = s->g;
  bool prog = false;
  // completions
  for (size_t i = 0; i < s->jobs.size(); ++i) {
    if (!s->job_busy[i]) continue;
    int rounds = 0;
    const int r = sssp_job_poll(g, s->jobs[i], &rounds);
    if (r != 0) {
      Query q = s->job_q[i];
      q.supersteps = rounds;
      emit(s, q, r == 1 ? GRAPH_OK : r, s->now());
      s->job_busy[i] = 0;
      prog = true;
    }
  }
  for (size_t i = 0; i < s->bjobs.size(); ++i) {
    if (!s->bjob_busy[i]) continue;
    int rounds = 0;
    const int r = sb_job_poll(g, s->bjobs[i], &rounds);
    if (r != 0) {
      const double t = s->now();
      for (Query q : s->bjob_q[i]) {
        q.supersteps = rounds;
        emit(s, q, r == 1 ? GRAPH_OK : r, t);
      }
      s->sssp_batched += s->bjob_q[i].size();
      s->bjob_q[i].clear();
      s->bjob_busy[i] = 0;
      prog = true;
    }
  }
  // admission, oldest first
  const size_t width = sb_job_lanes();
  while (!pend.empty()) {
    int fs = -1, fb = -1;
    for (size_t i = 0; i < s->jobs.size() && fs < 0; ++i)
      if (!s->job_busy[i]) fs = (int)i;
    for (size_t i = 0; i < s->bjobs.size() && fb < 0; ++i)
      if (!s->bjob_busy[i]) fb = (int)i;
    if (fb >= 0 && (fs < 0 || pend.size() >= width / 2)) {
      const size_t k = pend.size() < width ? pend.size() : width;
      std::vector<Query> qs;
      uint32_t src[GRAPH_SSSP_BATCH_MAX];
      uint32_t* outs[GRAPH_SSSP_BATCH_MAX];
      const double t = s->now();
      for (size_t l = 0; l < k; ++l) {
        Query q = pend.front();
        pend.pop_front();
        q.t_admit = t;
        src[l] = q.source;
        outs[l] = q.out;
        qs.push_back(q);
      }
      // plain rounds: a shared near-far threshold staggers the lanes, so a vertex would
      // read its edges again for each lane it waited in, losing the shared reads
      const graph_status st = sb_job_start(g, s->bjobs[fb], src, (uint32_t)k, outs, s->out_mem, 0);
      if (st != GRAPH_OK) {
        for (const Query& q : qs) emit(s, q, st, s->now());
      } else {
        s->bjob_q[fb] = std::move(qs);
        s->bjob_busy[fb] = 1;
      }
      prog = true;
      continue;
    }
    if (fs < 0) break;
    Query q = pend.front();
    pend.pop_front();
    q.t_admit = s->now();
    const graph_status st =
        sssp_job_start(g, s->jobs[fs], q.source, q.out, s->out_mem, s->sssp_delta);
    if (st != GRAPH_OK) {
      emit(s, q, st, s->now());
    } else {
      s->job_q[fs] = q;
      s->job_busy[fs] = 1;
    }
    prog = true;
  }
  if (s->jobs.empty() && s->bjobs.empty())
    while (!pend.empty()) {
      emit(s, pend.front(), GRAPH_EINVAL, s->now());
      pend.pop_front();
    }
  uint32_t busy = 0, bbusy = 0;
  for (char b : s->job_busy) busy += b ? 1 : 0;
  for (char b : s->bjob_busy) bbusy += b ? 1 : 0;
  bump(s->max_slots_busy, busy);
  bump(s->max_batch_busy, bbusy);
  return prog;
}

bool idle(const graph_server* s) {
  if (s->lanes && (bfs_lanes_busy(s->lanes) || bfs_lanes_free(s->lanes) !=
                   (s->nlanes >= 64 ? ~0ull : ((1ull << s->nlanes) - 1))))
    return false;
  if (!s->lane_batches.empty()) return false;
  for (char b : s->job_busy)
    if (b) return false;
  for (char b : s->bjob_busy)
    if (b) return false;
  return true;
}

void run(graph_server* s) {
  cudaSetDevice(s->g->device);
  std::deque<Query> pb, ps;
  for (;;) {
    bool stopping;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      while (!s->q_bfs.empty()) {
        pb.push_back(s->q_bfs.front());
        s->q_bfs.pop_front();
      }
      while (!s->q_sssp.empty()) {
        ps.push_back(s->q_sssp.front());
        s->q_sssp.pop_front();
      }
      stopping = s->stop;
    }
    bool prog = step_lanes(s, pb);
    prog |= finish_lane_batches(s);
    prog |= step_jobs(s, ps);
    if (prog) continue;
    if (stopping && pb.empty() && ps.empty() && idle(s)) break;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_work.wait_for(lk, std::chrono::microseconds(50),
                        [&] { return !s->q_bfs.empty() || !s->q_sssp.empty(); });
  }
}

void destroy_parts(graph_server* s) {
  graph* g = s->g;
  if (s->lanes) bfs_lanes_destroy(g, s->lanes);
  for (SsspJob* j : s->jobs) sssp_job_destroy(g, j);
  for (SbJob* j : s->bjobs) sb_job_destroy(g, j);
  for (cudaEvent_t e : s->ev_free) cudaEventDestroy(e);
  for (LaneBatch& b : s->lane_batches) cudaEventDestroy(b.ev);
  s->lanes = nullptr;
  s->jobs.clear();
  s->bjobs.clear();
  s->ev_free.clear();
  s->lane_batches.clear();
}

graph_status build(graph_server* s, const graph_server_attr& at) {
  graph* g = s->g;
  size_t fr = 0, tot = 0;
  GG_CUDA(cudaMemGetInfo(&fr, &tot));
  s->budget = at.mem_budget ? at.mem_budget : fr / 2;
  uint32_t nl = at.bfs_lanes ? at.bfs_lanes : GRAPH_BATCH_MAX;
  while (nl > 0 && bfs_lanes_bytes(g, nl) > s->budget) nl >>= 1;
  s->nlanes = nl;
  s->bytes_lanes = nl ? bfs_lanes_bytes(g, nl) : 0;
  s->bytes_job = sssp_job_bytes(g);
  s->bytes_bjob = s->sssp_batch ? sb_job_bytes(g) : 0;
  uint64_t slots = 0, bslots = 0;
  if (g->weighted) {
    uint64_t avail = s->budget - s->bytes_lanes;
    if (s->sssp_batch) {
      // batched jobs: up to half of the SSSP share of the budget, at most 8
      bslots = (avail / 2) / s->bytes_bjob;
      if (bslots > 8) bslots = 8;
      avail -= bslots * s->bytes_bjob;
    }
    slots = avail / s->bytes_job;
    // With batched jobs, fewer single-query slots serve a light or moderate load at the
    // lower latency of a single search; under a heavy load the waiting queries gather into
    // batches (16 balanced the two on RMAT-23: 4 gave 5% more peak throughput but 2.6x the
    // median latency at the plain form's capacity).
    const uint64_t cap = at.max_sssp ? at.max_sssp : (s->sssp_batch && bslots ? 16 : 64);
    if (slots > cap) slots = cap;
  }
  if (nl == 0 && slots == 0 && bslots == 0) {
    set_error("mem_budget %llu holds neither a BFS lane set nor an SSSP job",
              (unsigned long long)s->budget);
    return GRAPH_ENOMEM;
  }
  if (nl) GG_TRY(bfs_lanes_create(g, nl, &s->lanes));
  for (uint64_t i = 0; i < slots; ++i) {
    SsspJob* j = nullptr;
    GG_TRY(sssp_job_create(g, &j));
    s->jobs.push_back(j);
  }
  s->job_q.assign(s->jobs.size(), Query());
  s->job_busy.assign(s->jobs.size(), 0);
  for (uint64_t i = 0; i < bslots; ++i) {
    SbJob* j = nullptr;
    GG_TRY(sb_job_create(g, &j));
    s->bjobs.push_back(j);
  }
  s->bjob_q.assign(s->bjobs.size(), std::vector<Query>());
  s->bjob_busy.assign(s->bjobs.size(), 0);
  for (uint32_t i = 0; i < nl + 2; ++i) {
    cudaEvent_t e;
    GG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    s->ev_free.push_back(e);
  }
  return GRAPH_OK;
}

}  // namespace

extern "C" {

graph_status graph_server_create(graph_t* g, const graph_server_attr* attr,
                                 graph_server_t** out) {
  if (!g || !out) {
    set_error("graph or out is NULL");
    return GRAPH_EINVAL;
  }
  *out = nullptr;
  if (!g->partitioned) {
    set_error("graph_partition must run before graph_server_create");
    return GRAPH_ESTATE;
  }
  graph_server_attr at;
  memset(&at, 0, sizeof(at));
  if (attr) at = *attr;
  if ((at.out_mem != GRAPH_MEM_HOST && at.out_mem != GRAPH_MEM_DEVICE) ||
      at.bfs_lanes > GRAPH_BATCH_MAX) {
    set_error("bad server attributes");
    return GRAPH_EINVAL;
  }
  graph_server* s = new (std::nothrow) graph_server();
  if (!s) return GRAPH_ENOMEM;
  s->g = g;
  s->out_mem = at.out_mem;
  s->sssp_delta = at.sssp_delta;
  s->sssp_batch = at.sssp_batch != 0;
  s->t0 = Clock::now();
  graph_status st = build(s, at);
  if (st == GRAPH_OK) {
    try {
      s->worker = std::thread(run, s);
    } catch (...) {
      set_error("cannot start the server thread");
      st = GRAPH_ENOMEM;
    }
  }
  if (st != GRAPH_OK) {
    destroy_parts(s);
    delete s;
    return st;
  }
  *out = s;
  return GRAPH_OK;
}

graph_status graph_server_submit(graph_server_t* s, int kind, uint32_t source, uint32_t* out,
                                 uint64_t* ticket) {
  if (!s || !out || (kind != GRAPH_QUERY_BFS && kind != GRAPH_QUERY_SSSP)) {
    set_error("server or out is NULL, or bad query kind");
    return GRAPH_EINVAL;
  }
  if (source >= s->g->n) {
    set_error("source %u >= n %u", source, s->g->n);
    return GRAPH_EINVAL;
  }
  if ((kind == GRAPH_QUERY_SSSP && s->jobs.empty() && s->bjobs.empty()) ||
      (kind == GRAPH_QUERY_BFS && !s->lanes)) {
    set_error("the server has no %s capacity", kind == GRAPH_QUERY_SSSP ? "SSSP" : "BFS");
    return GRAPH_EINVAL;
  }
  Query q;
  q.kind = kind;
  q.source = source;
  q.out = out;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q.ticket = s->next_ticket++;
    q.t_submit = s->now();
    (kind == GRAPH_QUERY_BFS ? s->q_bfs : s->q_sssp).push_back(q);
    s->submitted++;
  }
  s->cv_work.notify_one();
  if (ticket) *ticket = q.ticket;
  return GRAPH_OK;
}

graph_status graph_server_poll(graph_server_t* s, graph_completion* done, uint32_t cap,
                               uint32_t* count, int wait_ms) {
  if (!s || !count || (cap && !done)) {
    set_error("server, done or count is NULL");
    return GRAPH_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  uint32_t k = 0;
  while (k < cap && !s->done.empty()) {
    done[k++] = s->done.front();
    s->done.pop_front();
  }
  *count = k;
  return GRAPH_OK;
}

graph_status graph_server_info_get(graph_server_t* s, graph_server_info* info) {
  if (!s || !info) {
    set_error("server or info is NULL");
    return GRAPH_EINVAL;
  }
  memset(info, 0, sizeof(*info));
  info->bfs_lanes = s->nlanes;
  info->sssp_slots = (uint32_t)s->jobs.size();
  info->bytes_lanes = s->bytes_lanes;
  info->bytes_per_sssp = s->bytes_job;
  info->mem_budget = s->budget;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    info->submitted = s->submitted;
    info->completed = s->completed;
    info->pending = s->submitted - s->completed;
  }
  info->max_lanes_busy = s->max_lanes_busy.load();
  info->max_slots_busy = s->max_slots_busy.load();
  info->bfs_supersteps = s->bfs_steps.load();
  info->sssp_batch_slots = (uint32_t)s->bjobs.size();
  info->max_batch_busy = s->max_batch_busy.load();
  info->bytes_per_sssp_batch = s->bytes_bjob;
  info->sssp_batched = s->sssp_batched.load();
  return GRAPH_OK;
}

graph_status graph_server_destroy(graph_server_t* s) {
  if (!s) return GRAPH_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  destroy_parts(s);
  delete s;
  return GRAPH_OK;
}

}  // extern "C"
