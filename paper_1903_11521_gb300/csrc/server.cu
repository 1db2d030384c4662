// Serving runtime: independent ADER-DG solves submitted at any time, admitted while their
// device memory fits an HBM budget, and advanced together (continuous batching).
//
// Two threads share the work:
//  * the worker only enqueues device work: each "tick" advances every active solve by one
//    step, with ONE local and ONE neighbour kernel launch per polynomial degree over the
//    tiles of all active solves of that degree (a per-CTA tile table points each CTA at
//    its solve's buffers, tile index and time step), the degrees on separate streams.  It
//    never waits for the device except to keep at most kAhead ticks in flight per degree
//    stream.  A solve enters the tick set once its set-up is enqueued (the degree stream
//    waits for the set-up's event on the device); after its last step the worker records
//    a completion event and hands it to the second thread.
//  * the lifecycle thread admits requests (solver creation with stream-ordered memory on
//    its own stream, DOF upload, per-element set-up kernel) and finishes solves (waits
//    for the completion event, copies the DOFs out, frees the solver on its stream), so
//    neither admission nor copy-out stalls the ticks of other solves.
// Admission: in arrival order while the budget allows; when the head request does not
// fit, later requests that fit may go ahead of it for up to kBackfillS seconds after it
// reached the head (after that, memory is reserved for it).  Every tile is computed
// exactly as in a solve alone (no data crosses solve boundaries), so a result does not
// depend on the mix it was computed in.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.h"
#include "solver_internal.h"
#include "tables.h"

using namespace yt;

namespace {

constexpr int kAhead = 2;              // ticks in flight per degree stream
constexpr int kSlots = kAhead + 1;     // tile-table buffers per degree
constexpr double kBackfillS = 0.5;

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum ReqState { kPending = 0, kAdmitting = 1, kReady = 2, kActive = 3, kFinishing = 4, kDone = 5, kFailed = 6 };

struct Request {
  int64_t id = 0;
  int order = 0;
  int64_t E = 0;
  double dt = 0.0;
  int steps = 0, enqueued_steps = 0;
  std::vector<double> material, jacobian, dofs, result;
  std::vector<int32_t> neighbours;
  std::vector<int8_t> faces, orient;
  size_t bytes = 0;
  int state = kPending;
  yt_status status = YT_OK;
  std::string error;
  double t_submit = 0, t_admit = 0, t_done = 0;
  yt_solver* solver = nullptr;
  cudaEvent_t ready = nullptr, done = nullptr;
};

// Tile tables of one degree: kSlots pinned host / device buffer pairs, each with the
// event of the last tick that read it.
struct Tables {
  TileRef* host[kSlots] = {};
  TileRef* dev[kSlots] = {};
  size_t cap[kSlots] = {};
  cudaEvent_t used[kSlots] = {};
  int cur = -1;
  size_t n = 0;
};

}  // namespace

struct yt_server {
  size_t budget = 0, in_use = 0, peak = 0;
  yt_precision prec = YT_F32;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_life, cv_done;
  bool stop = false;
  std::deque<Request*> pending;
  std::vector<Request*> ready, active, finishing;
  int admitting = 0;
  double head_since = 0.0;          // when the current head request reached the head
  int64_t head_id = 0;
  std::map<int64_t, std::unique_ptr<Request>> requests;
  int64_t next_id = 1;
  int64_t completed = 0, failed = 0, ticks = 0, max_active = 0;
  double element_updates = 0.0;
  std::thread worker, lifecycle;
  cudaStream_t streams[8] = {};     // per degree (worker)
  cudaStream_t life = nullptr;      // admissions and copy-out (lifecycle thread)
  cudaEvent_t tick_ev[8][kAhead] = {};
  int64_t stream_ticks[8] = {};
  Tables tables[8];
  bool dirty[8] = {};
  std::string fatal;            // set when a tick failed: the server then fails every request
  int64_t fail_at_tick = -1;    // diagnostics: a tick number treated as failed (host side)
  ~yt_server();
};

namespace {

// ------------------------------------------------------------------ lifecycle thread
// Creates the device solver of an admitted request on the lifecycle stream and records
// its ready event (host copies are released).
void activate(yt_server* sv, Request* r) {
  yt_mesh_desc m{};
  m.n_elements = r->E;
  m.material = r->material.data();
  m.jacobian = r->jacobian.data();
  m.neighbours = r->neighbours.data();
  m.faces = r->faces.data();
  m.orient = r->orient.data();
  yt_scheme_desc sch{};
  sch.order = r->order;
  sch.dt = r->dt;
  sch.precision = sv->prec;
  yt_solver* s = nullptr;
  yt_status rc = solver_create_stream_ordered(&m, &sch, sv->life, &s);
  if (rc == YT_OK) rc = yt_solver_set_dofs(s, r->dofs.data(), YT_MEM_HOST, reinterpret_cast<yt_stream>(sv->life));
  if (rc == YT_OK && (cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming) != cudaSuccess ||
                      cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess ||
                      cudaEventRecord(r->ready, sv->life) != cudaSuccess))
    rc = YT_ERR_CUDA;
  if (rc != YT_OK) {
    r->status = rc;
    r->error = yt_last_error();
    if (s) yt_solver_destroy(s);
    throw Error(rc, r->error);
  }
  r->solver = s;
  std::vector<double>().swap(r->dofs);
  std::vector<double>().swap(r->material);
  std::vector<double>().swap(r->jacobian);
}

// Copies the final DOFs of a finished solve out and frees it (its last step is complete).
yt_status finish(yt_server* sv, Request* r) {
  r->result.resize((size_t)r->E * kNq * r->solver->B);
  yt_status rc = yt_solver_get(r->solver, YT_FIELD_DOFS, r->result.data(), YT_MEM_HOST,
                               reinterpret_cast<yt_stream>(sv->life));
  if (rc == YT_OK && cudaStreamSynchronize(sv->life) != cudaSuccess) rc = YT_ERR_CUDA;
  yt_solver_destroy(r->solver);
  r->solver = nullptr;
  return rc;
}

void release_events(Request* r) {
  if (r->ready) cudaEventDestroy(r->ready);
  if (r->done) cudaEventDestroy(r->done);
  r->ready = r->done = nullptr;
}

// Admission decision (sv->mu held): the next request to admit, or null.
Request* next_admission(yt_server* sv, double now) {
  while (!sv->pending.empty() && sv->pending.front()->bytes > sv->budget) {
    Request* r = sv->pending.front();        // can never run
    sv->pending.pop_front();
    r->state = kFailed;
    r->status = YT_ERR_OOM;
    r->error = "request needs more device memory than the whole budget";
    r->t_done = now;
    ++sv->failed;
    sv->cv_done.notify_all();
  }
  if (sv->pending.empty()) return nullptr;
  Request* head = sv->pending.front();
  if (head->id != sv->head_id) {
    sv->head_id = head->id;
    sv->head_since = now;
  }
  auto take = [&](std::deque<Request*>::iterator it) {
    Request* r = *it;
    sv->pending.erase(it);
    sv->in_use += r->bytes;
    sv->peak = std::max(sv->peak, sv->in_use);
    r->state = kAdmitting;
    ++sv->admitting;
    return r;
  };
  if (sv->in_use + head->bytes <= sv->budget) return take(sv->pending.begin());
  if (now - sv->head_since > kBackfillS) return nullptr;   // memory is reserved for the head
  for (auto it = sv->pending.begin() + 1; it != sv->pending.end(); ++it)
    if (sv->in_use + (*it)->bytes <= sv->budget) return take(it);
  return nullptr;
}

void lifecycle_loop(yt_server* sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    Request* admit = nullptr;
    std::vector<Request*> fin;
    {
      std::unique_lock<std::mutex> lock(sv->mu);
      for (;;) {
        for (Request* r : sv->finishing)
          if (cudaEventQuery(r->done) != cudaErrorNotReady) fin.push_back(r);
        for (Request* r : fin) sv->finishing.erase(std::find(sv->finishing.begin(), sv->finishing.end(), r));
        if (!fin.empty()) break;
        if (sv->fatal.empty()) admit = next_admission(sv, now_s());
        if (admit) break;
        if (sv->stop && sv->pending.empty() && sv->finishing.empty() && sv->active.empty() &&
            sv->ready.empty() && sv->admitting == 0)
          return;
        // poll the completion events while solves are finishing; otherwise sleep until
        // a submission, a completion hand-over or a budget change
        if (!sv->finishing.empty() || (!sv->pending.empty() && sv->fatal.empty()))
          sv->cv_life.wait_for(lock, std::chrono::microseconds(200));
        else
          sv->cv_life.wait(lock);
      }
    }
    for (Request* r : fin) {
      const yt_status rc = finish(sv, r);
      std::lock_guard<std::mutex> lock(sv->mu);
      release_events(r);
      r->t_done = now_s();
      r->state = rc == YT_OK ? kDone : kFailed;
      r->status = rc;
      if (rc == YT_OK) ++sv->completed;
      else ++sv->failed;
      sv->in_use -= r->bytes;
      sv->cv_done.notify_all();
    }
    if (admit) {
      bool ok = true;
      try {
        activate(sv, admit);
      } catch (const std::exception&) {
        ok = false;
      }
      std::lock_guard<std::mutex> lock(sv->mu);
      --sv->admitting;
      if (ok && sv->fatal.empty()) {
        admit->t_admit = now_s();
        admit->state = kReady;
        sv->ready.push_back(admit);
        sv->cv_work.notify_all();
      } else {
        if (admit->solver) {
          yt_solver_destroy(admit->solver);
          admit->solver = nullptr;
        }
        release_events(admit);
        admit->state = kFailed;
        if (admit->status == YT_OK) admit->status = YT_ERR_CUDA;
        if (admit->error.empty()) admit->error = sv->fatal;
        admit->t_done = now_s();
        sv->in_use -= admit->bytes;
        ++sv->failed;
        sv->cv_done.notify_all();
      }
    }
  }
}

// ---------------------------------------------------------------------- worker thread
// After a failed tick the device state of the active solves is unknown: every active,
// ready and finishing solve is freed and fails, every pending request fails, and later
// submissions are refused (sv->fatal).  Called with sv->mu held, the degree streams idle.
void fail_all(yt_server* sv, const std::string& why) {
  sv->fatal = why;
  const double t = now_s();
  auto drop = [&](Request* r) {
    if (r->solver) yt_solver_destroy(r->solver);
    r->solver = nullptr;
    release_events(r);
    sv->in_use -= r->bytes;
    r->state = kFailed;
    r->status = YT_ERR_CUDA;
    r->error = why;
    r->t_done = t;
    ++sv->failed;
  };
  for (Request* r : sv->active) drop(r);
  for (Request* r : sv->ready) drop(r);
  for (Request* r : sv->finishing) drop(r);
  sv->active.clear();
  sv->ready.clear();
  sv->finishing.clear();
  for (Request* r : sv->pending) {
    r->state = kFailed;
    r->status = YT_ERR_CUDA;
    r->error = "server stopped after a failed step: " + why;
    r->t_done = t;
    ++sv->failed;
  }
  sv->pending.clear();
  sv->cv_done.notify_all();
  sv->cv_life.notify_all();
}

// Writes the tile table of degree o into a free slot and uploads it on the degree's
// stream (the slot's previous reader has finished: its event is waited for first).
void upload_table(yt_server* sv, int o, const std::vector<Request*>& solves) {
  Tables& T = sv->tables[o];
  size_t n = 0;
  for (Request* r : solves) n += (size_t)r->solver->ntiles;
  const int k = (T.cur + 1) % kSlots;
  if (T.used[k]) cuda_check(cudaEventSynchronize(T.used[k]), "tile table slot");
  if (T.cap[k] < n) {
    const size_t cap = std::max<size_t>(n * 2, 4096);
    if (T.host[k]) cudaFreeHost(T.host[k]);
    if (T.dev[k]) cuda_check(cudaFreeAsync(T.dev[k], sv->streams[o]), "free tile table");
    T.host[k] = nullptr;
    T.dev[k] = nullptr;
    cuda_check(cudaMallocHost(reinterpret_cast<void**>(&T.host[k]), cap * sizeof(TileRef)), "pinned tile table");
    cuda_check(cudaMallocAsync(reinterpret_cast<void**>(&T.dev[k]), cap * sizeof(TileRef), sv->streams[o]),
               "tile table");
    T.cap[k] = cap;
  }
  size_t i = 0;
  for (Request* r : solves) {
    yt_solver* s = r->solver;
    for (int64_t t = 0; t < s->ntiles; ++t) {
      TileRef& ref = T.host[k][i++];
      ref.Q = s->Q;
      ref.I = s->I;
      ref.Pface = s->Pface;
      ref.Wloc = s->Wloc;
      ref.star = s->star_r;
      ref.floc = s->floc_r;
      ref.fnb = s->fnb_r;
      ref.conn = s->conn;
      ref.tile = t;
      ref.dt = s->dt;
    }
  }
  cuda_check(cudaMemcpyAsync(T.dev[k], T.host[k], n * sizeof(TileRef), cudaMemcpyHostToDevice, sv->streams[o]),
             "copy tile table");
  T.cur = k;
  T.n = n;
}

// Enqueues one step of every active solve: per degree, one shared local and one shared
// neighbour launch over the tile table of that degree's solves.
void tick(yt_server* sv, const std::vector<Request*>& act) {
  if (sv->fail_at_tick >= 0 && sv->ticks == sv->fail_at_tick)
    throw Error(YT_ERR_CUDA, "injected failure of tick " + std::to_string(sv->ticks));
  std::vector<Request*> by_order[8];
  for (Request* r : act) by_order[r->order].push_back(r);
  for (int o = 2; o <= 7; ++o) {
    if (by_order[o].empty()) continue;
    cudaStream_t st = sv->streams[o];
    // at most kAhead ticks in flight on this stream
    cudaEvent_t& ev = sv->tick_ev[o][sv->stream_ticks[o] % kAhead];
    if (sv->stream_ticks[o] >= kAhead) cuda_check(cudaEventSynchronize(ev), "tick lookahead");
    if (sv->dirty[o]) {
      upload_table(sv, o, by_order[o]);
      sv->dirty[o] = false;
    }
    yt_solver* s0 = by_order[o].front()->solver;
    AderLaunch L = solver_launch_args(s0, st);
    L.refs = sv->tables[o].dev[sv->tables[o].cur];
    L.ntiles = (int64_t)sv->tables[o].n;
    solver_launch_variant(s0, L, 0);
    solver_launch_variant(s0, L, 2);
    cuda_check(cudaEventRecord(ev, st), "tick event");
    cuda_check(cudaEventRecord(sv->tables[o].used[sv->tables[o].cur], st), "table event");
    ++sv->stream_ticks[o];
  }
}

void worker_loop(yt_server* sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    std::vector<Request*> act;
    {
      std::unique_lock<std::mutex> lock(sv->mu);
      sv->cv_work.wait(lock, [&] {
        return !sv->ready.empty() || !sv->active.empty() ||
               (sv->stop && sv->pending.empty() && sv->admitting == 0 && sv->finishing.empty());
      });
      if (sv->ready.empty() && sv->active.empty()) return;     // stopped and drained
      // newly set-up solves join: their degree stream waits for the set-up on the device
      bool ok = true;
      for (Request* r : sv->ready) {
        ok = ok && cudaStreamWaitEvent(sv->streams[r->order], r->ready, 0) == cudaSuccess;
        r->state = kActive;
        sv->active.push_back(r);
        sv->dirty[r->order] = true;
      }
      sv->ready.clear();
      sv->max_active = std::max<int64_t>(sv->max_active, (int64_t)sv->active.size());
      if (!ok) {
        for (int o = 2; o <= 7; ++o) (void)cudaStreamSynchronize(sv->streams[o]);
        fail_all(sv, "cudaStreamWaitEvent failed");
        continue;
      }
      act = sv->active;
    }
    try {
      tick(sv, act);
    } catch (const std::exception& e) {
      for (int o = 2; o <= 7; ++o) (void)cudaStreamSynchronize(sv->streams[o]);
      std::lock_guard<std::mutex> lock(sv->mu);
      fail_all(sv, e.what());
      continue;
    }
    std::lock_guard<std::mutex> lock(sv->mu);
    ++sv->ticks;
    bool ok = true;
    for (Request* r : act) {
      ++r->enqueued_steps;
      sv->element_updates += (double)r->E;
      if (r->enqueued_steps >= r->steps) {
        // its last step is enqueued: the lifecycle thread copies it out once it is done
        ok = ok && cudaEventRecord(r->done, sv->streams[r->order]) == cudaSuccess;
        r->state = kFinishing;
        sv->active.erase(std::find(sv->active.begin(), sv->active.end(), r));
        sv->finishing.push_back(r);
        sv->dirty[r->order] = true;
      }
    }
    if (!ok) {
      for (int o = 2; o <= 7; ++o) (void)cudaStreamSynchronize(sv->streams[o]);
      fail_all(sv, "cudaEventRecord failed");
    }
    sv->cv_life.notify_all();
  }
}

}  // namespace

yt_server::~yt_server() {
  {
    std::lock_guard<std::mutex> lock(mu);
    stop = true;
  }
  cv_work.notify_all();
  cv_life.notify_all();
  if (lifecycle.joinable()) lifecycle.join();
  {
    std::lock_guard<std::mutex> lock(mu);
  }
  cv_work.notify_all();
  if (worker.joinable()) worker.join();
  for (auto& kv : requests) {
    if (kv.second->solver) yt_solver_destroy(kv.second->solver);
    release_events(kv.second.get());
  }
  for (int o = 0; o < 8; ++o) {
    if (streams[o]) cudaStreamSynchronize(streams[o]);
    for (int k = 0; k < kSlots; ++k) {
      if (tables[o].host[k]) cudaFreeHost(tables[o].host[k]);
      if (tables[o].dev[k]) cudaFreeAsync(tables[o].dev[k], streams[o]);
      if (tables[o].used[k]) cudaEventDestroy(tables[o].used[k]);
    }
    for (int k = 0; k < kAhead; ++k)
      if (tick_ev[o][k]) cudaEventDestroy(tick_ev[o][k]);
    if (streams[o]) {
      cudaStreamSynchronize(streams[o]);
      cudaStreamDestroy(streams[o]);
    }
  }
  if (life) {
    cudaStreamSynchronize(life);
    cudaStreamDestroy(life);
  }
}

extern "C" yt_status yt_server_create(const yt_server_desc* desc, yt_server** out) {
  return guarded([&] {
    YT_REQUIRE(desc && out, YT_ERR_INVALID, "null argument");
    *out = nullptr;
    YT_REQUIRE(desc->hbm_budget_bytes > 0, YT_ERR_INVALID, "budget must be positive");
    YT_REQUIRE(desc->precision == YT_F64 || desc->precision == YT_F32, YT_ERR_UNSUPPORTED, "precision");
    YT_REQUIRE(desc->flags == 0, YT_ERR_INVALID, "flags must be 0");
    auto sv = std::make_unique<yt_server>();
    sv->budget = (size_t)desc->hbm_budget_bytes;
    sv->prec = desc->precision;
    cuda_check(cudaGetDevice(&sv->device), "cudaGetDevice");
    // freed solver memory stays in the device's stream-ordered pool for the next ones
    cudaMemPool_t pool = nullptr;
    cuda_check(cudaDeviceGetDefaultMemPool(&pool, sv->device), "default memory pool");
    uint64_t keep = UINT64_MAX;
    cuda_check(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep), "pool threshold");
    for (int o = 0; o < 8; ++o) {
      cuda_check(cudaStreamCreateWithFlags(&sv->streams[o], cudaStreamNonBlocking), "stream");
      for (int k = 0; k < kAhead; ++k)
        cuda_check(cudaEventCreateWithFlags(&sv->tick_ev[o][k], cudaEventDisableTiming), "event");
      for (int k = 0; k < kSlots; ++k)
        cuda_check(cudaEventCreateWithFlags(&sv->tables[o].used[k], cudaEventDisableTiming), "event");
    }
    cuda_check(cudaStreamCreateWithFlags(&sv->life, cudaStreamNonBlocking), "stream");
    sv->worker = std::thread(worker_loop, sv.get());
    sv->lifecycle = std::thread(lifecycle_loop, sv.get());
    *out = sv.release();
  });
}

extern "C" yt_status yt_server_submit(yt_server* sv, const yt_mesh_desc* mesh, int32_t order,
                                      double dt, const double* dofs, int32_t n_steps,
                                      int64_t* request_id) {
  return guarded([&] {
    YT_REQUIRE(sv && mesh && dofs && request_id, YT_ERR_INVALID, "null argument");
    YT_REQUIRE(mesh->n_elements > 1 && mesh->material && mesh->jacobian && mesh->neighbours &&
                   mesh->faces && mesh->orient, YT_ERR_INVALID, "mesh needs full connectivity");
    YT_REQUIRE(!mesh->attenuation, YT_ERR_UNSUPPORTED, "servers: 9-quantity solves");
    YT_REQUIRE(order >= 2 && order <= 7, YT_ERR_UNSUPPORTED, "order");
    YT_REQUIRE(n_steps > 0, YT_ERR_INVALID, "n_steps must be positive");
    YT_REQUIRE(dt > 0, YT_ERR_INVALID, "dt must be positive");
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      YT_REQUIRE(sv->fatal.empty(), YT_ERR_CUDA, "server stopped after a failed step: " + sv->fatal);
    }
    auto r = std::make_unique<Request>();
    const int64_t E = mesh->n_elements;
    const size_t B = n_basis(order - 1);
    r->order = order;
    r->E = E;
    r->dt = dt;
    r->steps = n_steps;
    r->material.assign(mesh->material, mesh->material + E * 3);
    r->jacobian.assign(mesh->jacobian, mesh->jacobian + E * 9);
    r->neighbours.assign(mesh->neighbours, mesh->neighbours + E * 4);
    r->faces.assign(mesh->faces, mesh->faces + E * 4);
    r->orient.assign(mesh->orient, mesh->orient + E * 4);
    r->dofs.assign(dofs, dofs + (size_t)E * kNq * B);
    r->bytes = solver_device_bytes(order, sv->prec, E);
    r->t_submit = now_s();
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      r->id = sv->next_id++;
      *request_id = r->id;
      sv->pending.push_back(r.get());
      sv->requests[r->id] = std::move(r);
    }
    sv->cv_life.notify_all();
  });
}

extern "C" yt_status yt_server_wait(yt_server* sv, int64_t request_id, double* dofs_out,
                                    double* latency_s, double* queue_s) {
  return guarded([&] {
    YT_REQUIRE(sv, YT_ERR_INVALID, "null server");
    std::unique_lock<std::mutex> lock(sv->mu);
    auto it = sv->requests.find(request_id);
    YT_REQUIRE(it != sv->requests.end(), YT_ERR_INVALID, "unknown request id");
    Request* r = it->second.get();
    sv->cv_done.wait(lock, [&] { return r->state == kDone || r->state == kFailed; });
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    if (queue_s) *queue_s = (r->t_admit > 0 ? r->t_admit : r->t_done) - r->t_submit;
    if (r->state == kFailed) throw Error(r->status == YT_OK ? YT_ERR_CUDA : r->status, r->error);
    if (dofs_out) std::memcpy(dofs_out, r->result.data(), r->result.size() * sizeof(double));
  });
}

extern "C" yt_status yt_server_stats_get(yt_server* sv, yt_server_stats* out) {
  return guarded([&] {
    YT_REQUIRE(sv && out, YT_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lock(sv->mu);
    out->submitted = sv->next_id - 1;
    out->completed = sv->completed;
    out->failed = sv->failed;
    out->pending = (int64_t)sv->pending.size();
    out->active = (int64_t)(sv->active.size() + sv->ready.size() + sv->finishing.size()) + sv->admitting;
    out->max_active = sv->max_active;
    out->ticks = sv->ticks;
    out->budget_bytes = (int64_t)sv->budget;
    out->peak_bytes = (int64_t)sv->peak;
    out->element_updates = sv->element_updates;
  });
}

extern "C" yt_status yt_server_fail_tick(yt_server* sv, int64_t at_tick) {
  return guarded([&] {
    YT_REQUIRE(sv, YT_ERR_INVALID, "null server");
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->fail_at_tick = at_tick;
  });
}

extern "C" void yt_server_destroy(yt_server* sv) { delete sv; }
