// Serving runtime: independent ADER-DG solves submitted at any time, admitted while their
// device memory fits an HBM budget, and advanced together (continuous batching).
//
// A worker thread owns the device work.  Every iteration ("tick") it admits pending
// requests in arrival order while the budget allows, then advances every active solve by
// one step: for each polynomial degree, ONE local and ONE neighbour kernel launch cover
// the tiles of all active solves of that degree (a per-CTA tile table points each CTA at
// its solve's buffers, tile index and time step), and the degrees run on separate
// streams, so work of different solves overlaps on the device.  A solve that has taken
// its last step is copied out and freed at once, which frees budget for the next
// admissions.  Every tile is computed exactly as in a solve alone (no data crosses solve
// boundaries), so a result does not depend on the mix it was computed in.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
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

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum ReqState { kPending = 0, kActive = 1, kDone = 2, kFailed = 3 };

struct Request {
  int64_t id = 0;
  int order = 0;
  int64_t E = 0;
  double dt = 0.0;
  int steps = 0, done_steps = 0;
  std::vector<double> material, jacobian, dofs, result;
  std::vector<int32_t> neighbours;
  std::vector<int8_t> faces, orient;
  size_t bytes = 0;
  int state = kPending;
  yt_status status = YT_OK;
  std::string error;
  double t_submit = 0, t_admit = 0, t_done = 0;
  yt_solver* solver = nullptr;
};

}  // namespace

struct yt_server {
  size_t budget = 0, in_use = 0, peak = 0;
  yt_precision prec = YT_F32;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::deque<Request*> pending;
  std::vector<Request*> active;
  std::map<int64_t, std::unique_ptr<Request>> requests;
  int64_t next_id = 1;
  int64_t completed = 0, failed = 0, ticks = 0, max_active = 0;
  double element_updates = 0.0;
  std::thread worker;
  cudaStream_t streams[8] = {};
  TileRef* d_refs[8] = {};
  size_t ref_capacity[8] = {};
  std::vector<TileRef> h_refs[8];
  bool refs_dirty = true;
  std::string fatal;            // set when a tick failed: the server then fails every request
  int64_t fail_at_tick = -1;    // diagnostics: a tick number treated as failed (host side)
  ~yt_server();
};

namespace {

// Creates the device solver of an admitted request (host copies are released).
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
  yt_status rc = yt_solver_create(&m, &sch, nullptr, &s);
  if (rc == YT_OK) rc = yt_solver_set_dofs(s, r->dofs.data(), YT_MEM_HOST, nullptr);
  if (rc == YT_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) rc = YT_ERR_CUDA;
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

// After a failed tick the device state of the active solves is unknown: every active
// solve is destroyed and its budget released, every pending request fails, and later
// submissions are refused (sv->fatal).  Called with sv->mu held.
void fail_all(yt_server* sv, const std::string& why) {
  sv->fatal = why;
  const double t = now_s();
  for (Request* r : sv->active) {
    if (r->solver) yt_solver_destroy(r->solver);
    r->solver = nullptr;
    sv->in_use -= r->bytes;
    r->state = kFailed;
    r->status = YT_ERR_CUDA;
    r->error = why;
    r->t_done = t;
    ++sv->failed;
  }
  sv->active.clear();
  for (Request* r : sv->pending) {
    r->state = kFailed;
    r->status = YT_ERR_CUDA;
    r->error = "server stopped after a failed step: " + why;
    r->t_done = t;
    ++sv->failed;
  }
  sv->pending.clear();
  sv->refs_dirty = true;
  sv->cv_done.notify_all();
}

// One step of every active solve: per degree, one shared local and one shared neighbour
// launch over the tile table of that degree's solves.
void tick(yt_server* sv, const std::vector<Request*>& act) {
  if (sv->fail_at_tick >= 0 && sv->ticks == sv->fail_at_tick)
    throw Error(YT_ERR_CUDA, "injected failure of tick " + std::to_string(sv->ticks));
  std::vector<Request*> by_order[8];
  for (Request* r : act) by_order[r->order].push_back(r);
  for (int o = 2; o <= 7; ++o) {
    if (by_order[o].empty()) continue;
    auto& refs = sv->h_refs[o];
    if (sv->refs_dirty) {
      refs.clear();
      for (Request* r : by_order[o]) {
        yt_solver* s = r->solver;
        for (int64_t t = 0; t < s->ntiles; ++t) {
          TileRef ref;
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
          refs.push_back(ref);
        }
      }
      if (refs.size() > sv->ref_capacity[o]) {
        if (sv->d_refs[o]) cudaFree(sv->d_refs[o]);
        sv->d_refs[o] = nullptr;
        const size_t cap = refs.size() * 2;
        cuda_check(cudaMalloc(&sv->d_refs[o], cap * sizeof(TileRef)), "cudaMalloc tile table");
        sv->ref_capacity[o] = cap;
      }
      cuda_check(cudaMemcpyAsync(sv->d_refs[o], refs.data(), refs.size() * sizeof(TileRef),
                                 cudaMemcpyHostToDevice, sv->streams[o]), "copy tile table");
    }
    yt_solver* s0 = by_order[o].front()->solver;
    AderLaunch L = solver_launch_args(s0, sv->streams[o]);
    L.refs = sv->d_refs[o];
    L.ntiles = (int64_t)refs.size();
    solver_launch_variant(s0, L, 0);
    solver_launch_variant(s0, L, 2);
  }
  for (int o = 2; o <= 7; ++o)
    if (!by_order[o].empty()) cuda_check(cudaStreamSynchronize(sv->streams[o]), "tick");
  sv->refs_dirty = false;
}

void worker_loop(yt_server* sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    std::vector<Request*> admit;
    {
      std::unique_lock<std::mutex> lock(sv->mu);
      sv->cv_work.wait(lock, [&] { return sv->stop || !sv->pending.empty() || !sv->active.empty(); });
      if (sv->stop && sv->pending.empty() && sv->active.empty()) return;
      // admission in arrival order while the budget allows (a request larger than the
      // whole budget can never run and fails)
      while (!sv->pending.empty()) {
        Request* r = sv->pending.front();
        if (r->bytes > sv->budget) {
          sv->pending.pop_front();
          r->state = kFailed;
          r->status = YT_ERR_OOM;
          r->error = "request needs more device memory than the whole budget";
          r->t_done = now_s();
          ++sv->failed;
          sv->cv_done.notify_all();
          continue;
        }
        if (sv->in_use + r->bytes > sv->budget) break;
        sv->pending.pop_front();
        sv->in_use += r->bytes;
        sv->peak = std::max(sv->peak, sv->in_use);
        admit.push_back(r);
      }
    }
    for (Request* r : admit) {
      try {
        activate(sv, r);
        r->t_admit = now_s();
        std::lock_guard<std::mutex> lock(sv->mu);
        r->state = kActive;
        sv->active.push_back(r);
        sv->refs_dirty = true;
        sv->max_active = std::max<int64_t>(sv->max_active, (int64_t)sv->active.size());
      } catch (const std::exception&) {
        std::lock_guard<std::mutex> lock(sv->mu);
        r->state = kFailed;
        r->t_done = now_s();
        sv->in_use -= r->bytes;
        ++sv->failed;
        sv->cv_done.notify_all();
      }
    }
    std::vector<Request*> act;
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      act = sv->active;
    }
    if (act.empty()) continue;
    try {
      tick(sv, act);
    } catch (const std::exception& e) {
      for (int o = 2; o <= 7; ++o) (void)cudaStreamSynchronize(sv->streams[o]);
      std::lock_guard<std::mutex> lock(sv->mu);
      fail_all(sv, e.what());
      continue;
    }
    std::vector<Request*> finished;
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      ++sv->ticks;
      for (Request* r : act) {
        ++r->done_steps;
        sv->element_updates += (double)r->E;
        if (r->done_steps >= r->steps) finished.push_back(r);
      }
    }
    for (Request* r : finished) {
      r->result.resize((size_t)r->E * kNq * r->solver->B);
      yt_status rc = yt_solver_get(r->solver, YT_FIELD_DOFS, r->result.data(), YT_MEM_HOST, nullptr);
      if (rc == YT_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) rc = YT_ERR_CUDA;
      yt_solver_destroy(r->solver);
      r->solver = nullptr;
      std::lock_guard<std::mutex> lock(sv->mu);
      r->t_done = now_s();
      r->state = rc == YT_OK ? kDone : kFailed;
      r->status = rc;
      if (rc == YT_OK) ++sv->completed;
      else ++sv->failed;
      sv->in_use -= r->bytes;
      sv->active.erase(std::find(sv->active.begin(), sv->active.end(), r));
      sv->refs_dirty = true;
      sv->cv_done.notify_all();
    }
  }
}

}  // namespace

yt_server::~yt_server() {
  {
    std::lock_guard<std::mutex> lock(mu);
    stop = true;
  }
  cv_work.notify_all();
  if (worker.joinable()) worker.join();
  for (auto& kv : requests)
    if (kv.second->solver) yt_solver_destroy(kv.second->solver);
  for (int o = 0; o < 8; ++o) {
    if (d_refs[o]) cudaFree(d_refs[o]);
    if (streams[o]) cudaStreamDestroy(streams[o]);
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
    for (int o = 0; o < 8; ++o)
      cuda_check(cudaStreamCreateWithFlags(&sv->streams[o], cudaStreamNonBlocking), "stream");
    sv->worker = std::thread(worker_loop, sv.get());
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
    sv->cv_work.notify_all();
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
    out->active = (int64_t)sv->active.size();
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
