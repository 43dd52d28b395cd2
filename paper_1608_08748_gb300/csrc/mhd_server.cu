// mhd_server.cu -- continuous-batching server of simulation requests (include/mhd.h, "Serving").
// Host code only: a scheduler thread admits requests by HBM budget, advances the admitted
// requests of each (lane, precision, CFL) group one step at a time with one batched launch per
// kernel class (mhd_batch_*), the groups independently on streams of their lane's priority, and
// retires finished requests to host memory and frees their device memory.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "mhd.h"

namespace mhd_rt {
int set_error(int code, const std::string& msg);  // mhd.cu
int last_error_code();                            // mhd.cu
}

namespace {

enum ReqState { WAITING, RUNNING, DONE, FAILED };

struct Req {
  int64_t id = 0;
  mhd_request r{};
  std::vector<char> init[9];  // initial fields, caller dtype (rho, m x3, E, B x3, rho_H2)
  bool has_h2 = false;
  size_t bytes = 0;
  ReqState st = WAITING;
  bool cancel = false;  // running: retire at the end of the current batched step
  mhd_sim* sim = nullptr;
  mhd_result res{};
  std::vector<double> out[9];  // final state (float64, B cell-centred)
};

// (lane, precision, cfl).  Lane 0 holds the requests below the bulk size and runs at high
// stream priority; lane 1 the bulk requests at low priority, so that a large box's long steps do
// not hold the small ones back: each group steps on its own stream as soon as its previous step
// has finished, and the block scheduler starts the high-priority blocks first as SMs free up.
struct GroupKey {
  int lane;
  int precision;
  double cfl;
  bool operator<(const GroupKey& o) const {
    if (lane != o.lane) return lane < o.lane;
    if (precision != o.precision) return precision < o.precision;
    return cfl < o.cfl;
  }
};

struct Group {
  std::vector<Req*> active;   // the members of the batch (of the step in flight, if any)
  std::vector<Req*> joining;  // admitted while a step was in flight: join at the next launch
  mhd_batch* batch = nullptr;
  bool dirty = true;
  bool inflight = false;  // a batched step is queued or running on the batch's stream
};

}  // namespace

struct mhd_server {
  size_t budget = 0;
  int max_active = 1;
  int policy = MHD_SERVE_FIFO;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::deque<int64_t> waiting;
  std::unordered_map<int64_t, std::unique_ptr<Req>> reqs;
  std::map<GroupKey, Group> groups;  // scheduler thread only
  size_t used = 0;
  int nactive = 0;
  int64_t next_id = 0;
  int64_t unfinished = 0;
  bool stop = false;
  bool paused = false;
  int64_t bulk_cells = 1ll << 24;  // requests with at least this many cells run in the bulk lane
  std::thread th;
  std::chrono::steady_clock::time_point t0;
  std::atomic<int64_t> iterations{0};
  int64_t peak_bytes = 0;
  int peak_active = 0;
};

namespace {

double now_s(const mhd_server* S) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - S->t0).count();
}

size_t dsize(int dtype) { return dtype == MHD_F32 ? 4 : 8; }

// create the device simulation of an admitted request; returns MHD_OK or an error code
int start_request(mhd_server* S, Req* q) {
  const mhd_request& r = q->r;
  mhd_sim* sim = mhd_create(r.nx, r.ny, r.nz, r.gamma, r.dx);
  if (!sim) {
    const int code = mhd_rt::last_error_code();
    return code < 0 ? code : MHD_ENOMEM;
  }
  int rc = MHD_OK;
  if (r.precision) rc = mhd_set_option(sim, MHD_OPT_PRECISION, 1.0);
  if (rc == MHD_OK) rc = mhd_set_option(sim, MHD_OPT_CHEM, r.chem ? 1.0 : 0.0);
  for (int d = 0; d < 3 && rc == MHD_OK; ++d) rc = mhd_set_option(sim, MHD_OPT_BC_X + d, r.bc[d] ? 1.0 : 0.0);
  if (rc == MHD_OK) {
    mhd_fields f{};
    f.rho = q->init[0].data();
    for (int d = 0; d < 3; ++d) {
      f.mom[d] = q->init[1 + d].data();
      f.B[d] = q->init[5 + d].data();
    }
    f.E = q->init[4].data();
    f.rho_h2 = q->has_h2 ? q->init[8].data() : nullptr;
    f.dtype = r.state.dtype;
    f.on_device = 0;
    rc = mhd_set_state(sim, &f);
  }
  if (rc != MHD_OK) {
    mhd_destroy(sim);
    return rc;
  }
  for (auto& v : q->init) std::vector<char>().swap(v);  // the host copy is no longer needed
  q->sim = sim;
  return MHD_OK;
}

// copy a finished request's state to host memory and release its device memory
int finish_request(mhd_server* S, Req* q) {
  const size_t N = (size_t)q->r.nx * q->r.ny * q->r.nz;
  for (auto& v : q->out) v.assign(N, 0.0);
  mhd_fields f{};
  f.rho = q->out[0].data();
  for (int d = 0; d < 3; ++d) {
    f.mom[d] = q->out[1 + d].data();
    f.B[d] = q->out[5 + d].data();
  }
  f.E = q->out[4].data();
  f.rho_h2 = q->out[8].data();
  f.dtype = MHD_F64;
  f.on_device = 0;
  int rc = mhd_get_state(q->sim, &f);
  mhd_diag dg{};
  if (rc == MHD_OK) rc = mhd_diagnostics(q->sim, &dg);
  q->res.t = dg.t;
  mhd_destroy(q->sim);
  q->sim = nullptr;
  return rc;
}

void scheduler(mhd_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<Req*> admit;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop) break;
      if (S->paused) {
        // admission held: nothing leaves the queue
      } else if (S->policy == MHD_SERVE_FIFO) {
        // strict arrival order: the head waits until it fits
        while (!S->waiting.empty()) {
          Req* q = S->reqs[S->waiting.front()].get();
          if (S->nactive >= S->max_active || S->used + q->bytes > S->budget) break;
          S->waiting.pop_front();
          S->used += q->bytes;
          S->nactive += 1;
          q->st = RUNNING;
          admit.push_back(q);
        }
      } else {
        // smallest work first: among the waiting requests that fit, the fewest cell-updates
        // (cells x steps), ties by arrival
        while (!S->waiting.empty() && S->nactive < S->max_active) {
          auto best = S->waiting.end();
          double best_work = 0.0;
          for (auto it = S->waiting.begin(); it != S->waiting.end(); ++it) {
            const Req* q = S->reqs[*it].get();
            if (S->used + q->bytes > S->budget) continue;
            const double work = (double)q->res.cells * q->r.nsteps;
            if (best == S->waiting.end() || work < best_work) {
              best = it;
              best_work = work;
            }
          }
          if (best == S->waiting.end()) break;
          Req* q = S->reqs[*best].get();
          S->waiting.erase(best);
          S->used += q->bytes;
          S->nactive += 1;
          q->st = RUNNING;
          admit.push_back(q);
        }
      }
      if (admit.empty() && S->nactive == 0) {
        S->cv.wait(lk, [&] { return S->stop || (!S->paused && !S->waiting.empty()); });
        continue;
      }
      if ((int64_t)S->used > S->peak_bytes) S->peak_bytes = (int64_t)S->used;
      if (S->nactive > S->peak_active) S->peak_active = S->nactive;
    }
    for (Req* q : admit) {
      int rc = start_request(S, q);
      std::lock_guard<std::mutex> lk(S->mu);
      q->res.t_admit = now_s(S);
      if (rc != MHD_OK) {
        q->st = FAILED;
        q->res.status = rc;
        S->used -= q->bytes;
        S->nactive -= 1;
        S->unfinished -= 1;
        S->cv_done.notify_all();
        continue;
      }
      const int64_t cells = (int64_t)q->r.nx * q->r.ny * q->r.nz;
      Group& G = S->groups[GroupKey{cells >= S->bulk_cells ? 1 : 0, q->r.precision, q->r.cfl}];
      G.joining.push_back(q);
    }
    // every group whose previous step has finished: take its results, then queue its next step
    bool progressed = !admit.empty();
    for (auto it = S->groups.begin(); it != S->groups.end();) {
      Group& G = it->second;
      if (G.inflight) {
        const int qrc = mhd_batch_query(G.batch);
        if (qrc == MHD_PENDING) {
          ++it;
          continue;
        }
        G.inflight = false;
        progressed = true;
        std::vector<Req*> keep, done;
        std::vector<int> qrcs;
        for (Req* q : G.active) {
          int r1 = qrc;
          if (qrc == MHD_ENONPHYS) {  // find the members that flagged it
            mhd_diag dg{};
            r1 = (mhd_diagnostics(q->sim, &dg) == MHD_OK && !(dg.error_flags & 1)) ? MHD_OK : MHD_ENONPHYS;
          }
          qrcs.push_back(r1);
        }
        {
          std::lock_guard<std::mutex> lk(S->mu);
          for (size_t k = 0; k < G.active.size(); ++k) {
            Req* q = G.active[k];
            if (qrcs[k] == MHD_OK) q->res.steps_done += 1;
            if (q->cancel) {
              q->res.status = MHD_ECANCELED;
              done.push_back(q);
            } else if (qrcs[k] != MHD_OK || q->res.steps_done >= q->r.nsteps) {
              if (qrcs[k] != MHD_OK) q->res.status = qrcs[k];
              done.push_back(q);
            } else {
              keep.push_back(q);
            }
          }
        }
        if (!done.empty()) {
          if (G.batch) mhd_batch_destroy(G.batch);
          G.batch = nullptr;
          G.dirty = true;
          for (Req* q : done) {
            int frc = MHD_OK;
            if (q->res.status == MHD_ECANCELED) {  // no result is kept: release the device memory
              mhd_destroy(q->sim);
              q->sim = nullptr;
            } else {
              frc = finish_request(S, q);
            }
            std::lock_guard<std::mutex> lk(S->mu);
            if (q->res.status == MHD_PENDING) q->res.status = frc;
            else if (q->res.status == MHD_OK && frc != MHD_OK) q->res.status = frc;
            q->res.t_done = now_s(S);
            q->st = q->res.status == MHD_OK ? DONE : FAILED;
            S->used -= q->bytes;
            S->nactive -= 1;
            S->unfinished -= 1;
          }
          S->cv_done.notify_all();
        }
        G.active.swap(keep);
      }
      if (!G.joining.empty()) {  // no step in flight here: the admitted requests join now
        G.active.insert(G.active.end(), G.joining.begin(), G.joining.end());
        G.joining.clear();
        G.dirty = true;
      }
      if (G.active.empty()) {
        if (G.batch) mhd_batch_destroy(G.batch);
        it = S->groups.erase(it);
        continue;
      }
      int rc = MHD_OK;
      if (G.dirty) {
        if (G.batch) mhd_batch_destroy(G.batch);
        std::vector<mhd_sim*> sims;
        for (Req* q : G.active) sims.push_back(q->sim);
        G.batch = mhd_batch_create(sims.data(), (int)sims.size());
        rc = G.batch ? MHD_OK : MHD_ECUDA;
        if (rc == MHD_OK) rc = mhd_batch_set_priority(G.batch, it->first.lane == 0 ? 1 : 0);
        G.dirty = false;
      }
      if (rc == MHD_OK) rc = mhd_batch_step(G.batch, it->first.cfl);
      if (rc == MHD_OK) {
        G.inflight = true;
        S->iterations += 1;
      } else {
        // the group cannot step: its requests end with the error
        std::lock_guard<std::mutex> lk(S->mu);
        for (Req* q : G.active) {
          if (q->sim) mhd_destroy(q->sim);
          q->sim = nullptr;
          q->res.status = rc;
          q->res.t_done = now_s(S);
          q->st = FAILED;
          S->used -= q->bytes;
          S->nactive -= 1;
          S->unfinished -= 1;
        }
        S->cv_done.notify_all();
        G.active.clear();
        if (G.batch) mhd_batch_destroy(G.batch);
        G.batch = nullptr;
        it = S->groups.erase(it);
        continue;
      }
      ++it;
    }
    if (!progressed) {
      // nothing finished: wait a little for the device (or for a submission or a stop)
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait_for(lk, std::chrono::microseconds(200), [&] { return S->stop; });
    }
  }
  for (auto& kv : S->groups) {
    if (kv.second.batch) mhd_batch_destroy(kv.second.batch);
    for (auto* list : {&kv.second.active, &kv.second.joining})
      for (Req* q : *list)
        if (q->sim) {
          mhd_destroy(q->sim);
          q->sim = nullptr;
        }
  }
  S->groups.clear();
}

}  // namespace

extern "C" {

mhd_server* mhd_server_create(size_t hbm_budget_bytes, int max_active) {
  if (hbm_budget_bytes == 0 || max_active < 1) {
    mhd_rt::set_error(MHD_EINVAL, "mhd_server_create: need a budget > 0 and max_active >= 1");
    return nullptr;
  }
  mhd_server* S = new (std::nothrow) mhd_server();
  if (!S) {
    mhd_rt::set_error(MHD_ENOMEM, "mhd_server_create: host allocation failed");
    return nullptr;
  }
  S->budget = hbm_budget_bytes;
  S->max_active = max_active;
  cudaGetDevice(&S->device);
  S->t0 = std::chrono::steady_clock::now();
  S->th = std::thread(scheduler, S);
  return S;
}

void mhd_server_destroy(mhd_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->th.joinable()) S->th.join();
  delete S;
}

int mhd_server_set_policy(mhd_server* S, int policy) {
  if (!S || (policy != MHD_SERVE_FIFO && policy != MHD_SERVE_SMALLEST_WORK))
    return mhd_rt::set_error(MHD_EINVAL, "mhd_server_set_policy: policy must be MHD_SERVE_FIFO or MHD_SERVE_SMALLEST_WORK");
  std::lock_guard<std::mutex> lk(S->mu);
  S->policy = policy;
  return MHD_OK;
}

int64_t mhd_submit(mhd_server* S, const mhd_request* r) {
  if (!S || !r) return mhd_rt::set_error(MHD_EINVAL, "mhd_submit: null argument");
  if (r->nx < 1 || r->ny < 1 || r->nz < 1 || !(r->gamma > 1.0) || !(r->dx > 0.0) || r->nsteps < 1 ||
      !(r->cfl > 0.0) || (r->precision != 0 && r->precision != 1) ||
      (r->state.dtype != MHD_F64 && r->state.dtype != MHD_F32) || r->state.on_device)
    return mhd_rt::set_error(MHD_EINVAL, "mhd_submit: bad request (sizes, gamma, dx, cfl, nsteps, host state)");
  const void* src[9] = {r->state.rho, r->state.mom[0], r->state.mom[1], r->state.mom[2], r->state.E,
                        r->state.B[0], r->state.B[1], r->state.B[2], r->state.rho_h2};
  for (int q = 0; q < 8; ++q)
    if (!src[q]) return mhd_rt::set_error(MHD_EINVAL, "mhd_submit: rho, mom[3], E and B[3] are required");
  auto q = std::make_unique<Req>();
  q->r = *r;
  q->bytes = mhd_bytes_needed(r->nx, r->ny, r->nz, r->precision, r->chem);
  if (q->bytes > S->budget)
    return mhd_rt::set_error(MHD_ECAPACITY, "mhd_submit: request needs " + std::to_string(q->bytes) +
                                                " bytes, more than the whole budget");
  const size_t bytes = (size_t)r->nx * r->ny * r->nz * dsize(r->state.dtype);
  for (int k = 0; k < 9; ++k) {
    if (!src[k]) continue;
    q->init[k].resize(bytes);
    std::memcpy(q->init[k].data(), src[k], bytes);
  }
  q->has_h2 = src[8] != nullptr;
  for (auto& p : {&q->r.state.rho, &q->r.state.E, &q->r.state.rho_h2}) *p = nullptr;
  for (int d = 0; d < 3; ++d) q->r.state.mom[d] = q->r.state.B[d] = nullptr;
  q->res.status = MHD_PENDING;
  q->res.cells = (int64_t)r->nx * r->ny * r->nz;
  std::lock_guard<std::mutex> lk(S->mu);
  q->id = S->next_id++;
  q->res.t_submit = now_s(S);
  int64_t id = q->id;
  S->waiting.push_back(id);
  S->reqs.emplace(id, std::move(q));
  S->unfinished += 1;
  S->cv.notify_all();
  return id;
}

int mhd_poll(mhd_server* S, int64_t id, mhd_result* out) {
  if (!S || !out) return mhd_rt::set_error(MHD_EINVAL, "mhd_poll: null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return mhd_rt::set_error(MHD_ENOTFOUND, "mhd_poll: unknown request id");
  *out = it->second->res;
  if (it->second->st == WAITING || it->second->st == RUNNING) return MHD_PENDING;
  return it->second->res.status;
}

int mhd_fetch(mhd_server* S, int64_t id, mhd_fields* out) {
  if (!S || !out || out->on_device) return mhd_rt::set_error(MHD_EINVAL, "mhd_fetch: bad argument");
  std::unique_ptr<Req> q;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return mhd_rt::set_error(MHD_ENOTFOUND, "mhd_fetch: unknown request id");
    if (it->second->st == WAITING || it->second->st == RUNNING) return MHD_PENDING;
    if (it->second->st == FAILED) {
      int rc = it->second->res.status;
      S->reqs.erase(it);
      return mhd_rt::set_error(rc, "mhd_fetch: the request failed");
    }
    q = std::move(it->second);
    S->reqs.erase(it);
  }
  void* dst[9] = {out->rho, out->mom[0], out->mom[1], out->mom[2], out->E, out->B[0], out->B[1], out->B[2], out->rho_h2};
  const size_t N = (size_t)q->r.nx * q->r.ny * q->r.nz;
  for (int k = 0; k < 9; ++k) {
    if (!dst[k]) continue;
    if (out->dtype == MHD_F32) {
      float* d = (float*)dst[k];
      for (size_t i = 0; i < N; ++i) d[i] = (float)q->out[k][i];
    } else {
      std::memcpy(dst[k], q->out[k].data(), N * sizeof(double));
    }
  }
  return MHD_OK;
}

int mhd_cancel(mhd_server* S, int64_t id) {
  if (!S) return mhd_rt::set_error(MHD_EINVAL, "mhd_cancel: null server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return mhd_rt::set_error(MHD_ENOTFOUND, "mhd_cancel: unknown request id");
  Req* q = it->second.get();
  if (q->st == WAITING) {
    for (auto w = S->waiting.begin(); w != S->waiting.end(); ++w)
      if (*w == id) {
        S->waiting.erase(w);
        break;
      }
    q->st = FAILED;
    q->res.status = MHD_ECANCELED;
    q->res.t_done = now_s(S);
    S->unfinished -= 1;
    S->cv_done.notify_all();
    return MHD_OK;
  }
  if (q->st == RUNNING) {
    q->cancel = true;
    return MHD_OK;
  }
  return mhd_rt::set_error(MHD_EINVAL, "mhd_cancel: the request has already finished");
}

int mhd_server_pause(mhd_server* S, int paused) {
  if (!S || (paused != 0 && paused != 1)) return mhd_rt::set_error(MHD_EINVAL, "mhd_server_pause: paused must be 0 or 1");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->paused = paused != 0;
  }
  S->cv.notify_all();
  return MHD_OK;
}

int mhd_server_set_budget(mhd_server* S, size_t hbm_budget_bytes) {
  if (!S || hbm_budget_bytes == 0) return mhd_rt::set_error(MHD_EINVAL, "mhd_server_set_budget: need a budget > 0");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->budget = hbm_budget_bytes;
    for (auto w = S->waiting.begin(); w != S->waiting.end();) {
      Req* q = S->reqs[*w].get();
      if (q->bytes > S->budget) {
        q->st = FAILED;
        q->res.status = MHD_ECAPACITY;
        q->res.t_done = now_s(S);
        S->unfinished -= 1;
        w = S->waiting.erase(w);
      } else {
        ++w;
      }
    }
    S->cv_done.notify_all();
  }
  S->cv.notify_all();
  return MHD_OK;
}

int mhd_server_set_bulk_cells(mhd_server* S, int64_t cells) {
  if (!S || cells < 1) return mhd_rt::set_error(MHD_EINVAL, "mhd_server_set_bulk_cells: need cells >= 1");
  std::lock_guard<std::mutex> lk(S->mu);
  S->bulk_cells = cells;
  return MHD_OK;
}

int mhd_server_drain(mhd_server* S, double timeout_s) {
  if (!S) return mhd_rt::set_error(MHD_EINVAL, "mhd_server_drain: null server");
  std::unique_lock<std::mutex> lk(S->mu);
  bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return S->unfinished == 0; });
  return ok ? MHD_OK : mhd_rt::set_error(MHD_ETIMEOUT, "mhd_server_drain: requests still running");
}

double mhd_server_clock(mhd_server* S) { return S ? now_s(S) : 0.0; }

int mhd_server_stats(mhd_server* S, int64_t* iterations, int64_t* peak_bytes, int* peak_active) {
  if (!S) return mhd_rt::set_error(MHD_EINVAL, "mhd_server_stats: null server");
  std::lock_guard<std::mutex> lk(S->mu);
  if (iterations) *iterations = S->iterations.load();
  if (peak_bytes) *peak_bytes = S->peak_bytes;
  if (peak_active) *peak_active = S->peak_active;
  return MHD_OK;
}

}  // extern "C"
