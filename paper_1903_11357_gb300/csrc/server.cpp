// Serving: continuous batching of ASPCG solve requests on one GPU.
//
// dgasm_submit plans the request on the caller's thread (partition, ordering, envelope: host work)
// and estimates its device footprint (factors, coarse operator, Krylov state).  A scheduler thread
// admits queued requests in arrival order while a slot is free and the footprint fits in the memory
// budget next to the admitted ones, and runs rounds of ROUND_ITERS batched PCG iterations over the
// active requests together (one launch per kernel for the whole batch).  A setup thread builds the
// preconditioners of admitted requests and runs their initial step on a stream of its own, so that
// this device work overlaps the rounds of the requests already active; a request joins the active
// batch at the first round after its setup completes.  Finished requests are retired between rounds
// and their memory returned.  Each problem's arithmetic and reduction order are independent of the
// batch it runs in, so results are bitwise identical alone and in the mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include <cuda_runtime.h>

#include "common.h"
#include "engine.h"
#include "solver.h"

using namespace dgasm;

namespace {

enum ReqState { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2 };
constexpr int ROUND_ITERS = 8;

struct Request {
  uint64_t ticket = 0;
  dgasm_system_s* sys = nullptr;
  dgasm_setup_opts so{};
  std::vector<int> sub, agg;
  int nrhs = 1;
  const double* b = nullptr;
  double* x = nullptr;
  dgasm_solve_opts o{};
  int state = Q_QUEUED;
  int rc = DGASM_OK;
  std::vector<dgasm_stats> st;
  std::unique_ptr<dgasm_prec_s> pc;
  size_t bytes = 0;
  std::chrono::steady_clock::time_point t_submit, t_admit;
};

}  // namespace

struct dgasm_server_s {
  size_t budget = 0;
  int max_slots = 1;
  int device = 0;
  cudaStream_t stream = nullptr, own_stream = nullptr, setup_stream = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_setup;
  std::deque<Request*> queue;
  std::deque<Request*> setup_queue;   // admitted, waiting for their device setup
  std::vector<Request*> ready;        // set up and initialised, joining the batch at the next round
  int in_setup = 0;                   // admitted requests not active yet
  bool stop_setup = false;
  std::vector<Request*> active;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  size_t in_use = 0;
  int64_t n_done = 0, rounds = 0, stalls = 0;
  std::thread th, setup_th;
  std::unique_ptr<Engine> engine, engine_aux;
  bool active_changed = true;

  void run();
  void setup_run();
  void finish_request(Request* r, int rc, const char* msg);
};

void dgasm_server_s::finish_request(Request* r, int rc, const char* msg) {
  // called with mu held
  r->rc = rc;
  r->state = Q_DONE;
  if (rc < 0 && r->st.empty()) r->st.assign(r->nrhs, dgasm_stats{});
  (void)msg;
  in_use -= std::min(in_use, r->bytes);
  r->bytes = 0;
  ++n_done;
  cv_done.notify_all();
}

// setup thread: device setup (preconditioner, local-solve variant) and initial step of admitted requests,
// one at a time, on setup_stream
void dgasm_server_s::setup_run() {
  cudaSetDevice(device);
  Engine eng;
  while (true) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_setup.wait(lk, [&] { return stop_setup || !setup_queue.empty(); });
      if (setup_queue.empty()) break;
      r = setup_queue.front();
      setup_queue.pop_front();
    }
    dgasm_prec_s* pc = r->pc.get();
    int rc = prec_build(pc);
    // the same local-solve variant a solve of this problem alone would take (measured once per shape)
    if (rc >= 0) rc = tune_local_variant(pc, r->nrhs, r->b, setup_stream);
    const dgasm_solve_opts* o = &r->o;
    if (rc >= 0) rc = eng.build(1, &pc, &r->nrhs, &r->b, &r->x, &o, setup_stream, -1);
    if (rc >= 0) rc = eng.reset_state();
    if (rc >= 0) rc = eng.init();
    if (rc >= 0 && cudaStreamSynchronize(setup_stream) != cudaSuccess) rc = cuda_error(cudaGetLastError(), "init");
    std::lock_guard<std::mutex> lk(mu);
    if (rc < 0) {
      --in_setup;
      finish_request(r, rc, "setup failed");
      r->pc.reset();
    } else {
      ready.push_back(r);
    }
    cv_work.notify_all();
  }
}

void dgasm_server_s::run() {
  cudaSetDevice(device);
  engine.reset(new Engine());
  engine_aux.reset(new Engine());
  while (true) {
    {
      std::unique_lock<std::mutex> lk(mu);
      // admissible: a queued request, a free slot and room in the budget for the first in line
      auto admissible = [&] {
        return !stop && !queue.empty() && (int)(active.size() + in_setup) < max_slots &&
               in_use + queue.front()->bytes <= budget;
      };
      cv_work.wait(lk, [&] { return stop || !active.empty() || !ready.empty() || admissible(); });
      if (stop && active.empty() && queue.empty() && ready.empty() && in_setup == 0) break;
      // admission in arrival order while a slot is free and the footprint fits
      while (!stop && !queue.empty() && (int)(active.size() + in_setup) < max_slots) {
        Request* r = queue.front();
        if (in_use + r->bytes > budget) {
          ++stalls;
          break;
        }
        queue.pop_front();
        in_use += r->bytes;
        r->state = Q_RUNNING;
        r->t_admit = std::chrono::steady_clock::now();
        setup_queue.push_back(r);
        ++in_setup;
        cv_setup.notify_one();
      }
      // requests whose setup completed join this round
      for (Request* r : ready) {
        active.push_back(r);
        --in_setup;
        active_changed = true;
      }
      ready.clear();
      if (active.empty()) {
        // nothing to iterate yet: wait for a setup to complete (or shut down when nothing is left)
        if (stop && queue.empty() && in_setup == 0) break;
        cv_work.wait(lk, [&] { return !ready.empty() || (stop && in_setup == 0) || admissible(); });
        continue;
      }
    }
    if (active.empty()) continue;
    // one round of batched iterations over every admitted request
    std::vector<dgasm_prec_s*> pcs;
    std::vector<int> nr;
    std::vector<const double*> bs;
    std::vector<double*> xs;
    std::vector<const dgasm_solve_opts*> os;
    for (Request* r : active) {
      pcs.push_back(r->pc.get());
      nr.push_back(r->nrhs);
      bs.push_back(r->b);
      xs.push_back(r->x);
      os.push_back(&r->o);
    }
    int rc = DGASM_OK;
    std::vector<int> done;
    int open_rhs = 0;
    if (active_changed) {
      // count the right-hand sides still open (some finish in their initial step)
      rc = engine->build((int)active.size(), pcs.data(), nr.data(), bs.data(), xs.data(), os.data(), stream, 0);
      if (rc >= 0) rc = engine->read_done(done, &open_rhs);
      if (rc >= 0) rc = engine->build((int)active.size(), pcs.data(), nr.data(), bs.data(), xs.data(), os.data(), stream, open_rhs);
      active_changed = false;
    } else {
      // unchanged batch: the device counter still holds the open right-hand sides
      open_rhs = 1;
    }
    if (rc >= 0 && open_rhs > 0) {
      int ran = 0;
      rc = engine->iterate(ROUND_ITERS, &ran);
    }
    if (rc >= 0) rc = engine->read_done(done, nullptr);
    std::vector<Request*> fin;
    if (rc < 0) {
      fin = active;
    } else {
      for (size_t i = 0; i < active.size(); ++i)
        if (done[i]) fin.push_back(active[i]);
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      ++rounds;
    }
    if (fin.empty()) continue;
    // retire: true residual (requests whose true residual misses rtol restart from it and stay),
    // caller-order solution, statistics
    std::vector<int> rcs(fin.size(), rc);
    if (rc >= 0) {
      std::vector<dgasm_prec_s*> fp;
      std::vector<int> fn;
      std::vector<const double*> fb;
      std::vector<double*> fx;
      std::vector<const dgasm_solve_opts*> fo;
      int total = 0;
      auto gather = [&]() {
        fp.clear(); fn.clear(); fb.clear(); fx.clear(); fo.clear();
        total = 0;
        for (Request* r : fin) {
          fp.push_back(r->pc.get());
          fn.push_back(r->nrhs);
          fb.push_back(r->b);
          fx.push_back(r->x);
          fo.push_back(&r->o);
          total += r->nrhs;
        }
      };
      gather();
      int frc = engine_aux->build((int)fin.size(), fp.data(), fn.data(), fb.data(), fx.data(), fo.data(), stream, 0);
      if (frc >= 0) frc = engine_aux->true_residual();
      int nre = 0;
      if (frc >= 0) frc = engine_aux->restart(&nre);
      if (frc >= 0 && nre > 0) {
        std::vector<int> d2;
        frc = engine_aux->read_done(d2, nullptr);
        if (frc >= 0) {
          std::vector<Request*> keep;
          for (size_t i = 0; i < fin.size(); ++i)
            if (d2[i]) keep.push_back(fin[i]);
          fin.swap(keep);
          rcs.assign(fin.size(), rc);
          active_changed = true;   // restarted requests continue in the next rounds
          if (fin.empty()) continue;
          gather();
          frc = engine_aux->build((int)fin.size(), fp.data(), fn.data(), fb.data(), fx.data(), fo.data(), stream, 0);
        }
      }
      std::vector<dgasm_stats> st(total);
      if (frc >= 0) frc = engine_aux->finish();
      if (frc >= 0 && cudaStreamSynchronize(stream) != cudaSuccess) frc = cuda_error(cudaGetLastError(), "finish");
      if (frc >= 0) {
        std::vector<int> prc;
        engine_aux->collect(st.data(), 0.0, &prc);
        clear_error();
        int off = 0;
        for (size_t i = 0; i < fin.size(); ++i) {
          fin[i]->st.assign(st.begin() + off, st.begin() + off + fin[i]->nrhs);
          double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - fin[i]->t_submit).count();
          for (auto& s : fin[i]->st) s.solve_ms = ms;
          off += fin[i]->nrhs;
          rcs[i] = prc[i];
        }
      } else {
        std::fill(rcs.begin(), rcs.end(), frc);
      }
    }
    std::lock_guard<std::mutex> lk(mu);
    for (size_t i = 0; i < fin.size(); ++i) {
      Request* r = fin[i];
      r->pc.reset();
      active.erase(std::find(active.begin(), active.end(), r));
      finish_request(r, rcs[i], nullptr);
    }
    active_changed = true;
  }
  engine.reset();
  engine_aux.reset();
}

extern "C" int dgasm_server_create(size_t hbm_budget, int max_slots, void* stream, dgasm_server_t* out) {
  clear_error();
  if (!out) return set_error(DGASM_EINVAL, "dgasm_server_create: out is NULL");
  *out = nullptr;
  if (max_slots < 1 || hbm_budget == 0) return set_error(DGASM_EINVAL, "need max_slots >= 1 and a positive budget");
  std::unique_ptr<dgasm_server_s> sv(new (std::nothrow) dgasm_server_s());
  if (!sv) return set_error(DGASM_ENOMEM, "host allocation failed");
  sv->budget = hbm_budget;
  sv->max_slots = max_slots;
  DG_CUDA(cudaGetDevice(&sv->device));
  if (stream) {
    sv->stream = (cudaStream_t)stream;
  } else {
    DG_CUDA(cudaStreamCreateWithFlags(&sv->own_stream, cudaStreamNonBlocking));
    sv->stream = sv->own_stream;
  }
  DG_CUDA(cudaStreamCreateWithFlags(&sv->setup_stream, cudaStreamNonBlocking));
  dgasm_server_s* raw = sv.get();
  sv->th = std::thread([raw] { raw->run(); });
  sv->setup_th = std::thread([raw] { raw->setup_run(); });
  *out = sv.release();
  return DGASM_OK;
}

extern "C" int dgasm_submit(dgasm_server_t sv, dgasm_system_t sys, const dgasm_setup_opts* so, int nrhs,
                            const double* b, double* x, const dgasm_solve_opts* o, uint64_t* ticket) {
  clear_error();
  if (!sv || !sys || !so || !b || !x || !ticket) return set_error(DGASM_EINVAL, "dgasm_submit: NULL argument");
  if (nrhs < 1 || nrhs > KMAX) return set_error(DGASM_EINVAL, "nrhs=%d must lie in [1, %d]", nrhs, KMAX);
  if (o && (o->x0_given || o->host_buffers))
    return set_error(DGASM_EINVAL, "dgasm_submit: device buffers and zero initial guesses only");
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return set_error(DGASM_ENOMEM, "host allocation failed");
  r->sys = sys;
  r->so = *so;
  const int ne = sys->mesh->m.ne;
  if (so->sub_of_elem) {
    r->sub.assign(so->sub_of_elem, so->sub_of_elem + ne);
    r->so.sub_of_elem = r->sub.data();
  }
  if (so->agg_of_elem) {
    r->agg.assign(so->agg_of_elem, so->agg_of_elem + ne);
    r->so.agg_of_elem = r->agg.data();
  }
  r->so.stream = sv->setup_stream;   // the preconditioner is built by the setup thread
  r->nrhs = nrhs;
  r->b = b;
  r->x = x;
  if (o) r->o = *o;
  r->o.stream = sv->stream;
  r->t_submit = std::chrono::steady_clock::now();
  // host planning on the caller's thread, then the footprint estimate
  DG_TRY(prec_plan(sys, &r->so, r->pc));
  const int maxit = r->o.fixed_iters > 0 ? r->o.fixed_iters : (r->o.maxit > 0 ? r->o.maxit : 10000);
  r->bytes = prec_estimate_bytes(*r->pc, nrhs, maxit);
  if (r->bytes > sv->budget)
    return set_error(DGASM_ETOOBIG, "request needs about %zu bytes, more than the whole budget of %zu", r->bytes, sv->budget);
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) return set_error(DGASM_EINVAL, "server is shutting down");
  r->ticket = sv->next_ticket++;
  *ticket = r->ticket;
  sv->queue.push_back(r.get());
  sv->reqs[r->ticket] = std::move(r);
  sv->cv_work.notify_all();
  return DGASM_OK;
}

static int take_result(dgasm_server_s* sv, std::unordered_map<uint64_t, std::unique_ptr<Request>>::iterator it,
                       dgasm_stats* st) {
  Request* r = it->second.get();
  if (st) for (int i = 0; i < r->nrhs && i < (int)r->st.size(); ++i) st[i] = r->st[i];
  int rc = r->rc;
  sv->reqs.erase(it);
  if (rc < 0) return set_error(rc, "request failed with code %d", rc);
  return rc;
}

extern "C" int dgasm_poll(dgasm_server_t sv, uint64_t ticket, dgasm_stats* st) {
  clear_error();
  if (!sv) return set_error(DGASM_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return set_error(DGASM_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  if (it->second->state != Q_DONE) return DGASM_PENDING;
  return take_result(sv, it, st);
}

extern "C" int dgasm_wait(dgasm_server_t sv, uint64_t ticket, int timeout_ms, dgasm_stats* st) {
  clear_error();
  if (!sv) return set_error(DGASM_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto pred = [&] {
    auto it = sv->reqs.find(ticket);
    return it == sv->reqs.end() || it->second->state == Q_DONE;
  };
  if (timeout_ms < 0) sv->cv_done.wait(lk, pred);
  else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
    return set_error(DGASM_ETIMEOUT, "ticket %llu not finished after %d ms", (unsigned long long)ticket, timeout_ms);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return set_error(DGASM_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  return take_result(sv, it, st);
}

extern "C" int dgasm_cancel(dgasm_server_t sv, uint64_t ticket) {
  clear_error();
  if (!sv) return set_error(DGASM_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return set_error(DGASM_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  Request* r = it->second.get();
  if (r->state != Q_QUEUED) return r->state == Q_RUNNING ? DGASM_PENDING : DGASM_OK;
  sv->queue.erase(std::find(sv->queue.begin(), sv->queue.end(), r));
  r->pc.reset();
  r->st.assign(r->nrhs, dgasm_stats{});
  r->rc = DGASM_ECANCELLED;
  r->state = Q_DONE;
  sv->cv_done.notify_all();
  return DGASM_OK;
}

extern "C" int dgasm_server_stats(dgasm_server_t sv, int64_t* done, int64_t* rounds, int64_t* stalls, int64_t* bytes) {
  if (!sv) return set_error(DGASM_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (done) *done = sv->n_done;
  if (rounds) *rounds = sv->rounds;
  if (stalls) *stalls = sv->stalls;
  if (bytes) *bytes = (int64_t)sv->in_use;
  return DGASM_OK;
}

extern "C" int dgasm_server_destroy(dgasm_server_t sv) {
  if (!sv) return DGASM_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    // queued requests are cancelled; admitted ones run to completion
    for (Request* r : sv->queue) {
      r->pc.reset();
      r->rc = DGASM_ECANCELLED;
      r->state = Q_DONE;
    }
    sv->queue.clear();
    sv->cv_work.notify_all();
  }
  if (sv->th.joinable()) sv->th.join();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop_setup = true;
    sv->cv_setup.notify_all();
  }
  if (sv->setup_th.joinable()) sv->setup_th.join();
  if (sv->setup_stream) cudaStreamDestroy(sv->setup_stream);
  if (sv->own_stream) cudaStreamDestroy(sv->own_stream);
  delete sv;
  return DGASM_OK;
}
