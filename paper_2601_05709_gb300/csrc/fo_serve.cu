// Request server: continuous batching of optimisation-step requests of uneven sizes on one GPU.
//
// A request is one step of the level-set algorithm without the transport (state solve,
// explicit adjoint solve, cost and constraint, shape derivative, velocity) on its own box
// mesh.  Requests wait in a FIFO queue.  `executors` host threads each own a library context
// with its own CUDA stream; an idle executor admits the request at the head of the queue as
// soon as the device memory of the requests in flight plus the head's own estimate fits in
// the budget, runs it through the public calls on its context, and frees everything before
// taking the next.  Requests on different executors overlap on the device: a small
// request's persistent kernels occupy a few SMs and run beside the others.  Each request's
// launches depend on its own sizes only, so its results are the same alone and in a mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fo_internal.cuh"

namespace {

struct Job {
  uint64_t ticket = 0;
  fo_request rq{};
  std::vector<double> f, centers, phi;   // copies of the request's host arrays
  size_t bytes = 0;
  int state = 0;                          // 0 queued, 1 running, 2 done
  fo_result res{};
};

double now_ms(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct fo_server {
  fo_server_opts o{};
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_admit, cv_done;
  std::deque<Job *> queue;
  std::unordered_map<uint64_t, Job *> jobs;
  uint64_t next_ticket = 1;
  size_t bytes_in_flight = 0;
  int in_flight = 0;
  bool stopping = false;
  fo_server_stats st{};
  std::vector<std::thread> threads;
};

extern "C" void fo_server_opts_default(fo_server_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->executors = 8;
  o->mem_budget = (size_t)8 << 30;
  o->queue_capacity = 4096;
  o->dry_run_ms = 0.0;
  o->grid_share = 4;
  o->policy = FO_SERVE_FIFO;
}

extern "C" size_t fo_request_device_bytes(const fo_request *rq) {
  if (!rq || (rq->dim != 2 && rq->dim != 3)) return 0;
  Grid g0;
  const double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  if (!fo_grid_make(rq->dim, rq->n, lo, hi, g0)) return 0;
  // multigrid where asked for and where the grid coarsens far enough to use it; solver
  // scratch: multigrid CG 6 (state) / 7 (velocity) vectors, Jacobi CG 8, mixed refinement 11
  const int nc = rq->model.kind == FO_ELASTIC ? rq->dim : 1;
  const bool smg = rq->state.precond == FO_PC_MG && fo_mg_applicable(g0, nc);
  const bool vmg = rq->velocity.precond == FO_PC_MG && fo_mg_applicable(g0, rq->dim);
  const int svecs = smg ? 6 : (rq->state.precision == FO_MIXED ? 11 : 8);
  size_t b = fo_problem_footprint(rq->dim, rq->n, rq->model.kind, svecs, vmg ? 7 : 8, rq->n_bumps);
  if (smg) b += fo_mg_bytes(rq->dim, rq->n, nc, nc * nc, false, rq->state.mg_bf16 != 0);
  if (vmg) b += fo_mg_bytes(rq->dim, rq->n, rq->dim, rq->dim, true, rq->velocity.mg_bf16 != 0);
  return b;
}

static bool request_valid(const fo_request *rq) {
  if (rq->dim != 2 && rq->dim != 3) return false;
  for (int a = 0; a < rq->dim; ++a)
    if (rq->n[a] < 1 || !(rq->hi[a] > rq->lo[a])) return false;
  if (rq->model.kind != FO_HEAT && rq->model.kind != FO_ELASTIC) return false;
  if (rq->model.n_inst != 0) return false;
  if (rq->n_bumps > 0) return rq->bump_centers && rq->bump_width > 0;
  return rq->phi != nullptr;
}

// The device work of one request on the executor's context.
static void run_request(fo_ctx *ctx, Job *j) {
  fo_result &r = j->res;
  const fo_request &rq = j->rq;
  auto chk = [&](fo_status s) {
    if (s != FO_OK && (r.status == FO_OK || r.status == FO_ENOCONV) && s != FO_ENOCONV) {
      r.status = s;
      snprintf(r.message, sizeof r.message, "%s", fo_last_error(ctx));
    } else if (s == FO_ENOCONV && r.status == FO_OK) {
      r.status = s;
    }
    return r.status == FO_OK || r.status == FO_ENOCONV;
  };
  fo_mesh *m = nullptr;
  fo_problem *p = nullptr;
  fo_model_desc desc = rq.model;
  desc.f_nodal = j->f.empty() ? nullptr : j->f.data();
  double J = 0, C = 0, Btt = 0;
  if (chk(fo_mesh_box(ctx, rq.dim, rq.n, rq.lo, rq.hi, &m)) && chk(fo_problem_create(m, &desc, &p))) {
    fo_mesh_info mi;
    fo_mesh_query(m, &mi);
    r.dofs = mi.num_nodes * (desc.kind == FO_ELASTIC ? rq.dim : 1);
    bool ok = rq.n_bumps > 0 ? chk(fo_levelset_bumps(p, rq.n_bumps, j->centers.data(), rq.bump_width, rq.bump_offset))
                             : chk(fo_set_levelset(p, j->phi.data(), 0));
    ok = ok && chk(fo_coefficients(p));
    ok = ok && chk(fo_state_solve(p, &rq.state, &r.state));
    ok = ok && chk(fo_adjoint_solve(p, &rq.state, &r.adjoint));
    ok = ok && chk(fo_functionals(p, &J, &C));
    ok = ok && chk(fo_shape_derivative(p, rq.lambda, nullptr));
    ok = ok && chk(fo_descent(p, &rq.velocity, &Btt, &r.velocity));
    if (ok && rq.theta_out) chk(fo_get(p, FO_FIELD_THETA, rq.theta_out));
  }
  r.J = J;
  r.C = C;
  r.Btt = Btt;
  if (p) fo_problem_destroy(p);
  if (m) fo_mesh_destroy(m);
}

static void executor(fo_server *s) {
  fo_ctx *ctx = nullptr;
  if (s->o.dry_run_ms <= 0.0 && fo_ctx_create(s->device, nullptr, 0, &ctx) != FO_OK) ctx = nullptr;
  if (ctx) fo_ctx_set_grid_share(ctx, s->o.grid_share);
  for (;;) {
    Job *j = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // the request to admit next: the queue's head (FIFO), or its smallest footprint (ties in
      // submission order), which then must fit in what the budget leaves
      auto pick = [&]() -> std::deque<Job *>::iterator {
        if (s->queue.empty()) return s->queue.end();
        auto it = s->queue.begin();
        if (s->o.policy == FO_SERVE_SMALLEST_FIRST)
          for (auto k = s->queue.begin(); k != s->queue.end(); ++k)
            if ((*k)->bytes < (*it)->bytes) it = k;
        return s->bytes_in_flight + (*it)->bytes <= s->o.mem_budget ? it : s->queue.end();
      };
      std::deque<Job *>::iterator it;
      s->cv_admit.wait(lk, [&] { return s->stopping || (it = pick()) != s->queue.end(); });
      if (s->stopping) break;
      j = *it;
      s->queue.erase(it);
      j->state = 1;
      j->res.start_ms = now_ms(s->t0);
      s->bytes_in_flight += j->bytes;
      s->in_flight += 1;
      s->st.peak_in_flight = std::max<int64_t>(s->st.peak_in_flight, s->in_flight);
      s->st.peak_bytes = std::max(s->st.peak_bytes, s->bytes_in_flight);
    }
    if (s->o.dry_run_ms > 0.0) {
      std::this_thread::sleep_for(std::chrono::duration<double, std::milli>(s->o.dry_run_ms));
    } else if (!ctx) {
      j->res.status = FO_ECUDA;
      snprintf(j->res.message, sizeof j->res.message, "executor could not create a context");
    } else {
      run_request(ctx, j);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      j->res.end_ms = now_ms(s->t0);
      j->state = 2;
      s->bytes_in_flight -= j->bytes;
      s->in_flight -= 1;
      s->st.completed += 1;
      if (j->res.status != FO_OK && j->res.status != FO_ENOCONV) s->st.failed += 1;
    }
    s->cv_admit.notify_all();
    s->cv_done.notify_all();
  }
  if (ctx) fo_ctx_destroy(ctx);
}

extern "C" fo_status fo_server_create(fo_ctx *ctx, const fo_server_opts *opts, fo_server **out) {
  if (!out) return FO_EINVAL;
  *out = nullptr;
  fo_server_opts o;
  fo_server_opts_default(&o);
  if (opts) o = *opts;
  if (!ctx && !(o.dry_run_ms > 0.0)) return FO_EINVAL;
  if (o.executors < 1 || o.executors > 256 || o.queue_capacity < 1 || o.mem_budget == 0 || o.grid_share < 1 ||
      o.grid_share > 16 || (o.policy != FO_SERVE_FIFO && o.policy != FO_SERVE_SMALLEST_FIRST))
    return ctx ? fo_fail(ctx, FO_EINVAL, "bad server options") : FO_EINVAL;
  fo_server *s = new fo_server();
  s->o = o;
  s->device = ctx ? ctx->device : 0;
  s->t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < o.executors; ++i) s->threads.emplace_back(executor, s);
  *out = s;
  return FO_OK;
}

extern "C" fo_status fo_server_destroy(fo_server *s) {
  if (!s) return FO_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    for (Job *j : s->queue) {
      j->state = 2;
      j->res.status = FO_ESTATE;
      snprintf(j->res.message, sizeof j->res.message, "server destroyed before the request ran");
    }
    s->queue.clear();
  }
  s->cv_admit.notify_all();
  s->cv_done.notify_all();
  for (auto &t : s->threads) t.join();   // a running request ends with its own (bounded) solves
  for (auto &e : s->jobs) delete e.second;
  delete s;
  return FO_OK;
}

extern "C" fo_status fo_submit(fo_server *s, const fo_request *rq, uint64_t *ticket) {
  if (!s || !rq || !ticket) return FO_EINVAL;
  if (!request_valid(rq)) return FO_EINVAL;
  const size_t bytes = fo_request_device_bytes(rq);
  Job *j = new Job();
  j->rq = *rq;
  j->bytes = bytes;
  long long NN = 1;
  for (int a = 0; a < rq->dim; ++a) NN *= rq->n[a] + 1;
  if (rq->model.f_nodal) j->f.assign(rq->model.f_nodal, rq->model.f_nodal + NN);
  if (rq->n_bumps > 0) j->centers.assign(rq->bump_centers, rq->bump_centers + (size_t)rq->n_bumps * rq->dim);
  else j->phi.assign(rq->phi, rq->phi + NN);
  j->rq.model.f_nodal = nullptr;
  j->rq.bump_centers = nullptr;
  j->rq.phi = nullptr;
  j->res.device_bytes = bytes;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) {
      delete j;
      return FO_ESTATE;
    }
    if (bytes > s->o.mem_budget) {
      s->st.rejected += 1;
      delete j;
      return FO_ENOMEM_BUDGET;
    }
    if ((int)s->queue.size() >= s->o.queue_capacity) {
      s->st.rejected += 1;
      delete j;
      return FO_EBUSY;
    }
    j->ticket = s->next_ticket++;
    j->res.submit_ms = now_ms(s->t0);
    s->jobs[j->ticket] = j;
    s->queue.push_back(j);
    s->st.submitted += 1;
    *ticket = j->ticket;
  }
  s->cv_admit.notify_one();
  return FO_OK;
}

extern "C" fo_status fo_poll(fo_server *s, uint64_t ticket, fo_result *res, int *done) {
  if (!s || !done) return FO_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return FO_EINVAL;
  *done = it->second->state == 2;
  if (*done && res) *res = it->second->res;
  return FO_OK;
}

extern "C" fo_status fo_wait(fo_server *s, uint64_t ticket, double timeout_s, fo_result *res) {
  if (!s || !(timeout_s >= 0)) return FO_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return FO_EINVAL;
  Job *j = it->second;
  const auto limit = std::chrono::duration<double>(std::min(timeout_s, 1e7));
  if (!s->cv_done.wait_for(lk, limit, [&] { return j->state == 2; })) return FO_ETIMEOUT;
  if (res) *res = j->res;
  return FO_OK;
}

extern "C" fo_status fo_release(fo_server *s, uint64_t ticket) {
  if (!s) return FO_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end() || it->second->state != 2) return FO_EINVAL;
  delete it->second;
  s->jobs.erase(it);
  return FO_OK;
}

extern "C" fo_status fo_server_get_stats(fo_server *s, fo_server_stats *out) {
  if (!s || !out) return FO_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  return FO_OK;
}
