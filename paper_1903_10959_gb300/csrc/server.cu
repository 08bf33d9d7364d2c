// Continuous-batching eigensolve server.
//
// Requests (one periodic / Dirichlet system + a sequence of perturbed
// potentials) wait in a FIFO queue; a scheduler thread admits the head of the
// queue as soon as an execution slot is free and the request's device-memory
// estimate fits in the remaining budget.  Every admitted request runs on its
// own worker thread and CUDA stream, so the kernels of concurrently admitted
// requests overlap on the GPU and a request arriving while others run starts
// as soon as slots and memory allow.  A request keeps its wavefunction block
// and its Chebyshev upper bound resident on the device across its solves: the
// first solve starts from the seeded random block, each following solve
// rebuilds the cell matrices for the perturbed potential and restarts ChFSI
// from the previous eigenvectors (warm start, as in an SCF sequence).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "ctx.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

struct Job {
  uint64_t ticket = 0;
  chfsi_request req{};
  std::vector<double> xyz, depth, width, depth_seq;
  size_t bytes = 0;
  Clock::time_point submitted;
  // results
  bool done = false;
  chfsi_status status = CHFSI_OK;
  std::string err;
  std::vector<double> evals;       // (resolves + 1) x n
  std::vector<double> res, gres;   // max residuals of the lowest n_check pairs per solve
  std::vector<double> solve_ms;    // host wall time per solve
  double queue_ms = 0, first_ms = 0, total_ms = 0;
  size_t used_bytes = 0;
  std::vector<int> iters;          // ChFSI iterations run by each solve
};

}  // namespace

struct chfsi_server {
  size_t budget = 0, used = 0;
  int max_active = 1, active = 0;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv;        // scheduler wake-up
  std::condition_variable done_cv;   // poll wake-up
  std::deque<std::shared_ptr<Job>> queue;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  std::vector<std::thread> workers;
  std::thread scheduler;
  int device = 0;
};

namespace {

// Device bytes a request will hold: what its context allocates (cell
// matrices, their packed binary32 split copy, the mesh tables, the filter,
// rotation and residual scratch, the Gram partial sums and the solver
// workspace, at the default filter block of 200 columns) plus the block X.
size_t estimate_bytes(const chfsi_request& r) {
  const chfsi_mesh_desc& d = r.mesh;
  const size_t p = (size_t)d.p, ne = (p + 1) * (p + 1) * (p + 1);
  size_t ncells = 1, M = 1;
  for (int a = 0; a < 3; ++a) {
    ncells *= (size_t)d.ncell[a];
    M *= d.periodic[a] ? (size_t)d.ncell[a] * p : (size_t)d.ncell[a] * p - 1;
  }
  const bool mixed = r.prec != CHFSI_FP64;
  const size_t es = mixed ? 4 : 8, n = (size_t)r.n, B = std::min<size_t>(200, n);
  const size_t mt = (ne + 127) / 128, nk = (ne + 7) / 8;
  size_t b = ncells * ne * ne * 8;                                  // binary64 cell matrices
  if (mixed) b += ncells * nk * 2 * mt * 1024 * 4;                  // packed hi / lo TF32 copies
  if (r.prec == CHFSI_MIXED_BF16X3) b += ncells * ((ne + 15) / 16) * 3 * mt * 4096;   // BF16x3 terms
  if (r.prec == CHFSI_MIXED_F16X2) b += ncells * ((ne + 15) / 16) * 2 * mt * 4096 + ncells * 4 + n * 12;
  b += ncells * ne * 9 + ncells * 4 + M * 16 + 4096;                // dof map, modes, rows, mass
  b += M * n * es;                                                  // X
  b += std::max(M * n * es, M * B * 16);                            // rotation / binary64 pair
  b += M * B * es + M * B * 8;                                      // filter block, binary64 apply
  if (mixed) b += ncells * ne * B * 4;                              // dense cell blocks R_e
  b += std::max(n * n * 128 + (mixed ? ((size_t)64 << 20) : 0), n * 12288);  // Gram partials
  b += n * n * 8 * 5 + n * 64 + 4096;                               // N x N (S / H^, L^{-1}), solver workspace
  b += M * 24 + ((size_t)16 << 20);                                 // vectors, library slack
  if (mixed && r.polish_iters > 0)                                  // binary64 polish: staging
    b += M * n * 8 + M * n * 4 + M * B * 4;                         //  block, rotation, filter
  return b;
}

void run_job(chfsi_server* sv, std::shared_ptr<Job> job) {
  Job& J = *job;
  const chfsi_request& r = J.req;
  cudaSetDevice(sv->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  chfsi_ctx* ctx = nullptr;
  void* X = nullptr;
  const size_t es = r.prec == CHFSI_FP64 ? 8 : 4;
  const bool polish = r.polish_iters > 0 && r.prec != CHFSI_FP64;
  auto finish = [&](chfsi_status s, const std::string& msg) {
    J.status = s;
    J.err = msg;
  };
  chfsi_status s = chfsi_create(&r.mesh, st, &ctx);
  if (s != CHFSI_OK) {
    finish(s, "create");
  } else {
    const int64_t M = chfsi_num_dofs(ctx);
    const int n = r.n;
    J.evals.assign((size_t)(r.resolves + 1) * n, 0.0);
    double b = 0.0;
    if (cudaMalloc(&X, (size_t)M * n * es) != cudaSuccess) {
      cudaGetLastError();
      finish(CHFSI_ERR_OOM, "X");
    } else {
      for (int k = 0; k <= r.resolves && J.status == CHFSI_OK; ++k) {
        const double* dep = k == 0 ? J.depth.data() : J.depth_seq.data() + (size_t)(k - 1) * r.nwells;
        auto t0 = Clock::now();
        s = chfsi_set_potential_gaussians(ctx, r.nwells, J.xyz.data(), dep, J.width.data());
        if (s == CHFSI_OK) s = chfsi_build(ctx);
        if (s == CHFSI_OK && k == 0) {
          s = chfsi_bounds(ctx, 20, r.seed, &b);
          b *= 1.02;   // margin: later potentials move the spectrum slightly
          if (s == CHFSI_OK) s = chfsi_fill_uniform(ctx, X, n, M, n, r.seed, 1, r.prec);
        }
        int done = 0;
        const int its = k == 0 ? r.iters : r.warm_iters;
        double* ev = J.evals.data() + (size_t)k * n;
        if (s == CHFSI_OK && polish)
          s = chfsi_solve_polish(ctx, (float*)X, n, n, its, r.degree, b, r.tol, r.n_check, r.prec,
                                 r.polish_iters, r.polish_degree > 0 ? r.polish_degree : r.degree,
                                 nullptr, 0, ev, &done);
        else if (s == CHFSI_OK)
          s = chfsi_solve(ctx, X, n, n, its, r.degree, b, r.tol, r.n_check, r.prec, ev, &done);
        J.iters.push_back(done);
        double mx = 0.0, gmx = 0.0;
        if (s == CHFSI_OK && r.n_check > 0) {
          std::vector<double> res(r.n_check), gres(r.n_check);
          s = chfsi_residuals(ctx, X, n, r.n_check, r.prec, J.evals.data() + (size_t)k * n,
                              res.data(), gres.data());
          for (int i = 0; i < r.n_check; ++i) {
            mx = std::max(mx, res[i]);
            gmx = std::max(gmx, gres[i]);
          }
        }
        J.res.push_back(mx);
        J.gres.push_back(gmx);
        J.solve_ms.push_back(ms_since(t0));
        if (k == 0) J.first_ms = ms_since(J.submitted);
        if (s != CHFSI_OK) finish(s, chfsi_last_error(ctx));
      }
      J.used_bytes = (size_t)chfsi_device_bytes(ctx) + (size_t)M * n * es;
    }
  }
  if (X) cudaFree(X);
  if (ctx) chfsi_destroy(ctx);
  cudaStreamDestroy(st);
  std::lock_guard<std::mutex> lk(sv->mu);
  J.total_ms = ms_since(J.submitted);
  J.done = true;
  sv->used -= J.bytes;
  sv->active -= 1;
  sv->cv.notify_all();
  sv->done_cv.notify_all();
}

void scheduler_loop(chfsi_server* sv) {
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    sv->cv.wait(lk, [&] {
      if (sv->stop) return true;
      if (sv->queue.empty() || sv->active >= sv->max_active) return false;
      const auto& h = sv->queue.front();
      return sv->used + h->bytes <= sv->budget || sv->active == 0;
    });
    if (sv->stop && sv->queue.empty()) return;
    if (sv->stop) {   // fail what is still queued
      for (auto& j : sv->queue) {
        j->status = CHFSI_ERR_STATE;
        j->err = "server stopped";
        j->done = true;
      }
      sv->queue.clear();
      sv->done_cv.notify_all();
      return;
    }
    auto job = sv->queue.front();
    sv->queue.pop_front();
    if (job->bytes > sv->budget) {
      job->status = CHFSI_ERR_OOM;
      job->err = "request exceeds the device-memory budget";
      job->done = true;
      sv->done_cv.notify_all();
      continue;
    }
    sv->used += job->bytes;
    sv->active += 1;
    job->queue_ms = ms_since(job->submitted);
    sv->workers.emplace_back(run_job, sv, job);
  }
}

}  // namespace

extern "C" {

chfsi_status chfsi_server_create(size_t hbm_budget_bytes, int max_active, chfsi_server** out) {
  if (!out || max_active < 1 || hbm_budget_bytes == 0) return CHFSI_ERR_ARG;
  chfsi_server* sv = new chfsi_server();
  sv->budget = hbm_budget_bytes;
  sv->max_active = max_active;
  cudaGetDevice(&sv->device);
  sv->scheduler = std::thread(scheduler_loop, sv);
  *out = sv;
  return CHFSI_OK;
}

chfsi_status chfsi_server_submit(chfsi_server* sv, const chfsi_request* r, uint64_t* ticket) {
  if (!sv || !r || !ticket || r->n < 1 || r->nwells < 0 || r->resolves < 0 || r->degree < 1 ||
      r->iters < 0 || r->warm_iters < 0 || (r->nwells > 0 && (!r->xyz || !r->depth || !r->width)) ||
      (r->resolves > 0 && r->nwells > 0 && !r->depth_seq) || r->resolves + 1 > CHFSI_MAX_SOLVES ||
      r->mesh.p < 1 || r->n_check > r->n || r->polish_iters < 0 || r->polish_degree < 0)
    return CHFSI_ERR_ARG;
  auto job = std::make_shared<Job>();
  job->req = *r;
  job->xyz.assign(r->xyz, r->xyz + 3 * (size_t)r->nwells);
  job->depth.assign(r->depth, r->depth + r->nwells);
  job->width.assign(r->width, r->width + r->nwells);
  if (r->resolves > 0)
    job->depth_seq.assign(r->depth_seq, r->depth_seq + (size_t)r->resolves * r->nwells);
  job->req.xyz = job->req.depth = job->req.width = job->req.depth_seq = nullptr;
  job->bytes = estimate_bytes(*r);
  job->submitted = Clock::now();
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) return CHFSI_ERR_STATE;
  job->ticket = sv->next_ticket++;
  sv->jobs[job->ticket] = job;
  sv->queue.push_back(job);
  *ticket = job->ticket;
  sv->cv.notify_all();
  return CHFSI_OK;
}

chfsi_status chfsi_server_poll(chfsi_server* sv, uint64_t ticket, int wait, chfsi_result* out,
                               double* evals_out) {
  if (!sv || !out) return CHFSI_ERR_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return CHFSI_ERR_ARG;
  auto job = it->second;
  if (wait) sv->done_cv.wait(lk, [&] { return job->done; });
  std::memset(out, 0, sizeof(*out));
  out->done = job->done ? 1 : 0;
  if (!job->done) return CHFSI_OK;
  out->status = job->status;
  out->nsolves = (int)job->solve_ms.size();
  out->queue_ms = job->queue_ms;
  out->first_ms = job->first_ms;
  out->total_ms = job->total_ms;
  out->est_bytes = job->bytes;
  out->used_bytes = job->used_bytes;
  std::snprintf(out->error, sizeof(out->error), "%s", job->err.c_str());
  for (int k = 0; k < out->nsolves && k < CHFSI_MAX_SOLVES; ++k) {
    out->solve_ms[k] = job->solve_ms[k];
    out->max_residual[k] = job->res[k];
    out->max_gresidual[k] = job->gres[k];
    out->iters[k] = job->iters[k];
  }
  if (evals_out && !job->evals.empty())
    std::memcpy(evals_out, job->evals.data(), job->evals.size() * sizeof(double));
  return CHFSI_OK;
}

size_t chfsi_server_estimate(const chfsi_request* r) { return r ? estimate_bytes(*r) : 0; }

chfsi_status chfsi_server_destroy(chfsi_server* sv) {
  if (!sv) return CHFSI_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv.notify_all();
  }
  sv->scheduler.join();
  for (auto& w : sv->workers) w.join();
  delete sv;
  return CHFSI_OK;
}

}  // extern "C"
