// Batched mode: many independent FCM problems of uneven grid size, degree
// and geometry.  Every instance is a full handle (its own level hierarchy,
// CUDA stream and captured V-cycle graphs); a pool of host worker threads
// sets instances up and drives their solves, so the GPU runs many
// instances' kernels concurrently on their streams.  Instances never
// exchange data.
#include <atomic>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "fcm_internal.h"

struct fcm_batch {
  std::vector<fcm_handle*> h;
};

namespace {

int worker_count(int n, int threads) {
  int t = threads > 0 ? threads : (int)std::thread::hardware_concurrency();
  if (t < 1) t = 1;
  if (t > 64) t = 64;
  return t < n ? t : n;
}

// Run f(i) for i in [0, n) on `threads` workers; returns the first failing
// status (in instance order) and its message.
template <typename F>
fcm_status run_pool(int n, int threads, F&& f, std::string* msg) {
  std::vector<fcm_status> st(n, FCM_OK);
  std::vector<std::string> err(n);
  std::atomic<int> next(0);
  auto work = [&]() {
    for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) {
      st[i] = f(i);
      if (st[i] != FCM_OK) err[i] = fcm_last_error();
    }
  };
  int t = worker_count(n, threads);
  std::vector<std::thread> pool;
  for (int k = 1; k < t; ++k) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  for (int i = 0; i < n; ++i)
    if (st[i] != FCM_OK) {
      *msg = "instance " + std::to_string(i) + ": " + err[i];
      return st[i];
    }
  return FCM_OK;
}

}  // namespace

extern "C" {

fcm_status fcm_setup_batch(int n, const fcm_grid* grids, const fcm_geometry* geoms,
                           const fcm_physics* phys, const fcm_solver_opts* opts, int threads,
                           void* stream, fcm_batch** out) {
  if (!out || n < 1 || !grids || !geoms || !phys || !opts) {
    fcm::set_last_error("fcm_setup_batch: invalid argument");
    return FCM_E_INVALID;
  }
  *out = nullptr;
  std::unique_ptr<fcm_batch> b(new fcm_batch());
  b->h.assign(n, nullptr);
  std::string msg;
  fcm_status st = run_pool(
      n, threads,
      [&](int i) {
        return fcm_setup(&grids[i], &geoms[i], &phys[i], &opts[i], stream, &b->h[i]);
      },
      &msg);
  if (st != FCM_OK) {
    for (fcm_handle* h : b->h)
      if (h) fcm_destroy(h);
    fcm::set_last_error(msg.c_str());
    return st;
  }
  *out = b.release();
  return FCM_OK;
}

fcm_status fcm_batch_size(const fcm_batch* b, int* n) {
  if (!b || !n) {
    fcm::set_last_error("fcm_batch_size: null argument");
    return FCM_E_INVALID;
  }
  *n = (int)b->h.size();
  return FCM_OK;
}

fcm_status fcm_batch_handle(const fcm_batch* b, int i, fcm_handle** h) {
  if (!b || !h || i < 0 || i >= (int)b->h.size()) {
    fcm::set_last_error("fcm_batch_handle: invalid argument");
    return FCM_E_INVALID;
  }
  *h = b->h[i];
  return FCM_OK;
}

fcm_status fcm_pcg_solve_batch(fcm_batch* b, double* const* x_dev, double rtol, int maxit,
                               int prec, int threads, fcm_info* infos) {
  if (!b || !x_dev) {
    fcm::set_last_error("fcm_pcg_solve_batch: null argument");
    return FCM_E_INVALID;
  }
  const int n = (int)b->h.size();
  for (int i = 0; i < n; ++i)
    if (!x_dev[i]) {
      fcm::set_last_error("fcm_pcg_solve_batch: x_dev has a NULL entry");
      return FCM_E_INVALID;
    }
  // lockstep: all instances in flight, driven by this thread (threads < 0:
  // one graph launch per CG phase for all running instances)
  if (threads <= 0)
    return fcm::pcg_solve_lockstep(b->h.data(), n, x_dev, rtol, maxit, prec, infos, threads < 0);
  std::string msg;
  fcm_status st = run_pool(
      n, threads,
      [&](int i) {
        return fcm_pcg_solve(b->h[i], nullptr, x_dev[i], rtol, maxit, prec,
                             infos ? &infos[i] : nullptr);
      },
      &msg);
  if (st != FCM_OK) fcm::set_last_error(msg.c_str());
  return st;
}

void fcm_batch_destroy(fcm_batch* b) {
  if (!b) return;
  for (fcm_handle* h : b->h)
    if (h) fcm_destroy(h);
  delete b;
}

}  // extern "C"
