// pf_server.cu -- continuous batching of PF solves behind pf_submit / pf_poll.
//
// A fixed pool of worker threads (one per slot) takes requests from a FIFO queue as soon as a
// slot is free and the request's device state fits the remaining HBM budget (first request in
// arrival order that fits).  Each worker owns a non-blocking CUDA stream; it builds the grid,
// runs the same nonlinear solve as pf_nonlinear_solve on that stream, copies the outputs to
// host memory and frees the device state at once, so admitted problems overlap on the GPU and
// memory returns to the budget when a solve ends.  Results are bitwise those of a standalone
// solve on the same problem: the kernels, launch shapes and reduction orders depend only on the
// problem.
#include <cuda_runtime.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pf_gb300.h"

size_t pf_internal_grid_bytes(int nx, int ny, int nz, int accel_depth);  // pf_api.cu

namespace {

struct Request {
  uint64_t ticket = 0;
  int nx = 0, ny = 0, nz = 0;
  double h = 1.0, origin[3] = {0, 0, 0};
  std::vector<double> eps, charges;
  std::vector<uint8_t> solvent;
  std::vector<pf_species> species;
  pf_coeffs coeffs{};
  pf_nl_opts opts{};
  size_t bytes = 0;
  long N = 0;
  // results
  std::vector<double> phi, C, S, G;
  pf_result res{};
  int status = PF_PENDING;
  std::string error;
  bool done = false;
};

}  // namespace

struct pf_server {
  size_t budget = 0, used = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> all;
  std::vector<std::thread> workers;
  bool stop = false;
  uint64_t next = 1;
};

namespace {

void run_request(Request* r, cudaStream_t stream) {
  pf_grid* g = nullptr;
  pf_status s = pf_create_grid(r->nx, r->ny, r->nz, r->h, r->origin, stream, &g);
  if (s == PF_OK) s = pf_set_coeffs(g, &r->coeffs);
  if (s == PF_OK) {
    r->phi.assign(r->N, 0.0);
    r->C.assign((size_t)r->N * r->species.size(), 0.0);
    r->S.assign(r->N, 0.0);
    r->G.assign(r->N, 0.0);
    pf_result res{};
    res.phi_V = r->phi.data();
    res.C_M = r->C.data();
    res.S = r->S.data();
    res.Gamma = r->G.data();
    res.mem = PF_MEM_HOST;
    s = pf_nonlinear_solve(g, &r->opts, &res);
    r->res = res;
  }
  if (s != PF_OK) r->error = pf_last_error();
  pf_destroy_grid(g);
  r->status = s;
  r->res.status = s;
}

void worker_main(pf_server* sv) {
  cudaSetDevice(sv->device);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    Request* pick = nullptr;
    sv->cv.wait(lk, [&] {
      if (sv->stop) return true;
      for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it)
        if (sv->used + (*it)->bytes <= sv->budget) return true;
      return false;
    });
    if (sv->stop) break;
    for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
      if (sv->used + (*it)->bytes <= sv->budget) {
        pick = *it;
        sv->queue.erase(it);
        break;
      }
    }
    if (!pick) continue;
    sv->used += pick->bytes;
    lk.unlock();
    run_request(pick, stream);
    lk.lock();
    sv->used -= pick->bytes;
    pick->done = true;
    sv->cv.notify_all();
  }
  lk.unlock();
  if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

pf_status pf_server_create(size_t hbm_budget_bytes, int max_slots, pf_server** out) {
  if (!out || max_slots < 1 || hbm_budget_bytes == 0) return PF_E_INVAL;
  pf_server* sv = new pf_server();
  sv->budget = hbm_budget_bytes;
  cudaGetDevice(&sv->device);
  for (int i = 0; i < max_slots; ++i) sv->workers.emplace_back(worker_main, sv);
  *out = sv;
  return PF_OK;
}

pf_status pf_submit(pf_server* sv, const pf_request* q, uint64_t* ticket) {
  if (!sv || !q || !ticket) return PF_E_INVAL;
  const pf_coeffs& c = q->coeffs;
  if (q->nx < 2 || q->ny < 2 || q->nz < 3 || !(q->h_A > 0) || !c.eps || !c.solvent || c.n_species < 1 ||
      c.n_species > PF_MAX_SPECIES || !c.species || c.n_charges < 0 || (c.n_charges > 0 && !c.charges))
    return PF_E_INVAL;
  Request* r = new Request();
  r->nx = q->nx;
  r->ny = q->ny;
  r->nz = q->nz;
  r->h = q->h_A;
  for (int a = 0; a < 3; ++a) r->origin[a] = q->origin_A[a];
  r->N = (long)q->nx * q->ny * q->nz;
  r->bytes = pf_internal_grid_bytes(r->nx, r->ny, r->nz, q->opts.accel_depth);
  if (r->bytes > sv->budget) {
    delete r;
    return PF_E_OOM;
  }
  r->eps.assign(c.eps, c.eps + r->N);
  r->solvent.assign(c.solvent, c.solvent + r->N);
  r->charges.assign(c.charges ? c.charges : nullptr, c.charges ? c.charges + 4 * c.n_charges : nullptr);
  r->species.assign(c.species, c.species + c.n_species);
  r->coeffs = c;
  r->coeffs.eps = r->eps.data();
  r->coeffs.solvent = r->solvent.data();
  r->coeffs.charges = r->charges.empty() ? nullptr : r->charges.data();
  r->coeffs.species = r->species.data();
  r->opts = q->opts;
  std::lock_guard<std::mutex> lk(sv->mu);
  r->ticket = sv->next++;
  sv->all[r->ticket] = r;
  sv->queue.push_back(r);
  *ticket = r->ticket;
  sv->cv.notify_all();
  return PF_OK;
}

pf_status pf_poll(pf_server* sv, uint64_t ticket, pf_result* res, int* done) {
  if (!sv || !done) return PF_E_INVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return PF_E_INVAL;
  Request* r = it->second;
  if (!r->done) {
    *done = 0;
    return PF_PENDING;
  }
  if (!res) {
    *done = 1;
    return PF_OK;
  }
  if (res->mem != PF_MEM_HOST) return PF_E_INVAL;
  *done = 1;
  auto put = [](double* dst, const std::vector<double>& src) {
    if (dst && !src.empty()) memcpy(dst, src.data(), src.size() * sizeof(double));
  };
  put(res->phi_V, r->phi);
  put(res->C_M, r->C);
  put(res->S, r->S);
  put(res->Gamma, r->G);
  res->status = r->status;
  res->outer_iters = r->res.outer_iters;
  res->lin_iters_total = r->res.lin_iters_total;
  res->lin_iters_first = r->res.lin_iters_first;
  res->delta = r->res.delta;
  res->time_ms = r->res.time_ms;
  const pf_status st = (pf_status)r->status;
  sv->all.erase(it);
  delete r;
  return st;
}

pf_status pf_server_destroy(pf_server* sv) {
  if (!sv) return PF_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->queue.clear();
  }
  sv->cv.notify_all();
  for (auto& t : sv->workers) t.join();
  for (auto& kv : sv->all) delete kv.second;
  delete sv;
  return PF_OK;
}

}  // extern "C"
