// pf_server.cu -- continuous batching of PF solves behind pf_submit / pf_poll.
//
// One scheduler thread owns a batched engine (pf_batch.cu).  Between two engine steps it admits queued
// requests, first fit in arrival order, while a slot is free and the request's device state fits the
// remaining HBM budget: it creates the request's grid on the engine's stream and adds it as a member.
// Every engine step runs one outer iteration of all members in shared batched launches (members that
// just joined get their operators and initial potential first), so requests that arrive while others are
// on the GPU join the running launches at the next step.  A member that finishes has its outputs written
// to host memory, its grid freed at once (its bytes return to the budget), and its ticket completed.  The
// state of every request in flight (potential, concentrations, Krylov vectors) stays on the device.
// A request's arithmetic depends only on the request (the engine splits every grid into blocks the same
// way), so its result is bitwise that of a batch of this problem alone with the engine's tiles per block.
#include <cuda_runtime.h>
#include <string.h>

#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pf_grid.cuh"

size_t pf_internal_grid_bytes(int nx, int ny, int nz, int accel_depth);  // pf_api.cu

namespace {

struct Request {
  uint64_t ticket = 0;
  int nx = 0, ny = 0, nz = 0;
  double h = 1.0, origin[3] = {0, 0, 0};
  std::vector<double> eps, charges, phi0;
  std::vector<uint8_t> solvent;
  std::vector<pf_species> species;
  pf_coeffs coeffs{};
  pf_nl_opts opts{};
  size_t bytes = 0;
  long N = 0;
  pf_grid* g = nullptr;  // while in flight
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
  int device = 0, max_slots = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> all;
  std::thread scheduler;
  bool stop = false;
  uint64_t next = 1;
};

namespace {

void complete(pf_server* sv, Request* r, pf_status s, const std::string& err) {
  if (r->g) pf_destroy_grid(r->g);
  r->g = nullptr;
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->used -= r->bytes;
  r->status = s;
  r->res.status = s;
  r->error = err;
  r->done = true;
  sv->cv.notify_all();
}

// Creates the request's grid on the engine's stream and makes it a member; false (request completed
// with the failure) when that fails.
bool join(pf_server* sv, pf_batch* E, Request* r) {
  pf_status s = pf_create_grid(r->nx, r->ny, r->nz, r->h, r->origin, pfi::engine_stream(E), &r->g);
  if (s == PF_OK) s = pf_set_coeffs(r->g, &r->coeffs);
  if (s == PF_OK && !r->phi0.empty()) {
    s = pf_set_potential(r->g, r->phi0.data(), PF_MEM_HOST);
    r->opts.warm_start = 1;
  }
  if (s == PF_OK) {
    r->phi.assign(r->N, 0.0);
    r->C.assign((size_t)r->N * r->species.size(), 0.0);
    r->S.assign(r->N, 0.0);
    r->G.assign(r->N, 0.0);
    r->res = pf_result{};
    r->res.phi_V = r->phi.data();
    r->res.C_M = r->C.data();
    r->res.S = r->S.data();
    r->res.Gamma = r->G.data();
    r->res.mem = PF_MEM_HOST;
    s = pfi::engine_add(E, r->g, &r->res, r->opts, (long long)r->ticket);
  }
  if (s != PF_OK) {
    complete(sv, r, s, pf_last_error());
    return false;
  }
  return true;
}

void scheduler_main(pf_server* sv) {
  cudaSetDevice(sv->device);
  pf_batch* E = nullptr;
  pf_status es = pfi::engine_create(sv->max_slots, &E);  // while not PF_OK, every admitted request fails with it
  std::unordered_map<long long, Request*> inflight;
  for (;;) {
    std::vector<Request*> admit;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      auto admissible = [&] {
        if ((int)inflight.size() >= sv->max_slots) return false;
        for (Request* r : sv->queue)
          if (sv->used + r->bytes <= sv->budget) return true;
        return false;
      };
      sv->cv.wait(lk, [&] { return sv->stop || !inflight.empty() || admissible(); });
      if (sv->stop) break;
      for (auto it = sv->queue.begin(); it != sv->queue.end();) {
        if ((int)(inflight.size() + admit.size()) >= sv->max_slots) break;
        if (sv->used + (*it)->bytes <= sv->budget) {
          sv->used += (*it)->bytes;
          admit.push_back(*it);
          it = sv->queue.erase(it);
        } else {
          ++it;
        }
      }
    }
    for (Request* r : admit) {
      if (es != PF_OK) {
        complete(sv, r, es, "the serving engine could not be created");
        continue;
      }
      if (join(sv, E, r)) inflight[(long long)r->ticket] = r;
    }
    if (inflight.empty()) continue;
    std::vector<long long> fin;
    const pf_status s = pfi::engine_step(E, &fin);
    if (s != PF_OK) {
      // a failure of the engine itself (not of a problem): fail every request in flight and start afresh
      const std::string err = pf_last_error();
      pf_batch_destroy(E);
      E = nullptr;
      for (auto& kv : inflight) complete(sv, kv.second, s, err);
      inflight.clear();
      es = pfi::engine_create(sv->max_slots, &E);
      if (es != PF_OK) E = nullptr;  // later requests are completed with the failure instead of waiting
      continue;
    }
    for (long long t : fin) {
      Request* r = inflight[t];
      inflight.erase(t);
      complete(sv, r, (pf_status)r->res.status, r->res.status == PF_OK ? "" : "solve failed");
    }
  }
  for (auto& kv : inflight) {
    if (kv.second->g) pf_destroy_grid(kv.second->g);
    kv.second->g = nullptr;
  }
  if (E) pf_batch_destroy(E);
}

}  // namespace

extern "C" {

pf_status pf_server_create(size_t hbm_budget_bytes, int max_slots, pf_server** out) {
  if (!out || max_slots < 1 || hbm_budget_bytes == 0) return PF_E_INVAL;
  pf_server* sv = new pf_server();
  sv->budget = hbm_budget_bytes;
  sv->max_slots = max_slots;
  cudaGetDevice(&sv->device);
  sv->scheduler = std::thread(scheduler_main, sv);
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
  if (q->phi0_V) r->phi0.assign(q->phi0_V, q->phi0_V + r->N);
  else if (r->opts.warm_start) {
    delete r;
    return PF_E_INVAL;  // a fresh grid has no potential to start from
  }
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
  if (sv->scheduler.joinable()) sv->scheduler.join();
  for (auto& kv : sv->all) delete kv.second;
  delete sv;
  return PF_OK;
}

}  // extern "C"
