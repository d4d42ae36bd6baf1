// Serving loop: continuous batching of impurity solves on one GPU.
//
// Independent impurity problems (the paper's task parallelism over
// inequivalent sites, Sec. 6.9) become requests.  A pool of worker threads,
// each owning one CUDA stream, takes requests in arrival order as soon as a
// slot is free and the request's estimated device memory fits the budget;
// requests that arrive while others are on the GPU are admitted as slots and
// memory free up, and their kernels overlap on the device.  Results stay in
// the server until polled.  Every wait on the host is bounded.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

ed_status ed_solve_impl(const ed_model *model, int nup, int ndw, const ed_solve_opts *o,
                        ed_solve_result *res, double *host_G, void *d_psi_out, cudaStream_t cs);

namespace {

struct OwnedRequest {
  uint64_t ticket = 0;
  ed_model model;
  std::vector<double> e_imp, e_bath, v_bath;
  int nup = 0, ndw = 0;
  ed_solve_opts opts;
  int64_t mem_estimate = 0;
  double t_submit = 0;
};

struct Done {
  ed_result res;
  std::vector<double> G;
};

double clock_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

uint64_t binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  uint64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
  return r;
}

}  // namespace

struct ed_server_s {
  ed_server_opts opts;
  int device = 0;
  int64_t budget = 0;
  int64_t in_use = 0;
  int injected_failures = 0;
  bool stopping = false;
  uint64_t next_ticket = 1;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work;   // workers wait for admissible requests
  std::condition_variable cv_done;   // ed_wait waits for results
  std::deque<std::unique_ptr<OwnedRequest>> queue;
  std::unordered_map<uint64_t, int> running;  // ticket -> 1
  std::unordered_map<uint64_t, Done> done;
  std::vector<std::thread> workers;

  void worker_main();
};

// Device bytes a solve needs besides the small sector tables: three Lanczos
// vectors and psi in the ground precision, two FP64 vectors for the polish,
// three vectors of the largest neighbour sector for each Green's function
// chain that runs concurrently (up to 8), plus a fixed allowance.
static int64_t estimate_bytes(const OwnedRequest &r) {
  const int ns = r.model.norb * (r.model.nbath + 1);
  const int64_t d = (int64_t)binom(ns, r.nup) * (int64_t)binom(ns, r.ndw);
  const int64_t dn = std::max<int64_t>(
      std::max<int64_t>((int64_t)binom(ns, r.nup + 1) * binom(ns, r.ndw),
                        (int64_t)binom(ns, r.nup - 1) * binom(ns, r.ndw)),
      std::max<int64_t>((int64_t)binom(ns, r.nup) * binom(ns, r.ndw + 1),
                        (int64_t)binom(ns, r.nup) * binom(ns, r.ndw - 1)));
  const int elem = r.opts.lanczos.precision == ED_FP64 ? 8 : 4;
  const int gelem = r.opts.gf_precision == ED_FP64 ? 8 : 4;
  int64_t b = d * (4 * elem + 8 + (r.opts.lanczos.precision == ED_FP32_POLISH ? 5 * 8 : 8));
  const int64_t chains = std::min(8, 4 * r.model.norb);
  if (r.opts.nmats > 0) b += chains * dn * 3 * gelem;
  // the Krylov basis kept by the ground state: at most basis_mib MiB, about
  // 128 vectors for a typical run
  if (r.opts.lanczos.basis_mib > 0)
    b += std::min<int64_t>((int64_t)r.opts.lanczos.basis_mib << 20, d * elem * 128);
  return b + (32ll << 20);
}

void ed_server_s::worker_main() {
  cudaSetDevice(device);
  cudaStream_t cs = nullptr;
  cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  for (;;) {
    std::unique_ptr<OwnedRequest> req;
    bool inject = false;
    {
      std::unique_lock<std::mutex> lk(mu);
      // bounded waits: wake at least every 100 ms to re-check the state
      while (!stopping) {
        if (!queue.empty()) {
          const int64_t need = queue.front()->mem_estimate;
          if (in_use == 0 || in_use + need <= budget) break;
        }
        cv_work.wait_for(lk, std::chrono::milliseconds(100));
      }
      if (stopping && queue.empty()) break;
      if (stopping) break;
      req = std::move(queue.front());
      queue.pop_front();
      in_use += req->mem_estimate;
      running[req->ticket] = 1;
      if (injected_failures > 0) {
        --injected_failures;
        inject = true;
      }
    }
    Done d;
    memset(&d.res, 0, sizeof(d.res));
    d.res.t_submit_s = req->t_submit;
    d.res.t_start_s = clock_s(t0);
    d.res.norb = req->model.norb;
    d.res.nmats = req->opts.nmats;
    d.G.assign((size_t)2 * 2 * req->model.norb * std::max(0, req->opts.nmats), 0.0);
    if (inject) {
      d.res.status = ED_ERR_OOM;
    } else {
      ed_solve_result sr;
      d.res.status = ed_solve_impl(&req->model, req->nup, req->ndw, &req->opts, &sr,
                                   d.G.empty() ? nullptr : d.G.data(), nullptr, cs);
      d.res.ground = sr.ground;
      d.res.e0 = sr.ground.e0;
    }
    d.res.t_done_s = clock_s(t0);
    {
      std::lock_guard<std::mutex> lk(mu);
      in_use -= req->mem_estimate;
      running.erase(req->ticket);
      done[req->ticket] = std::move(d);
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
  if (cs) cudaStreamDestroy(cs);
}

extern "C" ed_status ed_server_create(const ed_server_opts *opts, ed_server *out) {
  if (!out) return ED_ERR_ARG;
  *out = nullptr;
  ed_server s = new ed_server_s();
  if (opts) s->opts = *opts;
  else memset(&s->opts, 0, sizeof(s->opts));
  if (s->opts.slots <= 0) s->opts.slots = 8;
  if (s->opts.queue_capacity <= 0) s->opts.queue_capacity = 65536;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) {
    ed_set_cuda_error(e, "cudaGetDevice", __FILE__, __LINE__);
    delete s;
    return ED_ERR_CUDA;
  }
  if (s->opts.device_mem_budget > 0) {
    s->budget = s->opts.device_mem_budget;
  } else {
    size_t avail = 0;
    const ed_status as = ed_device_available(&avail);
    if (as != ED_OK) {
      delete s;
      return as;
    }
    s->budget = (int64_t)(avail / 2);
  }
  ed_status bs = ed_upload_binomials();
  if (bs != ED_OK) {
    delete s;
    return bs;
  }
  s->t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < s->opts.slots; ++i) s->workers.emplace_back([s] { s->worker_main(); });
  *out = s;
  return ED_OK;
}

extern "C" ed_status ed_submit(ed_server s, const ed_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return ED_ERR_ARG;
  const ed_model &m = req->model;
  ed_status st = ED_OK;
  ModelParams mp = ed_model_params(&m, &st);
  if (st != ED_OK) return st;
  if (req->nup < 0 || req->ndw < 0 || req->nup > mp.ns || req->ndw > mp.ns) return ED_ERR_ARG;
  if (req->opts.nmats < 0) return ED_ERR_ARG;
  auto r = std::make_unique<OwnedRequest>();
  r->e_imp.assign(m.e_imp, m.e_imp + 2 * m.norb);
  size_t nb = (size_t)2 * m.norb * m.nbath;
  if (nb) {
    r->e_bath.assign(m.e_bath, m.e_bath + nb);
    r->v_bath.assign(m.v_bath, m.v_bath + nb);
  }
  r->model = m;
  r->model.e_imp = r->e_imp.data();
  r->model.e_bath = nb ? r->e_bath.data() : nullptr;
  r->model.v_bath = nb ? r->v_bath.data() : nullptr;
  r->nup = req->nup;
  r->ndw = req->ndw;
  r->opts = req->opts;
  // requests share the device: unless the request says otherwise, each keeps
  // at most 2 GiB of Krylov basis (beyond that its ground state uses the
  // second pass)
  if (r->opts.lanczos.basis_mib == 0) r->opts.lanczos.basis_mib = 2048;
  r->mem_estimate = estimate_bytes(*r);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->mem_estimate > s->budget) return ED_ERR_OOM;
    if ((int64_t)s->queue.size() >= s->opts.queue_capacity) return ED_ERR_BUSY;
    r->ticket = s->next_ticket++;
    r->t_submit = clock_s(s->t0);
    *ticket = r->ticket;
    s->queue.push_back(std::move(r));
  }
  s->cv_work.notify_one();
  return ED_OK;
}

extern "C" ed_status ed_poll(ed_server s, uint64_t ticket, ed_result *out, double *host_G) {
  if (!s || !out) return ED_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) {
    if (s->running.count(ticket)) return ED_PENDING;
    for (auto &q : s->queue)
      if (q->ticket == ticket) return ED_PENDING;
    return ED_ERR_NOT_FOUND;
  }
  *out = it->second.res;
  if (host_G) {
    if (!it->second.G.empty())
      memcpy(host_G, it->second.G.data(), it->second.G.size() * sizeof(double));
    s->done.erase(it);
  }
  return ED_OK;
}

extern "C" ed_status ed_wait(ed_server s, uint64_t ticket, double timeout_s) {
  if (!s) return ED_ERR_ARG;
  auto deadline = std::chrono::steady_clock::now() +
                  std::chrono::microseconds((int64_t)(std::max(0.0, timeout_s) * 1e6));
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    if (s->done.count(ticket)) return ED_OK;
    bool known = s->running.count(ticket) > 0;
    if (!known)
      for (auto &q : s->queue)
        if (q->ticket == ticket) known = true;
    if (!known) return ED_ERR_NOT_FOUND;
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !s->done.count(ticket))
      return ED_ERR_TIMEOUT;
  }
}

extern "C" ed_status ed_server_inject_alloc_failure(ed_server s, int32_t count) {
  if (!s || count < 0) return ED_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->injected_failures = count;
  return ED_OK;
}

extern "C" ed_status ed_server_destroy(ed_server s) {
  if (!s) return ED_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto &t : s->workers) t.join();
  delete s;
  return ED_OK;
}
