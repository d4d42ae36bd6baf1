// C ABI glue: error reporting, launch counter, status strings and the
// one-call impurity solve (Sec. 6.9 main flow: sector, ground state, G).
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include <algorithm>

#include "internal.cuh"

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void ed_set_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  g_last_error = buf;
}

void ed_set_error_msg(const char *msg) { g_last_error = msg ? msg : ""; }

void ed_count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

extern "C" int64_t ed_kernel_launches(void) { return g_launches.load(); }

extern "C" const char *ed_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *ed_status_string(ed_status st) {
  switch (st) {
    case ED_OK: return "ok";
    case ED_PENDING: return "pending";
    case ED_ERR_ARG: return "invalid argument";
    case ED_ERR_UNSUPPORTED: return "unsupported model or size";
    case ED_ERR_OOM: return "device memory exhausted";
    case ED_ERR_CUDA: return "CUDA error";
    case ED_ERR_TIMEOUT: return "timed out";
    case ED_ERR_NOT_CONVERGED: return "Lanczos not converged";
    case ED_ERR_BUSY: return "queue full";
    case ED_ERR_NOT_FOUND: return "unknown ticket";
  }
  return "unknown status";
}

ed_status ed_gf_impl(ed_sector s, ed_precision prec, const void *d_psi, double e0, int orb,
                     int spin, int nsteps, double beta, int nmats, double *host_G,
                     ed_gf_info *info, cudaStream_t cs, const double *host_z = nullptr);
ed_status ed_gf_chain_job(ed_sector s, ed_precision prec, const void *d_psi, double e0, int orb,
                          int spin, int create, int nsteps, double beta, int nmats,
                          double *host_G, double *weight, int *steps, int64_t *dim,
                          cudaEvent_t after);
ed_status ed_gf_prepare(ed_sector s, int spin, int create, int elem, cudaStream_t cs);
bool ed_gf_batchable(ed_sector s, int spin, int create);
ed_status ed_gf_chain_batch(ed_sector s, ed_precision prec, const void *d_psi, double e0,
                            int nsteps, double beta, int nmats, int njobs, const int *orb,
                            const int *spin, const int *create, double *host_G, double *weight,
                            int *steps, int64_t *dim, cudaStream_t cs);

void ed_gf_batch_announce(int delta);

static double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

static uint64_t binom_u(int n, int k) {
  if (k < 0 || k > n) return 0;
  uint64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
  return r;
}

// Marks a solve whose chains will be small enough for the batched launch
// (every N+-1 sector at most 2^14 states, before padding) as under way, so
// that a batch leader knows other members may still join.
struct BatchAnnounce {
  bool on = false;
  BatchAnnounce(const ed_model *m, int nup, int ndw, int nmats) {
    if (nmats <= 0) return;
    const int ns = m->norb * (m->nbath + 1);
    uint64_t d = 0;
    for (int ds = -1; ds <= 1; ds += 2) {
      d = std::max(d, binom_u(ns, nup + ds) * binom_u(ns, ndw));
      d = std::max(d, binom_u(ns, nup) * binom_u(ns, ndw + ds));
    }
    on = d <= (1u << 14);
    if (on) ed_gf_batch_announce(1);
  }
  ~BatchAnnounce() {
    if (on) ed_gf_batch_announce(-1);
  }
};

ed_status ed_solve_impl(const ed_model *model, int nup, int ndw, const ed_solve_opts *o,
                        ed_solve_result *res, double *host_G, void *d_psi_out, cudaStream_t cs) {
  if (!model || !o || !res) return ED_ERR_ARG;
  memset(res, 0, sizeof(*res));
  const int nmats = o->nmats;
  if (nmats < 0 || (nmats > 0 && !host_G)) return ED_ERR_ARG;
  if (nmats > 0) memset(host_G, 0, sizeof(double) * 2 * 2 * (size_t)model->norb * nmats);
  const ed_precision gp = o->lanczos.precision;
  const bool psi_double = gp != ED_FP32;
  const bool chain32 = o->gf_precision != ED_FP64;
  if (nmats > 0 && !psi_double && !chain32) return ED_ERR_ARG;
  const ed_precision gfp = psi_double ? (chain32 ? ED_FP32_POLISH : ED_FP64) : ED_FP32;

  const BatchAnnounce announce(model, nup, ndw, nmats);
  double t0 = now_s();
  ed_sector s = nullptr;
  ED_TRY(ed_sector_build(model, nup, ndw, cs, &s));
  double t1 = now_s();
  res->t_build_s = t1 - t0;
  void *psi = nullptr;
  ed_status rs = ED_OK;
  ed_lanczos_opts lo = o->lanczos;
  lo.want_vector = (nmats > 0 || d_psi_out) ? 1 : lo.want_vector;
  if (d_psi_out) {
    psi = d_psi_out;  // the caller's buffer holds psi for the chains too
  } else if (lo.want_vector) {
    rs = ed_dmalloc(&psi, s->dim * (psi_double ? 8 : 4), cs, "psi");
  }
  if (rs == ED_OK) {
    rs = ed_lanczos_ground_impl(s, &lo, &res->ground, psi, cs);
    if (rs == ED_ERR_NOT_CONVERGED) rs = ED_OK;  // reported in res->ground.stop_reason
  }
  double t2 = now_s();
  res->t_ground_s = t2 - t1;
  if (rs == ED_OK && nmats > 0) {
    const int steps = o->gf_steps > 0 ? o->gf_steps : 200;
    const double beta = o->beta > 0 ? o->beta : 100.0;
    const int norb = s->mp.norb;
    const bool copy_dw = nup == ndw && s->spin_symmetric;
    const int elem = gfp == ED_FP64 ? 8 : 4;
    struct Job {
      int orb, spin, create;
      std::vector<double> G;
      double weight = 0;
      int steps = 0;
      int64_t dim = 0;
      ed_status st = ED_OK;
    };
    std::vector<Job> jobs;
    for (int spin = 0; spin < 2; ++spin) {
      if (spin == 1 && copy_dw) continue;
      for (int create = 1; create >= -1; create -= 2) {
        if (rs == ED_OK) rs = ed_gf_prepare(s, spin, create, elem, cs);
        for (int orb = 0; orb < norb; ++orb) {
          Job j;
          j.orb = orb;
          j.spin = spin;
          j.create = create;
          j.G.assign(2 * (size_t)nmats, 0.0);
          jobs.push_back(std::move(j));
        }
      }
    }
    // small sectors: every chain in one batched launch on the solve's stream
    bool batch = rs == ED_OK;
    for (const Job &j : jobs) batch = batch && ed_gf_batchable(s, j.spin, j.create);
    if (batch) {
      const int nj = (int)jobs.size();
      std::vector<int> jo(nj), js(nj), jc(nj), jsteps(nj);
      std::vector<double> jw(nj), jG((size_t)nj * 2 * nmats);
      std::vector<int64_t> jd(nj);
      for (int q = 0; q < nj; ++q) {
        jo[q] = jobs[q].orb;
        js[q] = jobs[q].spin;
        jc[q] = jobs[q].create;
      }
      rs = ed_gf_chain_batch(s, gfp, psi, res->ground.e0, steps, beta, nmats, nj, jo.data(),
                             js.data(), jc.data(), jG.data(), jw.data(), jsteps.data(), jd.data(),
                             cs);
      for (int q = 0; q < nj && rs == ED_OK; ++q) {
        jobs[q].weight = jw[q];
        jobs[q].steps = jsteps[q];
        jobs[q].dim = jd[q];
        memcpy(jobs[q].G.data(), jG.data() + 2 * (size_t)nmats * q, 2 * sizeof(double) * nmats);
      }
    }
    cudaEvent_t ready = nullptr;
    if (rs == ED_OK && !batch &&
        cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess)
      rs = ED_ERR_CUDA;
    if (rs == ED_OK && !batch && cudaEventRecord(ready, cs) != cudaSuccess) rs = ED_ERR_CUDA;
    int dev = 0;
    cudaGetDevice(&dev);
    // larger sectors: chains run concurrently on their own streams, at most
    // kMaxChains at a time
    const size_t kMaxChains = 8;
    for (size_t b = 0; rs == ED_OK && !batch && b < jobs.size(); b += kMaxChains) {
      std::vector<std::thread> th;
      for (size_t k = b; k < std::min(jobs.size(), b + kMaxChains); ++k) {
        th.emplace_back([&, k] {
          cudaSetDevice(dev);
          Job &j = jobs[k];
          j.st = ed_gf_chain_job(s, gfp, psi, res->ground.e0, j.orb, j.spin, j.create, steps, beta,
                                 nmats, j.G.data(), &j.weight, &j.steps, &j.dim, ready);
        });
      }
      for (auto &t : th) t.join();
    }
    if (ready) cudaEventDestroy(ready);
    for (auto &j : jobs) {
      if (rs == ED_OK && j.st != ED_OK) rs = j.st;
      double *G = host_G + 2 * (size_t)nmats * (j.spin * norb + j.orb);
      for (int n = 0; n < 2 * nmats; ++n) G[n] += j.G[n];
      res->gf_chains += j.steps > 0 ? 1 : 0;
      res->gf_steps_total += j.steps;
      res->gf_product_bytes += (double)j.steps * (double)j.dim * 2.0 * elem;
    }
    if (copy_dw)
      for (int orb = 0; orb < norb; ++orb)
        memcpy(host_G + 2 * (size_t)nmats * (norb + orb), host_G + 2 * (size_t)nmats * orb,
               2 * sizeof(double) * nmats);
  }
  res->t_gf_s = now_s() - t2;
  if (psi && psi != d_psi_out) ed_dfree(psi, cs);
  // every chain job has synchronised its own stream; after this the sector's
  // tables have no reader left and are released stream-ordered on cs
  cudaError_t e = cudaStreamSynchronize(cs);
  ed_sector_release(s, cs);
  if (rs == ED_OK && e != cudaSuccess) {
    ed_set_cuda_error(e, "solve stream", __FILE__, __LINE__);
    rs = ED_ERR_CUDA;
  }
  return rs;
}

extern "C" ed_status ed_solve(const ed_model *model, int32_t nup, int32_t ndw,
                              const ed_solve_opts *opts, ed_solve_result *res, double *host_G,
                              void *d_psi, void *stream) {
  return ed_solve_impl(model, nup, ndw, opts, res, host_G, d_psi, (cudaStream_t)stream);
}
