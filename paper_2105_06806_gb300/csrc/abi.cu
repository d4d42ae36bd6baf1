// C ABI glue: error reporting, launch counter, status strings and the
// one-call impurity solve (Sec. 6.9 main flow: sector, ground state, G).
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <string>

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
                     ed_gf_info *info, cudaStream_t cs);

static double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

ed_status ed_solve_impl(const ed_model *model, int nup, int ndw, const ed_solve_opts *o,
                        ed_solve_result *res, double *host_G, cudaStream_t cs) {
  if (!model || !o || !res) return ED_ERR_ARG;
  memset(res, 0, sizeof(*res));
  const int nmats = o->nmats;
  if (nmats < 0 || (nmats > 0 && !host_G)) return ED_ERR_ARG;
  const ed_precision gp = o->lanczos.precision;
  const bool psi_double = gp != ED_FP32;
  const bool chain32 = o->gf_precision != ED_FP64;
  if (nmats > 0 && !psi_double && !chain32) return ED_ERR_ARG;
  const ed_precision gfp = psi_double ? (chain32 ? ED_FP32_POLISH : ED_FP64) : ED_FP32;

  double t0 = now_s();
  ed_sector s = nullptr;
  ED_TRY(ed_sector_build(model, nup, ndw, cs, &s));
  double t1 = now_s();
  res->t_build_s = t1 - t0;
  void *psi = nullptr;
  ed_status rs = ED_OK;
  ed_lanczos_opts lo = o->lanczos;
  lo.want_vector = nmats > 0 ? 1 : lo.want_vector;
  if (lo.want_vector) {
    cudaError_t e = cudaMallocAsync(&psi, s->dim * (psi_double ? 8 : 4), cs);
    if (e != cudaSuccess) {
      ed_set_cuda_error(e, "cudaMallocAsync(psi)", __FILE__, __LINE__);
      rs = ED_ERR_OOM;
    }
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
    for (int spin = 0; spin < 2 && rs == ED_OK; ++spin) {
      for (int orb = 0; orb < norb && rs == ED_OK; ++orb) {
        double *G = host_G + 2 * (size_t)nmats * (spin * norb + orb);
        if (spin == 1 && nup == ndw && s->spin_symmetric) {
          memcpy(G, host_G + 2 * (size_t)nmats * orb, 2 * sizeof(double) * nmats);
          continue;
        }
        rs = ed_gf_impl(s, gfp, psi, res->ground.e0, orb, spin, steps, beta, nmats, G, nullptr,
                        cs);
      }
    }
  }
  res->t_gf_s = now_s() - t2;
  if (psi) cudaFreeAsync(psi, cs);
  cudaStreamSynchronize(cs);
  ed_sector_free(s);
  return rs;
}

extern "C" ed_status ed_solve(const ed_model *model, int32_t nup, int32_t ndw,
                              const ed_solve_opts *opts, ed_solve_result *res, double *host_G,
                              void *stream) {
  return ed_solve_impl(model, nup, ndw, opts, res, host_G, (cudaStream_t)stream);
}
