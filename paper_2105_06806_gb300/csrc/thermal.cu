// Several low-lying states and finite temperature (Sec. 6.2 eigenspace list
// with its annealing truncation; App. A thermal averages of Eq. KLgf).
//
// The k-th state of a sector is the lowest eigenpair of the shift-deflated
// operator H + sigma sum_{j<k} |psi_j><psi_j|, solved with the
// operator-generic Lanczos driver on the block-major vectors: the product
// kernels, then one pass forming the k overlaps <psi_j, v> (v read once, every
// CTA a partial of each overlap) and one pass adding sigma <psi_j, v> psi_j.
// sigma puts the states already found above the top of the spectrum (the
// highest Ritz value of the first run plus 5% of the span), so that rounding
// that leaks them back into the Krylov space cannot produce them again.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int TH_THREADS = 256;
constexpr int TH_PARTS = 512;
constexpr int TH_STATES_PER_PASS = 16;  // overlaps formed by one pass

unsigned th_grid(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 4 * TH_THREADS - 1) / (4 * TH_THREADS),
                                                          TH_PARTS));
}

// parts[q * gridDim.x + cta] = sum over the CTA's elements of psi_q[i] v[i],
// q < nq (FP64 partials; states psi_q = st[q0 + q])
template <typename T>
__global__ void __launch_bounds__(TH_THREADS) k_defl_dots(T *const *st, int q0, int nq,
                                                          const T *v, int64_t n, double *parts) {
  __shared__ double red[TH_THREADS / 32][TH_STATES_PER_PASS];
  double acc[TH_STATES_PER_PASS];
  for (int q = 0; q < TH_STATES_PER_PASS; ++q) acc[q] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = (double)v[i];
    for (int q = 0; q < nq; ++q) acc[q] += (double)st[q0 + q][i] * x;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < nq; ++q) {
    double x = acc[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[wid][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < nq) {
    double t = 0.0;
    for (int k = 0; k < TH_THREADS / 32; ++k) t += red[k][threadIdx.x];
    parts[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}

// coef[q0 + q] = sigma * sum of the partials of overlap q (fixed order)
__global__ void k_defl_coef(const double *parts, int nq, int np, double sigma, double *coef,
                            int q0) {
  const int q = threadIdx.x;
  if (q >= nq) return;
  double t = 0.0;
  for (int k = 0; k < np; ++k) t += parts[(int64_t)q * np + k];
  coef[q0 + q] = sigma * t;
}

// w += sum_{q < k} coef[q] psi_q
template <typename T>
__global__ void k_defl_add(T *w, T *const *st, int k, const double *coef, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double x = (double)w[i];
    for (int q = 0; q < k; ++q) x += coef[q] * (double)st[q][i];
    w[i] = (T)x;
  }
}

// seeded start vector in padded block-major order (padding zero)
template <typename T>
__global__ void k_states_start(T *v, int64_t n, int64_t stride, const int32_t *padinv,
                               uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / stride, pc = i - r * stride;
    T x = T(0);
    if (padinv[pc] >= 0) {
      const double u = (double)(ed_splitmix64_at(seed, (uint64_t)i) >> 11) *
                       (1.0 / 9007199254740992.0);
      x = (T)(u - 0.5);
    }
    v[i] = x;
  }
}

struct Mem {
  void *p = nullptr;
  cudaStream_t cs = nullptr;
  ~Mem() {
    if (p) ed_dfree(p, cs);
  }
  ed_status alloc(size_t bytes, cudaStream_t st, const char *what) {
    cs = st;
    return ed_dmalloc(&p, std::max<size_t>(bytes, 256), st, what);
  }
};

// The deflated operator of one precision: states in block-major order
template <typename T>
struct Deflated {
  ed_sector s = nullptr;
  int64_t n = 0;
  double sigma = 0.0;
  int k = 0;                 // states deflated
  T *const *d_states = nullptr;
  double *parts = nullptr;   // TH_STATES_PER_PASS * TH_PARTS
  double *coef = nullptr;    // ED_MAX_STATES
  LinOp<T> op() const {
    LinOp<T> o;
    o.n = n;
    const Deflated<T> self = *this;
    o.apply = [self](const T *v, T *w, cudaStream_t cs) -> ed_status {
      ED_TRY(ed_launch_hv<T>(self.s, ed_hv_tables<T>(self.s, 1), HV_PLAIN, v, w, nullptr,
                             nullptr, nullptr, nullptr, nullptr, cs));
      if (self.k == 0) return ED_OK;
      const unsigned g = th_grid(self.n);
      for (int q0 = 0; q0 < self.k; q0 += TH_STATES_PER_PASS) {
        const int nq = std::min(TH_STATES_PER_PASS, self.k - q0);
        k_defl_dots<T><<<g, TH_THREADS, 0, cs>>>(self.d_states, q0, nq, v, self.n, self.parts);
        ED_LAUNCHED(1);
        k_defl_coef<<<1, TH_STATES_PER_PASS, 0, cs>>>(self.parts, nq, (int)g, self.sigma,
                                                      self.coef, q0);
        ED_LAUNCHED(1);
      }
      k_defl_add<T><<<g, TH_THREADS, 0, cs>>>(w, self.d_states, self.k, self.coef, self.n);
      ED_LAUNCHED(1);
      return ED_OK;
    };
    return o;
  }
};

// kept states (lowest first, Boltzmann factor >= cutoff, at most ntotal) and
// their normalised weights
void boltzmann(const std::vector<double> &E, double beta, double cutoff, int ntotal,
               std::vector<double> &w, int *nkept) {
  const size_t n = E.size();
  w.assign(n, 0.0);
  *nkept = 0;
  if (n == 0) return;
  std::vector<size_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return E[a] < E[b]; });
  const double e0 = E[order[0]];
  double z = 0.0;
  for (size_t t = 0; t < n && *nkept < ntotal; ++t) {
    const double f = exp(-beta * (E[order[t]] - e0));
    if (f >= cutoff) {
      w[order[t]] = f;
      z += f;
      ++*nkept;
    }
  }
  for (double &x : w) x /= z;
}

template <typename T>
ed_status solve_state(ed_sector s, Deflated<T> &d, int maxit, double tol, uint64_t seed,
                      const T *start, T *psi, OpRun *run, cudaStream_t cs) {
  Mem v0;
  if (!start) {
    ED_TRY(v0.alloc((size_t)d.n * sizeof(T), cs, "state start vector"));
    k_states_start<T><<<th_grid(d.n), TH_THREADS, 0, cs>>>((T *)v0.p, d.n, s->bstride, s->padinv,
                                                           seed);
    ED_LAUNCHED(1);
    start = (const T *)v0.p;
  }
  return ed_op_lanczos<T>(d.op(), start, maxit, tol, true, run, nullptr, psi, cs);
}

}  // namespace

extern "C" ed_status ed_espace_truncate(int32_t nsectors, const int32_t *counts,
                                        const double *energies, double beta, double cutoff,
                                        int32_t ntotal, int32_t step, double *weights,
                                        int32_t *next_counts, int32_t *nkept) {
  if (nsectors < 0 || (nsectors > 0 && (!counts || !weights)) || !isfinite(beta) ||
      !(cutoff >= 0.0))
    return ED_ERR_ARG;
  int64_t total = 0;
  for (int q = 0; q < nsectors; ++q) {
    if (counts[q] < 0) return ED_ERR_ARG;
    total += counts[q];
  }
  if (total > 0 && !energies) return ED_ERR_ARG;
  if (cutoff > 1.0) return ED_ERR_ARG;  // the lowest state's factor is 1
  const std::vector<double> E(energies, energies + total);
  std::vector<double> w;
  int nk = 0;
  boltzmann(E, beta, cutoff, ntotal > 0 ? ntotal : INT32_MAX, w, &nk);
  size_t o = 0;
  for (int q = 0; q < nsectors; ++q) {
    int kept = 0;
    for (int i = 0; i < counts[q]; ++i) {
      weights[o + i] = w[o + i];
      kept += w[o + i] > 0.0;
    }
    const bool top = counts[q] > 0 && w[o + counts[q] - 1] > 0.0;
    if (next_counts) next_counts[q] = top ? counts[q] + step : kept + 1;
    o += counts[q];
  }
  if (nkept) *nkept = nk;
  return ED_OK;
}

extern "C" ed_status ed_lanczos_states(ed_sector s, const ed_lanczos_opts *o, int32_t nstates,
                                       double *host_e, ed_lanczos_result *res, void *d_psis,
                                       void *stream) {
  if (!s || !o || !host_e) return ED_ERR_ARG;
  if (nstates < 1 || nstates > ED_MAX_STATES || nstates > s->dim) return ED_ERR_ARG;
  const ed_precision prec = o->precision;
  if (prec != ED_FP64 && prec != ED_FP32 && prec != ED_FP32_POLISH) return ED_ERR_ARG;
  const int maxit = o->max_iter > 0 ? o->max_iter : 512;
  if (maxit > ED_MAX_LANCZOS) return ED_ERR_ARG;
  const double tol = o->tol > 0 ? o->tol : (prec == ED_FP64 ? 1e-12 : 1e-6);
  const int steps = o->polish_steps > 0 ? o->polish_steps : 4;
  cudaStream_t cs = (cudaStream_t)stream;
  const int64_t n = s->bdim;
  const bool f32 = prec != ED_FP64;
  ED_TRY(ed_build_items(s, 1, 8));
  if (f32) ED_TRY(ed_build_items(s, 1, 4));
  const size_t vb8 = ((size_t)n * 8 + 255) & ~(size_t)255, vb4 = ((size_t)n * 4 + 255) & ~(size_t)255;
  // FP64 states (the output), FP32 states (FP32 runs), pointer tables,
  // partials and coefficients
  Mem mem;
  const size_t tb = ((size_t)ED_MAX_STATES * sizeof(void *) + 255) & ~(size_t)255;
  const size_t pb = ((size_t)(TH_STATES_PER_PASS * TH_PARTS + ED_MAX_STATES) * 8 + 255) & ~(size_t)255;
  ED_TRY(mem.alloc(nstates * vb8 + (f32 ? nstates * vb4 : 0) + 2 * tb + 2 * pb, cs, "excited states"));
  char *p = (char *)mem.p;
  std::vector<double *> s64(nstates);
  std::vector<float *> s32(nstates);
  for (int k = 0; k < nstates; ++k) s64[k] = (double *)(p + k * vb8);
  p += nstates * vb8;
  if (f32) {
    for (int k = 0; k < nstates; ++k) s32[k] = (float *)(p + k * vb4);
    p += nstates * vb4;
  }
  double **t64 = (double **)p;
  float **t32 = (float **)(p + tb);
  p += 2 * tb;
  double *parts64 = (double *)p, *coef64 = parts64 + TH_STATES_PER_PASS * TH_PARTS;
  double *parts32 = (double *)(p + pb), *coef32 = parts32 + TH_STATES_PER_PASS * TH_PARTS;
  ED_TRY_CUDA(cudaMemcpyAsync(t64, s64.data(), nstates * sizeof(double *), cudaMemcpyHostToDevice, cs));
  if (f32)
    ED_TRY_CUDA(cudaMemcpyAsync(t32, s32.data(), nstates * sizeof(float *), cudaMemcpyHostToDevice, cs));
  Deflated<double> d64;
  d64.s = s;
  d64.n = n;
  d64.d_states = t64;
  d64.parts = parts64;
  d64.coef = coef64;
  Deflated<float> d32;
  d32.s = s;
  d32.n = n;
  d32.d_states = t32;
  d32.parts = parts32;
  d32.coef = coef32;
  ed_status rs = ED_OK;
  for (int k = 0; k < nstates && rs == ED_OK; ++k) {
    OpRun run, pol;
    const uint64_t seed = o->seed + 0x9E3779B97F4A7C15ull * (uint64_t)k;
    ed_lanczos_result r;
    memset(&r, 0, sizeof(r));
    d64.k = d32.k = k;
    if (!f32) {
      rs = solve_state<double>(s, d64, maxit, tol, seed, nullptr, s64[k], &run, cs);
      r.e0 = r.e0_raw = run.theta;
      r.matvecs = r.matvecs_fp64 = run.matvecs;
    } else {
      rs = solve_state<float>(s, d32, maxit, tol, seed, nullptr, s32[k], &run, cs);
      r.e0 = r.e0_raw = run.theta;
      r.matvecs = run.matvecs;
      if (rs == ED_OK) rs = ed_op_normalised_copy<float, double>(s32[k], s64[k], n, cs);
      if (rs == ED_OK && prec == ED_FP32_POLISH) {
        Mem start;
        rs = start.alloc(vb8, cs, "polish start");
        if (rs == ED_OK && cudaMemcpyAsync(start.p, s64[k], (size_t)n * 8, cudaMemcpyDeviceToDevice,
                                           cs) != cudaSuccess)
          rs = ED_ERR_CUDA;
        if (rs == ED_OK)
          rs = solve_state<double>(s, d64, steps, 1e-300, 0, (const double *)start.p, s64[k],
                                   &pol, cs);
        r.e0 = pol.theta;
        r.polish_iterations = pol.k;
        r.matvecs += pol.matvecs;
        r.matvecs_fp64 = pol.matvecs;
      }
    }
    if (rs != ED_OK) break;
    if (k == 0) {
      // the shift: above the top of the spectrum seen by the first run
      const double span = std::max(run.theta_max - run.theta, 0.0);
      d64.sigma = d32.sigma = 1.05 * span + 1e-6;
    }
    r.iterations = run.k;
    r.residual_estimate = run.resid_est;
    r.stop_reason = run.stop;
    // residual with the undeflated H
    LinOp<double> h;
    h.n = n;
    h.apply = [s](const double *v, double *w, cudaStream_t st) {
      return ed_launch_hv<double>(s, ed_hv_tables<double>(s, 1), HV_PLAIN, v, w, nullptr, nullptr,
                                  nullptr, nullptr, nullptr, st);
    };
    double e = 0.0, resid = 0.0;
    rs = ed_op_residual(h, s64[k], &e, &resid, cs);
    r.residual = resid;
    r.matvecs += 1;
    r.matvecs_fp64 += 1;
    host_e[k] = r.e0;
    if (res) res[k] = r;
    if (rs == ED_OK && d_psis) {
      if (prec == ED_FP32)
        rs = ed_permute_vec(s, ED_FP32, false, s32[k], (float *)d_psis + (int64_t)k * s->dim, cs);
      else
        rs = ed_permute_vec(s, ED_FP64, false, s64[k], (double *)d_psis + (int64_t)k * s->dim, cs);
    }
  }
  if (cudaStreamSynchronize(cs) != cudaSuccess && rs == ED_OK) rs = ED_ERR_CUDA;
  return rs;
}

extern "C" ed_status ed_gf_thermal_z(int32_t nstates, const ed_sector *sectors,
                                     const void *const *d_psis, const double *energies,
                                     double beta, double cutoff, int32_t ntotal,
                                     ed_precision prec, int32_t orb, int32_t spin, int32_t nsteps,
                                     const double *host_z, int32_t nz, double *host_G,
                                     double *host_w, void *stream) {
  if (nstates < 1 || !sectors || !d_psis || !energies || !host_G || nz < 0 ||
      (nz > 0 && !host_z) || !isfinite(beta) || !(cutoff >= 0.0) || cutoff > 1.0)
    return ED_ERR_ARG;
  std::vector<double> E(energies, energies + nstates), w;
  int nk = 0;
  boltzmann(E, beta, cutoff, ntotal > 0 ? ntotal : INT32_MAX, w, &nk);
  if (host_w) std::copy(w.begin(), w.end(), host_w);
  std::vector<double> G(2 * (size_t)std::max(nz, 1), 0.0), Gi(2 * (size_t)std::max(nz, 1));
  for (int i = 0; i < nstates; ++i) {
    if (w[i] == 0.0) continue;
    if (!sectors[i] || !d_psis[i]) return ED_ERR_ARG;
    ED_TRY(ed_gf_lanczos_z(sectors[i], prec, d_psis[i], E[i], orb, spin, nsteps, host_z, nz,
                           Gi.data(), nullptr, stream));
    for (int64_t t = 0; t < 2 * (int64_t)nz; ++t) G[t] += w[i] * Gi[t];
  }
  std::copy(G.begin(), G.begin() + 2 * (size_t)nz, host_G);
  return ED_OK;
}
