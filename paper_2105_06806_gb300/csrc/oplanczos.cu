// Operator-generic Lanczos (Sec. 6.6, and the chains of Sec. 6.8) for
// operators assembled from the product kernels: the electron-phonon sector of
// Sec. 4 (the electronic product on every phonon slice plus the phonon
// terms) and the deflated sector operator of the excited-state solver.
//
// Plain Lanczos in the Paige form without re-orthogonalisation, as in the
// fused driver: w = A v_j, alpha_j = <v_j, w>, w -= alpha_j v_j + beta_j
// v_{j-1}, beta_{j+1} = ||w||, v_{j+1} = w / beta_{j+1}.  The reductions sum
// at most OP_FLUSH products per thread in the vector type and everything
// else in FP64; alpha_j and beta_{j+1} are written into a device
// LanczosState (so that the continued-fraction kernels read the chain
// directly) and copied to the host after every step, where the stopping rule
// (lowest Ritz value of T_j, Sturm bisection, and beta_{j+1} |y_j|) runs.
// The ground-state vector comes from the second pass of Sec. 6.6: the same
// recurrence regenerated from v_0 with the stored coefficients.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int OP_THREADS = 256;
constexpr int OP_FLUSH = 16;
constexpr int OP_MAX_PARTS = 1024;

int64_t op_grid(int64_t n) {
  return std::max<int64_t>(1, std::min<int64_t>((n + 4 * OP_THREADS - 1) / (4 * OP_THREADS),
                                                OP_MAX_PARTS));
}

template <typename T>
__device__ __forceinline__ T op_fma(T a, T b, T c);
template <>
__device__ __forceinline__ float op_fma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double op_fma<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ double op_block_sum(double x, double *red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
  return t;
}

// parts[cta] = sum over the CTA's elements of x_i y_i
template <typename T>
__global__ void __launch_bounds__(OP_THREADS) k_op_dot(const T *x, const T *y, int64_t n,
                                                       double *parts) {
  __shared__ double red[OP_THREADS / 32];
  double acc = 0.0;
  T t = T(0);
  int cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    t = op_fma<T>(x[i], y[i], t);
    if (++cnt == OP_FLUSH) {
      acc += (double)t;
      t = T(0);
      cnt = 0;
    }
  }
  acc += (double)t;
  const double s = op_block_sum(acc, red);
  if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

// dst = sum of the parts (fixed order), or its square root (SQRT)
template <bool SQRT>
__global__ void k_op_finish(const double *parts, int np, double *dst) {
  __shared__ double red[OP_THREADS / 32];
  double acc = 0.0;
  for (int k = threadIdx.x; k < np; k += blockDim.x) acc += parts[k];
  const double s = op_block_sum(acc, red);
  if (threadIdx.x == 0) dst[0] = SQRT ? sqrt(fmax(s, 0.0)) : s;
}

// w = w - alpha v - beta vp (vp may be null), parts = ||w||^2 per CTA
template <typename T>
__global__ void __launch_bounds__(OP_THREADS) k_op_update(T *w, const T *v, const T *vp,
                                                          const double *alpha,
                                                          const double *beta, int64_t n,
                                                          double *parts) {
  __shared__ double red[OP_THREADS / 32];
  const T a = (T)alpha[0], b = vp ? (T)beta[0] : T(0);
  double acc = 0.0;
  T t = T(0);
  int cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T x = op_fma<T>(-a, v[i], w[i]);
    if (vp) x = op_fma<T>(-b, vp[i], x);
    w[i] = x;
    t = op_fma<T>(x, x, t);
    if (++cnt == OP_FLUSH) {
      acc += (double)t;
      t = T(0);
      cnt = 0;
    }
  }
  acc += (double)t;
  const double s = op_block_sum(acc, red);
  if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

// y = x / norm[0] (0 when the norm is 0), converting the type
template <typename Ti, typename To>
__global__ void k_op_scale(const Ti *x, To *y, const double *norm, int64_t n) {
  const double nv = norm[0];
  const Ti inv = nv > 0.0 ? (Ti)(1.0 / nv) : Ti(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (To)(x[i] * inv);
}

// y += a x
template <typename T>
__global__ void k_op_axpy(T *y, const T *x, T a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = op_fma<T>(a, x[i], y[i]);
}

__global__ void k_op_set_j(LanczosState *st, int j, int done) {
  st->j = j;
  st->done = done;
  st->beta[0] = 0.0;
}

// ---------------------------------------------------------------- host tridiagonal

// Number of eigenvalues of T_k below x (Sturm sequence of the LDL^T pivots).
int sturm_below(const std::vector<double> &a, const std::vector<double> &b, int k, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < k; ++i) {
    const double bb = i ? b[i] * b[i] : 0.0;
    q = a[i] - x - (i ? bb / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// Largest eigenvalue of T_k (Sturm bisection): the top of the spectrum seen
// by the run, used to place deflated states above it.
double highest_ritz(const std::vector<double> &a, const std::vector<double> &b, int k) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < k; ++i) {
    const double r = (i ? fabs(b[i]) : 0.0) + (i + 1 < k ? fabs(b[i + 1]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_below(a, b, k, mid) >= k)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

double lowest_ritz(const std::vector<double> &a, const std::vector<double> &b, int k) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < k; ++i) {
    const double r = (i ? fabs(b[i]) : 0.0) + (i + 1 < k ? fabs(b[i + 1]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, fabs(lo)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_below(a, b, k, mid) >= 1)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Eigenvector of T_k for the eigenvalue th: inverse iteration with the
// tridiagonal LU (Thomas) of T_k - th, tiny pivots guarded, three sweeps.
std::vector<double> ritz_vector_host(const std::vector<double> &a, const std::vector<double> &b,
                                     int k, double th) {
  std::vector<double> y(k, 1.0), c(k), d(k);
  const double tiny = 1e-300, eps = 1e-15 * std::max(1.0, fabs(th));
  for (int sweep = 0; sweep < 3; ++sweep) {
    // forward elimination
    double piv = a[0] - th;
    if (fabs(piv) < eps) piv = piv < 0 ? -eps : eps;
    d[0] = y[0] / piv;
    for (int i = 1; i < k; ++i) {
      c[i - 1] = b[i] / piv;
      piv = a[i] - th - b[i] * c[i - 1];
      if (fabs(piv) < eps) piv = piv < 0 ? -eps : eps;
      d[i] = (y[i] - b[i] * d[i - 1]) / piv;
    }
    // back substitution
    y[k - 1] = d[k - 1];
    for (int i = k - 2; i >= 0; --i) y[i] = d[i] - c[i] * y[i + 1];
    double nrm = 0.0;
    for (int i = 0; i < k; ++i) nrm += y[i] * y[i];
    nrm = sqrt(std::max(nrm, tiny));
    for (int i = 0; i < k; ++i) y[i] /= nrm;
  }
  return y;
}

struct OpWork {
  void *mem = nullptr;
  cudaStream_t cs = nullptr;
  ~OpWork() {
    if (mem) ed_dfree(mem, cs);
  }
};

}  // namespace

template <typename T>
ed_status ed_op_norm(const T *x, int64_t n, double *d_out, double *parts, cudaStream_t cs) {
  const int64_t g = op_grid(n);
  k_op_dot<T><<<(unsigned)g, OP_THREADS, 0, cs>>>(x, x, n, parts);
  ED_LAUNCHED(1);
  k_op_finish<true><<<1, OP_THREADS, 0, cs>>>(parts, (int)g, d_out);
  ED_LAUNCHED(1);
  return ED_OK;
}

template <typename T>
ed_status ed_op_lanczos(const LinOp<T> &op, const T *v0, int maxit, double tol, bool ground,
                        OpRun *out, LanczosState *dst, T *psi, cudaStream_t cs) {
  *out = OpRun();
  const int64_t n = op.n;
  if (n <= 0 || maxit <= 0 || maxit > ED_MAX_LANCZOS) return ED_ERR_ARG;
  const int64_t g = op_grid(n);
  const size_t vb = ((size_t)n * sizeof(T) + 255) & ~(size_t)255;
  OpWork ws;
  ws.cs = cs;
  const size_t sb = (sizeof(LanczosState) + 255) & ~(size_t)255;
  ED_TRY(ed_dmalloc(&ws.mem, 3 * vb + sb + (size_t)(OP_MAX_PARTS + 8) * sizeof(double), cs,
                    "operator Lanczos"));
  char *p = (char *)ws.mem;
  T *buf[3] = {(T *)p, (T *)(p + vb), (T *)(p + 2 * vb)};
  LanczosState *st = dst ? dst : (LanczosState *)(p + 3 * vb);
  double *parts = (double *)(p + 3 * vb + sb);
  double *scal = parts + OP_MAX_PARTS;  // [0] ||v0||
  ED_TRY_CUDA(cudaMemsetAsync(ws.mem, 0, 3 * vb, cs));
  k_op_set_j<<<1, 1, 0, cs>>>(st, 0, 0);
  ED_LAUNCHED(1);
  // v_0 = v0 / ||v0||
  ED_TRY(ed_op_norm<T>(v0, n, scal, parts, cs));
  k_op_scale<T, T><<<(unsigned)g, OP_THREADS, 0, cs>>>(v0, buf[0], scal, n);
  ED_LAUNCHED(1);
  double h[3] = {0, 0, 0};
  ED_TRY_CUDA(cudaMemcpyAsync(h, scal, sizeof(double), cudaMemcpyDeviceToHost, cs));
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  out->weight = h[0] * h[0];
  if (!(h[0] > 0.0)) {
    out->stop = 1;
    return ED_OK;
  }
  std::vector<double> &A = out->alpha, &B = out->beta;
  A.clear();
  B.assign(1, 0.0);
  double tnorm = 0.0;
  int j = 0;
  for (;; ++j) {
    T *v = buf[j % 3], *w = buf[(j + 1) % 3], *vp = j > 0 ? buf[(j + 2) % 3] : nullptr;
    ED_TRY(op.apply(v, w, cs));
    ++out->matvecs;
    k_op_dot<T><<<(unsigned)g, OP_THREADS, 0, cs>>>(v, w, n, parts);
    ED_LAUNCHED(1);
    k_op_finish<false><<<1, OP_THREADS, 0, cs>>>(parts, (int)g, st->alpha + j);
    ED_LAUNCHED(1);
    k_op_update<T><<<(unsigned)g, OP_THREADS, 0, cs>>>(w, v, vp, st->alpha + j, st->beta + j, n,
                                                       parts);
    ED_LAUNCHED(1);
    k_op_finish<true><<<1, OP_THREADS, 0, cs>>>(parts, (int)g, st->beta + j + 1);
    ED_LAUNCHED(1);
    ED_TRY_CUDA(cudaMemcpyAsync(h, st->alpha + j, sizeof(double), cudaMemcpyDeviceToHost, cs));
    ED_TRY_CUDA(cudaMemcpyAsync(h + 1, st->beta + j + 1, sizeof(double), cudaMemcpyDeviceToHost, cs));
    ED_TRY_CUDA(cudaStreamSynchronize(cs));
    A.push_back(h[0]);
    tnorm = std::max(tnorm, std::max(fabs(h[0]), h[1]));
    const int k = j + 1;
    bool stop = false;
    if (h[1] <= 1e-13 * tnorm) {
      out->stop = 1;  // invariant subspace
      stop = true;
    }
    if (ground && (stop || k % 4 == 0 || k == maxit)) {
      out->theta = lowest_ritz(A, B, k);
      out->theta_max = highest_ritz(A, B, k);
      out->y = ritz_vector_host(A, B, k, out->theta);
      out->resid_est = h[1] * fabs(out->y[k - 1]);
      if (!stop && out->resid_est <= tol * std::max(1.0, fabs(out->theta))) {
        out->stop = 0;
        stop = true;
      }
    }
    if (!stop && k == maxit) {
      out->stop = 2;
      stop = true;
    }
    if (stop) {
      out->k = k;
      break;
    }
    B.push_back(h[1]);
    // v_{j+1} = w / beta_{j+1}, written over w in place
    k_op_scale<T, T><<<(unsigned)g, OP_THREADS, 0, cs>>>(w, w, st->beta + j + 1, n);
    ED_LAUNCHED(1);
  }
  k_op_set_j<<<1, 1, 0, cs>>>(st, out->k, 1);
  ED_LAUNCHED(1);
  if (ground && psi) {
    // second pass: the same recurrence from v_0 with the stored alpha, beta;
    // psi = sum_j y_j v_j, then normalised
    const int k = out->k;
    ED_TRY_CUDA(cudaMemsetAsync(psi, 0, (size_t)n * sizeof(T), cs));
    k_op_scale<T, T><<<(unsigned)g, OP_THREADS, 0, cs>>>(v0, buf[0], scal, n);
    ED_LAUNCHED(1);
    for (int i = 0; i < k; ++i) {
      T *v = buf[i % 3], *w = buf[(i + 1) % 3], *vp = i > 0 ? buf[(i + 2) % 3] : nullptr;
      k_op_axpy<T><<<(unsigned)g, OP_THREADS, 0, cs>>>(psi, v, (T)out->y[i], n);
      ED_LAUNCHED(1);
      if (i + 1 == k) break;
      ED_TRY(op.apply(v, w, cs));
      ++out->matvecs;
      k_op_update<T><<<(unsigned)g, OP_THREADS, 0, cs>>>(w, v, vp, st->alpha + i, st->beta + i,
                                                         n, parts);
      ED_LAUNCHED(1);
      k_op_scale<T, T><<<(unsigned)g, OP_THREADS, 0, cs>>>(w, w, st->beta + i + 1, n);
      ED_LAUNCHED(1);
    }
    ED_TRY(ed_op_norm<T>(psi, n, scal + 1, parts, cs));
    k_op_scale<T, T><<<(unsigned)g, OP_THREADS, 0, cs>>>(psi, psi, scal + 1, n);
    ED_LAUNCHED(1);
  }
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  return ED_OK;
}

// ||A psi - e psi|| / ||psi|| and e = <psi, A psi> / <psi, psi> in FP64
ed_status ed_op_residual(const LinOp<double> &op, const double *psi, double *e, double *r,
                         cudaStream_t cs) {
  const int64_t n = op.n, g = op_grid(n);
  const size_t vb = ((size_t)n * sizeof(double) + 255) & ~(size_t)255;
  OpWork ws;
  ws.cs = cs;
  ED_TRY(ed_dmalloc(&ws.mem, vb + (OP_MAX_PARTS + 8) * sizeof(double), cs, "residual"));
  double *w = (double *)ws.mem;
  double *parts = (double *)((char *)ws.mem + vb), *scal = parts + OP_MAX_PARTS;
  ED_TRY_CUDA(cudaMemsetAsync(w, 0, vb, cs));
  ED_TRY(op.apply(psi, w, cs));
  k_op_dot<double><<<(unsigned)g, OP_THREADS, 0, cs>>>(psi, w, n, parts);
  ED_LAUNCHED(1);
  k_op_finish<false><<<1, OP_THREADS, 0, cs>>>(parts, (int)g, scal);
  ED_LAUNCHED(1);
  k_op_dot<double><<<(unsigned)g, OP_THREADS, 0, cs>>>(psi, psi, n, parts);
  ED_LAUNCHED(1);
  k_op_finish<false><<<1, OP_THREADS, 0, cs>>>(parts, (int)g, scal + 1);
  ED_LAUNCHED(1);
  double h[2];
  ED_TRY_CUDA(cudaMemcpyAsync(h, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, cs));
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  const double nn = h[1];
  *e = nn > 0 ? h[0] / nn : 0.0;
  // w - e psi
  k_op_axpy<double><<<(unsigned)g, OP_THREADS, 0, cs>>>(w, psi, -*e, n);
  ED_LAUNCHED(1);
  ED_TRY(ed_op_norm<double>(w, n, scal + 2, parts, cs));
  ED_TRY_CUDA(cudaMemcpyAsync(h, scal + 2, sizeof(double), cudaMemcpyDeviceToHost, cs));
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  *r = nn > 0 ? h[0] / sqrt(nn) : 0.0;
  return ED_OK;
}

// y = x / ||x|| (FP64 norm), converting the type
template <typename Ti, typename To>
ed_status ed_op_normalised_copy(const Ti *x, To *y, int64_t n, cudaStream_t cs) {
  const int64_t g = op_grid(n);
  OpWork ws;
  ws.cs = cs;
  ED_TRY(ed_dmalloc(&ws.mem, (OP_MAX_PARTS + 8) * sizeof(double), cs, "normalised copy"));
  double *parts = (double *)ws.mem, *scal = parts + OP_MAX_PARTS;
  ED_TRY(ed_op_norm<Ti>(x, n, scal, parts, cs));
  k_op_scale<Ti, To><<<(unsigned)g, OP_THREADS, 0, cs>>>(x, y, scal, n);
  ED_LAUNCHED(1);
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  return ED_OK;
}

template ed_status ed_op_lanczos<float>(const LinOp<float> &, const float *, int, double, bool,
                                        OpRun *, LanczosState *, float *, cudaStream_t);
template ed_status ed_op_lanczos<double>(const LinOp<double> &, const double *, int, double, bool,
                                         OpRun *, LanczosState *, double *, cudaStream_t);
template ed_status ed_op_normalised_copy<float, double>(const float *, double *, int64_t,
                                                        cudaStream_t);
template ed_status ed_op_normalised_copy<double, double>(const double *, double *, int64_t,
                                                         cudaStream_t);
template ed_status ed_op_normalised_copy<double, float>(const double *, float *, int64_t,
                                                        cudaStream_t);
template ed_status ed_op_normalised_copy<float, float>(const float *, float *, int64_t,
                                                       cudaStream_t);
