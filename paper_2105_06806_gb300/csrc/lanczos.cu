// Lanczos ground state on the device (Sec. 6.6): plain Lanczos in the Paige
// form without re-orthogonalisation, FP64 scalars, lowest Ritz pair of the
// tridiagonal matrix by Sturm multisection, second pass for the ground-state
// vector, and an FP64 polish for the FP32 modes.
//
// Per step j the host enqueues four kernels (captured in a CUDA graph and
// replayed in chunks; every kernel exits at once when the device-side state
// says the recurrence has stopped):
//   k_hv<LANCZOS>   H v_j, block partials of <v_j, H v_j>
//   k_alpha         alpha_j = <v_j, H v_j> - beta_j <v_j, v_{j-1}> (Paige's
//                   <v_j, H v_j - beta_j v_{j-1}> by linearity; partials
//                   summed in a fixed order)
//   k_axpy_norm     w = H v_j - beta_j v_{j-1} - alpha_j v_j, block partials of
//                   ||w||^2 and <w, v_j>
//   k_beta          beta_{j+1}, lazy scale of v_{j+1} = w / beta_{j+1},
//                   Ritz value, residual estimate, stop test
// Vectors rotate over three buffers (v_j in buffer j%3) and carry a lazy
// scale factor so that no normalisation pass is needed.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

constexpr int SCALAR_THREADS = 512;
constexpr int AXPY_THREADS = 256;
// Reductions of the FP32 modes sum at most FLUSH products per thread in FP32
// before adding them into an FP64 accumulator (every partial across threads,
// warps and CTAs is FP64): the FP64 pipe is slow on this GPU, so the
// elementwise products stay FP32, but no FP32 sum runs over more than FLUSH
// terms.
constexpr int FLUSH = 16;

// ----------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Deterministic sum of n partials by one CTA: thread t adds the strided
// subsequence t, t+T, ... in order, then a fixed tree.
__device__ double cta_sum_parts(const double *p, int64_t n, double *red) {
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = s;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += red[k];
    red[0] = tot;
  }
  __syncthreads();
  tot = red[0];
  __syncthreads();
  return tot;
}

template <typename T>
__device__ __forceinline__ T fmaT(T a, T b, T c);
template <>
__device__ __forceinline__ float fmaT<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fmaT<double>(double a, double b, double c) {
  return __fma_rn(a, b, c);
}
template <typename T>
__device__ __forceinline__ T mulT(T a, T b);
template <>
__device__ __forceinline__ float mulT<float>(float a, float b) { return __fmul_rn(a, b); }
template <>
__device__ __forceinline__ double mulT<double>(double a, double b) { return __dmul_rn(a, b); }

// ----------------------------------------------------------------- tridiagonal

// The helpers below read T_k from shared-memory copies: a[i] = alpha_i,
// b[i] = beta_i, b2[i] = beta_i^2 (i < k; b[0] unused), so that their serial
// recurrences wait on shared rather than global loads.

// FP64 is the slow pipe of this part, so the recurrences below keep only
// their arithmetic there: the sign, zero and range tests read the bits of a
// double in the integer pipe.  The rescaling multiplies by a power of two,
// which is exact, so where it happens does not change any result.
__device__ __forceinline__ bool neg_bit(double x) { return __double2hiint(x) < 0; }
__device__ __forceinline__ bool is_zero(double x) { return (__double_as_longlong(x) << 1) == 0; }
// biased exponent of |x| (0 for zero and subnormals)
__device__ __forceinline__ int bexp(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }
// |x| above about 1e200 or (nonzero and) below about 1e-200
__device__ __forceinline__ bool out_of_range(int e) { return e > 1023 + 664 || e < 1023 - 664; }
// 2^(1022 - e): brings a double of biased exponent e into [0.5, 1) in magnitude
__device__ __forceinline__ double rescale_factor(int e) {
  return __hiloint2double((2045 - e) << 20, 0);
}

// Sturm count: eigenvalues of T_k below x = sign changes of the leading
// principal minors p_i = det(T_i - x) (division-free recurrence, rescaled by
// powers of two; an exact zero counts as a change, as a tiny negative pivot).
__device__ int sturm_count(const double *a, const double *b2, int k, double x) {
  double pm = 1.0, p = a[0] - x;
  int cnt = 0;
  if (p <= 0.0) {
    if (p == 0.0) p = -1e-300;
    cnt = 1;
  }
  for (int i = 1; i < k; ++i) {
    double pn = (a[i] - x) * p - b2[i] * pm;
    if (is_zero(pn)) pn = neg_bit(p) ? 1e-300 : -1e-300;
    cnt += neg_bit(pn) != neg_bit(p);
    pm = p;
    p = pn;
    const int e = bexp(p);
    if (out_of_range(e)) {
      const double f = rescale_factor(e);
      p *= f;
      pm *= f;
    }
  }
  return cnt;
}

// Squared last component of the normalised eigenvector of T_k for the
// eigenvalue theta: -p_{k-1}(theta) / p_k'(theta).
__device__ double last_component_sq(const double *a, const double *b2, int k, double x) {
  double pm = 1.0, p = a[0] - x;
  double dpm = 0.0, dp = -1.0;
  for (int i = 1; i < k; ++i) {
    double pn = (a[i] - x) * p - b2[i] * pm;
    double dpn = -p + (a[i] - x) * dp - b2[i] * dpm;
    pm = p;
    p = pn;
    dpm = dp;
    dp = dpn;
    // rescaled by the largest magnitude of the four (none when all are zero)
    const int e = max(max(bexp(p), bexp(pm)), max(bexp(dp), bexp(dpm)));
    if (e > 1023 + 664 ||
        (e < 1023 - 664 && !(is_zero(p) && is_zero(pm) && is_zero(dp) && is_zero(dpm)))) {
      const double f = rescale_factor(e);
      p *= f;
      pm *= f;
      dp *= f;
      dpm *= f;
    }
  }
  if (dp == 0.0) return 0.0;
  double r = -pm / dp;
  return r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
}

// Ritz vector of T_k for theta by inverse iteration with the tridiagonal
// (Thomas) solver: `sweeps` sweeps from a flat start, normalised, largest
// entry positive.  One thread.  The factorisation is formed once: rpiv[i] =
// 1 / pivot_i and mult[i] = beta_i / pivot_{i-1} (scratch of k entries each);
// y receives k entries.
__device__ void ritz_vector(const double *a, const double *b, int k, double th, int sweeps,
                            double *rpiv, double *mult, double *y) {
  const double shift = th - 1e-13 * fmax(1.0, fabs(th));
  double piv = a[0] - shift;
  if (piv == 0.0) piv = 1e-300;
  rpiv[0] = 1.0 / piv;
  for (int i = 1; i < k; ++i) {
    const double m = b[i] * rpiv[i - 1];
    mult[i] = m;
    double di = a[i] - shift - m * b[i];
    if (di == 0.0) di = 1e-300;
    rpiv[i] = 1.0 / di;
  }
  const double y0 = 1.0 / sqrt((double)k);
  for (int i = 0; i < k; ++i) y[i] = y0;
  for (int it = 0; it < sweeps; ++it) {
    double yp = y[0];
    for (int i = 1; i < k; ++i) {
      yp = y[i] - mult[i] * yp;
      y[i] = yp;
    }
    yp = yp * rpiv[k - 1];
    y[k - 1] = yp;
    double s = yp * yp;
    for (int i = k - 2; i >= 0; --i) {
      yp = (y[i] - b[i + 1] * yp) * rpiv[i];
      y[i] = yp;
      s += yp * yp;
    }
    s = 1.0 / sqrt(s);
    for (int i = 0; i < k; ++i) y[i] *= s;
  }
  int im = 0;
  for (int i = 1; i < k; ++i)
    if (fabs(y[i]) > fabs(y[im])) im = i;
  if (y[im] < 0.0)
    for (int i = 0; i < k; ++i) y[i] = -y[i];
}

// Copies T_k of the device state into shared memory (all threads).
__device__ void stage_tridiag(const LanczosState *st, int k, double *a, double *b, double *b2) {
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    a[i] = st->alpha[i];
    const double bi = st->beta[i];
    b[i] = bi;
    b2[i] = bi * bi;
  }
  __syncthreads();
}

// Lowest eigenvalue of T_k by multisection on one warp: each of the 32 lanes
// evaluates the Sturm count at one interior point, the bracket shrinks by 33
// per round.  (FP64 is the slow pipe on this part: 32 counts per round cost
// far less than a CTA-wide section, at a few more rounds.)  Called by the
// whole CTA; the result is returned to every thread.
__device__ double lowest_eigenvalue(const double *a, const double *b, const double *b2, int k,
                                    double hint_hi, double hint_lo) {
  __shared__ double s_theta;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const unsigned full = 0xffffffffu;
    // Gershgorin bracket
    double lo = 1e300, hi = -1e300;
    for (int i = lane; i < k; i += 32) {
      const double rad = (i > 0 ? fabs(b[i]) : 0.0) + (i + 1 < k ? fabs(b[i + 1]) : 0.0);
      lo = fmin(lo, a[i] - rad);
      hi = fmax(hi, a[i] + rad);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(full, lo, o));
      hi = fmax(hi, __shfl_xor_sync(full, hi, o));
    }
    // warm bracket [hint_lo, hint_hi] when it provably contains the minimum
    if (hint_hi < hi && hint_lo > lo && hint_lo < hint_hi) {
      int c = 0;
      if (lane == 0) c = sturm_count(a, b2, k, hint_lo) == 0;
      if (lane == 1) c = sturm_count(a, b2, k, hint_hi) >= 1;
      const int c0 = __shfl_sync(full, c, 0), c1 = __shfl_sync(full, c, 1);
      if (c0 && c1) {
        lo = hint_lo;
        hi = hint_hi;
      }
    }
    for (int round = 0; round < 128; ++round) {
      if (!(hi - lo > 4e-16 * fmax(1.0, fmax(fabs(lo), fabs(hi))))) break;
      const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
      const bool below = x > lo && x < hi && sturm_count(a, b2, k, x) >= 1;
      const unsigned m = __ballot_sync(full, below);
      const int f = m ? __ffs(m) - 1 : 32;
      const double nlo = f == 0 ? lo : lo + (hi - lo) * (double)f / 33.0;
      double nhi = f == 32 ? hi : lo + (hi - lo) * (double)(f + 1) / 33.0;
      if (nlo == lo && nhi == hi) nhi = lo;  // no progress possible: stop
      lo = nlo;
      hi = fmax(nhi, nlo);
    }
    if (lane == 0) s_theta = 0.5 * (lo + hi);
  }
  __syncthreads();
  const double th = s_theta;
  __syncthreads();
  return th;
}

// ----------------------------------------------------------------- kernels

// alpha_j = <v_j, H v_j - beta_j v_{j-1}> = <v_j, H v_j> - beta_j <v_j, v_{j-1}>:
// the product leaves the partials of <v_j, H v_j>; <v_j, v_{j-1}> comes from
// the previous step's update (k_axpy_norm, k_beta).
__global__ void k_alpha(LanczosState *st, const double *part, const int64_t nparts) {
  __shared__ double red[SCALAR_THREADS / 32];
  if (st->done) return;
  double s = cta_sum_parts(part, nparts, red);
  if (threadIdx.x == 0) {
    const int j = st->j;
    st->alpha[j] = j > 0 ? s - st->beta[j] * st->cvv : s;
  }
}

// w = H v_j - beta_j v_{j-1} - alpha_j v_j in place of H v_j (the product's
// output), with block partials of ||w||^2 (part[0, g)) and of <w, v_j>
// (part[g, 2g), g = gridDim.x) for the next step's <v_{j+1}, v_j>.  The
// operations per element are those of the second pass's product epilogue,
// so both passes form the same vectors bit for bit.
// 16-byte vector of the element type: 4 floats or 2 doubles.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using V = float4;
  static constexpr int N = 4;
  __device__ static void get(const V &v, float *x) { x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w; }
  __device__ static V make(const float *x) { return make_float4(x[0], x[1], x[2], x[3]); }
};
template <>
struct Vec16<double> {
  using V = double2;
  static constexpr int N = 2;
  __device__ static void get(const V &v, double *x) { x[0] = v.x; x[1] = v.y; }
  __device__ static V make(const double *x) { return make_double2(x[0], x[1]); }
};

template <typename T>
__global__ void __launch_bounds__(AXPY_THREADS) k_axpy_norm(LanczosState *st, T *b0, T *b1, T *b2,
                                                            T *const *basis, int64_t n,
                                                            double *part, T *psi = nullptr) {
  __shared__ double red[2][AXPY_THREADS / 32];
  if (st->done) return;
  const int j = st->j;
  T *bufs[3] = {b0, b1, b2};
  const T *v = basis ? basis[j] : bufs[j % 3];
  const T *prev = basis ? basis[j > 0 ? j - 1 : 0] : bufs[(j + 2) % 3];
  T *w = basis ? basis[j + 1] : bufs[(j + 1) % 3];
  const T s = (T)st->scale[j % 3];
  const T s_prev = (T)st->scale[(j + 2) % 3];
  const T al = (T)st->alpha[j];
  const T be = (T)st->beta[j];
  // Block-major vectors are 16-byte aligned and their length is a multiple
  // of 4 elements: 16-byte accesses, one vector per thread and iteration.
  // Per-thread sums in T over at most FLUSH elements, then into FP64.
  using VT = Vec16<T>;
  constexpr int NV = VT::N;
  constexpr int GROUP = FLUSH / NV;  // vectors per FP64 flush
  const typename VT::V *vv = reinterpret_cast<const typename VT::V *>(v);
  const typename VT::V *pv = reinterpret_cast<const typename VT::V *>(prev);
  typename VT::V *wv = reinterpret_cast<typename VT::V *>(w);
  // second pass of a two-pass sector, every other step: psi += y_{j-1} v_{j-1}
  // then psi += y_j v_j (v_{j-1} is read for the update anyway; the same two
  // operations as two one-vector steps, so the same psi bit for bit, at half
  // its traffic)
  typename VT::V *psv = reinterpret_cast<typename VT::V *>(psi);
  const T yj = psi ? (T)st->y[j] : T(0);
  const T yp = psi && j > 0 ? (T)st->y[j - 1] : T(0);
  const int64_t nv = n / NV;
  double accd = 0.0, cvvd = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  while (i < nv) {
    T acc = T(0), cvv = T(0);
#pragma unroll
    for (int g = 0; g < GROUP; ++g, i += stride) {
      if (i >= nv) break;
      T x[NV], pr[NV], vi[NV];
      VT::get(wv[i], x);
      VT::get(vv[i], vi);
      if (j > 0) VT::get(pv[i], pr);
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        if (j > 0) x[q] = fmaT<T>(-be, mulT<T>(pr[q], s_prev), x[q]);
        vi[q] = mulT<T>(vi[q], s);
        x[q] = fmaT<T>(-al, vi[q], x[q]);
        acc = fmaT<T>(x[q], x[q], acc);
        cvv = fmaT<T>(x[q], vi[q], cvv);
      }
      wv[i] = VT::make(x);
      if (psi) {
        T ps[NV];
        VT::get(psv[i], ps);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          ps[q] = fmaT<T>(yp, mulT<T>(pr[q], s_prev), ps[q]);
          ps[q] = fmaT<T>(yj, vi[q], ps[q]);
        }
        psv[i] = VT::make(ps);
      }
    }
    accd += (double)acc;
    cvvd += (double)cvv;
  }
  double d = warp_sum(accd), c = warp_sum(cvvd);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = d;
    red[1][wid] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0, totc = 0.0;
    for (int k = 0; k < AXPY_THREADS / 32; ++k) {
      tot += red[0][k];
      totc += red[1][k];
    }
    part[blockIdx.x] = tot;
    part[gridDim.x + blockIdx.x] = totc;
  }
}

// beta_{j+1}, scale, Ritz value and stop test.  The Ritz value is evaluated
// at steps 1 and 2, at the scheduled steps (next_check) and at the last step.
__global__ void k_beta(LanczosState *st, const double *part, int64_t nparts) {
  __shared__ double red[SCALAR_THREADS / 32];
  __shared__ int stop;
  // T_k, its squared off-diagonal, then (inverse iteration) pivots and y
  __shared__ double s_a[ED_MAX_LANCZOS], s_b[ED_MAX_LANCZOS], s_b2[ED_MAX_LANCZOS];
  __shared__ double s_rp[ED_MAX_LANCZOS], s_y[ED_MAX_LANCZOS];
  __shared__ double s_be, s_hint[2];
  if (st->done) return;
  double s2 = cta_sum_parts(part, nparts, red);
  const double c2 = cta_sum_parts(part + nparts, nparts, red);  // <w, v_j>
  const int j = st->j;
  // scalar work once, by thread 0 (FP64 is the slow pipe)
  if (threadIdx.x == 0) {
    const double al = st->alpha[j];
    const double be = sqrt(fmax(s2, 0.0));
    s_be = be;
    st->beta[j + 1] = be;
    st->cvv = be > 0.0 ? c2 / be : 0.0;
    st->scale[(j + 1) % 3] = be > 0.0 ? 1.0 / be : 0.0;
    st->tnorm = fmax(st->tnorm, fmax(fabs(al), be));
    stop = 0;
    if (be <= 1e-13 * st->tnorm) stop = 2;
    else if (j + 1 >= st->maxit) stop = 3;
  }
  __syncthreads();
  const int k = j + 1;
  const bool scheduled = k >= st->next_check;
  const bool want = st->tol > 0.0 && (stop != 0 || scheduled || k <= 2);
  if (want) {
    stage_tridiag(st, k, s_a, s_b, s_b2);
    const double prev = st->theta;
    if (threadIdx.x == 0) {
      const double dl = isfinite(st->acc[3]) ? fabs(st->acc[3]) : 0.0;
      s_hint[0] = (k > 1 && isfinite(prev)) ? prev : 1e300;
      s_hint[1] = (k > 1 && isfinite(prev)) ? prev - fmax(8.0 * dl, 1e-9 * fmax(1.0, fabs(prev)))
                                             : -1e300;
    }
    __syncthreads();
    const double th = lowest_eigenvalue(s_a, s_b, s_b2, k, s_hint[0], s_hint[1]);
    __shared__ int ritz;
    if (threadIdx.x == 0) {
      const double be = s_be;
      double y2 = last_component_sq(s_a, s_b2, k, th);
      double rest = be * sqrt(y2);
      // The polynomial formula loses relative accuracy once the Ritz value
      // has converged; near convergence use inverse iteration instead.
      ritz = rest < 1e-6 * fmax(1.0, fabs(th));
      if (ritz) {
        // the last component is tiny near convergence: three sweeps push the
        // other eigencomponents well below it
        ritz_vector(s_a, s_b, k, th, 3, s_rp, s_b2, s_y);
        rest = be * fabs(s_y[k - 1]);
      }
      st->acc[3] = isfinite(prev) ? th - prev : 1e300;
      st->theta = th;
      st->rest = rest;
      // converged, also when the test falls on the max_iter step
      if ((stop == 0 || stop == 3) && rest <= st->tol * fmax(1.0, fabs(th)) && k >= 2) stop = 1;
      if (scheduled)
        st->next_check = k + max(st->check_every, (int)ceil(st->check_growth * (double)k));
    }
    __syncthreads();
    if (ritz)
      for (int i = threadIdx.x; i < k; i += blockDim.x) st->y[i] = s_y[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (stop) st->done = stop;
    st->j = k;
  }
}

// Start vector: element i = u_i - 1/2 with u_i the uniform double of output i
// of a SplitMix64 stream seeded with `seed` (Steele, Lea, Flood 2014; top 53
// bits times 2^-53), in sector order.  Partial sums of squares per CTA.

// The vector lives in padded block-major order: element (r', pc) holds the
// start value of sector index pidx_dw[r'] * D_up + pidx_up[padinv[pc]], and
// padding columns (padinv < 0) hold zero.
template <typename T>
__global__ void __launch_bounds__(AXPY_THREADS) k_start_vector(T *v, int64_t n, uint64_t seed,
                                                               const int32_t *pidx_up,
                                                               const int32_t *pidx_dw,
                                                               const int32_t *padinv,
                                                               int64_t stride, int64_t dup,
                                                               double *part) {
  __shared__ double red[AXPY_THREADS / 32];
  double accd = 0.0;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;) {
    T acc = T(0);
    for (int k = 0; k < FLUSH && i < n; ++k, i += step) {
      const int64_t r = i / stride, pc = i - r * stride;
      const int32_t cb = padinv[pc];
      T x = T(0);
      if (cb >= 0) {
        const uint64_t p = (uint64_t)pidx_dw[r] * (uint64_t)dup + (uint64_t)pidx_up[cb];
        double u = (double)(ed_splitmix64_at(seed, p) >> 11) * (1.0 / 9007199254740992.0);
        x = (T)(u - 0.5);
      }
      v[i] = x;
      acc = fmaT<T>(x, x, acc);
    }
    accd += (double)acc;
  }
  double d = warp_sum(accd);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int k = 0; k < AXPY_THREADS / 32; ++k) tot += red[k];
    part[blockIdx.x] = tot;
  }
}

// Sum of squares of a vector (partials per CTA).
template <typename T>
__global__ void __launch_bounds__(AXPY_THREADS) k_norm2(const T *v, int64_t n, double *part) {
  __shared__ double red[AXPY_THREADS / 32];
  double accd = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;) {
    T acc = T(0);
    for (int k = 0; k < FLUSH && i < n; ++k, i += stride) acc = fmaT<T>(v[i], v[i], acc);
    accd += (double)acc;
  }
  double d = warp_sum(accd);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int k = 0; k < AXPY_THREADS / 32; ++k) tot += red[k];
    part[blockIdx.x] = tot;
  }
}

// Initialise the recurrence state: v_0 = buffer 0 scaled by 1/||buffer 0||.
__global__ void k_state_init(LanczosState *st, const double *part, int64_t nparts, int maxit,
                             double tol, int check_every, double check_growth) {
  __shared__ double red[SCALAR_THREADS / 32];
  double s = cta_sum_parts(part, nparts, red);
  if (threadIdx.x == 0) {
    st->j = 0;
    st->done = s > 0.0 ? 0 : 2;
    st->maxit = maxit;
    st->check_every = check_every;
    st->next_check = check_every;
    st->check_growth = check_growth;
    st->tol = tol;
    st->tnorm = 0.0;
    st->theta = INFINITY;
    st->rest = INFINITY;
    st->scale[0] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    st->scale[1] = 0.0;
    st->scale[2] = 0.0;
    st->beta[0] = 0.0;
    st->cvv = 0.0;
    st->acc[0] = s;
    st->acc[1] = st->acc[2] = 0.0;
    st->acc[3] = INFINITY;
  }
}

// Final Ritz vector of T_k (4 inverse-iteration sweeps): staged by the CTA,
// solved by one thread.  Dynamic shared memory: 5 * ED_MAX_LANCZOS doubles.
constexpr int TRIDIAG_THREADS = 128;
__global__ void k_tridiag_vector(LanczosState *st, int k) {
  extern __shared__ double sh[];
  double *a = sh, *b = sh + ED_MAX_LANCZOS, *b2 = sh + 2 * ED_MAX_LANCZOS;
  double *rp = sh + 3 * ED_MAX_LANCZOS, *y = sh + 4 * ED_MAX_LANCZOS;
  stage_tridiag(st, k, a, b, b2);
  if (threadIdx.x == 0) ritz_vector(a, b, k, st->theta, 4, rp, b2, y);
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) st->y[i] = y[i];
}

// Second pass bookkeeping: v_{j+1} = w / beta_{j+1}.
__global__ void k_second_advance(LanczosState *st) {
  const int j = st->j;
  const double be = st->beta[j + 1];
  st->scale[(j + 1) % 3] = be > 0.0 ? 1.0 / be : 0.0;
  st->j = j + 1;
}

// Second pass resumed at step m from the stored v_{m-1}, v_m (buffers
// (m-1) % 3 and m % 3 of the pass): the step counter and the two scales.
__global__ void k_second_resume(LanczosState *st, int m) {
  const double s0 = st->acc[0] > 0.0 ? 1.0 / sqrt(st->acc[0]) : 0.0;  // v_0 = start / ||start||
  st->j = m;
  st->done = 0;  // the Lanczos-mode kernels of the split second pass test it
  st->scale[m % 3] = m == 0 ? s0 : (st->beta[m] > 0.0 ? 1.0 / st->beta[m] : 0.0);
  if (m > 0)
    st->scale[(m - 1) % 3] = m == 1 ? s0 : (st->beta[m - 1] > 0.0 ? 1.0 / st->beta[m - 1] : 0.0);
}

// psi += y_j * scale * buf (last vector of the second pass), preceded by
// psi += y_{j-1} v_{j-1} when that vector is still pending (paired steps).
template <typename T>
__global__ void k_psi_tail(const LanczosState *st, const T *b0, const T *b1, const T *b2, T *psi,
                           int64_t n, int pending) {
  const int j = st->j;
  const T *bufs[3] = {b0, b1, b2};
  const T *v = bufs[j % 3];
  const T s = (T)st->scale[j % 3];
  const T y = (T)st->y[j];
  const T *vp = bufs[(j + 2) % 3];
  const T sp = (T)st->scale[(j + 2) % 3];
  const T yp = pending && j > 0 ? (T)st->y[j - 1] : T(0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    T p = psi[i];
    if (pending) p = fmaT<T>(yp, mulT<T>(vp[i], sp), p);
    psi[i] = fmaT<T>(y, mulT<T>(v[i], s), p);
  }
}

template <typename Ti, typename To>
__global__ void k_scale_copy(const Ti *x, To *y, int64_t n, const double *part, int64_t nparts) {
  __shared__ double red[AXPY_THREADS / 32];
  __shared__ double sc;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    sc = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
  }
  __syncthreads();
  const double f = sc;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = (To)((double)x[i] * f);
}

// Layout changes between sector order ([D_dw][D_up], ascending strings) and
// padded block-major order ([D_dw][bstride]):
//   blocked[r'][pc] = sector[pidx_dw[r']][pidx_up[padinv[pc]]]  (0 at padding)
//   sector[r][c]    = blocked[inv_dw[r]][colpos[inv_up[c]]]
// One grid row per output row; the gathers stay inside one input row.
template <typename Ti, typename To>
__global__ void k_to_blocked(const Ti *in, To *out, const int32_t *pidx_dw,
                             const int32_t *pidx_up, const int32_t *padinv, int64_t dup,
                             int64_t stride, int64_t ddw) {
  for (int64_t r = blockIdx.y; r < ddw; r += gridDim.y) {
    const Ti *src = in + (int64_t)pidx_dw[r] * dup;
    To *dst = out + r * stride;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < stride;
         c += (int64_t)gridDim.x * blockDim.x) {
      const int32_t cb = padinv[c];
      dst[c] = cb < 0 ? To(0) : (To)src[pidx_up[cb]];
    }
  }
}

template <typename Ti, typename To>
__global__ void k_from_blocked(const Ti *in, To *out, const int32_t *inv_dw, const int32_t *inv_up,
                               const int32_t *colpos, int64_t dup, int64_t stride, int64_t ddw) {
  for (int64_t r = blockIdx.y; r < ddw; r += gridDim.y) {
    const Ti *src = in + (int64_t)inv_dw[r] * stride;
    To *dst = out + r * dup;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < dup;
         c += (int64_t)gridDim.x * blockDim.x)
      dst[c] = (To)src[colpos[inv_up[c]]];
  }
}

template <typename Ti, typename To>
static ed_status permute_layout(ed_sector s, const Ti *in, To *out, bool to_blocked,
                                cudaStream_t cs) {
  const int64_t dup = s->sp[0].dim, ddw = s->sp[1].dim, stride = s->bstride;
  const int64_t cols = to_blocked ? stride : dup;
  dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((cols + 255) / 256, 64)),
            (unsigned)std::max<int64_t>(1, std::min<int64_t>(ddw, 65535)));
  if (to_blocked)
    k_to_blocked<Ti, To><<<grid, 256, 0, cs>>>(in, out, s->bi[1].pidx, s->bi[0].pidx, s->padinv,
                                               dup, stride, ddw);
  else
    k_from_blocked<Ti, To><<<grid, 256, 0, cs>>>(in, out, s->bi[1].inv, s->bi[0].inv, s->colpos,
                                                 dup, stride, ddw);
  ED_LAUNCHED(1);
  return ED_OK;
}

// Residual of psi: pass 1 forms <psi,w> and ||psi||^2 per CTA (w = H psi),
// k_rq_final the Rayleigh quotient e; pass 2 forms ||w - e psi||^2 directly
// (no cancellation), k_resid_final the normalised residual.
__global__ void __launch_bounds__(AXPY_THREADS) k_rq_parts(const double *psi, const double *w,
                                                           int64_t n, double *part,
                                                           int64_t nparts) {
  __shared__ double red[2][AXPY_THREADS / 32];
  double a = 0, c = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    a = fma(psi[i], w[i], a);
    c = fma(psi[i], psi[i], c);
  }
  a = warp_sum(a);
  c = warp_sum(c);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0, tc = 0;
    for (int k = 0; k < AXPY_THREADS / 32; ++k) {
      ta += red[0][k];
      tc += red[1][k];
    }
    part[blockIdx.x] = ta;
    part[nparts + blockIdx.x] = tc;
  }
}

__global__ void k_rq_final(const double *part, int64_t nparts, double *out) {
  __shared__ double red[SCALAR_THREADS / 32];
  double a = cta_sum_parts(part, nparts, red);
  double c = cta_sum_parts(part + nparts, nparts, red);
  if (threadIdx.x == 0) {
    out[0] = a / c;
    out[2] = c;
  }
}

__global__ void __launch_bounds__(AXPY_THREADS) k_resid_parts(const double *psi, const double *w,
                                                              int64_t n, const double *out,
                                                              double *part) {
  __shared__ double red[AXPY_THREADS / 32];
  const double e = out[0];
  double b = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const double r = fma(-e, psi[i], w[i]);
    b = fma(r, r, b);
  }
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < AXPY_THREADS / 32; ++k) t += red[k];
    part[blockIdx.x] = t;
  }
}

__global__ void k_resid_final(const double *part, int64_t nparts, double *out) {
  __shared__ double red[SCALAR_THREADS / 32];
  double b = cta_sum_parts(part, nparts, red);
  if (threadIdx.x == 0) out[1] = sqrt(b / out[2]);
}

// Ground state from a stored Krylov basis: psi = sum_{j<k} y_j (s_j v_j), in
// j order and with the operations of the second pass (s_j = 1/beta_j, the
// scale the first pass gave v_j), so psi is the one the second pass builds.
template <typename T>
__global__ void k_basis_coeffs(const LanczosState *st, int k, T *coef) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double sj;
    if (j == 0) sj = st->acc[0] > 0.0 ? 1.0 / sqrt(st->acc[0]) : 0.0;
    else sj = st->beta[j] > 0.0 ? 1.0 / st->beta[j] : 0.0;
    coef[j] = (T)st->y[j];
    coef[ED_MAX_LANCZOS + 2 + j] = (T)sj;
  }
}

template <typename T>
__global__ void __launch_bounds__(AXPY_THREADS) k_basis_combine(T *const *basis, const T *coef,
                                                                int k, T *psi, int64_t n) {
  __shared__ const T *s_v[ED_MAX_LANCZOS + 2];
  __shared__ T s_y[ED_MAX_LANCZOS + 2], s_s[ED_MAX_LANCZOS + 2];
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    s_v[j] = basis[j];
    s_y[j] = coef[j];
    s_s[j] = coef[ED_MAX_LANCZOS + 2 + j];
  }
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    T acc = T(0);
#pragma unroll 8
    for (int j = 0; j < k; ++j) acc = fmaT<T>(s_y[j], mulT<T>(s_v[j][i], s_s[j]), acc);
    psi[i] = acc;
  }
}

// ----------------------------------------------------------------- host driver

struct Workspace {
  void *mem = nullptr;
  cudaStream_t st = nullptr;
  ed_status alloc(size_t bytes, cudaStream_t s) {
    st = s;
    return ed_dmalloc(&mem, std::max<size_t>(bytes, 256), s, "Lanczos workspace");
  }
  ~Workspace() { ed_dfree(mem, st); }
};

static int64_t reduce_grid(int64_t n) {
  int64_t g = (n + AXPY_THREADS * 8 - 1) / (AXPY_THREADS * 8);
  return std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8));
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// CUDA graph capture is not allowed on the legacy default stream, so the
// captured Lanczos chunks run on the calling thread's private stream, ordered
// after and before the caller's stream by events.
struct StreamJoin {
  cudaEvent_t ev = nullptr;
  ~StreamJoin() {
    if (ev) cudaEventDestroy(ev);
  }
  ed_status order(cudaStream_t from, cudaStream_t to) {
    if (!ev) ED_TRY_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    ED_TRY_CUDA(cudaEventRecord(ev, from));
    ED_TRY_CUDA(cudaStreamWaitEvent(to, ev, 0));
    return ED_OK;
  }
};

// Krylov basis kept on the device during the first pass, so that the ground
// state needs no second pass (the paper's second pass trades a second run of
// the recurrence for memory; this part has the memory).  Vectors are
// allocated as the run reaches them, up to a byte budget; table[j] is the
// device address of v_j.  Past the budget the run goes on in the three
// rotating buffers (table[j] = rot[j % 3]) and the caller falls back to the
// second pass.  v_0 stays in the workspace buffer where the start vector is
// written; the rotation uses the other two and psi's buffer, which is only
// written after the run.
template <typename T>
struct BasisStore {
  T **d_table = nullptr;         // device table, maxit + 2 entries
  std::vector<T *> table;        // host copy
  std::vector<void *> owned;     // stored vectors v_1 .. v_{cap-1}
  T *v0 = nullptr;               // workspace buffer of the start vector
  T *rot[3] = {nullptr, nullptr, nullptr};  // rotation past the budget
  int cap = 1;                   // v_j with j < cap are kept
  bool full = false;             // budget reached: nothing more is stored
  int filled = 0;                // table entries uploaded
  size_t vbytes = 0, budget = 0, used = 0;
  cudaStream_t st = nullptr;
  ~BasisStore() {
    for (void *p : owned) ed_dfree(p, st);
  }
  // table entries 0 .. upto exist on the device (ordered on cs)
  ed_status ensure(int upto, cudaStream_t cs) {
    st = cs;
    upto = std::min<int>(upto, (int)table.size() - 1);
    if (upto < filled) return ED_OK;
    const int first = filled;
    for (int j = filled; j <= upto; ++j) {
      T *p = nullptr;
      if (j == 0) {
        p = v0;
      } else if (!full && j == cap && used + vbytes <= budget) {
        void *q = nullptr;
        if (ed_dmalloc(&q, vbytes, cs, "Krylov basis") != ED_OK) {
          cudaGetLastError();  // an allocation refused here only ends the storing
          ed_set_error_msg("");
        } else {
          owned.push_back(q);
          used += vbytes;
          ED_TRY_CUDA(cudaMemsetAsync(q, 0, vbytes, cs));  // padding entries stay zero
          p = (T *)q;
          cap = j + 1;
        }
      }
      if (!p) {
        full = true;
        p = rot[j % 3];
      }
      table[j] = p;
    }
    ED_TRY_CUDA(cudaMemcpyAsync(d_table + first, table.data() + first,
                                (upto + 1 - first) * sizeof(T *), cudaMemcpyHostToDevice, cs));
    filled = upto + 1;
    return ED_OK;
  }
};

// Runs Lanczos steps until the device state stops: chunks of `chunk` steps,
// each chunk one CUDA graph launch, then a 4-byte read of the stop flag.
template <typename T>
static ed_status run_steps(ed_sector s, const HvTables<T> &tb, T *const *bufs, LanczosState *st,
                           double *part, double *part2, int64_t n, int maxit, cudaStream_t caller,
                           int *steps_out, int32_t *h_flag, BasisStore<T> *bs = nullptr) {
  int64_t np1 = 0;
  const int64_t g2 = reduce_grid(n);
  int chunk = n < (1 << 20) ? 16 : 4;
  chunk = std::min(chunk, std::max(1, maxit));
  ed_status ps = ED_OK;
  cudaStream_t cs = ed_private_stream(&ps);
  if (ps != ED_OK) return ps;
  StreamJoin join;
  ED_TRY(join.order(caller, cs));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ED_TRY(ed_hv_prepare<T>());
  // product kernels per step: two for the two-pass product, else one; plus
  // the H_nd kernel with spin exchange or pair hopping
  const int64_t hv_per_step = ((tb.ditems && !tb.small_cols) ? 2 : 1) + (tb.nd_up ? 1 : 0);
  ED_TRY_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  ed_status rs = ED_OK;
  for (int it = 0; it < chunk && rs == ED_OK; ++it) {
    T *const *table = bs ? bs->d_table : nullptr;
    rs = ed_launch_hv<T>(s, tb, HV_LANCZOS, nullptr, nullptr, bufs, nullptr, st, part, &np1, cs,
                         table);
    if (rs != ED_OK) break;
    k_alpha<<<1, SCALAR_THREADS, 0, cs>>>(st, part, np1);
    k_axpy_norm<T><<<(unsigned)g2, AXPY_THREADS, 0, cs>>>(st, bufs[0], bufs[1], bufs[2], table, n,
                                                          part2);
    k_beta<<<1, SCALAR_THREADS, 0, cs>>>(st, part2, g2);
  }
  cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  // the captured product launches run inside the graph: count them per replay
  const int64_t hv_launches = hv_per_step * chunk;
  ed_count_launches(-hv_launches);
  if (rs != ED_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rs;
  }
  ED_TRY_CUDA(ce);
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  ED_TRY_CUDA(ce);
  int launched = 0;
  ed_status out = ED_OK;
  while (launched < maxit) {
    if (bs) {
      out = bs->ensure(launched + chunk, cs);  // v_0 .. v_{launched+chunk}
      if (out != ED_OK) break;
    }
    cudaError_t e = cudaGraphLaunch(exec, cs);
    if (e != cudaSuccess) {
      ed_set_cuda_error(e, "cudaGraphLaunch", __FILE__, __LINE__);
      out = ED_ERR_CUDA;
      break;
    }
    ed_count_launches(hv_launches + 3 * (int64_t)chunk);
    launched += chunk;
    e = cudaMemcpyAsync(h_flag, &st->done, sizeof(int32_t), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
      ed_set_cuda_error(e, "Lanczos stop flag", __FILE__, __LINE__);
      out = ED_ERR_CUDA;
      break;
    }
    if (*h_flag) break;
  }
  cudaGraphExecDestroy(exec);
  ed_status js = join.order(cs, caller);
  if (out == ED_OK) out = js;
  if (steps_out) *steps_out = launched;
  return out;
}

// Second pass: rebuild v_{j0+1}..v_{k-1} from the stored coefficients and
// accumulate psi += sum_{j >= j0} y_j v_j (j0 = 0: from the start vector
// with psi zeroed; j0 > 0: psi already holds the terms j < j0 and the state
// was resumed at step j0).
template <typename T>
static ed_status second_pass(ed_sector s, const HvTables<T> &tb, T *const *bufs, T *psi,
                             LanczosState *st, int j0, int k, int64_t n, double *part,
                             double *part2, cudaStream_t cs) {
  if (j0 == 0) ED_TRY_CUDA(cudaMemsetAsync(psi, 0, n * sizeof(T), cs));
  const int64_t g = reduce_grid(n);
  // Two-pass product: the first pass's own kernels (the Lanczos-mode product,
  // then the streaming update, which here also adds y_j v_j into psi) instead
  // of the fused second-pass H_dw epilogue: 14.3 + 3 ms against 19.6 ms per
  // step at Ns=18; the same operations, so the same vectors bit for bit.
  const bool split = tb.ditems && !tb.small_cols;
  for (int j = j0; j + 1 < k; ++j) {
    if (split) {
      int64_t np1 = 0;
      ED_TRY(ed_launch_hv<T>(s, tb, HV_LANCZOS, nullptr, nullptr, bufs, nullptr, st, part, &np1,
                             cs));
      // psi takes v_{j-1} and v_j on every other step (see k_axpy_norm)
      k_axpy_norm<T><<<(unsigned)g, AXPY_THREADS, 0, cs>>>(st, bufs[0], bufs[1], bufs[2], nullptr,
                                                            n, part2,
                                                            ((j - j0) & 1) ? psi : nullptr);
      ED_LAUNCHED(1);
    } else {
      ED_TRY(ed_launch_hv<T>(s, tb, HV_SECOND, nullptr, nullptr, bufs, psi, st, nullptr, nullptr,
                             cs));
    }
    k_second_advance<<<1, 1, 0, cs>>>(st);
    ED_LAUNCHED(1);
  }
  // with paired steps, v_{k-2} is still pending when the pass ran an odd
  // number of steps
  const int pending = split && ((k - 1 - j0) & 1) ? 1 : 0;
  k_psi_tail<T><<<(unsigned)g, AXPY_THREADS, 0, cs>>>(st, bufs[0], bufs[1], bufs[2], psi, n,
                                                       pending);
  ED_LAUNCHED(1);
  return ED_OK;
}

// Spacing of the Ritz-value tests.  A test at step k costs about
// kTestCostMs * k (the FP64 recurrences over T_k in sturm_count and
// last_component_sq, on one warp), a step about step_ms (the product and its
// reductions, estimated from the bytes they move at 1 TB/s plus the launch
// cost).  Testing every d steps spends kTestCostMs * k / d per step and runs
// d / 2 steps past convergence on average; d = k sqrt(2 kTestCostMs /
// step_ms) balances the two, so the tests fall on geometrically spaced steps
// with this growth.  The schedule depends on the sector size only, never on
// a timing, so a solve stops at the same step on every run.
constexpr double kTestCostMs = 3e-3;  // per unit of k, measured on GB300 (k_beta launches)
static double test_growth(int64_t n, size_t elem) {
  const double step_ms = 0.012 + 2.0 * (double)n * (double)elem * 1e-9;
  return sqrt(2.0 * kTestCostMs / step_ms);
}

// One Lanczos solve in precision T on sector s, starting from either the
// seeded vector or (start != nullptr) a given vector in precision T.
template <typename T>
static ed_status lanczos_solve(ed_sector s, int maxit, double tol, uint64_t seed, const T *start,
                               bool want_vector, T *psi_out, LanczosState *h_state,
                               cudaStream_t cs, int *matvecs, int basis_mib) {
  const int64_t n = s->bdim;  // padded block-major vectors
  ED_TRY(ed_build_items(s, 1, (int)sizeof(T)));
  const int64_t np1 = ed_hv_num_parts(s, 1, (int)sizeof(T));
  const int64_t g2 = reduce_grid(n);
  const int64_t nparts = std::max<int64_t>(np1, 3 * g2);
  size_t vb = align256(n * sizeof(T));
  const size_t tbytes = align256((size_t)(maxit + 2) * sizeof(T *));
  const size_t cbytes = align256(2 * (size_t)(ED_MAX_LANCZOS + 2) * sizeof(T));
  size_t bytes = 3 * vb + (want_vector ? vb + tbytes + cbytes : 0) +
                 align256(sizeof(LanczosState)) + 2 * align256(nparts * sizeof(double));
  Workspace ws;
  ED_TRY(ws.alloc(bytes, cs));
  char *p = (char *)ws.mem;
  T *bufs[3];
  for (int b = 0; b < 3; ++b) {
    bufs[b] = (T *)p;
    p += vb;
  }
  T *psi = nullptr;
  if (want_vector) {
    psi = (T *)p;
    p += vb;
  }
  LanczosState *st = (LanczosState *)p;
  p += align256(sizeof(LanczosState));
  double *part = (double *)p;
  p += align256(nparts * sizeof(double));
  double *part2 = (double *)p;
  p += align256(nparts * sizeof(double));
  // padding entries must stay zero in every vector
  ED_TRY_CUDA(cudaMemsetAsync(ws.mem, 0, (3 + (want_vector ? 1 : 0)) * vb, cs));
  // with a vector wanted, the first pass keeps its Krylov basis while the
  // budget allows (see BasisStore)
  BasisStore<T> bs;
  T *coef = nullptr;
  if (want_vector) {
    bs.d_table = (T **)p;
    p += tbytes;
    coef = (T *)p;
    bs.table.assign(maxit + 2, nullptr);
    bs.v0 = bufs[0];
    bs.rot[0] = psi;
    bs.rot[1] = bufs[1];
    bs.rot[2] = bufs[2];
    bs.vbytes = vb;
    if (basis_mib < 0) {
      bs.budget = 0;
    } else if (basis_mib > 0) {
      bs.budget = (size_t)basis_mib << 20;
    } else {
      size_t avail = 0;
      bs.budget = ed_device_available(&avail) == ED_OK ? (size_t)(0.6 * (double)avail) : 0;
    }
  }

  PinnedFlag flag;
  if (!flag.p) {
    ed_set_error_msg("page-locked stop flag allocation failed");
    return ED_ERR_OOM;
  }
  // Ritz-value tests cost FP64 latency on one warp: below 2^20 elements a
  // Lanczos step is cheaper than a test, so test at most every 8 steps there
  const int check_every = n > (1 << 22) ? 1 : (n > (1 << 20) ? 4 : 8);
  const double growth = test_growth(n, sizeof(T));
  auto init = [&]() -> ed_status {
    if (start) {
      ED_TRY_CUDA(cudaMemcpyAsync(bufs[0], start, n * sizeof(T), cudaMemcpyDeviceToDevice, cs));
      k_norm2<T><<<(unsigned)g2, AXPY_THREADS, 0, cs>>>(bufs[0], n, part);
    } else {
      k_start_vector<T><<<(unsigned)g2, AXPY_THREADS, 0, cs>>>(
          bufs[0], n, seed, s->bi[0].pidx, s->bi[1].pidx, s->padinv, s->bstride, s->sp[0].dim,
          part);
    }
    ED_LAUNCHED(1);
    k_state_init<<<1, SCALAR_THREADS, 0, cs>>>(st, part, g2, maxit, tol, check_every, growth);
    ED_LAUNCHED(1);
    return ED_OK;
  };
  ED_TRY(init());
  HvTables<T> tb = ed_hv_tables<T>(s, 1);
  int launched = 0;
  ED_TRY(run_steps<T>(s, tb, bufs, st, part, part2, n, maxit, cs, &launched, flag.p,
                      want_vector ? &bs : nullptr));
  bs.st = cs;  // the stored vectors are released after their last reader below
  ED_TRY_CUDA(cudaMemcpyAsync(h_state, st, sizeof(LanczosState), cudaMemcpyDeviceToHost, cs));
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  const int k = h_state->j;
  int mv = k;
  if (want_vector && k > 0) {
    k_tridiag_vector<<<1, TRIDIAG_THREADS, 5 * sizeof(double) * ED_MAX_LANCZOS, cs>>>(st, k);
    ED_LAUNCHED(1);
    if (k <= bs.cap) {
      // v_0 .. v_{k-1} are all stored: one pass over them
      k_basis_coeffs<T><<<1, 256, 0, cs>>>(st, k, coef);
      ED_LAUNCHED(1);
      k_basis_combine<T><<<(unsigned)g2, AXPY_THREADS, 0, cs>>>(bs.d_table, coef, k, psi, n);
      ED_LAUNCHED(1);
    } else if (bs.cap >= 3) {
      // v_0 .. v_{cap-1} are stored: psi from the stored vectors up to step
      // m - 1 = cap - 2, then the second pass resumed at step m from the
      // stored v_{m-1}, v_m (the same sums in the same order: bit-identical to
      // the full second pass).  The stored pair becomes the pass's rotation,
      // with the free workspace buffer 1 as its third member.
      const int m = bs.cap - 1;
      k_basis_coeffs<T><<<1, 256, 0, cs>>>(st, m, coef);
      ED_LAUNCHED(1);
      k_basis_combine<T><<<(unsigned)g2, AXPY_THREADS, 0, cs>>>(bs.d_table, coef, m, psi, n);
      ED_LAUNCHED(1);
      T *rot2[3];
      rot2[m % 3] = bs.table[m];
      rot2[(m + 2) % 3] = bs.table[m - 1];
      rot2[(m + 1) % 3] = bufs[1];
      k_second_resume<<<1, 1, 0, cs>>>(st, m);
      ED_LAUNCHED(1);
      ED_TRY(second_pass<T>(s, tb, rot2, psi, st, m, k, n, part, part2, cs));
      mv += k - 1 - m;
    } else {
      // restart the recurrence bookkeeping for the second pass
      ED_TRY(init());
      ED_TRY(second_pass<T>(s, tb, bufs, psi, st, 0, k, n, part, part2, cs));
      mv += k - 1;
    }
    // normalise psi into the output
    k_norm2<T><<<(unsigned)g2, AXPY_THREADS, 0, cs>>>(psi, n, part2);
    ED_LAUNCHED(1);
    k_scale_copy<T, T><<<(unsigned)g2, AXPY_THREADS, 0, cs>>>(psi, psi_out, n, part2, g2);
    ED_LAUNCHED(1);
    ED_TRY_CUDA(cudaMemcpyAsync(h_state->y, st->y, sizeof(double) * k, cudaMemcpyDeviceToHost, cs));
  }
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  if (matvecs) *matvecs += mv;
  return ED_OK;
}

// FP64 residual of a normalised FP64 vector in block-major order: returns
// (Rayleigh quotient, ||H psi - e psi||).
static ed_status fp64_residual(ed_sector s, const double *psi, double *e, double *r,
                               cudaStream_t cs) {
  ED_TRY(ed_build_items(s, 1, 8));
  const int64_t n = s->bdim;
  const int64_t g2 = reduce_grid(n);
  size_t bytes = align256(n * sizeof(double)) + align256(3 * g2 * sizeof(double)) + 256;
  Workspace ws;
  ED_TRY(ws.alloc(bytes, cs));
  double *w = (double *)ws.mem;
  double *part = (double *)((char *)ws.mem + align256(n * sizeof(double)));
  double *out = (double *)((char *)part + align256(3 * g2 * sizeof(double)));  // 3 doubles
  ED_TRY_CUDA(cudaMemsetAsync(w, 0, n * sizeof(double), cs));  // padding of H psi
  ED_TRY(ed_launch_hv<double>(s, ed_hv_tables<double>(s, 1), HV_PLAIN, psi, w, nullptr,
                              nullptr, nullptr, nullptr, nullptr, cs));
  k_rq_parts<<<(unsigned)g2, AXPY_THREADS, 0, cs>>>(psi, w, n, part, g2);
  ED_LAUNCHED(1);
  k_rq_final<<<1, SCALAR_THREADS, 0, cs>>>(part, g2, out);
  ED_LAUNCHED(1);
  k_resid_parts<<<(unsigned)g2, AXPY_THREADS, 0, cs>>>(psi, w, n, out, part);
  ED_LAUNCHED(1);
  k_resid_final<<<1, SCALAR_THREADS, 0, cs>>>(part, g2, out);
  ED_LAUNCHED(1);
  double h[3];
  ED_TRY_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, cs));
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  *e = h[0];
  *r = h[1];
  return ED_OK;
}

static void fill_result(const LanczosState &h, ed_lanczos_result *res) {
  res->e0_raw = h.theta;
  res->e0 = h.theta;
  res->residual_estimate = h.rest;
  res->iterations = h.j;
  res->stop_reason = h.done == 1 ? 0 : (h.done == 2 ? 1 : 2);
}

ed_status ed_lanczos_ground_impl(ed_sector s, const ed_lanczos_opts *o, ed_lanczos_result *res,
                                 void *d_psi, cudaStream_t cs) {
  memset(res, 0, sizeof(*res));
  int maxit = o->max_iter > 0 ? o->max_iter : 512;
  if (maxit > ED_MAX_LANCZOS) return ED_ERR_ARG;
  const ed_precision prec = o->precision;
  if (prec != ED_FP64 && prec != ED_FP32 && prec != ED_FP32_POLISH) return ED_ERR_ARG;
  double tol = o->tol > 0 ? o->tol : (prec == ED_FP64 ? 1e-12 : 1e-6);
  const bool want = o->want_vector != 0 || prec == ED_FP32_POLISH || d_psi != nullptr;
  if (s->dim <= 0) return ED_ERR_ARG;
  const int64_t n = s->bdim;  // padded block-major vectors
  std::vector<char> hbuf(sizeof(LanczosState));
  LanczosState *h = (LanczosState *)hbuf.data();
  int mv = 0, mv32 = 0;
  const int64_t g2 = reduce_grid(n);
  if (prec == ED_FP64) {
    Workspace psi;   // block-major ground state
    if (want) ED_TRY(psi.alloc(n * sizeof(double), cs));
    double *bpsi = (double *)psi.mem;
    ED_TRY(lanczos_solve<double>(s, maxit, tol, o->seed, nullptr, want, bpsi, h, cs, &mv,
                                 o->basis_mib));
    fill_result(*h, res);
    if (want) {
      double e, r;
      ED_TRY(fp64_residual(s, bpsi, &e, &r, cs));
      res->residual = r;
      ++mv;
      if (d_psi) ED_TRY((permute_layout<double, double>(s, bpsi, (double *)d_psi, false, cs)));
    }
  } else {
    Workspace psi32;
    if (want) ED_TRY(psi32.alloc(n * sizeof(float), cs));
    float *fpsi = (float *)psi32.mem;
    ED_TRY(lanczos_solve<float>(s, maxit, tol, o->seed, nullptr, want, fpsi, h, cs, &mv,
                                o->basis_mib));
    mv32 = mv;  // the FP32 first pass (and second pass, if any)
    fill_result(*h, res);
    if (want) {
      // FP64 copy of the FP32 ground state (normalised in FP64)
      Workspace start, prt;
      ED_TRY(start.alloc(n * sizeof(double), cs));
      ED_TRY(prt.alloc(g2 * sizeof(double), cs));
      k_norm2<float><<<(unsigned)g2, AXPY_THREADS, 0, cs>>>(fpsi, n, (double *)prt.mem);
      ED_LAUNCHED(1);
      k_scale_copy<float, double><<<(unsigned)g2, AXPY_THREADS, 0, cs>>>(
          fpsi, (double *)start.mem, n, (double *)prt.mem, g2);
      ED_LAUNCHED(1);
      if (prec == ED_FP32_POLISH) {
        // FP64 Lanczos restarted from the FP32 ground state (a6): a few FP64
        // steps, their Ritz pair, and the FP64 residual of the result.
        const int steps = o->polish_steps > 0 ? o->polish_steps : 4;
        Workspace psi64;
        ED_TRY(psi64.alloc(n * sizeof(double), cs));
        std::vector<char> h2buf(sizeof(LanczosState));
        LanczosState *h2 = (LanczosState *)h2buf.data();
        ED_TRY(lanczos_solve<double>(s, steps, 1e-300, 0, (const double *)start.mem, true,
                                     (double *)psi64.mem, h2, cs, &mv, o->basis_mib));
        res->e0 = h2->theta;
        res->polish_iterations = h2->j;
        double e, r;
        ED_TRY(fp64_residual(s, (const double *)psi64.mem, &e, &r, cs));
        res->residual = r;
        ++mv;
        if (d_psi)
          ED_TRY((permute_layout<double, double>(s, (const double *)psi64.mem, (double *)d_psi,
                                                 false, cs)));
      } else {
        double e, r;
        ED_TRY(fp64_residual(s, (const double *)start.mem, &e, &r, cs));
        res->residual = r;
        ++mv;
        if (d_psi) ED_TRY((permute_layout<float, float>(s, fpsi, (float *)d_psi, false, cs)));
      }
    }
  }
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  res->matvecs = mv;
  res->matvecs_fp64 = mv - mv32;
  if (res->stop_reason == 2) {
    ed_set_error_msg("max_iter reached before the Lanczos tolerance");
    return ED_ERR_NOT_CONVERGED;
  }
  return ED_OK;
}

// ----------------------------------------------------------------- chains (GF)

// A Lanczos chain of `nsteps` steps from a start vector (already in bufs[0]
// with partial squares in `part`): coefficients left in the device state.
template <typename T>
ed_status ed_lanczos_chain(ed_sector s, T *const *bufs, LanczosState *st, double *part,
                           double *part2, int64_t nparts_start, int nsteps, cudaStream_t cs,
                           int32_t *h_flag, const HvTables<T> *tables) {
  k_state_init<<<1, SCALAR_THREADS, 0, cs>>>(st, part, nparts_start, nsteps, 0.0, 1, 0.0);
  ED_LAUNCHED(1);
  ED_TRY(ed_build_items(s, 1, (int)sizeof(T)));
  const HvTables<T> tb = tables ? *tables : ed_hv_tables<T>(s, 1);
  int launched = 0;
  return run_steps<T>(s, tb, bufs, st, part, part2, s->bdim, nsteps, cs, &launched, h_flag);
}

template ed_status ed_lanczos_chain<float>(ed_sector, float *const *, LanczosState *, double *,
                                           double *, int64_t, int, cudaStream_t, int32_t *,
                                           const HvTables<float> *);
template ed_status ed_lanczos_chain<double>(ed_sector, double *const *, LanczosState *, double *,
                                            double *, int64_t, int, cudaStream_t, int32_t *,
                                            const HvTables<double> *);

int64_t ed_reduce_grid(int64_t n) { return reduce_grid(n); }

extern "C" ed_status ed_lanczos_ground(ed_sector s, const ed_lanczos_opts *opts,
                                       ed_lanczos_result *res, void *d_psi, void *stream) {
  if (!s || !opts || !res) return ED_ERR_ARG;
  return ed_lanczos_ground_impl(s, opts, res, d_psi, (cudaStream_t)stream);
}

ed_status ed_permute_vec(ed_sector s, ed_precision prec, bool to_blocked, const void *in,
                         void *out, cudaStream_t cs) {
  if (prec == ED_FP64)
    return permute_layout<double, double>(s, (const double *)in, (double *)out, to_blocked, cs);
  return permute_layout<float, float>(s, (const float *)in, (float *)out, to_blocked, cs);
}

extern "C" ed_status ed_sector_permute(ed_sector s, ed_precision prec, int32_t to_blocked,
                                       const void *d_in, int64_t n_in, void *d_out, int64_t n_out,
                                       void *stream) {
  if (!s || !d_in || !d_out || d_in == d_out) return ED_ERR_ARG;
  if (n_in != (to_blocked ? s->dim : s->bdim) || n_out != (to_blocked ? s->bdim : s->dim)) {
    ed_set_error_msg("vector length does not match the sector layout");
    return ED_ERR_ARG;
  }
  cudaStream_t cs = (cudaStream_t)stream;
  if (prec == ED_FP64)
    return permute_layout<double, double>(s, (const double *)d_in, (double *)d_out,
                                          to_blocked != 0, cs);
  if (prec == ED_FP32 || prec == ED_FP32_POLISH)
    return permute_layout<float, float>(s, (const float *)d_in, (float *)d_out, to_blocked != 0,
                                        cs);
  return ED_ERR_ARG;
}
