// Impurity Green's function on the Matsubara axis (Sec. 6.8, Eq. KLgf at
// T = 0): start vectors c^+_{a s}|gs> and c_{a s}|gs> built on the device in
// gather form, Lanczos chains on the N+-1 sectors, continued fractions.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "internal.cuh"

constexpr int GF_THREADS = 256;

__device__ __forceinline__ double gf_warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

struct ApplyArgs {
  // target sector (dst) in block-major order, source psi in sector order
  const uint32_t *dst_map;     // strings of the spin that changes, block-major order
  const int32_t *dst_pother;   // sector index of the unchanged spin's block-major index
  const int32_t *dst_padinv;   // padded column -> block-major up column (-1: padding)
  int64_t dst_stride, dst_dim; // padded row length, D_dw * stride
  int64_t src_dup;
  int level;                 // level a of the operator (impurity orbital)
  int create;                // +1: c^+, -1: c
  int spin;
  int nup_src;               // N_up of the source (sign of down operators)
};

// phi[r',c'] = sign * psi[r,c] where the changed spin string of the target
// element, with level a removed (c^+) or added (c), is the source string;
// sign = (-1)^(occupied modes before (a,s)) in the order 1up..Ns up,
// 1dw..Ns dw (Sec. 2.3).  phi is written in the target's block-major order,
// psi is read in sector order (sector index = colex rank of the strings).
// Partial sums of phi^2 per CTA.
template <typename Ti, typename To>
__global__ void __launch_bounds__(GF_THREADS) k_apply_op(ApplyArgs a, const Ti *psi, To *phi,
                                                         double *part) {
  __shared__ double red[GF_THREADS / 32];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const uint32_t bit = 1u << a.level;
  const uint32_t below = bit - 1u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.dst_dim; i += stride) {
    const int64_t r2 = i / a.dst_stride;
    const int32_t c2 = a.dst_padinv[i - r2 * a.dst_stride];
    To out = To(0);
    const uint32_t I2 = c2 < 0 ? 0u : a.dst_map[a.spin == 0 ? (int64_t)c2 : r2];
    const bool occ = (I2 & bit) != 0u;
    if (c2 >= 0 && occ == (a.create > 0)) {
      const uint32_t I = I2 ^ bit;
      const int64_t src_idx = ed_rank(I);
      int parity = __popc(I & below);
      if (a.spin == 1) parity += a.nup_src;
      const int64_t r = a.spin == 0 ? (int64_t)a.dst_pother[r2] : src_idx;
      const int64_t c = a.spin == 0 ? src_idx : (int64_t)a.dst_pother[c2];
      const Ti x = psi[r * a.src_dup + c];
      out = (To)((parity & 1) ? -x : x);
    }
    phi[i] = out;
    acc += (double)out * (double)out;
  }
  acc = gf_warp_sum(acc);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < GF_THREADS / 32; ++k) t += red[k];
    part[blockIdx.x] = t;
  }
}

// Continued fraction of one chain: G[n] += sgn * weight / f(z_n) with
// z_n = e0 + sgn * i w_n and f from the backward recurrence
// f = z - a_{k-1};  f = z - a_m - b_{m+1}^2 / f  (m = k-2 .. 0).
__global__ void k_cfrac(const LanczosState *st, double weight, double e0, double beta, int nmats,
                        int sgn, double2 *G) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nmats) return;
  const int k = st->j;
  if (k <= 0 || weight == 0.0) return;
  const double wn = (2.0 * n + 1.0) * M_PI / beta;
  const double zr = e0, zi = sgn * wn;
  double fr = zr - st->alpha[k - 1], fi = zi;
  for (int m = k - 2; m >= 0; --m) {
    const double b2 = st->beta[m + 1] * st->beta[m + 1];
    // b2 / f = b2 * conj(f) / |f|^2 (one FP64 division per level)
    const double inv = 1.0 / (fr * fr + fi * fi);
    const double qr = b2 * fr * inv, qi = -b2 * fi * inv;
    fr = zr - st->alpha[m] - qr;
    fi = zi - qi;
  }
  const double inv = 1.0 / (fr * fr + fi * fi);
  const double gr = weight * fr * inv, gi = -weight * fi * inv;
  G[n].x += sgn * gr;
  G[n].y += sgn * gi;
}

// The same continued fraction at arbitrary complex frequencies z_n (the real
// axis: z = w + i eta): G[n] += sgn * weight * [(E0 + sgn z_n - T)^-1]_00,
// the particle term (sgn = +1) and the hole term (sgn = -1) of Eq. KLgf.
// For z_n = i w_n this is k_cfrac's arithmetic.
__global__ void k_cfrac_z(const LanczosState *st, double weight, double e0, const double2 *z,
                          int nz, int sgn, double2 *G) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nz) return;
  const int k = st->j;
  if (k <= 0 || weight == 0.0) return;
  const double zr = e0 + sgn * z[n].x, zi = sgn * z[n].y;
  double fr = zr - st->alpha[k - 1], fi = zi;
  for (int m = k - 2; m >= 0; --m) {
    const double b2 = st->beta[m + 1] * st->beta[m + 1];
    const double inv = 1.0 / (fr * fr + fi * fi);
    const double qr = b2 * fr * inv, qi = -b2 * fi * inv;
    fr = zr - st->alpha[m] - qr;
    fi = zi - qi;
  }
  const double inv = 1.0 / (fr * fr + fi * fi);
  const double gr = weight * fr * inv, gi = -weight * fi * inv;
  G[n].x += sgn * gr;
  G[n].y += sgn * gi;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// c^+ / c of (orb, spin) from psi (sector order of s) into phi (block-major
// order of the neighbour sector nb): one launch of k_apply_op.
template <typename Ti, typename To>
ed_status ed_apply_op_launch(ed_sector s, ed_sector nb, const Ti *psi, To *phi, int orb, int spin,
                             int create, cudaStream_t cs) {
  const int64_t n = nb->bdim;
  const int64_t g2 = ed_reduce_grid(n);
  void *part = nullptr;
  ED_TRY(ed_dmalloc(&part, g2 * sizeof(double), cs, "apply partials"));
  ApplyArgs a;
  a.dst_map = nb->bk[spin].map;
  a.dst_pother = nb->bi[1 - spin].pidx;
  a.dst_padinv = nb->padinv;
  a.dst_stride = nb->bstride;
  a.dst_dim = n;
  a.src_dup = s->sp[0].dim;
  a.level = orb;  // impurity orbital alpha is level alpha
  a.create = create;
  a.spin = spin;
  a.nup_src = s->nup;
  k_apply_op<Ti, To><<<(unsigned)g2, GF_THREADS, 0, cs>>>(a, psi, phi, (double *)part);
  ed_count_launches(1);
  const cudaError_t e = cudaGetLastError();
  ed_dfree(part, cs);
  if (e != cudaSuccess) {
    ed_set_cuda_error(e, "k_apply_op", __FILE__, __LINE__);
    return ED_ERR_CUDA;
  }
  return ED_OK;
}
template ed_status ed_apply_op_launch<double, double>(ed_sector, ed_sector, const double *, double *,
                                                      int, int, int, cudaStream_t);
template ed_status ed_apply_op_launch<double, float>(ed_sector, ed_sector, const double *, float *,
                                                     int, int, int, cudaStream_t);
template ed_status ed_apply_op_launch<float, float>(ed_sector, ed_sector, const float *, float *,
                                                    int, int, int, cudaStream_t);

// ----------------------------------------------------------------- FP32 chains on H - sigma
//
// An FP32 chain runs on H - sigma with sigma = the energy the continued
// fraction is centred on (E0 of the state the chain starts from).  The
// diagonal of the product is E_up[c] + E_dw[r] + W in FP32 from tables
// rounded to FP32; each rounding costs up to 2^-24 of the entry's magnitude,
// and for total energies of order |E0| that puts the poles near E0 off by
// about |E0| 2^-24, which the low Matsubara frequencies magnify (a pole error
// d shifts G(i w) by about weight d / (w^2 + eps^2)).  The shifted tables
// E_up - s_up and E_dw - (sigma - s_up), s_up = min E_up, are formed in FP64
// and rounded once, so that the diagonal entries of the low-lying states are
// of the order of their excitation energy; alpha_j comes out shifted by
// -sigma and the continued fraction takes e0 - sigma.  The vectors, the
// product and the recurrence are unchanged.
__global__ void k_shift_diag(const double *eu, int64_t nu, const double *ed, int64_t nd,
                             double sigma, float *ou, float *od) {
  __shared__ double red[32];
  double m = 1e300;
  for (int64_t i = threadIdx.x; i < nu; i += blockDim.x) m = fmin(m, eu[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  double su = red[0];
  for (int k = 1; k < (int)(blockDim.x >> 5); ++k) su = fmin(su, red[k]);
  if (nu == 0) su = 0.0;
  const double sd = sigma - su;
  for (int64_t i = threadIdx.x; i < nu; i += blockDim.x) ou[i] = (float)(eu[i] - su);
  for (int64_t i = threadIdx.x; i < nd; i += blockDim.x) od[i] = (float)(ed[i] - sd);
}

size_t ed_shift_diag_bytes(ed_sector s) {
  return al256((size_t)s->bk[0].dim * sizeof(float)) + al256((size_t)s->bk[1].dim * sizeof(float));
}

ed_status ed_shift_diag32(ed_sector s, double sigma, void *mem, HvTables<float> *tb,
                          cudaStream_t cs) {
  float *ou = (float *)mem;
  float *od = (float *)((char *)mem + al256((size_t)s->bk[0].dim * sizeof(float)));
  k_shift_diag<<<1, 1024, 0, cs>>>(s->bk[0].ediag, s->bk[0].dim, s->bk[1].ediag, s->bk[1].dim,
                                   sigma, ou, od);
  ED_LAUNCHED(1);
  tb->e_up = ou;
  tb->e_dw = od;
  return ED_OK;
}

// G[n] += sgn * weight * [(e0 + sgn z_n - T)^-1]_00 for the chain held in st
ed_status ed_cfrac_z_launch(const LanczosState *st, double weight, double e0, const double2 *dz,
                            int nz, int sgn, double2 *dG, cudaStream_t cs) {
  if (nz <= 0) return ED_OK;
  k_cfrac_z<<<(nz + 31) / 32, 32, 0, cs>>>(st, weight, e0, dz, nz, sgn, dG);
  ED_LAUNCHED(1);
  return ED_OK;
}

// ----------------------------------------------------------------- batched chains
//
// All chains of a solve whose sectors are small run in one persistent launch:
// each CTA takes a chain from a device counter and runs it to the end alone
// (start vector c^+-|gs>, nsteps of the recurrence of lanczos.cu with the
// element-parallel product, FP64 scalars), so a chain costs one CTA and no
// host round trip.  The chains of a solve have different lengths (the
// c^+ and c sectors differ in dimension); a CTA that finishes takes the next.
// v_j is staged in shared memory every step, so every gather of the product
// is a shared-memory load.
constexpr int CHAIN_THREADS = 1024;
// padded elements of a batched chain's sector (FP64: 128 KB of shared memory)
constexpr int64_t CHAIN_MAX_DIM = 1 << 14;

template <typename Ti, typename To>
struct ChainTask {
  HvTables<To> tb;     // target sector, block-major, element-parallel form
  ApplyArgs a;         // start vector gather
  const Ti *psi;       // ground state, sector order
  To *b0, *b1, *b2;    // three vectors of a.dst_dim elements
  LanczosState *st;    // output: alpha, beta, j, acc[0] = ||phi||^2
  int nsteps;
};

// Sum over the CTA, the same value in every thread, fixed order, in FP64
// (each thread's partial covers at most n / CHAIN_THREADS <= 16 elements of
// a chain's sector, summed in the vector type).
template <typename T>
__device__ double chain_allsum(T xt, double *red) {
  double x = (double)xt;
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = (double)x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    red[32] = t;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

template <typename T>
__device__ __forceinline__ T ch_fma(T a, T b, T c);
template <>
__device__ __forceinline__ float ch_fma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double ch_fma<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename Ti, typename To>
__global__ void __launch_bounds__(CHAIN_THREADS) k_chain_batch(const ChainTask<Ti, To> *tasks,
                                                               int ntasks, int *next) {
  extern __shared__ __align__(16) unsigned char chain_smem[];
  To *S = reinterpret_cast<To *>(chain_smem);  // v_j (unscaled) of the current step
  __shared__ double red[33];
  __shared__ double s_scal[2];
  __shared__ int s_task, s_done;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(next, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= ntasks) return;
    const ChainTask<Ti, To> &tk = tasks[t];
    const HvTables<To> &tb = tk.tb;
    const ApplyArgs &a = tk.a;
    const int64_t n = a.dst_dim, stride = a.dst_stride;
    const float inv_stride = 1.0f / (float)stride;
    To *bufs[3] = {tk.b0, tk.b1, tk.b2};
    // start vector into b0 (the gather of k_apply_op), b1 = b2 = 0
    double sq = 0.0;
    {
      const uint32_t bit = 1u << a.level, below = bit - 1u;
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        // exact row index: (i + 1/2) / stride lies 1/(2 stride) from an integer
        const int64_t r2 = __float2int_rz(((float)i + 0.5f) * inv_stride);
        const int32_t c2 = a.dst_padinv[i - r2 * stride];
        To out = To(0);
        const uint32_t I2 = c2 < 0 ? 0u : a.dst_map[a.spin == 0 ? (int64_t)c2 : r2];
        if (c2 >= 0 && ((I2 & bit) != 0u) == (a.create > 0)) {
          const uint32_t I = I2 ^ bit;
          const int64_t src_idx = ed_rank(I);
          int parity = __popc(I & below);
          if (a.spin == 1) parity += a.nup_src;
          const int64_t r = a.spin == 0 ? (int64_t)a.dst_pother[r2] : src_idx;
          const int64_t c = a.spin == 0 ? src_idx : (int64_t)a.dst_pother[c2];
          const Ti x = tk.psi[r * a.src_dup + c];
          out = (To)((parity & 1) ? -x : x);
        }
        tk.b0[i] = out;
        tk.b1[i] = To(0);
        tk.b2[i] = To(0);
        sq += (double)out * (double)out;
      }
    }
    const double weight = chain_allsum<double>(sq, red);
    LanczosState *st = tk.st;
    double scale[3] = {weight > 0.0 ? 1.0 / sqrt(weight) : 0.0, 0.0, 0.0};
    double beta_j = 0.0, tnorm = 0.0;
    int j = 0, done = weight > 0.0 ? 0 : 2;
    if (threadIdx.x == 0) {
      st->acc[0] = weight;
      st->beta[0] = 0.0;
    }
    while (!done) {
      const To *g = bufs[j % 3];
      const To *prev = bufs[(j + 2) % 3];
      To *out = bufs[(j + 1) % 3];
      const To s_cur = (To)scale[j % 3], s_prev = (To)scale[(j + 2) % 3];
      const To bj = (To)beta_j;
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) S[i] = g[i];
      __syncthreads();
      // w1 = H v_j - beta_j v_{j-1} (padding columns are skipped: they stay 0)
      To dot = To(0);  // per-thread partials in the vector type; FP64 across warps
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t r = __float2int_rz(((float)i + 0.5f) * inv_stride);
        const int pc = (int)(i - r * stride);
        const int4 ci = __ldg(tb.small_cols + pc);
        if (ci.x < 0) continue;
        const To x = S[i];
        const To *row = S + r * stride + ci.z;
        const int deg = ci.w & 255, ncp = ci.w >> 8;
        const int mu = (int)tb.m_up[ci.x] * tb.nmask;
        To acc = (tb.e_up[ci.x] + tb.e_dw[r] + tb.W[mu + tb.m_dw[r]]) * x;
        for (int e = 0; e < deg; ++e) {
          const int o = ci.y + e * ncp;
          acc = ch_fma<To>(__ldg(tb.ell_val + o), row[__ldg(tb.ell_col + o)], acc);
        }
        const int32_t d0 = __ldg(tb.rp_dw + r), d1 = __ldg(tb.rp_dw + r + 1);
        for (int32_t k = d0; k < d1; ++k)
          acc = ch_fma<To>(__ldg(tb.val_dw + k), S[(int64_t)__ldg(tb.col_dw + k) * stride + pc], acc);
        if (tb.nd_up)  // spin exchange and pair hopping
          acc += ed_nd_terms<To>(tb, S, stride, r, pc, (int)tb.m_up[ci.x], (int)tb.m_dw[r]);
        const To v = x * s_cur;
        To w1 = acc * s_cur;
        if (j > 0) w1 = ch_fma<To>(-bj, prev[i] * s_prev, w1);
        out[i] = w1;
        dot = ch_fma<To>(v, w1, dot);
      }
      const double al = chain_allsum<To>(dot, red);
      // w = w1 - alpha_j v_j, ||w||^2
      const To alT = (To)al;
      To ss = To(0);
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const To w = ch_fma<To>(-alT, S[i] * s_cur, out[i]);
        out[i] = w;
        ss = ch_fma<To>(w, w, ss);
      }
      const double ss_tot = chain_allsum<To>(ss, red);
      // scalar bookkeeping once, by thread 0
      if (threadIdx.x == 0) {
        const double be = sqrt(fmax(ss_tot, 0.0));
        tnorm = fmax(tnorm, fmax(fabs(al), be));
        st->alpha[j] = al;
        st->beta[j + 1] = be;
        s_scal[0] = be;
        s_scal[1] = be > 0.0 ? 1.0 / be : 0.0;
        s_done = be <= 1e-13 * tnorm ? 2 : (j + 1 >= tk.nsteps ? 3 : 0);
      }
      __syncthreads();
      beta_j = s_scal[0];
      scale[(j + 1) % 3] = s_scal[1];
      done = s_done;
      ++j;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      st->j = j;
      st->done = done;
    }
    __syncthreads();
  }
}

// Continued fractions of a batch of chains (grid.y = chain): the arithmetic
// of k_cfrac, with the weight ||phi||^2 read from the chain's state and the
// ground energy of the chain's solve.
__global__ void k_cfrac_batch(const LanczosState *const *sts, const int *sgns, const double *e0s,
                              double beta, int nmats, double2 *G) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (n >= nmats) return;
  const double e0 = e0s[c];
  const LanczosState *st = sts[c];
  const int k = st->j;
  const double weight = st->acc[0];
  double2 out = make_double2(0.0, 0.0);
  if (k > 0 && weight != 0.0) {
    const int sgn = sgns[c];
    const double wn = (2.0 * n + 1.0) * M_PI / beta;
    const double zr = e0, zi = sgn * wn;
    double fr = zr - st->alpha[k - 1], fi = zi;
    for (int m = k - 2; m >= 0; --m) {
      const double b2 = st->beta[m + 1] * st->beta[m + 1];
      const double inv = 1.0 / (fr * fr + fi * fi);
      const double qr = b2 * fr * inv, qi = -b2 * fi * inv;
      fr = zr - st->alpha[m] - qr;
      fi = zi - qi;
    }
    const double inv = 1.0 / (fr * fr + fi * fi);
    out.x = sgn * (weight * fr * inv);
    out.y = sgn * (-weight * fi * inv);
  }
  G[(size_t)c * nmats + n] = out;
}

template <typename Ti, typename To>
static ed_status one_chain(ed_sector s, const Ti *psi, int orb, int spin, int create, int nsteps,
                           double e0, double beta, int nmats, double2 *dG, double *weight,
                           int *steps, cudaStream_t cs, const double2 *dz = nullptr) {
  *weight = 0.0;
  *steps = 0;
  ed_sector nb = nullptr;
  ED_TRY(ed_neighbor_sector(s, spin, create, cs, &nb));
  if (!nb || nb->dim == 0) return ED_OK;
  const int64_t n = nb->bdim;  // padded block-major vectors
  const int64_t np1 = ed_hv_num_parts(nb, 1, (int)sizeof(To));
  const int64_t g2 = ed_reduce_grid(n);
  const int64_t nparts = std::max<int64_t>(np1, 3 * g2);
  const size_t vb = al256(n * sizeof(To));
  constexpr bool shift = std::is_same<To, float>::value;  // FP32 chains run on H - e0
  const size_t bytes = 3 * vb + al256(sizeof(LanczosState)) + 2 * al256(nparts * sizeof(double)) +
                       (shift ? ed_shift_diag_bytes(nb) : 0);
  void *mem = nullptr;
  ED_TRY(ed_dmalloc(&mem, bytes, cs, "gf chain workspace"));
  cudaError_t e = cudaSuccess;
  char *p = (char *)mem;
  To *bufs[3];
  for (int b = 0; b < 3; ++b) {
    bufs[b] = (To *)p;
    p += vb;
  }
  LanczosState *st = (LanczosState *)p;
  p += al256(sizeof(LanczosState));
  double *part = (double *)p;
  p += al256(nparts * sizeof(double));
  double *part2 = (double *)p;
  p += al256(nparts * sizeof(double));

  ApplyArgs a;
  a.dst_map = nb->bk[spin].map;
  a.dst_pother = nb->bi[1 - spin].pidx;
  a.dst_padinv = nb->padinv;
  a.dst_stride = nb->bstride;
  a.dst_dim = n;
  a.src_dup = s->sp[0].dim;
  a.level = orb;  // impurity orbital alpha is level alpha
  a.create = create;
  a.spin = spin;
  a.nup_src = s->nup;
  ed_status rs = ED_OK;
  // padding entries must stay zero in every chain vector
  if (cudaMemsetAsync(mem, 0, 3 * vb, cs) != cudaSuccess) rs = ED_ERR_CUDA;
  PinnedFlag flag;
  if (rs == ED_OK && !flag.p) rs = ED_ERR_OOM;
  if (rs == ED_OK) {
    k_apply_op<Ti, To><<<(unsigned)g2, GF_THREADS, 0, cs>>>(a, psi, bufs[0], part);
    ed_count_launches(1);
    if (cudaGetLastError() != cudaSuccess) rs = ED_ERR_CUDA;
  }
  // the product's tables: shifted by sigma = e0 for FP32 chains
  if (rs == ED_OK) rs = ed_build_items(nb, 1, (int)sizeof(To));
  HvTables<To> tb = ed_hv_tables<To>(nb, 1);
  const double sigma = shift ? e0 : 0.0;
  if constexpr (shift) {
    if (rs == ED_OK) rs = ed_shift_diag32(nb, sigma, p, &tb, cs);
  }
  if (rs == ED_OK) rs = ed_lanczos_chain<To>(nb, bufs, st, part, part2, g2, nsteps, cs, flag.p, &tb);
  double hw[2] = {0, 0};
  int32_t hj = 0;
  if (rs == ED_OK) {
    // weight = ||phi||^2 was stored by the state initialisation in acc[0]
    e = cudaMemcpyAsync(hw, &st->acc[0], sizeof(double), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hj, &st->j, sizeof(int32_t), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
      ed_set_cuda_error(e, "gf chain read-back", __FILE__, __LINE__);
      rs = ED_ERR_CUDA;
    }
  }
  if (rs == ED_OK && hw[0] > 0.0 && nmats > 0) {
    // 32 frequencies per CTA: the FP64 recurrences spread over many SMs
    if (dz)  // nmats arbitrary complex frequencies
      k_cfrac_z<<<(nmats + 31) / 32, 32, 0, cs>>>(st, hw[0], e0 - sigma, dz, nmats, create, dG);
    else
      k_cfrac<<<(nmats + 31) / 32, 32, 0, cs>>>(st, hw[0], e0 - sigma, beta, nmats, create, dG);
    ed_count_launches(1);
    if (cudaGetLastError() != cudaSuccess) rs = ED_ERR_CUDA;
  }
  *weight = hw[0];
  *steps = hj;
  ed_dfree(mem, cs);
  return rs;
}

ed_status ed_gf_impl(ed_sector s, ed_precision prec, const void *d_psi, double e0, int orb,
                     int spin, int nsteps, double beta, int nmats, double *host_G,
                     ed_gf_info *info, cudaStream_t cs, const double *host_z = nullptr) {
  if (!s || !d_psi || orb < 0 || orb >= s->mp.norb || spin < 0 || spin > 1 || nsteps <= 0 ||
      nsteps > ED_MAX_LANCZOS || nmats < 0 ||
      (nmats > 0 && (!host_G || (!host_z && !(beta > 0)))))
    return ED_ERR_ARG;
  double2 *dG = nullptr;
  // [0, nmats): G; with host_z, then the nmats frequencies
  const size_t nz = host_z ? (size_t)nmats : 0;
  ED_TRY(ed_dmalloc((void **)&dG, (std::max(1, nmats) + nz) * sizeof(double2), cs,
                    "gf accumulator"));
  ed_status rs = ED_OK;
  if (cudaMemsetAsync(dG, 0, std::max(1, nmats) * sizeof(double2), cs) != cudaSuccess) rs = ED_ERR_CUDA;
  const double2 *dz = nz ? dG + std::max(1, nmats) : nullptr;
  if (rs == ED_OK && nz &&
      cudaMemcpyAsync((void *)dz, host_z, nz * sizeof(double2), cudaMemcpyHostToDevice, cs) !=
          cudaSuccess)
    rs = ED_ERR_CUDA;
  double wp = 0, wh = 0;
  int sp = 0, sh = 0;
  for (int create = 1; create >= -1 && rs == ED_OK; create -= 2) {
    double *w = create > 0 ? &wp : &wh;
    int *k = create > 0 ? &sp : &sh;
    if (prec == ED_FP64)
      rs = one_chain<double, double>(s, (const double *)d_psi, orb, spin, create, nsteps, e0, beta,
                                     nmats, dG, w, k, cs, dz);
    else if (prec == ED_FP32)
      rs = one_chain<float, float>(s, (const float *)d_psi, orb, spin, create, nsteps, e0, beta,
                                   nmats, dG, w, k, cs, dz);
    else
      rs = one_chain<double, float>(s, (const double *)d_psi, orb, spin, create, nsteps, e0, beta,
                                    nmats, dG, w, k, cs, dz);
  }
  if (rs == ED_OK && nmats > 0) {
    cudaError_t e = cudaMemcpyAsync(host_G, dG, nmats * sizeof(double2), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
      ed_set_cuda_error(e, "gf result copy", __FILE__, __LINE__);
      rs = ED_ERR_CUDA;
    }
  }
  ed_dfree(dG, cs);
  if (info) {
    info->weight_particle = wp;
    info->weight_hole = wh;
    info->steps_particle = sp;
    info->steps_hole = sh;
  }
  return rs;
}

// One chain (particle: create = +1, hole: -1) of G_{orb,spin}, on its own
// stream ordered after `after`; its contribution to G goes to host_G
// (2*nmats doubles, overwritten).  Used by ed_solve to run the chains of a
// solve concurrently; the neighbour sector and its work lists must already
// exist (ed_gf_prepare) so that concurrent jobs share no mutable state.
ed_status ed_gf_chain_job(ed_sector s, ed_precision prec, const void *d_psi, double e0, int orb,
                          int spin, int create, int nsteps, double beta, int nmats,
                          double *host_G, double *weight, int *steps, int64_t *dim,
                          cudaEvent_t after) {
  *weight = 0.0;
  *steps = 0;
  *dim = 0;
  cudaStream_t cs = nullptr;
  ED_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  ed_status rs = ED_OK;
  if (after && cudaStreamWaitEvent(cs, after, 0) != cudaSuccess) rs = ED_ERR_CUDA;
  double2 *dG = nullptr;
  if (rs == ED_OK)
    rs = ed_dmalloc((void **)&dG, std::max(1, nmats) * sizeof(double2), cs, "gf accumulator");
  if (rs == ED_OK && cudaMemsetAsync(dG, 0, std::max(1, nmats) * sizeof(double2), cs) != cudaSuccess)
    rs = ED_ERR_CUDA;
  if (rs == ED_OK) {
    if (prec == ED_FP64)
      rs = one_chain<double, double>(s, (const double *)d_psi, orb, spin, create, nsteps, e0,
                                     beta, nmats, dG, weight, steps, cs);
    else if (prec == ED_FP32)
      rs = one_chain<float, float>(s, (const float *)d_psi, orb, spin, create, nsteps, e0, beta,
                                   nmats, dG, weight, steps, cs);
    else
      rs = one_chain<double, float>(s, (const double *)d_psi, orb, spin, create, nsteps, e0,
                                    beta, nmats, dG, weight, steps, cs);
  }
  if (rs == ED_OK && nmats > 0) {
    cudaError_t e = cudaMemcpyAsync(host_G, dG, nmats * sizeof(double2), cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) rs = ED_ERR_CUDA;
  }
  ed_dfree(dG, cs);
  if (cudaStreamSynchronize(cs) != cudaSuccess && rs == ED_OK) rs = ED_ERR_CUDA;
  cudaStreamDestroy(cs);
  ed_sector nb = s->nb[spin][create > 0 ? 1 : 0];
  *dim = nb ? nb->dim : 0;
  return rs;
}

// Builds the neighbour sector of a chain and its product work lists on the
// calling thread (before concurrent chain jobs start).
ed_status ed_gf_prepare(ed_sector s, int spin, int create, int elem, cudaStream_t cs) {
  ed_sector nb = nullptr;
  ED_TRY(ed_neighbor_sector(s, spin, create, cs, &nb));
  if (nb && nb->dim > 0) ED_TRY(ed_build_items(nb, 1, elem));
  return ED_OK;
}

// True when the chain of (spin, create) can run in the batched launch: its
// sector exists, has the element-parallel tables and at most CHAIN_MAX_DIM
// padded elements (ed_gf_prepare must have run).
bool ed_gf_batchable(ed_sector s, int spin, int create) {
  const ed_sector nb = s->nb[spin][create > 0 ? 1 : 0];
  if (!nb || nb->dim == 0) return true;  // an empty chain
  return nb->bdim <= CHAIN_MAX_DIM && nb->small_cols != nullptr;
}

// ----------------------------------------------------------------- cross-request batches
//
// Solves that reach their small-sector chains at about the same time (the
// requests a server runs concurrently, or several host threads calling
// ed_solve) share one launch of k_chain_batch / k_cfrac_batch: the first
// caller of a (device, precision, grid) group leads it, waits a short window
// for the others while other small solves are under way, then launches every
// member's chains at once on its own stream after the members' streams.  A
// chain runs on one CTA from its own task and workspace, so its coefficients
// and G do not depend on which other chains share the launch: a solve gives
// the same result alone and in any mix.
namespace {

constexpr double kBatchWindowS = 1e-3;  // the leader's wait for more members
constexpr double kMemberWaitS = 300.0;    // a member's bound on the leader's launch

struct BatchMember {
  int key = 0;
  int nmats = 0;
  double beta = 0;
  size_t task_bytes = 0;              // bytes of one ChainTask of this precision
  std::vector<unsigned char> tasks;   // nt tasks, device pointers inside
  int nt = 0;
  std::vector<LanczosState *> sts;
  std::vector<int> sgn;
  std::vector<double> e0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ready = nullptr;        // recorded on the member's stream: workspace written
  // filled by the leader
  std::vector<double> G;
  std::vector<int32_t> steps;
  std::vector<double> weight;
  ed_status st = ED_OK;
  bool done = false;
};

struct BatchGroup {
  std::vector<BatchMember *> members;
};

struct Batcher {
  std::mutex mu;
  std::condition_variable cv;
  std::map<std::tuple<int, int, int, double>, BatchGroup *> open;  // (device, key, nmats, beta)
  int active = 0;  // small solves under way (ed_gf_batch_announce)
  int64_t launches = 0, chains = 0, max_members = 0;
};
Batcher &batcher() {
  static Batcher b;
  return b;
}

// Launches the chains of every member of a closed group on the leader's stream.
template <typename Ti, typename To>
ed_status run_group(const std::vector<BatchMember *> &ms, cudaStream_t cs) {
  int nt = 0;
  for (const BatchMember *m : ms) nt += m->nt;
  const int nmats = ms[0]->nmats;
  const double beta = ms[0]->beta;
  std::vector<ChainTask<Ti, To>> tasks(nt);
  std::vector<LanczosState *> sts(nt);
  std::vector<int> sgn(nt);
  std::vector<double> e0(nt);
  int64_t nmax = 1;
  {
    int i = 0;
    for (const BatchMember *m : ms)
      for (int q = 0; q < m->nt; ++q, ++i) {
        memcpy(&tasks[i], m->tasks.data() + (size_t)q * sizeof(ChainTask<Ti, To>),
               sizeof(ChainTask<Ti, To>));
        sts[i] = m->sts[q];
        sgn[i] = m->sgn[q];
        e0[i] = m->e0[q];
        nmax = std::max<int64_t>(nmax, tasks[i].a.dst_dim);
      }
  }
  const size_t o_tasks = 0, o_sts = al256(nt * sizeof(ChainTask<Ti, To>));
  const size_t o_sgn = o_sts + al256(nt * sizeof(LanczosState *));
  const size_t o_e0 = o_sgn + al256(nt * sizeof(int));
  const size_t o_G = o_e0 + al256(nt * sizeof(double));
  const size_t o_next = o_G + al256((size_t)nt * std::max(nmats, 1) * sizeof(double2));
  void *mem = nullptr;
  ED_TRY(ed_dmalloc(&mem, o_next + 256, cs, "batched chains"));
  char *base = (char *)mem;
  ed_status rs = ED_OK;
  for (const BatchMember *m : ms)
    if (rs == ED_OK && m->stream != cs && cudaStreamWaitEvent(cs, m->ready, 0) != cudaSuccess)
      rs = ED_ERR_CUDA;
  auto h2d = [&](size_t o, const void *src, size_t n) {
    if (rs == ED_OK && cudaMemcpyAsync(base + o, src, n, cudaMemcpyHostToDevice, cs) != cudaSuccess)
      rs = ED_ERR_CUDA;
  };
  h2d(o_tasks, tasks.data(), nt * sizeof(ChainTask<Ti, To>));
  h2d(o_sts, sts.data(), nt * sizeof(LanczosState *));
  h2d(o_sgn, sgn.data(), nt * sizeof(int));
  h2d(o_e0, e0.data(), nt * sizeof(double));
  if (rs == ED_OK && cudaMemsetAsync(base + o_next, 0, sizeof(int), cs) != cudaSuccess) rs = ED_ERR_CUDA;
  if (rs == ED_OK && cudaFuncSetAttribute(k_chain_batch<Ti, To>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(CHAIN_MAX_DIM * sizeof(To))) != cudaSuccess)
    rs = ED_ERR_CUDA;
  if (rs == ED_OK) {
    k_chain_batch<Ti, To><<<(unsigned)std::min(nt, 2 * 152), CHAIN_THREADS,
                            (size_t)nmax * sizeof(To), cs>>>(
        (const ChainTask<Ti, To> *)(base + o_tasks), nt, (int *)(base + o_next));
    ed_count_launches(1);
    if (nmats > 0) {
      k_cfrac_batch<<<dim3((nmats + 31) / 32, nt), 32, 0, cs>>>(
          (const LanczosState *const *)(base + o_sts), (const int *)(base + o_sgn),
          (const double *)(base + o_e0), beta, nmats, (double2 *)(base + o_G));
      ed_count_launches(1);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      ed_set_cuda_error(e, "batched chains launch", __FILE__, __LINE__);
      rs = ED_ERR_CUDA;
    }
  }
  std::vector<double> G((size_t)nt * 2 * std::max(nmats, 0));
  std::vector<int32_t> hj(nt, 0);
  std::vector<double> hw(nt, 0.0);
  if (rs == ED_OK && nmats > 0 &&
      cudaMemcpyAsync(G.data(), base + o_G, G.size() * sizeof(double), cudaMemcpyDeviceToHost,
                      cs) != cudaSuccess)
    rs = ED_ERR_CUDA;
  for (int i = 0; i < nt && rs == ED_OK; ++i) {
    if (cudaMemcpyAsync(&hj[i], &sts[i]->j, sizeof(int32_t), cudaMemcpyDeviceToHost, cs) !=
            cudaSuccess ||
        cudaMemcpyAsync(&hw[i], &sts[i]->acc[0], sizeof(double), cudaMemcpyDeviceToHost, cs) !=
            cudaSuccess)
      rs = ED_ERR_CUDA;
  }
  cudaError_t e = cudaStreamSynchronize(cs);
  if (rs == ED_OK && e != cudaSuccess) {
    ed_set_cuda_error(e, "batched chains", __FILE__, __LINE__);
    rs = ED_ERR_CUDA;
  }
  ed_dfree(mem, cs);
  int i = 0;
  for (BatchMember *m : ms) {
    m->st = rs;
    m->G.assign(G.begin() + (size_t)i * 2 * std::max(nmats, 0),
                G.begin() + (size_t)(i + m->nt) * 2 * std::max(nmats, 0));
    m->steps.assign(hj.begin() + i, hj.begin() + i + m->nt);
    m->weight.assign(hw.begin() + i, hw.begin() + i + m->nt);
    i += m->nt;
  }
  return rs;
}

// Joins (or leads) the group of m's kind; returns when m's chains have run.
template <typename Ti, typename To>
ed_status join_group(BatchMember &m) {
  Batcher &B = batcher();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ED_ERR_CUDA;
  const auto key = std::make_tuple(dev, m.key, m.nmats, m.beta);
  std::unique_lock<std::mutex> lk(B.mu);
  auto it = B.open.find(key);
  if (it != B.open.end()) {
    it->second->members.push_back(&m);
    B.cv.notify_all();
    // bounded: the leader's launch ends with a synchronisation of its stream
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::microseconds((int64_t)(kMemberWaitS * 1e6));
    while (!m.done)
      if (B.cv.wait_until(lk, deadline) == std::cv_status::timeout && !m.done) {
        ed_set_error_msg("batched chains: the leading solve did not finish in time");
        return ED_ERR_TIMEOUT;
      }
    return m.st;
  }
  BatchGroup *g = new BatchGroup();
  g->members.push_back(&m);
  B.open[key] = g;
  // wait a short window for the other small solves under way to join
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::microseconds((int64_t)(kBatchWindowS * 1e6));
  while ((int)g->members.size() < B.active &&
         B.cv.wait_until(lk, deadline) != std::cv_status::timeout) {
  }
  B.open.erase(key);
  lk.unlock();
  const ed_status rs = run_group<Ti, To>(g->members, m.stream);
  lk.lock();
  B.launches += 1;
  int64_t nt = 0;
  for (BatchMember *x : g->members) {
    nt += x->nt;
    x->done = true;
  }
  B.chains += nt;
  B.max_members = std::max<int64_t>(B.max_members, (int64_t)g->members.size());
  delete g;
  lk.unlock();
  B.cv.notify_all();
  return rs;
}

}  // namespace

// Small solves under way: a leader only waits for more members while more
// than one is (see join_group).
void ed_gf_batch_announce(int delta) {
  Batcher &B = batcher();
  {
    std::lock_guard<std::mutex> lk(B.mu);
    B.active = std::max(0, B.active + delta);
  }
  B.cv.notify_all();
}

extern "C" ed_status ed_batch_stats(int64_t *launches, int64_t *chains, int64_t *max_solves) {
  if (!launches || !chains || !max_solves) return ED_ERR_ARG;
  Batcher &B = batcher();
  std::lock_guard<std::mutex> lk(B.mu);
  *launches = B.launches;
  *chains = B.chains;
  *max_solves = B.max_members;
  return ED_OK;
}

template <typename Ti, typename To>
static ed_status chain_batch(ed_sector s, const Ti *psi, double e0, int nsteps, double beta,
                             int nmats, int njobs, const int *orb, const int *spin,
                             const int *create, double *host_G, double *weight, int *steps,
                             int64_t *dim, cudaStream_t cs) {
  constexpr bool shift = std::is_same<To, float>::value;  // FP32 chains run on H - e0
  std::vector<ChainTask<Ti, To>> tasks;
  std::vector<int> job_of, sgn;
  std::vector<size_t> off;
  std::vector<ed_sector> nbs;
  size_t bytes = 0;
  for (int q = 0; q < njobs; ++q) {
    weight[q] = 0.0;
    steps[q] = 0;
    dim[q] = 0;
    if (nmats > 0) memset(host_G + 2 * (size_t)nmats * q, 0, 2 * sizeof(double) * nmats);
    const ed_sector nb = s->nb[spin[q]][create[q] > 0 ? 1 : 0];
    if (!nb || nb->dim == 0) continue;
    dim[q] = nb->dim;
    if (!nb->small_cols || nb->bdim > CHAIN_MAX_DIM) return ED_ERR_UNSUPPORTED;
    ChainTask<Ti, To> t;
    memset(&t, 0, sizeof(t));
    t.tb = ed_hv_tables<To>(nb, 1);
    t.a.dst_map = nb->bk[spin[q]].map;
    t.a.dst_pother = nb->bi[1 - spin[q]].pidx;
    t.a.dst_padinv = nb->padinv;
    t.a.dst_stride = nb->bstride;
    t.a.dst_dim = nb->bdim;
    t.a.src_dup = s->sp[0].dim;
    t.a.level = orb[q];  // impurity orbital alpha is level alpha
    t.a.create = create[q];
    t.a.spin = spin[q];
    t.a.nup_src = s->nup;
    t.psi = psi;
    t.nsteps = nsteps;
    off.push_back(bytes);
    bytes += 3 * al256(nb->bdim * sizeof(To)) + al256(sizeof(LanczosState)) +
             (shift ? ed_shift_diag_bytes(nb) : 0);
    nbs.push_back(nb);
    tasks.push_back(t);
    job_of.push_back(q);
    sgn.push_back(create[q]);
  }
  const int nt = (int)tasks.size();
  if (nt == 0) return ED_OK;
  // the chains' vectors and states, on this solve's stream
  void *mem = nullptr;
  ED_TRY(ed_dmalloc(&mem, bytes + 256, cs, "batched chain workspace"));
  char *base = (char *)mem;
  BatchMember m;
  m.key = std::is_same<Ti, double>::value * 2 + std::is_same<To, double>::value;
  m.nmats = nmats;
  m.beta = beta;
  m.nt = nt;
  m.stream = cs;
  for (int i = 0; i < nt; ++i) {
    char *p = base + off[i];
    const size_t vb = al256(tasks[i].a.dst_dim * sizeof(To));
    tasks[i].b0 = (To *)p;
    tasks[i].b1 = (To *)(p + vb);
    tasks[i].b2 = (To *)(p + 2 * vb);
    tasks[i].st = (LanczosState *)(p + 3 * vb);
    m.sts.push_back(tasks[i].st);
    m.sgn.push_back(sgn[i]);
    m.e0.push_back(shift ? 0.0 : e0);  // the continued fraction's e0 - sigma
  }
  ed_status rs = ED_OK;
  if constexpr (shift) {
    for (int i = 0; i < nt && rs == ED_OK; ++i)
      rs = ed_shift_diag32(nbs[i], e0,
                           base + off[i] + 3 * al256(tasks[i].a.dst_dim * sizeof(To)) +
                               al256(sizeof(LanczosState)),
                           &tasks[i].tb, cs);
  }
  if (rs != ED_OK) {
    ed_dfree(mem, cs);
    return rs;
  }
  m.tasks.resize((size_t)nt * sizeof(ChainTask<Ti, To>));
  memcpy(m.tasks.data(), tasks.data(), m.tasks.size());
  if (cudaEventCreateWithFlags(&m.ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(m.ready, cs) != cudaSuccess)
    rs = ED_ERR_CUDA;
  if (rs == ED_OK) rs = join_group<Ti, To>(m);
  if (m.ready) cudaEventDestroy(m.ready);
  if (rs == ED_ERR_TIMEOUT) return rs;  // the leader may still use the workspace: keep it
  ed_dfree(mem, cs);
  if (rs != ED_OK) return rs;
  for (int i = 0; i < nt; ++i) {
    const int q = job_of[i];
    weight[q] = m.weight[i];
    steps[q] = m.steps[i];
    if (nmats > 0)
      memcpy(host_G + 2 * (size_t)nmats * q, m.G.data() + 2 * (size_t)nmats * i,
             2 * sizeof(double) * nmats);
  }
  return ED_OK;
}

// The chains of a solve in one batched launch (see k_chain_batch); per job q:
// host_G[q] (2 * nmats doubles, overwritten), weight, steps and the
// dimension of its sector.  ED_ERR_UNSUPPORTED when a chain is not batchable.
ed_status ed_gf_chain_batch(ed_sector s, ed_precision prec, const void *d_psi, double e0,
                            int nsteps, double beta, int nmats, int njobs, const int *orb,
                            const int *spin, const int *create, double *host_G, double *weight,
                            int *steps, int64_t *dim, cudaStream_t cs) {
  if (nsteps <= 0 || nsteps > ED_MAX_LANCZOS) return ED_ERR_ARG;
  if (prec == ED_FP64)
    return chain_batch<double, double>(s, (const double *)d_psi, e0, nsteps, beta, nmats, njobs, orb,
                                       spin, create, host_G, weight, steps, dim, cs);
  if (prec == ED_FP32)
    return chain_batch<float, float>(s, (const float *)d_psi, e0, nsteps, beta, nmats, njobs, orb,
                                     spin, create, host_G, weight, steps, dim, cs);
  return chain_batch<double, float>(s, (const double *)d_psi, e0, nsteps, beta, nmats, njobs, orb,
                                    spin, create, host_G, weight, steps, dim, cs);
}

extern "C" ed_status ed_gf_lanczos(ed_sector s, ed_precision prec, const void *d_psi, double e0,
                                   int32_t orb, int32_t spin, int32_t nsteps, double beta,
                                   int32_t nmats, double *host_G, ed_gf_info *info, void *stream) {
  if (prec != ED_FP64 && prec != ED_FP32 && prec != ED_FP32_POLISH) return ED_ERR_ARG;
  return ed_gf_impl(s, prec, d_psi, e0, orb, spin, nsteps, beta, nmats, host_G, info,
                    (cudaStream_t)stream);
}

extern "C" ed_status ed_gf_lanczos_z(ed_sector s, ed_precision prec, const void *d_psi, double e0,
                                     int32_t orb, int32_t spin, int32_t nsteps,
                                     const double *host_z, int32_t nz, double *host_G,
                                     ed_gf_info *info, void *stream) {
  if (prec != ED_FP64 && prec != ED_FP32 && prec != ED_FP32_POLISH) return ED_ERR_ARG;
  if (nz < 0 || (nz > 0 && (!host_z || !host_G))) return ED_ERR_ARG;
  static const double none[2] = {0.0, 0.0};
  return ed_gf_impl(s, prec, d_psi, e0, orb, spin, nsteps, 0.0, nz, host_G, info,
                    (cudaStream_t)stream, host_z ? host_z : none);
}
