// Impurity susceptibilities at T = 0 (Sec. 6.8: Eq. KLgf with the bosonic
// sign), C_O(z) = n+ [(E0 + z - T+)^-1]_00 + n- [(E0 - z - T-)^-1]_00 for
// the spin (S^z), charge (n) and s-wave pair (d_dw d_up) operators of one
// orbital.
//
// Spin and charge are diagonal in the basis: one pass forms <O> (FP64
// partials of O |psi|^2 and |psi|^2 over the impurity masks of each
// element), one pass writes (O - <O>) psi into the block-major order of the
// same sector, and one chain serves both terms.  The pair operator changes
// both electron numbers: two c^+ (or c) applications through the Green's
// function's gather kernel with a layout permutation between them, one chain
// per term.  The chains run through the operator-generic Lanczos driver and
// the continued fractions through the Green's function's kernel.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int CHI_THREADS = 256;
constexpr int CHI_PARTS = 1024;

struct OTable {
  double v[1 << ED_MAX_NORB][1 << ED_MAX_NORB];  // O on impurity masks (m_up, m_dw)
};

// O = sum_a wts[a] O_a on the impurity masks (O_a the spin or charge
// operator of orbital a)
OTable make_table(int norb, int kind, const int *wts) {
  OTable t;
  memset(&t, 0, sizeof(t));
  for (int mu = 0; mu < (1 << norb); ++mu)
    for (int md = 0; md < (1 << norb); ++md) {
      double v = 0.0;
      for (int a = 0; a < norb; ++a) {
        const double nu = (mu >> a) & 1, nd = (md >> a) & 1;
        v += wts[a] * (kind == ED_CHI_SPIN ? 0.5 * (nu - nd) : nu + nd);
      }
      t.v[mu][md] = v;
    }
  return t;
}

// parts[cta] = sum O psi^2, parts[CHI_PARTS + cta] = sum psi^2 (sector order)
template <typename T>
__global__ void __launch_bounds__(CHI_THREADS) k_chi_expect(const T *psi, int64_t dup, int64_t n,
                                                            const uint8_t *mup,
                                                            const uint8_t *mdw, OTable ot,
                                                            double *parts) {
  __shared__ double red[2][CHI_THREADS / 32];
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / dup, c = i - r * dup;
    const double x = (double)psi[i];
    a += ot.v[mup[c]][mdw[r]] * x * x;
    b += x * x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < CHI_THREADS / 32; ++k) {
      sa += red[0][k];
      sb += red[1][k];
    }
    parts[blockIdx.x] = sa;
    parts[CHI_PARTS + blockIdx.x] = sb;
  }
}

// avg[0] = sum of the O psi^2 partials / sum of the psi^2 partials (fixed order)
__global__ void k_chi_avg(const double *parts, int np, double *avg) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < np; ++k) {
    a += parts[k];
    b += parts[CHI_PARTS + k];
  }
  avg[0] = b > 0.0 ? a / b : 0.0;
}

// phi (padded block-major) = (O - <O>) psi (sector order), padding zero
template <typename Ti, typename To>
__global__ void k_chi_apply(const Ti *psi, To *phi, const int32_t *pidx_dw, const int32_t *pidx_up,
                            const int32_t *padinv, const uint8_t *bk_mup, const uint8_t *bk_mdw,
                            int64_t dup, int64_t stride, int64_t ddw, OTable ot,
                            const double *avg) {
  const double o0 = avg[0];
  for (int64_t r = blockIdx.y; r < ddw; r += gridDim.y) {
    const Ti *src = psi + (int64_t)pidx_dw[r] * dup;
    To *dst = phi + r * stride;
    const int md = bk_mdw[r];
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < stride;
         c += (int64_t)gridDim.x * blockDim.x) {
      const int32_t cb = padinv[c];
      dst[c] = cb < 0 ? To(0) : (To)((ot.v[bk_mup[cb]][md] - o0) * (double)src[pidx_up[cb]]);
    }
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

// Imaginary-time output of a susceptibility call: C(tau) at ntau host times
// in [0, beta], accumulated on the host.
struct TauOut {
  const double *tau;
  int ntau;
  double beta;
  double *C;
};

// Eigenvalues lam and squared first eigenvector components w of the
// symmetric tridiagonal T_k (a[0..k-1], b[1..k-1]) by cyclic Jacobi rotations
// on its dense form: each rotation J (cos c, sin s in the plane p, q) zeroes
// the element (p, q) of J^T T J; only the first row of the accumulated
// rotations is kept, since the weights are its squares.  Sweeps until the
// off-diagonal part is below 1e-28 of the diagonal's squared norm.
void tridiag_poles(const double *a, const double *b, int k, std::vector<double> &lam,
                   std::vector<double> &w) {
  std::vector<double> A((size_t)k * k, 0.0), v(k, 0.0);
  for (int i = 0; i < k; ++i) {
    A[(size_t)i * k + i] = a[i];
    if (i > 0) A[(size_t)i * k + i - 1] = A[(size_t)(i - 1) * k + i] = b[i];
  }
  v[0] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int p = 0; p < k; ++p) {
      dia += A[(size_t)p * k + p] * A[(size_t)p * k + p];
      for (int q = p + 1; q < k; ++q) off += A[(size_t)p * k + q] * A[(size_t)p * k + q];
    }
    if (off <= 1e-28 * dia || off == 0.0) break;
    for (int p = 0; p + 1 < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = A[(size_t)p * k + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * k + p], aqq = A[(size_t)q * k + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        for (int r = 0; r < k; ++r) {
          if (r == p || r == q) continue;
          const double arp = A[(size_t)r * k + p], arq = A[(size_t)r * k + q];
          A[(size_t)r * k + p] = A[(size_t)p * k + r] = c * arp - sn * arq;
          A[(size_t)r * k + q] = A[(size_t)q * k + r] = sn * arp + c * arq;
        }
        A[(size_t)p * k + p] = app - t * apq;
        A[(size_t)q * k + q] = aqq + t * apq;
        A[(size_t)p * k + q] = A[(size_t)q * k + p] = 0.0;
        const double vp = v[p], vq = v[q];
        v[p] = c * vp - sn * vq;
        v[q] = sn * vp + c * vq;
      }
  }
  lam.resize(k);
  w.resize(k);
  for (int i = 0; i < k; ++i) {
    lam[i] = A[(size_t)i * k + i];
    w[i] = v[i] * v[i];
  }
}

// C(tau) += sgn-terms of the chain held in st (k steps): weight * sum_m w_m
// exp(-t (lam_m - e0)), t = tau for the O^+ chain (sgn +1), beta - tau for
// the O chain (sgn -1)
ed_status tau_accumulate(const LanczosState *st, int k, double weight, double e0, bool both,
                         int which, const TauOut &to, cudaStream_t cs) {
  std::vector<double> a(k), b(k);
  ED_TRY_CUDA(cudaMemcpyAsync(a.data(), st->alpha, k * sizeof(double), cudaMemcpyDeviceToHost, cs));
  ED_TRY_CUDA(cudaMemcpyAsync(b.data(), st->beta, k * sizeof(double), cudaMemcpyDeviceToHost, cs));
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  std::vector<double> lam, w;
  tridiag_poles(a.data(), b.data(), k, lam, w);
  for (int sg = +1; sg >= -1; sg -= 2) {
    if (!both && which != sg) continue;
    for (int i = 0; i < to.ntau; ++i) {
      const double t = sg > 0 ? to.tau[i] : to.beta - to.tau[i];
      double acc = 0.0;
      for (int m = 0; m < k; ++m) acc += w[m] * exp(-t * (lam[m] - e0));
      to.C[i] += weight * acc;
    }
  }
  return ED_OK;
}

// chain on sector nb from phi (block-major), then C += sgn-term (see ed_chi_z)
template <typename T>
ed_status chain_and_cfrac(ed_sector nb, const T *phi, int nsteps, double e0, const double2 *dz,
                          int nz, bool both, int which, double2 *dC, LanczosState *st,
                          double *weight, cudaStream_t cs, double coef = 1.0,
                          const TauOut *tout = nullptr) {
  ED_TRY(ed_build_items(nb, 1, (int)sizeof(T)));
  // FP32 chains run on H - e0, with the one-body diagonal tables shifted in
  // FP64 before their rounding (as the Green's-function chains)
  HvTables<T> tb = ed_hv_tables<T>(nb, 1);
  Mem shifted;
  double sigma = 0.0;
  if constexpr (std::is_same<T, float>::value) {
    ED_TRY(shifted.alloc(ed_shift_diag_bytes(nb), cs, "shifted diagonal"));
    ED_TRY(ed_shift_diag32(nb, e0, shifted.p, &tb, cs));
    sigma = e0;
  }
  LinOp<T> op;
  op.n = nb->bdim;
  op.apply = [nb, tb](const T *v, T *w, cudaStream_t s2) {
    return ed_launch_hv<T>(nb, tb, HV_PLAIN, v, w, nullptr, nullptr, nullptr, nullptr, nullptr, s2);
  };
  OpRun run;
  ED_TRY(ed_op_lanczos<T>(op, phi, nsteps, 0.0, false, &run, st, nullptr, cs));
  *weight = run.weight;
  if (run.weight <= 0.0 || run.k <= 0) return ED_OK;
  e0 -= sigma;
  if (tout) return tau_accumulate(st, run.k, coef * run.weight, e0, both, which, *tout, cs);
  // n+ [(e0 + z - T)^-1]_00 (sgn +1) and + n- [(e0 - z - T)^-1]_00: the
  // launcher adds sgn * weight * [(e0 + sgn z - T)^-1]_00, so the second
  // term takes sgn = -1 with weight -n-
  if (both || which > 0) ED_TRY(ed_cfrac_z_launch(st, coef * run.weight, e0, dz, nz, +1, dC, cs));
  if (both || which < 0) ED_TRY(ed_cfrac_z_launch(st, -coef * run.weight, e0, dz, nz, -1, dC, cs));
  return ED_OK;
}

// (spin and charge: O = sum_a wts[a] O_a, nullable wts = orbital `orb` alone;
// the chain's terms enter C with the factor `coef`)
template <typename Ti, typename To>
ed_status chi_impl(ed_sector s, ed_precision prec, const Ti *psi, double e0, int kind, int orb,
                   int nsteps, const double2 *dz, int nz, double2 *dC, LanczosState *st,
                   double *w, cudaStream_t cs, const int *wts = nullptr, double coef = 1.0,
                   const TauOut *tout = nullptr) {
  if (kind == ED_CHI_SPIN || kind == ED_CHI_CHARGE) {
    int one[ED_MAX_NORB] = {0};
    one[orb] = 1;
    const OTable ot = make_table(s->mp.norb, kind, wts ? wts : one);
    const int64_t n = s->dim, bn = s->bdim, dup = s->sp[0].dim, ddw = s->sp[1].dim;
    Mem scratch, phi;
    ED_TRY(scratch.alloc((2 * CHI_PARTS + 8) * sizeof(double), cs, "susceptibility partials"));
    ED_TRY(phi.alloc((size_t)bn * sizeof(To), cs, "susceptibility start vector"));
    double *parts = (double *)scratch.p, *avg = parts + 2 * CHI_PARTS;
    const unsigned g = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((n + 4 * CHI_THREADS - 1) / (4 * CHI_THREADS), CHI_PARTS));
    k_chi_expect<Ti><<<g, CHI_THREADS, 0, cs>>>(psi, dup, n, s->sp[0].imask, s->sp[1].imask, ot,
                                                parts);
    ED_LAUNCHED(1);
    k_chi_avg<<<1, 32, 0, cs>>>(parts, (int)g, avg);
    ED_LAUNCHED(1);
    const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((s->bstride + 255) / 256, 64)),
                    (unsigned)std::max<int64_t>(1, std::min<int64_t>(ddw, 65535)));
    k_chi_apply<Ti, To><<<grid, 256, 0, cs>>>(psi, (To *)phi.p, s->bi[1].pidx, s->bi[0].pidx,
                                              s->padinv, s->bk[0].imask, s->bk[1].imask, dup,
                                              s->bstride, ddw, ot, avg);
    ED_LAUNCHED(1);
    double wt = 0.0;
    ED_TRY(chain_and_cfrac<To>(s, (const To *)phi.p, nsteps, e0, dz, nz, true, 0, dC, st, &wt, cs,
                               coef, tout));
    w[0] = w[1] = wt;
    return ED_OK;
  }
  // pair: O^+ = d^+_up d^+_dw (d^+_dw first), O = d_dw d_up (d_up first)
  const ed_precision sp = sizeof(To) == 8 ? ED_FP64 : ED_FP32;
  for (int term = +1; term >= -1; term -= 2) {
    const int first = term > 0 ? 1 : 0, second = term > 0 ? 0 : 1;
    ed_sector s1 = nullptr, s2 = nullptr;
    ED_TRY(ed_neighbor_sector(s, first, term, cs, &s1));
    if (!s1 || s1->dim == 0) continue;
    ED_TRY(ed_neighbor_sector(s1, second, term, cs, &s2));
    if (!s2 || s2->dim == 0) continue;
    Mem a, b, c;
    ED_TRY(a.alloc((size_t)s1->bdim * sizeof(To), cs, "pair operator"));
    ED_TRY(b.alloc((size_t)s1->dim * sizeof(To), cs, "pair operator"));
    ED_TRY(c.alloc((size_t)s2->bdim * sizeof(To), cs, "pair operator"));
    ED_TRY((ed_apply_op_launch<Ti, To>(s, s1, psi, (To *)a.p, orb, first, term, cs)));
    ED_TRY(ed_permute_vec(s1, sp, false, a.p, b.p, cs));
    ED_TRY((ed_apply_op_launch<To, To>(s1, s2, (const To *)b.p, (To *)c.p, orb, second, term, cs)));
    double wt = 0.0;
    ED_TRY(chain_and_cfrac<To>(s2, (const To *)c.p, nsteps, e0, dz, nz, false, term, dC, st, &wt,
                               cs, 1.0, tout));
    w[term > 0 ? 0 : 1] = wt;
  }
  (void)prec;
  return ED_OK;
}

// ----------------------------------------------------------------- excitonic function
//
// O = sum_sigma (c^+_a c_b + c^+_b c_a) of an orbital pair: out = O x on the
// padded block-major layout, each element gathering the two moves between
// impurity levels a and b of its up string (same row) and of its dw string
// (same column) from the move tables (entry (index << 1) | sign, or -1);
// padding columns stay zero.  At most four terms of +-x, summed in FP64.
template <typename T>
__global__ void k_exciton_apply(const T *x, T *out, const int32_t *mup, const int32_t *mdw,
                                const int32_t *padinv, int64_t stride, int64_t ddw, int k1,
                                int k2) {
  for (int64_t r = blockIdx.y; r < ddw; r += gridDim.y) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < stride;
         c += (int64_t)gridDim.x * blockDim.x) {
      double acc = 0.0;
      if (padinv[c] >= 0) {
        for (int q = 0; q < 2; ++q) {
          const int k = q ? k2 : k1;
          const int32_t eu = mup[(int64_t)k * stride + c];
          if (eu >= 0) {
            const double v = (double)x[r * stride + (eu >> 1)];
            acc += (eu & 1) ? -v : v;
          }
          const int32_t ed = mdw[(int64_t)k * ddw + r];
          if (ed >= 0) {
            const double v = (double)x[(int64_t)(ed >> 1) * stride + c];
            acc += (ed & 1) ? -v : v;
          }
        }
      }
      out[r * stride + c] = (T)acc;
    }
  }
}

// parts[cta] = sum x y, parts[CHI_PARTS + cta] = sum x x (FP64)
template <typename T>
__global__ void __launch_bounds__(CHI_THREADS) k_exciton_dots(const T *x, const T *y, int64_t n,
                                                              double *parts) {
  __shared__ double red[2][CHI_THREADS / 32];
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double xi = (double)x[i];
    a += xi * (double)y[i];
    b += xi * xi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < CHI_THREADS / 32; ++k) {
      sa += red[0][k];
      sb += red[1][k];
    }
    parts[blockIdx.x] = sa;
    parts[CHI_PARTS + blockIdx.x] = sb;
  }
}

// phi = y - <O> x (the connected operator applied to psi)
template <typename Ti, typename To>
__global__ void k_exciton_phi(const Ti *x, const Ti *y, To *phi, int64_t n, const double *avg) {
  const double o0 = avg[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    phi[i] = (To)((double)y[i] - o0 * (double)x[i]);
}

template <typename Ti, typename To>
ed_status exciton_impl(ed_sector s, const Ti *psi, double e0, int a, int b, int nsteps,
                       const double2 *dz, int nz, double2 *dC, LanczosState *st, double *w,
                       cudaStream_t cs) {
  const int no = s->mp.norb;
  const int64_t bn = s->bdim, stride = s->bstride, ddw = s->sp[1].dim;
  Mem xb, ob, tabs, scratch, phi;
  ED_TRY(xb.alloc((size_t)bn * sizeof(Ti), cs, "excitonic operator"));
  ED_TRY(ob.alloc((size_t)bn * sizeof(Ti), cs, "excitonic operator"));
  ED_TRY(tabs.alloc((size_t)no * no * (stride + ddw) * sizeof(int32_t), cs, "move tables"));
  ED_TRY(scratch.alloc((2 * CHI_PARTS + 8) * sizeof(double), cs, "susceptibility partials"));
  ED_TRY(phi.alloc((size_t)bn * sizeof(To), cs, "susceptibility start vector"));
  int32_t *mup = (int32_t *)tabs.p, *mdw = mup + (size_t)no * no * stride;
  double *parts = (double *)scratch.p, *avg = parts + 2 * CHI_PARTS;
  ED_TRY(ed_move_tables(s, mup, mdw, cs));
  ED_TRY(ed_permute_vec(s, sizeof(Ti) == 8 ? ED_FP64 : ED_FP32, true, psi, xb.p, cs));
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((stride + 255) / 256, 64)),
                  (unsigned)std::max<int64_t>(1, std::min<int64_t>(ddw, 65535)));
  k_exciton_apply<Ti><<<grid, 256, 0, cs>>>((const Ti *)xb.p, (Ti *)ob.p, mup, mdw, s->padinv,
                                            stride, ddw, b * no + a, a * no + b);
  ED_LAUNCHED(1);
  const unsigned g = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((bn + 4 * CHI_THREADS - 1) / (4 * CHI_THREADS), CHI_PARTS));
  k_exciton_dots<Ti><<<g, CHI_THREADS, 0, cs>>>((const Ti *)xb.p, (const Ti *)ob.p, bn, parts);
  ED_LAUNCHED(1);
  k_chi_avg<<<1, 32, 0, cs>>>(parts, (int)g, avg);
  ED_LAUNCHED(1);
  k_exciton_phi<Ti, To><<<g, CHI_THREADS, 0, cs>>>((const Ti *)xb.p, (const Ti *)ob.p,
                                                   (To *)phi.p, bn, avg);
  ED_LAUNCHED(1);
  double wt = 0.0;
  ED_TRY(chain_and_cfrac<To>(s, (const To *)phi.p, nsteps, e0, dz, nz, true, 0, dC, st, &wt, cs));
  w[0] = w[1] = wt;
  return ED_OK;
}

// The device buffers of a susceptibility call (the frequencies, the
// accumulated C, one Lanczos state) around `run`, then C and the weights to
// the host.
template <typename F>
ed_status chi_call(const double *host_z, int32_t nz, double *host_C, double *host_w,
                   cudaStream_t cs, F run) {
  Mem buf;
  const size_t zb = (size_t)std::max(nz, 1) * sizeof(double2);
  ED_TRY(buf.alloc(2 * zb + ((sizeof(LanczosState) + 255) & ~(size_t)255), cs, "susceptibility"));
  double2 *dz = (double2 *)buf.p, *dC = (double2 *)((char *)buf.p + zb);
  LanczosState *st = (LanczosState *)((char *)buf.p + 2 * zb);
  if (nz > 0) {
    ED_TRY_CUDA(cudaMemcpyAsync(dz, host_z, nz * sizeof(double2), cudaMemcpyHostToDevice, cs));
    ED_TRY_CUDA(cudaMemsetAsync(dC, 0, nz * sizeof(double2), cs));
  }
  double w[2] = {0.0, 0.0};
  ED_TRY(run(dz, dC, st, w));
  if (nz > 0)
    ED_TRY_CUDA(cudaMemcpyAsync(host_C, dC, nz * sizeof(double2), cudaMemcpyDeviceToHost, cs));
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  if (host_w) {
    host_w[0] = w[0];
    host_w[1] = w[1];
  }
  return ED_OK;
}

// chi_impl in the precisions of `prec`
ed_status chi_prec(ed_sector s, ed_precision prec, const void *d_psi, double e0, int kind, int orb,
                   int nsteps, const double2 *dz, int nz, double2 *dC, LanczosState *st,
                   double *w, cudaStream_t cs, const int *wts = nullptr, double coef = 1.0,
                   const TauOut *tout = nullptr) {
  if (prec == ED_FP64)
    return chi_impl<double, double>(s, prec, (const double *)d_psi, e0, kind, orb, nsteps, dz, nz,
                                    dC, st, w, cs, wts, coef, tout);
  if (prec == ED_FP32)
    return chi_impl<float, float>(s, prec, (const float *)d_psi, e0, kind, orb, nsteps, dz, nz, dC,
                                  st, w, cs, wts, coef, tout);
  return chi_impl<double, float>(s, prec, (const double *)d_psi, e0, kind, orb, nsteps, dz, nz, dC,
                                 st, w, cs, wts, coef, tout);
}

}  // namespace

extern "C" ed_status ed_chi_z(ed_sector s, ed_precision prec, const void *d_psi, double e0,
                              int32_t kind, int32_t orb, int32_t nsteps, const double *host_z,
                              int32_t nz, double *host_C, double *host_w, void *stream) {
  if (!s || !d_psi || !host_C || nz < 0 || (nz > 0 && !host_z)) return ED_ERR_ARG;
  if (kind != ED_CHI_SPIN && kind != ED_CHI_CHARGE && kind != ED_CHI_PAIR) return ED_ERR_ARG;
  if (orb < 0 || orb >= s->mp.norb) return ED_ERR_ARG;
  if (prec != ED_FP64 && prec != ED_FP32 && prec != ED_FP32_POLISH) return ED_ERR_ARG;
  if (nsteps <= 0) nsteps = 200;
  if (nsteps > ED_MAX_LANCZOS) return ED_ERR_ARG;
  cudaStream_t cs = (cudaStream_t)stream;
  return chi_call(host_z, nz, host_C, host_w, cs,
                  [&](const double2 *dz, double2 *dC, LanczosState *st, double *w) {
                    return chi_prec(s, prec, d_psi, e0, kind, orb, nsteps, dz, nz, dC, st, w, cs);
                  });
}

// Imaginary time: C(tau) from each chain's poles and weights (tau_accumulate)
extern "C" ed_status ed_chi_tau(ed_sector s, ed_precision prec, const void *d_psi, double e0,
                                int32_t kind, int32_t orb, int32_t nsteps, double beta,
                                const double *host_tau, int32_t ntau, double *host_C,
                                void *stream) {
  if (!s || !d_psi || ntau < 0 || (ntau > 0 && (!host_tau || !host_C))) return ED_ERR_ARG;
  if (kind != ED_CHI_SPIN && kind != ED_CHI_CHARGE && kind != ED_CHI_PAIR) return ED_ERR_ARG;
  if (orb < 0 || orb >= s->mp.norb || !(beta > 0.0)) return ED_ERR_ARG;
  for (int i = 0; i < ntau; ++i)
    if (!(host_tau[i] >= 0.0 && host_tau[i] <= beta)) return ED_ERR_ARG;
  if (prec != ED_FP64 && prec != ED_FP32 && prec != ED_FP32_POLISH) return ED_ERR_ARG;
  if (nsteps <= 0) nsteps = 200;
  if (nsteps > ED_MAX_LANCZOS) return ED_ERR_ARG;
  cudaStream_t cs = (cudaStream_t)stream;
  for (int i = 0; i < ntau; ++i) host_C[i] = 0.0;
  const TauOut to{host_tau, ntau, beta, host_C};
  double unused[2];
  return chi_call(nullptr, 0, unused, nullptr, cs,
                  [&](const double2 *dz, double2 *dC, LanczosState *st, double *w) {
                    return chi_prec(s, prec, d_psi, e0, kind, orb, nsteps, dz, 0, dC, st, w, cs,
                                    nullptr, 1.0, &to);
                  });
}

// Inter-orbital spin / charge function: the auxiliary-operator construction
// of Sec. 6.8, C_ab = [C(O_a + O_b) - C_aa - C_bb] / 2 (real operators, real
// symmetric H: C_ab = C_ba), three chains accumulated into one C.  The
// excitonic kind: C_O of O = sum_sigma (c^+_a c_b + c^+_b c_a), one chain.
extern "C" ed_status ed_chi_ab_z(ed_sector s, ed_precision prec, const void *d_psi, double e0,
                                 int32_t kind, int32_t orb_a, int32_t orb_b, int32_t nsteps,
                                 const double *host_z, int32_t nz, double *host_C, void *stream) {
  if (!s || !d_psi || !host_C || nz < 0 || (nz > 0 && !host_z)) return ED_ERR_ARG;
  if (kind != ED_CHI_SPIN && kind != ED_CHI_CHARGE && kind != ED_CHI_EXCITON) return ED_ERR_ARG;
  const int norb = s->mp.norb;
  if (orb_a < 0 || orb_a >= norb || orb_b < 0 || orb_b >= norb) return ED_ERR_ARG;
  if (kind == ED_CHI_EXCITON && orb_a == orb_b) return ED_ERR_ARG;
  if (prec != ED_FP64 && prec != ED_FP32 && prec != ED_FP32_POLISH) return ED_ERR_ARG;
  if (nsteps <= 0) nsteps = 200;
  if (nsteps > ED_MAX_LANCZOS) return ED_ERR_ARG;
  cudaStream_t cs = (cudaStream_t)stream;
  if (kind == ED_CHI_EXCITON)
    return chi_call(host_z, nz, host_C, nullptr, cs,
                    [&](const double2 *dz, double2 *dC, LanczosState *st, double *w) {
                      if (prec == ED_FP64)
                        return exciton_impl<double, double>(s, (const double *)d_psi, e0, orb_a,
                                                            orb_b, nsteps, dz, nz, dC, st, w, cs);
                      if (prec == ED_FP32)
                        return exciton_impl<float, float>(s, (const float *)d_psi, e0, orb_a,
                                                          orb_b, nsteps, dz, nz, dC, st, w, cs);
                      return exciton_impl<double, float>(s, (const double *)d_psi, e0, orb_a,
                                                         orb_b, nsteps, dz, nz, dC, st, w, cs);
                    });
  int wab[ED_MAX_NORB] = {0}, wa[ED_MAX_NORB] = {0}, wb[ED_MAX_NORB] = {0};
  wab[orb_a] += 1;
  wab[orb_b] += 1;  // a = b: 2 O_a, and the combination gives C_aa
  wa[orb_a] = 1;
  wb[orb_b] = 1;
  return chi_call(host_z, nz, host_C, nullptr, cs,
                  [&](const double2 *dz, double2 *dC, LanczosState *st, double *w) {
                    ED_TRY(chi_prec(s, prec, d_psi, e0, kind, orb_a, nsteps, dz, nz, dC, st, w,
                                    cs, wab, 0.5));
                    ED_TRY(chi_prec(s, prec, d_psi, e0, kind, orb_a, nsteps, dz, nz, dC, st, w,
                                    cs, wa, -0.5));
                    return chi_prec(s, prec, d_psi, e0, kind, orb_b, nsteps, dz, nz, dC, st, w, cs,
                                    wb, -0.5);
                  });
}
