// Sector product w = H v (Sec. 6.7 without MPI, Eq. Hbuild) with optional
// Lanczos epilogues (Sec. 6.6).
//
// Layout: v is a row-major [D_dw][D_up] array (Eq. Vmatrix); row r is one
// down configuration.  One CTA owns R consecutive rows; it stages them in
// shared memory (coalesced loads), applies the diagonal and H_up along each
// row from shared memory, and adds the H_dw part by reading the neighbour
// rows k of r at the same columns (coalesced row segments, L2 resident for
// small sectors).  No transpose is formed: the strided axis of Sec. 3.2 is
// read directly by row segments.
#include <algorithm>
#include <mutex>

#include "internal.cuh"

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) {
  return __fmaf_rn(a, b, c);
}
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) {
  return __fma_rn(a, b, c);
}
template <typename T>
__device__ __forceinline__ T mul_t(T a, T b);
template <>
__device__ __forceinline__ float mul_t<float>(float a, float b) { return __fmul_rn(a, b); }
template <>
__device__ __forceinline__ double mul_t<double>(double a, double b) { return __dmul_rn(a, b); }
template <typename T>
__device__ __forceinline__ T add_t(T a, T b);
template <>
__device__ __forceinline__ float add_t<float>(float a, float b) { return __fadd_rn(a, b); }
template <>
__device__ __forceinline__ double add_t<double>(double a, double b) { return __dadd_rn(a, b); }

template <typename T>
HvTables<T> ed_hv_tables(ed_sector s);
template <>
HvTables<double> ed_hv_tables<double>(ed_sector s) {
  HvTables<double> t;
  t.dup = s->sp[0].dim;
  t.ddw = s->sp[1].dim;
  t.rp_up = s->sp[0].rowptr;
  t.col_up = s->sp[0].col;
  t.val_up = s->sp[0].val;
  t.e_up = s->sp[0].ediag;
  t.m_up = s->sp[0].imask;
  t.rp_dw = s->sp[1].rowptr;
  t.col_dw = s->sp[1].col;
  t.val_dw = s->sp[1].val;
  t.e_dw = s->sp[1].ediag;
  t.m_dw = s->sp[1].imask;
  t.W = s->W;
  t.nmask = 1 << s->mp.norb;
  return t;
}
template <>
HvTables<float> ed_hv_tables<float>(ed_sector s) {
  HvTables<float> t;
  t.dup = s->sp[0].dim;
  t.ddw = s->sp[1].dim;
  t.rp_up = s->sp[0].rowptr;
  t.col_up = s->sp[0].col;
  t.val_up = s->sp[0].val32;
  t.e_up = s->sp[0].ediag32;
  t.m_up = s->sp[0].imask;
  t.rp_dw = s->sp[1].rowptr;
  t.col_dw = s->sp[1].col;
  t.val_dw = s->sp[1].val32;
  t.e_dw = s->sp[1].ediag32;
  t.m_dw = s->sp[1].imask;
  t.W = s->W32;
  t.nmask = 1 << s->mp.norb;
  return t;
}

template <typename T>
struct HvLaunch {
  HvTables<T> tb;
  int rows_per_cta;
  int use_smem;
  const T *v;
  T *w;
  T *b0, *b1, *b2;
  T *psi;
  LanczosState *st;
  double *part;
};

constexpr int HV_THREADS = 512;
constexpr size_t HV_SMEM_MAX = 112 * 1024;

template <typename T>
__device__ __forceinline__ double block_sum(double x, double *red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  }
  return s;
}

// One output element: diagonal + H_up (row from `row`) + H_dw (neighbour rows
// of the global array `g`).  The summation order is fixed so that the two
// Lanczos passes reproduce each other bit for bit.
template <typename T>
__device__ __forceinline__ T hv_element(const HvTables<T> &tb, const T *__restrict__ row,
                                        const T *__restrict__ g, int64_t r, int64_t c) {
  const T x = row[c];
  T d = add_t<T>(add_t<T>(tb.e_up[c], tb.e_dw[r]), tb.W[(int)tb.m_up[c] * tb.nmask + tb.m_dw[r]]);
  T acc = mul_t<T>(d, x);
  const int32_t u0 = __ldg(tb.rp_up + c), u1 = __ldg(tb.rp_up + c + 1);
  for (int32_t k = u0; k < u1; ++k) acc = fma_t<T>(__ldg(tb.val_up + k), row[__ldg(tb.col_up + k)], acc);
  const int32_t d0 = __ldg(tb.rp_dw + r), d1 = __ldg(tb.rp_dw + r + 1);
  for (int32_t k = d0; k < d1; ++k)
    acc = fma_t<T>(__ldg(tb.val_dw + k), __ldg(g + (int64_t)__ldg(tb.col_dw + k) * tb.dup + c), acc);
  return acc;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(HV_THREADS) k_hv(HvLaunch<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[HV_THREADS / 32];
  T *srow = reinterpret_cast<T *>(smem_raw);
  const HvTables<T> &tb = a.tb;

  int j = 0;
  T s_cur = T(1), s_prev = T(0), beta_j = T(0), alpha_j = T(0), y_j = T(0);
  const T *g;
  const T *prev = nullptr;
  T *out;
  if (MODE == HV_PLAIN) {
    g = a.v;
    out = a.w;
  } else {
    const LanczosState *st = a.st;
    if (MODE == HV_LANCZOS && st->done) return;
    j = st->j;
    T *bufs[3] = {a.b0, a.b1, a.b2};
    g = bufs[j % 3];
    prev = bufs[(j + 2) % 3];
    out = bufs[(j + 1) % 3];
    s_cur = (T)st->scale[j % 3];
    s_prev = (T)st->scale[(j + 2) % 3];
    beta_j = (T)st->beta[j];
    if (MODE == HV_SECOND) {
      alpha_j = (T)st->alpha[j];
      y_j = (T)st->y[j];
    }
  }

  const int64_t R = a.rows_per_cta;
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int64_t r1 = min(r0 + R, tb.ddw);
  const int64_t dup = tb.dup;
  const int64_t nel = (r1 - r0) * dup;
  const int64_t base = r0 * dup;
  const T *rows = g + base;
  if (a.use_smem) {
    for (int64_t e = threadIdx.x; e < nel; e += blockDim.x) srow[e] = rows[e];
    __syncthreads();
    rows = srow;
  }

  T dot = T(0);
  auto epilogue = [&](int64_t e, T acc) {
    const int64_t gi = base + e;
    if (MODE == HV_PLAIN) {
      out[gi] = acc;
    } else {
      const T v = mul_t<T>(rows[e], s_cur);
      T w1 = mul_t<T>(acc, s_cur);
      if (j > 0) w1 = fma_t<T>(-beta_j, mul_t<T>(prev[gi], s_prev), w1);
      if (MODE == HV_LANCZOS) {
        out[gi] = w1;
        dot = fma_t<T>(v, w1, dot);
      } else {
        out[gi] = fma_t<T>(-alpha_j, v, w1);
        a.psi[gi] = fma_t<T>(y_j, v, a.psi[gi]);
      }
    }
  };

  if (dup >= (int64_t)blockDim.x) {
    for (int64_t lr = 0; lr < r1 - r0; ++lr) {
      const T *row = rows + lr * dup;
      for (int64_t c = threadIdx.x; c < dup; c += blockDim.x)
        epilogue(lr * dup + c, hv_element<T>(tb, row, g, r0 + lr, c));
    }
  } else {
    for (int64_t e = threadIdx.x; e < nel; e += blockDim.x) {
      const int64_t lr = e / dup, c = e - lr * dup;
      epilogue(e, hv_element<T>(tb, rows + lr * dup, g, r0 + lr, c));
    }
  }
  if (MODE == HV_LANCZOS) {
    double s = block_sum<T>((double)dot, red);
    if (threadIdx.x == 0) a.part[blockIdx.x] = s;
  }
}

static void hv_geometry(int64_t dup, int64_t ddw, int elem, int *R, int *use_smem, int64_t *nblk,
                        size_t *smem) {
  int64_t r = std::max<int64_t>(1, (2048 + dup - 1) / std::max<int64_t>(dup, 1));
  r = std::min<int64_t>(r, std::max<int64_t>(ddw, 1));
  size_t bytes = (size_t)(r * dup) * elem;
  while (r > 1 && bytes > HV_SMEM_MAX) {
    --r;
    bytes = (size_t)(r * dup) * elem;
  }
  *R = (int)r;
  *use_smem = bytes <= HV_SMEM_MAX ? 1 : 0;
  *smem = *use_smem ? bytes : 0;
  *nblk = (ddw + r - 1) / r;
}

int64_t ed_hv_num_parts(ed_sector s, int elem_size) {
  int R, us;
  int64_t nb;
  size_t sm;
  hv_geometry(s->sp[0].dim, s->sp[1].dim, elem_size, &R, &us, &nb, &sm);
  return nb;
}

// Opt the product kernels into large dynamic shared memory, once per device
// (outside any stream capture).
template <typename T>
ed_status ed_hv_prepare() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  ED_TRY_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && done[dev]) return ED_OK;
  ED_TRY_CUDA(cudaFuncSetAttribute(k_hv<T, HV_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)HV_SMEM_MAX));
  ED_TRY_CUDA(cudaFuncSetAttribute(k_hv<T, HV_LANCZOS>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HV_SMEM_MAX));
  ED_TRY_CUDA(cudaFuncSetAttribute(k_hv<T, HV_SECOND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)HV_SMEM_MAX));
  if (dev < 64) done[dev] = true;
  return ED_OK;
}
template ed_status ed_hv_prepare<float>();
template ed_status ed_hv_prepare<double>();

template <typename T, int MODE>
static ed_status launch_mode(const HvLaunch<T> &a, int64_t nblk, size_t smem, cudaStream_t st) {
  k_hv<T, MODE><<<(unsigned)nblk, HV_THREADS, smem, st>>>(a);
  ED_LAUNCHED(1);
  return ED_OK;
}

template <typename T>
ed_status ed_launch_hv(ed_sector s, const HvTables<T> &tb, int mode, const T *v, T *w,
                       T *const *bufs, T *psi, LanczosState *state, double *part,
                       int64_t *nparts, cudaStream_t st) {
  ED_TRY(ed_hv_prepare<T>());
  HvLaunch<T> a;
  a.tb = tb;
  int64_t nblk;
  size_t smem;
  hv_geometry(tb.dup, tb.ddw, (int)sizeof(T), &a.rows_per_cta, &a.use_smem, &nblk, &smem);
  if (nparts) *nparts = nblk;
  if (nblk == 0 || tb.dup == 0) return ED_OK;
  a.v = v;
  a.w = w;
  a.b0 = bufs ? bufs[0] : nullptr;
  a.b1 = bufs ? bufs[1] : nullptr;
  a.b2 = bufs ? bufs[2] : nullptr;
  a.psi = psi;
  a.st = state;
  a.part = part;
  if (mode == HV_PLAIN) return launch_mode<T, HV_PLAIN>(a, nblk, smem, st);
  if (mode == HV_LANCZOS) return launch_mode<T, HV_LANCZOS>(a, nblk, smem, st);
  return launch_mode<T, HV_SECOND>(a, nblk, smem, st);
}

template ed_status ed_launch_hv<float>(ed_sector, const HvTables<float> &, int, const float *,
                                       float *, float *const *, float *, LanczosState *, double *,
                                       int64_t *, cudaStream_t);
template ed_status ed_launch_hv<double>(ed_sector, const HvTables<double> &, int, const double *,
                                        double *, double *const *, double *, LanczosState *,
                                        double *, int64_t *, cudaStream_t);

extern "C" ed_status ed_matvec(ed_sector s, ed_precision prec, const void *d_v, void *d_w,
                               void *stream) {
  if (!s || !d_v || !d_w || d_v == d_w) return ED_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == ED_FP64) ED_TRY(ed_hv_prepare<double>());
  else ED_TRY(ed_hv_prepare<float>());
  if (prec == ED_FP64)
    return ed_launch_hv<double>(s, ed_hv_tables<double>(s), HV_PLAIN, (const double *)d_v,
                                (double *)d_w, nullptr, nullptr, nullptr, nullptr, nullptr, st);
  if (prec == ED_FP32 || prec == ED_FP32_POLISH)
    return ed_launch_hv<float>(s, ed_hv_tables<float>(s), HV_PLAIN, (const float *)d_v,
                               (float *)d_w, nullptr, nullptr, nullptr, nullptr, nullptr, st);
  return ED_ERR_ARG;
}
