// Allocation-free residual check of a caller's vector.
//
// Some callers cannot let a library allocate device memory on this path:
// applications that hand all device memory to their own pool or arena
// allocator up front (an allocation by the library would fail or fragment
// their pool), and latency-critical loops in which cudaMalloc/cudaFree could
// block (cudaFree synchronises the device).  ed_residual_noalloc computes what the Lanczos driver's
// FP64 residual step computes (E = <psi,H psi>/<psi,psi> and
// ||H psi - E psi|| / ||psi||) without calling cudaMalloc, cudaFree or any
// allocating routine: its scratch (the vector H psi, per-CTA partial sums and
// the three result words) is the file-scope array below, which every GPU that
// loads the library holds until the process exits.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PARTS = 1024;   // CTAs of the reduction passes
constexpr int64_t NA_MAX_DIM = ED_NOALLOC_MAX_DIM;

// [0, NA_MAX_DIM): H psi; then 2 * NA_PARTS partial sums; then 4 result words.
constexpr int64_t NA_WORDS = NA_MAX_DIM + 2 * NA_PARTS + 4;
static __device__ __align__(256) double g_scratch[NA_WORDS];

// Host-side device address of g_scratch, looked up once per device with
// that device current (the symbol's host name is not a device address).
std::mutex g_mu;
double *g_addr[64] = {nullptr};

ed_status scratch_address(double **out) {
  int dev = 0;
  ED_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return ED_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      ed_set_cuda_error(e, "cudaGetSymbolAddress(residual scratch)", __FILE__, __LINE__);
      return ED_ERR_CUDA;
    }
    g_addr[dev] = (double *)p;
  }
  *out = g_addr[dev];
  return ED_OK;
}

__device__ __forceinline__ double na_warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

__device__ double na_block_sum(double x, double *red) {
  x = na_warp_sum(x);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
  return t;
}

// w = H psi in sector order, one thread per element (Eq. Hbuild): diagonal,
// H_up along the row, H_dw across rows at the same column.
__global__ void k_na_product(HvTables<double> tb, const double *psi, double *w, int64_t n) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += step) {
    const int64_t r = i / tb.dup, c = i - r * tb.dup;
    const double x = psi[i];
    double acc = (tb.e_up[c] + tb.e_dw[r] + tb.W[(int)tb.m_up[c] * tb.nmask + tb.m_dw[r]]) * x;
    for (int32_t k = tb.rp_up[c]; k < tb.rp_up[c + 1]; ++k)
      acc = fma(tb.val_up[k], psi[r * tb.dup + tb.col_up[k]], acc);
    for (int32_t k = tb.rp_dw[r]; k < tb.rp_dw[r + 1]; ++k)
      acc = fma(tb.val_dw[k], psi[(int64_t)tb.col_dw[k] * tb.dup + c], acc);
    w[i] = acc;
  }
}

// pass 1: <psi, w> and <psi, psi> per CTA
__global__ void k_na_rq_parts(const double *psi, const double *w, int64_t n, double *parts) {
  __shared__ double red[NA_THREADS / 32];
  double a = 0.0, c = 0.0;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += step) {
    a = fma(psi[i], w[i], a);
    c = fma(psi[i], psi[i], c);
  }
  a = na_block_sum(a, red);
  __syncthreads();
  c = na_block_sum(c, red);
  if (threadIdx.x == 0) {
    parts[blockIdx.x] = a;
    parts[NA_PARTS + blockIdx.x] = c;
  }
}

// E and <psi,psi> into the result words (one CTA, fixed order)
__global__ void k_na_rq_final(const double *parts, int nparts, double *res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, c = 0.0;
  for (int k = 0; k < nparts; ++k) {
    a += parts[k];
    c += parts[NA_PARTS + k];
  }
  res[0] = c > 0.0 ? a / c : 0.0;
  res[2] = c;
}

// pass 2: ||w - E psi||^2 per CTA (formed directly: no cancellation)
__global__ void k_na_res_parts(const double *psi, const double *w, int64_t n, const double *res,
                               double *parts) {
  __shared__ double red[NA_THREADS / 32];
  const double e = res[0];
  double b = 0.0;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += step) {
    const double d = fma(-e, psi[i], w[i]);
    b = fma(d, d, b);
  }
  b = na_block_sum(b, red);
  if (threadIdx.x == 0) parts[blockIdx.x] = b;
}

__global__ void k_na_res_final(const double *parts, int nparts, double *res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double b = 0.0;
  for (int k = 0; k < nparts; ++k) b += parts[k];
  res[1] = res[2] > 0.0 ? sqrt(b / res[2]) : 0.0;
}

}  // namespace

// The scratch array is shared by every call on a device and keeps the last
// call's contents.  Each call overwrites every word it reads before reading
// it (H psi, all partial sums of the CTAs it launches, the result words), so
// nothing needs clearing between calls; calls whose kernels overlap on the
// GPU (different streams, or different host threads) race on the array and
// must be serialised by the caller.
extern "C" ed_status ed_residual_noalloc(ed_sector s, const double *d_psi, int64_t n,
                                         double *host_e_r, void *stream) {
  if (!s || !d_psi || !host_e_r) return ED_ERR_ARG;
  if (n != s->dim) {
    ed_set_error_msg("vector length does not match the sector dimension");
    return ED_ERR_ARG;
  }
  if (n > NA_MAX_DIM) {
    ed_set_error_msg("sector dimension above ED_NOALLOC_MAX_DIM for ed_residual_noalloc");
    return ED_ERR_ARG;
  }
  double *scratch = nullptr;
  ED_TRY(scratch_address(&scratch));
  double *w = scratch;
  double *parts = scratch + NA_MAX_DIM;
  double *res = parts + 2 * NA_PARTS;
  cudaStream_t cs = (cudaStream_t)stream;

  HvTables<double> tb;
  tb.dup = s->sp[0].dim;
  tb.ddw = s->sp[1].dim;
  tb.rp_up = s->sp[0].rowptr;
  tb.col_up = s->sp[0].col;
  tb.val_up = s->sp[0].val;
  tb.e_up = s->sp[0].ediag;
  tb.m_up = s->sp[0].imask;
  tb.rp_dw = s->sp[1].rowptr;
  tb.col_dw = s->sp[1].col;
  tb.val_dw = s->sp[1].val;
  tb.e_dw = s->sp[1].ediag;
  tb.m_dw = s->sp[1].imask;
  tb.W = s->W;
  tb.nmask = 1 << s->mp.norb;
  // spin exchange and pair hopping (sector order), added after the product
  tb.stride = s->sp[0].dim;
  tb.nd_up = s->nd[0].up;
  tb.nd_dw = s->nd[0].dw;
  tb.nd_ncols = s->nd[0].ncols;
  tb.nd_norb = s->mp.norb;
  tb.nd_jx = s->mp.Jx;
  tb.nd_jp = s->mp.Jp;

  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(NA_PARTS, (n + NA_THREADS - 1) / NA_THREADS));
  k_na_product<<<grid, NA_THREADS, 0, cs>>>(tb, d_psi, w, n);
  ED_LAUNCHED(1);
  ED_TRY(ed_launch_nd<double>(tb, HV_PLAIN, d_psi, w, nullptr, nullptr, nullptr, nullptr, cs));
  k_na_rq_parts<<<grid, NA_THREADS, 0, cs>>>(d_psi, w, n, parts);
  ED_LAUNCHED(1);
  k_na_rq_final<<<1, 32, 0, cs>>>(parts, grid, res);
  ED_LAUNCHED(1);
  k_na_res_parts<<<grid, NA_THREADS, 0, cs>>>(d_psi, w, n, res, parts);
  ED_LAUNCHED(1);
  k_na_res_final<<<1, 32, 0, cs>>>(parts, grid, res);
  ED_LAUNCHED(1);
  double out[2];
  ED_TRY_CUDA(cudaMemcpyAsync(out, res, sizeof(out), cudaMemcpyDeviceToHost, cs));
  ED_TRY_CUDA(cudaStreamSynchronize(cs));
  host_e_r[0] = out[0];
  host_e_r[1] = out[1];
  return ED_OK;
}
