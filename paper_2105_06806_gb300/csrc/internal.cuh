// Internal declarations of the GB300 exact-diagonalisation library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "edgb.h"

// ----------------------------------------------------------------- errors

void ed_set_cuda_error(cudaError_t e, const char *what, const char *file, int line);
void ed_set_error_msg(const char *msg);
void ed_count_launches(int64_t n);

#define ED_TRY_CUDA(call)                                                   \
  do {                                                                      \
    cudaError_t e__ = (call);                                               \
    if (e__ != cudaSuccess) {                                               \
      ed_set_cuda_error(e__, #call, __FILE__, __LINE__);                    \
      return e__ == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA;   \
    }                                                                       \
  } while (0)

#define ED_TRY(call)                          \
  do {                                        \
    ed_status st__ = (call);                  \
    if (st__ != ED_OK) return st__;           \
  } while (0)

#define ED_LAUNCHED(n)                                                      \
  do {                                                                      \
    ed_count_launches(n);                                                   \
    cudaError_t e__ = cudaGetLastError();                                   \
    if (e__ != cudaSuccess) {                                               \
      ed_set_cuda_error(e__, "kernel launch", __FILE__, __LINE__);          \
      return ED_ERR_CUDA;                                                   \
    }                                                                       \
  } while (0)

// ----------------------------------------------------------------- memory (memory.cu)

// Stream-ordered device allocation from the library's pool (never
// synchronises the device); ed_dfree orders the release on `st`.
ed_status ed_dmalloc(void **p, size_t bytes, cudaStream_t st, const char *what);
void ed_dfree(void *p, cudaStream_t st);
// Device memory a new allocation can use: free device memory plus the
// blocks cached in the library's pool (current device).
ed_status ed_device_available(size_t *bytes);
// Non-blocking stream private to the calling host thread (current device).
cudaStream_t ed_private_stream(ed_status *st);
// Page-locked 4-byte host word for polling a device flag, from a recycled pool.
int32_t *ed_pinned_flag_acquire();
void ed_pinned_flag_release(int32_t *f);

struct PinnedFlag {
  int32_t *p = ed_pinned_flag_acquire();
  PinnedFlag() = default;
  PinnedFlag(const PinnedFlag &) = delete;
  PinnedFlag &operator=(const PinnedFlag &) = delete;
  ~PinnedFlag() { ed_pinned_flag_release(p); }
};

// ----------------------------------------------------------------- model

// Level energies and hybridisations indexed by level (Sec. 2.1): level a < Norb
// is impurity orbital a; level Norb + alpha*Nbath + nu is bath level nu of
// orbital alpha.  Passed by value to the table-building kernels.
struct ModelParams {
  int norb, nbath, ns;
  double eps[2][ED_MAX_NS];   // one-body level energies per spin
  double V[2][ED_MAX_NS];     // V of the bath level (0 for impurity levels)
  int orb_of_level[ED_MAX_NS];  // orbital alpha owning the level
  double U, Ust, Jh;
  double Jx, Jp;              // spin exchange, pair hopping (H_nd of Eq. Ham1)
};

// Per-spin basis and hopping tables of a sector (device pointers).
struct SpinTables {
  int n = 0;               // electrons of this spin
  int64_t dim = 0;         // D_sigma
  int64_t nnz = 0;
  uint32_t *map = nullptr;     // [dim] Ns-bit strings, ascending
  uint8_t *imask = nullptr;    // [dim] impurity occupation bits
  double *ediag = nullptr;     // [dim] E_sigma (FP64)
  float *ediag32 = nullptr;    // [dim] E_sigma rounded to FP32
  int32_t *rowptr = nullptr;   // [dim+1]
  int32_t *col = nullptr;      // [nnz] sorted per row
  double *val = nullptr;       // [nnz]
  float *val32 = nullptr;      // [nnz]
};

// Block-major order of one spin basis.  With a diagonal H^loc, a normal bath
// and the density-density interaction, the number of spin-s electrons in
// each orbital group {impurity level alpha} + {bath levels of alpha} is
// conserved (the per-orbital quantum numbers of Sec. 2.2; H_sigma then splits
// into a Kronecker sum over orbitals, Sec. 2.4).  The states of a total-N
// sector are therefore grouped into blocks by the tuple (n_0..n_{Norb-1}),
// blocks in lexicographic order of the tuple; inside a block the index is
// the mixed-radix number of the group strings (group 0 slowest), each group
// string ranked in colex order.  H_sigma maps every block to itself.
struct BlockView {
  int norb, nbath, g, nblocks;
  const int64_t *offset;    // [nblocks + 1]
  const int8_t *keys;       // [nblocks][norb]
  const int32_t *code2blk;  // [(g+1)^norb] -> block index or -1
};

struct BlockInfo {
  int nblocks = 0;
  std::vector<int64_t> offset;   // host copy, nblocks + 1
  std::vector<int8_t> keys;      // host copy
  int64_t *d_offset = nullptr;
  int8_t *d_keys = nullptr;
  int32_t *d_code2blk = nullptr;
  int32_t *pidx = nullptr;       // [dim] blocked index -> sector (paper) index
  int32_t *inv = nullptr;        // [dim] sector (paper) index -> blocked index
};

struct HvItem {
  int32_t r0, nr, c0, nc;  // rows [r0, r0+nr) x columns [c0, c0+nc), one block pair
  int32_t c0p;             // first column in the vector layout (padded in block-major)
  int32_t deg;             // ELL width of the up block (block-major), 0: use CSR
  int32_t ell_off;         // first ELL entry of the up block
  int32_t ncp;             // ELL row length (padded block width)
};

// Work item of the H_dw pass of the two-pass product: rows [r0, r0 + nr) of
// one dw block x padded columns [c0p, c0p + nc) of one up block (nc real
// columns, c0p a multiple of 4).
struct DwItem {
  int32_t r0, nr, c0p, nc;
};

struct ItemList {
  HvItem *d_items = nullptr;
  int64_t nitems = 0;
  size_t smem = 0;
  DwItem *d_ditems = nullptr;  // non-null: two-pass product (block pairs larger than L2)
  int64_t nditems = 0;
};

struct LanczosState;

// Move tables of the spin-exchange and pair-hopping terms (H_nd of Eq. Ham1)
// in one vector layout.  Both terms move one electron of each spin between
// two impurity orbitals, and each factorises into a move on the up string
// times a move on the dw string (the two N_up-dependent signs of the dw
// operators cancel): entry k = from * Norb + to of index i is the layout
// index of the string with the electron moved, shifted left by one, with
// bit 0 the sign (-1)^(occupied impurity levels strictly between), or -1
// where the move does not apply (and on padding columns).
struct NdTables {
  int32_t *up = nullptr;   // [Norb^2][ncols]
  int32_t *dw = nullptr;   // [Norb^2][D_dw]
  int64_t ncols = 0;       // columns of the layout (padded in block-major)
};

struct ed_sector_s {
  ModelParams mp;
  std::vector<double> e_imp, e_bath, v_bath;  // host copies (for neighbours)
  double U = 0, Ust = 0, Jh = 0;
  int nup = 0, ndw = 0;
  int64_t dim = 0;
  SpinTables sp[2];   // sector (paper) order: ascending strings
  SpinTables bk[2];   // block-major order (Lanczos vectors live in this order)
  BlockInfo bi[2];
  ItemList items[2][2];  // [layout 0 sector / 1 blocked][0 FP32 / 1 FP64]
  // Block-major vectors pad every up block to a multiple of 4 columns (16-byte
  // aligned row segments): row length bstride, length bdim = D_dw * bstride.
  int64_t bstride = 0, bdim = 0;
  std::vector<int64_t> up_off_pad;   // padded column offset of every up block
  int32_t *colpos = nullptr;         // [D_up] block-major column -> padded column
  int32_t *padinv = nullptr;         // [bstride] padded column -> column or -1
  // H_up of every up block as a column-major ELL table (entry e of local
  // column c at ell_off + e * ncp + c; padded with zero values): coalesced
  // reads when consecutive threads own consecutive columns.
  std::vector<int32_t> ell_deg, ell_off;  // host, per up block
  int32_t *ell_col = nullptr;             // local column of the entry
  float *ell_v32 = nullptr;
  double *ell_v64 = nullptr;
  // Per padded column of a block-major row (small sectors only): {column in
  // block-major up order or -1 for padding, its first ELL entry, first padded
  // column of its up block, (ELL row length << 8) | ELL width}.
  int4 *small_cols = nullptr;
  // block-major product kernel per precision [FP32, FP64]: -1 undecided,
  // 0 tiled (one- or two-pass), 1 element-parallel; pinned or autotuned
  int8_t hv_kernel[2] = {-1, -1};
  bool hv_pinned[2] = {false, false};
  double tune_ms[2][2] = {{-1.0, -1.0}, {-1.0, -1.0}};  // [precision][tiled, element-parallel]
  NdTables nd[2];          // [layout]; empty when J_X = J_P = 0
  double *W = nullptr;     // [2^norb][2^norb]
  float *W32 = nullptr;
  ed_sector nb[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [spin][0:c,1:c+]
  int64_t device_bytes = 0;
  bool spin_symmetric = false;
};

// Binomial table C[n][k], n,k <= 32, in constant memory.  Built at compile
// time (Pascal's rule) so every translation unit holds its own copy and no
// upload or relocatable device code is needed.
struct BinomTable {
  uint64_t v[33][33];
};
constexpr BinomTable ed_make_binom() {
  BinomTable t{};
  for (int n = 0; n <= 32; ++n) {
    t.v[n][0] = 1;
    for (int k = 1; k <= n; ++k) t.v[n][k] = t.v[n - 1][k - 1] + (k <= n - 1 ? t.v[n - 1][k] : 0);
  }
  return t;
}
static __constant__ BinomTable c_binom_tab = ed_make_binom();
#define c_binom (c_binom_tab.v)
inline ed_status ed_upload_binomials() { return ED_OK; }

// Output i of a SplitMix64 stream seeded with `seed` (Steele, Lea, Flood
// 2014): the seeded start vectors of the Lanczos drivers.
__device__ __forceinline__ uint64_t ed_splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t ed_unrank(uint64_t r, int ns, int n) {
  // Combinatorial number system: the r-th Ns-bit string with n set bits in
  // ascending order has set bits p_1 < ... < p_n with r = sum_k C(p_k, k).
  uint32_t I = 0;
  for (int k = n; k >= 1; --k) {
    int p = k - 1;
    while (p + 1 < ns && c_binom[p + 1][k] <= r) ++p;
    r -= c_binom[p][k];
    I |= 1u << p;
  }
  return I;
}

__device__ __forceinline__ int64_t ed_rank(uint32_t I) {
  int64_t r = 0;
  int k = 0;
  while (I) {
    int p = __ffs(I) - 1;
    ++k;
    r += (int64_t)c_binom[p][k];
    I &= I - 1;
  }
  return r;
}

__device__ __forceinline__ uint32_t ed_group_string(uint32_t I, int a, int norb, int nbath) {
  return ((I >> a) & 1u) | (((I >> (norb + a * nbath)) & ((1u << nbath) - 1u)) << 1);
}
__device__ __forceinline__ uint32_t ed_group_expand(uint32_t gs, int a, int norb, int nbath) {
  return ((gs & 1u) << a) | ((gs >> 1) << (norb + a * nbath));
}

__device__ __forceinline__ int64_t ed_blocked_rank(const BlockView &bv, uint32_t I) {
  int code = 0;
  uint32_t gs[ED_MAX_NORB];
  int n[ED_MAX_NORB];
  for (int a = 0; a < bv.norb; ++a) {
    gs[a] = ed_group_string(I, a, bv.norb, bv.nbath);
    n[a] = __popc(gs[a]);
    code = code * (bv.g + 1) + n[a];
  }
  const int b = bv.code2blk[code];
  int64_t idx = 0;
  for (int a = 0; a < bv.norb; ++a) idx = idx * (int64_t)c_binom[bv.g][n[a]] + ed_rank(gs[a]);
  return bv.offset[b] + idx;
}

__device__ __forceinline__ uint32_t ed_blocked_unrank(const BlockView &bv, int64_t i) {
  int lo = 0, hi = bv.nblocks - 1;
  while (lo < hi) {  // last block with offset <= i
    int mid = (lo + hi + 1) >> 1;
    if (bv.offset[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  int64_t w = i - bv.offset[lo];
  uint32_t I = 0;
  for (int a = bv.norb - 1; a >= 0; --a) {
    const int na = bv.keys[lo * bv.norb + a];
    const int64_t cnt = (int64_t)c_binom[bv.g][na];
    const int64_t r = w % cnt;
    w /= cnt;
    I |= ed_group_expand(ed_unrank((uint64_t)r, bv.g, na), a, bv.norb, bv.nbath);
  }
  return I;
}

// ----------------------------------------------------------------- kernels/launchers

// sector.cu
ed_status ed_build_sector_impl(const ModelParams &mp, double U, double Ust, double Jh,
                               int nup, int ndw, cudaStream_t st, ed_sector s);
ModelParams ed_model_params(const ed_model *m, ed_status *st);

// matvec.cu
template <typename T>
struct HvTables {
  int64_t dup, ddw;
  const int32_t *rp_up, *col_up, *rp_dw, *col_dw;
  const T *val_up, *val_dw, *e_up, *e_dw, *W;
  const uint8_t *m_up, *m_dw;
  int nmask;  // 2^norb
  const HvItem *items;
  int64_t nitems;
  size_t smem;
  int64_t stride;   // row length of the vector layout
  const int32_t *ell_col;
  const T *ell_val;
  const DwItem *ditems;    // non-null: two-pass product (H_up pass, then H_dw pass)
  int64_t nditems;
  const int4 *small_cols;  // non-null: element-parallel product (small sectors)
  int64_t small_grid;      // its CTAs (= block partials of the Lanczos mode)
  int32_t small_chunk;     // its elements per thread
  bool passa_wide;         // two-pass product: the wide shape of the H_up pass
  // H_nd (spin exchange, pair hopping): move tables of this layout, or null
  const int32_t *nd_up = nullptr, *nd_dw = nullptr;
  int64_t nd_ncols = 0;
  int nd_norb = 0;
  T nd_jx = T(0), nd_jp = T(0);
};

// Sum of the H_nd terms of Eq. Ham1 for the basis state of row r (impurity
// mask md) and column c (mask mu) of a layout: every up move b -> a (b
// occupied, a empty in mu) pairs with the dw move a -> b (spin exchange,
// +J_X: -J_X d+_{a up} d_{a dw} d+_{b dw} d_{b up} = +J_X (d+_{a up} d_{b up})
// (d+_{b dw} d_{a dw})) or b -> a (pair hopping, +J_P), whichever md allows.
// H_nd is real symmetric, so the terms applied to the output state give its
// row.  v is read at [row * stride + column] of the moved strings.
template <typename T>
__device__ __forceinline__ T ed_nd_terms(const HvTables<T> &tb, const T *v, int64_t stride,
                                         int64_t r, int64_t c, int mu, int md) {
  T acc = T(0);
  const int no = tb.nd_norb;
  for (int b = 0; b < no; ++b) {
    if (!((mu >> b) & 1)) continue;
    for (int a = 0; a < no; ++a) {
      if ((mu >> a) & 1) continue;
      int kd;
      T cf;
      if (((md >> a) & 1) && !((md >> b) & 1)) {
        kd = a * no + b;
        cf = tb.nd_jx;
      } else if (((md >> b) & 1) && !((md >> a) & 1)) {
        kd = b * no + a;
        cf = tb.nd_jp;
      } else {
        continue;
      }
      if (cf == T(0)) continue;
      const int32_t eu = __ldg(tb.nd_up + (int64_t)(b * no + a) * tb.nd_ncols + c);
      const int32_t ed = __ldg(tb.nd_dw + (int64_t)kd * tb.ddw + r);
      const T x = v[(int64_t)(ed >> 1) * stride + (eu >> 1)];
      acc += ((eu ^ ed) & 1) ? -cf * x : cf * x;
    }
  }
  return acc;
}

ed_status ed_build_nd_tables(ed_sector s, cudaStream_t st);
void ed_free_nd_tables(ed_sector s, cudaStream_t st);
// The block-major move tables of both spins (the format of NdTables: entry
// k = b * norb + a moves an electron from impurity level b to a) into caller
// device memory: up norb^2 * bstride, dw norb^2 * D_dw int32.
ed_status ed_move_tables(ed_sector s, int32_t *up, int32_t *dw, cudaStream_t st);
// CTAs (= partial sums of the Lanczos and dot modes) of the H_nd kernel
int64_t ed_nd_grid(int64_t ddw, int64_t ncols);
// Adds the H_nd terms after the factorised product (modes of k_hv; ND_DOT:
// part[cta] = sum_i v_i (H_nd v)_i, nothing written).
enum { ND_DOT = 3 };
template <typename T>
ed_status ed_launch_nd(const HvTables<T> &tb, int mode, const T *v, T *w, T *const *bufs,
                       T *const *basis, const struct LanczosState *state, double *part,
                       cudaStream_t st);
// layout 0: sector (paper) order; 1: block-major order
template <typename T>
HvTables<T> ed_hv_tables(ed_sector s, int layout);
ed_status ed_build_items(ed_sector s, int layout, int elem);
ed_status ed_build_ell(ed_sector s, cudaStream_t st);

// Lanczos device state (lanczos.cu).
struct LanczosState {
  int32_t j;          // completed steps
  int32_t done;       // 0 running, 1 converged, 2 breakdown, 3 max_iter
  int32_t maxit;
  int32_t check_every;  // fewest steps between two Ritz-value tests
  int32_t next_check;   // step of the next scheduled test
  int32_t pad_;
  double check_growth;  // a test at step k schedules the next one
                        // max(check_every, ceil(check_growth * k)) steps later
  double tol;
  double tnorm;
  double theta, rest;
  double scale[3];    // logical vector = scale[b] * buffer b
  double alpha[ED_MAX_LANCZOS];
  double beta[ED_MAX_LANCZOS + 1];
  double y[ED_MAX_LANCZOS];
  double acc[4];      // scratch reductions
  double cvv;         // <v_j, v_{j-1}>, from the update of the previous step
};

// Modes of the fused product kernel.
enum { HV_PLAIN = 0, HV_LANCZOS = 1, HV_SECOND = 2 };

template <typename T>
ed_status ed_launch_hv(ed_sector s, const HvTables<T> &tb, int mode, const T *v, T *w,
                       T *const *bufs, T *psi, LanczosState *state, double *part,
                       int64_t *nparts, cudaStream_t st,
                       T *const *basis = nullptr);

int64_t ed_hv_num_parts(ed_sector s, int layout, int elem_size);
template <typename T>
ed_status ed_hv_prepare();

// lanczos.cu
int64_t ed_reduce_grid(int64_t n);
// a chain of nsteps from bufs[0]; `tables` (nullable) replaces the sector's
// product tables (the shifted diagonal of FP32 chains)
template <typename T>
ed_status ed_lanczos_chain(ed_sector s, T *const *bufs, LanczosState *st, double *part,
                           double *part2, int64_t nparts_start, int nsteps, cudaStream_t cs,
                           int32_t *h_flag, const HvTables<T> *tables = nullptr);
ed_status ed_lanczos_ground_impl(ed_sector s, const ed_lanczos_opts *o, ed_lanczos_result *res,
                                 void *d_psi, cudaStream_t cs);

// sector.cu
ed_status ed_neighbor_sector(ed_sector s, int spin, int create, cudaStream_t st, ed_sector *out);
// Releases s (and its neighbour sectors) ordered on st, without
// synchronising the device; no work that reads s may be pending elsewhere.
void ed_sector_release(ed_sector s, cudaStream_t st);

// ----------------------------------------------------------------- operator Lanczos (oplanczos.cu)

#include <functional>

// A linear operator on device vectors of n elements (padding included; it
// must leave padding entries of w zero when those of v are zero).
template <typename T>
struct LinOp {
  int64_t n = 0;
  std::function<ed_status(const T *v, T *w, cudaStream_t)> apply;
};

struct OpRun {
  std::vector<double> alpha, beta;  // beta[0] = 0; beta[j] couples v_{j-1}, v_j
  int k = 0;                        // steps taken
  int stop = 0;                     // 0 converged, 1 breakdown, 2 step limit
  double theta = 0.0;               // lowest Ritz value (ground runs)
  double theta_max = 0.0;           // highest Ritz value (ground runs)
  double resid_est = 0.0;           // beta_{k+1} |y_k|
  double weight = 0.0;              // ||v0||^2
  std::vector<double> y;            // Ritz vector of theta
  int matvecs = 0;
};

// Lanczos from v0 (normalised inside): ground = stop on the lowest Ritz
// value's residual estimate (checked every 4 steps), else run to maxit or
// breakdown (a Green's-function chain).  alpha/beta also land in dst (device,
// nullable).  With ground and psi: the second pass writes the normalised
// Ritz vector into psi.
template <typename T>
ed_status ed_op_lanczos(const LinOp<T> &op, const T *v0, int maxit, double tol, bool ground,
                        OpRun *out, LanczosState *dst, T *psi, cudaStream_t cs);
ed_status ed_op_residual(const LinOp<double> &op, const double *psi, double *e, double *r,
                         cudaStream_t cs);
template <typename Ti, typename To>
ed_status ed_op_normalised_copy(const Ti *x, To *y, int64_t n, cudaStream_t cs);

// gf.cu: one c^+ / c application into a block-major slice, one continued fraction
template <typename Ti, typename To>
ed_status ed_apply_op_launch(ed_sector s, ed_sector nb, const Ti *psi, To *phi, int orb, int spin,
                             int create, cudaStream_t cs);
ed_status ed_cfrac_z_launch(const LanczosState *st, double weight, double e0, const double2 *dz,
                            int nz, int sgn, double2 *dG, cudaStream_t cs);
// gf.cu: the FP32 product tables of an FP32 chain on H - sigma (the one-body
// diagonal tables shifted in FP64, then rounded): ed_shift_diag_bytes(s) bytes
// of device scratch at `mem` receive them, tb->e_up / tb->e_dw point there
size_t ed_shift_diag_bytes(ed_sector s);
ed_status ed_shift_diag32(ed_sector s, double sigma, void *mem, HvTables<float> *tb,
                          cudaStream_t cs);
// lanczos.cu: sector order <-> block-major order of one vector
ed_status ed_permute_vec(ed_sector s, ed_precision prec, bool to_blocked, const void *in,
                         void *out, cudaStream_t cs);


