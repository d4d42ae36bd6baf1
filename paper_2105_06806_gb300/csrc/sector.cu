// Sector set-up on the device: basis enumeration, ranks, per-spin CSR
// hopping matrices and diagonal tables (Sec. 2.3-2.4, Sec. 6.3).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "internal.cuh"

static uint64_t host_binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  uint64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
  return r;
}

ModelParams ed_model_params(const ed_model *m, ed_status *st) {
  ModelParams mp;
  memset(&mp, 0, sizeof(mp));
  *st = ED_OK;
  if (!m || m->norb < 1 || m->nbath < 0 || !m->e_imp || (m->nbath > 0 && (!m->e_bath || !m->v_bath))) {
    *st = ED_ERR_ARG;
    return mp;
  }
  if (m->norb > ED_MAX_NORB || m->norb * (m->nbath + 1) > ED_MAX_NS) {
    *st = ED_ERR_UNSUPPORTED;
    return mp;
  }
  mp.norb = m->norb;
  mp.nbath = m->nbath;
  mp.ns = m->norb * (m->nbath + 1);
  mp.U = m->U;
  mp.Ust = m->Ust;
  mp.Jh = m->Jh;
  mp.Jx = m->Jx;
  mp.Jp = m->Jp;
  for (int s = 0; s < 2; ++s) {
    for (int a = 0; a < m->norb; ++a) {
      mp.eps[s][a] = m->e_imp[s * m->norb + a];
      mp.V[s][a] = 0.0;
      mp.orb_of_level[a] = a;
      for (int nu = 0; nu < m->nbath; ++nu) {
        int lev = m->norb + a * m->nbath + nu;
        mp.eps[s][lev] = m->e_bath[(s * m->norb + a) * m->nbath + nu];
        mp.V[s][lev] = m->v_bath[(s * m->norb + a) * m->nbath + nu];
        mp.orb_of_level[lev] = a;
      }
    }
  }
  return mp;
}

// ----------------------------------------------------------------- kernels

template <int ORDER>
__device__ __forceinline__ uint32_t order_unrank(const BlockView &bv, int64_t i, int ns, int n) {
  return ORDER == 0 ? ed_unrank((uint64_t)i, ns, n) : ed_blocked_unrank(bv, i);
}
template <int ORDER>
__device__ __forceinline__ int64_t order_rank(const BlockView &bv, uint32_t I) {
  return ORDER == 0 ? ed_rank(I) : ed_blocked_rank(bv, I);
}

// One thread per basis state: the string, impurity mask, diagonal energy
// E_sigma = sum_a eps_a n_a + (U'-J) sum_{alpha<beta} n_alpha n_beta, and for
// the block-major order the permutation to and from sector order.
template <int ORDER>
__global__ void k_spin_basis(ModelParams mp, BlockView bv, int spin, int n, int64_t dim,
                             uint32_t *map, uint8_t *imask, double *ediag, float *ediag32,
                             int32_t *pidx, int32_t *inv) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= dim) return;
  uint32_t I = order_unrank<ORDER>(bv, i, mp.ns, n);
  map[i] = I;
  uint32_t m = I & ((1u << mp.norb) - 1u);
  imask[i] = (uint8_t)m;
  double e = 0.0;
  for (int a = 0; a < mp.ns; ++a)
    if ((I >> a) & 1u) e += mp.eps[spin][a];
  int k = __popc(m);
  e += (mp.Ust - mp.Jh) * (double)(k * (k - 1) / 2);
  ediag[i] = e;
  ediag32[i] = (float)e;
  if (ORDER == 1) {
    const int32_t p = (int32_t)ed_rank(I);
    pidx[i] = p;
    inv[p] = (int32_t)i;
  }
}

// Hops of one state: for each bath level b of orbital alpha, exactly one of
// (impurity level alpha, b) occupied -> one matrix element of H_sigma.
__device__ __forceinline__ int hop_count(const ModelParams &mp, uint32_t I) {
  int c = 0;
  for (int b = mp.norb; b < mp.ns; ++b) {
    int d = mp.orb_of_level[b];
    c += (int)(((I >> d) ^ (I >> b)) & 1u);
  }
  return c;
}

__global__ void k_row_counts(ModelParams mp, int64_t dim, const uint32_t *map, int32_t *cnt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= dim) return;
  cnt[i] = hop_count(mp, map[i]);
}

// Exclusive scan of the row counts into rowptr (one CTA, fixed order).
__global__ void k_scan_rowptr(int64_t dim, const int32_t *cnt, int32_t *rowptr) {
  __shared__ int32_t sums[1024];
  const int T = blockDim.x;
  const int t = threadIdx.x;
  int64_t chunk = (dim + T - 1) / T;
  int64_t lo = t * chunk, hi = min(dim, lo + chunk);
  int32_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += cnt[i];
  sums[t] = s;
  __syncthreads();
  if (t == 0) {
    int32_t run = 0;
    for (int k = 0; k < T; ++k) {
      int32_t x = sums[k];
      sums[k] = run;
      run += x;
    }
  }
  __syncthreads();
  int32_t run = sums[t];
  for (int64_t i = lo; i < hi; ++i) {
    rowptr[i] = run;
    run += cnt[i];
  }
  if (hi == dim && lo < hi) rowptr[dim] = run;
  if (dim == 0 && t == 0) rowptr[0] = 0;
}

// CSR fill: H_sigma[i, j] = V * (-1)^(occupied levels strictly between the
// two levels) for J = I with the electron moved (Eq. Hbuild, Sec. 2.3 signs).
template <int ORDER>
__global__ void k_fill_csr(ModelParams mp, BlockView bv, int spin, int64_t dim, const uint32_t *map,
                           const int32_t *rowptr, int32_t *col, double *val, float *val32) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= dim) return;
  uint32_t I = map[i];
  int32_t cs[ED_MAX_NS];
  double vs[ED_MAX_NS];
  int m = 0;
  for (int b = mp.norb; b < mp.ns; ++b) {
    int d = mp.orb_of_level[b];
    if ((((I >> d) ^ (I >> b)) & 1u) == 0u) continue;
    uint32_t J = I ^ (1u << d) ^ (1u << b);
    int lo = d < b ? d : b, hi = d < b ? b : d;
    uint32_t between = ((1u << hi) - 1u) & ~((2u << lo) - 1u);
    double sg = (__popc(I & between) & 1) ? -1.0 : 1.0;
    int32_t c = (int32_t)order_rank<ORDER>(bv, J);
    double v = sg * mp.V[spin][b];
    // insertion keeps the row sorted by column
    int p = m;
    while (p > 0 && cs[p - 1] > c) {
      cs[p] = cs[p - 1];
      vs[p] = vs[p - 1];
      --p;
    }
    cs[p] = c;
    vs[p] = v;
    ++m;
  }
  int32_t o = rowptr[i];
  for (int k = 0; k < m; ++k) {
    col[o + k] = cs[k];
    val[o + k] = vs[k];
    val32[o + k] = (float)vs[k];
  }
}

// W[m_up][m_dw] = U sum_a n_a,up n_a,dw + U' sum_{a != b} n_a,up n_b,dw.
__global__ void k_wtable(ModelParams mp, double *W, float *W32) {
  int nm = 1 << mp.norb;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nm * nm) return;
  int mu = t / nm, md = t % nm;
  double w = 0.0;
  for (int a = 0; a < mp.norb; ++a)
    for (int b = 0; b < mp.norb; ++b)
      if (((mu >> a) & 1) && ((md >> b) & 1)) w += (a == b) ? mp.U : mp.Ust;
  W[t] = w;
  W32[t] = (float)w;
}

// ----------------------------------------------------------------- host

template <typename P>
static ed_status dalloc(ed_sector s, cudaStream_t st, P **p, size_t count) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(P);
  ED_TRY(ed_dmalloc((void **)p, bytes, st, "sector table"));
  s->device_bytes += (int64_t)bytes;
  return ED_OK;
}

// Blocks of the block-major order: all tuples (n_0..n_{Norb-1}) with
// 0 <= n_alpha <= Nbath+1 and sum N, in lexicographic order (host metadata).
static void enumerate_blocks(int norb, int g, int n, int a, std::vector<int8_t> &cur,
                             std::vector<int8_t> &keys) {
  if (a == norb) {
    if (n == 0) keys.insert(keys.end(), cur.begin(), cur.end());
    return;
  }
  for (int k = 0; k <= std::min(g, n); ++k) {
    cur[a] = (int8_t)k;
    enumerate_blocks(norb, g, n - k, a + 1, cur, keys);
  }
}

static ed_status build_blocks(ed_sector s, int spin, int n, cudaStream_t st, BlockView *bv) {
  const ModelParams &mp = s->mp;
  BlockInfo &b = s->bi[spin];
  const int g = mp.nbath + 1;
  std::vector<int8_t> cur(mp.norb, 0);
  b.keys.clear();
  enumerate_blocks(mp.norb, g, n, 0, cur, b.keys);
  b.nblocks = (int)(b.keys.size() / mp.norb);
  b.offset.assign(b.nblocks + 1, 0);
  int ncode = 1;
  for (int a = 0; a < mp.norb; ++a) ncode *= (g + 1);
  std::vector<int32_t> code2blk(ncode, -1);
  for (int k = 0; k < b.nblocks; ++k) {
    int64_t sz = 1;
    int code = 0;
    for (int a = 0; a < mp.norb; ++a) {
      sz *= (int64_t)host_binom(g, b.keys[k * mp.norb + a]);
      code = code * (g + 1) + b.keys[k * mp.norb + a];
    }
    b.offset[k + 1] = b.offset[k] + sz;
    code2blk[code] = k;
  }
  ED_TRY(dalloc(s, st, &b.d_offset, b.nblocks + 1));
  ED_TRY(dalloc(s, st, &b.d_keys, std::max<size_t>(b.keys.size(), 1)));
  ED_TRY(dalloc(s, st, &b.d_code2blk, ncode));
  ED_TRY_CUDA(cudaMemcpyAsync(b.d_offset, b.offset.data(), (b.nblocks + 1) * sizeof(int64_t),
                              cudaMemcpyHostToDevice, st));
  if (!b.keys.empty())
    ED_TRY_CUDA(cudaMemcpyAsync(b.d_keys, b.keys.data(), b.keys.size(), cudaMemcpyHostToDevice, st));
  ED_TRY_CUDA(cudaMemcpyAsync(b.d_code2blk, code2blk.data(), ncode * sizeof(int32_t),
                              cudaMemcpyHostToDevice, st));
  // the host vectors must outlive the asynchronous copies: the sector build
  // synchronises the stream before returning
  bv->norb = mp.norb;
  bv->nbath = mp.nbath;
  bv->g = g;
  bv->nblocks = b.nblocks;
  bv->offset = b.d_offset;
  bv->keys = b.d_keys;
  bv->code2blk = b.d_code2blk;
  return ED_OK;
}

BlockView ed_block_view(ed_sector s, int spin) {
  BlockView bv;
  const BlockInfo &b = s->bi[spin];
  bv.norb = s->mp.norb;
  bv.nbath = s->mp.nbath;
  bv.g = s->mp.nbath + 1;
  bv.nblocks = b.nblocks;
  bv.offset = b.d_offset;
  bv.keys = b.d_keys;
  bv.code2blk = b.d_code2blk;
  return bv;
}

template <int ORDER>
static ed_status build_spin(ed_sector s, int spin, int n, cudaStream_t st, const BlockView &bv) {
  const ModelParams &mp = s->mp;
  SpinTables &t = ORDER == 0 ? s->sp[spin] : s->bk[spin];
  t.n = n;
  t.dim = (int64_t)host_binom(mp.ns, n);
  // every bath level contributes 2*C(Ns-2, n-1) hops (exactly one of the two
  // levels occupied)
  t.nnz = (int64_t)mp.norb * mp.nbath * 2 * (int64_t)host_binom(mp.ns - 2, n - 1);
  if (t.nnz >= (int64_t)INT32_MAX || t.dim >= (int64_t)INT32_MAX) return ED_ERR_UNSUPPORTED;
  ED_TRY(dalloc(s, st, &t.map, t.dim));
  ED_TRY(dalloc(s, st, &t.imask, t.dim));
  ED_TRY(dalloc(s, st, &t.ediag, t.dim));
  ED_TRY(dalloc(s, st, &t.ediag32, t.dim));
  ED_TRY(dalloc(s, st, &t.rowptr, t.dim + 1));
  ED_TRY(dalloc(s, st, &t.col, t.nnz));
  ED_TRY(dalloc(s, st, &t.val, t.nnz));
  ED_TRY(dalloc(s, st, &t.val32, t.nnz));
  int32_t *pidx = nullptr, *inv = nullptr;
  if (ORDER == 1) {
    ED_TRY(dalloc(s, st, &s->bi[spin].pidx, t.dim));
    ED_TRY(dalloc(s, st, &s->bi[spin].inv, t.dim));
    pidx = s->bi[spin].pidx;
    inv = s->bi[spin].inv;
  }
  int32_t *cnt = nullptr;
  ED_TRY(ed_dmalloc((void **)&cnt, std::max<int64_t>(t.dim, 1) * sizeof(int32_t), st, "row counts"));
  int threads = 256;
  int blocks = (int)((t.dim + threads - 1) / threads);
  if (t.dim > 0) {
    k_spin_basis<ORDER><<<blocks, threads, 0, st>>>(mp, bv, spin, n, t.dim, t.map, t.imask,
                                                    t.ediag, t.ediag32, pidx, inv);
    ED_LAUNCHED(1);
    k_row_counts<<<blocks, threads, 0, st>>>(mp, t.dim, t.map, cnt);
    ED_LAUNCHED(1);
  }
  k_scan_rowptr<<<1, 1024, 0, st>>>(t.dim, cnt, t.rowptr);
  ED_LAUNCHED(1);
  if (t.dim > 0) {
    k_fill_csr<ORDER><<<blocks, threads, 0, st>>>(mp, bv, spin, t.dim, t.map, t.rowptr, t.col,
                                                  t.val, t.val32);
    ED_LAUNCHED(1);
  }
  ed_dfree(cnt, st);
  return ED_OK;
}

ed_status ed_build_sector_impl(const ModelParams &mp, double U, double Ust, double Jh, int nup,
                               int ndw, cudaStream_t st, ed_sector s) {
  ED_TRY(ed_upload_binomials());
  s->mp = mp;
  s->U = U;
  s->Ust = Ust;
  s->Jh = Jh;
  s->nup = nup;
  s->ndw = ndw;
  BlockView none;
  memset(&none, 0, sizeof(none));
  for (int spin = 0; spin < 2; ++spin) {
    const int n = spin == 0 ? nup : ndw;
    ED_TRY(build_spin<0>(s, spin, n, st, none));
    BlockView bv;
    ED_TRY(build_blocks(s, spin, n, st, &bv));
    ED_TRY(build_spin<1>(s, spin, n, st, bv));
  }
  s->dim = s->sp[0].dim * s->sp[1].dim;
  // padded block-major columns: every up block rounded up to 4 columns
  {
    const BlockInfo &b = s->bi[0];
    s->up_off_pad.assign(b.nblocks + 1, 0);
    for (int k = 0; k < b.nblocks; ++k)
      s->up_off_pad[k + 1] = s->up_off_pad[k] + (b.offset[k + 1] - b.offset[k] + 3) / 4 * 4;
    s->bstride = s->up_off_pad[b.nblocks];
    s->bdim = s->bstride * s->sp[1].dim;
    std::vector<int32_t> colpos(s->sp[0].dim), padinv(std::max<int64_t>(s->bstride, 1), -1);
    for (int k = 0; k < b.nblocks; ++k)
      for (int64_t c = b.offset[k]; c < b.offset[k + 1]; ++c) {
        const int64_t pc = s->up_off_pad[k] + (c - b.offset[k]);
        colpos[c] = (int32_t)pc;
        padinv[pc] = (int32_t)c;
      }
    ED_TRY(dalloc(s, st, &s->colpos, colpos.size()));
    ED_TRY(dalloc(s, st, &s->padinv, padinv.size()));
    ED_TRY_CUDA(cudaMemcpyAsync(s->colpos, colpos.data(), colpos.size() * 4, cudaMemcpyHostToDevice, st));
    ED_TRY_CUDA(cudaMemcpyAsync(s->padinv, padinv.data(), padinv.size() * 4, cudaMemcpyHostToDevice, st));
  }
  // spin exchange and pair hopping (J_X, J_P != 0): move tables of both layouts
  ED_TRY(ed_build_nd_tables(s, st));
  int nm = 1 << mp.norb;
  ED_TRY(dalloc(s, st, &s->W, nm * nm));
  ED_TRY(dalloc(s, st, &s->W32, nm * nm));
  k_wtable<<<(nm * nm + 63) / 64, 64, 0, st>>>(mp, s->W, s->W32);
  ED_LAUNCHED(1);
  bool sym = true;
  for (int a = 0; a < mp.ns; ++a)
    if (mp.eps[0][a] != mp.eps[1][a] || mp.V[0][a] != mp.V[1][a]) sym = false;
  s->spin_symmetric = sym;
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  return ED_OK;
}

static void free_spin(SpinTables &t, cudaStream_t st) {
  ed_dfree(t.map, st);
  ed_dfree(t.imask, st);
  ed_dfree(t.ediag, st);
  ed_dfree(t.ediag32, st);
  ed_dfree(t.rowptr, st);
  ed_dfree(t.col, st);
  ed_dfree(t.val, st);
  ed_dfree(t.val32, st);
  t = SpinTables();
}

// Releases the device tables of s and of its cached neighbour sectors,
// ordered on `st`; work on other streams that reads them must already be
// complete or ordered before `st`.
static void sector_destroy(ed_sector s, cudaStream_t st) {
  if (!s) return;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) sector_destroy(s->nb[a][b], st);
  for (int sp = 0; sp < 2; ++sp) {
    free_spin(s->sp[sp], st);
    free_spin(s->bk[sp], st);
    ed_dfree(s->bi[sp].d_offset, st);
    ed_dfree(s->bi[sp].d_keys, st);
    ed_dfree(s->bi[sp].d_code2blk, st);
    ed_dfree(s->bi[sp].pidx, st);
    ed_dfree(s->bi[sp].inv, st);
    for (int e = 0; e < 2; ++e) {
      ed_dfree(s->items[sp][e].d_items, st);
      ed_dfree(s->items[sp][e].d_ditems, st);
    }
  }
  ed_dfree(s->colpos, st);
  ed_dfree(s->padinv, st);
  ed_dfree(s->ell_col, st);
  ed_dfree(s->ell_v32, st);
  ed_dfree(s->ell_v64, st);
  ed_dfree(s->small_cols, st);
  ed_dfree(s->W, st);
  ed_dfree(s->W32, st);
  ed_free_nd_tables(s, st);
  delete s;
}

void ed_sector_release(ed_sector s, cudaStream_t st) { sector_destroy(s, st); }

extern "C" ed_status ed_sector_build(const ed_model *model, int32_t nup, int32_t ndw,
                                     void *stream, ed_sector *out) {
  if (!out) return ED_ERR_ARG;
  *out = nullptr;
  ed_status st = ED_OK;
  ModelParams mp = ed_model_params(model, &st);
  if (st != ED_OK) return st;
  if (nup < 0 || ndw < 0 || nup > mp.ns || ndw > mp.ns) return ED_ERR_ARG;
  ed_sector s = new ed_sector_s();
  s->e_imp.assign(model->e_imp, model->e_imp + 2 * model->norb);
  size_t nb = (size_t)2 * model->norb * model->nbath;
  if (nb) {
    s->e_bath.assign(model->e_bath, model->e_bath + nb);
    s->v_bath.assign(model->v_bath, model->v_bath + nb);
  }
  st = ed_build_sector_impl(mp, model->U, model->Ust, model->Jh, nup, ndw,
                            (cudaStream_t)stream, s);
  if (st != ED_OK) {
    sector_destroy(s, (cudaStream_t)stream);
    return st;
  }
  *out = s;
  return ED_OK;
}

// Neighbour sector for the Green's function chains (cached in `s`).
ed_status ed_neighbor_sector(ed_sector s, int spin, int create, cudaStream_t st, ed_sector *out) {
  int slot = create > 0 ? 1 : 0;
  if (s->nb[spin][slot]) {
    *out = s->nb[spin][slot];
    return ED_OK;
  }
  int nup = s->nup + (spin == 0 ? create : 0);
  int ndw = s->ndw + (spin == 1 ? create : 0);
  if (nup < 0 || ndw < 0 || nup > s->mp.ns || ndw > s->mp.ns) {
    *out = nullptr;
    return ED_OK;
  }
  ed_sector n = new ed_sector_s();
  n->e_imp = s->e_imp;
  n->e_bath = s->e_bath;
  n->v_bath = s->v_bath;
  ed_status r = ed_build_sector_impl(s->mp, s->U, s->Ust, s->Jh, nup, ndw, st, n);
  if (r != ED_OK) {
    sector_destroy(n, st);
    return r;
  }
  s->nb[spin][slot] = n;
  *out = n;
  return ED_OK;
}

extern "C" ed_status ed_sector_get_info(ed_sector s, ed_sector_info *out) {
  if (!s || !out) return ED_ERR_ARG;
  out->ns = s->mp.ns;
  out->norb = s->mp.norb;
  out->nbath = s->mp.nbath;
  out->nup = s->nup;
  out->ndw = s->ndw;
  out->dim_up = s->sp[0].dim;
  out->dim_dw = s->sp[1].dim;
  out->dim = s->dim;
  out->nnz_up = s->sp[0].nnz;
  out->nnz_dw = s->sp[1].nnz;
  out->device_bytes = s->device_bytes;
  out->blocked_stride = s->bstride;
  out->blocked_dim = s->bdim;
  return ED_OK;
}

extern "C" ed_status ed_sector_copy_tables(ed_sector s, int32_t spin, uint32_t *host_map,
                                           int32_t *host_rowptr, int32_t *host_col,
                                           double *host_val, double *host_ediag,
                                           uint8_t *host_imask) {
  if (!s || spin < 0 || spin > 1) return ED_ERR_ARG;
  const SpinTables &t = s->sp[spin];
  if (host_map) ED_TRY_CUDA(cudaMemcpy(host_map, t.map, t.dim * 4, cudaMemcpyDeviceToHost));
  if (host_rowptr)
    ED_TRY_CUDA(cudaMemcpy(host_rowptr, t.rowptr, (t.dim + 1) * 4, cudaMemcpyDeviceToHost));
  if (host_col) ED_TRY_CUDA(cudaMemcpy(host_col, t.col, t.nnz * 4, cudaMemcpyDeviceToHost));
  if (host_val) ED_TRY_CUDA(cudaMemcpy(host_val, t.val, t.nnz * 8, cudaMemcpyDeviceToHost));
  if (host_ediag)
    ED_TRY_CUDA(cudaMemcpy(host_ediag, t.ediag, t.dim * 8, cudaMemcpyDeviceToHost));
  if (host_imask) ED_TRY_CUDA(cudaMemcpy(host_imask, t.imask, t.dim, cudaMemcpyDeviceToHost));
  return ED_OK;
}

extern "C" ed_status ed_sector_copy_w(ed_sector s, double *host_w) {
  if (!s || !host_w) return ED_ERR_ARG;
  int nm = 1 << s->mp.norb;
  ED_TRY_CUDA(cudaMemcpy(host_w, s->W, nm * nm * 8, cudaMemcpyDeviceToHost));
  return ED_OK;
}

extern "C" ed_status ed_sector_free(ed_sector s) {
  if (!s) return ED_ERR_ARG;
  // the caller's streams are not known here: wait for all work of the
  // device, then release on this thread's private stream
  ed_status ps = ED_OK;
  cudaStream_t cs = ed_private_stream(&ps);
  cudaError_t e = cudaDeviceSynchronize();
  sector_destroy(s, cs);
  if (ps != ED_OK) return ps;
  if (e != cudaSuccess) {
    ed_set_cuda_error(e, "cudaDeviceSynchronize", __FILE__, __LINE__);
    return ED_ERR_CUDA;
  }
  return ED_OK;
}
