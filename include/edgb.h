/*
 * edgb.h — C ABI of the GB300 exact-diagonalisation hot path.
 *
 * The library computes, on one GPU, the Lanczos ground state and the impurity
 * Green's function of a multi-orbital Anderson impurity model in one
 * (N_up, N_dw) Fock sector, following A. Amaricci et al., "EDIpack: a parallel
 * exact diagonalization package for quantum impurity problems":
 *
 *   - the model is Eq. Ham1 with diagonal H^loc and bath h and a "normal"
 *     bath (each impurity orbital has its own Nbath levels,
 *     Ns = Norb (Nbath + 1), Sec. 2.1 and Sec. 6.4); the interaction is the
 *     density-density part (U, U', U' - J) plus, when J_X or J_P != 0, the
 *     spin exchange and pair hopping H_nd;
 *   - the sector basis is the product of two ascending lists of Ns-bit strings
 *     with N_up and N_dw set bits (Sec. 2.3, Sec. 6.3);
 *   - the sector Hamiltonian has the split H = H_d + H_up x 1 + 1 x H_dw of
 *     Eq. Hdecomp with the matrix elements of Eq. Hbuild (Sec. 2.4);
 *   - the product w = H v is the serial form of Sec. 6.7 (diagonal, up part
 *     along contiguous rows, down part along the strided axis, Sec. 3.2),
 *     plus H_nd v over the whole sector when J_X or J_P != 0 (Sec. 3.2);
 *   - the ground state comes from plain Lanczos without re-orthogonalisation
 *     (Sec. 6.6); G(i w_n) from Lanczos chains and continued fractions
 *     (Sec. 6.8, Eq. KLgf).
 *
 * Conventions (fixed by this header; the paper is 1-based):
 *   - level a of a spin string is bit a.  Impurity orbital alpha is level
 *     alpha (alpha < Norb); bath level nu of orbital alpha is level
 *     Norb + alpha*Nbath + nu.
 *   - sector index i = i_up + i_dw * D_up (0-based Eq. SectorIndxDecomp): a
 *     sector vector is a row-major [D_dw][D_up] array (Eq. Vmatrix).
 *   - fermionic signs use the mode order 1up..Ns up, 1dw..Ns dw (Sec. 2.3).
 *   - spin index 0 = up, 1 = down.
 *
 * Memory and errors:
 *   - every call returns an ed_status; nothing aborts or throws across the ABI.
 *   - pointers named d_* are DEVICE pointers owned by the caller; host_* are
 *     host pointers owned by the caller.  Model arrays are copied at the call.
 *   - handles (ed_sector, ed_server) are owned by the library and released by
 *     the matching *_free / *_destroy call.
 *   - stream arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream).  Calls that return host results synchronise the
 *     stream before returning; ed_matvec is asynchronous.
 *   - a CUDA error is reported as ED_ERR_CUDA and its text is available from
 *     ed_last_error(); the device context stays usable unless the CUDA error
 *     itself is sticky.
 */
#ifndef EDGB_H
#define EDGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EDGB_VERSION_MAJOR 1
#define EDGB_VERSION_MINOR 0

/* Largest supported values (strings are 32-bit; tables sized statically). */
#define ED_MAX_NS 24
#define ED_MAX_NORB 5
#define ED_MAX_LANCZOS 1024

typedef enum {
  ED_OK = 0,
  ED_PENDING = 1,            /* ed_poll: request not finished yet            */
  ED_ERR_ARG = -1,           /* invalid argument (NULL, out of range, size)  */
  ED_ERR_UNSUPPORTED = -2,   /* Ns or Norb above the limits                  */
  ED_ERR_OOM = -3,           /* device allocation failed                     */
  ED_ERR_CUDA = -4,          /* a CUDA runtime call failed                   */
  ED_ERR_TIMEOUT = -5,       /* a bounded wait ran out                       */
  ED_ERR_NOT_CONVERGED = -6, /* Lanczos reached max_iter before tolerance    */
  ED_ERR_BUSY = -7,          /* server queue full                            */
  ED_ERR_NOT_FOUND = -8      /* unknown ticket                               */
} ed_status;

typedef enum {
  ED_FP64 = 0,        /* FP64 vectors, matrix elements and accumulation          */
  ED_FP32 = 1,        /* FP32 vectors and elements, FP32 row sums, FP64 scalars  */
  ED_FP32_POLISH = 2  /* ED_FP32 Lanczos, then FP64 Lanczos steps from the FP32
                         ground state (energy and vector reported in FP64)       */
} ed_precision;

/* Model parameters of Eq. Ham1 (host arrays, copied). */
typedef struct {
  int32_t norb;            /* impurity orbitals, 1..ED_MAX_NORB              */
  int32_t nbath;           /* bath levels per orbital, >= 0                  */
  double U;                /* intra-orbital U                                */
  double Ust;              /* inter-orbital opposite-spin U'                 */
  double Jh;               /* Hund J: same-spin inter-orbital term is U'-J   */
  double Jx, Jp;           /* spin exchange J_X, pair hopping J_P: the terms
                              -J_X d+_{a up} d_{a dw} d+_{b dw} d_{b up} and
                              +J_P d+_{a up} d+_{a dw} d_{b dw} d_{b up},
                              a != b impurity orbitals (0: term absent)      */
  const double *e_imp;     /* [2][norb]        impurity levels (H^loc diag)  */
  const double *e_bath;    /* [2][norb][nbath] bath energies                 */
  const double *v_bath;    /* [2][norb][nbath] hybridisations V^nu_{alpha s} */
} ed_model;

typedef struct ed_sector_s *ed_sector;

typedef struct {
  int32_t ns, norb, nbath, nup, ndw;
  int64_t dim_up, dim_dw, dim;     /* D_up, D_dw, D = D_up * D_dw           */
  int64_t nnz_up, nnz_dw;          /* stored entries of H_up and H_dw        */
  int64_t device_bytes;            /* device memory held by the handle       */
  int64_t blocked_stride;          /* row length of block-major vectors      */
  int64_t blocked_dim;             /* D_dw * blocked_stride                  */
} ed_sector_info;

/* Sector set-up (Sec. 6.3 build_sector, Sec. 2.4 / Eq. Hbuild): enumerates
 * both spin bases on the device (ascending Ns-bit strings with N_sigma set
 * bits, ranked by the combinatorial number system, which gives the same
 * order as the paper's scan + binary search), and builds the per-spin CSR
 * hopping matrices (columns sorted, FP64 and FP32 values) and the diagonal
 * tables: E_sigma[i] (one-body energies + (U'-J) same-spin pairs) and
 * W[m_up][m_dw] (U and U' terms over impurity occupation masks).  With
 * J_X or J_P != 0 it also tabulates, per spin and vector layout, the string
 * reached by moving one electron between two impurity orbitals (its index
 * and the sign of the move), Norb^2 int32 entries per string: the product
 * then adds H_nd v with one gather kernel (every entry point that applies H,
 * the GF chains and the interaction energy of ed_observables included).
 * Returns ED_ERR_ARG for nup/ndw outside 0..Ns, ED_ERR_UNSUPPORTED for
 * Norb > ED_MAX_NORB or Ns > ED_MAX_NS.  Synchronises `stream`. */
ed_status ed_sector_build(const ed_model *model, int32_t nup, int32_t ndw,
                          void *stream, ed_sector *out);
ed_status ed_sector_get_info(ed_sector s, ed_sector_info *out);
/* Test hook: copies spin `spin`'s tables to host arrays (each may be NULL):
 * map[D_s] (uint32 strings, sector order), rowptr[D_s+1], col[nnz], val[nnz]
 * (FP64), ediag[D_s] (FP64 E_sigma), imask[D_s] (impurity bits).  The W table
 * ([2^norb][2^norb] FP64) is copied by ed_sector_copy_w. */
ed_status ed_sector_copy_tables(ed_sector s, int32_t spin, uint32_t *host_map,
                                int32_t *host_rowptr, int32_t *host_col,
                                double *host_val, double *host_ediag,
                                uint8_t *host_imask);
ed_status ed_sector_copy_w(ed_sector s, double *host_w);
ed_status ed_sector_free(ed_sector s);

/* w = H v on the sector (Sec. 6.7 without MPI; Eq. Hbuild):
 *   w[r,c] = (E_up[c] + E_dw[r] + W[m_up[c]][m_dw[r]]) v[r,c]
 *          + sum_k H_up[c,k] v[r,k] + sum_k H_dw[r,k] v[k,c].
 * d_v, d_w: device arrays of n = D elements, double for ED_FP64, float for
 * ED_FP32 / ED_FP32_POLISH; must not overlap.  ED_ERR_ARG when n != D.
 * Asynchronous on `stream`. */
ed_status ed_matvec(ed_sector s, ed_precision prec, const void *d_v, void *d_w, int64_t n,
                    void *stream);

/* Block-major layout.  With a diagonal H^loc, a normal bath and the
 * density-density interaction, each orbital group (impurity level alpha and
 * its bath levels) conserves its number of spin-s electrons (the per-orbital
 * quantum numbers of Sec. 2.2; H_sigma is a Kronecker sum over orbitals,
 * Sec. 2.4).  In block-major order the states of each spin are grouped by
 * the tuple of group occupations (tuples in lexicographic order; inside a
 * block the mixed-radix index of the group strings, group 0 slowest, each
 * group string in colex order), so H maps every (dw block, up block)
 * rectangle of the [D_dw][D_up] array to itself.  The library's Lanczos
 * vectors live in this order; inputs and outputs of the calls below that
 * say "sector order" are converted at the boundary.
 *
 * Block-major vectors are [D_dw][blocked_stride] arrays: every up block is
 * padded to a multiple of 4 columns (16-byte aligned row segments) and the
 * padding entries are zero (ed_sector_info gives blocked_stride and
 * blocked_dim = D_dw * blocked_stride).
 *
 * ed_matvec_blocked: w = H v with v, w block-major vectors of
 * n = blocked_dim elements (same element types as ed_matvec), both 16-byte
 * aligned (ED_ERR_ARG otherwise); the padding of w is not written.  ed_sector_permute: converts between a sector-order
 * D-vector and a block-major vector (to_blocked = 1: sector -> blocked,
 * padding written as zero); n_in / n_out are the element counts of the two
 * arrays; d_in and d_out must not overlap.  Both return ED_ERR_ARG when a
 * count does not match the layout, and are asynchronous. */
ed_status ed_matvec_blocked(ed_sector s, ed_precision prec, const void *d_v, void *d_w,
                            int64_t n, void *stream);

/* Which product kernel serves the block-major layout of s in precision prec
 * (builds the block-major work tables if they do not exist yet; synchronous):
 *   ED_KERNEL_TILED       rows of a work item staged in shared memory, H_up
 *                         from an ELL table, H_dw from neighbour rows;
 *   ED_KERNEL_ELEMENTWISE one thread per vector element (small sectors; the
 *                         autotuner below decides between it and the tiled
 *                         kernel);
 *   ED_KERNEL_TWO_PASS    the tiled kernel without H_dw, then an H_dw pass over
 *                         column chunks (sectors whose largest dw block x up
 *                         block slice of a vector exceeds 160 MiB: the
 *                         neighbour rows of one pass would not stay in L2).
 * The result is the same w = H v bit for bit whichever kernel runs.
 * ED_ERR_ARG for a null handle or output or an unknown precision. */
#define ED_KERNEL_TILED 0
#define ED_KERNEL_ELEMENTWISE 1
#define ED_KERNEL_TWO_PASS 2
ed_status ed_sector_blocked_kernel(ed_sector s, ed_precision prec, int32_t *kernel);

/* Autotuner (no counterpart in the paper).  Sectors of at most 2^17 padded
 * elements use the element-parallel kernel; above that the first sector of
 * each model shape (Norb, Nbath, precision) times the tiled family and
 * the element-parallel kernel (one warm-up and three launches each, on two
 * scratch vectors of the sector's size) when its block-major tables are
 * built, and every sector of that shape in the process then uses the faster
 * one.
 * ed_sector_tune_info returns the kernel in use and host_ms[0..1], the
 * measured milliseconds of the tiled and the element-parallel product
 * (-1 where this sector did not time them).  ed_sector_set_kernel pins a
 * kernel for one sector and precision: ED_KERNEL_ELEMENTWISE or the tiled
 * family (ED_KERNEL_TILED, or
 * ED_KERNEL_TWO_PASS where the block sizes call for two passes); other
 * requests give ED_ERR_UNSUPPORTED.  All kernels compute the same w = H v bit
 * for bit; Lanczos runs differ only in the summation order of <v, w>. */
ed_status ed_sector_tune_info(ed_sector s, ed_precision prec, int32_t *kernel, double *host_ms);
ed_status ed_sector_set_kernel(ed_sector s, ed_precision prec, int32_t kernel);
ed_status ed_sector_permute(ed_sector s, ed_precision prec, int32_t to_blocked,
                            const void *d_in, int64_t n_in, void *d_out, int64_t n_out,
                            void *stream);

typedef struct {
  ed_precision precision;
  int32_t max_iter;      /* first-pass Lanczos steps, <= ED_MAX_LANCZOS (0: 512) */
  double tol;            /* stop when beta_{k+1}|y_k| <= tol*max(1,|theta|)      */
                         /* (0: 1e-12 for FP64, 1e-6 for the FP32 modes)         */
  uint64_t seed;         /* start vector: v0_i = u_i - 1/2, u_i = SplitMix64(seed)
                            output i, sector order, then normalised               */
  int32_t polish_steps;  /* FP64 Lanczos steps of ED_FP32_POLISH (0: 4)          */
  int32_t want_vector;   /* 1: psi and its FP64 residual                         */
  int32_t basis_mib;     /* Krylov basis kept on the device during the first
                            pass, so that psi needs no second pass (or one
                            resumed after the stored vectors): 0 = up to 60%
                            of the available device memory, > 0 = at most this
                            many MiB, -1 = none (always the second pass)      */
  int32_t reserved;      /* 0                                                    */
} ed_lanczos_opts;

typedef struct {
  double e0;                /* reported ground energy                          */
  double e0_raw;            /* lowest Ritz value of the first (FP32/FP64) pass */
  double residual;          /* ||H psi - e0 psi|| / ||psi|| in FP64 (vector)   */
  double residual_estimate; /* beta_{k+1}|y_k| of the first pass               */
  int32_t iterations;       /* first-pass steps k                              */
  int32_t polish_iterations;
  int32_t stop_reason;      /* 0 converged, 1 breakdown, 2 max_iter            */
  int32_t matvecs;          /* total products performed                        */
  int32_t matvecs_fp64;     /* of which in FP64 (all of them for ED_FP64; the
                               polish steps and residual products otherwise)   */
  int32_t reserved;         /* 0                                               */
} ed_lanczos_result;

/* Lanczos ground state of the sector (Sec. 6.6): plain Lanczos, Paige form,
 * no re-orthogonalisation; lowest eigenpair of the tridiagonal matrix by
 * Sturm multisection (FP64); psi = sum_j y_j v_j from the Krylov basis kept
 * during the first pass when it fits the basis_mib budget, else from the
 * paper's second pass (the same recurrence run again); both give the same
 * psi, bit for bit.
 * d_psi (nullable, requires want_vector) receives psi, normalised, in
 * sector order: double for ED_FP64 / ED_FP32_POLISH, float for ED_FP32.
 * Work vectors are allocated stream-ordered on the device and released
 * before return.  Synchronises `stream`.  Returns ED_ERR_NOT_CONVERGED (with
 * `res` filled) when max_iter is reached before the tolerance. */
ed_status ed_lanczos_ground(ed_sector s, const ed_lanczos_opts *opts,
                            ed_lanczos_result *res, void *d_psi, void *stream);

typedef struct {
  double weight_particle;  /* ||c^+ psi||^2                                    */
  double weight_hole;      /* ||c psi||^2                                      */
  int32_t steps_particle;  /* chain lengths actually used (breakdown stops)    */
  int32_t steps_hole;
} ed_gf_info;

/* Impurity Green's function G_{orb,spin}(i w_n), w_n = (2n+1) pi / beta,
 * n = 0..nmats-1, at T = 0 (Sec. 6.8, Eq. KLgf with "+" for fermions):
 *   G = n+ [(z - T+)^-1]_00 at z = e0 + i w_n  -  n- [(z - T-)^-1]_00 at
 *   z = e0 - i w_n,
 * where T+- are the tridiagonal matrices of `nsteps`-step Lanczos chains
 * started from c^+_{orb,spin} psi and c_{orb,spin} psi and n+- their squared
 * norms.  d_psi is the normalised ground state of `s` in sector order
 * (double for ED_FP64 / ED_FP32_POLISH, float for ED_FP32); chains run in
 * the precision `prec` (ED_FP32_POLISH runs them in FP32).  The N+-1 sectors
 * are built on first use and cached in `s`.  host_G receives 2*nmats doubles
 * (re, im interleaved).  Synchronises `stream`. */
ed_status ed_gf_lanczos(ed_sector s, ed_precision prec, const void *d_psi, double e0,
                        int32_t orb, int32_t spin, int32_t nsteps, double beta,
                        int32_t nmats, double *host_G, ed_gf_info *info,
                        void *stream);

/* The same Green's function at arbitrary complex frequencies z_n (Sec. 6.8,
 * Eq. KLgf; App. B for the real axis): host_z holds nz complex values (re, im
 * interleaved) and host_G receives 2*nz doubles,
 *   G(z) = n+ [(e0 + z - T+)^-1]_00 - n- [(e0 - z - T-)^-1]_00,
 * so z = i w_n gives the Matsubara function of ed_gf_lanczos and z = w + i eta
 * (eta > 0) the retarded function on the real axis.  Arguments otherwise as
 * ed_gf_lanczos.  Synchronises `stream`. */
ed_status ed_gf_lanczos_z(ed_sector s, ed_precision prec, const void *d_psi, double e0,
                          int32_t orb, int32_t spin, int32_t nsteps, const double *host_z,
                          int32_t nz, double *host_G, ed_gf_info *info, void *stream);

/* Impurity self-energy by the Dyson equation (Sec. 6.8, App. B):
 *   Sigma(z) = G0(z)^-1 - G(z)^-1,
 *   G0_{orb,spin}(z)^-1 = z - e_imp[spin][orb]
 *                         - sum_nu v_bath[spin][orb][nu]^2 / (z - e_bath[spin][orb][nu])
 * (the non-interacting impurity function of the normal bath of `model`).
 * host_z and host_G: nz complex values each (re, im interleaved), host_sigma
 * receives 2*nz doubles; all host arrays owned by the caller.  ED_ERR_ARG for
 * a null pointer, nz < 0 or orb / spin out of range.  Synchronises `stream`. */
ed_status ed_sigma(const ed_model *model, int32_t orb, int32_t spin, const double *host_z,
                   int32_t nz, const double *host_G, double *host_sigma, void *stream);

/* Local observables of a sector-order state psi of n = D elements (device;
 * double for ED_FP64 / ED_FP32_POLISH, float for ED_FP32), normalised by the
 * call (App. B: densities and double occupancies of the impurity).
 * host_out receives 2*norb + 4*norb*norb + 2 doubles:
 *   dens[s][a]        <n_{a s}>                          (2*norb)
 *   nn[s][t][a][b]    <n_{a s} n_{b t}>                  (4*norb*norb; the
 *                     double occupancy of orbital a is nn[0][1][a][a])
 *   e_int             <H_int> = U sum_a nn[0][1][a][a] + U' sum_{a!=b} nn[0][1][a][b]
 *                     + (U' - J) sum_{a<b} (nn[0][0][a][b] + nn[1][1][a][b])
 *                     + <psi|H_nd|psi> / <psi, psi> (spin exchange and pair
 *                     hopping; summed in FP32 for ED_FP32 vectors)
 *   norm              <psi, psi> before normalisation.
 * ED_ERR_ARG when n != D.  Synchronises `stream`. */
ed_status ed_observables(ed_sector s, ed_precision prec, const void *d_psi, int64_t n,
                         double *host_out, void *stream);

/* Per-orbital sectors (Sec. 2.2, N_ud = Norb): with J_X = J_P = 0, a diagonal
 * H^loc and a normal bath the electron number of every orbital group (the
 * impurity level and its bath levels) is conserved per spin, and S[N_up,
 * N_dw] splits into finer sectors labelled by the per-orbital occupations
 * nup_orb[alpha], ndw_orb[alpha] (sums N_up, N_dw).  ed_orbital_sector_dims
 * gives the finer sector's D_up, D_dw (ED_ERR_ARG when no state of s has
 * those occupations).  ed_lanczos_ground_orbital finds its ground state: the
 * product kernels run over that block pair's work items only, on vectors of
 * the finer sector alone, through the operator-generic Lanczos driver
 * (options and result as ed_lanczos_ground); d_psi (nullable) receives psi
 * as a sector-order vector of s (D elements, zero outside the finer
 * sector).  ED_ERR_UNSUPPORTED when J_X or J_P != 0. */
ed_status ed_orbital_sector_dims(ed_sector s, const int32_t *nup_orb, const int32_t *ndw_orb,
                                 int64_t *dim_up, int64_t *dim_dw);
ed_status ed_lanczos_ground_orbital(ed_sector s, const int32_t *nup_orb, const int32_t *ndw_orb,
                                    const ed_lanczos_opts *opts, ed_lanczos_result *res,
                                    void *d_psi, void *stream);

/* Impurity susceptibility at T = 0 (Sec. 6.8: Eq. KLgf with the bosonic sign),
 *   C_O(z) = <O (z - (H - E0))^-1 O^+> - <O^+ (z + (H - E0))^-1 O>
 *          = n+ [(e0 + z - T+)^-1]_00 + n- [(e0 - z - T-)^-1]_00,
 * T+- the tridiagonal matrices of `nsteps`-step chains started from O^+ psi
 * and O psi, n+- their squared norms.  kind: ED_CHI_SPIN, O = S^z_orb =
 * (n_{orb up} - n_{orb dw})/2, and ED_CHI_CHARGE, O = n_orb, both as the
 * connected O - <O> (one chain serves both terms); ED_CHI_PAIR, O =
 * d_{orb dw} d_{orb up} (chains on the (N_up+1, N_dw+1) and (N_up-1, N_dw-1)
 * sectors).  d_psi, prec, host_z / host_C (nz complex values each) as for
 * ed_gf_lanczos_z; host_w (nullable) receives n+ and n-.  Synchronises
 * `stream`. */
enum { ED_CHI_SPIN = 0, ED_CHI_CHARGE = 1, ED_CHI_PAIR = 2, ED_CHI_EXCITON = 3 };
ed_status ed_chi_z(ed_sector s, ed_precision prec, const void *d_psi, double e0, int32_t kind,
                   int32_t orb, int32_t nsteps, const double *host_z, int32_t nz, double *host_C,
                   double *host_w, void *stream);

/* Susceptibility in imaginary time at T = 0 (Sec. 6.8 evaluates the
 * susceptibilities on the imaginary-time axis as well): for tau in [0, beta],
 *   C(tau) = n+ sum_m w+_m exp(-tau (E+_m - e0))
 *          + n- sum_m w-_m exp(-(beta - tau)(E-_m - e0)),
 * from the two chains of ed_chi_z (the O^+ psi chain decays over tau, the
 * O psi chain over beta - tau), E_m and w_m the eigenvalues of each chain's
 * tridiagonal matrix and the squared first components of its eigenvectors
 * (computed on the host by Jacobi rotations, at most ED_MAX_LANCZOS
 * steps).  Its bosonic Fourier transform is -C(i nu_n) of ed_chi_z up to
 * exp(-beta (E_m - e0)) terms; for spin and charge C(tau) = C(beta - tau).
 * kind, orb, prec, nsteps as ed_chi_z; host_tau: ntau times in [0, beta]
 * (ED_ERR_ARG otherwise, or for beta <= 0); host_C receives ntau doubles.
 * Synchronises `stream`. */
ed_status ed_chi_tau(ed_sector s, ed_precision prec, const void *d_psi, double e0, int32_t kind,
                     int32_t orb, int32_t nsteps, double beta, const double *host_tau,
                     int32_t ntau, double *host_C, void *stream);

/* Inter-orbital spin or charge function (Sec. 6.8, the auxiliary-operator
 * construction of non-diagonal correlation functions):
 *   C_ab(z) = <A (z - (H - E0))^-1 B> - <B (z + (H - E0))^-1 A>,
 * A = O_a - <O_a>, B = O_b - <O_b>, O the ED_CHI_SPIN or ED_CHI_CHARGE
 * operator of one orbital, from the chains of O_a + O_b, O_a and O_b:
 * C_ab = [C(O_a + O_b) - C_aa - C_bb] / 2 (for these real operators and a
 * real symmetric H, C_ab = C_ba, so the paper's second auxiliary operator
 * A - iB is not needed); orb_a = orb_b gives ed_chi_z's C_aa.
 * kind = ED_CHI_EXCITON: the excitonic function of the orbital pair
 * (orb_a != orb_b), C_O with O = sum_sigma (c^+_{a sigma} c_{b sigma} +
 * c^+_{b sigma} c_{a sigma}) (the singlet inter-orbital particle-hole
 * operator, hermitian, same sector) as its connected O - <O>, from one chain
 * as for spin and charge.  Arguments, precisions and outputs as ed_chi_z (no
 * weights); ED_ERR_ARG for ED_CHI_PAIR, an orbital out of range or an
 * excitonic pair with orb_a = orb_b.  Synchronises `stream`. */
ed_status ed_chi_ab_z(ed_sector s, ed_precision prec, const void *d_psi, double e0, int32_t kind,
                      int32_t orb_a, int32_t orb_b, int32_t nsteps, const double *host_z,
                      int32_t nz, double *host_C, void *stream);

/* ---------------------------------------------------------------- several states, finite T
 * The nstates lowest eigenpairs of the sector (the states of the eigenspace
 * list, Sec. 6.2; the paper takes them from P-ARPACK, Sec. 5): Lanczos on
 * the block-major vectors, state k found as the lowest eigenpair of
 *   H + sigma sum_{j<k} |psi_j><psi_j|
 * (shift deflation: the states already found are moved above the top of the
 * spectrum; sigma = 1.05 (theta_max - E_0) + 1e-6, theta_max the highest Ritz
 * value of the first run), each with the stopping rule and the second pass
 * of ed_lanczos_ground; ED_FP32_POLISH runs every state in FP32, then
 * polish_steps FP64 steps on the FP64 deflated operator.  host_e receives the
 * nstates energies in the order found (ascending up to the tolerance), res
 * (nullable) nstates results (residuals of the undeflated H), d_psis
 * (nullable) nstates consecutive normalised vectors of D elements in sector
 * order (double for ED_FP64 / ED_FP32_POLISH, float for ED_FP32).
 * ED_ERR_ARG unless 1 <= nstates <= min(D, ED_MAX_STATES).  Synchronises
 * `stream`. */
#define ED_MAX_STATES 256
ed_status ed_lanczos_states(ed_sector s, const ed_lanczos_opts *opts, int32_t nstates,
                            double *host_e, ed_lanczos_result *res, void *d_psis, void *stream);

/* Annealing truncation of the eigenspace list (Sec. 6.2; host only).  The
 * states of nsectors sectors, counts[q] of sector q with their energies
 * ascending and consecutive in `energies`: E0 the lowest; a state is kept when
 * e^{-beta (E - E0)} >= cutoff (the paper's "<" read as the condition for
 * dropping it), lowest first, at most ntotal states; weights (one per state,
 * 0 for a dropped one) = e^{-beta (E - E0)} / Z over the kept states.
 * next_counts[q]: counts[q] + step when the highest computed state of sector
 * q was kept (the sector may hold more states under the threshold), else one
 * more than the sector kept.  *nkept receives the kept count. */
ed_status ed_espace_truncate(int32_t nsectors, const int32_t *counts, const double *energies,
                             double beta, double cutoff, int32_t ntotal, int32_t step,
                             double *weights, int32_t *next_counts, int32_t *nkept);

/* Finite-temperature Green's function (App. A: the thermal average over the
 * eigenstates of Eq. KLgf): G(z) = sum_i w_i G_i(z), G_i the
 * ed_gf_lanczos_z function of state i (sector sectors[i], normalised vector
 * d_psis[i] in sector order, energy energies[i]) and w_i the weights of
 * ed_espace_truncate over the nstates states (one list).  host_w (nullable)
 * receives the weights; dropped states run no chains.  Other arguments as
 * ed_gf_lanczos_z.  Synchronises `stream`. */
ed_status ed_gf_thermal_z(int32_t nstates, const ed_sector *sectors, const void *const *d_psis,
                          const double *energies, double beta, double cutoff, int32_t ntotal,
                          ed_precision prec, int32_t orb, int32_t spin, int32_t nsteps,
                          const double *host_z, int32_t nz, double *host_G, double *host_w,
                          void *stream);

/* ---------------------------------------------------------------- electron-phonon
 * One local phonon mode coupled to the impurity densities (Sec. 4):
 *   H = H_e + w0 b^+ b + sum_{alpha sigma} g_alpha d^+_{alpha sigma} d_{alpha sigma} (b + b^+),
 * phonon number cut off at nph (states |0>..|nph>, D_ph = nph + 1).  A
 * coupled sector is an electronic sector times the phonon space, phonon
 * index slowest (Eq. Vdecomp2): element i_e + p * D of a vector of
 * D * D_ph elements, i_e the electronic sector index; its matrix is
 * Eq. HephBuild, 1 (x) H_e + H_ph (x) 1 + (b + b^+) (x) N_g with
 * N_g = sum_alpha g_alpha (n_{alpha up} + n_{alpha dw}). */
typedef struct {
  double w0;               /* phonon frequency                               */
  double g[ED_MAX_NORB];   /* coupling g_alpha of orbital alpha (unused: 0)  */
  int32_t nph;             /* phonon cut-off N_ph, 0..ED_MAX_NPH             */
  int32_t reserved;        /* 0                                              */
} ed_phonon;
#define ED_MAX_NPH 4095

/* w = H v on the coupled sector of s (Eq. HephBuild): the electronic product
 * of ed_matvec on every phonon slice, then the phonon terms
 * w[p] += w0 p v[p] + N_g (sqrt(p) v[p-1] + sqrt(p+1) v[p+1]) in one pass over
 * the slices.  v, w: device, n = D * (nph + 1) elements in the precision's
 * type, distinct.  ED_ERR_ARG for a bad size, pointer or phonon record. */
ed_status ed_eph_matvec(ed_sector s, const ed_phonon *ph, ed_precision prec, const void *d_v,
                        void *d_w, int64_t n, void *stream);

/* Lanczos ground state of the coupled sector (Sec. 4 with Sec. 6.6): plain
 * Lanczos on the device (the vectors in padded block-major slices), the
 * stopping rule of ed_lanczos_ground checked every 4 steps, psi from the
 * second pass.  ED_FP32_POLISH runs `polish_steps` FP64 steps from the FP32
 * vector.  d_psi (nullable) receives psi in coupled sector order (double for
 * ED_FP64 / ED_FP32_POLISH, float for ED_FP32).  Fields of ed_lanczos_opts as
 * for ed_lanczos_ground (basis_mib unused: always the second pass).
 * Synchronises `stream`. */
ed_status ed_eph_lanczos_ground(ed_sector s, const ed_phonon *ph, const ed_lanczos_opts *opts,
                                ed_lanczos_result *res, void *d_psi, void *stream);

/* G(z) of the coupled model at T = 0 (Eq. KLgf with the coupled H): chains
 * started from c^+ psi and c psi, c acting on every phonon slice, on the
 * coupled N+-1 sectors; arguments and output as ed_gf_lanczos_z, d_psi in
 * coupled sector order. */
ed_status ed_eph_gf_lanczos_z(ed_sector s, const ed_phonon *ph, ed_precision prec,
                              const void *d_psi, double e0, int32_t orb, int32_t spin,
                              int32_t nsteps, const double *host_z, int32_t nz, double *host_G,
                              ed_gf_info *info, void *stream);

/* One impurity solve: sector build, ground state, and G for every orbital and
 * both spins (the down spin is copied from the up spin when N_up = N_dw and
 * the model is spin symmetric, Sec. 6.6 twin symmetry).  The particle and
 * hole chains of all orbitals run concurrently, each on its own stream.  host_G receives
 * [2][norb][nmats] complex values as 2*2*norb*nmats doubles (may be NULL when
 * nmats == 0). */
typedef struct {
  ed_lanczos_opts lanczos;
  int32_t gf_steps;      /* lanc_ngfiter (0: 200)  */
  int32_t nmats;         /* Matsubara points (>= 0) */
  double beta;           /* inverse temperature setting the grid */
  ed_precision gf_precision;
} ed_solve_opts;

typedef struct {
  ed_lanczos_result ground;
  double t_build_s, t_ground_s, t_gf_s;  /* wall time of each phase */
  int32_t gf_chains;         /* Lanczos chains run for G                   */
  int32_t gf_steps_total;    /* products of all chains                     */
  double gf_product_bytes;   /* algorithmic bytes of those products
                                (read v + write w per product)              */
} ed_solve_result;

/* d_psi (nullable, device): receives the normalised ground state in sector
 * order, D elements, double unless the ground precision is ED_FP32 (float). */
ed_status ed_solve(const ed_model *model, int32_t nup, int32_t ndw,
                   const ed_solve_opts *opts, ed_solve_result *res,
                   double *host_G, void *d_psi, void *stream);

/* ---------------------------------------------------------------- serving
 * A request loop on a host thread: requests are admitted while their
 * estimated device memory fits the budget and a slot is free, run
 * concurrently on a pool of CUDA streams (continuous batching: a request
 * that arrives while others run starts as soon as a slot and memory free
 * up), and their results are kept until polled.  Results are bit-identical
 * to ed_solve with the same request (deterministic reductions). */
typedef struct ed_server_s *ed_server;

typedef struct {
  int32_t slots;               /* concurrent solves (streams), 0: 8           */
  int64_t device_mem_budget;   /* bytes for admitted solves, 0: 50% of free   */
  int32_t queue_capacity;      /* pending requests, 0: 65536                  */
} ed_server_opts;

typedef struct {
  ed_model model;              /* arrays copied at submit                    */
  int32_t nup, ndw;
  ed_solve_opts opts;
} ed_request;

typedef struct {
  ed_status status;            /* status of the solve                        */
  double e0;
  ed_lanczos_result ground;
  int32_t norb, nmats;
  double t_submit_s, t_start_s, t_done_s;  /* server clock (seconds)         */
} ed_result;

ed_status ed_server_create(const ed_server_opts *opts, ed_server *out);
/* Copies the request; returns ED_ERR_BUSY when the queue is full and
 * ED_ERR_OOM when the request alone exceeds the memory budget. */
ed_status ed_submit(ed_server srv, const ed_request *req, uint64_t *ticket);
/* Never blocks.  ED_PENDING while the request runs; otherwise fills `out`
 * and, when host_G is not NULL, copies G ([2][norb][nmats] complex) and
 * forgets the ticket. */
ed_status ed_poll(ed_server srv, uint64_t ticket, ed_result *out, double *host_G);
/* Blocks up to timeout_s seconds for the request; ED_ERR_TIMEOUT otherwise. */
ed_status ed_wait(ed_server srv, uint64_t ticket, double timeout_s);
ed_status ed_server_destroy(ed_server srv);
/* Batched Green's-function launches of this process (no counterpart in the
 * paper; the task parallelism over independent impurity problems of Sec. 6.9
 * on one GPU).  The chains of solves whose N+-1 sectors are small (at most
 * 2^14 states) run in one persistent launch, one CTA per chain; solves that
 * reach that phase at about the same time -- concurrent server requests,
 * or several host threads calling ed_solve -- share one launch (the first
 * one leads and waits at most 1 ms for the others).  A chain's result does
 * not depend on the chains it shares a launch with.  Returns the number of
 * such launches, of chains run in them, and the largest number of solves
 * merged into one launch. */
ed_status ed_batch_stats(int64_t *launches, int64_t *chains, int64_t *max_solves);
/* Test hook: the next `count` admissions fail as if the device allocation
 * had failed (the request completes with ED_ERR_OOM). */
ed_status ed_server_inject_alloc_failure(ed_server srv, int32_t count);

/* ---------------------------------------------------------------- no allocation
 * Residual check that allocates nothing (the paper has no counterpart: this
 * is a service of this library).  It is meant for callers that cannot let a
 * library allocate device memory: applications that hand all device memory
 * to their own pool or arena allocator up front (a cudaMalloc by the library
 * would then fail or fragment their pool), and latency-critical loops in
 * which cudaMalloc/cudaFree could block (cudaFree synchronises the device).
 * For a caller's vector psi of n = D elements in sector order (double,
 * device memory) it computes
 *   host_e_r[0] = <psi, H psi> / <psi, psi>,
 *   host_e_r[1] = ||H psi - host_e_r[0] psi|| / ||psi||,
 * enqueued on `stream`, then copies the two words to the host and
 * synchronises `stream` before returning.
 * It calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * (H psi, partial sums, result words) is a file-scope device array of
 * ED_NOALLOC_MAX_DIM + 2052 doubles (about 8 MiB).  Every GPU that loads the
 * library's module holding the array reserves it until the process exits;
 * under CUDA's default lazy module loading that happens on the module's first
 * use, which is this entry point's first call on the device.  D above
 * ED_NOALLOC_MAX_DIM (or n != D) returns ED_ERR_ARG.  The first call on a
 * device also looks up the array's device address (with that device
 * current): make that first call at set-up time, before any stream capture.
 * Every call overwrites the scratch words it reads before reading them, so
 * no clearing is needed; calls whose kernels overlap on the GPU (other
 * streams or threads) race on the shared array and must be serialised by
 * the caller. */
#define ED_NOALLOC_MAX_DIM (1 << 20)
ed_status ed_residual_noalloc(ed_sector s, const double *d_psi, int64_t n, double *host_e_r,
                              void *stream);

/* Device memory of the library (current device).  Every device buffer comes
 * from one stream-ordered pool per device, and freed blocks stay cached in
 * it for later allocations (the first use of fresh device memory costs about
 * 5.6 ms per GB on GB300, a large share of a solve that allocates its Krylov
 * basis as it goes).  Other allocators in the process (PyTorch's, for one)
 * cannot use the cached blocks: ed_memory_trim returns the cached blocks
 * beyond keep_bytes (>= 0; 0 returns all that are not in use) to the device,
 * as torch.cuda.empty_cache does for PyTorch.  ed_memory_cached reports the
 * pool's reserved bytes and the part of them in use by live buffers.  The
 * budgets that look at free memory (the Krylov basis of ed_lanczos_ground,
 * the admission of ed_server_create with device_mem_budget = 0) count the
 * cached blocks as available.  ED_ERR_ARG on a negative keep_bytes or a
 * NULL output. */
ed_status ed_memory_trim(int64_t keep_bytes);
ed_status ed_memory_cached(int64_t *reserved, int64_t *used);

const char *ed_status_string(ed_status st);
const char *ed_last_error(void);
/* Number of kernels this library has launched in the calling process. */
int64_t ed_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* EDGB_H */
