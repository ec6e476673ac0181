/*
 * tnt_gb300.h -- C-ABI of the GB300 (sm_103a) two-site-update library.
 *
 * The library computes the hot path of the MPS algorithms of "The Tensor Network Theory
 * Library" (arXiv:1610.02244): the effective-Hamiltonian matvec L.W.W.R.theta that the
 * eigensolver applies in DMRG (Sec. 4.2 Listing 1, Sec. 4.3 Listing 2), the two-site
 * gate of TEBD (Sec. 3, Sec. 5), and the reshape plus truncated SVD of theta that follows
 * both (App. B.1.2, Eq. 3), on Bose-Hubbard chains (Sec. 5, Eq. 2), spin-S Heisenberg
 * chains (Sec. 6) or any hand-built MPO (Sec. 4.3), with optional U(1) labels (App. A.1.1);
 * around it, the DMRG sweep (two-site, and single-site with subspace expansion), the TEBD
 * step and the observables of the paper's examples.
 *
 * Conventions for every call
 *   - Every call returns an int status (TNT_OK = 0 or a TNT_E_* code); results go through
 *     out-pointers.  After a failure tnt_last_error(ctx) describes it.
 *   - Complex numbers are interleaved {double re, im} (tnt_cplx), tensors are dense,
 *     row-major (C order), with the leg orders below.  Sizes are int64_t.
 *       MPS site tensor   A[a, s, b]           (left bond, physical, right bond)
 *       two-site tensor   theta[a, s1, s2, b]
 *       MPO tensor        W[w, w', s', s]      (s' out/bra, s in/ket)
 *       left environment  L[a', w, a]          (a' bra side, a ket side)
 *       right environment R[b', w, b]
 *   - Pointers named d_* are DEVICE pointers (CUDA global memory on the context's device);
 *     they are borrowed for the duration of the call, never freed or retained.  Pointers
 *     named h_* are HOST pointers, copied during the call.
 *   - Work is enqueued on the context's stream.  Calls that return host scalars
 *     synchronise that stream before returning; calls with device outputs only do not.
 *   - All computation runs on the GPU; there is no CPU fallback.  A missing or
 *     unusable GPU makes tnt_ctx_create fail with TNT_E_CUDA.
 *   - Handles (tnt_ctx, tnt_mpo, tnt_mps, tnt_dmrg) are opaque, created by the library
 *     and freed only by their *_destroy call.
 */
#ifndef TNT_GB300_H
#define TNT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Everything declared here is exported from the shared library; nothing else is. */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

/* ------------------------------------------------------------------ status codes */
enum {
  TNT_OK = 0,
  TNT_E_INVALID = 1,     /* bad argument (null pointer, non-positive size, bad enum)   */
  TNT_E_ALLOC = 2,       /* device or pinned host allocation failed                     */
  TNT_E_CUDA = 3,        /* a CUDA runtime/driver call or kernel launch failed          */
  TNT_E_NOCONV = 4,      /* an iterative solver hit its iteration cap unconverged       */
  TNT_E_TIMEOUT = 5,     /* a bounded device-side wait gave up                          */
  TNT_E_BOUNDS = 6,      /* a device-side index check failed                            */
  TNT_E_NAN = 7,         /* a NaN/Inf was detected in a result                          */
  TNT_E_UNSUPPORTED = 8  /* shape or mode not supported by this library                 */
};

enum { TNT_PREC_FP64 = 0, TNT_PREC_MIXED = 1 };
/* Truncation error functions of App. B.1.2: Eq. 3 (2-norm), sum of squares, 1-norm. */
enum { TNT_TRUNC_2NORM = 0, TNT_TRUNC_SUMSQ = 1, TNT_TRUNC_1NORM = 2 };
/* Which factor of M = U S V^H the truncated SVD keeps orthonormal. */
enum { TNT_SVD_LEFT = 0, TNT_SVD_RIGHT = 1 };

typedef struct { double re, im; } tnt_cplx;

typedef struct tnt_ctx tnt_ctx;
typedef struct tnt_mpo tnt_mpo;
typedef struct tnt_mps tnt_mps;
typedef struct tnt_dmrg tnt_dmrg;
typedef struct tnt_tebd tnt_tebd;

/*
 * Simulation parameters (the library's system settings, App. A.3 and App. B.5).
 * Defaults (tnt_params_default) are the printed defaults of App. A.3 Listing 5:
 * relative truncation tolerance 1e-16, absolute tolerance -1 (off), truncation error
 * tolerance 1e-8, truncation type 2norm, eigensolver iteration cap 300.
 */
typedef struct {
  int64_t chi_max;      /* bond-dimension cap (truncation rule 1)                 */
  double trunc_abs;     /* rule 2: discard lambda_i < trunc_abs; <= 0 disables      */
  double trunc_rel;     /* rule 3: discard lambda_i / lambda_0 < trunc_rel          */
  double trunc_err;     /* rule 4: largest discard with error < trunc_err           */
  int trunc_type;       /* TNT_TRUNC_*: error function of rule 4                   */
  double lanczos_tol;   /* relative eigenvalue-change and residual tolerance        */
  int lanczos_maxit;    /* total matvec cap per eigensolve                          */
  int krylov_cap;       /* Krylov vectors before a restart (<= 64)                  */
  int precision;        /* TNT_PREC_FP64 or TNT_PREC_MIXED for H_eff.theta          */
  uint64_t seed;        /* reserved for library-side random draws                  */
} tnt_params;

/* Result of one eigensolve (Lanczos on H_eff, Sec. 4.3). */
typedef struct {
  double E;             /* Ritz value of the last Krylov step                       */
  double E_rq;          /* FP64 Rayleigh quotient <x|H x>/<x|x> of the returned x    */
  double resid;         /* Lanczos residual estimate beta_k |y_k|                    */
  double resid_fp64;    /* |H x - E_rq x| with H applied in FP64                     */
  int n_matvec;         /* matvecs spent (mixed + FP64)                              */
  int converged;        /* 1 if the stopping rule was met before the cap             */
} tnt_lanczos_result;

/* Result of one truncated SVD (App. B.1.2). */
typedef struct {
  int64_t chi;          /* kept singular values                                     */
  double err;           /* truncation error (trunc_type) of the normalised discards  */
  double disc;          /* discarded weight: sum of raw discarded lambda^2           */
  double norm2;         /* sum of all lambda^2                                       */
  int n_blocks;         /* charge blocks decomposed                                  */
  int tie_at_cut;       /* 1 if lambda_chi and lambda_chi+1 agree to 1e-10 lambda_0  */
} tnt_trunc_result;

/* Per-sweep DMRG statistics (one sweep = 2(L-1) two-site updates). */
typedef struct {
  double E;             /* energy after the sweep (FP64 Rayleigh quotient)           */
  double max_err;       /* largest truncation error of the sweep                     */
  double max_disc;      /* largest discarded weight of the sweep                     */
  int64_t max_chi;      /* largest bond dimension after the sweep                    */
  int total_matvecs;    /* matvecs of all eigensolves                                */
  int unconverged;      /* eigensolves that hit the cap                              */
  double seconds;       /* wall time of the sweep (CUDA events)                      */
  double t_plan;        /* seconds per phase, summed over the sweep's updates (stream  */
  double t_eig;         /*   time between events, host gaps included): eigensolve      */
  double t_svd;         /*   planning (block tables, operator upload), the eigensolve, */
  double t_env;         /*   theta formation + truncated SVD, environment growth        */
} tnt_sweep_stats;

/* Per-step TEBD statistics (second-order Trotter step). */
typedef struct {
  double err_sum;       /* sum of the step's truncation errors (Eq. 3)               */
  double disc_sum;      /* sum of the step's discarded weights                       */
  int64_t max_chi;
  double seconds;
} tnt_step_stats;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`, enqueueing on `stream` (a cudaStream_t, or
 * NULL for the legacy default stream).  Fails with TNT_E_CUDA if no usable GPU exists. */
int tnt_ctx_create(int device, void* stream, tnt_ctx** out);

/* Device allocator supplied by the caller (the paper's tntSystem owns the library's
 * resources, App. A.3; here an application that manages device memory itself, e.g. through
 * PyTorch's caching allocator, hands the library its alloc/free pair).  alloc(bytes, user)
 * returns device memory on the context's device, aligned to at least 256 bytes, or NULL
 * (the call that needed it then fails with TNT_E_ALLOC); free(ptr, user) receives only
 * pointers alloc returned.  Both are called on the thread that called into the library,
 * never from a kernel; before memory goes back through free the library synchronises the
 * device, so nothing of its own still uses it. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} tnt_allocator;

/* tnt_ctx_create with every device allocation of the context, and of the MPO, MPS, DMRG
 * and TEBD handles made from it (scratch arena, status word, FP64 product slices, site
 * tensors, environments), made through *alloc (copied; alloc->user must outlive them).
 * TNT_E_INVALID if alloc or either callback is NULL. */
int tnt_ctx_create_with_allocator(int device, void* stream, const tnt_allocator* alloc,
                                  tnt_ctx** out);
int tnt_ctx_destroy(tnt_ctx* ctx);
/* Replace the stream used by later calls. */
int tnt_set_stream(tnt_ctx* ctx, void* stream);
/* Text of the last error on this context (static storage owned by the context). */
const char* tnt_last_error(const tnt_ctx* ctx);
/* Number of kernels this library has launched on the context (diagnostics). */
int64_t tnt_launch_count(const tnt_ctx* ctx);
/* Diagnostics: time every launch of one kernel class with CUDA events recorded on the
 * context's stream, and sum its algorithmic work.  Classes and their work unit:
 *   "cgemm_tf32x3" (useful FLOPs 8 M N K of the complex product), "zgemm_f64" (8 M N K),
 *   "op_apply" (FLOPs), "op_mixed", "split_theta" (bytes read plus written), "multidot",
 *   "multiaxpy" (FP64 FLOPs), "heig_tridiag" (FLOPs), "heig_tridiag_eig" (none),
 *   "heig_backtransform" (FLOPs), "cgemm_grouped", "zgemm_grouped", "oz_gemm" (useful
 *   FLOPs), "u1_wop", "u1_pack_theta", "u1_gather", "oz_slice" (bytes).
 * NULL or "" switches timing off.  At most 16384 launches are recorded between reads. */
int tnt_profile_select(tnt_ctx* ctx, const char* kernel_class);
/* Synchronise the stream; return the summed duration (ms), the number of timed launches
 * and their summed work since the last read; reset the counters. */
int tnt_profile_read(tnt_ctx* ctx, double* total_ms, int64_t* launches, double* work);

/* Parameter handling (App. A.3: the system settings and their defaults). */
int tnt_params_default(tnt_params* p);
int tnt_params_set(tnt_ctx* ctx, const tnt_params* p);
int tnt_params_get(const tnt_ctx* ctx, tnt_params* p);
/* Summary of the settings in the layout of App. A.3 Listing 5, NUL-terminated into buf. */
int tnt_sys_info(const tnt_ctx* ctx, char* buf, size_t n);

/* ------------------------------------------------------------------ model (host, FP64) */

/* One site's Bose-Hubbard MPO tensor W[4][4][d][d], d = n_max + 1, for site j (1-based)
 * of Eq. 2 plus -mu n: lower-triangular hand construction (Sec. 4.3),
 *   W[0][0] = I, W[1][0] = b, W[2][0] = b+, W[3][0] = U/2 n(n-1) + (V (j-j_c)^2 - mu) n,
 *   W[3][1] = -J b+, W[3][2] = -J b, W[3][3] = I.
 * Left boundary vector e_3, right boundary e_0.  h_W: host, 16 d^2 elements.
 * TNT_E_INVALID for n_max < 0, a NULL output or a non-finite parameter. */
int tnt_bh_mpo_site(int n_max, double J, double U, double mu, double V, double j,
                    double j_c, tnt_cplx* h_W);
/* Trotter gate exp(-i tau h) of the bond term
 *   h = -J (b+ (x) b + b (x) b+) + c1 h_site (x) I + c2 I (x) h_site,
 * h_site = U/2 n(n-1) - mu n, as a d^2 x d^2 matrix G[(s1' s2'), (s1 s2)] (host).
 * TNT_E_INVALID for n_max < 0, a NULL output or a non-finite parameter. */
int tnt_bh_bond_gate(int n_max, double J, double U, double mu, double c1, double c2,
                     double tau, tnt_cplx* h_G);
/* Spin-S Heisenberg chain (the performance model of Sec. 6, Tables 1 and 2, is the
 * isotropic spin-1 case: two_s = 2, Jz = J, hz = 0):
 *   H = sum_j [J/2 (S+_j S-_{j+1} + S-_j S+_{j+1}) + Jz S^z_j S^z_{j+1}] - hz sum_j S^z_j.
 * Basis |s>, s = 0..two_s, magnetisation m = s - S, so that s counts quanta like a boson
 * number: the U(1) label of a bond (the sum of s to its left) is S^z_left + S * sites,
 * the sector S^z_total = 0 is N = L S, and every U(1) entry point of this library applies
 * unchanged.  <s+1|S+|s> = sqrt(S(S+1) - m(m+1)).
 * tnt_spin_mpo_site: W[5][5][d][d], d = two_s + 1, lower-triangular like the Bose-Hubbard
 *   MPO: W[0][0] = I, W[1][0] = S-, W[2][0] = S+, W[3][0] = S^z, W[4][0] = -hz S^z,
 *   W[4][1] = J/2 S+, W[4][2] = J/2 S-, W[4][3] = Jz S^z, W[4][4] = I; left boundary
 *   e_4, right boundary e_0; MPO bond charges wq = {0, +1, -1, 0, 0}.
 * tnt_spin_bond_h: the bond term with the field split c1 / c2 between the two sites,
 *   h[(s1' s2'), (s1 s2)] (host, d^4 values).
 * two_s in 1..15; TNT_E_INVALID otherwise, or for a non-finite parameter. */
int tnt_spin_mpo_site(int two_s, double J, double Jz, double hz, tnt_cplx* h_W);
int tnt_spin_bond_h(int two_s, double J, double Jz, double hz, double c1, double c2,
                    tnt_cplx* h_h);
/* G = exp(-i tau h) of a Hermitian n x n host matrix h (row-major; its Hermitian part is
 * used), by host cyclic Jacobi in FP64: the Trotter gate of any nearest-neighbour bond
 * term (Sec. 3).  n in 1..256.  TNT_E_INVALID for n out of range, a NULL pointer, or a
 * non-finite tau or entry of h. */
int tnt_bond_gate(int n, const tnt_cplx* h_h, double tau, tnt_cplx* h_G);

/* ------------------------------------------------------------------ two-site kernels */

/* a1. theta[a,s1,s2,b] = sum_m A[a,s1,m] B[m,s2,b]  (Sec. 3 contraction, App. B.1.1).
 * d_A: chl x d x chm, d_B: chm x d x chr, d_theta: chl x d x d x chr (device). */
int tnt_theta_form(tnt_ctx* ctx, const tnt_cplx* d_A, const tnt_cplx* d_B, int64_t chl,
                   int64_t d, int64_t chm, int64_t chr, tnt_cplx* d_theta);

/* a2. out[a,s1',s2',b] = sum G[(s1' s2'),(s1 s2)] theta[a,s1,s2,b]  (TEBD gate, Sec. 3).
 * d_G: d^2 x d^2 (device); d_out must not alias d_theta. */
int tnt_gate_apply(tnt_ctx* ctx, const tnt_cplx* d_G, const tnt_cplx* d_theta, int64_t chl,
                   int64_t d, int64_t chr, tnt_cplx* d_out);

/* a3. y = H_eff theta:
 *   y[a',s1',s2',b'] = sum L[a',w,a] W1[w,w1,s1',s1] W2[w1,w2,s2',s2] R[b',w2,b] theta[a,s1,s2,b]
 * (two-site form of the Listing 1 contractor), contracted as (L.theta).W1.W2.R.
 * precision = TNT_PREC_FP64: FP64 throughout.  TNT_PREC_MIXED: the two chi^3 contractions
 * on tcgen05 tensor cores in split TF32 (hi*hi + hi*lo + lo*hi, FP32 accumulation),
 * relative error ~1e-6 of |y|; the W contraction and the output stay FP64.
 * d_L: chl x D x chl, d_W1, d_W2: D x D x d x d, d_R: chr x D x chr, d_theta, d_y:
 * chl x d x d x chr (device; d_y must not alias inputs). */
int tnt_heff_apply(tnt_ctx* ctx, const tnt_cplx* d_L, const tnt_cplx* d_W1,
                   const tnt_cplx* d_W2, const tnt_cplx* d_R, const tnt_cplx* d_theta,
                   int64_t chl, int64_t d, int64_t D, int64_t chr, int precision,
                   tnt_cplx* d_y);

/* The FP64 path of tnt_heff_apply for callers that cannot allocate device memory (the
 * paper has no counterpart: this is an interface for embedding).  A plug-in inside a host
 * application that owns all device memory (its own pool, or a budget fixed at start-up),
 * or a process sharing its GPU with a framework that reserved the rest, cannot call
 * cudaMalloc; this call makes none (nor cudaFree, nor any allocating library routine).
 * Its intermediates (the dense operator W1.W2, L.theta and W1.W2.L.theta) live in one
 * file-scope device array of 16 MiB that every GPU loading the library holds until the
 * process exits, so it accepts only d^2 D <= 256 and chl * D * d * d * chr <= 491,520
 * (e.g. chi = 64, d = 5, D = 4); larger shapes return TNT_E_UNSUPPORTED with the limit in
 * the message.  The first call on a device looks the array's device address up (once,
 * with that device current, which may initialise the module); make that first call before
 * any stream capture.  All calls share the array and it keeps the last call's contents:
 * calls that overlap on the GPU (other streams, or other host threads on the same device)
 * race on it.  Arguments, layouts and results are those of tnt_heff_apply with
 * TNT_PREC_FP64; the call enqueues its four kernels on the context's stream and returns
 * without synchronising. */
int tnt_heff_apply_noalloc(tnt_ctx* ctx, const tnt_cplx* d_L, const tnt_cplx* d_W1,
                           const tnt_cplx* d_W2, const tnt_cplx* d_R, const tnt_cplx* d_theta,
                           int64_t chl, int64_t d, int64_t D, int64_t chr, tnt_cplx* d_y);

/* a8. Environment growth (Sec. 4.3 <psi|H|psi> network, Listing 2 H_prepare):
 *   left:  Lout[m',w',m] = sum conj(A[a',s',m']) L[a',w,a] W[w,w',s',s] A[a,s,m]
 *          d_L: chl x D x chl, d_A: chl x d x chr, d_Lout: chr x D x chr
 *   right: Rout[a',w,a] = sum conj(B[a',s',b']) R[b',w',b] W[w,w',s',s] B[a,s,b]
 *          d_R: chr x D x chr, d_B: chl x d x chr, d_Rout: chl x D x chl      (FP64) */
int tnt_env_left(tnt_ctx* ctx, const tnt_cplx* d_L, const tnt_cplx* d_W,
                 const tnt_cplx* d_A, int64_t chl, int64_t d, int64_t D, int64_t chr,
                 tnt_cplx* d_Lout);
int tnt_env_right(tnt_ctx* ctx, const tnt_cplx* d_R, const tnt_cplx* d_W,
                  const tnt_cplx* d_B, int64_t chl, int64_t d, int64_t D, int64_t chr,
                  tnt_cplx* d_Rout);

/* a4 + a9. Lowest eigenpair of H_eff (Lanczos, full re-orthogonalisation by classical
 * Gram-Schmidt, repeated once when the first pass cancelled more than 99% of the vector,
 * FP64 vectors and tridiagonal solve; restart from the Ritz vector
 * every krylov_cap steps; at most lanczos_maxit matvecs; the library's eigensolver role of
 * Sec. 4.3).  Matvecs use ctx precision; with TNT_PREC_MIXED one more FP64 matvec gives
 * E_rq and resid_fp64.  d_theta (chl x d x d x chr) is the start vector on entry and the
 * unit-norm eigenvector on exit.  Returns TNT_E_NOCONV (with the result filled) if the cap
 * was hit unconverged. */
int tnt_lanczos_ground(tnt_ctx* ctx, const tnt_cplx* d_L, const tnt_cplx* d_W1,
                       const tnt_cplx* d_W2, const tnt_cplx* d_R, int64_t chl, int64_t d,
                       int64_t D, int64_t chr, tnt_cplx* d_theta, tnt_lanczos_result* res);

/* a5 + a6. Truncated SVD of M (m x n, device) read as block diagonal under U(1) labels
 * h_row_q (m) and h_col_q (n) (host; pass all zeros, or NULL for both, for a dense matrix),
 * with the four truncation rules of the context parameters (App. B.1.2; smallest chi wins)
 * and global order lambda desc, then charge asc, then in-block index.
 * side = TNT_SVD_LEFT:  d_U (m x chi) orthonormal columns, d_X = S V^H (chi x n) = U^H M.
 * side = TNT_SVD_RIGHT: d_X = V^H (chi x n) orthonormal rows, d_U = U S (m x chi) = M V.
 * renorm != 0 rescales the kept S to sum S^2 = 1 (DMRG); 0 keeps it (TEBD).
 * Capacity: d_U holds m * cap, d_X holds cap * n, h_S and h_bond_q hold cap values, with
 * cap = min(m, n, chi_max); outputs are written densely with leading dimension chi.
 * Kept indices are ordered by charge ascending, then lambda descending.
 * Per block an FP64 Gram matrix and its leading eigenvectors (Householder tridiagonal form,
 * bisection, inverse iteration); each sigma is the norm of a projection (a row of U^H M or
 * a column of M V), so its absolute error is ~eps |M|: values far below eps^(1/2) sigma_0
 * keep their absolute, not their relative, accuracy. */
/* Automatic blocking (Sec. 6, Fig. of the blocked array; the library's SVD zeroing
 * tolerance, off (-1) by default as in its system listing, App. B): with tol >= 0, every
 * truncated SVD of a matrix without charge labels (tnt_svd_trunc with NULL labels, and the
 * SVDs of unlabelled MPS in DMRG and TEBD) first sets the entries with |M_ij| <= tol to
 * zero, then groups rows and columns into the connected components of the remaining
 * non-zero pattern (a row and a column are joined by a non-zero entry) and runs the block
 * SVD on those blocks, exactly as for charge blocks; the bond labels returned are the
 * component numbers (ascending in each component's first row).  tol < 0 switches it off.
 * TNT_E_INVALID for a NaN tolerance. */
int tnt_set_svd_zero_tol(tnt_ctx* ctx, double tol);
/* The host half of automatic blocking (no GPU needed): the connected components of a
 * bipartite non-zero pattern, rows 0..m-1 and columns 0..n-1, bit (j % 32) of
 * h_mask[i * ceil(n/32) + j / 32] set where M_ij is non-zero.  h_row_q (m) and h_col_q (n)
 * get component numbers: numbered by each component's first row, components of columns
 * alone after them in column order; *h_count their number.  Host arrays, the caller's.
 * TNT_E_INVALID on a null pointer or m, n < 1. */
int tnt_autoblock_components(int64_t m, int64_t n, const uint32_t* h_mask, int64_t* h_row_q,
                             int64_t* h_col_q, int64_t* h_count);
int tnt_svd_trunc(tnt_ctx* ctx, const tnt_cplx* d_M, int64_t m, int64_t n,
                  const int64_t* h_row_q, const int64_t* h_col_q, int side, int renorm,
                  tnt_cplx* d_U, tnt_cplx* d_X, double* h_S, int64_t* h_bond_q,
                  tnt_trunc_result* res);

/* ------------------------------------------------------------------ MPO / MPS / DMRG */

/* Bose-Hubbard MPO on L sites (Eq. 2 plus -mu N), device-resident. */
int tnt_mpo_bose_hubbard(tnt_ctx* ctx, int L, int n_max, double J, double U, double mu,
                         double V, double j_c, tnt_mpo** out);
/* Spin-S Heisenberg MPO of tnt_spin_mpo_site on L sites (device-resident, U(1) charges
 * wq = {0, +1, -1, 0, 0}). */
int tnt_mpo_spin_heisenberg(tnt_ctx* ctx, int L, int two_s, double J, double Jz, double hz,
                            tnt_mpo** out);
/* Any MPO from host tensors (Sec. 4.3: MPOs are built by hand): h_W[j] = W_j[D][D][d][d]
 * (W[w][w'][s'][s], s' the bra index), h_left / h_right the D boundary vectors (the
 * operator is left^T W_1 ... W_L right), h_wq (D values, or NULL) the U(1) charges of the
 * MPO bond index (L[a',w,a] non-zero only where q_a' = q_a + wq[w]); with NULL the DMRG
 * sweep runs the dense path.  Host arrays are copied.  d in 1..16, D in 1..64. */
int tnt_mpo_create(tnt_ctx* ctx, int L, int d, int D, const tnt_cplx* const* h_W,
                   const tnt_cplx* h_left, const tnt_cplx* h_right, const int* h_wq,
                   tnt_mpo** out);
int tnt_mpo_destroy(tnt_mpo* mpo);

/* MPS from host data: h_chi[0..L] bond dimensions (h_chi[0] = h_chi[L] = 1), h_sites[j]
 * chi[j] x d x chi[j+1] tensors, h_charges[k] (chi[k] labels of bond k, bosons to the
 * left) or h_charges = NULL for no labels.  Device capacity per bond is
 * min(chi_cap, d^k, d^(L-k)) with chi_cap >= every h_chi. */
int tnt_mps_create(tnt_ctx* ctx, int L, int d, int64_t chi_cap, const int64_t* h_chi,
                   const tnt_cplx* const* h_sites, const int64_t* const* h_charges,
                   tnt_mps** out);
/* Product (Fock) state |n_1 ... n_L> with bond labels (e.g. the Mott state |1,...,1>). */
int tnt_mps_product(tnt_ctx* ctx, int L, int d, int64_t chi_cap, const int* h_occupations,
                    tnt_mps** out);
int tnt_mps_destroy(tnt_mps* mps);
int tnt_mps_length(const tnt_mps* mps, int* L, int* d);
int tnt_mps_bond_dim(const tnt_mps* mps, int bond, int64_t* chi);
/* Copy site j (chi[j] x d x chi[j+1]) to host; cap is the host buffer length in elements. */
int tnt_mps_get_site(tnt_ctx* ctx, const tnt_mps* mps, int site, tnt_cplx* h_out,
                     int64_t cap);
int tnt_mps_get_charges(const tnt_mps* mps, int bond, int64_t* h_out, int64_t cap);
/* <psi|O|psi> (FP64 environment pass) and <psi|psi>. */
int tnt_mps_expect_mpo(tnt_ctx* ctx, const tnt_mps* mps, const tnt_mpo* mpo, double* E);
int tnt_mps_norm2(tnt_ctx* ctx, const tnt_mps* mps, double* norm2);

/* <a|b> of two MPS of equal length and physical dimension (the <psi|O|psi> network of
 * Sec. 4.3 with O = 1 and two different states), FP64, contracted site by site from the
 * left (two GEMMs per site); labels are not used.  Host output; synchronises the stream.
 * TNT_E_INVALID on mismatched L or d. */
int tnt_mps_overlap(tnt_ctx* ctx, const tnt_mps* a, const tnt_mps* b, tnt_cplx* out);

/* Replace the U(1) labels of bond `bond` (App. A.1.1: tntNodeSetQN sets the quantum numbers
 * of a leg; here a bond label counts the bosons to the left of the bond).  h_q holds
 * chi[bond] labels (host, copied).  Accepted only if every non-zero entry of the two sites
 * next to the bond keeps q_left + s = q_right under the new labels (checked on the device);
 * otherwise TNT_E_INVALID with the count of violating entries, and the labels are left as
 * they were.  The MPS must carry labels; the boundary bonds' labels are fixed. */
int tnt_mps_set_charges(tnt_ctx* ctx, tnt_mps* mps, int bond, const int64_t* h_q);

/* File output and input of an MPS (App. B.5: the library writes its networks with their
 * block labels and its system settings, and a file written by one calculation is the input
 * of the next).  The file (native byte order) holds: the 8 bytes "TNTMPS01"; int32 L, d
 * and a labels flag; the context's tnt_params; int64 chi[0..L]; with labels, chi[k] int64
 * labels per bond; every site tensor (chi[j] x d x chi[j+1] tnt_cplx, row-major).
 * tnt_mps_load creates a new MPS (storage cap chi_cap, as tnt_mps_create) and, if
 * restore_params != 0, sets the context's parameters to the saved ones.  TNT_E_INVALID on
 * an unreadable, truncated or foreign file, or a bond above chi_cap. */
int tnt_mps_save(tnt_ctx* ctx, const tnt_mps* mps, const char* path);
int tnt_mps_load(tnt_ctx* ctx, const char* path, int64_t chi_cap, int restore_params,
                 tnt_mps** out);

/* Observables of Sec. 5's examples, FP64, for any (not necessarily normalised) MPS:
 * h_n[j] = <n_j> / <psi|psi> (L values), and the single-particle density matrix
 * h_rho[i*L + j] = <b+_i b_j> / <psi|psi> (L x L, Hermitian), by transfer environments
 * (O(L) environment growths for the density, O(L^2) for the matrix).  Host outputs. */
int tnt_mps_density(tnt_ctx* ctx, const tnt_mps* mps, double* h_n);
int tnt_mps_bdagb(tnt_ctx* ctx, const tnt_mps* mps, tnt_cplx* h_rho);

/* Two-site DMRG (Sec. 4.3 Listing 2 in two-site form).  Create brings the MPS to
 * right-canonical unit-norm form by exact SVD moves and builds the right environments.
 * One sweep = bonds 0..L-2 left to right, then L-2..0 right to left; each update forms
 * theta (a1), runs the eigensolve (a3, a4), splits theta by the truncated SVD (a5, a6)
 * with S renormalised (a7), and grows the environment (a8).  With TNT_PREC_MIXED each
 * eigensolve runs its split-TF32 Lanczos and then an FP64 Lanczos from that vector on a
 * budget of its own (lanczos_maxit matvecs), so the sweep's energies and states have the
 * FP64 path's accuracy; the split-TF32 phase supplies the start. */
int tnt_dmrg_create(tnt_ctx* ctx, tnt_mps* mps, const tnt_mpo* mpo, tnt_dmrg** out);
int tnt_dmrg_sweep(tnt_ctx* ctx, tnt_dmrg* dmrg, tnt_sweep_stats* stats);
/* One single-site sweep with subspace expansion on the same handle (the sweep of Sec. 4.3
 * on one site at a time; App. B's direct sums): sites 0..L-2 left to right, then L-1..1
 * right to left.  At site i the FP64 eigensolve of L . W . R . M (the one-site H_eff) gives
 * M; M is enlarged along the bond it hands over by a direct sum with the expansion term
 * alpha L.W.M (left to right, new index (w', b) with U(1) label q_b + wq[w']) or
 * alpha W.R.M (right to left, (w, a) with q_a + wq[w]), the neighbour by a zero block, and
 * the truncated SVD of the enlarged tensor (context parameters, S renormalised) splits it
 * back.  alpha = 0 is a plain one-site sweep, which cannot enlarge any bond.  Bonds are
 * capped by the MPS storage (chi_cap).  TNT_E_INVALID for alpha < 0 or non-finite. */
int tnt_dmrg_sweep1(tnt_ctx* ctx, tnt_dmrg* dmrg, double alpha, tnt_sweep_stats* stats);
/* The energy of every update of the last sweep on this handle (Sec. 4.3 Listing 2: the
 * local eigensolve's ground-state energy, here the FP64 Rayleigh quotient of its
 * eigenvector), in update order: 2(L-1) values after tnt_dmrg_sweep (bonds 0..L-2, then
 * L-2..0) or tnt_dmrg_sweep1 (sites 0..L-2, then L-1..1), fewer after a sweep that stopped
 * at an error, none before the first sweep.  *n receives the count; min(cap, *n) values
 * are copied to h_E (host memory; NULL allowed with cap = 0).  Host only, no GPU work.
 * TNT_E_INVALID for a NULL handle or n, cap < 0, or a NULL h_E with cap > 0. */
int tnt_dmrg_update_energies(const tnt_dmrg* dmrg, double* h_E, int64_t cap, int64_t* n);
/* One sweep of n independent chains in lock step (the batched phase scan: chains at
 * different U/J, seeds or fillings).  The chains' DMRG handles (each made by
 * tnt_dmrg_create, with U(1) labels on its MPS and MPO, all of one length L, no two sharing
 * an MPS) are swept together bond by bond: at each bond the n two-site eigenproblems are
 * solved by one lock-step Lanczos whose matvec is one grouped launch per contraction stage
 * over every block of every chain (as tnt_lanczos_ground_u1_batched, with the FP64 finish
 * of tnt_dmrg_sweep), then each chain's truncated SVD and environment growth follow.  Each
 * chain's result is that of tnt_dmrg_sweep on it alone, up to rounding.  stats[p] (host,
 * n entries) receives chain p's statistics, seconds being those of the whole batched
 * sweep.  TNT_E_INVALID for unlabelled chains, different lengths, a shared MPS, or a handle
 * whose centre is not on site 0. */
int tnt_dmrg_sweep_batched(tnt_ctx* ctx, int n, tnt_dmrg* const* handles, tnt_sweep_stats* stats);

/* One two-site update on bond (bond, bond + 1) of the handle's MPS (Sec. 4.3 Listing 2:
 * one local optimisation, in two-site form): theta, the eigensolve, the truncated SVD with
 * S renormalised and the environment growth, exactly as inside tnt_dmrg_sweep.  dir = +1
 * leaves the orthogonality centre on site bond + 1 (A_bond <- U) and grows the left
 * environment; dir = -1 leaves it on site bond (A_bond+1 <- V^H) and grows the right one.
 * The centre must be on site bond or bond + 1 and the environments of the bond current
 * (after tnt_dmrg_create the centre is on site 0, and a sweep ends there), else
 * TNT_E_INVALID.  Results in *lz and *tr; TNT_E_NOCONV if the eigensolve hit its cap (the
 * update is still applied).  A sweep requires the centre back on site 0. */
int tnt_dmrg_update(tnt_ctx* ctx, tnt_dmrg* dmrg, int bond, int dir, tnt_lanczos_result* lz,
                    tnt_trunc_result* tr);
int tnt_dmrg_destroy(tnt_dmrg* dmrg);

/* ------------------------------------------------------------------ FP64 matrix products */

/* C = op(A) op(B) in FP64 accuracy: the matrix form of a tensor contraction (App. B.1.1:
 * contraction as a matrix product after a reshape; here any leg order is expressed by
 * strides, nothing is permuted).  A(i,k) = d_A[i*a_rs + k*a_cs] (conjugated if conj_a),
 * B(k,j) = d_B[k*b_rs + j*b_cs] (conjugated if conj_b), C(i,j) = d_C[i*c_rs + j] (out;
 * must not alias A or B).  Device pointers, borrowed.  The engine is the context's FP64
 * GEMM setting: FMA (FP64 units) or TC (exact integer slices of the operands multiplied
 * on the TF32 tensor cores with exact FP32 sums, added in FP64: error within the size of
 * FP64 rounding, see tnt_set_fp64_gemm).  TNT_E_INVALID on bad sizes. */
int tnt_matmul(tnt_ctx* ctx, int64_t M, int64_t N, int64_t K, const tnt_cplx* d_A, int64_t a_rs,
               int64_t a_cs, int conj_a, const tnt_cplx* d_B, int64_t b_rs, int64_t b_cs,
               int conj_b, tnt_cplx* d_C, int64_t c_rs);

enum { TNT_FP64_GEMM_FMA = 0, TNT_FP64_GEMM_TC = 1 };
/* Engine of the library's FP64 matrix products (the FP64 H_eff.theta, theta, the
 * environments, the SVD's Gram matrices and projections).
 * TNT_FP64_GEMM_TC (default): each row of A and column of B is scaled by a power of two
 * to below 1 and cut into 9 integer slices of 6 bits (exact FP64 steps); slice products
 * run as TF32 MMAs whose FP32 sums over K chunks of 224 stay below 2^24 and so are exact;
 * the 45 slice pairs p + q <= 10 are added in FP64.  The error is below
 * 11 * 2^-54 * K * sigma_i * tau_j, sigma_i and tau_j the powers of two just above
 * max_k|A_ik| and max_k|B_kj|: the size of FP64's own rounding bound.
 * Small products (and calls that must not allocate) use FMA. */
int tnt_set_fp64_gemm(tnt_ctx* ctx, int engine);

/* ------------------------------------------------------------------ U(1) blocks, grouped */

/* One two-site H_eff problem with U(1) boson-number labels (App. A.1.1: every leg carries
 * quantum numbers; here a bond label counts the bosons to the left of the bond, and the
 * physical index s is its own boson number).  theta[a,s1,s2,b] is non-zero only where
 * q_b = q_a + s1 + s2, L[a',w,a] only where q_a' = q_a + wq[w], R[b',w,b] only where
 * q_b' = q_b + wq[w]; wq are the charges of the MPO bond index (the hand-built
 * Bose-Hubbard MPO of tnt_bh_mpo_site: wq = {0, +1, -1, 0}).  Environments and W are the
 * dense device arrays of tnt_heff_apply (entries outside the blocks are never read);
 * h_qa, h_qb, h_wq are host arrays, copied; labels must be non-decreasing.
 *
 * Compact theta (the vectors of the calls below): the blocks only, left sectors in
 * ascending charge; within sector q the slab [a in q][(s1, s2) row-major][b in the right
 * sector of charge q + s1 + s2] (pairs whose right sector is absent are skipped). */
typedef struct {
  const tnt_cplx* d_L;   /* chl x D x chl */
  const tnt_cplx* d_W1;  /* D x D x d x d, site i   */
  const tnt_cplx* d_W2;  /* D x D x d x d, site i+1 */
  const tnt_cplx* d_R;   /* chr x D x chr */
  int64_t chl, d, D, chr;
  const int64_t* h_qa;   /* chl labels of the left bond  */
  const int64_t* h_qb;   /* chr labels of the right bond */
  const int* h_wq;       /* D charges of the MPO bond index */
} tnt_u1_problem;

/* Length of the compact theta of one problem (host only; TNT_E_INVALID on bad labels). */
int tnt_u1_size(const tnt_u1_problem* prob, int64_t* n);
/* Dense theta (chl x d x d x chr, device) -> compact (device), and back (the dense result
 * is zero outside the blocks).  Integer index work only (App. B.1.2 reshape). */
int tnt_u1_pack(tnt_ctx* ctx, const tnt_u1_problem* prob, const tnt_cplx* d_theta, tnt_cplx* d_x);
int tnt_u1_unpack(tnt_ctx* ctx, const tnt_u1_problem* prob, const tnt_cplx* d_x, tnt_cplx* d_theta);
/* a3 over U(1) blocks, several problems at once (independent chains, each with its own
 * environments, MPO and labels): y_p = H_eff,p x_p (Sec. 4.2 Listing 1 order) where x and
 * y hold the problems' compact vectors back to back.  All blocks of all problems go into
 * one grouped launch per contraction stage; precision TNT_PREC_FP64 (FP64 grouped GEMM)
 * or TNT_PREC_MIXED (split TF32 on tcgen05, FP32 accumulate, tile shape autotuned once
 * per block structure and cached in the context).  h_flops (optional) receives the
 * algorithmic FLOPs of the block-sparse matvec.  x and y must not alias.  Returns
 * TNT_E_TIMEOUT if a tensor-core pipeline wait expired (the result is then invalid). */
int tnt_heff_apply_u1(tnt_ctx* ctx, int nprob, const tnt_u1_problem* probs, const tnt_cplx* d_x,
                      tnt_cplx* d_y, int precision, double* h_flops);
/* a4 over U(1) blocks: the Lanczos ground state of tnt_lanczos_ground on a compact theta
 * (in: start vector, out: ground state, unit norm), with the grouped matvec replayed as a
 * CUDA graph and, in TNT_PREC_MIXED, the FP64 grouped matvec for the win-back. */
int tnt_lanczos_ground_u1(tnt_ctx* ctx, const tnt_u1_problem* prob, tnt_cplx* d_x,
                          tnt_lanczos_result* res);
/* a4 for several independent problems at once (e.g. chains at different U/J): one
 * Lanczos recurrence per problem, run in lock step so that every Krylov step is one
 * grouped matvec over all problems; inner products, norms, the tridiagonal eigenpairs and
 * the stop rule are per problem, and a converged problem is frozen while the others go
 * on.  d_x holds the compact start vectors back to back (out: ground states, unit norm
 * each); h_res receives nprob results.  TNT_E_NOCONV if any problem hit the cap. */
int tnt_lanczos_ground_u1_batched(tnt_ctx* ctx, int nprob, const tnt_u1_problem* probs,
                                  tnt_cplx* d_x, tnt_lanczos_result* h_res);
/* Graph replay of the grouped matvec on (1, default) or off (plain launches; also off
 * while a kernel class is being profiled). */
int tnt_set_graphs(tnt_ctx* ctx, int on);
/* The autotuner's choice for these problems' block structure: h_tiles[0] = N tile of the
 * L.theta stage, [1] = N tile of the T3.R stage, [2] = its split-K.  TNT_E_INVALID if the
 * structure has not been tuned yet by a call above. */
int tnt_u1_tiles(tnt_ctx* ctx, int nprob, const tnt_u1_problem* probs, int* h_tiles);

/* Second-order Trotter TEBD (Sec. 3, Trotterised update; Sec. 5, real-time evolution with
 * the accumulated truncation error and 1 - <psi|psi> tracked).  The paper prints no scheme;
 * one step is exp(-i H_odd dt/2) exp(-i H_even dt) exp(-i H_odd dt/2), odd bonds (1,2),
 * (3,4), ... (1-based), hbar = 1, with the Bose-Hubbard bond term
 *   h = -J (b+ (x) b + b (x) b+) + c1 h_site (x) I + c2 I (x) h_site,
 *   h_site = U/2 n(n-1) - mu n,  c = 1 on the end sites, 1/2 elsewhere.
 * Gates within a layer go in ascending bond order; before each the orthogonality centre
 * moves to the bond by exact SVD moves, then theta = A_i A_{i+1} (a1), theta' = G theta
 * (a2), truncated SVD by the context's parameters (a5, a6), A_i <- U, A_{i+1} <- S V^H
 * (a7).  The state is NOT renormalised: the discarded weight leaves <psi|psi>.
 * create: the MPS (borrowed; it must outlive the handle and is updated in place) gets its
 *   centre at site 0 by exact moves; n_max + 1 must equal the MPS's d; the gates are built
 *   on the host in FP64.  TNT_E_INVALID on bad arguments.
 * step: one Trotter step; stats gets the sums of the step's truncation errors (Eq. 3) and
 *   discarded weights, the largest bond and the step's device time.  Bond dimensions are
 *   capped by the context's chi_max and by the MPS's storage (its chi_cap). */
int tnt_tebd_create(tnt_ctx* ctx, tnt_mps* mps, int n_max, double J, double U, double mu,
                    double dt, tnt_tebd** out);
/* The same Trotter step for the spin-S Heisenberg chain (the bond term of
 * tnt_spin_bond_h with c1, c2 as above; two_s + 1 must equal the MPS's d). */
int tnt_tebd_create_spin(tnt_ctx* ctx, tnt_mps* mps, int two_s, double J, double Jz,
                         double hz, double dt, tnt_tebd** out);
/* The same Trotter step for any nearest-neighbour Hamiltonian: h_bond[i] (host, d^2 x d^2,
 * rows (s1' s2'), columns (s1 s2)) is the term of bond (i, i+1), i = 0..L-2, with the
 * on-site parts already split between bonds.  Copied; TNT_E_NAN on a non-finite entry.
 * With U(1)-labelled MPS bonds each term must conserve s1 + s2. */
int tnt_tebd_create_bonds(tnt_ctx* ctx, tnt_mps* mps, const tnt_cplx* const* h_bond,
                          double dt, tnt_tebd** out);
int tnt_tebd_step(tnt_ctx* ctx, tnt_tebd* tebd, tnt_step_stats* stats);
/* One two-site gate on bond (bond, bond + 1) through the TEBD handle, which tracks the
 * orthogonality centre (Sec. 3's Trotterised update is a sequence of these): the centre is
 * moved to site bond or bond + 1 by exact SVD moves, theta' = G theta with h_gate the
 * d^2 x d^2 matrix G[(s1' s2'), (s1 s2)] (host, row-major, copied; e.g. from tnt_bond_gate),
 * then the truncated SVD with the context's parameters and no renormalisation; dir = +1
 * leaves the centre on site bond + 1 (A_bond <- U), dir = -1 on site bond.  The SVD's
 * result in *tr.  TNT_E_NAN for a non-finite gate entry. */
int tnt_tebd_gate(tnt_ctx* ctx, tnt_tebd* tebd, int bond, const tnt_cplx* h_gate, int dir,
                  tnt_trunc_result* tr);
/* The site holding the orthogonality centre of the TEBD handle's MPS. */
int tnt_tebd_centre(const tnt_tebd* tebd, int* centre);
int tnt_tebd_destroy(tnt_tebd* tebd);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* TNT_GB300_H */
