// Internal declarations of the GB300 two-site-update library (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/tnt_gb300.h"

namespace tnt {

// ---------------------------------------------------------------- complex helpers
typedef double2 z;  // complex128 stored {re, im}, the same bytes as tnt_cplx

__host__ __device__ __forceinline__ z zmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ z zadd(z a, z b) { return zmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ z zsub(z a, z b) { return zmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ z zmul(z a, z b) {
  return zmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ z zconj(z a) { return zmk(a.x, -a.y); }
__host__ __device__ __forceinline__ z zscale(z a, double s) { return zmk(a.x * s, a.y * s); }
// acc += a * b
__host__ __device__ __forceinline__ void zfma(z& acc, z a, z b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// ---------------------------------------------------------------- context
struct Arena {
  // A bump allocator over one device block; grown (reallocated) only between calls.
  char* base = nullptr;
  size_t cap = 0;
  size_t top = 0;
};

// Device allocator of a context and of the handles made from it: cudaMalloc / cudaFree,
// or the caller's callbacks (tnt_ctx_create_with_allocator).
struct DevAlloc {
  void* (*alloc)(size_t bytes, void* user) = nullptr;
  void (*free)(void* ptr, void* user) = nullptr;
  void* user = nullptr;
};
// 0 on success; *p = nullptr on failure
int dev_alloc(const DevAlloc& a, void** p, size_t bytes);
// synchronises the device first when the memory goes back to the caller's allocator
void dev_free(const DevAlloc& a, void* p);

struct Ctx {
  int device = 0;
  DevAlloc dalloc;
  cudaStream_t stream = 0;
  tnt_params params;
  Arena ws;               // per-call scratch
  std::string err;        // last error message
  double* h_pinned = nullptr;  // small pinned host buffer for scalar read-back
  size_t h_pinned_cap = 0;
  // device status word written by kernels (bounds / NaN / timeout flags)
  int* d_status = nullptr;
  // arrival counters of the kernels that finish their reduction in the last CTA to arrive
  // (zero between launches: that CTA resets its counter)
  unsigned* d_count = nullptr;
  // counters (diagnostics, not hot-path state)
  int64_t launches = 0;
  // optional CUDA-event timing of one kernel class (tnt_profile_select)
  std::string prof_cls;
  std::vector<cudaEvent_t> prof_ev;  // pairs: start, end
  size_t prof_n = 0;
  double prof_work = 0;  // algorithmic FLOPs or bytes of the timed launches
  // grouped U(1) matvec: replay as a CUDA graph (off while kernel classes are profiled),
  // and the autotuner's tile choice per block-structure signature
  bool use_graphs = true;
  std::map<std::string, std::vector<int>> tune;
  // FP64 GEMM engine for large products: 1 = integer-slice emulation on the tensor cores
  // (FP64-accurate), 0 = FP64 FMA only; its slice buffer is owned by the context
  int oz_mode = 1;
  double svd_zero_tol = -1.0;  // automatic blocking of unlabelled SVDs (< 0: off)
  // split-TF32 eigensolves end with an FP64 Lanczos from their vector, on a budget of
  // their own (set by the DMRG sweep around its eigensolves)
  bool fp64_finish = false;
  void* oz_buf = nullptr;
  size_t oz_cap = 0;
  // second stream for the Lanczos T_k eigenproblem, one Krylov step behind the vector
  // work on `stream`, and the events that order the two (created on first use)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_main[2] = {nullptr, nullptr}, ev_side[2] = {nullptr, nullptr};
};

// Records CUDA events around the launches of one kernel class when that class is
// selected, and adds the launch's algorithmic work (FLOPs or bytes, per class).
struct ProfScope {
  Ctx* c;
  bool on;
  ProfScope(Ctx* cc, const char* cls, double work = 0)
      : c(cc), on(!cc->prof_cls.empty() && cc->prof_cls == cls && 2 * cc->prof_n + 1 < cc->prof_ev.size()) {
    if (on) {
      cudaEventRecord(c->prof_ev[2 * c->prof_n], c->stream);
      c->prof_work += work;
    }
  }
  ~ProfScope() {
    if (on) {
      cudaEventRecord(c->prof_ev[2 * c->prof_n + 1], c->stream);
      c->prof_n++;
    }
  }
};

// error plumbing: every entry point returns through these
int set_err(Ctx* c, int code, const char* fmt, ...);
#define TNT_CUDA_TRY(ctx, expr)                                                     \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return ::tnt::set_err((ctx), TNT_E_CUDA, "%s failed: %s (%s:%d)", #expr,      \
                            cudaGetErrorString(e_), __FILE__, __LINE__);            \
  } while (0)
#define TNT_TRY(expr)              \
  do {                             \
    int r_ = (expr);               \
    if (r_ != TNT_OK) return r_;   \
  } while (0)
#define TNT_CHECK_LAUNCH(ctx) TNT_CUDA_TRY(ctx, cudaGetLastError())

// scratch: reserve() grows the arena (synchronising the stream) before a call's
// allocations; alloc() then only bumps.  Everything is released by reset().
int ws_reserve(Ctx* c, size_t bytes);
void* ws_alloc(Ctx* c, size_t bytes);
inline void ws_reset(Ctx* c) { c->ws.top = 0; }
inline size_t ws_round(size_t b) { return (b + 255) & ~size_t(255); }
int pinned_reserve(Ctx* c, size_t bytes);

// ---------------------------------------------------------------- kernels (FP64 path)
// Strided complex GEMM: C[i,j] = alpha * sum_k opA(i,k) opB(k,j) + beta * C[i,j]
// opA(i,k) = A[i*a_rs + k*a_cs] (conjugated if conj_a), likewise B; batched by stride.
struct ZGemm {
  int64_t M, N, K;
  const z* A;
  int64_t a_rs, a_cs, a_bs;
  const z* B;
  int64_t b_rs, b_cs, b_bs;
  z* C;
  int64_t c_rs, c_bs;
  int conj_a, conj_b;
  z alpha, beta;
  int64_t batch;
  int lower_only;  // Hermitian result: skip 64x64 tiles strictly above the diagonal
};
int zgemm(Ctx* c, const ZGemm& g);
// FP64-accurate C = A B on the tensor cores by exact integer slicing (oz.cu); zgemm routes
// large products with alpha = 1, beta = 0, batch = 1 there when the context allows it
bool ozgemm_eligible(const Ctx* c, const ZGemm& g);
int ozgemm(Ctx* c, const ZGemm& g);
// FP64 FMA GEMMs only while the guard lives (paths that must not allocate)
struct OzOff {
  Ctx* c;
  int saved;
  explicit OzOff(Ctx* cc) : c(cc), saved(cc->oz_mode) { c->oz_mode = 0; }
  ~OzOff() { c->oz_mode = saved; }
};
// G[i][j] = conj(G[j][i]) for i < j (complete a Hermitian matrix from its lower part)
int herm_mirror(Ctx* c, z* G, int64_t n);

// Sparse small operator acting on a group of legs with strided batches:
// out[b0*os0 + b1*os1 + b2*os2 + out_off[i]] (+)= sum_j op[i,j] in[b0*is0 + ... + in_off[j]]
// op is given in CSR form (row_ptr over i, col j, value).
struct OpApply {
  const z* in;
  z* out;
  int nI, nJ, nnz;
  const int* row_ptr;     // device, nI+1
  const int* col;         // device, nnz
  const z* val;           // device, nnz
  const int64_t* in_off;  // device, nJ
  const int64_t* out_off; // device, nI
  int64_t B0, B1, B2;
  int64_t is0, is1, is2, os0, os1, os2;
  int accumulate;
};
int op_apply(Ctx* c, const OpApply& a);

// Upload a dense op (nI x nJ, host) as CSR plus the two offset tables into scratch.
int op_upload(Ctx* c, const std::vector<z>& dense, int nI, int nJ,
              const std::vector<int64_t>& in_off, const std::vector<int64_t>& out_off,
              OpApply* a);

// Vector kernels (FP64, deterministic two-level reductions).
// dots[i] = <V_i | w> for i < k   (V_i = V + i*ld).  With d_skip set and *d_skip != 0 at
// run time, the kernels return without work (a pass decided on the device to be unneeded).
int vec_multidot(Ctx* c, const z* V, int64_t ld, int k, const z* w, int64_t n, z* d_dots,
                 const int* d_skip = nullptr);
// w -= sum_i coef[i] V_i ; then d_norm2 = |w|^2   (coef on device); skipped as above, in
// which case w and d_norm2 keep their values
int vec_multiaxpy_norm(Ctx* c, const z* V, int64_t ld, int k, const z* d_coef, z* w,
                       int64_t n, double* d_norm2, const int* d_skip = nullptr);
// The same two passes with FP32 arithmetic on the FP64 vectors (FP64 sums over blocks, FP64
// subtraction from w): for a Lanczos phase whose matvec error is already ~2^-22.
int vec_multidot_f32(Ctx* c, const z* V, int64_t ld, int k, const z* w, int64_t n, z* d_dots);
int vec_multiaxpy_norm_f32(Ctx* c, const z* V, int64_t ld, int k, const z* d_coef, z* w,
                           int64_t n, double* d_norm2);
// y = x * (1 / sqrt(*d_norm2))  (d_norm2 on device); if x == y scales in place
int vec_normalize(Ctx* c, const z* x, z* y, int64_t n, const double* d_norm2);
int vec_norm2(Ctx* c, const z* x, int64_t n, double* d_norm2);
int vec_dot(Ctx* c, const z* x, const z* y, int64_t n, z* d_dot);

// Lanczos tridiagonal: lowest eigenpair of T (k x k) given alpha[0..k-1], beta[0..k-2];
// writes out[0] = E, out[1] = |y_{k-1}|, and y[0..k-1].
int tridiag_lowest(Ctx* c, const double* d_alpha, const double* d_beta, int k, double* d_out,
                   double* d_y);
// The same on stream st (the Lanczos runs it on the context's side stream)
int tridiag_lowest_on(Ctx* c, cudaStream_t st, const double* d_alpha, const double* d_beta, int k,
                      double* d_out, double* d_y);
// Creates the context's side stream and its events on first use
int side_stream(Ctx* c);
// the same for nprob problems at once: problem p's alpha, beta, y at p * 64, out at p * 2;
// problems with d_skip[p] != 0 are left untouched
int tridiag_lowest_batched(Ctx* c, const double* d_alpha, const double* d_beta, int k,
                           double* d_out, double* d_y, int nprob, const int* d_skip);

// Hermitian eigensolvers of the truncated SVD's Gram blocks (heig.cu, FP64: Householder
// tridiagonalisation, bisection, inverse iteration, back-transformation).
// One large block: leading k eigenpairs, the reduction spread over the whole GPU.
// U: n x k with leading dimension ldu; ev: device, k values.
size_t heig_scratch_bound(int64_t n, int64_t k);
int heig_top(Ctx* c, z* G, int64_t n, int64_t k, z* U, int64_t ldu, double* ev);
// Many small blocks (n <= 256) at once, one CTA per block for the reduction.  A block of
// heig_small_blocks: offset of its n x n Gram block (and of its eigenvector columns,
// leading dimension n), its size and the number of eigenvectors wanted
struct SmallEig {
  int64_t goff, n, k;
};
int heig_small_blocks(Ctx* c, z* G, const std::vector<SmallEig>& blocks, z* U, double* ev);

// Helpers: gather / scatter / conversion
int gather2d(Ctx* c, const z* src, int64_t src_ld, const int64_t* d_rows, int64_t nr,
             const int64_t* d_cols, int64_t nc, z* dst, int64_t dst_ld, int conj_t);
int zfill(Ctx* c, z* p, int64_t n, z v);
int zscale_inplace(Ctx* c, z* p, int64_t n, const double* d_scale, int mode);

// Truncated SVD (svd.cu) and its scratch bound
size_t svd_scratch_bound(int64_t m, int64_t n);
int svd_trunc_impl(Ctx* c, const z* M, int64_t m, int64_t n, const int64_t* h_rq,
                   const int64_t* h_cq, int side, int renorm, z* U, z* X, double* h_S,
                   int64_t* h_bq, tnt_trunc_result* res);

// H_eff internals
int heff_f64(Ctx* c, const z* L, const z* W1, const z* W2, const z* R, const z* theta,
             int64_t chl, int64_t d, int64_t D, int64_t chr, z* y);
int heff_mixed(Ctx* c, const z* L, const z* W1, const z* W2, const z* R, const z* theta,
               int64_t chl, int64_t d, int64_t D, int64_t chr, z* y);

// host copies of MPO tensors are needed to build the CSR ops: read back W (tiny)
int read_small(Ctx* c, const void* dsrc, void* hdst, size_t bytes);

int bh_mpo_site_host(int n_max, double J, double U, double mu, double V, double j, double jc,
                     z* W);
int bh_bond_gate_host(int n_max, double J, double U, double mu, double c1, double c2,
                      double tau, z* G);
// exp(-i tau h) of a Hermitian n x n host matrix (row-major), by host Jacobi
int bond_gate_host(int n, const z* h, double tau, z* G);
// spin-S Heisenberg pieces (two_s = 2S): MPO site tensor [5][5][d][d], bond term d^2 x d^2
int spin_mpo_site_host(int two_s, double J, double Jz, double hz, z* W);
int spin_bond_h_host(int two_s, double J, double Jz, double hz, double c1, double c2, z* h);

// release the call's scratch on every return path
struct Scope {
  Ctx* c;
  explicit Scope(Ctx* cc) : c(cc) { ws_reset(c); }
  ~Scope() { ws_reset(c); }
};

}  // namespace tnt

struct tnt_ctx {
  tnt::Ctx c;
};
