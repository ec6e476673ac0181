// C-ABI entry points (include/tnt_gb300.h): context, parameters, model builders and the
// two-site kernels.  Argument checking happens here; the work is in the other units.
#include <cmath>
#include <cstdarg>
#include <initializer_list>
#include <vector>

#include "heff_plan.cuh"

namespace tnt {

int set_err(Ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

int dev_alloc(const DevAlloc& a, void** p, size_t bytes) {
  *p = nullptr;
  if (a.alloc) {
    *p = a.alloc(bytes, a.user);
    return *p ? 0 : 1;
  }
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    *p = nullptr;
    return 1;
  }
  return 0;
}

void dev_free(const DevAlloc& a, void* p) {
  if (!p) return;
  if (a.free) {
    cudaDeviceSynchronize();  // no kernel of this library may still use the memory
    a.free(p, a.user);
  } else {
    cudaFree(p);
  }
}

int ws_reserve(Ctx* c, size_t bytes) {
  if (bytes <= c->ws.cap) return TNT_OK;
  if (c->ws.top != 0)
    return set_err(c, TNT_E_ALLOC,
                   "scratch of %zu bytes needed while %zu bytes are in use (reserve first)", bytes,
                   c->ws.top);
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  dev_free(c->dalloc, c->ws.base);
  c->ws.base = nullptr;
  c->ws.cap = 0;
  size_t cap = ws_round(bytes + bytes / 8);
  void* base = nullptr;
  if (dev_alloc(c->dalloc, &base, cap) != 0)
    return set_err(c, TNT_E_ALLOC, "device allocation of %zu bytes of scratch failed", cap);
  c->ws.base = (char*)base;
  c->ws.cap = cap;
  return TNT_OK;
}

void* ws_alloc(Ctx* c, size_t bytes) {
  bytes = ws_round(bytes);
  if (c->ws.top + bytes > c->ws.cap) return nullptr;
  void* p = c->ws.base + c->ws.top;
  c->ws.top += bytes;
  return p;
}

int pinned_reserve(Ctx* c, size_t bytes) {
  if (bytes <= c->h_pinned_cap) return TNT_OK;
  if (c->h_pinned) {
    TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    cudaFreeHost(c->h_pinned);
  }
  c->h_pinned = nullptr;
  c->h_pinned_cap = 0;
  if (cudaMallocHost((void**)&c->h_pinned, bytes) != cudaSuccess)
    return set_err(c, TNT_E_ALLOC, "pinned host allocation of %zu bytes failed", bytes);
  c->h_pinned_cap = bytes;
  return TNT_OK;
}


// ---------------------------------------------------------------- Bose-Hubbard (host)
static void local_ops(int n_max, std::vector<double>* b) {
  const int d = n_max + 1;
  b->assign((size_t)d * d, 0.0);
  for (int n = 1; n < d; ++n) (*b)[(size_t)(n - 1) * d + n] = std::sqrt((double)n);
}

int bh_mpo_site_host(int n_max, double J, double U, double mu, double V, double j, double jc,
                     z* W) {
  const int d = n_max + 1, D = 4;
  std::vector<double> b;
  local_ops(n_max, &b);
  for (int e = 0; e < D * D * d * d; ++e) W[e] = zmk(0, 0);
  auto at = [&](int w, int v, int so, int si) -> z& { return W[((w * D + v) * d + so) * d + si]; };
  for (int so = 0; so < d; ++so)
    for (int si = 0; si < d; ++si) {
      const double bb = b[(size_t)so * d + si];      // <so|b|si>
      const double bd = b[(size_t)si * d + so];      // <so|b+|si>
      const double id = (so == si) ? 1.0 : 0.0;
      const double nn = (so == si) ? (double)si : 0.0;
      at(0, 0, so, si) = zmk(id, 0);
      at(1, 0, so, si) = zmk(bb, 0);
      at(2, 0, so, si) = zmk(bd, 0);
      at(3, 0, so, si) = zmk(0.5 * U * nn * (nn - id) + (V * (j - jc) * (j - jc) - mu) * nn, 0);
      at(3, 1, so, si) = zmk(-J * bd, 0);
      at(3, 2, so, si) = zmk(-J * bb, 0);
      at(3, 3, so, si) = zmk(id, 0);
    }
  return TNT_OK;
}

// Hermitian eigendecomposition on the host (cyclic Jacobi, tiny matrices: the d^2 x d^2
// bond term) for the gate exp(-i tau h).
static void herm_eig_host(int n, std::vector<z>& A, std::vector<double>* lam, std::vector<z>* V) {
  V->assign((size_t)n * n, zmk(0, 0));
  for (int i = 0; i < n; ++i) (*V)[(size_t)i * n + i] = zmk(1, 0);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0, dg = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double a = std::hypot(A[(size_t)i * n + j].x, A[(size_t)i * n + j].y);
        if (i == j) dg = std::max(dg, a); else off = std::max(off, a);
      }
    if (off <= 1e-16 * dg || off < 1e-300) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        z apq = A[(size_t)p * n + q];
        double ab = std::hypot(apq.x, apq.y);
        if (ab < 1e-300) continue;
        double app = A[(size_t)p * n + p].x, aqq = A[(size_t)q * n + q].x;
        z e = zmk(apq.x / ab, apq.y / ab);
        double tau = (aqq - app) / (2 * ab);
        double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
        double cs = 1 / std::sqrt(1 + t * t), sn = t * cs;
        for (int jx = 0; jx < n; ++jx) {  // rows: A <- J^H A
          z gp = A[(size_t)p * n + jx], gq = zmul(e, A[(size_t)q * n + jx]);
          A[(size_t)p * n + jx] = zsub(zscale(gp, cs), zscale(gq, sn));
          A[(size_t)q * n + jx] = zadd(zscale(gp, sn), zscale(gq, cs));
        }
        z ec = zconj(e);
        for (int i = 0; i < n; ++i) {  // columns: A <- A J, V <- V J
          z gp = A[(size_t)i * n + p], gq = zmul(A[(size_t)i * n + q], ec);
          A[(size_t)i * n + p] = zsub(zscale(gp, cs), zscale(gq, sn));
          A[(size_t)i * n + q] = zadd(zscale(gp, sn), zscale(gq, cs));
          z vp = (*V)[(size_t)i * n + p], vq = zmul((*V)[(size_t)i * n + q], ec);
          (*V)[(size_t)i * n + p] = zsub(zscale(vp, cs), zscale(vq, sn));
          (*V)[(size_t)i * n + q] = zadd(zscale(vp, sn), zscale(vq, cs));
        }
      }
  }
  lam->resize(n);
  for (int i = 0; i < n; ++i) (*lam)[i] = A[(size_t)i * n + i].x;
}

int bh_bond_gate_host(int n_max, double J, double U, double mu, double c1, double c2,
                      double tau, z* G) {
  const int d = n_max + 1, n = d * d;
  std::vector<double> b;
  local_ops(n_max, &b);
  std::vector<z> h((size_t)n * n, zmk(0, 0));
  auto hs = [&](int s) { return 0.5 * U * s * (s - 1) - mu * s; };
  for (int s1o = 0; s1o < d; ++s1o)
    for (int s2o = 0; s2o < d; ++s2o)
      for (int s1 = 0; s1 < d; ++s1)
        for (int s2 = 0; s2 < d; ++s2) {
          // -J (b+ (x) b + b (x) b+)
          double v = -J * (b[(size_t)s1 * d + s1o] * b[(size_t)s2o * d + s2] +
                           b[(size_t)s1o * d + s1] * b[(size_t)s2 * d + s2o]);
          if (s1o == s1 && s2o == s2) v += c1 * hs(s1) + c2 * hs(s2);
          h[(size_t)(s1o * d + s2o) * n + (s1 * d + s2)] = zmk(v, 0);
        }
  return bond_gate_host(n, h.data(), tau, G);
}

int bond_gate_host(int n, const z* h_in, double tau, z* G) {
  if (n < 1) return TNT_E_INVALID;
  std::vector<z> h(h_in, h_in + (size_t)n * n);
  for (int i = 0; i < n; ++i)  // Hermitian part only (h is Hermitian up to rounding)
    for (int j = 0; j <= i; ++j) {
      const z a = h[(size_t)i * n + j], b = zconj(h[(size_t)j * n + i]);
      const z m = zmk(0.5 * (a.x + b.x), 0.5 * (a.y + b.y));
      h[(size_t)i * n + j] = m;
      h[(size_t)j * n + i] = zconj(m);
    }
  std::vector<double> lam;
  std::vector<z> Q;
  herm_eig_host(n, h, &lam, &Q);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      z acc = zmk(0, 0);
      for (int k = 0; k < n; ++k) {
        z ph = zmk(std::cos(-tau * lam[k]), std::sin(-tau * lam[k]));
        zfma(acc, zmul(Q[(size_t)i * n + k], ph), zconj(Q[(size_t)j * n + k]));
      }
      G[(size_t)i * n + j] = acc;
    }
  return TNT_OK;
}

// ---------------------------------------------------------------- spin-S Heisenberg (host)
// Basis |s>, s = 0..2S, magnetisation m = s - S, so that s counts quanta like a boson
// number and the U(1) label of a bond (the sum of s to its left) is S^z_left + S * sites.
//   <s+1| S+ |s> = sqrt(S(S+1) - m(m+1)),  S- = (S+)^H,  S^z = diag(m).
static void spin_ops(int two_s, std::vector<double>* sp, std::vector<double>* sz) {
  const int d = two_s + 1;
  sp->assign((size_t)d * d, 0.0);
  sz->assign((size_t)d * d, 0.0);
  for (int s = 0; s < d; ++s) {
    const double m2 = 2.0 * s - two_s;  // 2m
    (*sz)[(size_t)s * d + s] = 0.5 * m2;
    if (s + 1 < d)  // S(S+1) - m(m+1) = (2S (2S + 2) - 2m (2m + 2)) / 4
      (*sp)[(size_t)(s + 1) * d + s] = 0.5 * std::sqrt((double)two_s * (two_s + 2) - m2 * (m2 + 2));
  }
}

// H = sum_j [J/2 (S+_j S-_{j+1} + S-_j S+_{j+1}) + Jz S^z_j S^z_{j+1}] - hz sum_j S^z_j,
// MPO of bond dimension 5 in the lower-triangular form of the Bose-Hubbard MPO: rows
//   0: I;  1: S-;  2: S+;  3: S^z;  4: -hz S^z, J/2 S+, J/2 S-, Jz S^z, I
// (left boundary row 4, right boundary column 0).
int spin_mpo_site_host(int two_s, double J, double Jz, double hz, z* W) {
  const int d = two_s + 1, D = 5;
  std::vector<double> sp, sz;
  spin_ops(two_s, &sp, &sz);
  for (int e = 0; e < D * D * d * d; ++e) W[e] = zmk(0, 0);
  auto at = [&](int w, int v, int so, int si) -> z& { return W[((w * D + v) * d + so) * d + si]; };
  for (int so = 0; so < d; ++so)
    for (int si = 0; si < d; ++si) {
      const double p = sp[(size_t)so * d + si];  // <so|S+|si>
      const double m = sp[(size_t)si * d + so];  // <so|S-|si>
      const double zz = sz[(size_t)so * d + si];
      const double id = (so == si) ? 1.0 : 0.0;
      at(0, 0, so, si) = zmk(id, 0);
      at(1, 0, so, si) = zmk(m, 0);
      at(2, 0, so, si) = zmk(p, 0);
      at(3, 0, so, si) = zmk(zz, 0);
      at(4, 0, so, si) = zmk(-hz * zz, 0);
      at(4, 1, so, si) = zmk(0.5 * J * p, 0);
      at(4, 2, so, si) = zmk(0.5 * J * m, 0);
      at(4, 3, so, si) = zmk(Jz * zz, 0);
      at(4, 4, so, si) = zmk(id, 0);
    }
  return TNT_OK;
}

// bond term with the field split c1 / c2 between the two sites (as the on-site energy of
// the Bose-Hubbard bond term): rows (s1' s2'), columns (s1 s2)
int spin_bond_h_host(int two_s, double J, double Jz, double hz, double c1, double c2, z* h) {
  const int d = two_s + 1, n = d * d;
  std::vector<double> sp, sz;
  spin_ops(two_s, &sp, &sz);
  for (int s1o = 0; s1o < d; ++s1o)
    for (int s2o = 0; s2o < d; ++s2o)
      for (int s1 = 0; s1 < d; ++s1)
        for (int s2 = 0; s2 < d; ++s2) {
          const double pm = sp[(size_t)s1o * d + s1] * sp[(size_t)s2 * d + s2o];  // S+ (x) S-
          const double mp = sp[(size_t)s1 * d + s1o] * sp[(size_t)s2o * d + s2];  // S- (x) S+
          double v = 0.5 * J * (pm + mp);
          if (s1o == s1 && s2o == s2) {
            const double m1 = sz[(size_t)s1 * d + s1], m2 = sz[(size_t)s2 * d + s2];
            v += Jz * m1 * m2 - hz * (c1 * m1 + c2 * m2);
          }
          h[(size_t)(s1o * d + s2o) * n + (s1 * d + s2)] = zmk(v, 0);
        }
  return TNT_OK;
}

}  // namespace tnt

using namespace tnt;

// every model parameter of a host builder must be a finite number
static bool all_finite(std::initializer_list<double> v) {
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

#define CTX_CHECK(ctx)                   \
  do {                                   \
    if (!(ctx)) return TNT_E_INVALID;    \
  } while (0)
#define ARG_CHECK(ctx, cond, ...)                                       \
  do {                                                                  \
    if (!(cond)) return set_err(&(ctx)->c, TNT_E_INVALID, __VA_ARGS__); \
  } while (0)

extern "C" {

int tnt_params_default(tnt_params* p) {
  if (!p) return TNT_E_INVALID;
  p->chi_max = (int64_t)1 << 40;
  p->trunc_abs = -1.0;
  p->trunc_rel = 1e-16;
  p->trunc_err = 1e-8;
  p->trunc_type = TNT_TRUNC_2NORM;
  p->lanczos_tol = 1e-12;
  p->lanczos_maxit = 300;
  p->krylov_cap = 32;
  p->precision = TNT_PREC_FP64;
  p->seed = 0;
  return TNT_OK;
}

static int ctx_create(int device, void* stream, const DevAlloc& a, tnt_ctx** out) {
  if (!out) return TNT_E_INVALID;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= device || device < 0) return TNT_E_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return TNT_E_CUDA;
  tnt_ctx* t = new tnt_ctx();
  t->c.device = device;
  t->c.stream = (cudaStream_t)stream;
  t->c.dalloc = a;
  tnt_params_default(&t->c.params);
  void* st = nullptr;
  if (dev_alloc(a, &st, 256) != 0) {
    delete t;
    return a.alloc ? TNT_E_ALLOC : TNT_E_CUDA;
  }
  t->c.d_status = (int*)st;
  void* cnt = nullptr;
  if (dev_alloc(a, &cnt, 256) != 0) {
    dev_free(a, st);
    delete t;
    return a.alloc ? TNT_E_ALLOC : TNT_E_CUDA;
  }
  t->c.d_count = (unsigned*)cnt;
  cudaMemsetAsync(t->c.d_status, 0, 256, t->c.stream);
  cudaMemsetAsync(t->c.d_count, 0, 256, t->c.stream);
  if (pinned_reserve(&t->c, 4096) != TNT_OK || cudaStreamSynchronize(t->c.stream) != cudaSuccess) {
    dev_free(a, t->c.d_status);
    dev_free(a, t->c.d_count);
    delete t;
    return TNT_E_ALLOC;
  }
  *out = t;
  return TNT_OK;
}

int tnt_ctx_create(int device, void* stream, tnt_ctx** out) {
  return ctx_create(device, stream, DevAlloc{}, out);
}

int tnt_ctx_create_with_allocator(int device, void* stream, const tnt_allocator* alloc,
                                  tnt_ctx** out) {
  if (!out) return TNT_E_INVALID;
  *out = nullptr;
  if (!alloc || !alloc->alloc || !alloc->free) return TNT_E_INVALID;
  DevAlloc a;
  a.alloc = alloc->alloc;
  a.free = alloc->free;
  a.user = alloc->user;
  return ctx_create(device, stream, a, out);
}

int tnt_ctx_destroy(tnt_ctx* ctx) {
  if (!ctx) return TNT_E_INVALID;
  cudaStreamSynchronize(ctx->c.stream);
  if (ctx->c.side) {
    cudaStreamSynchronize(ctx->c.side);
    cudaStreamDestroy(ctx->c.side);
    for (int i = 0; i < 2; ++i) {
      cudaEventDestroy(ctx->c.ev_main[i]);
      cudaEventDestroy(ctx->c.ev_side[i]);
    }
  }
  for (auto& e : ctx->c.prof_ev) cudaEventDestroy(e);
  dev_free(ctx->c.dalloc, ctx->c.ws.base);
  if (ctx->c.h_pinned) cudaFreeHost(ctx->c.h_pinned);
  dev_free(ctx->c.dalloc, ctx->c.d_status);
  dev_free(ctx->c.dalloc, ctx->c.d_count);
  dev_free(ctx->c.dalloc, ctx->c.oz_buf);
  delete ctx;
  return TNT_OK;
}

int tnt_set_stream(tnt_ctx* ctx, void* stream) {
  CTX_CHECK(ctx);
  ctx->c.stream = (cudaStream_t)stream;
  return TNT_OK;
}

const char* tnt_last_error(const tnt_ctx* ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

int64_t tnt_launch_count(const tnt_ctx* ctx) { return ctx ? ctx->c.launches : -1; }

int tnt_profile_select(tnt_ctx* ctx, const char* cls) {
  CTX_CHECK(ctx);
  Ctx* c = &ctx->c;
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->prof_n = 0;
  c->prof_work = 0;
  c->prof_cls = cls ? cls : "";
  if (!c->prof_cls.empty() && c->prof_ev.empty()) {
    c->prof_ev.resize(2 * 16384);
    for (auto& e : c->prof_ev) TNT_CUDA_TRY(c, cudaEventCreate(&e));
  }
  return TNT_OK;
}

int tnt_profile_read(tnt_ctx* ctx, double* total_ms, int64_t* launches, double* work) {
  CTX_CHECK(ctx);
  ARG_CHECK(ctx, total_ms && launches && work, "null pointer");
  Ctx* c = &ctx->c;
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  double t = 0;
  for (size_t i = 0; i < c->prof_n; ++i) {
    float ms = 0;
    TNT_CUDA_TRY(c, cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]));
    t += ms;
  }
  *total_ms = t;
  *launches = (int64_t)c->prof_n;
  *work = c->prof_work;
  c->prof_n = 0;
  c->prof_work = 0;
  return TNT_OK;
}

int tnt_params_set(tnt_ctx* ctx, const tnt_params* p) {
  CTX_CHECK(ctx);
  ARG_CHECK(ctx, p, "null params");
  ARG_CHECK(ctx, p->chi_max >= 1, "chi_max must be >= 1");
  ARG_CHECK(ctx, p->trunc_type >= 0 && p->trunc_type <= 2, "bad trunc_type %d", p->trunc_type);
  ARG_CHECK(ctx, p->krylov_cap >= 2 && p->krylov_cap <= 64, "krylov_cap must be in [2, 64]");
  ARG_CHECK(ctx, p->lanczos_maxit >= 1, "lanczos_maxit must be >= 1");
  ARG_CHECK(ctx, p->precision == TNT_PREC_FP64 || p->precision == TNT_PREC_MIXED, "bad precision");
  ctx->c.params = *p;
  return TNT_OK;
}

int tnt_params_get(const tnt_ctx* ctx, tnt_params* p) {
  if (!ctx || !p) return TNT_E_INVALID;
  *p = ctx->c.params;
  return TNT_OK;
}

int tnt_sys_info(const tnt_ctx* ctx, char* buf, size_t n) {
  if (!ctx || !buf || n == 0) return TNT_E_INVALID;
  const tnt_params& p = ctx->c.params;
  const char* tt = p.trunc_type == TNT_TRUNC_2NORM ? "2norm" : p.trunc_type == TNT_TRUNC_SUMSQ ? "sumsq" : "1norm";
  snprintf(buf, n,
           "------------- System Information -------------\n"
           "Symmetry type: U(1) boson number (per call, optional).\n"
           "Basis operator: boson number n.\n"
           "Relative truncation tolerance is %g.\n"
           "Absolute truncation tolerance is %g.\n"
           "Truncation error tolerance is %g.\n"
           "Tolerance for automatic blocking is %g.\n"
           "Current truncation type is %s.\n"
           "SVD type is FP64 Gram plus tridiagonal eigensolver (GPU).\n"
           "Maximum bond dimension is %lld.\n"
           "Maximum number of iterations for eigenvalue solver is %d.\n"
           "Krylov vectors before restart: %d; eigensolver tolerance %g.\n"
           "H_eff precision: %s.\n",
           p.trunc_rel, p.trunc_abs, p.trunc_err, ctx->c.svd_zero_tol, tt, (long long)p.chi_max, p.lanczos_maxit,
           p.krylov_cap, p.lanczos_tol, p.precision == TNT_PREC_MIXED ? "split TF32 (tcgen05)" : "FP64");
  return TNT_OK;
}

int tnt_bh_mpo_site(int n_max, double J, double U, double mu, double V, double j, double j_c,
                    tnt_cplx* h_W) {
  if (n_max < 0 || !h_W || !all_finite({J, U, mu, V, j, j_c})) return TNT_E_INVALID;
  return bh_mpo_site_host(n_max, J, U, mu, V, j, j_c, (z*)h_W);
}

int tnt_spin_mpo_site(int two_s, double J, double Jz, double hz, tnt_cplx* h_W) {
  if (two_s < 1 || two_s > 15 || !h_W || !all_finite({J, Jz, hz})) return TNT_E_INVALID;
  return spin_mpo_site_host(two_s, J, Jz, hz, (z*)h_W);
}

int tnt_spin_bond_h(int two_s, double J, double Jz, double hz, double c1, double c2,
                    tnt_cplx* h_h) {
  if (two_s < 1 || two_s > 15 || !h_h || !all_finite({J, Jz, hz, c1, c2})) return TNT_E_INVALID;
  return spin_bond_h_host(two_s, J, Jz, hz, c1, c2, (z*)h_h);
}

int tnt_bond_gate(int n, const tnt_cplx* h_h, double tau, tnt_cplx* h_G) {
  if (n < 1 || n > 256 || !h_h || !h_G || !std::isfinite(tau)) return TNT_E_INVALID;
  for (int64_t i = 0; i < (int64_t)n * n; ++i)
    if (!std::isfinite(h_h[i].re) || !std::isfinite(h_h[i].im)) return TNT_E_INVALID;
  return bond_gate_host(n, (const z*)h_h, tau, (z*)h_G);
}

int tnt_bh_bond_gate(int n_max, double J, double U, double mu, double c1, double c2, double tau,
                     tnt_cplx* h_G) {
  if (n_max < 0 || !h_G || !all_finite({J, U, mu, c1, c2, tau})) return TNT_E_INVALID;
  return bh_bond_gate_host(n_max, J, U, mu, c1, c2, tau, (z*)h_G);
}

int tnt_theta_form(tnt_ctx* ctx, const tnt_cplx* d_A, const tnt_cplx* d_B, int64_t chl, int64_t d,
                   int64_t chm, int64_t chr, tnt_cplx* d_theta) {
  CTX_CHECK(ctx);
  ARG_CHECK(ctx, d_A && d_B && d_theta, "null pointer");
  ARG_CHECK(ctx, chl > 0 && d > 0 && chm > 0 && chr > 0, "non-positive dimension");
  Scope s(&ctx->c);
  return theta_form_impl(&ctx->c, (const z*)d_A, (const z*)d_B, chl, d, chm, chr, (z*)d_theta);
}

int tnt_gate_apply(tnt_ctx* ctx, const tnt_cplx* d_G, const tnt_cplx* d_theta, int64_t chl,
                   int64_t d, int64_t chr, tnt_cplx* d_out) {
  CTX_CHECK(ctx);
  ARG_CHECK(ctx, d_G && d_theta && d_out && d_out != d_theta, "null or aliased pointer");
  ARG_CHECK(ctx, chl > 0 && d > 0 && chr > 0 && d * d <= 256, "bad dimension");
  Scope s(&ctx->c);
  TNT_TRY(ws_reserve(&ctx->c, 1 << 20));
  std::vector<z> G((size_t)(d * d * d * d));
  TNT_TRY(read_small(&ctx->c, d_G, G.data(), G.size() * sizeof(z)));
  return gate_apply_impl(&ctx->c, G, (const z*)d_theta, chl, d, chr, (z*)d_out);
}

int tnt_heff_apply(tnt_ctx* ctx, const tnt_cplx* d_L, const tnt_cplx* d_W1, const tnt_cplx* d_W2,
                   const tnt_cplx* d_R, const tnt_cplx* d_theta, int64_t chl, int64_t d, int64_t D,
                   int64_t chr, int precision, tnt_cplx* d_y) {
  CTX_CHECK(ctx);
  ARG_CHECK(ctx, d_L && d_W1 && d_W2 && d_R && d_theta && d_y, "null pointer");
  ARG_CHECK(ctx, d_y != d_theta, "d_y aliases d_theta");
  ARG_CHECK(ctx, chl > 0 && d > 0 && D > 0 && chr > 0, "non-positive dimension");
  ARG_CHECK(ctx, precision == TNT_PREC_FP64 || precision == TNT_PREC_MIXED, "bad precision");
  ARG_CHECK(ctx, d * d * D <= 256, "d^2 D = %lld exceeds 256", (long long)(d * d * D));
  Ctx* c = &ctx->c;
  Scope s(c);
  TNT_TRY(ws_reserve(c, heff_scratch_bound(chl, d, D, chr, precision)));
  HeffPlan p;
  TNT_TRY(heff_prepare(c, (const z*)d_L, (const z*)d_W1, (const z*)d_W2, (const z*)d_R, chl, d, D,
                       chr, precision, &p));
  return heff_run(c, p, (const z*)d_theta, (z*)d_y, precision);
}

int tnt_env_left(tnt_ctx* ctx, const tnt_cplx* d_L, const tnt_cplx* d_W, const tnt_cplx* d_A,
                 int64_t chl, int64_t d, int64_t D, int64_t chr, tnt_cplx* d_Lout) {
  CTX_CHECK(ctx);
  ARG_CHECK(ctx, d_L && d_W && d_A && d_Lout, "null pointer");
  ARG_CHECK(ctx, chl > 0 && d > 0 && D > 0 && chr > 0 && d * D <= 256, "bad dimension");
  Scope s(&ctx->c);
  TNT_TRY(ws_reserve(&ctx->c, env_scratch_bound(chl, d, D, chr)));
  return env_left_impl(&ctx->c, (const z*)d_L, (const z*)d_W, (const z*)d_A, chl, d, D, chr,
                       (z*)d_Lout);
}

int tnt_env_right(tnt_ctx* ctx, const tnt_cplx* d_R, const tnt_cplx* d_W, const tnt_cplx* d_B,
                  int64_t chl, int64_t d, int64_t D, int64_t chr, tnt_cplx* d_Rout) {
  CTX_CHECK(ctx);
  ARG_CHECK(ctx, d_R && d_W && d_B && d_Rout, "null pointer");
  ARG_CHECK(ctx, chl > 0 && d > 0 && D > 0 && chr > 0 && d * D <= 256, "bad dimension");
  Scope s(&ctx->c);
  TNT_TRY(ws_reserve(&ctx->c, env_scratch_bound(chl, d, D, chr)));
  return env_right_impl(&ctx->c, (const z*)d_R, (const z*)d_W, (const z*)d_B, chl, d, D, chr,
                        (z*)d_Rout);
}

int tnt_lanczos_ground(tnt_ctx* ctx, const tnt_cplx* d_L, const tnt_cplx* d_W1,
                       const tnt_cplx* d_W2, const tnt_cplx* d_R, int64_t chl, int64_t d,
                       int64_t D, int64_t chr, tnt_cplx* d_theta, tnt_lanczos_result* res) {
  CTX_CHECK(ctx);
  ARG_CHECK(ctx, d_L && d_W1 && d_W2 && d_R && d_theta && res, "null pointer");
  ARG_CHECK(ctx, chl > 0 && d > 0 && D > 0 && chr > 0 && d * d * D <= 256, "bad dimension");
  Ctx* c = &ctx->c;
  Scope s(c);
  const int64_t n = chl * d * d * chr;
  TNT_TRY(ws_reserve(c, heff_scratch_bound(chl, d, D, chr, c->params.precision) +
                            lanczos_scratch_bound(n, c->params.krylov_cap)));
  HeffPlan p;
  TNT_TRY(heff_prepare(c, (const z*)d_L, (const z*)d_W1, (const z*)d_W2, (const z*)d_R, chl, d, D,
                       chr, c->params.precision, &p));
  return lanczos_impl(c, p, (z*)d_theta, res);
}

int tnt_set_svd_zero_tol(tnt_ctx* ctx, double tol) {
  CTX_CHECK(ctx);
  ARG_CHECK(ctx, !std::isnan(tol), "tolerance is NaN");
  ctx->c.svd_zero_tol = tol < 0 ? -1.0 : tol;
  return TNT_OK;
}

int tnt_svd_trunc(tnt_ctx* ctx, const tnt_cplx* d_M, int64_t m, int64_t n, const int64_t* h_row_q,
                  const int64_t* h_col_q, int side, int renorm, tnt_cplx* d_U, tnt_cplx* d_X,
                  double* h_S, int64_t* h_bond_q, tnt_trunc_result* res) {
  CTX_CHECK(ctx);
  ARG_CHECK(ctx, d_M && d_U && d_X && h_S && h_bond_q && res, "null pointer");
  ARG_CHECK(ctx, m > 0 && n > 0, "non-positive dimension");
  ARG_CHECK(ctx, (h_row_q == nullptr) == (h_col_q == nullptr), "give both charge arrays or neither");
  ARG_CHECK(ctx, side == TNT_SVD_LEFT || side == TNT_SVD_RIGHT, "bad side");
  Scope s(&ctx->c);
  return svd_trunc_impl(&ctx->c, (const z*)d_M, m, n, h_row_q, h_col_q, side, renorm, (z*)d_U,
                        (z*)d_X, h_S, h_bond_q, res);
}

}  // extern "C"
