// Lanczos ground states of several independent problems in lock step (the eigensolver of
// Sec. 4.3 run for many chains at once).  The problems' vectors lie back to back; each
// Krylov step applies one grouped matvec to all of them and then runs the same FP64
// recurrence as the single-problem solver (classical Gram-Schmidt applied twice, beta_k,
// lowest eigenpair of T_k, stop rule) with every inner product,
// norm and scalar kept per problem: the vector kernels work on chunks that never cross a
// problem boundary and reduce per problem in a fixed order.  A problem that has converged
// is frozen (its chunks, scalars and tridiagonal solves are skipped) while the others go
// on; restarts after krylov_cap steps and the FP64 win-back of the split-TF32 path are
// per problem as well.
#include <algorithm>
#include <cmath>
#include <vector>

#include "heff_plan.cuh"
#include "f32conv.cuh"

namespace tnt {

namespace {
constexpr int ST = 256;  // threads per chunk block
constexpr int SKB = 8;   // vectors per dot pass
constexpr int KMAX = 64; // Krylov vectors per problem (stride of the per-problem scalars)

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double bsum(double v, double* sh) {
  v = wsum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0;
  if (w == 0) {
    r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    r = wsum(r);
  }
  __syncthreads();
  return r;
}

// chunk b covers [ch[3b+1], ch[3b+2]) of problem ch[3b]
template <int KV>
__global__ void __launch_bounds__(ST) k_sdot(const z* __restrict__ V, int64_t ld,
                                             const z* __restrict__ w, const int64_t* __restrict__ ch,
                                             int nch, z* __restrict__ partial,
                                             const int* __restrict__ skip) {
  const int b = blockIdx.x;
  const int p = (int)ch[3 * b];
  if (skip[p]) return;
  __shared__ double sh[32];
  double ar[KV], ai[KV];
#pragma unroll
  for (int v = 0; v < KV; ++v) ar[v] = ai[v] = 0.0;
  for (int64_t e = ch[3 * b + 1] + threadIdx.x; e < ch[3 * b + 2]; e += blockDim.x) {
    const z x = w[e];
    z u[KV];
#pragma unroll
    for (int v = 0; v < KV; ++v) u[v] = V[(int64_t)v * ld + e];
#pragma unroll
    for (int v = 0; v < KV; ++v) {
      ar[v] = fma(u[v].x, x.x, fma(u[v].y, x.y, ar[v]));
      ai[v] = fma(u[v].x, x.y, fma(-u[v].y, x.x, ai[v]));
    }
  }
#pragma unroll
  for (int v = 0; v < KV; ++v) {
    const double r = bsum(ar[v], sh), i = bsum(ai[v], sh);
    if (threadIdx.x == 0) partial[(int64_t)v * nch + b] = zmk(r, i);
  }
}

// dots[p * KMAX + v0 + v] = sum of problem p's chunk partials, in chunk order
__global__ void k_sreduce_dots(const z* __restrict__ partial, int nch, const int* __restrict__ first,
                               int kv, int v0, z* __restrict__ dots, const int* __restrict__ skip) {
  const int p = blockIdx.x;
  if (skip[p]) return;
  __shared__ double sh[32];
  for (int v = 0; v < kv; ++v) {
    double r = 0, i = 0;
    for (int b = first[p] + threadIdx.x; b < first[p + 1]; b += blockDim.x) {
      const z q = partial[(int64_t)v * nch + b];
      r += q.x;
      i += q.y;
    }
    r = bsum(r, sh);
    i = bsum(i, sh);
    if (threadIdx.x == 0) dots[p * KMAX + v0 + v] = zmk(r, i);
  }
}

// w -= sum_v coef[p][v] V_v on problem p's chunks; partial[b] = |w|^2 over the chunk
// (kper, if given, caps k per problem: vectors beyond a problem's own count are never read)
__global__ void __launch_bounds__(ST) k_saxpy_norm(const z* __restrict__ V, int64_t ld, int k,
                                                   const z* __restrict__ coef, z* __restrict__ w,
                                                   const int64_t* __restrict__ ch,
                                                   double* __restrict__ partial,
                                                   const int* __restrict__ skip,
                                                   const int* __restrict__ kper) {
  const int b = blockIdx.x;
  const int p = (int)ch[3 * b];
  if (skip[p]) return;
  if (kper) k = min(k, kper[p]);
  __shared__ z sc[KMAX];
  __shared__ double sh[32];
  for (int t = threadIdx.x; t < k; t += blockDim.x) sc[t] = coef[p * KMAX + t];
  __syncthreads();
  double acc = 0;
  for (int64_t e = ch[3 * b + 1] + threadIdx.x; e < ch[3 * b + 2]; e += blockDim.x) {
    z x = w[e];
    int v = 0;
    for (; v + 8 <= k; v += 8) {
      z u[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) u[q] = V[(int64_t)(v + q) * ld + e];
#pragma unroll
      for (int q = 0; q < 8; ++q) {  // x -= cv u as four FMAs
        const z cv = sc[v + q];
        x.x = fma(-cv.x, u[q].x, fma(cv.y, u[q].y, x.x));
        x.y = fma(-cv.x, u[q].y, fma(-cv.y, u[q].x, x.y));
      }
    }
    for (; v < k; ++v) {
      const z u = V[(int64_t)v * ld + e];
      const z cv = sc[v];
      x.x = fma(-cv.x, u.x, fma(cv.y, u.y, x.x));
      x.y = fma(-cv.x, u.y, fma(-cv.y, u.x, x.y));
    }
    w[e] = x;
    acc = fma(x.x, x.x, fma(x.y, x.y, acc));
  }
  const double s = bsum(acc, sh);
  if (threadIdx.x == 0) partial[b] = s;
}

// The same two passes in FP32 arithmetic on the FP64 vectors (the products, the sums per
// thread, warp and chunk; FP64 sums over a problem's chunks and FP64 subtraction from w):
// for the Gram-Schmidt passes of a split-TF32 phase, whose matvec error (~2^-22) is above
// this rounding, and which in FP64 are bound by GB300's FP64 pipe
template <int KV>
__global__ void __launch_bounds__(ST) k_sdot32(const z* __restrict__ V, int64_t ld,
                                               const z* __restrict__ w, const int64_t* __restrict__ ch,
                                               int nch, z* __restrict__ partial,
                                               const int* __restrict__ skip) {
  const int b = blockIdx.x;
  const int p = (int)ch[3 * b];
  if (skip[p]) return;
  float ar[KV], ai[KV];
#pragma unroll
  for (int v = 0; v < KV; ++v) ar[v] = ai[v] = 0.f;
  for (int64_t e = ch[3 * b + 1] + threadIdx.x; e < ch[3 * b + 2]; e += blockDim.x) {
    const z xd = w[e];
    z u[KV];
#pragma unroll
    for (int v = 0; v < KV; ++v) u[v] = V[(int64_t)v * ld + e];
    const float xr = f32_of(xd.x), xi = f32_of(xd.y);
#pragma unroll
    for (int v = 0; v < KV; ++v) {  // conj(u) x
      const float ur = f32_of(u[v].x), ui = f32_of(u[v].y);
      ar[v] = fmaf(ur, xr, fmaf(ui, xi, ar[v]));
      ai[v] = fmaf(ur, xi, fmaf(-ui, xr, ai[v]));
    }
  }
  __shared__ float shp[ST / 32][2 * KV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < KV; ++v) {
    ar[v] = warp_sum_f(ar[v]);
    ai[v] = warp_sum_f(ai[v]);
  }
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < KV; ++v) {
      shp[wid][2 * v] = ar[v];
      shp[wid][2 * v + 1] = ai[v];
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * KV) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < ST / 32; ++q) t += shp[q][threadIdx.x];
    ((double*)(partial + (int64_t)(threadIdx.x >> 1) * nch + b))[threadIdx.x & 1] = f64_of(t);
  }
}

__global__ void __launch_bounds__(ST) k_saxpy_norm32(const z* __restrict__ V, int64_t ld, int k,
                                                     const z* __restrict__ coef, z* __restrict__ w,
                                                     const int64_t* __restrict__ ch,
                                                     double* __restrict__ partial,
                                                     const int* __restrict__ skip) {
  const int b = blockIdx.x;
  const int p = (int)ch[3 * b];
  if (skip[p]) return;
  __shared__ float2 sc[KMAX];
  __shared__ float shw[ST / 32];
  for (int t = threadIdx.x; t < k; t += blockDim.x)
    sc[t] = make_float2(f32_of(coef[p * KMAX + t].x), f32_of(coef[p * KMAX + t].y));
  __syncthreads();
  float acc = 0.f;
  for (int64_t e = ch[3 * b + 1] + threadIdx.x; e < ch[3 * b + 2]; e += blockDim.x) {
    float sr = 0.f, si = 0.f;
    int v = 0;
    for (; v + 8 <= k; v += 8) {
      z u[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) u[q] = V[(int64_t)(v + q) * ld + e];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float2 cv = sc[v + q];
        const float ur = f32_of(u[q].x), ui = f32_of(u[q].y);
        sr = fmaf(cv.x, ur, fmaf(-cv.y, ui, sr));
        si = fmaf(cv.x, ui, fmaf(cv.y, ur, si));
      }
    }
    for (; v < k; ++v) {
      const z u = V[(int64_t)v * ld + e];
      const float2 cv = sc[v];
      const float ur = f32_of(u.x), ui = f32_of(u.y);
      sr = fmaf(cv.x, ur, fmaf(-cv.y, ui, sr));
      si = fmaf(cv.x, ui, fmaf(cv.y, ur, si));
    }
    z x = w[e];
    x.x -= f64_of(sr);
    x.y -= f64_of(si);
    w[e] = x;
    const float xr = f32_of(x.x), xi = f32_of(x.y);
    acc = fmaf(xr, xr, fmaf(xi, xi, acc));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  acc = warp_sum_f(acc);
  if (lane == 0) shw[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < ST / 32; ++q) t += shw[q];
    partial[b] = f64_of(t);
  }
}

__global__ void __launch_bounds__(ST) k_snorm2(const z* __restrict__ x, const int64_t* __restrict__ ch,
                                               double* __restrict__ partial, const int* __restrict__ skip) {
  const int b = blockIdx.x;
  if (skip[(int)ch[3 * b]]) return;
  __shared__ double sh[32];
  double acc = 0;
  for (int64_t e = ch[3 * b + 1] + threadIdx.x; e < ch[3 * b + 2]; e += blockDim.x) {
    const z v = x[e];
    acc = fma(v.x, v.x, fma(v.y, v.y, acc));
  }
  const double s = bsum(acc, sh);
  if (threadIdx.x == 0) partial[b] = s;
}

__global__ void k_sreduce_real(const double* __restrict__ partial, const int* __restrict__ first,
                               double* __restrict__ out, const int* __restrict__ skip) {
  const int p = blockIdx.x;
  if (skip[p]) return;
  __shared__ double sh[32];
  double r = 0;
  for (int b = first[p] + threadIdx.x; b < first[p + 1]; b += blockDim.x) r += partial[b];
  r = bsum(r, sh);
  if (threadIdx.x == 0) out[p] = r;
}

// y = x / sqrt(norm2[p]) on problem p's chunks (zero if the norm vanished)
__global__ void __launch_bounds__(ST) k_snormalize(const z* __restrict__ x, z* __restrict__ y,
                                                   const int64_t* __restrict__ ch,
                                                   const double* __restrict__ norm2,
                                                   const int* __restrict__ skip) {
  const int b = blockIdx.x;
  const int p = (int)ch[3 * b];
  if (skip[p]) return;
  __shared__ double s_s;  // by one thread: the FP64 square root and division outweigh the chunk's scaling
  if (threadIdx.x == 0) s_s = norm2[p] > 0.0 ? 1.0 / sqrt(norm2[p]) : 0.0;
  __syncthreads();
  const double s = s_s;
  for (int64_t e = ch[3 * b + 1] + threadIdx.x; e < ch[3 * b + 2]; e += blockDim.x) y[e] = zscale(x[e], s);
}

// r = Hx - E x on problem p's chunks (E = Re dot[p])
__global__ void __launch_bounds__(ST) k_sresid(const z* __restrict__ Hx, const z* __restrict__ x,
                                               const z* __restrict__ dot, z* __restrict__ r,
                                               const int64_t* __restrict__ ch,
                                               const int* __restrict__ skip) {
  const int b = blockIdx.x;
  const int p = (int)ch[3 * b];
  if (skip[p]) return;
  const double e = dot[p * KMAX].x;
  for (int64_t i = ch[3 * b + 1] + threadIdx.x; i < ch[3 * b + 2]; i += blockDim.x)
    r[i] = zsub(Hx[i], zscale(x[i], e));
}

__global__ void k_sfill(z* __restrict__ w, const int64_t* __restrict__ ch, const int* __restrict__ skip) {
  const int b = blockIdx.x;
  if (skip[(int)ch[3 * b]]) return;
  for (int64_t e = ch[3 * b + 1] + threadIdx.x; e < ch[3 * b + 2]; e += blockDim.x) w[e] = zmk(0, 0);
}

// per problem: alpha_k = Re dots[k], beta_k = sqrt(norm2) (also to bk[p] for read-back)
__global__ void k_sscalars(const z* __restrict__ dots, int k, const double* __restrict__ norm2,
                           double* __restrict__ alpha, double* __restrict__ beta,
                           double* __restrict__ bk, int P, const int* __restrict__ skip) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P || skip[p]) return;
  alpha[p * KMAX + k] = dots[p * KMAX + k].x;
  beta[p * KMAX + k] = sqrt(norm2[p]);
  bk[p] = beta[p * KMAX + k];
}
// Ritz coefficients: coef[p][i] = -y[p][i] for i < kk[p], zero beyond
__global__ void k_sritz(const double* __restrict__ y, const int* __restrict__ kk, z* __restrict__ coef,
                        int P) {
  const int p = blockIdx.x;
  if (p >= P) return;
  for (int i = threadIdx.x; i < KMAX; i += blockDim.x) coef[p * KMAX + i] = zmk(i < kk[p] ? -y[p * KMAX + i] : 0.0, 0.0);
}

template <int KV>
void launch_sdot(int nch, cudaStream_t st, const z* V, int64_t ld, const z* w, const int64_t* ch, z* part,
                 const int* skip) {
  k_sdot<KV><<<nch, ST, 0, st>>>(V, ld, w, ch, nch, part, skip);
}
void sdot_kv(int kv, int nch, cudaStream_t st, const z* V, int64_t ld, const z* w, const int64_t* ch,
             z* part, const int* skip) {
  switch (kv) {
    case 1: launch_sdot<1>(nch, st, V, ld, w, ch, part, skip); break;
    case 2: launch_sdot<2>(nch, st, V, ld, w, ch, part, skip); break;
    case 3: launch_sdot<3>(nch, st, V, ld, w, ch, part, skip); break;
    case 4: launch_sdot<4>(nch, st, V, ld, w, ch, part, skip); break;
    case 5: launch_sdot<5>(nch, st, V, ld, w, ch, part, skip); break;
    case 6: launch_sdot<6>(nch, st, V, ld, w, ch, part, skip); break;
    case 7: launch_sdot<7>(nch, st, V, ld, w, ch, part, skip); break;
    default: launch_sdot<8>(nch, st, V, ld, w, ch, part, skip); break;
  }
}

void sdot32_kv(int kv, int nch, cudaStream_t st, const z* V, int64_t ld, const z* w,
               const int64_t* ch, z* part, const int* skip) {
  switch (kv) {
    case 1: k_sdot32<1><<<nch, ST, 0, st>>>(V, ld, w, ch, nch, part, skip); break;
    case 2: k_sdot32<2><<<nch, ST, 0, st>>>(V, ld, w, ch, nch, part, skip); break;
    case 3: k_sdot32<3><<<nch, ST, 0, st>>>(V, ld, w, ch, nch, part, skip); break;
    case 4: k_sdot32<4><<<nch, ST, 0, st>>>(V, ld, w, ch, nch, part, skip); break;
    case 5: k_sdot32<5><<<nch, ST, 0, st>>>(V, ld, w, ch, nch, part, skip); break;
    case 6: k_sdot32<6><<<nch, ST, 0, st>>>(V, ld, w, ch, nch, part, skip); break;
    case 7: k_sdot32<7><<<nch, ST, 0, st>>>(V, ld, w, ch, nch, part, skip); break;
    default: k_sdot32<8><<<nch, ST, 0, st>>>(V, ld, w, ch, nch, part, skip); break;
  }
}

// device scratch of one batched solve
struct BScratch {
  int P = 0, nch = 0;
  int64_t n = 0;
  int64_t* ch = nullptr;
  int* first = nullptr;
  z* V = nullptr;  // KMAX-capped basis: cap x n
  z* w = nullptr;
  z* w2 = nullptr;
  z* part = nullptr;      // SKB x nch
  double* rpart = nullptr;  // nch
  z* dots = nullptr;      // P x KMAX
  z* coef = nullptr;      // P x KMAX
  double *alpha = nullptr, *beta = nullptr, *y = nullptr, *tri = nullptr;  // P x KMAX, tri 3 P
  double *n2 = nullptr;  // P
  int *frozen = nullptr, *skip2 = nullptr, *kk = nullptr, *done = nullptr;  // P
  int* none = nullptr;    // P zeros
  double* h = nullptr;    // pinned: tri (2P) + beta_k (P)
};

// dots[p][v] = <B_v | w> over problem p for v < k, B_v = basis + v * n
// (f32: FP32 arithmetic, the Gram-Schmidt passes of a split-TF32 phase)
int sdots(Ctx* c, BScratch& s, const z* basis, int k, const z* w, z* dots_out, const int* skip,
          bool f32 = false) {
  for (int v0 = 0; v0 < k; v0 += SKB) {
    const int kv = std::min(SKB, k - v0);
    const bool all = skip == s.frozen || skip == s.none;
    if (f32) {
      ProfScope ps(c, all ? "multidot32" : "multidot_cond", all ? 16.0 * (double)(kv + 1) * (double)s.n : 0.0);
      sdot32_kv(kv, s.nch, c->stream, basis + (int64_t)v0 * s.n, s.n, w, s.ch, s.part, skip);
    } else {
      ProfScope ps(c, all ? "multidot" : "multidot_cond", all ? 8.0 * (double)kv * (double)s.n : 0.0);
      sdot_kv(kv, s.nch, c->stream, basis + (int64_t)v0 * s.n, s.n, w, s.ch, s.part, skip);
    }
    k_sreduce_dots<<<s.P, 256, 0, c->stream>>>(s.part, s.nch, s.first, kv, v0, dots_out, skip);
    c->launches += 2;
  }
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}
int saxpy(Ctx* c, BScratch& s, int k, const z* coef, z* w, double* norm2, const int* skip,
          const int* kper = nullptr, bool f32 = false) {
  const bool all = skip == s.frozen || skip == s.none;
  if (f32 && !kper) {
    ProfScope ps(c, all ? "multiaxpy32" : "multiaxpy_cond", all ? 16.0 * ((double)k + 2.0) * (double)s.n : 0.0);
    k_saxpy_norm32<<<s.nch, ST, 0, c->stream>>>(s.V, s.n, k, coef, w, s.ch, s.rpart, skip);
  } else {
    ProfScope ps(c, all ? "multiaxpy" : "multiaxpy_cond",
                 all ? (8.0 * (double)k + 4.0) * (double)s.n : 0.0);
    k_saxpy_norm<<<s.nch, ST, 0, c->stream>>>(s.V, s.n, k, coef, w, s.ch, s.rpart, skip, kper);
  }
  k_sreduce_real<<<s.P, 256, 0, c->stream>>>(s.rpart, s.first, norm2, skip);
  c->launches += 2;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}
int snorm2(Ctx* c, BScratch& s, const z* x, double* norm2, const int* skip) {
  k_snorm2<<<s.nch, ST, 0, c->stream>>>(x, s.ch, s.rpart, skip);
  k_sreduce_real<<<s.P, 256, 0, c->stream>>>(s.rpart, s.first, norm2, skip);
  c->launches += 2;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}
int snormalize(Ctx* c, BScratch& s, const z* x, z* y, const double* norm2, const int* skip) {
  k_snormalize<<<s.nch, ST, 0, c->stream>>>(x, y, s.ch, norm2, skip);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

// Krylov cycles for every problem not yet done (done[p] on entry: skip entirely).
// x: in start vectors, out Ritz vectors of the problems that ran.
// resid_only: a split-TF32 phase that an FP64 continuation follows stops on the residual
// test alone (as in the single-problem solver)
int cycles(Ctx* c, const MatVec& A, BScratch& s, z* x, int precision, int max_matvec,
           std::vector<int>& done, std::vector<tnt_lanczos_result>& res, bool resid_only = false) {
  const tnt_params& P = c->params;
  const int cap = P.krylov_cap, NP = s.P;
  const double u = (precision == TNT_PREC_MIXED) ? std::ldexp(1.0, -22) : std::ldexp(1.0, -52);
  const double tol = P.lanczos_tol, rtol = std::max(tol, 10.0 * u);
  // Gram-Schmidt in FP32 arithmetic while the matvec is split TF32 (the Ritz vectors are
  // assembled in FP64)
  const bool f32_gs = (precision == TNT_PREC_MIXED);
  std::vector<int> frozen(done), total((size_t)NP, 0), kk((size_t)NP, 0), conv((size_t)NP, 0);
  std::vector<double> E((size_t)NP, 0), Eprev((size_t)NP, 0), resid((size_t)NP, 0);
  std::vector<int> have_prev((size_t)NP, 0);
  auto push_frozen = [&]() -> int {
    TNT_CUDA_TRY(c, cudaMemcpyAsync(s.frozen, frozen.data(), sizeof(int) * NP, cudaMemcpyHostToDevice, c->stream));
    TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return TNT_OK;
  };
  TNT_TRY(push_frozen());
  // v_0 = x / |x| per problem
  TNT_TRY(snorm2(c, s, x, s.n2, s.frozen));
  TNT_TRY(snormalize(c, s, x, s.V, s.n2, s.frozen));
  int running = 0;
  for (int p = 0; p < NP; ++p) running += frozen[(size_t)p] ? 0 : 1;
  int mv = 0;
  while (running > 0) {
    std::vector<int> active_in_cycle(frozen);  // 0 where the problem takes part
    int k = 0;
    for (; k < cap; ++k) {
      TNT_TRY(A.apply(c, s.V + (int64_t)k * s.n, s.w, precision));
      ++mv;
      TNT_TRY(sdots(c, s, s.V, k + 1, s.w, s.dots, s.frozen, f32_gs));
      TNT_TRY(saxpy(c, s, k + 1, s.dots, s.w, s.n2, s.frozen, nullptr, f32_gs));
      k_sscalars<<<(NP + 63) / 64, 64, 0, c->stream>>>(s.dots, k, s.n2, s.alpha, s.beta, s.tri + 2 * NP, NP, s.frozen);
      c->launches += 1;
      TNT_TRY(sdots(c, s, s.V, k + 1, s.w, s.coef, s.frozen, f32_gs));  // second pass, always
      TNT_TRY(saxpy(c, s, k + 1, s.coef, s.w, s.n2, s.frozen, nullptr, f32_gs));
      k_sscalars<<<(NP + 63) / 64, 64, 0, c->stream>>>(s.dots, k, s.n2, s.alpha, s.beta, s.tri + 2 * NP, NP, s.frozen);
      c->launches++;
      TNT_TRY(tridiag_lowest_batched(c, s.alpha, s.beta, k + 1, s.tri, s.y, NP, s.frozen));
      TNT_CUDA_TRY(c, cudaMemcpyAsync(s.h, s.tri, sizeof(double) * 3 * NP, cudaMemcpyDeviceToHost, c->stream));
      TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      bool changed = false;
      for (int p = 0; p < NP; ++p) {
        if (frozen[(size_t)p]) continue;
        total[(size_t)p]++;
        const double e = s.h[2 * p], yk = s.h[2 * p + 1], bk = s.h[2 * NP + p];
        if (!std::isfinite(e) || !std::isfinite(bk))
          return set_err(c, TNT_E_NAN, "batched Lanczos: non-finite value in problem %d", p);
        E[(size_t)p] = e;
        resid[(size_t)p] = bk * yk;
        kk[(size_t)p] = k + 1;
        bool cv = (resid_only || (have_prev[(size_t)p] && std::fabs(e - Eprev[(size_t)p]) <= tol * std::fabs(e))) &&
                  resid[(size_t)p] <= rtol * std::fabs(e);
        if (bk <= rtol * std::fabs(e) * 1e-3 || bk == 0.0) cv = true;
        have_prev[(size_t)p] = 1;
        Eprev[(size_t)p] = e;
        if (cv || total[(size_t)p] + res[(size_t)p].n_matvec >= max_matvec) {
          conv[(size_t)p] = cv ? 1 : 0;
          frozen[(size_t)p] = 1;
          changed = true;
          --running;
        }
      }
      if (changed) TNT_TRY(push_frozen());
      if (running == 0 || k + 1 == cap) break;
      TNT_TRY(snormalize(c, s, s.w, s.V + (int64_t)(k + 1) * s.n, s.n2, s.frozen));
    }
    // Ritz vectors of every problem that took part in this cycle
    std::vector<int> skip_ritz((size_t)NP);
    for (int p = 0; p < NP; ++p) skip_ritz[(size_t)p] = active_in_cycle[(size_t)p];
    TNT_CUDA_TRY(c, cudaMemcpyAsync(s.kk, kk.data(), sizeof(int) * NP, cudaMemcpyHostToDevice, c->stream));
    TNT_CUDA_TRY(c, cudaMemcpyAsync(s.skip2, skip_ritz.data(), sizeof(int) * NP, cudaMemcpyHostToDevice, c->stream));
    k_sritz<<<NP, 64, 0, c->stream>>>(s.y, s.kk, s.coef, NP);
    c->launches++;
    k_sfill<<<s.nch, ST, 0, c->stream>>>(s.w, s.ch, s.skip2);
    c->launches++;
    int kmax = 1;
    for (int p = 0; p < NP; ++p)
      if (!active_in_cycle[(size_t)p]) kmax = std::max(kmax, kk[(size_t)p]);
    TNT_TRY(saxpy(c, s, kmax, s.coef, s.w, s.n2, s.skip2, s.kk));
    // finished problems: Ritz vector to x; the others restart from it
    std::vector<int> to_x((size_t)NP), to_v((size_t)NP);
    for (int p = 0; p < NP; ++p) {
      const bool took = !active_in_cycle[(size_t)p];
      to_x[(size_t)p] = (took && frozen[(size_t)p]) ? 0 : 1;   // 0 = write
      to_v[(size_t)p] = (took && !frozen[(size_t)p]) ? 0 : 1;
    }
    TNT_CUDA_TRY(c, cudaMemcpyAsync(s.done, to_x.data(), sizeof(int) * NP, cudaMemcpyHostToDevice, c->stream));
    TNT_TRY(snormalize(c, s, s.w, x, s.n2, s.done));
    TNT_CUDA_TRY(c, cudaMemcpyAsync(s.skip2, to_v.data(), sizeof(int) * NP, cudaMemcpyHostToDevice, c->stream));
    TNT_TRY(snormalize(c, s, s.w, s.V, s.n2, s.skip2));
    TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // the host flag arrays above are reused
    for (int p = 0; p < NP; ++p) {
      if (active_in_cycle[(size_t)p]) continue;
      if (frozen[(size_t)p]) {
        tnt_lanczos_result& r = res[(size_t)p];
        r.E = E[(size_t)p];
        r.resid = resid[(size_t)p];
        r.n_matvec += total[(size_t)p];
        r.converged = conv[(size_t)p];
      }
    }
    (void)mv;
  }
  for (int p = 0; p < NP; ++p) done[(size_t)p] = 1;
  return TNT_OK;
}
}  // namespace

size_t lanczos_batched_scratch_bound(int64_t n, int nprob, int krylov_cap) {
  const int64_t nch = n / 2048 + nprob + 1;
  return ws_round(sizeof(z) * (size_t)n * krylov_cap) + 3 * ws_round(sizeof(z) * (size_t)n) +
         ws_round(sizeof(int64_t) * 3 * nch) + ws_round(sizeof(z) * SKB * nch) + ws_round(sizeof(double) * nch) +
         16 * ws_round(sizeof(double) * KMAX * (nprob + 1) * 2) + (size_t)(4 << 20);
}

int lanczos_batched(Ctx* c, const MatVec& A, const std::vector<int64_t>& off, z* x,
                    std::vector<tnt_lanczos_result>* out) {
  const tnt_params& Pm = c->params;
  const int cap = Pm.krylov_cap;
  if (cap < 2 || cap > KMAX) return set_err(c, TNT_E_INVALID, "krylov_cap %d outside [2, %d]", cap, KMAX);
  const int NP = (int)off.size() - 1;
  BScratch s;
  s.P = NP;
  s.n = off[(size_t)NP];
  if (s.n != A.n) return set_err(c, TNT_E_INVALID, "batched Lanczos: offsets do not match the operator");
  // chunks of at most CH elements, never crossing a problem boundary
  const int64_t CH = std::max<int64_t>(2048, (s.n + 607) / 608);
  std::vector<int64_t> ch;
  std::vector<int> first(1, 0);
  for (int p = 0; p < NP; ++p) {
    for (int64_t lo = off[(size_t)p]; lo < off[(size_t)p + 1]; lo += CH) {
      ch.push_back(p);
      ch.push_back(lo);
      ch.push_back(std::min(off[(size_t)p + 1], lo + CH));
    }
    if (off[(size_t)p + 1] == off[(size_t)p]) return set_err(c, TNT_E_INVALID, "batched Lanczos: empty problem %d", p);
    first.push_back((int)(ch.size() / 3));
  }
  s.nch = (int)(ch.size() / 3);
  TNT_TRY(pinned_reserve(c, sizeof(double) * (3 * NP + 8)));
  s.h = c->h_pinned;
  auto al = [&](size_t b) { return ws_alloc(c, ws_round(std::max<size_t>(b, 8))); };
  s.V = (z*)al(sizeof(z) * (size_t)s.n * cap);
  s.w = (z*)al(sizeof(z) * (size_t)s.n);
  s.w2 = (z*)al(sizeof(z) * (size_t)s.n);
  s.ch = (int64_t*)al(sizeof(int64_t) * ch.size());
  s.first = (int*)al(sizeof(int) * first.size());
  s.part = (z*)al(sizeof(z) * SKB * s.nch);
  s.rpart = (double*)al(sizeof(double) * s.nch);
  s.dots = (z*)al(sizeof(z) * KMAX * NP);
  s.coef = (z*)al(sizeof(z) * KMAX * NP);
  s.alpha = (double*)al(sizeof(double) * KMAX * NP);
  s.beta = (double*)al(sizeof(double) * KMAX * NP);
  s.y = (double*)al(sizeof(double) * KMAX * NP);
  s.tri = (double*)al(sizeof(double) * 3 * NP);  // (E, |y_k|) per problem, then beta_k
  s.n2 = (double*)al(sizeof(double) * NP);
  s.frozen = (int*)al(sizeof(int) * NP);
  s.skip2 = (int*)al(sizeof(int) * NP);
  s.kk = (int*)al(sizeof(int) * NP);
  s.done = (int*)al(sizeof(int) * NP);
  s.none = (int*)al(sizeof(int) * NP);
  if (!s.V || !s.w || !s.w2 || !s.ch || !s.first || !s.part || !s.rpart || !s.dots || !s.coef ||
      !s.alpha || !s.beta || !s.y || !s.tri || !s.n2 || !s.frozen || !s.skip2 || !s.kk ||
      !s.done || !s.none)
    return set_err(c, TNT_E_ALLOC, "scratch exhausted (batched Lanczos)");
  TNT_CUDA_TRY(c, cudaMemcpyAsync(s.ch, ch.data(), sizeof(int64_t) * ch.size(), cudaMemcpyHostToDevice, c->stream));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(s.first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice, c->stream));
  TNT_CUDA_TRY(c, cudaMemsetAsync(s.none, 0, sizeof(int) * NP, c->stream));
  TNT_CUDA_TRY(c, cudaMemsetAsync(s.alpha, 0, sizeof(double) * KMAX * NP, c->stream));
  TNT_CUDA_TRY(c, cudaMemsetAsync(s.beta, 0, sizeof(double) * KMAX * NP, c->stream));
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  out->assign((size_t)NP, tnt_lanczos_result{});
  std::vector<int> done((size_t)NP, 0);
  const int prec = Pm.precision;
  TNT_TRY(cycles(c, A, s, x, prec, Pm.lanczos_maxit, done, *out,
                 prec == TNT_PREC_MIXED && c->fp64_finish));
  if (prec == TNT_PREC_MIXED) {
    // win-back: one FP64 grouped matvec for all problems, Rayleigh quotients and residuals
    TNT_TRY(A.apply(c, x, s.w, TNT_PREC_FP64));
    TNT_TRY(sdots(c, s, x, 1, s.w, s.dots, s.none));
    k_sresid<<<s.nch, ST, 0, c->stream>>>(s.w, x, s.dots, s.w2, s.ch, s.none);
    c->launches++;
    TNT_TRY(snorm2(c, s, s.w2, s.n2, s.none));
    std::vector<z> hd((size_t)KMAX * NP);
    std::vector<double> hn((size_t)NP);
    TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    TNT_CUDA_TRY(c, cudaMemcpy(hd.data(), s.dots, sizeof(z) * KMAX * NP, cudaMemcpyDeviceToHost));
    TNT_CUDA_TRY(c, cudaMemcpy(hn.data(), s.n2, sizeof(double) * NP, cudaMemcpyDeviceToHost));
    std::vector<int> again((size_t)NP, 1);  // 1 = done
    bool any = false;
    // a problem continues in FP64 from its vector when its residual is not accurate enough
    // for the FP64 energy (within what is left of its budget), or always, on a budget of
    // its own, when the caller asks for FP64 accuracy (the DMRG sweeps)
    const bool finish = c->fp64_finish;
    for (int p = 0; p < NP; ++p) {
      tnt_lanczos_result& r = (*out)[(size_t)p];
      r.n_matvec += 1;
      r.E_rq = hd[(size_t)p * KMAX].x;
      r.resid_fp64 = std::sqrt(hn[(size_t)p]);
      if (finish || (r.resid_fp64 > 1e-5 * std::fabs(r.E_rq) && r.n_matvec < Pm.lanczos_maxit)) {
        again[(size_t)p] = 0;
        any = true;
      }
    }
    if (any) {
      const std::vector<int> cont(again);
      // the budget of cycles() counts the matvecs a problem has already spent; with the
      // FP64 finish the continuation gets lanczos_maxit of its own
      std::vector<int> spent((size_t)NP, 0);
      if (finish)
        for (int p = 0; p < NP; ++p)
          if (!cont[(size_t)p]) std::swap(spent[(size_t)p], (*out)[(size_t)p].n_matvec);
      TNT_TRY(cycles(c, A, s, x, TNT_PREC_FP64, Pm.lanczos_maxit, again, *out));
      for (int p = 0; p < NP; ++p) {
        if (cont[(size_t)p]) continue;
        tnt_lanczos_result& r = (*out)[(size_t)p];
        r.n_matvec += spent[(size_t)p];
        r.E_rq = r.E;
        r.resid_fp64 = r.resid;
      }
    }
    return TNT_OK;
  }
  for (int p = 0; p < NP; ++p) {
    (*out)[(size_t)p].E_rq = (*out)[(size_t)p].E;
    (*out)[(size_t)p].resid_fp64 = (*out)[(size_t)p].resid;
  }
  return TNT_OK;
}

}  // namespace tnt
