// Leading eigenpairs of a large Hermitian FP64 matrix (the Gram matrix of one charge block
// of the truncated SVD, App. B.1.2): k largest eigenvalues and their eigenvectors.
//
//   1. Householder reduction to real tridiagonal form G = Q T Q^H: for each column j the
//      reflector H_j = I - tau v v^H maps the part below the diagonal to beta e_1 (beta
//      real), and the trailing block is updated as A <- H_j^H A H_j through
//      p = tau A v, w = p - (tau/2)(p^H v) v, A <- A - v w^H - w v^H.
//   2. Bisection on Sturm counts of T for eigenvalues n-1, ..., n-k (one thread each).
//   3. Inverse iteration on T - lambda I (pivoted tridiagonal LU, three sweeps, shifts of
//      coincident eigenvalues separated by 10 eps |T|).
//   4. Back-transformation U = H_0 H_1 ... H_{n-2} Y.
//   5. One Newton-Schulz step U <- U (3 I - U^H U) / 2 in FP64 to restore orthonormality
//      lost to close eigenvalues.
// All arithmetic is FP64.  The cost is O(n^3) once, against O(sweeps n^3) for Jacobi.
#include <cmath>

#include "heff_plan.cuh"

namespace tnt {

namespace {
constexpr double EPS = 2.220446049250313e-16;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum; valid in every thread on return
__device__ double block_sum_all(double v, double* sh) {
  v = warp_sum_d(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  return r;
}

// reflector of column j from row j of the (Hermitian, fully stored) trailing matrix
__global__ void k_hh_reflector(const z* __restrict__ G, int64_t n, int64_t j, z* __restrict__ Hv,
                               z* __restrict__ tau, double* __restrict__ d,
                               double* __restrict__ e) {
  __shared__ double sh[32];
  __shared__ double s_xn2;
  const int64_t m = n - j - 1;
  const z* row = G + j * n + j + 1;  // x_r = conj(row[r])
  double acc = 0;
  for (int64_t r = 1 + threadIdx.x; r < m; r += blockDim.x) {
    const z v = row[r];
    acc = fma(v.x, v.x, fma(v.y, v.y, acc));
  }
  acc = block_sum_all(acc, sh);
  if (threadIdx.x == 0) s_xn2 = acc;
  __syncthreads();
  const double xn2 = s_xn2;
  const z alpha = m > 0 ? zconj(row[0]) : zmk(0, 0);
  double beta;
  z t, scale;
  if (m == 0 || (xn2 == 0.0 && alpha.y == 0.0)) {
    t = zmk(0, 0);
    beta = alpha.x;
    scale = zmk(0, 0);
  } else {
    const double nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2);
    beta = alpha.x >= 0 ? -nrm : nrm;
    t = zmk((beta - alpha.x) / beta, -alpha.y / beta);
    const z den = zmk(alpha.x - beta, alpha.y);  // 1 / (alpha - beta)
    const double dd = den.x * den.x + den.y * den.y;
    scale = zmk(den.x / dd, -den.y / dd);
  }
  z* v = Hv + j * n;
  for (int64_t r = threadIdx.x; r < m; r += blockDim.x)
    v[r] = (r == 0) ? zmk(1, 0) : zmul(zconj(row[r]), scale);
  if (threadIdx.x == 0) {
    tau[j] = t;
    d[j] = G[j * n + j].x;
    if (m > 0) e[j] = beta;
  }
}

// p = tau A v (A = trailing block), one warp per row; partial[b] = sum over the block's
// rows of conj(p_r) v_r
__global__ void k_hh_gemv(const z* __restrict__ G, int64_t n, int64_t j, const z* __restrict__ Hv,
                          const z* __restrict__ tau, z* __restrict__ p, z* __restrict__ partial) {
  __shared__ double shr[8], shi[8];
  const int64_t m = n - j - 1;
  const z* v = Hv + j * n;
  const z t = tau[j];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double pr = 0, pi = 0;
  for (int64_t r = (int64_t)blockIdx.x * 8 + warp; r < m; r += (int64_t)gridDim.x * 8) {
    const z* a = G + (j + 1 + r) * n + j + 1;
    double sr = 0, si = 0;
    for (int64_t c = lane; c < m; c += 32) {
      const z x = a[c], y = v[c];
      sr = fma(x.x, y.x, fma(-x.y, y.y, sr));
      si = fma(x.x, y.y, fma(x.y, y.x, si));
    }
    sr = warp_sum_d(sr);
    si = warp_sum_d(si);
    if (lane == 0) {
      const z pv = zmul(t, zmk(sr, si));
      p[r] = pv;
      const z vr = v[r];
      pr += pv.x * vr.x + pv.y * vr.y;  // conj(p) v
      pi += pv.x * vr.y - pv.y * vr.x;
    }
  }
  if (lane == 0) {
    shr[warp] = pr;
    shi[warp] = pi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int i = 0; i < 8; ++i) {
      a += shr[i];
      b += shi[i];
    }
    partial[blockIdx.x] = zmk(a, b);
  }
}

// A <- A - v w^H - w v^H with w = p - (tau s / 2) v, s = p^H v (sum of partials)
__global__ void k_hh_update(z* __restrict__ G, int64_t n, int64_t j, const z* __restrict__ Hv,
                            const z* __restrict__ tau, const z* __restrict__ p,
                            const z* __restrict__ partial, int nparts) {
  __shared__ z s_c;
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int i = 0; i < nparts; ++i) {
      a += partial[i].x;
      b += partial[i].y;
    }
    const z ts = zmul(tau[j], zmk(a, b));
    s_c = zmk(-0.5 * ts.x, -0.5 * ts.y);
  }
  __syncthreads();
  const z cf = s_c;
  const int64_t m = n - j - 1;
  const z* v = Hv + j * n;
  const int64_t tot = m * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / m, c = e % m;
    const z vr = v[r], vc = v[c];
    const z wr = zadd(p[r], zmul(cf, vr)), wc = zadd(p[c], zmul(cf, vc));
    z* a = G + (j + 1 + r) * n + j + 1 + c;
    z x = *a;
    x = zsub(x, zmul(vr, zconj(wc)));
    x = zsub(x, zmul(wr, zconj(vc)));
    *a = x;
  }
}

__device__ int sturm_lt(const double* d, const double* e, int64_t n, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (q < 0) cnt++;
  for (int64_t i = 1; i < n; ++i) {
    if (fabs(q) < pivmin) q = -pivmin;
    q = (d[i] - x) - e[i - 1] * e[i - 1] / q;
    if (q < 0) cnt++;
  }
  return cnt;
}

// eigenvalue of ascending index n-1-i for i < k, by bisection; ev[i] descending
__global__ void k_bisect(const double* __restrict__ d, const double* __restrict__ e, int64_t n,
                         int64_t k, double* __restrict__ ev, double* __restrict__ tnorm_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double lo = d[0], hi = d[0], tn = 0, emax2 = 0;
  for (int64_t r = 0; r < n; ++r) {
    const double rad = (r > 0 ? fabs(e[r - 1]) : 0.0) + (r < n - 1 ? fabs(e[r]) : 0.0);
    lo = fmin(lo, d[r] - rad);
    hi = fmax(hi, d[r] + rad);
    tn = fmax(tn, fabs(d[r]) + rad);
    if (r < n - 1) emax2 = fmax(emax2, e[r] * e[r]);
  }
  if (i == 0 && tnorm_out) tnorm_out[0] = tn;
  if (i >= k) return;
  const double pivmin = fmax(1e-300, EPS * EPS * fmax(emax2, 1e-300)) + 1e-300;
  const int64_t idx = n - 1 - i;
  const double pad = 2 * EPS * tn + 1e-300;
  lo -= pad;
  hi += pad;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (hi - lo <= 2 * EPS * fmax(fabs(lo), fabs(hi)) + 1e-300 || mid <= lo || mid >= hi) break;
    if (sturm_lt(d, e, n, mid, pivmin) <= idx) lo = mid; else hi = mid;
  }
  ev[i] = 0.5 * (lo + hi);
}

// inverse iteration, one thread per eigenvalue; work arrays interleaved by thread:
// element r of thread i at [r * k + i]
__global__ void k_inviter(const double* __restrict__ d, const double* __restrict__ e, int64_t n,
                          const double* __restrict__ ev, int64_t k, const double* __restrict__ tnorm,
                          double* __restrict__ work, double* __restrict__ Y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const double tn = fmax(tnorm[0], 1e-300);
  double lam = ev[i];
  // separate coincident shifts (descending order): keep a gap of 10 eps |T|
  for (int64_t t = i; t > 0; --t) {
    if (ev[t - 1] - ev[t] >= 10 * EPS * tn) break;
    lam = fmin(lam, ev[t - 1] - 10 * EPS * tn * (double)(i - t + 1));
  }
  double* dl = work;
  double* dm = work + n * k;
  double* du = work + 2 * n * k;
  double* du2 = work + 3 * n * k;
  double* y = work + 4 * n * k;
  int8_t* piv = (int8_t*)(work + 5 * n * k);
#define W(a, r) a[(r) * k + i]
  // start vector: deterministic, free of structure
  uint32_t h = 2166136261u ^ (uint32_t)(i * 2654435761u);
  for (int64_t r = 0; r < n; ++r) {
    h ^= (uint32_t)r;
    h *= 16777619u;
    W(y, r) = 0.5 + (double)(h & 0xffff) / 65536.0;
  }
  const double small = EPS * tn;
  // LU with partial pivoting of T - lam I (tridiagonal, textbook)
  for (int64_t r = 0; r < n; ++r) {
    W(dm, r) = d[r] - lam;
    W(du, r) = r < n - 1 ? e[r] : 0.0;
    W(dl, r) = r < n - 1 ? e[r] : 0.0;
    W(du2, r) = 0.0;
  }
  for (int64_t r = 0; r < n - 1; ++r) {
    const double a = W(dm, r), b = W(dl, r);
    if (fabs(a) >= fabs(b)) {
      const double aa = fabs(a) < small ? (a < 0 ? -small : small) : a;
      W(dm, r) = aa;
      const double f = b / aa;
      W(dl, r) = f;
      W(dm, r + 1) -= f * W(du, r);
      piv[r * k + i] = 0;
    } else {
      const double f = a / b;
      W(dm, r) = b;
      W(dl, r) = f;
      const double t = W(du, r);
      W(du, r) = W(dm, r + 1);
      W(dm, r + 1) = t - f * W(du, r);
      if (r < n - 2) {
        W(du2, r) = W(du, r + 1);
        W(du, r + 1) = -f * W(du, r + 1);
      }
      piv[r * k + i] = 1;
    }
  }
  if (fabs(W(dm, n - 1)) < small) W(dm, n - 1) = W(dm, n - 1) < 0 ? -small : small;
  for (int sweep = 0; sweep < 3; ++sweep) {
    for (int64_t r = 0; r < n - 1; ++r) {
      if (piv[r * k + i] == 0) {
        W(y, r + 1) -= W(dl, r) * W(y, r);
      } else {
        const double t = W(y, r);
        W(y, r) = W(y, r + 1);
        W(y, r + 1) = t - W(dl, r) * W(y, r);
      }
    }
    W(y, n - 1) /= W(dm, n - 1);
    if (n > 1) W(y, n - 2) = (W(y, n - 2) - W(du, n - 2) * W(y, n - 1)) / W(dm, n - 2);
    for (int64_t r = n - 3; r >= 0; --r)
      W(y, r) = (W(y, r) - W(du, r) * W(y, r + 1) - W(du2, r) * W(y, r + 2)) / W(dm, r);
    double nrm = 0;
    for (int64_t r = 0; r < n; ++r) nrm = fma(W(y, r), W(y, r), nrm);
    nrm = 1.0 / sqrt(nrm);
    for (int64_t r = 0; r < n; ++r) W(y, r) *= nrm;
  }
  for (int64_t r = 0; r < n; ++r) Y[i * n + r] = W(y, r);
#undef W
}

// U[:, i] = H_0 ... H_{n-2} y_i; one CTA per eigenvector, the vector in shared memory
__global__ void __launch_bounds__(256) k_backtransform(const double* __restrict__ Y,
                                                       const z* __restrict__ Hv,
                                                       const z* __restrict__ tau, int64_t n,
                                                       z* __restrict__ U, int64_t ldu) {
  extern __shared__ double sm_bt[];
  z* y = (z*)sm_bt;
  __shared__ double shr[8], shi[8];
  const int64_t i = blockIdx.x;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) y[r] = zmk(Y[i * n + r], 0);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t j = n - 2; j >= 0; --j) {
    const z t = tau[j];
    if (t.x == 0.0 && t.y == 0.0) continue;
    const int64_t m = n - j - 1;
    const z* v = Hv + j * n;
    double sr = 0, si = 0;  // s = v^H y[j+1:]
    for (int64_t r = threadIdx.x; r < m; r += blockDim.x) {
      const z a = v[r], b = y[j + 1 + r];
      sr = fma(a.x, b.x, fma(a.y, b.y, sr));
      si = fma(a.x, b.y, fma(-a.y, b.x, si));
    }
    sr = warp_sum_d(sr);
    si = warp_sum_d(si);
    if (lane == 0) {
      shr[warp] = sr;
      shi[warp] = si;
    }
    __syncthreads();
    double a = 0, b = 0;
    for (int q = 0; q < 8; ++q) {
      a += shr[q];
      b += shi[q];
    }
    const z ts = zmul(t, zmk(a, b));
    for (int64_t r = threadIdx.x; r < m; r += blockDim.x)
      y[j + 1 + r] = zsub(y[j + 1 + r], zmul(ts, v[r]));
    __syncthreads();
  }
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) U[r * ldu + i] = y[r];
}

// S <- 1.5 I - 0.5 S  (k x k)
__global__ void k_ns_coef(z* S, int64_t k) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < k * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k, c = e % k;
    z v = zscale(S[e], -0.5);
    if (r == c) v.x += 1.5;
    S[e] = v;
  }
}

__global__ void k_copy_cols(const z* __restrict__ src, int64_t n, int64_t k, int64_t lds,
                            z* __restrict__ dst, int64_t ldd) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k, c = e % k;
    dst[r * ldd + c] = src[r * lds + c];
  }
}

unsigned gsz(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return (unsigned)b;
}
}  // namespace

size_t heig_scratch_bound(int64_t n, int64_t k) {
  return ws_round(sizeof(z) * n * n) + 2 * ws_round(sizeof(z) * n) + 3 * ws_round(sizeof(double) * n) +
         ws_round(sizeof(z) * 1216) + ws_round(sizeof(double) * k) + ws_round(sizeof(double) * (6 * n * k + k)) +
         ws_round(sizeof(double) * n * k) + 2 * ws_round(sizeof(z) * n * k) + 2 * ws_round(sizeof(z) * k * k) +
         (size_t)(1 << 20);
}

// G (n x n, row-major, Hermitian, destroyed); U (n x k, leading dimension ldu): the
// eigenvectors of the k largest eigenvalues, in descending order; ev (device, k).
int heig_top(Ctx* c, z* G, int64_t n, int64_t k, z* U, int64_t ldu, double* ev) {
  if (k < 1 || k > n) return set_err(c, TNT_E_INVALID, "heig_top: k = %lld of n = %lld", (long long)k, (long long)n);
  if (n > 8192) return set_err(c, TNT_E_UNSUPPORTED, "heig_top: n = %lld > 8192", (long long)n);
  const size_t top = c->ws.top;
  z* Hv = (z*)ws_alloc(c, ws_round(sizeof(z) * n * n));
  z* tau = (z*)ws_alloc(c, ws_round(sizeof(z) * n));
  z* p = (z*)ws_alloc(c, ws_round(sizeof(z) * n));
  double* d = (double*)ws_alloc(c, ws_round(sizeof(double) * n));
  double* e = (double*)ws_alloc(c, ws_round(sizeof(double) * n));
  double* tn = (double*)ws_alloc(c, ws_round(sizeof(double) * n));
  z* part = (z*)ws_alloc(c, ws_round(sizeof(z) * 1216));
  double* work = (double*)ws_alloc(c, ws_round(sizeof(double) * (6 * n * k + k)));
  double* Y = (double*)ws_alloc(c, ws_round(sizeof(double) * n * k));
  z* U0 = (z*)ws_alloc(c, ws_round(sizeof(z) * n * k));
  z* S = (z*)ws_alloc(c, ws_round(sizeof(z) * k * k));
  if (!Hv || !tau || !p || !d || !e || !tn || !part || !work || !Y || !U0 || !S) {
    c->ws.top = top;
    return set_err(c, TNT_E_ALLOC, "scratch exhausted (heig_top n=%lld k=%lld)", (long long)n, (long long)k);
  }
  cudaStream_t st = c->stream;
  {
    ProfScope ps(c, "heig_tridiag");
    for (int64_t j = 0; j < n; ++j) {
      k_hh_reflector<<<1, 256, 0, st>>>(G, n, j, Hv, tau, d, e);
      const int64_t m = n - j - 1;
      if (m <= 0) break;
      const int nb = (int)std::min<int64_t>((m + 7) / 8, 1216);
      k_hh_gemv<<<nb, 256, 0, st>>>(G, n, j, Hv, tau, p, part);
      k_hh_update<<<gsz(m * m), 256, 0, st>>>(G, n, j, Hv, tau, p, part, nb);
      c->launches += 3;
    }
    c->launches += 1;
    TNT_CHECK_LAUNCH(c);
  }
  {
    ProfScope ps(c, "heig_tridiag_eig");
    k_bisect<<<(unsigned)((k + 127) / 128), 128, 0, st>>>(d, e, n, k, ev, tn);
    k_inviter<<<(unsigned)((k + 63) / 64), 64, 0, st>>>(d, e, n, ev, k, tn, work, Y);
    c->launches += 2;
    TNT_CHECK_LAUNCH(c);
  }
  {
    ProfScope ps(c, "heig_backtransform");
    const size_t smem = sizeof(z) * n;
    TNT_CUDA_TRY(c, cudaFuncSetAttribute(k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_backtransform<<<(unsigned)k, 256, smem, st>>>(Y, Hv, tau, n, U0, k);
    c->launches++;
    TNT_CHECK_LAUNCH(c);
  }
  // Newton-Schulz: S = U0^H U0; S <- 1.5 I - 0.5 S; U = U0 S
  ZGemm g{};
  g.M = k; g.N = k; g.K = n;
  g.A = U0; g.a_rs = 1; g.a_cs = k; g.conj_a = 1;
  g.B = U0; g.b_rs = k; g.b_cs = 1;
  g.C = S; g.c_rs = k;
  g.alpha = zmk(1, 0); g.beta = zmk(0, 0); g.batch = 1;
  int r = zgemm(c, g);
  if (r == TNT_OK) {
    k_ns_coef<<<gsz(k * k), 256, 0, st>>>(S, k);
    c->launches++;
    ZGemm h{};
    h.M = n; h.N = k; h.K = k;
    h.A = U0; h.a_rs = k; h.a_cs = 1;
    h.B = S; h.b_rs = k; h.b_cs = 1;
    h.C = U; h.c_rs = ldu;
    h.alpha = zmk(1, 0); h.beta = zmk(0, 0); h.batch = 1;
    r = zgemm(c, h);
  }
  c->ws.top = top;
  return r;
}

}  // namespace tnt
