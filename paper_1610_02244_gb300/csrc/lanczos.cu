// Lanczos ground-state eigensolver for H_eff (the external sparse eigensolver the library
// calls with the contractor of Listing 1 as its matvec; Sec. 4.3, iteration cap 300 of
// App. A.3).  Vectors, sums over blocks and the tridiagonal eigenproblem are FP64 on the
// GPU; the matvec may run in split TF32, and with it the Gram-Schmidt products in FP32.
// Per Krylov step k:
//   w = H v_k;  c = V^H w;  alpha_k = Re c_k;  w -= V c   (classical Gram-Schmidt; in FP32
//   arithmetic on the FP64 vectors while the matvec is split TF32), then
//   the same pass once more ("twice is enough": one pass leaves w's components along
//   converged Ritz directions at the size of the cancellation error, and a restarted
//   Lanczos on a DMRG effective Hamiltonian then stalls short of its tolerance)
//   beta_k = |w|;  (E_k, y) = lowest eigenpair of T_k;  resid = beta_k |y_k|
//   stop if |E_k - E_{k-1}| <= tol |E_k| and resid <= max(tol, 10 u)|E_k|, u the matvec's
//   unit roundoff (2^-52 FP64, 2^-22 split TF32), or if beta_k vanishes (a split-TF32
//   phase that an FP64 continuation follows stops on the residual test alone)
//   v_{k+1} = w / beta_k;  restart from the Ritz vector after krylov_cap steps.
// (The three-term subtraction alpha v_k + beta v_{k-1} is contained in the first
// Gram-Schmidt pass, whose coefficient on v_k is alpha_k.)
#include <cmath>

#include "heff_plan.cuh"

namespace tnt {

namespace {
// alpha[k] = Re dots[k]; beta[k] = sqrt(norm2)
__global__ void k_lz_scalars(const z* dots, int k, const double* norm2, double* alpha,
                             double* beta) {
  if (threadIdx.x == 0) {
    alpha[k] = dots[k].x;
    beta[k] = sqrt(norm2[0]);
  }
}

// coef[i] = -y[i] (so that multiaxpy on a zero vector builds sum_i y_i V_i)
__global__ void k_lz_ritz_coef(const double* y, int k, z* coef) {
  int i = threadIdx.x;
  if (i < k) coef[i] = zmk(-y[i], 0.0);
}

// out = a - e b (elementwise), partial |.|^2 in norm-ready form
__global__ void k_resid(const z* __restrict__ Hx, const z* __restrict__ x, const double* E,
                        z* __restrict__ r, int64_t n) {
  const double e = E[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] = zsub(Hx[i], zscale(x[i], e));
}
__global__ void k_copy_re(const z* src, double* dst) {
  if (threadIdx.x == 0) dst[0] = src[0].x;
}
}  // namespace

constexpr int64_t MIXED_MIN_N = 1 << 16;

size_t lanczos_scratch_bound(int64_t n, int krylov_cap) {
  return ws_round(sizeof(z) * (size_t)n * krylov_cap) + 2 * ws_round(sizeof(z) * (size_t)n) +
         (size_t)(2 << 20);
}

// resid_only: stop on the residual estimate alone (a split-TF32 phase followed by an FP64
// continuation, which applies the energy test itself: the split-TF32 Ritz values move at
// the matvec's noise level from one restart to the next, and waiting for them to settle
// to 1e-12 |E| spent up to 160 matvecs on bonds whose start vector was already converged)
static int lanczos_cycle_loop(Ctx* c, const MatVec& A, z* theta, int precision,
                              int max_matvec, tnt_lanczos_result* res, z* V, z* w,
                              double* dsc, bool resid_only = false) {
  const tnt_params& P = c->params;
  const int64_t n = A.n;
  const int cap = P.krylov_cap;
  z* dots = (z*)dsc;                  // 64 complex
  double* norm2 = dsc + 128;          // 1
  double* alpha = dsc + 136;          // 64
  double* beta = dsc + 200;           // 64
  z* coef = (z*)(dsc + 336);          // 64 complex
  double* tri2 = dsc + 464;           // 2 x 2: (E, |y_k|) of even / odd steps
  double* y2 = dsc + 512;             // 2 x 64: y of even / odd steps
  const double u = (precision == TNT_PREC_MIXED) ? std::ldexp(1.0, -22) : std::ldexp(1.0, -52);
  const double tol = P.lanczos_tol;
  const double rtol = std::max(tol, 10.0 * u);
  // with split-TF32 matvecs the Gram-Schmidt passes run in FP32 arithmetic (their rounding,
  // u_32 |V c|, stays below the matvec's own ~2^-22 error); the Ritz vector is assembled
  // in FP64, as its norm enters the FP64 Rayleigh quotient
  const bool f32_gs = (precision == TNT_PREC_MIXED);
  double* hp = c->h_pinned;
  // v_0 = theta / |theta| (a zero or non-finite start vector is reported, not iterated)
  TNT_TRY(vec_norm2(c, theta, n, norm2));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(hp, norm2, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (!(hp[0] > 0.0) || !std::isfinite(hp[0]))
    return set_err(c, TNT_E_NAN, "Lanczos start vector has |x|^2 = %g (n = %lld)", hp[0], (long long)n);
  TNT_TRY(vec_normalize(c, theta, V, n, norm2));
  int total = 0;
  bool have_prev = false;
  double E_prev = 0;
  // T_k's lowest eigenpair runs on the side stream one Krylov step behind the vector work:
  // step k's scalars are handed over by an event, its result comes back into pinned slot
  // k & 1, and the host checks step k - 1 while step k runs.  A solve that converges at
  // k - 1 has computed one step more than it uses (not counted in n_matvec); the Ritz
  // vector is that of step k - 1, from V[0..k-1] and y of slot (k-1) & 1.
  TNT_TRY(side_stream(c));
  int last_side = -1;  // slot of the last side-stream launch
  auto launch_tk = [&](int k) -> int {
    double* tk = tri2 + 2 * (k & 1);
    TNT_CUDA_TRY(c, cudaEventRecord(c->ev_main[k & 1], c->stream));
    TNT_CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_main[k & 1], 0));
    TNT_TRY(tridiag_lowest_on(c, c->side, alpha, beta, k + 1, tk, y2 + 64 * (k & 1)));
    TNT_CUDA_TRY(c, cudaMemcpyAsync(hp + 4 * (k & 1), tk, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->side));
    TNT_CUDA_TRY(c, cudaMemcpyAsync(hp + 4 * (k & 1) + 2, beta + k, sizeof(double), cudaMemcpyDeviceToHost, c->side));
    TNT_CUDA_TRY(c, cudaEventRecord(c->ev_side[k & 1], c->side));
    last_side = k & 1;
    return TNT_OK;
  };
  double E = 0, resid = 0;
  int kk = 0;
  // step j's result: E_j, the residual estimate, and whether the solve may stop there
  auto check_step = [&](int j, bool* cv) -> int {
    TNT_CUDA_TRY(c, cudaEventSynchronize(c->ev_side[j & 1]));
    const double* h = hp + 4 * (j & 1);
    E = h[0];
    const double bk = h[2];
    resid = bk * h[1];
    kk = j + 1;
    *cv = (resid_only || (have_prev && std::fabs(E - E_prev) <= tol * std::fabs(E))) &&
          resid <= rtol * std::fabs(E);
    if (bk <= rtol * std::fabs(E) * 1e-3 || bk == 0.0) *cv = true;
    if (!std::isfinite(E) || !std::isfinite(bk))
      return set_err(c, TNT_E_NAN, "Lanczos produced a non-finite value at step %d (E = %g, beta = %g, %s matvec)",
                     total, E, bk, precision == TNT_PREC_MIXED ? "split-TF32" : "FP64");
    have_prev = true;
    E_prev = E;
    return TNT_OK;
  };
  for (;;) {
    bool stop = false, conv = false;
    int use = 0;  // the step whose Ritz pair the cycle ends with
    for (int k = 0; k < cap; ++k) {
      z* vk = V + (int64_t)k * n;
      TNT_TRY(A.apply(c, vk, w, precision));
      ++total;
      if (f32_gs) {
        TNT_TRY(vec_multidot_f32(c, V, n, k + 1, w, n, dots));
        TNT_TRY(vec_multiaxpy_norm_f32(c, V, n, k + 1, dots, w, n, norm2));
      } else {
        TNT_TRY(vec_multidot(c, V, n, k + 1, w, n, dots));
        TNT_TRY(vec_multiaxpy_norm(c, V, n, k + 1, dots, w, n, norm2));
      }
      k_lz_scalars<<<1, 32, 0, c->stream>>>(dots, k, norm2, alpha, beta);  // alpha_k from pass 1
      c->launches += 1;
      if (f32_gs) {
        TNT_TRY(vec_multidot_f32(c, V, n, k + 1, w, n, coef));
        TNT_TRY(vec_multiaxpy_norm_f32(c, V, n, k + 1, coef, w, n, norm2));
      } else {
        TNT_TRY(vec_multidot(c, V, n, k + 1, w, n, coef));
        TNT_TRY(vec_multiaxpy_norm(c, V, n, k + 1, coef, w, n, norm2));
      }
      // beta_k from pass 2 (overwrite), then the tridiagonal eigenpair of T_k on the side
      k_lz_scalars<<<1, 32, 0, c->stream>>>(dots, k, norm2, alpha, beta);
      c->launches++;
      TNT_TRY(launch_tk(k));
      if (k > 0) {
        bool cv = false;
        TNT_TRY(check_step(k - 1, &cv));
        if (cv) {
          conv = stop = true;
          use = k - 1;
          --total;  // step k was not needed
          break;
        }
      }
      if (k + 1 == cap || total >= max_matvec) {
        bool cv = false;
        TNT_TRY(check_step(k, &cv));
        conv = cv;
        stop = cv || total >= max_matvec;
        use = k;
        break;
      }
      // v_{k+1}, except after the last step of a cycle: the basis holds cap vectors, and
      // the restart begins from the Ritz vector instead
      TNT_TRY(vec_normalize(c, w, V + (int64_t)(k + 1) * n, n, norm2));
    }
    // the side stream's work is done before the main stream reuses its buffers
    TNT_CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev_side[last_side], 0));
    // Ritz vector x = sum_i y_i v_i  (built in w, normalised)
    k_lz_ritz_coef<<<1, 64, 0, c->stream>>>(y2 + 64 * (use & 1), kk, coef);
    c->launches++;
    TNT_TRY(zfill(c, w, n, zmk(0, 0)));
    TNT_TRY(vec_multiaxpy_norm(c, V, n, kk, coef, w, n, norm2));
    if (stop) {
      TNT_TRY(vec_normalize(c, w, theta, n, norm2));
      res->E = E;
      res->resid = resid;
      res->n_matvec += total;
      res->converged = conv ? 1 : 0;
      return TNT_OK;
    }
    TNT_TRY(vec_normalize(c, w, V, n, norm2));  // restart
  }
}

namespace {
struct HeffMatVec : MatVec {
  const HeffPlan& p;
  explicit HeffMatVec(const HeffPlan& pp) : p(pp) { n = pp.chl * pp.d * pp.d * pp.chr; }
  int apply(Ctx* c, const z* x, z* y, int precision) const override {
    return heff_run(c, p, x, y, precision);
  }
};
}  // namespace

int lanczos_impl(Ctx* c, const HeffPlan& p, z* theta, tnt_lanczos_result* res) {
  return lanczos_run(c, HeffMatVec(p), theta, res);
}

int lanczos_run(Ctx* c, const MatVec& A, z* theta, tnt_lanczos_result* res) {
  const tnt_params& P = c->params;
  const int64_t n = A.n;
  const int cap = P.krylov_cap;
  if (cap < 2 || cap > 64) return set_err(c, TNT_E_INVALID, "krylov_cap %d outside [2, 64]", cap);
  TNT_TRY(pinned_reserve(c, 64 * sizeof(double)));
  z* V = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)n * cap));
  z* w = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)n));
  z* w2 = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)n));
  double* dsc = (double*)ws_alloc(c, ws_round(sizeof(double) * 1024));
  if (!V || !w || !w2 || !dsc) return set_err(c, TNT_E_ALLOC, "scratch exhausted (Lanczos)");
  *res = tnt_lanczos_result{};
  // below MIXED_MIN_N entries a matvec is a handful of small launches whichever the
  // arithmetic, and the split-TF32 phase only adds the FP64 finish on top: such problems
  // run their matvecs in FP64 from the start (the result is the FP64 path's)
  const int prec = (P.precision == TNT_PREC_MIXED && n < MIXED_MIN_N) ? TNT_PREC_FP64 : P.precision;
  TNT_TRY(lanczos_cycle_loop(c, A, theta, prec, P.lanczos_maxit, res, V, w, dsc,
                             prec == TNT_PREC_MIXED && c->fp64_finish));
  if (prec == TNT_PREC_MIXED) {
    // accuracy win-back: one FP64 matvec for the Rayleigh quotient and the true residual
    double* hp = c->h_pinned;
    z* dot = (z*)dsc;
    double* norm2 = dsc + 128;
    double* Erq = dsc + 130;
    TNT_TRY(A.apply(c, theta, w, TNT_PREC_FP64));
    res->n_matvec += 1;
    TNT_TRY(vec_dot(c, theta, w, n, dot));
    k_copy_re<<<1, 32, 0, c->stream>>>(dot, Erq);
    k_resid<<<1216, 256, 0, c->stream>>>(w, theta, Erq, w2, n);
    c->launches += 2;
    TNT_TRY(vec_norm2(c, w2, n, norm2));
    TNT_CUDA_TRY(c, cudaMemcpyAsync(hp, Erq, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    TNT_CUDA_TRY(c, cudaMemcpyAsync(hp + 1, norm2, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    res->E_rq = hp[0];
    res->resid_fp64 = std::sqrt(hp[1]);
    // continue in FP64 from this vector when its residual is not accurate enough for the
    // FP64 energy, within what is left of the budget; or always, on a budget of its own,
    // when the caller asks for FP64 accuracy (a residual scaled by |E| says little where a
    // constant offset inflates |E| over small gaps)
    const bool finish = c->fp64_finish;
    const int budget = finish ? P.lanczos_maxit : P.lanczos_maxit - res->n_matvec;
    if ((finish || res->resid_fp64 > 1e-5 * std::fabs(res->E_rq)) && budget > 0) {
      tnt_lanczos_result r2{};
      TNT_TRY(lanczos_cycle_loop(c, A, theta, TNT_PREC_FP64, budget, &r2, V, w, dsc));
      res->n_matvec += r2.n_matvec;
      res->E = r2.E;
      res->E_rq = r2.E;
      res->resid = r2.resid;
      res->resid_fp64 = r2.resid;
      res->converged = r2.converged;
    }
  } else {
    res->E_rq = res->E;
    res->resid_fp64 = res->resid;
  }
  return res->converged ? TNT_OK : TNT_E_NOCONV;
}

}  // namespace tnt
