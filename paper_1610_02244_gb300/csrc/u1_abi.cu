// C-ABI entry points of the U(1) block-sparse grouped matvec and its Lanczos solve.
#include <vector>

#include "heff_plan.cuh"
#include "u1.cuh"

namespace tnt {
namespace {

int spec_of(Ctx* c, const tnt_u1_problem* p, U1Spec* s) {
  if (!p || !p->d_L || !p->d_W1 || !p->d_W2 || !p->d_R || !p->h_qa || !p->h_qb || !p->h_wq)
    return set_err(c, TNT_E_INVALID, "U(1) problem: null pointer");
  if (p->chl < 1 || p->chr < 1 || p->d < 1 || p->D < 1 || p->d * p->d * p->D > 256)
    return set_err(c, TNT_E_INVALID, "U(1) problem: bad dimension");
  s->L = (const z*)p->d_L;
  s->R = (const z*)p->d_R;
  s->W1 = (const z*)p->d_W1;
  s->W2 = (const z*)p->d_W2;
  s->chl = p->chl;
  s->chr = p->chr;
  s->d = p->d;
  s->D = p->D;
  s->qa.assign(p->h_qa, p->h_qa + p->chl);
  s->qb.assign(p->h_qb, p->h_qb + p->chr);
  s->wq.assign(p->h_wq, p->h_wq + p->D);
  return u1_check(c, *s);
}

// a kernel's bounded wait expired: report it and clear the flag for the next call
int status_check(Ctx* c) {
  int h = 0;
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  TNT_CUDA_TRY(c, cudaMemcpy(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    cudaMemset(c->d_status, 0, sizeof(int));
    return set_err(c, TNT_E_TIMEOUT, "grouped tensor-core GEMM: an mbarrier wait expired");
  }
  return TNT_OK;
}

}  // namespace
}  // namespace tnt

using namespace tnt;

extern "C" {

int tnt_u1_size(const tnt_u1_problem* prob, int64_t* n) {
  if (!prob || !n || !prob->h_qa || !prob->h_qb || prob->chl < 1 || prob->chr < 1 || prob->d < 1)
    return TNT_E_INVALID;
  U1Spec s;
  s.chl = prob->chl;
  s.chr = prob->chr;
  s.d = prob->d;
  s.qa.assign(prob->h_qa, prob->h_qa + prob->chl);
  s.qb.assign(prob->h_qb, prob->h_qb + prob->chr);
  for (size_t i = 1; i < s.qa.size(); ++i) if (s.qa[i] < s.qa[i - 1]) return TNT_E_INVALID;
  for (size_t i = 1; i < s.qb.size(); ++i) if (s.qb[i] < s.qb[i - 1]) return TNT_E_INVALID;
  *n = u1_compact_size(s);
  return TNT_OK;
}

int tnt_u1_pack(tnt_ctx* ctx, const tnt_u1_problem* prob, const tnt_cplx* d_theta, tnt_cplx* d_x) {
  if (!ctx) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  if (!d_theta || !d_x) return set_err(c, TNT_E_INVALID, "null pointer");
  U1Spec s;
  TNT_TRY(spec_of(c, prob, &s));
  Scope sc(c);
  TNT_TRY(ws_reserve(c, (size_t)(3 * 8) * (size_t)(s.chl * s.d * s.d) + (1 << 20)));
  return u1_convert(c, s, (const z*)d_theta, (z*)d_x, 1);
}

int tnt_u1_unpack(tnt_ctx* ctx, const tnt_u1_problem* prob, const tnt_cplx* d_x, tnt_cplx* d_theta) {
  if (!ctx) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  if (!d_theta || !d_x) return set_err(c, TNT_E_INVALID, "null pointer");
  U1Spec s;
  TNT_TRY(spec_of(c, prob, &s));
  Scope sc(c);
  TNT_TRY(ws_reserve(c, (size_t)(3 * 8) * (size_t)(s.chl * s.d * s.d) + (1 << 20)));
  return u1_convert(c, s, (const z*)d_x, (z*)d_theta, 0);
}

int tnt_heff_apply_u1(tnt_ctx* ctx, int nprob, const tnt_u1_problem* probs, const tnt_cplx* d_x,
                      tnt_cplx* d_y, int precision, double* h_flops) {
  if (!ctx) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  if (nprob < 1 || !probs || !d_x || !d_y || d_x == d_y)
    return set_err(c, TNT_E_INVALID, "bad problem count or null / aliased vector");
  if (precision != TNT_PREC_FP64 && precision != TNT_PREC_MIXED)
    return set_err(c, TNT_E_INVALID, "bad precision");
  std::vector<U1Spec> specs((size_t)nprob);
  for (int i = 0; i < nprob; ++i) TNT_TRY(spec_of(c, &probs[i], &specs[(size_t)i]));
  Scope sc(c);
  U1Plan p;
  TNT_TRY(u1_layout(c, specs, &p));
  TNT_TRY(ws_reserve(c, p.bytes));
  TNT_TRY(u1_prepare(c, specs, &p));
  if (h_flops) *h_flops = p.flops;
  TNT_TRY(u1_run(c, p, (const z*)d_x, (z*)d_y, precision));
  return status_check(c);
}

int tnt_lanczos_ground_u1(tnt_ctx* ctx, const tnt_u1_problem* prob, tnt_cplx* d_x,
                          tnt_lanczos_result* res) {
  if (!ctx) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  if (!d_x || !res) return set_err(c, TNT_E_INVALID, "null pointer");
  std::vector<U1Spec> specs(1);
  TNT_TRY(spec_of(c, prob, &specs[0]));
  Scope sc(c);
  U1Plan p;
  TNT_TRY(u1_layout(c, specs, &p));
  TNT_TRY(ws_reserve(c, p.bytes + lanczos_scratch_bound(p.n, c->params.krylov_cap)));
  TNT_TRY(u1_prepare(c, specs, &p));
  const int r = lanczos_run(c, U1MatVec(p), (z*)d_x, res);
  TNT_TRY(status_check(c));
  return r;
}

int tnt_lanczos_ground_u1_batched(tnt_ctx* ctx, int nprob, const tnt_u1_problem* probs,
                                  tnt_cplx* d_x, tnt_lanczos_result* h_res) {
  if (!ctx) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  if (nprob < 1 || !probs || !d_x || !h_res) return set_err(c, TNT_E_INVALID, "bad arguments");
  std::vector<U1Spec> specs((size_t)nprob);
  for (int i = 0; i < nprob; ++i) TNT_TRY(spec_of(c, &probs[i], &specs[(size_t)i]));
  Scope sc(c);
  U1Plan p;
  TNT_TRY(u1_layout(c, specs, &p));
  TNT_TRY(ws_reserve(c, p.bytes + lanczos_batched_scratch_bound(p.n, nprob, c->params.krylov_cap)));
  TNT_TRY(u1_prepare(c, specs, &p));
  std::vector<int64_t> off(p.x_off);
  off.push_back(p.n);
  std::vector<tnt_lanczos_result> res;
  TNT_TRY(lanczos_batched(c, U1MatVec(p), off, (z*)d_x, &res));
  TNT_TRY(status_check(c));
  bool all = true;
  for (int i = 0; i < nprob; ++i) {
    h_res[i] = res[(size_t)i];
    all = all && res[(size_t)i].converged;
  }
  return all ? TNT_OK : TNT_E_NOCONV;
}

int tnt_matmul(tnt_ctx* ctx, int64_t M, int64_t N, int64_t K, const tnt_cplx* d_A, int64_t a_rs,
               int64_t a_cs, int conj_a, const tnt_cplx* d_B, int64_t b_rs, int64_t b_cs,
               int conj_b, tnt_cplx* d_C, int64_t c_rs) {
  if (!ctx) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  if (!d_A || !d_B || !d_C || M < 1 || N < 1 || K < 1 || c_rs < N)
    return set_err(c, TNT_E_INVALID, "bad matmul arguments");
  if ((const void*)d_C == (const void*)d_A || (const void*)d_C == (const void*)d_B)
    return set_err(c, TNT_E_INVALID, "matmul output aliases an input");
  ZGemm g{};
  g.M = M; g.N = N; g.K = K;
  g.A = (const z*)d_A; g.a_rs = a_rs; g.a_cs = a_cs; g.conj_a = conj_a ? 1 : 0;
  g.B = (const z*)d_B; g.b_rs = b_rs; g.b_cs = b_cs; g.conj_b = conj_b ? 1 : 0;
  g.C = (z*)d_C; g.c_rs = c_rs;
  g.alpha = zmk(1, 0); g.beta = zmk(0, 0); g.batch = 1;
  TNT_TRY(zgemm(c, g));
  return status_check(c);
}

int tnt_set_fp64_gemm(tnt_ctx* ctx, int engine) {
  if (!ctx) return TNT_E_INVALID;
  if (engine != TNT_FP64_GEMM_FMA && engine != TNT_FP64_GEMM_TC)
    return set_err(&ctx->c, TNT_E_INVALID, "unknown FP64 GEMM engine %d", engine);
  ctx->c.oz_mode = engine;
  return TNT_OK;
}

int tnt_set_graphs(tnt_ctx* ctx, int on) {
  if (!ctx) return TNT_E_INVALID;
  ctx->c.use_graphs = (on != 0);
  return TNT_OK;
}

int tnt_u1_tiles(tnt_ctx* ctx, int nprob, const tnt_u1_problem* probs, int* h_tiles) {
  if (!ctx) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  if (nprob < 1 || !probs || !h_tiles) return set_err(c, TNT_E_INVALID, "bad arguments");
  std::vector<U1Spec> specs((size_t)nprob);
  for (int i = 0; i < nprob; ++i) TNT_TRY(spec_of(c, &probs[i], &specs[(size_t)i]));
  U1Plan p;
  TNT_TRY(u1_layout(c, specs, &p));
  auto it = c->tune.find(p.sig);
  if (it == c->tune.end()) return set_err(c, TNT_E_INVALID, "block structure not tuned yet");
  for (int i = 0; i < 3; ++i) h_tiles[i] = it->second[(size_t)i];
  return TNT_OK;
}

}  // extern "C"
