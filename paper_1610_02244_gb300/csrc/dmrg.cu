// MPO / MPS handles and the two-site DMRG sweep (Sec. 4.3, Listing 2 in two-site form).
// The sweep is host orchestration of the device kernels: theta formation (a1), Lanczos on
// H_eff (a3, a4), truncated SVD (a5, a6) with S renormalised (a7), environment growth (a8).
#include <algorithm>
#include <cmath>
#include <vector>

#include "heff_plan.cuh"
#include "mps.cuh"
#include "u1.cuh"

namespace tnt {

int64_t ipow_cap(int64_t d, int64_t k, int64_t cap) {
  int64_t r = 1;
  for (int64_t i = 0; i < k; ++i) {
    r *= d;
    if (r >= cap) return cap;
  }
  return std::min(r, cap);
}

std::vector<int64_t> labels_or_zero(const tnt_mps* m, int bond) {
  if (m->labelled) return m->q[bond];
  return std::vector<int64_t>((size_t)m->chi[bond], 0);
}

// exact SVD parameters for gauge moves (no truncation beyond exact zeros)
tnt_params exact_params(const tnt_params& p) {
  tnt_params e = p;
  e.chi_max = (int64_t)1 << 40;
  e.trunc_abs = -1.0;
  e.trunc_err = 0.0;
  return e;
}

// grow Lenv over one site: Lout = env_left(Lin, W, A)
static int dmrg_env_left(Ctx* c, tnt_dmrg* g, int i) {
  tnt_mps* m = g->mps;
  size_t top = c->ws.top;
  int r = env_left_impl(c, g->Lenv[i], g->mpo->W[i], m->A[i], m->chi[i], m->d, g->mpo->D,
                        m->chi[i + 1], g->Lenv[i + 1], g->mpo->hW[(size_t)i].data());
  c->ws.top = top;
  return r;
}

static int dmrg_env_right(Ctx* c, tnt_dmrg* g, int j) {
  // Renv[j] from Renv[j+1] and site j
  tnt_mps* m = g->mps;
  size_t top = c->ws.top;
  int r = env_right_impl(c, g->Renv[j + 1], g->mpo->W[j], m->A[j], m->chi[j], m->d, g->mpo->D,
                         m->chi[j + 1], g->Renv[j], g->mpo->hW[(size_t)j].data());
  c->ws.top = top;
  return r;
}

// One two-site update on bond (i, i+1); dir > 0 left-to-right, dir < 0 right-to-left.
static int dmrg_update(Ctx* c, tnt_dmrg* g, int i, int dir, tnt_lanczos_result* lz,
                       tnt_trunc_result* tr, bool marks) {
  tnt_mps* m = g->mps;
  const int64_t d = m->d, D = g->mpo->D;
  const int64_t chl = m->chi[i], chm = m->chi[i + 1], chr = m->chi[i + 2];
  const int64_t n = chl * d * d * chr;
  // labelled bonds with sorted labels: the eigensolve runs on the U(1) blocks only
  std::vector<U1Spec> spec;
  U1Plan up;
  if (m->labelled && (int64_t)g->mpo->wq.size() == D &&
      std::is_sorted(m->q[i].begin(), m->q[i].end()) &&
      std::is_sorted(m->q[i + 2].begin(), m->q[i + 2].end())) {
    spec.resize(1);
    U1Spec& s = spec[0];
    s.L = g->Lenv[i]; s.R = g->Renv[i + 2]; s.W1 = g->mpo->W[i]; s.W2 = g->mpo->W[i + 1];
    s.chl = chl; s.chr = chr; s.d = d; s.D = D;
    s.qa = m->q[i]; s.qb = m->q[i + 2]; s.wq = g->mpo->wq;
    s.hW1 = g->mpo->hW[(size_t)i].data(); s.hW2 = g->mpo->hW[(size_t)i + 1].data();
    TNT_TRY(u1_layout(c, spec, &up));
    if (c->ws.top == 0)
      TNT_TRY(ws_reserve(c, std::max(g->scratch, ws_round(sizeof(z) * n) + ws_round(sizeof(z) * up.n) + up.bytes +
                                                     lanczos_scratch_bound(up.n, c->params.krylov_cap) + (4 << 20))));
  }
  const size_t top = c->ws.top;
  z* theta = (z*)ws_alloc(c, ws_round(sizeof(z) * n));
  if (!theta) return set_err(c, TNT_E_ALLOC, "scratch exhausted (theta)");
  TNT_TRY(theta_form_impl(c, m->A[i], m->A[i + 1], chl, d, chm, chr, theta));
  if (!spec.empty()) {
    size_t t2 = c->ws.top;
    z* x = (z*)ws_alloc(c, ws_round(sizeof(z) * up.n));
    if (!x) return set_err(c, TNT_E_ALLOC, "scratch exhausted (compact theta)");
    TNT_TRY(u1_convert(c, spec[0], theta, x, 1));
    TNT_TRY(u1_prepare(c, spec, &up));
    if (marks) cudaEventRecord(g->ev[1], c->stream);
    c->fp64_finish = true;  // the sweep's energies and states are FP64-accurate
    int r = lanczos_run(c, U1MatVec(up), x, lz);
    c->fp64_finish = false;
    if (r == TNT_E_NAN)  // name the update in the message
      return set_err(c, r, "bond %d (%s, chi %lld|%lld|%lld, compact length %lld): %s", i,
                     dir > 0 ? "left to right" : "right to left", (long long)chl, (long long)chm,
                     (long long)chr, (long long)up.n, std::string(c->err).c_str());
    if (r != TNT_OK && r != TNT_E_NOCONV) return r;
    TNT_TRY(u1_convert(c, spec[0], x, theta, 0));
    c->ws.top = t2;
  } else {
    HeffPlan p;
    size_t t2 = c->ws.top;
    TNT_TRY(heff_prepare(c, g->Lenv[i], g->mpo->W[i], g->mpo->W[i + 1], g->Renv[i + 2], chl, d, D,
                         chr, c->params.precision, &p, g->mpo->hW[(size_t)i].data(),
                         g->mpo->hW[(size_t)i + 1].data()));
    if (marks) cudaEventRecord(g->ev[1], c->stream);
    c->fp64_finish = true;
    int r = lanczos_impl(c, p, theta, lz);
    c->fp64_finish = false;
    if (r != TNT_OK && r != TNT_E_NOCONV) return r;
    c->ws.top = t2;
  }
  if (marks) cudaEventRecord(g->ev[2], c->stream);
  // SVD of M[(a s1), (s2 b)] with labels q_a + s1 and q_b - s2
  std::vector<int64_t> ql = labels_or_zero(m, i), qr = labels_or_zero(m, i + 2);
  std::vector<int64_t> rq((size_t)(chl * d)), cq((size_t)(d * chr));
  for (int64_t a = 0; a < chl; ++a)
    for (int64_t s = 0; s < d; ++s) rq[(size_t)(a * d + s)] = m->labelled ? ql[(size_t)a] + s : 0;
  for (int64_t s = 0; s < d; ++s)
    for (int64_t b = 0; b < chr; ++b) cq[(size_t)(s * chr + b)] = m->labelled ? qr[(size_t)b] - s : 0;
  const int64_t capk = std::min<int64_t>(m->cap[i + 1], std::min(chl * d, d * chr));
  std::vector<double> S((size_t)capk);
  std::vector<int64_t> bq((size_t)capk);
  // U -> A_i (chl x d x k), X -> A_{i+1} (k x d x chr): the kernels write densely with
  // leading dimension k, exactly the site layouts
  {
    tnt_params pp = c->params;  // the site storage bounds the kept dimension
    pp.chi_max = std::min(pp.chi_max, m->cap[i + 1]);
    ParamsGuard pg(c, pp);
    TNT_TRY(svd_trunc_impl(c, theta, chl * d, d * chr, rq.data(), cq.data(),
                           dir > 0 ? TNT_SVD_LEFT : TNT_SVD_RIGHT, 1, m->A[i], m->A[i + 1],
                           S.data(), bq.data(), tr));
  }
  m->chi[i + 1] = tr->chi;
  if (m->labelled) m->q[i + 1].assign(bq.begin(), bq.begin() + tr->chi);
  c->ws.top = top;
  return TNT_OK;
}

// ---------------------------------------------------------------- one-site sweep
// Single-site DMRG with subspace expansion by direct sums (Sec. 4.3 sweep on one site at a
// time; App. B node algebra: the direct sum that expands one leg, and the one that pads a
// leg with zeros).  One-site H_eff.M = L . W . R . M in FP64: T1 = L M (GEMM over a), T2 =
// W T1 (sparse over (w, s)), y = T2 R^T (GEMM over (w', b)).  Left to right, T2 of the
// optimised M scaled by alpha is the expansion term P[(a' s'), (w' b)]: M~ = [M | P], the
// neighbour gets zero rows (so only its first chr rows meet the SVD's S V^H), and the new
// index (w', b) carries the label q_b + wq[w'].  Right to left, the mirror stages give
// P[(w a), (s' b')] with labels q_a + wq[w]: M~ = [M ; P], the left neighbour gets zero
// columns.  The SVD of M~ then decides which of the offered directions to keep.
namespace {
struct OneSitePlan {
  const z* R = nullptr;
  int64_t chl = 0, d = 0, D = 0, chr = 0;
  const z* L = nullptr;
  z* X = nullptr;  // T1, chl D x d chr
  z* Y = nullptr;  // T2, chl d x D chr
  OpApply op{};
};

// T1 = scale L M, T2 = W T1 (the first two stages of the left environment growth)
int onesite_left_stages(Ctx* c, const OneSitePlan& p, const z* M, z scale) {
  ZGemm g{};
  g.M = p.chl * p.D; g.N = p.d * p.chr; g.K = p.chl;
  g.A = p.L; g.a_rs = p.chl; g.a_cs = 1;
  g.B = M; g.b_rs = p.d * p.chr; g.b_cs = 1;
  g.C = p.X; g.c_rs = p.d * p.chr;
  g.alpha = scale; g.beta = zmk(0, 0); g.batch = 1;
  TNT_TRY(zgemm(c, g));
  OpApply a = p.op;
  a.in = p.X;
  a.out = p.Y;
  return op_apply(c, a);
}

int onesite_prepare(Ctx* c, const z* Lenv, const z* Renv, const z* hW, int64_t chl, int64_t d,
                    int64_t D, int64_t chr, OneSitePlan* p) {
  p->L = Lenv;
  p->R = Renv;
  p->chl = chl;
  p->d = d;
  p->D = D;
  p->chr = chr;
  const size_t nx = (size_t)chl * D * d * chr;
  p->X = (z*)ws_alloc(c, ws_round(sizeof(z) * nx));
  p->Y = (z*)ws_alloc(c, ws_round(sizeof(z) * nx));
  if (!p->X || !p->Y) return set_err(c, TNT_E_ALLOC, "scratch exhausted (one-site plan)");
  // Y[a'][(s' w')][m] = sum_{w,s} W[w,w',s',s] X[a'][(w s)][m]
  const int nI = (int)(d * D), nJ = (int)(D * d);
  std::vector<z> op((size_t)nI * nJ);
  for (int64_t so = 0; so < d; ++so)
    for (int64_t wo = 0; wo < D; ++wo)
      for (int64_t w = 0; w < D; ++w)
        for (int64_t s = 0; s < d; ++s)
          op[(size_t)((so * D + wo) * nJ + (w * d + s))] = hW[(size_t)(((w * D + wo) * d + so) * d + s)];
  std::vector<int64_t> in_off(nJ), out_off(nI);
  for (int j = 0; j < nJ; ++j) in_off[j] = (int64_t)j * chr;
  for (int i = 0; i < nI; ++i) out_off[i] = (int64_t)i * chr;
  TNT_TRY(op_upload(c, op, nI, nJ, in_off, out_off, &p->op));
  p->op.B0 = chl; p->op.B1 = 1; p->op.B2 = chr;
  p->op.is0 = D * d * chr; p->op.os0 = d * D * chr;
  p->op.is2 = p->op.os2 = 1;
  return TNT_OK;
}

struct OneSiteMatVec : MatVec {
  const OneSitePlan& p;
  explicit OneSiteMatVec(const OneSitePlan& pp) : p(pp) { n = pp.chl * pp.d * pp.chr; }
  int apply(Ctx* c, const z* x, z* y, int) const override {
    TNT_TRY(onesite_left_stages(c, p, x, zmk(1, 0)));
    // y[(a' s')][b'] = sum_{(w' b)} T2[(a' s')][(w' b)] R[b'][(w' b)]
    ZGemm g{};
    g.M = p.chl * p.d; g.N = p.chr; g.K = p.D * p.chr;
    g.A = p.Y; g.a_rs = p.D * p.chr; g.a_cs = 1;
    g.B = p.R; g.b_rs = 1; g.b_cs = p.D * p.chr;
    g.C = y; g.c_rs = p.chr;
    g.alpha = zmk(1, 0); g.beta = zmk(0, 0); g.batch = 1;
    return zgemm(c, g);
  }
};

// P[(w a)][(s' b')] = scale sum W[w,w',s',s] R[b',w',b] M[a,s,b] (the first two stages of
// the right environment growth), written to out
int onesite_right_expansion(Ctx* c, const z* Renv, const z* hW, const z* M, int64_t chl,
                            int64_t d, int64_t D, int64_t chr, z scale, z* out) {
  const size_t nx = (size_t)chl * d * chr * D;
  z* X = (z*)ws_alloc(c, ws_round(sizeof(z) * nx));
  if (!X) return set_err(c, TNT_E_ALLOC, "scratch exhausted (one-site expansion)");
  ZGemm g{};
  g.M = chl * d; g.N = chr * D; g.K = chr;
  g.A = M; g.a_rs = chr; g.a_cs = 1;
  g.B = Renv; g.b_rs = 1; g.b_cs = chr;
  g.C = X; g.c_rs = chr * D;
  g.alpha = scale; g.beta = zmk(0, 0); g.batch = 1;
  TNT_TRY(zgemm(c, g));
  const int nI = (int)(D * d), nJ = (int)(d * D);
  std::vector<z> op((size_t)nI * nJ);
  for (int64_t w = 0; w < D; ++w)
    for (int64_t so = 0; so < d; ++so)
      for (int64_t s = 0; s < d; ++s)
        for (int64_t wi = 0; wi < D; ++wi)
          op[(size_t)((w * d + so) * nJ + (s * D + wi))] = hW[(size_t)(((w * D + wi) * d + so) * d + s)];
  std::vector<int64_t> in_off(nJ), out_off(nI);
  for (int64_t s = 0; s < d; ++s)
    for (int64_t wi = 0; wi < D; ++wi) in_off[(size_t)(s * D + wi)] = s * chr * D + wi;
  for (int64_t w = 0; w < D; ++w)
    for (int64_t so = 0; so < d; ++so) out_off[(size_t)(w * d + so)] = w * chl * d * chr + so * chr;
  OpApply a{};
  TNT_TRY(op_upload(c, op, nI, nJ, in_off, out_off, &a));
  a.in = X; a.out = out;
  a.B0 = chl; a.B1 = 1; a.B2 = chr;
  a.is0 = d * chr * D; a.is2 = D;
  a.os0 = d * chr; a.os2 = 1;
  return op_apply(c, a);
}
}  // namespace

// one single-site update at site i; dir > 0 hands the centre to i + 1, dir < 0 to i - 1
static int dmrg1_update(Ctx* c, tnt_dmrg* g, int i, int dir, double alpha,
                        tnt_lanczos_result* lz, tnt_trunc_result* tr) {
  tnt_mps* m = g->mps;
  const tnt_mpo* o = g->mpo;
  const int64_t d = m->d, D = o->D, chl = m->chi[i], chr = m->chi[i + 1];
  const int64_t n = chl * d * chr;
  const size_t top = c->ws.top;
  OneSitePlan p;
  TNT_TRY(onesite_prepare(c, g->Lenv[i], g->Renv[i + 1], o->hW[(size_t)i].data(), chl, d, D, chr, &p));
  z* x = (z*)ws_alloc(c, ws_round(sizeof(z) * n));
  if (!x) return set_err(c, TNT_E_ALLOC, "scratch exhausted (one-site tensor)");
  TNT_CUDA_TRY(c, cudaMemcpyAsync(x, m->A[i], sizeof(z) * n, cudaMemcpyDeviceToDevice, c->stream));
  {
    tnt_params pp = c->params;  // the one-site matvec is FP64
    pp.precision = TNT_PREC_FP64;
    ParamsGuard pg(c, pp);
    const int r = lanczos_run(c, OneSiteMatVec(p), x, lz);
    if (r != TNT_OK && r != TNT_E_NOCONV) return r;
  }
  std::vector<int> wq((size_t)D, 0);
  if ((int64_t)o->wq.size() == D) wq = o->wq;
  const z sc = zmk(alpha, 0);
  if (dir > 0) {
    const std::vector<int64_t> ql = labels_or_zero(m, i), qr = labels_or_zero(m, i + 1);
    const int64_t ncol = chr + (alpha > 0 ? D * chr : 0);
    z* Mt = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(chl * d * ncol)));
    if (!Mt) return set_err(c, TNT_E_ALLOC, "scratch exhausted (expanded tensor)");
    TNT_CUDA_TRY(c, cudaMemcpy2DAsync(Mt, sizeof(z) * ncol, x, sizeof(z) * chr, sizeof(z) * chr,
                                      (size_t)(chl * d), cudaMemcpyDeviceToDevice, c->stream));
    std::vector<int64_t> rq((size_t)(chl * d)), cq((size_t)ncol);
    for (int64_t a = 0; a < chl; ++a)
      for (int64_t s = 0; s < d; ++s) rq[(size_t)(a * d + s)] = m->labelled ? ql[(size_t)a] + s : 0;
    for (int64_t b = 0; b < chr; ++b) cq[(size_t)b] = m->labelled ? qr[(size_t)b] : 0;
    if (alpha > 0) {
      TNT_TRY(onesite_left_stages(c, p, x, sc));
      TNT_CUDA_TRY(c, cudaMemcpy2DAsync(Mt + chr, sizeof(z) * ncol, p.Y, sizeof(z) * D * chr,
                                        sizeof(z) * D * chr, (size_t)(chl * d),
                                        cudaMemcpyDeviceToDevice, c->stream));
      for (int64_t w = 0; w < D; ++w)
        for (int64_t b = 0; b < chr; ++b)
          cq[(size_t)(chr + w * chr + b)] = m->labelled ? qr[(size_t)b] + wq[(size_t)w] : 0;
    }
    const int64_t capk = std::min<int64_t>(m->cap[i + 1], std::min(chl * d, ncol));
    z* Xs = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(capk * ncol)));
    if (!Xs) return set_err(c, TNT_E_ALLOC, "scratch exhausted (expanded factor)");
    std::vector<double> S((size_t)capk);
    std::vector<int64_t> bq((size_t)capk);
    {
      tnt_params pp = c->params;
      pp.chi_max = std::min(pp.chi_max, m->cap[i + 1]);
      ParamsGuard pg(c, pp);
      TNT_TRY(svd_trunc_impl(c, Mt, chl * d, ncol, rq.data(), cq.data(), TNT_SVD_LEFT, 1, m->A[i],
                             Xs, S.data(), bq.data(), tr));
    }
    const int64_t k = tr->chi, chn = m->chi[i + 2];
    // A_{i+1} <- (S V^H)[:, :chr] A_{i+1}: the zero rows of the padded neighbour drop out
    z* Bn = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(k * d * chn)));
    if (!Bn) return set_err(c, TNT_E_ALLOC, "scratch exhausted (one-site neighbour)");
    ZGemm gm{};
    gm.M = k; gm.N = d * chn; gm.K = chr;
    gm.A = Xs; gm.a_rs = ncol; gm.a_cs = 1;
    gm.B = m->A[i + 1]; gm.b_rs = d * chn; gm.b_cs = 1;
    gm.C = Bn; gm.c_rs = d * chn;
    gm.alpha = zmk(1, 0); gm.beta = zmk(0, 0); gm.batch = 1;
    TNT_TRY(zgemm(c, gm));
    TNT_CUDA_TRY(c, cudaMemcpyAsync(m->A[i + 1], Bn, sizeof(z) * (size_t)(k * d * chn),
                                    cudaMemcpyDeviceToDevice, c->stream));
    m->chi[i + 1] = k;
    if (m->labelled) m->q[i + 1].assign(bq.begin(), bq.begin() + k);
  } else {
    const std::vector<int64_t> ql = labels_or_zero(m, i), qr = labels_or_zero(m, i + 1);
    const int64_t nrow = chl + (alpha > 0 ? D * chl : 0);
    z* Mt = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(nrow * d * chr)));
    if (!Mt) return set_err(c, TNT_E_ALLOC, "scratch exhausted (expanded tensor)");
    TNT_CUDA_TRY(c, cudaMemcpyAsync(Mt, x, sizeof(z) * n, cudaMemcpyDeviceToDevice, c->stream));
    std::vector<int64_t> rq((size_t)nrow), cq((size_t)(d * chr));
    for (int64_t a = 0; a < chl; ++a) rq[(size_t)a] = m->labelled ? ql[(size_t)a] : 0;
    for (int64_t s = 0; s < d; ++s)
      for (int64_t b = 0; b < chr; ++b) cq[(size_t)(s * chr + b)] = m->labelled ? qr[(size_t)b] - s : 0;
    if (alpha > 0) {
      TNT_TRY(onesite_right_expansion(c, g->Renv[i + 1], o->hW[(size_t)i].data(), x, chl, d, D, chr,
                                      sc, Mt + n));
      for (int64_t w = 0; w < D; ++w)
        for (int64_t a = 0; a < chl; ++a)
          rq[(size_t)(chl + w * chl + a)] = m->labelled ? ql[(size_t)a] + wq[(size_t)w] : 0;
    }
    const int64_t capk = std::min<int64_t>(m->cap[i], std::min(nrow, d * chr));
    z* US = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(nrow * capk)));
    if (!US) return set_err(c, TNT_E_ALLOC, "scratch exhausted (expanded factor)");
    std::vector<double> S((size_t)capk);
    std::vector<int64_t> bq((size_t)capk);
    {
      tnt_params pp = c->params;
      pp.chi_max = std::min(pp.chi_max, m->cap[i]);
      ParamsGuard pg(c, pp);
      TNT_TRY(svd_trunc_impl(c, Mt, nrow, d * chr, rq.data(), cq.data(), TNT_SVD_RIGHT, 1, US,
                             m->A[i], S.data(), bq.data(), tr));
    }
    const int64_t k = tr->chi, chp = m->chi[i - 1];
    // A_{i-1} <- A_{i-1} (U S)[:chl, :]: the zero columns of the padded neighbour drop out
    z* An = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(chp * d * k)));
    if (!An) return set_err(c, TNT_E_ALLOC, "scratch exhausted (one-site neighbour)");
    ZGemm gm{};
    gm.M = chp * d; gm.N = k; gm.K = chl;
    gm.A = m->A[i - 1]; gm.a_rs = chl; gm.a_cs = 1;
    gm.B = US; gm.b_rs = k; gm.b_cs = 1;
    gm.C = An; gm.c_rs = k;
    gm.alpha = zmk(1, 0); gm.beta = zmk(0, 0); gm.batch = 1;
    TNT_TRY(zgemm(c, gm));
    TNT_CUDA_TRY(c, cudaMemcpyAsync(m->A[i - 1], An, sizeof(z) * (size_t)(chp * d * k),
                                    cudaMemcpyDeviceToDevice, c->stream));
    m->chi[i] = k;
    if (m->labelled) m->q[i].assign(bq.begin(), bq.begin() + k);
  }
  c->ws.top = top;
  return TNT_OK;
}

static size_t dmrg1_scratch_bound(const tnt_mps* m, int D, const tnt_params& p) {
  size_t best = 0;
  for (int i = 0; i < m->L; ++i) {
    const int64_t chl = m->cap[i], chr = m->cap[i + 1], d = m->d;
    const int64_t n = chl * d * chr;
    const size_t plan = 2 * ws_round(sizeof(z) * (size_t)(chl * D * d * chr)) + (size_t)(1 << 20);
    size_t b = plan + ws_round(sizeof(z) * n) + lanczos_scratch_bound(n, p.krylov_cap);
    const int64_t wide = chr * (1 + D), tall = chl * (1 + D);
    b = std::max(b, plan + ws_round(sizeof(z) * n) + 3 * ws_round(sizeof(z) * (size_t)(chl * d * wide)) +
                        svd_scratch_bound(chl * d, wide) + ws_round(sizeof(z) * (size_t)(chl * d * chr)));
    b = std::max(b, plan + ws_round(sizeof(z) * n) + 3 * ws_round(sizeof(z) * (size_t)(tall * d * chr)) +
                        svd_scratch_bound(tall, d * chr) + ws_round(sizeof(z) * (size_t)(chl * d * chr * D)));
    best = std::max(best, b);
  }
  return best + (size_t)(8 << 20);
}

static size_t dmrg_scratch_bound(const tnt_mps* m, int D, const tnt_params& p) {
  size_t best = 0;
  for (int i = 0; i + 1 < m->L; ++i) {
    const int64_t chl = m->cap[i], chr = m->cap[i + 2], d = m->d;
    const int64_t n = chl * d * d * chr;
    size_t b = ws_round(sizeof(z) * n) + heff_scratch_bound(chl, d, D, chr, p.precision) +
               lanczos_scratch_bound(n, p.krylov_cap);
    b = std::max(b, ws_round(sizeof(z) * n) + svd_scratch_bound(chl * d, d * chr));
    b = std::max(b, env_scratch_bound(std::max(chl, m->cap[i + 1]), d, D,
                                      std::max(chr, m->cap[i + 1])));
    best = std::max(best, b);
  }
  return best + (size_t)(8 << 20);
}

// sweeps start and end with the centre on site 0 and every right environment current
static int sweep_ready(Ctx* c, const tnt_dmrg* g) {
  if (g->centre != 0 || g->rvalid > 1)
    return set_err(c, TNT_E_INVALID,
                   "a sweep starts with the centre on site 0 (it is on site %d; move it back "
                   "with right-to-left updates)", g->centre);
  return TNT_OK;
}

// One two-site update on bond (i, i+1) of several chains in lock step (the batched form
// of dmrg_update): every chain's theta, one lock-step Lanczos over all chains whose matvec
// is one grouped launch per contraction stage over all their U(1) blocks (with the FP64
// finish of a sweep), then each chain's truncated SVD.  The chains are independent; they
// share only the launches.
static int batched_update(Ctx* c, const std::vector<tnt_dmrg*>& gs, int i, int dir,
                          std::vector<tnt_lanczos_result>* lz, std::vector<tnt_trunc_result>* tr) {
  const int P = (int)gs.size();
  std::vector<U1Spec> specs((size_t)P);
  std::vector<int64_t> nth((size_t)P);
  size_t th_bytes = 0, svd_bytes = 0, scratch = 0;
  for (int p = 0; p < P; ++p) {
    tnt_dmrg* g = gs[(size_t)p];
    tnt_mps* m = g->mps;
    const int64_t d = m->d, D = g->mpo->D;
    const int64_t chl = m->chi[i], chr = m->chi[i + 2];
    U1Spec& sp = specs[(size_t)p];
    sp.L = g->Lenv[i]; sp.R = g->Renv[i + 2]; sp.W1 = g->mpo->W[i]; sp.W2 = g->mpo->W[i + 1];
    sp.chl = chl; sp.chr = chr; sp.d = d; sp.D = D;
    sp.qa = m->q[i]; sp.qb = m->q[i + 2]; sp.wq = g->mpo->wq;
    sp.hW1 = g->mpo->hW[(size_t)i].data(); sp.hW2 = g->mpo->hW[(size_t)i + 1].data();
    nth[(size_t)p] = chl * d * d * chr;
    th_bytes += ws_round(sizeof(z) * nth[(size_t)p]);
    svd_bytes = std::max(svd_bytes, svd_scratch_bound(chl * d, d * chr));
    scratch = std::max(scratch, g->scratch);
  }
  U1Plan up;
  TNT_TRY(u1_layout(c, specs, &up));
  const size_t eig_bytes = ws_round(sizeof(z) * up.n) + up.bytes +
                           lanczos_batched_scratch_bound(up.n, P, c->params.krylov_cap);
  ws_reset(c);
  TNT_TRY(ws_reserve(c, std::max(scratch, th_bytes + std::max(eig_bytes, svd_bytes) + (size_t)(8 << 20))));
  std::vector<z*> th((size_t)P);
  for (int p = 0; p < P; ++p) {
    th[(size_t)p] = (z*)ws_alloc(c, ws_round(sizeof(z) * nth[(size_t)p]));
    if (!th[(size_t)p]) return set_err(c, TNT_E_ALLOC, "scratch exhausted (batched theta)");
  }
  const size_t top = c->ws.top;
  z* x = (z*)ws_alloc(c, ws_round(sizeof(z) * up.n));
  if (!x) return set_err(c, TNT_E_ALLOC, "scratch exhausted (batched compact theta)");
  for (int p = 0; p < P; ++p) {
    tnt_mps* m = gs[(size_t)p]->mps;
    TNT_TRY(theta_form_impl(c, m->A[i], m->A[i + 1], m->chi[i], m->d, m->chi[i + 1], m->chi[i + 2],
                            th[(size_t)p]));
    TNT_TRY(u1_convert(c, specs[(size_t)p], th[(size_t)p], x + up.x_off[(size_t)p], 1));
  }
  TNT_TRY(u1_prepare(c, specs, &up));
  std::vector<int64_t> off(up.x_off);
  off.push_back(up.n);
  c->fp64_finish = true;
  int r = lanczos_batched(c, U1MatVec(up), off, x, lz);
  c->fp64_finish = false;
  if (r != TNT_OK && r != TNT_E_NOCONV) return r;
  for (int p = 0; p < P; ++p)
    TNT_TRY(u1_convert(c, specs[(size_t)p], x + up.x_off[(size_t)p], th[(size_t)p], 0));
  c->ws.top = top;  // the plan's buffers are free again; the thetas stay
  tr->assign((size_t)P, tnt_trunc_result{});
  for (int p = 0; p < P; ++p) {
    tnt_mps* m = gs[(size_t)p]->mps;
    const int64_t d = m->d, chl = m->chi[i], chr = m->chi[i + 2];
    const std::vector<int64_t>& ql = m->q[i];
    const std::vector<int64_t>& qr = m->q[i + 2];
    std::vector<int64_t> rq((size_t)(chl * d)), cq((size_t)(d * chr));
    for (int64_t a = 0; a < chl; ++a)
      for (int64_t s2 = 0; s2 < d; ++s2) rq[(size_t)(a * d + s2)] = ql[(size_t)a] + s2;
    for (int64_t s2 = 0; s2 < d; ++s2)
      for (int64_t b = 0; b < chr; ++b) cq[(size_t)(s2 * chr + b)] = qr[(size_t)b] - s2;
    const int64_t capk = std::min<int64_t>(m->cap[i + 1], std::min(chl * d, d * chr));
    std::vector<double> S((size_t)capk);
    std::vector<int64_t> bq((size_t)capk);
    tnt_params pp = c->params;
    pp.chi_max = std::min(pp.chi_max, m->cap[i + 1]);
    {
      ParamsGuard pg(c, pp);
      const size_t t2 = c->ws.top;
      r = svd_trunc_impl(c, th[(size_t)p], chl * d, d * chr, rq.data(), cq.data(),
                         dir > 0 ? TNT_SVD_LEFT : TNT_SVD_RIGHT, 1, m->A[i], m->A[i + 1], S.data(),
                         bq.data(), &(*tr)[(size_t)p]);
      c->ws.top = t2;
    }
    if (r != TNT_OK) return set_err(c, r, "chain %d, bond %d: %s", p, i, std::string(c->err).c_str());
    m->chi[i + 1] = (*tr)[(size_t)p].chi;
    m->q[i + 1].assign(bq.begin(), bq.begin() + (*tr)[(size_t)p].chi);
  }
  ws_reset(c);
  return TNT_OK;
}

}  // namespace tnt

using namespace tnt;

extern "C" {

int tnt_dmrg_sweep_batched(tnt_ctx* ctx, int n, tnt_dmrg* const* handles, tnt_sweep_stats* stats) {
  if (!ctx || n < 1 || !handles || !stats) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  std::vector<tnt_dmrg*> gs((size_t)n);
  int L = -1;
  for (int p = 0; p < n; ++p) {
    tnt_dmrg* g = handles[p];
    if (!g || g->ctx != ctx) return set_err(c, TNT_E_INVALID, "handle %d is NULL or of another context", p);
    for (int q = 0; q < p; ++q)
      if (handles[q] == g || handles[q]->mps == g->mps)
        return set_err(c, TNT_E_INVALID, "handles %d and %d share an MPS", q, p);
    const tnt_mps* m = g->mps;
    if (L < 0) L = m->L;
    if (m->L != L) return set_err(c, TNT_E_INVALID, "chain %d has %d sites, chain 0 has %d", p, m->L, L);
    if (!m->labelled || (int64_t)g->mpo->wq.size() != g->mpo->D)
      return set_err(c, TNT_E_INVALID, "chain %d: the batched sweep needs U(1) labels on the MPS and the MPO", p);
    for (int k = 0; k <= L; ++k)
      if (!std::is_sorted(m->q[k].begin(), m->q[k].end()))
        return set_err(c, TNT_E_INVALID, "chain %d: labels of bond %d are not sorted", p, k);
    TNT_TRY(sweep_ready(c, g));
    gs[(size_t)p] = g;
    g->last_E.clear();
    stats[p] = tnt_sweep_stats{};
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c->stream);
  std::vector<double> E((size_t)n, 0.0);
  int r = TNT_OK;
  auto account = [&](const std::vector<tnt_lanczos_result>& lz, const std::vector<tnt_trunc_result>& tr) {
    for (int p = 0; p < n; ++p) {
      tnt_sweep_stats& st = stats[p];
      st.total_matvecs += lz[(size_t)p].n_matvec;
      st.unconverged += lz[(size_t)p].converged ? 0 : 1;
      st.max_err = std::max(st.max_err, tr[(size_t)p].err);
      st.max_disc = std::max(st.max_disc, tr[(size_t)p].disc);
      E[(size_t)p] = lz[(size_t)p].E_rq;
      gs[(size_t)p]->last_E.push_back(lz[(size_t)p].E_rq);
    }
  };
  for (int i = 0; i + 1 < L && r == TNT_OK; ++i) {
    std::vector<tnt_lanczos_result> lz;
    std::vector<tnt_trunc_result> tr;
    r = batched_update(c, gs, i, +1, &lz, &tr);
    for (int p = 0; p < n && r == TNT_OK; ++p) r = dmrg_env_left(c, gs[(size_t)p], i);
    if (r == TNT_OK) account(lz, tr);
  }
  for (int i = L - 2; i >= 0 && r == TNT_OK; --i) {
    std::vector<tnt_lanczos_result> lz;
    std::vector<tnt_trunc_result> tr;
    r = batched_update(c, gs, i, -1, &lz, &tr);
    for (int p = 0; p < n && r == TNT_OK; ++p) r = dmrg_env_right(c, gs[(size_t)p], i + 1);
    if (r == TNT_OK) account(lz, tr);
  }
  ws_reset(c);
  cudaEventRecord(e1, c->stream);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int p = 0; p < n; ++p) {
    tnt_dmrg* g = gs[(size_t)p];
    stats[p].seconds = ms * 1e-3;
    stats[p].E = E[(size_t)p];
    stats[p].max_chi = *std::max_element(g->mps->chi.begin(), g->mps->chi.end());
    g->centre = r == TNT_OK ? 0 : -1;
    g->lvalid = 0;
    g->rvalid = r == TNT_OK ? 1 : g->mps->L + 1;
  }
  return r;
}

}  // extern "C"

namespace tnt {
// uploads host site tensors and boundary vectors into a new MPO handle
static int mpo_upload(Ctx* c, int L, int d, int D, const std::vector<std::vector<z>>& sites,
                      const std::vector<z>& lb, const std::vector<z>& rb, std::vector<int> wq,
                      tnt_mpo** out) {
  tnt_mpo* o = new tnt_mpo();
  o->dalloc = c->dalloc;
  o->L = L;
  o->d = d;
  o->D = D;
  o->wq = std::move(wq);
  o->hleft = lb;
  o->hright = rb;
  const size_t nW = (size_t)D * D * d * d;
  for (int j = 0; j < L; ++j) {
    z* dW = nullptr;
    if (dev_alloc(c->dalloc, (void**)&dW, nW * sizeof(z)) != 0) {
      tnt_mpo_destroy(o);
      return set_err(c, TNT_E_ALLOC, "device allocation for the MPO failed");
    }
    o->W.push_back(dW);
    o->hW.push_back(sites[(size_t)j]);
    if (cudaMemcpy(dW, sites[(size_t)j].data(), nW * sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess) {
      tnt_mpo_destroy(o);
      return set_err(c, TNT_E_CUDA, "MPO upload failed");
    }
  }
  if (dev_alloc(c->dalloc, (void**)&o->left, sizeof(z) * D) != 0 ||
      dev_alloc(c->dalloc, (void**)&o->right, sizeof(z) * D) != 0 ||
      cudaMemcpy(o->left, lb.data(), sizeof(z) * D, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(o->right, rb.data(), sizeof(z) * D, cudaMemcpyHostToDevice) != cudaSuccess) {
    tnt_mpo_destroy(o);
    return set_err(c, TNT_E_ALLOC, "MPO boundary upload failed");
  }
  *out = o;
  return TNT_OK;
}

// boundary vectors of the lower-triangular form: left e_{D-1}, right e_0
static void triangular_boundaries(int D, std::vector<z>* lb, std::vector<z>* rb) {
  lb->assign((size_t)D, zmk(0, 0));
  rb->assign((size_t)D, zmk(0, 0));
  (*lb)[(size_t)(D - 1)] = zmk(1, 0);
  (*rb)[0] = zmk(1, 0);
}
}  // namespace tnt

extern "C" {

int tnt_mpo_bose_hubbard(tnt_ctx* ctx, int L, int n_max, double J, double U, double mu, double V,
                         double j_c, tnt_mpo** out) {
  if (!ctx || !out || L < 2 || n_max < 0) return TNT_E_INVALID;
  const int d = n_max + 1, D = 4;
  std::vector<std::vector<z>> sites((size_t)L, std::vector<z>((size_t)D * D * d * d));
  for (int j = 0; j < L; ++j)
    bh_mpo_site_host(n_max, J, U, mu, V, (double)(j + 1), j_c, sites[(size_t)j].data());
  std::vector<z> lb, rb;
  triangular_boundaries(D, &lb, &rb);
  // b+ placed to the left: the bra has one boson more (w = 1)
  return mpo_upload(&ctx->c, L, d, D, sites, lb, rb, {0, 1, -1, 0}, out);
}

int tnt_mpo_spin_heisenberg(tnt_ctx* ctx, int L, int two_s, double J, double Jz, double hz,
                            tnt_mpo** out) {
  if (!ctx || !out || L < 2 || two_s < 1 || two_s > 15) return TNT_E_INVALID;
  const int d = two_s + 1, D = 5;
  std::vector<std::vector<z>> sites((size_t)L, std::vector<z>((size_t)D * D * d * d));
  for (int j = 0; j < L; ++j) spin_mpo_site_host(two_s, J, Jz, hz, sites[(size_t)j].data());
  std::vector<z> lb, rb;
  triangular_boundaries(D, &lb, &rb);
  // channel 1 follows an S+ to the left (the bra carries one quantum more), channel 2 an S-
  return mpo_upload(&ctx->c, L, d, D, sites, lb, rb, {0, 1, -1, 0, 0}, out);
}

int tnt_mpo_create(tnt_ctx* ctx, int L, int d, int D, const tnt_cplx* const* h_W,
                   const tnt_cplx* h_left, const tnt_cplx* h_right, const int* h_wq,
                   tnt_mpo** out) {
  if (!ctx || !out || L < 2 || d < 1 || d > 16 || D < 1 || D > 64 || !h_W || !h_left || !h_right)
    return TNT_E_INVALID;
  const size_t nW = (size_t)D * D * d * d;
  std::vector<std::vector<z>> sites((size_t)L);
  for (int j = 0; j < L; ++j) {
    if (!h_W[j]) return set_err(&ctx->c, TNT_E_INVALID, "MPO site %d is NULL", j);
    const z* w = (const z*)h_W[j];
    sites[(size_t)j].assign(w, w + nW);
  }
  std::vector<z> lb((const z*)h_left, (const z*)h_left + D), rb((const z*)h_right, (const z*)h_right + D);
  std::vector<int> wq;
  if (h_wq) wq.assign(h_wq, h_wq + D);
  return mpo_upload(&ctx->c, L, d, D, sites, lb, rb, std::move(wq), out);
}

int tnt_mpo_destroy(tnt_mpo* mpo) {
  if (!mpo) return TNT_E_INVALID;
  for (z* w : mpo->W) dev_free(mpo->dalloc, w);
  dev_free(mpo->dalloc, mpo->left);
  dev_free(mpo->dalloc, mpo->right);
  delete mpo;
  return TNT_OK;
}

int tnt_mps_create(tnt_ctx* ctx, int L, int d, int64_t chi_cap, const int64_t* h_chi,
                   const tnt_cplx* const* h_sites, const int64_t* const* h_charges, tnt_mps** out) {
  if (!ctx || !out || L < 2 || d < 1 || !h_chi || !h_sites || chi_cap < 1) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  if (h_chi[0] != 1 || h_chi[L] != 1) return set_err(c, TNT_E_INVALID, "boundary bonds must be 1");
  tnt_mps* m = new tnt_mps();
  m->dalloc = c->dalloc;
  m->L = L;
  m->d = d;
  m->chi.assign(h_chi, h_chi + L + 1);
  m->cap.resize(L + 1);
  for (int k = 0; k <= L; ++k) {
    m->cap[k] = std::min(ipow_cap(d, k, chi_cap), ipow_cap(d, L - k, chi_cap));
    if (m->chi[k] < 1 || m->chi[k] > m->cap[k]) {
      tnt_mps_destroy(m);
      return set_err(c, TNT_E_INVALID, "bond %d dimension %lld outside [1, %lld]", k,
                     (long long)h_chi[k], (long long)m->cap[k]);
    }
  }
  m->labelled = (h_charges != nullptr);
  m->q.resize(L + 1);
  if (m->labelled)
    for (int k = 0; k <= L; ++k) m->q[k].assign(h_charges[k], h_charges[k] + m->chi[k]);
  for (int j = 0; j < L; ++j) {
    z* p = nullptr;
    const size_t capn = (size_t)(m->cap[j] * d * m->cap[j + 1]);
    if (dev_alloc(c->dalloc, (void**)&p, capn * sizeof(z)) != 0) {
      tnt_mps_destroy(m);
      return set_err(c, TNT_E_ALLOC, "device allocation for MPS site %d failed", j);
    }
    m->A.push_back(p);
    const size_t nn = (size_t)(m->chi[j] * d * m->chi[j + 1]);
    if (cudaMemcpy(p, h_sites[j], nn * sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess) {
      tnt_mps_destroy(m);
      return set_err(c, TNT_E_CUDA, "copy of MPS site %d failed", j);
    }
  }
  *out = m;
  return TNT_OK;
}

int tnt_mps_product(tnt_ctx* ctx, int L, int d, int64_t chi_cap, const int* h_occ, tnt_mps** out) {
  if (!ctx || !h_occ || L < 2) return TNT_E_INVALID;
  std::vector<int64_t> chi(L + 1, 1);
  std::vector<std::vector<tnt_cplx>> sites(L, std::vector<tnt_cplx>((size_t)d, tnt_cplx{0, 0}));
  std::vector<const tnt_cplx*> ptr(L);
  std::vector<std::vector<int64_t>> q(L + 1, std::vector<int64_t>(1, 0));
  std::vector<const int64_t*> qp(L + 1);
  int64_t tot = 0;
  for (int j = 0; j < L; ++j) {
    if (h_occ[j] < 0 || h_occ[j] >= d) return set_err(&ctx->c, TNT_E_INVALID, "occupation out of range");
    sites[j][(size_t)h_occ[j]] = tnt_cplx{1.0, 0.0};
    ptr[j] = sites[j].data();
    tot += h_occ[j];
    q[j + 1][0] = tot;
  }
  for (int k = 0; k <= L; ++k) qp[k] = q[k].data();
  return tnt_mps_create(ctx, L, d, chi_cap, chi.data(), ptr.data(), qp.data(), out);
}

int tnt_mps_destroy(tnt_mps* m) {
  if (!m) return TNT_E_INVALID;
  for (z* p : m->A) dev_free(m->dalloc, p);
  delete m;
  return TNT_OK;
}

int tnt_mps_length(const tnt_mps* m, int* L, int* d) {
  if (!m || !L || !d) return TNT_E_INVALID;
  *L = m->L;
  *d = m->d;
  return TNT_OK;
}

int tnt_mps_bond_dim(const tnt_mps* m, int bond, int64_t* chi) {
  if (!m || !chi || bond < 0 || bond > m->L) return TNT_E_INVALID;
  *chi = m->chi[bond];
  return TNT_OK;
}

int tnt_mps_get_site(tnt_ctx* ctx, const tnt_mps* m, int site, tnt_cplx* h_out, int64_t cap) {
  if (!ctx || !m || !h_out || site < 0 || site >= m->L) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  const int64_t nn = m->chi[site] * m->d * m->chi[site + 1];
  if (cap < nn) return set_err(c, TNT_E_INVALID, "host buffer holds %lld < %lld", (long long)cap, (long long)nn);
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  TNT_CUDA_TRY(c, cudaMemcpy(h_out, m->A[site], (size_t)nn * sizeof(z), cudaMemcpyDeviceToHost));
  return TNT_OK;
}

int tnt_mps_get_charges(const tnt_mps* m, int bond, int64_t* h_out, int64_t cap) {
  if (!m || !h_out || bond < 0 || bond > m->L || !m->labelled) return TNT_E_INVALID;
  if (cap < m->chi[bond]) return TNT_E_INVALID;
  std::copy(m->q[bond].begin(), m->q[bond].end(), h_out);
  return TNT_OK;
}

int tnt_mps_expect_mpo(tnt_ctx* ctx, const tnt_mps* m, const tnt_mpo* o, double* E) {
  if (!ctx || !m || !o || !E || m->L != o->L || m->d != o->d) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  ws_reset(c);
  int64_t mx = *std::max_element(m->chi.begin(), m->chi.end());
  size_t need = 2 * ws_round(sizeof(z) * (size_t)(mx * o->D * mx)) +
                env_scratch_bound(mx, m->d, o->D, mx);
  TNT_TRY(ws_reserve(c, need));
  z* Ea = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(mx * o->D * mx)));
  z* Eb = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(mx * o->D * mx)));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(Ea, o->left, sizeof(z) * o->D, cudaMemcpyDeviceToDevice, c->stream));
  for (int j = 0; j < m->L; ++j) {
    size_t top = c->ws.top;
    int r = env_left_impl(c, Ea, o->W[j], m->A[j], m->chi[j], m->d, o->D, m->chi[j + 1], Eb,
                          o->hW[(size_t)j].data());
    c->ws.top = top;
    if (r != TNT_OK) { ws_reset(c); return r; }
    std::swap(Ea, Eb);
  }
  std::vector<z> h((size_t)o->D);
  int r = read_small(c, Ea, h.data(), sizeof(z) * o->D);
  ws_reset(c);
  if (r != TNT_OK) return r;
  double e = 0;  // contract with the right boundary vector
  for (int w = 0; w < o->D; ++w) e += h[(size_t)w].x * o->hright[(size_t)w].x - h[(size_t)w].y * o->hright[(size_t)w].y;
  *E = e;
  return TNT_OK;
}

int tnt_mps_norm2(tnt_ctx* ctx, const tnt_mps* m, double* norm2) {
  if (!ctx || !m || !norm2) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  ws_reset(c);
  const int64_t d = m->d;
  int64_t mx = *std::max_element(m->chi.begin(), m->chi.end());
  size_t need = 2 * ws_round(sizeof(z) * (size_t)(mx * mx)) + ws_round(sizeof(z) * d * d) +
                env_scratch_bound(mx, d, 1, mx);
  TNT_TRY(ws_reserve(c, need));
  z* Ea = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(mx * mx)));
  z* Eb = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(mx * mx)));
  z* Wid = (z*)ws_alloc(c, ws_round(sizeof(z) * d * d));
  std::vector<z> hid((size_t)(d * d), zmk(0, 0));
  for (int64_t s = 0; s < d; ++s) hid[(size_t)(s * d + s)] = zmk(1, 0);
  z one = zmk(1, 0);
  TNT_CUDA_TRY(c, cudaMemcpyAsync(Wid, hid.data(), sizeof(z) * d * d, cudaMemcpyHostToDevice, c->stream));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(Ea, &one, sizeof(z), cudaMemcpyHostToDevice, c->stream));
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (int j = 0; j < m->L; ++j) {
    size_t top = c->ws.top;
    int r = env_left_impl(c, Ea, Wid, m->A[j], m->chi[j], d, 1, m->chi[j + 1], Eb);
    c->ws.top = top;
    if (r != TNT_OK) { ws_reset(c); return r; }
    std::swap(Ea, Eb);
  }
  z h;
  int r = read_small(c, Ea, &h, sizeof(z));
  ws_reset(c);
  if (r != TNT_OK) return r;
  *norm2 = h.x;
  return TNT_OK;
}

int tnt_dmrg_create(tnt_ctx* ctx, tnt_mps* m, const tnt_mpo* o, tnt_dmrg** out) {
  if (!ctx || !m || !o || !out || m->L != o->L || m->d != o->d) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  tnt_dmrg* g = new tnt_dmrg();
  g->ctx = ctx;
  g->dalloc = c->dalloc;
  g->mps = m;
  g->mpo = o;
  const int L = m->L;
  g->Lenv.assign(L + 1, nullptr);
  g->Renv.assign(L + 1, nullptr);
  for (cudaEvent_t& e : g->ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      tnt_dmrg_destroy(g);
      return set_err(c, TNT_E_CUDA, "event creation failed");
    }
  for (int k = 0; k <= L; ++k) {
    const size_t ne = (size_t)(m->cap[k] * o->D * m->cap[k]);
    if (dev_alloc(c->dalloc, (void**)&g->Lenv[k], ne * sizeof(z)) != 0 ||
        dev_alloc(c->dalloc, (void**)&g->Renv[k], ne * sizeof(z)) != 0) {
      tnt_dmrg_destroy(g);
      return set_err(c, TNT_E_ALLOC, "device allocation for environments failed");
    }
  }
  g->scratch = dmrg_scratch_bound(m, o->D, c->params);
  ws_reset(c);
  int r = ws_reserve(c, g->scratch);
  if (r != TNT_OK) { tnt_dmrg_destroy(g); return r; }
  // right-canonical form by exact SVD moves from the right end, then unit norm
  {
    ParamsGuard pg(c, exact_params(c->params));
    const int64_t d = m->d;
    for (int j = L - 1; j >= 1; --j) {
      const int64_t chl = m->chi[j], chr = m->chi[j + 1];
      std::vector<int64_t> ql = labels_or_zero(m, j), qr = labels_or_zero(m, j + 1);
      std::vector<int64_t> cq((size_t)(d * chr));
      for (int64_t s = 0; s < d; ++s)
        for (int64_t b = 0; b < chr; ++b) cq[(size_t)(s * chr + b)] = m->labelled ? qr[(size_t)b] - s : 0;
      const int64_t capk = std::min(chl, d * chr);
      std::vector<double> S((size_t)capk);
      std::vector<int64_t> bq((size_t)capk);
      z* M = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(chl * d * chr)));
      z* US = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(chl * capk)));
      z* Anew = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(m->chi[j - 1] * d * capk)));
      if (!M || !US || !Anew) { ws_reset(c); tnt_dmrg_destroy(g); return set_err(c, TNT_E_ALLOC, "scratch (canonicalise)"); }
      cudaMemcpyAsync(M, m->A[j], sizeof(z) * (size_t)(chl * d * chr), cudaMemcpyDeviceToDevice, c->stream);
      tnt_trunc_result tr{};
      r = svd_trunc_impl(c, M, chl, d * chr, ql.data(), cq.data(), TNT_SVD_RIGHT, 0, US, m->A[j],
                         S.data(), bq.data(), &tr);
      if (r != TNT_OK) { ws_reset(c); tnt_dmrg_destroy(g); return r; }
      const int64_t k = tr.chi;
      // A_{j-1} <- A_{j-1} (US)
      ZGemm gm{};
      gm.M = m->chi[j - 1] * d; gm.N = k; gm.K = chl;
      gm.A = m->A[j - 1]; gm.a_rs = chl; gm.a_cs = 1;
      gm.B = US; gm.b_rs = k; gm.b_cs = 1;
      gm.C = Anew; gm.c_rs = k;
      gm.alpha = zmk(1, 0); gm.beta = zmk(0, 0); gm.batch = 1;
      r = zgemm(c, gm);
      if (r != TNT_OK) { ws_reset(c); tnt_dmrg_destroy(g); return r; }
      cudaMemcpyAsync(m->A[j - 1], Anew, sizeof(z) * (size_t)(m->chi[j - 1] * d * k), cudaMemcpyDeviceToDevice, c->stream);
      m->chi[j] = k;
      if (m->labelled) m->q[j].assign(bq.begin(), bq.begin() + k);
      ws_reset(c);
      TNT_TRY(ws_reserve(c, g->scratch));
    }
    // normalise site 0
    const int64_t n0 = m->chi[0] * d * m->chi[1];
    double* nrm = (double*)ws_alloc(c, 256);
    r = vec_norm2(c, m->A[0], n0, nrm);
    if (r == TNT_OK) r = zscale_inplace(c, m->A[0], n0, nrm, 1);
    ws_reset(c);
    if (r != TNT_OK) { tnt_dmrg_destroy(g); return r; }
  }
  // environments
  TNT_CUDA_TRY(c, cudaMemcpyAsync(g->Lenv[0], o->left, sizeof(z) * o->D, cudaMemcpyDeviceToDevice, c->stream));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(g->Renv[L], o->right, sizeof(z) * o->D, cudaMemcpyDeviceToDevice, c->stream));
  for (int j = L - 1; j >= 1; --j) {
    r = dmrg_env_right(c, g, j);
    if (r != TNT_OK) { ws_reset(c); tnt_dmrg_destroy(g); return r; }
  }
  ws_reset(c);
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  g->centre = 0;
  g->lvalid = 0;
  g->rvalid = 1;
  *out = g;
  return TNT_OK;
}

int tnt_dmrg_update(tnt_ctx* ctx, tnt_dmrg* g, int bond, int dir, tnt_lanczos_result* lz,
                    tnt_trunc_result* tr) {
  if (!ctx || !g || !lz || !tr || g->ctx != ctx) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  tnt_mps* m = g->mps;
  const int i = bond;
  if (i < 0 || i + 1 >= m->L || (dir != 1 && dir != -1))
    return set_err(c, TNT_E_INVALID, "bond %d / direction %d (bonds 0..%d, direction +1 or -1)",
                   bond, dir, m->L - 2);
  if ((g->centre != i && g->centre != i + 1) || g->lvalid < i || g->rvalid > i + 2)
    return set_err(c, TNT_E_INVALID,
                   "bond %d needs the centre on site %d or %d and its environments current "
                   "(centre on site %d)", i, i, i + 1, g->centre);
  *lz = tnt_lanczos_result{};
  *tr = tnt_trunc_result{};
  ws_reset(c);
  TNT_TRY(ws_reserve(c, g->scratch));
  int r = dmrg_update(c, g, i, dir, lz, tr, false);
  if (r == TNT_OK) r = dir > 0 ? dmrg_env_left(c, g, i) : dmrg_env_right(c, g, i + 1);
  ws_reset(c);
  if (r != TNT_OK) return r;
  if (dir > 0) {
    g->centre = i + 1;
    g->lvalid = i + 1;
    g->rvalid = std::max(g->rvalid, i + 2);
  } else {
    g->centre = i;
    g->rvalid = i + 1;
    g->lvalid = std::min(g->lvalid, i);
  }
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return lz->converged ? TNT_OK : TNT_E_NOCONV;
}

int tnt_dmrg_sweep(tnt_ctx* ctx, tnt_dmrg* g, tnt_sweep_stats* st) {
  if (!ctx || !g || !st || g->ctx != ctx) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  TNT_TRY(sweep_ready(c, g));
  tnt_mps* m = g->mps;
  const int L = m->L;
  *st = tnt_sweep_stats{};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c->stream);
  ws_reset(c);
  g->last_E.clear();
  TNT_TRY(ws_reserve(c, g->scratch));
  double E = 0;
  auto account = [&](const tnt_lanczos_result& lz, const tnt_trunc_result& tr) {
    st->total_matvecs += lz.n_matvec;
    st->unconverged += lz.converged ? 0 : 1;
    st->max_err = std::max(st->max_err, tr.err);
    st->max_disc = std::max(st->max_disc, tr.disc);
    E = lz.E_rq;
  };
  // phase marks: ev[0] update start, ev[1] eigensolve start, ev[2] eigensolve end,
  // ev[3] SVD end, ev[4] environment end (the update already synchronises on its SVD)
  auto phases = [&]() {
    float a = 0, b = 0, d = 0, e = 0;
    cudaEventSynchronize(g->ev[4]);
    cudaEventElapsedTime(&a, g->ev[0], g->ev[1]);
    cudaEventElapsedTime(&b, g->ev[1], g->ev[2]);
    cudaEventElapsedTime(&d, g->ev[2], g->ev[3]);
    cudaEventElapsedTime(&e, g->ev[3], g->ev[4]);
    st->t_plan += 1e-3 * a;
    st->t_eig += 1e-3 * b;
    st->t_svd += 1e-3 * d;
    st->t_env += 1e-3 * e;
  };
  int r = TNT_OK;
  for (int i = 0; i + 1 < L && r == TNT_OK; ++i) {
    tnt_lanczos_result lz{};
    tnt_trunc_result tr{};
    cudaEventRecord(g->ev[0], c->stream);
    r = dmrg_update(c, g, i, +1, &lz, &tr, true);
    cudaEventRecord(g->ev[3], c->stream);
    if (r == TNT_OK) r = dmrg_env_left(c, g, i);
    cudaEventRecord(g->ev[4], c->stream);
    if (r == TNT_OK) phases();
    account(lz, tr);
    if (r == TNT_OK) g->last_E.push_back(lz.E_rq);
  }
  for (int i = L - 2; i >= 0 && r == TNT_OK; --i) {
    tnt_lanczos_result lz{};
    tnt_trunc_result tr{};
    cudaEventRecord(g->ev[0], c->stream);
    r = dmrg_update(c, g, i, -1, &lz, &tr, true);
    cudaEventRecord(g->ev[3], c->stream);
    if (r == TNT_OK) r = dmrg_env_right(c, g, i + 1);
    cudaEventRecord(g->ev[4], c->stream);
    if (r == TNT_OK) phases();
    account(lz, tr);
    if (r == TNT_OK) g->last_E.push_back(lz.E_rq);
  }
  ws_reset(c);
  cudaEventRecord(e1, c->stream);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  st->seconds = ms * 1e-3;
  st->E = E;
  st->max_chi = *std::max_element(m->chi.begin(), m->chi.end());
  // a sweep that stopped at an error leaves the gauge unknown: no single update until the
  // next full sweep is asked for, which then reports the state instead of running
  g->centre = r == TNT_OK ? 0 : -1;
  g->lvalid = 0;
  g->rvalid = r == TNT_OK ? 1 : m->L + 1;
  return r;
}

int tnt_dmrg_sweep1(tnt_ctx* ctx, tnt_dmrg* g, double alpha, tnt_sweep_stats* st) {
  if (!ctx || !g || !st || g->ctx != ctx || !(alpha >= 0) || !std::isfinite(alpha)) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  TNT_TRY(sweep_ready(c, g));
  tnt_mps* m = g->mps;
  const int L = m->L;
  *st = tnt_sweep_stats{};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c->stream);
  ws_reset(c);
  g->last_E.clear();
  TNT_TRY(ws_reserve(c, std::max(g->scratch, dmrg1_scratch_bound(m, g->mpo->D, c->params))));
  double E = 0;
  auto account = [&](const tnt_lanczos_result& lz, const tnt_trunc_result& tr) {
    st->total_matvecs += lz.n_matvec;
    st->unconverged += lz.converged ? 0 : 1;
    st->max_err = std::max(st->max_err, tr.err);
    st->max_disc = std::max(st->max_disc, tr.disc);
    E = lz.E_rq;
  };
  int r = TNT_OK;
  for (int i = 0; i + 1 < L && r == TNT_OK; ++i) {
    tnt_lanczos_result lz{};
    tnt_trunc_result tr{};
    r = dmrg1_update(c, g, i, +1, alpha, &lz, &tr);
    if (r == TNT_OK) r = dmrg_env_left(c, g, i);
    account(lz, tr);
    if (r == TNT_OK) g->last_E.push_back(lz.E_rq);
  }
  for (int i = L - 1; i >= 1 && r == TNT_OK; --i) {
    tnt_lanczos_result lz{};
    tnt_trunc_result tr{};
    r = dmrg1_update(c, g, i, -1, alpha, &lz, &tr);
    if (r == TNT_OK) r = dmrg_env_right(c, g, i);
    account(lz, tr);
    if (r == TNT_OK) g->last_E.push_back(lz.E_rq);
  }
  ws_reset(c);
  cudaEventRecord(e1, c->stream);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  st->seconds = ms * 1e-3;
  st->E = E;
  st->max_chi = *std::max_element(m->chi.begin(), m->chi.end());
  g->centre = r == TNT_OK ? 0 : -1;
  g->lvalid = 0;
  g->rvalid = r == TNT_OK ? 1 : m->L + 1;
  return r;
}

int tnt_dmrg_update_energies(const tnt_dmrg* g, double* h_E, int64_t cap, int64_t* n) {
  if (!g || !n || cap < 0 || (cap > 0 && !h_E)) return TNT_E_INVALID;
  *n = (int64_t)g->last_E.size();
  const int64_t k = std::min(cap, *n);
  for (int64_t i = 0; i < k; ++i) h_E[i] = g->last_E[(size_t)i];
  return TNT_OK;
}

int tnt_dmrg_destroy(tnt_dmrg* g) {
  if (!g) return TNT_E_INVALID;
  for (cudaEvent_t e : g->ev)
    if (e) cudaEventDestroy(e);
  for (z* p : g->Lenv) dev_free(g->dalloc, p);
  for (z* p : g->Renv) dev_free(g->dalloc, p);
  delete g;
  return TNT_OK;
}

}  // extern "C"
