// Second-order Trotter TEBD on the device MPS handle (Sec. 3, Trotterised update; Sec. 5,
// real-time evolution from a product state with the accumulated truncation error and
// 1 - <psi|psi> tracked).  The paper names the update but prints no scheme; the step is the
// symmetric split
//   U(dt) = exp(-i H_odd dt/2) exp(-i H_even dt) exp(-i H_odd dt/2),
// odd bonds (1,2), (3,4), ... and even bonds (2,3), ... (1-based), hbar = 1.  The bond term
// carries the on-site energy with weight 1/2 in the interior and 1 on the two end sites.
// Each gate: move the orthogonality centre to site i by exact SVD moves, theta = A_i A_{i+1}
// (a1), theta' = G theta (a2), truncated SVD of theta'[(a s1),(s2 b)] (a5, a6), A_i <- U,
// A_{i+1} <- S V^H (a7).  No renormalisation: the discarded weight leaves the norm.
#include <algorithm>
#include <cmath>
#include <vector>

#include "heff_plan.cuh"
#include "mps.cuh"

struct tnt_tebd {
  tnt_ctx* ctx = nullptr;
  tnt_mps* mps = nullptr;
  int centre = 0;
  bool up = true;  // direction of the next layer (alternates layer by layer, across steps)
  std::vector<std::vector<tnt::z>> G_half, G_full;  // per bond, d^2 x d^2 (host)
  size_t scratch = 0;
};

namespace tnt {

static size_t tebd_scratch_bound(const tnt_mps* m) {
  size_t best = 0;
  const int64_t d = m->d;
  for (int i = 0; i + 1 < m->L; ++i) {
    const int64_t chl = m->cap[i], chr = m->cap[i + 2];
    const int64_t n = chl * d * d * chr;
    best = std::max(best, 2 * ws_round(sizeof(z) * n) + svd_scratch_bound(chl * d, d * chr));
  }
  // centre moves: the site copy, the factor and the product each fit in the largest site
  int64_t site = 0;
  for (int j = 0; j < m->L; ++j) site = std::max(site, m->cap[j] * d * m->cap[j + 1]);
  for (int j = 0; j < m->L; ++j) {
    const int64_t chl = m->cap[j], chr = m->cap[j + 1];
    best = std::max(best, 3 * ws_round(sizeof(z) * site) +
                              std::max(svd_scratch_bound(chl * d, chr), svd_scratch_bound(chl, d * chr)));
  }
  return best + (size_t)(8 << 20);
}

// centre j -> j+1:  A_j = U (left-orthonormal), A_{j+1} <- (S V^H) A_{j+1}
static int tebd_move_right(Ctx* c, tnt_tebd* t) {
  tnt_mps* m = t->mps;
  const int j = t->centre;
  const int64_t d = m->d, chl = m->chi[j], chr = m->chi[j + 1], chn = m->chi[j + 2];
  const size_t top = c->ws.top;
  std::vector<int64_t> ql = labels_or_zero(m, j), qr = labels_or_zero(m, j + 1);
  std::vector<int64_t> rq((size_t)(chl * d));
  for (int64_t a = 0; a < chl; ++a)
    for (int64_t s = 0; s < d; ++s) rq[(size_t)(a * d + s)] = m->labelled ? ql[(size_t)a] + s : 0;
  const int64_t capk = std::min(chl * d, chr);
  z* M = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(chl * d * chr)));
  z* X = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(capk * chr)));
  z* B = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(capk * d * chn)));
  if (!M || !X || !B) return set_err(c, TNT_E_ALLOC, "scratch exhausted (centre move)");
  TNT_CUDA_TRY(c, cudaMemcpyAsync(M, m->A[j], sizeof(z) * (size_t)(chl * d * chr),
                                  cudaMemcpyDeviceToDevice, c->stream));
  std::vector<double> S((size_t)capk);
  std::vector<int64_t> bq((size_t)capk);
  tnt_trunc_result tr{};
  {
    ParamsGuard pg(c, exact_params(c->params));
    TNT_TRY(svd_trunc_impl(c, M, chl * d, chr, rq.data(), qr.data(), TNT_SVD_LEFT, 0, m->A[j], X,
                           S.data(), bq.data(), &tr));
  }
  const int64_t k = tr.chi;
  ZGemm g{};
  g.M = k; g.N = d * chn; g.K = chr;
  g.A = X; g.a_rs = chr; g.a_cs = 1;
  g.B = m->A[j + 1]; g.b_rs = d * chn; g.b_cs = 1;
  g.C = B; g.c_rs = d * chn;
  g.alpha = zmk(1, 0); g.beta = zmk(0, 0); g.batch = 1;
  TNT_TRY(zgemm(c, g));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(m->A[j + 1], B, sizeof(z) * (size_t)(k * d * chn),
                                  cudaMemcpyDeviceToDevice, c->stream));
  m->chi[j + 1] = k;
  if (m->labelled) m->q[j + 1].assign(bq.begin(), bq.begin() + k);
  t->centre = j + 1;
  c->ws.top = top;
  return TNT_OK;
}

// centre j -> j-1:  A_j = V^H (right-orthonormal), A_{j-1} <- A_{j-1} (U S)
static int tebd_move_left(Ctx* c, tnt_tebd* t) {
  tnt_mps* m = t->mps;
  const int j = t->centre;
  const int64_t d = m->d, chl = m->chi[j], chr = m->chi[j + 1], chp = m->chi[j - 1];
  const size_t top = c->ws.top;
  std::vector<int64_t> ql = labels_or_zero(m, j), qr = labels_or_zero(m, j + 1);
  std::vector<int64_t> cq((size_t)(d * chr));
  for (int64_t s = 0; s < d; ++s)
    for (int64_t b = 0; b < chr; ++b) cq[(size_t)(s * chr + b)] = m->labelled ? qr[(size_t)b] - s : 0;
  const int64_t capk = std::min(chl, d * chr);
  z* M = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(chl * d * chr)));
  z* US = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(chl * capk)));
  z* A = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(chp * d * capk)));
  if (!M || !US || !A) return set_err(c, TNT_E_ALLOC, "scratch exhausted (centre move)");
  TNT_CUDA_TRY(c, cudaMemcpyAsync(M, m->A[j], sizeof(z) * (size_t)(chl * d * chr),
                                  cudaMemcpyDeviceToDevice, c->stream));
  std::vector<double> S((size_t)capk);
  std::vector<int64_t> bq((size_t)capk);
  tnt_trunc_result tr{};
  {
    ParamsGuard pg(c, exact_params(c->params));
    TNT_TRY(svd_trunc_impl(c, M, chl, d * chr, ql.data(), cq.data(), TNT_SVD_RIGHT, 0, US,
                           m->A[j], S.data(), bq.data(), &tr));
  }
  const int64_t k = tr.chi;
  ZGemm g{};
  g.M = chp * d; g.N = k; g.K = chl;
  g.A = m->A[j - 1]; g.a_rs = chl; g.a_cs = 1;
  g.B = US; g.b_rs = k; g.b_cs = 1;
  g.C = A; g.c_rs = k;
  g.alpha = zmk(1, 0); g.beta = zmk(0, 0); g.batch = 1;
  TNT_TRY(zgemm(c, g));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(m->A[j - 1], A, sizeof(z) * (size_t)(chp * d * k),
                                  cudaMemcpyDeviceToDevice, c->stream));
  m->chi[j] = k;
  if (m->labelled) m->q[j].assign(bq.begin(), bq.begin() + k);
  t->centre = j - 1;
  c->ws.top = top;
  return TNT_OK;
}

// one gate on bond (i, i+1): the centre is moved into {i, i+1} (theta = A_i A_{i+1} is
// then the centre's two-site tensor); side TNT_SVD_LEFT leaves it at i+1 (A_i <- U,
// A_{i+1} <- S V^H), TNT_SVD_RIGHT at i (A_i <- U S, A_{i+1} <- V^H)
static int tebd_gate(Ctx* c, tnt_tebd* t, int i, const std::vector<z>& G, int side,
                     tnt_step_stats* st, tnt_trunc_result* tr_out = nullptr) {
  tnt_mps* m = t->mps;
  while (t->centre < i) TNT_TRY(tebd_move_right(c, t));
  while (t->centre > i + 1) TNT_TRY(tebd_move_left(c, t));
  const int64_t d = m->d, chl = m->chi[i], chm = m->chi[i + 1], chr = m->chi[i + 2];
  const int64_t n = chl * d * d * chr;
  const size_t top = c->ws.top;
  z* theta = (z*)ws_alloc(c, ws_round(sizeof(z) * n));
  z* theta2 = (z*)ws_alloc(c, ws_round(sizeof(z) * n));
  if (!theta || !theta2) return set_err(c, TNT_E_ALLOC, "scratch exhausted (theta)");
  TNT_TRY(theta_form_impl(c, m->A[i], m->A[i + 1], chl, d, chm, chr, theta));
  TNT_TRY(gate_apply_impl(c, G, theta, chl, d, chr, theta2));
  std::vector<int64_t> ql = labels_or_zero(m, i), qr = labels_or_zero(m, i + 2);
  std::vector<int64_t> rq((size_t)(chl * d)), cq((size_t)(d * chr));
  for (int64_t a = 0; a < chl; ++a)
    for (int64_t s = 0; s < d; ++s) rq[(size_t)(a * d + s)] = m->labelled ? ql[(size_t)a] + s : 0;
  for (int64_t s = 0; s < d; ++s)
    for (int64_t b = 0; b < chr; ++b) cq[(size_t)(s * chr + b)] = m->labelled ? qr[(size_t)b] - s : 0;
  const int64_t capk = std::min<int64_t>(m->cap[i + 1], std::min(chl * d, d * chr));
  std::vector<double> S((size_t)capk);
  std::vector<int64_t> bq((size_t)capk);
  tnt_trunc_result tr{};
  {
    tnt_params pp = c->params;  // the site storage bounds the kept dimension
    pp.chi_max = std::min(pp.chi_max, m->cap[i + 1]);
    ParamsGuard pg(c, pp);
    TNT_TRY(svd_trunc_impl(c, theta2, chl * d, d * chr, rq.data(), cq.data(), side, 0,
                           m->A[i], m->A[i + 1], S.data(), bq.data(), &tr));
  }
  m->chi[i + 1] = tr.chi;
  if (m->labelled) m->q[i + 1].assign(bq.begin(), bq.begin() + tr.chi);
  t->centre = (side == TNT_SVD_LEFT) ? i + 1 : i;
  st->err_sum += tr.err;
  st->disc_sum += tr.disc;
  if (tr_out) *tr_out = tr;
  c->ws.top = top;
  return TNT_OK;
}

}  // namespace tnt

using namespace tnt;

extern "C" {

}  // extern "C"

namespace tnt {
// gates from per-bond Hamiltonians (rows (s1' s2'), columns (s1 s2)), then the
// orthogonality centre to site 0 by exact right-to-left moves (a gauge change only)
static int tebd_from_bonds(tnt_ctx* ctx, tnt_mps* m, const std::vector<std::vector<z>>& h,
                           double dt, tnt_tebd** out) {
  Ctx* c = &ctx->c;
  const int L = m->L, d2 = m->d * m->d;
  tnt_tebd* t = new tnt_tebd();
  t->ctx = ctx;
  t->mps = m;
  t->G_half.assign((size_t)(L - 1), std::vector<z>((size_t)d2 * d2));
  t->G_full.assign((size_t)(L - 1), std::vector<z>((size_t)d2 * d2));
  for (int i = 0; i + 1 < L; ++i) {
    bond_gate_host(d2, h[(size_t)i].data(), 0.5 * dt, t->G_half[(size_t)i].data());
    bond_gate_host(d2, h[(size_t)i].data(), dt, t->G_full[(size_t)i].data());
  }
  t->scratch = tebd_scratch_bound(m);
  ws_reset(c);
  int r = ws_reserve(c, t->scratch);
  t->centre = L - 1;
  while (r == TNT_OK && t->centre > 0) r = tebd_move_left(c, t);
  ws_reset(c);
  if (r == TNT_OK) r = cudaStreamSynchronize(c->stream) == cudaSuccess ? TNT_OK : TNT_E_CUDA;
  if (r != TNT_OK) {
    delete t;
    return r;
  }
  *out = t;
  return TNT_OK;
}

// on-site weights of the bond terms: 1/2 in the interior, 1 on the two end sites
static void bond_weights(int L, int i, double* c1, double* c2) {
  *c1 = (i == 0) ? 1.0 : 0.5;
  *c2 = (i + 2 == L) ? 1.0 : 0.5;
}
}  // namespace tnt

extern "C" {

int tnt_tebd_create(tnt_ctx* ctx, tnt_mps* m, int n_max, double J, double U, double mu,
                    double dt, tnt_tebd** out) {
  if (!ctx || !m || !out || n_max + 1 != m->d || !std::isfinite(dt)) return TNT_E_INVALID;
  if (m->d * m->d > 256) return set_err(&ctx->c, TNT_E_INVALID, "d^2 = %d exceeds 256", m->d * m->d);
  const int L = m->L, d = m->d, d2 = d * d;
  std::vector<std::vector<z>> h((size_t)(L - 1), std::vector<z>((size_t)d2 * d2));
  std::vector<double> b((size_t)d * d, 0.0);  // <s'|b|s>
  for (int n = 1; n < d; ++n) b[(size_t)(n - 1) * d + n] = std::sqrt((double)n);
  auto hs = [&](int s) { return 0.5 * U * s * (s - 1) - mu * s; };
  for (int i = 0; i + 1 < L; ++i) {
    double c1, c2;
    bond_weights(L, i, &c1, &c2);
    // -J (b+ (x) b + b (x) b+) + c1 h_site (x) 1 + c2 1 (x) h_site
    for (int s1o = 0; s1o < d; ++s1o)
      for (int s2o = 0; s2o < d; ++s2o)
        for (int s1 = 0; s1 < d; ++s1)
          for (int s2 = 0; s2 < d; ++s2) {
            double v = -J * (b[(size_t)s1 * d + s1o] * b[(size_t)s2o * d + s2] +
                             b[(size_t)s1o * d + s1] * b[(size_t)s2 * d + s2o]);
            if (s1o == s1 && s2o == s2) v += c1 * hs(s1) + c2 * hs(s2);
            h[(size_t)i][(size_t)(s1o * d + s2o) * d2 + (s1 * d + s2)] = zmk(v, 0);
          }
  }
  return tebd_from_bonds(ctx, m, h, dt, out);
}

int tnt_tebd_create_spin(tnt_ctx* ctx, tnt_mps* m, int two_s, double J, double Jz, double hz,
                         double dt, tnt_tebd** out) {
  if (!ctx || !m || !out || two_s < 1 || two_s + 1 != m->d || !std::isfinite(dt))
    return TNT_E_INVALID;
  const int L = m->L, d2 = m->d * m->d;
  std::vector<std::vector<z>> h((size_t)(L - 1), std::vector<z>((size_t)d2 * d2));
  for (int i = 0; i + 1 < L; ++i) {
    double c1, c2;
    bond_weights(L, i, &c1, &c2);
    spin_bond_h_host(two_s, J, Jz, hz, c1, c2, h[(size_t)i].data());
  }
  return tebd_from_bonds(ctx, m, h, dt, out);
}

int tnt_tebd_create_bonds(tnt_ctx* ctx, tnt_mps* m, const tnt_cplx* const* h_bond, double dt,
                          tnt_tebd** out) {
  if (!ctx || !m || !out || !h_bond || !std::isfinite(dt)) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  if (m->d * m->d > 256) return set_err(c, TNT_E_INVALID, "d^2 = %d exceeds 256", m->d * m->d);
  const int L = m->L;
  const size_t n2 = (size_t)m->d * m->d * m->d * m->d;
  std::vector<std::vector<z>> h((size_t)(L - 1));
  for (int i = 0; i + 1 < L; ++i) {
    if (!h_bond[i]) return set_err(c, TNT_E_INVALID, "bond term %d is NULL", i);
    const z* p = (const z*)h_bond[i];
    for (size_t e = 0; e < n2; ++e)
      if (!std::isfinite(p[e].x) || !std::isfinite(p[e].y))
        return set_err(c, TNT_E_NAN, "bond term %d has a non-finite entry", i);
    h[(size_t)i].assign(p, p + n2);
  }
  return tebd_from_bonds(ctx, m, h, dt, out);
}

int tnt_tebd_step(tnt_ctx* ctx, tnt_tebd* t, tnt_step_stats* st) {
  if (!ctx || !t || !st || t->ctx != ctx) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  tnt_mps* m = t->mps;
  const int L = m->L;
  *st = tnt_step_stats{};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c->stream);
  ws_reset(c);
  int r = ws_reserve(c, t->scratch);
  // odd bonds (0-based i even) at dt/2, even bonds at dt, odd bonds at dt/2.  The gates of
  // a layer commute; each layer runs opposite to the one before (ascending gates leave the
  // centre on their right site, descending ones on their left), so consecutive gates are
  // one centre move apart and no layer starts with a walk across the chain.
  for (int layer = 0; layer < 3 && r == TNT_OK; ++layer) {
    const int first = (layer == 1) ? 1 : 0;
    const auto& G = (layer == 1) ? t->G_full : t->G_half;
    if (first + 1 < L) {
      int last = first;
      while (last + 2 + 1 < L) last += 2;
      if (t->up) {
        for (int i = first; i <= last && r == TNT_OK; i += 2)
          r = tebd_gate(c, t, i, G[(size_t)i], TNT_SVD_LEFT, st);
      } else {
        for (int i = last; i >= first && r == TNT_OK; i -= 2)
          r = tebd_gate(c, t, i, G[(size_t)i], TNT_SVD_RIGHT, st);
      }
    }
    t->up = !t->up;
  }
  ws_reset(c);
  cudaEventRecord(e1, c->stream);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  st->seconds = ms * 1e-3;
  st->max_chi = *std::max_element(m->chi.begin(), m->chi.end());
  return r;
}

int tnt_tebd_gate(tnt_ctx* ctx, tnt_tebd* t, int bond, const tnt_cplx* h_gate, int dir,
                  tnt_trunc_result* tr) {
  if (!ctx || !t || !h_gate || !tr || t->ctx != ctx) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  tnt_mps* m = t->mps;
  if (bond < 0 || bond + 1 >= m->L || (dir != 1 && dir != -1))
    return set_err(c, TNT_E_INVALID, "bond %d / direction %d (bonds 0..%d, direction +1 or -1)",
                   bond, dir, m->L - 2);
  const size_t n2 = (size_t)m->d * m->d * m->d * m->d;
  const z* p = (const z*)h_gate;
  for (size_t e = 0; e < n2; ++e)
    if (!std::isfinite(p[e].x) || !std::isfinite(p[e].y))
      return set_err(c, TNT_E_NAN, "gate has a non-finite entry");
  std::vector<z> G(p, p + n2);
  tnt_step_stats st{};
  *tr = tnt_trunc_result{};
  ws_reset(c);
  int r = ws_reserve(c, t->scratch);
  if (r == TNT_OK) r = tebd_gate(c, t, bond, G, dir > 0 ? TNT_SVD_LEFT : TNT_SVD_RIGHT, &st, tr);
  ws_reset(c);
  if (r == TNT_OK) TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return r;
}

int tnt_tebd_centre(const tnt_tebd* t, int* centre) {
  if (!t || !centre) return TNT_E_INVALID;
  *centre = t->centre;
  return TNT_OK;
}

int tnt_tebd_destroy(tnt_tebd* t) {
  if (!t) return TNT_E_INVALID;
  delete t;
  return TNT_OK;
}

}  // extern "C"
