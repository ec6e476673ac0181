// Two-site contractions on the GPU: H_eff.theta (Listing 1 in two-site form), environment
// growth (Sec. 4.3), theta formation and the TEBD gate (Sec. 3).  Every index reorder the
// library performs before its matrix products (App. B.1.1) is folded into GEMM strides or
// the operator offset tables here; nothing is permuted in memory.
#include <algorithm>

#include "heff_plan.cuh"

namespace tnt {

int read_small(Ctx* c, const void* dsrc, void* hdst, size_t bytes) {
  TNT_CUDA_TRY(c, cudaMemcpyAsync(hdst, dsrc, bytes, cudaMemcpyDeviceToHost, c->stream));
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return TNT_OK;
}

size_t heff_scratch_bound(int64_t chl, int64_t d, int64_t D, int64_t chr, int precision) {
  const size_t t = (size_t)chl * D * d * d * chr;  // T1 and T3 elements
  size_t b = 2 * ws_round(sizeof(z) * t) + (size_t)(1 << 20);
  if (precision == TNT_PREC_MIXED) b += heff_mixed_scratch_bound(chl, d, D, chr);
  return b;
}

// W12[(s1',s2',w2),(w,s1,s2)] = sum_w1 W1[w,w1,s1',s1] W2[w1,w2,s2',s2]  (host, tiny)
static void build_w12(const std::vector<z>& W1, const std::vector<z>& W2, int64_t d, int64_t D,
                      std::vector<z>* W12) {
  const int64_t nI = d * d * D, nJ = D * d * d;
  W12->assign((size_t)(nI * nJ), zmk(0, 0));
  auto at1 = [&](int64_t w, int64_t v, int64_t so, int64_t si) {
    return W1[(size_t)(((w * D + v) * d + so) * d + si)];
  };
  auto at2 = [&](int64_t w, int64_t v, int64_t so, int64_t si) {
    return W2[(size_t)(((w * D + v) * d + so) * d + si)];
  };
  for (int64_t s1o = 0; s1o < d; ++s1o)
    for (int64_t s2o = 0; s2o < d; ++s2o)
      for (int64_t w2 = 0; w2 < D; ++w2) {
        const int64_t i = (s1o * d + s2o) * D + w2;
        for (int64_t w = 0; w < D; ++w)
          for (int64_t s1 = 0; s1 < d; ++s1)
            for (int64_t s2 = 0; s2 < d; ++s2) {
              const int64_t j = (w * d + s1) * d + s2;
              z acc = zmk(0, 0);
              for (int64_t w1 = 0; w1 < D; ++w1) zfma(acc, at1(w, w1, s1o, s1), at2(w1, w2, s2o, s2));
              (*W12)[(size_t)(i * nJ + j)] = acc;
            }
      }
}

int heff_prepare(Ctx* c, const z* L, const z* W1, const z* W2, const z* R, int64_t chl,
                 int64_t d, int64_t D, int64_t chr, int precision, HeffPlan* p, const z* hW1,
                 const z* hW2) {
  p->L = L;
  p->R = R;
  p->chl = chl;
  p->d = d;
  p->D = D;
  p->chr = chr;
  p->precision = precision;
  const size_t nW = (size_t)(D * D * d * d);
  std::vector<z> h1(nW), h2(nW), w12;
  if (hW1) std::copy(hW1, hW1 + nW, h1.begin());
  else TNT_TRY(read_small(c, W1, h1.data(), nW * sizeof(z)));
  if (hW2) std::copy(hW2, hW2 + nW, h2.begin());
  else TNT_TRY(read_small(c, W2, h2.data(), nW * sizeof(z)));
  build_w12(h1, h2, d, D, &w12);
  const int nI = (int)(d * d * D), nJ = (int)(D * d * d);
  std::vector<int64_t> in_off(nJ), out_off(nI);
  for (int j = 0; j < nJ; ++j) in_off[j] = (int64_t)j * chr;   // T1[a'][(w s1 s2)][b]
  for (int i = 0; i < nI; ++i) out_off[i] = (int64_t)i * chr;  // T3[a'][(s1' s2' w2)][b]
  TNT_TRY(op_upload(c, w12, nI, nJ, in_off, out_off, &p->op));
  const size_t t = (size_t)chl * D * d * d * chr;
  p->T1 = (z*)ws_alloc(c, ws_round(sizeof(z) * t));
  p->T3 = (z*)ws_alloc(c, ws_round(sizeof(z) * t));
  if (!p->T1 || !p->T3) return set_err(c, TNT_E_ALLOC, "scratch exhausted (H_eff intermediates)");
  p->op.in = p->T1;
  p->op.out = p->T3;
  p->op.B0 = chl;
  p->op.B1 = 1;
  p->op.B2 = chr;
  p->op.is0 = D * d * d * chr;
  p->op.os0 = d * d * D * chr;
  p->op.is1 = p->op.os1 = 0;
  p->op.is2 = p->op.os2 = 1;
  p->op.accumulate = 0;
  if (precision == TNT_PREC_MIXED) TNT_TRY(heff_mixed_prepare(c, p));
  return TNT_OK;
}

// FP64: T1 = L.theta (GEMM), T3 = W12 . T1 (sparse op), y = T3 . R^T (GEMM)
int heff_run_f64(Ctx* c, const HeffPlan& p, const z* theta, z* y) {
  const int64_t chl = p.chl, d = p.d, D = p.D, chr = p.chr;
  ZGemm g1{};
  g1.M = chl * D;
  g1.N = d * d * chr;
  g1.K = chl;
  g1.A = p.L;  // L[(a' w)][a]
  g1.a_rs = chl;
  g1.a_cs = 1;
  g1.B = theta;  // theta[a][(s1 s2 b)]
  g1.b_rs = d * d * chr;
  g1.b_cs = 1;
  g1.C = p.T1;
  g1.c_rs = d * d * chr;
  g1.alpha = zmk(1, 0);
  g1.beta = zmk(0, 0);
  g1.batch = 1;
  TNT_TRY(zgemm(c, g1));
  TNT_TRY(op_apply(c, p.op));
  ZGemm g4{};
  g4.M = chl * d * d;
  g4.N = chr;
  g4.K = D * chr;
  g4.A = p.T3;  // T3[(a' s1' s2')][(w2 b)]
  g4.a_rs = D * chr;
  g4.a_cs = 1;
  g4.B = p.R;  // B(k=(w2 b), j=b') = R[b'][(w2 b)]
  g4.b_rs = 1;
  g4.b_cs = D * chr;
  g4.C = y;
  g4.c_rs = chr;
  g4.alpha = zmk(1, 0);
  g4.beta = zmk(0, 0);
  g4.batch = 1;
  return zgemm(c, g4);
}

int heff_run(Ctx* c, const HeffPlan& p, const z* theta, z* y, int precision) {
  if (precision == TNT_PREC_MIXED) return heff_run_mixed(c, p, theta, y);
  return heff_run_f64(c, p, theta, y);
}

// ---------------------------------------------------------------- environments
size_t env_scratch_bound(int64_t chl, int64_t d, int64_t D, int64_t chr) {
  const size_t x = (size_t)std::max(chl, chr) * D * d * std::max(chl, chr);
  return 2 * ws_round(sizeof(z) * x) + (size_t)(1 << 20);
}

int env_left_impl(Ctx* c, const z* Lenv, const z* W, const z* A, int64_t chl, int64_t d,
                  int64_t D, int64_t chr, z* Lout, const z* hWin) {
  // X[a'][w][s][m] = sum_a L[(a' w)][a] A[a][(s m)]
  const size_t nx = (size_t)chl * D * d * chr;
  z* X = (z*)ws_alloc(c, ws_round(sizeof(z) * nx));
  z* Y = (z*)ws_alloc(c, ws_round(sizeof(z) * nx));
  if (!X || !Y) return set_err(c, TNT_E_ALLOC, "scratch exhausted (env_left)");
  ZGemm g{};
  g.M = chl * D; g.N = d * chr; g.K = chl;
  g.A = Lenv; g.a_rs = chl; g.a_cs = 1;
  g.B = A; g.b_rs = d * chr; g.b_cs = 1;
  g.C = X; g.c_rs = d * chr;
  g.alpha = zmk(1, 0); g.beta = zmk(0, 0); g.batch = 1;
  TNT_TRY(zgemm(c, g));
  // Y[a'][(s' w')][m] = sum_{w,s} W[w,w',s',s] X[a'][(w s)][m]
  const size_t nW = (size_t)(D * D * d * d);
  std::vector<z> hW(nW);
  if (hWin) std::copy(hWin, hWin + nW, hW.begin());
  else TNT_TRY(read_small(c, W, hW.data(), nW * sizeof(z)));
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
  OpApply a{};
  TNT_TRY(op_upload(c, op, nI, nJ, in_off, out_off, &a));
  a.in = X; a.out = Y;
  a.B0 = chl; a.B1 = 1; a.B2 = chr;
  a.is0 = D * d * chr; a.os0 = d * D * chr;
  a.is2 = a.os2 = 1;
  TNT_TRY(op_apply(c, a));
  // Lout[m'][(w' m)] = sum_{(a' s')} conj(A[(a' s')][m']) Y[(a' s')][(w' m)]
  ZGemm h{};
  h.M = chr; h.N = D * chr; h.K = chl * d;
  h.A = A; h.a_rs = 1; h.a_cs = chr; h.conj_a = 1;
  h.B = Y; h.b_rs = D * chr; h.b_cs = 1;
  h.C = Lout; h.c_rs = D * chr;
  h.alpha = zmk(1, 0); h.beta = zmk(0, 0); h.batch = 1;
  return zgemm(c, h);
}

int env_right_impl(Ctx* c, const z* Renv, const z* W, const z* B, int64_t chl, int64_t d,
                   int64_t D, int64_t chr, z* Rout, const z* hWin) {
  // X[a][s][b'][w'] = sum_b B[(a s)][b] R[(b' w')][b]
  const size_t nx = (size_t)chl * d * chr * D;
  z* X = (z*)ws_alloc(c, ws_round(sizeof(z) * nx));
  z* Y = (z*)ws_alloc(c, ws_round(sizeof(z) * nx));
  if (!X || !Y) return set_err(c, TNT_E_ALLOC, "scratch exhausted (env_right)");
  ZGemm g{};
  g.M = chl * d; g.N = chr * D; g.K = chr;
  g.A = B; g.a_rs = chr; g.a_cs = 1;
  g.B = Renv; g.b_rs = 1; g.b_cs = chr;
  g.C = X; g.c_rs = chr * D;
  g.alpha = zmk(1, 0); g.beta = zmk(0, 0); g.batch = 1;
  TNT_TRY(zgemm(c, g));
  // Y[w][a][s'][b'] = sum_{s,w'} W[w,w',s',s] X[a][s][b'][w']
  const size_t nW = (size_t)(D * D * d * d);
  std::vector<z> hW(nW);
  if (hWin) std::copy(hWin, hWin + nW, hW.begin());
  else TNT_TRY(read_small(c, W, hW.data(), nW * sizeof(z)));
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
  a.in = X; a.out = Y;
  a.B0 = chl; a.B1 = 1; a.B2 = chr;
  a.is0 = d * chr * D; a.is2 = D;
  a.os0 = d * chr; a.os2 = 1;
  TNT_TRY(op_apply(c, a));
  // Rout[a'][(w a)] = sum_{(s' b')} conj(B[a'][(s' b')]) Y[(w a)][(s' b')]
  ZGemm h{};
  h.M = chl; h.N = D * chl; h.K = d * chr;
  h.A = B; h.a_rs = d * chr; h.a_cs = 1; h.conj_a = 1;
  h.B = Y; h.b_rs = 1; h.b_cs = d * chr;
  h.C = Rout; h.c_rs = D * chl;
  h.alpha = zmk(1, 0); h.beta = zmk(0, 0); h.batch = 1;
  return zgemm(c, h);
}

// ---------------------------------------------------------------- theta and gate
int theta_form_impl(Ctx* c, const z* A, const z* B, int64_t chl, int64_t d, int64_t chm,
                    int64_t chr, z* theta) {
  ZGemm g{};
  g.M = chl * d; g.N = d * chr; g.K = chm;
  g.A = A; g.a_rs = chm; g.a_cs = 1;
  g.B = B; g.b_rs = d * chr; g.b_cs = 1;
  g.C = theta; g.c_rs = d * chr;
  g.alpha = zmk(1, 0); g.beta = zmk(0, 0); g.batch = 1;
  return zgemm(c, g);
}

int gate_apply_impl(Ctx* c, const std::vector<z>& G, const z* theta, int64_t chl, int64_t d,
                    int64_t chr, z* out) {
  const int nI = (int)(d * d), nJ = (int)(d * d);
  std::vector<int64_t> off(nJ);
  for (int j = 0; j < nJ; ++j) off[j] = (int64_t)j * chr;
  OpApply a{};
  TNT_TRY(op_upload(c, G, nI, nJ, off, off, &a));
  a.in = theta; a.out = out;
  a.B0 = chl; a.B1 = 1; a.B2 = chr;
  a.is0 = a.os0 = d * d * chr;
  a.is2 = a.os2 = 1;
  return op_apply(c, a);
}

}  // namespace tnt
