// MPS overlap, file input/output and U(1) labels of an existing MPS handle.
//
//   <a|b>: the <psi|O|psi> network of Sec. 4.3 with O = 1 and two different states,
//     contracted from the left: E_0 = 1, E_{j+1}[al', be'] = sum conj(A_j[al, s, al'])
//     E_j[al, be] B_j[be, s, be'] as two FP64 GEMMs per site.
//   save / load (App. B.5: the library writes networks with their block labels and the
//     system settings, and a file written by one run is input to the next): one binary
//     file holding the bond dimensions, the U(1) bond labels, every site tensor and the
//     context's parameters; loading restores the MPS and, on request, the parameters.
//   labels (App. A.1.1, tntNodeSetQN): a bond's U(1) labels are replaced after checking,
//     on the device, that both neighbouring site tensors vanish outside the blocks the new
//     labels allow (q_left + s = q_right for every non-zero A[a, s, b]).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "heff_plan.cuh"
#include "mps.cuh"

namespace tnt {
namespace {

// one FP64 transfer step of the overlap: E' = A^H (E B)
int overlap_step(Ctx* c, const z* E, const z* A, const z* B, int64_t ca, int64_t cb,
                 int64_t ca2, int64_t cb2, int64_t d, z* T, z* Eout) {
  ZGemm g{};  // T[al][(s be')] = sum_be E[al][be] B[be][(s be')]
  g.M = ca; g.N = d * cb2; g.K = cb;
  g.A = E; g.a_rs = cb; g.a_cs = 1;
  g.B = B; g.b_rs = d * cb2; g.b_cs = 1;
  g.C = T; g.c_rs = d * cb2;
  g.alpha = zmk(1, 0); g.beta = zmk(0, 0); g.batch = 1;
  TNT_TRY(zgemm(c, g));
  ZGemm h{};  // E'[al'][be'] = sum_{(al s)} conj(A[(al s)][al']) T[(al s)][be']
  h.M = ca2; h.N = cb2; h.K = ca * d;
  h.A = A; h.a_rs = 1; h.a_cs = ca2; h.conj_a = 1;
  h.B = T; h.b_rs = cb2; h.b_cs = 1;
  h.C = Eout; h.c_rs = cb2;
  h.alpha = zmk(1, 0); h.beta = zmk(0, 0); h.batch = 1;
  return zgemm(c, h);
}

// count of entries A[a, s, b] with |A| > 0 outside q_left[a] + s == q_right[b]
__global__ void k_label_violations(const z* __restrict__ A, int64_t chl, int64_t d, int64_t chr,
                                   const int64_t* __restrict__ ql, const int64_t* __restrict__ qr,
                                   unsigned long long* __restrict__ bad) {
  const int64_t n = chl * d * chr;
  unsigned long long cnt = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e % chr, s = (e / chr) % d, a = e / (chr * d);
    const z v = A[e];
    if ((v.x != 0.0 || v.y != 0.0) && ql[a] + s != qr[b]) ++cnt;
  }
  if (cnt) atomicAdd(bad, cnt);
}

constexpr char MPS_MAGIC[8] = {'T', 'N', 'T', 'M', 'P', 'S', '0', '1'};

struct FileCloser {
  FILE* f;
  ~FileCloser() {
    if (f) fclose(f);
  }
};
}  // namespace
}  // namespace tnt

using namespace tnt;

extern "C" {

int tnt_mps_overlap(tnt_ctx* ctx, const tnt_mps* a, const tnt_mps* b, tnt_cplx* out) {
  if (!ctx || !a || !b || !out) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  if (a->L != b->L || a->d != b->d)
    return set_err(c, TNT_E_INVALID, "overlap of MPS with L, d = %d, %d and %d, %d", a->L, a->d,
                   b->L, b->d);
  const int64_t d = a->d;
  const int64_t ma = *std::max_element(a->chi.begin(), a->chi.end());
  const int64_t mb = *std::max_element(b->chi.begin(), b->chi.end());
  ws_reset(c);
  TNT_TRY(ws_reserve(c, 2 * ws_round(sizeof(z) * (size_t)(ma * mb)) +
                            ws_round(sizeof(z) * (size_t)(ma * d * mb)) + 4096));
  z* Ea = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(ma * mb)));
  z* Eb = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(ma * mb)));
  z* T = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(ma * d * mb)));
  const z one = zmk(1, 0);
  TNT_CUDA_TRY(c, cudaMemcpyAsync(Ea, &one, sizeof(z), cudaMemcpyHostToDevice, c->stream));
  for (int j = 0; j < a->L; ++j) {
    const int r = overlap_step(c, Ea, a->A[j], b->A[j], a->chi[j], b->chi[j], a->chi[j + 1],
                               b->chi[j + 1], d, T, Eb);
    if (r != TNT_OK) {
      ws_reset(c);
      return r;
    }
    std::swap(Ea, Eb);
  }
  z h;
  const int r = read_small(c, Ea, &h, sizeof(z));
  ws_reset(c);
  if (r != TNT_OK) return r;
  out->re = h.x;
  out->im = h.y;
  return TNT_OK;
}

int tnt_mps_set_charges(tnt_ctx* ctx, tnt_mps* m, int bond, const int64_t* h_q) {
  if (!ctx || !m || !h_q) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  if (bond < 0 || bond > m->L) return set_err(c, TNT_E_INVALID, "bond %d outside 0..%d", bond, m->L);
  const int64_t chi = m->chi[bond];
  if (!m->labelled) return set_err(c, TNT_E_INVALID, "the MPS carries no U(1) labels (create it with charges)");
  if ((bond == 0 || bond == m->L) && h_q[0] != m->q[bond][0])
    return set_err(c, TNT_E_INVALID, "the boundary label of bond %d is fixed at %lld", bond,
                   (long long)m->q[bond][0]);
  std::vector<int64_t> nq(h_q, h_q + chi);
  // both neighbouring sites must vanish outside the blocks the new labels allow
  ws_reset(c);
  int64_t mx = *std::max_element(m->chi.begin(), m->chi.end());
  TNT_TRY(ws_reserve(c, 3 * ws_round(sizeof(int64_t) * (size_t)mx) + 4096));
  int64_t* dq = (int64_t*)ws_alloc(c, ws_round(sizeof(int64_t) * (size_t)mx));
  int64_t* dl = (int64_t*)ws_alloc(c, ws_round(sizeof(int64_t) * (size_t)mx));
  unsigned long long* bad = (unsigned long long*)ws_alloc(c, 256);
  TNT_CUDA_TRY(c, cudaMemsetAsync(bad, 0, sizeof(unsigned long long), c->stream));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(dq, nq.data(), sizeof(int64_t) * chi, cudaMemcpyHostToDevice, c->stream));
  for (int side = 0; side < 2; ++side) {
    const int j = side == 0 ? bond - 1 : bond;  // site left of the bond, then right of it
    if (j < 0 || j >= m->L) continue;
    const int other = side == 0 ? j : j + 1;   // the site's other bond
    TNT_CUDA_TRY(c, cudaMemcpyAsync(dl, m->q[other].data(), sizeof(int64_t) * m->chi[other],
                                    cudaMemcpyHostToDevice, c->stream));
    const int64_t n = m->chi[j] * m->d * m->chi[j + 1];
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 1216);
    k_label_violations<<<blocks, 256, 0, c->stream>>>(m->A[j], m->chi[j], m->d, m->chi[j + 1],
                                                      side == 0 ? dl : dq, side == 0 ? dq : dl, bad);
    c->launches++;
    TNT_CHECK_LAUNCH(c);
    TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // dl is reused by the next side
  }
  unsigned long long h_bad = 0;
  const int r = read_small(c, bad, &h_bad, sizeof(h_bad));
  ws_reset(c);
  if (r != TNT_OK) return r;
  if (h_bad)
    return set_err(c, TNT_E_INVALID,
                   "%llu non-zero entries of the sites next to bond %d break the new labels", h_bad, bond);
  m->q[bond] = nq;
  return TNT_OK;
}

int tnt_mps_save(tnt_ctx* ctx, const tnt_mps* m, const char* path) {
  if (!ctx || !m || !path) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  FILE* f = fopen(path, "wb");
  if (!f) return set_err(c, TNT_E_INVALID, "cannot open %s for writing", path);
  FileCloser fc{f};
  const int32_t hdr[3] = {m->L, m->d, m->labelled ? 1 : 0};
  bool ok = fwrite(MPS_MAGIC, 1, 8, f) == 8 && fwrite(hdr, sizeof(int32_t), 3, f) == 3 &&
            fwrite(&c->params, sizeof(tnt_params), 1, f) == 1 &&
            fwrite(m->chi.data(), sizeof(int64_t), m->L + 1, f) == (size_t)(m->L + 1);
  if (ok && m->labelled)
    for (int k = 0; k <= m->L && ok; ++k)
      ok = fwrite(m->q[k].data(), sizeof(int64_t), m->chi[k], f) == (size_t)m->chi[k];
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  std::vector<z> h;
  for (int j = 0; j < m->L && ok; ++j) {
    const size_t n = (size_t)(m->chi[j] * m->d * m->chi[j + 1]);
    h.resize(n);
    TNT_CUDA_TRY(c, cudaMemcpy(h.data(), m->A[j], n * sizeof(z), cudaMemcpyDeviceToHost));
    ok = fwrite(h.data(), sizeof(z), n, f) == n;
  }
  if (!ok) return set_err(c, TNT_E_INVALID, "short write to %s", path);
  return TNT_OK;
}

int tnt_mps_load(tnt_ctx* ctx, const char* path, int64_t chi_cap, int restore_params,
                 tnt_mps** out) {
  if (!ctx || !path || !out || chi_cap < 1) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return set_err(c, TNT_E_INVALID, "cannot open %s", path);
  FileCloser fc{f};
  char magic[8];
  int32_t hdr[3];
  tnt_params p{};
  if (fread(magic, 1, 8, f) != 8 || memcmp(magic, MPS_MAGIC, 8) != 0 ||
      fread(hdr, sizeof(int32_t), 3, f) != 3 || fread(&p, sizeof(tnt_params), 1, f) != 1)
    return set_err(c, TNT_E_INVALID, "%s is not an MPS file of this library", path);
  const int L = hdr[0], d = hdr[1];
  const bool labelled = hdr[2] != 0;
  if (L < 2 || L > (1 << 20) || d < 1 || d > (1 << 16))
    return set_err(c, TNT_E_INVALID, "%s: L = %d, d = %d out of range", path, L, d);
  std::vector<int64_t> chi((size_t)L + 1);
  if (fread(chi.data(), sizeof(int64_t), L + 1, f) != (size_t)(L + 1))
    return set_err(c, TNT_E_INVALID, "%s: truncated header", path);
  for (int k = 0; k <= L; ++k)
    if (chi[(size_t)k] < 1 || chi[(size_t)k] > chi_cap)
      return set_err(c, TNT_E_INVALID, "%s: bond %d has dimension %lld (cap %lld)", path, k,
                     (long long)chi[(size_t)k], (long long)chi_cap);
  std::vector<std::vector<int64_t>> q;
  std::vector<const int64_t*> qp;
  if (labelled) {
    q.resize((size_t)L + 1);
    for (int k = 0; k <= L; ++k) {
      q[(size_t)k].resize((size_t)chi[(size_t)k]);
      if (fread(q[(size_t)k].data(), sizeof(int64_t), chi[(size_t)k], f) != (size_t)chi[(size_t)k])
        return set_err(c, TNT_E_INVALID, "%s: truncated labels", path);
      qp.push_back(q[(size_t)k].data());
    }
  }
  std::vector<std::vector<tnt_cplx>> sites((size_t)L);
  std::vector<const tnt_cplx*> sp((size_t)L);
  for (int j = 0; j < L; ++j) {
    const size_t n = (size_t)(chi[(size_t)j] * d * chi[(size_t)j + 1]);
    sites[(size_t)j].resize(n);
    if (fread(sites[(size_t)j].data(), sizeof(tnt_cplx), n, f) != n)
      return set_err(c, TNT_E_INVALID, "%s: truncated site %d", path, j);
    sp[(size_t)j] = sites[(size_t)j].data();
  }
  TNT_TRY(tnt_mps_create(ctx, L, d, chi_cap, chi.data(), sp.data(), labelled ? qp.data() : nullptr, out));
  if (restore_params) {
    const int r = tnt_params_set(ctx, &p);
    if (r != TNT_OK) {
      tnt_mps_destroy(*out);
      *out = nullptr;
      return r;
    }
  }
  return TNT_OK;
}

}  // extern "C"
