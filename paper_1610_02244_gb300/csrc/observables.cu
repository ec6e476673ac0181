// One-site and two-site expectation values of the device MPS (Sec. 5: the density <n_j>
// and the single-particle density matrix <b+_i b_j> the paper's examples print), FP64.
//
// With the identity transfer environments E_j (sites 0..j-1, from the left) and F_j
// (sites j..L-1, from the right), all D = 1 environments grown by the FP64 environment
// kernels (a8):
//   <n_j>      = sum_{b',b} [E_j (x) n at site j](b',b) F_{j+1}(b',b) / <psi|psi>
//   <b+_i b_j> = the same with b+ at site i, identity on i+1..j-1, b at site j (i < j);
//                <b+_j b_i> = conj(<b+_i b_j>).
// <psi|psi> is the fully grown E_L.  No normalisation of the state is assumed.
#include <algorithm>
#include <cmath>
#include <vector>

#include "heff_plan.cuh"
#include "mps.cuh"

namespace tnt {

namespace {
// out[0] = sum_i x_i y_i (no conjugation), one block, fixed order
__global__ void k_hsum(const z* __restrict__ x, const z* __restrict__ y, int64_t n, z* __restrict__ out) {
  __shared__ double sr[256], si[256];
  double ar = 0, ai = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const z a = x[i], b = y[i];
    ar = fma(a.x, b.x, fma(-a.y, b.y, ar));
    ai = fma(a.x, b.y, fma(a.y, b.x, ai));
  }
  sr[threadIdx.x] = ar;
  si[threadIdx.x] = ai;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      si[threadIdx.x] += si[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = zmk(sr[0], si[0]);
}

struct Obs {
  z* Wid = nullptr;   // D = 1 operators [1][1][d][d]: identity, n, b+, b
  z* Wn = nullptr;
  z* Wbd = nullptr;
  z* Wb = nullptr;
  std::vector<z*> E, F;  // E[j]: chi_j x chi_j (sites 0..j-1); F[j]: sites j..L-1
  z* T0 = nullptr;    // running environments
  z* T1 = nullptr;
  z* out = nullptr;   // device results
};

size_t obs_bound(const tnt_mps* m, int64_t nout) {
  size_t b = 0;
  int64_t mx = 1;
  for (int k = 0; k <= m->L; ++k) {
    b += 2 * ws_round(sizeof(z) * (size_t)(m->chi[k] * m->chi[k]));
    mx = std::max(mx, m->chi[k]);
  }
  b += 2 * ws_round(sizeof(z) * (size_t)(mx * mx)) + 4 * ws_round(sizeof(z) * m->d * m->d) +
       ws_round(sizeof(z) * (size_t)nout) + env_scratch_bound(mx, m->d, 1, mx);
  return b + (size_t)(1 << 20);
}

int obs_setup(Ctx* c, const tnt_mps* m, Obs* o, int64_t nout) {
  const int64_t d = m->d;
  const int L = m->L;
  std::vector<z> id((size_t)(d * d), zmk(0, 0)), nn(id), bd(id), bb(id);
  for (int64_t s = 0; s < d; ++s) {
    id[(size_t)(s * d + s)] = zmk(1, 0);
    nn[(size_t)(s * d + s)] = zmk((double)s, 0);
    if (s + 1 < d) {
      bd[(size_t)((s + 1) * d + s)] = zmk(std::sqrt((double)(s + 1)), 0);  // <s+1|b+|s>
      bb[(size_t)(s * d + s + 1)] = zmk(std::sqrt((double)(s + 1)), 0);    // <s|b|s+1>
    }
  }
  z** ws[4] = {&o->Wid, &o->Wn, &o->Wbd, &o->Wb};
  const std::vector<z>* hs[4] = {&id, &nn, &bd, &bb};
  for (int i = 0; i < 4; ++i) {
    *ws[i] = (z*)ws_alloc(c, ws_round(sizeof(z) * d * d));
    if (!*ws[i]) return set_err(c, TNT_E_ALLOC, "scratch exhausted (observables)");
    TNT_CUDA_TRY(c, cudaMemcpyAsync(*ws[i], hs[i]->data(), sizeof(z) * d * d, cudaMemcpyHostToDevice, c->stream));
  }
  int64_t mx = 1;
  for (int k = 0; k <= L; ++k) mx = std::max(mx, m->chi[k]);
  o->E.assign((size_t)L + 1, nullptr);
  o->F.assign((size_t)L + 1, nullptr);
  for (int k = 0; k <= L; ++k) {
    o->E[(size_t)k] = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(m->chi[k] * m->chi[k])));
    o->F[(size_t)k] = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(m->chi[k] * m->chi[k])));
    if (!o->E[(size_t)k] || !o->F[(size_t)k]) return set_err(c, TNT_E_ALLOC, "scratch exhausted (observables)");
  }
  o->T0 = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(mx * mx)));
  o->T1 = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)(mx * mx)));
  o->out = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)std::max<int64_t>(nout, 1)));
  if (!o->T0 || !o->T1 || !o->out) return set_err(c, TNT_E_ALLOC, "scratch exhausted (observables)");
  const z one = zmk(1, 0);
  TNT_CUDA_TRY(c, cudaMemcpyAsync(o->E[0], &one, sizeof(z), cudaMemcpyHostToDevice, c->stream));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(o->F[(size_t)L], &one, sizeof(z), cudaMemcpyHostToDevice, c->stream));
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // the host constants above are stack values
  for (int j = 0; j < L; ++j) {
    const size_t top = c->ws.top;
    TNT_TRY(env_left_impl(c, o->E[(size_t)j], o->Wid, m->A[(size_t)j], m->chi[(size_t)j], d, 1,
                          m->chi[(size_t)j + 1], o->E[(size_t)j + 1]));
    c->ws.top = top;
  }
  for (int j = L - 1; j >= 0; --j) {
    const size_t top = c->ws.top;
    TNT_TRY(env_right_impl(c, o->F[(size_t)j + 1], o->Wid, m->A[(size_t)j], m->chi[(size_t)j], d, 1,
                           m->chi[(size_t)j + 1], o->F[(size_t)j]));
    c->ws.top = top;
  }
  return TNT_OK;
}

// env over site j with operator W from Ein into Eout
int grow(Ctx* c, const tnt_mps* m, int j, const z* Ein, const z* W, z* Eout) {
  const size_t top = c->ws.top;
  const int r = env_left_impl(c, Ein, W, m->A[(size_t)j], m->chi[(size_t)j], m->d, 1,
                              m->chi[(size_t)j + 1], Eout);
  c->ws.top = top;
  return r;
}

int close(Ctx* c, const tnt_mps* m, int j, const z* X, const Obs& o, z* dst) {
  const int64_t n = m->chi[(size_t)j + 1] * m->chi[(size_t)j + 1];
  k_hsum<<<1, 256, 0, c->stream>>>(X, o.F[(size_t)j + 1], n, dst);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}
}  // namespace

}  // namespace tnt

using namespace tnt;

extern "C" {

int tnt_mps_density(tnt_ctx* ctx, const tnt_mps* m, double* h_n) {
  if (!ctx || !m || !h_n) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  const int L = m->L;
  Scope sc(c);
  TNT_TRY(ws_reserve(c, obs_bound(m, L + 1)));
  Obs o;
  TNT_TRY(obs_setup(c, m, &o, L + 1));
  for (int j = 0; j < L; ++j) {
    TNT_TRY(grow(c, m, j, o.E[(size_t)j], o.Wn, o.T0));
    TNT_TRY(close(c, m, j, o.T0, o, o.out + j));
  }
  TNT_CUDA_TRY(c, cudaMemcpyAsync(o.out + L, o.E[(size_t)L], sizeof(z), cudaMemcpyDeviceToDevice, c->stream));
  std::vector<z> h((size_t)L + 1);
  TNT_TRY(read_small(c, o.out, h.data(), sizeof(z) * (L + 1)));
  const double norm = h[(size_t)L].x;
  if (!(norm > 0)) return set_err(c, TNT_E_NAN, "state norm is not positive");
  for (int j = 0; j < L; ++j) h_n[j] = h[(size_t)j].x / norm;
  return TNT_OK;
}

int tnt_mps_bdagb(tnt_ctx* ctx, const tnt_mps* m, tnt_cplx* h_rho) {
  if (!ctx || !m || !h_rho) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  const int L = m->L;
  Scope sc(c);
  TNT_TRY(ws_reserve(c, obs_bound(m, (int64_t)L * L + 1)));
  Obs o;
  TNT_TRY(obs_setup(c, m, &o, (int64_t)L * L + 1));
  for (int i = 0; i < L; ++i) {
    TNT_TRY(grow(c, m, i, o.E[(size_t)i], o.Wn, o.T0));
    TNT_TRY(close(c, m, i, o.T0, o, o.out + (int64_t)i * L + i));
    if (i + 1 == L) break;
    TNT_TRY(grow(c, m, i, o.E[(size_t)i], o.Wbd, o.T0));  // b+ at site i
    for (int j = i + 1; j < L; ++j) {
      TNT_TRY(grow(c, m, j, o.T0, o.Wb, o.T1));          // b at site j
      TNT_TRY(close(c, m, j, o.T1, o, o.out + (int64_t)i * L + j));
      if (j + 1 < L) {
        TNT_TRY(grow(c, m, j, o.T0, o.Wid, o.T1));        // identity on site j
        std::swap(o.T0, o.T1);
      }
    }
  }
  TNT_CUDA_TRY(c, cudaMemcpyAsync(o.out + (int64_t)L * L, o.E[(size_t)L], sizeof(z), cudaMemcpyDeviceToDevice, c->stream));
  std::vector<z> h((size_t)L * L + 1);
  TNT_TRY(read_small(c, o.out, h.data(), sizeof(z) * h.size()));
  const double norm = h[(size_t)L * L].x;
  if (!(norm > 0)) return set_err(c, TNT_E_NAN, "state norm is not positive");
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j) {
      z v;
      if (i <= j) v = h[(size_t)i * L + j];
      else v = zconj(h[(size_t)j * L + i]);
      h_rho[(size_t)i * L + j] = tnt_cplx{v.x / norm, v.y / norm};
    }
  return TNT_OK;
}

}  // extern "C"
