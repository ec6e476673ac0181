// Device-resident MPO and MPS handles shared by the DMRG sweep and the TEBD step.
#pragma once

#include <vector>

#include "tnt_internal.cuh"

struct tnt_mpo {
  int L = 0, d = 0, D = 4;
  tnt::DevAlloc dalloc;     // allocator of the context that made it
  std::vector<tnt::z*> W;  // per site, D x D x d x d (device)
  tnt::z* left = nullptr;   // boundary environment L_0[0,w,0] (device, D)
  tnt::z* right = nullptr;  // boundary R_{L}[0,w,0]
  std::vector<int> wq;      // U(1) charge of each MPO bond index (empty: none)
  std::vector<std::vector<tnt::z>> hW;  // host copies of W (no read-back per update)
  std::vector<tnt::z> hleft, hright;    // host copies of the boundary vectors
};

struct tnt_mps {
  int L = 0, d = 0;
  tnt::DevAlloc dalloc;               // allocator of the context that made it
  std::vector<int64_t> chi, cap;      // bonds 0..L
  std::vector<tnt::z*> A;             // sites 0..L-1, capacity cap[j] x d x cap[j+1]
  std::vector<std::vector<int64_t>> q;  // bond labels (empty vectors: no labels)
  bool labelled = false;
};

struct tnt_dmrg {
  tnt_ctx* ctx = nullptr;
  tnt::DevAlloc dalloc;
  tnt_mps* mps = nullptr;
  const tnt_mpo* mpo = nullptr;
  std::vector<tnt::z*> Lenv, Renv;  // Lenv[i]: sites 0..i-1 (i = 0..L); Renv[i]: sites i..L-1
  size_t scratch = 0;
  cudaEvent_t ev[5] = {};  // phase marks of one update (sweep statistics)
  std::vector<double> last_E;  // energy of each update of the last sweep, in update order
  // gauge bookkeeping for single updates: the site holding the orthogonality centre, and
  // the environments consistent with the current sites (Lenv[0..lvalid], Renv[rvalid..L])
  int centre = 0, lvalid = 0, rvalid = 1;
};

namespace tnt {
// exact SVD parameters for gauge moves (no truncation beyond exact zeros)
tnt_params exact_params(const tnt_params& p);
std::vector<int64_t> labels_or_zero(const tnt_mps* m, int bond);
int64_t ipow_cap(int64_t d, int64_t k, int64_t cap);

// swaps in parameters for the lifetime of the guard (exact gauge moves)
struct ParamsGuard {
  Ctx* c;
  tnt_params saved;
  ParamsGuard(Ctx* cc, const tnt_params& p) : c(cc), saved(cc->params) { c->params = p; }
  ~ParamsGuard() { c->params = saved; }
};
}  // namespace tnt
