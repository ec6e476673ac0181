// Host replay of the grouped U(1) H_eff.theta plan (test infrastructure, no GPU).
//
// Builds the library's own plan with tnt::u1_layout for one or several problems whose
// environments, MPO tensors and compact theta are host arrays, then carries out, in FP64
// on the host, exactly the data movement and arithmetic the device kernels take from the
// plan's tables: the packed L blocks (PackSeg), the transposed theta slabs (TSlab), the
// stage-1 tasks, the W1 W2 contraction over block pairs (WPair / WOut / WIn), the packed R
// blocks, the stage-4 tasks and the gather of output rows (GRow).  The result is compared
// by the calling test with the oracle's dense contraction, so a wrong table (a block sent
// to the wrong place, a sector pairing missed) shows here without a GPU.
//
// Input (binary, little endian): int64 nprob, then per problem int64 chl, chr, d, D, the
// labels qa[chl], qb[chr], wq[D] (int64), then complex128 L[chl][D][chl], W1[D][D][d][d],
// W2[D][D][d][d], R[chr][D][chr]; then int64 n and complex128 x[n] (all problems' compact
// theta back to back).  Output: int64 n, complex128 y[n], then int64 coverage errors (the
// compact entries not written exactly once by the gather).
#include <cstdint>
#include <cstdio>
#include <vector>

#include "u1.cuh"

namespace {
template <typename T>
bool rd(FILE* f, T* p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

struct Prob {
  int64_t chl, chr, d, D;
  std::vector<int64_t> qa, qb, wq;
  std::vector<tnt::z> L, W1, W2, R;
};

inline void fma_z(tnt::z& acc, const tnt::z& a, const tnt::z& b) {
  acc.x += a.x * b.x - a.y * b.y;
  acc.y += a.x * b.y + a.y * b.x;
}
}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: %s input output\n", argv[0]);
    return 2;
  }
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int64_t nprob = 0;
  if (!rd(f, &nprob, 1) || nprob < 1) return 2;
  std::vector<Prob> P((size_t)nprob);
  for (Prob& p : P) {
    int64_t h[4];
    if (!rd(f, h, 4)) return 2;
    p.chl = h[0]; p.chr = h[1]; p.d = h[2]; p.D = h[3];
    p.qa.resize((size_t)p.chl); p.qb.resize((size_t)p.chr); p.wq.resize((size_t)p.D);
    p.L.resize((size_t)(p.chl * p.D * p.chl));
    p.W1.resize((size_t)(p.D * p.D * p.d * p.d));
    p.W2.resize(p.W1.size());
    p.R.resize((size_t)(p.chr * p.D * p.chr));
    if (!rd(f, p.qa.data(), p.qa.size()) || !rd(f, p.qb.data(), p.qb.size()) ||
        !rd(f, p.wq.data(), p.wq.size()) || !rd(f, p.L.data(), p.L.size()) ||
        !rd(f, p.W1.data(), p.W1.size()) || !rd(f, p.W2.data(), p.W2.size()) ||
        !rd(f, p.R.data(), p.R.size()))
      return 2;
  }
  int64_t n = 0;
  if (!rd(f, &n, 1)) return 2;
  std::vector<tnt::z> x((size_t)n);
  if (!rd(f, x.data(), x.size())) return 2;
  fclose(f);

  std::vector<tnt::U1Spec> specs((size_t)nprob);
  for (size_t i = 0; i < P.size(); ++i) {
    tnt::U1Spec& s = specs[i];
    const Prob& p = P[i];
    s.L = p.L.data(); s.R = p.R.data(); s.W1 = p.W1.data(); s.W2 = p.W2.data();
    s.hW1 = p.W1.data(); s.hW2 = p.W2.data();
    s.chl = p.chl; s.chr = p.chr; s.d = p.d; s.D = p.D;
    s.qa = p.qa; s.qb = p.qb;
    s.wq.assign(p.wq.begin(), p.wq.end());
  }
  tnt::Ctx c;
  tnt::U1Plan plan;
  if (tnt::u1_layout(&c, specs, &plan) != 0) {
    fprintf(stderr, "u1_layout: %s\n", c.err.c_str());
    return 3;
  }
  if (plan.n != n) {
    fprintf(stderr, "compact length %lld, input has %lld\n", (long long)plan.n, (long long)n);
    return 4;
  }
  using tnt::z;
  const z zero = tnt::zmk(0, 0);
  // stage-1 operands: packed L blocks and transposed theta slabs
  std::vector<z> A1((size_t)(plan.rowsA1 * plan.KA1), zero), B1((size_t)(plan.rowsB1 * plan.KA1), zero);
  for (const tnt::PackSeg& s : plan.segA1)
    for (int64_t i = 0; i < s.len; ++i) A1[(size_t)(s.dst + i)] = s.src[i];
  for (const tnt::TSlab& sb : plan.slabs)
    for (int64_t k = 0; k < sb.K; ++k)
      for (int64_t j = 0; j < sb.N; ++j)
        B1[(size_t)((sb.dst_row0 + j) * plan.KA1 + k)] = x[(size_t)(sb.src + k * sb.N + j)];
  std::vector<z> T1((size_t)plan.P1, zero);
  for (const tnt::TaskDesc& t : plan.s1)
    for (int64_t i = 0; i < t.M; ++i)
      for (int64_t j = 0; j < t.N; ++j) {
        z acc = zero;
        for (int64_t k = 0; k < t.K; ++k)
          fma_z(acc, A1[(size_t)((t.a_row0 + i) * plan.KA1 + k)], B1[(size_t)((t.b_row0 + j) * plan.KA1 + k)]);
        T1[(size_t)(t.c_off + i * t.ldc + j)] = acc;
      }
  // W1 W2 contraction into the stage-4 A operand
  std::vector<z> A4((size_t)(plan.rowsA4 * plan.KA4), zero);
  for (const tnt::WPair& pr : plan.pairs)
    for (int o = pr.out0; o < pr.out0 + pr.nout; ++o) {
      const tnt::WOut& w = plan.outs[(size_t)o];
      for (int64_t ia = 0; ia < pr.n_a; ++ia)
        for (int64_t jb = 0; jb < pr.n_b; ++jb) {
          z acc = zero;
          for (int r = w.r0; r < w.r1; ++r) {
            const tnt::WIn& in = plan.ins[(size_t)r];
            fma_z(acc, in.val, T1[(size_t)(in.base + ia * in.rs + jb)]);
          }
          A4[(size_t)(w.base + ia * plan.KA4 + jb)] = acc;
        }
    }
  // stage-4 B operand: packed R blocks; stage-4 tasks; gather
  std::vector<z> B4((size_t)(plan.rowsB4 * plan.KA4), zero);
  for (const tnt::PackSeg& s : plan.segB4)
    for (int64_t i = 0; i < s.len; ++i) B4[(size_t)(s.dst + i)] = s.src[i];
  std::vector<z> Y((size_t)plan.P4, zero);
  for (const tnt::TaskDesc& t : plan.s4)
    for (int64_t i = 0; i < t.M; ++i)
      for (int64_t j = 0; j < t.N; ++j) {
        z acc = zero;
        for (int64_t k = 0; k < t.K; ++k)
          fma_z(acc, A4[(size_t)((t.a_row0 + i) * plan.KA4 + k)], B4[(size_t)((t.b_row0 + j) * plan.KA4 + k)]);
        Y[(size_t)(t.c_off + i * t.ldc + j)] = acc;
      }
  std::vector<z> y((size_t)n, zero);
  std::vector<int> hits((size_t)n, 0);
  for (const tnt::GRow& g : plan.rows)
    for (int64_t j = 0; j < g.n; ++j) {
      y[(size_t)(g.dst + j)] = Y[(size_t)(g.src + j)];
      hits[(size_t)(g.dst + j)]++;
    }
  int64_t bad = 0;
  for (int h : hits) bad += (h != 1);
  FILE* o = fopen(argv[2], "wb");
  if (!o) return 2;
  fwrite(&n, sizeof(n), 1, o);
  fwrite(y.data(), sizeof(z), y.size(), o);
  fwrite(&bad, sizeof(bad), 1, o);
  fclose(o);
  return 0;
}
