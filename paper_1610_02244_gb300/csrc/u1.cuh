// U(1) block-sparse H_eff.theta over one or several problems in grouped launches.
//
// With boson-number labels on every bond (App. A.1.1; labels count the bosons to the
// left), theta[a,s1,s2,b] is non-zero only for q_b = q_a + s1 + s2, L[a',w,a] only for
// q_a' = q_a + c_w and R[b',w,b] only for q_b' = q_b + c_w, c_w the charge of the MPO bond
// index (Bose-Hubbard: c = (0, +1, -1, 0)).  The matvec of Listing 1 (Sec. 4.2) then splits
// into dense blocks: stage 1 (L . theta) has one task per left sector q of a, with rows
// (w, a' in q + c_w), K = a in q and columns (s1, s2, b in q + s1 + s2); the W contraction
// maps those to stage 4 (T3 . R^T) tasks, one per right sector Q of b', with rows
// (q', s1', s2', a' in q') for q' + s1' + s2' = Q and K = (w2, b in Q - c_w2).  Every task
// of every problem goes into one grouped launch per stage (App. B.1.2: the per-block work
// the paper's library dispatches one call at a time).
//
// Compact theta: left sectors in ascending charge, and within sector q the slab
// [a in q][(s1, s2) row-major][b in right sector q + s1 + s2]; problems are concatenated.
#pragma once

#include <cuda.h>

#include <string>
#include <vector>

#include "heff_plan.cuh"

namespace tnt {

struct Sector {
  int64_t q, start, size;
};

// one problem as given by the caller (device pointers borrowed, host labels copied)
struct U1Spec {
  const z *L = nullptr, *R = nullptr, *W1 = nullptr, *W2 = nullptr;
  const z *hW1 = nullptr, *hW2 = nullptr;  // optional host copies of W1, W2
  int64_t chl = 0, chr = 0, d = 0, D = 0;
  std::vector<int64_t> qa, qb;
  std::vector<int> wq;
};

// grouped tcgen05 task: rows a_row0.. of the packed A planes, b_row0.. of the packed B
// planes, output re plane at c_off (+ split * split_stride), leading dimension ldc
struct GTask {
  int a_row0, b_row0;
  int M, N;
  int kb_total, kb_per_split;
  int64_t c_off;
  int64_t ldc;
};
// grouped FP64 task: C[c_off + i c_rs + j] = sum_k A[a_off + i a_rs + k a_cs] B[b_off + k b_rs + j b_cs]
struct ZTask {
  int64_t M, N, K;
  int64_t a_off, a_rs, a_cs;
  int64_t b_off, b_rs, b_cs;
  int64_t c_off, c_rs;
};
// contiguous run copied (and split, for the TF32 planes) by the pack kernel; src is an
// absolute device address (environments of several problems), dst an element offset
struct PackSeg {
  const z* src;
  int64_t dst;
  int64_t len;
};
// theta slab [K][N] at src, written transposed to packed rows dst_row0 + n, column k
struct TSlab {
  int64_t src, N, K, dst_row0;
};
// W contraction for one (a' sector, b sector) pair: element (i, j), i < n_a, j < n_b
struct WPair {
  int64_t n_a, n_b;
  int out0, nout;
};
struct WOut {
  int64_t base;  // output element (0, 0)
  int r0, r1;    // input terms [r0, r1) in the WIn table
};
struct WIn {
  int64_t base, rs;  // input element (i, j) at base + i rs + j
  z val;
};
// one output row of stage 4: Y row at src, compact-theta row at dst, n entries
struct GRow {
  int64_t src, dst;
  int64_t n;
};

// host description of one stage's grouped GEMM (before tiling)
struct TaskDesc {
  int64_t a_row0, b_row0, M, N, K, c_off, ldc;
};

// kernel arguments (one struct per kernel, so that a graph node's input or output
// pointer can be patched before a replay)
struct TPArgs {   // theta slabs -> transposed split-TF32 planes
  const z* x;
  const TSlab* slabs;
  const int4* tiles;  // (slab, n0, k0, -)
  int ntiles;
  float* dst;
  int64_t KA, plane;
};
struct GArgs {    // grouped split-TF32 complex GEMM
  const GTask* tasks;
  const int4* tiles;  // (task, m0, n0, split)
  int ntiles;
  float* C;
  int64_t plane, split_stride;
  int* status;
};
struct ZGArgs {   // grouped FP64 complex GEMM
  const ZTask* tasks;
  const int4* tiles;  // (task, m0, n0, -)
  int ntiles;
  const z* A;
  const z* B;
  z* C;
};
struct WArgs {    // W1 W2 contraction between the stages
  const WPair* pairs;
  const WOut* outs;
  const WIn* ins;
  const int2* tiles;  // (pair, first element)
  int ntiles;
  const float* t1f;   // FP32 re plane; im plane at + p1
  int64_t p1;
  const z* t1z;
  float* a4f;         // split planes of p4 elements each
  int64_t p4;
  z* a4z;
  int64_t out_rs;
};
struct GthArgs {  // stage-4 rows -> compact y
  const GRow* rows;
  int nrows;
  const float* yf;    // FP32 re plane; im at + plane; split s at + s sstride
  int64_t plane, sstride;
  int nsplit;
  const z* yz;
  z* y;
};

struct U1Plan {
  // host layout (u1_layout), kept until the tables are uploaded
  std::vector<PackSeg> segA1, segB4;
  std::vector<TSlab> slabs;
  std::vector<int4> ttiles;
  std::vector<WPair> pairs;
  std::vector<WOut> outs;
  std::vector<WIn> ins;
  std::vector<int2> wtiles;
  std::vector<GRow> rows;
  size_t bytes = 0;                 // device scratch the plan takes
  int nprob = 0;
  int64_t n = 0;                    // compact length over all problems
  std::vector<int64_t> x_off;       // per problem
  std::string sig;                  // block-structure signature (autotuner key)
  double flops = 0;                 // algorithmic FLOPs of one matvec (blocks only)
  double dense_flops = 0;           // the same problems without the U(1) blocks
  // stage 1
  std::vector<TaskDesc> s1, s4;
  int64_t KA1 = 0, rowsA1 = 0, rowsB1 = 0, KA4 = 0, rowsA4 = 0, rowsB4 = 0;
  int64_t P1 = 0, P4 = 0;           // elements per plane of T1 and of Y
  // split-TF32 operands (4 planes each) and FP32 intermediates
  float *A1p = nullptr, *B1p = nullptr, *T1f = nullptr, *A4p = nullptr, *B4p = nullptr, *Yf = nullptr;
  // FP64 operands and intermediates
  z *A1z = nullptr, *T1z = nullptr, *A4z = nullptr, *B4z = nullptr, *Yz = nullptr;
  // device tables
  TSlab* d_slabs = nullptr; int4* d_ttiles = nullptr; int n_ttiles = 0;
  WPair* d_pairs = nullptr; WOut* d_outs = nullptr; WIn* d_ins = nullptr;
  int2* d_wtiles = nullptr; int n_wtiles = 0;
  GRow* d_rows = nullptr; int n_rows = 0;
  ZTask* d_z1 = nullptr; int4* d_z1tiles = nullptr; int n_z1tiles = 0;
  ZTask* d_z4 = nullptr; int4* d_z4tiles = nullptr; int n_z4tiles = 0;
  GTask* d_g1 = nullptr; int4* d_g1tiles = nullptr; int n_g1tiles = 0;
  GTask* d_g4 = nullptr; int4* d_g4tiles = nullptr; int n_g4tiles = 0;
  int cap_g1tiles = 0, cap_g4tiles = 0;
  // tile choice (autotuned): N tile of stage 1 and stage 4, split-K of stage 4
  int bn1 = 128, bn4 = 128, split4 = 1;
  int ztile = 64;                   // FP64 grouped tiles: 64 x 64, or 16 x 16 for small structures
  CUtensorMap tmA1, tmB1, tmA4, tmB4;  // B maps are rebuilt for the chosen N tile
  // CUDA graphs of one matvec per precision (input / output pointers patched per replay)
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaGraphNode_t in_node[2] = {nullptr, nullptr}, out_node[2] = {nullptr, nullptr};
  TPArgs in_tp{};
  ZGArgs in_zg{};
  GthArgs out_g[2]{};
  U1Plan() = default;
  U1Plan(const U1Plan&) = delete;
  U1Plan& operator=(const U1Plan&) = delete;
  ~U1Plan();
};

// host layout of the grouped matvec (no device work); sets p->bytes
int u1_layout(Ctx* c, const std::vector<U1Spec>& probs, U1Plan* p);
// device buffers from the scratch arena (p->bytes must fit), packed constant operands,
// tables, and the autotuned tile choice
int u1_prepare(Ctx* c, const std::vector<U1Spec>& probs, U1Plan* p);
int u1_run(Ctx* c, U1Plan& p, const z* x, z* y, int precision);
// compact length of one problem, and dense <-> compact conversion of theta
int64_t u1_compact_size(const U1Spec& s);
int u1_convert(Ctx* c, const U1Spec& s, const z* src, z* dst, int to_compact);
// validates labels (non-decreasing) and sizes; TNT_OK or TNT_E_INVALID with a message
int u1_check(Ctx* c, const U1Spec& s);

// the grouped matvec as the Lanczos operator
struct U1MatVec : MatVec {
  U1Plan& p;
  explicit U1MatVec(U1Plan& pp) : p(pp) { n = pp.n; }
  int apply(Ctx* c, const z* x, z* y, int precision) const override {
    return u1_run(c, p, x, y, precision);
  }
};

}  // namespace tnt
