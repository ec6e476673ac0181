// Prepared H_eff.theta contraction: operator tables and scratch for repeated matvecs.
#pragma once

#include <cuda.h>  // CUtensorMap (type only; the encoder is fetched from the driver)

#include "tnt_internal.cuh"

namespace tnt {

// Split-TF32 operands of the two chi^3 contractions (tc_mixed.cu).  Every operand is four
// FP32 planes (re_hi, re_lo, im_hi, im_lo), K-major, rows padded to 128 and K to 16 with
// zeros; a 3-D TMA map [plane][row][k] addresses each.
struct MixedPlan {
  int64_t M1, N1, K1, Mp1, Np1, Kp1;  // stage 1: T1[(a' w)][(s1 s2 b)] = L . theta
  int64_t M4, N4, K4, Mp4, Np4, Kp4;  // stage 4: y[(a' s1' s2')][b'] = T3 . R^T
  int split4 = 1;                     // split-K factor of stage 4
  float* Lp = nullptr;      // 4 x Mp1 x Kp1
  float* Thp = nullptr;     // 4 x Np1 x Kp1   (theta transposed)
  float* T1 = nullptr;      // 2 x M1 x N1     (re, im accumulators of stage 1)
  float* T3p = nullptr;     // 4 x Mp4 x Kp4
  float* Rp = nullptr;      // 4 x Np4 x Kp4
  float* Yp = nullptr;      // split4 x 2 x M4 x N4
  OpApply op{};             // W12 on T1 -> T3 planes (offsets in plane units)
  CUtensorMap tmL, tmTh, tmT3, tmR;
};

struct HeffPlan {
  const z* L = nullptr;
  const z* R = nullptr;
  int64_t chl = 0, d = 0, D = 0, chr = 0;
  int precision = TNT_PREC_FP64;
  OpApply op{};        // W12 acting T1 -> T3
  z* T1 = nullptr;     // [a'][w][s1][s2][b]
  z* T3 = nullptr;     // [a'][s1'][s2'][w2][b]
  MixedPlan mixed{};   // used when precision == TNT_PREC_MIXED
};

size_t heff_scratch_bound(int64_t chl, int64_t d, int64_t D, int64_t chr, int precision);
int heff_prepare(Ctx* c, const z* L, const z* W1, const z* W2, const z* R, int64_t chl,
                 int64_t d, int64_t D, int64_t chr, int precision, HeffPlan* p,
                 const z* hW1 = nullptr, const z* hW2 = nullptr);
int heff_run(Ctx* c, const HeffPlan& p, const z* theta, z* y, int precision);
int heff_run_f64(Ctx* c, const HeffPlan& p, const z* theta, z* y);

// split-TF32 tensor-core path
// 3-D TMA map over planes[4][rows][K] (FP32, K % 4 == 0): box 16 x box_rows x 1, 64 B swizzle
int tma_map_planes(Ctx* c, CUtensorMap* tm, float* base, int64_t rows, int64_t K, int box_rows);
int tma_map_planes_n(Ctx* c, CUtensorMap* tm, float* base, int64_t rows, int64_t K, int box_rows,
                     int nplanes);
size_t heff_mixed_scratch_bound(int64_t chl, int64_t d, int64_t D, int64_t chr);
int heff_mixed_prepare(Ctx* c, HeffPlan* p);
int heff_run_mixed(Ctx* c, const HeffPlan& p, const z* theta, z* y);

size_t env_scratch_bound(int64_t chl, int64_t d, int64_t D, int64_t chr);
// hW (optional): a host copy of W, which spares the read-back of the device tensor
int env_left_impl(Ctx* c, const z* Lenv, const z* W, const z* A, int64_t chl, int64_t d,
                  int64_t D, int64_t chr, z* Lout, const z* hW = nullptr);
int env_right_impl(Ctx* c, const z* Renv, const z* W, const z* B, int64_t chl, int64_t d,
                   int64_t D, int64_t chr, z* Rout, const z* hW = nullptr);
int theta_form_impl(Ctx* c, const z* A, const z* B, int64_t chl, int64_t d, int64_t chm,
                    int64_t chr, z* theta);
int gate_apply_impl(Ctx* c, const std::vector<z>& G, const z* theta, int64_t chl, int64_t d,
                    int64_t chr, z* out);

// Lanczos (lanczos.cu) on any Hermitian operator given as a matvec y = A x over n complex
// entries; precision selects the matvec path (the win-back asks for TNT_PREC_FP64).
struct MatVec {
  int64_t n = 0;
  virtual int apply(Ctx* c, const z* x, z* y, int precision) const = 0;
  virtual ~MatVec() = default;
};
size_t lanczos_scratch_bound(int64_t n, int krylov_cap);
int lanczos_run(Ctx* c, const MatVec& A, z* theta, tnt_lanczos_result* res);
int lanczos_impl(Ctx* c, const HeffPlan& p, z* theta, tnt_lanczos_result* res);
// independent problems in lock step: off[p] .. off[p+1] is problem p's part of the vectors
// (A must be block diagonal over those parts); one result per problem
size_t lanczos_batched_scratch_bound(int64_t n, int nprob, int krylov_cap);
int lanczos_batched(Ctx* c, const MatVec& A, const std::vector<int64_t>& off, z* x,
                    std::vector<tnt_lanczos_result>* out);

}  // namespace tnt
