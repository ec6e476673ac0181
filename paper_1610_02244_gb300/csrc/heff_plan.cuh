// Prepared H_eff.theta contraction: operator tables and scratch for repeated matvecs.
#pragma once

#include "tnt_internal.cuh"

namespace tnt {

struct MixedPlan;  // split-TF32 tensor-core operands (tc_mixed.cu)

struct HeffPlan {
  const z* L = nullptr;
  const z* R = nullptr;
  int64_t chl = 0, d = 0, D = 0, chr = 0;
  int precision = TNT_PREC_FP64;
  OpApply op{};        // W12 acting T1 -> T3
  z* T1 = nullptr;     // [a'][w][s1][s2][b]
  z* T3 = nullptr;     // [a'][s1'][s2'][w2][b]
  MixedPlan* mixed = nullptr;  // lives in scratch
};

size_t heff_scratch_bound(int64_t chl, int64_t d, int64_t D, int64_t chr, int precision);
int heff_prepare(Ctx* c, const z* L, const z* W1, const z* W2, const z* R, int64_t chl,
                 int64_t d, int64_t D, int64_t chr, int precision, HeffPlan* p);
int heff_run(Ctx* c, const HeffPlan& p, const z* theta, z* y, int precision);
int heff_run_f64(Ctx* c, const HeffPlan& p, const z* theta, z* y);

// split-TF32 tensor-core path
size_t heff_mixed_scratch_bound(int64_t chl, int64_t d, int64_t D, int64_t chr);
int heff_mixed_prepare(Ctx* c, HeffPlan* p);
int heff_run_mixed(Ctx* c, const HeffPlan& p, const z* theta, z* y);

size_t env_scratch_bound(int64_t chl, int64_t d, int64_t D, int64_t chr);
int env_left_impl(Ctx* c, const z* Lenv, const z* W, const z* A, int64_t chl, int64_t d,
                  int64_t D, int64_t chr, z* Lout);
int env_right_impl(Ctx* c, const z* Renv, const z* W, const z* B, int64_t chl, int64_t d,
                   int64_t D, int64_t chr, z* Rout);
int theta_form_impl(Ctx* c, const z* A, const z* B, int64_t chl, int64_t d, int64_t chm,
                    int64_t chr, z* theta);
int gate_apply_impl(Ctx* c, const std::vector<z>& G, const z* theta, int64_t chl, int64_t d,
                    int64_t chr, z* out);

// Lanczos (lanczos.cu)
size_t lanczos_scratch_bound(int64_t n, int krylov_cap);
int lanczos_impl(Ctx* c, const HeffPlan& p, z* theta, tnt_lanczos_result* res);

}  // namespace tnt
