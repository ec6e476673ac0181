// placeholder replaced by the tensor-core path
#include "heff_plan.cuh"
namespace tnt {
size_t heff_mixed_scratch_bound(int64_t, int64_t, int64_t, int64_t) { return 0; }
int heff_mixed_prepare(Ctx* c, HeffPlan*) { return set_err(c, TNT_E_UNSUPPORTED, "mixed precision not built"); }
int heff_run_mixed(Ctx* c, const HeffPlan&, const z*, z*) { return set_err(c, TNT_E_UNSUPPORTED, "mixed precision not built"); }
}
