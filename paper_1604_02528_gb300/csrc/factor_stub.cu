// placeholder, replaced by the factorization/adjoint kernels
#include "plan.h"
namespace selinv { void factor_release(selinv_plan_s *) {} }
extern "C" int selinv_plan_set_matrix(selinv_plan, int32_t, const int64_t *, const int32_t *) { return SELINV_ERR_UNSUPPORTED; }
extern "C" int selinv_factor(selinv_plan, selinv_dtype, const void *, void *, void *, void *) { return SELINV_ERR_UNSUPPORTED; }
extern "C" int selinv_adjoint(selinv_plan, selinv_dtype, const void *, const void *, const void *, const void *, void *, void *, void *) { return SELINV_ERR_UNSUPPORTED; }
extern "C" int selinv_factor_adjoint(selinv_plan, selinv_dtype, const void *, const void *, const void *, const void *, void *, void *) { return SELINV_ERR_UNSUPPORTED; }
