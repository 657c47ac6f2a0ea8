// placeholder, replaced by the adjoint kernels
#include "plan.h"
namespace selinv { void adjoint_release(void *) {} }
extern "C" int selinv_adjoint(selinv_plan, selinv_dtype, const void *, const void *, const void *, const void *, void *, void *, void *) { return SELINV_ERR_UNSUPPORTED; }
extern "C" int selinv_factor_adjoint(selinv_plan, selinv_dtype, const void *, const void *, const void *, const void *, void *, void *) { return SELINV_ERR_UNSUPPORTED; }
