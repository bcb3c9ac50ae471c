// adjoint.cu -- discrete adjoint of the fluid step (placeholder until the
// adjoint kernels land).
#include "../../include/melbm.h"
#include "melbm_adjoint.h"

namespace melbm {
struct AdjointState {};
void adjoint_free(AdjointState* a) { delete a; }
}  // namespace melbm

extern "C" {
int melbm_forward_checkpointed(melbm_t, const float*, int, int) { return MELBM_EINVAL; }
int melbm_backward(melbm_t, const float*, float*, float*) { return MELBM_EINVAL; }
}
