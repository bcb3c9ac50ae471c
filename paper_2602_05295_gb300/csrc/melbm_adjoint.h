// melbm_adjoint.h -- internal interface of the discrete-adjoint translation unit.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace melbm {
struct AdjointState;
void adjoint_free(AdjointState* a);
}  // namespace melbm
