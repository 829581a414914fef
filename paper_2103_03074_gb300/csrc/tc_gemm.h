// Tensor-core (tcgen05) split-precision complex GEMM forms.
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"
#include "tn.h"

namespace tn {

// true if `form` has a tensor-core GEMM in this build
bool tc_form_available(tn_form form);

// Same contract as launch_gemm_f32, computed in the split form `form`.
cudaError_t launch_gemm_tc(const GemmArgs &a, tn_form form, cudaStream_t s);

}  // namespace tn
