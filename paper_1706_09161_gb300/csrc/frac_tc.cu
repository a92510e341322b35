// Fractional terms on the tensor cores (split-precision forms): not built yet.
#include "lbm_internal.h"

namespace lbm {

cudaError_t launch_frac_tc(const lbm_s*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_split_C(const lbm_s*, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace lbm
