// k_iterate_256x2: k_iterate compiled for 256 threads per block, at least 2 resident blocks per SM, for the
// batch's plain integrals.
#include "mbpt_kernels.cuh"
#include "mbpt_kernels.h"

namespace mbpt {

__global__ void __launch_bounds__(256, 2) k_iterate_256x2(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist) {
    k_iterate_body<256, 0>(hdr, items, csum, chist);
}

}  // namespace mbpt
