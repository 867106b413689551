// k_iterate_128x4_grp: k_iterate compiled for 128 threads per block, at least 4 resident blocks per SM, for the
// batch's group integrals.
#include "mbpt_kernels.cuh"
#include "mbpt_kernels.h"

namespace mbpt {

__global__ void __launch_bounds__(128, 4) k_iterate_128x4_grp(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist) {
    k_iterate_body<128, 2>(hdr, items, csum, chist);
}

}  // namespace mbpt
