// k_iterate_128x3_reg: k_iterate compiled for 128 threads per block, at least 3 resident blocks per SM, for the
// batch's plain integrals with the denominator regulator.
#include "mbpt_kernels.cuh"
#include "mbpt_kernels.h"

namespace mbpt {

__global__ void __launch_bounds__(128, 3) k_iterate_128x3_reg(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist) {
    k_iterate_body<128, 1>(hdr, items, csum, chist);
}

}  // namespace mbpt
