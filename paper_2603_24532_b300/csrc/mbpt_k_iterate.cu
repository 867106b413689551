// k_iterate for one launch shape and one batch part, chosen when the unit is compiled: MBPT_TPB threads
// per block, at least MBPT_MINB resident blocks per SM (which caps the registers per thread), batch part
// MBPT_PART (bit 0: integrals with the denominator regulator, bit 1: group integrals, bit 2: sixth order).
// The build compiles this unit once per (shape, part), so that each kernel carries only its own
// instantiations and the instantiations compile in parallel.
#include "mbpt_kernels.cuh"
#include "mbpt_kernels.h"

#if !defined(MBPT_TPB) || !defined(MBPT_MINB) || !defined(MBPT_PART)
#error "compile with -DMBPT_TPB=<threads> -DMBPT_MINB=<blocks per SM> -DMBPT_PART=<0..7>"
#endif

namespace mbpt {

__global__ void __launch_bounds__(MBPT_TPB, MBPT_MINB)
    MBPT_K_ITERATE(MBPT_TPB, MBPT_MINB, MBPT_PART)(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist) {
    k_iterate_body<MBPT_TPB, MBPT_PART>(hdr, items, csum, chist);
}

}  // namespace mbpt
