// Declarations of the __global__ entry points of libmbpt (defined in mbpt_k_*.cu).
#pragma once
#include <stdint.h>

#include "mbpt_internal.h"

namespace mbpt {

// sample evaluation: persistent, chunks from an atomic counter; one definition per launch shape
// (threads per block x minimum resident blocks per SM) and batch part (_reg: integrals with the
// denominator regulator; _grp: group integrals)
__global__ void k_iterate_256x2(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_128x4(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_256x1(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_128x3(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_256x2_reg(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_128x4_reg(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_256x1_reg(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_128x3_reg(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_256x2_grp(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_128x4_grp(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_256x1_grp(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_128x3_grp(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_256x2_grp_reg(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_128x4_grp_reg(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_256x1_grp_reg(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);
__global__ void k_iterate_128x3_grp_reg(WorkHeader* hdr, const WorkItem* items, double* csum, float* chist);

// per integral: fixed-order reduction of the chunk slots, combination, convergence, refinement
__global__ void k_finalize(WorkHeader* hdr, const WorkItem* items, const double* csum, const float* chist,
                           double* const* last_hist);
// test hooks
__global__ void k_dump(const DiagRec* rec, int n_members, const double* grid, uint64_t seed, uint32_t sid, uint32_t iter,
                       uint64_t first, uint64_t count, double* xo, double* wo);
__global__ void k_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                         uint64_t count, uint32_t* out);

}  // namespace mbpt
