// Declarations of the __global__ entry points of libmbpt (defined in mbpt_k_iterate.cu and mbpt_k_misc.cu).
#pragma once
#include <stdint.h>

#include "mbpt_internal.h"

// Name of the sample-evaluation kernel of one launch shape (threads per block t x minimum resident blocks
// per SM b) and batch part p (bit 0: integrals with the denominator regulator, bit 1: group integrals,
// bit 2: sixth order): k_iterate_<t>x<b> followed by _o6, _grp and _reg as the bits say.
#define MBPT_PSUF_0
#define MBPT_PSUF_1 _reg
#define MBPT_PSUF_2 _grp
#define MBPT_PSUF_3 _grp_reg
#define MBPT_PSUF_4 _o6
#define MBPT_PSUF_5 _o6_reg
#define MBPT_PSUF_6 _o6_grp
#define MBPT_PSUF_7 _o6_grp_reg
#define MBPT_PSUF_I(p) MBPT_PSUF_##p
#define MBPT_PSUF(p) MBPT_PSUF_I(p)
#define MBPT_KNAME_I(t, b, suf) k_iterate_##t##x##b##suf
#define MBPT_KNAME(t, b, suf) MBPT_KNAME_I(t, b, suf)
#define MBPT_K_ITERATE(t, b, p) MBPT_KNAME(t, b, MBPT_PSUF(p))

// the parts of one shape, in part order
#define MBPT_K_ITERATE_PARTS(t, b)                                                                          \
    MBPT_K_ITERATE(t, b, 0), MBPT_K_ITERATE(t, b, 1), MBPT_K_ITERATE(t, b, 2), MBPT_K_ITERATE(t, b, 3),     \
        MBPT_K_ITERATE(t, b, 4), MBPT_K_ITERATE(t, b, 5), MBPT_K_ITERATE(t, b, 6), MBPT_K_ITERATE(t, b, 7)

namespace mbpt {

#define MBPT_DECLARE_K_ITERATE(t, b, p) \
    __global__ void MBPT_K_ITERATE(t, b, p)(WorkHeader * hdr, const WorkItem* items, double* csum, float* chist);
#define MBPT_DECLARE_SHAPE(t, b)                                                                                \
    MBPT_DECLARE_K_ITERATE(t, b, 0) MBPT_DECLARE_K_ITERATE(t, b, 1) MBPT_DECLARE_K_ITERATE(t, b, 2)            \
    MBPT_DECLARE_K_ITERATE(t, b, 3) MBPT_DECLARE_K_ITERATE(t, b, 4) MBPT_DECLARE_K_ITERATE(t, b, 5)            \
    MBPT_DECLARE_K_ITERATE(t, b, 6) MBPT_DECLARE_K_ITERATE(t, b, 7)

// sample evaluation: persistent, chunks from an atomic counter; one definition per launch shape and batch part
MBPT_DECLARE_SHAPE(256, 2)
MBPT_DECLARE_SHAPE(128, 4)
MBPT_DECLARE_SHAPE(256, 1)
MBPT_DECLARE_SHAPE(128, 3)
#undef MBPT_DECLARE_SHAPE
#undef MBPT_DECLARE_K_ITERATE

// per integral: fixed-order reduction of the chunk slots, combination, convergence, refinement
__global__ void k_finalize(WorkHeader* hdr, const WorkItem* items, const double* csum, const float* chist,
                           double* const* last_hist);
// batched estimate: the first `words` 16-byte words of each listed integral's state, into one array
__global__ void k_gather_heads(const DiagState* const* src, int k, int words, uint4* out);
// test hooks
__global__ void k_dump(const DiagRec* rec, int n_members, const double* grid, uint64_t seed, uint32_t sid, uint32_t iter,
                       uint64_t first, uint64_t count, uint32_t spin, double* xo, double* wo);
__global__ void k_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                         uint64_t count, uint32_t* out);

}  // namespace mbpt
