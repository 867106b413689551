// Device kernels of libmbpt (internal): chunk scheduling, the per-chunk sample loop, reductions,
// refinement.  Templates and inline functions only; the __global__ entry points are defined in
// separate translation units (one per compiled launch shape) so they build in parallel.
#pragma once
#include <stdint.h>

#include "mbpt_device.cuh"
#include "mbpt_internal.h"

namespace mbpt {

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
// pre-test rounds between evaluation phases (longer phases keep the instruction cache warmer; a
// group chunk has only as many rounds as its samples per thread, so the group parts take short
// phases and spend the shared memory on per-sample slots), and the per-warp stack length: one
// phase of both classes (a phase's stacks are evaluated in full before the next phase)
__host__ __device__ constexpr int class_rounds(int part) {
    return (part & 3) == 3 ? 4 : ((part & 3) == 2 ? 16 : 32);
}
__host__ __device__ constexpr int group_slots(int part) { return (part & 3) == 3 ? kGroupSlotsReg : kGroupSlotsPlain; }
__host__ __device__ constexpr int queue_len(int part) { return 32 * class_rounds(part); }

// Shared memory of one k_iterate block; the regulator and group arrays exist only in their parts
// (PART bit 0: regulator, bit 1: group; the sixth-order bit does not change the layout), which leaves the
// plain kernel room for long pre-test phases.
template <int NW, int PART = 0>
struct alignas(16) ChunkSmemT {
    DiagRec rec;
    Grid2 grid[kCells];
    float hist[NW][kCells];                  // warp-private FP32 histograms, or (kHistBlockF64) the first
                                             // 8 kCells bytes hold one block-shared FP64 histogram
    double cacc[(PART & 1) ? 2 * kComp : 1][NW * 32];   // per-thread sums of the regulator components
    double gacc[(PART & 2) ? group_slots(PART) : 1][NW * 32];  // group integrals: per-sample sums over the members
    uint32_t queue[NW][queue_len(PART)];     // per-warp stacks of samples past the pre-test
                                             // (away from a Fermi surface from the bottom, near one from the top)
    int rem[2][NW];                          // per warp: far and near samples of the phase on its stacks
    double red[2][NW];
    double redc[(PART & 1) ? 2 * kComp : 1][NW];
    uint32_t chunk, item, iter, skip;
};
using ChunkSmem = ChunkSmemT<kWarps, 0>;
static_assert(sizeof(double) * kCells <= sizeof(float) * 4 * kCells, "the FP64 histogram fits the FP32 ones of 4 warps");

__device__ __forceinline__ void load_record(DiagRec* dst, const DiagRec* src) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(DiagRec) / 16); i += blockDim.x) d[i] = s[i];
}

// The FP32 sampling map needs every bin wider than float resolution; an iteration whose grid has a
// narrower bin samples with the FP64 map instead (decided per integral and iteration, so every chunk
// of the integral takes the same path).  Must be called by every thread of the block.
__device__ __forceinline__ int effective_precision(int prec, const double* grid, int d, int nb) {
    if (prec != MBPT_MIXED) return prec;
    int bad = 0;
    for (int idx = threadIdx.x; idx < d * nb; idx += blockDim.x) {
        const int a = idx / nb, i = idx - a * nb;
        const double e0 = grid[a * (nb + 1) + i], e1 = grid[a * (nb + 1) + i + 1];
        if (e1 > e0 && !((float)e1 > (float)e0)) bad = 1;
    }
    return __syncthreads_or(bad) ? MBPT_MIXED_MAP64 : prec;
}

__device__ __forceinline__ void load_grid(Grid2* gs, const double* grid, int d, int nb, int prec) {
    const int stride = grid_stride(d);
    for (int idx = threadIdx.x; idx < d * nb; idx += blockDim.x) {
        const int a = idx / nb, i = idx - a * nb;
        const double e0 = grid[a * (nb + 1) + i], e1 = grid[a * (nb + 1) + i + 1];
        const double de = e1 - e0;
        if (prec == MBPT_MIXED) {
            // FP32 bins tile [0, 1] exactly: width = difference of the rounded edges
            Grid4f g;
            g.e = (float)e0;
            g.de = (float)e1 - g.e;
            g.pad0 = 0.0f;
            g.pad1 = 0.0f;
            reinterpret_cast<Grid4f*>(gs)[a * stride + i] = g;
        } else {
            Grid2 g;
            g.de = de;
            g.a = (prec == MBPT_FP64) ? e0 : e0 - de;
            gs[a * stride + i] = g;
        }
    }
}

// Histogram of w^2 over the sample's bins: warp-private FP32 bins (clamped below FLT_MAX), or
// (layout kHistBlockF64) one FP64 histogram shared by the block at the start of the same array.
template <int D>
__device__ __forceinline__ void hist_add(float* hist, float* hist_block, uint32_t layout, int nb,
                                         const uint32_t* binpack, double w) {
    if (layout == kHistBlockF64) {
        double* h = reinterpret_cast<double*>(hist_block);
        const double w2 = w * w;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const uint32_t i = (binpack[a >> 2] >> (8 * (a & 3))) & 0xffu;
            atomicAdd(&h[a * nb + i], w2);
        }
        return;
    }
    const float wf = narrow_trunc(w);
    float w2 = wf * wf;
    if (!(w2 <= 3.0e38f)) w2 = 3.0e38f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const uint32_t i = (binpack[a >> 2] >> (8 * (a & 3))) & 0xffu;
        atomicAdd(&hist[a * nb + i], w2);
    }
}

// Bin indices of sample s alone (the same integer map as eval_sample: i = floor((u + 1/2) 2^-32 nb), bin_split).
template <int D>
__device__ __forceinline__ void sample_bins(uint32_t s, uint32_t t, uint32_t sid, uint32_t k0, uint32_t k1,
                                            uint32_t nb, uint32_t* binpack) {
    constexpr int NBLK = (D + 3) / 4;
#pragma unroll
    for (int w = 0; w < kBinWords; ++w) binpack[w] = 0;
#pragma unroll
    for (int j = 0; j < NBLK; ++j) {
        uint32_t u[4];
        philox4x32_10(s, t, sid, (uint32_t)j, k0, k1, u);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int a = 4 * j + q;
            if (a < D) {
                uint32_t i, lo;
                bin_split(u[q], nb, i, lo);
                binpack[a >> 2] |= i << (8 * (a & 3));
            }
        }
    }
}

// One chunk: samples first + j*blockDim + tid, j < spt.
//  Plain integrals, every precision: the FP64 pipe issues per warp instruction, so a warp whose
//  lanes hold a mix of zero and live samples pays for the zero ones, and (mixed mode) one whose lanes
//  take both sampling maps pays for both.  Each warp therefore alternates two phases, each a tight loop over
//  its own code: class_rounds() rounds of the FP32 front and Fermi-step pre-test, pushing the samples
//  that may be live onto one of two shared-memory stacks by class (away from / near a Fermi
//  surface; ballot + prefix count); then, behind a barrier, the block evaluates all its warps' stacks
//  together in groups of 32 of one class, spread round-robin over the warps, so a phase leaves at most one
//  partial group per class in the whole block and every warp gets the same number of groups to within one.
//  Which thread sums which sample depends only on the chunk, so results stay deterministic.
//  A group integral (n_members > 1; its own kernel, GRP) evaluates every member at each sample, member
//  by member with the record swapped in shared memory, each member's samples through the phases
//  above, adding the weights per sample into gacc, zeroed per chunk (spt x (1 + regulator components)
//  <= group_slots() slots per thread); sums, squares and the histogram then see the group's integrand.
template <int N, int PREC, int MAPK, bool REG, bool GRP, int NW>
__device__ __forceinline__ void run_chunk(ChunkSmemT<NW, (REG ? 1 : 0) | (GRP ? 2 : 0)>& S, const WorkItem& W,
                                          uint32_t chunk_local, double& sw, double& sw2) {
    const DiagRec& R = S.rec;
    const int w_spt = W.spt;
    const uint64_t w_samples = W.samples;
    const uint32_t w_sid = W.stream_id;
    const double* const w_grid = W.grid;
    const uint32_t cs = blockDim.x * (uint32_t)w_spt;
    const uint64_t first = (uint64_t)chunk_local * cs;
    const uint32_t t = S.iter;
    const uint32_t k0 = (uint32_t)W.seed, k1 = (uint32_t)(W.seed >> 32);
    float* hist = S.hist[threadIdx.x >> 5];
    float* hist_block = &S.hist[0][0];
    const uint32_t layout = W.hist_layout;
    const uint32_t spin = W.spin_sum;
    uint32_t* q = S.queue[threadIdx.x >> 5];
    const uint32_t lane = threadIdx.x & 31u;
    const int nb = R.nb;
    constexpr int D = 3 * (N + 1) - 3 * MAPK;
    constexpr int PER = REG ? 1 + kComp : 1;        // group slots per sample
    constexpr int kRounds = class_rounds((REG ? 1 : 0) | (GRP ? 2 : 0));
    constexpr int kQ = queue_len((REG ? 1 : 0) | (GRP ? 2 : 0));
    // (the plain kernels keep the direct loop as a runtime branch that never runs: with the loop
    // structure fixed at compile time their register allocation is worse -- measured 1 KB stack
    // frame instead of 120 B, and 2 % slower)
    const int nm = GRP ? (int)W.n_members : 1;
    const bool compact = GRP || W.n_members <= 1;
    for (int m = 0; m < nm; ++m) {
        if (m > 0) {
            __syncthreads();
            load_record(&S.rec, W.rec + m);
            __syncthreads();
        }
        // Phases: every warp classifies rounds [j0, j0 + kRounds) of the chunk onto its two stacks; after a
        // barrier the block evaluates the concatenation of all warps' far stacks (warp order), then of their
        // near stacks, in groups of 32, group g by warp g mod NW (so at most one partial group per class and
        // phase, the groups spread evenly over the warps, and the assignment depends only on the chunk);
        // a second barrier before the stacks are filled again.  pf / pn: lane w < NW holds the inclusive
        // prefix sum of the far / near counts of warps 0..w.
        int j0 = 0, g = -1, n_gf = 0, n_g = 0, pf = 0, pn = 0;
        for (;;) {
            uint64_t s;
            bool have, use_near = false;
            if (compact) {
                if (g < 0 || g >= n_g) {
                    if (g >= 0) __syncthreads();   // end of a phase: the stacks are reused
                    if (j0 >= w_spt) break;
                    const int jend = (j0 + kRounds < w_spt) ? j0 + kRounds : w_spt;
                    int nf = 0, nn = 0;
                    for (int j = j0; j < jend; ++j) {
                        const uint64_t sc = first + (uint64_t)j * blockDim.x + threadIdx.x;
                        const int cls = sc < w_samples
                                            ? sample_class<N, MAPK, PREC>(R, S.grid, (uint32_t)sc, t, w_sid, k0, k1)
                                            : kClassZero;
                        const uint32_t lt = (1u << lane) - 1u;
                        const uint32_t b0 = __ballot_sync(0xffffffffu, cls == kClassFar);
                        const uint32_t b1 = __ballot_sync(0xffffffffu, cls == kClassNear);
                        if (cls == kClassFar) q[nf + __popc(b0 & lt)] = (uint32_t)sc;
                        if (cls == kClassNear) q[kQ - 1 - (nn + __popc(b1 & lt))] = (uint32_t)sc;
                        nf += __popc(b0);
                        nn += __popc(b1);
                    }
                    j0 = jend;
                    const int warp = (int)(threadIdx.x >> 5);
                    if (lane == 0) {
                        S.rem[0][warp] = nf;
                        S.rem[1][warp] = nn;
                    }
                    __syncthreads();
                    pf = ((int)lane < NW) ? S.rem[0][lane] : 0;
                    pn = ((int)lane < NW) ? S.rem[1][lane] : 0;
#pragma unroll
                    for (int o = 1; o < NW; o <<= 1) {
                        const int a = __shfl_up_sync(0xffffffffu, pf, o), b = __shfl_up_sync(0xffffffffu, pn, o);
                        if ((int)lane >= o) {
                            pf += a;
                            pn += b;
                        }
                    }
                    n_gf = (__shfl_sync(0xffffffffu, pf, NW - 1) + 31) >> 5;
                    n_g = n_gf + ((__shfl_sync(0xffffffffu, pn, NW - 1) + 31) >> 5);
                    g = warp;
                    if (g >= n_g) continue;
                }
                use_near = g >= n_gf;
                const int src = use_near ? pn : pf;
                const int e = (use_near ? g - n_gf : g) * 32 + (int)lane;
                have = e < __shfl_sync(0xffffffffu, src, NW - 1);
                // owner warp of entry e: the first w with prefix(w) > e (binary search over the NW prefixes)
                int w = 0;
#pragma unroll
                for (int step = NW / 2; step >= 1; step >>= 1) {
                    const int v = __shfl_sync(0xffffffffu, src, w + step - 1);
                    if (v <= e) w += step;
                }
                const int prev = __shfl_sync(0xffffffffu, src, w > 0 ? w - 1 : 0);
                const int k = e - (w > 0 ? prev : 0);
                s = !have ? 0u : (use_near ? S.queue[w][kQ - 1 - k] : S.queue[w][k]);
                g += NW;
            } else {
                if (j0 >= w_spt) break;
                s = first + (uint64_t)j0 * blockDim.x + threadIdx.x;
                have = s < w_samples;
                ++j0;
            }
            if (have) {
                const SampleOut o = eval_sample<N, PREC, MAPK, REG>(
                        R, S.grid, w_grid, (uint32_t)s, t, w_sid, k0, k1, nullptr,
                        !compact ? kClassUnknown : (use_near ? kClassNear : kClassFar), spin);
                if constexpr (GRP) {
                    // the sample's slot belongs to the thread that owns it in the chunk layout (sample
                    // first + js * blockDim + own), whichever warp evaluates it; each slot gets one add per member
                    const uint32_t off = (uint32_t)(s - first);
                    const int js = (int)(off / blockDim.x), own = (int)(off - (uint32_t)js * blockDim.x);
                    S.gacc[js * PER][own] += o.w;
                    if constexpr (REG) {
#pragma unroll
                        for (int c = 0; c < kComp; ++c) S.gacc[js * PER + 1 + c][own] += o.wc[c];
                    }
                } else {
                    if (nonzero(o.w)) {          // a zero weight leaves both sums unchanged: no FP64 work
                        sw += o.w;
                        sw2 = fma(o.w, o.w, sw2);
                        hist_add<D>(hist, hist_block, layout, nb, o.binpack, o.w);
                    }
                    if constexpr (REG) {
#pragma unroll
                        for (int c = 0; c < kComp; ++c) {
                            S.cacc[2 * c][threadIdx.x] += o.wc[c];
                            S.cacc[2 * c + 1][threadIdx.x] = fma(o.wc[c], o.wc[c], S.cacc[2 * c + 1][threadIdx.x]);
                        }
                    }
                }
            }
        }
    }
    if constexpr (!GRP) return;
    __syncthreads();                           // slots were filled by the block's warps
    for (int j = 0; j < w_spt; ++j) {
        const uint64_t s = first + (uint64_t)j * blockDim.x + threadIdx.x;
        if (s >= w_samples) continue;
        const double w = S.gacc[j * PER][threadIdx.x];
        sw += w;
        sw2 = fma(w, w, sw2);
        if constexpr (REG) {
#pragma unroll
            for (int c = 0; c < kComp; ++c) {
                const double v = S.gacc[j * PER + 1 + c][threadIdx.x];
                S.cacc[2 * c][threadIdx.x] += v;
                S.cacc[2 * c + 1][threadIdx.x] = fma(v, v, S.cacc[2 * c + 1][threadIdx.x]);
            }
        }
        if (nonzero(w)) {
            uint32_t bp[kBinWords];
            sample_bins<D>((uint32_t)s, t, w_sid, k0, k1, (uint32_t)nb, bp);
            hist_add<D>(hist, hist_block, layout, nb, bp, w);
        }
    }
}

// Sum over n chunk slots of one histogram entry (col[c * stride]): eight FP32 partial sums
// (independent loads in flight), widened and combined in FP64 in a fixed order.
__device__ __forceinline__ double hist_column_sum(const float* __restrict__ col, size_t stride, uint32_t n) {
    float p[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    uint32_t c = 0;
    for (; c + 8 <= n; c += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) p[u] += col[(size_t)(c + u) * stride];
    }
    for (; c < n; ++c) p[0] += col[(size_t)c * stride];
    return ((widen_f(p[0]) + widen_f(p[1])) + (widen_f(p[2]) + widen_f(p[3]))) +
           ((widen_f(p[4]) + widen_f(p[5])) + (widen_f(p[6]) + widen_f(p[7])));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Persistent kernel: blocks take chunks (a fixed range of one integral's samples) from a global
// counter; each chunk's sum w, sum w^2 and histogram go to the chunk's own slot, so the result of a
// chunk does not depend on which block ran it or what else is in the batch.
// Compiled in several launch shapes (threads per block x minimum resident blocks, i.e. a register cap);
// the autotuner picks one per context.
// The batch is run by kParts kernels, one per part, each carrying only its own instantiations: PART
// bit 0 = the integrals carry the denominator regulator, bit 1 = group integrals, bit 2 = sixth order.
template <int TPB, int PART>
__device__ __forceinline__ void k_iterate_body(WorkHeader* hdr, const WorkItem* __restrict__ items,
                                               double* __restrict__ csum, float* __restrict__ chist) {
    constexpr int NW = TPB / 32;
    constexpr int LAYOUT = PART & (kPartReg | kPartGrp);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ChunkSmemT<NW, LAYOUT>& S = *reinterpret_cast<ChunkSmemT<NW, LAYOUT>*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr bool REGP = (PART & kPartReg) != 0, GRPP = (PART & kPartGrp) != 0, O6P = (PART & kPartO6) != 0;
    static_assert(NW >= 4, "the FP64 block histogram overlays the FP32 histograms of four warps");
    static_assert((NW & (NW - 1)) == 0 && NW <= 32, "the search for the warp that holds a pooled entry halves the range of warps");
    uint32_t item0 = 0, chunk0 = 0;
#pragma unroll
    for (int p = 0; p < PART; ++p) {
        item0 += hdr->part_items[p];
        chunk0 += hdr->part_chunks[p];
    }
    const uint32_t n_items = hdr->part_items[PART], total = hdr->part_chunks[PART];
    for (;;) {
        if (tid == 0) {
            const uint32_t cl = atomicAdd(&hdr->part_counter[PART], 1u);
            uint32_t it = item0;
            if (cl < total) {
                const uint32_t c = chunk0 + cl;
                uint32_t lo = item0, hi = item0 + n_items;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (items[mid].chunk_begin <= c) lo = mid;
                    else hi = mid;
                }
                it = lo;
                if (c - items[it].chunk_begin >= items[it].n_chunks) atomicOr(&hdr->error, 1u);
                if ((items[it].rec->n_shifts != 0) != REGP || (items[it].n_members > 1) != GRPP ||
                    (items[it].rec->order == 6) != O6P)
                    atomicOr(&hdr->error, 4u);
            }
            S.chunk = (cl < total) ? chunk0 + cl : 0xFFFFFFFFu;
            S.item = it;
            S.skip = (cl < total) ? (uint32_t)items[it].state->converged |
                                        (uint32_t)((items[it].rec->n_shifts != 0) != REGP ||
                                                   (items[it].n_members > 1) != GRPP ||
                                                   (items[it].rec->order == 6) != O6P)
                                  : 1u;
            S.iter = (cl < total) ? (uint32_t)items[it].state->iter : 0u;
        }
        __syncthreads();
        const uint32_t chunk = S.chunk;
        if (chunk == 0xFFFFFFFFu) break;
        if (S.skip) {
            __syncthreads();
            continue;
        }
        const WorkItem& W = items[S.item];
        load_record(&S.rec, W.rec);
        __syncthreads();
        const int d = S.rec.d, nb = S.rec.nb, order = S.rec.order;
        const int prec = effective_precision(S.rec.precision, W.grid, d, nb);
        load_grid(S.grid, W.grid, d, nb, prec);
        for (int i = tid; i < NW * kCells; i += blockDim.x) (&S.hist[0][0])[i] = 0.0f;
        if constexpr (REGP)
            for (int c = 0; c < 2 * kComp; ++c) S.cacc[c][tid] = 0.0;
        if constexpr (GRPP)
            for (int c = 0; c < group_slots(PART); ++c) S.gacc[c][tid] = 0.0;
        __syncthreads();
        double sw = 0.0, sw2 = 0.0;
        const uint32_t cl = chunk - W.chunk_begin;
        const int key = (order * 3 + prec) * 2 + S.rec.map_kind;
#define MBPT_CASE(N_, P_, M_) \
    case (N_ * 3 + P_) * 2 + M_: run_chunk<N_, P_, M_, REGP, GRPP, NW>(S, W, cl, sw, sw2); break;
#define MBPT_CASES(N_) \
    MBPT_CASE(N_, MBPT_FP64, 0) MBPT_CASE(N_, MBPT_MIXED, 0) MBPT_CASE(N_, MBPT_MIXED_MAP64, 0) \
    MBPT_CASE(N_, MBPT_FP64, 1) MBPT_CASE(N_, MBPT_MIXED, 1) MBPT_CASE(N_, MBPT_MIXED_MAP64, 1)
        if constexpr (O6P) {
            switch (key) {
                MBPT_CASES(6)
                default:
                    if (tid == 0) atomicOr(&hdr->error, 2u);
            }
        } else {
            switch (key) {
                MBPT_CASES(2)
                MBPT_CASES(3)
                MBPT_CASES(4)
                MBPT_CASES(5)
                default:
                    if (tid == 0) atomicOr(&hdr->error, 2u);
            }
        }
#undef MBPT_CASES
#undef MBPT_CASE
        sw = warp_sum(sw);
        sw2 = warp_sum(sw2);
        if (lane == 0) {
            S.red[0][warp] = sw;
            S.red[1][warp] = sw2;
        }
        __syncthreads();
        if constexpr (REGP) {
            for (int c = 0; c < 2 * kComp; ++c) {
                const double v = warp_sum(S.cacc[c][tid]);
                if (lane == 0) S.redc[c][warp] = v;
            }
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < NW; ++w) {
                a += S.red[0][w];
                b += S.red[1][w];
            }
            csum[kSumStride * (size_t)chunk] = a;
            csum[kSumStride * (size_t)chunk + 1] = b;
            if constexpr (REGP)
                for (int c = 0; c < 2 * kComp; ++c) {
                    double v = 0.0;
                    for (int w = 0; w < NW; ++w) v += S.redc[c][w];
                    csum[kSumStride * (size_t)chunk + 2 + c] = v;
                }
        }
        float* dst = chist + (size_t)chunk * (size_t)W.hist_stride;
        if (W.hist_layout == kHistBlockF64) {
            const double* h = reinterpret_cast<const double*>(&S.hist[0][0]);
            for (int i = tid; i < d * nb; i += blockDim.x) dst[i] = (float)h[i];
        } else {
            for (int i = tid; i < d * nb; i += blockDim.x) {
                float v = 0.0f;
                for (int w = 0; w < NW; ++w) v += S.hist[w][i];
                dst[i] = v;
            }
        }
        __syncthreads();
    }
}

}  // namespace mbpt
