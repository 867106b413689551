// Non-templated kernels of libmbpt: finalize (reduction, combination, refinement), sample dump
// and Philox test hooks.
#include "mbpt_kernels.cuh"
#include "mbpt_kernels.h"

namespace mbpt {

// Grid refinement of one axis (Lepage 1978 with (7,1)/8 and (1,6,1)/8 smoothing):
// dbar -> r = dbar/sum -> m = ((r-1)/ln r)^alpha -> new edges at equal shares of the
// piecewise-linear cumulative of m.
// Grid refinement (Lepage 1978), split so that the per-bin work runs on the whole block:
//  refine_weights (thread per bin): smoothing (7,1)/8, (1,6,1)/8, (1,7)/8 of the bin's w^2 sums, then,
//   once the axis total is known, the compressed importance m = ((r - 1)/ln r)^alpha of r = smoothed/total;
//  refine_rebin (thread per axis): new edges that give every bin an equal share of sum m, by linear
//   interpolation inside the old bins.  Totals are summed in bin order, as a sequential refinement would.
__device__ __forceinline__ double refine_smooth(const double* h, int i, int nb) {
    if (i == 0) return (7.0 * h[0] + h[1]) / 8.0;
    if (i == nb - 1) return (h[nb - 2] + 7.0 * h[nb - 1]) / 8.0;
    return (h[i - 1] + 6.0 * h[i] + h[i + 1]) / 8.0;
}

__device__ __forceinline__ double refine_importance(double smoothed, double tot, double alpha) {
    const double r = smoothed / tot;
    if (r <= 0.0) return 0.0;
    if (r >= 1.0) return 1.0;
    return pow((r - 1.0) / log(r), alpha);
}

__device__ void refine_rebin(double* grid, const double* old, const double* m, int nb) {
    double msum = 0.0;
    for (int i = 0; i < nb; ++i) msum += m[i];
    const double share = msum / nb;
    int j = 0;
    double cum = 0.0;
    for (int k = 1; k < nb; ++k) {
        const double target = k * share;
        while (j < nb - 1 && cum + m[j] < target) {
            cum += m[j];
            ++j;
        }
        double frac = m[j] > 0.0 ? (target - cum) / m[j] : 0.0;
        if (frac > 1.0) frac = 1.0;
        if (frac < 0.0) frac = 0.0;
        grid[k] = old[j] + frac * (old[j + 1] - old[j]);
    }
    grid[0] = old[0];
    grid[nb] = old[nb];
}

// Per integral: fixed-order reduction of the chunk slots, combination of the iteration into the
// running estimate (inverse-variance weights, or with MBPT_COMBINE_POOLED the pooled sums of the
// evaluation phase on the frozen grid), convergence test and grid refinement.
__global__ void __launch_bounds__(256) k_finalize(WorkHeader* hdr, const WorkItem* __restrict__ items,
                                                 const double* __restrict__ csum, const float* __restrict__ chist,
                                                 double* const* __restrict__ last_hist) {
    __shared__ double hsum[kCells];
    __shared__ double tmp[kCells];
    __shared__ double old[kCells + kMaxD];
    __shared__ double red[2][8];
    __shared__ double redq[2 * kComp][8];
    __shared__ double axis_tot[kMaxD];
    __shared__ int s_skip, s_refine;
    const int tid = threadIdx.x;
    for (uint32_t ii = blockIdx.x; ii < hdr->n_items; ii += gridDim.x) {
        const WorkItem& W = items[ii];
        DiagState* st = W.state;
        if (tid == 0) s_skip = st->converged;
        __syncthreads();
        if (s_skip) {
            __syncthreads();
            continue;
        }
        double a = 0.0, b = 0.0;
        for (uint32_t c = tid; c < W.n_chunks; c += blockDim.x) {
            a += csum[kSumStride * (size_t)(W.chunk_begin + c)];
            b += csum[kSumStride * (size_t)(W.chunk_begin + c) + 1];
        }
        const int nsh = W.rec->n_shifts;
        if (nsh) {
            for (int q = 0; q < 2 * kComp; ++q) {
                double v = 0.0;
                for (uint32_t c = tid; c < W.n_chunks; c += blockDim.x)
                    v += csum[kSumStride * (size_t)(W.chunk_begin + c) + 2 + q];
                v = warp_sum(v);
                if ((tid & 31) == 0) redq[q][tid >> 5] = v;
            }
        }
        a = warp_sum(a);
        b = warp_sum(b);
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = a;
            red[1][tid >> 5] = b;
        }
        const int d = W.rec->d, nb = W.rec->nb;
        for (int i = tid; i < d * nb; i += blockDim.x) {
            const double acc = hist_column_sum(chist + (size_t)W.chunk_begin * (size_t)W.hist_stride + i,
                                               (size_t)W.hist_stride, W.n_chunks);
            hsum[i] = acc;
            last_hist[ii][i] = acc;
        }
        for (int i = tid; i < d * (nb + 1); i += blockDim.x) old[i] = W.grid[i];
        __syncthreads();
        if (tid == 0) {
            double A = 0.0, B = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                A += red[0][w];
                B += red[1][w];
            }
            const double M = (double)W.samples;
            const double I = A / M;
            const double var = (B / M - I * I) / (M - 1.0);
            const int t = st->iter;
            if (t < kMaxIters) {
                st->hist_mean[t] = I;
                st->hist_var[t] = var;
            }
            st->last_mean = I;
            st->last_var = var;
            if (!isfinite(I) || !isfinite(var)) st->status = MBPT_ENUMERIC;
            const bool training = (uint32_t)t < W.train_iters;   // grid training only
            const bool pooled = W.combine == MBPT_COMBINE_POOLED;
            double mean, sigma, chi2 = 0.0;
            if (pooled) {
                // evaluation phase: every sample of every evaluation iteration carries the same weight
                if (!training) {
                    st->pool_s1 += A;
                    st->pool_s2 += B;
                    st->pool_n += M;
                    st->n_used += 1;
                }
                if (st->pool_n > 1.0) {
                    const double N = st->pool_n;
                    mean = st->pool_s1 / N;
                    const double v = (st->pool_s2 / N - mean * mean) / (N - 1.0);
                    sigma = v > 0.0 ? sqrt(v) : 0.0;
                    const int T = t + 1 < kMaxIters ? t + 1 : kMaxIters;
                    if (st->n_used > 1) {
                        double c2 = 0.0;
                        for (int k = (int)W.train_iters; k < T; ++k)
                            if (st->hist_var[k] > 0.0) {
                                const double dd = st->hist_mean[k] - mean;
                                c2 += dd * dd / st->hist_var[k];
                            }
                        chi2 = c2 / (st->n_used - 1);
                    }
                } else {
                    mean = I;                    // no evaluation iteration yet
                    sigma = (double)INFINITY;
                }
            } else {
                if (var > 0.0 && !training) {
                    st->sum_inv_var += 1.0 / var;
                    st->sum_mean_w += I / var;
                    st->n_used += 1;
                }
                if (st->sum_inv_var > 0.0) {
                    mean = st->sum_mean_w / st->sum_inv_var;
                    sigma = sqrt(1.0 / st->sum_inv_var);
                    const int T = t + 1 < kMaxIters ? t + 1 : kMaxIters;
                    if (st->n_used > 1) {
                        double c2 = 0.0;
                        for (int k = (int)W.train_iters; k < T; ++k)
                            if (st->hist_var[k] > 0.0) {
                                const double dd = st->hist_mean[k] - mean;
                                c2 += dd * dd / st->hist_var[k];
                            }
                        chi2 = c2 / (st->n_used - 1);
                    }
                } else if (training) {
                    mean = I;                    // no combined estimate yet
                    sigma = (double)INFINITY;
                } else {
                    mean = I;
                    sigma = 0.0;
                }
            }
            st->mean = mean;
            st->sigma = sigma;
            st->chi2 = chi2;
            if (nsh) {
                // regulator components: same combination as the main estimate
                for (int q = 0; q < kComp; ++q) {
                    double Aq = 0.0, Bq = 0.0;
                    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                        Aq += redq[2 * q][w];
                        Bq += redq[2 * q + 1][w];
                    }
                    const double Iq = Aq / M;
                    const double vq = (Bq / M - Iq * Iq) / (M - 1.0);
                    if (pooled) {
                        if (!training) {
                            st->comp_pool_s1[q] += Aq;
                            st->comp_pool_s2[q] += Bq;
                        }
                        if (st->pool_n > 1.0) {
                            const double N = st->pool_n, mq = st->comp_pool_s1[q] / N;
                            const double v = (st->comp_pool_s2[q] / N - mq * mq) / (N - 1.0);
                            st->comp_mean[q] = mq;
                            st->comp_sigma[q] = v > 0.0 ? sqrt(v) : 0.0;
                        } else {
                            st->comp_mean[q] = Iq;
                            st->comp_sigma[q] = (double)INFINITY;
                        }
                        continue;
                    }
                    if (vq > 0.0 && !training) {
                        st->comp_inv_var[q] += 1.0 / vq;
                        st->comp_mean_w[q] += Iq / vq;
                    }
                    if (st->comp_inv_var[q] > 0.0) {
                        st->comp_mean[q] = st->comp_mean_w[q] / st->comp_inv_var[q];
                        st->comp_sigma[q] = sqrt(1.0 / st->comp_inv_var[q]);
                    } else {
                        st->comp_mean[q] = Iq;
                        st->comp_sigma[q] = training ? (double)INFINITY : 0.0;
                    }
                }
            }
            st->n_evals += (int64_t)W.samples;
            st->iter = t + 1;
            const bool has_target = (W.target_rel > 0.0) || (W.target_abs > 0.0);
            const double goal = fmax(W.target_rel * fabs(mean), W.target_abs);
            if (has_target && (uint32_t)st->iter >= W.train_iters + 2u && sigma <= goal) st->converged = 1;
            // the grid is refined after every iteration until freeze_after iterations have run; in the
            // pooled combination it is frozen once the training iterations are done
            s_refine = ((W.freeze_after == 0u) || ((uint32_t)st->iter < W.freeze_after)) &&
                       (!pooled || (uint32_t)st->iter <= W.train_iters);
        }
        __syncthreads();
        if (s_refine) {
            for (int idx = tid; idx < d * nb; idx += blockDim.x) {
                const int a = idx / nb, i = idx - a * nb;
                tmp[idx] = refine_smooth(hsum + a * nb, i, nb);
            }
            __syncthreads();
            if (tid < d) {
                double tot = 0.0;
                for (int i = 0; i < nb; ++i) tot += tmp[tid * nb + i];
                axis_tot[tid] = tot;
            }
            __syncthreads();
            for (int idx = tid; idx < d * nb; idx += blockDim.x) {
                const int a = idx / nb;
                if (axis_tot[a] > 0.0) tmp[idx] = refine_importance(tmp[idx], axis_tot[a], W.alpha);
            }
            __syncthreads();
            // an axis without weight keeps its grid
            if (tid < d && axis_tot[tid] > 0.0)
                refine_rebin(W.grid + tid * (nb + 1), old + tid * (nb + 1), tmp + tid * nb, nb);
        }
        __syncthreads();
    }
}

// Test hook kernel: samples [first, first+count) of iteration `iter`, mapped point and weight (the spin sum
// with the context's Goldstone-sum strategy, as k_iterate evaluates it).
template <int N, int PREC, int MAPK>
__device__ void dump_one(const DiagRec& R, const Grid2* gs, const double* grid64, uint32_t s, uint32_t t,
                         uint32_t sid, uint32_t k0, uint32_t k1, uint32_t spin, double* x, double* w) {
    const SampleOut o = eval_sample<N, PREC, MAPK, false>(R, gs, grid64, s, t, sid, k0, k1, x, kClassUnknown, spin);
    *w = o.w;
}

__global__ void __launch_bounds__(256) k_dump(const DiagRec* rec, int n_members, const double* grid, uint64_t seed,
                                             uint32_t sid, uint32_t iter, uint64_t first, uint64_t count,
                                             uint32_t spin, double* xo, double* wo) {
    __shared__ DiagRec R;
    __shared__ Grid2 gs[kCells];
    load_record(&R, rec);
    __syncthreads();
    const int prec = effective_precision(R.precision, grid, R.d, R.nb);
    load_grid(gs, grid, R.d, R.nb, prec);
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < count;
    const uint32_t s = (uint32_t)(first + i);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    double* x = (xo && active) ? xo + i * R.d : nullptr;
    double acc = 0.0;
    // a group integral: the sum of its members' weights at the same point
    for (int m = 0; m < n_members; ++m) {
        if (m > 0) load_record(&R, rec + m);
        __syncthreads();
        double w = 0.0;
        if (active) {
            switch ((R.order * 3 + prec) * 2 + R.map_kind) {
#define MBPT_CASE(N_, P_, M_) \
    case (N_ * 3 + P_) * 2 + M_: dump_one<N_, P_, M_>(R, gs, grid, s, iter, sid, k0, k1, spin, m == 0 ? x : nullptr, &w); break;
#define MBPT_CASES(N_) \
    MBPT_CASE(N_, MBPT_FP64, 0) MBPT_CASE(N_, MBPT_MIXED, 0) MBPT_CASE(N_, MBPT_MIXED_MAP64, 0) \
    MBPT_CASE(N_, MBPT_FP64, 1) MBPT_CASE(N_, MBPT_MIXED, 1) MBPT_CASE(N_, MBPT_MIXED_MAP64, 1)
                MBPT_CASES(2)
                MBPT_CASES(3)
                MBPT_CASES(4)
                MBPT_CASES(5)
                MBPT_CASES(6)
#undef MBPT_CASES
#undef MBPT_CASE
                default: w = 0.0;
            }
        }
        acc = (m == 0) ? w : acc + w;
        __syncthreads();
    }
    if (active) wo[i] = acc;
}

// FP64 throughput probe for the roofline denominator: every thread runs eight independent chains
// a <- a * b + c (no dependency between consecutive DFMAs of one chain's neighbours), so the FP64 pipe, not
// latency, bounds the loop.  The sink store never happens (the chains stay positive) but keeps the loop.
__device__ double g_dfma_sink;

// One 16-byte word per thread: word w of the state of integral s, at out[s * words + w].
__global__ void __launch_bounds__(256) k_gather_heads(const DiagState* const* src, int k, int words, uint4* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k * words) return;
    const int s = i / words, w = i - s * words;
    out[i] = reinterpret_cast<const uint4*>(src[s])[w];
}

__global__ void __launch_bounds__(256) k_dfma_rate(int iters) {
    const double b = 0.9999999, c = 1.0e-7;
    double a0 = 1.0 + 1e-9 * threadIdx.x, a1 = a0 + 0.1, a2 = a0 + 0.2, a3 = a0 + 0.3;
    double a4 = a0 + 0.4, a5 = a0 + 0.5, a6 = a0 + 0.6, a7 = a0 + 0.7;
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, b, c);
        a1 = fma(a1, b, c);
        a2 = fma(a2, b, c);
        a3 = fma(a3, b, c);
        a4 = fma(a4, b, c);
        a5 = fma(a5, b, c);
        a6 = fma(a6, b, c);
        a7 = fma(a7, b, c);
    }
    const double s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s < 0.0) g_dfma_sink = s;
}

__global__ void k_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                         uint64_t count, uint32_t* out) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    uint32_t o[4];
    philox4x32_10(c0 + (uint32_t)i, c1, c2, c3, k0, k1, o);
    for (int j = 0; j < 4; ++j) out[4 * i + j] = o[j];
}

}  // namespace mbpt
