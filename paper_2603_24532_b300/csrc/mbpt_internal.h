// Internal data layout shared by the host runtime and the device kernels of
// libmbpt (not part of the public ABI).
#pragma once
#include <stdint.h>

#include <vector>

#include "../../include/mbpt.h"

namespace mbpt {

constexpr int kMaxD = 3 * (MBPT_MAX_DEVICE_ORDER + 1);   // 21 dimensions at order 6
constexpr int kMaxTerms = 1 << MBPT_MAX_DEVICE_ORDER;    // 64 spin-sum terms
constexpr int kMaxLoops = MBPT_MAX_DEVICE_ORDER + 1;     // loops of one term: at most n+1
constexpr int kBinWords = (kMaxD + 3) / 4;               // words of a sample's packed bin indices (8 bits per axis)
// Shared-memory grid rows and histograms of one integral hold at most kCells = d x n_bins entries;
// grid row a starts at a * grid_stride(d) (MBPT_MAX_BINS up to d = 18, 54 at d = 21)
constexpr int kCells = MBPT_MAX_GRID_CELLS;
#if defined(__CUDACC__)
#define MBPT_HOST_DEVICE __host__ __device__
#else
#define MBPT_HOST_DEVICE
#endif
MBPT_HOST_DEVICE constexpr int grid_stride(int d) {
    return d * MBPT_MAX_BINS <= kCells ? MBPT_MAX_BINS : kCells / d;
}
static_assert(18 * MBPT_MAX_BINS <= kCells, "orders 2..5 keep MBPT_MAX_BINS bins");
constexpr int kMaxIters = 512;                           // iteration history kept per integral
constexpr int kThreads = 256;                            // threads per block of the iterate kernel
constexpr int kShifts = 3;                               // denominator-regulator components
constexpr int kComp = kShifts + 1;                       // ... plus their extrapolation to zero shift
constexpr int kSumStride = 2 + 2 * kComp;                // doubles per chunk-sum slot
// grouped evaluation: per-thread shared-memory slots holding per-sample sums over the members
// (one per sample; with the regulator, one per sample and component), i.e. samples per thread per chunk
constexpr int kGroupSlotsPlain = 16;
constexpr int kGroupSlotsReg = 15;
constexpr int kWarps = kThreads / 32;
// samples per thread of a chunk by order (index = order) for a fresh context and for the allocation-free
// iteration, which promises the same chunking.  32 at every order: measured on a B300 with 256 x 2 blocks,
// 32 against 16 samples per thread is 12 % faster on 198 fourth-order integrals x 2^24, 8 % on all 2004
// fifth-order integrals x 2^20 and 9 % on 11269 sixth-order integrals x 2^16 (longer chunks leave fewer
// partial warps in the evaluation phases; 64 and more gain little or lose)
constexpr int kDefaultSpt[MBPT_MAX_DEVICE_ORDER + 1] = {0, 0, 32, 32, 32, 32, 32};
// the batch is run by eight k_iterate kernels, one per part: bit 0 = the integrals carry the denominator
// regulator, bit 1 = group integrals, bit 2 = sixth order (its instantiations have their own kernels, so that
// their registers and stack do not weigh on the orders 2..5)
constexpr int kParts = 8;
constexpr int kPartReg = 1, kPartGrp = 2, kPartO6 = 4;
// per-chunk histogram layouts of k_iterate (the autotuner picks one): warp-private FP32 bins, or one
// block-shared FP64 histogram
constexpr int kHistWarpF32 = 0, kHistBlockF64 = 1;

// Compiled, device-resident description of one integral (diagram x physics x VEGAS setup).
//
// Line momenta live in "slots": slots 0..n are the chords (the integration
// variables), slots n+1..2n-1 the remaining (tree) lines in an order in which
// each tree line follows from momentum conservation at one vertex whose other
// three lines are already known:  k[slot] = k[tree_a] + k[tree_b] - k[tree_c].
// All bit masks below are over slots.
struct alignas(16) DiagRec {
    int32_t order, n_lines, n_chords, d;
    int32_t nb, precision, asym, reg_half;      // asym: per-loop species sums; reg_half = r/2
    uint32_t hole_slots;                         // slots holding hole lines
    uint32_t all_slots;                          // (1 << 2n) - 1
    int8_t tree_a[MBPT_MAX_DEVICE_ORDER], tree_b[MBPT_MAX_DEVICE_ORDER], tree_c[MBPT_MAX_DEVICE_ORDER];
    // energy denominators, built cut by cut: D~_m = D~_{m-1} + sum_k sign[m][k] |k_slot[m][k]|^2
    // over the four lines of vertex m in increasing slot order (D~_-1 = 0); D_m = (hbar^2/2m) D~_m
    int8_t cut_slot[MBPT_MAX_DEVICE_ORDER][4];
    int8_t cut_neg[MBPT_MAX_DEVICE_ORDER][4];    // 1: subtract
    // vertex v = <o1 o2|V|i1 i2>: slots of o1, o2, i1, i2
    int8_t port_slot[MBPT_MAX_DEVICE_ORDER][4];
    // P_v = k_o1 - k_o2 and P'_v = k_i1 - k_i2 as chord combinations (coefficients -2..2)
    float vcoef_out[MBPT_MAX_DEVICE_ORDER][8];
    float vcoef_in[MBPT_MAX_DEVICE_ORDER][8];
    // tree line in slot n+1+j as a chord combination (coefficients -1..1), for the FP32 step pre-test
    float tcoef[MBPT_MAX_DEVICE_ORDER][8];
    // spin(-isospin) sum, term t: bit v of t set = vertex v taken in exchange
    double gcoef_d[kMaxTerms];                   // (-1)^L(t) g^L(t)   (one Fermi momentum)
    // the same sum with V_e = V_d - Delta at every vertex: term A (bit v set = factor Delta_v, else V_d)
    // carries (-1)^|A| sum over the terms t whose exchange set contains A of gcoef(t)
    float gdel_f[kMaxTerms];
    float gsign_f[kMaxTerms];                    // (-1)^L(t)           (per-loop species sums)
    int8_t nloops[kMaxTerms];
    uint16_t loop_mask[kMaxTerms][kMaxLoops];    // slots of each loop (2n <= 12 bits)
    // chord sampling: radial range [lo, lo + rng]
    double chord_lo[8], chord_rng[8];
    float chord_lo_f[8], chord_rng_f[8];
    // physics
    double kf2_n, kf2_p;                         // squared Fermi momenta (0 = species absent)
    double CS, CY4, mpi2_4;                      // with P = 2p: V = [C_S + 4C_Y/(|P-P'|^2 + 4m_pi^2)] F
    double regc;                                 // (|P|^2 regc)^reg_half = (p/Lambda)^r
    double pref;                                 // all constant factors of the weight
    float pref_mf;                               // |pref| = pref_mf 2^pref_e, pref_mf in [1, 2) (rounded to FP32)
    int32_t pref_e;
    uint32_t pref_sign_hi;                       // sign bit of pref in the high word of a double
    float near_f;                                // MBPT_MIXED: FP64-map band around a Fermi surface (units of kF^2)
    float CSf, CY4f, mpi2_4f, regc2f;            // FP32 copies; regc2f folds in log2(e)^(1/reg_half)
    int8_t line_slot[MBPT_MAX_LINES];            // slot of each descriptor line
    int32_t map_kind;                            // 0: full chord directions; 1: rotational reduction
    int32_t n_shifts;                            // 0 or kShifts
    float kf2_nf, kf2_pf;                        // FP32 copies of kf2_n, kf2_p (Fermi-step pre-test)
    int32_t spectrum;                            // 0 free, 1 Hartree-Fock (table below)
    float hf_hinv_f;                             // 1 / knot spacing, FP32
    const double* hf_tab;                        // per interval i: k_i and the cubic's a, b, c, d (D~ units)
    const float* hf_tab_f;                       // the same in FP32 (mixed precision)
    int32_t hf_n;                                // intervals (knots - 1)
    int32_t pad_h;
    int32_t pad_s;
    double eta[kShifts];                         // shifts in units of hbar^2/2m (D~ units)
    double lag[kShifts];                         // Lagrange weights of the quadratic at zero shift
};

// Per-integral running state (device).
struct alignas(16) DiagState {
    double sum_inv_var;     // sum over iterations with non-zero variance of 1/sigma_t^2
    double sum_mean_w;      // ... of I_t/sigma_t^2
    double last_mean, last_var;
    double mean, sigma, chi2;
    int64_t n_evals;
    int32_t iter;           // iterations done; Philox counter word 1 of the next iteration
    int32_t converged;
    int32_t status;
    int32_t n_used;         // iterations entering the weighted mean
    double hist_mean[kMaxIters];
    double hist_var[kMaxIters];
    // regulator components (shift 0..2, extrapolation): running inverse-variance sums and estimates
    double comp_inv_var[kComp], comp_mean_w[kComp], comp_mean[kComp], comp_sigma[kComp];
    // evaluation phase of MBPT_COMBINE_POOLED: sum w, sum w^2 and samples over the evaluation iterations
    double pool_s1, pool_s2, pool_n;
    double comp_pool_s1[kComp], comp_pool_s2[kComp];
    double pad_pool;
};
// the Python binding reads state images at fixed offsets (mbpt.py: STATE_HEADER_BYTES, DIAGSTATE_BYTES)
static_assert(sizeof(DiagState) == 8496, "DiagState layout changed: update the binding's offsets");

// One entry of the batch work table.
struct alignas(16) WorkItem {
    const DiagRec* rec;
    DiagState* state;
    double* grid;          // d rows of nb+1 edges
    uint64_t samples;      // per iteration
    uint64_t seed;
    uint32_t stream_id;
    uint32_t chunk_begin;  // first global chunk of this integral
    uint32_t n_chunks;
    uint32_t freeze_after;
    double alpha, target_rel, target_abs;
    int32_t spt;           // samples per thread per chunk
    int32_t hist_stride;   // floats per chunk histogram slot
    uint32_t train_iters;  // leading iterations not combined into the estimate
    uint32_t n_members;    // records at rec[0..n_members): > 1 is a group integral (sum of the members)
    uint32_t combine;      // MBPT_COMBINE_INVVAR or MBPT_COMBINE_POOLED
    uint32_t hist_layout;  // kHistWarpF32 or kHistBlockF64
    uint32_t spin_sum;     // MBPT_SPIN_TABLE or MBPT_SPIN_FOLD
    uint32_t pad_w;
};

struct alignas(16) WorkHeader {
    uint32_t n_items;         // all items of the batch (k_finalize)
    uint32_t total_chunks;
    uint32_t error;           // non-zero: a kernel saw an out-of-range index or a misplaced item
    uint32_t pad0;
    uint64_t hist_floats;     // size of the chunk histogram scratch
    // the batch is split in kParts parts, each run by its own k_iterate kernel, in part order (bits as for
    // kParts); part p holds part_items[p] consecutive items and part_chunks[p] consecutive chunks
    uint32_t part_items[kParts];
    uint32_t part_chunks[kParts];
    uint32_t part_counter[kParts];   // dynamic chunk scheduling, reset before every iterate launch
};

// host-side helpers (mbpt_host.cpp)
int compile_record(const mbpt_diagram_desc& desc, const mbpt_physics& ph, const mbpt_vegas_cfg& cfg,
                   DiagRec* rec, char* err, size_t errlen);
int validate_descriptor(const mbpt_diagram_desc& desc, char* err, size_t errlen);
// reorder a descriptor's chords hole chords first (stable), permuting the columns of line_coef alike
void hole_chords_first(mbpt_diagram_desc& desc);
// the weight's constant factor and its FP32 mantissa / exponent / sign fields
void set_pref(DiagRec* rec, double pref);
int build_hf_table(const mbpt_physics& ph, std::vector<double>& tab, char* err, size_t errlen);
double hf_eval(const std::vector<double>& tab, double hinv, double k);

}  // namespace mbpt
