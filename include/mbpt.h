/*
 * mbpt.h -- C ABI of the B300 (sm_103a) Monte Carlo evaluator of
 * zero-temperature Hugenholtz diagrams for the energy per particle of infinite
 * nucleon matter (arXiv:2603.24532, "Many-body perturbation theory for the
 * nuclear equation of state up to fifth order").
 *
 * What the library computes (Sec. II, Eqs. (2)-(6); Sec. III.C):
 *   for a diagram G of order n (n = 2..6 vertices, 2n lines, n+1 loop momenta)
 *   and a physics point (Fermi momenta kF_n, kF_p, potential V(p,p')),
 *     E_G/N = (1/n_dens) (-1)^(h+l0) 2^(-n_eq)
 *             sum_{spins, isospins} int prod_c d^3l_c/(2pi)^3
 *             prod_lines Theta_l  prod_vertices <o1 o2|V|i1 i2>  / prod_cuts D_m
 *   with Theta_l = n_k (holes) or 1 - n_k (particles), n_k = theta(kF - k),
 *   D_m = sum_{holes in cut m} eps - sum_{particles in cut m} eps,
 *   eps(k) = (hbar^2/2m) k^2 (free spectrum), estimated by VEGAS importance
 *   sampling (Lepage) with Philox4x32-10 random numbers.
 *
 * Conventions for every call:
 *   - Every function returns an mbpt_status; nothing throws across the ABI.
 *     Out-parameters are written only when MBPT_OK is returned.  On error,
 *     mbpt_last_error() returns a message for the calling thread.
 *   - Input structs are owned by the caller and copied during the call.
 *   - Device memory is owned by the context: it either lives in a caller
 *     supplied device arena (mbpt_ctx_create with arena != NULL, e.g. a
 *     torch-allocated buffer) or in one cudaMalloc'ed arena of the requested
 *     size that mbpt_ctx_destroy frees.  Per-integral state is carved out of
 *     that arena; when it is full, creation fails with MBPT_ENOMEM.
 *   - A context is bound to one device and one CUDA stream and is not
 *     thread-safe: one host thread drives it.  Work is queued asynchronously
 *     on the context stream; mbpt_estimate / mbpt_get_state synchronise it.
 *   - Units: momenta fm^-1, energies MeV, hbar^2/m MeV fm^2, C_S MeV fm^3,
 *     C_Y MeV fm.  Results are contributions to E/N in MeV.
 */
#ifndef MBPT_H
#define MBPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mbpt_ctx mbpt_ctx;     /* opaque: device, stream, arena, graphs */
typedef struct mbpt_diag mbpt_diag;   /* opaque: one integral = diagram x physics point */

typedef enum {
    MBPT_OK = 0,
    MBPT_EINVAL = -1,     /* invalid argument or descriptor */
    MBPT_ENOMEM = -2,     /* arena or host allocation exhausted */
    MBPT_ECUDA = -3,      /* a CUDA runtime call failed (message has the CUDA error) */
    MBPT_EDEVICE = -4,    /* a kernel reported an out-of-range index in its error word */
    MBPT_ETIMEOUT = -5,   /* a bounded device wait gave up */
    MBPT_ENUMERIC = -6,   /* NaN or Inf in an integral's accumulators */
    MBPT_EBUSY = -7       /* operation not allowed while work is queued */
} mbpt_status;

typedef enum {
    MBPT_FP64 = 0,        /* every step in FP64 */
    MBPT_MIXED = 1,       /* potential matrix elements (exp, Yukawa), their products
                             and the spin sum in FP32; the sampling map (VEGAS map,
                             chord magnitudes and directions, Jacobians) in FP32,
                             placing each chord momentum at an exact FP64 point;
                             line momenta, Fermi steps, energy denominators,
                             weights, sums and the grid update in FP64 */
    MBPT_MIXED_MAP64 = 2  /* as MBPT_MIXED but with the sampling map in FP64 */
} mbpt_precision;

#define MBPT_MAX_ORDER 6          /* generator */
#define MBPT_MAX_DEVICE_ORDER 6   /* the device path runs 2..6 (Table I's sixth order: d = 21) */
#define MBPT_MAX_LINES 12
#define MBPT_MAX_CHORDS 7
#define MBPT_MAX_BINS 64
#define MBPT_MAX_GRID_CELLS 1152  /* d x n_bins of one integral (grid and histograms stay in shared
                                     memory): at most 64 bins up to d = 18, 54 at d = 21 */
#define MBPT_MAX_GROUP 1024       /* members of one group integral */
#define MBPT_HF_KNOTS 1024        /* knots of the Hartree-Fock self-energy table */
#define MBPT_HF_QUAD 64           /* Gauss-Legendre nodes per dimension of each knot's integral */

/* descriptor flags */
#define MBPT_FLAG_ANOMALOUS   1   /* a hole and a particle forced to equal momentum: zero at T = 0 */
#define MBPT_FLAG_SELF_MIRROR 2   /* equal to its own time-and-arrow reversal */
#define MBPT_FLAG_REPEATED_DENOMINATOR 4   /* two cuts with the same energy denominator (a 1/D^2 factor) */

/*
 * One Hugenholtz diagram with two-body vertices (Sec. II, Table I).
 * Vertices 0..order-1 are in time order (0 = earliest).  Line l runs from
 * vertex line_src[l] to line_dst[l]; line_src < line_dst is a particle line,
 * line_src > line_dst a hole line.  Vertex v stands for the antisymmetrised
 * matrix element <vtx_out[v][0] vtx_out[v][1]|V|vtx_in[v][0] vtx_in[v][1]>
 * (lines leaving v on the left, lines entering v on the right).  The n+1
 * chords are lines whose momenta are the integration variables; every line
 * momentum is k_l = sum_c line_coef[l][c] * k_chord(c), coefficients in
 * {-1,0,1}.  The sign (-1)^(h+l0), the weight 2^(-n_eq), the energy-
 * denominator cuts and the spin-sum table are derived from this description
 * by the library; line_coef is checked against momentum conservation.
 */
typedef struct {
    int32_t order;
    int32_t n_lines;
    int8_t line_src[MBPT_MAX_LINES];
    int8_t line_dst[MBPT_MAX_LINES];
    int8_t vtx_out[MBPT_MAX_ORDER][2];
    int8_t vtx_in[MBPT_MAX_ORDER][2];
    int8_t n_chords;
    int8_t chord_line[MBPT_MAX_CHORDS];
    int8_t line_coef[MBPT_MAX_LINES][MBPT_MAX_CHORDS];
    int32_t diagram_id;      /* position in mbpt_generate's order */
    int32_t mirror_id;       /* diagram_id of the time-and-arrow-reversed partner */
    int32_t flags;           /* MBPT_FLAG_* */
} mbpt_diagram_desc;

/*
 * Physics point.  V(p, p') = [C_S + C_Y/(|p - p'|^2 + m_pi^2)] exp(-(p/Lambda)^r - (p'/Lambda)^r)
 * with r = reg_power (nonlocal regulator of Sec. III.B); p, p' are half the
 * relative momenta of the outgoing and incoming pairs of a vertex.
 * A species with kF = 0 is absent: pure neutron matter has kF_p = 0,
 * symmetric matter kF_n = kF_p.  Hole chords are sampled in [0, max kF],
 * particle chords in [smallest present kF, K_max].
 * map_kind 0: every chord momentum from (k, cos theta, phi), rational azimuth;
 * d = 3(order+1) dimensions.  map_kind 1: rotational invariance of the
 * integrand (Sec. III.C, "N_dim - 3"): chord 0 along z (k only), chord 1 in the
 * xz plane (k, cos theta), the fixed angles integrated analytically (4 pi 2 pi);
 * d = 3 order.
 * spectrum 0: free single-particle energies eps(k) = (hbar^2/2m) k^2.  spectrum 1:
 * Hartree-Fock energies eps(k) = (hbar^2/2m) k^2 + Sigma(k) (Eq. (7)), with
 *   Sigma(k) = (2 pi)^-3 int_{k' < kF} d^3k' [g V(p, p) - V(p, -p)],  p = (k - k')/2,
 * g = 2 (neutron matter) or 4 (symmetric matter), tabulated once per integral at
 * 1024 knots k_i = i h, h = 2 K_max / 1023, each by a 64 x 64-point Gauss-Legendre
 * rule over (|k'|, cos angle), and interpolated by the cubic spline with zero slope
 * at k = 0 and zero curvature at the last knot; Sigma = 0 beyond the last knot
 * (the sampling-time interpolation of the paper, Sec. II).  The Hartree-Fock
 * spectrum needs one Fermi momentum (kF_n = kF_p or kF_p = 0) and a spectrum that
 * increases with k (MBPT_EINVAL otherwise).
 */
typedef struct {
    double kF_n, kF_p;
    double hbar2_over_m;
    double C_S, C_Y, m_pi, Lambda;
    int32_t reg_power;       /* even, 2..8 */
    int32_t map_kind;        /* 0 or 1 */
    double K_max;
    int32_t spectrum;        /* 0 free, 1 Hartree-Fock */
    int32_t reserved;        /* 0 */
} mbpt_physics;

/*
 * VEGAS settings of one integral (Lepage 1978; Sec. III.C).  Sample s of the
 * integral's iteration t uses Philox4x32-10 with key (seed low word, seed high
 * word) and counter (s, t, stream_id, j), j = 0..ceil(d/4)-1; axis a takes word
 * a.  The grid is refined after every iteration (smoothing (7,1)/8 and
 * (1,6,1)/8, compression exponent alpha) until `freeze_after` iterations have
 * run (0 = never freeze).  The first `train_iters` iterations only train the
 * grid: their estimates are recorded but not combined (PVegas' training phase,
 * Sec. III.C).  The integral stops iterating once its combined standard error
 * is <= max(target_rel*|mean|, target_abs) (0, 0 = never).
 *
 * Combination of the iterations (`combine`):
 *   MBPT_COMBINE_INVVAR (0): Lepage's inverse-variance weighted mean of the iteration estimates
 *     from iteration train_iters on, sigma = (sum 1/sigma_t^2)^(-1/2).  With heavy-tailed weights
 *     the iterations that missed the tail have both the smaller |I_t| and the smaller sigma_t, so
 *     this mean is biased toward them and its sigma is too small.
 *   MBPT_COMBINE_POOLED (1): PVegas' split into a training and an evaluation phase (Sec. III.C).
 *     The first train_iters iterations train the grid (refined after each) and are not combined;
 *     from then on the grid is frozen and every evaluation sample carries the same weight: with
 *     S1 = sum w, S2 = sum w^2 and N samples over all evaluation iterations, mean = S1/N and
 *     sigma^2 = (S2/N - mean^2)/(N - 1), the plain Monte Carlo estimator of one long run on one
 *     grid (unbiased whatever the tails).  chi2_dof compares the evaluation iterations' own
 *     estimates with that mean.  freeze_after, if set, can only freeze earlier.
 *
 * Denominator regulator (Sec. III.A): with n_shifts = 3 every sample also
 * evaluates the integrand with each energy denominator D_m replaced by
 * D_m - shift[k] (D_m < 0 on the integration domain, so the shift moves the
 * pole away), and the quadratic through the three components extrapolated to
 * zero shift, sum_k L_k w_k with the Lagrange weights L_k of the three shifts;
 * all four are accumulated and combined like the main estimate (the grid still
 * adapts to the unshifted integrand).  Read them with mbpt_estimate_shifts.
 */
typedef struct {
    int32_t n_bins;            /* 2..MBPT_MAX_BINS and d x n_bins <= MBPT_MAX_GRID_CELLS (50 in the
                                  paper's setup) */
    int32_t precision;         /* mbpt_precision */
    double alpha;              /* grid compression exponent, 1.5 */
    uint64_t seed;
    uint32_t stream_id;        /* identifies the integral's random stream */
    uint32_t freeze_after;
    uint64_t samples_per_iter; /* >= 2, < 2^32 */
    double target_rel;
    double target_abs;
    uint32_t train_iters;      /* leading iterations excluded from the combined estimate */
    uint32_t n_shifts;         /* 0, or 3: denominator regulator components (below) */
    double shift[3];           /* MeV, positive and distinct */
    uint32_t combine;          /* MBPT_COMBINE_INVVAR or MBPT_COMBINE_POOLED (above) */
    float near_band;           /* MBPT_MIXED: width of the band around each Fermi surface, in units of
                                  kF^2, inside which a sample is placed with the FP64 map (the FP64
                                  mode's point) instead of the FP32 map; 0 = the library default
                                  (2^-10 up to fourth order, 2^-7 from fifth order on), else in
                                  [2^-16, 1/2] */
} mbpt_vegas_cfg;

#define MBPT_COMBINE_INVVAR 0
#define MBPT_COMBINE_POOLED 1

typedef struct {
    double mean;               /* inverse-variance weighted mean over iterations (MeV) */
    double sigma;              /* its standard error */
    double chi2_dof;           /* chi^2 of the iteration estimates per degree of freedom */
    double last_mean;          /* estimate of the last iteration alone */
    double last_sigma;
    int64_t n_iter;            /* iterations combined */
    int64_t n_evals;           /* integrand evaluations so far */
    int32_t converged;         /* 1 once the target error was reached */
    int32_t status;            /* MBPT_OK or MBPT_ENUMERIC */
} mbpt_result;

/* ---- generator (CPU) ------------------------------------------------------ */

/*
 * Enumerate all connected order-n Hugenholtz diagrams with two-body vertices
 * (Table I: 1, 3, 39, 840, 27300 for n = 2..6) in a deterministic order:
 * adjacency matrices A (A[i][j] = lines from vertex i to j; zero diagonal,
 * row and column sums 2) sorted by their row-major entries; lines listed in
 * row-major order of A; ports in increasing line index; chords chosen by a
 * spanning forest that takes particle lines first, then hole lines, and listed
 * hole chords first, then particle chords (each in line order), so that
 * diagrams with equally many hole chords map a sampled point to the same loop
 * momenta (see mbpt_create_group).
 * out may be NULL to query the count.  Returns MBPT_EINVAL for n outside 2..6
 * and MBPT_ENOMEM when cap is too small (*count still receives the count).
 */
int mbpt_generate(int order, mbpt_diagram_desc* out, int cap, int* count);

/*
 * Grouping key of a descriptor (grouped evaluation, Sec. III.A and Table I's N_grp): the number of
 * its loop momenta (chords) that are hole lines, i.e. how many integration momenta lie in the Fermi
 * ball.  Diagrams of one order with equal keys share the integration domain; at orders 2..6 the key
 * takes 1, 2, 4, 5 and 6 distinct values.  MBPT_EINVAL for a NULL argument or bad chord index.
 */
int mbpt_hole_chords(const mbpt_diagram_desc* desc, int* out);

/*
 * The Hartree-Fock self-energy Sigma(k) (MeV) of the physics point's spectrum table (see
 * mbpt_physics, spectrum 1) at n momenta k[i] (fm^-1), evaluated on the host in FP64 from the same
 * per-interval cubic coefficients the device uses.  MBPT_EINVAL for invalid physics or two
 * different Fermi momenta.
 */
int mbpt_hf_self_energy(const mbpt_physics* physics, int n, const double* k, double* sigma);

/* ---- context ------------------------------------------------------------- */

/*
 * Create a context on `device`.  If arena != NULL it must be a device pointer
 * to arena_bytes of memory (256-byte aligned) owned by the caller that stays
 * valid until mbpt_ctx_destroy; otherwise the library cudaMallocs arena_bytes.
 * `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).
 */
int mbpt_ctx_create(mbpt_ctx** ctx, int device, void* arena, size_t arena_bytes, void* cuda_stream);
int mbpt_ctx_destroy(mbpt_ctx* ctx);
/* Bytes of the arena in use and free (largest block) -- for admission control. */
int mbpt_ctx_mem(const mbpt_ctx* ctx, size_t* used, size_t* largest_free);
/* Device bytes one integral with this descriptor and configuration needs (with the Hartree-Fock
 * spectrum, one more block of (MBPT_HF_KNOTS - 1) x 60 bytes for its table). */
int mbpt_diag_bytes(const mbpt_diagram_desc* desc, const mbpt_vegas_cfg* cfg, size_t* bytes);
/* The same for a group integral of k members (mbpt_create_group); the members' order is that of descs[0]. */
int mbpt_group_bytes(const mbpt_diagram_desc* descs, int k, const mbpt_vegas_cfg* cfg, size_t* bytes);

/*
 * Launch shape of mbpt_vegas_iterate.  The sample-evaluation kernel is compiled
 * in a few shapes (threads per block x minimum resident blocks per SM, which
 * caps registers per thread); mbpt_kernel_variants lists them (count first,
 * then up to cap shapes).  mbpt_ctx_set_kernel selects one for a context and
 * mbpt_ctx_set_launch sets the samples per thread of a chunk (1..256) for one
 * order; a chunk is threads x samples_per_thread consecutive samples of one
 * integral.  The autotuner sets these.  Results of an integral depend on its
 * chunking (summation order), not on the rest of the batch.
 */
int mbpt_kernel_variants(int* threads_per_block, int* min_blocks_per_sm, int cap, int* count);
int mbpt_ctx_set_kernel(mbpt_ctx* ctx, int threads_per_block, int min_blocks_per_sm);
int mbpt_ctx_set_launch(mbpt_ctx* ctx, int order, int samples_per_thread);
int mbpt_ctx_get_launch(const mbpt_ctx* ctx, int order, int* threads_per_block, int* min_blocks_per_sm,
                        int* samples_per_thread);
/*
 * Per-chunk histogram layout of the sample-evaluation kernel (an autotuner choice; the context starts with
 * MBPT_HIST_WARP_F32).  MBPT_HIST_WARP_F32: every warp adds w^2 to its own FP32 bins (FP32 shared-memory
 * atomics without contention between warps; results bitwise reproducible).  MBPT_HIST_BLOCK_F64: one FP64
 * histogram per block (FP64 shared-memory atomics from every warp; the order of the additions, and so the
 * last bits of the histogram and of the refined grid, can vary from run to run).  Either way a chunk's
 * histogram is stored in FP32 and the chunks are summed in FP64 in a fixed order.
 */
int mbpt_ctx_set_hist_layout(mbpt_ctx* ctx, int layout);
int mbpt_ctx_get_hist_layout(const mbpt_ctx* ctx, int* layout);
#define MBPT_HIST_WARP_F32 0
#define MBPT_HIST_BLOCK_F64 1

/*
 * Goldstone-sum strategy of the mixed-precision modes in matter with one Fermi momentum (an autotuner
 * choice; the context starts with MBPT_SPIN_TABLE).  The spin(-isospin) sum of Sec. II / App. B is the
 * multilinear polynomial sum_A c'(A) prod_{v in A} Delta_v prod_{v not in A} V_v over the subsets A of the
 * n vertices (V_v the direct matrix element, Delta_v the direct minus the exchange one, c' the
 * difference-form Goldstone table).  MBPT_SPIN_TABLE forms the 2^n vertex products and sums them with the
 * table; MBPT_SPIN_FOLD folds the table vertex by vertex (T(A) <- T(A) V_v + T(A + {v}) Delta_v), the
 * same polynomial with 2^n - 2 fewer FP32 products and fewer live registers.  The two agree to FP32
 * rounding.  FP64 mode and asymmetric matter always use their product tables.
 */
int mbpt_ctx_set_spin_sum(mbpt_ctx* ctx, int strategy);
int mbpt_ctx_get_spin_sum(const mbpt_ctx* ctx, int* strategy);
#define MBPT_SPIN_TABLE 0
#define MBPT_SPIN_FOLD 1

/*
 * Device time of the last mbpt_vegas_iterate iteration: the sample-evaluation
 * launch and the reduce/combine/refine launch, in milliseconds, from CUDA
 * events recorded around them on the context stream.  Synchronises on the
 * last iteration.  MBPT_EINVAL if nothing has run yet.
 */
int mbpt_ctx_last_timing(mbpt_ctx* ctx, double* iterate_ms, double* finalize_ms);
/* The CUDA stream the context queues its work on (its own stream when created with NULL). */
int mbpt_ctx_stream(const mbpt_ctx* ctx, void** cuda_stream);

/* ---- integrals ------------------------------------------------------------ */

/*
 * Validate and compile a descriptor for a physics point into a device-resident
 * integral with a uniform VEGAS grid.  Returns MBPT_EINVAL for an invalid
 * descriptor (ports not matching lines, chords not completing a spanning tree,
 * line_coef violating momentum conservation, order outside 2..6), invalid
 * physics (kF < 0, both kF zero, K_max <= kF, odd reg_power) or configuration
 * (including d x n_bins above MBPT_MAX_GRID_CELLS, i.e. more than 54 bins at order 6),
 * and MBPT_ENOMEM when the arena cannot hold its state.
 */
int mbpt_create_diagram(mbpt_ctx* ctx, const mbpt_diagram_desc* desc, const mbpt_physics* physics,
                        const mbpt_vegas_cfg* cfg, mbpt_diag** out);
/*
 * Grouped evaluation (Sec. III.A): one integral whose integrand is the sum of k diagrams of the same
 * order, member m scaled by scale[m] (NULL: all 1; e.g. 2 for one diagram standing for a mirror
 * pair), evaluated at the same loop momenta: each member's chords are taken hole chords first (the
 * order mbpt_generate lists them in; other descriptors are reordered), so members with equally many
 * hole chords -- the grouping key, mbpt_hole_chords -- map a sampled point x to the same chord
 * momenta.  One VEGAS grid then adapts to the sum, and the members' singular regions and
 * fluctuations coincide and partly cancel.  One physics point and
 * configuration for all members; the result (mbpt_estimate, the regulator components, the state
 * image) is that of the sum.  Each sample costs k integrand evaluations; a chunk holds
 * 16 samples per thread (3 with the regulator).  MBPT_EINVAL for k outside
 * 1..MBPT_MAX_GROUP, mixed orders, a non-finite scale or any member that create_diagram would reject.
 * mbpt_dump_samples of a group returns the summed weight.
 */
int mbpt_create_group(mbpt_ctx* ctx, const mbpt_diagram_desc* descs, int k, const double* scale,
                      const mbpt_physics* physics, const mbpt_vegas_cfg* cfg, mbpt_diag** out);
int mbpt_destroy_diagram(mbpt_diag* diag);
/*
 * Change an integral's samples per iteration, freeze point, training iterations and targets for its
 * next iterations (PVegas' adaptive number of samples per iteration, Sec. III.C).
 * Seed, stream id, bins, alpha and precision must be unchanged (MBPT_EINVAL).
 */
int mbpt_set_config(mbpt_diag* diag, const mbpt_vegas_cfg* cfg);

/*
 * Run n_iters VEGAS iterations on the k integrals as one batch: per
 * iteration one persistent launch evaluates all samples of all integrals not
 * yet converged (Sec. III.C "integrand evaluation distributed ... via CUDA"),
 * then a second launch reduces the per-chunk sums in a fixed order, combines
 * the iteration into each integral's running estimate and refines its grid.
 * The pair is captured once per context in a CUDA graph and replayed.
 * Asynchronous on the context stream.  All diags must belong to ctx.
 */
int mbpt_vegas_iterate(mbpt_ctx* ctx, mbpt_diag* const* diags, int k, int n_iters);

/* Synchronise and read an integral's estimate. */
int mbpt_estimate(const mbpt_diag* diag, mbpt_result* out);
/* The same for k integrals of one context with a single synchronisation; out[i] for diags[i].  A small
 * kernel gathers the integrals' estimates on the device and one copy brings them back (device and pinned
 * host staging held by the context, grown to the largest k); without room for the staging it reads
 * the integrals one copy each instead of failing. */
int mbpt_estimate_batch(mbpt_diag* const* diags, int k, mbpt_result* out);
/* Regulator components: mean[k], sigma[k] for shift k = 0..2 and, at index 3, the
 * extrapolation to zero shift.  MBPT_EINVAL if the integral has no shifts. */
int mbpt_estimate_shifts(const mbpt_diag* diag, double mean[4], double sigma[4]);

/*
 * Checkpoint: the grid, the iteration history and counters as a host byte
 * image.  With buf == NULL (or cap too small) *need receives the size and
 * MBPT_ENOMEM is returned if buf != NULL.  mbpt_set_state restores an image
 * taken from an integral with the same descriptor shape and configuration.
 */
int mbpt_get_state(const mbpt_diag* diag, void* buf, size_t cap, size_t* need);
int mbpt_set_state(mbpt_diag* diag, const void* buf, size_t len);

/*
 * Test hook: evaluate samples [first, first + count) of iteration `iter` with
 * the integral's current grid and copy to host memory the mapped points
 * x[count][d] (in [0,1]^d) and weights w[count] = J_vegas * f(x), evaluated as
 * mbpt_vegas_iterate evaluates them (the context's Goldstone-sum strategy).  Does
 * not touch the integral's accumulators.  x may be NULL.
 */
int mbpt_dump_samples(mbpt_diag* diag, int64_t iter, int64_t first, int64_t count, double* x, double* w);

/* Test hook: Philox4x32-10 on the device for counters (ctr0 + i, ctr1, ctr2,
 * ctr3), i < count; out receives 4*count words. */
int mbpt_philox_device(mbpt_ctx* ctx, const uint32_t ctr[4], const uint32_t key[2], int64_t count, uint32_t* out);

/*
 * One VEGAS iteration of one integral without any device allocation.  The
 * paper has no counterpart: this serves callers that must not allocate device
 * memory once running (device memory owned by another allocator or a fixed
 * budget; loops where cudaMalloc's implicit synchronisation is unacceptable).
 *
 * Evaluates samples 0..samples_per_iter-1 of iteration `iter` (Philox counter
 * word 1) on the caller's grid and writes, in a fixed summation order,
 *   out[0] = sum w, out[1] = sum w^2, out[2 + a*n_bins + i] = histogram of w^2
 * (axis a, bin i).  grid: device pointer, d rows of n_bins+1 edges
 * (d = 3(order+1)); out: device pointer to 2 + d*n_bins doubles.  Neither is
 * retained.  Same integrand, launch shape and chunking as a fresh context's
 * mbpt_vegas_iterate, so the sums agree with that path.  No refinement or
 * combination.  Asynchronous on `cuda_stream` (NULL = legacy default stream).
 *
 * Scratch: one file-scope device array of 32 MiB per device, held from the
 * library's load to process exit and shared by every call.  Requests that
 * need more (with 50 bins: above about 3.8e7 samples at order 5, 1.1e8 at
 * order 3) fail with MBPT_EINVAL and a message giving the limit.  The
 * first call on a device looks up the array's device address and sets kernel
 * attributes for that device.  Every call copies its work description from
 * host stack memory with cudaMemcpyAsync.  Calls that overlap on the GPU
 * (different streams, or different host threads) race on the shared array:
 * serialise them.  Each call resets
 * the parts that must start at zero; the rest of the array keeps the last
 * call's contents.
 *
 * Errors: invalid arguments are rejected on the host (MBPT_EINVAL) before
 * anything is queued, and out is left untouched.  Should the kernel report an
 * error in its device error word (an out-of-range chunk or a record that no
 * compiled case matches -- validated input does not produce one), the call has
 * already returned, so every element of out (the sums and the histogram) is
 * set to NaN instead.
 */
int mbpt_vegas_iteration_noalloc(int device, const mbpt_diagram_desc* desc, const mbpt_physics* physics,
                                 const mbpt_vegas_cfg* cfg, uint32_t iter, const double* grid, double* out,
                                 void* cuda_stream);

/*
 * Measurement helper (the paper has no counterpart): FP64 thread operations per second that a
 * dependency-free DFMA loop (eight independent fused multiply-add chains per thread, 2048 threads per
 * SM) reaches on `device` now, timed with CUDA events on `cuda_stream` (best of three launches after a
 * warm-up launch; synchronises the stream).  It is the denominator of the roofline fraction of the
 * FP64-bound sample-evaluation kernel, measured at the clock the GPU runs at.
 */
int mbpt_fp64_rate(int device, void* cuda_stream, double* ops_per_s);

const char* mbpt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MBPT_H */
