/*
 * oracle.c -- plain, slow FP64 CPU oracle for the Monte Carlo evaluation of
 * zero-temperature Hugenholtz diagrams (arXiv:2603.24532, Sec. II and III.C).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it.  It shares no code, header, table or constant with the
 * CUDA path: it has its own Philox4x32-10, its own reading of a diagram
 * (sign, weight, cuts, loop momenta), an explicit spin/isospin enumeration of
 * the antisymmetrised vertices, and its own VEGAS map, histogram and grid
 * refinement.  Every step is written in the order the paper (or the cited
 * textbook method) states it, with no fusion or reordering.
 *
 * Diagram input (the oracle's own convention, documented in oracle/__init__.py):
 *   n            order = number of vertices, 2..6 (vertex index = time order,
 *                0 = earliest)
 *   lines[2*nl]  (src, dst) per line, nl = 2n; src < dst => particle,
 *                src > dst => hole (Sec. II: particles a,b,.. and holes i,j,..)
 *   ports[4*n]   per vertex (o1, o2, i1, i2): the vertex is <o1 o2|V|i1 i2>,
 *                o = lines leaving the vertex, i = lines entering it
 *   chords[n+1]  lines whose momenta are the free loop momenta
 *
 * Parity status of each function (what pins it; see tests/):
 *   oracle_philox4x32_10   pinned: published known-answer vectors + cuRAND
 *   oracle_derive          pinned: Eqs. (2)-(5) prefactors, toy-space RSPT
 *   oracle_integrand       pinned: closed forms at first order, Gauss-Legendre
 *                          quadrature of Eq. (2), scaling laws, mirror pairs
 *   oracle_first_order_integrand  pinned: C_S n (g-1)/(2g) closed form, 1D GL
 *   oracle_discrete_diagram pinned: exact Rayleigh-Schroedinger coefficients
 *   oracle_vegas_samples / oracle_refine  pinned: separable test integrals
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stdint.h>
#include <string.h>

#define O_MAXN 6
#define O_MAXL 12
#define O_MAXC 7

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11 "Parallel random numbers:
 * as easy as 1, 2, 3").  Ten rounds of the S-box
 *   (c0,c1,c2,c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
 * with the key bumped by the Weyl constants between rounds.
 * ------------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) { k0 += W0; k1 += W1; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ---------------------------------------------------------------------------
 * Derived description of a diagram.  Layout of the int array `info`:
 * ------------------------------------------------------------------------- */
enum {
    OI_N = 0, OI_NL, OI_NC, OI_H, OI_NEQ, OI_L0, OI_OK,
    OI_SRC = 8,
    OI_DST = OI_SRC + O_MAXL,
    OI_PORT = OI_DST + O_MAXL,          /* 4 per vertex */
    OI_CHORD = OI_PORT + 4 * O_MAXN,
    OI_COEF = OI_CHORD + O_MAXC,        /* coef[l*O_MAXC + c] in {-1,0,1} */
    OI_END = OI_COEF + O_MAXL * O_MAXC
};
int oracle_info_ints(void) { return OI_END; }

/* Solve A z = b for a small dense system by Gaussian elimination with partial
 * pivoting.  Returns 0 if singular. */
static int solve_dense(int m, double A[O_MAXN][O_MAXN], double b[O_MAXN], double z[O_MAXN]) {
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (fabs(A[piv][col]) < 1e-12) return 0;
        if (piv != col) {
            for (int k = 0; k < m; ++k) { double t = A[col][k]; A[col][k] = A[piv][k]; A[piv][k] = t; }
            double t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        for (int r = col + 1; r < m; ++r) {
            double f = A[r][col] / A[col][col];
            for (int k = col; k < m; ++k) A[r][k] -= f * A[col][k];
            b[r] -= f * b[col];
        }
    }
    for (int r = m - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < m; ++k) s -= A[r][k] * z[k];
        z[r] = s / A[r][r];
    }
    return 1;
}

/*
 * oracle_derive: from the raw diagram, compute
 *   h     = number of hole lines,
 *   n_eq  = number of ordered vertex pairs joined by two lines of the same
 *           direction (equivalent lines),
 *   l0    = number of closed loops when every vertex <o1 o2|V|i1 i2> pairs
 *           i1 -> o1 and i2 -> o2,
 *   coef  = k_line = sum_c coef[line][c] * l_c from momentum conservation
 *           (sum of momenta entering a vertex = sum leaving it),
 * and returns 1 on success, 0 if the input is not a valid diagram.
 * The Hugenholtz rule applied later is (-1)^(h + l0) / 2^n_eq (textbook
 * Hugenholtz rules; reproduces the prefactors of Eqs. (2)-(5)).
 */
int oracle_derive(int n, const int* lines, const int* ports, const int* chords, int* info) {
    memset(info, 0, sizeof(int) * OI_END);
    int nl = 2 * n, nc = n + 1;
    if (n < 2 || n > O_MAXN) return 0;
    info[OI_N] = n; info[OI_NL] = nl; info[OI_NC] = nc;
    for (int l = 0; l < nl; ++l) {
        int s = lines[2 * l], d = lines[2 * l + 1];
        if (s < 0 || s >= n || d < 0 || d >= n || s == d) return 0;
        info[OI_SRC + l] = s; info[OI_DST + l] = d;
    }
    /* ports must list each line exactly once as an out-port of its src and
     * once as an in-port of its dst */
    for (int v = 0; v < n; ++v) {
        for (int k = 0; k < 4; ++k) {
            int l = ports[4 * v + k];
            if (l < 0 || l >= nl) return 0;
            info[OI_PORT + 4 * v + k] = l;
            if (k < 2 && lines[2 * l] != v) return 0;
            if (k >= 2 && lines[2 * l + 1] != v) return 0;
        }
        if (ports[4 * v] == ports[4 * v + 1] || ports[4 * v + 2] == ports[4 * v + 3]) return 0;
    }
    int h = 0;
    for (int l = 0; l < nl; ++l) if (lines[2 * l] > lines[2 * l + 1]) ++h;
    info[OI_H] = h;
    int neq = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            int cnt = 0;
            for (int l = 0; l < nl; ++l) if (lines[2 * l] == i && lines[2 * l + 1] == j) ++cnt;
            if (cnt == 2) ++neq;
        }
    info[OI_NEQ] = neq;
    /* loops of the direct pairing: a line entering vertex v through port i1
     * continues on the line leaving through o1; i2 continues on o2 */
    int seen[O_MAXL] = {0}, loops = 0;
    for (int start = 0; start < nl; ++start) {
        if (seen[start]) continue;
        ++loops;
        int l = start;
        while (!seen[l]) {
            seen[l] = 1;
            int v = lines[2 * l + 1];
            if (ports[4 * v + 2] == l) l = ports[4 * v + 0];
            else l = ports[4 * v + 1];
        }
    }
    info[OI_L0] = loops;
    /* chords */
    int is_chord[O_MAXL] = {0};
    for (int c = 0; c < nc; ++c) {
        int l = chords[c];
        if (l < 0 || l >= nl || is_chord[l]) return 0;
        is_chord[l] = 1;
        info[OI_CHORD + c] = l;
    }
    /* tree lines: the remaining n-1 lines; unknown momenta z_t.  Conservation
     * at vertices 1..n-1 (vertex 0's equation is implied). */
    int tree[O_MAXL], nt = 0;
    for (int l = 0; l < nl; ++l) if (!is_chord[l]) tree[nt++] = l;
    if (nt != n - 1) return 0;
    for (int c = 0; c < nc; ++c) {
        double A[O_MAXN][O_MAXN], b[O_MAXN], z[O_MAXN];
        for (int r = 0; r < n - 1; ++r) {
            int v = r + 1;
            b[r] = 0.0;
            for (int t = 0; t < nt; ++t) {
                int l = tree[t];
                double a = 0.0;
                if (lines[2 * l + 1] == v) a += 1.0;   /* entering */
                if (lines[2 * l] == v) a -= 1.0;       /* leaving */
                A[r][t] = a;
            }
            /* chord c carries unit momentum; move it to the right-hand side */
            int lc = chords[c];
            double a = 0.0;
            if (lines[2 * lc + 1] == v) a += 1.0;
            if (lines[2 * lc] == v) a -= 1.0;
            b[r] = -a;
        }
        if (!solve_dense(n - 1, A, b, z)) return 0;
        for (int l = 0; l < nl; ++l) info[OI_COEF + l * O_MAXC + c] = 0;
        info[OI_COEF + chords[c] * O_MAXC + c] = 1;
        for (int t = 0; t < nt; ++t) {
            double r = floor(z[t] + 0.5);
            if (fabs(z[t] - r) > 1e-9 || fabs(r) > 1.0) return 0;
            info[OI_COEF + tree[t] * O_MAXC + c] = (int)r;
        }
    }
    /* verify conservation at every vertex, including vertex 0 */
    for (int v = 0; v < n; ++v)
        for (int c = 0; c < nc; ++c) {
            int s = 0;
            for (int l = 0; l < nl; ++l) {
                int cf = info[OI_COEF + l * O_MAXC + c];
                if (lines[2 * l + 1] == v) s += cf;
                if (lines[2 * l] == v) s -= cf;
            }
            if (s != 0) return 0;
        }
    info[OI_OK] = 1;
    return 1;
}

/* ---------------------------------------------------------------------------
 * Physics parameters, array `ph`:
 *   ph[0] kF_n, ph[1] kF_p (fm^-1; a species with kF = 0 is absent)
 *   ph[2] hbar^2/m (MeV fm^2)
 *   ph[3] C_S (MeV fm^3), ph[4] C_Y (MeV fm), ph[5] m_pi (fm^-1),
 *   ph[6] Lambda (fm^-1), ph[7] regulator exponent (even integer),
 *   ph[8] K_max: upper end of the radial range of particle chords (fm^-1)
 *   ph[9] chord map: 0 full directions, 1 rotational reduction (see chord_momenta)
 *   ph[10] denominator shift s (MeV): every D_m below is replaced by D_m - s
 *          (the regulator of Sec. III.A; 0 = the diagram itself)
 *   ph[11] single-particle spectrum: 0 free, eps = (hbar^2/2m) k^2; 1 Hartree-Fock,
 *          eps = (hbar^2/2m) k^2 + Sigma(k) (Eq. (7)) with Sigma from the cubic spline whose
 *          knots follow: ph[12] number of knots N, ph[13] knot spacing h (knot i at k = i h),
 *          ph[14 .. 14+N) Sigma at the knots (MeV), ph[14+N .. 14+2N) the spline's second
 *          derivatives (oracle_spline_build); Sigma = 0 beyond the last knot
 * The potential is V(p, p') = [C_S + C_Y / (|p - p'|^2 + m_pi^2)]
 *                             * exp(-(|p|/Lambda)^r - (|p'|/Lambda)^r).
 * ------------------------------------------------------------------------- */
static double vpot(const double* ph, const double p[3], const double pp[3]) {
    double q2 = 0.0, p2 = 0.0, pp2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        q2 += (p[k] - pp[k]) * (p[k] - pp[k]);
        p2 += p[k] * p[k];
        pp2 += pp[k] * pp[k];
    }
    double r = ph[7];
    double reg = exp(-pow(sqrt(p2) / ph[6], r) - pow(sqrt(pp2) / ph[6], r));
    return (ph[3] + ph[4] / (q2 + ph[5] * ph[5])) * reg;
}

/* Radial range of chord momenta: a hole chord lies in [0, kF_max], a particle
 * chord in [kF_min, K_max], where kF_min is the smallest Fermi momentum of a
 * species that is present. */
static void chord_range(const double* ph, int hole, double* lo, double* hi) {
    double kfn = ph[0], kfp = ph[1];
    double kmax = kfn > kfp ? kfn : kfp;
    double kmin = kmax;
    if (kfn > 0.0 && kfn < kmin) kmin = kfn;
    if (kfp > 0.0 && kfp < kmin) kmin = kfp;
    if (hole) { *lo = 0.0; *hi = kmax; }
    else { *lo = kmin; *hi = ph[8]; }
}

/*
 * Map three unit-interval coordinates to a chord momentum (spherical
 * coordinates with a rational azimuth):
 *   k      = lo + (hi - lo) x0
 *   cos(t) = 2 x1 - 1,   sin(t) = 2 sqrt(x1 (1 - x1))
 *   a = x2 (1 - x2), b = x2 - 1/2, m = a^2 + b^2 ... = (1/2 - a)^2,
 *   cos(phi) = (a^2 - b^2)/mm, sin(phi) = 2ab/mm with mm = a^2 + b^2,
 *   which sweeps phi over (-pi, pi) with d(phi)/d(x2) = 2/(1/2 - a).
 * Returns the Jacobian of d^3k = k^2 dk dcos(t) dphi with respect to x.
 */
static double chord_map(const double x[3], double lo, double hi, double out[3]) {
    double k = lo + (hi - lo) * x[0];
    double ct = 2.0 * x[1] - 1.0;
    double st = 2.0 * sqrt(x[1] * (1.0 - x[1]));
    double a = x[2] * (1.0 - x[2]);
    double b = x[2] - 0.5;
    double mm = a * a + b * b;
    double cphi = (a * a - b * b) / mm;
    double sphi = 2.0 * a * b / mm;
    out[0] = k * st * cphi;
    out[1] = k * st * sphi;
    out[2] = k * ct;
    double dphi = 2.0 / (0.5 - a);
    return (hi - lo) * k * k * 2.0 * dphi;
}

/* Explicit spin-isospin enumeration state */
typedef struct {
    int n, nl;
    const int* info;
    int nlab;                 /* labels per line = 2 spins x number of species */
    int lab_species[4];       /* species of label index (0 = n, 1 = p) */
    int lab_spin[4];
    double ksq[O_MAXL];       /* |k_l|^2 */
    double kf2[2];            /* kF^2 per species */
    double Vd[O_MAXN], Ve[O_MAXN];
    int label[O_MAXL];
    int last_line_of_vertex[O_MAXN];
    int absmode;              /* 1: sum |terms| (condition number of the spin sum) */
} spin_enum;

static int line_is_hole(const int* info, int l) { return info[OI_SRC + l] > info[OI_DST + l]; }

/* step function of line l for label `lab`: hole -> k^2 < kF^2, particle -> k^2 >= kF^2 */
static int step_ok(const spin_enum* S, int l, int lab) {
    double kf2 = S->kf2[S->lab_species[lab]];
    if (line_is_hole(S->info, l)) return S->ksq[l] < kf2;
    return S->ksq[l] >= kf2;
}

/* value of the antisymmetrised vertex <o1 o2|V|i1 i2> for the current labels:
 * delta(o1,i1) delta(o2,i2) V(p,p') - delta(o1,i2) delta(o2,i1) V(p,-p') */
static double vertex_value(const spin_enum* S, int v) {
    const int* pt = S->info + OI_PORT + 4 * v;
    int o1 = S->label[pt[0]], o2 = S->label[pt[1]], i1 = S->label[pt[2]], i2 = S->label[pt[3]];
    double val = 0.0;
    if (S->absmode) {
        if (o1 == i1 && o2 == i2) val += fabs(S->Vd[v]);
        if (o1 == i2 && o2 == i1) val += fabs(S->Ve[v]);
        return val;
    }
    if (o1 == i1 && o2 == i2) val += S->Vd[v];
    if (o1 == i2 && o2 == i1) val -= S->Ve[v];
    return val;
}

static double enumerate(spin_enum* S, int l, double acc) {
    if (l == S->nl) return acc;
    double total = 0.0;
    for (int lab = 0; lab < S->nlab; ++lab) {
        if (!step_ok(S, l, lab)) continue;
        S->label[l] = lab;
        double a = acc;
        for (int v = 0; v < S->n && a != 0.0; ++v)
            if (S->last_line_of_vertex[v] == l) a *= vertex_value(S, v);
        if (a == 0.0) continue;
        total += enumerate(S, l + 1, a);
    }
    return total;
}

/* Sum over the spin (and isospin) labels of every line of
 *   prod_l Theta_l * prod_v <o1 o2|V|i1 i2>_v. */
static double spin_sum(spin_enum* S) {
    for (int v = 0; v < S->n; ++v) {
        int m = -1;
        for (int k = 0; k < 4; ++k) {
            int l = S->info[OI_PORT + 4 * v + k];
            if (l > m) m = l;
        }
        S->last_line_of_vertex[v] = m;
    }
    return enumerate(S, 0, 1.0);
}

static void setup_labels(spin_enum* S, const double* ph) {
    S->nlab = 0;
    for (int sp = 0; sp < 2; ++sp) {
        if (!(ph[sp] > 0.0)) continue;
        for (int sg = 0; sg < 2; ++sg) {
            S->lab_species[S->nlab] = sp;
            S->lab_spin[S->nlab] = sg;
            ++S->nlab;
        }
    }
    S->kf2[0] = ph[0] * ph[0];
    S->kf2[1] = ph[1] * ph[1];
}

/* Total nucleon density n = (kF_n^3 + kF_p^3) / (3 pi^2) (two spin states per
 * species; Sec. II, kF = (3 pi^2 n_tau)^(1/3)). */
static double density(const double* ph) {
    return (ph[0] * ph[0] * ph[0] + ph[1] * ph[1] * ph[1]) / (3.0 * M_PI * M_PI);
}

/* ---------------------------------------------------------------------------
 * Hartree-Fock spectrum (Eq. (7)).
 * ------------------------------------------------------------------------- */

/* Gauss-Legendre nodes and weights on [-1, 1]: Newton iteration on the Legendre polynomial P_n
 * (three-term recurrence) from the Chebyshev-like starting guess cos(pi (i + 3/4)/(n + 1/2)). */
void oracle_gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Hartree-Fock self-energy (MeV) of a nucleon of momentum k in matter with one Fermi momentum kF and
 * g occupied labels (2 neutron matter, 4 symmetric matter), for the spin-isospin independent
 * potential: the direct term <ij|V|ij> counts every label of j, the exchange term only j with i's
 * label, so
 *   Sigma(k) = (1/(2 pi)^3) int_{k' < kF} d^3k' [g V(p, p) - V(p, -p)],  p = (k - k')/2,
 * reduced by azimuthal symmetry to 1/(4 pi^2) int_0^kF dk' k'^2 int_{-1}^{1} dc [...], with
 * |p|^2 = (k^2 + k'^2 - 2 k k' c)/4, on n_rad x n_ang Gauss-Legendre nodes. */
double oracle_hf_self_energy(const double* ph, double k, int n_rad, int n_ang) {
    double kf = ph[0] > 0.0 ? ph[0] : ph[1];
    double g = (ph[0] > 0.0 ? 2.0 : 0.0) + (ph[1] > 0.0 ? 2.0 : 0.0);
    double xr[256], wr[256], xa[256], wa[256];
    if (n_rad > 256 || n_ang > 256) return NAN;
    oracle_gauss_legendre(n_rad, xr, wr);
    oracle_gauss_legendre(n_ang, xa, wa);
    double tot = 0.0;
    for (int i = 0; i < n_rad; ++i) {
        double kp = 0.5 * kf * (xr[i] + 1.0), wk = 0.5 * kf * wr[i];
        double inner = 0.0;
        for (int j = 0; j < n_ang; ++j) {
            double c = xa[j];
            double p2 = 0.25 * (k * k + kp * kp - 2.0 * k * kp * c);
            if (p2 < 0.0) p2 = 0.0;
            /* p along z and p' = +-p: V(p, p) has q = 0, V(p, -p) has |q|^2 = 4 p^2 */
            double pv[3] = {0.0, 0.0, sqrt(p2)}, mv[3] = {0.0, 0.0, -sqrt(p2)};
            inner += wa[j] * (g * vpot(ph, pv, pv) - vpot(ph, pv, mv));
        }
        tot += wk * kp * kp * inner;
    }
    return tot / (4.0 * M_PI * M_PI);
}

/* Cubic spline through y_i at k_i = i h (i < n) with zero slope at k = 0 (Sigma is even in k) and
 * zero curvature at the last knot; m receives the second derivatives (tridiagonal system solved by
 * forward elimination and back substitution). */
void oracle_spline_build(int n, double h, const double* y, double* m) {
    double c[4096], d[4096];
    if (n < 3 || n > 4096) return;
    /* row 0: 2 m0 + m1 = 6 (y1 - y0)/h^2; rows 1..n-2: m_{i-1} + 4 m_i + m_{i+1} = 6 (y_{i-1} - 2 y_i + y_{i+1})/h^2 */
    double b0 = 2.0;
    c[0] = 1.0 / b0;
    d[0] = 6.0 * (y[1] - y[0]) / (h * h) / b0;
    for (int i = 1; i < n - 1; ++i) {
        double rhs = 6.0 * (y[i - 1] - 2.0 * y[i] + y[i + 1]) / (h * h);
        double den = 4.0 - c[i - 1];
        c[i] = 1.0 / den;
        d[i] = (rhs - d[i - 1]) / den;
    }
    m[n - 1] = 0.0;
    for (int i = n - 2; i >= 0; --i) m[i] = d[i] - c[i] * m[i + 1];
}

double oracle_spline_eval(int n, double h, const double* y, const double* m, double k) {
    if (!(k < (n - 1) * h)) return 0.0;
    int i = (int)floor(k / h);
    if (i > n - 2) i = n - 2;
    double t = k - i * h;
    double slope = (y[i + 1] - y[i]) / h - h * (2.0 * m[i] + m[i + 1]) / 6.0;
    return y[i] + t * slope + t * t * m[i] / 2.0 + t * t * t * (m[i + 1] - m[i]) / (6.0 * h);
}

/* Single-particle energy (MeV) of a line with |k|^2 = ksq; *mag receives |kinetic| + |Sigma| for the
 * rounding estimate. */
static double sp_energy(const double* ph, double ksq, double* mag) {
    double kin = 0.5 * ph[2] * ksq;
    if (ph[11] == 0.0) {
        *mag = kin;
        return kin;
    }
    int n = (int)ph[12];
    double sg = oracle_spline_eval(n, ph[13], ph + 14, ph + 14 + n, sqrt(ksq));
    *mag = kin + fabs(sg);
    return kin + sg;
}

/*
 * oracle_integrand: the contribution of one diagram to E/N at a point
 * x in [0,1]^(3(n+1)) of the chord coordinates:
 *
 *   f(x) = (-1)^(h+l0) 2^(-n_eq) / n_dens * J_chords(x) / (2 pi)^(3(n+1))
 *          * sum_labels prod_l Theta_l prod_v <o1 o2|V|i1 i2>_v / prod_m D_m
 *
 * with D_m = sum_{holes crossing cut m} eps - sum_{particles crossing cut m} eps,
 * eps = (hbar^2/2m) k^2, cut m lying between vertices m and m+1 (Sec. II,
 * Eqs. (2)-(6) with the free spectrum).  `count_D` (optional) receives the
 * condition number sum_m (sum_{l in C_m} eps_l) / |D_m| used by the parity
 * tolerance.
 */
/*
 * Chord momenta of the point x and the Jacobian of the chord map.  ph[9] selects the map:
 *   0: every chord from chord_map on axes 3c..3c+2;
 *   1: rotational invariance of the integrand (Sec. III.C): chord 0 = (0, 0, k) from axis 0 with
 *      Jacobian 4 pi range k^2 (all its directions integrated out), chord 1 =
 *      k (sin t, 0, cos t) from axes 1, 2 (cos t = 2 x - 1) with Jacobian 2 pi 2 range k^2 (all its
 *      azimuths integrated out), chords c >= 2 from chord_map on axes 3c-3..3c-1.
 */
static double chord_momenta(const int* info, const double* ph, const double* x, double* chord_k) {
    int nc = info[OI_NC];
    int mapk = (int)ph[9];
    double jac = 1.0;
    for (int c = 0; c < nc; ++c) {
        int l = info[OI_CHORD + c];
        double lo, hi;
        chord_range(ph, line_is_hole(info, l), &lo, &hi);
        double* out = chord_k + 3 * c;
        if (mapk == 1 && c == 0) {
            double k = lo + (hi - lo) * x[0];
            out[0] = 0.0; out[1] = 0.0; out[2] = k;
            jac *= 4.0 * M_PI * (hi - lo) * k * k;
        } else if (mapk == 1 && c == 1) {
            double k = lo + (hi - lo) * x[1];
            double ct = 2.0 * x[2] - 1.0;
            double st = 2.0 * sqrt(x[2] * (1.0 - x[2]));
            out[0] = k * st; out[1] = 0.0; out[2] = k * ct;
            jac *= 2.0 * M_PI * 2.0 * (hi - lo) * k * k;
        } else {
            int off = mapk == 1 ? 3 * c - 3 : 3 * c;
            jac *= chord_map(x + off, lo, hi, out);
        }
    }
    return jac;
}

double oracle_integrand_momenta(const int* info, const double* ph, const double* chord_k_flat, double* cond);

double oracle_integrand(const int* info, const double* ph, const double* x, double* cond) {
    int nc = info[OI_NC];
    double chord_k[O_MAXC * 3];
    if (cond) *cond = 0.0;
    double jac = chord_momenta(info, ph, x, chord_k);
    double core = oracle_integrand_momenta(info, ph, chord_k, cond);
    if (core == 0.0) return 0.0;
    return jac * core / pow(2.0 * M_PI, 3.0 * nc);
}

/*
 * The integrand at given chord momenta, without the chord-map Jacobian and the
 * (2 pi)^(-3(n+1)) measure:
 *   (-1)^(h+l0) 2^(-n_eq) / n_dens * sum_labels prod_l Theta_l prod_v <o1 o2|V|i1 i2>_v / prod_m D_m
 */
double oracle_integrand_momenta(const int* info, const double* ph, const double* chord_k_flat, double* cond) {
    int n = info[OI_N], nl = info[OI_NL], nc = info[OI_NC];
    if (cond) *cond = 0.0;
    spin_enum S;
    memset(&S, 0, sizeof(S));
    S.n = n; S.nl = nl; S.info = info;
    setup_labels(&S, ph);
    double k[O_MAXL][3];
    for (int l = 0; l < nl; ++l) {
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int c = 0; c < nc; ++c) s += info[OI_COEF + l * O_MAXC + c] * chord_k_flat[3 * c + a];
            k[l][a] = s;
        }
        S.ksq[l] = k[l][0] * k[l][0] + k[l][1] * k[l][1] + k[l][2] * k[l][2];
    }
    for (int v = 0; v < n; ++v) {
        const int* pt = info + OI_PORT + 4 * v;
        double p[3], pp[3], mpp[3];
        for (int a = 0; a < 3; ++a) {
            p[a] = 0.5 * (k[pt[0]][a] - k[pt[1]][a]);
            pp[a] = 0.5 * (k[pt[2]][a] - k[pt[3]][a]);
            mpp[a] = -pp[a];
        }
        S.Vd[v] = vpot(ph, p, pp);
        S.Ve[v] = vpot(ph, p, mpp);
    }
    double ssum = spin_sum(&S);
    if (ssum == 0.0) return 0.0;
    double dprod = 1.0, condsum = 0.0;
    for (int m = 0; m < n - 1; ++m) {
        double D = 0.0, mag = 0.0;
        for (int l = 0; l < nl; ++l) {
            int s = info[OI_SRC + l], d = info[OI_DST + l];
            int lo = s < d ? s : d, hi = s < d ? d : s;
            if (!(lo <= m && m < hi)) continue;
            double emag;
            double eps = sp_energy(ph, S.ksq[l], &emag);
            if (line_is_hole(info, l)) D += eps;
            else D -= eps;
            mag += emag;
        }
        if (!(D < 0.0)) return 0.0;   /* only on a measure-zero set */
        D -= ph[10];
        dprod *= D;
        condsum += mag / fabs(D);
    }
    if (cond) {
        /* rounding amplification: energy denominators plus the cancellation in the
         * spin sum, sum |terms| / |sum| */
        S.absmode = 1;
        double sabs = spin_sum(&S);
        *cond = condsum + sabs / fabs(ssum);
    }
    int h = info[OI_H], l0 = info[OI_L0], neq = info[OI_NEQ];
    double sign = ((h + l0) % 2 == 0) ? 1.0 : -1.0;
    return sign / pow(2.0, neq) / density(ph) * ssum / dprod;
}

/* Squared line momenta |k_l|^2 at the point x (chord map + momentum routing), for
 * classifying samples that sit within rounding of a Fermi surface. */
void oracle_line_ksq(const int* info, const double* ph, const double* x, double* out) {
    int nl = info[OI_NL], nc = info[OI_NC];
    double chord_k[O_MAXC * 3];
    chord_momenta(info, ph, x, chord_k);
    for (int l = 0; l < nl; ++l) {
        double k[3];
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int c = 0; c < nc; ++c) s += info[OI_COEF + l * O_MAXC + c] * chord_k[3 * c + a];
            k[a] = s;
        }
        out[l] = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    }
}

/*
 * First-order (Hartree-Fock) potential energy per particle, the one diagram
 * with a single vertex whose two lines are holes closing on themselves
 * (Eq. (1)): E/N = (1/n) (1/2) sum_{labels} int d^3k1 d^3k2/(2pi)^6 n1 n2 <12|V|12>.
 * x in [0,1]^6 maps the two hole momenta with chord_map on [0, kF_max].
 */
double oracle_first_order_integrand(const double* ph, const double* x) {
    double k1[3], k2[3], lo, hi;
    chord_range(ph, 1, &lo, &hi);
    double jac = chord_map(x, lo, hi, k1) * chord_map(x + 3, lo, hi, k2);
    spin_enum S;
    memset(&S, 0, sizeof(S));
    setup_labels(&S, ph);
    double ks1 = k1[0] * k1[0] + k1[1] * k1[1] + k1[2] * k1[2];
    double ks2 = k2[0] * k2[0] + k2[1] * k2[1] + k2[2] * k2[2];
    double p[3], mp[3];
    for (int a = 0; a < 3; ++a) { p[a] = 0.5 * (k1[a] - k2[a]); mp[a] = -p[a]; }
    double vd = vpot(ph, p, p), ve = vpot(ph, p, mp);
    double total = 0.0;
    for (int a = 0; a < S.nlab; ++a) {
        if (!(ks1 < S.kf2[S.lab_species[a]])) continue;
        for (int b = 0; b < S.nlab; ++b) {
            if (!(ks2 < S.kf2[S.lab_species[b]])) continue;
            /* <ab|V|ab>: direct delta(a,a)delta(b,b) = 1, exchange delta(a,b) */
            double val = vd;
            if (a == b) val -= ve;
            total += val;
        }
    }
    return 0.5 * total * jac / pow(2.0 * M_PI, 6.0) / density(ph);
}

/* ---------------------------------------------------------------------------
 * VEGAS (Lepage, J. Comput. Phys. 27 (1978) 192), one iteration's samples.
 *
 * Sample s of iteration t of the integral with stream id `sid` draws
 * Philox4x32-10 blocks j = 0..ceil(d/4)-1 with key (seed_lo, seed_hi) and
 * counter (s, t, sid, j); axis a uses word a of the concatenated output and
 * y_a = (u_a + 1/2) 2^-32.  The map:  i = floor(y N_b),
 *   x = e_i + (y N_b - i)(e_{i+1} - e_i),  J = prod_a N_b (e_{i+1} - e_i),
 * and w = J f(x).  Accumulates sum w, sum w^2 and per-axis, per-bin sums of
 * w^2 in sample order.  `grid` holds d rows of N_b+1 edges.
 * kind: 0 = diagram (info, ph), 1 = first-order diagram, 2 = test integrand
 * (separable Gaussian product, params in ph: centre ph[0], width ph[1]),
 * 3 = test integrand (product of pi/2 sin(pi x)).
 * ------------------------------------------------------------------------- */
static double test_integrand(int kind, const double* ph, const double* x, int d) {
    double f = 1.0;
    for (int a = 0; a < d; ++a) {
        if (kind == 2) {
            double z = (x[a] - ph[0]) / ph[1];
            f *= exp(-0.5 * z * z) / (ph[1] * sqrt(2.0 * M_PI));
        } else {
            f *= 0.5 * M_PI * sin(M_PI * x[a]);
        }
    }
    return f;
}

static void vegas_samples_impl(int kind, int n_members, const int* info, const double* scale,
                               const double* ph, int d, int nb, const double* grid, uint64_t seed,
                               uint32_t sid, uint32_t t, uint64_t s_begin, uint64_t s_end, double* sums,
                               double* hist, double* dump_x, double* dump_w) {
    double sw = 0.0, sw2 = 0.0;
    for (uint64_t s = s_begin; s < s_end; ++s) {
        uint32_t words[4 * ((O_MAXC * 3 + 3) / 4 + 1)];
        int nblk = (d + 3) / 4;
        for (int j = 0; j < nblk; ++j) {
            uint32_t ctr[4] = {(uint32_t)s, t, sid, (uint32_t)j};
            uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
            oracle_philox4x32_10(ctr, key, words + 4 * j);
        }
        double x[O_MAXC * 3];
        int bin[O_MAXC * 3];
        double jac = 1.0;
        for (int a = 0; a < d; ++a) {
            double y = ((double)words[a] + 0.5) * (1.0 / 4294967296.0);
            double yn = y * nb;
            int i = (int)floor(yn);
            if (i >= nb) i = nb - 1;
            const double* e = grid + (size_t)a * (nb + 1);
            x[a] = e[i] + (yn - i) * (e[i + 1] - e[i]);
            jac *= nb * (e[i + 1] - e[i]);
            bin[a] = i;
        }
        double f;
        if (kind == 0) {
            /* a group integrand is the plain sum of its members' integrands at the same point,
             * each through its own chord map (Sec. III.A, grouped evaluation) */
            f = 0.0;
            for (int m = 0; m < n_members; ++m)
                f += scale[m] * oracle_integrand(info + (size_t)m * OI_END, ph, x, NULL);
        } else if (kind == 1) f = oracle_first_order_integrand(ph, x);
        else f = test_integrand(kind, ph, x, d);
        double w = jac * f;
        sw += w;
        sw2 += w * w;
        if (hist)
            for (int a = 0; a < d; ++a) hist[(size_t)a * nb + bin[a]] += w * w;
        if (dump_x) {
            uint64_t r = s - s_begin;
            for (int a = 0; a < d; ++a) dump_x[r * d + a] = x[a];
            dump_w[r] = w;
        }
    }
    sums[0] += sw;
    sums[1] += sw2;
}

void oracle_vegas_samples(int kind, const int* info, const double* ph, int d, int nb,
                          const double* grid, uint64_t seed, uint32_t sid, uint32_t t,
                          uint64_t s_begin, uint64_t s_end,
                          double* sums, double* hist, double* dump_x, double* dump_w) {
    const double one = 1.0;
    vegas_samples_impl(kind, 1, info, &one, ph, d, nb, grid, seed, sid, t, s_begin, s_end, sums, hist, dump_x,
                       dump_w);
}

/* The same for the sum of n_members diagrams (infos: n_members consecutive info blocks), member m
 * scaled by scale[m]. */
void oracle_vegas_samples_group(int n_members, const int* infos, const double* scale, const double* ph, int d,
                                int nb, const double* grid, uint64_t seed, uint32_t sid, uint32_t t,
                                uint64_t s_begin, uint64_t s_end, double* sums, double* hist, double* dump_x,
                                double* dump_w) {
    vegas_samples_impl(0, n_members, infos, scale, ph, d, nb, grid, seed, sid, t, s_begin, s_end, sums, hist,
                       dump_x, dump_w);
}

/*
 * Grid refinement of one axis (Lepage 1978, with the smoothing used in the
 * current `vegas` package):
 *   dbar_0 = (7 d_0 + d_1)/8, dbar_i = (d_{i-1} + 6 d_i + d_{i+1})/8,
 *   dbar_{N-1} = (d_{N-2} + 7 d_{N-1})/8;  r_i = dbar_i / sum dbar;
 *   m_i = ((r_i - 1)/ln r_i)^alpha  (m_i = 0 where r_i = 0, 1 where r_i = 1);
 * then new edges place equal shares sum(m)/N of the piecewise-linear
 * cumulative of m in every new bin.  If every d_i is zero the grid is kept.
 */
void oracle_refine(const double* hist, const double* grid, int nb, double alpha, double* out) {
    double dbar[1024], m[1024];
    if (nb < 2 || nb > 1024) { memcpy(out, grid, sizeof(double) * (nb + 1)); return; }
    dbar[0] = (7.0 * hist[0] + hist[1]) / 8.0;
    for (int i = 1; i < nb - 1; ++i) dbar[i] = (hist[i - 1] + 6.0 * hist[i] + hist[i + 1]) / 8.0;
    dbar[nb - 1] = (hist[nb - 2] + 7.0 * hist[nb - 1]) / 8.0;
    double tot = 0.0;
    for (int i = 0; i < nb; ++i) tot += dbar[i];
    if (!(tot > 0.0)) { memcpy(out, grid, sizeof(double) * (nb + 1)); return; }
    double msum = 0.0;
    for (int i = 0; i < nb; ++i) {
        double r = dbar[i] / tot;
        if (r <= 0.0) m[i] = 0.0;
        else if (r >= 1.0) m[i] = 1.0;
        else m[i] = pow((r - 1.0) / log(r), alpha);
        msum += m[i];
    }
    double share = msum / nb;
    out[0] = grid[0];
    out[nb] = grid[nb];
    int j = 0;
    double cum = 0.0;      /* sum of m over bins before j */
    for (int k = 1; k < nb; ++k) {
        double target = k * share;
        while (j < nb - 1 && cum + m[j] < target) { cum += m[j]; ++j; }
        double frac = m[j] > 0.0 ? (target - cum) / m[j] : 0.0;
        if (frac > 1.0) frac = 1.0;
        if (frac < 0.0) frac = 0.0;
        out[k] = grid[j] + frac * (grid[j + 1] - grid[j]);
    }
}

/* ---------------------------------------------------------------------------
 * Discrete-label evaluation of a diagram in a finite single-particle space
 * (holes 0..nh-1 with energies eps[0..nh-1], particles nh..nh+np-1), for the
 * Rayleigh-Schroedinger check of the diagram rules:
 *   E_G = (-1)^(h+l0) 2^(-n_eq) sum_{labels} prod_v wbar[o1,o2,i1,i2] / prod_m D_m
 * with unrestricted label sums (exclusion-principle-violating terms kept).
 * wbar is N^4 row-major (N = nh+np), antisymmetric in each index pair.
 * ------------------------------------------------------------------------- */
typedef struct {
    const int* info; int n, nl, nh, np, N;
    const double* w; const double* eps;
    int label[O_MAXL];
} disc_state;

static double disc_rec(disc_state* D, int l) {
    if (l == D->nl) {
        double val = 1.0;
        for (int v = 0; v < D->n; ++v) {
            const int* pt = D->info + OI_PORT + 4 * v;
            size_t N = (size_t)D->N;
            val *= D->w[((D->label[pt[0]] * N + D->label[pt[1]]) * N + D->label[pt[2]]) * N + D->label[pt[3]]];
        }
        if (val == 0.0) return 0.0;
        for (int m = 0; m < D->n - 1; ++m) {
            double den = 0.0;
            for (int k = 0; k < D->nl; ++k) {
                int s = D->info[OI_SRC + k], d = D->info[OI_DST + k];
                int lo = s < d ? s : d, hi = s < d ? d : s;
                if (!(lo <= m && m < hi)) continue;
                if (s > d) den += D->eps[D->label[k]];
                else den -= D->eps[D->label[k]];
            }
            val /= den;
        }
        return val;
    }
    int hole = D->info[OI_SRC + l] > D->info[OI_DST + l];
    int first = hole ? 0 : D->nh, last = hole ? D->nh : D->nh + D->np;
    double total = 0.0;
    for (int lab = first; lab < last; ++lab) {
        D->label[l] = lab;
        total += disc_rec(D, l + 1);
    }
    return total;
}

double oracle_discrete_diagram(const int* info, int nh, int np, const double* wbar, const double* eps) {
    disc_state D;
    memset(&D, 0, sizeof(D));
    D.info = info; D.n = info[OI_N]; D.nl = info[OI_NL];
    D.nh = nh; D.np = np; D.N = nh + np; D.w = wbar; D.eps = eps;
    double s = disc_rec(&D, 0);
    int h = info[OI_H], l0 = info[OI_L0], neq = info[OI_NEQ];
    double sign = ((h + l0) % 2 == 0) ? 1.0 : -1.0;
    return sign / pow(2.0, neq) * s;
}
