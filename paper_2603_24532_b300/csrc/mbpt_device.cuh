// Device code of libmbpt: Philox4x32-10, the VEGAS map, the Hugenholtz-diagram
// integrand and the per-chunk sample loop (arXiv:2603.24532 Sec. II, III.C).
//
// Cost model on B300: an FP64 instruction costs ~64 FP32/INT instructions, so
// every step that does not need FP64 runs in FP32 or integer arithmetic, and the
// FP64 instruction count per sample is fixed by the order n alone (no
// data-dependent predication of FP64 work): structure that varies between
// diagrams is applied through integer selects on uniform indices.
#pragma once
#include <stdint.h>

#include "mbpt_internal.h"

namespace mbpt {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of
// (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)),
// key bumped by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t* out) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// v[lo + k] for a uniform 0 <= k < n (lo and n constants after unrolling) with integer selects, no
// predicated FP64 work: a tournament on the bits of k -- level b keeps, of each pair of entries b apart, the
// one that bit b of k picks -- so n - 1 selects of log2(n) depth, and one bit test per level shared by
// every call with the same k
template <int NS>
__device__ __forceinline__ double sel_bits(const double (&v)[16], int k, int lo, int n) {
    double r[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) r[j] = (j < n) ? v[(lo + j) & 15] : 0.0;
#pragma unroll
    for (int b = 1; b < NS; b <<= 1) {
#pragma unroll
        for (int j = 0; j + b < NS; j += 2 * b)
            if (j + b < n) r[j] = (k & b) ? r[j + b] : r[j];
    }
    return r[0];
}

__device__ __forceinline__ double neg_if(double x, int neg) {
    // flip the sign bit with an integer op
    long long b = __double_as_longlong(x) ^ ((long long)(neg != 0) << 63);
    return __longlong_as_double(b);
}

// Exact widening of a positive normal float to double with integer operations only (keeps the
// conversion off the FP64 pipe): rebias the exponent (127 -> 1023) and move the 23-bit mantissa up.
__device__ __forceinline__ double widen_pos_normal(float f) {
    const unsigned long long b = (unsigned long long)__float_as_uint(f);
    const unsigned long long e = ((b >> 23) & 0xFFull) + (1023ull - 127ull);
    return __longlong_as_double((long long)((e << 52) | ((b & 0x7FFFFFull) << 29)));
}

// double -> float with integer operations only (the hardware conversion runs on the FP64 pipe):
// keep the sign, rebias the exponent (1023 -> 127), truncate the mantissa to 23 bits; values below
// the normal float range become signed zero, values above it infinity.  Relative error < 2^-23.
__device__ __forceinline__ float narrow_trunc(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FFull) - 1023 + 127;
    const unsigned int m = (unsigned int)(b >> 29) & 0x7FFFFFu;
    unsigned int r = sign | ((unsigned int)e << 23) | m;
    r = (e <= 0) ? sign : r;
    r = (e >= 255) ? (sign | 0x7F800000u) : r;
    return __uint_as_float(r);
}

// float -> double exactly with integer operations; zero and subnormal floats give signed zero.
__device__ __forceinline__ double widen_f(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned int ef = (u >> 23) & 0xFFu;
    const unsigned long long body =
        ((unsigned long long)(ef + (1023u - 127u)) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)(sign | (ef == 0u ? 0ull : body)));
}

// x != 0 without an FP64 compare
__device__ __forceinline__ bool nonzero(double x) {
    return (((unsigned long long)__double_as_longlong(x)) << 1) != 0ull;
}

// sqrt(q), q >= 0: Newton-Raphson on s^2 = q started from the FP32 hardware reciprocal square
// root y ~ 1/sqrt(q) (relative error e0 ~ 1e-7): s <- s + (y/2)(q - s^2).  With the slope held at
// y/2 the error goes e -> -e0 e - e^2/2, so two steps reach FP64 rounding (5 FP64 operations
// instead of the ~9 DADD-equivalents of the IEEE square root on this part).
__device__ __forceinline__ double sqrt_nr(double q) {
    const float y = rsqrtf(fmaxf(narrow_trunc(q), 1.17549435e-38f));
    const double h = widen_pos_normal(0.5f * y);
    double s = q * widen_pos_normal(y);
    s = fma(h, fma(-s, s, q), s);
    s = fma(h, fma(-s, s, q), s);
    return s;
}

// 1/m for m > 0 in a range where m and the FP32 reciprocal are normal floats: Newton-Raphson r <- r + r (1 - m r)
// from the FP32 estimate, two steps (error e -> e^2 each).
__device__ __forceinline__ double rcp_nr(double m) {
    double r = widen_pos_normal(__frcp_rn(narrow_trunc(m)));
    r = fma(r, fma(-m, r, 1.0), r);
    r = fma(r, fma(-m, r, 1.0), r);
    return r;
}

// 1/D for a finite, normal, non-zero D: scale |D| into [1, 2) by exponent arithmetic, take the
// Newton-refined reciprocal there and move the exponent back (4 FP64 operations instead of an
// IEEE division).
__device__ __forceinline__ double rcp_scaled(double D) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(D);
    const long long e = (long long)((b >> 52) & 0x7FFull) - 1023;
    const double m = __longlong_as_double((long long)((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
    const double r = rcp_nr(m);                        // in (1/2, 1]
    const unsigned long long rb = (unsigned long long)__double_as_longlong(r) - ((unsigned long long)e << 52);
    return __longlong_as_double((long long)(rb | (b & 0x8000000000000000ull)));
}

// Bin index and fraction bits of y = (u + 1/2) 2^-32 on nb equal bins: with q = u nb + floor(nb/2) (one
// 32 x 32 -> 64-bit multiply-add), (2u + 1) nb = 2q + (nb & 1), so i = floor(y nb) = q >> 32 and the 33-bit
// fraction of y nb is 2 (q mod 2^32) + (nb & 1): the same integers as the 64-bit product (2u + 1) nb, in
// fewer instructions.  lo = q mod 2^32.
__device__ __forceinline__ void bin_split(uint32_t u, uint32_t nb, uint32_t& i, uint32_t& lo) {
    const uint64_t q = (uint64_t)u * nb + (nb >> 1);
    i = (uint32_t)(q >> 32);
    lo = (uint32_t)q;
}

// Grid entry in shared memory (16 bytes).  FP64 map: (e_i, de_i) in FP64 mode, (e_i - de_i, de_i)
// with the FP32 potentials; FP32 map (MBPT_MIXED): floats (e_i, de_i, -, -).
struct Grid2 {
    double a, de;
};
struct Grid4f {
    float e, de, pad0, pad1;
};


// Result of one sample.
struct SampleOut {
    double w;              // J_vegas * f(x)
    uint32_t binpack[kBinWords];   // bin index of axis a in byte (a & 3) of word a >> 2
    double wc[kComp];      // regulator components (shifted denominators, extrapolation); if n_shifts
};

// V(p, p) and Delta = V(p, p') - V(p, -p') for one vertex, FP32, from P = 2p and P' = 2p'.  The
// difference is formed without cancellation: the contact parts cancel exactly and
// 1/(|P-P'|^2 + 4m^2) - 1/(|P+P'|^2 + 4m^2) = 4 P.P' / ((|P-P'|^2 + 4m^2)(|P+P'|^2 + 4m^2)), so Delta keeps
// FP32 relative accuracy where V_d and V_e nearly agree (small momentum transfer), the region in which
// the exchange cancellation of the spin sum is strongest.
__device__ __forceinline__ void vertex_pot_delta_f32(const DiagRec& R, float Px, float Py, float Pz, float Qx, float Qy,
                                                     float Qz, float& vd, float& dl) {
    const float pp = fmaf(Px, Px, fmaf(Py, Py, Pz * Pz));
    const float qq = fmaf(Qx, Qx, fmaf(Qy, Qy, Qz * Qz));
    const float pq = fmaf(Px, Qx, fmaf(Py, Qy, Pz * Qz));
    const float s = pp + qq;
    const float rd = __fdividef(1.0f, fmaf(-2.0f, pq, s) + R.mpi2_4f);   // 1/(|P - P'|^2 + 4 m^2)
    const float re = __fdividef(1.0f, fmaf(2.0f, pq, s) + R.mpi2_4f);    // 1/(|P + P'|^2 + 4 m^2)
    const float a = pp * R.regc2f, b = qq * R.regc2f;
    float ah = a, bh = b;
    for (int i = 1; i < R.reg_half; ++i) { ah *= a; bh *= b; }
    const float F = exp2f(-(ah + bh));
    vd = fmaf(R.CY4f, rd, R.CSf) * F;
    dl = (R.CY4f * 4.0f * pq) * (rd * re) * F;
}

// V(p, p') for one vertex, FP32, from P = 2p and P' = 2p'.
__device__ __forceinline__ void vertex_pot_f32(const DiagRec& R, float Px, float Py, float Pz, float Qx, float Qy,
                                               float Qz, float& vd, float& ve) {
    const float pp = fmaf(Px, Px, fmaf(Py, Py, Pz * Pz));
    const float qq = fmaf(Qx, Qx, fmaf(Qy, Qy, Qz * Qz));
    const float pq = fmaf(Px, Qx, fmaf(Py, Qy, Pz * Qz));
    const float s = pp + qq;
    const float qd = fmaf(-2.0f, pq, s);      // |P - P'|^2
    const float qe = fmaf(2.0f, pq, s);       // |P + P'|^2
    const float a = pp * R.regc2f, b = qq * R.regc2f;
    float ah = a, bh = b;
    for (int i = 1; i < R.reg_half; ++i) { ah *= a; bh *= b; }
    const float F = exp2f(-(ah + bh));        // exp(-(p/L)^r - (p'/L)^r)
    vd = (R.CSf + __fdividef(R.CY4f, qd + R.mpi2_4f)) * F;
    ve = (R.CSf + __fdividef(R.CY4f, qe + R.mpi2_4f)) * F;
}

// V(p, p') for one vertex, FP64.
__device__ __forceinline__ void vertex_pot_f64(const DiagRec& R, double Px, double Py, double Pz, double Qx,
                                               double Qy, double Qz, double& vd, double& ve) {
    const double pp = fma(Px, Px, fma(Py, Py, Pz * Pz));
    const double qq = fma(Qx, Qx, fma(Qy, Qy, Qz * Qz));
    const double pq = fma(Px, Qx, fma(Py, Qy, Pz * Qz));
    const double s = pp + qq;
    const double qd = fma(-2.0, pq, s);
    const double qe = fma(2.0, pq, s);
    const double a = pp * R.regc, b = qq * R.regc;
    double ah = a, bh = b;
    for (int i = 1; i < R.reg_half; ++i) { ah *= a; bh *= b; }
    const double F = exp(-(ah + bh));
    vd = (R.CS + R.CY4 / (qd + R.mpi2_4)) * F;
    ve = (R.CS + R.CY4 / (qe + R.mpi2_4)) * F;
}

// ---------------------------------------------------------------------------
// One sample of an order-N diagram.
//  s: sample index within the iteration, t: iteration, sid: stream id, (k0,k1): key
//  x_out (optional): the mapped point in [0,1]^d
// ---------------------------------------------------------------------------
// Axes of chord c: map 0 gives every chord (k, cos t, phi) on axes 3c..3c+2.  Map 1 (rotational
// invariance, Sec. III.C) puts chord 0 on the z axis (k only, axis 0) and chord 1 in the xz plane
// (k, cos t on axes 1, 2); chords c >= 2 use axes 3c-3..3c-1.  The fixed angles integrate to
// 4 pi x 2 pi, folded into pref with the other constant Jacobian factors.
template <int MAPK>
__device__ __forceinline__ constexpr int chord_axis(int c) {
    return MAPK == 0 ? 3 * c : (c == 0 ? 0 : (c == 1 ? 1 : 3 * c - 3));
}
template <int MAPK>
__device__ __forceinline__ constexpr int chord_kind(int c) {   // 0 full direction, 1 z axis, 2 xz plane
    return MAPK == 0 ? 0 : (c == 0 ? 1 : (c == 1 ? 2 : 0));
}

// Hartree-Fock self-energy of a line with |k|^2 = u, in units of hbar^2/2m (the spectrum table's cubic
// on the interval of k; 0 beyond the table).  FP32 in the mixed mode, FP64 otherwise.
template <int PREC>
__device__ __forceinline__ double hf_sigma(const DiagRec& R, double u) {
    const float kf = sqrtf(narrow_trunc(u));
    const int i = (int)(kf * R.hf_hinv_f);
    if (i >= R.hf_n) return 0.0;
    if (PREC == MBPT_MIXED) {
        const float* c = R.hf_tab_f + 5 * i;
        const float t = kf - __ldg(c);
        return widen_f(fmaf(fmaf(fmaf(__ldg(c + 4), t, __ldg(c + 3)), t, __ldg(c + 2)), t, __ldg(c + 1)));
    } else {
        const double* c = R.hf_tab + 5 * i;
        const double t = sqrt_nr(u) - __ldg(c);
        return fma(fma(fma(__ldg(c + 4), t, __ldg(c + 3)), t, __ldg(c + 2)), t, __ldg(c + 1));
    }
}

// FP64 chord momenta, |l|^2 and chord Jacobian from an FP64 point x (FP64 and FP64-map modes, and the
// mixed mode's samples near a Fermi surface).  k = lo + rng x0, cos(t) = 2 x1 - 1,
// sin(t) = 2 sqrt(x1 (1 - x1)), rational azimuth a = x2 (1 - x2), b = x2 - 1/2:
// cos(phi) = (a^2 - b^2)/(a^2 + b^2), sin(phi) = 2ab/(a^2 + b^2), dphi/dx2 = 2/(1/2 - a); Jacobian
// k^2 (1/2 - a)/(a^2 + b^2) times the constant 4 rng folded into pref.
template <int N, int PREC, int MAPK, int D>
__device__ __forceinline__ void chords_fp64(const DiagRec& R, const double (&x)[D], double (&K)[3][16],
                                            double (&U)[16], float (&lf)[3][N + 1], double& jc) {
#pragma unroll
    for (int c = 0; c < N + 1; ++c) {
        const int ax = chord_axis<MAPK>(c), kind = chord_kind<MAPK>(c);
        const double k = fma(R.chord_rng[c], x[ax], R.chord_lo[c]);
        const double k2 = k * k;
        if (kind == 1) {
            K[0][c] = 0.0;
            K[1][c] = 0.0;
            K[2][c] = k;
            jc *= k2;
        } else if (kind == 2) {
            const double x1 = x[ax + 1];
            const double ct = fma(2.0, x1, -1.0);
            const double sq = sqrt_nr(fma(-x1, x1, x1));
            K[0][c] = (k + k) * sq;
            K[1][c] = 0.0;
            K[2][c] = k * ct;
            jc *= k2;
        } else {
            const double x1 = x[ax + 1], x2 = x[ax + 2];
            const double ct = fma(2.0, x1, -1.0);
            const double sq = sqrt_nr(fma(-x1, x1, x1));
            const double a = fma(-x2, x2, x2);
            const double b = x2 - 0.5;
            const double bb = b * b;
            const double mm = fma(a, a, bb);
            const double rr = rcp_nr(mm);           // mm = (1/2 - a)^2 in [1/16, 1/4]
            const double ncos = fma(a, a, -bb);
            const double nsin = (a + a) * b;
            const double R2 = (k + k) * sq * rr;
            K[0][c] = R2 * ncos;
            K[1][c] = R2 * nsin;
            K[2][c] = k * ct;
            jc *= k2 * ((0.5 - a) * rr);
        }
        U[c] = k2;
        if (PREC != MBPT_FP64) {
            lf[0][c] = narrow_trunc(K[0][c]);
            lf[1][c] = narrow_trunc(K[1][c]);
            lf[2][c] = narrow_trunc(K[2][c]);
        }
    }
}

// FP32 front of a mixed-precision sample: the VEGAS map on the FP32 grid (point, bins), chord
// magnitudes, unit directions (kind 1: along z; kind 2: in the xz plane; kind 0: rational azimuth) and
// FP32 chord momenta; the VEGAS and chord Jacobians as one mantissa product and exponent sum (so that
// it cannot underflow; a zero or subnormal factor sets zero_bin).
// GRID selects the shared-memory grid: 0 the FP32 grid of the mixed mode (e, de); 1 the FP64 grid of
// the FP64 mode (x = a + frac de); 2 the FP64 grid of the FP64-map mode (x = a + (1 + frac) de).  With
// an FP64 grid the point is an FP32 approximation of the one the exact path uses (for the pre-test
// only), and the Jacobian outputs are not computed.
template <int N, int MAPK, int D, int GRID = 0>
__device__ __forceinline__ void mixed_front(const DiagRec& R, const Grid2* __restrict__ gs, const uint32_t* u,
                                            uint32_t nb, float (&xf)[D], uint32_t (&binpack)[kBinWords], float& mp,
                                            int& ex, bool& zero_bin, float (&kmag)[N + 1],
                                            float (&kdir)[3][N + 1], float (&lf)[3][N + 1]) {
    mp = 1.0f;
    ex = 0;
    zero_bin = false;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        uint32_t i, lo;
        bin_split(u[a], nb, i, lo);
        const uint32_t fb = lo >> 9;                                       // top 23 bits of the fraction
        const float frac = __uint_as_float(0x3F800000u | fb) - 1.0f;
        if constexpr (GRID == 0) {
            const Grid4f g = reinterpret_cast<const Grid4f*>(gs)[a * grid_stride(D) + i];
            xf[a] = fmaf(frac, g.de, g.e);
            const uint32_t bits = __float_as_uint(g.de);
            zero_bin |= (bits == 0u);
            ex += (int)(bits >> 23) - 127;
            mp *= __uint_as_float((bits & 0x7FFFFFu) | 0x3F800000u);
        } else {
            const Grid2 g = gs[a * grid_stride(D) + i];
            xf[a] = fmaf(GRID == 1 ? frac : 1.0f + frac, narrow_trunc(g.de), narrow_trunc(g.a));
        }
        binpack[a >> 2] |= i << (8 * (a & 3));
    }
#pragma unroll
    for (int c = 0; c < N + 1; ++c) {
        const int ax = chord_axis<MAPK>(c), kind = chord_kind<MAPK>(c);
        const float k = fmaf(R.chord_rng_f[c], xf[ax], R.chord_lo_f[c]);
        kmag[c] = k;
        float jc;
        if (kind == 1) {
            kdir[0][c] = 0.0f;
            kdir[1][c] = 0.0f;
            kdir[2][c] = 1.0f;
            jc = k * k;
        } else if (kind == 2) {
            const float x1 = xf[ax + 1];
            kdir[0][c] = 2.0f * sqrtf(fmaf(-x1, x1, x1));
            kdir[1][c] = 0.0f;
            kdir[2][c] = fmaf(2.0f, x1, -1.0f);
            jc = k * k;
        } else {
            const float x1 = xf[ax + 1], x2 = xf[ax + 2];
            const float ct = fmaf(2.0f, x1, -1.0f);
            const float sq = sqrtf(fmaf(-x1, x1, x1));
            const float a = fmaf(-x2, x2, x2);
            const float b = x2 - 0.5f;
            const float bb = b * b;
            const float mm = fmaf(a, a, bb);
            const float rr = __frcp_rn(mm);
            const float R2 = 2.0f * sq * rr;
            kdir[0][c] = R2 * fmaf(a, a, -bb);
            kdir[1][c] = R2 * ((a + a) * b);
            kdir[2][c] = ct;
            jc = k * k * ((0.5f - a) * rr);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) lf[q][c] = k * kdir[q][c];
        if constexpr (GRID == 0) {
            const uint32_t jb = __float_as_uint(jc);
            zero_bin |= (jb & 0x7F800000u) == 0u;
            ex += (int)(jb >> 23) - 127;
            mp *= __uint_as_float((jb & 0x7FFFFFu) | 0x3F800000u);
        }
    }
}

// Fermi-step pre-test in FP32 of the mixed mode.  Returns true when some line fails its step for
// every species by more than the FP32 error bound of |k|^2: the sample is zero.  Bound: the FP32
// chord components are within 2^-24 of the exact FP64 products that the exact path uses, a line is
// accumulated from at most N+1 chords by fused multiply-adds with coefficients -1..1, so with
// S_l = sum over its chords of |coefficient| |k_c|, |k_f^2 - k^2| < 2^-19 S_l^2; the margin is
// 2^-16 S_l^2 plus 2^-20 kF^2 for the FP32 copy of kF^2.  near: some line lies within the margin plus
// near_f kF^2 of a Fermi surface (the band in which the caller places the sample with the FP64 map;
// 2^-10 up to fourth order, 2^-7 from fifth order on by default).
// SLACK (FP64 and FP64-map modes, whose exact path places the sample with the FP64 map): the FP32
// point differs from the FP64 one by < 2^-20 per axis, which moves a chord magnitude by
// < 2^-18 (rng + k) and its unit direction by < 2^-7 (the sin(theta) = 2 sqrt(x1 (1 - x1)) factor is
// only 1/2-Hoelder: a change d of x1 moves it by < 2 sqrt(d)), so the line moves by
// < 2^-6.9 S_l + 2^-18 Q_l with Q_l = sum of |coefficient| rng_c, and |k|^2 by < 2^-5.9 S_l^2 +
// 2^-17 S_l Q_l + (that)^2; the margin adds 2^-5 S_l^2 + 2^-16 S_l Q_l.
template <int N, bool SLACK = false>
__device__ __forceinline__ bool pretest_dead(const DiagRec& R, const float (&lf)[3][N + 1],
                                             const float (&kmag)[N + 1], bool& near) {
    constexpr int L = N + 1;
    bool dead = false;
    near = false;
#pragma unroll
    for (int l = 0; l < 2 * N; ++l) {
        float x, y, z, S;
        float Q = 0.0f;
        if (l < L) {
            x = lf[0][l];
            y = lf[1][l];
            z = lf[2][l];
            S = kmag[l];
            if (SLACK) Q = R.chord_rng_f[l];
        } else {
            x = 0.0f;
            y = 0.0f;
            z = 0.0f;
            S = 0.0f;
#pragma unroll
            for (int c = 0; c < L; ++c) {
                const float cf = R.tcoef[l - L][c];
                x = fmaf(cf, lf[0][c], x);
                y = fmaf(cf, lf[1][c], y);
                z = fmaf(cf, lf[2][c], z);
                S = fmaf(fabsf(cf), kmag[c], S);
                if (SLACK) Q = fmaf(fabsf(cf), R.chord_rng_f[c], Q);
            }
        }
        const float uf = fmaf(x, x, fmaf(y, y, z * z));
        float mg = 1.52587890625e-05f * S * S;
        if (SLACK) mg = fmaf(0.03125f * S, S, fmaf(1.52587890625e-05f * S, Q, mg));
        const bool hole = (R.hole_slots >> l) & 1u;
        const float mn = fmaf(9.5367431640625e-07f, R.kf2_nf, mg);
        const float dn = uf - R.kf2_nf;
        bool f = hole ? (dn > mn) : (dn < -mn);
        bool nr = fabsf(dn) <= fmaf(R.near_f, R.kf2_nf, mn);
        if (R.asym) {
            const float mp2 = fmaf(9.5367431640625e-07f, R.kf2_pf, mg);
            const float dp = uf - R.kf2_pf;
            f = f && (hole ? (dp > mp2) : (dp < -mp2));
            nr = nr || (fabsf(dp) <= fmaf(R.near_f, R.kf2_pf, mp2));
        }
        if (l >= L) dead |= f;    // a chord lies in its own step's range (hole chords in [0, kF_max], particle
                                  // chords in [kF_min, K_max]) and passes it for some species
        near |= nr;
    }
    return dead;
}

// Spin sum of one Fermi momentum in FP32 (mixed precision): products of V_d and Delta = V_d - V_e over
// the vertices, summed with the difference-form table gdel_f.  P_v = k_o1 - k_o2 and P'_v = k_i1 - k_i2
// from the FP32 chord momenta lf.
template <int N>
__device__ __forceinline__ float spin_sum_diff_f32(const DiagRec& R, const float (&lf)[3][N + 1]) {
    constexpr int L = N + 1;
    float prod[1 << N];
    prod[0] = 1.0f;
#pragma unroll
    for (int v = 0; v < N; ++v) {
        float P[3], Q[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float p = 0.0f, qq = 0.0f;
#pragma unroll
            for (int c = 0; c < L; ++c) {
                p = fmaf(R.vcoef_out[v][c], lf[q][c], p);
                qq = fmaf(R.vcoef_in[v][c], lf[q][c], qq);
            }
            P[q] = p;
            Q[q] = qq;
        }
        float vd, dl;
        vertex_pot_delta_f32(R, P[0], P[1], P[2], Q[0], Q[1], Q[2], vd, dl);
#pragma unroll
        for (int j = 0; j < (1 << v); ++j) {
            prod[j + (1 << v)] = prod[j] * dl;
            prod[j] *= vd;
        }
    }
    float sum = 0.0f;
#pragma unroll
    for (int tt = 0; tt < (1 << N); ++tt) sum = fmaf(R.gdel_f[tt], prod[tt], sum);
    return sum;
}

// The same sum folded vertex by vertex (the Horner form of the multilinear polynomial, MBPT_SPIN_FOLD): the
// table index's bit v selects Delta_v over V_v, so folding vertex 0 pairs entries 2b and 2b + 1 into
// T(b) = c'(2b) V_0 + c'(2b + 1) Delta_0, and every later vertex folds the remaining table the same way;
// after n folds one entry, the sum, is left.  2 (2^n - 1) FP32 operations against the 2^(n+1) - 4 products
// and 2^n fused multiply-adds of the table, and at most 2^(n-1) partial sums live.
template <int N>
__device__ __forceinline__ float spin_sum_fold_f32(const DiagRec& R, const float (&lf)[3][N + 1]) {
    constexpr int L = N + 1;
    float T[1 << (N - 1)];
#pragma unroll
    for (int v = 0; v < N; ++v) {
        float P[3], Q[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float p = 0.0f, qq = 0.0f;
#pragma unroll
            for (int c = 0; c < L; ++c) {
                p = fmaf(R.vcoef_out[v][c], lf[q][c], p);
                qq = fmaf(R.vcoef_in[v][c], lf[q][c], qq);
            }
            P[q] = p;
            Q[q] = qq;
        }
        float vd, dl;
        vertex_pot_delta_f32(R, P[0], P[1], P[2], Q[0], Q[1], Q[2], vd, dl);
#pragma unroll
        for (int b = 0; b < (1 << (N - 1 - v)); ++b) {
            if (v == 0) T[b] = fmaf(R.gdel_f[2 * b + 1], dl, R.gdel_f[2 * b] * vd);
            else T[b] = fmaf(T[2 * b + 1], dl, T[2 * b] * vd);
        }
    }
    return T[0];
}

// Spin-isospin sum in asymmetric matter, FP32: products of V_d and V_e over the vertices, each Goldstone
// term weighted by its loop factors, which depend on the per-line Fermi steps of both species (bit l of
// okn / okp: line l passes its neutron / proton step).
template <int N>
__device__ __forceinline__ float spin_sum_asym_f32(const DiagRec& R, const float (&lf)[3][N + 1], uint32_t okn,
                                                   uint32_t okp) {
    constexpr int L = N + 1;
    float prod[1 << N];
    prod[0] = 1.0f;
#pragma unroll
    for (int v = 0; v < N; ++v) {
        float P[3], Q[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float p = 0.0f, qq = 0.0f;
#pragma unroll
            for (int c = 0; c < L; ++c) {
                p = fmaf(R.vcoef_out[v][c], lf[q][c], p);
                qq = fmaf(R.vcoef_in[v][c], lf[q][c], qq);
            }
            P[q] = p;
            Q[q] = qq;
        }
        float vd, ve;
        vertex_pot_f32(R, P[0], P[1], P[2], Q[0], Q[1], Q[2], vd, ve);
#pragma unroll
        for (int j = 0; j < (1 << v); ++j) {
            prod[j + (1 << v)] = prod[j] * ve;
            prod[j] *= vd;
        }
    }
    float sum = 0.0f;
#pragma unroll
    for (int tt = 0; tt < (1 << N); ++tt) {
        float f = R.gsign_f[tt];
        const int nlp = R.nloops[tt];
        for (int lp = 0; lp < nlp; ++lp) {
            const uint32_t msk = R.loop_mask[tt][lp];
            const int fn = (msk & ~okn) == 0u;
            const int fp = (msk & ~okp) == 0u;
            f *= (float)(2 * (fn + fp));
        }
        sum = fmaf(f, prod[tt], sum);
    }
    return sum;
}

// Classes of a sample after the FP32 front and pre-test (sample_class): zero, live away from every Fermi
// surface, live near one (mixed mode: placed with the FP64 map); kClassUnknown: not classified.
constexpr int kClassZero = 0, kClassFar = 1, kClassNear = 2, kClassUnknown = 3;

// REG: the integral carries the denominator regulator (a separate instantiation, so that the
// registers of the plain integrand are not spent on it).
template <int N, int PREC, int MAPK, bool REG>
__device__ __forceinline__ SampleOut eval_sample(const DiagRec& R, const Grid2* __restrict__ gs,
                                                 const double* __restrict__ grid64, uint32_t s, uint32_t t,
                                                 uint32_t sid, uint32_t k0, uint32_t k1, double* x_out,
                                                 int known = kClassUnknown, uint32_t spin = MBPT_SPIN_TABLE) {
    constexpr int L = N + 1;          // chords
    constexpr int D = 3 * L - 3 * MAPK;   // dimensions
    constexpr int NL = 2 * N;         // lines
    constexpr int NBLK = (D + 3) / 4; // Philox blocks
    SampleOut o;
    const uint32_t nb = (uint32_t)R.nb;

    // --- counter-based random numbers
    uint32_t u[4 * NBLK];
#pragma unroll
    for (int j = 0; j < NBLK; ++j) philox4x32_10(s, t, sid, (uint32_t)j, k0, k1, &u[4 * j]);

    // --- VEGAS map: y = (u + 1/2) 2^-32, i = floor(y nb), x = e_i + (y nb - i) de_i, J = prod nb de_i
    // (nb^d is folded into pref).  (2u+1) nb < 2^39, so the bin index and the fraction are exact
    // integer arithmetic.
    // --- chord momenta (chords_fp64, mixed_front)
    double K[3][16];
    double U[16];
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        K[0][l] = 0.0;
        K[1][l] = 0.0;
        K[2][l] = 0.0;
        U[l] = 0.0;
    }
    float lf[3][L];           // chord momenta in FP32 for the potentials
    double jv = 1.0, jc = 1.0;
#pragma unroll
    for (int w = 0; w < kBinWords; ++w) o.binpack[w] = 0;
    if (PREC == MBPT_MIXED) {
        // Sampling map in FP32.  It only decides where the sample lies: each chord momentum is the
        // exact FP64 product of an FP32 magnitude and an FP32 unit direction, so lines, steps and
        // energy denominators below are evaluated in FP64 at that point; the map's Jacobian is
        // good to FP32 rounding (a relative weight error ~1e-7 per sample).  Samples whose lines
        // come within ~1e-3 kF^2 of a Fermi surface -- where the energy denominators can vanish and
        // a step decision could depend on where the FP32 map rounds the point -- are placed with the
        // FP64 map instead (the FP64 mode's point, bins unchanged).
        // known: the caller has already classified the sample (sample_class): near a surface, or away
        // from every surface and not dead (the pre-test below would find the same, so it is skipped).
        const bool force64 = known == kClassNear;
        float xf[D];
        float mp = 1.0f;
        int ex = 0;
        bool zero_bin = false;
        float kmag[L], kdir[3][L];
        bool near = force64;
        if (!force64) mixed_front<N, MAPK, D>(R, gs, u, nb, xf, o.binpack, mp, ex, zero_bin, kmag, kdir, lf);
        if (known == kClassUnknown && pretest_dead<N>(R, lf, kmag, near)) {
            if (x_out) {
#pragma unroll
                for (int a = 0; a < D; ++a) x_out[a] = widen_f(xf[a]);
            }
            o.w = 0.0;
            if (REG) {
#pragma unroll
                for (int k = 0; k < kComp; ++k) o.wc[k] = 0.0;
            }
            return o;
        }
        if (near) {
            double x[D];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                uint32_t i, lo;
                bin_split(u[a], nb, i, lo);
                const uint64_t fb = ((uint64_t)lo << 1) | (uint64_t)(nb & 1u);   // the 33 fraction bits
                const double m = __longlong_as_double((long long)(0x3FF0000000000000ull | (fb << 19)));
                const double e0 = grid64[a * (nb + 1) + i];
                const double de = grid64[a * (nb + 1) + i + 1] - e0;
                x[a] = fma(m - 1.0, de, e0);
                jv *= de;
                o.binpack[a >> 2] |= i << (8 * (a & 3));
                if (x_out) x_out[a] = x[a];
            }
            chords_fp64<N, MBPT_MIXED, MAPK, D>(R, x, K, U, lf, jc);
            jv = R.pref * (jv * jc);
        } else {
            if (x_out) {
#pragma unroll
                for (int a = 0; a < D; ++a) x_out[a] = widen_f(xf[a]);
            }
            // the weight's constant factor, VEGAS and chord Jacobians together (mixed_front): one FP32
            // mantissa product and an exponent sum, no FP64 work
            jv = (zero_bin || R.pref_mf == 0.0f)
                     ? 0.0
                     : __longlong_as_double(
                                (long long)((unsigned long long)(__double_as_longlong(widen_pos_normal(mp * R.pref_mf)) +
                                                                 ((long long)(ex + R.pref_e) << 52)) |
                                            ((unsigned long long)R.pref_sign_hi << 32)));
            // exact FP64 chord momenta: products of the FP32 magnitude and direction (24 x 24 bits)
#pragma unroll
            for (int c = 0; c < L; ++c) {
                const int kind = chord_kind<MAPK>(c);
                const double kd = widen_f(kmag[c]);
                if (kind == 1) {
                    K[0][c] = 0.0;
                    K[1][c] = 0.0;
                    K[2][c] = kd;
                    U[c] = kd * kd;
                } else if (kind == 2) {
                    K[0][c] = kd * widen_f(kdir[0][c]);
                    K[1][c] = 0.0;
                    K[2][c] = kd * widen_f(kdir[2][c]);
                    U[c] = fma(K[0][c], K[0][c], K[2][c] * K[2][c]);
                } else {
                    K[0][c] = kd * widen_f(kdir[0][c]);
                    K[1][c] = kd * widen_f(kdir[1][c]);
                    K[2][c] = kd * widen_f(kdir[2][c]);
                    U[c] = fma(K[0][c], K[0][c], fma(K[1][c], K[1][c], K[2][c] * K[2][c]));
                }
            }
        }
    } else {
        double x[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            uint32_t i, lo;
            bin_split(u[a], nb, i, lo);
            const uint64_t fb = ((uint64_t)lo << 1) | (uint64_t)(nb & 1u);   // the 33 fraction bits
            const double m = __longlong_as_double((long long)(0x3FF0000000000000ull | (fb << 19)));   // 1 + frac
            const Grid2 g = gs[a * grid_stride(D) + i];
            if (PREC == MBPT_FP64) x[a] = fma(m - 1.0, g.de, g.a);
            else x[a] = fma(m, g.de, g.a);
            jv *= g.de;
            o.binpack[a >> 2] |= i << (8 * (a & 3));
            if (x_out) x_out[a] = x[a];
        }
        chords_fp64<N, PREC, MAPK, D>(R, x, K, U, lf, jc);
        jv = R.pref * (jv * jc);
    }

    // --- spin sum of one Fermi momentum, FP32, before the FP64 work: it needs only the FP32 chord momenta,
    // which are then no longer live through the FP64 section (fewer spills; measured 5 % faster at
    // fifth order).  Asymmetric matter needs the Fermi steps of every line and sums below.
    const float s_f32 = (PREC != MBPT_FP64 && !R.asym)
                            ? (spin == MBPT_SPIN_FOLD ? spin_sum_fold_f32<N>(R, lf) : spin_sum_diff_f32<N>(R, lf))
                            : 0.0f;

    // --- tree lines from momentum conservation: k = k_a + k_b - k_c
#pragma unroll
    for (int j = 0; j < N - 1; ++j) {
        const int ia = R.tree_a[j], ib = R.tree_b[j], ic = R.tree_c[j];
#pragma unroll
        for (int q = 0; q < 3; ++q)
            K[q][L + j] = (sel_bits<NL>(K[q], ia, 0, L + j) + sel_bits<NL>(K[q], ib, 0, L + j)) -
                          sel_bits<NL>(K[q], ic, 0, L + j);
        U[L + j] = fma(K[0][L + j], K[0][L + j], fma(K[1][L + j], K[1][L + j], K[2][L + j] * K[2][L + j]));
    }

    // --- Fermi-sea steps: hole k^2 < kF^2, particle k^2 >= kF^2 (non-negative doubles compare
    // as their bit patterns)
    uint32_t okn = 0, okp = 0;
    if (PREC == MBPT_MIXED && known == kClassFar && !R.asym) {
        // classified away from the Fermi surface: the pre-test found every line on its passing side by
        // more than the near band, far beyond the error of its FP32 |k|^2
        okn = R.all_slots;
    } else {
        const long long bn = __double_as_longlong(R.kf2_n), bp = __double_as_longlong(R.kf2_p);
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const long long bu = __double_as_longlong(U[l]);
            const bool hole = (R.hole_slots >> l) & 1u;
            const bool on = hole ? (bu < bn) : (bu >= bn);
            const bool op = hole ? (bu < bp) : (bu >= bp);
            okn |= (uint32_t)on << l;
            okp |= (uint32_t)op << l;
        }
    }
    const uint32_t all = R.all_slots;
    bool live;
    if (R.asym) live = ((okn | okp) == all);
    else live = (okn == all);
    if (!live) {
        o.w = 0.0;
        if (REG) {
#pragma unroll
            for (int k = 0; k < kComp; ++k) o.wc[k] = 0.0;
        }
        return o;
    }

    // --- Hartree-Fock spectrum (Eq. (7)): single-particle energy (hbar^2/2m)(|k|^2 + Sigma~(|k|)) on every
    // line; the Fermi steps above test |k|^2 itself
    if (R.spectrum) {
#pragma unroll
        for (int l = 0; l < NL; ++l) U[l] += hf_sigma<PREC>(R, U[l]);
    }

    // --- energy denominators (FP64): D~_m = D~_{m-1} + sum over the four lines of vertex m
    double Dprod = 1.0;
    double Dcut[(REG && N > 1) ? N - 1 : 1];
    {
        double Dm = 0.0;
#pragma unroll
        for (int m = 0; m < N - 1; ++m) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double uv = neg_if(sel_bits<NL>(U, R.cut_slot[m][k] - k, k, NL - 3), R.cut_neg[m][k]);
                if (m == 0 && k == 0) Dm = uv;
                else Dm += uv;
            }
            if (REG) Dcut[m] = Dm;
            Dprod = (m == 0) ? Dm : Dprod * Dm;
        }
    }

    // --- spin(-isospin) sum of the antisymmetrised vertex products
    double S;
    if (PREC != MBPT_FP64 && !R.asym) {
        S = widen_f(s_f32);
    } else if (PREC != MBPT_FP64) {
        // asymmetric matter (per-sample loop factors): products of V_d and V_e
        S = widen_f(spin_sum_asym_f32<N>(R, lf, okn, okp));
    } else {
        double prod[1 << N];
        prod[0] = 1.0;
#pragma unroll
        for (int v = 0; v < N; ++v) {
            double P[3], Q[3];
            const int o1 = R.port_slot[v][0], o2 = R.port_slot[v][1], i1 = R.port_slot[v][2], i2 = R.port_slot[v][3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                P[q] = sel_bits<NL>(K[q], o1, 0, NL) - sel_bits<NL>(K[q], o2, 0, NL);
                Q[q] = sel_bits<NL>(K[q], i1, 0, NL) - sel_bits<NL>(K[q], i2, 0, NL);
            }
            double vd, ve;
            vertex_pot_f64(R, P[0], P[1], P[2], Q[0], Q[1], Q[2], vd, ve);
#pragma unroll
            for (int j = 0; j < (1 << v); ++j) {
                prod[j + (1 << v)] = prod[j] * ve;
                prod[j] *= vd;
            }
        }
        double sum = 0.0;
        if (!R.asym) {
#pragma unroll
            for (int tt = 0; tt < (1 << N); ++tt) sum = fma(R.gcoef_d[tt], prod[tt], sum);
        } else {
#pragma unroll
            for (int tt = 0; tt < (1 << N); ++tt) {
                float f = R.gsign_f[tt];
                const int nlp = R.nloops[tt];
                for (int lp = 0; lp < nlp; ++lp) {
                    const uint32_t msk = R.loop_mask[tt][lp];
                    const int fn = (msk & ~okn) == 0u;
                    const int fp = (msk & ~okp) == 0u;
                    f *= (float)(2 * (fn + fp));
                }
                sum = fma((double)f, prod[tt], sum);
            }
        }
        S = sum;
    }

    // --- weight: w = pref * J_vegas * J_chords * S / prod_m D~_m, jv holding pref * J_vegas * J_chords.
    // A spin sum that is exactly zero (asymmetric matter: every line passes its step for some species,
    // but no species assignment is consistent along the loops, e.g. a hole and a particle of equal
    // momentum in different species) gives zero; the cut of such a pair can have D = 0, so the
    // division is skipped.
    if (!nonzero(S)) o.w = 0.0;
    else if (PREC == MBPT_FP64) o.w = (jv * S) / Dprod;
    else o.w = (jv * S) * rcp_scaled(Dprod);
    // --- denominator regulator: every D~_m -> D~_m - eta_k (pole moved away from the domain), and
    // the quadratic through the three components evaluated at zero shift
    if constexpr (REG) {
        const double num = nonzero(S) ? jv * S : 0.0;
        double ext = 0.0;
#pragma unroll
        for (int k = 0; k < kShifts; ++k) {
            double P = 1.0;
#pragma unroll
            for (int m = 0; m < N - 1; ++m) P *= (Dcut[m] - R.eta[k]);
            const double wk = nonzero(num) ? ((PREC == MBPT_FP64) ? num / P : num * rcp_scaled(P)) : 0.0;
            o.wc[k] = wk;
            ext = fma(R.lag[k], wk, ext);
        }
        o.wc[kShifts] = ext;
    }
    return o;
}

// Class of sample s after an FP32 front and Fermi-step pre-test (Philox and FP32 work only):
// 0 zero (eval_sample would find it zero), 1 live or undecided (mixed mode: and away from every Fermi
// surface, FP32 placement), 2 (mixed mode) near a surface, placed with the FP64 map.  In the FP64 and
// FP64-map modes the pre-test works on an FP32 approximation of the FP64 point, with the extra
// margin for the difference, and every survivor is class 1.
template <int N, int MAPK, int PREC>
__device__ __forceinline__ int sample_class(const DiagRec& R, const Grid2* __restrict__ gs, uint32_t s, uint32_t t,
                                            uint32_t sid, uint32_t k0, uint32_t k1) {
    constexpr int L = N + 1;
    constexpr int D = 3 * L - 3 * MAPK;
    constexpr int NBLK = (D + 3) / 4;
    constexpr int GRID = PREC == MBPT_MIXED ? 0 : (PREC == MBPT_FP64 ? 1 : 2);
    uint32_t u[4 * NBLK];
#pragma unroll
    for (int j = 0; j < NBLK; ++j) philox4x32_10(s, t, sid, (uint32_t)j, k0, k1, &u[4 * j]);
    float xf[D];
    uint32_t bp[kBinWords] = {};
    float mp, kmag[L], kdir[3][L], lf[3][L];
    int ex;
    bool zero_bin, near;
    mixed_front<N, MAPK, D, GRID>(R, gs, u, (uint32_t)R.nb, xf, bp, mp, ex, zero_bin, kmag, kdir, lf);
    if (pretest_dead<N, GRID != 0>(R, lf, kmag, near)) return kClassZero;
    return (GRID == 0 && near) ? kClassNear : kClassFar;
}

}  // namespace mbpt
