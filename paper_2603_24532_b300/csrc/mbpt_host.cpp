// Host side of libmbpt: the diagram generator (Table I of arXiv:2603.24532),
// descriptor validation and the compilation of a descriptor + physics point +
// VEGAS setup into the device record DiagRec.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <array>
#include <map>
#include <vector>

#include "mbpt_internal.h"

namespace mbpt {
namespace {

using Mat = std::array<int8_t, 36>;   // row-major n x n, n <= 6

void fill_rows(int n, int i, std::vector<std::array<int8_t, 6>>& rows) {
    // all rows with zero at i, non-negative entries summing to 2, ascending lexicographic order
    rows.clear();
    std::vector<std::array<int8_t, 6>> tmp;
    for (int a = 0; a < n; ++a) {
        if (a == i) continue;
        for (int b = a; b < n; ++b) {
            if (b == i) continue;
            std::array<int8_t, 6> r{};
            r[a] += 1;
            r[b] += 1;
            tmp.push_back(r);
        }
    }
    std::sort(tmp.begin(), tmp.end(), [n](const std::array<int8_t, 6>& x, const std::array<int8_t, 6>& y) {
        for (int k = 0; k < n; ++k)
            if (x[k] != y[k]) return x[k] < y[k];
        return false;
    });
    rows = tmp;
}

bool connected(int n, const Mat& A) {
    int seen = 1, stack[6], sp = 0;
    stack[sp++] = 0;
    while (sp) {
        int v = stack[--sp];
        for (int u = 0; u < n; ++u)
            if ((A[v * n + u] || A[u * n + v]) && !(seen >> u & 1)) {
                seen |= 1 << u;
                stack[sp++] = u;
            }
    }
    return seen == (1 << n) - 1;
}

void enumerate_rec(int n, int i, Mat& A, int colsum[6], const std::vector<std::vector<std::array<int8_t, 6>>>& rows,
                   std::vector<Mat>& out) {
    if (i == n) {
        for (int j = 0; j < n; ++j)
            if (colsum[j] != 2) return;
        if (connected(n, A)) out.push_back(A);
        return;
    }
    for (const auto& r : rows[i]) {
        bool ok = true;
        for (int j = 0; j < n; ++j)
            if (colsum[j] + r[j] > 2) { ok = false; break; }
        if (!ok) continue;
        for (int j = 0; j < n; ++j) { A[i * n + j] = r[j]; colsum[j] += r[j]; }
        enumerate_rec(n, i + 1, A, colsum, rows, out);
        for (int j = 0; j < n; ++j) { colsum[j] -= r[j]; A[i * n + j] = 0; }
    }
}

std::vector<Mat> all_matrices(int n) {
    std::vector<std::vector<std::array<int8_t, 6>>> rows(n);
    for (int i = 0; i < n; ++i) fill_rows(n, i, rows[i]);
    std::vector<Mat> out;
    Mat A{};
    int colsum[6] = {0};
    enumerate_rec(n, 0, A, colsum, rows, out);
    return out;   // nested loops over lexicographically sorted rows: already in row-major lexicographic order
}

int find_root(int* parent, int a) {
    while (parent[a] != a) a = parent[a] = parent[parent[a]];
    return a;
}

// Momentum routing: for chord c, walk the tree path from the chord's end back to its start;
// tree lines traversed along their arrow get +1, against it -1.
bool route_chords(int n, int nl, const int8_t* src, const int8_t* dst, const int8_t* chords, int nc,
                  int8_t coef[MBPT_MAX_LINES][MBPT_MAX_CHORDS]) {
    bool is_chord[MBPT_MAX_LINES] = {false};
    for (int c = 0; c < nc; ++c) is_chord[chords[c]] = true;
    for (int l = 0; l < nl; ++l)
        for (int c = 0; c < MBPT_MAX_CHORDS; ++c) coef[l][c] = 0;
    for (int c = 0; c < nc; ++c) {
        int lc = chords[c];
        coef[lc][c] = 1;
        // BFS over tree lines from dst(lc) to src(lc)
        int prev_line[6], prev_v[6];
        for (int v = 0; v < n; ++v) prev_line[v] = -2;
        int q[6], qh = 0, qt = 0;
        int start = dst[lc], goal = src[lc];
        prev_line[start] = -1;
        q[qt++] = start;
        while (qh < qt) {
            int v = q[qh++];
            for (int l = 0; l < nl; ++l) {
                if (is_chord[l]) continue;
                int u = -1;
                if (src[l] == v) u = dst[l];
                else if (dst[l] == v) u = src[l];
                if (u < 0 || prev_line[u] != -2) continue;
                prev_line[u] = l;
                prev_v[u] = v;
                q[qt++] = u;
            }
        }
        if (prev_line[goal] == -2) return false;
        for (int v = goal; v != start; v = prev_v[v]) {
            int l = prev_line[v];
            int from = prev_v[v];
            // traversal goes from `from` to `v`
            if (src[l] == from && dst[l] == v) coef[l][c] += 1;
            else coef[l][c] -= 1;
        }
    }
    return true;
}

void build_desc(int n, const Mat& A, int id, mbpt_diagram_desc& d) {
    memset(&d, 0, sizeof(d));
    d.order = n;
    d.n_lines = 2 * n;
    int nl = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < A[i * n + j]; ++k) {
                d.line_src[nl] = (int8_t)i;
                d.line_dst[nl] = (int8_t)j;
                ++nl;
            }
    for (int v = 0; v < n; ++v) {
        int no = 0, ni = 0;
        for (int l = 0; l < nl; ++l) {
            if (d.line_src[l] == v) d.vtx_out[v][no++] = (int8_t)l;
            if (d.line_dst[l] == v) d.vtx_in[v][ni++] = (int8_t)l;
        }
    }
    int parent[6];
    for (int v = 0; v < n; ++v) parent[v] = v;
    int order_l[MBPT_MAX_LINES], no = 0;
    for (int l = 0; l < nl; ++l) if (d.line_src[l] < d.line_dst[l]) order_l[no++] = l;
    for (int l = 0; l < nl; ++l) if (d.line_src[l] > d.line_dst[l]) order_l[no++] = l;
    bool chord[MBPT_MAX_LINES] = {false};
    for (int k = 0; k < nl; ++k) {
        int l = order_l[k];
        int a = find_root(parent, d.line_src[l]), b = find_root(parent, d.line_dst[l]);
        if (a == b) chord[l] = true;
        else parent[a] = b;
    }
    // hole chords first, then particle chords, each in line order: diagrams with the same number of hole
    // chords then map a sampled point to the same loop momenta (aligned group members)
    int nc = 0;
    for (int l = 0; l < nl; ++l) if (chord[l] && d.line_src[l] > d.line_dst[l]) d.chord_line[nc++] = (int8_t)l;
    for (int l = 0; l < nl; ++l) if (chord[l] && d.line_src[l] < d.line_dst[l]) d.chord_line[nc++] = (int8_t)l;
    d.n_chords = (int8_t)nc;
    route_chords(n, nl, d.line_src, d.line_dst, d.chord_line, nc, d.line_coef);
    d.diagram_id = id;
}

bool anomalous(const mbpt_diagram_desc& d) {
    int nl = d.n_lines, nc = d.n_chords;
    for (int a = 0; a < nl; ++a) {
        if (!(d.line_src[a] > d.line_dst[a])) continue;
        for (int b = 0; b < nl; ++b) {
            if (!(d.line_src[b] < d.line_dst[b])) continue;
            bool eq = true, neg = true;
            for (int c = 0; c < nc; ++c) {
                if (d.line_coef[a][c] != d.line_coef[b][c]) eq = false;
                if (d.line_coef[a][c] != -d.line_coef[b][c]) neg = false;
            }
            if (eq || neg) return true;
        }
    }
    return false;
}

// Two cuts whose energy denominators are the same function of the loop momenta.  With
// k_l = sum_c coef_lc l_c, D~_m = sum_{lines of cut m} (+1 hole, -1 particle) |k_l|^2 is the quadratic form
// Q_m[c][c'] = sum_l s_l coef_lc coef_lc' in the loop momenta; equal integer matrices mean equal
// denominators, and the weight carries 1/D^2 (e.g. a self-energy insertion between the two cuts).
bool repeated_denominator(const mbpt_diagram_desc& d) {
    const int n = d.order, nl = d.n_lines, nc = d.n_chords;
    std::vector<std::vector<int>> Q((size_t)(n > 1 ? n - 1 : 0), std::vector<int>((size_t)(nc * nc), 0));
    for (int m = 0; m < n - 1; ++m)
        for (int l = 0; l < nl; ++l) {
            const int lo = std::min(d.line_src[l], d.line_dst[l]), hi = std::max(d.line_src[l], d.line_dst[l]);
            if (!(lo <= m && m < hi)) continue;
            const int sgn = d.line_src[l] > d.line_dst[l] ? 1 : -1;
            for (int a = 0; a < nc; ++a)
                for (int b = 0; b < nc; ++b) Q[(size_t)m][(size_t)(a * nc + b)] += sgn * d.line_coef[l][a] * d.line_coef[l][b];
        }
    for (int a = 0; a < n - 1; ++a)
        for (int b = a + 1; b < n - 1; ++b)
            if (Q[(size_t)a] == Q[(size_t)b]) return true;
    return false;
}

Mat mirror(int n, const Mat& A) {
    Mat M{};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) M[i * n + j] = A[(n - 1 - j) * n + (n - 1 - i)];
    return M;
}

void set_err(char* err, size_t len, const char* msg) {
    if (err && len) snprintf(err, len, "%s", msg);
}

}  // namespace

int validate_descriptor(const mbpt_diagram_desc& d, char* err, size_t errlen) {
    int n = d.order;
    if (n < 2 || n > MBPT_MAX_DEVICE_ORDER) { set_err(err, errlen, "order must be 2..6"); return MBPT_EINVAL; }
    int nl = d.n_lines;
    if (nl != 2 * n) { set_err(err, errlen, "n_lines must be 2*order"); return MBPT_EINVAL; }
    for (int l = 0; l < nl; ++l) {
        int s = d.line_src[l], t = d.line_dst[l];
        if (s < 0 || s >= n || t < 0 || t >= n || s == t) { set_err(err, errlen, "line endpoints out of range"); return MBPT_EINVAL; }
    }
    for (int v = 0; v < n; ++v) {
        int no = 0, ni = 0;
        for (int l = 0; l < nl; ++l) { no += d.line_src[l] == v; ni += d.line_dst[l] == v; }
        if (no != 2 || ni != 2) { set_err(err, errlen, "every vertex needs two outgoing and two incoming lines"); return MBPT_EINVAL; }
        for (int k = 0; k < 2; ++k) {
            int lo = d.vtx_out[v][k], li = d.vtx_in[v][k];
            if (lo < 0 || lo >= nl || li < 0 || li >= nl || d.line_src[lo] != v || d.line_dst[li] != v) {
                set_err(err, errlen, "vertex ports do not match the lines");
                return MBPT_EINVAL;
            }
        }
        if (d.vtx_out[v][0] == d.vtx_out[v][1] || d.vtx_in[v][0] == d.vtx_in[v][1]) {
            set_err(err, errlen, "a vertex lists the same line twice");
            return MBPT_EINVAL;
        }
    }
    int nc = d.n_chords;
    if (nc != n + 1) { set_err(err, errlen, "n_chords must be order+1"); return MBPT_EINVAL; }
    bool is_chord[MBPT_MAX_LINES] = {false};
    for (int c = 0; c < nc; ++c) {
        int l = d.chord_line[c];
        if (l < 0 || l >= nl || is_chord[l]) { set_err(err, errlen, "invalid chord list"); return MBPT_EINVAL; }
        is_chord[l] = true;
    }
    int parent[8];
    for (int v = 0; v < n; ++v) parent[v] = v;
    for (int l = 0; l < nl; ++l) {
        if (is_chord[l]) continue;
        int a = find_root(parent, d.line_src[l]), b = find_root(parent, d.line_dst[l]);
        if (a == b) { set_err(err, errlen, "non-chord lines contain a cycle"); return MBPT_EINVAL; }
        parent[a] = b;
    }
    for (int v = 1; v < n; ++v)
        if (find_root(parent, v) != find_root(parent, 0)) { set_err(err, errlen, "diagram is not connected"); return MBPT_EINVAL; }
    for (int l = 0; l < nl; ++l)
        for (int c = 0; c < nc; ++c)
            if (d.line_coef[l][c] < -1 || d.line_coef[l][c] > 1) { set_err(err, errlen, "line_coef outside {-1,0,1}"); return MBPT_EINVAL; }
    for (int c = 0; c < nc; ++c)
        for (int cc = 0; cc < nc; ++cc)
            if (d.line_coef[d.chord_line[c]][cc] != (c == cc)) { set_err(err, errlen, "chord rows of line_coef must be unit vectors"); return MBPT_EINVAL; }
    for (int v = 0; v < n; ++v)
        for (int c = 0; c < nc; ++c) {
            int s = 0;
            for (int l = 0; l < nl; ++l) {
                if (d.line_dst[l] == v) s += d.line_coef[l][c];
                if (d.line_src[l] == v) s -= d.line_coef[l][c];
            }
            if (s) { set_err(err, errlen, "line_coef violates momentum conservation"); return MBPT_EINVAL; }
        }
    return MBPT_OK;
}

void set_pref(DiagRec* r, double pref) {
    r->pref = pref;
    // FP32 mantissa and exponent of |pref| (far-class mixed samples fold it into the FP32 Jacobian);
    // pref_mf = 0 for pref = 0
    int e = 0;
    float m = (float)(2.0 * std::frexp(std::fabs(pref), &e));   // in [1, 2] (0 for pref = 0), rounded to nearest
    e -= 1;
    if (m >= 2.0f) {
        m = 1.0f;
        e += 1;
    }
    r->pref_mf = m;
    r->pref_e = pref == 0.0 ? 0 : e;
    r->pref_sign_hi = std::signbit(pref) ? 0x80000000u : 0u;
}

void hole_chords_first(mbpt_diagram_desc& d) {
    const int nc = d.n_chords, nl = d.n_lines;
    if (nc < 1 || nc > MBPT_MAX_CHORDS || nl < 1 || nl > MBPT_MAX_LINES) return;   // left to validation
    for (int c = 0; c < nc; ++c)
        if (d.chord_line[c] < 0 || d.chord_line[c] >= nl) return;
    int perm[MBPT_MAX_CHORDS], k = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int c = 0; c < nc; ++c) {
            const int l = d.chord_line[c];
            const bool hole = d.line_src[l] > d.line_dst[l];
            if (hole == (pass == 0)) perm[k++] = c;
        }
    const mbpt_diagram_desc o = d;
    for (int j = 0; j < nc; ++j) {
        d.chord_line[j] = o.chord_line[perm[j]];
        for (int l = 0; l < nl; ++l) d.line_coef[l][j] = o.line_coef[l][perm[j]];
    }
}

int compile_record(const mbpt_diagram_desc& d, const mbpt_physics& ph, const mbpt_vegas_cfg& cfg, DiagRec* r,
                   char* err, size_t errlen) {
    int st = validate_descriptor(d, err, errlen);
    if (st) return st;
    if (!(ph.kF_n >= 0.0) || !(ph.kF_p >= 0.0) || !(ph.kF_n > 0.0 || ph.kF_p > 0.0)) {
        set_err(err, errlen, "Fermi momenta must be >= 0 and not both zero");
        return MBPT_EINVAL;
    }
    double kfmax = ph.kF_n > ph.kF_p ? ph.kF_n : ph.kF_p;
    double kfmin = kfmax;
    if (ph.kF_n > 0.0 && ph.kF_n < kfmin) kfmin = ph.kF_n;
    if (ph.kF_p > 0.0 && ph.kF_p < kfmin) kfmin = ph.kF_p;
    if (!(ph.K_max > kfmax) || !(ph.hbar2_over_m > 0.0) || !(ph.Lambda > 0.0) || !(ph.m_pi >= 0.0) ||
        ph.reg_power < 2 || ph.reg_power > 8 || (ph.reg_power & 1) || ph.map_kind < 0 || ph.map_kind > 1) {
        set_err(err, errlen, "invalid physics parameters (K_max > kF, hbar2_over_m > 0, Lambda > 0, even reg_power 2..8, map_kind 0 or 1)");
        return MBPT_EINVAL;
    }
    if (ph.spectrum != 0 && ph.spectrum != 1) {
        set_err(err, errlen, "spectrum must be 0 (free) or 1 (Hartree-Fock)");
        return MBPT_EINVAL;
    }
    if (ph.spectrum == 1 && ph.kF_n > 0.0 && ph.kF_p > 0.0 && ph.kF_n != ph.kF_p) {
        set_err(err, errlen, "the Hartree-Fock spectrum needs one Fermi momentum (neutron or symmetric matter)");
        return MBPT_EINVAL;
    }
    if (cfg.n_bins < 2 || cfg.n_bins > MBPT_MAX_BINS || cfg.samples_per_iter < 2 ||
        cfg.samples_per_iter >= (1ull << 32) || !(cfg.alpha >= 0.0) ||
        (cfg.precision != MBPT_FP64 && cfg.precision != MBPT_MIXED && cfg.precision != MBPT_MIXED_MAP64) || !(cfg.target_rel >= 0.0) ||
        !(cfg.target_abs >= 0.0)) {
        set_err(err, errlen, "invalid VEGAS configuration");
        return MBPT_EINVAL;
    }
    if (cfg.n_shifts != 0 && cfg.n_shifts != (uint32_t)kShifts) {
        set_err(err, errlen, "n_shifts must be 0 or 3");
        return MBPT_EINVAL;
    }
    if (cfg.combine != MBPT_COMBINE_INVVAR && cfg.combine != MBPT_COMBINE_POOLED) {
        set_err(err, errlen, "combine must be MBPT_COMBINE_INVVAR or MBPT_COMBINE_POOLED");
        return MBPT_EINVAL;
    }
    if (!(cfg.near_band == 0.0f || (cfg.near_band >= 1.52587890625e-05f && cfg.near_band <= 0.5f))) {
        set_err(err, errlen, "near_band must be 0 (default) or in [2^-16, 1/2]");
        return MBPT_EINVAL;
    }
    if (cfg.n_shifts) {
        for (int k = 0; k < kShifts; ++k)
            if (!(cfg.shift[k] > 0.0) || !(cfg.shift[k] < 1e6)) {
                set_err(err, errlen, "regulator shifts must be positive (MeV)");
                return MBPT_EINVAL;
            }
        if (cfg.shift[0] == cfg.shift[1] || cfg.shift[0] == cfg.shift[2] || cfg.shift[1] == cfg.shift[2]) {
            set_err(err, errlen, "regulator shifts must be distinct");
            return MBPT_EINVAL;
        }
    }
    memset(r, 0, sizeof(*r));
    int n = d.order, nl = d.n_lines, nc = d.n_chords;
    r->order = n;
    r->n_lines = nl;
    r->n_chords = nc;
    r->map_kind = ph.map_kind;
    r->d = 3 * nc - 3 * ph.map_kind;
    r->nb = cfg.n_bins;
    if (r->nb > grid_stride(r->d)) {
        if (err && errlen)
            snprintf(err, errlen, "n_bins %d too large for d = %d (at most %d: d x n_bins <= %d)", r->nb, r->d,
                     grid_stride(r->d), kCells);
        return MBPT_EINVAL;
    }
    r->precision = cfg.precision;
    r->reg_half = ph.reg_power / 2;
    r->all_slots = (1u << nl) - 1u;
    // --- slots: chords first, then tree lines in post-order of a spanning tree rooted at vertex 0
    int slot_of[MBPT_MAX_LINES];
    bool is_chord[MBPT_MAX_LINES] = {false};
    for (int l = 0; l < nl; ++l) slot_of[l] = -1;
    for (int c = 0; c < nc; ++c) {
        slot_of[(int)d.chord_line[c]] = c;
        is_chord[(int)d.chord_line[c]] = true;
    }
    int parent_edge[8], depth[8], order_v[8], nv = 0;
    for (int v = 0; v < n; ++v) { parent_edge[v] = -2; depth[v] = 0; }
    parent_edge[0] = -1;
    order_v[nv++] = 0;
    for (int qh = 0; qh < nv; ++qh) {
        int v = order_v[qh];
        for (int l = 0; l < nl; ++l) {
            if (is_chord[l]) continue;
            int u = -1;
            if (d.line_src[l] == v) u = d.line_dst[l];
            else if (d.line_dst[l] == v) u = d.line_src[l];
            if (u < 0 || parent_edge[u] != -2) continue;
            parent_edge[u] = l;
            depth[u] = depth[v] + 1;
            order_v[nv++] = u;
        }
    }
    int next_slot = nc, t = 0;
    for (int k = nv - 1; k >= 1; --k) {     // reverse BFS order: children before parents
        int v = order_v[k];
        int e = parent_edge[v];
        // the other three lines at v: same side as e (C) and opposite side (A, B)
        bool e_in = d.line_dst[e] == v;
        int A, B, C;
        if (e_in) {
            A = d.vtx_out[v][0]; B = d.vtx_out[v][1];
            C = d.vtx_in[v][0] == e ? d.vtx_in[v][1] : d.vtx_in[v][0];
        } else {
            A = d.vtx_in[v][0]; B = d.vtx_in[v][1];
            C = d.vtx_out[v][0] == e ? d.vtx_out[v][1] : d.vtx_out[v][0];
        }
        if (slot_of[A] < 0 || slot_of[B] < 0 || slot_of[C] < 0) {
            set_err(err, errlen, "internal: momentum routing order");
            return MBPT_EINVAL;
        }
        r->tree_a[t] = (int8_t)slot_of[A];
        r->tree_b[t] = (int8_t)slot_of[B];
        r->tree_c[t] = (int8_t)slot_of[C];
        slot_of[e] = next_slot++;
        ++t;
    }
    for (int l = 0; l < nl; ++l) r->line_slot[l] = (int8_t)slot_of[l];
    for (int l = 0; l < nl; ++l)
        if (slot_of[l] >= nc)
            for (int c = 0; c < nc; ++c) r->tcoef[slot_of[l] - nc][c] = (float)d.line_coef[l][c];
    int h = 0;
    for (int l = 0; l < nl; ++l)
        if (d.line_src[l] > d.line_dst[l]) { r->hole_slots |= 1u << slot_of[l]; ++h; }
    // --- ranges of the chord momenta
    for (int c = 0; c < nc; ++c) {
        bool hole = d.line_src[(int)d.chord_line[c]] > d.line_dst[(int)d.chord_line[c]];
        r->chord_lo[c] = hole ? 0.0 : kfmin;
        r->chord_rng[c] = hole ? kfmax : ph.K_max - kfmin;
        r->chord_lo_f[c] = (float)r->chord_lo[c];
        r->chord_rng_f[c] = (float)r->chord_rng[c];
    }
    // --- vertices
    for (int v = 0; v < n; ++v) {
        int o1 = d.vtx_out[v][0], o2 = d.vtx_out[v][1], i1 = d.vtx_in[v][0], i2 = d.vtx_in[v][1];
        r->port_slot[v][0] = (int8_t)slot_of[o1];
        r->port_slot[v][1] = (int8_t)slot_of[o2];
        r->port_slot[v][2] = (int8_t)slot_of[i1];
        r->port_slot[v][3] = (int8_t)slot_of[i2];
        for (int c = 0; c < nc; ++c) {
            r->vcoef_out[v][c] = (float)(d.line_coef[o1][c] - d.line_coef[o2][c]);
            r->vcoef_in[v][c] = (float)(d.line_coef[i1][c] - d.line_coef[i2][c]);
        }
    }
    // --- energy denominators: cut m lies between vertices m and m+1 and holds the lines with
    // min(src,dst) <= m < max(src,dst).  D~_m = sum_holes k^2 - sum_particles k^2 over the cut,
    // updated at vertex m: lines starting there enter, lines ending there leave.
    for (int m = 0; m < n - 1; ++m) {
        int k = 0;
        for (int l = 0; l < nl; ++l) {
            int s = d.line_src[l], tt = d.line_dst[l];
            if (s != m && tt != m) continue;
            int lo = s < tt ? s : tt;
            bool hole = s > tt;
            bool enter = (lo == m);
            bool add = (hole == enter);     // hole entering: +, particle entering: -, leaving: opposite
            r->cut_slot[m][k] = (int8_t)slot_of[l];
            r->cut_neg[m][k] = add ? 0 : 1;
            ++k;
        }
        if (k != 4) {
            set_err(err, errlen, "internal: vertex without four lines");
            return MBPT_EINVAL;
        }        // increasing slot order (distinct slots: term k lies in k .. 2n-4+k)
        for (int a = 1; a < 4; ++a)
            for (int b = a; b > 0 && r->cut_slot[m][b - 1] > r->cut_slot[m][b]; --b) {
                std::swap(r->cut_slot[m][b - 1], r->cut_slot[m][b]);
                std::swap(r->cut_neg[m][b - 1], r->cut_neg[m][b]);
            }
    }
    // --- equivalent line pairs
    int neq = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            int cnt = 0;
            for (int l = 0; l < nl; ++l) cnt += (d.line_src[l] == i && d.line_dst[l] == j);
            if (cnt == 2) ++neq;
        }
    // --- spin-sum terms: loops when vertex v continues i1->o1, i2->o2 (direct) or
    // i1->o2, i2->o1 (exchange)
    bool sym = (ph.kF_p == 0.0) || (ph.kF_n == 0.0) || (ph.kF_n == ph.kF_p);
    int species = (ph.kF_n > 0.0) + (ph.kF_p > 0.0);
    double g = 2.0 * species;
    r->asym = sym ? 0 : 1;
    for (int term = 0; term < (1 << n); ++term) {
        int seen = 0, loops = 0;
        for (int start = 0; start < nl; ++start) {
            if ((seen >> start) & 1) continue;
            uint32_t mask = 0;
            int l = start;
            while (!((seen >> l) & 1)) {
                seen |= 1 << l;
                mask |= 1u << slot_of[l];
                int v = d.line_dst[l];
                bool ex = (term >> v) & 1;
                bool first = d.vtx_in[v][0] == l;
                l = (first != ex) ? d.vtx_out[v][0] : d.vtx_out[v][1];
            }
            if (loops < kMaxLoops) r->loop_mask[term][loops] = (uint16_t)mask;
            ++loops;
        }
        if (loops > kMaxLoops) {
            set_err(err, errlen, "internal: too many loops");
            return MBPT_EINVAL;
        }
        r->nloops[term] = (int8_t)loops;
        r->gsign_f[term] = (loops & 1) ? -1.0f : 1.0f;
        double c = ((loops & 1) ? -1.0 : 1.0) * pow(g, loops);
        r->gcoef_d[term] = c;
    }
    // difference form: superset sums of the coefficients, signed by the subset size (exact integers)
    for (int a = 0; a < (1 << n); ++a) {
        double acc = 0.0;
        for (int term = 0; term < (1 << n); ++term)
            if ((term & a) == a) acc += r->gcoef_d[term];
        r->gdel_f[a] = (float)((__builtin_popcount(a) & 1) ? -acc : acc);
    }
    // --- physics
    if (sym) {
        double kf = ph.kF_n > 0.0 ? ph.kF_n : ph.kF_p;
        r->kf2_n = kf * kf;
        r->kf2_p = kf * kf;
    } else {
        r->kf2_n = ph.kF_n * ph.kF_n;
        r->kf2_p = ph.kF_p * ph.kF_p;
    }
    r->kf2_nf = (float)r->kf2_n;
    r->kf2_pf = (float)r->kf2_p;
    r->spectrum = ph.spectrum;
    r->hf_n = MBPT_HF_KNOTS - 1;
    r->hf_hinv_f = (float)((MBPT_HF_KNOTS - 1) / (2.0 * ph.K_max));
    r->CS = ph.C_S;
    r->CY4 = 4.0 * ph.C_Y;
    r->mpi2_4 = 4.0 * ph.m_pi * ph.m_pi;
    r->regc = 1.0 / (4.0 * ph.Lambda * ph.Lambda);
    r->CSf = (float)r->CS;
    r->CY4f = (float)r->CY4;
    r->mpi2_4f = (float)r->mpi2_4;
    r->regc2f = (float)(r->regc * pow(1.4426950408889634, 1.0 / r->reg_half));
    const double pi = 3.14159265358979323846;
    double dens = (ph.kF_n * ph.kF_n * ph.kF_n + ph.kF_p * ph.kF_p * ph.kF_p) / (3.0 * pi * pi);
    // (-1)^h 2^-n_eq / n_dens * (2pi)^-3(n+1) * (2/(hbar^2/m))^(n-1) * N_b^d * chord constants:
    // 4 range_c per full chord (dcos/dx = 2, dphi/dx = 2/(1/2 - a) with the 1/(1/2 - a) per sample);
    // with the rotational reduction 4 pi range_0 (all directions of chord 0) and
    // 2 x 2 pi range_1 (polar angle, all azimuths of chord 1)
    double pref = ((h & 1) ? -1.0 : 1.0) / pow(2.0, neq) / pow(2.0 * pi, 3.0 * nc) / dens *
                  pow(2.0 / ph.hbar2_over_m, n - 1) * pow((double)cfg.n_bins, (double)r->d);
    for (int c = 0; c < nc; ++c) {
        if (ph.map_kind == 1 && c < 2) pref *= 4.0 * pi * r->chord_rng[c];
        else pref *= 4.0 * r->chord_rng[c];
    }
    set_pref(r, pref);
    // denominator regulator: D_m - shift in D~ units (D = (hbar^2/2m) D~), Lagrange weights at 0
    r->n_shifts = (int32_t)cfg.n_shifts;
    // FP64-map band of the mixed mode: wider from fifth order on, where more lines (and the larger spin sums)
    // make the weight more sensitive to where the FP32 map puts a sample near a Fermi surface
    r->near_f = cfg.near_band != 0.0f ? cfg.near_band : (n >= 5 ? 0.0078125f : 0.0009765625f);
    for (int k = 0; k < kShifts; ++k) {
        r->eta[k] = cfg.n_shifts ? cfg.shift[k] / (0.5 * ph.hbar2_over_m) : 0.0;
        double L = 1.0;
        for (int j = 0; j < kShifts; ++j)
            if (j != k) L *= (0.0 - cfg.shift[j]) / (cfg.shift[k] - cfg.shift[j]);
        r->lag[k] = cfg.n_shifts ? L : 0.0;
    }
    return MBPT_OK;
}

// ---------------------------------------------------------------------------
// Hartree-Fock single-particle spectrum (Eq. (7)) for one Fermi momentum.
// ---------------------------------------------------------------------------
namespace {

// Gauss-Legendre rule on [-1, 1]: roots of P_n by Newton's method (P_n and P_n' from the three-term
// recurrence), weights 2 / ((1 - x^2) P_n'(x)^2).
void gl_rule(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dpn = 1.0;
        for (int it = 0; it < 100; ++it) {
            double pm1 = 1.0, pn = z;
            for (int j = 2; j <= n; ++j) {
                const double pj = ((2 * j - 1) * z * pn - (j - 1) * pm1) / j;
                pm1 = pn;
                pn = pj;
            }
            dpn = n * (z * pn - pm1) / (z * z - 1.0);
            const double step = pn / dpn;
            z -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dpn * dpn);
    }
}

}  // namespace

// Sigma at the knots k_i = i h (MeV): 1/(4 pi^2) int_0^kF dk' k'^2 int_{-1}^{1} dc [g V_d - V_e] with
// V_d = [C_S + C_Y/m_pi^2] exp(-2 (p/L)^r), V_e = [C_S + C_Y/(4p^2 + m_pi^2)] exp(-2 (p/L)^r),
// p^2 = (k^2 + k'^2 - 2 k k' c)/4.  Then the cubic spline (zero slope at 0, zero curvature at the end)
// as per-interval polynomials in t = k - k_i, in units of hbar^2/2m: tab[5 i .. 5 i + 4] = k_i, a, b, c, d.
int build_hf_table(const mbpt_physics& ph, std::vector<double>& tab, char* err, size_t errlen) {
    const int n = MBPT_HF_KNOTS, nq = MBPT_HF_QUAD;
    const double kf = ph.kF_n > 0.0 ? ph.kF_n : ph.kF_p;
    const double g = (ph.kF_n > 0.0 ? 2.0 : 0.0) + (ph.kF_p > 0.0 ? 2.0 : 0.0);
    const double h = 2.0 * ph.K_max / (n - 1);
    const double pi = 3.14159265358979323846;
    std::vector<double> xg, wg;
    gl_rule(nq, xg, wg);
    const double L2 = ph.Lambda * ph.Lambda, mpi2 = ph.m_pi * ph.m_pi, rh = 0.5 * ph.reg_power;
    std::vector<double> y(n), m(n);
    for (int i = 0; i < n; ++i) {
        const double k = i * h;
        double acc = 0.0;
        for (int a = 0; a < nq; ++a) {
            const double kp = 0.5 * kf * (xg[a] + 1.0);
            double inner = 0.0;
            for (int b = 0; b < nq; ++b) {
                double p2 = 0.25 * (k * k + kp * kp - 2.0 * k * kp * xg[b]);
                if (p2 < 0.0) p2 = 0.0;
                const double F = std::exp(-2.0 * std::pow(p2 / L2, rh));
                const double vd = (ph.C_S + ph.C_Y / mpi2) * F;
                const double ve = (ph.C_S + ph.C_Y / (4.0 * p2 + mpi2)) * F;
                inner += wg[b] * (g * vd - ve);
            }
            acc += 0.5 * kf * wg[a] * kp * kp * inner;
        }
        y[i] = acc / (4.0 * pi * pi);
    }
    // spline second derivatives: 2 m0 + m1 = 6 (y1 - y0)/h^2; m_{i-1} + 4 m_i + m_{i+1} = 6 (y_{i-1} - 2 y_i + y_{i+1})/h^2;
    // m_{n-1} = 0.  Thomas algorithm.
    std::vector<double> cp(n), dp(n);
    cp[0] = 0.5;
    dp[0] = 3.0 * (y[1] - y[0]) / (h * h);
    for (int i = 1; i < n - 1; ++i) {
        const double den = 4.0 - cp[i - 1];
        cp[i] = 1.0 / den;
        dp[i] = (6.0 * (y[i - 1] - 2.0 * y[i] + y[i + 1]) / (h * h) - dp[i - 1]) / den;
    }
    m[n - 1] = 0.0;
    for (int i = n - 2; i >= 0; --i) m[i] = dp[i] - cp[i] * m[i + 1];
    const double e = 0.5 * ph.hbar2_over_m;
    tab.assign((size_t)5 * (n - 1), 0.0);
    double prev = -1e300;
    for (int i = 0; i < n - 1; ++i) {
        tab[5 * i + 0] = i * h;
        tab[5 * i + 1] = y[i] / e;
        tab[5 * i + 2] = ((y[i + 1] - y[i]) / h - h * (2.0 * m[i] + m[i + 1]) / 6.0) / e;
        tab[5 * i + 3] = 0.5 * m[i] / e;
        tab[5 * i + 4] = (m[i + 1] - m[i]) / (6.0 * h) / e;
        const double eps = i * h * i * h + y[i] / e;    // in units of hbar^2/2m
        if (i > 0 && !(eps > prev)) {
            set_err(err, errlen, "the Hartree-Fock spectrum does not increase with k");
            return MBPT_EINVAL;
        }
        prev = eps;
    }
    return MBPT_OK;
}

// Sigma(k)/(hbar^2/2m) from the table (FP64), 0 beyond the last knot.
double hf_eval(const std::vector<double>& tab, double hinv, double k) {
    const int nint = (int)(tab.size() / 5);
    int i = (int)std::floor(k * hinv);
    if (i < 0) i = 0;
    if (i >= nint) return 0.0;
    const double* c = &tab[5 * (size_t)i];
    const double t = k - c[0];
    return std::fma(std::fma(std::fma(c[4], t, c[3]), t, c[2]), t, c[1]);
}

}  // namespace mbpt

using namespace mbpt;

extern "C" int mbpt_generate(int order, mbpt_diagram_desc* out, int cap, int* count) {
    if (order < 2 || order > MBPT_MAX_ORDER || !count) return MBPT_EINVAL;
    std::vector<Mat> mats = all_matrices(order);
    int total = (int)mats.size();
    *count = total;
    if (!out) return MBPT_OK;
    if (cap < total) return MBPT_ENOMEM;
    std::map<Mat, int> index;
    for (int k = 0; k < total; ++k) index[mats[k]] = k;
    for (int k = 0; k < total; ++k) {
        build_desc(order, mats[k], k, out[k]);
        Mat M = mirror(order, mats[k]);
        out[k].mirror_id = index.count(M) ? index[M] : -1;
        int flags = 0;
        if (anomalous(out[k])) flags |= MBPT_FLAG_ANOMALOUS;
        if (out[k].mirror_id == k) flags |= MBPT_FLAG_SELF_MIRROR;
        if (repeated_denominator(out[k])) flags |= MBPT_FLAG_REPEATED_DENOMINATOR;
        out[k].flags = flags;
    }
    return MBPT_OK;
}

extern "C" int mbpt_hole_chords(const mbpt_diagram_desc* d, int* out) {
    if (!d || !out || d->n_chords < 0 || d->n_chords > MBPT_MAX_CHORDS || d->n_lines < 0 ||
        d->n_lines > MBPT_MAX_LINES)
        return MBPT_EINVAL;
    int h = 0;
    for (int c = 0; c < d->n_chords; ++c) {
        const int l = d->chord_line[c];
        if (l < 0 || l >= d->n_lines) return MBPT_EINVAL;
        h += d->line_src[l] > d->line_dst[l];   // src above dst in time: a hole line
    }
    *out = h;
    return MBPT_OK;
}

extern "C" int mbpt_hf_self_energy(const mbpt_physics* ph, int n, const double* k, double* sigma) {
    if (!ph || n < 0 || (n > 0 && (!k || !sigma))) return MBPT_EINVAL;
    if (!(ph->kF_n >= 0.0) || !(ph->kF_p >= 0.0) || !(ph->kF_n > 0.0 || ph->kF_p > 0.0) ||
        (ph->kF_n > 0.0 && ph->kF_p > 0.0 && ph->kF_n != ph->kF_p) || !(ph->K_max > 0.0) ||
        !(ph->hbar2_over_m > 0.0) || !(ph->Lambda > 0.0) || ph->reg_power < 2)
        return MBPT_EINVAL;
    std::vector<double> tab;
    char err[128];
    int st = build_hf_table(*ph, tab, err, sizeof(err));
    if (st) return st;
    const double hinv = (MBPT_HF_KNOTS - 1) / (2.0 * ph->K_max), e = 0.5 * ph->hbar2_over_m;
    for (int i = 0; i < n; ++i) sigma[i] = e * hf_eval(tab, hinv, k[i]);
    return MBPT_OK;
}
