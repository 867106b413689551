"""Deterministic quadratures that pin the oracle to the mathematics of the paper
(independent formulations, not a re-typing of the oracle's integrand).

* first_order_full_v: E^(1)/N for a spin-independent potential reduced to a 1D
  integral over the half relative momentum of two points in the Fermi sphere.
* second_order: E^(2)/N of Eq. (2) in centre-of-mass / relative momenta with the
  Pauli restrictions written as explicit integration limits, product
  Gauss-Legendre in six variables.
"""
from __future__ import annotations

import math

import numpy as np


def first_order_from_sigma(kF, g, sigma, n=200):
    """E_HF/N = (g/2n) int d^3k/(2 pi)^3 theta(kF - k) Sigma(k) = (g/(4 pi^2 n)) int_0^kF k^2 Sigma(k) dk."""
    nd = g * kF ** 3 / (6.0 * math.pi ** 2)
    x, w = gl(0.0, kF, n)
    return g / (4.0 * math.pi ** 2 * nd) * float(np.sum(w * x ** 2 * sigma(x)))


def gl(a: float, b: float, n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def vpot(C_S, C_Y, m_pi, Lam, r, p, pp, q2):
    return (C_S + C_Y / (q2 + m_pi ** 2)) * np.exp(-(p / Lam) ** r - (pp / Lam) ** r)


def first_order_full_v(kF, g, C_S, C_Y, m_pi, Lam, r=4, npts=200):
    """E/N = (n/2) int_0^kF P(p) [V_d(p) - V_e(p)/g] dp with
    P(p) = (24 p^2/kF^3)(1 - 3p/(2kF) + p^3/(2kF^3)) the distribution of
    p = |k1 - k2|/2 for k1, k2 uniform in the Fermi ball, V_d = V(p, p) and
    V_e = V(p, -p); n = g kF^3 / (6 pi^2)."""
    n = g * kF ** 3 / (6.0 * math.pi ** 2)
    p, w = gl(0.0, kF, npts)
    P = 24.0 * p ** 2 / kF ** 3 * (1.0 - 1.5 * p / kF + 0.5 * p ** 3 / kF ** 3)
    vd = vpot(C_S, C_Y, m_pi, Lam, r, p, p, 0.0)
    ve = vpot(C_S, C_Y, m_pi, Lam, r, p, p, 4.0 * p ** 2)
    return 0.5 * n * float(np.sum(w * P * (vd - ve / g)))


def first_order_contact(kF, g, C_S):
    """Unregulated contact: E/N = C_S n (g - 1)/(2 g)."""
    n = g * kF ** 3 / (6.0 * math.pi ** 2)
    return C_S * n * (g - 1) / (2.0 * g)


def second_order(kF, g, hbar2_over_m, C_S, C_Y, m_pi, Lam, r=4, n_rad=12, n_ang=10, pmax=8.0, cross=True,
                 shift=0.0, sigma=None):
    """E^(2)/N = (1/n) (1/4) sum_spins int d^3k_i d^3k_j d^3k_a/(2pi)^9 |<ab|V|ij>|^2 / D
    with P = (k_i + k_j)/2, p = (k_i - k_j)/2, p' = (k_a - k_b)/2 (Jacobian 8),
    D = (hbar^2/m)(p^2 - p'^2), spin sum g^2 (V_d^2 + V_e^2) - 2 g V_d V_e.
    P along z, p in the xz-plane; holes need P^2 + p^2 + 2Pp|cos t_p| < kF^2,
    particles P^2 + p'^2 - 2Pp'|cos t'| >= kF^2.  shift s replaces D by D - s.  sigma (a vectorised
    function of |k|) adds a self-energy to every single-particle energy: the lines are then
    k_i,j = P +- p, k_a,b = P +- p' and D = eps_i + eps_j - eps_a - eps_b - s."""
    n = g * kF ** 3 / (6.0 * math.pi ** 2)
    Pn, Pw = gl(0.0, kF, n_rad)
    total = 0.0
    # cos(t_p) -> -cos(t_p) together with cos(t') -> -cos(t') leaves the integrand
    # unchanged, and phi' -> 2pi - phi' too: integrate cos(t_p) >= 0 and phi' in [0, pi], times 4.
    phn, phw = gl(0.0, math.pi, n_ang)
    for P, wP in zip(Pn, Pw):
        q0 = math.sqrt(kF ** 2 - P ** 2)
        # hole relative momentum panels
        p_nodes, p_w = [], []
        for a, b in ((0.0, kF - P), (kF - P, q0)):
            if b > a:
                x, w = gl(a, b, n_rad)
                p_nodes.append(x)
                p_w.append(w)
        p_nodes = np.concatenate(p_nodes)
        p_w = np.concatenate(p_w)
        pp_nodes, pp_w = [], []
        edges = [q0, kF + P, kF + P + 0.5, 2.5, 4.0, pmax]
        for a, b in zip(edges[:-1], edges[1:]):
            if b > a:
                x, w = gl(a, b, n_rad)
                pp_nodes.append(x)
                pp_w.append(w)
        pp_nodes = np.concatenate(pp_nodes)
        pp_w = np.concatenate(pp_w)
        for p, wp in zip(p_nodes, p_w):
            ch = (kF ** 2 - P ** 2 - p ** 2) / (2.0 * P * p)
            ch = min(max(ch, 0.0), 1.0)
            if ch <= 0.0:
                continue
            ct, wct = gl(0.0, ch, n_ang)
            st = np.sqrt(1.0 - ct ** 2)
            cp = (P ** 2 + pp_nodes ** 2 - kF ** 2) / (2.0 * P * pp_nodes)
            cp = np.clip(cp, 0.0, 1.0)
            u, wu = np.polynomial.legendre.leggauss(n_ang)
            # cos(t') in [-cp, cp]: nodes per p'
            ctp = cp[:, None] * u[None, :]                     # (np', nang)
            wctp = cp[:, None] * wu[None, :]
            stp = np.sqrt(np.maximum(0.0, 1.0 - ctp ** 2))
            # full grid: (ct, p', ct', phi')
            CT = ct[:, None, None, None]
            ST = st[:, None, None, None]
            PP = pp_nodes[None, :, None, None]
            CTP = ctp[None, :, :, None]
            STP = stp[None, :, :, None]
            PH = phn[None, None, None, :]
            dot = p * PP * (ST * STP * np.cos(PH) + CT * CTP)
            qd2 = p ** 2 + PP ** 2 - 2.0 * dot
            qe2 = p ** 2 + PP ** 2 + 2.0 * dot
            reg = np.exp(-(p / Lam) ** r - (PP / Lam) ** r)
            vd = (C_S + C_Y / (qd2 + m_pi ** 2)) * reg
            ve = (C_S + C_Y / (qe2 + m_pi ** 2)) * reg
            S = g * g * (vd ** 2 + ve ** 2) - (2.0 * g * vd * ve if cross else 0.0)
            Dn = hbar2_over_m * (p ** 2 - PP ** 2) - shift
            if sigma is not None:
                # P along z, p in the xz plane at polar angle t_p, p' at (t', phi')
                pz = p * CT
                ppz = PP * CTP
                ki = np.sqrt(np.maximum(P ** 2 + p ** 2 + 2 * P * pz, 0.0))
                kj = np.sqrt(np.maximum(P ** 2 + p ** 2 - 2 * P * pz, 0.0))
                ka = np.sqrt(np.maximum(P ** 2 + PP ** 2 + 2 * P * ppz, 0.0))
                kb = np.sqrt(np.maximum(P ** 2 + PP ** 2 - 2 * P * ppz, 0.0))
                Dn = Dn + sigma(ki) + sigma(kj) - sigma(ka) - sigma(kb)
            W = (wct[:, None, None, None] * (pp_w * pp_nodes ** 2)[None, :, None, None]
                 * wctp[None, :, :, None] * phw[None, None, None, :])
            inner = float(np.sum(W * S / Dn)) * 4.0
            total += wP * 4.0 * math.pi * P ** 2 * wp * 2.0 * math.pi * p ** 2 * inner
    return 2.0 / ((2.0 * math.pi) ** 9 * n) * total
