"""Pins of the oracle's force matrices and equilibria.

K^h (Eq. "eq:hh_Kk_hh"), K^H (Eq. "eq:H_Kk"): exact identities the paper
states for the discrete momentum derivative (zero mass moment, Sec. III.B;
moments of order < Q recovered, Sec. IV.B.4) and the derivative of the
discrete Maxwellian.  Equilibria (Eqs. "eq:hh_gk", "eq:H_gk"): brute-force
projection integrals, and the moments they must reproduce.
"""
import math
from decimal import Decimal

import numpy as np
import pytest
from scipy import integrate

from oracle import model
from oracle.model import (VelocitySet, h_equilibrium, h_force_matrix, hh_equilibrium,
                          hh_force_matrix, p_polys)
from oracle.quadrature import _ctx, dec_inv_sqrt_2pi, gauss_hermite, half_range_hermite, poly_eval, to_f64


def _half_moment_identity_residual(K, p, Q):
    """max over s in [1, Q-1], halves sigma, columns k' of
    | sum_{k in sigma} p_k^s K_kk' + s p_k'^{s-1} [k' in sigma] |, relative to
    the size sum_{k in sigma} |p_k^s K_kk'| of the terms summed."""
    worst = 0.0
    for s in range(1, Q):
        for sl in (slice(0, Q), slice(Q, 2 * Q)):
            terms = p[sl, None] ** s * K[sl, :]
            lhs = terms.sum(0)
            rhs = np.zeros(2 * Q)
            rhs[sl] = -s * p[sl] ** (s - 1)
            worst = max(worst, (np.abs(lhs - rhs) / np.abs(terms).sum(0)).max())
    return worst


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 6, 8, 12, 16])
def test_hh_force_matrix_identities(Q):
    K = hh_force_matrix(Q)
    vs = VelocitySet(Q)
    p, w = vs.px, vs.wx
    scale = np.abs(K).max()
    # zero mass moment of dp f: sum_k K_kk' = 0 for every column (Sec. III.B)
    assert np.abs(K.sum(axis=0)).max() <= 1e-15 * scale * 2 * Q
    # half-range moments of order 1..Q-1: int_half p^s dp f = -s int_half p^{s-1} f
    assert _half_moment_identity_residual(K, p, Q) < 1e-15 * Q
    # derivative of the discrete Maxwellian at T = 1: dp(omega) = -p omega
    np.testing.assert_allclose(K @ w, -p * w, atol=1e-14 * np.abs(p * w).max() * Q)
    # the jump term is the only coupling between the two halves, rank one
    cross = K[:Q, Q:]
    assert np.linalg.matrix_rank(cross, tol=1e-10 * np.abs(cross).max()) == 1


def _hh_force_matrix_without_delta(Q):
    """K built from Eq. "eq:dfpm" alone (the delta(p) jump term dropped):
    the cross-half term becomes -omega(0) Phi0 Phi0 restricted to each half."""
    d = half_range_hermite(Q)
    C, z, w = d["C"], d["z"], d["w"]
    K = hh_force_matrix(Q).copy()
    with _ctx():
        s2pi = dec_inv_sqrt_2pi()
        H = [[poly_eval(C[l][: l + 1], zk) for l in range(Q)] for zk in z]
        Phi0 = [sum(C[s][0] * H[k][s] for s in range(Q)) for k in range(Q)]
        for k in range(2 * Q):
            for kp in range(2 * Q):
                sk, skp = (1 if k < Q else -1), (1 if kp < Q else -1)
                extra = s2pi / 2 * Phi0[k % Q] * Phi0[kp % Q]   # undo the printed -1/2 term
                if sk == skp:
                    extra -= s2pi * Phi0[k % Q] * Phi0[kp % Q]   # same-half -omega(0) f(0)
                K[k, kp] += float(w[k % Q] * sk * extra)
    return K


@pytest.mark.parametrize("Q", [4, 8])
def test_dropping_the_delta_term_breaks_mass_conservation(Q):
    # Planted mistake: without the distributional jump term the zeroth moment
    # of dp f is no longer zero (the mass bias the paper's construction removes).
    bad = _hh_force_matrix_without_delta(Q)
    assert np.abs(bad.sum(axis=0)).max() > 1e-3
    # ... and a transposed operand also fails the column identity.
    assert np.abs(hh_force_matrix(Q).T.sum(axis=0)).max() > 1e-3


@pytest.mark.parametrize("Q", [2, 4, 6, 8, 16])
def test_h_force_matrix_identities(Q):
    K = h_force_matrix(Q)
    d = gauss_hermite(Q)
    z, w = to_f64(d["z"]), to_f64(d["w"])
    scale = np.abs(K).max()
    assert np.abs(K.sum(axis=0)).max() <= 1e-14 * scale * Q
    for s in range(1, Q):
        lhs = (z[:, None] ** s * K).sum(0)
        np.testing.assert_allclose(lhs, -s * z ** (s - 1), atol=1e-12 * scale * Q ** 2)
    np.testing.assert_allclose(K @ w, -z * w, atol=1e-14 * Q)


def test_p_polynomials_against_hermite():
    # P_s^-(x) = (-1)^s H_s(x) (Rodrigues) and P_s^+(x) = (-i)^s H_s(i x),
    # with the physicists' Hermite polynomials of numpy.
    Pp, Pm, Ps = p_polys(10)
    xs = np.linspace(-1.5, 1.5, 7)
    for s in range(11):
        c = np.zeros(s + 1)
        c[s] = 1.0
        Hs = np.polynomial.hermite.herm2poly(c)
        np.testing.assert_allclose(np.polyval(list(reversed(Pm[s])), xs),
                                   (-1) ** s * np.polyval(Hs[::-1], xs), rtol=1e-12, atol=1e-9)
        plus = ((-1j) ** s * np.polynomial.hermite.hermval(1j * xs, c)).real
        np.testing.assert_allclose(np.polyval(list(reversed(Pp[s])), xs), plus, rtol=1e-12, atol=1e-9)
    # P_s^* at s = 1, 2 by hand: P_1^* = 1, P_2^* = P_1^- + 2 P_1^+ ... expanded
    assert list(Ps[1]) == [1]
    assert list(Ps[2]) == [0, 2]          # C(2,0) P_0^+ P_1^- + C(2,1) P_1^+ P_0^- = -2x + 4x


def _g(p, u, T):
    return math.exp(-(p - u) ** 2 / (2 * T)) / math.sqrt(2 * math.pi * T)


@pytest.mark.parametrize("Q,u,T", [(4, 0.3, 1.4), (4, -0.6, 0.5), (8, 0.2, 2.0), (8, -0.1, 0.7),
                                   (16, 0.25, 1.3)])
def test_hh_equilibrium_by_projection_integrals(Q, u, T):
    # g_k = w_k sum_{l<=N} G_l^{+-} h_l(z_k) with G_l^{+-} = int_0^inf g(+-p) h_l(p) dp
    # computed by adaptive quadrature (not by the closed form of Eq. "eq:hh_gk").
    N = Q - 1
    d = half_range_hermite(Q)
    C, z, w = d["C"], to_f64(d["z"]), to_f64(d["w"])
    h = lambda l, x: sum(float(C[l][s]) * x ** s for s in range(l + 1))
    ref = np.zeros(2 * Q)
    for sgn, off in ((1, 0), (-1, Q)):
        G = [integrate.quad(lambda p: _g(sgn * p, u, T) * h(l, p), 0, np.inf,
                            epsabs=1e-14, epsrel=1e-13, limit=400)[0] for l in range(N + 1)]
        for k in range(Q):
            ref[off + k] = w[k] * sum(G[l] * h(l, z[k]) for l in range(N + 1))
    got = hh_equilibrium(Q, N, u, T)
    tol = {4: 1e-12, 8: 1e-10, 16: 1e-6}[Q]   # quad's own error grows with |h_l|
    np.testing.assert_allclose(got, ref, atol=tol * np.abs(ref).max())


@pytest.mark.parametrize("Q", [3, 4, 8, 16])
def test_hh_equilibrium_moments(Q):
    vs = VelocitySet(Q)
    u = np.array([0.0, 0.3, -0.45, 0.1])
    T = np.array([1.0, 1.4, 0.6, 2.2])
    g = hh_equilibrium(Q, Q - 1, u, T)
    p = vs.px
    np.testing.assert_allclose(g.sum(-1), 1.0, rtol=1e-13)
    np.testing.assert_allclose((g * p).sum(-1), u, atol=1e-13)
    np.testing.assert_allclose(((p[None] - u[:, None]) ** 2 * g).sum(-1), T, rtol=1e-13)
    # half-range moments too (exact for orders <= N): int_0^inf p g dp
    from scipy.special import erf
    zeta = u / np.sqrt(2 * T)
    half0 = 0.5 * (1 + erf(zeta))
    np.testing.assert_allclose(g[:, :Q].sum(-1), half0, rtol=1e-12)
    # at rest and unit temperature the equilibrium is the weight vector
    np.testing.assert_allclose(hh_equilibrium(Q, Q - 1, 0.0, 1.0), vs.wx, rtol=1e-13)


def test_hh_equilibrium_decimal_path_agrees_with_fp64():
    # Forcing the 80-digit path on a well-conditioned case gives the same numbers.
    u, T = np.array([0.2, -0.3]), np.array([1.1, 0.8])
    fast = hh_equilibrium(4, 3, u, T)
    slow = hh_equilibrium(4, 3, u, T, tol=0.0)
    np.testing.assert_allclose(fast, slow, rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("Q,u,T", [(4, 0.3, 1.4), (8, -0.5, 0.6), (16, 0.2, 1.7)])
def test_h_equilibrium_by_projection_integrals(Q, u, T):
    # G_l = int g He_l dp by adaptive quadrature; g_k = w_k sum G_l He_l(z_k)/l!.
    N = Q - 1
    d = gauss_hermite(Q)
    z, w = to_f64(d["z"]), to_f64(d["w"])
    He = lambda l, x: np.polynomial.hermite_e.hermeval(x, [0] * l + [1])
    G = [integrate.quad(lambda p: _g(p, u, T) * He(l, p), -np.inf, np.inf,
                        epsabs=1e-14, epsrel=1e-13, limit=400)[0] for l in range(N + 1)]
    ref = np.array([w[k] * sum(G[l] * He(l, z[k]) / math.factorial(l) for l in range(N + 1))
                    for k in range(Q)])
    np.testing.assert_allclose(h_equilibrium(Q, N, u, T), ref, atol=1e-10 * np.abs(ref).max())
    g = h_equilibrium(Q, N, u, T)
    assert g.sum() == pytest.approx(1.0, rel=1e-13)
    assert (g * z).sum() == pytest.approx(u, abs=1e-13)
    assert ((z - u) ** 2 * g).sum() == pytest.approx(T, rel=1e-13)


@pytest.mark.parametrize("Qx", [4, 8])
def test_full_range_x_set_layout_and_moments(Qx):
    # The HLB set along p_x (x_full): the Gauss-Hermite nodes re-ordered as
    # +z (ascending) then -z, with weights, K^H and g_x permuted the same way.
    # Pinned by the node layout, the K^H identities in that order (mass:
    # sum_k K_kk' = 0; momentum: sum_k p_k K_kk' = -1 per column, the discrete
    # form of int p d_p f = -int f) and exact equilibrium moments.
    from oracle.quadrature import gauss_hermite, to_f64
    vs = VelocitySet(Qx, 4, 0, x_full=True)
    z = np.sort(np.abs(to_f64(gauss_hermite(Qx)["z"])))[::2]
    np.testing.assert_allclose(vs.px, np.concatenate([z, -z]), rtol=1e-14)
    assert vs.QH == Qx // 2 and (vs.px[:Qx // 2] > 0).all()
    np.testing.assert_allclose(vs.Kx.sum(axis=0), 0.0, atol=1e-12)
    np.testing.assert_allclose((vs.px[:, None] * vs.Kx).sum(axis=0), -1.0, atol=1e-12)
    n, ux, uy, T = 1.1, 0.3, -0.2, 0.9
    f = vs.equilibrium(np.float64(n), ux, uy, 0.0, np.float64(T))
    px, py = vs.px[None, None, :], vs.py[None, :, None]
    assert f.sum() == pytest.approx(n, rel=1e-13)
    assert (f * px).sum() / n == pytest.approx(ux, abs=1e-13)
    assert (f * py).sum() / n == pytest.approx(uy, abs=1e-13)
    assert (f * ((px - ux) ** 2 + (py - uy) ** 2)).sum() / (2 * n) == pytest.approx(T, rel=1e-13)
    # the permuted g_x is the full-range equilibrium at the permuted nodes
    from oracle.model import h_equilibrium
    g = h_equilibrium(Qx, Qx - 1, ux, T)
    zz = to_f64(gauss_hermite(Qx)["z"])
    for k, p in enumerate(vs.px):
        assert vs.g_x(ux, T)[k] == pytest.approx(g[int(np.argmin(np.abs(zz - p)))], rel=1e-14)


@pytest.mark.parametrize("Q", [1, 3, 8, 16])
def test_gauss_laguerre_half_quadrature(Q):
    # Half-range Gauss-Laguerre (Sec. IV.B, weights of Eq. "eq:wk_half"):
    # exact on z^s exp(-z) for s <= 2Q - 1 (int = s!), and the nodes/weights
    # of numpy's laggauss (a library routine).
    import math
    from oracle.quadrature import gauss_laguerre_half, to_f64
    d = gauss_laguerre_half(Q)
    z, w = to_f64(d["z"]), to_f64(d["w"])
    for s_ in range(2 * Q):
        assert (w * z ** s_).sum() == pytest.approx(math.factorial(s_), rel=1e-12)
    x0, w0 = np.polynomial.laguerre.laggauss(Q)
    np.testing.assert_allclose(z, x0, rtol=1e-12)
    np.testing.assert_allclose(w, w0, rtol=1e-10, atol=1e-300)


@pytest.mark.parametrize("Q", [3, 4, 8])
def test_hl_force_matrix_identities(Q):
    # K^L of Eq. "eq:hh_Kk_L": the discrete d/dp conserves mass (sum_k K = 0),
    # gives -1 for the momentum (sum_k p_k K_kk' = -1) and -2 p_k' for the
    # energy; without the jump term (-Phi0 Phi0 / 2) mass is not conserved.
    from oracle.model import hl_force_matrix
    vs = VelocitySet(Q, x_laguerre=True)
    K, p = vs.Kx, vs.px
    scale = np.abs(K).max()
    np.testing.assert_allclose(K.sum(axis=0), 0.0, atol=1e-12 * scale)
    np.testing.assert_allclose((p[:, None] * K).sum(axis=0), -1.0, atol=1e-12 * scale)
    np.testing.assert_allclose((p[:, None] ** 2 * K).sum(axis=0), -2 * p, atol=1e-12 * scale * p.max())
    # planted mistake: the jump term replaced by what differentiating each half
    # separately gives (-omega(0) Phi0 Phi0 within a half, omega(0) = 1), as in
    # the half-range Hermite test above: mass is no longer conserved
    from oracle.quadrature import gauss_laguerre_half, to_f64
    d = gauss_laguerre_half(Q)
    w = to_f64(d["w"])
    Phi0 = np.array([sum(float(poly_eval(d["L"][l], zk)) for l in range(Q)) for zk in d["z"]])
    P, W = np.concatenate([Phi0, Phi0]), np.concatenate([w, -w])
    same = np.kron(np.eye(2), np.ones((Q, Q)))
    bad = hl_force_matrix(Q) + W[:, None] * (0.5 - same) * np.outer(P, P)
    assert np.abs(bad.sum(axis=0)).max() > 1e-3


@pytest.mark.parametrize("u,T", [(0.0, 1.0), (0.4, 0.8), (-0.7, 1.5)])
def test_hl_equilibrium_by_projection_integrals(u, T):
    # G_l^{+-} = int_0^inf g(+-p) L_l(p) dp by adaptive quadrature (scipy), and
    # the moments n, u, T of the projected equilibrium (exact for N >= 2).
    from scipy.integrate import quad
    from scipy.special import eval_laguerre
    from oracle.model import hl_equilibrium
    from oracle.quadrature import gauss_laguerre_half, to_f64
    Q, N = 6, 5
    d = gauss_laguerre_half(Q)
    z, w = to_f64(d["z"]), to_f64(d["w"])
    g = lambda p: math.exp(-(p - u) ** 2 / (2 * T)) / math.sqrt(2 * math.pi * T)
    ref = np.zeros(2 * Q)
    for half, sgn in ((0, 1), (1, -1)):
        G = [quad(lambda p: g(sgn * p) * eval_laguerre(l, p), 0, np.inf, epsabs=1e-14, epsrel=1e-13)[0]
             for l in range(N + 1)]
        for k in range(Q):
            ref[half * Q + k] = w[k] * sum(eval_laguerre(l, z[k]) * G[l] for l in range(N + 1))
    got = hl_equilibrium(Q, N, u, T)
    np.testing.assert_allclose(got, ref, atol=1e-11)
    vs = VelocitySet(Q, x_laguerre=True)
    assert got.sum() == pytest.approx(1.0, rel=1e-12)
    assert (got * vs.px).sum() == pytest.approx(u, abs=1e-12)
    assert (got * (vs.px - u) ** 2).sum() == pytest.approx(T, rel=1e-11)


def test_direct_product_equilibrium_moments():
    # App. A: feq = n g_x g_y g_z reproduces n, u and T = sum |p-u|^2 f/(D n).
    vs = VelocitySet(4, 4, 4)   # N = Q - 1 >= 2 on every axis
    n, ux, uy, uz, T = 1.3, 0.2, -0.1, 0.05, 1.2
    f = vs.equilibrium(np.float64(n), ux, uy, uz, np.float64(T))
    px, py, pz = vs.px[None, None, :], vs.py[None, :, None], vs.pz[:, None, None]
    assert f.sum() == pytest.approx(n, rel=1e-13)
    assert (f * px).sum() / n == pytest.approx(ux, abs=1e-13)
    assert (f * py).sum() / n == pytest.approx(uy, abs=1e-13)
    assert (f * pz).sum() / n == pytest.approx(uz, abs=1e-13)
    c2 = (px - ux) ** 2 + (py - uy) ** 2 + (pz - uz) ** 2
    assert (f * c2).sum() / (3 * n) == pytest.approx(T, rel=1e-13)
