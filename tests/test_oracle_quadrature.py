"""Pins of the oracle's quadratures against closed forms, brute force and numpy.

Half-range Hermite quadrature: Sec. IV.B.1 (Eqs. "eq:hh_quad", "eq:wk_half"),
App. B.  Full-range Gauss-Hermite: Sec. IV.A.1 (Eqs. "eq:H_quad", "eq:H_wk").
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle.quadrature import gauss_hermite, half_range_hermite, to_f64


def mu(s):
    """int_0^inf z^s exp(-z^2/2)/sqrt(2 pi) dz via the Gamma function."""
    return 2.0 ** ((s - 1) / 2.0) * math.gamma((s + 1) / 2.0) / math.sqrt(2 * math.pi)


def test_q1_closed_form():
    # h_1 is proportional to z - mu_1/mu_0: root sqrt(2/pi), weight mu_0 = 1/2.
    d = half_range_hermite(1)
    assert float(d["z"][0]) == pytest.approx(math.sqrt(2 / math.pi), rel=1e-15)
    assert float(d["w"][0]) == pytest.approx(0.5, rel=1e-15)


def test_q2_closed_form():
    # Monic pi_2 = z^2 + a z + b orthogonal to 1 and z; roots by the quadratic
    # formula; weights from sum_k w_k z_k^s = mu_s for s = 0, 1.
    m = [mu(s) for s in range(4)]
    A = np.array([[m[1], m[0]], [m[2], m[1]]])
    a, b = np.linalg.solve(A, [-m[2], -m[3]])
    r = np.sort(np.roots([1.0, a, b]).real)
    w = np.linalg.solve(np.vstack([np.ones(2), r]), [m[0], m[1]])
    d = half_range_hermite(2)
    np.testing.assert_allclose(to_f64(d["z"]), r, rtol=1e-13)
    np.testing.assert_allclose(to_f64(d["w"]), w, rtol=1e-13)


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 5, 8, 12, 16])
def test_half_range_exactness_brute_force(Q):
    # Gauss rule of order Q is exact for degree < 2Q (Sec. IV.B.1), and not beyond.
    d = half_range_hermite(Q)
    z, w = to_f64(d["z"]), to_f64(d["w"])
    assert np.all(z > 0) and np.all(np.diff(z) > 0) and np.all(w > 0)
    for s in range(2 * Q):
        assert np.sum(w * z ** s) == pytest.approx(mu(s), rel=2e-13)
    if Q <= 8:   # the degree-2Q defect shrinks fast with Q; FP64 resolves it up to Q = 8
        assert abs(np.sum(w * z ** (2 * Q)) - mu(2 * Q)) > 1e-9 * mu(2 * Q)


@pytest.mark.parametrize("Q", [2, 4, 8])
def test_half_range_orthonormality_by_integration(Q):
    # <h_l, h_l'> = delta over [0, inf) with omega, integrated numerically.
    C = half_range_hermite(Q)["C"]
    om = lambda z: math.exp(-z * z / 2) / math.sqrt(2 * math.pi)
    h = lambda l, z: sum(float(C[l][s]) * z ** s for s in range(l + 1))
    for l in range(Q + 1):
        for lp in range(l + 1):
            val, _ = integrate.quad(lambda z: om(z) * h(l, z) * h(lp, z), 0, np.inf,
                                    epsabs=1e-13, epsrel=1e-12, limit=200)
            assert val == pytest.approx(1.0 if l == lp else 0.0, abs=1e-9)
        assert float(C[l][l]) > 0


@pytest.mark.parametrize("Q", [2, 4, 8, 16])
def test_half_range_christoffel_weights(Q):
    # For orthonormal polynomials the Gauss weights are 1 / sum_{l<Q} h_l(z_k)^2,
    # a different formula from Eq. "eq:wk_half" used by the oracle.
    d = half_range_hermite(Q)
    C = d["C"]
    from oracle.quadrature import poly_eval
    for zk, wk in zip(d["z"], d["w"]):
        s = sum(poly_eval(C[l][: l + 1], zk) ** 2 for l in range(Q))
        assert float(1 / s) == pytest.approx(float(wk), rel=1e-14)


@pytest.mark.parametrize("Q", range(1, 17))
def test_half_range_envelope(Q):
    # All half-range Hermite points lie within +-2.5 sqrt(Q) (Fig. "hh_hyp" caption).
    z = to_f64(half_range_hermite(Q)["z"])
    assert z.max() < 2.5 * math.sqrt(Q)


@pytest.mark.parametrize("Q", [2, 4, 6, 8, 16])
def test_gauss_hermite_matches_numpy(Q):
    # Probabilists' Gauss-Hermite with omega normalised to unit mass.
    x, w = np.polynomial.hermite_e.hermegauss(Q)
    d = gauss_hermite(Q)
    np.testing.assert_allclose(to_f64(d["z"]), x, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(to_f64(d["w"]), w / math.sqrt(2 * math.pi), rtol=1e-12)
    assert np.abs(to_f64(d["z"])).max() < 2 * math.sqrt(Q)   # envelope +-2 sqrt(Q)


# --- orders up to the paper's HHLB(20;200) (oracle/highorder.py; needs mpmath) ----
@pytest.mark.parametrize("Q", [4, 16, 32])
def test_highorder_route_matches_the_80_digit_route(Q):
    # Two independent constructions (monomial coefficients in Decimal; the
    # Golub-Welsch recurrence in mpmath): nodes, weights and K^h agree to the
    # last FP64 bit.
    pytest.importorskip("mpmath")
    from oracle.highorder import half_range_hermite_hp, hh_force_matrix_hp
    from oracle.model import hh_force_matrix
    hp, dec = half_range_hermite_hp(Q), half_range_hermite(Q)
    np.testing.assert_allclose([float(x) for x in hp["z"]], to_f64(dec["z"]), rtol=1e-15)
    np.testing.assert_allclose([float(x) for x in hp["w"]], to_f64(dec["w"]), rtol=1e-14)
    K0 = hh_force_matrix(Q)
    np.testing.assert_allclose(hh_force_matrix_hp(Q), K0, atol=1e-14 * np.abs(K0).max())


@pytest.mark.slow
def test_highorder_quadrature_at_order_200():
    # HHLB(20;200)'s half-range quadrature (Sec. V): exact on z^s omega(z) for
    # every s < 2Q = 400 (relative to mu_s, at the working precision), all
    # nodes inside the 2.5 sqrt(Q) envelope of the paper's Fig. "fig:hh_hyp",
    # positive weights summing to mu_0 = 1/2.
    mp = pytest.importorskip("mpmath")
    from oracle.highorder import half_moment_mp, half_range_hermite_hp
    Q = 200
    d = half_range_hermite_hp(Q)
    z, w = d["z"], d["w"]
    with mp.workdps(d["dps"]):
        worst = max(abs(mp.fsum(wk * zk ** s for zk, wk in zip(z, w)) / half_moment_mp(s) - 1) for s in range(2 * Q))
        assert worst < mp.mpf(10) ** -300
        assert abs(mp.fsum(w) - mp.mpf(1) / 2) < mp.mpf(10) ** -300
    assert all(x > 0 for x in w)
    assert 0 < float(z[0]) and float(z[-1]) < 2.5 * Q ** 0.5
    assert all(float(z[k]) < float(z[k + 1]) for k in range(Q - 1))


def test_highorder_force_matrix_identities():
    # K^h at Q = 64 from the recurrence-based route: per column, mass
    # (sum_k K = 0), momentum (sum_k p_k K = -1) and the derivative of the rest
    # Maxwellian (K w = -p w), each relative to the column's magnitude (the
    # entries span 30 orders of magnitude at this order).
    pytest.importorskip("mpmath")
    from oracle.highorder import half_range_hermite_hp, hh_force_matrix_hp
    Q = 64
    d = half_range_hermite_hp(Q)
    K = hh_force_matrix_hp(Q)
    z = np.array([float(x) for x in d["z"]])
    w = np.array([float(x) for x in d["w"]])
    p, W = np.concatenate([z, -z]), np.concatenate([w, w])
    assert (np.abs(K.sum(axis=0)) / np.abs(K).sum(axis=0)).max() < 1e-14
    assert (np.abs((p[:, None] * K).sum(axis=0) + 1) / np.abs(p[:, None] * K).sum(axis=0)).max() < 1e-14
    assert np.abs(K @ W + p * W).max() < 1e-12 * np.abs(p * W).max()


def test_stored_order_200_tables_match_the_mpmath_construction():
    # tests/golden/half_range_hermite_q200.txt (written by
    # tests/golden/make_half_range_tables.py from oracle.highorder) holds the
    # 560-digit tables rounded to 40 digits.
    mp = pytest.importorskip("mpmath")
    from oracle.highorder import half_range_hermite_hp, read_store, store_path
    Q = 200
    st = read_store(store_path(Q))
    d = half_range_hermite_hp(Q)
    with mp.workdps(60):
        for key in ("z", "w"):
            assert max(abs(mp.mpf(str(x)) / y - 1) for x, y in zip(st[key], d[key])) < mp.mpf(10) ** -38
        for key in ("a", "b"):
            assert max(abs(mp.mpf(str(x)) / y - 1) for x, y in zip(st[key], d[key][:Q + 1])) < mp.mpf(10) ** -38
        assert abs(mp.mpf(str(st["h0"])) / d["h0"] - 1) < mp.mpf(10) ** -38


@pytest.mark.parametrize("Q", [16, 64])
def test_fp64_force_matrix_from_the_recurrence_matches_mpmath(Q):
    # hh_force_matrix_rec (FP64 values h_l(z_k) by the recurrence) against the
    # mpmath evaluation of the same formula, per column.
    pytest.importorskip("mpmath")
    from oracle.highorder import hh_force_matrix_hp, hh_force_matrix_rec
    K, ref = hh_force_matrix_rec(Q), hh_force_matrix_hp(Q)
    assert (np.abs(K - ref) / np.abs(ref).max(axis=0)[None, :]).max() < 1e-12


def test_order_200_velocity_set_reproduces_moments_and_derivatives():
    # The oracle's HHLB(20;200) set (stored tables, no mpmath): the order-20
    # projection of a Maxwellian keeps n, u and T (Eq. "eq:hh_gk" preserves
    # the moments up to order N), K^h acts as -d/dp on moments (sum_k p_k^s
    # (K f)_k = -s sum_k p_k^(s-1) f_k for s <= 3: integration by parts with
    # the jump at p = 0 included), and K^h annihilates nothing of the mass.
    from oracle.model import VelocitySet
    vs = VelocitySet(200, Nx=20)
    assert vs.V == 400 and vs.px.max() < 2.5 * 200 ** 0.5
    for u, T in ((0.0, 1.0), (0.3, 0.7), (-0.5, 1.6)):
        f = vs.g_x(np.array(u), np.array(T))
        n = f.sum()
        j = (vs.px * f).sum()
        E = (vs.px ** 2 * f).sum()
        assert n == pytest.approx(1.0, rel=1e-13)
        assert j / n == pytest.approx(u, abs=1e-13)
        assert E / n - (j / n) ** 2 == pytest.approx(T, rel=1e-13)
        Kf = vs.Kx @ f
        for s in range(4):
            lhs = (vs.px ** s * Kf).sum()
            rhs = -s * (vs.px ** (s - 1) * f).sum() if s else 0.0
            assert lhs == pytest.approx(rhs, abs=1e-12 * max(1.0, abs(rhs)))
