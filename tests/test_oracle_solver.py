"""Pins of the oracle's time step: WENO-5 limits, orders of accuracy, RK-3,
the homogeneous-force closed form, the free-molecular closed form, the
isothermal barometric profile and conservation of the particle number.

Sections: Sec. IV.C (numerical method), Sec. V (numerical results), App. A.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.solver import Config, Solver, face_fluxes, grid_x, weno5_face, weno5_weights

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _weno_table():
    rows = []
    with open(os.path.join(GOLDEN, "weno_zero_limits.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "eq":
                pattern, w = None, tok[1:]
            else:
                pattern, w = [int(t) for t in tok[:3]], tok[3:]
            rows.append((pattern, [float(Fraction(x)) for x in w]))
    return rows


@pytest.mark.parametrize("pattern,expect", _weno_table())
def test_weno_zero_limits_table(pattern, expect):
    # Tab. "weno": every listed zero pattern of the smoothness indicators.
    rng = np.random.default_rng(1)
    if pattern is None:
        for v in (0.0, 0.37, 5.0):
            got = weno5_weights(v, v, v)
            np.testing.assert_allclose(got, expect, rtol=1e-15)
        return
    s = [0.0 if z == 0 else rng.uniform(0.1, 3.0) for z in pattern]
    np.testing.assert_allclose(weno5_weights(*s), expect, rtol=1e-15, atol=0)


def test_weno_weights_limit_is_continuous():
    # delta_q / sigma_q^2 tends to the table entry as sigma_1 -> 0.
    w = weno5_weights(1e-30, 0.5, 0.7)
    assert w[0] == pytest.approx(1.0, abs=1e-12)


def _periodic_divergence(fun, n, scheme, v=1.0):
    x = (np.arange(n) + 0.5) / n
    f = fun(x)
    fe = np.concatenate([f[-3:], f, f[:3]])
    F = face_fluxes(fe, np.array(v), 0, scheme)
    return x, (F[1:] - F[:-1]) * n


@pytest.mark.parametrize("scheme,l1_order,linf_order", [("weno5", 3.8, 2.8), ("upwind2", 1.9, 1.9)])
@pytest.mark.parametrize("v", [1.0, -1.0])
def test_advection_order_of_accuracy(scheme, l1_order, linf_order, v):
    # Smooth periodic profile: error of v d_x f falls as a power of dx.  WENO-5
    # without epsilon keeps its 5th-order candidates away from critical points
    # but, as ``sigma -> 0`` there, drops to 3rd order pointwise (the effect the
    # paper's reference on mapped WENO describes); the L1 rate stays above 4.
    fun = lambda x: 1.5 + np.sin(2 * np.pi * x) + 0.3 * np.cos(4 * np.pi * x)
    dfun = lambda x: 2 * np.pi * np.cos(2 * np.pi * x) - 1.2 * np.pi * np.sin(4 * np.pi * x)
    e1, einf = [], []
    for n in (80, 160, 320, 640):
        x, div = _periodic_divergence(fun, n, scheme, v)
        err = np.abs(div - v * dfun(x))
        e1.append(err.mean())
        einf.append(err.max())
    r1 = [math.log2(e1[i] / e1[i + 1]) for i in range(3)]
    rinf = [math.log2(einf[i] / einf[i + 1]) for i in range(3)]
    assert min(r1) > l1_order and min(rinf) > linf_order, (r1, rinf)


def test_weno_face_reconstructs_quadratics_exactly():
    # Each candidate is exact for quadratics, so WENO is too, for any weights.
    q = lambda x: 0.3 * x * x - 1.1 * x + 2.0
    cells = [q(i) for i in range(-2, 3)]
    # cell-centred point values: the face value at +1/2 of the quadratic
    # interpolant through the point values is a fixed linear combination.
    F = weno5_face(*cells)
    # candidate 2 (symmetric) evaluated by hand
    F2 = -cells[1] / 6 + 5 * cells[2] / 6 + cells[3] / 3
    assert F == pytest.approx(F2, rel=1e-14)


def test_rk3_stability_polynomial():
    # TVD RK-3 (Eq. "eq:rk3") applied to f' = lam f multiplies f by
    # 1 + z + z^2/2 + z^3/6 with z = lam dt (3rd order, Tab. "rk3").
    s = Solver(Config(Qx=1, nx=4, Kn=math.inf))
    lam = -0.7 + 0.0
    s.rhs = lambda f: lam * f
    s.f = np.ones_like(s.f)
    z = lam * s.dt
    s.step(1)
    np.testing.assert_allclose(s.f, 1 + z + z * z / 2 + z ** 3 / 6, rtol=1e-15)


@pytest.mark.parametrize("Qx,Qy,Qz,ax,ay,az", [(4, 0, 0, -0.3, 0, 0), (4, 4, 0, 0.2, -0.4, 0),
                                             (3, 4, 4, -0.1, 0.2, 0.3)])
def test_homogeneous_force_and_bgk_closed_form(Qx, Qy, Qz, ax, ay, az):
    # Without advection n is constant, u(t) = u0 + a t and T is constant,
    # for any Kn and a non-Maxwellian start: the K identities make the moment
    # equations polynomial in t of degree <= 2, which RK-3 integrates exactly.
    s = Solver(Config(Qx=Qx, Qy=Qy, Qz=Qz, nx=3, ax=ax, ay=ay, az=az, Kn=0.3, dt=0.01))
    s.init_equilibrium(1.2, 0.1, -0.05, 0.9)
    rng = np.random.default_rng(3)
    s.f = s.f * (1 + 0.1 * rng.uniform(-1, 1, s.f.shape))
    n0, u0, T0, _ = s.moments()
    for _ in range(50):
        f = s.f
        f1 = f + s.dt * s.source(f)
        f2 = 0.75 * f + 0.25 * f1 + 0.25 * s.dt * s.source(f1)
        s.f = f / 3 + 2 / 3 * f2 + 2 / 3 * s.dt * s.source(f2)
    t = 50 * s.dt
    n, u, T, _ = s.moments()
    np.testing.assert_allclose(n, n0, rtol=1e-13)
    np.testing.assert_allclose(u, u0 + np.array([ax, ay, az]) * t, atol=1e-13)
    np.testing.assert_allclose(T, T0, rtol=1e-12)


def test_homogeneous_force_and_bgk_closed_form_order_200():
    # The same closed form with the HHLB(20;200) set of Sec. V (stored tables):
    # K^h of order 200 and the order-20 projected equilibrium keep n and T and
    # move u by a t exactly, with 400 velocities whose weights reach 5e-221.
    s = Solver(Config(Qx=200, Nx_eq=20, nx=3, ax=-0.3, Kn=0.3, dt=0.001))
    s.init_equilibrium(1.2, 0.1, -0.05, 0.9)
    rng = np.random.default_rng(3)
    s.f = s.f * (1 + 0.1 * rng.uniform(-1, 1, s.f.shape))
    n0, u0, T0, _ = s.moments()
    for _ in range(20):
        f = s.f
        f1 = f + s.dt * s.source(f)
        f2 = 0.75 * f + 0.25 * f1 + 0.25 * s.dt * s.source(f1)
        s.f = f / 3 + 2 / 3 * f2 + 2 / 3 * s.dt * s.source(f2)
    n, u, T, _ = s.moments()
    np.testing.assert_allclose(n, n0, rtol=1e-13)
    np.testing.assert_allclose(u, u0 + np.array([-0.3, 0.0, 0.0]) * 20 * s.dt, atol=1e-13)
    np.testing.assert_allclose(T, T0, rtol=1e-12)


@pytest.mark.parametrize("Qx,Qy,Qz", [(4, 0, 0), (8, 4, 0), (6, 4, 4)])
def test_homogeneous_force_closed_form_full_range_x(Qx, Qy, Qz):
    # The same closed form for the HLB set along p_x (K^H, no jump term).
    ax, ay, az = -0.25, 0.15, -0.1
    s = Solver(Config(Qx=Qx, Qy=Qy, Qz=Qz, nx=3, ax=ax, ay=ay, az=az, Kn=0.3, dt=0.01, x_basis=1))
    s.init_equilibrium(1.1, 0.1, -0.05, 0.95)
    rng = np.random.default_rng(4)
    s.f = s.f * (1 + 0.1 * rng.uniform(-1, 1, s.f.shape))
    n0, u0, T0, _ = s.moments()
    for _ in range(50):
        f = s.f
        f1 = f + s.dt * s.source(f)
        f2 = 0.75 * f + 0.25 * f1 + 0.25 * s.dt * s.source(f1)
        s.f = f / 3 + 2 / 3 * f2 + 2 / 3 * s.dt * s.source(f2)
    a = np.array([ax, ay if Qy else 0.0, az if Qz else 0.0])
    n, u, T, _ = s.moments()
    np.testing.assert_allclose(n, n0, rtol=1e-13)
    np.testing.assert_allclose(u, u0 + a * 50 * s.dt, atol=1e-13)
    np.testing.assert_allclose(T, T0, rtol=1e-12)


@pytest.mark.parametrize("Qx,Qy", [(4, 0), (8, 4)])
def test_free_molecular_discrete_closed_form_full_range_x(Qx, Qy):
    # HLB along p_x between walls at T_L != T_R, g = 0, Kn = inf: the steady
    # state is f = n_L g_L (p_x > 0), n_R g_R (p_x < 0) at every node, with the
    # zero-flux condition n_L J(T_L) = n_R J(T_R), J(T) = sum_{p_x > 0} p_x g_x(0, T)
    # (the Gauss-Hermite half sums are not the continuous half-range moments,
    # which is why HLB is inexact at walls, Sec. V).  So n = n_L A_L + n_R A_R with
    # A(T) = sum_{p_x > 0} g_x(0, T), uniform in x.
    TL, TR = 0.8, 1.7
    s = Solver(Config(Qx=Qx, Qy=Qy, nx=12, advection="upwind2", T_left=TL, T_right=TR, x_basis=1))
    s.init_equilibrium()
    for _ in range(200):
        fo = s.f.copy()
        s.step(100)
        if s.residual(fo, s.f) < 1e-13:
            break
    vs = s.vs
    h = vs.QH
    J = lambda T: float((vs.px[:h] * vs.g_x(0.0, T)[:h]).sum())
    A = lambda T: float(vs.g_x(0.0, T)[:h].sum())
    nl, nr = s.last_wall_density
    np.testing.assert_allclose(nl * J(TL), nr * J(TR), rtol=1e-11)
    n, u, T, q = s.moments()
    np.testing.assert_allclose(n, nl[0] * A(TL) + nr[0] * A(TR), rtol=1e-11)
    np.testing.assert_allclose(u, 0.0, atol=1e-11)


def test_barometric_interior_residual_full_range_x():
    # f = exp(-g x) g(0, 1) is the steady state for the HLB set too (K^H maps
    # the Maxwellian at rest exactly); interior residual O(dx^2) for upwind2.
    g = 0.5
    res = []
    for nx in (32, 64, 128):
        s = Solver(Config(Qx=8, Qy=4, nx=nx, advection="upwind2", ax=-g, Kn=0.3, x_basis=1))
        n = np.exp(-g * s.xc)
        s.f = n[None, :, None, None, None] * s.vs.equilibrium(np.float64(1.0), 0.0, 0.0, 0.0, np.float64(1.0))[None, None]
        res.append(np.abs(s.rhs(s.f)[:, 5:-5]).max())
    assert res[0] / res[1] > 3.5 and res[1] / res[2] > 3.5


@pytest.mark.parametrize("x_basis", [1, 2])
def test_half_range_laguerre_and_full_range_x_closed_forms(x_basis):
    # The closed forms of the tests above for the other p_x families: the
    # homogeneous force (u = u0 + a t exactly, n and T constant), the
    # free-molecular state in its discrete form (n_L J(T_L) = n_R J(T_R),
    # J(T) = sum_{p_x > 0} p_x g_x(0, T); n = n_L A(T_L) + n_R A(T_R)), and the
    # second-order barometric residual (Gauss-Hermite only: the Laguerre weight
    # exp(-z) does not match the Maxwellian, so the projected rest state is not
    # mapped exactly by K^L and the residual stays O(1) at small Q, a model
    # error, not a discretisation one).  x_basis 2 is the half-range
    # Gauss-Laguerre set (K^L of Eq. "eq:hh_Kk_L").
    Qx = 4 if x_basis == 2 else 8
    s = Solver(Config(Qx=Qx, Qy=4, nx=3, ax=-0.25, ay=0.15, Kn=0.3, dt=0.005, x_basis=x_basis))
    s.init_equilibrium(1.1, 0.1, -0.05, 0.95)
    rng = np.random.default_rng(5)
    s.f = s.f * (1 + 0.1 * rng.uniform(-1, 1, s.f.shape))
    n0, u0, T0, _ = s.moments()
    for _ in range(40):
        f = s.f
        f1 = f + s.dt * s.source(f)
        f2 = 0.75 * f + 0.25 * f1 + 0.25 * s.dt * s.source(f1)
        s.f = f / 3 + 2 / 3 * f2 + 2 / 3 * s.dt * s.source(f2)
    n, u, T, _ = s.moments()
    np.testing.assert_allclose(n, n0, rtol=1e-12)
    np.testing.assert_allclose(u, u0 + np.array([-0.25, 0.15, 0.0]) * 40 * s.dt, atol=1e-12)
    np.testing.assert_allclose(T, T0, rtol=1e-11)
    TL, TR = 0.8, 1.7
    s = Solver(Config(Qx=Qx, nx=10, advection="upwind2", T_left=TL, T_right=TR, x_basis=x_basis))
    s.init_equilibrium()
    for _ in range(400):
        fo = s.f.copy()
        s.step(100)
        if s.residual(fo, s.f) < 1e-13:
            break
    vs, h = s.vs, s.vs.QH
    J = lambda T_: float((vs.px[:h] * vs.g_x(0.0, T_)[:h]).sum())
    A = lambda T_: float(vs.g_x(0.0, T_)[:h].sum())
    nl, nr = s.last_wall_density
    np.testing.assert_allclose(nl * J(TL), nr * J(TR), rtol=1e-10)
    np.testing.assert_allclose(s.moments()[0], nl[0] * A(TL) + nr[0] * A(TR), rtol=1e-10)
    if x_basis == 2:
        return
    g = 0.5
    res = []
    for nx in (32, 64, 128):
        s = Solver(Config(Qx=Qx, nx=nx, advection="upwind2", ax=-g, Kn=0.3, x_basis=x_basis))
        n = np.exp(-g * s.xc)
        s.f = n[None, :, None, None, None] * s.vs.equilibrium(np.float64(1.0), 0.0, 0.0, 0.0, np.float64(1.0))[None, None]
        res.append(np.abs(s.rhs(s.f)[:, 5:-5]).max())
    assert res[0] / res[1] > 3.5 and res[1] / res[2] > 3.5


@pytest.mark.parametrize("Qx,Qy,Qz", [(4, 0, 0), (4, 4, 0), (3, 4, 4)])
def test_homogeneous_force_field_closed_form(Qx, Qy, Qz):
    # A per-node acceleration field on top of the uniform one: without
    # advection every node evolves on its own, so n and T stay constant and
    # u(t) = u0 + a(node) t exactly at every node (the closed form above, node
    # by node).  A field applied to the wrong nodes, or transposed, fails it.
    rng = np.random.default_rng(11)
    ny, nx = 2, 3
    fields = {k: rng.uniform(-0.4, 0.4, (ny, nx)) for k in ("ax_field", "ay_field", "az_field")}
    uni = (0.1, -0.05, 0.2)
    s = Solver(Config(Qx=Qx, Qy=Qy, Qz=Qz, nx=nx, ny=ny, ax=uni[0], ay=uni[1], az=uni[2], Kn=0.3, dt=0.01,
                      **fields))
    s.init_equilibrium(1.2, 0.1, -0.05, 0.9)
    s.f = s.f * (1 + 0.1 * rng.uniform(-1, 1, s.f.shape))
    n0, u0, T0, _ = s.moments()
    for _ in range(40):
        f = s.f
        f1 = f + s.dt * s.source(f)
        f2 = 0.75 * f + 0.25 * f1 + 0.25 * s.dt * s.source(f1)
        s.f = f / 3 + 2 / 3 * f2 + 2 / 3 * s.dt * s.source(f2)
    t = 40 * s.dt
    n, u, T, _ = s.moments()
    a = np.stack([uni[0] + fields["ax_field"], uni[1] + fields["ay_field"], uni[2] + fields["az_field"]], axis=-1)
    for k, Qk in enumerate((Qx, Qy, Qz)):
        if k and not Qk:
            a[..., k] = 0.0          # an absent momentum axis feels no force
    np.testing.assert_allclose(n, n0, rtol=1e-13)
    np.testing.assert_allclose(u, u0 + a * t, atol=1e-13)
    np.testing.assert_allclose(T, T0, rtol=1e-12)


def test_potential_barometric_interior_residual_is_second_order():
    # A gas at rest in a potential V(x) between walls at T = 1: f = n(x) w_k
    # with n = exp(-V(x)) is the exact steady state of Eq. "eq:boltz_force"
    # with a = -V'(x) (the isothermal profile of Eq. "eq:iso_n" for a general
    # potential).  Away from the walls the discrete L[f] is the upwind2
    # truncation error, O(dx^2); a field with the wrong sign (O(1)) or one
    # evaluated a node off (O(dx)) leaves ten times more at nx = 64.
    g, c = 0.4, 0.15
    V = lambda x: g * x + c * np.sin(2 * np.pi * x)
    dV = lambda x: g + 2 * np.pi * c * np.cos(2 * np.pi * x)
    res = []
    for nx in (32, 64, 128):
        xc = grid_x(nx, 1.0, 0.0)[1]
        s = Solver(Config(Qx=4, Qy=4, nx=nx, advection="upwind2", Kn=0.3, ax_field=-dV(xc)[None, :]))
        n = np.exp(-V(s.xc))
        s.f = n[None, :, None, None, None] * s.vs.equilibrium(np.float64(1.0), 0.0, 0.0, 0.0, np.float64(1.0))[None, None]
        res.append(np.abs(s.rhs(s.f)[:, 5:-5]).max())
    assert res[0] / res[1] > 3.5 and res[1] / res[2] > 3.5
    xc = grid_x(64, 1.0, 0.0)[1]
    for wrong in (+dV(xc), -np.roll(dV(xc), 1)):   # planted: sign flipped; field one node off
        s = Solver(Config(Qx=4, Qy=4, nx=64, advection="upwind2", Kn=0.3, ax_field=wrong[None, :]))
        n = np.exp(-V(s.xc))
        s.f = n[None, :, None, None, None] * s.vs.equilibrium(np.float64(1.0), 0.0, 0.0, 0.0, np.float64(1.0))[None, None]
        assert np.abs(s.rhs(s.f)[:, 5:-5]).max() > 10 * res[1]


@pytest.mark.parametrize("Qx,Qy,adv", [(4, 0, "weno5"), (4, 4, "upwind2"), (6, 4, "weno5")])
def test_free_molecular_closed_form(Qx, Qy, adv):
    # g = 0, Kn = inf, walls at T_L != T_R (Sec. V.D at g = 0): f is n_L g_L for
    # p_x > 0 and n_R g_R for p_x < 0 everywhere, with n_L sqrt(T_L) = n_R sqrt(T_R)
    # = c; n = c (T_L^-1/2 + T_R^-1/2)/2, T = sqrt(T_L T_R), u = 0,
    # (exact in the discrete model once N >= 3 along p_x and N >= 2 along p_y)
    # q_x = c (D + 1)(T_L - T_R) / (2 sqrt(2 pi))  (Eq. "eq:bal_q" for D = 1).
    TL, TR = 0.8, 1.7
    s = Solver(Config(Qx=Qx, Qy=Qy, nx=12, advection=adv, T_left=TL, T_right=TR))
    s.init_equilibrium()
    for _ in range(200):
        fo = s.f.copy()
        s.step(100)
        if s.residual(fo, s.f) < 1e-13:
            break
    n, u, T, q = s.moments()
    D = s.vs.D
    c = n.mean() * 2 / (TL ** -0.5 + TR ** -0.5)
    np.testing.assert_allclose(n, n.mean(), rtol=1e-11)
    np.testing.assert_allclose(T, math.sqrt(TL * TR), rtol=1e-11)
    np.testing.assert_allclose(u, 0.0, atol=1e-11)
    np.testing.assert_allclose(q, c * (D + 1) * (TL - TR) / (2 * math.sqrt(2 * math.pi)), rtol=1e-10)
    nl, nr = s.last_wall_density
    np.testing.assert_allclose(nl * math.sqrt(TL), nr * math.sqrt(TR), rtol=1e-11)


def test_barometric_interior_residual_is_second_order():
    # f = n(x) w_k with n ~ exp(-g x) (T_w = 1) is the exact steady state of
    # Eq. "eq:boltz_force" (Eq. "eq:iso_n"); away from the walls the discrete
    # L[f] is the upwind2 truncation error, O(dx^2).  A wrong force sign or
    # a wrong K makes it O(1).
    g = 0.5
    res = []
    for nx in (32, 64, 128):
        s = Solver(Config(Qx=4, Qy=4, nx=nx, advection="upwind2", ax=-g, Kn=0.3))
        n = np.exp(-g * s.xc)
        s.f = n[None, :, None, None, None] * s.vs.equilibrium(np.float64(1.0), 0.0, 0.0, 0.0, np.float64(1.0))[None, None]
        L = s.rhs(s.f)
        res.append(np.abs(L[:, 5:-5]).max())
    assert res[0] / res[1] > 3.5 and res[1] / res[2] > 3.5
    # planted mistake: the force with the wrong sign leaves an O(1) residual
    s = Solver(Config(Qx=4, nx=64, advection="upwind2", ax=+g, Kn=0.3))
    n = np.exp(-g * s.xc)
    s.f = n[None, :, None, None, None] * s.vs.wx[None, None, None, None, :]
    assert np.abs(s.rhs(s.f)[:, 5:-5]).max() > 1e-2


@pytest.mark.slow
def test_barometric_steady_state_converges():
    # Time-marched steady state vs Eq. "eq:iso_n" with the walls' ghost rule:
    # the density error falls at (at least) first order in dx, T at second.
    g = 0.5
    errs, terrs = [], []
    for nx in (16, 32):
        s = Solver(Config(Qx=4, nx=nx, advection="upwind2", ax=-g, Kn=1.0))
        n = np.exp(-g * s.xc)
        n /= (n * s.dx).sum()
        s.f = n[None, :, None, None, None] * s.vs.wx[None, None, None, None, :]
        for _ in range(100):
            fo = s.f.copy()
            s.step(200)
            if s.residual(fo, s.f) < 1e-9:
                break
        nn, u, T, _ = s.moments()
        N = s.total_number()
        ana = g * N * np.exp(-g * s.xc) / (1 - np.exp(-g))
        errs.append(np.abs(nn[0] - ana).max() / ana.max())
        terrs.append(np.abs(T - 1).max())
    assert errs[0] < 4e-3 and errs[0] / errs[1] > 1.8
    assert terrs[0] / terrs[1] > 3.0


@pytest.mark.parametrize("adv", ["upwind2", "weno5"])
def test_particle_number_is_conserved(adv):
    # N = int n dx dy (Eq. "eq:Ndef") is conserved step by step: zero net wall
    # flux, zero mass moment of K, BGK conserves n.
    s = Solver(Config(Qx=3, Qy=4, nx=10, ny=6, Ly=0.6, stretch_A=0.7, advection=adv,
                      T_left=0.7, T_right=1.6, ax=-0.4, ay=0.3, Kn=0.2))
    s.init_equilibrium(1.0, 0.1, 0.0, 1.1)
    rng = np.random.default_rng(5)
    s.f *= 1 + 0.2 * rng.uniform(-1, 1, s.f.shape)
    N0 = s.total_number()
    s.step(25)
    assert s.total_number() == pytest.approx(N0, rel=1e-13)


def test_wall_emitted_flux_is_wall_maxwellian():
    # Eqs. "eq:weno_flux_eq", "eq:weno_populate": with the three ghosts equal,
    # sigma_1 = 0 and the emitted flux at the wall face is p_k n_w g_k^w exactly;
    # the total flux through the wall face vanishes.
    s = Solver(Config(Qx=4, Qy=2, nx=8, advection="weno5", T_left=0.6, T_right=1.4))
    s.init_equilibrium(1.0, 0.2, 0.0, 1.0)
    rng = np.random.default_rng(7)
    s.f *= 1 + 0.1 * rng.uniform(-1, 1, s.f.shape)
    fe, nl, nr = s._extend_x(s.f)
    F = face_fluxes(fe, s.vx, 1, "weno5")
    Q = s.vs.Qx
    emit_l = F[:, 0, ..., :Q]
    np.testing.assert_allclose(emit_l, (nl[:, None, None, None] * s.vs.px[:Q] * s.gw[0][None, ..., :Q]),
                               rtol=1e-14)
    assert abs(F[:, 0].sum()) < 1e-14 * np.abs(F[:, 0]).sum()
    assert abs(F[:, -1].sum()) < 1e-14 * np.abs(F[:, -1]).sum()


def test_stretched_grid():
    # Eqs. "eq:x_eta", "eq:etai": edges tile [0, L], symmetric, refined at the walls.
    edges, xc, dx = grid_x(512, 1.0, 0.9)
    assert edges[0] == pytest.approx(0.0, abs=1e-15) and edges[-1] == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(dx, dx[::-1], rtol=1e-12)
    assert dx.min() == pytest.approx(dx[0]) and dx.max() == pytest.approx(dx[255])
    # first cell: x(eta) = L/2 + L/(2A) tanh(eta) between -artanh A and -artanh A + d_eta
    de = 2 * math.atanh(0.9) / 512
    assert dx[0] == pytest.approx((math.tanh(-math.atanh(0.9) + de) + 0.9) / 1.8, rel=1e-12)


def test_ballistic_reference_profiles():
    # The free-streaming solution of Sec. V (Eq. "eq:f_bal") that the paper's
    # convergence test uses as reference, pinned by: zero mass flux everywhere
    # (its moments against Eq. "eq:bal_npnm"); equal wall temperatures giving
    # the isothermal barometric profile n = N (g/T) e^{-g x/T} / (1 - e^{-g L/T})
    # at T = T_w (Eq. "eq:iso_n"); g -> 0 giving the free-molecular state
    # (uniform n, T = sqrt(T_L T_R)).
    from oracle.ballistic import ballistic_profiles, epsilon
    x = np.linspace(0.0, 1.0, 41)
    n, u, T = ballistic_profiles(x, 1.0, 0.1, 1.4, 0.6)
    np.testing.assert_allclose(u, 0.0, atol=1e-14)
    from scipy.integrate import trapezoid
    xf = np.linspace(0.0, 1.0, 4001)
    assert trapezoid(ballistic_profiles(xf, 1.0, 0.1, 1.4, 0.6)[0], xf) == pytest.approx(1.0, rel=1e-6)
    g, Tw = 0.7, 1.3
    n, u, T = ballistic_profiles(x, 1.0, g, Tw, Tw, N=2.0)
    np.testing.assert_allclose(n, 2.0 * (g / Tw) * np.exp(-g * x / Tw) / (1 - np.exp(-g / Tw)), rtol=1e-12)
    np.testing.assert_allclose(T, Tw, rtol=1e-12)
    # (the turning momentum c(x) = sqrt(g (L - 2x')) makes the limit O(sqrt g))
    n, u, T = ballistic_profiles(x, 1.0, 1e-16, 0.8, 1.7)
    np.testing.assert_allclose(n, 1.0, rtol=1e-7)
    np.testing.assert_allclose(T, math.sqrt(0.8 * 1.7), rtol=1e-7)
    assert epsilon([1.0, 1.2], [1.0, 1.0]) == pytest.approx(1.0)     # 0.2 / max(0.2, 0.1)
    assert epsilon([1.0, 1.01], [1.0, 1.0]) == pytest.approx(0.1)    # 0.01 / 0.1 (spread floor)


def test_weno_face_is_homogeneous_down_to_tiny_populations():
    # Eq. "eq:weno5_omega": the weights depend on ratios of sigmas only, so the
    # face value scales with the stencil.  Scaling by a power of two is exact
    # in FP64, also at 2^-700 (populations of the Q = 200 set reach 5e-221,
    # where sigma^2 of the raw values would underflow); a stencil spanning 300
    # orders of magnitude still gives finite weights (delta/sigma^2 beyond the
    # FP64 range) that pick the flattest sub-stencil.
    rng = np.random.default_rng(5)
    cells = rng.uniform(0.5, 2.0, size=(5, 64))
    F = weno5_face(*cells)
    for k in (-700, -300, 200):
        np.testing.assert_array_equal(weno5_face(*(np.ldexp(cells, k))), np.ldexp(F, k))
    st = np.array([1.0, 0.5, 1e-100, 3e-100, 2e-100])
    got = weno5_face(*st)
    # sigma_1, sigma_2 = O(1), sigma_3 = O(1e-200): delta_3/sigma_3^2 ~ 1e400,
    # so the third candidate takes the whole weight
    F3 = st[2] / 3.0 + 5.0 * st[3] / 6.0 - st[4] / 6.0
    assert np.isfinite(got) and got == pytest.approx(F3, rel=1e-12)


# --- the Navier-Stokes regime (Sec. V, oracle/hydrodynamic.py) -------------------
@pytest.mark.parametrize("g,TL,TR", [(0.5, 0.8, 1.2), (1.0, 1.4, 0.6), (0.1, 1.0, 1.0), (0.0, 0.8, 1.2)])
def test_navier_stokes_profiles_closed_forms(g, TL, TR):
    # Eqs. "eq:NS_temp", "eq:NS_n": N particles, the wall temperatures at the
    # walls, T^2 linear (constant heat flux with kappa ~ T), hydrostatic
    # balance d(nT)/dx = -g n, and the barometric Eq. "eq:iso_n" at equal
    # wall temperatures; g -> 0 is continuous.
    from scipy.integrate import quad
    from oracle.hydrodynamic import ns_profiles
    N = quad(lambda s: ns_profiles(s, 1.0, g, TL, TR, N=0.7)[0], 0.0, 1.0, epsabs=1e-14, epsrel=1e-13)[0]
    assert N == pytest.approx(0.7, rel=1e-12)
    _, Tw = ns_profiles(np.array([0.0, 1.0]), 1.0, g, TL, TR)
    np.testing.assert_allclose(Tw, [TL, TR], rtol=1e-14)
    x = np.linspace(0.05, 0.95, 19)
    n, T = ns_profiles(x, 1.0, g, TL, TR)
    np.testing.assert_allclose(np.diff(T ** 2) / np.diff(x), TR ** 2 - TL ** 2, rtol=1e-9, atol=1e-12)
    h = 1e-5
    (n1, T1), (n0, T0) = ns_profiles(x + h, 1.0, g, TL, TR), ns_profiles(x - h, 1.0, g, TL, TR)
    np.testing.assert_allclose((n1 * T1 - n0 * T0) / (2 * h), -g * n, rtol=1e-7, atol=1e-9)
    if TL == TR:
        Tw = TL
        iso = g * np.exp(-g * (x - 0.5) / Tw) / (2 * Tw * math.sinh(g / (2 * Tw)))
        np.testing.assert_allclose(n, iso, rtol=1e-13)
    if g == 0.0:
        np.testing.assert_allclose(n, ns_profiles(x, 1.0, 1e-7, TL, TR)[0], rtol=1e-6)


@pytest.mark.slow
def test_oracle_approaches_the_navier_stokes_profiles():
    # HHLB(3;4), 24 cells, WENO5, g = 0.5, walls at 0.8 and 1.2, Kn = 0.02:
    # the stationary n and T lie within O(Kn) of Eqs. "eq:NS_n", "eq:NS_temp"
    # (measured eps = 2.8 % and 5.4 % here; 1.5 % and 2.7 % at Kn = 0.01,
    # 0.7 % and 1.3 % at Kn = 0.005: first order in Kn, the temperature jump and
    # Knudsen layers at the walls), and the heat flux approaches Eq. "eq:NS_q".
    from oracle.ballistic import epsilon
    from oracle.hydrodynamic import ns_heat_flux, ns_profiles
    g, TL, TR, Kn = 0.5, 0.8, 1.2, 0.02
    s = Solver(Config(Qx=4, nx=24, advection="weno5", T_left=TL, T_right=TR, ax=-g, Kn=Kn, cfl=0.5))
    s.init_equilibrium(1.0, 0.0, 0.0, 1.0)
    s.step(6000)
    n, u, T, q = (a.ravel() for a in s.moments())
    _, xc, dx = grid_x(24, 1.0, 0.0)
    rn, rT = ns_profiles(xc, 1.0, g, TL, TR, N=float((n * dx).sum()))
    assert epsilon(n, rn) < 0.04
    assert epsilon(T, rT) < 0.07
    assert 0.03 < epsilon(T, rT)                       # not converged past the O(Kn) error
    q_ns = ns_heat_flux(1.0, Kn, TL, TR)
    assert np.abs(q[6:-6] - q_ns).max() < 0.25 * abs(q_ns)
