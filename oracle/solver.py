"""The FP64 time step of the oracle: advection, walls, force, BGK, RK-3.

Test infrastructure only (see the package docstring).  One instance is a
channel with diffuse-reflecting walls at x = 0 and x = Lx (the paper's x_+ =
-L/2 and x_- = +L/2, shifted by L/2) and, for ny > 1, periodic in y.

State layout: f[y, x, kz, jy, ix] (ix fastest), FP64.

Steps of one evaluation of L[f] (Eq. "eq:L_def", multi-D form Eq.
"eq:boltz_multi_k"), in the paper's order:
  1. walls (Sec. IV.C.3): quadratic extrapolation of the incident
     populations into the ghost cells; the incident fluxes at the wall
     interface; the emitted density n_w from zero net mass flux (Eq.
     "eq:nplus_def", read with the v_k of the continuous form in the
     denominator); ghosts of the emitted populations = n_w g_k^w (Eq.
     "eq:weno_populate");
  2. fluxes F_{i+1/2} by WENO-5 without epsilon (Sec. IV.C.2, Tab. "weno")
     or 2nd-order upwind, and their divergence over the cell width
     x(eta_{i+1/2}) - x(eta_{i-1/2}) (Eq. "eq:x_eta");
  3. moments n, u, T (Eq. "eq:fmoms"), tau = Kn/n (Eq. "eq:tau");
  4. feq = n g_x g_y g_z (App. A) with the projected equilibria;
  5. force term -sum_a a_a (K_a f) along each momentum axis (App. A;
     a = F/m; a = -g x gives the +mg dp f of Eq. "eq:L_def"); a_a is the
     uniform value plus an optional per-node field;
  6. L = -div - force - (f - feq)/tau;  then the RK-3 of Eq. "eq:rk3".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .model import VelocitySet

UPWIND2, WENO5 = "upwind2", "weno5"

# Ideal WENO-5 weights delta_q (Sec. IV.C.2).
_DELTA = (0.1, 0.6, 0.3)


@dataclass
class Config:
    Qx: int
    Qy: int = 0
    Qz: int = 0
    Nx_eq: int = -1
    Ny_eq: int = -1
    Nz_eq: int = -1
    nx: int = 64
    ny: int = 1
    Lx: float = 1.0
    Ly: float = 1.0
    stretch_A: float = 0.0
    advection: str = WENO5
    cfl: float = 0.5
    dt: float = 0.0
    T_left: float = 1.0
    T_right: float = 1.0
    ax: float = 0.0
    ay: float = 0.0
    az: float = 0.0
    Kn: float = math.inf
    # Optional per-node acceleration fields, arrays of shape (ny, nx), added
    # to the uniform (ax, ay, az): e.g. a force from a potential, a = -grad V / m.
    # The paper's tests use a constant force only; its conclusion (Sec.
    # "sec:conc") presents the force-term formalism as general, and the force
    # term of App. A acts node by node, so a(x) enters it pointwise.
    ax_field: object = None
    ay_field: object = None
    az_field: object = None
    # 0: half-range Hermite along p_x (the HHLB models); 1: full-range
    # Gauss-Hermite of order Qx (the HLB models the paper compares with, Sec. V);
    # 2: half-range Gauss-Laguerre (Sec. IV.B, Eq. "eq:hh_Kk_L")
    x_basis: int = 0
    extra: dict = field(default_factory=dict)


def config_from(d: dict) -> Config:
    """Config from a plain workload dict (advection 0 = upwind2, 1 = weno5)."""
    kw = {k: v for k, v in d.items() if k in Config.__dataclass_fields__}
    adv = d.get("advection", WENO5)
    kw["advection"] = {0: UPWIND2, 1: WENO5}.get(adv, adv)
    return Config(**kw)


# ----------------------------------------------------------------------------
# grid (Eqs. "eq:x_eta", "eq:etai")
# ----------------------------------------------------------------------------
def grid_x(nx: int, L: float, A: float):
    """Cell edges, centres and widths on [0, L].

    A = 0: uniform.  0 < A < 1: eta_i = (i - (nx+1)/2) d_eta with
    d_eta = 2 artanh(A)/nx, x(eta) = L/2 + (L/(2A)) tanh(eta); the edges are
    x(eta_i -+ d_eta/2) and the centres x(eta_i).
    """
    if A == 0.0:
        edges = np.linspace(0.0, L, nx + 1)
        centres = 0.5 * (edges[:-1] + edges[1:])
    else:
        d_eta = 2.0 * math.atanh(A) / nx
        i = np.arange(1, nx + 1, dtype=np.float64)
        eta_c = (i - (nx + 1) / 2.0) * d_eta
        eta_e = np.concatenate([eta_c - d_eta / 2.0, eta_c[-1:] + d_eta / 2.0])
        edges = L / 2.0 + L / (2.0 * A) * np.tanh(eta_e)
        centres = L / 2.0 + L / (2.0 * A) * np.tanh(eta_c)
    return edges, centres, np.diff(edges)


# ----------------------------------------------------------------------------
# fluxes
# ----------------------------------------------------------------------------
def weno5_weights(s1, s2, s3):
    """Normalised weights of Eq. "eq:weno5_omega" with the zero limits of Tab. "weno".

    If any sigma_q is exactly zero, the weights are delta_q renormalised over
    the set of zero sigmas (the limits of delta_q/sigma_q^2 as those sigmas
    vanish); otherwise w_q = (delta_q/sigma_q^2) / sum_r (delta_r/sigma_r^2).
    Where a nonzero sigma is so small (below ~1e-154) that these quotients
    overflow FP64, they are formed again in numpy's long double (exponent
    range to 1e4932 on x86 and Arm; only those entries, since long double is
    a software type on Arm).
    """
    s = (np.asarray(s1, float), np.asarray(s2, float), np.asarray(s3, float))
    z = [si == 0.0 for si in s]
    anyz = z[0] | z[1] | z[2]
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        wt = [np.where(anyz, np.where(z[q], _DELTA[q], 0.0), _DELTA[q] / (s[q] * s[q])) for q in range(3)]
        tot = wt[0] + wt[1] + wt[2]
        out = [wt[q] / tot for q in range(3)]
    wide = ~np.isfinite(tot)
    if np.any(wide):
        sw = [np.asarray(np.broadcast_to(si, wide.shape)[wide], dtype=np.longdouble) for si in s]
        zw = [si == 0 for si in sw]
        anyw = zw[0] | zw[1] | zw[2]
        with np.errstate(divide="ignore", invalid="ignore"):
            ww = [np.where(anyw, np.where(zw[q], _DELTA[q], 0.0), np.longdouble(_DELTA[q]) / (sw[q] * sw[q]))
                  for q in range(3)]
        totw = ww[0] + ww[1] + ww[2]
        out = [np.array(np.broadcast_to(o, wide.shape), dtype=np.float64) for o in out]
        for q in range(3):
            out[q][wide] = (ww[q] / totw).astype(np.float64)
    return tuple(out)


def weno5_face(a, b, c, d, e):
    """WENO-5 reconstruction at the face downwind of c for a positive velocity.

    (a, b, c, d, e) = f at cells i-2 .. i+2 for the face i+1/2 (Sec. IV.C.2).
    Returns sum_q w_q F^q / (p/m), i.e. the flux per unit velocity.
    """
    F1 = a / 3.0 - 7.0 * b / 6.0 + 11.0 * c / 6.0
    F2 = -b / 6.0 + 5.0 * c / 6.0 + d / 3.0
    F3 = c / 3.0 + 5.0 * d / 6.0 - e / 6.0
    # The weights of Eq. "eq:weno5_omega" are invariant under f -> c f (each
    # sigma_q scales as c^2), so the sigmas are formed from the stencil times
    # the power of two 2^-k that brings its largest magnitude into [1/2, 1):
    # exact in FP64, and sigma_q^2 stays in range for populations as small as
    # the 5e-221 weights of the Q = 200 quadrature.
    m = np.maximum(np.maximum(np.maximum(np.abs(a), np.abs(b)), np.maximum(np.abs(c), np.abs(d))), np.abs(e))
    k = np.maximum(np.frexp(m)[1], -1020)
    sc = np.ldexp(1.0, -k)
    a, b, c, d, e = a * sc, b * sc, c * sc, d * sc, e * sc
    s1 = 13.0 / 12.0 * (a - 2 * b + c) ** 2 + 0.25 * (a - 4 * b + 3 * c) ** 2
    s2 = 13.0 / 12.0 * (b - 2 * c + d) ** 2 + 0.25 * (b - d) ** 2
    s3 = 13.0 / 12.0 * (c - 2 * d + e) ** 2 + 0.25 * (3 * c - 4 * d + e) ** 2
    w1, w2, w3 = weno5_weights(s1, s2, s3)
    return w1 * F1 + w2 * F2 + w3 * F3


def upwind2_face(b, c):
    """Linear 2nd-order upwind value at the face downwind of c: (3c - b)/2."""
    return 1.5 * c - 0.5 * b


def face_fluxes(fe, v, axis: int, scheme: str):
    """Fluxes at all faces of a ghost-extended array along ``axis``.

    ``fe`` has 3 ghost cells on each side along ``axis`` (n + 6 entries);
    ``v`` holds the velocity of each population, broadcast against ``fe``
    with a length-1 ``axis``; every population's velocity must be non-zero.
    Face j (j = 0..n) lies between cells j-1 and j.  For v > 0 the stencil
    of face j is cells j-3..j+1; for v < 0 it is the mirror image
    (cells j+2..j-2, Sec. IV.C.2 "without loss of generality p_k > 0").
    """
    n = fe.shape[axis] - 6

    def cell(c):               # cells c .. c+n of the extended array, c in [-3, 2]
        return np.take(fe, np.arange(c + 3, c + 3 + n + 1), axis=axis)

    if scheme == WENO5:
        pos = weno5_face(cell(-3), cell(-2), cell(-1), cell(0), cell(1))
        neg = weno5_face(cell(2), cell(1), cell(0), cell(-1), cell(-2))
    else:
        pos = upwind2_face(cell(-2), cell(-1))
        neg = upwind2_face(cell(1), cell(0))
    return v * np.where(v > 0, pos, neg)


# ----------------------------------------------------------------------------
# the solver
# ----------------------------------------------------------------------------
class Solver:
    """One channel instance; ``f`` is advanced in place by ``step``."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        if cfg.nx < 3:
            raise ValueError("nx >= 3 (quadratic wall extrapolation)")
        self.vs = VelocitySet(cfg.Qx, cfg.Qy, cfg.Qz, cfg.Nx_eq, cfg.Ny_eq, cfg.Nz_eq, x_full=cfg.x_basis == 1,
                              x_laguerre=cfg.x_basis == 2)
        vs = self.vs
        self.edges, self.xc, self.dx = grid_x(cfg.nx, cfg.Lx, cfg.stretch_A)
        self.two_d = cfg.ny > 1
        self.dy = cfg.Ly / cfg.ny
        self.vx = vs.px[None, None, None, None, :]
        self.vy = vs.py[None, None, None, :, None]
        if cfg.dt > 0:
            self.dt = cfg.dt
        else:
            rate = np.abs(vs.px).max() / self.dx.min()
            if self.two_d:
                rate += np.abs(vs.py).max() / self.dy
            self.dt = cfg.cfl / rate
        self.set_walls(cfg.T_left, cfg.T_right)
        self.f = np.zeros((cfg.ny, cfg.nx) + vs.shape)
        self.time = 0.0
        self.nsteps = 0

    # -- walls -------------------------------------------------------------
    def set_walls(self, T_left: float, T_right: float):
        """Wall Maxwellians g^w = g_x(0, T_w) g_y(0, T_w) g_z(0, T_w) (Eq. "eq:fwall")."""
        vs = self.vs
        self.gw = []
        self.gw_den = []
        for Tw, emit in ((T_left, vs.px > 0), (T_right, vs.px < 0)):
            g = vs.equilibrium(np.float64(1.0), 0.0, 0.0, 0.0, np.float64(Tw))
            self.gw.append(g)
            # sum over emitted populations of v_x g^w (denominator of n_w)
            self.gw_den.append(float(np.sum((vs.px * g)[..., emit])))

    def _extend_x(self, f):
        """Ghost-extended copy along x with the diffuse-reflection walls.

        Returns (fe, n_left, n_right); n_* has shape (ny,).
        """
        nx = f.shape[1]
        vs = self.vs
        Q = vs.QH
        pos = slice(0, Q)          # p_x = +z_k (Eq. "eq:hh_pk")
        neg = slice(Q, 2 * Q)      # p_x = -z_k
        fe = np.full((f.shape[0], nx + 6) + f.shape[2:], np.nan)
        fe[:, 3:nx + 3] = f
        f0, f1, f2 = f[:, 0], f[:, 1], f[:, 2]
        fe[:, 2, ..., neg] = (3 * f0 - 3 * f1 + f2)[..., neg]          # cell -1 (paper's 0)
        fe[:, 1, ..., neg] = (6 * f0 - 8 * f1 + 3 * f2)[..., neg]      # cell -2 (paper's -1)
        g0, g1, g2 = f[:, nx - 1], f[:, nx - 2], f[:, nx - 3]
        fe[:, nx + 3, ..., pos] = (3 * g0 - 3 * g1 + g2)[..., pos]
        fe[:, nx + 4, ..., pos] = (6 * g0 - 8 * g1 + 3 * g2)[..., pos]
        # incident fluxes at the two wall faces
        scheme = self.cfg.advection
        left = face_fluxes(fe[:, 0:7], self.vx, 1, scheme)[:, 0]      # face 0
        right = face_fluxes(fe[:, nx - 1:nx + 6], self.vx, 1, scheme)[:, -1]   # face nx
        n_left = -np.sum(left[..., neg], axis=(-1, -2, -3)) / self.gw_den[0]
        n_right = -np.sum(right[..., pos], axis=(-1, -2, -3)) / self.gw_den[1]
        for c in range(3):
            fe[:, c, ..., pos] = (n_left[:, None, None, None] * self.gw[0][None])[..., pos]
            fe[:, nx + 3 + c, ..., neg] = (n_right[:, None, None, None] * self.gw[1][None])[..., neg]
        return fe, n_left, n_right

    # -- moments -----------------------------------------------------------
    def moments(self, f=None):
        """n, u (3 components), T, q_x per node (Eq. "eq:fmoms", App. A).

        T = sum |p - u|^2 f / (D n) with D the number of momentum axes;
        q_x = sum (p_x - u_x) |p - u|^2 f / 2.
        """
        f = self.f if f is None else f
        vs = self.vs
        px = vs.px[None, None, :]
        py = vs.py[None, :, None]
        pz = vs.pz[:, None, None]
        n = f.sum(axis=(-1, -2, -3))
        ux = (f * px).sum(axis=(-1, -2, -3)) / n
        uy = (f * py).sum(axis=(-1, -2, -3)) / n
        uz = (f * pz).sum(axis=(-1, -2, -3)) / n
        cx = px - ux[..., None, None, None]
        cy = py - uy[..., None, None, None]
        cz = pz - uz[..., None, None, None]
        c2 = cx * cx + cy * cy + cz * cz
        T = (f * c2).sum(axis=(-1, -2, -3)) / (vs.D * n)
        q = 0.5 * (f * cx * c2).sum(axis=(-1, -2, -3))
        return n, np.stack([ux, uy, uz], axis=-1), T, q

    def total_number(self, f=None):
        """N = int n dx (dy) (Eq. "eq:Ndef")."""
        f = self.f if f is None else f
        n = f.sum(axis=(-1, -2, -3))
        return float((n * self.dx[None, :]).sum() * (self.dy if self.two_d else 1.0))

    # -- right-hand side -----------------------------------------------------
    def acceleration(self, axis: int):
        """a_axis at every node, shape (ny, nx, 1, 1, 1): the uniform value
        plus the per-node field, if any."""
        cfg = self.cfg
        a = np.full((cfg.ny, cfg.nx), (cfg.ax, cfg.ay, cfg.az)[axis], dtype=np.float64)
        fld = (cfg.ax_field, cfg.ay_field, cfg.az_field)[axis]
        if fld is not None:
            a = a + np.asarray(fld, dtype=np.float64).reshape(cfg.ny, cfg.nx)
        return a[:, :, None, None, None]

    def source(self, f):
        """Local part of L[f]: -sum_a a_a (K_a f) - (f - feq)/tau (no advection)."""
        cfg, vs = self.cfg, self.vs
        S = np.zeros_like(f)
        ax, ay, az = (self.acceleration(k) for k in range(3))
        if np.any(ax):
            S -= ax * np.einsum("ij,...j->...i", vs.Kx, f)
        if vs.Qy and np.any(ay):
            S -= ay * np.einsum("ij,...jk->...ik", vs.Ky, f)
        if vs.Qz and np.any(az):
            S -= az * np.einsum("ij,...jkl->...ikl", vs.Kz, f)
        if math.isfinite(cfg.Kn):
            n, u, T, _ = self.moments(f)
            feq = vs.equilibrium(n, u[..., 0], u[..., 1], u[..., 2], T)
            tau = cfg.Kn / n
            S -= (f - feq) / tau[..., None, None, None]
        return S

    def rhs(self, f):
        cfg, vs = self.cfg, self.vs
        fe, n_l, n_r = self._extend_x(f)
        Fx = face_fluxes(fe, self.vx, 1, cfg.advection)             # (ny, nx+1, ...)
        div = (Fx[:, 1:] - Fx[:, :-1]) / self.dx[None, :, None, None, None]
        if self.two_d:
            fy = np.concatenate([f[-3:], f, f[:3]], axis=0)
            Fy = face_fluxes(fy, self.vy, 0, cfg.advection)
            div = div + (Fy[1:] - Fy[:-1]) / self.dy
        L = -div + self.source(f)
        self.last_wall_density = (n_l, n_r)
        return L

    # -- time stepping (Eq. "eq:rk3") ---------------------------------------
    def step(self, nsteps: int = 1):
        dt = self.dt
        for _ in range(nsteps):
            f = self.f
            f1 = f + dt * self.rhs(f)
            f2 = 0.75 * f + 0.25 * f1 + 0.25 * dt * self.rhs(f1)
            self.f = f / 3.0 + 2.0 / 3.0 * f2 + 2.0 / 3.0 * dt * self.rhs(f2)
            self.time += dt
            self.nsteps += 1
        return self.f

    def init_equilibrium(self, n=1.0, ux=0.0, uy=0.0, T=1.0):
        cfg = self.cfg
        shape = (cfg.ny, cfg.nx)
        full = lambda v: np.broadcast_to(np.asarray(v, dtype=np.float64), shape)
        self.f = self.vs.equilibrium(full(n), full(ux), full(uy), np.zeros(shape), full(T)).copy()
        return self.f

    def residual(self, f_old, f_new):
        """max |f^{n+1} - f^n| / (dt max f)."""
        return float(np.abs(f_new - f_old).max() / (self.dt * np.abs(f_new).max()))
