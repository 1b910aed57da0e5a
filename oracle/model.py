"""Force matrices, projected equilibria and the direct-product velocity set.

Test infrastructure only (see the package docstring).  m = 1 and p_0 = 1
throughout, so momenta and velocities coincide (p_k = z_k).

* ``hh_force_matrix(Q)``: K^h_{kk'} of Eq. "eq:hh_Kk_hh" (Sec. IV.B.4), the
  2Q x 2Q discrete momentum derivative for the half-range Hermite quadrature,
  evaluated term by term in Decimal and rounded once to FP64.  Index order:
  k = 0..Q-1 are +z_k (sigma = +1), k = Q..2Q-1 are -z_{k-Q} (sigma = -1).
* ``h_force_matrix(Q)``: K^H_{kk'} of Eq. "eq:H_Kk" (Sec. IV.A.4).
* ``hh_equilibrium(Q, N, u, T)``: g_k of Eq. "eq:hh_gk" (Sec. IV.B.3), with
  zeta = u / sqrt(2T), P_s^{+-} = exp(-+zeta^2) d^s/dzeta^s exp(+-zeta^2) and
  P_s^* = sum_{j<s} C(s,j) P_j^+ P_{s-j-1}^-, Phi_s^N of Eq. "eq:Phi_def".
* ``h_equilibrium(Q, N, u, T)``: g_k of Eq. "eq:H_gk" with
  G_l = sum_s l!/(2^s s! (l-2s)!) (T-1)^s u^{l-2s}.  The printed exponent of
  (T - 1) is "2"; it is read as s (the only reading with G_l(u=0, T=1) =
  delta_{l0}, i.e. g_k = w_k at rest and unit temperature).
* ``hl_force_matrix(Q)``: K^L_{kk'} of Eq. "eq:hh_Kk_L", the half-range
  Gauss-Laguerre counterpart (same index order).
* ``hl_equilibrium(Q, N, u, T)``: the half-range projection of the
  Maxwellian on the Laguerre basis, g_k = w_k sum_{l<=N} L_l(z_k) G_l^{+-} with
  G_l^{+-} = int_0^inf g(+-p) L_l(p) dp written out from the half-range moments
  M_s^{+-} = int_0^inf p^s g(+-p) dp.
* ``VelocitySet``: the mixed quadrature of App. A: half-range along p_x
  (Hermite, Laguerre, or full-range Gauss-Hermite), full-range along p_y and
  p_z (an axis with Q = 0 is absent).
"""
from __future__ import annotations

import math
from decimal import Decimal
from functools import lru_cache

import numpy as np
from scipy.special import erf as _erf

from .quadrature import (PREC, _ctx, dec_inv_sqrt_2pi, dec_pi, gauss_hermite, gauss_laguerre_half,
                         half_hermite_coeffs, half_range_hermite, poly_eval, to_f64)

# Orders above this come from oracle/highorder.py (the 80-digit monomial route
# of quadrature.half_range_hermite loses about 2.5 digits per order).
HH_DECIMAL_MAX_Q = 32


def half_range_nodes(Q: int) -> dict:
    """Nodes z and weights w (Decimal, ascending) of the half-range Hermite
    quadrature of order Q: the 80-digit route up to Q = 32, the stored or
    mpmath tables of ``highorder.half_range_data`` beyond."""
    if Q <= HH_DECIMAL_MAX_Q:
        return half_range_hermite(Q)
    from . import highorder
    return highorder.half_range_data(Q)


# ----------------------------------------------------------------------------
# half-range Hermite: K^h  (Eq. "eq:hh_Kk_hh")
# ----------------------------------------------------------------------------
@lru_cache(maxsize=None)
def hh_force_matrix(Q: int) -> np.ndarray:
    if Q > HH_DECIMAL_MAX_Q:
        from . import highorder
        return highorder.hh_force_matrix_rec(Q)
    d = half_range_hermite(Q)
    C, z, w = d["C"], d["z"], d["w"]
    with _ctx():
        s2pi = dec_inv_sqrt_2pi()
        # h_l(z_k) for l <= Q - 1 (h_Q(z_k) = 0 by construction)
        H = [[poly_eval(C[l][: l + 1], zk) for l in range(Q)] for zk in z]
        h0 = [C[l][0] for l in range(Q)]          # h_{l,0} = h_l(0)
        lead = [C[l][l] for l in range(Q)]        # h_{l,l}
        # Phi_0^Q(z_k) = sum_{s=0}^{Q-1} h_{s,0} h_s(z_k)   (Eq. "eq:Phi_def_hh")
        Phi0 = [sum(h0[s] * H[k][s] for s in range(Q)) for k in range(Q)]
        # Same-half bracket: B[k][k'] = sum_{l=0}^{Q-2} h_l(z_k') [
        #   h_{l,0}/sqrt(2pi) sum_{s=l+1}^{Q-1} h_{s,0} h_s(z_k)
        #   - (h_{l,l}/h_{l+1,l+1}) h_{l+1}(z_k) ]
        def same_half(k: int, kp: int) -> Decimal:
            acc = Decimal(0)
            for l in range(Q - 1):
                inner = sum(h0[s] * H[k][s] for s in range(l + 1, Q))
                acc += H[kp][l] * (h0[l] * s2pi * inner - lead[l] / lead[l + 1] * H[k][l + 1])
            return acc

        K = np.zeros((2 * Q, 2 * Q))
        for k in range(2 * Q):
            sk = 1 if k < Q else -1
            kk = k % Q
            for kp in range(2 * Q):
                skp = 1 if kp < Q else -1
                kkp = kp % Q
                val = Decimal(0)
                if sk == skp:
                    val += same_half(kk, kkp)
                val -= s2pi / 2 * Phi0[kk] * Phi0[kkp]
                K[k, kp] = float(w[kk] * sk * val)
    return K


# ----------------------------------------------------------------------------
# half-range Gauss-Laguerre: K^L  (Eq. "eq:hh_Kk_L")
# ----------------------------------------------------------------------------
@lru_cache(maxsize=None)
def hl_force_matrix(Q: int) -> np.ndarray:
    d = gauss_laguerre_half(Q)
    L, z, w = d["L"], d["z"], d["w"]
    with _ctx():
        Lv = [[poly_eval(L[l], zk) for l in range(Q)] for zk in z]       # L_l(z_k), l <= Q-1
        Phi0 = [sum(Lv[k]) for k in range(Q)]                            # sum_{s<Q} L_s(z_k)
        # same-half bracket: B[k][k'] = sum_{l=0}^{Q-2} L_l(z_k') sum_{s=l+1}^{Q-1} L_s(z_k)
        K = np.zeros((2 * Q, 2 * Q))
        for k in range(2 * Q):
            kk, sk = k % Q, (1 if k < Q else -1)
            for kp in range(2 * Q):
                kkp, skp = kp % Q, (1 if kp < Q else -1)
                acc = Decimal(0)
                if sk == skp:
                    for l in range(Q - 1):
                        acc += Lv[kkp][l] * sum(Lv[kk][s] for s in range(l + 1, Q))
                acc -= Phi0[kk] * Phi0[kkp] / 2
                K[k, kp] = float(w[kk] * sk * acc)
    return K


def _hl_moments_dec(N: int, u: float, T: float, sgn: int):
    """M_s = int_0^inf p^s g(sgn p) dp, s <= N, for g = exp(-(p-u)^2/(2T))/sqrt(2 pi T)
    (Decimal): M_0 = (1 + erf(sgn u/sqrt(2T)))/2, M_1 = sgn u M_0 + T g(0),
    M_{s+1} = sgn u M_s + s T M_{s-1} (integration by parts of (p - sgn u) g)."""
    with _ctx():
        uD, TD = Decimal(float(u)) * sgn, Decimal(float(T))
        g0 = (-(uD * uD) / (2 * TD)).exp() / (2 * dec_pi() * TD).sqrt()
        M = [(1 + _dec_erf(uD / (2 * TD).sqrt())) / 2]
        if N >= 1:
            M.append(uD * M[0] + TD * g0)
        for s_ in range(1, N):
            M.append(uD * M[s_] + s_ * TD * M[s_ - 1])
    return M


def hl_equilibrium(Q: int, N: int, u, T) -> np.ndarray:
    """Half-range Gauss-Laguerre projection of the Maxwellian, shape u.shape + (2Q,)
    (entries 0..Q-1 at +z_k, Q..2Q-1 at -z_k), n = 1; each node in Decimal."""
    if not 0 <= N < Q:
        raise ValueError("0 <= N < Q")
    d = gauss_laguerre_half(Q)
    L, z, w = d["L"], d["z"], d["w"]
    u = np.asarray(u, dtype=np.float64)
    T = np.broadcast_to(np.asarray(T, dtype=np.float64), u.shape)
    out = np.zeros(u.shape + (2 * Q,))
    with _ctx():
        Lz = [[poly_eval(L[l], zk) for l in range(N + 1)] for zk in z]
        for ix in np.ndindex(u.shape):
            for half, sgn in ((0, 1), (1, -1)):
                M = _hl_moments_dec(N, float(u[ix]), float(T[ix]), sgn)
                G = [sum(L[l][s_] * M[s_] for s_ in range(l + 1)) for l in range(N + 1)]
                for k in range(Q):
                    out[ix + (half * Q + k,)] = float(w[k] * sum(Lz[k][l] * G[l] for l in range(N + 1)))
    return out


# ----------------------------------------------------------------------------
# full-range Hermite: K^H  (Eq. "eq:H_Kk")
# ----------------------------------------------------------------------------
@lru_cache(maxsize=None)
def h_force_matrix(Q: int) -> np.ndarray:
    d = gauss_hermite(Q)
    z, w, He = d["z"], d["w"], d["He"]
    with _ctx():
        Hv = [[poly_eval([Decimal(c) for c in He[l]], zk) for l in range(Q)] for zk in z]
        K = np.zeros((Q, Q))
        for k in range(Q):
            for kp in range(Q):
                acc = Decimal(0)
                for l in range(Q - 1):
                    acc += Hv[k][l + 1] * Hv[kp][l] / math.factorial(l)
                K[k, kp] = float(-w[k] * acc)
    return K


# ----------------------------------------------------------------------------
# equilibria
# ----------------------------------------------------------------------------
def _poly_mul(a, b):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


@lru_cache(maxsize=None)
def p_polys(N: int):
    """Integer coefficients (ascending) of P_s^+, P_s^-, P_s^* for s <= N.

    d/dzeta [p(zeta) e^{+-zeta^2}] = (p' +- 2 zeta p) e^{+-zeta^2}, applied s
    times to p = 1 gives P_s^{+-}; P_s^* is the binomial convolution of the
    definition under Eq. "eq:hh_gk".
    """
    Pp, Pm = [[1]], [[1]]
    for s in range(N):
        for P, sign in ((Pp, 1), (Pm, -1)):
            cur = P[-1]
            nxt = [0] * (len(cur) + 1)
            for i, c in enumerate(cur):          # derivative
                if i:
                    nxt[i - 1] += i * c
            for i, c in enumerate(cur):          # +- 2 zeta p
                nxt[i + 1] += sign * 2 * c
            P.append(nxt)
    Ps = [[0]]
    for s in range(1, N + 1):
        acc = [0]
        for j in range(s):
            prod = _poly_mul(Pp[j], Pm[s - j - 1])
            prod = [math.comb(s, j) * c for c in prod]
            if len(prod) > len(acc):
                acc = acc + [0] * (len(prod) - len(acc))
            for i, c in enumerate(prod):
                acc[i] += c
        Ps.append(acc)
    return tuple(map(tuple, Pp)), tuple(map(tuple, Pm)), tuple(map(tuple, Ps))


def _polyval_asc(coeffs, x):
    acc = np.zeros_like(x, dtype=np.float64)
    for c in reversed(coeffs):
        acc = acc * x + float(c)
    return acc


@lru_cache(maxsize=None)
def hh_phi_table_dec(Q: int, N: int):
    """Phi_s^N(z_k) = sum_{l=s}^N h_{l,s} h_l(z_k) (Eq. "eq:Phi_def"), Decimal, [k][s].
    Only the coefficients of h_0 .. h_N enter (the rows of the Cholesky inverse
    do not depend on how many are formed)."""
    C = half_hermite_coeffs(N + 1)
    z = half_range_nodes(Q)["z"]
    with _ctx():
        out = []
        for zk in z:
            hl = [poly_eval(C[l][: l + 1], zk) for l in range(N + 1)]
            out.append(tuple(sum(C[l][s] * hl[l] for l in range(s, N + 1)) for s in range(N + 1)))
    return tuple(out)


def hh_phi_table(Q: int, N: int) -> np.ndarray:
    return np.array([[float(x) for x in row] for row in hh_phi_table_dec(Q, N)])


def _dec_erf(x: Decimal) -> Decimal:
    """erf by its Maclaurin series, 2/sqrt(pi) sum_n (-1)^n x^{2n+1}/(n!(2n+1))."""
    with _ctx() as c:
        c.prec = PREC + 30      # the alternating series cancels for |x| ~ O(few)
        x2 = x * x
        term, total, n = x, x, 0
        eps = Decimal(10) ** (-(PREC + 5))
        while abs(term) > eps * abs(total) or n < 2:
            n += 1
            term *= -x2 / n
            total += term / (2 * n + 1)
        return +(total * 2 / dec_pi().sqrt())


def _hh_equilibrium_node(Q: int, N: int, u: float, T: float):
    """g_k of Eq. "eq:hh_gk" for one (u, T), evaluated term by term in Decimal.

    The expansion sums (T/2)^{s/2} Phi_s^N(z_k) [...] over s with terms far
    larger than their sum (|Phi_s^N| reaches 1e11 at Q = 16), so FP64 would
    lose up to nine digits; 80-digit arithmetic returns g_k correctly rounded.
    """
    w = half_range_nodes(Q)["w"]
    Phi = hh_phi_table_dec(Q, N)
    Pp, _, Ps = p_polys(N)
    with _ctx():
        uD, TD = Decimal(float(u)), Decimal(float(T))
        zeta = uD / (2 * TD).sqrt()
        e = (-zeta * zeta).exp() * 2 / dec_pi().sqrt()
        root = (TD / 2).sqrt()
        out = []
        for sgn in (1, -1):
            zs = sgn * zeta
            one_erf = 1 + _dec_erf(zs)
            A = []
            scale = Decimal(1)
            for s in range(N + 1):
                pp = poly_eval([Decimal(c) for c in Pp[s]], zs)
                ps = poly_eval([Decimal(c) for c in Ps[s]], zs)
                A.append(scale * (one_erf * pp + e * ps))
                scale *= root
            for k in range(Q):
                out.append(float(w[k] / 2 * sum(A[s] * Phi[k][s] for s in range(N + 1))))
    return out


def hh_equilibrium(Q: int, N: int, u, T, tol: float = 1e-12) -> np.ndarray:
    """Half-range equilibrium g_k(u, T), Eq. "eq:hh_gk"; shape u.shape + (2Q,).

    Entries 0..Q-1 belong to +z_k, entries Q..2Q-1 to -z_k.  The formula is
    first evaluated in FP64 together with the standard rounding-error bound
    of a sum, (N + 3) eps sum_s |term_s|; every node whose bound exceeds
    ``tol`` relative to |g_k| is evaluated again in 80-digit Decimal
    (``_hh_equilibrium_node``).  At Q <= 8 FP64 suffices; at Q = 16 the
    terms are up to 1e9 times their sum and Decimal takes over.
    """
    if not 0 <= N < Q:
        raise ValueError("0 <= N < Q")
    u = np.asarray(u, dtype=np.float64)
    T = np.broadcast_to(np.asarray(T, dtype=np.float64), u.shape)
    w = to_f64(half_range_nodes(Q)["w"])
    Phi = hh_phi_table(Q, N)                         # (Q, N+1)
    Pp, _, Ps = p_polys(N)
    zeta = u / np.sqrt(2.0 * T)
    e = np.exp(-zeta * zeta) * (2.0 / math.sqrt(math.pi))
    out = np.zeros(u.shape + (2 * Q,))
    bound = np.zeros(u.shape + (2 * Q,))
    for sgn, sl in ((1.0, slice(0, Q)), (-1.0, slice(Q, 2 * Q))):
        zs = sgn * zeta
        one_erf = 1.0 + _erf(zs)
        acc = np.zeros(u.shape + (Q,))
        mag = np.zeros(u.shape + (Q,))
        for s in range(N + 1):
            A = (T / 2.0) ** (s / 2.0) * (one_erf * _polyval_asc(Pp[s], zs)
                                         + e * _polyval_asc(Ps[s], zs))
            term = A[..., None] * Phi[:, s]
            acc += term
            mag += np.abs(term)
        out[..., sl] = 0.5 * w * acc
        bound[..., sl] = 0.5 * w * mag * (N + 3) * np.finfo(np.float64).eps
    bad = np.any(bound > tol * np.abs(out), axis=-1)
    if np.any(bad):
        idx = np.argwhere(bad)
        for ix in map(tuple, idx):
            out[ix] = _hh_equilibrium_node(Q, N, float(u[ix]), float(T[ix]))
    return out


def h_equilibrium(Q: int, N: int, u, T) -> np.ndarray:
    """Full-range equilibrium g_k(u, T), Eq. "eq:H_gk"; shape u.shape + (Q,)."""
    if not 0 <= N < Q:
        raise ValueError("0 <= N < Q")
    u = np.asarray(u, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    d = gauss_hermite(Q)
    z, w, He = to_f64(d["z"]), to_f64(d["w"]), d["He"]
    out = np.zeros(u.shape + (Q,))
    for l in range(N + 1):
        G = np.zeros_like(u)
        for s in range(l // 2 + 1):
            coef = math.factorial(l) / (2 ** s * math.factorial(s) * math.factorial(l - 2 * s))
            G = G + coef * (T - 1.0) ** s * u ** (l - 2 * s)
        Hel = np.array([sum(c * zk ** i for i, c in enumerate(He[l])) for zk in z])
        out += G[..., None] * (w * Hel / math.factorial(l))
    return out


# ----------------------------------------------------------------------------
# velocity set (App. A)
# ----------------------------------------------------------------------------
class VelocitySet:
    """Direct product p_{ijk} = (p_x,i, p_y,j, p_z,k); f index order (kz, jy, ix).

    Qx >= 1 half-range points per half (2 Qx values of p_x), or with
    x_full=True an even full-range order Qx (Qx values of p_x); Qy, Qz in
    {0, 2, 4, ...} (0 = axis absent, which contributes a single p = 0 with
    weight 1 and no degree of freedom).  N* = equilibrium orders.  QH is the
    number of p_x > 0 values; they come first.
    """

    def __init__(self, Qx: int, Qy: int = 0, Qz: int = 0, Nx=None, Ny=None, Nz=None, x_full: bool = False,
                 x_laguerre: bool = False):
        if Qx < 1:
            raise ValueError("Qx >= 1")
        for q in (Qy, Qz) + ((Qx,) if x_full else ()):
            if q < 0 or q % 2:
                raise ValueError("full-range orders must be 0 or even (Sec. IV.A.1)")
        self.Qx, self.Qy, self.Qz = Qx, Qy, Qz
        self.x_full = bool(x_full)
        self.x_laguerre = bool(x_laguerre) and not x_full
        self.Nx = Qx - 1 if Nx is None or Nx < 0 else Nx
        self.Ny = (Qy - 1 if Ny is None or Ny < 0 else Ny) if Qy else 0
        self.Nz = (Qz - 1 if Nz is None or Nz < 0 else Nz) if Qz else 0
        if x_full:
            # the HLB(N; Q) models of Sec. V along p_x: full-range Gauss-Hermite
            # of order Qx, K^H (Eq. "eq:H_Kk", no jump term) and Eq. "eq:H_gk";
            # nodes ordered +z_1 < ... < +z_{Q/2}, then -z_1, ..., -z_{Q/2}, the
            # layout of the half-range set (px > 0 first)
            d = gauss_hermite(Qx)
            z = to_f64(d["z"])                      # ascending
            h = Qx // 2
            self._xperm = np.concatenate([np.arange(h, Qx), np.arange(h - 1, -1, -1)])
            self.px = z[self._xperm]
            self.wx = to_f64(d["w"])[self._xperm]
            self.Kx = h_force_matrix(Qx)[np.ix_(self._xperm, self._xperm)]
            self.QH = h
        elif x_laguerre:
            # the half-range Gauss-Laguerre family (Sec. IV.B, Eq. "eq:hh_Kk_L")
            d = gauss_laguerre_half(Qx)
            zx, wx = to_f64(d["z"]), to_f64(d["w"])
            self.px = np.concatenate([zx, -zx])
            self.wx = np.concatenate([wx, wx])
            self.Kx = hl_force_matrix(Qx)
            self.QH = Qx
        else:
            zx = to_f64(half_range_nodes(Qx)["z"])
            wx = to_f64(half_range_nodes(Qx)["w"])
            self.px = np.concatenate([zx, -zx])
            self.wx = np.concatenate([wx, wx])
            self.Kx = hh_force_matrix(Qx)
            self.QH = Qx                            # velocities with p_x > 0
        if Qy:
            gy = gauss_hermite(Qy)
            self.py, self.wy = to_f64(gy["z"]), to_f64(gy["w"])
            self.Ky = h_force_matrix(Qy)
        else:
            self.py, self.wy, self.Ky = np.zeros(1), np.ones(1), np.zeros((1, 1))
        if Qz:
            gz = gauss_hermite(Qz)
            self.pz, self.wz = to_f64(gz["z"]), to_f64(gz["w"])
            self.Kz = h_force_matrix(Qz)
        else:
            self.pz, self.wz, self.Kz = np.zeros(1), np.ones(1), np.zeros((1, 1))
        self.D = 1 + (Qy > 0) + (Qz > 0)
        self.shape = (len(self.pz), len(self.py), len(self.px))
        self.V = int(np.prod(self.shape))

    def g_x(self, u, T):
        if self.x_full:
            return h_equilibrium(self.Qx, self.Nx, u, T)[..., self._xperm]
        if self.x_laguerre:
            return hl_equilibrium(self.Qx, self.Nx, u, T)
        return hh_equilibrium(self.Qx, self.Nx, u, T)

    def g_y(self, u, T):
        if not self.Qy:
            return np.ones(np.shape(u) + (1,))
        return h_equilibrium(self.Qy, self.Ny, u, T)

    def g_z(self, u, T):
        if not self.Qz:
            return np.ones(np.shape(u) + (1,))
        return h_equilibrium(self.Qz, self.Nz, u, T)

    def equilibrium(self, n, ux, uy, uz, T):
        """feq_{ijk} = n g_x,i g_y,j g_z,k (App. A); shape n.shape + (Vz, Vy, Vx)."""
        gx = self.g_x(ux, T)
        gy = self.g_y(uy, T)
        gz = self.g_z(uz, T)
        n = np.asarray(n, dtype=np.float64)
        return (n[..., None, None, None] * gz[..., :, None, None]
                * gy[..., None, :, None] * gx[..., None, None, :])
