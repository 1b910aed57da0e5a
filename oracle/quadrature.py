"""Quadratures of the oracle, in 80-digit ``decimal`` arithmetic.

Test infrastructure only (see the package docstring).

Half-range Hermite polynomials h_l (App. B, Eq. "eq:hh_omega"): orthonormal on
[0, inf) with weight omega(z) = exp(-z^2/2)/sqrt(2 pi), gamma_l = 1, positive
leading coefficient.  They are built here by the most literal route: the Gram
matrix of the monomials, <z^i, z^j> = mu_{i+j} with the half-range moments
mu_s = int_0^inf omega z^s dz, is Cholesky-factorised, G = L L^T, and the rows
of L^{-1} are the coefficients h_{l,s} of Eq. "eq:phi_expl".

The half-range Gauss quadrature of order Q (Sec. IV.B.1, Eq. "eq:hh_quad")
takes the Q (positive) roots z_k of h_Q, and the weights of Eq. "eq:wk_half":
    w_k = z_k a_Q^2 / ( h_{Q+1}(z_k)^2 [z_k + h_{Q,0}^2 / sqrt(2 pi)] ),
with a_Q = h_{Q+1,Q+1} / h_{Q,Q} (Eq. "eq:a_def").  The full velocity set is
p_k = z_k, p_{k+Q} = -z_k (Eq. "eq:hh_pk", p_0 = 1).

Half-range Gauss-Laguerre (Sec. IV.B, weight exp(-z) on [0, inf)): roots of
L_Q, weights z_k / ((Q+1)^2 L_{Q+1}(z_k)^2) (Eq. "eq:wk_half").

Full-range Gauss-Hermite (Sec. IV.A.1): roots of the probabilists' Hermite
polynomial He_Q (Eq. "eq:H_ortho" normalisation <He_l, He_l'> = l! delta),
weights w_k = Q! / He_{Q+1}(z_k)^2 (Eq. "eq:H_wk"), summing to 1.
"""
from __future__ import annotations

import functools
import math
from decimal import Decimal, localcontext

import numpy as np

PREC = 80  # decimal digits used for every table


def _ctx():
    return localcontext(prec=PREC)


@functools.lru_cache(maxsize=None)
def dec_pi() -> Decimal:
    """pi to PREC digits by Machin's formula pi = 16 atan(1/5) - 4 atan(1/239)."""
    with localcontext(prec=PREC + 10):

        def atan_inv(n: int) -> Decimal:
            x = Decimal(1) / n
            x2 = x * x
            term, total, k = x, x, 1
            eps = Decimal(10) ** (-(PREC + 8))
            while abs(term) > eps:
                term *= -x2
                total += term / (2 * k + 1)
                k += 1
            return total

        return +(16 * atan_inv(5) - 4 * atan_inv(239))


@functools.lru_cache(maxsize=None)
def dec_inv_sqrt_2pi() -> Decimal:
    with _ctx():
        return Decimal(1) / (2 * dec_pi()).sqrt()


def half_moment(s: int) -> Decimal:
    """mu_s = int_0^inf z^s exp(-z^2/2)/sqrt(2 pi) dz.

    Even s: (s-1)!!/2.  Odd s: 2^{(s-1)/2} ((s-1)/2)! / sqrt(2 pi).
    (Substitute t = z^2/2 in the Gamma integral.)
    """
    with _ctx():
        if s % 2 == 0:
            df = 1
            for j in range(s - 1, 0, -2):
                df *= j
            return Decimal(df) / 2
        m = (s - 1) // 2
        return Decimal(2 ** m * math.factorial(m)) * dec_inv_sqrt_2pi()


@functools.lru_cache(maxsize=None)
def half_hermite_coeffs(M: int):
    """Coefficients C[l][s] of h_l(z) = sum_s C[l][s] z^s for l < M (Decimal).

    Cholesky G = L L^T of the Hankel moment matrix G_ij = mu_{i+j}; then
    C = L^{-1} (lower triangular, positive diagonal).
    """
    with _ctx():
        mu = [half_moment(s) for s in range(2 * M)]
        G = [[mu[i + j] for j in range(M)] for i in range(M)]
        L = [[Decimal(0)] * M for _ in range(M)]
        for i in range(M):
            for j in range(i + 1):
                acc = G[i][j] - sum(L[i][k] * L[j][k] for k in range(j))
                if i == j:
                    L[i][i] = acc.sqrt()
                else:
                    L[i][j] = acc / L[j][j]
        # C = L^{-1} by forward substitution, column by column.
        C = [[Decimal(0)] * M for _ in range(M)]
        for col in range(M):
            for i in range(col, M):
                rhs = Decimal(1) if i == col else Decimal(0)
                rhs -= sum(L[i][k] * C[k][col] for k in range(col, i))
                C[i][col] = rhs / L[i][i]
        return tuple(tuple(row) for row in C)


def poly_eval(coeffs, z: Decimal) -> Decimal:
    """Horner evaluation of sum_s coeffs[s] z^s (Decimal)."""
    with _ctx():
        acc = Decimal(0)
        for c in reversed(coeffs):
            acc = acc * z + c
        return acc


def _poly_deriv_eval(coeffs, z: Decimal) -> Decimal:
    with _ctx():
        acc = Decimal(0)
        n = len(coeffs)
        for s in range(n - 1, 0, -1):
            acc = acc * z + s * coeffs[s]
        return acc


def _newton_polish(coeffs, x0: float, iters: int = 60) -> Decimal:
    with _ctx():
        x = Decimal(repr(float(x0)))
        eps = Decimal(10) ** (-(PREC - 8))
        for _ in range(iters):
            dx = poly_eval(coeffs, x) / _poly_deriv_eval(coeffs, x)
            x -= dx
            if abs(dx) <= eps * (1 + abs(x)):
                break
        return x


@functools.lru_cache(maxsize=None)
def half_range_hermite(Q: int):
    """Half-range Gauss-Hermite quadrature of order Q >= 1 (Decimal data).

    Returns a dict with
      C     : coefficients h_{l,s} for l <= Q + 1 (Decimal, lower-triangular),
      z     : the Q positive roots of h_Q, ascending (Decimal),
      w     : weights of Eq. "eq:wk_half" (Decimal),
      a     : a_l = h_{l+1,l+1}/h_{l,l} for l <= Q (Decimal).
    """
    if Q < 1:
        raise ValueError("Q >= 1")
    C = half_hermite_coeffs(Q + 2)
    with _ctx():
        a = [C[l + 1][l + 1] / C[l][l] for l in range(Q + 1)]
        # Initial guesses: FP64 eigenvalues of the Jacobi matrix of the
        # orthonormal recurrence z h_l = (1/a_l) h_{l+1} + beta_l h_l + ...;
        # the diagonal beta_l = <h_l, z h_l> follows from the coefficients:
        # z h_l has z^{l+1} coefficient C[l][l] and z^l coefficient C[l][l-1],
        # so beta_l = (C[l][l-1] - C[l][l] * C[l+1][l] / C[l+1][l+1]) / C[l][l].
        diag = []
        for l in range(Q):
            lower = C[l][l - 1] if l >= 1 else Decimal(0)
            beta = (lower - C[l][l] * C[l + 1][l] / C[l + 1][l + 1]) / C[l][l]
            diag.append(float(beta))
        off = [float(1 / a[l]) for l in range(Q - 1)]
        J = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
        guesses = np.sort(np.linalg.eigvalsh(J))
        hQ = C[Q][: Q + 1]
        z = [_newton_polish(hQ, g) for g in guesses]
        s2pi = dec_inv_sqrt_2pi()
        hQ1 = C[Q + 1][: Q + 2]
        w = []
        for zk in z:
            h1 = poly_eval(hQ1, zk)
            w.append(zk * a[Q] ** 2 / (h1 * h1 * (zk + C[Q][0] ** 2 * s2pi)))
    return {"C": C, "z": z, "w": w, "a": a}


def _he_coeffs(M: int):
    """Integer coefficients of He_0..He_{M-1}: He_{n+1} = z He_n - n He_{n-1}."""
    He = [[1], [0, 1]]
    for n in range(1, M - 1):
        nxt = [0] * (n + 2)
        for s, c in enumerate(He[n]):
            nxt[s + 1] += c
        for s, c in enumerate(He[n - 1]):
            nxt[s] -= n * c
        He.append(nxt)
    return He[:M]


@functools.lru_cache(maxsize=None)
def gauss_hermite(Q: int):
    """Full-range Gauss-Hermite quadrature of order Q (Decimal data).

    Roots of He_Q (probabilists'), Newton-polished in Decimal from the FP64
    nodes of numpy's hermegauss; weights Q!/He_{Q+1}(z_k)^2 (Eq. "eq:H_wk").
    Returns dict(z=..., w=..., He=integer coefficient lists for l <= Q+1).
    """
    if Q < 1:
        raise ValueError("Q >= 1")
    He = _he_coeffs(Q + 2)
    x0, _ = np.polynomial.hermite_e.hermegauss(Q)
    with _ctx():
        cQ = [Decimal(c) for c in He[Q]]
        cQ1 = [Decimal(c) for c in He[Q + 1]]
        z = [_newton_polish(cQ, g) for g in np.sort(x0)]
        # exact zero for the middle root of odd Q
        z = [Decimal(0) if abs(zz) < Decimal(10) ** (-(PREC - 10)) else zz for zz in z]
        fac = Decimal(math.factorial(Q))
        w = [fac / poly_eval(cQ1, zk) ** 2 for zk in z]
    return {"z": z, "w": w, "He": He}


def _laguerre_coeffs(M: int):
    """Exact coefficients (Fractions, ascending) of the Laguerre polynomials
    L_0..L_{M-1}: L_n(z) = sum_s (-1)^s C(n, s) z^s / s!, orthonormal on
    [0, inf) with weight exp(-z)."""
    from fractions import Fraction
    return [[Fraction((-1) ** s * math.comb(n, s), math.factorial(s)) for s in range(n + 1)] for n in range(M)]


@functools.lru_cache(maxsize=None)
def gauss_laguerre_half(Q: int):
    """Half-range Gauss-Laguerre quadrature of order Q (Decimal data), the
    first half-range family of Sec. IV.B (weight omega(z) = exp(-z), gamma = 1).

    Roots z_k of L_Q, Newton-polished in Decimal from numpy's laggauss nodes;
    weights w_k = z_k / ((Q + 1)^2 L_{Q+1}(z_k)^2) (the Gauss-Laguerre form of
    Eq. "eq:wk_half").  Returns dict(z=..., w=..., L=coefficient lists for
    l <= Q + 1 as Decimals).
    """
    if Q < 1:
        raise ValueError("Q >= 1")
    Lf = _laguerre_coeffs(Q + 2)
    x0, _ = np.polynomial.laguerre.laggauss(Q)
    with _ctx():
        L = [[Decimal(c.numerator) / Decimal(c.denominator) for c in row] for row in Lf]
        z = [_newton_polish(L[Q], g) for g in np.sort(x0)]
        w = [zk / ((Q + 1) ** 2 * poly_eval(L[Q + 1], zk) ** 2) for zk in z]
    return {"z": z, "w": w, "L": L}


def to_f64(seq) -> np.ndarray:
    return np.array([float(x) for x in seq], dtype=np.float64)
