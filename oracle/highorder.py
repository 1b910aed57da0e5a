"""High-order half-range Gauss-Hermite quadrature and force matrix (orders up
to the Q = 200 per half of the paper's HHLB(20;200) model, Sec. V).

Test infrastructure only (see the package docstring).

The 80-digit route of ``quadrature.half_range_hermite`` (monomial coefficients
of h_l) cannot reach these orders: the Hankel moment matrix loses about 2.5
digits per order, and the monomial coefficients of h_200 cancel over hundreds
of digits.  Here, with mpmath at ``2.5 Q + 60`` digits:

1. the Hankel matrix G_ij = mu_{i+j} of the half-range moments
   mu_s = int_0^inf z^s omega(z) dz = 2^{s/2} Gamma((s+1)/2) / (2 sqrt(pi)),
   omega(z) = exp(-z^2/2)/sqrt(2 pi), is Cholesky-factorised, G = L L^T;
2. the three-term recurrence of the orthonormal h_l (App. B) follows from L
   (Golub-Welsch): z h_l = b_{l+1} h_{l+1} + a_l h_l + b_l h_{l-1} with
   b_{l+1} = L_{l+1,l+1}/L_{l,l} and a_l = L_{l+1,l}/L_{l,l} - L_{l,l-1}/L_{l-1,l-1};
3. the nodes z_k are the roots of h_Q: eigenvalues of the Jacobi matrix in FP64,
   then Newton on h_Q evaluated by the recurrence (stable) at full precision;
4. the weights are those of Eq. "eq:wk_half",
   w_k = z_k a_Q^2 / (h_{Q+1}(z_k)^2 [z_k + h_Q(0)^2 / sqrt(2 pi)]), with
   a_Q = h_{Q+1,Q+1}/h_{Q,Q} = 1/b_{Q+1};
5. K^h of Eq. "eq:hh_Kk_hh" from the values h_l(z_k) and the derivative
   expansion of the orthonormal basis (Eqs. "eq:phip", "eq:hh_varphi"):
   h_l' = h_{l-1}/a_{l-1} - omega(0) h_l(0) sum_{s<l} h_s(0) h_s.

Pinned (tests/test_oracle_quadrature.py): agreement with the 80-digit route
at Q <= 32; exactness sum_k w_k z_k^s = mu_s for s < 2Q at Q = 200; the node
envelope of the paper's Fig. "fig:hh_hyp" (all |z_k| < 2.5 sqrt(Q)); the
recurrence at two precisions; the K^h identities at Q = 64.

Stored tables.  mpmath is not available everywhere the oracle runs, and Q = 200
takes about 40 s, so ``write_store`` keeps z_k, w_k and the recurrence of one
order as 40-digit decimal text (tests/golden/half_range_hermite_q<Q>.txt,
written by tests/golden/make_half_range_tables.py, which calls only this
module).  ``half_range_data(Q)`` reads that file when it exists (whatever
mpmath's presence, so that the oracle's results do not depend on it) and
computes the tables otherwise.  ``hh_force_matrix_rec`` forms K^h from these
data in FP64 by the same recurrence-value formula as ``hh_force_matrix_hp``;
from exact recurrence coefficients FP64 suffices (1e-13 of each column's
largest entry at Q = 100, pinned against the mpmath matrix).
"""
from __future__ import annotations

import functools
import os
from decimal import Decimal

import numpy as np

STORE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")
STORE_DIGITS = 40


class _LazyMpmath:
    """mpmath, imported on first use (the stored tables need no mpmath)."""

    def __getattr__(self, name):
        import mpmath
        return getattr(mpmath, name)


mp = _LazyMpmath()


def _dps(Q: int) -> int:
    return int(2.5 * Q) + 60


def half_moment_mp(s: int):
    return mp.power(2, mp.mpf(s) / 2) * mp.gamma(mp.mpf(s + 1) / 2) / (2 * mp.sqrt(mp.pi))


@functools.lru_cache(maxsize=None)
def half_range_recurrence_hp(Q: int, dps: int | None = None):
    """(a_l, b_{l+1}) for l = 0..Q of the orthonormal half-range Hermite
    polynomials (h_0 = 1/sqrt(mu_0)), as mpmath numbers at ``dps`` digits."""
    dps = dps or _dps(Q)
    with mp.workdps(dps):
        n = Q + 2
        mu = [half_moment_mp(s) for s in range(2 * n)]
        G = mp.matrix(n, n)
        for i in range(n):
            for j in range(n):
                G[i, j] = mu[i + j]
        L = mp.cholesky(G)
        a = [L[l + 1, l] / L[l, l] - (L[l, l - 1] / L[l - 1, l - 1] if l else 0) for l in range(n - 1)]
        b = [L[l + 1, l + 1] / L[l, l] for l in range(n - 1)]      # b[l] = b_{l+1}
        return tuple(a), tuple(b), 1 / mp.sqrt(mu[0])


def _values(Q: int, z, a, b, h0, L: int):
    """h_0(z) .. h_L(z) by the recurrence."""
    h = [h0, (z - a[0]) * h0 / b[0]]
    for l in range(1, L):
        h.append(((z - a[l]) * h[l] - b[l - 1] * h[l - 1]) / b[l])
    return h[:L + 1]


@functools.lru_cache(maxsize=None)
def half_range_hermite_hp(Q: int):
    """Nodes and weights (mpmath, ascending nodes) of the half-range
    Gauss-Hermite quadrature of order Q, and the recurrence."""
    dps = _dps(Q)
    a, b, h0 = half_range_recurrence_hp(Q, dps)
    from scipy.linalg import eigh_tridiagonal
    guesses = eigh_tridiagonal(np.array([float(x) for x in a[:Q]]), np.array([float(x) for x in b[:Q - 1]]),
                               eigvals_only=True)
    with mp.workdps(dps):
        z = []
        eps = mp.mpf(10) ** (-(dps - 10))
        for g in np.sort(guesses):
            x = mp.mpf(float(g))
            for _ in range(100):
                # h_Q and its derivative by the recurrence (differentiated)
                p, dp = [h0, (x - a[0]) * h0 / b[0]], [mp.mpf(0), h0 / b[0]]
                for l in range(1, Q):
                    p.append(((x - a[l]) * p[l] - b[l - 1] * p[l - 1]) / b[l])
                    dp.append((p[l] + (x - a[l]) * dp[l] - b[l - 1] * dp[l - 1]) / b[l])
                step = p[Q] / dp[Q]
                x -= step
                if abs(step) <= eps * (1 + abs(x)):
                    break
            z.append(x)
        aQ = 1 / b[Q]
        hQ0 = _values(Q, mp.mpf(0), a, b, h0, Q)[Q]
        w = []
        for zk in z:
            hQ1 = _values(Q, zk, a, b, h0, Q + 1)[Q + 1]
            w.append(zk * aQ ** 2 / (hQ1 ** 2 * (zk + hQ0 ** 2 / mp.sqrt(2 * mp.pi))))
    return {"z": tuple(z), "w": tuple(w), "a": a, "b": b, "h0": h0, "dps": dps}


@functools.lru_cache(maxsize=None)
def hh_force_matrix_hp(Q: int) -> np.ndarray:
    """K^h (2Q x 2Q, FP64) of Eq. "eq:hh_Kk_hh" from the recurrence-based
    values h_l(z_k), h_l(0); order +z_k then -z_k as in ``model.hh_force_matrix``."""
    d = half_range_hermite_hp(Q)
    a, b, h0, z, w = d["a"], d["b"], d["h0"], d["z"], d["w"]
    with mp.workdps(40 + Q // 2):
        om0 = 1 / mp.sqrt(2 * mp.pi)
        H = [_values(Q, zk, a, b, h0, Q) for zk in z]          # h_l(z_k), l <= Q
        c0 = _values(Q, mp.mpf(0), a, b, h0, Q)               # h_l(0)
        Phi0 = [sum(c0[s] * H[k][s] for s in range(Q)) for k in range(Q)]
        # tail[k][l] = sum_{s=l+1}^{Q-1} h_s(0) h_s(z_k)
        tail = []
        for k in range(Q):
            acc, row = mp.mpf(0), [None] * Q
            for l in range(Q - 1, -1, -1):
                row[l] = acc
                acc += c0[l] * H[k][l]
            tail.append(row)
        # same-half bracket B[k][k'] = sum_{l<=Q-2} h_l(z_k') (omega(0) h_l(0) tail[k][l] - h_{l+1}(z_k)/a_l)
        # with 1/a_l = b_{l+1} (h_{l+1}' = h_l/a_l - ...)
        inner = [[om0 * c0[l] * tail[k][l] - b[l] * H[k][l + 1] for l in range(Q - 1)] for k in range(Q)]
        K = np.zeros((2 * Q, 2 * Q))
        for k in range(Q):
            for kp in range(Q):
                same = sum(H[kp][l] * inner[k][l] for l in range(Q - 1))
                jump = om0 * Phi0[k] * Phi0[kp] / 2
                for sk, skp in ((0, 0), (0, 1), (1, 0), (1, 1)):
                    sign = 1 if sk == 0 else -1
                    val = (same if sk == skp else 0) - jump
                    K[sk * Q + k, skp * Q + kp] = float(w[k] * sign * val)
    return K


def to_f64(seq) -> np.ndarray:
    return np.array([float(x) for x in seq], dtype=np.float64)


# ----------------------------------------------------------------------------
# stored tables
# ----------------------------------------------------------------------------
def store_path(Q: int) -> str:
    return os.path.join(STORE_DIR, f"half_range_hermite_q{Q}.txt")


def write_store(Q: int, path: str | None = None) -> str:
    """Write z_k, w_k (k < Q), a_l, b_{l+1} (l <= Q) and h_0 of order Q as
    STORE_DIGITS-digit decimal text, one value per line after a header."""
    d = half_range_hermite_hp(Q)
    path = path or store_path(Q)
    with mp.workdps(d["dps"]):
        def fmt(x):
            return mp.nstr(x, STORE_DIGITS, strip_zeros=False, min_fixed=1, max_fixed=0)
        lines = [f"# half-range Gauss-Hermite quadrature of order {Q} (App. B, Eq. \"eq:wk_half\"),",
                 f"# written by oracle.highorder.write_store from the mpmath tables at {d['dps']} digits",
                 f"Q {Q}", f"h0 {fmt(d['h0'])}"]
        lines += [f"z {fmt(x)}" for x in d["z"]]
        lines += [f"w {fmt(x)}" for x in d["w"]]
        lines += [f"a {fmt(x)}" for x in d["a"][:Q + 1]]
        lines += [f"b {fmt(x)}" for x in d["b"][:Q + 1]]
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    return path


def read_store(path: str) -> dict:
    """The stored tables as Decimal tuples: z, w (ascending nodes), a, b, h0."""
    out = {"z": [], "w": [], "a": [], "b": []}
    Q = h0 = None
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, val = line.split()
            if key == "Q":
                Q = int(val)
            elif key == "h0":
                h0 = Decimal(val)
            else:
                out[key].append(Decimal(val))
    if Q is None or h0 is None or len(out["z"]) != Q or len(out["w"]) != Q or len(out["a"]) != Q + 1 \
            or len(out["b"]) != Q + 1:
        raise ValueError(f"{path}: malformed half-range table")
    return {"Q": Q, "h0": h0, **{k: tuple(v) for k, v in out.items()}}


@functools.lru_cache(maxsize=None)
def half_range_data(Q: int) -> dict:
    """z, w, a, b, h0 of order Q as Decimal tuples: from the stored file if it
    exists, else computed with mpmath (rounded to STORE_DIGITS digits)."""
    path = store_path(Q)
    if os.path.exists(path):
        return read_store(path)
    d = half_range_hermite_hp(Q)
    with mp.workdps(d["dps"]):
        def dec(x):
            return Decimal(mp.nstr(x, STORE_DIGITS, strip_zeros=False, min_fixed=1, max_fixed=0))
        return {"Q": Q, "h0": dec(d["h0"]), "z": tuple(map(dec, d["z"])), "w": tuple(map(dec, d["w"])),
                "a": tuple(map(dec, d["a"][:Q + 1])), "b": tuple(map(dec, d["b"][:Q + 1]))}


@functools.lru_cache(maxsize=None)
def hh_force_matrix_rec(Q: int) -> np.ndarray:
    """K^h (2Q x 2Q, FP64) of Eq. "eq:hh_Kk_hh" from ``half_range_data(Q)``:
    the values h_l(z_k), h_l(0) by the three-term recurrence in FP64, then the
    formula of ``hh_force_matrix_hp`` (same-half bracket with the derivative
    expansion of Eqs. "eq:phip", "eq:hh_varphi", and the jump term
    -omega(0)/2 Phi_0(z_k) Phi_0(z_k') in every block)."""
    d = half_range_data(Q)
    z, w = to_f64(d["z"]), to_f64(d["w"])
    a, b, h0 = to_f64(d["a"]), to_f64(d["b"]), float(d["h0"])
    om0 = 1.0 / np.sqrt(2.0 * np.pi)

    def values(x):
        H = np.zeros((len(x), Q + 1))
        H[:, 0] = h0
        H[:, 1] = (x - a[0]) * h0 / b[0]
        for l in range(1, Q):
            H[:, l + 1] = ((x - a[l]) * H[:, l] - b[l - 1] * H[:, l - 1]) / b[l]
        return H

    H = values(z)[:, :Q]                        # h_l(z_k), l < Q
    c0 = values(np.zeros(1))[0, :Q]             # h_l(0)
    Phi0 = H @ c0
    tail = np.zeros((Q, Q))                     # tail[k, l] = sum_{s=l+1}^{Q-1} h_s(0) h_s(z_k)
    for l in range(Q - 2, -1, -1):
        tail[:, l] = tail[:, l + 1] + c0[l + 1] * H[:, l + 1]
    inner = om0 * c0[None, :Q - 1] * tail[:, :Q - 1] - b[None, :Q - 1] * H[:, 1:Q]
    same = inner @ H[:, :Q - 1].T               # [k, k']
    jump = om0 * np.outer(Phi0, Phi0) / 2.0
    K = np.zeros((2 * Q, 2 * Q))
    for sk in (0, 1):
        sign = 1.0 if sk == 0 else -1.0
        for skp in (0, 1):
            blk = (same if sk == skp else 0.0) - jump
            K[sk * Q:(sk + 1) * Q, skp * Q:(skp + 1) * Q] = (sign * w)[:, None] * blk
    return K
