// Host-side tables of libhlb: quadratures, force matrices, equilibrium
// recurrences and the grid, in FP64.
//
// Half-range Hermite (App. B, weight omega(z) = exp(-z^2/2)/sqrt(2 pi) on
// [0, inf), gamma_l = 1): the recurrence coefficients of the orthonormal
// polynomials h_l come from the Stieltjes procedure run on a discretisation
// of the weight (composite Gauss-Legendre on panels of width 1/2), in its
// orthonormal (Lanczos-like) form.  The discrete measure must integrate
// h_l^2 omega, of degree 2l, to rounding: 20 nodes per panel do so for the
// first 34 terms, 60 up to the 202 terms of Q = 200 (with 20 the coefficients
// drift from l ~ 50 on, by 1e-3 at l = 100; the procedure itself is not the
// limit, a reorthogonalised Lanczos run on the same nodes drifts alike).  The Q quadrature points are the
// eigenvalues of the Jacobi matrix (Sturm bisection, then Newton on h_Q);
// the weights are the Christoffel numbers 1 / sum_{l<Q} h_l(z_k)^2, equal to
// Eq. "eq:wk_half".  Full-range Gauss-Hermite (Sec. IV.A.1) uses the known
// recurrence He_{l+1} = z He_l - l He_{l-1} the same way.
//
// Force matrices: K^h of Eq. "eq:hh_Kk_hh" (with h_{l,0} = h_l(0) and
// h_{l,l}/h_{l+1,l+1} = 1/a_l, Eq. "eq:a_def") and K^H of Eq. "eq:H_Kk".
//
// Equilibrium (per node, also on the device): g_k = w_k sum_{l<=N} G_l h_l(z_k)
// with G_l^{+-} = int_0^inf g(+-p) h_l(p) dp.  Instead of the monomial
// expansion of Eq. "eq:hh_gk" (whose terms exceed their sum by up to 1e9 at
// Q = 16), G_l is generated in the orthonormal basis: integrating by parts
// with (p - u) g = -T dg/dp and the derivative expansion of h_l (Eqs.
// "eq:phip", "eq:hh_varphi": h_l' = h_{l-1}/a_{l-1} - omega(0) h_l(0)
// sum_{s<l} h_s(0) h_s),
//   int_0^inf p g h_l = u G_l + T [ g(0) h_l(0) + G_{l-1}/a_{l-1}
//                                   - omega(0) h_l(0) sum_{s<l} h_s(0) G_s ],
// and the three-term recurrence gives G_{l+1} = a_l (int p g h_l) + b_l G_l
// + c_l G_{l-1}, starting from G_0 = h_0 (1 + erf(u/sqrt(2T)))/2.
// Full-range (Eq. "eq:H_gk"): G_{l+1} = u G_l + l (T - 1) G_{l-1}, G_0 = 1,
// G_1 = u, which is the sum printed there with the exponent of (T - 1) read as s.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "hlb_internal.h"

namespace hlb {
namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

// Gauss-Legendre nodes/weights on [-1, 1] (Newton on P_n from cos guesses).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            // P_n = p1, P_{n-1} = p0
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Orthonormal recurrence z p_l = sb[l+1] p_{l+1} + alpha[l] p_l + sb[l] p_{l-1},
// p_0 = 1/sb[0] (sb = sqrt(beta), beta_0 = total mass).
struct Recurrence {
    std::vector<double> alpha, sb;
};

// Discretised Stieltjes procedure for the half-range Gaussian weight; M terms.
Recurrence half_range_recurrence(int M) {
    const double zmax = 14.0 + 2.5 * std::sqrt((double)M + 2.0);
    const int per = M <= 34 ? 20 : 60;
    const double width = 0.5;
    const int panels = (int)std::ceil(zmax / width);
    std::vector<double> gx, gw;
    gauss_legendre(per, gx, gw);
    std::vector<double> t, lam;
    t.reserve(panels * per);
    lam.reserve(panels * per);
    for (int pnl = 0; pnl < panels; ++pnl) {
        double a = pnl * width, b = a + width;
        for (int i = 0; i < per; ++i) {
            double z = 0.5 * (a + b) + 0.5 * (b - a) * gx[i];
            t.push_back(z);
            lam.push_back(0.5 * (b - a) * gw[i] * std::exp(-0.5 * z * z) / std::sqrt(2.0 * kPi));
        }
    }
    const size_t n = t.size();
    Recurrence r;
    r.alpha.assign(M, 0.0);
    r.sb.assign(M + 1, 0.0);
    double mass = 0.0;
    for (size_t j = 0; j < n; ++j) mass += lam[j];
    r.sb[0] = std::sqrt(mass);
    std::vector<double> prev(n, 0.0), cur(n, 1.0 / r.sb[0]), nxt(n);
    for (int l = 0; l < M; ++l) {
        double a = 0.0;
        for (size_t j = 0; j < n; ++j) a += lam[j] * t[j] * cur[j] * cur[j];
        r.alpha[l] = a;
        double nb = 0.0;
        for (size_t j = 0; j < n; ++j) {
            nxt[j] = (t[j] - a) * cur[j] - (l ? r.sb[l] : 0.0) * prev[j];
            nb += lam[j] * nxt[j] * nxt[j];
        }
        r.sb[l + 1] = std::sqrt(nb);
        for (size_t j = 0; j < n; ++j) {
            prev[j] = cur[j];
            cur[j] = nxt[j] / r.sb[l + 1];
        }
    }
    return r;
}

// Probabilists' Hermite, unit-mass weight: alpha = 0, beta_l = l, beta_0 = 1.
Recurrence hermite_recurrence(int M) {
    Recurrence r;
    r.alpha.assign(M, 0.0);
    r.sb.assign(M + 1, 0.0);
    r.sb[0] = 1.0;
    for (int l = 1; l <= M; ++l) r.sb[l] = std::sqrt((double)l);
    return r;
}

// Laguerre, weight exp(-z) on [0, inf) (unit mass): with p_l = (-1)^l L_l
// (positive leading coefficient), z p_l = (l+1) p_{l+1} + (2l+1) p_l + l p_{l-1}.
Recurrence laguerre_recurrence(int M) {
    Recurrence r;
    r.alpha.resize(M);
    for (int l = 0; l < M; ++l) r.alpha[l] = 2.0 * l + 1.0;
    r.sb.assign(M + 1, 0.0);
    r.sb[0] = 1.0;
    for (int l = 1; l <= M; ++l) r.sb[l] = (double)l;
    return r;
}

// Orthonormal polynomial values p_0..p_L at z, and p_L'(z).
void ortho_values(const Recurrence& r, int L, double z, double* vals, double* dL = nullptr) {
    double pm = 0.0, p = 1.0 / r.sb[0];
    double dm = 0.0, d = 0.0;
    vals[0] = p;
    for (int l = 0; l < L; ++l) {
        double pn = ((z - r.alpha[l]) * p - (l ? r.sb[l] * pm : 0.0)) / r.sb[l + 1];
        double dn = (p + (z - r.alpha[l]) * d - (l ? r.sb[l] * dm : 0.0)) / r.sb[l + 1];
        pm = p;
        p = pn;
        dm = d;
        d = dn;
        vals[l + 1] = p;
    }
    if (dL) *dL = d;
}

// Eigenvalues of the Q x Q Jacobi matrix (ascending) by Sturm bisection,
// polished by Newton on p_Q.
std::vector<double> gauss_nodes(const Recurrence& r, int Q) {
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < Q; ++i) {
        double rad = (i > 0 ? r.sb[i] : 0.0) + (i + 1 < Q ? r.sb[i + 1] : 0.0);
        lo = std::min(lo, r.alpha[i] - rad);
        hi = std::max(hi, r.alpha[i] + rad);
    }
    auto count_below = [&](double x) {
        int c = 0;
        double q = 1.0;
        for (int i = 0; i < Q; ++i) {
            double e2 = i ? r.sb[i] * r.sb[i] : 0.0;
            q = (r.alpha[i] - x) - (i ? e2 / q : 0.0);
            if (q == 0.0) q = -1e-300;
            if (q < 0) ++c;
        }
        return c;
    };
    std::vector<double> z(Q);
    std::vector<double> vals(Q + 2);
    for (int k = 0; k < Q; ++k) {
        double a = lo, b = hi;
        for (int it = 0; it < 200 && b - a > 1e-15 * std::max(1.0, std::fabs(a) + std::fabs(b)); ++it) {
            double m = 0.5 * (a + b);
            if (count_below(m) > k) b = m; else a = m;
        }
        double x = 0.5 * (a + b);
        for (int it = 0; it < 5; ++it) {
            double d;
            ortho_values(r, Q, x, vals.data(), &d);
            if (d == 0.0) break;
            double dx = vals[Q] / d;
            if (!std::isfinite(dx) || std::fabs(dx) > 1e-6 * std::max(1.0, std::fabs(x))) break;
            x -= dx;
        }
        z[k] = x;
    }
    return z;
}

}  // namespace

void absent_axis(AxisTables& out) {
    out = AxisTables();
    out.count = 1;
    out.p = {0.0};
    out.w = {1.0};
    out.K = {0.0};
    out.N = 0;
    out.T = {1.0};
}

// Both half-range families (App. B): the orthonormal p_l of the weight omega
// on [0, inf) with derivative expansion
//   p_l' = d_l p_{l-1} - omega(0) p_l(0) sum_{s<l} p_s(0) p_s,
// half-range Hermite: omega(z) = exp(-z^2/2)/sqrt(2 pi), d_l = 1/a_{l-1}
// (Eqs. "eq:phip", "eq:hh_varphi"); Gauss-Laguerre: omega(z) = exp(-z),
// d_l = 0 (L_l' = -sum_{s<l} L_s, in the sign convention p_l = (-1)^l L_l).
// K of Eq. "eq:hh_Kk" then reads, for k, k' on the same half,
//   w_k s_k [ sum_{l<=Q-2} p_l(z_k') (omega(0) p_l(0) sum_{s=l+1}^{Q-1} p_s(0) p_s(z_k) - d_{l+1} p_{l+1}(z_k))
//            - omega(0)/2 Phi0(z_k) Phi0(z_k') ],
// and only the last term across halves (Eqs. "eq:hh_Kk_hh", "eq:hh_Kk_L").
std::string build_half_axis(int Q, int N, AxisTables& out, bool laguerre) {
    if (Q < 1 || Q > (laguerre ? kMaxQLaguerre : kMaxQHalf))
        return laguerre ? "Gauss-Laguerre Qx must be in [1, 16]" : "Qx must be in [1, 200]";
    if (N < 0 || N >= Q) return "Nx_eq must be in [0, Qx - 1]";
    const Recurrence r = laguerre ? laguerre_recurrence(Q + 2) : half_range_recurrence(Q + 2);
    const double om0 = laguerre ? 1.0 : 1.0 / std::sqrt(2.0 * kPi);
    out = AxisTables();
    out.om0 = om0;
    out.Q = Q;
    out.half = true;
    out.count = 2 * Q;
    out.N = N;
    std::vector<double> z = gauss_nodes(r, Q);
    std::vector<double> w(Q);
    std::vector<std::vector<double>> H(Q, std::vector<double>(Q + 2));
    for (int k = 0; k < Q; ++k) {
        ortho_values(r, Q + 1, z[k], H[k].data());
        double s = 0.0;
        for (int l = 0; l < Q; ++l) s += H[k][l] * H[k][l];
        w[k] = 1.0 / s;
    }
    std::vector<double> h0(Q + 2);
    ortho_values(r, Q + 1, 0.0, h0.data());
    out.p.resize(2 * Q);
    out.w.resize(2 * Q);
    for (int k = 0; k < Q; ++k) {
        out.p[k] = z[k];
        out.p[Q + k] = -z[k];
        out.w[k] = out.w[Q + k] = w[k];
    }
    // K^h, Eq. "eq:hh_Kk_hh" (p_0 = 1, gamma = 1); lead ratio h_{l,l}/h_{l+1,l+1} = sb[l+1].
    std::vector<double> Phi0(Q, 0.0);
    for (int k = 0; k < Q; ++k)
        for (int s = 0; s < Q; ++s) Phi0[k] += h0[s] * H[k][s];
    // tail[k][l] = sum_{s=l+1}^{Q-1} h_{s,0} h_s(z_k)
    std::vector<std::vector<double>> tail(Q, std::vector<double>(Q, 0.0));
    for (int k = 0; k < Q; ++k) {
        double acc = 0.0;
        for (int l = Q - 1; l >= 0; --l) {
            tail[k][l] = acc;
            acc += h0[l] * H[k][l];
        }
    }
    out.jc.resize(2 * Q);
    out.jd.resize(2 * Q);
    for (int k = 0; k < 2 * Q; ++k) {
        out.jc[k] = -0.5 * om0 * w[k % Q] * (k < Q ? 1.0 : -1.0) * Phi0[k % Q];
        out.jd[k] = Phi0[k % Q];
    }
    out.K.assign(4 * Q * Q, 0.0);
    for (int k = 0; k < 2 * Q; ++k) {
        const int kk = k % Q;
        const double sk = k < Q ? 1.0 : -1.0;
        for (int kp = 0; kp < 2 * Q; ++kp) {
            const int kkp = kp % Q;
            const double skp = kp < Q ? 1.0 : -1.0;
            double val = 0.0;
            if (sk == skp) {
                for (int l = 0; l <= Q - 2; ++l)
                    val += H[kkp][l] * (h0[l] * om0 * tail[kk][l] - (laguerre ? 0.0 : r.sb[l + 1]) * H[kk][l + 1]);
            }
            val -= 0.5 * om0 * Phi0[kk] * Phi0[kkp];
            out.K[k * 2 * Q + kp] = w[kk] * sk * val;
        }
    }
    // equilibrium tables
    out.T.assign(Q * (N + 1), 0.0);
    for (int k = 0; k < Q; ++k)
        for (int l = 0; l <= N; ++l) out.T[k * (N + 1) + l] = w[k] * H[k][l];
    out.ra.resize(N);
    out.rb.resize(N);
    out.rc.resize(N);
    out.dcoef.resize(N);
    out.h0.assign(h0.begin(), h0.begin() + N + 1);
    for (int l = 0; l < N; ++l) {
        // h_{l+1} = ((z - alpha_l) h_l - sb_l h_{l-1}) / sb_{l+1}
        out.ra[l] = 1.0 / r.sb[l + 1];
        out.rb[l] = -r.alpha[l] / r.sb[l + 1];
        out.rc[l] = l ? -r.sb[l] / r.sb[l + 1] : 0.0;
        out.dcoef[l] = laguerre ? 0.0 : r.sb[l + 1];      // d_{l+1}: coefficient of p_l in p_{l+1}'
    }
    return "";
}

std::string build_full_axis(int Q, int N, AxisTables& out) {
    if (Q < 2 || Q > kMaxQ || (Q % 2)) return "full-range orders must be 0 or even in [2, 32]";
    if (N < 0 || N >= Q) return "equilibrium order must be in [0, Q - 1]";
    const Recurrence r = hermite_recurrence(Q + 1);
    out = AxisTables();
    out.Q = Q;
    out.half = false;
    out.count = Q;
    out.N = N;
    std::vector<double> z = gauss_nodes(r, Q);
    // odd-free: Q even, so no zero node; symmetrise the computed pairs
    for (int k = 0; k < Q / 2; ++k) {
        double m = 0.5 * (z[Q - 1 - k] - z[k]);
        z[k] = -m;
        z[Q - 1 - k] = m;
    }
    out.p = z;
    out.w.resize(Q);
    std::vector<std::vector<double>> He(Q, std::vector<double>(Q + 1));
    for (int k = 0; k < Q; ++k) {
        // He_l(z) (unnormalised) by its recurrence
        He[k][0] = 1.0;
        He[k][1] = z[k];
        for (int l = 1; l < Q; ++l) He[k][l + 1] = z[k] * He[k][l] - l * He[k][l - 1];
        double s = 0.0, fact = 1.0;
        for (int l = 0; l < Q; ++l) {
            if (l) fact *= l;
            s += He[k][l] * He[k][l] / fact;
        }
        out.w[k] = 1.0 / s;
    }
    out.K.assign(Q * Q, 0.0);
    for (int k = 0; k < Q; ++k)
        for (int kp = 0; kp < Q; ++kp) {
            double acc = 0.0, fact = 1.0;
            for (int l = 0; l <= Q - 2; ++l) {
                if (l) fact *= l;
                acc += He[k][l + 1] * He[kp][l] / fact;
            }
            out.K[k * Q + kp] = -out.w[k] * acc;
        }
    out.T.assign(Q * (N + 1), 0.0);
    for (int k = 0; k < Q; ++k) {
        double fact = 1.0;
        for (int l = 0; l <= N; ++l) {
            if (l) fact *= l;
            out.T[k * (N + 1) + l] = out.w[k] * He[k][l] / fact;
        }
    }
    return "";
}

std::string build_full_x_axis(int Q, int N, AxisTables& out) {
    AxisTables full;
    std::string e = build_full_axis(Q, N, full);
    if (!e.empty()) return e;
    const int h = Q / 2;
    std::vector<int> perm(Q);
    for (int i = 0; i < h; ++i) {
        perm[i] = h + i;            // +z_{i+1}
        perm[h + i] = h - 1 - i;    // -z_{i+1}
    }
    out = AxisTables();
    out.Q = h;
    out.half = false;
    out.mirror = true;
    out.count = Q;
    out.N = N;
    out.p.resize(Q);
    out.w.resize(Q);
    out.K.assign((size_t)Q * Q, 0.0);
    for (int i = 0; i < Q; ++i) {
        out.p[i] = full.p[perm[i]];
        out.w[i] = full.w[perm[i]];
        for (int j = 0; j < Q; ++j) out.K[(size_t)i * Q + j] = full.K[(size_t)perm[i] * Q + perm[j]];
    }
    out.T.assign((size_t)h * (N + 1), 0.0);
    for (int k = 0; k < h; ++k)
        for (int l = 0; l <= N; ++l) out.T[(size_t)k * (N + 1) + l] = full.T[(size_t)perm[k] * (N + 1) + l];
    return "";
}

// G_l = int_0^inf g(p) h_l(p) dp for l <= N (g the Gaussian of mean us and
// temperature T) by composite Gauss-Legendre quadrature over [0, max(us, 0) +
// 40 sqrt(T)] (panels of width min(1, sqrt T)/4, 20 nodes each), h_l(p) by
// the three-term recurrence.  The error is absolute, about eps times the
// largest term; the integration-by-parts recurrence below instead carries its
// rounding along a solution that grows about threefold per order (1e-11 of the
// largest g_k at N = 10, 5e-7 at N = 20, 1e-1 at N = 31 at rest).
void half_range_projection_quadrature(const AxisTables& ax, double us, double T, double* G) {
    struct Rule { std::vector<double> x, w; };
    static const Rule rule = [] { Rule r; gauss_legendre(20, r.x, r.w); return r; }();   // thread-safe init
    const std::vector<double>& gx = rule.x;
    const std::vector<double>& gw = rule.w;
    const int N = ax.N;
    const double width = 0.25 * std::min(1.0, std::sqrt(T));
    const double top = std::max(us, 0.0) + 40.0 * std::sqrt(T);
    const int panels = (int)std::ceil(top / width);
    const double norm = 1.0 / std::sqrt(2.0 * kPi * T);
    for (int l = 0; l <= N; ++l) G[l] = 0.0;
    for (int pnl = 0; pnl < panels; ++pnl) {
        const double a = pnl * width;
        for (int i = 0; i < 20; ++i) {
            const double p = a + 0.5 * width * (1.0 + gx[i]);
            const double d = p - us;
            const double wt = 0.5 * width * gw[i] * norm * std::exp(-d * d / (2.0 * T));
            double hm = 0.0, h = ax.h0[0];
            G[0] += wt * h;
            for (int l = 0; l < N; ++l) {
                const double hn = (ax.ra[l] * p + ax.rb[l]) * h + ax.rc[l] * hm;
                hm = h;
                h = hn;
                G[l + 1] += wt * h;
            }
        }
    }
}

void axis_equilibrium(const AxisTables& ax, double u, double T, double* g) {
    if (ax.count == 1 && !ax.half && ax.Q == 0) {
        g[0] = 1.0;
        return;
    }
    const int N = ax.N;
    double G[kMaxN + 2];
    if (ax.half && N > kStableRecurrenceN) {
        const int Q = ax.Q;
        for (int sgn = 0; sgn < 2; ++sgn) {
            half_range_projection_quadrature(ax, sgn ? -u : u, T, G);
            for (int k = 0; k < Q; ++k) {
                double acc = 0.0;
                for (int l = 0; l <= N; ++l) acc += ax.T[k * (N + 1) + l] * G[l];
                g[sgn * Q + k] = acc;
            }
        }
    } else if (ax.half) {
        const int Q = ax.Q;
        const double om0 = ax.om0;
        const double g0 = std::exp(-u * u / (2.0 * T)) / std::sqrt(2.0 * kPi * T);
        for (int sgn = 0; sgn < 2; ++sgn) {
            const double us = sgn ? -u : u;
            G[0] = ax.h0[0] * 0.5 * (1.0 + std::erf(us / std::sqrt(2.0 * T)));
            double S = 0.0;
            for (int l = 0; l < N; ++l) {
                const double gm1 = l ? G[l - 1] : 0.0;
                const double ig = (l ? gm1 * ax.dcoef[l - 1] : 0.0) - om0 * ax.h0[l] * S;
                const double pg = us * G[l] + T * (g0 * ax.h0[l] + ig);
                G[l + 1] = ax.ra[l] * pg + ax.rb[l] * G[l] + ax.rc[l] * gm1;
                S += ax.h0[l] * G[l];
            }
            for (int k = 0; k < Q; ++k) {
                double acc = 0.0;
                for (int l = 0; l <= N; ++l) acc += ax.T[k * (N + 1) + l] * G[l];
                g[sgn * Q + k] = acc;
            }
        }
    } else if (ax.mirror) {
        // rows of the +z nodes; the -z nodes with -u (He_l(-z) = (-1)^l He_l(z))
        for (int sgn = 0; sgn < 2; ++sgn) {
            const double us = sgn ? -u : u;
            G[0] = 1.0;
            if (N >= 1) G[1] = us;
            for (int l = 1; l < N; ++l) G[l + 1] = us * G[l] + l * (T - 1.0) * G[l - 1];
            for (int k = 0; k < ax.Q; ++k) {
                double acc = 0.0;
                for (int l = 0; l <= N; ++l) acc += ax.T[k * (N + 1) + l] * G[l];
                g[sgn * ax.Q + k] = acc;
            }
        }
    } else {
        G[0] = 1.0;
        if (N >= 1) G[1] = u;
        for (int l = 1; l < N; ++l) G[l + 1] = u * G[l] + l * (T - 1.0) * G[l - 1];
        for (int k = 0; k < ax.Q; ++k) {
            double acc = 0.0;
            for (int l = 0; l <= N; ++l) acc += ax.T[k * (N + 1) + l] * G[l];
            g[k] = acc;
        }
    }
}

void grid_widths(int nx, double L, double A, std::vector<double>& dx) {
    dx.assign(nx, L / nx);
    if (A <= 0.0) return;
    const double deta = 2.0 * std::atanh(A) / nx;
    auto x_of = [&](double eta) { return 0.5 * L + L / (2.0 * A) * std::tanh(eta); };
    for (int i = 1; i <= nx; ++i) {
        const double eta = (i - 0.5 * (nx + 1)) * deta;
        dx[i - 1] = x_of(eta + 0.5 * deta) - x_of(eta - 0.5 * deta);
    }
}

void gauss_legendre_rule(int n, std::vector<double>& x, std::vector<double>& w) { gauss_legendre(n, x, w); }

}  // namespace hlb
