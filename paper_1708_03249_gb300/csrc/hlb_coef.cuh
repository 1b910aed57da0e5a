// Equilibrium factor lines in double-float (FP32 groups with equilibrium
// orders up to 15): the coefficient recurrences of the half- and full-range
// projections (App. A, Eqs. "eq:hh_gk", "eq:H_gk") and their compensated dot
// products with the quadrature tables.  Used by the node pass (hlb_node.cu)
// and the persistent batched kernel (hlb_persist.cu).
#pragma once

#include <cuda_runtime.h>

#include "hlb_device.cuh"
#include "hlb_internal.h"

namespace hlb {

// The sizes factor_line_df reads, copied out of a GroupDev (a small value to
// pass to a function that is not inlined).
struct FactorDims {
    int Nx, Ny, Nz, Qx, QX2, VY, VZ, ncp, Qy, Qz, x_full;
    float2 m_om0f;
    __device__ explicit FactorDims(const GroupDev& g)
        : Nx(g.Nx), Ny(g.Ny), Nz(g.Nz), Qx(g.Qx), QX2(g.QX2), VY(g.VY), VZ(g.VZ), ncp(g.ncp), Qy(g.Qy), Qz(g.Qz),
          x_full(g.x_full), m_om0f(g.m_om0f) {}
};

// FP32 groups whose equilibrium orders are all below NM (double-float path,
// orders up to 15): one thread per node, coefficients in registers.  The FP64 prelude (erf,
// exp, sqrt) runs once per node on full warps; each role's recurrence is
// followed at once by its dot products with the quadrature tables (broadcast
// reads from shared memory); a warp's 32 factor lines are assembled in shared
// memory and written out contiguously.
template <int NM>
__device__ __forceinline__ void half_range_G_df(int r, const NodeDF& in, const float2* recf, int Nx, float2 m_om0,
                                                float2 (&G)[NM]) {
    const float2* ra = recf;
    const float2* rb = recf + Nx;
    const float2* rc = recf + 2 * Nx;
    const float2* h0 = recf + 3 * Nx;
    const float2* inv_ra = recf + 4 * Nx + 1;
    const float sg = r ? -1.0f : 1.0f;
    const float2 us = make_float2(sg * in.ux.x, sg * in.ux.y);
    const float2 half = df_add(make_float2(0.5f, 0.0f), make_float2(0.5f * sg * in.erf_z.x, 0.5f * sg * in.erf_z.y));
    G[0] = df_mul(h0[0], half);
    float2 S = make_float2(0.0f, 0.0f), gm1 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int l = 0; l < NM - 1; ++l) {
        if (l < Nx) {
            float2 ig = df_mul(df_mul(m_om0, h0[l]), S);
            if (l) ig = df_add(ig, df_mul(gm1, inv_ra[l - 1]));
            const float2 pg = df_add(df_mul(us, G[l]), df_mul(in.T, df_add(df_mul(in.g0, h0[l]), ig)));
            G[l + 1] = df_add(df_add(df_mul(ra[l], pg), df_mul(rb[l], G[l])), df_mul(rc[l], gm1));
            S = df_add(S, df_mul(h0[l], G[l]));
            gm1 = G[l];
        }
    }
}

template <int NM>
__device__ __forceinline__ void full_range_G_df(float2 u, float2 Tm1, int N, float2 (&G)[NM]) {
    G[0] = make_float2(1.0f, 0.0f);
    G[1] = u;
#pragma unroll
    for (int l = 1; l < NM - 1; ++l)
        if (l < N) G[l + 1] = df_add(df_mul(u, G[l]), df_mul(df_mul(make_float2((float)l, 0.0f), Tm1), G[l - 1]));
}

// Two dot products at once (table rows 2k and 2k+1, one per lane of the f32x2
// registers) with the same double-float coefficients G, by the compensated
// dot product Dot2 of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005):
// TwoProduct of the high parts, TwoSum into the running sum, the rounding
// errors and the products with the low parts of the table and of G summed in
// the error term.  The result is as accurate as a double-float evaluation
// (about twice the FP32 precision, times the condition number) at a third of
// its instructions.  P[l] = (T_2k,l hi, T_2k+1,l hi, T_2k,l lo, T_2k+1,l lo).
template <int NM>
__device__ __forceinline__ void dot2_pair(const float4* P, const float2 (&G)[NM], int N, float2& r0, float2& r1) {
    float2 acc = f2(0.0f), err = f2(0.0f);
#pragma unroll
    for (int l = 0; l < NM; ++l) {
        if (l <= N) {
            const float4 t = P[l];
            const float2 th = make_float2(t.x, t.y), tl = make_float2(t.z, t.w);
            const float2 gh = f2(G[l].x), gl = f2(G[l].y);
            const float2 q = __fmul2_rn(th, f2(-G[l].x));        // -p, p = fl(th gh)
            const float2 e = __ffma2_rn(th, gh, q);               // th gh - p, exact
            const float2 sum = fsub2(acc, q);                     // acc + p
            const float2 bb = fsub2(sum, acc);
            const float2 t2 = fsub2(fsub2(acc, fsub2(sum, bb)), __fadd2_rn(q, bb));   // (acc + p) - sum, exact
            acc = sum;
            err = __fadd2_rn(err, __fadd2_rn(t2, e));
            err = __ffma2_rn(th, gl, __ffma2_rn(tl, gh, err));
        }
    }
    r0 = df_add(make_float2(acc.x, 0.0f), make_float2(err.x, 0.0f));
    r1 = df_add(make_float2(acc.y, 0.0f), make_float2(err.y, 0.0f));
}

// line[k] = (row k of a paired table . G) (times scale when given), k < nrows
template <int NM>
__device__ __forceinline__ void lines_dot2(float* line, const float4* P, int nrows, const float2 (&G)[NM], int N,
                                           const float2* scale) {
    for (int k = 0; k < nrows; k += 2) {
        float2 v0, v1;
        dot2_pair<NM>(P + (k >> 1) * (N + 1), G, N, v0, v1);
        if (scale) { v0 = df_mul(v0, *scale); v1 = df_mul(v1, *scale); }
        line[k] = v0.x + v0.y;
        if (k + 1 < nrows) line[k + 1] = v1.x + v1.y;
    }
}

// The factor line { n g_x (2Qx), g_y (VY), g_z (VZ), 1/tau, zeros to ncp } of
// one node from its n, u, T (FP64) and 1/tau; sPx, sPy, sPz the paired tables
// (dot2_pair layout), sRec the double-float recurrence table.  GD is GroupDev
// or FactorDims (the fields read here).
template <int NM, typename GD>
__device__ __forceinline__ void factor_line_df_in(const GD& g, const NodeDF& in, double itau, const float4* sPx,
                                                  const float4* sPy, const float4* sPz, const float2* sRec,
                                                  float* line) {
    const int Nx = g.Nx, Ny = g.Ny, Nz = g.Nz, Qx = g.Qx, QX2 = g.QX2, VY = g.VY, VZ = g.VZ, ncp = g.ncp;
    for (int o = QX2 + VY + VZ; o < ncp; ++o) line[o] = 0.0f;
    line[QX2 + VY + VZ] = (float)itau;
    if (itau == 0.0) {
        for (int o = 0; o < QX2 + VY + VZ; ++o) line[o] = 0.0f;
        return;
    }
    float2 G[NM];
#pragma unroll 1
    for (int r = 0; r < 2; ++r) {                    // n g_x, p_x > 0 then p_x < 0
        if (g.x_full)                                 // full-range p_x: G_l(+-u_x)
            full_range_G_df<NM>(r ? make_float2(-in.ux.x, -in.ux.y) : in.ux, in.Tm1, Nx, G);
        else
            half_range_G_df<NM>(r, in, sRec, Nx, g.m_om0f, G);
        lines_dot2<NM>(line + r * Qx, sPx, Qx, G, Nx, &in.n);
    }
    if (g.Qy) {
        full_range_G_df<NM>(in.uy, in.Tm1, Ny, G);
        lines_dot2<NM>(line + QX2, sPy, VY, G, Ny, nullptr);
    } else {
        line[QX2] = 1.0f;
    }
    if (g.Qz) {
        full_range_G_df<NM>(in.uz, in.Tm1, Nz, G);
        lines_dot2<NM>(line + QX2 + VY, sPz, VZ, G, Nz, nullptr);
    } else {
        line[QX2 + VY] = 1.0f;
    }
}

template <int NM, typename GD>
__device__ __forceinline__ void factor_line_df(const GD& g, double n, double ux, double uy, double uz, double T,
                                               double itau, const float4* sPx, const float4* sPy, const float4* sPz,
                                               const float2* sRec, float* line) {
    NodeDF in;
    if (itau != 0.0) node_inputs_df(n, ux, uy, uz, T, g.Nx, in);
    factor_line_df_in<NM>(g, in, itau, sPx, sPy, sPz, sRec, line);
}

// s + e = a + b exactly (TwoSum), whatever the magnitudes.
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return make_float2(s, (a - (s - bb)) + (b - bb));
}

// 1/x in double-float: the FP32 reciprocal refined by one Newton step
// (r + r (1 - x r), the residual formed exactly enough in double-float).
__device__ __forceinline__ float2 df_recip(float2 x) {
    const float r = 1.0f / x.x;
    const float2 res = df_add(make_float2(1.0f, 0.0f), df_mul(make_float2(-x.x, -x.y), make_float2(r, 0.0f)));
    return df_add(make_float2(r, 0.0f), df_mul(make_float2(r, 0.0f), res));
}

// sqrt(x) in double-float (x > 0): the FP32 root s refined by one Newton step
// s + (x - s^2) / (2 s), with s^2 by TwoProduct.
__device__ __forceinline__ float2 df_sqrt(float2 x) {
    const float s = sqrtf(x.x);
    const float p = s * s, e = fmaf(s, s, -p);
    const float2 res = df_add(x, make_float2(-p, -e));
    return df_fast_two_sum(s, res.x / (2.0f * s));
}

// The per-node inputs of the recurrences (NodeDF) from the compensated FP32
// moment sums (running sum and error term of n, j_x, j_y, j_z, E at sm[0..4]
// and sm[8..12]) entirely in double-float: n = s + c, u = j / n, T = (E - n
// |u|^2) / (D n), sqrt(T) and 1/sqrt(T) by Newton steps, and exp, erf as in
// node_inputs_df (FP64 where |u_x| / sqrt(2T) > 2.5).  For equilibrium orders
// up to 10: the relative error, about 1e-14, grows threefold per order in the
// recurrence and stays below FP32 resolution there.  Returns n (FP64) for 1/tau.
__device__ inline double node_inputs_from_sums_df(const float* sm, int D, NodeDF& o) {
    const float2 n = df_two_sum(sm[0], sm[8]);
    const float2 in = df_recip(n);
    const float2 ux = df_mul(df_two_sum(sm[1], sm[9]), in), uy = df_mul(df_two_sum(sm[2], sm[10]), in),
                 uz = df_mul(df_two_sum(sm[3], sm[11]), in);
    const float2 u2 = df_add(df_add(df_mul(ux, ux), df_mul(uy, uy)), df_mul(uz, uz));
    const float2 E = df_two_sum(sm[4], sm[12]);
    float2 T = df_mul(df_add(E, df_mul(make_float2(-n.x, -n.y), u2)), in);
    if (D == 3) T = df_mul(T, make_float2(0.3333333432674408f, -9.934107758624577e-09f));   // 1/3
    else if (D == 2) T = make_float2(0.5f * T.x, 0.5f * T.y);
    o.n = n;
    o.ux = ux;
    o.uy = uy;
    o.uz = uz;
    o.T = T;
    o.Tm1 = df_add(T, make_float2(-1.0f, 0.0f));
    const float2 irt = df_recip(df_sqrt(T));
    const float2 z = df_mul(ux, df_mul(irt, make_float2(0.7071067690849304f, 1.2101617485882343e-08f)));
    const float2 inv_sqrt2pi = make_float2(0.3989422917366028f, -1.1335170135851058e-08f);
    if (fabsf(z.x) <= 2.5f) {
        const float2 z2 = df_mul(z, z);
        const float2 Ez = df_exp_nonpos(make_float2(-z2.x, -z2.y));
        o.erf_z = df_erf_series(z, z2, Ez);
        o.g0 = df_mul(df_mul(Ez, inv_sqrt2pi), irt);
    } else {
        const double zd = (double)z.x + (double)z.y;
        o.erf_z = df_from_double(erf(zd));
        o.g0 = df_mul(df_mul(df_from_double(exp(-zd * zd)), inv_sqrt2pi), irt);
    }
    return (double)n.x + (double)n.y;
}

}  // namespace hlb
