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
__device__ __forceinline__ void factor_line_df(const GD& g, double n, double ux, double uy, double uz, double T,
                                               double itau, const float4* sPx, const float4* sPy, const float4* sPz,
                                               const float2* sRec, float* line) {
    const int Nx = g.Nx, Ny = g.Ny, Nz = g.Nz, Qx = g.Qx, QX2 = g.QX2, VY = g.VY, VZ = g.VZ, ncp = g.ncp;
    for (int o = QX2 + VY + VZ; o < ncp; ++o) line[o] = 0.0f;
    line[QX2 + VY + VZ] = (float)itau;
    if (itau == 0.0) {
        for (int o = 0; o < QX2 + VY + VZ; ++o) line[o] = 0.0f;
        return;
    }
    NodeDF in;
    node_inputs_df(n, ux, uy, uz, T, Nx, in);
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

}  // namespace hlb
