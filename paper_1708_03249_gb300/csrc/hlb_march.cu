// The RK-3 stage as two kernels (sm_103a):
//
// node_kernel   one warp per node: moments of the stage input (Eq. "eq:fmoms"),
//               then the per-node equilibrium coefficients in FP64 (App. A;
//               half-range recurrence in the orthonormal basis, full-range
//               Hermite recurrence), written as a factor line
//               coef[node] = { n g_x (2Qx), g_y (Qy), g_z (Qz), 1/tau }.
//
// march_kernel  one CTA per (instance, kz slab, strip of TY rows, x-segment);
//               one thread per velocity of the slab (all 2Qx x Qy velocities of
//               one p_z, so both K contractions stay inside the CTA).  Each
//               thread marches along x holding a 6-cell register window of its
//               velocity per row, so every x-face flux (WENO-5 / upwind2) is
//               evaluated once and carried to the next cell; the window
//               rotation is unrolled six ways so that no register moves.  Per
//               x-step the centre values and the node's factor line are staged
//               in double-buffered shared memory behind one barrier, then the
//               force term sum_a a_a (K_a f) (Eqs. "eq:hh_Kk_hh", "eq:H_Kk";
//               K rows in registers), BGK, the y-faces (periodic) and the RK-3
//               combination (Eq. "eq:rk3") finish the node.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "hlb_device.cuh"
#include "hlb_internal.h"

namespace hlb {
namespace {

// ---------------------------------------------------------------------------
// node kernel
// ---------------------------------------------------------------------------
// Per-node equilibrium factors, in two passes with no block-wide barrier:
//   sums_kernel   streams the stage input once (one warp per node) and writes
//                 the five quadrature sums n, j_x, j_y, j_z, E per node;
//   coef_kernel   one warp per 32 nodes, one lane per node: n, u, T, then the
//                 coefficient recurrences of all four roles, then the factor
//                 line (dot products shared across the warp).
// FP64 runs at 1/64 of FP32 here and a warp instruction costs the same
// whatever its mask, so every FP64 instruction runs on full warps; FP32
// groups with Nx <= 15 run the recurrences and dot products in double-float
// (FP64 only for erf, exp, sqrt, once per node).
template <typename R>
__global__ void __launch_bounds__(256) sums_kernel(const GroupDev g, const R* __restrict__ fs, R* __restrict__ sums) {
    extern __shared__ __align__(16) double ssm[];
    using R4 = typename std::conditional<sizeof(R) == 4, float4, double4>::type;
    const int QX2 = g.QX2, VY = g.VY, VZ = g.VZ, V = g.V;
    const int tid = threadIdx.x, bs = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = bs >> 5;
    R4* sM = reinterpret_cast<R4*>(ssm);                 // [V]: p_x, p_y, p_z, |p|^2
    R4* sYZ = sM + V;                                    // [VY * VZ]: p_y, p_z, p_y^2 + p_z^2
    const R* px = static_cast<const R*>(g.p);
    const R* py = px + QX2;
    const R* pz = py + VY;
    for (int v = tid; v < V; v += bs) {
        const int ix = v % QX2, jy = (v / QX2) % VY, kz = v / (QX2 * VY);
        const R a = px[ix], b = py[jy], c = pz[kz];
        R4 m4;
        m4.x = a; m4.y = b; m4.z = c; m4.w = a * a + b * b + c * c;
        sM[v] = m4;
    }
    for (int bq = tid; bq < VY * VZ; bq += bs) {
        const R b = py[bq % VY], c = pz[bq / VY];
        R4 y4;
        y4.x = b; y4.y = c; y4.z = b * b + c * c; y4.w = R(0);
        sYZ[bq] = y4;
    }
    __syncthreads();
    // 4-vector loads need 4 | 2Qx and 2Qx | 128 (2Qx a power of two up to 128):
    // then 4 consecutive velocities share (jy, kz) and a lane's p_x never change
    const bool vec4 = (QX2 & 3) == 0 && (QX2 & (QX2 - 1)) == 0 && QX2 <= 128;
    for (int node = blockIdx.x * nw + warp; node < g.nnodes; node += gridDim.x * nw) {
        const int ii = g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0;
        const InstDev& I = g.inst[ii];
        const R* f = fs + (size_t)I.f_off + (size_t)(node - I.node_off) * V;
        R a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
        if (vec4) {
            const R4* f4 = reinterpret_cast<const R4*>(f);
            const int x0 = (4 * lane) % QX2;
            const R pxa = sM[x0].x, pxb = sM[x0 + 1].x, pxc = sM[x0 + 2].x, pxd = sM[x0 + 3].x;
#pragma unroll 4
            for (int q = lane; q < (V >> 2); q += 32) {
                const R4 x = f4[q];
                const R4 yz = sYZ[(q << 2) / QX2];
                const R s = (x.x + x.y) + (x.z + x.w);
                a0 += s;
                a1 += pxa * x.x + pxb * x.y + pxc * x.z + pxd * x.w;
                a2 += yz.x * s;
                a3 += yz.y * s;
                a4 += pxa * pxa * x.x + pxb * pxb * x.y + pxc * pxc * x.z + pxd * pxd * x.w + yz.z * s;
            }
        } else {
            for (int v = lane; v < V; v += 32) {
                const R val = f[v];
                const R4 mw = sM[v];
                a0 += val;
                a1 += mw.x * val;
                a2 += mw.y * val;
                a3 += mw.z * val;
                a4 += mw.w * val;
            }
        }
        a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2); a3 = warp_sum(a3); a4 = warp_sum(a4);
        if (lane == 0) {
            R* o = sums + (size_t)node * 8;
            o[0] = a0; o[1] = a1; o[2] = a2; o[3] = a3; o[4] = a4;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(32) coef_kernel(const GroupDev g, const R* __restrict__ sums) {
    extern __shared__ __align__(16) double csm[];
    const int Nx = g.Nx, Ny = g.Ny, Nz = g.Nz;
    const int nrec = 5 * Nx + 1;
    const int nT = g.Qx * (Nx + 1) + g.VY * (Ny + 1) + g.VZ * (Nz + 1);
    const int ncoef = 2 * (Nx + 1) + (Ny + 1) + (Nz + 1);
    const int QX2 = g.QX2, VY = g.VY, VZ = g.VZ;
    const int tid = threadIdx.x, bs = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = bs >> 5;
    const bool df = g.use_df != 0;
    double* sRec = csm;
    double* sT = sRec + nrec;
    double* sW = sT + nT;                                // per warp: [32][ncoef] coefficients + [32] state
    const int per_warp = 32 * ncoef + 32 * 2 + 32 * (int)(sizeof(NodeDF) / 8);
    double* sG = sW + warp * per_warp;
    double* sNT = sG + 32 * ncoef;                       // [32][2]: n, 1/tau
    NodeDF* sIn = reinterpret_cast<NodeDF*>(sNT + 64);   // [32]
    float2* sRecF = reinterpret_cast<float2*>(sRec);
    float2* sTF = reinterpret_cast<float2*>(sT);
    float2* sGF = reinterpret_cast<float2*>(sG);
    if (df) {
        for (int i = tid; i < nrec; i += bs) sRecF[i] = g.recf[i];
        for (int i = tid; i < nT; i += bs) sTF[i] = g.Tf[i];
    } else {
        for (int i = tid; i < nrec; i += bs) sRec[i] = g.rec[i];
        for (int i = tid; i < nT; i += bs) sT[i] = g.Td[i];
    }
    __syncthreads();
    const double* sTx = sT;
    const double* sTy = sTx + g.Qx * (Nx + 1);
    const double* sTz = sTy + VY * (Ny + 1);
    const float2* sTxF = sTF;
    const float2* sTyF = sTxF + g.Qx * (Nx + 1);
    const float2* sTzF = sTyF + VY * (Ny + 1);
    R* coef = static_cast<R*>(g.coef);
    const int nf = QX2 + VY + VZ;
    const int nbatches = (g.nnodes + 31) / 32;
    for (int bt = blockIdx.x * nw + warp; bt < nbatches; bt += gridDim.x * nw) {
        const int base = bt * 32;
        const int nb = min(32, g.nnodes - base);
        // 1. lane = node: n, u, T, 1/tau; the recurrences' FP64 inputs
        bool active = false;
        if (lane < nb) {
            const int node = base + lane;
            const int ii = g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0;
            const double inv_Kn = g.inst[ii].inv_Kn;
            const R* sm = sums + (size_t)node * 8;
            active = inv_Kn != 0.0;
            double ux, uy, uz, T, n;
            if (df) {
                const float nf32 = (float)sm[0];
                const float fx = (float)sm[1] / nf32, fy = (float)sm[2] / nf32, fz = (float)sm[3] / nf32;
                const float fT = ((float)sm[4] - nf32 * (fx * fx + fy * fy + fz * fz)) / (g.D * nf32);
                n = nf32; ux = fx; uy = fy; uz = fz; T = fT;
            } else {
                n = (double)sm[0];
                ux = (double)sm[1] / n; uy = (double)sm[2] / n; uz = (double)sm[3] / n;
                T = ((double)sm[4] - n * (ux * ux + uy * uy + uz * uz)) / (g.D * n);
            }
            sNT[2 * lane] = n;
            sNT[2 * lane + 1] = n * inv_Kn;
            if (active) {
                if (df) {
                    node_inputs_df(n, ux, uy, uz, T, sIn[lane]);
                    for (int role = 0; role < 4; ++role)
                        node_coefficients_df(g, role, sIn[lane], sRecF, sGF + lane * ncoef);
                } else {
                    for (int role = 0; role < 4; ++role)
                        node_coefficients(g, role, ux, uy, uz, T, sRec, sG + lane * ncoef);
                }
            }
        }
        __syncwarp();
        // 2. factor lines: lanes over (node, output), one loop per output kind
        //    so that the lanes of a warp follow the same path
        for (int t = lane; t < nb * QX2; t += 32) {          // n g_x
            const int k = t / QX2, o = t - k * QX2;
            R* line = coef + (size_t)(base + k) * g.ncp;
            if (sNT[2 * k + 1] == 0.0) { line[o] = R(0); continue; }
            const int kk = o % g.Qx, sg = o / g.Qx;
            if (df) {
                const float2* Gs = sGF + k * ncoef + sg * (Nx + 1);
                const float2* Tr = sTxF + kk * (Nx + 1);
                float2 acc = df_mul(Tr[0], Gs[0]);
                for (int l = 1; l <= Nx; ++l) acc = df_add(acc, df_mul(Tr[l], Gs[l]));
                acc = df_mul(acc, sIn[k].n);
                line[o] = (R)(acc.x + acc.y);
            } else {
                const double* Gs = sG + k * ncoef + sg * (Nx + 1);
                const double* Tr = sTx + kk * (Nx + 1);
                double acc = 0.0;
                for (int l = 0; l <= Nx; ++l) acc += Tr[l] * Gs[l];
                line[o] = (R)(acc * sNT[2 * k]);
            }
        }
        for (int t = lane; t < nb * VY; t += 32) {           // g_y
            const int k = t / VY, j = t - k * VY;
            R* line = coef + (size_t)(base + k) * g.ncp + QX2;
            if (sNT[2 * k + 1] == 0.0) { line[j] = R(0); continue; }
            if (!g.Qy) { line[j] = R(1); continue; }
            if (df) {
                const float2* Gy = sGF + k * ncoef + 2 * (Nx + 1);
                const float2* Tr = sTyF + j * (Ny + 1);
                float2 acc = df_mul(Tr[0], Gy[0]);
                for (int l = 1; l <= Ny; ++l) acc = df_add(acc, df_mul(Tr[l], Gy[l]));
                line[j] = (R)(acc.x + acc.y);
            } else {
                const double* Gy = sG + k * ncoef + 2 * (Nx + 1);
                const double* Tr = sTy + j * (Ny + 1);
                double acc = 0.0;
                for (int l = 0; l <= Ny; ++l) acc += Tr[l] * Gy[l];
                line[j] = (R)acc;
            }
        }
        for (int t = lane; t < nb * VZ; t += 32) {           // g_z
            const int k = t / VZ, j = t - k * VZ;
            R* line = coef + (size_t)(base + k) * g.ncp + QX2 + VY;
            if (sNT[2 * k + 1] == 0.0) { line[j] = R(0); continue; }
            if (!g.Qz) { line[j] = R(1); continue; }
            if (df) {
                const float2* Gz = sGF + k * ncoef + 2 * (Nx + 1) + (Ny + 1);
                const float2* Tr = sTzF + j * (Nz + 1);
                float2 acc = df_mul(Tr[0], Gz[0]);
                for (int l = 1; l <= Nz; ++l) acc = df_add(acc, df_mul(Tr[l], Gz[l]));
                line[j] = (R)(acc.x + acc.y);
            } else {
                const double* Gz = sG + k * ncoef + 2 * (Nx + 1) + (Ny + 1);
                const double* Tr = sTz + j * (Nz + 1);
                double acc = 0.0;
                for (int l = 0; l <= Nz; ++l) acc += Tr[l] * Gz[l];
                line[j] = (R)acc;
            }
        }
        if (lane < nb) coef[(size_t)(base + lane) * g.ncp + nf] = (R)sNT[2 * lane + 1];   // 1/tau
        __syncwarp();
    }
}

// FP32 groups whose equilibrium orders are all below NM (double-float path, orders up to 15):
// one thread per node, coefficients in registers.  The FP64 prelude (erf,
// exp, sqrt) runs once per node on full warps; each role's recurrence is
// followed at once by its dot products with the quadrature tables (broadcast
// reads from shared memory); a warp's 32 factor lines are assembled in shared
// memory and written out contiguously.
template <int NM>
__device__ __forceinline__ void half_range_G_df(int r, const NodeDF& in, const float2* recf, int Nx, float2 (&G)[NM]) {
    const float2* ra = recf;
    const float2* rb = recf + Nx;
    const float2* rc = recf + 2 * Nx;
    const float2* h0 = recf + 3 * Nx;
    const float2* inv_ra = recf + 4 * Nx + 1;
    const float sg = r ? -1.0f : 1.0f;
    const float2 us = make_float2(sg * in.ux.x, sg * in.ux.y);
    const float2 half = df_add(make_float2(0.5f, 0.0f), make_float2(0.5f * sg * in.erf_z.x, 0.5f * sg * in.erf_z.y));
    G[0] = df_mul(h0[0], half);
    const float2 m_om0 = make_float2(-3.989422917e-01f, 1.133517014e-08f);   // -1/sqrt(2 pi)
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

template <int NM>
__device__ __forceinline__ float2 dot_df(const float2* Trow, const float2 (&G)[NM], int N) {
    float2 acc = df_mul(Trow[0], G[0]);
#pragma unroll
    for (int l = 1; l < NM; ++l)
        if (l <= N) acc = df_add(acc, df_mul(Trow[l], G[l]));
    return acc;
}

template <int NM>
__global__ void __launch_bounds__(128) coef_df_kernel(const GroupDev g, const float* __restrict__ sums) {
    extern __shared__ __align__(16) float2 cdf[];
    const int Nx = g.Nx, Ny = g.Ny, Nz = g.Nz, Qx = g.Qx, QX2 = g.QX2, VY = g.VY, VZ = g.VZ, ncp = g.ncp;
    const int nrec = 5 * Nx + 1;
    const int nT = Qx * (Nx + 1) + VY * (Ny + 1) + VZ * (Nz + 1);
    float2* sRec = cdf;
    float2* sT = sRec + nrec;
    float* sLine = reinterpret_cast<float*>(cdf + ((nrec + nT + 1) & ~1)) + (threadIdx.x >> 5) * 32 * ncp;   // [32][ncp] per warp
    for (int i = threadIdx.x; i < nrec; i += blockDim.x) sRec[i] = g.recf[i];
    for (int i = threadIdx.x; i < nT; i += blockDim.x) sT[i] = g.Tf[i];
    __syncthreads();
    const float2* sTx = sT;
    const float2* sTy = sTx + Qx * (Nx + 1);
    const float2* sTz = sTy + VY * (Ny + 1);
    const int lane = threadIdx.x & 31;
    const int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    const int node = base + lane;
    float* line = sLine + lane * ncp;
    if (node < g.nnodes) {
        const int ii = g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0;
        const double inv_Kn = g.inst[ii].inv_Kn;
        const float* sm = sums + (size_t)node * 8;
        const float n = sm[0];
        const float ux = sm[1] / n, uy = sm[2] / n, uz = sm[3] / n;
        const float T = (sm[4] - n * (ux * ux + uy * uy + uz * uz)) / (g.D * n);
        const double itau = (double)n * inv_Kn;
        for (int o = QX2 + VY + VZ; o < ncp; ++o) line[o] = 0.0f;
        line[QX2 + VY + VZ] = (float)itau;
        if (itau == 0.0) {
            for (int o = 0; o < QX2 + VY + VZ; ++o) line[o] = 0.0f;
        } else {
            NodeDF in;
            node_inputs_df(n, ux, uy, uz, T, in);
            float2 G[NM];
#pragma unroll 1
            for (int r = 0; r < 2; ++r) {                    // n g_x, p_x > 0 then p_x < 0
                half_range_G_df<NM>(r, in, sRec, Nx, G);
                for (int kk = 0; kk < Qx; ++kk) {
                    const float2 v = df_mul(dot_df<NM>(sTx + kk * (Nx + 1), G, Nx), in.n);
                    line[r * Qx + kk] = v.x + v.y;
                }
            }
            if (g.Qy) {
                full_range_G_df<NM>(in.uy, in.Tm1, Ny, G);
                for (int j = 0; j < VY; ++j) {
                    const float2 v = dot_df<NM>(sTy + j * (Ny + 1), G, Ny);
                    line[QX2 + j] = v.x + v.y;
                }
            } else {
                line[QX2] = 1.0f;
            }
            if (g.Qz) {
                full_range_G_df<NM>(in.uz, in.Tm1, Nz, G);
                for (int j = 0; j < VZ; ++j) {
                    const float2 v = dot_df<NM>(sTz + j * (Nz + 1), G, Nz);
                    line[QX2 + VY + j] = v.x + v.y;
                }
            } else {
                line[QX2 + VY] = 1.0f;
            }
        }
    }
    __syncwarp();
    // the warp's lines are contiguous in the factor-line buffer
    const int nb = min(32, g.nnodes - base);
    if (nb > 0) {
        float4* dst = reinterpret_cast<float4*>(static_cast<float*>(g.coef) + (size_t)base * ncp);
        const float4* src = reinterpret_cast<const float4*>(sLine);
        for (int i = lane; i < nb * ncp / 4; i += 32) dst[i] = src[i];
    }
}

// ---------------------------------------------------------------------------
// march kernel
// ---------------------------------------------------------------------------
// Flux per unit velocity at the face between cells c2 and c3 of the window
// c0..c5 (x-2 .. x+3): the upwind stencil is c0..c4 for v > 0 and c5..c1 for
// v < 0 (Sec. IV.C.2, mirrored for negative velocities).
template <typename R, int ADV>
__device__ __forceinline__ R face_value(bool pos, R sv, R c0, R c1, R c2, R c3, R c4, R c5) {
    if (ADV == HLB_WENO5_) {
        const R a = pos ? c0 : c5, b = pos ? c1 : c4, c = pos ? c2 : c3, d = pos ? c3 : c2,
                e = pos ? c4 : c1;
        return weno5_face_sv(a, b, c, d, e, sv);
    } else {
        const R b = pos ? c1 : c4, c = pos ? c2 : c3;
        return upwind2_face(b, c);
    }
}

// One x-step's inputs, filled by bulk copies: the head cell x+3 of each strip
// row, cell x of the six y-halo rows (2D), f^n at cell x (stages 2 and 3) and
// the factor lines of the strip's nodes at x.
template <typename R, int QX2, int VY, int TY>
struct StepBuf {
    static constexpr int S = QX2 * VY;
    static constexpr int NH = TY > 1 ? 6 : 1;
    static constexpr int NCPMAX = (QX2 + VY + 32 + 1 + 3) / 4 * 4;
    R head[TY][S];
    R halo[NH][S];
    R fnr[TY][S];
    R coef[TY][NCPMAX];
};

constexpr int kDepth = 4;    // x-steps in flight

template <typename R, int QX2, int VY, int TY>
constexpr size_t march_smem_bytes() {
    return kDepth * sizeof(StepBuf<R, QX2, VY, TY>) + 2 * TY * QX2 * VY * sizeof(R) + kDepth * 8 + 16;   // + abort flag
}

// The marching kernel.  Offsets inside an instance are 32-bit (the host
// only takes this path when an instance holds fewer than 2^31 values).
template <typename R, int ADV, int QX2, int VY, int TY>
__global__ void __launch_bounds__(QX2 * VY, (QX2 * VY <= 32 ? 16 : (QX2 * VY <= 128 ? 4 : 1)))
march_kernel(const GroupDev g, const Work* __restrict__ works, const R* __restrict__ fs,
             const R* __restrict__ fn, R* __restrict__ fo, int stage) {
    constexpr int S = QX2 * VY;
    constexpr int QX = QX2 / 2;
    using Buf = StepBuf<R, QX2, VY, TY>;
    extern __shared__ __align__(128) unsigned char msm[];
    Buf* buf = reinterpret_cast<Buf*>(msm);
    R* sF = reinterpret_cast<R*>(msm + kDepth * sizeof(Buf));              // [2][TY][S]
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(sF + 2 * TY * S);
    int* sAbort = reinterpret_cast<int*>(bars + kDepth);

    const Work W = works[blockIdx.x];
    const InstDev& I = g.inst[W.inst];
    const int t = threadIdx.x;
    const int ix = t % QX2, jy = t / QX2, kz = W.kz;
    const int V = g.V, nx = I.nx, ny = I.ny, ncp = g.ncp;
    const int v = (kz * VY + jy) * QX2 + ix;
    const R* P = static_cast<const R*>(g.p);
    const R vx = P[ix], vy = P[QX2 + jy];
    const bool xpos = ix < QX, ypos = vy > R(0);
    const R sv = static_cast<const R*>(g.wscale)[v];
    const R* K = static_cast<const R*>(g.K);
    R kx[QX2], ky[VY];
#pragma unroll
    for (int i = 0; i < QX2; ++i) kx[i] = K[ix * QX2 + i];
#pragma unroll
    for (int j = 0; j < VY; ++j) ky[j] = K[QX2 * QX2 + jy * VY + j];
    const R ax = (R)I.ax, ay = (R)I.ay, dt = (R)I.dt, inv_dy = (R)I.inv_dy;
    const R* invdx = static_cast<const R*>(g.inv_dx) + I.dx_off;
    const int rs = nx * V;
    const R* fsI = fs + I.f_off;                 // instance base (slab offset added per copy)
    const R* fnI = fn + I.f_off;
    const R* fsv = fsI + v;
    R* fov = fo + I.f_off + v;
    const R* cI = static_cast<const R*>(g.coef) + (size_t)I.node_off * ncp;
    const int csrc_z = QX2 + VY + kz, csrc_t = QX2 + VY + g.VZ;
    const R* gw = static_cast<const R*>(g.gw) + I.gw_off;
    const R gwl = gw[v], gwr = gw[V + v];
    int roff[TY], crow[TY];
    bool valid[TY];
    R nwl_g[TY], nwr_g[TY];
#pragma unroll
    for (int r = 0; r < TY; ++r) {
        const int y = W.y0 + r;
        valid[r] = y < ny;
        const int yy = y % ny;
        roff[r] = yy * rs;
        crow[r] = yy * nx;
        nwl_g[r] = (R)g.nw[(size_t)(I.row_off + yy) * 2 + 0] * gwl;
        nwr_g[r] = (R)g.nw[(size_t)(I.row_off + yy) * 2 + 1] * gwr;
    }
    const int xa = W.xa, xb = W.xb;
    const int slab = kz * S;

    // producer (thread 0): the copies of step xs into buffer (xs - xa) % kDepth
    auto issue = [&](int xs) {
        if (xs >= xb) return;
        if (g.inject_stall && xs == xa + 1) return;     // bounded-wait test: this step's copies never come
        Buf& B = buf[(xs - xa) % kDepth];
        unsigned long long* bar = &bars[(xs - xa) % kDepth];
        const uint32_t row_bytes = S * sizeof(R);
        uint32_t bytes = TY * ncp * sizeof(R);
        if (xs + 3 < nx) bytes += TY * row_bytes;
        if (TY > 1) bytes += 6 * row_bytes;
        if (stage > 0) bytes += TY * row_bytes;
        fence_proxy_async_smem();
        mbar_expect_tx(bar, bytes);
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            if (xs + 3 < nx) bulk_g2s(B.head[r], fsI + roff[r] + (xs + 3) * V + slab, row_bytes, bar);
            if (stage > 0) bulk_g2s(B.fnr[r], fnI + roff[r] + xs * V + slab, row_bytes, bar);
            bulk_g2s(B.coef[r], cI + (crow[r] + xs) * ncp, ncp * sizeof(R), bar);
        }
        if (TY > 1) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int ylo = ((W.y0 - 3 + k) % ny + ny) % ny;
                const int yhi = (W.y0 + TY + k) % ny;
                bulk_g2s(B.halo[k], fsI + ylo * rs + xs * V + slab, row_bytes, bar);
                bulk_g2s(B.halo[3 + k], fsI + yhi * rs + xs * V + slab, row_bytes, bar);
            }
        }
    };

    if (t == 0) {
        for (int d = 0; d < kDepth; ++d) mbar_init(&bars[d], 1);
        *sAbort = 0;
        mbar_init_fence();
    }
    __syncthreads();
    if (t == 0)
        for (int xs = xa; xs < xa + kDepth - 1; ++xs) issue(xs);

    // window of cells xa-3 .. xa+2 (walls: ghosts of Sec. IV.C.3) and the face xa-1/2
    R w[TY][6], Fm[TY];
#pragma unroll
    for (int r = 0; r < TY; ++r) {
        const R* f = fsv + roff[r];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const int x = xa - 3 + j;
            R val;
            if (x >= 0 && x < nx) val = f[x * V];
            else if (x < 0) {
                if (xpos) val = nwl_g[r];
                else if (x < -2) val = R(0);          // never read by a negative velocity
                else {
                    const R f0 = f[0], f1 = f[V], f2 = f[2 * V];
                    val = x == -1 ? R(3) * f0 - R(3) * f1 + f2 : R(6) * f0 - R(8) * f1 + R(3) * f2;
                }
            } else if (!xpos) val = nwr_g[r];
            else if (x > nx + 1) val = R(0);          // never read by a positive velocity
            else {
                const R f0 = f[(nx - 1) * V], f1 = f[(nx - 2) * V], f2 = f[(nx - 3) * V];
                val = x == nx ? R(3) * f0 - R(3) * f1 + f2 : R(6) * f0 - R(8) * f1 + R(3) * f2;
            }
            w[r][j] = val;
        }
        Fm[r] = vx * face_value<R, ADV>(xpos, sv, w[r][0], w[r][1], w[r][2], w[r][3], w[r][4], w[r][5]);
    }

    int xab = xa;
#pragma unroll 1
    for (int x = xa; x < xb; ++x) {
        const int step = x - xa;
        const Buf& B = buf[step % kDepth];
        if (!mbar_wait(&bars[step % kDepth], (step / kDepth) & 1, g.err, g.wait_ns)) *sAbort = 1;
        xab = x;
        const int b = x & 1;
        R fc[TY];
#pragma unroll
        for (int r = 0; r < TY; ++r) {
#pragma unroll
            for (int j = 0; j < 5; ++j) w[r][j] = w[r][j + 1];
            const int h = x + 3;
            R hv;
            if (h < nx) hv = B.head[r][t];
            else if (!xpos) hv = nwr_g[r];                          // emitted at the right wall
            else if (h == nx) hv = R(3) * w[r][4] - R(3) * w[r][3] + w[r][2];
            else if (h == nx + 1) hv = R(6) * w[r][3] - R(8) * w[r][2] + R(3) * w[r][1];
            else hv = R(0);                                       // never read by v > 0
            w[r][5] = hv;
            fc[r] = w[r][2];
            sF[(b * TY + r) * S + t] = fc[r];
        }
        // x faces: x+1/2 from the window, x-1/2 carried from the previous cell
        R divx[TY];
        const R idx = invdx[x];
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            const R Fp = vx * face_value<R, ADV>(xpos, sv, w[r][0], w[r][1], w[r][2], w[r][3], w[r][4], w[r][5]);
            divx[r] = (Fp - Fm[r]) * idx;
            Fm[r] = Fp;
        }
        // y faces (periodic) from column x of rows y0-3 .. y0+TY+2
        R divy[TY];
#pragma unroll
        for (int r = 0; r < TY; ++r) divy[r] = R(0);
        if (TY > 1) {
            R col[TY + 6];
#pragma unroll
            for (int k = 0; k < 3; ++k) col[k] = B.halo[k][t];
#pragma unroll
            for (int r = 0; r < TY; ++r) col[3 + r] = fc[r];
#pragma unroll
            for (int k = 0; k < 3; ++k) col[TY + 3 + k] = B.halo[3 + k][t];
            R Gf[TY + 1];
#pragma unroll
            for (int i = 0; i <= TY; ++i)      // face between col[i+2] and col[i+3]
                Gf[i] = vy * face_value<R, ADV>(ypos, sv, col[i], col[i + 1], col[i + 2], col[i + 3],
                                                col[i + 4], col[i + 5]);
#pragma unroll
            for (int r = 0; r < TY; ++r) divy[r] = (Gf[r + 1] - Gf[r]) * inv_dy;
        }
        __syncthreads();
        if (*sAbort) break;
        if (t == 0) issue(x + kDepth - 1);
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            const R* fr = sF + (b * TY + r) * S;
            const R* fxr = fr + jy * QX2;
            R kxf = R(0), kyf = R(0);
#pragma unroll
            for (int i = 0; i < QX2; ++i) kxf += kx[i] * fxr[i];
            if (VY > 1) {
#pragma unroll
                for (int j = 0; j < VY; ++j) kyf += ky[j] * fr[j * QX2 + ix];
            }
            const R* cr = B.coef[r];
            const R feq = cr[ix] * cr[QX2 + jy] * cr[csrc_z];
            const R itau = cr[csrc_t];
            const R L = -divx[r] - divy[r] - (ax * kxf + ay * kyf) - (fc[r] - feq) * itau;
            R out;
            if (stage == 0) {
                out = fc[r] + dt * L;
            } else {
                const R fo_n = B.fnr[r][t];
                out = stage == 1 ? R(0.75) * fo_n + R(0.25) * fc[r] + R(0.25) * dt * L
                                 : fo_n * R(1.0 / 3.0) + R(2.0 / 3.0) * fc[r] + R(2.0 / 3.0) * dt * L;
            }
            if (valid[r]) fov[roff[r] + x * V] = out;
        }
    }
    if (*sAbort && t == 0) {
        // a wait ran out at step xab: let the copies issued since land before the CTA exits
        for (int s2 = xab - xa; s2 < xb - xa && s2 < xab - xa + kDepth - 1; ++s2)
            mbar_drain(&bars[s2 % kDepth], (s2 / kDepth) & 1, g.wait_ns);
    }
}

// FP32 pair kernel: each iteration advances two strip rows by two cells.
// The x faces pack the two rows into the lanes of f32x2 registers, the y faces
// pack the two cells, so every WENO evaluation is a full f32x2 one.  The
// window holds values pre-multiplied by the population's inverse weight, so
// that every WENO evaluation reads scaled stencils directly.
template <int QX2, int VY>
struct PairBuf {
    static constexpr int S = QX2 * VY;
    static constexpr int NCPMAX = (QX2 + VY + 32 + 1 + 3) / 4 * 4;
    float head[2][2][S];        // [cell x0+3+i][row]
    float halo[2][6][S];        // [cell x0+i][halo row y0-3, y0-2, y0-1, y0+2, y0+3, y0+4]
    float fnr[2][2][S];         // [cell x0+i][row]: f^n (stages 2, 3)
    float coef[2][2 * NCPMAX];  // [row]: factor lines of cells x0, x0+1
};

#ifndef HLB_PAIR_DEPTH
#define HLB_PAIR_DEPTH 2
#endif
#ifndef HLB_PAIR_MIN_BLOCKS
#define HLB_PAIR_MIN_BLOCKS 7
#endif
constexpr int kPairDepth = HLB_PAIR_DEPTH;   // pairs of cells in flight (copy buffers)

// The force term by warp-level tensor-core products when both contractions
// tile into 16 x 8 x 8 blocks.
template <int QX2, int VY>
// HLB_PAIR_MMA=1 takes the force term to the tensor cores (mma.sync, three
// TF32 products); on the 1024 x 512 channel with 16 x 8 x 8 velocities it
// measured 4.27 ms per stage launch against 3.87 ms for the FP32 FMA loop
// (the fragment loads, splits and stores cost more issue slots than the
// packed FMAs they replace), so it is off by default.
#ifndef HLB_PAIR_MMA
#define HLB_PAIR_MMA 0
#endif
__host__ __device__ constexpr bool pair_uses_mma() { return HLB_PAIR_MMA && QX2 % 8 == 0 && VY % 8 == 0; }

// FMA path: a_x K_x and a_y K_y rows in shared memory, every entry duplicated
// into an f32x2 pair, rows padded by two pairs (a warp's eight rows fall in
// distinct banks).
template <int QX2, int VY>
__host__ __device__ constexpr int pair_kdup_pairs() { return QX2 * (QX2 + 2) + VY * (VY + 2); }

template <int QX2, int VY>
constexpr size_t pair_smem_bytes() {
    return kPairDepth * sizeof(PairBuf<QX2, VY>) + (pair_uses_mma<QX2, VY>() ? 4 : 2) * VY * (QX2 + 1) * sizeof(float4) +
           (pair_uses_mma<QX2, VY>() ? 0 : pair_kdup_pairs<QX2, VY>() * sizeof(float2)) + (kPairDepth + 3) * 8 + 16;
}

// D += A B on the tensor cores, TF32 operands, FP32 accumulation
// (m16n8k8; A row-major 16 x 8, B column-major 8 x 8).
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// x = hi + lo with hi a TF32 value (round to nearest); lo keeps the rest
// (its own low bits are dropped by the tensor core).
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    lo = __float_as_uint(x - __uint_as_float(hi));
}

// D += A B in three TF32 products (A_lo B_hi + A_hi B_lo + A_hi B_hi), close
// to an FP32 product; a[k] are FP32 values, b{0,1}{h,l} split fragments.
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const float (&a)[4], uint32_t b0h, uint32_t b0l,
                                           uint32_t b1h, uint32_t b1l) {
    uint32_t ah[4], al[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) split_tf32(a[k], ah[k], al[k]);
    mma_tf32(d, al[0], al[1], al[2], al[3], b0h, b1h);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], b0l, b1l);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], b0h, b1h);
}

template <int ADV, int QX2, int VY>
__global__ void __launch_bounds__(QX2 * VY, (QX2 * VY <= 32 ? 16 : (QX2 * VY <= 128 ? HLB_PAIR_MIN_BLOCKS : 1)))
march_pair_kernel(const GroupDev g, const Work* __restrict__ works, const float* __restrict__ fs,
                  const float* __restrict__ fn, float* __restrict__ fo, int stage) {
    constexpr int S = QX2 * VY;
    constexpr int QX = QX2 / 2;
    constexpr int SP = QX2 + 1;            // padded sF row: the K_x reads of a warp hit distinct banks
    using Buf = PairBuf<QX2, VY>;
    extern __shared__ __align__(128) unsigned char msm[];
    Buf* buf = reinterpret_cast<Buf*>(msm);
    constexpr bool kMMA = pair_uses_mma<QX2, VY>();
    float4* sF = reinterpret_cast<float4*>(msm + kPairDepth * sizeof(Buf));   // [2][VY][SP]: (r0 x0, r1 x0, r0 x1, r1 x1)
    float4* sKx = sF + 2 * VY * SP;                   // [VY][SP]: a_x K_x f, same layout (tensor-core path)
    float4* sKy = sKx + VY * SP;                      // [VY][SP]: a_y K_y f
    float2* sKd = reinterpret_cast<float2*>(sF + (kMMA ? 4 : 2) * VY * SP);    // FMA path: duplicated a K rows
    constexpr int KXR = QX2 + 2, KYR = VY + 2;        // padded row lengths (pairs)
    unsigned long long* bars =
        reinterpret_cast<unsigned long long*>(sKd + (kMMA ? 0 : pair_kdup_pairs<QX2, VY>()));   // bulk-copy pipeline
    unsigned long long* xch = bars + kPairDepth;       // [2]: sF[b] written by every warp
    unsigned long long* xch2 = xch + 2;                // sKx, sKy written by every warp
    int* sAbort = reinterpret_cast<int*>(xch2 + 1);

    const Work W = works[blockIdx.x];
    const InstDev& I = g.inst[W.inst];
    const int t = threadIdx.x;
    // Thread -> velocity: when a sign quadrant of (p_x, p_y) fills whole warps,
    // each warp takes one quadrant, so the stencil orientation is warp-uniform;
    // otherwise ix runs fastest.
    constexpr int QH = QX2 / 2, YH = VY >= 2 ? VY / 2 : 1;
    constexpr bool kQuad = VY >= 2 && (QH * YH) % 32 == 0;
    int ix, jy;
    if (kQuad) {
        const int q = t / (QH * YH), rr = t % (QH * YH);
        ix = (q >> 1) * QH + rr % QH;
        jy = (q & 1) * YH + rr / QH;
    } else {
        ix = t % QX2;
        jy = t / QX2;
    }
    const int kz = W.kz;
    const int vl = jy * QX2 + ix;                  // velocity within the slab
    const int V = g.V, nx = I.nx, ny = I.ny, ncp = g.ncp;
    const int v = kz * S + vl;
    const float* P = static_cast<const float*>(g.p);
    const float vx = P[ix], vy = P[QX2 + jy];
    const bool xpos = ix < QX, ypos = vy > 0.0f;
    const float sv = static_cast<const float*>(g.wscale)[v];
    const float isv = 1.0f / sv;
    const float* K = static_cast<const float*>(g.K);
    const int warp = t >> 5, lane = t & 31;
    // FMA path: this thread's rows of K_x and K_y.  Tensor-core path: warp w
    // computes one 16 x 8 tile of (a_x K_x f)^T and one of (a_y K_y f)^T, the
    // contractions written as F^T K^T with F^T rows (j_y, cell/row) resp.
    // (i_x, cell/row); the B fragments (a K)^T stay in registers, split hi/lo.

    constexpr int XS = QX2 / 8, YS = VY / 8;        // k-steps (tensor-core path)
    uint32_t bxh[kMMA ? XS : 1][2], bxl[kMMA ? XS : 1][2], byh[kMMA ? YS : 1][2], byl[kMMA ? YS : 1][2];
    const int mX = warp / (QX2 / 8 > 0 ? QX2 / 8 : 1), nX = warp % (QX2 / 8 > 0 ? QX2 / 8 : 1);
    const int mY = warp / (VY / 8 > 0 ? VY / 8 : 1), nY = warp % (VY / 8 > 0 ? VY / 8 : 1);
    const int gq = lane >> 2, tq = lane & 3;
    if constexpr (kMMA) {
        const float axf = (float)I.ax, ayf = (float)I.ay;
#pragma unroll
        for (int ks = 0; ks < XS; ++ks)
#pragma unroll
            for (int h = 0; h < 2; ++h)      // B[k][n] = a_x K_x[8 nX + n][8 ks + k]
                split_tf32(axf * K[(8 * nX + gq) * QX2 + 8 * ks + tq + 4 * h], bxh[ks][h], bxl[ks][h]);
#pragma unroll
        for (int ks = 0; ks < YS; ++ks)
#pragma unroll
            for (int h = 0; h < 2; ++h)      // B[k][n] = a_y K_y[8 nY + n][8 ks + k]
                split_tf32(ayf * K[QX2 * QX2 + (8 * nY + gq) * VY + 8 * ks + tq + 4 * h], byh[ks][h], byl[ks][h]);
    } else {
        const float axf = (float)I.ax, ayf = (float)I.ay;
        for (int e = t; e < QX2 * QX2; e += S) sKd[(e / QX2) * KXR + e % QX2] = f2(axf * K[e]);
        for (int e = t; e < VY * VY; e += S) sKd[QX2 * KXR + (e / VY) * KYR + e % VY] = f2(ayf * K[QX2 * QX2 + e]);
    }
    (void)bxh; (void)bxl; (void)byh; (void)byl; (void)mX; (void)nX; (void)mY; (void)nY;
    const float2 dt2 = f2((float)I.dt);
    const float2 vxs = f2(vx * isv), vys = f2(vy * isv * (float)I.inv_dy), isv2 = f2(isv), sv2 = f2(sv);
    const float* invdx = static_cast<const float*>(g.inv_dx) + I.dx_off;
    const int rs = nx * V;
    const float* fsI = fs + I.f_off;
    const float* fnI = fn + I.f_off;
    float* fov = fo + I.f_off + v;
    const float* cI = static_cast<const float*>(g.coef) + (size_t)I.node_off * ncp;
    const int csrc_z = QX2 + VY + kz, csrc_t = QX2 + VY + g.VZ;
    const float* gw = static_cast<const float*>(g.gw) + I.gw_off;
    const float gwl = gw[v] * sv, gwr = gw[V + v] * sv;
    int roff[2], crow[2];
    bool valid[2];
    float nwl_g[2], nwr_g[2];          // scaled emitted ghosts
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int y = W.y0 + r;
        valid[r] = y < ny;
        const int yy = y % ny;
        roff[r] = yy * rs;
        crow[r] = yy * nx;
        nwl_g[r] = (float)g.nw[(size_t)(I.row_off + yy) * 2 + 0] * gwl;
        nwr_g[r] = (float)g.nw[(size_t)(I.row_off + yy) * 2 + 1] * gwr;
    }
    const int xa = W.xa, xb = W.xb;
    const int npairs = (xb - xa + 1) >> 1;
    const int slab = kz * S;
    const uint32_t row_bytes = S * sizeof(float);

    // producer (warp 0, one copy per lane): the inputs of pair p into buffer p % kPairDepth
    // Copy `lane` of pair p (22 lanes: 12 halo rows, 4 head rows, 4 f^n rows,
    // 2 factor-line runs): source, bytes and destination in B; false if the
    // lane has none for this pair.
    auto copy_of = [&](int lane, int p, Buf& B, const float*& src, uint32_t& bytes, float*& dst) -> bool {
        const int x0 = xa + 2 * p;
        const int n2 = min(2, xb - x0);
        bytes = row_bytes;
        if (lane < 12) {                                   // halo rows of cells x0, x0+1
            const int i = lane / 6, k = lane % 6;
            const int yk = k < 3 ? ((W.y0 - 3 + k) % ny + ny) % ny : (W.y0 + k - 1) % ny;
            src = fsI + yk * rs + (x0 + i) * V + slab;
            dst = B.halo[i][k];
            return i < n2;
        } else if (lane < 16) {                            // head cells x0+3, x0+4
            const int i = (lane - 12) >> 1, r = lane & 1;
            src = fsI + roff[r] + (x0 + 3 + i) * V + slab;
            dst = B.head[i][r];
            return i < n2 && x0 + 3 + i < nx;
        } else if (lane < 20) {                            // f^n of cells x0, x0+1
            const int i = (lane - 16) >> 1, r = lane & 1;
            src = fnI + roff[r] + (x0 + i) * V + slab;
            dst = B.fnr[i][r];
            return stage > 0 && i < n2;
        } else if (lane < 22) {                            // factor lines
            const int r = lane - 20;
            src = cI + (size_t)(crow[r] + x0) * ncp;
            bytes = n2 * ncp * (uint32_t)sizeof(float);
            dst = B.coef[r];
            return true;
        }
        return false;
    };
    // The copies are spread over the warps so that no warp carries them all:
    // with four or more warps, warps 0 and 1 take the halo rows of cells x0
    // and x0+1, warp 2 the head rows and factor lines, warp 3 the f^n rows; a
    // single warp takes all 22.  Thread 0 registers each pair's byte count
    // (arrive.expect_tx) before any warp can issue that pair's copies.
    int my_copy = -1;
    if (S / 32 >= 4) {
        if (warp < 2 && lane < 6) my_copy = 6 * warp + lane;
        else if (warp == 2 && lane < 6) my_copy = lane < 4 ? 12 + lane : 16 + lane;    // 12..15, 20..21
        else if (warp == 3 && lane < 4) my_copy = 16 + lane;
    } else if (warp == 0 && lane < 22) {
        my_copy = lane;
    }
    auto expect = [&](int p) {                     // thread 0 only
        if (p >= npairs || (g.inject_stall && p == 1)) return;   // test hook: pair 1 never arrives
        const int x0 = xa + 2 * p;
        const int n2 = min(2, xb - x0);
        const int nhead = (x0 + 3 < nx) + (n2 > 1 && x0 + 4 < nx);
        uint32_t bytes = n2 * (6 * row_bytes + 2 * ncp * (uint32_t)sizeof(float)) + 2 * nhead * row_bytes;
        if (stage > 0) bytes += 2 * n2 * row_bytes;
        mbar_expect_tx(&bars[p % kPairDepth], bytes);
    };
    auto issue = [&](int p) {
        if (my_copy < 0 || p >= npairs || (g.inject_stall && p == 1)) return;
        Buf& B = buf[p % kPairDepth];
        const float* src;
        uint32_t bytes;
        float* dst;
        fence_proxy_async_smem();
        if (copy_of(my_copy, p, B, src, bytes, dst)) bulk_g2s(dst, src, bytes, &bars[p % kPairDepth]);
    };

    if (t == 0) {
        for (int d = 0; d < kPairDepth; ++d) mbar_init(&bars[d], 1);
        mbar_init(&xch[0], S / 32);
        mbar_init(&xch[1], S / 32);
        mbar_init(xch2, S / 32);
        *sAbort = 0;
        mbar_init_fence();
        for (int p = 0; p < kPairDepth - 1; ++p) expect(p);
    }
    __syncthreads();
    for (int p = 0; p < kPairDepth - 1; ++p) issue(p);

    // scaled window of cells xa-3 .. xa+4 (wall ghosts of Sec. IV.C.3); w[0..5] filled here
    float2 w[8];
    {
        float wr[2][6];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float* f = fsI + v + roff[r];
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                const int x = xa - 3 + j;
                float val;
                if (x >= 0 && x < nx) val = f[x * V] * sv;
                else if (x < 0) {
                    if (xpos) val = nwl_g[r];
                    else if (x < -2) val = 0.0f;          // never read by a negative velocity
                    else {
                        const float f0 = f[0] * sv, f1 = f[V] * sv, f2v = f[2 * V] * sv;
                        val = x == -1 ? 3.0f * f0 - 3.0f * f1 + f2v : 6.0f * f0 - 8.0f * f1 + 3.0f * f2v;
                    }
                } else if (!xpos) val = nwr_g[r];
                else if (x > nx + 1) val = 0.0f;          // never read by a positive velocity
                else {
                    const float f0 = f[(nx - 1) * V] * sv, f1 = f[(nx - 2) * V] * sv, f2v = f[(nx - 3) * V] * sv;
                    val = x == nx ? 3.0f * f0 - 3.0f * f1 + f2v : 6.0f * f0 - 8.0f * f1 + 3.0f * f2v;
                }
                wr[r][j] = val;
            }
        }
#pragma unroll
        for (int j = 0; j < 6; ++j) w[j] = make_float2(wr[0][j], wr[1][j]);
        w[6] = w[7] = f2(0.0f);
    }
    // flux per unit velocity at the face between c[2] and c[3] of c[0..5]
    auto face = [&](bool pos, const float2* c) -> float2 {
        if (ADV == HLB_WENO5_) {
            if (pos) return weno5_scaled2(c[0], c[1], c[2], c[3], c[4]);
            return weno5_scaled2(c[5], c[4], c[3], c[2], c[1]);
        }
        return pos ? upwind2_face2(c[1], c[2]) : upwind2_face2(c[4], c[3]);
    };
    // a cell entering the window at position e (head row pair hd; right-wall
    // ghosts from the cells nx-1, nx-2, nx-3 already in the window)
    auto enter = [&](int h, const float* hd0, const float* hd1, float2 m1, float2 m2, float2 m3,
                     float2 m4) -> float2 {
        if (h < nx) return __fmul2_rn(make_float2(hd0[vl], hd1[vl]), sv2);
        if (!xpos) return make_float2(nwr_g[0], nwr_g[1]);                     // emitted at the right wall
        if (h == nx) return __ffma2_rn(f2(3.0f), __fadd2_rn(m1, __fmul2_rn(f2(-1.0f), m2)), m3);
        if (h == nx + 1) return __ffma2_rn(f2(6.0f), m2, __ffma2_rn(f2(-8.0f), m3, __fmul2_rn(f2(3.0f), m4)));
        return f2(0.0f);                                                        // never read by v > 0
    };
    float2 Fm = __fmul2_rn(vxs, face(xpos, w));

    // a_x K_x f and a_y K_y f of one pair on the tensor cores: warp w takes
    // the X tile (rows 16 mX.., columns 8 nX..) of (K_x-contraction)^T and the
    // Y tile (rows 16 mY.., columns 8 nY..) of (K_y-contraction)^T and stores
    // them in the layout of sF.
    auto force_mma = [&](const float4* fr) {
        const float* ff = reinterpret_cast<const float*>(fr);
        float* kxo = reinterpret_cast<float*>(sKx);
        float* kyo = reinterpret_cast<float*>(sKy);
        const int R0 = 16 * mX + gq, jy0 = R0 >> 2, rx = R0 & 3;       // X rows: (j_y, cell/row)
        float dx[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int ks = 0; ks < XS; ++ks) {
            const int i0 = 8 * ks + tq;
            const float a[4] = {ff[(jy0 * SP + i0) * 4 + rx], ff[((jy0 + 2) * SP + i0) * 4 + rx],
                                ff[(jy0 * SP + i0 + 4) * 4 + rx], ff[((jy0 + 2) * SP + i0 + 4) * 4 + rx]};
            mma_3xtf32(dx, a, bxh[ks][0], bxl[ks][0], bxh[ks][1], bxl[ks][1]);
        }
        const int ixo = 8 * nX + 2 * tq;
        kxo[(jy0 * SP + ixo) * 4 + rx] = dx[0];
        kxo[(jy0 * SP + ixo + 1) * 4 + rx] = dx[1];
        kxo[((jy0 + 2) * SP + ixo) * 4 + rx] = dx[2];
        kxo[((jy0 + 2) * SP + ixo + 1) * 4 + rx] = dx[3];
        const int Q0 = 16 * mY + gq, ix0 = Q0 >> 2, ry = Q0 & 3;       // Y rows: (i_x, cell/row)
        float dy[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int ks = 0; ks < YS; ++ks) {
            const int j0 = 8 * ks + tq;
            const float a[4] = {ff[(j0 * SP + ix0) * 4 + ry], ff[(j0 * SP + ix0 + 2) * 4 + ry],
                                ff[((j0 + 4) * SP + ix0) * 4 + ry], ff[((j0 + 4) * SP + ix0 + 2) * 4 + ry]};
            mma_3xtf32(dy, a, byh[ks][0], byl[ks][0], byh[ks][1], byl[ks][1]);
        }
        const int jyo = 8 * nY + 2 * tq;
        kyo[(jyo * SP + ix0) * 4 + ry] = dy[0];
        kyo[((jyo + 1) * SP + ix0) * 4 + ry] = dy[1];
        kyo[(jyo * SP + ix0 + 2) * 4 + ry] = dy[2];
        kyo[((jyo + 1) * SP + ix0 + 2) * 4 + ry] = dy[3];
    };

    // Per pair: wait for its copies; write the centre values to sF[b] and
    // arrive on xch[b]; evaluate the faces (the other warps catch up
    // meanwhile); wait on xch[b]; then the force term, which reads every
    // warp's sF[b].  On the tensor-core path the force term sits between the
    // x and the y faces and its tiles are exchanged through xch2.  Passing
    // xch[b] of pair p also means every warp is done with pair p-1, so its
    // copy buffer is refilled then.  Every wait is bounded, so no warp can be
    // left waiting for good.
    int pa = 0, slot = 0;
    uint32_t phase = 0;
#pragma unroll 1
    for (int p = 0; p < npairs; ++p) {
        const int x0 = xa + 2 * p;
        const bool two = x0 + 1 < xb;
        pa = p;
        const Buf& B = buf[slot];
        if (!mbar_wait(&bars[slot], phase, g.err, g.wait_ns)) *sAbort = 1;
        if (t == 0) expect(p + kPairDepth - 1);     // its slot's previous phase (pair p-1) is complete
        const int b = p & 1;
        w[6] = enter(x0 + 3, B.head[0][0], B.head[0][1], w[5], w[4], w[3], w[2]);
        w[7] = enter(x0 + 4, B.head[1][0], B.head[1][1], w[6], w[5], w[4], w[3]);
        const float2 fc0 = __fmul2_rn(w[3], isv2), fc1 = __fmul2_rn(w[4], isv2);
        sF[(b * VY + jy) * SP + ix] = make_float4(fc0.x, fc0.y, fc1.x, fc1.y);
        __syncwarp();
        if (lane == 0) mbar_arrive(&xch[b]);
        // x faces x0+1/2, x0+3/2 (rows packed); x0-1/2 carried
        const float2 Fp0 = __fmul2_rn(vxs, face(xpos, w + 1));
        const float2 Fp1 = __fmul2_rn(vxs, face(xpos, w + 2));
        const float2 divx0 = __fmul2_rn(fsub2(Fp0, Fm), f2(invdx[x0]));
        const float2 divx1 = __fmul2_rn(fsub2(Fp1, Fp0), f2(two ? invdx[x0 + 1] : 0.0f));
        Fm = Fp1;
        if constexpr (kMMA) {
            if (!mbar_wait(&xch[b], (p >> 1) & 1, g.err, g.wait_ns)) *sAbort = 1;
            if (*sAbort) break;
            issue(p + kPairDepth - 1);
            force_mma(sF + b * VY * SP);
            __syncwarp();
            if (lane == 0) mbar_arrive(xch2);
        }
        // y faces (periodic), cells packed: rows y0-3 .. y0+4 of columns x0, x0+1
        float2 col[8];
#pragma unroll
        for (int k = 0; k < 3; ++k) col[k] = __fmul2_rn(make_float2(B.halo[0][k][vl], B.halo[1][k][vl]), sv2);
        col[3] = make_float2(w[3].x, w[4].x);
        col[4] = make_float2(w[3].y, w[4].y);
#pragma unroll
        for (int k = 0; k < 3; ++k) col[5 + k] = __fmul2_rn(make_float2(B.halo[0][3 + k][vl], B.halo[1][3 + k][vl]), sv2);
        const float2 G0 = face(ypos, col), G1 = face(ypos, col + 1), G2 = face(ypos, col + 2);
        const float2 dy0 = __fmul2_rn(vys, fsub2(G1, G0));   // row y0, cells x0, x0+1
        const float2 dy1 = __fmul2_rn(vys, fsub2(G2, G1));   // row y0+1
        // shift the window by two cells
#pragma unroll
        for (int j = 0; j < 6; ++j) w[j] = w[j + 2];
        // force term at both cells (rows packed): a_x K_x f + a_y K_y f
        float2 fk0, fk1;
        if constexpr (kMMA) {
            if (!mbar_wait(xch2, p & 1, g.err, g.wait_ns)) *sAbort = 1;
            const float4 ex = sKx[jy * SP + ix], ey = sKy[jy * SP + ix];
            fk0 = __fadd2_rn(make_float2(ex.x, ex.y), make_float2(ey.x, ey.y));
            fk1 = __fadd2_rn(make_float2(ex.z, ex.w), make_float2(ey.z, ey.w));
        } else {
            if (!mbar_wait(&xch[b], (p >> 1) & 1, g.err, g.wait_ns)) *sAbort = 1;
            if (*sAbort) break;
            issue(p + kPairDepth - 1);
            const float4* fr = sF + b * VY * SP;
            const float4* kxr = reinterpret_cast<const float4*>(sKd + ix * KXR);            // (k, k) pairs, two per load
            const float4* kyr = reinterpret_cast<const float4*>(sKd + QX2 * KXR + jy * KYR);
            fk0 = f2(0.0f);
            fk1 = f2(0.0f);
#pragma unroll
            for (int i = 0; i < QX2; i += 2) {
                const float4 kk = kxr[i >> 1];
                const float4 fa = fr[jy * SP + i], fb = fr[jy * SP + i + 1];
                fk0 = __ffma2_rn(make_float2(kk.x, kk.y), make_float2(fa.x, fa.y), fk0);
                fk1 = __ffma2_rn(make_float2(kk.x, kk.y), make_float2(fa.z, fa.w), fk1);
                fk0 = __ffma2_rn(make_float2(kk.z, kk.w), make_float2(fb.x, fb.y), fk0);
                fk1 = __ffma2_rn(make_float2(kk.z, kk.w), make_float2(fb.z, fb.w), fk1);
            }
#pragma unroll
            for (int j = 0; j < VY; j += 2) {
                const float4 kk = kyr[j >> 1];
                const float4 fa = fr[j * SP + ix], fb = fr[(j + 1) * SP + ix];
                fk0 = __ffma2_rn(make_float2(kk.x, kk.y), make_float2(fa.x, fa.y), fk0);
                fk1 = __ffma2_rn(make_float2(kk.x, kk.y), make_float2(fa.z, fa.w), fk1);
                fk0 = __ffma2_rn(make_float2(kk.z, kk.w), make_float2(fb.x, fb.y), fk0);
                fk1 = __ffma2_rn(make_float2(kk.z, kk.w), make_float2(fb.z, fb.w), fk1);
            }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            if (i == 1 && !two) break;
            const float* c0 = B.coef[0] + i * ncp;
            const float* c1 = B.coef[1] + i * ncp;
            const float2 feq = __fmul2_rn(__fmul2_rn(make_float2(c0[ix], c1[ix]), make_float2(c0[QX2 + jy], c1[QX2 + jy])),
                                          make_float2(c0[csrc_z], c1[csrc_z]));
            const float2 itau = make_float2(c0[csrc_t], c1[csrc_t]);
            const float2 fc = i ? fc1 : fc0;
            const float2 divx = i ? divx1 : divx0;
            const float2 divy = i ? make_float2(dy0.y, dy1.y) : make_float2(dy0.x, dy1.x);
            // L = -div_x - div_y - (a_x K_x f + a_y K_y f) - (f - feq)/tau
            float2 L = __fadd2_rn(__fadd2_rn(divx, divy), i ? fk1 : fk0);
            L = __ffma2_rn(fsub2(fc, feq), itau, L);
            float2 out;      // fc + dt (-L), then the RK-3 combination (Eq. "eq:rk3")
            if (stage == 0) {
                out = fsub2(fc, __fmul2_rn(dt2, L));
            } else {
                const float2 fo_n = make_float2(B.fnr[i][0][vl], B.fnr[i][1][vl]);
                if (stage == 1)
                    out = __ffma2_rn(f2(0.75f), fo_n, __fmul2_rn(f2(0.25f), fsub2(fc, __fmul2_rn(dt2, L))));
                else
                    out = __ffma2_rn(f2(1.0f / 3.0f), fo_n, __fmul2_rn(f2(2.0f / 3.0f), fsub2(fc, __fmul2_rn(dt2, L))));
            }
            const int x = x0 + i;
            if (valid[0]) fov[roff[0] + x * V] = out.x;
            if (valid[1]) fov[roff[1] + x * V] = out.y;
        }
        if (++slot == kPairDepth) { slot = 0; phase ^= 1u; }
    }
    if (*sAbort && t == 0) {
        // a wait ran out at pair pa: let the copies of the pairs issued since
        // (pa .. pa + kPairDepth - 2) land before the CTA exits
        for (int s2 = pa; s2 < npairs && s2 < pa + kPairDepth - 1; ++s2)
            mbar_drain(&bars[s2 % kPairDepth], (s2 / kPairDepth) & 1, g.wait_ns);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t prepare_node() {
    cudaError_t e = cudaFuncSetAttribute(coef_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(coef_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(coef_df_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(coef_df_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(coef_df_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sums_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sums_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
}

// Node pass of a stage: the quadrature sums of every node, then the factor
// lines.  The sums live in the first 8 R of each node's factor line slot of
// an auxiliary buffer (g.sums).
void launch_node(int precision, const GroupDev& g, const void* fs, cudaStream_t st) {
    const size_t es = precision == HLB_FP64_ ? 8 : 4;
    const size_t smem_a = 4 * (g.V + g.VY * g.VZ) * es;
    const int blocks_a = (g.nnodes + 7) / 8 < 152 * 16 ? (g.nnodes + 7) / 8 : 152 * 16;
    const int nrec = 5 * g.Nx + 1;
    const int nT = g.Qx * (g.Nx + 1) + g.VY * (g.Ny + 1) + g.VZ * (g.Nz + 1);
    const int ncoef = 2 * (g.Nx + 1) + (g.Ny + 1) + (g.Nz + 1);
    const int block_b = 32;
    const size_t per_warp = 8 * (32 * ncoef + 64) + 32 * sizeof(NodeDF);
    const size_t smem_b = 8 * (nrec + nT) + (block_b / 32) * per_warp;
    const int batches = (g.nnodes + 31) / 32;
    const int blocks_b = batches;
    if (precision == HLB_FP64_) {
        sums_kernel<double><<<blocks_a, 256, smem_a, st>>>(g, (const double*)fs, (double*)g.sums);
        coef_kernel<double><<<blocks_b, block_b, smem_b, st>>>(g, (const double*)g.sums);
    } else {
        sums_kernel<float><<<blocks_a, 256, smem_a, st>>>(g, (const float*)fs, (float*)g.sums);
        const int nmax = max(g.Nx, max(g.Ny, g.Nz));
        if (g.use_df && nmax < 16) {
            const int nT = g.Qx * (g.Nx + 1) + g.VY * (g.Ny + 1) + g.VZ * (g.Nz + 1);
            const size_t smem_c = 8 * ((size_t)nrec + nT + 1) + 4 * 32 * (size_t)g.ncp * 4;
            const int blocks_c = (g.nnodes + 127) / 128;
            if (nmax < 8) coef_df_kernel<8><<<blocks_c, 128, smem_c, st>>>(g, (const float*)g.sums);
            else if (nmax < 12) coef_df_kernel<12><<<blocks_c, 128, smem_c, st>>>(g, (const float*)g.sums);
            else coef_df_kernel<16><<<blocks_c, 128, smem_c, st>>>(g, (const float*)g.sums);
        } else {
            coef_kernel<float><<<blocks_b, block_b, smem_b, st>>>(g, (const float*)g.sums);
        }
    }
}

#define HLB_MARCH_LIST(X)                                                              \
    X(float, 8, 4, 1) X(float, 8, 4, 2) X(float, 8, 1, 1) X(float, 16, 8, 1)              \
    X(float, 16, 8, 2) X(float, 16, 1, 1) X(float, 32, 16, 1) X(float, 32, 16, 2)         \
    X(float, 32, 1, 1) X(double, 8, 4, 1) X(double, 8, 1, 1) X(double, 16, 8, 1)          \
    X(double, 32, 16, 1) X(double, 16, 1, 1)

template <typename R, int ADV, int QX2, int VY, int TY>
static void launch_one(const GroupDev& g, const Work* works, int nworks, const void* fs, const void* fn,
                       void* fo, int stage, cudaStream_t st) {
    if constexpr (sizeof(R) == 4 && TY == 2) {
        march_pair_kernel<ADV, QX2, VY><<<nworks, QX2 * VY, pair_smem_bytes<QX2, VY>(), st>>>(
            g, works, (const float*)fs, (const float*)fn, (float*)fo, stage);
    } else {
        march_kernel<R, ADV, QX2, VY, TY><<<nworks, QX2 * VY, march_smem_bytes<R, QX2, VY, TY>(), st>>>(
            g, works, (const R*)fs, (const R*)fn, (R*)fo, stage);
    }
}

template <typename R, int ADV, int QX2, int VY, int TY>
static cudaError_t prepare_one() {
    if constexpr (sizeof(R) == 4 && TY == 2)
        return cudaFuncSetAttribute(march_pair_kernel<ADV, QX2, VY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)pair_smem_bytes<QX2, VY>());
    else
        return cudaFuncSetAttribute(march_kernel<R, ADV, QX2, VY, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)march_smem_bytes<R, QX2, VY, TY>());
}

bool march_available(int precision, int adv, int QX2, int VY, int TY) {
    (void)adv;
    const bool dbl = precision == HLB_FP64_;
#define HLB_AVAIL(RT, A, B, C) \
    if ((sizeof(RT) == 8) == dbl && QX2 == A && VY == B && TY == C) return true;
    HLB_MARCH_LIST(HLB_AVAIL)
#undef HLB_AVAIL
    return false;
}

cudaError_t prepare_march(int precision, int adv, int QX2, int VY, int TY) {
    const bool dbl = precision == HLB_FP64_;
#define HLB_PREP(RT, A, B, C)                                                        \
    if ((sizeof(RT) == 8) == dbl && QX2 == A && VY == B && TY == C)                  \
        return adv == HLB_WENO5_ ? prepare_one<RT, HLB_WENO5_, A, B, C>()          \
                                 : prepare_one<RT, HLB_UPWIND2_, A, B, C>();
    HLB_MARCH_LIST(HLB_PREP)
#undef HLB_PREP
    return cudaSuccess;
}

void launch_march(int precision, int adv, int QX2, int VY, int TY, const GroupDev& g, const Work* works,
                  int nworks, const void* fs, const void* fn, void* fo, int stage, cudaStream_t st) {
    const bool dbl = precision == HLB_FP64_;
#define HLB_LAUNCH(RT, A, B, C)                                                                      \
    if ((sizeof(RT) == 8) == dbl && QX2 == A && VY == B && TY == C) {                                \
        if (adv == HLB_WENO5_) launch_one<RT, HLB_WENO5_, A, B, C>(g, works, nworks, fs, fn, fo, stage, st); \
        else launch_one<RT, HLB_UPWIND2_, A, B, C>(g, works, nworks, fs, fn, fo, stage, st);              \
        return;                                                                                      \
    }
    HLB_MARCH_LIST(HLB_LAUNCH)
#undef HLB_LAUNCH
}

}  // namespace hlb
