// Node pass of an RK-3 stage (sm_103a): the quadrature sums of every node
// (Eq. "eq:fmoms"), then n, u, T, 1/tau and the per-node equilibrium factor
// line coef[node] = { n g_x (2Qx), g_y (Qy), g_z (Qz), 1/tau } (Eqs.
// "eq:hh_gk", "eq:H_gk", App. A; half-range recurrence in the orthonormal
// basis, full-range Hermite recurrence).
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "hlb_coef.cuh"
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
    // 4-vector loads with eight lanes per node, four nodes per warp: they need
    // 4 | 2Qx and 2Qx | 32 (2Qx a power of two up to 32), so that the four
    // velocities of a load share (jy, kz) and a lane's p_x never change.  The
    // compensated tree then has three levels, and each shuffle serves four
    // nodes.  Other sets: one warp per node, a table of all velocities.
    const bool vec4 = (QX2 & 3) == 0 && (QX2 & (QX2 - 1)) == 0 && QX2 <= 32 && V >= 32;
    auto store = [&](int node, R a0, R a1, R a2, R a3, R a4, R c0, R c1, R c2, R c3, R c4) {
        R* o = sums + (size_t)node * kSumStride;
        o[0] = a0; o[1] = a1; o[2] = a2; o[3] = a3; o[4] = a4;
        o[8] = c0; o[9] = c1; o[10] = c2; o[11] = c3; o[12] = c4;
    };
    if (vec4) {
        const int sl = lane & 7;
        const int x0 = (4 * sl) % QX2;
        const int lg = __ffs(QX2) - 1;                   // 2Qx = 2^lg
        const R pxa = sM[x0].x, pxb = sM[x0 + 1].x, pxc = sM[x0 + 2].x, pxd = sM[x0 + 3].x;
        for (int nb = (blockIdx.x * nw + warp) * 4; nb < g.nnodes; nb += gridDim.x * nw * 4) {
            const int node = nb + (lane >> 3);
            // compensated per-lane sums (FP32 states)
            R a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0, c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0;
            if (node < g.nnodes) {
                const int ii = g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0;
                const InstDev& I = g.inst[ii];
                const R4* f4 = reinterpret_cast<const R4*>(fs + (size_t)I.f_off + (size_t)(node - I.node_off) * V);
#pragma unroll 4
                for (int q = sl; q < (V >> 2); q += 8) {
                    const R4 x = f4[q];
                    const R4 yz = sYZ[(q << 2) >> lg];
                    const R sq = (x.x + x.y) + (x.z + x.w);
                    csum_add(a0, c0, sq);
                    csum_add(a1, c1, pxa * x.x + pxb * x.y + pxc * x.z + pxd * x.w);
                    csum_add(a2, c2, yz.x * sq);
                    csum_add(a3, c3, yz.y * sq);
                    csum_add(a4, c4, pxa * pxa * x.x + pxb * pxb * x.y + pxc * pxc * x.z + pxd * pxd * x.w + yz.z * sq);
                }
            }
            // compensated tree over the eight lanes of each node
            auto tree8 = [](R& sa, R& ca) {
#pragma unroll
                for (int o = 4; o > 0; o >>= 1) {
                    const R s2 = __shfl_xor_sync(0xffffffffu, sa, o), c2 = __shfl_xor_sync(0xffffffffu, ca, o);
                    csum_add(sa, ca, s2);
                    ca += c2;
                }
            };
            tree8(a0, c0); tree8(a1, c1); tree8(a2, c2); tree8(a3, c3); tree8(a4, c4);
            if (sl == 0 && node < g.nnodes) store(node, a0, a1, a2, a3, a4, c0, c1, c2, c3, c4);
        }
        return;
    }
    for (int node = blockIdx.x * nw + warp; node < g.nnodes; node += gridDim.x * nw) {
        const int ii = g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0;
        const InstDev& I = g.inst[ii];
        const R* f = fs + (size_t)I.f_off + (size_t)(node - I.node_off) * V;
        // compensated per-lane sums (FP32 states), compensated warp tree
        R a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0, c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0;
        for (int v = lane; v < V; v += 32) {
            const R val = f[v];
            const R4 mw = sM[v];
            csum_add(a0, c0, val);
            csum_add(a1, c1, mw.x * val);
            csum_add(a2, c2, mw.y * val);
            csum_add(a3, c3, mw.z * val);
            csum_add(a4, c4, mw.w * val);
        }
        csum_warp(a0, c0); csum_warp(a1, c1); csum_warp(a2, c2); csum_warp(a3, c3); csum_warp(a4, c4);
        if (lane == 0) store(node, a0, a1, a2, a3, a4, c0, c1, c2, c3, c4);
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
            const R* sm = sums + (size_t)node * kSumStride;
            active = inv_Kn != 0.0;
            // n, u, T in FP64 from the compensated sums (one division)
            const double n = (double)sm[0] + (double)sm[8], in = 1.0 / n;
            const double ux = ((double)sm[1] + (double)sm[9]) * in, uy = ((double)sm[2] + (double)sm[10]) * in,
                         uz = ((double)sm[3] + (double)sm[11]) * in;
            const double T = ((double)sm[4] + (double)sm[12] - n * (ux * ux + uy * uy + uz * uz)) * in *
                             (g.D == 3 ? 1.0 / 3.0 : (g.D == 2 ? 0.5 : 1.0));
            sNT[2 * lane] = n;
            sNT[2 * lane + 1] = n * inv_Kn;
            if (active) {
                if (df) {
                    node_inputs_df(n, ux, uy, uz, T, Nx, sIn[lane]);
                    for (int role = 0; role < 4; ++role)
                        node_coefficients_df(g, role, sIn[lane], sRecF, sGF + lane * ncoef);
                } else {
                    for (int role = 0; role < 4; ++role) {
                        if (g.quad_x && role < 2) {      // G^{+-} by quadrature (quad_coef_kernel)
                            const double* q = g.gquad + ((size_t)node * 2 + role) * (Nx + 1);
                            for (int l = 0; l <= Nx; ++l) sG[lane * ncoef + role * (Nx + 1) + l] = q[l];
                        } else {
                            node_coefficients(g, role, ux, uy, uz, T, sRec, sG + lane * ncoef);
                        }
                    }
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
        if (g.has_field && lane < nb) {              // a = a_uniform + a_field(node)
            const int node = base + lane;
            const InstDev& I = g.inst[g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0];
            R* fl = coef + (size_t)node * g.ncp + g.field_off;
            fl[0] = (R)(I.ax + g.afield[3 * (size_t)node]);
            fl[1] = (R)(I.ay + g.afield[3 * (size_t)node + 1]);
            fl[2] = (R)(I.az + g.afield[3 * (size_t)node + 2]);
        }
        __syncwarp();
    }
}

template <int NM>
__global__ void __launch_bounds__(128) coef_df_kernel(const GroupDev g, const float* __restrict__ sums) {
    extern __shared__ __align__(16) float2 cdf[];
    const int Nx = g.Nx, Ny = g.Ny, Nz = g.Nz, Qx = g.Qx, QX2 = g.QX2, VY = g.VY, VZ = g.VZ, ncp = g.ncp;
    const int nrec = 5 * Nx + 1;
    // the tables T_x (Qx rows), T_y (VY rows), T_z (VZ rows) of Nx+1, Ny+1,
    // Nz+1 double-float entries, re-laid as row pairs (dot2_pair); an odd last
    // row is paired with zeros
    const int px = (Qx + 1) >> 1, py = (VY + 1) >> 1, pz = (VZ + 1) >> 1;
    const int nP = px * (Nx + 1) + py * (Ny + 1) + pz * (Nz + 1);
    float4* sP = reinterpret_cast<float4*>(cdf);
    float2* sRec = reinterpret_cast<float2*>(sP + nP);
    float* sLine = reinterpret_cast<float*>(sP + nP + ((nrec + 1) >> 1)) + (threadIdx.x >> 5) * 32 * ncp;   // [32][ncp] per warp
    for (int i = threadIdx.x; i < nrec; i += blockDim.x) sRec[i] = g.recf[i];
    {
        const float2* Tx = g.Tf;
        const float2* Ty = Tx + Qx * (Nx + 1);
        const float2* Tz = Ty + VY * (Ny + 1);
        auto pairs = [&](float4* dst, const float2* T, int rows, int n1) {
            const int np = (rows + 1) >> 1;
            for (int i = threadIdx.x; i < np * n1; i += blockDim.x) {
                const int k = 2 * (i / n1), l = i % n1;
                const float2 a = T[k * n1 + l];
                const float2 b = k + 1 < rows ? T[(k + 1) * n1 + l] : make_float2(0.0f, 0.0f);
                dst[i] = make_float4(a.x, b.x, a.y, b.y);
            }
        };
        pairs(sP, Tx, Qx, Nx + 1);
        pairs(sP + px * (Nx + 1), Ty, VY, Ny + 1);
        pairs(sP + px * (Nx + 1) + py * (Ny + 1), Tz, VZ, Nz + 1);
    }
    __syncthreads();
    const float4* sPx = sP;
    const float4* sPy = sPx + px * (Nx + 1);
    const float4* sPz = sPy + py * (Ny + 1);
    const int lane = threadIdx.x & 31;
    const int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    const int node = base + lane;
    float* line = sLine + lane * ncp;
    if (node < g.nnodes) {
        const int ii = g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0;
        const double inv_Kn = g.inst[ii].inv_Kn;
        const float* sm = sums + (size_t)node * kSumStride;
        bool done = false;
        if constexpr (NM <= 12) {
            if (Nx <= HLB_DF_SPECIAL_MAX_N) {
                // n, u, T and the recurrences' start in double-float (no FP64
                // pipe work but for 1/tau and the rare |z| > 2.5)
                NodeDF nin;
                const double n = node_inputs_from_sums_df(sm, g.D, nin);
                factor_line_df_in<NM>(g, nin, n * inv_Kn, sPx, sPy, sPz, sRec, line);
                done = true;
            }
        }
        if (!done) {
            // n, u, T in FP64 from the compensated sums (one division)
            const double n = (double)sm[0] + (double)sm[8], in = 1.0 / n;
            const double ux = ((double)sm[1] + (double)sm[9]) * in, uy = ((double)sm[2] + (double)sm[10]) * in,
                         uz = ((double)sm[3] + (double)sm[11]) * in;
            const double T = ((double)sm[4] + (double)sm[12] - n * (ux * ux + uy * uy + uz * uz)) * in *
                             (g.D == 3 ? 1.0 / 3.0 : (g.D == 2 ? 0.5 : 1.0));
            factor_line_df<NM>(g, n, ux, uy, uz, T, (double)n * inv_Kn, sPx, sPy, sPz, sRec, line);
        }
        if (g.has_field) {                           // a = a_uniform + a_field(node)
            const InstDev& I = g.inst[ii];
            line[g.field_off] = (float)(I.ax + g.afield[3 * (size_t)node]);
            line[g.field_off + 1] = (float)(I.ay + g.afield[3 * (size_t)node + 1]);
            line[g.field_off + 2] = (float)(I.az + g.afield[3 * (size_t)node + 2]);
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


}  // namespace

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

// Blocks of `func` resident on the whole GPU at once (one wave), at most
// `want`: a grid-stride kernel then has no partly filled last wave.
static int one_wave(const void* func, int block, size_t smem, int want) {
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            nsm = 152;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, func, block, smem) != cudaSuccess || per < 1) per = 1;
    return want < nsm * per ? (want > 0 ? want : 1) : nsm * per;
}

__global__ void df_special_kernel(const double* __restrict__ z, int n, double* __restrict__ erf_out,
                                  double* __restrict__ exp_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 zd = df_from_double(z[i]);
    const float2 z2 = df_mul(zd, zd);
    const float2 E = df_exp_nonpos(make_float2(-z2.x, -z2.y));
    const float2 er = df_erf_series(zd, z2, E);
    erf_out[i] = (double)er.x + (double)er.y;
    exp_out[i] = (double)E.x + (double)E.y;
}

cudaError_t launch_df_special(const double* z, int n, double* erf_out, double* exp_out) {
    if (n > 0) df_special_kernel<<<(n + 127) / 128, 128>>>(z, n, erf_out, exp_out);
    const cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : cudaDeviceSynchronize();
}

// Node pass of a stage: the quadrature sums of every node, then the factor
// lines.  The sums live in the first 8 R of each node's factor line slot of
// an auxiliary buffer (g.sums).
void launch_node(int precision, const GroupDev& g, const void* fs, cudaStream_t st) {
    const size_t es = precision == HLB_FP64_ ? 8 : 4;
    const size_t smem_a = 4 * (g.V + g.VY * g.VZ) * es;
    const int want_a = (g.nnodes + 7) / 8;
    const int blocks_a = precision == HLB_FP64_
                             ? one_wave(reinterpret_cast<const void*>(&sums_kernel<double>), 256, smem_a, want_a)
                             : one_wave(reinterpret_cast<const void*>(&sums_kernel<float>), 256, smem_a, want_a);
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
            const int nP = (g.Qx + 1) / 2 * (g.Nx + 1) + (g.VY + 1) / 2 * (g.Ny + 1) + (g.VZ + 1) / 2 * (g.Nz + 1);
            const size_t smem_c = 16 * ((size_t)nP + (nrec + 1) / 2) + 4 * 32 * (size_t)g.ncp * 4;
            const int blocks_c = (g.nnodes + 127) / 128;
            if (nmax < 8) coef_df_kernel<8><<<blocks_c, 128, smem_c, st>>>(g, (const float*)g.sums);
            else if (nmax < 12) coef_df_kernel<12><<<blocks_c, 128, smem_c, st>>>(g, (const float*)g.sums);
            else coef_df_kernel<16><<<blocks_c, 128, smem_c, st>>>(g, (const float*)g.sums);
        } else {
            coef_kernel<float><<<blocks_b, block_b, smem_b, st>>>(g, (const float*)g.sums);
        }
    }
}

}  // namespace hlb
