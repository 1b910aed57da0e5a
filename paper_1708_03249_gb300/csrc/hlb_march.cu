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

#include "hlb_device.cuh"
#include "hlb_internal.h"

namespace hlb {
namespace {

// ---------------------------------------------------------------------------
// node kernel
// ---------------------------------------------------------------------------
// Node batch of one CTA.  FP64 runs at 1/64 of FP32 on this GPU and a warp
// instruction costs the same whatever its active mask, so the FP64 work
// (recurrences, dot products) is batched so that every lane is busy.
constexpr int kNodeBatch = 32;

template <typename R>
__global__ void __launch_bounds__(256) node_kernel(const GroupDev g, const R* __restrict__ fs) {
    extern __shared__ __align__(16) double nsm[];
    const int Nx = g.Nx, Ny = g.Ny, Nz = g.Nz;
    const int nrec = 5 * Nx + 1;
    const int nT = g.Qx * (Nx + 1) + g.VY * (Ny + 1) + g.VZ * (Nz + 1);
    const int ncoef = 2 * (Nx + 1) + (Ny + 1) + (Nz + 1);
    const int QX2 = g.QX2, VY = g.VY, VZ = g.VZ, V = g.V;
    const int tid = threadIdx.x, bs = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = bs >> 5;
    // shared: moment weights, FP64 tables, per-node sums / state / coefficients
    R* sM = reinterpret_cast<R*>(nsm);
    double* sRec = nsm + (4 * V * sizeof(R) + 7) / 8;
    double* sT = sRec + nrec;
    double* sSum = sT + nT;                              // [kNodeBatch][5]
    double* sState = sSum + 5 * kNodeBatch;              // [kNodeBatch][6]: n, ux, uy, uz, T, 1/tau
    double* sG = sState + 6 * kNodeBatch;                // [kNodeBatch][ncoef]
    const R* px = static_cast<const R*>(g.p);
    const R* py = px + QX2;
    const R* pz = py + VY;
    for (int v = tid; v < V; v += bs) {
        const int ix = v % QX2, jy = (v / QX2) % VY, kz = v / (QX2 * VY);
        const R a = px[ix], b = py[jy], c = pz[kz];
        sM[4 * v + 0] = a;
        sM[4 * v + 1] = b;
        sM[4 * v + 2] = c;
        sM[4 * v + 3] = a * a + b * b + c * c;
    }
    for (int i = tid; i < nrec; i += bs) sRec[i] = g.rec[i];
    for (int i = tid; i < nT; i += bs) sT[i] = g.Td[i];
    __syncthreads();
    const double* sTx = sT;
    const double* sTy = sTx + g.Qx * (Nx + 1);
    const double* sTz = sTy + VY * (Ny + 1);
    R* coef = static_cast<R*>(g.coef);
    const int nf = QX2 + VY + VZ;

    for (int base = blockIdx.x * kNodeBatch; base < g.nnodes; base += gridDim.x * kNodeBatch) {
        const int nb = min(kNodeBatch, g.nnodes - base);
        // 1. moment sums: one warp per node, FP32 lanes, pairwise tree
        for (int k = warp; k < nb; k += nw) {
            const int node = base + k;
            const int ii = g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0;
            const InstDev& I = g.inst[ii];
            const R* f = fs + (size_t)I.f_off + (size_t)(node - I.node_off) * V;
            R a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
            for (int v = lane; v < V; v += 32) {
                const R val = f[v];
                const R* mw = sM + 4 * v;
                a0 += val;
                a1 += mw[0] * val;
                a2 += mw[1] * val;
                a3 += mw[2] * val;
                a4 += mw[3] * val;
            }
            a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2); a3 = warp_sum(a3); a4 = warp_sum(a4);
            if (lane == 0) {
                double* sm = sSum + 5 * k;
                sm[0] = a0; sm[1] = a1; sm[2] = a2; sm[3] = a3; sm[4] = a4;
            }
        }
        __syncthreads();
        // 2. n, u, T, 1/tau per node (one lane per node)
        if (tid < nb) {
            const int node = base + tid;
            const int ii = g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0;
            const double* sm = sSum + 5 * tid;
            const double n = sm[0];
            const double ux = sm[1] / n, uy = sm[2] / n, uz = sm[3] / n;
            double* st = sState + 6 * tid;
            st[0] = n; st[1] = ux; st[2] = uy; st[3] = uz;
            st[4] = (sm[4] - n * (ux * ux + uy * uy + uz * uz)) / (g.D * n);
            st[5] = n * g.inst[ii].inv_Kn;
        }
        __syncthreads();
        // 3. coefficients: lane per (node, role); roles 0/1 = half-range G^{+-},
        //    2 = full-range p_y, 3 = p_z.  Consecutive lanes share a role.
        for (int t = tid; t < 4 * nb; t += bs) {
            const int role = t / nb, k = t - role * nb;
            const double* st = sState + 6 * k;
            if (st[5] != 0.0) node_coefficients(g, role, st[1], st[2], st[3], st[4], sRec, sG + k * ncoef);
        }
        __syncthreads();
        // 4. factor lines: lane per (node, output)
        for (int t = tid; t < nb * (nf + 1); t += bs) {
            const int k = t / (nf + 1), o = t - k * (nf + 1);
            const double* st = sState + 6 * k;
            const double* G = sG + k * ncoef;
            R* line = coef + (size_t)(base + k) * g.ncp;
            double acc = 0.0;
            if (st[5] == 0.0) {                  // collisionless: no equilibrium at all
                acc = 0.0;
            } else if (o < QX2) {
                const int kk = o % g.Qx, sg = o / g.Qx;
                const double* Gs = G + sg * (Nx + 1);
                for (int l = 0; l <= Nx; ++l) acc += sTx[kk * (Nx + 1) + l] * Gs[l];
                acc *= st[0];
            } else if (o < QX2 + VY) {
                const int j = o - QX2;
                if (g.Qy) {
                    const double* Gy = G + 2 * (Nx + 1);
                    for (int l = 0; l <= Ny; ++l) acc += sTy[j * (Ny + 1) + l] * Gy[l];
                } else {
                    acc = 1.0;
                }
            } else if (o < nf) {
                const int j = o - QX2 - VY;
                if (g.Qz) {
                    const double* Gz = G + 2 * (Nx + 1) + (Ny + 1);
                    for (int l = 0; l <= Nz; ++l) acc += sTz[j * (Nz + 1) + l] * Gz[l];
                } else {
                    acc = 1.0;
                }
            } else {
                acc = st[5];
            }
            line[o] = (R)acc;
        }
        __syncthreads();
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
    return kDepth * sizeof(StepBuf<R, QX2, VY, TY>) + 2 * TY * QX2 * VY * sizeof(R) + kDepth * 8 + 16;
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

#pragma unroll 1
    for (int x = xa; x < xb; ++x) {
        const int step = x - xa;
        const Buf& B = buf[step % kDepth];
        mbar_wait(&bars[step % kDepth], (step / kDepth) & 1, g.err);
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
}

// FP32, two strip rows packed into the lanes of f32x2 registers (x = row y0,
// y = row y0+1).  Same pipeline and arithmetic as march_kernel; the window
// holds values pre-multiplied by the population's inverse weight so that
// every WENO evaluation reads scaled stencils directly.
template <int ADV, int QX2, int VY>
__global__ void __launch_bounds__(QX2 * VY, (QX2 * VY <= 32 ? 16 : (QX2 * VY <= 128 ? 4 : 1)))
march2_kernel(const GroupDev g, const Work* __restrict__ works, const float* __restrict__ fs,
              const float* __restrict__ fn, float* __restrict__ fo, int stage) {
    constexpr int TY = 2;
    constexpr int S = QX2 * VY;
    constexpr int QX = QX2 / 2;
    using Buf = StepBuf<float, QX2, VY, TY>;
    extern __shared__ __align__(128) unsigned char msm[];
    Buf* buf = reinterpret_cast<Buf*>(msm);
    float2* sF = reinterpret_cast<float2*>(msm + kDepth * sizeof(Buf));     // [2][S] (row0, row1)
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(sF + 2 * S);

    const Work W = works[blockIdx.x];
    const InstDev& I = g.inst[W.inst];
    const int t = threadIdx.x;
    const int ix = t % QX2, jy = t / QX2, kz = W.kz;
    const int V = g.V, nx = I.nx, ny = I.ny, ncp = g.ncp;
    const int v = (kz * VY + jy) * QX2 + ix;
    const float* P = static_cast<const float*>(g.p);
    const float vx = P[ix], vy = P[QX2 + jy];
    const bool xpos = ix < QX, ypos = vy > 0.0f;
    const float sv = static_cast<const float*>(g.wscale)[v];
    const float isv = 1.0f / sv;
    const float* K = static_cast<const float*>(g.K);
    float2 kx[QX2], ky[VY];
#pragma unroll
    for (int i = 0; i < QX2; ++i) kx[i] = f2(K[ix * QX2 + i]);
#pragma unroll
    for (int j = 0; j < VY; ++j) ky[j] = f2(K[QX2 * QX2 + jy * VY + j]);
    const float2 ax2 = f2((float)I.ax), ay2 = f2((float)I.ay), dt2 = f2((float)I.dt);
    const float2 vxs = f2(vx * isv), vys = f2(vy * isv * (float)I.inv_dy), isv2 = f2(isv);
    const float* invdx = static_cast<const float*>(g.inv_dx) + I.dx_off;
    const int rs = nx * V;
    const float* fsI = fs + I.f_off;
    const float* fnI = fn + I.f_off;
    float* fov = fo + I.f_off + v;
    const float* cI = static_cast<const float*>(g.coef) + (size_t)I.node_off * ncp;
    const int csrc_z = QX2 + VY + kz, csrc_t = QX2 + VY + g.VZ;
    const float* gw = static_cast<const float*>(g.gw) + I.gw_off;
    const float gwl = gw[v] * sv, gwr = gw[V + v] * sv;
    int roff[TY], crow[TY];
    bool valid[TY];
    float nwl_g[TY], nwr_g[TY];        // scaled emitted ghosts
#pragma unroll
    for (int r = 0; r < TY; ++r) {
        const int y = W.y0 + r;
        valid[r] = y < ny;
        const int yy = y % ny;
        roff[r] = yy * rs;
        crow[r] = yy * nx;
        nwl_g[r] = (float)g.nw[(size_t)(I.row_off + yy) * 2 + 0] * gwl;
        nwr_g[r] = (float)g.nw[(size_t)(I.row_off + yy) * 2 + 1] * gwr;
    }
    const int xa = W.xa, xb = W.xb;
    const int slab = kz * S;

    auto issue = [&](int xs) {
        if (xs >= xb) return;
        Buf& B = buf[(xs - xa) % kDepth];
        unsigned long long* bar = &bars[(xs - xa) % kDepth];
        const uint32_t row_bytes = S * sizeof(float);
        uint32_t bytes = TY * ncp * sizeof(float) + 6 * row_bytes;
        if (xs + 3 < nx) bytes += TY * row_bytes;
        if (stage > 0) bytes += TY * row_bytes;
        fence_proxy_async_smem();
        mbar_expect_tx(bar, bytes);
#pragma unroll
        for (int r = 0; r < TY; ++r) {
            if (xs + 3 < nx) bulk_g2s(B.head[r], fsI + roff[r] + (xs + 3) * V + slab, row_bytes, bar);
            if (stage > 0) bulk_g2s(B.fnr[r], fnI + roff[r] + xs * V + slab, row_bytes, bar);
            bulk_g2s(B.coef[r], cI + (crow[r] + xs) * ncp, ncp * sizeof(float), bar);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int ylo = ((W.y0 - 3 + k) % ny + ny) % ny;
            const int yhi = (W.y0 + TY + k) % ny;
            bulk_g2s(B.halo[k], fsI + ylo * rs + xs * V + slab, row_bytes, bar);
            bulk_g2s(B.halo[3 + k], fsI + yhi * rs + xs * V + slab, row_bytes, bar);
        }
    };

    if (t == 0) {
        for (int d = 0; d < kDepth; ++d) mbar_init(&bars[d], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (t == 0)
        for (int xs = xa; xs < xa + kDepth - 1; ++xs) issue(xs);

    // scaled window of cells xa-3 .. xa+2 (wall ghosts of Sec. IV.C.3)
    float wr[TY][6];
#pragma unroll
    for (int r = 0; r < TY; ++r) {
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
    float2 w[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) w[j] = make_float2(wr[0][j], wr[1][j]);
    auto xface = [&](const float2* c) -> float2 {
        const float2 a = xpos ? c[0] : c[5], b = xpos ? c[1] : c[4], cc = xpos ? c[2] : c[3],
                     d = xpos ? c[3] : c[2], e = xpos ? c[4] : c[1];
        return ADV == HLB_WENO5_ ? weno5_scaled2(a, b, cc, d, e) : upwind2_face2(b, cc);
    };
    float2 Fm = __fmul2_rn(vxs, xface(w));

#pragma unroll 1
    for (int x = xa; x < xb; ++x) {
        const int step = x - xa;
        const Buf& B = buf[step % kDepth];
        mbar_wait(&bars[step % kDepth], (step / kDepth) & 1, g.err);
        const int b = x & 1;
#pragma unroll
        for (int j = 0; j < 5; ++j) w[j] = w[j + 1];
        const int h = x + 3;
        if (h < nx) w[5] = __fmul2_rn(make_float2(B.head[0][t], B.head[1][t]), f2(sv));
        else if (!xpos) w[5] = make_float2(nwr_g[0], nwr_g[1]);
        else if (h == nx) w[5] = __ffma2_rn(f2(3.0f), __fadd2_rn(w[4], __fmul2_rn(f2(-1.0f), w[3])), w[2]);
        else if (h == nx + 1)
            w[5] = __ffma2_rn(f2(6.0f), w[3], __ffma2_rn(f2(-8.0f), w[2], __fmul2_rn(f2(3.0f), w[1])));
        else w[5] = f2(0.0f);
        const float2 fc = __fmul2_rn(w[2], isv2);
        sF[b * S + t] = fc;
        // x faces
        const float2 Fp = __fmul2_rn(vxs, xface(w));
        const float2 divx = __fmul2_rn(__fadd2_rn(Fp, __fmul2_rn(f2(-1.0f), Fm)), f2(invdx[x]));
        Fm = Fp;
        // y faces (periodic): rows y0-3 .. y0+4 of column x, scaled
        float col[8];
#pragma unroll
        for (int k = 0; k < 3; ++k) col[k] = B.halo[k][t] * sv;
        col[3] = w[2].x;
        col[4] = w[2].y;
#pragma unroll
        for (int k = 0; k < 3; ++k) col[5 + k] = B.halo[3 + k][t] * sv;
        float2 G01;
        float G2;
        if (ADV == HLB_WENO5_) {
            if (ypos) {
                G01 = weno5_scaled2(make_float2(col[0], col[1]), make_float2(col[1], col[2]), make_float2(col[2], col[3]),
                                    make_float2(col[3], col[4]), make_float2(col[4], col[5]));
                G2 = weno5_scaled(col[2], col[3], col[4], col[5], col[6]);
            } else {
                G01 = weno5_scaled2(make_float2(col[5], col[6]), make_float2(col[4], col[5]), make_float2(col[3], col[4]),
                                    make_float2(col[2], col[3]), make_float2(col[1], col[2]));
                G2 = weno5_scaled(col[7], col[6], col[5], col[4], col[3]);
            }
        } else {
            if (ypos) {
                G01 = upwind2_face2(make_float2(col[1], col[2]), make_float2(col[2], col[3]));
                G2 = upwind2_face(col[3], col[4]);
            } else {
                G01 = upwind2_face2(make_float2(col[4], col[5]), make_float2(col[3], col[4]));
                G2 = upwind2_face(col[6], col[5]);
            }
        }
        const float2 divy = __fmul2_rn(vys, make_float2(G01.y - G01.x, G2 - G01.y));
        __syncthreads();
        if (t == 0) issue(x + kDepth - 1);
        const float2* fr = sF + b * S;
        float2 kxf = f2(0.0f), kyf = f2(0.0f);
#pragma unroll
        for (int i = 0; i < QX2; ++i) kxf = __ffma2_rn(kx[i], fr[jy * QX2 + i], kxf);
#pragma unroll
        for (int j = 0; j < VY; ++j) kyf = __ffma2_rn(ky[j], fr[j * QX2 + ix], kyf);
        const float* c0 = B.coef[0];
        const float* c1 = B.coef[1];
        const float2 feq = make_float2(c0[ix] * c0[QX2 + jy] * c0[csrc_z], c1[ix] * c1[QX2 + jy] * c1[csrc_z]);
        const float2 itau = make_float2(c0[csrc_t], c1[csrc_t]);
        // L = -div_x - div_y - (a_x K_x f + a_y K_y f) - (f - feq)/tau
        float2 L = __fadd2_rn(divx, divy);
        L = __ffma2_rn(ax2, kxf, L);
        L = __ffma2_rn(ay2, kyf, L);
        L = __ffma2_rn(__fadd2_rn(fc, __fmul2_rn(f2(-1.0f), feq)), itau, L);
        L = __fmul2_rn(f2(-1.0f), L);
        float2 out;
        if (stage == 0) {
            out = __ffma2_rn(dt2, L, fc);
        } else {
            const float2 fo_n = make_float2(B.fnr[0][t], B.fnr[1][t]);
            if (stage == 1)
                out = __ffma2_rn(f2(0.75f), fo_n, __fmul2_rn(f2(0.25f), __ffma2_rn(dt2, L, fc)));
            else
                out = __ffma2_rn(f2(1.0f / 3.0f), fo_n, __fmul2_rn(f2(2.0f / 3.0f), __ffma2_rn(dt2, L, fc)));
        }
        if (valid[0]) fov[roff[0] + x * V] = out.x;
        if (valid[1]) fov[roff[1] + x * V] = out.y;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_node(int precision, const GroupDev& g, const void* fs, cudaStream_t st) {
    const int block = 256;
    const int nrec = 5 * g.Nx + 1;
    const int nT = g.Qx * (g.Nx + 1) + g.VY * (g.Ny + 1) + g.VZ * (g.Nz + 1);
    const int ncoef = 2 * (g.Nx + 1) + (g.Ny + 1) + (g.Nz + 1);
    const size_t smem = (4 * g.V * (precision == HLB_FP64_ ? 8 : 4) + 7) / 8 * 8 +
                        sizeof(double) * (nrec + nT + kNodeBatch * (5 + 6 + ncoef));
    const int batches = (g.nnodes + kNodeBatch - 1) / kNodeBatch;
    const int grid = batches < 152 * 8 ? batches : 152 * 8;
    if (precision == HLB_FP64_) node_kernel<double><<<grid, block, smem, st>>>(g, (const double*)fs);
    else node_kernel<float><<<grid, block, smem, st>>>(g, (const float*)fs);
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
        march2_kernel<ADV, QX2, VY><<<nworks, QX2 * VY, march_smem_bytes<R, QX2, VY, TY>(), st>>>(
            g, works, (const float*)fs, (const float*)fn, (float*)fo, stage);
    } else {
        march_kernel<R, ADV, QX2, VY, TY><<<nworks, QX2 * VY, march_smem_bytes<R, QX2, VY, TY>(), st>>>(
            g, works, (const R*)fs, (const R*)fn, (R*)fo, stage);
    }
}

template <typename R, int ADV, int QX2, int VY, int TY>
static cudaError_t prepare_one() {
    if constexpr (sizeof(R) == 4 && TY == 2)
        return cudaFuncSetAttribute(march2_kernel<ADV, QX2, VY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)march_smem_bytes<R, QX2, VY, TY>());
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
