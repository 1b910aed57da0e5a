// The 1D FP32 stage kernel (sm_103a): one CTA per (instance row, p_z slab,
// x-segment), one thread per velocity of the slab.  Four cells per iteration:
// the x faces two at a time in f32x2 WENO evaluations, the force term and the
// update of cell pairs in f32x2, the four centre values exchanged as one
// 16-byte word, so every a K row loaded from shared memory serves four cells.
// Scaled branch-free WENO-5, a split exchange barrier and a bulk-copy ring, as
// in the 2D pair kernel.
// Included by hlb_line.cu (FMA force term) and hlb_tc.cu (force term on the
// tensor cores), which instantiate it.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "hlb_device.cuh"
#include "hlb_internal.h"

namespace hlb {
namespace {

// One iteration's inputs (four cells), filled by bulk copies.
template <int QX2, int VY>
struct LineBuf {
    static constexpr int S = QX2 * VY;
    static constexpr int NCPMAX = (QX2 + VY + 32 + 1 + 3 + 3) / 4 * 4;   // p_z up to 32, 1/tau, a_x a_y a_z
    float head[4][S];           // cells x0+3 .. x0+6
    float fnr[4][S];            // f^n of cells x0 .. x0+3 (stages 2, 3)
    float coef[4 * NCPMAX];     // factor lines of cells x0 .. x0+3
};

constexpr int kLineDepth = 2;   // iterations in flight

// The force term: the FP32 FMA loop (FM = kForceFMA), or the tensor cores
// (3xTF32 or split-BF16, hlb_device.cuh) for slabs that tile into 16 x 8 x 8
// blocks.  For 32 x 16 slabs the FMA form is bound by shared-memory
// wavefronts (each thread reads its a K row and the fibre's four-cell words
// for every term); the tensor-core form reads each fibre value once per tile
// and keeps a K in registers.  The library picks the form per velocity set.
template <int QX2, int VY, int FM>
__host__ __device__ constexpr bool line_uses_mma() { return FM != kForceFMA && QX2 % 8 == 0 && VY % 8 == 0; }

template <int QX2, int VY, int FM>
constexpr size_t line_smem_bytes() {
    return kLineDepth * sizeof(LineBuf<QX2, VY>) + (line_uses_mma<QX2, VY, FM>() ? 4 : 2) * VY * (QX2 + 1) * sizeof(float4) +
           (line_uses_mma<QX2, VY, FM>() ? 0 : pair_kdup_pairs<QX2, VY>() * sizeof(float2)) + (kLineDepth + 3) * 8 + 16;
}

// FF = 1: the group has a per-node acceleration field; the a K rows are then
// plain K rows, K_x f and K_y f are kept apart and scaled per cell by the a_x,
// a_y of the factor lines (uniform plus field).  SR = 1: the stage outputs are
// rounded stochastically (rk3_out_sr2, hlb_device.cuh).
template <int ADV, int QX2, int VY, int FM, int FF, int SR = 0>
__global__ void __launch_bounds__(QX2 * VY, (QX2 * VY <= 32 ? 16 : (QX2 * VY <= 128 ? 8 : (QX2 * VY <= 256 ? 4 : 2))))
march1_kernel(const GroupDev g, const Work* __restrict__ works, const float* __restrict__ fs,
              const float* __restrict__ fn, float* __restrict__ fo, int stage) {
    constexpr int S = QX2 * VY;
    static_assert(S % 32 == 0, "the exchange barrier counts whole warps");
    constexpr int QX = QX2 / 2;
    constexpr int SP = QX2 + 1;              // padded sF row (float4: cells x0 .. x0+3)
    constexpr int KXR = QX2 + 2, KYR = VY + 2;
    using Buf = LineBuf<QX2, VY>;
    constexpr bool kMMA = line_uses_mma<QX2, VY, FM>();
    static_assert(!FF || !kMMA, "force fields take the FMA form");
    extern __shared__ __align__(128) unsigned char msm[];
    Buf* buf = reinterpret_cast<Buf*>(msm);
    float4* sF = reinterpret_cast<float4*>(msm + kLineDepth * sizeof(Buf));    // [2][VY][SP]
    float4* sKx = sF + 2 * VY * SP;                   // [VY][SP]: a_x K_x f, four cells (tensor-core path)
    float4* sKy = sKx + VY * SP;                      // [VY][SP]: a_y K_y f
    float2* sKd = reinterpret_cast<float2*>(sF + (kMMA ? 4 : 2) * VY * SP);     // FMA path: duplicated a K rows
    unsigned long long* bars =
        reinterpret_cast<unsigned long long*>(sKd + (kMMA ? 0 : pair_kdup_pairs<QX2, VY>()));
    unsigned long long* xch = bars + kLineDepth;                                 // [2]: sF[b] written by every warp
    unsigned long long* xch2 = xch + 2;                                          // sKx, sKy written by every warp
    int* sAbort = reinterpret_cast<int*>(xch2 + 1);

    const Work W = works[blockIdx.x];
    const InstDev& I = g.inst[W.inst];
    const int t = threadIdx.x;
    // Thread -> velocity: when one sign half of p_x fills whole warps, each
    // warp takes one half (warp-uniform upwind orientation); otherwise ix
    // runs fastest.
    constexpr bool kHalf = (QX * VY) % 32 == 0;
    int ix, jy;
    if (kHalf) {
        const int h = t / (QX * VY), rr = t % (QX * VY);
        ix = h * QX + rr % QX;
        jy = rr / QX;
    } else {
        ix = t % QX2;
        jy = t / QX2;
    }
    const int kz = W.kz;
    const int vl = jy * QX2 + ix;
    const int V = g.V, nx = I.nx, ncp = g.ncp;
    const int v = kz * S + vl;
    const float* P = static_cast<const float*>(g.p);
    const float vx = P[ix];
    const bool xpos = ix < QX;
    const float sv = static_cast<const float*>(g.wscale)[v];
    const float isv = 1.0f / sv;
    const float* K = static_cast<const float*>(g.K);
    ForceTC<FM, QX2, VY> mma;
    if constexpr (kMMA) {
        mma.load(K, (float)I.ax, (float)I.ay, t >> 5, t & 31);
    } else {
        const float axf = FF ? 1.0f : (float)I.ax, ayf = FF ? 1.0f : (float)I.ay;
        for (int e = t; e < QX2 * QX2; e += S) sKd[(e / QX2) * KXR + e % QX2] = f2(axf * K[e]);
        for (int e = t; e < VY * VY; e += S) sKd[QX2 * KXR + (e / VY) * KYR + e % VY] = f2(ayf * K[QX2 * QX2 + e]);
    }
    (void)mma;
    const float2 dt2 = f2((float)I.dt), isv2 = f2(isv), vxs = f2(vx * isv);
    const float* invdx = static_cast<const float*>(g.inv_dx) + I.dx_off;
    const float* fsI = fs + I.f_off;
    const float* fnI = fn + I.f_off;
    float* fov = fo + I.f_off + v;
    const float* cI = static_cast<const float*>(g.coef) + (size_t)I.node_off * ncp;
    const int csrc_z = QX2 + VY + kz, csrc_t = QX2 + VY + g.VZ;
    const float* gw = static_cast<const float*>(g.gw) + I.gw_off;
    const int row = W.y0;                                   // 0 for a 1D instance
    const int roff = row * nx * V, crow = row * nx;
    const float nwl = (float)g.nw[(size_t)(I.row_off + row) * 2 + 0] * gw[v] * sv;        // scaled emitted ghosts
    const float nwr = (float)g.nw[(size_t)(I.row_off + row) * 2 + 1] * gw[V + v] * sv;
    const int xa = W.xa, xb = W.xb;
    const int niter = (xb - xa + 3) >> 2;
    const int slab = kz * S;
    const uint32_t row_bytes = S * sizeof(float);
    const int lane = t & 31;

    // warp 0 issues the (at most nine) copies of an iteration, one per lane;
    // thread 0 registers the byte count before any of them
    auto expect = [&](int p) {
        if (p >= niter || (g.inject_stall && p == 1)) return;   // test hook: iteration 1 never arrives
        const int x0 = xa + 4 * p;
        const int n4 = min(4, xb - x0);
        int nhead = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) nhead += (k < n4 && x0 + 3 + k < nx);
        uint32_t bytes = nhead * row_bytes + n4 * ncp * (uint32_t)sizeof(float);
        if (stage > 0) bytes += n4 * row_bytes;
        mbar_expect_tx(&bars[p % kLineDepth], bytes);
    };
    auto issue = [&](int p) {
        if (t >= 32 || p >= niter || (g.inject_stall && p == 1)) return;
        const int x0 = xa + 4 * p;
        const int n4 = min(4, xb - x0);
        Buf& B = buf[p % kLineDepth];
        unsigned long long* bar = &bars[p % kLineDepth];
        fence_proxy_async_smem();
        if (lane < 4) {
            if (lane < n4 && x0 + 3 + lane < nx)
                bulk_g2s(B.head[lane], fsI + roff + (x0 + 3 + lane) * V + slab, row_bytes, bar);
        } else if (lane < 8) {
            const int i = lane - 4;
            if (stage > 0 && i < n4) bulk_g2s(B.fnr[i], fnI + roff + (x0 + i) * V + slab, row_bytes, bar);
        } else if (lane == 8) {
            bulk_g2s(B.coef, cI + (size_t)(crow + x0) * ncp, n4 * ncp * (uint32_t)sizeof(float), bar);
        }
    };

    if (t == 0) {
        for (int d = 0; d < kLineDepth; ++d) mbar_init(&bars[d], 1);
        mbar_init(&xch[0], S / 32);
        mbar_init(&xch[1], S / 32);
        mbar_init(xch2, S / 32);
        *sAbort = 0;
        mbar_init_fence();
        for (int p = 0; p < kLineDepth - 1; ++p) expect(p);
    }
    __syncthreads();
    for (int p = 0; p < kLineDepth - 1; ++p) issue(p);

    // scaled window of cells xa-3 .. xa+6 (wall ghosts of Sec. IV.C.3); w[0..5] filled here
    float w[10];
    {
        const float* f = fsI + v + roff;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const int x = xa - 3 + j;
            float val;
            if (x >= 0 && x < nx) val = f[x * V] * sv;
            else if (x < 0) {
                if (xpos) val = nwl;
                else if (x < -2) val = 0.0f;          // never read by a negative velocity
                else {
                    const float f0 = f[0] * sv, f1 = f[V] * sv, f2v = f[2 * V] * sv;
                    val = x == -1 ? 3.0f * f0 - 3.0f * f1 + f2v : 6.0f * f0 - 8.0f * f1 + 3.0f * f2v;
                }
            } else if (!xpos) val = nwr;
            else if (x > nx + 1) val = 0.0f;          // never read by a positive velocity
            else {
                const float f0 = f[(nx - 1) * V] * sv, f1 = f[(nx - 2) * V] * sv, f2v = f[(nx - 3) * V] * sv;
                val = x == nx ? 3.0f * f0 - 3.0f * f1 + f2v : 6.0f * f0 - 8.0f * f1 + 3.0f * f2v;
            }
            w[j] = val;
        }
#pragma unroll
        for (int j = 6; j < 10; ++j) w[j] = 0.0f;
    }
    // the faces (c[2], c[3]) and (c[3], c[4]) of c[0..6], packed
    auto faces2 = [&](const float* c) -> float2 {
        if (ADV == HLB_WENO5_) {
            if (xpos)
                return weno5_scaled2(make_float2(c[0], c[1]), make_float2(c[1], c[2]), make_float2(c[2], c[3]),
                                     make_float2(c[3], c[4]), make_float2(c[4], c[5]));
            return weno5_scaled2(make_float2(c[5], c[6]), make_float2(c[4], c[5]), make_float2(c[3], c[4]),
                                 make_float2(c[2], c[3]), make_float2(c[1], c[2]));
        }
        return xpos ? upwind2_face2(make_float2(c[1], c[2]), make_float2(c[2], c[3]))
                    : upwind2_face2(make_float2(c[4], c[5]), make_float2(c[3], c[4]));
    };
    // the face between c[2] and c[3] of c[0..5]
    auto face1 = [&](const float* c) -> float {
        if (ADV == HLB_WENO5_)
            return xpos ? weno5_scaled(c[0], c[1], c[2], c[3], c[4]) : weno5_scaled(c[5], c[4], c[3], c[2], c[1]);
        return xpos ? 1.5f * c[2] - 0.5f * c[1] : 1.5f * c[3] - 0.5f * c[4];
    };
    // a cell entering the window (head row hd; right-wall ghosts from the
    // cells nx-1, nx-2, nx-3 already in the window)
    auto enter = [&](int h, const float* hd, float m1, float m2, float m3, float m4) -> float {
        if (h < nx) return hd[vl] * sv;
        if (!xpos) return nwr;                                  // emitted at the right wall
        if (h == nx) return 3.0f * (m1 - m2) + m3;
        if (h == nx + 1) return 6.0f * m2 - 8.0f * m3 + 3.0f * m4;
        return 0.0f;                                            // never read by v > 0
    };
    float Fm = vx * isv * face1(w);                             // face xa-1/2

    // Per iteration (cells x0 .. x0+3): wait for its copies; write the four
    // centre values to sF[b] and arrive on xch[b]; evaluate the faces; wait on
    // xch[b] (every warp is then done with the previous iteration, whose copy
    // buffer is refilled); the force term reads every warp's sF[b].  Every
    // wait is bounded.
    int pa = 0, slot = 0;
    uint32_t phase = 0;
#pragma unroll 1
    for (int p = 0; p < niter; ++p) {
        const int x0 = xa + 4 * p;
        const int n4 = min(4, xb - x0);
        pa = p;
        const Buf& B = buf[slot];
        if (!mbar_wait(&bars[slot], phase, g.err, g.wait_ns)) *sAbort = 1;
        if (t == 0) expect(p + kLineDepth - 1);
        const int b = p & 1;
#pragma unroll
        for (int k = 0; k < 4; ++k) w[6 + k] = enter(x0 + 3 + k, B.head[k], w[5 + k], w[4 + k], w[3 + k], w[2 + k]);
        const float2 fc01 = __fmul2_rn(make_float2(w[3], w[4]), isv2);      // cells x0, x0+1
        const float2 fc23 = __fmul2_rn(make_float2(w[5], w[6]), isv2);      // cells x0+2, x0+3
        sF[(b * VY + jy) * SP + ix] = make_float4(fc01.x, fc01.y, fc23.x, fc23.y);
        __syncwarp();
        if (lane == 0) mbar_arrive(&xch[b]);
        // faces x0+1/2 .. x0+7/2 in two packed evaluations; x0-1/2 carried
        const float2 Fp01 = __fmul2_rn(vxs, faces2(w + 1));
        const float2 Fp23 = __fmul2_rn(vxs, faces2(w + 3));
        float idx[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) idx[k] = k < n4 ? invdx[x0 + k] : 0.0f;
        const float2 divx01 = __fmul2_rn(fsub2(Fp01, make_float2(Fm, Fp01.x)), make_float2(idx[0], idx[1]));
        const float2 divx23 = __fmul2_rn(fsub2(Fp23, make_float2(Fp01.y, Fp23.x)), make_float2(idx[2], idx[3]));
        Fm = Fp23.y;
#pragma unroll
        for (int j = 0; j < 6; ++j) w[j] = w[j + 4];
        if (!mbar_wait(&xch[b], (p >> 1) & 1, g.err, g.wait_ns)) *sAbort = 1;
        if (*sAbort) break;
        issue(p + kLineDepth - 1);
        // a_x K_x f + a_y K_y f at the four cells
        const float4* fr = sF + b * VY * SP;
        float2 fk01 = f2(0.0f), fk23 = f2(0.0f), gy01 = f2(0.0f), gy23 = f2(0.0f);   // gy: K_y f apart (FF)
        if constexpr (kMMA) {
            // every warp's tiles, exchanged through xch2 (sKx, sKy are free
            // again: every warp passed xch[b] after reading them last time)
            mma.run(fr, sKx, sKy);
            __syncwarp();
            if (lane == 0) mbar_arrive(xch2);
            if (!mbar_wait(xch2, p & 1, g.err, g.wait_ns)) *sAbort = 1;
            const float4 ex = sKx[jy * SP + ix], ey = sKy[jy * SP + ix];
            fk01 = __fadd2_rn(make_float2(ex.x, ex.y), make_float2(ey.x, ey.y));
            fk23 = __fadd2_rn(make_float2(ex.z, ex.w), make_float2(ey.z, ey.w));
        } else {
            const float4* kxr = reinterpret_cast<const float4*>(sKd + ix * KXR);
            const float4* kyr = reinterpret_cast<const float4*>(sKd + QX2 * KXR + jy * KYR);
#pragma unroll
            for (int i = 0; i < QX2; i += 2) {
                const float4 kk = kxr[i >> 1], fa = fr[jy * SP + i], fb = fr[jy * SP + i + 1];
                fk01 = __ffma2_rn(make_float2(kk.x, kk.y), make_float2(fa.x, fa.y), fk01);
                fk23 = __ffma2_rn(make_float2(kk.x, kk.y), make_float2(fa.z, fa.w), fk23);
                fk01 = __ffma2_rn(make_float2(kk.z, kk.w), make_float2(fb.x, fb.y), fk01);
                fk23 = __ffma2_rn(make_float2(kk.z, kk.w), make_float2(fb.z, fb.w), fk23);
            }
            if (VY > 1) {
#pragma unroll
                for (int j = 0; j < VY; j += 2) {
                    const float4 kk = kyr[j >> 1], fa = fr[j * SP + ix], fb = fr[(j + 1) * SP + ix];
                    float2& y01 = FF ? gy01 : fk01;
                    float2& y23 = FF ? gy23 : fk23;
                    y01 = __ffma2_rn(make_float2(kk.x, kk.y), make_float2(fa.x, fa.y), y01);
                    y23 = __ffma2_rn(make_float2(kk.x, kk.y), make_float2(fa.z, fa.w), y23);
                    y01 = __ffma2_rn(make_float2(kk.z, kk.w), make_float2(fb.x, fb.y), y01);
                    y23 = __ffma2_rn(make_float2(kk.z, kk.w), make_float2(fb.z, fb.w), y23);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {                       // cells x0+2q, x0+2q+1
            if (2 * q >= n4) break;
            const float* c0 = B.coef + (2 * q) * ncp;
            const float* c1 = c0 + ncp;                     // stale beyond n4: its results are not stored
            const float2 feq = __fmul2_rn(__fmul2_rn(make_float2(c0[ix], c1[ix]), make_float2(c0[QX2 + jy], c1[QX2 + jy])),
                                          make_float2(c0[csrc_z], c1[csrc_z]));
            const float2 itau = make_float2(c0[csrc_t], c1[csrc_t]);
            const float2 fc = q ? fc23 : fc01;
            // L = -div_x - (a_x K_x f + a_y K_y f) - (f - feq)/tau
            float2 fk = q ? fk23 : fk01;
            if (FF) {      // a_x (K_x f) + a_y (K_y f) with the cells' a of the factor lines
                const int fo = g.field_off;
                fk = __ffma2_rn(make_float2(c0[fo + 1], c1[fo + 1]), q ? gy23 : gy01,
                                __fmul2_rn(make_float2(c0[fo], c1[fo]), fk));
            }
            const float2 L = __ffma2_rn(fsub2(fc, feq), itau, __fadd2_rn(q ? divx23 : divx01, fk));
            float2 out;  // fc + dt (-L), then the RK-3 combination (Eq. "eq:rk3")
            if constexpr (SR != 0) {
                const float2 fo_n = stage > 0 ? make_float2(B.fnr[2 * q][vl], B.fnr[2 * q + 1][vl]) : f2(0.0f);
                out = rk3_out_sr2(stage, fc, __fmul2_rn(dt2, L), fo_n, sr_key(fov + roff + (x0 + 2 * q) * V));
            } else if (stage == 0) {
                out = fsub2(fc, __fmul2_rn(dt2, L));
            } else {
                const float2 fo_n = make_float2(B.fnr[2 * q][vl], B.fnr[2 * q + 1][vl]);
                // c f^n + (1 - c) f' as f' + c (f^n - f'): the weights sum
                // to 1 exactly whatever the rounding of c (with 1/3 and 2/3
                // each rounded, FP32 gains mass 2^-25 per step)
                const float2 fp = fsub2(fc, __fmul2_rn(dt2, L));
                out = __ffma2_rn(f2(stage == 1 ? 0.75f : 1.0f / 3.0f), fsub2(fo_n, fp), fp);
            }
            fov[roff + (x0 + 2 * q) * V] = out.x;
            if (2 * q + 1 < n4) fov[roff + (x0 + 2 * q + 1) * V] = out.y;
        }
        if (++slot == kLineDepth) { slot = 0; phase ^= 1u; }
    }
    if (*sAbort && t == 0) {
        // a wait ran out at iteration pa: let the copies registered since
        // (less an iteration the test hook withheld) land before the CTA exits
        for (int s2 = pa; s2 < niter && s2 < pa + kLineDepth - 1; ++s2)
            if (!(g.inject_stall && s2 == 1)) mbar_drain(&bars[s2 % kLineDepth], (s2 / kLineDepth) & 1, g.wait_ns);
    }
}

template <int ADV, int QX2, int VY, int FM, int FF = 0, int SR = 0>
void launch_line_t(const GroupDev& g, const Work* works, int nworks, const void* fs, const void* fn, void* fo,
                   int stage, cudaStream_t st) {
    march1_kernel<ADV, QX2, VY, FM, FF, SR><<<nworks, QX2 * VY, line_smem_bytes<QX2, VY, FM>(), st>>>(
        g, works, (const float*)fs, (const float*)fn, (float*)fo, stage);
}

template <int ADV, int QX2, int VY, int FM, int FF = 0, int SR = 0>
cudaError_t prepare_line_t() {
    return cudaFuncSetAttribute(march1_kernel<ADV, QX2, VY, FM, FF, SR>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)line_smem_bytes<QX2, VY, FM>());
}

}  // namespace
}  // namespace hlb
