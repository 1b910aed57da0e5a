// The 2D FP32 stage kernel (sm_103a): one CTA per (instance, p_z slab, strip of
// two rows, x-segment), one thread per velocity of the slab; see
// march_pair_kernel below.  Included by hlb_pair.cu (FMA force term) and
// hlb_tc.cu (force term on the tensor cores), which instantiate it.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <type_traits>

#include "hlb_device.cuh"
#include "hlb_internal.h"

namespace hlb {
namespace {

// FP32 pair kernel: each iteration advances two strip rows by two cells.
// The x faces pack the two rows into the lanes of f32x2 registers, the y faces
// pack the two cells, so every WENO evaluation is a full f32x2 one.  The
// window holds values pre-multiplied by the population's inverse weight, so
// that every WENO evaluation reads scaled stencils directly.
template <int QX2, int VY>
struct PairBuf {
    static constexpr int S = QX2 * VY;
    static constexpr int NCPMAX = (QX2 + VY + 32 + 1 + 3 + 3) / 4 * 4;   // p_z up to 32, 1/tau, a_x a_y a_z
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

// The force term: the FP32 FMA loop (FM = kForceFMA; a K rows duplicated into
// f32x2 pairs in shared memory), or warp-level tensor-core products (3xTF32
// or split-BF16, hlb_device.cuh) when both contractions tile into 16 x 8 x 8
// blocks.  On the 1024 x 512 channel with 16 x 8 x 8 velocities the 3xTF32
// form measured 3.74 ms per stage launch against 3.51 ms for the FMA loop (the
// fragment loads, splits and stores cost more issue slots than the packed
// FMAs they replace); the library picks the form per velocity set.
template <int QX2, int VY, int FM>
__host__ __device__ constexpr bool pair_uses_mma() { return FM != kForceFMA && QX2 % 8 == 0 && VY % 8 == 0; }


template <int QX2, int VY, int FM>
constexpr size_t pair_smem_bytes() {
    return kPairDepth * sizeof(PairBuf<QX2, VY>) + (pair_uses_mma<QX2, VY, FM>() ? 4 : 2) * VY * (QX2 + 1) * sizeof(float4) +
           (pair_uses_mma<QX2, VY, FM>() ? 0 : pair_kdup_pairs<QX2, VY>() * sizeof(float2)) + (kPairDepth + 3) * 8 + 16;
}

// FF = 1: the group has a per-node acceleration field; the a K rows are then
// plain K rows, K_x f and K_y f are kept apart and scaled per cell by the a_x,
// a_y of the factor lines (uniform plus field).  SR = 1: the stage outputs are
// rounded stochastically (rk3_out_sr2, hlb_device.cuh).
template <int ADV, int QX2, int VY, int FM, int FF, int SR = 0>
__global__ void __launch_bounds__(QX2 * VY, (QX2 * VY <= 32 ? 16 : (QX2 * VY <= 128 ? HLB_PAIR_MIN_BLOCKS : 2)))
march_pair_kernel(const GroupDev g, const Work* __restrict__ works, const float* __restrict__ fs,
                  const float* __restrict__ fn, float* __restrict__ fo, int stage) {
    constexpr int S = QX2 * VY;
    constexpr int QX = QX2 / 2;
    constexpr int SP = QX2 + 1;            // padded sF row: the K_x reads of a warp hit distinct banks
    using Buf = PairBuf<QX2, VY>;
    extern __shared__ __align__(128) unsigned char msm[];
    Buf* buf = reinterpret_cast<Buf*>(msm);
    constexpr bool kMMA = pair_uses_mma<QX2, VY, FM>();
    static_assert(!FF || !kMMA, "force fields take the FMA form");
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
    // FMA path: this thread's rows of a K, duplicated into pairs in shared
    // memory.  Tensor-core path: the B fragments of warp w's tiles in
    // registers (ForceMMA).
    ForceTC<FM, QX2, VY> mma;
    if constexpr (kMMA) {
        mma.load(K, (float)I.ax, (float)I.ay, warp, lane);
    } else {
        const float axf = FF ? 1.0f : (float)I.ax, ayf = FF ? 1.0f : (float)I.ay;
        for (int e = t; e < QX2 * QX2; e += S) sKd[(e / QX2) * KXR + e % QX2] = f2(axf * K[e]);
        for (int e = t; e < VY * VY; e += S) sKd[QX2 * KXR + (e / VY) * KYR + e % VY] = f2(ayf * K[QX2 * QX2 + e]);
    }
    (void)mma;
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
    // This thread's copy, fixed for the whole segment (22 copies per pair: 12
    // halo rows, 4 head rows, 4 f^n rows, 2 factor-line runs): the source of
    // pair 0 and its step per pair, the destination's offset in a buffer, and
    // the cell i of the pair it belongs to (the copy exists while i < cells of
    // the pair).  Computed once, so the per-pair issue is an add and a copy.
    const float* cp_src = nullptr;
    long long cp_step = 2LL * V;
    size_t cp_dst = 0;
    int cp_i = 0, cp_kind = 0;                         // 0 halo, 1 head, 2 f^n, 3 factor lines
    if (my_copy >= 0 && my_copy < 12) {
        const int i = my_copy / 6, k = my_copy % 6;
        const int yk = k < 3 ? ((W.y0 - 3 + k) % ny + ny) % ny : (W.y0 + k - 1) % ny;
        cp_src = fsI + (size_t)yk * rs + (size_t)(xa + i) * V + slab;
        cp_dst = offsetof(Buf, halo) + ((size_t)i * 6 + k) * S * sizeof(float);
        cp_i = i; cp_kind = 0;
    } else if (my_copy >= 12 && my_copy < 16) {
        const int i = (my_copy - 12) >> 1, r = my_copy & 1;
        cp_src = fsI + roff[r] + (size_t)(xa + 3 + i) * V + slab;
        cp_dst = offsetof(Buf, head) + ((size_t)i * 2 + r) * S * sizeof(float);
        cp_i = i; cp_kind = 1;
    } else if (my_copy >= 16 && my_copy < 20) {
        const int i = (my_copy - 16) >> 1, r = my_copy & 1;
        cp_src = fnI + roff[r] + (size_t)(xa + i) * V + slab;
        cp_dst = offsetof(Buf, fnr) + ((size_t)i * 2 + r) * S * sizeof(float);
        cp_i = i; cp_kind = 2;
    } else if (my_copy >= 20 && my_copy < 22) {
        const int r = my_copy - 20;
        cp_src = cI + (size_t)(crow[r] + xa) * ncp;
        cp_step = 2LL * ncp;
        cp_dst = offsetof(Buf, coef) + (size_t)r * Buf::NCPMAX * 2 * sizeof(float);
        cp_kind = 3;
    }
    auto issue = [&](int p) {
        if (my_copy < 0 || p >= npairs || (g.inject_stall && p == 1)) return;
        const int x0 = xa + 2 * p;
        const int n2 = min(2, xb - x0);
        bool go = cp_i < n2;
        uint32_t bytes = row_bytes;
        if (cp_kind == 1) go = go && x0 + 3 + cp_i < nx;
        else if (cp_kind == 2) go = go && stage > 0;
        else if (cp_kind == 3) bytes = n2 * ncp * (uint32_t)sizeof(float);
        fence_proxy_async_smem();
        if (go)
            bulk_g2s(reinterpret_cast<unsigned char*>(&buf[p % kPairDepth]) + cp_dst, cp_src + p * cp_step, bytes,
                     &bars[p % kPairDepth]);
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

    // Per pair: wait for its copies; write the centre values to sF[b] and
    // arrive on xch[b]; evaluate the faces (the other warps catch up
    // meanwhile); wait on xch[b]; then the force term, which reads every
    // warp's sF[b].  On the tensor-core path the force term sits between the
    // x and the y faces and its tiles are exchanged through xch2.  Passing
    // xch[b] of pair p also means every warp is done with pair p-1, so its
    // copy buffer is refilled then.  Every wait is bounded, so no warp can be
    // left waiting for good.
    float* fo0 = fov + roff[0] + (size_t)xa * V;       // this thread's outputs at cell x0, rows y0, y0+1
    float* fo1 = fov + roff[1] + (size_t)xa * V;
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
            mma.run(sF + b * VY * SP, sKx, sKy);
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
        float2 fk0, fk1, gy0 = f2(0.0f), gy1 = f2(0.0f);     // gy: K_y f apart (FF)
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
                float2& y0 = FF ? gy0 : fk0;
                float2& y1 = FF ? gy1 : fk1;
                y0 = __ffma2_rn(make_float2(kk.x, kk.y), make_float2(fa.x, fa.y), y0);
                y1 = __ffma2_rn(make_float2(kk.x, kk.y), make_float2(fa.z, fa.w), y1);
                y0 = __ffma2_rn(make_float2(kk.z, kk.w), make_float2(fb.x, fb.y), y0);
                y1 = __ffma2_rn(make_float2(kk.z, kk.w), make_float2(fb.z, fb.w), y1);
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
            float2 fk = i ? fk1 : fk0;
            if (FF) {      // a_x (K_x f) + a_y (K_y f) with the cells' a of the factor lines
                const int fo = g.field_off;
                fk = __ffma2_rn(make_float2(c0[fo + 1], c1[fo + 1]), i ? gy1 : gy0,
                                __fmul2_rn(make_float2(c0[fo], c1[fo]), fk));
            }
            float2 L = __fadd2_rn(__fadd2_rn(divx, divy), fk);
            L = __ffma2_rn(fsub2(fc, feq), itau, L);
            float2 out;      // fc + dt (-L), then the RK-3 combination (Eq. "eq:rk3")
            if constexpr (SR != 0) {
                const float2 fo_n = stage > 0 ? make_float2(B.fnr[i][0][vl], B.fnr[i][1][vl]) : f2(0.0f);
                out = rk3_out_sr2(stage, fc, __fmul2_rn(dt2, L), fo_n, sr_key(fo0 + (size_t)i * V));
            } else if (stage == 0) {
                out = fsub2(fc, __fmul2_rn(dt2, L));
            } else {
                const float2 fo_n = make_float2(B.fnr[i][0][vl], B.fnr[i][1][vl]);
                // c f^n + (1 - c) f' as f' + c (f^n - f'): the weights sum
                // to 1 exactly whatever the rounding of c (with 1/3 and 2/3
                // each rounded, FP32 gains mass 2^-25 per step)
                const float2 fp = fsub2(fc, __fmul2_rn(dt2, L));
                out = __ffma2_rn(f2(stage == 1 ? 0.75f : 1.0f / 3.0f), fsub2(fo_n, fp), fp);
            }
            if (valid[0]) fo0[(size_t)i * V] = out.x;
            if (valid[1]) fo1[(size_t)i * V] = out.y;
        }
        fo0 += 2 * (size_t)V;
        fo1 += 2 * (size_t)V;
        if (++slot == kPairDepth) { slot = 0; phase ^= 1u; }
    }
    if (*sAbort && t == 0) {
        // a wait ran out at pair pa: let the copies of the pairs registered
        // since (pa .. pa + kPairDepth - 2, less a pair the test hook
        // withheld) land before the CTA exits
        for (int s2 = pa; s2 < npairs && s2 < pa + kPairDepth - 1; ++s2)
            if (!(g.inject_stall && s2 == 1)) mbar_drain(&bars[s2 % kPairDepth], (s2 / kPairDepth) & 1, g.wait_ns);
    }
}


template <int ADV, int QX2, int VY, int FM, int FF = 0, int SR = 0>
void launch_pair_t(const GroupDev& g, const Work* works, int nworks, const void* fs, const void* fn, void* fo,
                   int stage, cudaStream_t st) {
    march_pair_kernel<ADV, QX2, VY, FM, FF, SR><<<nworks, QX2 * VY, pair_smem_bytes<QX2, VY, FM>(), st>>>(
        g, works, (const float*)fs, (const float*)fn, (float*)fo, stage);
}

template <int ADV, int QX2, int VY, int FM, int FF = 0, int SR = 0>
cudaError_t prepare_pair_t() {
    return cudaFuncSetAttribute(march_pair_kernel<ADV, QX2, VY, FM, FF, SR>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair_smem_bytes<QX2, VY, FM>());
}

}  // namespace
}  // namespace hlb
