// The persistent batched stage kernel (sm_103a) for 1D FP32 channel groups
// (many independent instances of one velocity set, Q_z absent): one launch
// advances every instance of the group by one RK-3 step (Eq. "eq:rk3").
//
// Work queue.  The work of a stage is, per instance: its node chunks (up to
// one cell per thread each: the moment sums of Eq. "eq:fmoms" with
// compensated FP32 sums, the equilibrium factor lines n g_x, g_y, 1/tau of
// App. A in double-float, and, for a chunk that holds a wall cell, the
// emitted density n_w = -sum_inc F / sum_emit p_x g^w of Eq. "eq:nplus_def"
// in FP64), then its x-segments (the line kernel's marching update: WENO-5 /
// upwind2 advection, the force term a . K f, BGK and the RK-3 combination).
// The items of a launch are numbered stage-major (in a stage: all node
// chunks, then all segments), and every CTA takes the next number from a
// counter in global memory until they run out.  Two counters per instance order the work: a node item of stage s
// waits until all segments of stage s-1 of its instance are done (it reads
// their output), a segment of stage s until all node items of stage s of its
// instance are done (it reads their factor lines and wall densities, and its
// halo and inputs come from stage s-1, done before those).  Every item an
// item waits for has a smaller number, so it was taken by a CTA that is
// running: the waits end whatever the grid size, there is no grid-wide
// barrier, and the stages of different instances overlap.  Every wait is
// bounded (%globaltimer): when one runs out the CTA records HLB_ETIMEOUT and
// raises the launch's abort flag, and every CTA leaves at its next item.
// State reads that may follow another CTA's writes bypass L1 (ld.global.cg;
// bulk copies read L2).
#include <cuda_runtime.h>

#include <cstdint>

#include "hlb_coef.cuh"
#include "hlb_device.cuh"
#include "hlb_internal.h"

namespace hlb {
namespace {

constexpr int kPDepth = 2;          // iterations in flight (copy buffers)

// Launch-shape knobs (measured choices): CTAs per SM that the 512-thread
// slabs are compiled for (2: 64 registers per thread), and whether the
// marching body is inlined into the item loop (it then reads the group
// descriptor from the kernel's parameter space, as the per-stage kernels do)
// or called.
#ifndef HLB_PERSIST_MIN_BLOCKS_512
#define HLB_PERSIST_MIN_BLOCKS_512 2
#endif
#ifndef HLB_PERSIST_MARCH_INLINE
#define HLB_PERSIST_MARCH_INLINE 1
#endif
#if HLB_PERSIST_MARCH_INLINE
#define HLB_MARCH_ITEM_ATTR __forceinline__
#else
#define HLB_MARCH_ITEM_ATTR __noinline__
#endif

// One iteration's inputs (four cells), filled by bulk copies.
template <int QX2, int VY>
struct PersistBuf {
    static constexpr int S = QX2 * VY;
    static constexpr int NCP = (QX2 + VY + 2 + 3 + 3) / 4 * 4;     // factor line (VZ = 1; field slots)
    float head[4][S];               // cells x0+3 .. x0+6
    float fnr[4][S];                // f^n of cells x0 .. x0+3 (stages 2, 3)
    float coef[4 * NCP];            // factor lines of cells x0 .. x0+3
};

constexpr size_t al16(size_t x) { return (x + 15) / 16 * 16; }

// Shared-memory layout (bytes), the same on the host and the device; every
// block starts on a 16-byte boundary (float4 and bulk-copy destinations).
template <int QX2, int VY, int FM, int NM>
struct PersistLayout {
    static constexpr int S = QX2 * VY, SP = QX2 + 1, QX = QX2 / 2;
    static constexpr bool kMMA = FM != kForceFMA && QX2 % 8 == 0 && VY % 8 == 0;
    static constexpr int NCP = PersistBuf<QX2, VY>::NCP;
    static constexpr int PX = (QX + 1) / 2, PY = (VY + 1) / 2;  // row pairs of the tables
    static constexpr size_t ring = 0;
    static constexpr size_t sF = al16(ring + kPDepth * sizeof(PersistBuf<QX2, VY>));
    static constexpr size_t sK = al16(sF + 2 * VY * SP * sizeof(float4));
    static constexpr size_t sSum =
        al16(sK + (kMMA ? 2 * VY * SP * sizeof(float4) : pair_kdup_pairs<QX2, VY>() * sizeof(float2)));
    static constexpr size_t sPt = al16(sSum + (size_t)S * 8 * sizeof(float));
    static constexpr size_t sRec = al16(sPt + (size_t)(PX + PY) * NM * sizeof(float4));
    static constexpr size_t sPv = al16(sRec + (5 * NM + 2) * sizeof(float2));
    static constexpr size_t sRed = al16(sPv + 4 * (QX2 + VY) * sizeof(float));   // p, its remainder, p^2, its remainder
    static constexpr size_t bars = al16(sRed + (2 * (S / 32) + 2) * sizeof(double));
    static constexpr size_t ints = al16(bars + (kPDepth + 3) * sizeof(unsigned long long));
    static constexpr size_t bytes = ints + 4 * sizeof(int);
    static_assert(sizeof(PersistBuf<QX2, VY>) % 16 == 0, "bulk-copy rows on 16-byte boundaries");
    static_assert(bytes <= 227 * 1024, "shared memory of one CTA");
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Orders this thread's earlier generic-proxy accesses of global memory (the
// acquire of another CTA's results) before its later async-proxy reads of it
// (bulk copies).
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// One factor line (hlb_coef.cuh), kept out of line so that its registers do
// not weigh on the callers'.
template <int NM>
__device__ __noinline__ void factor_line_call(const FactorDims d, double n, double ux, double uy, double T, double itau,
                                              const float4* sPx, const float4* sPy, const float2* sRec, float* line) {
    factor_line_df<NM>(d, n, ux, uy, 0.0, T, itau, sPx, sPy, sPy, sRec, line);
}

// Node item: cells [it.a, it.b) of instance it.inst of the stage's input.  Moment sums one warp per cell (compensated),
// factor lines one thread per cell into the group's factor-line buffer, and
// the emitted density of each wall whose cell the chunk holds.
template <int ADV, int QX2, int VY, int FM, int NM>
__device__ __forceinline__ void node_item(const GroupDev& g, const PersistArgs& pa, const PersistItem it, int stage) {
    using L = PersistLayout<QX2, VY, FM, NM>;
    constexpr int S = QX2 * VY, NW = S / 32, V = S;
    extern __shared__ __align__(128) unsigned char msm[];
    float* sSum = reinterpret_cast<float*>(msm + L::sSum);
    const float4* sPt = reinterpret_cast<const float4*>(msm + L::sPt);
    const float2* sRec = reinterpret_cast<const float2*>(msm + L::sRec);
    const float* sPv = reinterpret_cast<const float*>(msm + L::sPv);
    double* sRed = reinterpret_cast<double*>(msm + L::sRed);
    const InstDev& I = g.inst[it.inst];
    const float* fin = pa.buf[stage == 0 ? pa.cur : (stage == 1 ? (pa.cur + 1) % 3 : (pa.cur + 2) % 3)] + I.f_off;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nx = I.nx, n = it.b - it.a;
    for (int c = warp; c < n; c += NW) {
        const float* fc = fin + (size_t)(it.a + c) * V;
        float s0 = 0, c0 = 0, s1 = 0, c1 = 0, s2 = 0, c2 = 0, s3 = 0, c3 = 0;
#pragma unroll
        for (int m = 0; m < S / 32; ++m) {
            const int vv = lane + 32 * m;
            const float f = __ldcg(fc + vv);
            // the FP64 momenta as rounding plus remainder (the node pass's
            // sums_kernel does the same; a fixed half-ulp error per velocity
            // is a heat and momentum source under strong collisions)
            const int ix = vv % QX2, jy = QX2 + vv / QX2;
            constexpr int P = QX2 + VY;
            csum_add(s0, c0, f);
            csum_add(s1, c1, __fmaf_rn(sPv[P + ix], f, sPv[ix] * f));
            csum_add(s2, c2, __fmaf_rn(sPv[P + jy], f, sPv[jy] * f));
            csum_add(s3, c3, __fmaf_rn(sPv[3 * P + ix] + sPv[3 * P + jy], f,
                                       __fmaf_rn(sPv[2 * P + ix], f, sPv[2 * P + jy] * f)));
        }
        csum_warp(s0, c0);
        csum_warp(s1, c1);
        csum_warp(s2, c2);
        csum_warp(s3, c3);
        if (lane == 0) {
            float* o = sSum + c * 8;
            o[0] = s0; o[1] = c0; o[2] = s1; o[3] = c1; o[4] = s2; o[5] = c2; o[6] = s3; o[7] = c3;
        }
    }
    const bool wl = it.a == 0, wr = it.b == nx;
    if (wl || wr) {
        // the incident fluxes at the wall faces from the quadratically
        // extrapolated ghosts (Sec. IV.C.3): thread t holds velocity t
        const int ix = t % QX2;
        const double pxd = g.pd[ix];
        const bool inc = pxd < 0 ? wl : wr;
        double accL = 0.0, accR = 0.0;
        if (inc) {
            const float sv = static_cast<const float*>(g.wscale)[t];
            const size_t a0 = pxd < 0 ? 0 : (size_t)(nx - 1) * V, st = pxd < 0 ? (size_t)V : (size_t)0 - (size_t)V;
            const float f0 = __ldcg(fin + a0 + t) * sv, f1 = __ldcg(fin + a0 + st + t) * sv,
                        f2v = __ldcg(fin + a0 + 2 * st + t) * sv;
            float face;
            if (ADV == HLB_WENO5_) {
                const float d = 3.0f * f0 - 3.0f * f1 + f2v, e = 6.0f * f0 - 8.0f * f1 + 3.0f * f2v;
                face = weno5_scaled(f2v, f1, f0, d, e);
            } else {
                face = upwind2_face<float>(f1, f0);
            }
            const double F = (double)((static_cast<const float*>(g.p)[ix] * (1.0f / sv)) * face);
            if (pxd < 0) accL = F; else accR = F;
        }
        accL = warp_sum(accL);
        accR = warp_sum(accR);
        if (lane == 0) { sRed[warp] = accL; sRed[NW + warp] = accR; }
    }
    __syncthreads();
    if (t == 0 && (wl || wr)) {
        double sl = 0.0, sr = 0.0;
        for (int w = 0; w < NW; ++w) { sl += sRed[w]; sr += sRed[NW + w]; }
        if (wl) g.nw[(size_t)I.row_off * 2 + 0] = -sl / I.den_left;
        if (wr) g.nw[(size_t)I.row_off * 2 + 1] = -sr / I.den_right;
    }
    if (t < n) {
        const float* m = sSum + t * 8;
        const double nn = (double)m[0] + (double)m[1], in = 1.0 / nn;
        const double ux = ((double)m[2] + (double)m[3]) * in, uy = ((double)m[4] + (double)m[5]) * in;
        const double T = ((double)m[6] + (double)m[7] - nn * (ux * ux + uy * uy)) * in / (double)g.D;
        float* line = static_cast<float*>(g.coef) + (size_t)(I.node_off + it.a + t) * g.ncp;
        factor_line_call<NM>(FactorDims(g), nn, ux, uy, T, nn * I.inv_Kn, sPt, sPt + L::PX * (g.Nx + 1), sRec, line);
    }
}

// March item: segment works[j] of stage `stage` (the line kernel's marching
// update of cells [W.xa, W.xb)) from the stage input, f^n and into the stage
// output of the launch's buffers; P0 the pipeline iterations consumed by
// earlier items (ring slot and barrier parities).  Returns P0 plus this
// item's iterations; on a failed wait it raises *sAbort (after the copies in
// flight have landed).
template <int ADV, int QX2, int VY, int FM, int NM>
__device__ HLB_MARCH_ITEM_ATTR uint32_t march_item(const GroupDev& g, const PersistArgs& a, const Work* works, int j,
                                                    int stage, uint32_t P0) {
    using L = PersistLayout<QX2, VY, FM, NM>;
    constexpr int S = QX2 * VY;
    constexpr int QX = QX2 / 2, SP = QX2 + 1, NCP = L::NCP;
    constexpr int KXR = QX2 + 2, KYR = VY + 2;
    constexpr int NW = S / 32;
    constexpr bool kMMA = L::kMMA;
    using Buf = PersistBuf<QX2, VY>;
    extern __shared__ __align__(128) unsigned char msm[];
    Buf* buf = reinterpret_cast<Buf*>(msm + L::ring);
    float4* sF = reinterpret_cast<float4*>(msm + L::sF);
    float4* sKx = reinterpret_cast<float4*>(msm + L::sK);
    float4* sKy = sKx + VY * SP;
    float2* sKd = reinterpret_cast<float2*>(msm + L::sK);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(msm + L::bars);
    unsigned long long* xch = bars + kPDepth;
    unsigned long long* xch2 = xch + 2;
    int* sAbort = reinterpret_cast<int*>(msm + L::ints) + 1;
    const Work W = works[j];
    const InstDev& I = g.inst[W.inst];
    // buffer roles of the stage: S -> X, (S, X) -> Y, (S, Y) -> X
    const float* fsI = a.buf[stage == 0 ? a.cur : (stage == 1 ? (a.cur + 1) % 3 : (a.cur + 2) % 3)] + I.f_off;
    float* foI = a.buf[stage == 1 ? (a.cur + 2) % 3 : (a.cur + 1) % 3] + I.f_off;
    const float* fnI = a.buf[a.cur] + I.f_off;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
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
    const int vl = jy * QX2 + ix, v = vl, V = S;
    const int nx = I.nx;
    const float* P = static_cast<const float*>(g.p);
    const float vx = P[ix];
    const bool xpos = ix < QX;
    const float sv = static_cast<const float*>(g.wscale)[v];
    const float isv = 1.0f / sv;
    const float* K = static_cast<const float*>(g.K);
    ForceTC<FM, QX2, VY> mma;
    if constexpr (kMMA) {
        mma.load(K, (float)I.ax, (float)I.ay, warp, lane);
    } else {
        const float axf = (float)I.ax, ayf = (float)I.ay;
        for (int e = t; e < QX2 * QX2; e += S) sKd[(e / QX2) * KXR + e % QX2] = f2(axf * K[e]);
        for (int e = t; e < VY * VY; e += S) sKd[QX2 * KXR + (e / VY) * KYR + e % VY] = f2(ayf * K[QX2 * QX2 + e]);
    }
    (void)mma;
    (void)NW;
    const float2 dt2 = f2((float)I.dt), isv2 = f2(isv), vxs = f2(vx * isv);
    const float* invdx = static_cast<const float*>(g.inv_dx) + I.dx_off;
    float* fov = foI + v;
    const float* cI = static_cast<const float*>(g.coef) + (size_t)I.node_off * NCP;
    const int csrc_t = QX2 + VY + 1;
    const float* gw = static_cast<const float*>(g.gw) + I.gw_off;
    const float nwl = (float)__ldcg(g.nw + (size_t)I.row_off * 2 + 0) * gw[v] * sv;      // scaled emitted ghosts
    const float nwr = (float)__ldcg(g.nw + (size_t)I.row_off * 2 + 1) * gw[V + v] * sv;
    const int xa = W.xa, xb = W.xb;
    const int niter = (xb - xa + 3) >> 2;
    const uint32_t row_bytes = S * sizeof(float);

    auto expect = [&](int p) {                      // thread 0
        if (p >= niter) return;
        const int x0 = xa + 4 * p;
        const int n4 = min(4, xb - x0);
        int nhead = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) nhead += (k < n4 && x0 + 3 + k < nx);
        uint32_t bytes = nhead * row_bytes + n4 * NCP * (uint32_t)sizeof(float);
        if (stage > 0) bytes += n4 * row_bytes;
        mbar_expect_tx(&bars[(P0 + p) % kPDepth], bytes);
    };
    auto issue = [&](int p) {                       // warp 0
        if (t >= 32 || p >= niter) return;
        const int x0 = xa + 4 * p;
        const int n4 = min(4, xb - x0);
        Buf& B = buf[(P0 + p) % kPDepth];
        unsigned long long* bar = &bars[(P0 + p) % kPDepth];
        fence_proxy_async_smem();
        if (lane < 4) {
            if (lane < n4 && x0 + 3 + lane < nx) bulk_g2s(B.head[lane], fsI + (x0 + 3 + lane) * V, row_bytes, bar);
        } else if (lane < 8) {
            const int i = lane - 4;
            if (stage > 0 && i < n4) bulk_g2s(B.fnr[i], fnI + (x0 + i) * V, row_bytes, bar);
        } else if (lane == 8) {
            bulk_g2s(B.coef, cI + (size_t)x0 * NCP, n4 * NCP * (uint32_t)sizeof(float), bar);
        }
    };
    if (t == 0)
        for (int p = 0; p < kPDepth - 1; ++p) expect(p);
    __syncthreads();
    for (int p = 0; p < kPDepth - 1; ++p) issue(p);

    // scaled window of cells xa-3 .. xa+6 (wall ghosts of Sec. IV.C.3)
    float w[10];
    {
        const float* f = fsI + v;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const int x = xa - 3 + j;
            float val;
            if (x >= 0 && x < nx) val = __ldcg(f + x * V) * sv;
            else if (x < 0) {
                if (xpos) val = nwl;
                else if (x < -2) val = 0.0f;          // never read by a negative velocity
                else {
                    const float f0 = __ldcg(f) * sv, f1 = __ldcg(f + V) * sv, f2v = __ldcg(f + 2 * V) * sv;
                    val = x == -1 ? 3.0f * f0 - 3.0f * f1 + f2v : 6.0f * f0 - 8.0f * f1 + 3.0f * f2v;
                }
            } else if (!xpos) val = nwr;
            else if (x > nx + 1) val = 0.0f;          // never read by a positive velocity
            else {
                const float f0 = __ldcg(f + (nx - 1) * V) * sv, f1 = __ldcg(f + (nx - 2) * V) * sv,
                            f2v = __ldcg(f + (nx - 3) * V) * sv;
                val = x == nx ? 3.0f * f0 - 3.0f * f1 + f2v : 6.0f * f0 - 8.0f * f1 + 3.0f * f2v;
            }
            w[j] = val;
        }
#pragma unroll
        for (int j = 6; j < 10; ++j) w[j] = 0.0f;
    }
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
    auto face1 = [&](const float* c) -> float {
        if (ADV == HLB_WENO5_)
            return xpos ? weno5_scaled(c[0], c[1], c[2], c[3], c[4]) : weno5_scaled(c[5], c[4], c[3], c[2], c[1]);
        return xpos ? 1.5f * c[2] - 0.5f * c[1] : 1.5f * c[3] - 0.5f * c[4];
    };
    auto enter = [&](int h, const float* hd, float m1, float m2, float m3, float m4) -> float {
        if (h < nx) return hd[vl] * sv;
        if (!xpos) return nwr;                                  // emitted at the right wall
        if (h == nx) return 3.0f * (m1 - m2) + m3;
        if (h == nx + 1) return 6.0f * m2 - 8.0f * m3 + 3.0f * m4;
        return 0.0f;                                            // never read by v > 0
    };
    float Fm = vx * isv * face1(w);

    int pa = 0;
#pragma unroll 1
    for (int p = 0; p < niter; ++p) {
        const uint32_t Pg = P0 + p;
        const int slot = Pg % kPDepth;
        const uint32_t phase = (Pg / kPDepth) & 1u;
        const int x0 = xa + 4 * p;
        const int n4 = min(4, xb - x0);
        pa = p;
        const Buf& B = buf[slot];
        if (!mbar_wait(&bars[slot], phase, g.err, g.wait_ns)) *sAbort = 1;
        if (t == 0) expect(p + kPDepth - 1);
        const int b = Pg & 1;
#pragma unroll
        for (int k = 0; k < 4; ++k) w[6 + k] = enter(x0 + 3 + k, B.head[k], w[5 + k], w[4 + k], w[3 + k], w[2 + k]);
        const float2 fc01 = __fmul2_rn(make_float2(w[3], w[4]), isv2);
        const float2 fc23 = __fmul2_rn(make_float2(w[5], w[6]), isv2);
        sF[(b * VY + jy) * SP + ix] = make_float4(fc01.x, fc01.y, fc23.x, fc23.y);
        __syncwarp();
        if (lane == 0) mbar_arrive(&xch[b]);
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
        if (!mbar_wait(&xch[b], (Pg >> 1) & 1, g.err, g.wait_ns)) *sAbort = 1;
        if (*sAbort) break;
        issue(p + kPDepth - 1);
        const float4* fr = sF + b * VY * SP;
        float2 fk01 = f2(0.0f), fk23 = f2(0.0f);
        if constexpr (kMMA) {
            mma.run(fr, sKx, sKy);
            __syncwarp();
            if (lane == 0) mbar_arrive(xch2);
            if (!mbar_wait(xch2, Pg & 1, g.err, g.wait_ns)) *sAbort = 1;
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
                    fk01 = __ffma2_rn(make_float2(kk.x, kk.y), make_float2(fa.x, fa.y), fk01);
                    fk23 = __ffma2_rn(make_float2(kk.x, kk.y), make_float2(fa.z, fa.w), fk23);
                    fk01 = __ffma2_rn(make_float2(kk.z, kk.w), make_float2(fb.x, fb.y), fk01);
                    fk23 = __ffma2_rn(make_float2(kk.z, kk.w), make_float2(fb.z, fb.w), fk23);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {                       // cells x0+2q, x0+2q+1
            if (2 * q >= n4) break;
            const float* c0 = B.coef + (2 * q) * NCP;
            const float* c1 = c0 + NCP;                     // stale beyond n4: its results are not stored
            const float2 feq = __fmul2_rn(make_float2(c0[ix], c1[ix]), make_float2(c0[QX2 + jy], c1[QX2 + jy]));
            const float2 itau = make_float2(c0[csrc_t], c1[csrc_t]);
            const float2 fc = q ? fc23 : fc01;
            const float2 Lv = __ffma2_rn(fsub2(fc, feq), itau, __fadd2_rn(q ? divx23 : divx01, q ? fk23 : fk01));
            float2 out;
            if (g.sround) {      // stochastic rounding of the stage output (hlb_device.cuh)
                const float2 fo_n = stage > 0 ? make_float2(B.fnr[2 * q][vl], B.fnr[2 * q + 1][vl]) : f2(0.0f);
                out = rk3_out_sr2(stage, fc, __fmul2_rn(dt2, Lv), fo_n, sr_key(fov + (x0 + 2 * q) * V));
            } else if (stage == 0) {
                out = fsub2(fc, __fmul2_rn(dt2, Lv));
            } else {
                const float2 fo_n = make_float2(B.fnr[2 * q][vl], B.fnr[2 * q + 1][vl]);
                // c f^n + (1 - c) f' as f' + c (f^n - f'): the weights sum
                // to 1 exactly whatever the rounding of c (with 1/3 and 2/3
                // each rounded, FP32 gains mass 2^-25 per step)
                const float2 fp = fsub2(fc, __fmul2_rn(dt2, Lv));
                out = __ffma2_rn(f2(stage == 1 ? 0.75f : 1.0f / 3.0f), fsub2(fo_n, fp), fp);
            }
            fov[(x0 + 2 * q) * V] = out.x;
            if (2 * q + 1 < n4) fov[(x0 + 2 * q + 1) * V] = out.y;
        }
    }
    if (*sAbort && t == 0) {
        // let the copies registered after the failed wait land before leaving
        for (int s2 = pa; s2 < niter && s2 < pa + kPDepth - 1; ++s2)
            mbar_drain(&bars[(P0 + s2) % kPDepth], ((P0 + s2) / kPDepth) & 1, g.wait_ns);
    }
    return P0 + niter;
}

template <int ADV, int QX2, int VY, int FM, int NM>
__global__ void __launch_bounds__(QX2 * VY, (QX2 * VY <= 32 ? 16 : (QX2 * VY <= 128 ? 8 : HLB_PERSIST_MIN_BLOCKS_512)))
persist_line_kernel(const GroupDev g, const Work* __restrict__ works, const PersistArgs a) {
    using L = PersistLayout<QX2, VY, FM, NM>;
    constexpr int S = QX2 * VY, NW = S / 32;
    static_assert(S % 32 == 0, "the exchange barriers count whole warps");
    constexpr int PX = L::PX, PY = L::PY;
    extern __shared__ __align__(128) unsigned char msm[];
    float4* sPt = reinterpret_cast<float4*>(msm + L::sPt);
    float2* sRec = reinterpret_cast<float2*>(msm + L::sRec);
    float* sPv = reinterpret_cast<float*>(msm + L::sPv);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(msm + L::bars);
    unsigned long long* xch = bars + kPDepth;
    unsigned long long* xch2 = xch + 2;
    int* sItem = reinterpret_cast<int*>(msm + L::ints);
    int* sAbort = sItem + 1;
    int* sSkip = sItem + 2;
    const int t = threadIdx.x;
    const int Nx = g.Nx, Ny = g.Ny, Qx = g.Qx;

    // the tables every item reads: momenta, the equilibrium tables as row
    // pairs (dot2_pair layout), the recurrence
    for (int i = t; i < QX2 + VY; i += S) {
        const double p = g.pd[i], p2 = p * p;
        const float hi = (float)p, hi2 = (float)p2;
        sPv[i] = hi;
        sPv[QX2 + VY + i] = (float)(p - (double)hi);
        sPv[2 * (QX2 + VY) + i] = hi2;
        sPv[3 * (QX2 + VY) + i] = (float)(p2 - (double)hi2);
    }
    {
        const float2* Tx = g.Tf;
        const float2* Ty = Tx + Qx * (Nx + 1);
        for (int i = t; i < PX * (Nx + 1); i += S) {
            const int k = 2 * (i / (Nx + 1)), l = i % (Nx + 1);
            const float2 p0 = Tx[k * (Nx + 1) + l];
            const float2 p1 = k + 1 < Qx ? Tx[(k + 1) * (Nx + 1) + l] : make_float2(0.0f, 0.0f);
            sPt[i] = make_float4(p0.x, p1.x, p0.y, p1.y);
        }
        for (int i = t; i < PY * (Ny + 1); i += S) {
            const int k = 2 * (i / (Ny + 1)), l = i % (Ny + 1);
            const float2 p0 = g.Qy ? Ty[k * (Ny + 1) + l] : make_float2(0.0f, 0.0f);
            const float2 p1 = g.Qy && k + 1 < VY ? Ty[(k + 1) * (Ny + 1) + l] : make_float2(0.0f, 0.0f);
            sPt[PX * (Nx + 1) + i] = make_float4(p0.x, p1.x, p0.y, p1.y);
        }
        for (int i = t; i < 5 * Nx + 1; i += S) sRec[i] = g.recf[i];
    }
    if (t == 0) {
        for (int d = 0; d < kPDepth; ++d) mbar_init(&bars[d], 1);
        mbar_init(&xch[0], NW);
        mbar_init(&xch[1], NW);
        mbar_init(xch2, NW);
        *sAbort = 0;
        *sSkip = 0;
        mbar_init_fence();
    }
    __syncthreads();

    const int total = 3 * a.nitems;
    uint32_t P0 = 0;                  // pipeline iterations consumed so far (ring slot, barrier parities)
#pragma unroll 1
    for (;;) {
        if (t == 0) *sItem = *(volatile int*)a.abort ? total : atomicAdd(a.head, 1);
        __syncthreads();
        const int item = *sItem;
        if (item >= total) break;
        const int s = item / a.nitems;
        const PersistItem it = a.items[item - s * a.nitems];
        // wait (bounded) for what the item reads
        if (t == 0) {
            const unsigned* ctr = it.kind == 0 ? a.prog_march + it.inst : a.prog_node + it.inst;
            const unsigned need = it.kind == 0 ? (unsigned)(s * a.nseg[it.inst]) : (unsigned)((s + 1) * a.nchunk[it.inst]);
            if (ld_acquire_gpu(ctr) < need) {
                const unsigned long long t0 = global_ns();
                while (ld_acquire_gpu(ctr) < need) {
                    if (*(volatile int*)a.abort) { *sSkip = 1; break; }
                    if (global_ns() - t0 > g.wait_ns) {
                        atomicExch(g.err, 4);       // HLB_ETIMEOUT
                        atomicExch(a.abort, 1);
                        *sSkip = 1;
                        break;
                    }
                    __nanosleep(256);
                }
            }
        }
        __syncthreads();
        if (*sSkip) break;
        if (it.kind == 0) {
            node_item<ADV, QX2, VY, FM, NM>(g, a, it, s);
        } else {
            // the lanes that issue bulk copies order the acquire above before
            // their async-proxy reads of the other CTAs' outputs
            if (t < 32) fence_proxy_async_global();
            P0 = march_item<ADV, QX2, VY, FM, NM>(g, a, works, it.a, s, P0);
        }
        // every thread is done with the item (normally or after a failed wait)
        __syncthreads();
        if (*sAbort) {
            if (t == 0) atomicExch(a.abort, 1);
            break;
        }
        if (t == 0) {
            __threadfence();
            // test hook: the first item's count never comes (a barrier that never opens)
            const bool withhold = g.inject_stall && item == 0;
            if (!withhold) atomicAdd(it.kind == 0 ? a.prog_node + it.inst : a.prog_march + it.inst, 1u);
        }
    }
}

template <int ADV, int QX2, int VY, int FM, int NM>
cudaError_t prepare_one() {
    return cudaFuncSetAttribute(persist_line_kernel<ADV, QX2, VY, FM, NM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PersistLayout<QX2, VY, FM, NM>::bytes);
}

template <int ADV, int QX2, int VY, int FM, int NM>
int occupancy_one() {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, persist_line_kernel<ADV, QX2, VY, FM, NM>, QX2 * VY,
                                                      PersistLayout<QX2, VY, FM, NM>::bytes) != cudaSuccess)
        return 0;
    return per;
}

template <int ADV, int QX2, int VY, int FM, int NM>
void launch_one(const GroupDev& g, const Work* works, const PersistArgs& a, int grid, cudaStream_t st) {
    persist_line_kernel<ADV, QX2, VY, FM, NM>
        <<<grid, QX2 * VY, PersistLayout<QX2, VY, FM, NM>::bytes, st>>>(g, works, a);
}

}  // namespace

// (2 Qx, Qy, force-term form, coefficient bound NM > max(Nx, Ny)): the line
// kernel's slabs with the form HLB_FP32 picks for them
#define HLB_PERSIST_LIST(X) X(8, 4, 0, 8) X(16, 8, 0, 8) X(32, 16, 1, 16) X(32, 1, 0, 16)

bool persist_available(int QX2, int VY, int form, int Nmax) {
#define HLB_AV(A, B, F, N) if (QX2 == A && VY == B && form == F && Nmax < N) return true;
    HLB_PERSIST_LIST(HLB_AV)
#undef HLB_AV
    return false;
}

size_t persist_smem_bytes(int QX2, int VY, int form) {
#define HLB_SM(A, B, F, N) if (QX2 == A && VY == B && form == F) return PersistLayout<A, B, F, N>::bytes;
    HLB_PERSIST_LIST(HLB_SM)
#undef HLB_SM
    return 0;
}

cudaError_t prepare_persist(int adv, int QX2, int VY, int form, int* blocks_per_sm) {
#define HLB_PR(A, B, F, N)                                                                                  \
    if (QX2 == A && VY == B && form == F) {                                                                 \
        cudaError_t e = adv == HLB_WENO5_ ? prepare_one<HLB_WENO5_, A, B, F, N>()                          \
                                          : prepare_one<HLB_UPWIND2_, A, B, F, N>();                        \
        if (e != cudaSuccess) return e;                                                                     \
        *blocks_per_sm = adv == HLB_WENO5_ ? occupancy_one<HLB_WENO5_, A, B, F, N>()                       \
                                           : occupancy_one<HLB_UPWIND2_, A, B, F, N>();                     \
        return *blocks_per_sm > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;                            \
    }
    HLB_PERSIST_LIST(HLB_PR)
#undef HLB_PR
    return cudaErrorInvalidValue;
}

void launch_persist(int adv, int QX2, int VY, int form, const GroupDev& g, const Work* works, const PersistArgs& a,
                    int grid, cudaStream_t st) {
#define HLB_LA(A, B, F, N)                                                                      \
    if (QX2 == A && VY == B && form == F) {                                                     \
        if (adv == HLB_WENO5_) launch_one<HLB_WENO5_, A, B, F, N>(g, works, a, grid, st);       \
        else launch_one<HLB_UPWIND2_, A, B, F, N>(g, works, a, grid, st);                       \
        return;                                                                                 \
    }
    HLB_PERSIST_LIST(HLB_LA)
#undef HLB_LA
}

}  // namespace hlb
