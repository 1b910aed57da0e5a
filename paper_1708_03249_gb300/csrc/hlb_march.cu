// The scalar marching stage kernel (sm_103a) and the dispatch of all
// marching kernels.
//
// march_kernel  one CTA per (instance, p_z slab, strip of TY rows, x-segment);
//               one thread per velocity of the slab (all 2Qx x Qy velocities of
//               one p_z, so both K contractions stay inside the CTA).  Each
//               thread marches along x holding a 6-cell register window of its
//               velocity per row, so every x-face flux (WENO-5 / upwind2) is
//               evaluated once and carried to the next cell.  Per x-step the
//               head cells, halo rows, f^n and the factor lines arrive by bulk
//               copies into a four-deep ring; the centre values are staged in
//               double-buffered shared memory behind one barrier, then the
//               force term sum_a a_a (K_a f) (Eqs. "eq:hh_Kk_hh", "eq:H_Kk";
//               K rows in registers), BGK, the y-faces (periodic) and the RK-3
//               combination (Eq. "eq:rk3") finish the node.
// It serves FP64 groups and FP32 1D slabs of fewer than 32 velocities; other
// FP32 groups run march_pair_kernel (2D, hlb_pair.cu) or march1_kernel (1D,
// hlb_line.cu).
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "hlb_device.cuh"
#include "hlb_internal.h"

namespace hlb {
namespace {

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
    static constexpr int NCPMAX = (QX2 + VY + 32 + 1 + 3 + 3) / 4 * 4;   // p_z up to 32, 1/tau, a_x a_y a_z
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
            // with a force field the node's a = a_uniform + a_field is in its factor line
            const R axr = g.has_field ? cr[g.field_off] : ax, ayr = g.has_field ? cr[g.field_off + 1] : ay;
            const R feq = cr[ix] * cr[QX2 + jy] * cr[csrc_z];
            const R itau = cr[csrc_t];
            const R L = -divx[r] - divy[r] - (axr * kxf + ayr * kyf) - (fc[r] - feq) * itau;
            R out;
            if constexpr (sizeof(R) == 4) {
                if (g.sround) {      // stochastic rounding of the stage output (hlb_device.cuh)
                    out = rk3_out_sr(stage, fc[r], -(dt * L), stage > 0 ? B.fnr[r][t] : R(0),
                                     sr_key(fov + roff[r] + x * V));
                    if (valid[r]) fov[roff[r] + x * V] = out;
                    continue;
                }
            }
            if (stage == 0) {
                out = fc[r] + dt * L;
            } else {
                const R fo_n = B.fnr[r][t];
                // c f^n + (1 - c) f' as f' + c (f^n - f'): the weights sum to
                // 1 exactly whatever the rounding of c
                const R fp = fc[r] + dt * L;
                out = fp + (stage == 1 ? R(0.75) : R(1.0 / 3.0)) * (fo_n - fp);
            }
            if (valid[r]) fov[roff[r] + x * V] = out;
        }
    }
    if (*sAbort && t == 0) {
        // a wait ran out at step xab: let the copies issued since (less a step
        // the test hook withheld) land before the CTA exits
        for (int s2 = xab - xa; s2 < xb - xa && s2 < xab - xa + kDepth - 1; ++s2)
            if (!(g.inject_stall && s2 == 1)) mbar_drain(&bars[s2 % kDepth], (s2 / kDepth) & 1, g.wait_ns);
    }
}


}  // namespace

#define HLB_MARCH_LIST(X)                                                              \
    X(float, 8, 1, 1) X(float, 16, 1, 1) X(double, 8, 4, 1) X(double, 8, 1, 1)             \
    X(double, 16, 8, 1) X(double, 32, 16, 1) X(double, 16, 1, 1)

namespace {
template <typename R, int ADV, int QX2, int VY, int TY>
void launch_one(const GroupDev& g, const Work* works, int nworks, const void* fs, const void* fn, void* fo,
                int stage, cudaStream_t st) {
    march_kernel<R, ADV, QX2, VY, TY><<<nworks, QX2 * VY, march_smem_bytes<R, QX2, VY, TY>(), st>>>(
        g, works, (const R*)fs, (const R*)fn, (R*)fo, stage);
}

template <typename R, int ADV, int QX2, int VY, int TY>
cudaError_t prepare_one() {
    return cudaFuncSetAttribute(march_kernel<R, ADV, QX2, VY, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)march_smem_bytes<R, QX2, VY, TY>());
}
}  // namespace

bool march_available(int precision, int adv, int QX2, int VY, int TY) {
    (void)adv;
    const bool dbl = precision == HLB_FP64_;
    if (!dbl && TY == 2) return pair_available(QX2, VY);
    if (!dbl && TY == 1 && line_available(QX2, VY)) return true;
#define HLB_AVAIL(RT, A, B, C) \
    if ((sizeof(RT) == 8) == dbl && QX2 == A && VY == B && TY == C) return true;
    HLB_MARCH_LIST(HLB_AVAIL)
#undef HLB_AVAIL
    return false;
}

cudaError_t prepare_march(int precision, int adv, int QX2, int VY, int TY, int form) {
    const bool dbl = precision == HLB_FP64_;
    if (!dbl && TY == 2) return prepare_pair(adv, QX2, VY, form);
    if (!dbl && TY == 1 && line_available(QX2, VY)) return prepare_line(adv, QX2, VY, form);
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
    if (!dbl && TY == 2) {
        launch_pair(adv, QX2, VY, g.force_form, g, works, nworks, fs, fn, fo, stage, st);
        return;
    }
    if (!dbl && TY == 1 && line_available(QX2, VY)) {
        launch_line(adv, QX2, VY, g.force_form, g, works, nworks, fs, fn, fo, stage, st);
        return;
    }
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
