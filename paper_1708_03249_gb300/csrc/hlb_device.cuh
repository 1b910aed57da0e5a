// Device helpers shared by the stage kernels (included by the .cu files).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "hlb_internal.h"

namespace hlb {

constexpr double kSqrt2Pi = 2.5066282746310005024157652848110;

template <typename R> __device__ __forceinline__ R rabs(R x) { return x < R(0) ? -x : x; }
template <typename R> __device__ __forceinline__ R rmax(R a, R b) { return a > b ? a : b; }

// 2^-k with m = x 2^k, x in [1/2, 1) (k clamped so that the result is finite).
__device__ __forceinline__ double pow2_inverse(double m) {
    int k;
    frexp(m, &k);
    return ldexp(1.0, -max(k, -1020));
}
__device__ __forceinline__ float pow2_inverse(float m) {
    int k;
    frexpf(m, &k);
    return ldexpf(1.0f, -max(k, -120));
}

// WENO-5 face value per unit velocity for a positive velocity: (a..e) are the
// values at cells i-2..i+2 of face i+1/2 (Sec. IV.C.2).  No epsilon: the
// weights are delta_q/sigma_q^2 normalised, or, if any sigma_q vanishes,
// delta_q over the vanishing set (Tab. "weno").
//  - The sigmas are formed from the stencil values times the power of two
//    that brings their largest magnitude into [1/2, 1) (the weights do not
//    change under a common scaling, and a power of two scales exactly), so
//    that small populations do not underflow sigma.
//  - delta_q/sigma_q^2 is evaluated as delta_q (sigma_min/sigma_q)^2, the
//    same ratios multiplied by sigma_min^2: every factor lies in [0, 1], so
//    nothing overflows, and a sigma far above sigma_min underflows to a zero
//    weight, its exact limit.
template <typename R>
__device__ __forceinline__ R weno5_face(R a, R b, R c, R d, R e) {
    const R F1 = (R(2) * a - R(7) * b + R(11) * c) * R(1.0 / 6.0);
    const R F2 = (-b + R(5) * c + R(2) * d) * R(1.0 / 6.0);
    const R F3 = (R(2) * c + R(5) * d - e) * R(1.0 / 6.0);
    const R m = rmax(rmax(rmax(rabs(a), rabs(b)), rmax(rabs(c), rabs(d))), rabs(e));
    if (m == R(0)) return R(0);
    const R r = pow2_inverse(m);
    const R A = a * r, B = b * r, C = c * r, Dd = d * r, E = e * r;
    const R t1 = A - R(2) * B + C, t2 = A - R(4) * B + R(3) * C;
    const R t3 = B - R(2) * C + Dd, t4 = B - Dd;
    const R t5 = C - R(2) * Dd + E, t6 = R(3) * C - R(4) * Dd + E;
    const R s1 = R(13.0 / 12.0) * t1 * t1 + R(0.25) * t2 * t2;
    const R s2 = R(13.0 / 12.0) * t3 * t3 + R(0.25) * t4 * t4;
    const R s3 = R(13.0 / 12.0) * t5 * t5 + R(0.25) * t6 * t6;
    const R smin = s1 < s2 ? (s1 < s3 ? s1 : s3) : (s2 < s3 ? s2 : s3);
    R w1, w2, w3;
    if (smin == R(0)) {
        w1 = s1 == R(0) ? R(0.1) : R(0);
        w2 = s2 == R(0) ? R(0.6) : R(0);
        w3 = s3 == R(0) ? R(0.3) : R(0);
    } else {
        const R u1 = smin / s1, u2 = smin / s2, u3 = smin / s3;
        w1 = R(0.1) * u1 * u1;
        w2 = R(0.6) * u2 * u2;
        w3 = R(0.3) * u3 * u3;
    }
    return (w1 * F1 + w2 * F2 + w3 * F3) / (w1 + w2 + w3);
}

// Same weights as weno5_face, for the marching kernel: the smoothness
// indicators are formed from the stencil values times a fixed per-velocity
// scale ``sv`` (the inverse quadrature weight of the population, so that the
// scaled values are O(n)), and the reciprocals use the fast FP32 unit.  A
// non-zero sigma below 1e-30 (far under FP32's resolution of an O(1) scaled
// stencil) is treated as 1e-30, which ties it with any other such sigma.
template <typename R>
__device__ __forceinline__ R weno5_face_sv(R a, R b, R c, R d, R e, R sv);

template <>
__device__ __forceinline__ double weno5_face_sv<double>(double a, double b, double c, double d, double e,
                                                        double sv) {
    (void)sv;
    return weno5_face<double>(a, b, c, d, e);
}

template <>
__device__ __forceinline__ float weno5_face_sv<float>(float a, float b, float c, float d, float e, float sv) {
    const float F1 = (2.0f * a - 7.0f * b + 11.0f * c) * (1.0f / 6.0f);
    const float F2 = (-b + 5.0f * c + 2.0f * d) * (1.0f / 6.0f);
    const float F3 = (2.0f * c + 5.0f * d - e) * (1.0f / 6.0f);
    const float A = a * sv, B = b * sv, C = c * sv, Dd = d * sv, E = e * sv;
    const float t1 = A - 2.0f * B + C, t2 = A - 4.0f * B + 3.0f * C;
    const float t3 = B - 2.0f * C + Dd, t4 = B - Dd;
    const float t5 = C - 2.0f * Dd + E, t6 = 3.0f * C - 4.0f * Dd + E;
    const float s1 = (13.0f / 12.0f) * t1 * t1 + 0.25f * t2 * t2;
    const float s2 = (13.0f / 12.0f) * t3 * t3 + 0.25f * t4 * t4;
    const float s3 = (13.0f / 12.0f) * t5 * t5 + 0.25f * t6 * t6;
    float w1, w2, w3;
    if (fminf(s1, fminf(s2, s3)) == 0.0f) {
        w1 = s1 == 0.0f ? 0.1f : 0.0f;
        w2 = s2 == 0.0f ? 0.6f : 0.0f;
        w3 = s3 == 0.0f ? 0.3f : 0.0f;
    } else {
        const float c1 = fmaxf(s1, 1e-30f), c2 = fmaxf(s2, 1e-30f), c3 = fmaxf(s3, 1e-30f);
        const float m = fminf(c1, fminf(c2, c3));
        const float u1 = m * __fdividef(1.0f, c1), u2 = m * __fdividef(1.0f, c2), u3 = m * __fdividef(1.0f, c3);
        w1 = 0.1f * u1 * u1;
        w2 = 0.6f * u2 * u2;
        w3 = 0.3f * u3 * u3;
    }
    return (w1 * F1 + w2 * F2 + w3 * F3) * __fdividef(1.0f, w1 + w2 + w3);
}

template <typename R>
__device__ __forceinline__ R upwind2_face(R b, R c) { return R(1.5) * c - R(0.5) * b; }

// Shared-memory footprint, in f32x2 pairs, of the a_x K_x and a_y K_y rows of
// the FP32 marching kernels: every entry duplicated into a pair, rows padded
// by two pairs so that a warp's rows fall in distinct banks.
template <int QX2, int VY>
__host__ __device__ constexpr int pair_kdup_pairs() { return QX2 * (QX2 + 2) + VY * (VY + 2); }

// ---------------------------------------------------------------------------
// The force term a_x K_x f + a_y K_y f of one exchange tile on the tensor cores
// (warp-level mma.sync, three TF32 products, FP32 accumulation).  The tile is
// sF[VY][QX2 + 1] of float4 (four cells or cell/row combinations c per
// velocity).  The two contractions are written as F^T K^T:
//   X rows (j_y, c), 4 VY of them, columns i_x:  (a_x K_x f)^T,
//   Y rows (i_x, c), 4 QX2 of them, columns j_y: (a_y K_y f)^T.
// Warp w computes one 16 x 8 tile of each (exactly S/32 tiles per product
// when 8 | QX2 and 8 | VY) and stores it into sKx / sKy in the layout of sF.
// The B fragments (a K)^T stay in registers, split into TF32 hi and lo parts.
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    // D += A B, m16n8k8, A row-major 16 x 8, B column-major 8 x 8
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

// x = hi + lo with hi the TF32 truncation of x (its low 13 mantissa bits
// cleared: one logic operation, where the rounding conversion takes several);
// lo = x - hi is exact and below 2^-10 |x|.
__device__ __forceinline__ void split_tf32_rz(float x, uint32_t& hi, uint32_t& lo) {
    hi = __float_as_uint(x) & 0xffffe000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
}

// D += A B in three TF32 products (A_lo B_hi + A_hi B_lo + A_hi B_hi), close
// to an FP32 product; a[k] are FP32 values (split here by truncation, once per
// use), b{0,1}{h,l} fragments split once by rounding.
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const float (&a)[4], uint32_t b0h, uint32_t b0l,
                                           uint32_t b1h, uint32_t b1l) {
    uint32_t ah[4], al[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) split_tf32_rz(a[k], ah[k], al[k]);
    mma_tf32(d, al[0], al[1], al[2], al[3], b0h, b1h);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], b0l, b1l);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], b0h, b1h);
}

template <int QX2, int VY>
struct ForceMMA {
    static constexpr int XS = QX2 / 8, YS = VY / 8, SP = QX2 + 1;   // k-steps; padded tile row
    static constexpr int XA = XS > 0 ? XS : 1, YA = YS > 0 ? YS : 1;
    uint32_t bxh[XA][2], bxl[XA][2], byh[YA][2], byl[YA][2];
    int mX, nX, mY, nY, gq, tq;

    // K: K_x (QX2 x QX2) then K_y (VY x VY), row-major; ax, ay the acceleration
    __device__ __forceinline__ void load(const float* K, float axf, float ayf, int warp, int lane) {
        mX = warp / XS; nX = warp % XS; mY = warp / YS; nY = warp % YS;
        gq = lane >> 2; tq = lane & 3;
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
    }

    __device__ __forceinline__ void run(const float4* fr, float4* sKx, float4* sKy) const {
        const float* ff = reinterpret_cast<const float*>(fr);
        float* kxo = reinterpret_cast<float*>(sKx);
        float* kyo = reinterpret_cast<float*>(sKy);
        const int R0 = 16 * mX + gq, jy0 = R0 >> 2, rx = R0 & 3;       // X rows: (j_y, c)
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
        const int Q0 = 16 * mY + gq, ix0 = Q0 >> 2, ry = Q0 & 3;       // Y rows: (i_x, c)
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
    }
};

// ---------------------------------------------------------------------------
// The same force term with split-BF16 products: every FP32 operand x is
// written as three bf16 terms, x = h + m + l + r with |m| <= 2^-9 |h|,
// |l| <= 2^-18 |x| and |r| <= 2^-27 |x| (each split step subtracts exactly in
// FP32), and A B is formed from the six products whose order is at most
// 2^-18 (h h, h m, m h, m m, h l, l h), smallest first, on mma.sync m16n8k8
// with bf16 inputs and FP32 accumulation.  The dropped products (m l, l m,
// l l) are below 2^-26 of |A| |B|, so the contraction keeps FP32 accuracy.
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    // D += A B, m16n8k8, A row-major 16 x 8 (two bf16 per register), B column-major 8 x 8
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

// (x0, x1) -> bf16x2 words h, m, l (x0 in the low halves): x_k = h_k + m_k + l_k
// up to 2^-27 |x_k|.  cvt.rn.bf16x2.f32 packs its first source in the high half.
__device__ __forceinline__ void split_bf16x3(float x0, float x1, uint32_t& h, uint32_t& m, uint32_t& l) {
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(x1), "f"(x0));
    const float r0 = x0 - __uint_as_float(h << 16), r1 = x1 - __uint_as_float(h & 0xffff0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(m) : "f"(r1), "f"(r0));
    const float s0 = r0 - __uint_as_float(m << 16), s1 = r1 - __uint_as_float(m & 0xffff0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(s1), "f"(s0));
}

__device__ __forceinline__ void mma_bf16x6(float (&d)[4], uint32_t ah0, uint32_t am0, uint32_t al0, uint32_t ah1,
                                           uint32_t am1, uint32_t al1, uint32_t bh, uint32_t bm, uint32_t bl) {
    mma_bf16(d, am0, am1, bm);
    mma_bf16(d, ah0, ah1, bl);
    mma_bf16(d, al0, al1, bh);
    mma_bf16(d, ah0, ah1, bm);
    mma_bf16(d, am0, am1, bh);
    mma_bf16(d, ah0, ah1, bh);
}

// Same tiles, layout and interface as ForceMMA; fragments of m16n8k8 bf16:
// A rows g and g+8, columns 2t and 2t+1; B rows (k) 2t and 2t+1, column g.
template <int QX2, int VY>
struct ForceMMABF16 {
    static constexpr int XS = QX2 / 8, YS = VY / 8, SP = QX2 + 1;
    static constexpr int XA = XS > 0 ? XS : 1, YA = YS > 0 ? YS : 1;
    uint32_t bx[XA][3], by[YA][3];       // (h, m, l) of each B fragment
    int mX, nX, mY, nY, gq, tq;

    __device__ __forceinline__ void load(const float* K, float axf, float ayf, int warp, int lane) {
        mX = warp / XS; nX = warp % XS; mY = warp / YS; nY = warp % YS;
        gq = lane >> 2; tq = lane & 3;
#pragma unroll
        for (int ks = 0; ks < XS; ++ks) {    // B[k][n] = a_x K_x[8 nX + n][8 ks + k]
            const float* r = K + (8 * nX + gq) * QX2 + 8 * ks + 2 * tq;
            split_bf16x3(axf * r[0], axf * r[1], bx[ks][0], bx[ks][1], bx[ks][2]);
        }
#pragma unroll
        for (int ks = 0; ks < YS; ++ks) {    // B[k][n] = a_y K_y[8 nY + n][8 ks + k]
            const float* r = K + QX2 * QX2 + (8 * nY + gq) * VY + 8 * ks + 2 * tq;
            split_bf16x3(ayf * r[0], ayf * r[1], by[ks][0], by[ks][1], by[ks][2]);
        }
    }

    __device__ __forceinline__ void run(const float4* fr, float4* sKx, float4* sKy) const {
        const float* ff = reinterpret_cast<const float*>(fr);
        float* kxo = reinterpret_cast<float*>(sKx);
        float* kyo = reinterpret_cast<float*>(sKy);
        const int R0 = 16 * mX + gq, jy0 = R0 >> 2, rx = R0 & 3;       // X rows: (j_y, c)
        float dx[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int ks = 0; ks < XS; ++ks) {
            const int i0 = 8 * ks + 2 * tq;
            uint32_t h0, m0, l0, h1, m1, l1;
            split_bf16x3(ff[(jy0 * SP + i0) * 4 + rx], ff[(jy0 * SP + i0 + 1) * 4 + rx], h0, m0, l0);
            split_bf16x3(ff[((jy0 + 2) * SP + i0) * 4 + rx], ff[((jy0 + 2) * SP + i0 + 1) * 4 + rx], h1, m1, l1);
            mma_bf16x6(dx, h0, m0, l0, h1, m1, l1, bx[ks][0], bx[ks][1], bx[ks][2]);
        }
        const int ixo = 8 * nX + 2 * tq;
        kxo[(jy0 * SP + ixo) * 4 + rx] = dx[0];
        kxo[(jy0 * SP + ixo + 1) * 4 + rx] = dx[1];
        kxo[((jy0 + 2) * SP + ixo) * 4 + rx] = dx[2];
        kxo[((jy0 + 2) * SP + ixo + 1) * 4 + rx] = dx[3];
        const int Q0 = 16 * mY + gq, ix0 = Q0 >> 2, ry = Q0 & 3;       // Y rows: (i_x, c)
        float dy[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int ks = 0; ks < YS; ++ks) {
            const int j0 = 8 * ks + 2 * tq;
            uint32_t h0, m0, l0, h1, m1, l1;
            split_bf16x3(ff[(j0 * SP + ix0) * 4 + ry], ff[((j0 + 1) * SP + ix0) * 4 + ry], h0, m0, l0);
            split_bf16x3(ff[(j0 * SP + ix0 + 2) * 4 + ry], ff[((j0 + 1) * SP + ix0 + 2) * 4 + ry], h1, m1, l1);
            mma_bf16x6(dy, h0, m0, l0, h1, m1, l1, by[ks][0], by[ks][1], by[ks][2]);
        }
        const int jyo = 8 * nY + 2 * tq;
        kyo[(jyo * SP + ix0) * 4 + ry] = dy[0];
        kyo[((jyo + 1) * SP + ix0) * 4 + ry] = dy[1];
        kyo[(jyo * SP + ix0 + 2) * 4 + ry] = dy[2];
        kyo[((jyo + 1) * SP + ix0 + 2) * 4 + ry] = dy[3];
    }
};

// Force-term forms of the FP32 marching kernels (template parameter FM).  The
// dispatch forms kForceField, kForceFMASR and kForceFieldSR select the FMA form
// with a per-node acceleration field (template parameter FF of the kernels),
// with stochastically rounded stage outputs (SR), or both.
constexpr int kForceFMA = 0, kForceTF32x3 = 1, kForceBF16x6 = 2, kForceField = 3, kForceFMASR = 4,
              kForceFieldSR = 5;
template <int FM, int QX2, int VY>
using ForceTC = typename std::conditional<FM == kForceBF16x6, ForceMMABF16<QX2, VY>, ForceMMA<QX2, VY>>::type;

// 1/x on the special-function unit (x >= 1e-30 here; beyond 1e38 it flushes to 0).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// WENO-5 face value from a stencil already divided by the population's
// weight (values O(1) wherever the population matters), without epsilon
// (Sec. IV.C.2), face between c and d of the upwind-ordered stencil a..e:
// - the candidates relative to c, q_k = c + R_k / 6, with R_1 = 2a - 7b + 5c,
//   R_2 = 2d - b - c, R_3 = 5d - 4c - e, and the indicators' t_k, s_k, all from
//   the differences of neighbouring stencil values;
// - the indicators scaled by 12/13, B_k = t_k^2 + (3/13) s_k^2 (a common factor
//   leaves the weights unchanged), with an additive floor of 1e-30, below which
//   FP32 cannot resolve them anyway;
// - the nonlinear weights from the ratios u_k = min_j B_j / B_k in (0, 1], so
//   nothing overflows, and a zero B_k takes the limit of Tab. "weno" (the
//   zero-indicator stencils share the weight in proportion to d_k);
// - face = c + (v_1 R_1 + 6 v_2 R_2 + 3 v_3 R_3) / (6 (v_1 + 6 v_2 + 3 v_3)) with
//   v_k = u_k^2: the linear weights (0.1, 0.6, 0.3) scaled by 10, so the
//   denominator is at least 1.
// The packed form below needs six constants (f32x2 instructions take no
// immediates).  The scalar form performs the same roundings in the same
// order (explicit _rn operations, no contraction), so a face gives the same
// bits in either form: the wall kernel's incident flux is the stage kernels'.
__device__ __forceinline__ float weno5_scaled(float a, float b, float c, float d, float e) {
    const float dmm = __fsub_rn(a, b), dm = __fsub_rn(c, b), dp = __fsub_rn(d, c), dpp = __fsub_rn(e, d);
    const float t1 = __fadd_rn(dm, dmm), s1 = __fmaf_rn(3.0f, dm, dmm);
    const float t2 = __fsub_rn(dp, dm), s2 = __fadd_rn(dm, dp);
    const float t3 = __fsub_rn(dpp, dp), s3 = __fmaf_rn(-3.0f, dp, dpp);
    const float R1 = __fadd_rn(__fadd_rn(t1, s1), dm), R2 = __fadd_rn(s2, dp), R3 = __fsub_rn(dp, s3);
    constexpr float k = 3.0f / 13.0f, fl = 1e-30f;
    const float B1 = __fmaf_rn(t1, t1, __fmaf_rn(__fmul_rn(k, s1), s1, fl));
    const float B2 = __fmaf_rn(t2, t2, __fmaf_rn(__fmul_rn(k, s2), s2, fl));
    const float B3 = __fmaf_rn(t3, t3, __fmaf_rn(__fmul_rn(k, s3), s3, fl));
    const float m = fminf(B1, fminf(B2, B3));
    const float u1 = __fmul_rn(m, rcp_approx(B1)), u2 = __fmul_rn(m, rcp_approx(B2)), u3 = __fmul_rn(m, rcp_approx(B3));
    const float v1 = __fmul_rn(u1, u1);
    const float V2 = __fmul_rn(6.0f, __fmul_rn(u2, u2)), V3 = __fmul_rn(3.0f, __fmul_rn(u3, u3));
    const float den = __fadd_rn(__fadd_rn(v1, V2), V3);
    const float num = __fmaf_rn(V3, R3, __fmaf_rn(V2, R2, __fmul_rn(v1, R1)));
    return __fmaf_rn(__fmul_rn(num, 1.0f / 6.0f), rcp_approx(den), c);
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// a - b in the packed FP32 pipe
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}

// Two independent faces at once in the packed FP32 pipe (f32x2 on sm_100+);
// the arithmetic of weno5_scaled, lane by lane.
__device__ __forceinline__ float2 weno5_scaled2(float2 a, float2 b, float2 c, float2 d, float2 e) {
    const float2 dmm = fsub2(a, b), dm = fsub2(c, b), dp = fsub2(d, c), dpp = fsub2(e, d);
    const float2 t1 = __fadd2_rn(dm, dmm), s1 = __ffma2_rn(f2(3.0f), dm, dmm);
    const float2 t2 = fsub2(dp, dm), s2 = __fadd2_rn(dm, dp);
    const float2 t3 = fsub2(dpp, dp), s3 = __ffma2_rn(f2(-3.0f), dp, dpp);
    const float2 R1 = __fadd2_rn(__fadd2_rn(t1, s1), dm), R2 = __fadd2_rn(s2, dp), R3 = fsub2(dp, s3);
    const float2 k = f2(3.0f / 13.0f), fl = f2(1e-30f);
    const float2 B1 = __ffma2_rn(t1, t1, __ffma2_rn(__fmul2_rn(k, s1), s1, fl));
    const float2 B2 = __ffma2_rn(t2, t2, __ffma2_rn(__fmul2_rn(k, s2), s2, fl));
    const float2 B3 = __ffma2_rn(t3, t3, __ffma2_rn(__fmul2_rn(k, s3), s3, fl));
    const float2 m = make_float2(fminf(B1.x, fminf(B2.x, B3.x)), fminf(B1.y, fminf(B2.y, B3.y)));
    const float2 u1 = __fmul2_rn(m, make_float2(rcp_approx(B1.x), rcp_approx(B1.y)));
    const float2 u2 = __fmul2_rn(m, make_float2(rcp_approx(B2.x), rcp_approx(B2.y)));
    const float2 u3 = __fmul2_rn(m, make_float2(rcp_approx(B3.x), rcp_approx(B3.y)));
    const float2 v1 = __fmul2_rn(u1, u1);
    const float2 V2 = __fmul2_rn(f2(6.0f), __fmul2_rn(u2, u2)), V3 = __fmul2_rn(f2(3.0f), __fmul2_rn(u3, u3));
    const float2 den = __fadd2_rn(__fadd2_rn(v1, V2), V3);
    const float2 num = __ffma2_rn(V3, R3, __ffma2_rn(V2, R2, __fmul2_rn(v1, R1)));
    return __ffma2_rn(__fmul2_rn(num, f2(1.0f / 6.0f)), make_float2(rcp_approx(den.x), rcp_approx(den.y)), c);
}

// ---------------------------------------------------------------------------
// Stochastic rounding of the FP32 stage outputs (optional, hlb_set_rounding).
// With round-to-nearest, a stage adds dt L to f and drops it when it is below
// half a unit in the last place (ulp): near a steady state the FP32 state
// stops where |dt L| < ulp / 2, short of L = 0 by about ulp / (dt x the
// slowest relaxation rate), which can exceed the 1e-5 parity bar when dt is
// small.  Here the stage output s = RN(v) comes with the error e of its last
// additions (s + e = v, by the TwoSum of Knuth and Moller), and s moves one
// ulp toward v with probability |e| / ulp, so that its expectation is v and
// the state keeps drifting toward L = 0.  The probability comes from a hash
// of the value's address, the stage and the bits of s and e: deterministic,
// no state, the same inside a captured graph.
// ---------------------------------------------------------------------------
// A 32-bit integer finaliser (xor-shift and multiply rounds, the constants of
// C. Wellons' "lowbias32" from his hash-prospector search).
__device__ __forceinline__ uint32_t sr_hash(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// s + e = a - b exactly (TwoSum of a and -b).
__device__ __forceinline__ void two_diff2(float2 a, float2 b, float2& s, float2& e) {
    s = fsub2(a, b);
    const float2 bb = fsub2(s, a);
    e = fsub2(fsub2(a, fsub2(s, bb)), __fadd2_rn(b, bb));
}
// s + e = a + b exactly (TwoSum).
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
    s = __fadd2_rn(a, b);
    const float2 bb = fsub2(s, a);
    e = __fadd2_rn(fsub2(a, fsub2(s, bb)), fsub2(b, bb));
}
__device__ __forceinline__ void two_diff(float a, float b, float& s, float& e) {
    s = __fsub_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fsub_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fadd_rn(b, bb));
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s rounded stochastically toward s + e (|e| <= ulp(s) / 2), r uniform in [0, 1).
__device__ __forceinline__ float sround(float s, float e, float r) {
    if (e == 0.0f || s == 0.0f || !(fabsf(s) < 3.0e38f)) return s;
    const uint32_t b = __float_as_uint(s);
    const float nxt = __uint_as_float((e > 0.0f) == (s > 0.0f) ? b + 1u : b - 1u);
    return fabsf(e) > r * fabsf(__fsub_rn(nxt, s)) ? nxt : s;
}

// The RK-3 stage output (Eq. "eq:rk3") from fc, dtL = dt L[fc] and, at stages
// 1 and 2, f^n, with stochastic rounding: stage 0 gives fc - dtL; stages 1
// and 2 give fp + c (f^n - fp) with fp = fc - dtL, c = 3/4 or 1/3, whose exact
// value is out + e2 + (1 - c) e1 for the errors e1 of fp and e2 of the final
// addition (the product's rounding is relative to the increment and left out).
// One hash serves both lanes (16 bits of probability each).
__device__ __forceinline__ float2 rk3_out_sr2(int stage, float2 fc, float2 dtL, float2 fn, uint32_t key) {
    float2 fp, e1;
    two_diff2(fc, dtL, fp, e1);
    float2 out = fp, e = e1;
    if (stage > 0) {
        const float c = stage == 1 ? 0.75f : 1.0f / 3.0f;
        float2 e2;
        two_sum2(fp, __fmul2_rn(f2(c), fsub2(fn, fp)), out, e2);
        e = __ffma2_rn(f2(1.0f - c), e1, e2);
    }
    const uint32_t h = sr_hash(key ^ ((uint32_t)stage * 0x85ebca77u) ^ __float_as_uint(out.x) ^
                               (__float_as_uint(e.x) * 0x9e3779b9u) ^
                               ((__float_as_uint(out.y) ^ __float_as_uint(e.y)) * 0xc2b2ae35u));
    return make_float2(sround(out.x, e.x, (float)(h & 0xffffu) * (1.0f / 65536.0f)),
                       sround(out.y, e.y, (float)(h >> 16) * (1.0f / 65536.0f)));
}
__device__ __forceinline__ float rk3_out_sr(int stage, float fc, float dtL, float fn, uint32_t key) {
    float fp, e1;
    two_diff(fc, dtL, fp, e1);
    float out = fp, e = e1;
    if (stage > 0) {
        const float c = stage == 1 ? 0.75f : 1.0f / 3.0f;
        float e2;
        two_sum(fp, __fmul_rn(c, __fsub_rn(fn, fp)), out, e2);
        e = __fmaf_rn(1.0f - c, e1, e2);
    }
    const uint32_t h = sr_hash(key ^ ((uint32_t)stage * 0x85ebca77u) ^ __float_as_uint(out) ^
                               (__float_as_uint(e) * 0x9e3779b9u));
    return sround(out, e, (float)(h >> 8) * (1.0f / 16777216.0f));
}
// The key of a value: its address in the stage output (unique within a launch).
__device__ __forceinline__ uint32_t sr_key(const void* p) {
    return (uint32_t)(reinterpret_cast<uintptr_t>(p) >> 2);
}

__device__ __forceinline__ float2 upwind2_face2(float2 b, float2 c) {
    return __ffma2_rn(f2(1.5f), c, __fmul2_rn(f2(-0.5f), b));
}

__device__ __forceinline__ int find_slot(const int* start, int n, int key) {
    int lo = 0, hi = n;            // start[lo] <= key < start[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(start + mid) <= key) lo = mid; else hi = mid;
    }
    return lo;
}

// Compensated summation (Kahan-Babuska / Neumaier): the running sum s and an
// error term c with s + c equal to the sum of the terms to about twice the
// working precision.  The FP32 form is the error-free TwoSum of Knuth; the FP64
// form is a plain sum (c stays 0).
__device__ __forceinline__ void csum_add(float& s, float& c, float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}
__device__ __forceinline__ void csum_add(double& s, double& c, double x) {
    (void)c;
    s += x;
}

// csum_add on two independent sums at once in the packed FP32 pipe.
__device__ __forceinline__ void csum_add2(float2& s, float2& c, float2 x) {
    const float2 t = __fadd2_rn(s, x);
    const float2 bp = fsub2(t, s);
    c = __fadd2_rn(c, __fadd2_rn(fsub2(s, fsub2(t, bp)), fsub2(x, bp)));
    s = t;
}

// Butterfly reduction of (s, c) over groups of 2 O consecutive lanes (O = 16:
// the whole warp); every lane of a group ends with the group's sum.
template <typename R, int O = 16>
__device__ __forceinline__ void csum_warp(R& s, R& c) {
#pragma unroll
    for (int o = O; o > 0; o >>= 1) {
        const R s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
        csum_add(s, c, s2);
        c += c2;
    }
}

// Slots of a node's moment sums: n, j_x, j_y, j_z, E at [0..4] and their
// compensation terms at [8..12] (zero for FP64 states).
constexpr int kSumStride = 16;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-node equilibrium coefficients in FP64.  Thread role r:
//   r = 0, 1: half-range G_l^{+-} (l <= Nx) by the recurrence in the
//             orthonormal basis (see hlb_tables.cpp);
//   r = 2:    full-range G_l along p_y;  r = 3: along p_z.
__device__ inline void node_coefficients(const GroupDev& g, int r, double ux, double uy, double uz,
                                  double T, const double* rec, double* coef) {
    const int Nx = g.Nx;
    if (r < 2 && g.x_full) {
        // full-range p_x (Eq. "eq:H_gk"): G_l(+-u_x) for the +z and -z rows
        const double u = r ? -ux : ux;
        double* G = coef + r * (Nx + 1);
        G[0] = 1.0;
        if (Nx >= 1) G[1] = u;
        for (int l = 1; l < Nx; ++l) G[l + 1] = u * G[l] + l * (T - 1.0) * G[l - 1];
    } else if (r < 2) {
        const double* ra = rec;
        (void)ra;
        const double* rb = rec + Nx;
        const double* rc = rec + 2 * Nx;
        const double* h0 = rec + 3 * Nx;
        const double* inv_ra = rec + 4 * Nx + 1;
        double* G = coef + r * (Nx + 1);
        const double us = r ? -ux : ux;
        const double g0 = exp(-ux * ux / (2.0 * T)) / (kSqrt2Pi * sqrt(T));
        G[0] = h0[0] * 0.5 * (1.0 + erf(us / sqrt(2.0 * T)));
        double S = 0.0;
        double gm1 = 0.0;
        for (int l = 0; l < Nx; ++l) {
            const double ig = (l ? gm1 * inv_ra[l - 1] : 0.0) - g.om0 * h0[l] * S;
            const double pg = us * G[l] + T * (g0 * h0[l] + ig);
            G[l + 1] = ra[l] * pg + rb[l] * G[l] + rc[l] * gm1;
            S += h0[l] * G[l];
            gm1 = G[l];
        }
    } else {
        const int N = r == 2 ? g.Ny : g.Nz;
        const double u = r == 2 ? uy : uz;
        double* G = coef + 2 * (Nx + 1) + (r == 2 ? 0 : g.Ny + 1);
        G[0] = 1.0;
        if (N >= 1) G[1] = u;
        for (int l = 1; l < N; ++l) G[l + 1] = u * G[l] + l * (T - 1.0) * G[l - 1];
    }
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (an unevaluated sum hi + lo of two FP32 numbers,
// about 48 significant bits), built from the error-free transformations
// TwoSum (Knuth) and TwoProduct by FMA.  Used for the per-node equilibrium
// recurrence, whose rounding errors grow by ~1e4 over eight terms: FP32 is
// too short and this GPU's FP64 rate is 1/64 of FP32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 df_fast_two_sum(float a, float b) {
    const float s = a + b;
    return make_float2(s, b - (s - a));
}

__device__ __forceinline__ float2 df_add(float2 x, float2 y) {
    const float s = x.x + y.x;
    const float bb = s - x.x;
    const float e = (x.x - (s - bb)) + (y.x - bb);
    return df_fast_two_sum(s, e + (x.y + y.y));
}

__device__ __forceinline__ float2 df_mul(float2 x, float2 y) {
    const float p = x.x * y.x;
    float e = fmaf(x.x, y.x, -p);
    e = fmaf(x.x, y.y, fmaf(x.y, y.x, e));
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ float2 df_from_double(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (global -> shared) completed on an mbarrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Plain arrival (release at CTA scope): the arriving thread's earlier
// shared-memory writes are visible to threads that then see the phase complete.
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// its later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// src 16-byte aligned; bytes a multiple of 16.  A hint: no completion to wait for.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// try_wait that may suspend the thread for up to hint_ns while the phase is
// incomplete (the thread resumes when it completes), so that a waiting warp
// does not spin through issue slots.
__device__ __forceinline__ bool mbar_try_wait_hint(unsigned long long* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after wait_ns nanoseconds, records HLB_ETIMEOUT in
// *err and returns false.  The caller then leaves its loop, so that no wait
// of the CTA is left pending.
constexpr uint32_t kSuspendHintNs = 100000;

__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, int* err,
                                          unsigned long long wait_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait_hint(bar, parity, kSuspendHintNs)) {
        if (global_ns() - t0 > wait_ns) {
            atomicExch(err, 4);   // HLB_ETIMEOUT
            return false;
        }
    }
    return true;
}

// After a wait ran out: wait for the phase of the given parity (the bulk
// copies it tracks) to complete before the CTA exits, so that no copy the CTA
// issued lands in shared memory after the CTA is gone.  Callers drain only
// phases whose byte count was registered (not the ones the test hook
// withholds); a copy that was issued always completes, normally within
// microseconds, so the bound here is generous (wait_ns + 1 s) and is only
// reached if a phase was registered but some of its copies were never issued
// (a warp that left the loop early), by which time the issued ones have long
// landed.  Records nothing.
__device__ __forceinline__ void mbar_drain(unsigned long long* bar, uint32_t parity, unsigned long long wait_ns) {
    const unsigned long long t0 = global_ns();
    const unsigned long long bound = wait_ns + 1000000000ull;
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > bound) return;
    }
}

// exp(y) in double-float for y in [-60, 0]: y = k ln 2 + r with |r| <= ln2 / 2
// (k ln 2 subtracted exactly: ln 2 as hi + lo, k hi by TwoProduct), exp(r) by
// its Taylor polynomial to degree 13 (remainder below 2e-17) evaluated by
// Horner's rule in double-float, then times 2^k (exact).
__device__ inline float2 df_exp_nonpos(float2 y) {
    // 1/n!, n = 0 .. 13, as double-float pairs (rounded from the exact rationals)
    const float fh[14] = {1.0f, 1.0f, 0.5f, 0.1666666716337204f, 0.0416666679084301f, 0.008333333767950535f,
                          0.0013888889225199819f, 0.00019841270113829523f, 2.4801587642286904e-05f,
                          2.7557318844628753e-06f, 2.755731998149713e-07f, 2.5052107943679403e-08f,
                          2.0876755879584152e-09f, 1.6059044372074283e-10f};
    const float fl[14] = {0.0f, 0.0f, 0.0f, -4.967053879312289e-09f, -1.2417634698280722e-09f,
                          -4.34617203337595e-10f, -3.3631094437103215e-11f, -2.725596874933456e-12f,
                          -3.40699609366682e-13f, 3.793571224297229e-14f, -7.575112209051195e-15f,
                          4.4176230446483665e-16f, 1.1082839147459852e-16f, -5.352526511562726e-18f};
    const float ln2h = 0.6931471824645996f, ln2l = -1.9046542121259336e-09f;
    const float k = rintf(y.x * 1.4426950408889634f);
    const float p = k * ln2h, e = fmaf(k, ln2h, -p);          // k ln2h = p + e exactly
    const float q = k * ln2l, eq = fmaf(k, ln2l, -q);
    float2 r = df_add(df_add(y, make_float2(-p, -e)), make_float2(-q, -eq));
    float2 sum = make_float2(fh[13], fl[13]);
#pragma unroll
    for (int n = 12; n >= 0; --n) sum = df_add(df_mul(sum, r), make_float2(fh[n], fl[n]));
    const int ki = (int)k;
    return make_float2(ldexpf(sum.x, ki), ldexpf(sum.y, ki));
}

// x / m in double-float for a small positive integer m: the high part's
// remainder x.hi - q1 m is exact (FMA), the low part carries it.
__device__ __forceinline__ float2 df_div_small(float2 x, float m) {
    const float q1 = __fdividef(x.x, m);
    const float rem = fmaf(-q1, m, x.x);
    return df_fast_two_sum(q1, __fdividef(rem + x.y, m));
}

// erf(z) in double-float for |z| <= 2.5 from E = exp(-z^2): erf z =
// (2/sqrt(pi)) E z sum_n (2 z^2)^n / (1 3 5 ... (2n+1)), a series of positive
// terms (no cancellation; they peak near n = z^2 and fall below 2^-52 of the
// sum by n = 40 at z = 2.5).
__device__ inline float2 df_erf_series(float2 z, float2 z2, float2 E) {
    const float2 w = make_float2(2.0f * z2.x, 2.0f * z2.y);
    float2 t = make_float2(1.0f, 0.0f), sum = t;
    for (int n = 1; n < 48; ++n) {
        t = df_div_small(df_mul(t, w), (float)(2 * n + 1));
        sum = df_add(sum, t);
        if (__all_sync(__activemask(), t.x < sum.x * 2.0e-16f)) break;
    }
    const float2 two_sqrtpi = make_float2(1.128379225730896f, -5.8635382771399236e-08f);
    return df_mul(df_mul(two_sqrtpi, E), df_mul(z, sum));
}

// The half-range coefficients G^{+-}_l (roles 0, 1) and the full-range ones
// (roles 2: p_y, 3: p_z) of node_coefficients, in double-float.  recf holds
// (hi, lo) pairs of ra, rb, rc, h0, 1/ra in the layout of rec; the values that
// start the recurrence come from FP64 n, u, T: sqrt(T) and 1/sqrt(T) in FP64,
// erf and exp in double-float where the recurrence's growth (about threefold
// per order) keeps their ~1e-13 error below FP32 resolution (orders up to 10),
// in FP64 above.
// Per-node inputs of node_coefficients_df, formed once per node in FP64:
// ux, uy, uz, T, and for the half-range recurrence
// E = erf(u_x / sqrt(2T)) and g(0) = exp(-u_x^2 / 2T) / sqrt(2 pi T).
struct NodeDF {
    float2 ux, uy, uz, T, Tm1, erf_z, g0, n;
};

#ifndef HLB_DF_SPECIAL_MAX_N
#define HLB_DF_SPECIAL_MAX_N 10
#endif
__device__ inline void node_inputs_df(double n, double ux, double uy, double uz, double T, int Nx, NodeDF& o) {
    o.n = df_from_double(n);
    o.ux = df_from_double(ux);
    o.uy = df_from_double(uy);
    o.uz = df_from_double(uz);
    o.T = df_from_double(T);
    o.Tm1 = df_from_double(T - 1.0);
    const double irt = 1.0 / sqrt(T);
    const double z = ux * irt * 0.70710678118654752440;     // u_x / sqrt(2T)
    if (Nx <= HLB_DF_SPECIAL_MAX_N && fabs(z) <= 2.5) {
        const float2 zd = df_from_double(z);
        const float2 z2 = df_mul(zd, zd);
        const float2 E = df_exp_nonpos(make_float2(-z2.x, -z2.y));          // exp(-u_x^2 / 2T)
        o.erf_z = df_erf_series(zd, z2, E);
        const float2 inv_sqrt2pi = make_float2(0.3989422917366028f, -1.1335170135851058e-08f);
        o.g0 = df_mul(df_mul(E, inv_sqrt2pi), df_from_double(irt));          // E / sqrt(2 pi T)
    } else {
        o.erf_z = df_from_double(erf(z));
        o.g0 = df_from_double(exp(-z * z) * (irt / kSqrt2Pi));
    }
}

// The half-range coefficients G^{+-}_l (roles 0, 1) and the full-range ones
// (roles 2: p_y, 3: p_z) of node_coefficients, in double-float; recf holds
// (hi, lo) pairs of ra, rb, rc, h0, 1/ra in the layout of rec.
__device__ inline void node_coefficients_df(const GroupDev& g, int r, const NodeDF& in, const float2* recf,
                                            float2* coef) {
    const int Nx = g.Nx;
    // same slots as node_coefficients: G^+ | G^- | G_y | G_z
    float2* G = coef + (r < 2 ? r * (Nx + 1) : 2 * (Nx + 1) + (r == 2 ? 0 : g.Ny + 1));
    if (r < 2 && g.x_full) {
        // full-range p_x (Eq. "eq:H_gk"): G_l(+-u_x) for the +z and -z rows
        const float2 u = r ? make_float2(-in.ux.x, -in.ux.y) : in.ux;
        G[0] = make_float2(1.0f, 0.0f);
        if (Nx >= 1) G[1] = u;
        for (int l = 1; l < Nx; ++l)
            G[l + 1] = df_add(df_mul(u, G[l]), df_mul(df_mul(make_float2((float)l, 0.0f), in.Tm1), G[l - 1]));
    } else if (r < 2) {
        const float2* ra = recf;
        const float2* rb = recf + Nx;
        const float2* rc = recf + 2 * Nx;
        const float2* h0 = recf + 3 * Nx;
        const float2* inv_ra = recf + 4 * Nx + 1;
        const float sg = r ? -1.0f : 1.0f;
        const float2 us = make_float2(sg * in.ux.x, sg * in.ux.y);
        // int_0^inf g(+-p) dp = (1 +- erf(u_x/sqrt(2T)))/2, with h_0 = h0[0]
        const float2 half = df_add(make_float2(0.5f, 0.0f), make_float2(0.5f * sg * in.erf_z.x, 0.5f * sg * in.erf_z.y));
        G[0] = df_mul(h0[0], half);
        const float2 m_om0 = g.m_om0f;                 // -omega(0) of the half-range family
        float2 S = make_float2(0.0f, 0.0f), gm1 = make_float2(0.0f, 0.0f);
        for (int l = 0; l < Nx; ++l) {
            float2 ig = df_mul(df_mul(m_om0, h0[l]), S);
            if (l) ig = df_add(ig, df_mul(gm1, inv_ra[l - 1]));
            const float2 pg = df_add(df_mul(us, G[l]), df_mul(in.T, df_add(df_mul(in.g0, h0[l]), ig)));
            G[l + 1] = df_add(df_add(df_mul(ra[l], pg), df_mul(rb[l], G[l])), df_mul(rc[l], gm1));
            S = df_add(S, df_mul(h0[l], G[l]));
            gm1 = G[l];
        }
    } else {
        const int N = r == 2 ? g.Ny : g.Nz;
        const float2 u = r == 2 ? in.uy : in.uz;
        G[0] = make_float2(1.0f, 0.0f);
        if (N >= 1) G[1] = u;
        for (int l = 1; l < N; ++l)
            G[l + 1] = df_add(df_mul(u, G[l]), df_mul(df_mul(make_float2((float)l, 0.0f), in.Tm1), G[l - 1]));
    }
}

}  // namespace hlb
