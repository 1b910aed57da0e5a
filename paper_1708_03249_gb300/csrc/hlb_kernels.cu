// Device kernels of libhlb (sm_103a).
//
// Per RK-3 stage (Eq. "eq:rk3") these kernels run (the marching kernels of
// hlb_march.cu, hlb_pair.cuh, hlb_line.cuh take the stage kernel's place
// where they apply):
//   quad_coef_kernel  FP64 half-range groups above order 12: the half-range
//                 equilibrium coefficients of every collisional node by
//                 quadrature of the projection integrals (see below).
//   wall_kernel   one or a few CTAs per (instance, y-row): incident fluxes at
//                 both wall faces from the quadratically extrapolated ghosts
//                 (Sec. IV.C.3), summed in FP64, give the emitted densities
//                 n_w = -sum_inc F / sum_emit p_x g^w (Eq. "eq:nplus_def").
//   stage_kernel  fused per node: moments (Eq. "eq:fmoms") by a block
//                 reduction, the equilibrium factors g_x, g_y, g_z (FP64
//                 recurrences, App. A), the force term sum_a a_a K_a f
//                 (Eqs. "eq:hh_Kk_hh", "eq:H_Kk"; a the uniform acceleration
//                 plus the node's field value), BGK with tau = Kn/n,
//                 WENO-5 / upwind2 fluxes along x (walls: Eq.
//                 "eq:weno_populate" ghosts) and y (periodic), and the RK-3
//                 combination; writes the stage output.  It serves the
//                 shapes the marching kernels do not, among them the
//                 half-range sets beyond Qx = 32 (the HHLB(20;200) model of
//                 Sec. V): there K_x stays in global memory, its cross-half
//                 blocks enter as their rank-one factor, and a node's
//                 velocities are split over several CTAs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "hlb_internal.h"
#include "hlb_device.cuh"

namespace hlb {

namespace {

// Shared-memory layout of the stage kernel (sizes in elements).
struct SmemLayout {
    int nK, nP, nT, nG;
    size_t offK, offP, offT, offF, offG;      // in R elements
    size_t offD;                              // in bytes (8-aligned)
    int nRec, nCoef;
    int nJ;                                   // doubles: per-fibre cross-half sums (kx_global)
    size_t bytes;
};

template <typename R>
__host__ __device__ inline SmemLayout smem_layout(const GroupDev& g, int nwarps) {
    SmemLayout L;
    L.nK = (g.kx_global ? 0 : g.QX2 * g.QX2) + g.VY * g.VY + g.VZ * g.VZ;
    L.nP = g.QX2 + g.VY + g.VZ;
    L.nT = g.Qx * (g.Nx + 1) + g.VY * (g.Ny + 1) + g.VZ * (g.Nz + 1);
    L.nG = g.QX2 + g.VY + g.VZ;
    L.offK = 0;
    L.offP = L.offK + L.nK;
    L.offT = L.offP + L.nP;
    L.offF = L.offT + L.nT;
    L.offG = L.offF + g.V;
    size_t rbytes = (L.offG + L.nG) * sizeof(R);
    L.offD = (rbytes + 15) & ~size_t(15);
    L.nRec = 5 * g.Nx + 1;
    L.nCoef = 2 * (g.Nx + 1) + (g.Ny + 1) + (g.Nz + 1);
    L.nJ = g.kx_global ? 2 * g.VY * g.VZ : 0;
    // doubles: rec, coef, 8 scalars, 5 * nwarps reduction slots, cross-half sums
    L.bytes = L.offD + sizeof(double) * (L.nRec + L.nCoef + 8 + 5 * nwarps + L.nJ);
    return L;
}

// Value of velocity v at x-position pos of a row (ghost rules at the walls).
template <typename R>
__device__ __forceinline__ R x_value(const R* __restrict__ frow, int pos, int nx, int V, int v,
                                     bool px_pos, R nwl_g, R nwr_g) {
    if (pos >= 0 && pos < nx) return frow[(size_t)pos * V + v];
    if (pos < 0) {
        if (px_pos) return nwl_g;                        // emitted: n_w g^w (3 ghosts)
        const R f0 = frow[v], f1 = frow[(size_t)V + v], f2 = frow[2 * (size_t)V + v];
        if (pos == -1) return R(3) * f0 - R(3) * f1 + f2;            // paper's cell 0
        return R(6) * f0 - R(8) * f1 + R(3) * f2;                     // paper's cell -1
    }
    if (!px_pos) return nwr_g;
    const R f0 = frow[(size_t)(nx - 1) * V + v], f1 = frow[(size_t)(nx - 2) * V + v],
            f2 = frow[(size_t)(nx - 3) * V + v];
    if (pos == nx) return R(3) * f0 - R(3) * f1 + f2;
    return R(6) * f0 - R(8) * f1 + R(3) * f2;
}

// Fluxes at the faces x+1/2 and x-1/2 (per unit velocity) from a 6-cell
// window; w[] holds cells x-3..x+2 for v > 0 and x-2..x+3 for v < 0.
template <typename R, int ADV>
__device__ __forceinline__ void face_pair(const R* w, bool pos, R& Fp, R& Fm) {
    if (ADV == HLB_WENO5_) {
        if (pos) {
            Fp = weno5_face(w[1], w[2], w[3], w[4], w[5]);
            Fm = weno5_face(w[0], w[1], w[2], w[3], w[4]);
        } else {
            Fp = weno5_face(w[5], w[4], w[3], w[2], w[1]);
            Fm = weno5_face(w[4], w[3], w[2], w[1], w[0]);
        }
    } else {
        if (pos) {
            Fp = upwind2_face(w[2], w[3]);
            Fm = upwind2_face(w[1], w[2]);
        } else {
            Fp = upwind2_face(w[4], w[3]);
            Fm = upwind2_face(w[3], w[2]);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// stage kernel
// ---------------------------------------------------------------------------
// CTAs per SM the generic stage kernel is compiled for (2: at most 128
// registers per thread, so that two 256-thread CTAs fit an SM; on the order-200
// set 0.0927 ms per stage launch against 0.0989 ms at 1, eight ballistic cases).
#ifndef HLB_STAGE_MIN_BLOCKS
#define HLB_STAGE_MIN_BLOCKS 2
#endif
template <typename R, int ADV>
__global__ void __launch_bounds__(256, HLB_STAGE_MIN_BLOCKS)
stage_kernel(const GroupDev g, const R* __restrict__ fs, const R* __restrict__ fn,
             R* __restrict__ fo, int stage) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nwarps = blockDim.x >> 5;
    const SmemLayout L = smem_layout<R>(g, nwarps);
    R* sR = reinterpret_cast<R*>(smem_raw);
    R* sK = sR + L.offK;
    R* sP = sR + L.offP;
    R* sT = sR + L.offT;
    R* sF = sR + L.offF;
    R* sG = sR + L.offG;
    double* sD = reinterpret_cast<double*>(smem_raw + L.offD);
    double* sRec = sD;
    double* sCoef = sRec + L.nRec;
    double* sScal = sCoef + L.nCoef;
    double* sRed = sScal + 8;
    double* sJ = sRed + 5 * nwarps;           // [fibre][2]: sum_{k' in half} d_k' f_k'

    const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, warp = tid >> 5;
    // Kx stays in global memory (read through KxT) when it exceeds the
    // shared-memory budget; sK then holds Ky and Kz only
    const R* gK = static_cast<const R*>(g.K) + (g.kx_global ? g.QX2 * g.QX2 : 0);
    const R* gP = static_cast<const R*>(g.p);
    const R* gT = static_cast<const R*>(g.Tt);
    for (int i = tid; i < L.nK; i += bs) sK[i] = gK[i];
    for (int i = tid; i < L.nP; i += bs) sP[i] = gP[i];
    for (int i = tid; i < L.nT; i += bs) sT[i] = gT[i];
    for (int i = tid; i < L.nRec; i += bs) sRec[i] = g.rec[i];
    __syncthreads();

    const int V = g.V, QX2 = g.QX2, VY = g.VY, VZ = g.VZ, Qx = g.Qx;
    const R* sKx = sK;
    const R* sKy = sK + (g.kx_global ? 0 : QX2 * QX2);
    const R* sKz = sKy + VY * VY;
    const R* sPx = sP;
    const R* sPy = sP + QX2;
    const R* sPz = sPy + VY;
    const R* sTx = sT;
    const R* sTy = sT + Qx * (g.Nx + 1);
    const R* sTz = sTy + VY * (g.Ny + 1);
    const R* gw = static_cast<const R*>(g.gw);

    // work items: (node, velocity range); one range per node unless Kx is
    // read from global memory (vchunks > 1)
    const int nvc = g.vchunks;
    for (int item = blockIdx.x; item < g.nnodes * nvc; item += gridDim.x) {
        const int node = item / nvc, chunk = item - node * nvc;
        const int v0 = (int)((long long)chunk * V / nvc), v1 = (int)((long long)(chunk + 1) * V / nvc);
        const int ii = g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0;
        const InstDev I = g.inst[ii];
        const int local = node - I.node_off;
        const int nx = I.nx;
        const int y = local / nx, x = local - y * nx;
        const size_t row_off = (size_t)I.f_off + (size_t)y * nx * V;
        const R* frow = fs + row_off;

        // Collisionless instances (Kn = +inf) have no BGK term at all: no
        // moments and no equilibrium are formed for them.
        const bool collide = I.inv_Kn != 0.0;
        // 1. node values and moment partial sums, accumulated in FP64 for
        // either state precision (T = (E - n|u|^2)/(D n) cancels digits, and
        // the FP32 state's sums are not compensated here)
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
        for (int v = tid; v < V; v += bs) {
            const R val_r = frow[(size_t)x * V + v];
            sF[v] = val_r;
            if (!collide) continue;
            const int ix = v % QX2, jy = (v / QX2) % VY, kz = v / (QX2 * VY);
            const double px = sPx[ix], py = sPy[jy], pz = sPz[kz], val = val_r;
            a0 += val;
            a1 += px * val;
            a2 += py * val;
            a3 += pz * val;
            a4 += (px * px + py * py + pz * pz) * val;
        }
        if (collide) {
        a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2); a3 = warp_sum(a3); a4 = warp_sum(a4);
        if (lane == 0) {
            sRed[warp * 5 + 0] = a0; sRed[warp * 5 + 1] = a1; sRed[warp * 5 + 2] = a2;
            sRed[warp * 5 + 3] = a3; sRed[warp * 5 + 4] = a4;
        }
        __syncthreads();
        if (tid < 4) {
            double m[5] = {0, 0, 0, 0, 0};
            for (int w = 0; w < nwarps; ++w)
                for (int k = 0; k < 5; ++k) m[k] += sRed[w * 5 + k];
            const double n = m[0];
            const double ux = m[1] / n, uy = m[2] / n, uz = m[3] / n;
            const double T = (m[4] - n * (ux * ux + uy * uy + uz * uz)) / (g.D * n);
            if (tid == 0) {
                sScal[0] = n;
                sScal[1] = n * I.inv_Kn;     // 1/tau
            }
            if (g.quad_x && tid < 2) {          // G^{+-} by quadrature (quad_coef_kernel)
                const double* q = g.gquad + ((size_t)node * 2 + tid) * (g.Nx + 1);
                for (int l = 0; l <= g.Nx; ++l) sCoef[tid * (g.Nx + 1) + l] = q[l];
            } else {
                node_coefficients(g, tid, ux, uy, uz, T, sRec, sCoef);
            }
        }
        __syncthreads();
        // 2. equilibrium factors g_x (times n), g_y, g_z
        {
            const int nf = QX2 + VY + VZ;
            // a velocity range of a 1D set (VY = VZ = 1) needs its own g_x only
            const bool x_range = nvc > 1 && VY * VZ == 1;
            for (int t = tid; t < nf; t += bs) {
                double acc = 0.0;
                if (t < QX2 && x_range && (t < v0 || t >= v1)) continue;
                if (t < QX2) {
                    const int k = t % Qx, sg = t / Qx;
                    const double* G = sCoef + sg * (g.Nx + 1);
                    for (int l = 0; l <= g.Nx; ++l) acc += (double)sTx[k * (g.Nx + 1) + l] * G[l];
                    acc *= sScal[0];
                } else if (t < QX2 + VY) {
                    const int j = t - QX2;
                    if (g.Qy) {
                        const double* G = sCoef + 2 * (g.Nx + 1);
                        for (int l = 0; l <= g.Ny; ++l) acc += (double)sTy[j * (g.Ny + 1) + l] * G[l];
                    } else {
                        acc = 1.0;
                    }
                } else {
                    const int k = t - QX2 - VY;
                    if (g.Qz) {
                        const double* G = sCoef + 2 * (g.Nx + 1) + (g.Ny + 1);
                        for (int l = 0; l <= g.Nz; ++l) acc += (double)sTz[k * (g.Nz + 1) + l] * G[l];
                    } else {
                        acc = 1.0;
                    }
                }
                sG[t] = (R)acc;
            }
        }
        }  // collide
        __syncthreads();
        if (g.kx_global) {
            // K^h = blockdiag(same-half blocks) + the rank-one jump term
            // c_k d_k' in every block (Eq. "eq:hh_Kk_hh"): the cross-half
            // blocks enter through one sum per fibre and half
            const double* jd = g.KxJ + QX2;
            const int nfib = VY * VZ;
            for (int fh = warp; fh < 2 * nfib; fh += nwarps) {
                const int fb = fh >> 1, h = fh & 1;
                const R* fr = sF + (size_t)fb * QX2 + h * Qx;
                double acc = 0.0;
                for (int i = lane; i < Qx; i += 32) acc += jd[h * Qx + i] * (double)fr[i];
                acc = warp_sum(acc);
                if (lane == 0) sJ[fh] = acc;
            }
            __syncthreads();
        }

        const R inv_tau = collide ? (R)sScal[1] : R(0);
        const R dt = (R)I.dt;
        const R inv_dx = (R)(1.0 / g.dx[I.dx_off + x]);
        const R inv_dy = (R)I.inv_dy;
        // the uniform acceleration plus the node's field value (hlb_set_force_field)
        const double* af = g.has_field ? g.afield + 3 * (size_t)node : nullptr;
        const R ax = (R)(I.ax + (af ? af[0] : 0.0)), ay = (R)(I.ay + (af ? af[1] : 0.0)),
                az = (R)(I.az + (af ? af[2] : 0.0));
        const double nwl = g.nw[(size_t)(I.row_off + y) * 2 + 0];
        const double nwr = g.nw[(size_t)(I.row_off + y) * 2 + 1];
        const R* gwl = gw + I.gw_off;
        const R* gwr = gwl + V;
        const int ny = I.ny;

        // 3. per velocity of the range
        for (int v = v0 + tid; v < v1; v += bs) {
            const int ix = v % QX2, jy = (v / QX2) % VY, kz = v / (QX2 * VY);
            const R f = sF[v];
            const R feq = collide ? sG[ix] * sG[QX2 + jy] * sG[QX2 + VY + kz] : R(0);
            // force: sum_a a_a (K_a f)
            R force = 0;
            if (ax != R(0)) {
                const R* fr = sF + (v - ix);
                R acc = 0;
                if (g.kx_global) {
                    // own half: column ix of Kx^T (consecutive threads read
                    // consecutive entries; four partial sums shorten the
                    // dependent chain); other half: c_ix times its fibre sum
                    const int h = ix < Qx ? 0 : 1;
                    const double* Kc = g.KxT + (size_t)h * Qx * QX2 + ix;
                    const R* fh = fr + h * Qx;
                    R a4[4] = {0, 0, 0, 0};
                    int i = 0;
                    for (; i + 4 <= Qx; i += 4) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) a4[q] += (R)Kc[(size_t)(i + q) * QX2] * fh[i + q];
                    }
                    for (; i < Qx; ++i) a4[0] += (R)Kc[(size_t)i * QX2] * fh[i];
                    const int fb = (v - ix) / QX2;
                    acc = (a4[0] + a4[1]) + (a4[2] + a4[3]) + (R)(g.KxJ[ix] * sJ[2 * fb + (1 - h)]);
                } else {
                    const R* Kr = sKx + ix * QX2;
                    for (int i = 0; i < QX2; ++i) acc += Kr[i] * fr[i];
                }
                force += ax * acc;
            }
            if (ay != R(0) && g.Qy) {
                const R* Kr = sKy + jy * VY;
                const R* fr = sF + (v - jy * QX2);
                R acc = 0;
                for (int j = 0; j < VY; ++j) acc += Kr[j] * fr[j * QX2];
                force += ay * acc;
            }
            if (az != R(0) && g.Qz) {
                const R* Kr = sKz + kz * VZ;
                const R* fr = sF + (v - kz * QX2 * VY);
                R acc = 0;
                for (int k = 0; k < VZ; ++k) acc += Kr[k] * fr[(size_t)k * QX2 * VY];
                force += az * acc;
            }
            // advection along x
            const R vx = sPx[ix];
            const bool xpos = ix < Qx;
            R w[6];
            const int base = xpos ? x - 3 : x - 2;
            const R nwl_g = (R)nwl * gwl[v], nwr_g = (R)nwr * gwr[v];
#pragma unroll
            for (int k = 0; k < 6; ++k) w[k] = x_value(frow, base + k, nx, V, v, xpos, nwl_g, nwr_g);
            R Fp, Fm;
            face_pair<R, ADV>(w, xpos, Fp, Fm);
            R Lval = -vx * (Fp - Fm) * inv_dx;
            // advection along y (periodic)
            if (ny > 1) {
                const R vy = sPy[jy];
                const bool ypos = vy > R(0);
                const int yb = ypos ? y - 3 : y - 2;
                const R* fcol = fs + (size_t)I.f_off + (size_t)x * V + v;
                const size_t rstride = (size_t)nx * V;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    int yy = yb + k;
                    yy += (yy < 0) ? ny : 0;
                    yy -= (yy >= ny) ? ny : 0;
                    w[k] = fcol[(size_t)yy * rstride];
                }
                R Gp, Gm;
                face_pair<R, ADV>(w, ypos, Gp, Gm);
                Lval -= vy * (Gp - Gm) * inv_dy;
            }
            Lval -= force;
            if (collide) Lval -= (f - feq) * inv_tau;
            R out;
            bool done = false;
            if constexpr (sizeof(R) == 4) {
                if (g.sround) {      // stochastic rounding of the stage output (hlb_device.cuh)
                    R* dst = fo + row_off + (size_t)x * V + v;
                    *dst = rk3_out_sr(stage, f, -(dt * Lval), stage > 0 ? fn[row_off + (size_t)x * V + v] : R(0),
                                      sr_key(dst));
                    done = true;
                }
            }
            if (!done) {
                if (stage == 0) {
                    out = f + dt * Lval;
                } else {
                    const R fnv = fn[row_off + (size_t)x * V + v];
                    // c f^n + (1 - c) f' as f' + c (f^n - f'): the weights sum to
                    // 1 exactly whatever the rounding of c
                    const R fp = f + dt * Lval;
                    out = fp + (stage == 1 ? R(0.75) : R(1.0 / 3.0)) * (fnv - fp);
                }
                fo[row_off + (size_t)x * V + v] = out;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// wall kernel: emitted densities of both walls of one (instance, y) row
// ---------------------------------------------------------------------------
template <typename R, int ADV>
__global__ void __launch_bounds__(256)
wall_kernel(const GroupDev g, const R* __restrict__ fs) {
    __shared__ double red[2][8];
    const int row = blockIdx.x / g.wchunks, chunk = blockIdx.x - row * g.wchunks;
    if (row >= g.nrows) return;
    const int ii = g.ninst > 1 ? find_slot(g.row_start, g.ninst, row) : 0;
    const InstDev I = g.inst[ii];
    const int y = row - I.row_off;
    const int nx = I.nx, V = g.V, QX2 = g.QX2;
    const R* frow = fs + (size_t)I.f_off + (size_t)y * nx * V;
    double accL = 0.0, accR = 0.0;
    const int Vc = (V + g.wchunks - 1) / g.wchunks, v0 = chunk * Vc, v1 = min(V, v0 + Vc);
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const int ix = v % QX2;
        const double px = g.pd[ix];
        const size_t a = px < 0 ? 0 : (size_t)(nx - 1) * V, step = px < 0 ? (size_t)V : (size_t)0 - (size_t)V;
        // incident on the left wall (face -1/2) or on the right one (face nx-1/2):
        // f0 the wall cell, f1 and f2 the next two inward
        double F;
        if constexpr (sizeof(R) == 4) {
            // the stage kernels' FP32 face: stencil scaled by 1/w, ghosts
            // extrapolated from the scaled values
            const float sv = static_cast<const float*>(g.wscale)[v];
            const float f0 = frow[a + v] * sv, f1 = frow[a + step + v] * sv, f2 = frow[a + 2 * step + v] * sv;
            float face;
            if (ADV == HLB_WENO5_) {
                const float d = 3.0f * f0 - 3.0f * f1 + f2, e = 6.0f * f0 - 8.0f * f1 + 3.0f * f2;
                face = weno5_scaled(f2, f1, f0, d, e);
            } else {
                face = upwind2_face<float>(f1, f0);
            }
            F = (double)(((float)px * (1.0f / sv)) * face);
        } else {
            const double f0 = frow[a + v], f1 = frow[a + step + v], f2 = frow[a + 2 * step + v];
            if (ADV == HLB_WENO5_) {
                const double d = 3.0 * f0 - 3.0 * f1 + f2, e = 6.0 * f0 - 8.0 * f1 + 3.0 * f2;
                F = px * weno5_face<double>(f2, f1, f0, d, e);
            } else {
                F = px * upwind2_face<double>(f1, f0);
            }
        }
        if (px < 0) accL += F; else accR += F;
    }
    accL = warp_sum(accL);
    accR = warp_sum(accR);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[0][warp] = accL; red[1][warp] = accR; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sl = 0.0, sr = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sl += red[0][w]; sr += red[1][w]; }
        if (g.wchunks > 1) {
            // this chunk's partial sums; the row's last CTA adds them in chunk
            // order (the same result whatever order the CTAs finish in)
            double* part = g.wpart + (size_t)row * g.wchunks * 2;
            part[2 * chunk] = sl;
            part[2 * chunk + 1] = sr;
            __threadfence();
            if (atomicAdd(g.wcount + row, 1u) != (unsigned)(g.wchunks - 1)) return;
            __threadfence();
            sl = sr = 0.0;
            for (int c = 0; c < g.wchunks; ++c) {
                sl += __ldcg(part + 2 * c);
                sr += __ldcg(part + 2 * c + 1);
            }
            atomicExch(g.wcount + row, 0u);
        }
        g.nw[(size_t)row * 2 + 0] = -sl / I.den_left;
        g.nw[(size_t)row * 2 + 1] = -sr / I.den_right;
    }
}

// ---------------------------------------------------------------------------
// The half-range equilibrium coefficients of FP64 groups above the
// recurrence's stable order: G^{+-}_l = int_0^inf g(+-p) h_l(p) dp (l <= Nx),
// g the Gaussian of the node's u_x and T (Sec. IV.B, the projection of Eq.
// "eq:hh_gk"), by composite Gauss-Legendre quadrature over [0, |u_x| +
// 15 sqrt(T)] in panels of width sqrt(T) (kQuadNodes points each; 300-440
// points; 1e-14 of max |G| against a 30-point rule on panels of 0.02
// sqrt(T)), h_l(p) by the three-term recurrence of the orthonormal basis
// (forward evaluation at a point is stable).  The integration-by-parts
// recurrence of node_coefficients carries its rounding (and that of its erf
// and exp start) along a solution that grows about threefold per order:
// 5e-7 of max g at N = 20.  One CTA per node, both signs from the same h_l(p);
// moments in FP64 as the stage kernel forms them.
// ---------------------------------------------------------------------------
template <int NMAX>
__global__ void __launch_bounds__(256) quad_coef_kernel(const GroupDev g, const double* __restrict__ fs) {
    __shared__ double red[8][2 * NMAX];
    __shared__ double sMom[8];
    const int node = blockIdx.x;
    const int ii = g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0;
    const InstDev& I = g.inst[ii];
    if (I.inv_Kn == 0.0) return;                // collisionless: no equilibrium is formed
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int V = g.V, QX2 = g.QX2, VY = g.VY, Nx = g.Nx;
    const double* f = fs + I.f_off + (size_t)(node - I.node_off) * V;
    // moments of the node
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, a4 = 0.0;
    for (int v = tid; v < V; v += blockDim.x) {
        const double val = f[v];
        const double px = g.pd[v % QX2], py = g.pd[QX2 + (v / QX2) % VY], pz = g.pd[QX2 + VY + v / (QX2 * VY)];
        a0 += val;
        a1 += px * val;
        a2 += py * val;
        a3 += pz * val;
        a4 += (px * px + py * py + pz * pz) * val;
    }
    a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2); a3 = warp_sum(a3); a4 = warp_sum(a4);
    if (lane == 0) { red[warp][0] = a0; red[warp][1] = a1; red[warp][2] = a2; red[warp][3] = a3; red[warp][4] = a4; }
    __syncthreads();
    if (tid == 0) {
        double m[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w < nw; ++w)
            for (int k = 0; k < 5; ++k) m[k] += red[w][k];
        const double n = m[0], ux = m[1] / n, uy = m[2] / n, uz = m[3] / n;
        sMom[0] = ux;
        sMom[1] = (m[4] - n * (ux * ux + uy * uy + uz * uz)) / (g.D * n);
    }
    __syncthreads();
    const double ux = sMom[0], T = sMom[1];
    const double sT = sqrt(T), width = sT;
    const int panels = (int)ceil((fabs(ux) + 15.0 * sT) / width);
    const int npts = panels * kQuadNodes;
    const double norm = 1.0 / (kSqrt2Pi * sT), i2T = 0.5 / T;
    const double* ra = g.rec;
    const double* rb = g.rec + Nx;
    const double* rc = g.rec + 2 * Nx;
    const double h00 = g.rec[3 * Nx];
    double Gp[NMAX], Gm[NMAX];
#pragma unroll
    for (int l = 0; l < NMAX; ++l) Gp[l] = Gm[l] = 0.0;
    for (int k = tid; k < npts; k += blockDim.x) {
        const int pnl = k / kQuadNodes, i = k - pnl * kQuadNodes;
        const double p = (pnl + 0.5 * (1.0 + g.glrule[i])) * width;
        const double w0 = 0.5 * width * g.glrule[kQuadNodes + i] * norm;
        const double dp = p - ux, dm = p + ux;
        const double wp = w0 * exp(-dp * dp * i2T), wm = w0 * exp(-dm * dm * i2T);
        double hm = 0.0, h = h00;
        Gp[0] += wp * h;
        Gm[0] += wm * h;
#pragma unroll
        for (int l = 0; l < NMAX - 1; ++l) {
            if (l < Nx) {
                const double hn = (ra[l] * p + rb[l]) * h + rc[l] * hm;
                hm = h;
                h = hn;
                Gp[l + 1] += wp * h;
                Gm[l + 1] += wm * h;
            }
        }
    }
    __syncthreads();                            // red[] is reused below
#pragma unroll
    for (int l = 0; l < NMAX; ++l) {
        if (l <= Nx) {
            const double sp = warp_sum(Gp[l]), sm = warp_sum(Gm[l]);
            if (lane == 0) { red[warp][l] = sp; red[warp][NMAX + l] = sm; }
        }
    }
    __syncthreads();
    double* out = g.gquad + (size_t)node * 2 * (Nx + 1);
    for (int t = tid; t < 2 * (Nx + 1); t += blockDim.x) {
        const int sg = t / (Nx + 1), l = t - sg * (Nx + 1);
        double acc = 0.0;
        for (int w = 0; w < nw; ++w) acc += red[w][sg * NMAX + l];
        out[t] = acc;
    }
}

// ---------------------------------------------------------------------------
// state initialisation, moments (FP64 output), residual
// ---------------------------------------------------------------------------
template <typename R>
__global__ void broadcast_kernel(R* __restrict__ f, const R* __restrict__ g, long long nvalues, int V) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvalues;
         i += (long long)gridDim.x * blockDim.x)
        f[i] = g[i % V];
}

// One warp per node, one pass over the node's values: the raw quadrature sums
// n, j, P_xa = sum p_x p_a f, E = sum |p|^2 f and Q = sum p_x |p|^2 f, from which
// (FP64, per node)
//   u = j/n,  T = (E - n|u|^2)/(D n),
//   q_x = (1/2) sum (p_x - u_x)|p - u|^2 f
//       = (1/2) [Q - 2 (u_x P_xx + u_y P_xy + u_z P_xz) - u_x E + 2 n u_x |u|^2].
// Lanes and the warp tree accumulate in the state's precision, compensated for
// FP32 states (sum and error term); the per-node combination is FP64.  With
// 4 | 2Q_x and 2Q_x | 128 the lanes read 4-vectors whose p_x are fixed per
// lane (as in sums_kernel); otherwise a shared table of (p_x, p_y, p_z) per
// velocity (up to kMomentTableMax velocities) or per-value index arithmetic.
template <typename R, typename R4>
__device__ __forceinline__ R4 velocity_of(const R* P, int v, int QX2, int VY) {
    R4 m;
    m.x = P[v % QX2]; m.y = P[QX2 + (v / QX2) % VY]; m.z = P[QX2 + VY + v / (QX2 * VY)]; m.w = R(0);
    return m;
}

constexpr int kMomentTableMax = 1536;

template <typename R, bool kTable>
__global__ void __launch_bounds__(256)
moments_kernel(const GroupDev g, const R* __restrict__ fs, double* n_out, double* u_out,
               double* T_out, double* q_out, int node_base, const long long* __restrict__ gnode) {
    using R4 = typename std::conditional<sizeof(R) == 4, float4, double4>::type;
    extern __shared__ __align__(16) unsigned char mom_smem[];
    R4* sP = reinterpret_cast<R4*>(mom_smem);            // [V]: p_x, p_y, p_z   (kTable)
    R4* sYZ = sP + (kTable ? g.V : 0);                   // [VY VZ]: p_y, p_z, p_y^2 + p_z^2
    const int V = g.V, QX2 = g.QX2, VY = g.VY, VZ = g.VZ;
    const R* P = static_cast<const R*>(g.p);
    const bool vec4 = (QX2 & 3) == 0 && (QX2 & (QX2 - 1)) == 0 && QX2 <= 128;
    if (kTable) {
        for (int v = threadIdx.x; v < V; v += blockDim.x) sP[v] = velocity_of<R, R4>(P, v, QX2, VY);
        for (int k = threadIdx.x; k < VY * VZ; k += blockDim.x) {
            R4 y;
            y.x = P[QX2 + k % VY]; y.y = P[QX2 + VY + k / VY]; y.z = y.x * y.x + y.y * y.y; y.w = R(0);
            sYZ[k] = y;
        }
        __syncthreads();
    }
    // Nodes go to warps in batches of 32: the warp forms the sums of each node
    // of its batch together (butterfly sums leave them in every lane) and lane
    // k keeps node k's; then every lane finishes its own node in FP64 (on full
    // warps: a lone lane's FP64 instruction costs a whole warp's) and the
    // outputs are written coalesced.
    const int warps = (blockDim.x >> 5) * gridDim.x;
    const int lane = threadIdx.x & 31;
    // 4-vector path with 2Q_x <= 32: eight lanes per node, four nodes of the
    // batch at a time; each lane's p_x stay fixed (its 4-vectors are 8 apart).
    const bool quad = kTable && vec4 && QX2 <= 32;
    for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < g.nnodes; base += warps * 32) {
        const int nb = min(32, g.nnodes - base);
        R mine[9], mine_c[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) mine[k] = mine_c[k] = R(0);
        if (quad) {
            const int sl = lane & 7, lg = __ffs(QX2) - 1;
            const int x0 = (4 * sl) & (QX2 - 1);
            R px[4], px2[4], px3[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                px[e] = P[x0 + e]; px2[e] = px[e] * px[e]; px3[e] = px2[e] * px[e];
            }
            for (int b = 0; 4 * b < nb; ++b) {
                const int node = base + 4 * b + (lane >> 3);
                // n, j_x, j_y, j_z, P_xx, E - P_xx, P_xy, P_xz, Q (compensated for FP32)
                R a[9] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
                R c[9] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
                if (node < base + nb) {
                    const int ii = g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0;
                    const InstDev& I = g.inst[ii];
                    const R4* f4 = reinterpret_cast<const R4*>(fs + (size_t)I.f_off + (size_t)(node - I.node_off) * V);
                    if constexpr (sizeof(R) == 4) {
                        // FP32: the nine sums in the lanes of f32x2 registers, compensated
                        // pairwise (n, j_x), (j_y, j_z), (P_xx, E - P_xx), (P_xy, P_xz), (Q, -)
                        float2 s2[5], c2[5];
#pragma unroll
                        for (int q = 0; q < 5; ++q) s2[q] = c2[q] = make_float2(0.0f, 0.0f);
                        float2 pjx[4], p13[4];                   // (p_x, p_x^2), (1, p_x^3) per element
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            pjx[e] = make_float2((float)px[e], (float)px2[e]);
                            p13[e] = make_float2(1.0f, (float)px3[e]);
                        }
#pragma unroll 4
                        for (int k = sl; k < (V >> 2); k += 8) {
                            const float4 x = reinterpret_cast<const float4*>(f4)[k];
                            const float4 yz = reinterpret_cast<const float4*>(sYZ)[k >> (lg - 2)];
                            const float xe[4] = {x.x, x.y, x.z, x.w};
                            float2 jp = make_float2(0.0f, 0.0f), sq = make_float2(0.0f, 0.0f);   // (j_x, P_xx), (n, Q_x)
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                jp = __ffma2_rn(pjx[e], f2(xe[e]), jp);
                                sq = __ffma2_rn(p13[e], f2(xe[e]), sq);
                            }
                            const float2 yzv = make_float2(yz.x, yz.y);
                            csum_add2(s2[0], c2[0], make_float2(sq.x, jp.x));
                            csum_add2(s2[1], c2[1], __fmul2_rn(yzv, f2(sq.x)));
                            csum_add2(s2[2], c2[2], make_float2(jp.y, yz.z * sq.x));
                            csum_add2(s2[3], c2[3], __fmul2_rn(yzv, f2(jp.x)));
                            csum_add2(s2[4], c2[4], make_float2(fmaf(yz.z, jp.x, sq.y), 0.0f));
                        }
#pragma unroll
                        for (int q = 0; q < 5; ++q) {
                            a[2 * q] = (R)s2[q].x; c[2 * q] = (R)c2[q].x;
                            if (q < 4) { a[2 * q + 1] = (R)s2[q].y; c[2 * q + 1] = (R)c2[q].y; }
                        }
                    } else {
#pragma unroll 4
                    for (int k = sl; k < (V >> 2); k += 8) {
                        const R4 x = f4[k];
                        const R4 yz = sYZ[k >> (lg - 2)];
                        const R sm = (x.x + x.y) + (x.z + x.w);
                        const R jx = px[0] * x.x + px[1] * x.y + px[2] * x.z + px[3] * x.w;
                        const R pxx = px2[0] * x.x + px2[1] * x.y + px2[2] * x.z + px2[3] * x.w;
                        const R pxxx = px3[0] * x.x + px3[1] * x.y + px3[2] * x.z + px3[3] * x.w;
                        csum_add(a[0], c[0], sm); csum_add(a[1], c[1], jx);
                        csum_add(a[2], c[2], yz.x * sm); csum_add(a[3], c[3], yz.y * sm);
                        csum_add(a[4], c[4], pxx); csum_add(a[5], c[5], yz.z * sm);
                        csum_add(a[6], c[6], yz.x * jx); csum_add(a[7], c[7], yz.y * jx);
                        csum_add(a[8], c[8], pxxx + yz.z * jx);
                    }
                    }
                }
                // eight-lane trees; lane L keeps node L's sums (lane 8 (L & 3) of sub-batch L >> 2)
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    csum_warp<R, 4>(a[k], c[k]);
                    const R s2 = __shfl_sync(0xffffffffu, a[k], 8 * (lane & 3));
                    const R c2 = __shfl_sync(0xffffffffu, c[k], 8 * (lane & 3));
                    if ((lane >> 2) == b) { mine[k] = s2; mine_c[k] = c2; }
                }
            }
        }
        for (int kn = 0; kn < (quad ? 0 : nb); ++kn) {
            const int node = base + kn;
            const int ii = g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0;
            const InstDev& I = g.inst[ii];
            const R* f = fs + (size_t)I.f_off + (size_t)(node - I.node_off) * V;
            // n, j_x, j_y, j_z, P_xx, E - P_xx, P_xy, P_xz, Q
            // compensated per-lane sums (FP32 states)
            R a[9] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
            R c[9] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
            if (kTable && vec4) {
                const R4* f4 = reinterpret_cast<const R4*>(f);
                const int x0 = (4 * lane) % QX2;
                R px[4], px2[4], px3[4];
    #pragma unroll
                for (int e = 0; e < 4; ++e) {
                    px[e] = P[x0 + e]; px2[e] = px[e] * px[e]; px3[e] = px2[e] * px[e];
                }
    #pragma unroll 4
                for (int k = lane; k < (V >> 2); k += 32) {
                    const R4 x = f4[k];
                    const R4 yz = sYZ[(k << 2) / QX2];
                    const R sm = (x.x + x.y) + (x.z + x.w);
                    const R jx = px[0] * x.x + px[1] * x.y + px[2] * x.z + px[3] * x.w;
                    const R pxx = px2[0] * x.x + px2[1] * x.y + px2[2] * x.z + px2[3] * x.w;
                    const R pxxx = px3[0] * x.x + px3[1] * x.y + px3[2] * x.z + px3[3] * x.w;
                    csum_add(a[0], c[0], sm); csum_add(a[1], c[1], jx);
                    csum_add(a[2], c[2], yz.x * sm); csum_add(a[3], c[3], yz.y * sm);
                    csum_add(a[4], c[4], pxx); csum_add(a[5], c[5], yz.z * sm);
                    csum_add(a[6], c[6], yz.x * jx); csum_add(a[7], c[7], yz.y * jx);
                    csum_add(a[8], c[8], pxxx + yz.z * jx);
                }
            } else {
                for (int v = lane; v < V; v += 32) {
                    const R val = f[v];
                    const R4 p = kTable ? sP[v] : velocity_of<R, R4>(P, v, QX2, VY);
                    const R jx = p.x * val, yz2 = p.y * p.y + p.z * p.z;
                    csum_add(a[0], c[0], val); csum_add(a[1], c[1], jx);
                    csum_add(a[2], c[2], p.y * val); csum_add(a[3], c[3], p.z * val);
                    csum_add(a[4], c[4], p.x * jx); csum_add(a[5], c[5], yz2 * val);
                    csum_add(a[6], c[6], p.y * jx); csum_add(a[7], c[7], p.z * jx);
                    csum_add(a[8], c[8], (p.x * p.x + yz2) * jx);
                }
            }
            // warp sums in the state's precision (FP64 adds run at 1/64 of FP32 here)
    #pragma unroll
            for (int k = 0; k < 9; ++k) {
                csum_warp(a[k], c[k]);
                if (lane == kn) { mine[k] = a[k]; mine_c[k] = c[k]; }
            }
        }
        if (lane < nb) {
            const int node = base + lane;
            double d[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) d[k] = (double)mine[k] + (double)mine_c[k];
            const double n = d[0];
            const double ux = d[1] / n, uy = d[2] / n, uz = d[3] / n;
            const double u2 = ux * ux + uy * uy + uz * uz;
            const double E = d[4] + d[5];
            const double Tn = (E - n * u2) / (g.D * n);
            const double qx = 0.5 * (d[8] - 2.0 * (ux * d[4] + uy * d[6] + uz * d[7]) - ux * E + 2.0 * n * ux * u2);
            long long o = node_base + node;
            if (gnode) {                    // the caller's layout: instance by instance
                const int k = find_slot(g.node_start, g.ninst, node);
                o = gnode[k] + (node - g.node_start[k]);
            }
            if (n_out) n_out[o] = n;
            if (u_out) { u_out[3 * o] = ux; u_out[3 * o + 1] = uy; u_out[3 * o + 2] = uz; }
            if (T_out) T_out[o] = Tn;
            if (q_out) q_out[o] = qx;
            if (!(isfinite(n) && isfinite(Tn))) *g.nonfinite = 1;
        }
    }
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// Per instance: max |a - b| and max |b| (non-negative doubles order like their bits).
template <typename R>
__global__ void residual_kernel(const GroupDev g, const R* __restrict__ a, const R* __restrict__ b,
                                double* out /* [ninst][2] */) {
    const int warps = (blockDim.x >> 5) * gridDim.x;
    const int lane = threadIdx.x & 31;
    for (int node = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); node < g.nnodes; node += warps) {
        const int ii = g.ninst > 1 ? find_slot(g.node_start, g.ninst, node) : 0;
        const InstDev I = g.inst[ii];
        const size_t off = (size_t)I.f_off + (size_t)(node - I.node_off) * g.V;
        double md = 0.0, mb = 0.0;
        for (int v = lane; v < g.V; v += 32) {
            const double bv = b[off + v];
            md = fmax(md, fabs(bv - (double)a[off + v]));
            mb = fmax(mb, fabs(bv));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
            mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
        }
        if (lane == 0) {
            atomic_max_nonneg(out + 2 * ii, md);
            atomic_max_nonneg(out + 2 * ii + 1, mb);
        }
    }
}

// ---------------------------------------------------------------------------
// host-side launchers (non-template entry points used by hlb_api.cu)
// ---------------------------------------------------------------------------
size_t stage_smem_bytes(const GroupDev& g, int precision, int block) {
    return precision == HLB_FP64_ ? smem_layout<double>(g, block / 32).bytes
                                  : smem_layout<float>(g, block / 32).bytes;
}

template <typename R, int ADV>
static cudaError_t set_attr(size_t smem) {
    return cudaFuncSetAttribute(stage_kernel<R, ADV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t prepare_stage(int precision, int adv, size_t smem) {
    if (precision == HLB_FP64_) return adv == HLB_WENO5_ ? set_attr<double, HLB_WENO5_>(smem) : set_attr<double, HLB_UPWIND2_>(smem);
    return adv == HLB_WENO5_ ? set_attr<float, HLB_WENO5_>(smem) : set_attr<float, HLB_UPWIND2_>(smem);
}

cudaError_t stage_occupancy(int precision, int adv, int block, size_t smem, int* blocks_per_sm) {
    const void* fn;
    if (precision == HLB_FP64_) fn = adv == HLB_WENO5_ ? (const void*)stage_kernel<double, HLB_WENO5_> : (const void*)stage_kernel<double, HLB_UPWIND2_>;
    else fn = adv == HLB_WENO5_ ? (const void*)stage_kernel<float, HLB_WENO5_> : (const void*)stage_kernel<float, HLB_UPWIND2_>;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}

void launch_stage(int precision, int adv, const GroupDev& g, const void* fs, const void* fn, void* fo,
                  int stage, int grid, int block, size_t smem, cudaStream_t st) {
    if (precision == HLB_FP64_) {
        if (adv == HLB_WENO5_) stage_kernel<double, HLB_WENO5_><<<grid, block, smem, st>>>(g, (const double*)fs, (const double*)fn, (double*)fo, stage);
        else stage_kernel<double, HLB_UPWIND2_><<<grid, block, smem, st>>>(g, (const double*)fs, (const double*)fn, (double*)fo, stage);
    } else {
        if (adv == HLB_WENO5_) stage_kernel<float, HLB_WENO5_><<<grid, block, smem, st>>>(g, (const float*)fs, (const float*)fn, (float*)fo, stage);
        else stage_kernel<float, HLB_UPWIND2_><<<grid, block, smem, st>>>(g, (const float*)fs, (const float*)fn, (float*)fo, stage);
    }
}

void launch_quad_coef(const GroupDev& g, const void* fs, cudaStream_t st) {
    if (g.Nx < 24) quad_coef_kernel<24><<<g.nnodes, 256, 0, st>>>(g, (const double*)fs);
    else quad_coef_kernel<32><<<g.nnodes, 256, 0, st>>>(g, (const double*)fs);
}

void launch_wall(int precision, int adv, const GroupDev& g, const void* fs, cudaStream_t st) {
    const int block = 128;
    if (precision == HLB_FP64_) {
        if (adv == HLB_WENO5_) wall_kernel<double, HLB_WENO5_><<<g.nrows * g.wchunks, block, 0, st>>>(g, (const double*)fs);
        else wall_kernel<double, HLB_UPWIND2_><<<g.nrows * g.wchunks, block, 0, st>>>(g, (const double*)fs);
    } else {
        if (adv == HLB_WENO5_) wall_kernel<float, HLB_WENO5_><<<g.nrows * g.wchunks, block, 0, st>>>(g, (const float*)fs);
        else wall_kernel<float, HLB_UPWIND2_><<<g.nrows * g.wchunks, block, 0, st>>>(g, (const float*)fs);
    }
}

void launch_broadcast(int precision, void* f, const void* gvec, long long nvalues, int V, cudaStream_t st) {
    const int block = 256;
    long long blocks = (nvalues + block - 1) / block;
    const int grid = (int)(blocks < 65535LL * 16 ? blocks : 65535LL * 16);
    if (precision == HLB_FP64_) broadcast_kernel<double><<<grid, block, 0, st>>>((double*)f, (const double*)gvec, nvalues, V);
    else broadcast_kernel<float><<<grid, block, 0, st>>>((float*)f, (const float*)gvec, nvalues, V);
}

void launch_moments(int precision, const GroupDev& g, const void* fs, double* n, double* u, double* T,
                    double* q, int node_base, cudaStream_t st, const long long* gnode) {
    const int block = 256;                               // 8 warps, 32 nodes per warp and batch
    const int grid = (g.nnodes + 255) / 256 < 152 * 8 ? (g.nnodes + 255) / 256 : 152 * 8;
    const bool table = g.V + g.VY * g.VZ <= kMomentTableMax;
    if (precision == HLB_FP64_) {
        if (table) moments_kernel<double, true><<<grid, block, (g.V + g.VY * g.VZ) * sizeof(double4), st>>>(g, (const double*)fs, n, u, T, q, node_base, gnode);
        else moments_kernel<double, false><<<grid, block, 0, st>>>(g, (const double*)fs, n, u, T, q, node_base, gnode);
    } else {
        if (table) moments_kernel<float, true><<<grid, block, (g.V + g.VY * g.VZ) * sizeof(float4), st>>>(g, (const float*)fs, n, u, T, q, node_base, gnode);
        else moments_kernel<float, false><<<grid, block, 0, st>>>(g, (const float*)fs, n, u, T, q, node_base, gnode);
    }
}

void launch_residual(int precision, const GroupDev& g, const void* a, const void* b, double* out, cudaStream_t st) {
    const int block = 256;
    const int grid = (g.nnodes + 7) / 8 < 4096 ? (g.nnodes + 7) / 8 : 4096;
    if (precision == HLB_FP64_) residual_kernel<double><<<grid, block, 0, st>>>(g, (const double*)a, (const double*)b, out);
    else residual_kernel<float><<<grid, block, 0, st>>>(g, (const float*)a, (const float*)b, out);
}

}  // namespace hlb

// ---------------------------------------------------------------------------
// FP32 FMA throughput of the device (the ALU roof of the FP32 stage kernels):
// every thread runs kFmaChains independent chains of dependent FMAs (scalar
// fmaf, or packed f32x2 __ffma2_rn counting two FMAs each), enough warps per SM
// to cover the pipeline latency; the result is written so that no chain is
// dropped.
// ---------------------------------------------------------------------------
namespace hlb {
namespace {
constexpr int kFmaChains = 8, kFmaIters = 4096;

__global__ void __launch_bounds__(256) fma_peak_kernel(float* out, float a, float b) {
    float x[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) x[c] = threadIdx.x * 1e-7f + c;
#pragma unroll 16
    for (int i = 0; i < kFmaIters; ++i)
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma2_peak_kernel(float* out, float a, float b) {
    float2 x[kFmaChains / 2];
#pragma unroll
    for (int c = 0; c < kFmaChains / 2; ++c) x[c] = make_float2(threadIdx.x * 1e-7f + c, c + 0.5f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 16
    for (int i = 0; i < kFmaIters; ++i)
#pragma unroll
        for (int c = 0; c < kFmaChains / 2; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kFmaChains / 2; ++c) s += x[c].x + x[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

cudaError_t measure_fp32_peak(int packed, double* tflops) {
    int dev = 0, nsm = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int block = 256, grid = nsm * 8;          // 64 warps per SM
    float* out = nullptr;
    e = cudaMalloc(&out, (size_t)grid * block * sizeof(float));
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 0.0f;
    for (int rep = 0; rep < 4; ++rep) {             // the first launch is a warm-up
        cudaEventRecord(e0);
        if (packed) fma2_peak_kernel<<<grid, block>>>(out, 0.999f, 1e-3f);
        else fma_peak_kernel<<<grid, block>>>(out, 0.999f, 1e-3f);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * kFmaChains * (double)kFmaIters * grid * block;
    *tflops = flops / (best * 1e-3) / 1e12;
    return cudaSuccess;
}
}  // namespace hlb
