// Internal declarations shared by the host tables, the API and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

namespace hlb {

// Mirrors of the public enums of hlb.h, usable in device code.
constexpr int HLB_UPWIND2_ = 0, HLB_WENO5_ = 1;
constexpr int HLB_FP64_ = 0, HLB_FP32_ = 1;

constexpr int kMaxQ = 32;          // largest quadrature order per axis
constexpr int kMaxQHalf = 200;     // half-range Hermite p_x (the HHLB(20;200) model): FP64 beyond kMaxQ
constexpr int kMaxQLaguerre = 16;  // half-range Gauss-Laguerre: beyond, weights < 1e-22 and |p| > 50
constexpr int kMaxN = kMaxQ;       // largest equilibrium order + 1
constexpr int kStableRecurrenceN = 12;   // host half-range projections above this order by quadrature

// One momentum axis of the direct-product velocity set (App. A).
struct AxisTables {
    int Q = 0;                       // quadrature order (per half for the half-range axis and
                                     // for the mirrored full-range p_x axis)
    bool half = false;               // half-range Hermite (p_x) or full-range Gauss-Hermite
    bool mirror = false;             // full-range p_x axis laid out +z then -z (two roles, +-u)
    int count = 1;                   // velocities on the axis: 2Q, Q, or 1 if absent
    int N = 0;                       // equilibrium order
    std::vector<double> p, w;        // [count]
    std::vector<double> K;           // [count * count], row-major K[k][k']
    // Equilibrium tables.  Half-range: T[k][l] = w_k h_l(z_k) (k < Q, l <= N),
    // recurrence h_{l+1} = (a_l z + b_l) h_l + c_l h_{l-1}, h0[l] = h_l(0).
    // Full-range: T[j][l] = w_j He_l(z_j) / l!.
    std::vector<double> T;
    std::vector<double> ra, rb, rc, h0;
    // half-range families: omega(0) and d_{l+1} of p_{l+1}' = d_{l+1} p_l - omega(0) p_{l+1}(0) sum ...
    double om0 = 0.0;
    std::vector<double> dcoef;
    // half-range families: the jump term of K, -omega(0)/2 w_k s_k Phi0(z_k) Phi0(z_k'),
    // as c_k = -omega(0)/2 w_k s_k Phi0(z_k) and d_k' = Phi0(z_k') (2Q each); it is
    // the whole of every cross-half block
    std::vector<double> jc, jd;
};

// Build the tables of a half-range (p_x) or full-range (p_y, p_z) axis.
// Returns "" on success or an error message.
std::string build_half_axis(int Q, int N, AxisTables& out, bool laguerre = false);
std::string build_full_axis(int Q, int N, AxisTables& out);
// Full-range Gauss-Hermite of even order Q along p_x, in the layout of the
// half-range axis: p = (+z_1 .. +z_{Q/2}, -z_1 .. -z_{Q/2}) with z ascending,
// w and K^H permuted alike; out.Q = Q/2 and T holds the rows of the +z nodes
// only (g at -z_k with u equals g at +z_k with -u).
std::string build_full_x_axis(int Q, int N, AxisTables& out);
void absent_axis(AxisTables& out);

// g(u, T) on the axis (count values), FP64, by the same recurrences the
// kernels use per node.
void axis_equilibrium(const AxisTables& ax, double u, double T, double* g);

// x-cell widths of the uniform (A = 0) or tanh-stretched grid.
void grid_widths(int nx, double L, double A, std::vector<double>& dx);

// ---------------------------------------------------------------------------
// Device-side descriptors (passed by value to kernels).
// ---------------------------------------------------------------------------
struct InstDev {
    long long f_off;     // first value of the instance in the state arrays
    int node_off;        // first node of the instance (flattened over the group)
    int row_off;         // first (instance, y) row
    int nx, ny;
    int dx_off;          // offset into the concatenated x-cell widths
    double inv_dy;       // 1/dy (0 for a 1D instance)
    double dt;
    double inv_Kn;       // 1/Kn (0: collisionless)
    double ax, ay, az;
    double den_left, den_right;   // sum over emitted populations of p_x g^w
    int gw_off;          // offset of [2][V] wall Maxwellians (values of R)
};

// One CTA of the marching stage kernel: instance, y-strip, x-segment, kz slab.
struct Work {
    int inst, y0, xa, xb, kz, pad0, pad1, pad2;
};

struct GroupDev {
    int V, QX2, VY, VZ, Qx, Nx, Ny, Nz, Qy, Qz, D;
    int ncp;                 // stride of a node's equilibrium-factor line
    void* coef;              // R: [node][ncp] = g_x * n (QX2), g_y (VY), g_z (VZ), 1/tau
    void* sums;              // R: [node][16] = n, j_x, j_y, j_z, E of the stage input at [0..4],
                             //    their compensation terms at [8..12]
    const void* inv_dx;      // R: 1/dx, concatenated per instance (same offsets as dx)
    const void* wscale;      // R: [V] the power of two nearest 1/(w_x w_y w_z) per velocity (WENO
                             //    smoothness scale; exact to apply and to undo)
    int ninst, nnodes, nrows;
    const InstDev* inst;
    const int* node_start;   // [ninst + 1]
    const int* row_start;    // [ninst + 1]
    const void* K;           // R: Kx [QX2^2], Ky [VY^2], Kz [VZ^2] concatenated
    const double* KxT;       // FP64 Kx transposed, [i'][i]: read from global memory by the
                             // generic stage kernel when Kx does not fit in shared memory
    const double* KxJ;       // FP64 [2][QX2]: c_k, d_k of the rank-one cross-half blocks
                             // K[k][k'] = c_k d_k' (k, k' on opposite halves; kx_global)
    int kx_global;           // 1: Kx is not staged in shared memory (KxT is read instead)
    int vchunks;             // CTAs per node of the generic stage kernel (velocity ranges)
    const void* p;           // R: px [QX2], py [VY], pz [VZ]
    const double* pd;        // FP64 copies of px, py, pz
    const void* Tt;          // R: Tx [Qx (Nx+1)], Ty [VY (Ny+1)], Tz [VZ (Nz+1)]
    const double* rec;       // FP64: ra[Nx], rb[Nx], rc[Nx], h0[Nx+1], 1/ra[Nx]
    const double* Td;        // FP64 copies of Tx, Ty, Tz
    const float2* recf;      // double-float (hi, lo) copies of rec
    const float2* Tf;        // double-float (hi, lo) copies of Tx, Ty, Tz
    int use_df;              // FP32 groups with Nx <= 11: equilibrium in double-float
    int x_full;              // p_x on the mirrored full-range axis: the x roles use the
                             // full-range recurrence with +-u_x (rec unused)
    double om0;              // omega(0) of the half-range family (1/sqrt(2 pi) Hermite, 1 Laguerre)
    float2 m_om0f;           // -omega(0) in double-float
    const double* dx;        // FP64 x-cell widths, concatenated per instance
    const void* gw;          // R: wall Maxwellians
    double* nw;              // FP64 [nrows][2] emitted densities
    int* err;                // device error word (0 = ok; else an hlb_status)
    int* nonfinite;          // set by the moments kernel when a node's n or T is not finite
    unsigned long long wait_ns;   // bound of every pipeline wait in the marching kernels
    int inject_stall;        // test hook: nonzero withholds the copies of a marching CTA's second step
    int sround;              // FP32 stage outputs rounded stochastically (hlb_set_rounding), else to nearest
    int force_form;          // FP32 marching kernels: force term by FMA (0), 3xTF32 (1) or split-BF16 (2)
                             // tensor-core products
    // FP64 half-range groups above the recurrence's stable order: the
    // coefficients G^{+-}_l of every collisional node by quadrature of the
    // projection integrals (quad_coef_kernel), read by the stage kernel
    int quad_x;              // 1: G^{+-} come from gquad
    double* gquad;           // [nnodes][2][Nx + 1]
    const double* glrule;    // [2][kQuadNodes]: Gauss-Legendre nodes and weights on [-1, 1]
    // wall kernel: each row's velocities over wchunks CTAs, their partial
    // incident fluxes in wpart [nrows][wchunks][2], summed in chunk order by the
    // row's last CTA (wcount [nrows], zero between launches)
    int wchunks;
    double* wpart;
    unsigned* wcount;
    // per-node acceleration field (hlb_set_force_field): the node pass writes
    // a = a_uniform + a_field(node) into slots field_off .. field_off+2 of the
    // factor line, which every line reserves; afield [nnodes][3] FP64
    int has_field;
    int field_off;
    const double* afield;
};
constexpr int kQuadNodes = 20;   // points per panel of the projection quadrature

}  // namespace hlb

// Launchers (hlb_kernels.cu, hlb_node.cu, hlb_march.cu, hlb_pair.cu, hlb_line.cu).
#include <cuda_runtime.h>
namespace hlb {
size_t stage_smem_bytes(const GroupDev& g, int precision, int block);
cudaError_t prepare_stage(int precision, int adv, size_t smem);
cudaError_t stage_occupancy(int precision, int adv, int block, size_t smem, int* blocks_per_sm);
void launch_stage(int precision, int adv, const GroupDev& g, const void* fs, const void* fn, void* fo,
                  int stage, int grid, int block, size_t smem, cudaStream_t st);
void launch_wall(int precision, int adv, const GroupDev& g, const void* fs, cudaStream_t st);
// G^{+-}_l (l <= Nx) of every collisional node of an FP64 half-range group by
// quadrature of the projection integrals (hlb_kernels.cu)
void launch_quad_coef(const GroupDev& g, const void* fs, cudaStream_t st);
void gauss_legendre_rule(int n, std::vector<double>& x, std::vector<double>& w);
void launch_node(int precision, const GroupDev& g, const void* fs, cudaStream_t st);
cudaError_t prepare_node();
// Marching stage kernel for (QX2, VY, TY); returns false if no instantiation exists.
bool march_available(int precision, int adv, int QX2, int VY, int TY);
cudaError_t prepare_march(int precision, int adv, int QX2, int VY, int TY, int form);
void launch_march(int precision, int adv, int QX2, int VY, int TY, const GroupDev& g, const Work* works,
                  int nworks, const void* fs, const void* fn, void* fo, int stage, cudaStream_t st);
// FP32 marching kernels of hlb_pair.cu (2D strips of two rows) and
// hlb_line.cu (1D rows).
// `form` is the force-term form (GroupDev::force_form); forms 1 and 2 exist for
// the slabs force_tc_available accepts (instantiated in hlb_tc.cu).
bool line_available(int QX2, int VY);
cudaError_t prepare_line(int adv, int QX2, int VY, int form);
void launch_line(int adv, int QX2, int VY, int form, const GroupDev& g, const Work* works, int nworks,
                 const void* fs, const void* fn, void* fo, int stage, cudaStream_t st);
bool pair_available(int QX2, int VY);
cudaError_t prepare_pair(int adv, int QX2, int VY, int form);
void launch_pair(int adv, int QX2, int VY, int form, const GroupDev& g, const Work* works, int nworks,
                 const void* fs, const void* fn, void* fo, int stage, cudaStream_t st);
bool force_tc_available(int QX2, int VY);
cudaError_t prepare_pair_tc(int adv, int QX2, int VY, int form);
cudaError_t prepare_line_tc(int adv, int QX2, int VY, int form);
void launch_pair_tc(int adv, int QX2, int VY, int form, const GroupDev& g, const Work* works, int nworks,
                    const void* fs, const void* fn, void* fo, int stage, cudaStream_t st);
void launch_line_tc(int adv, int QX2, int VY, int form, const GroupDev& g, const Work* works, int nworks,
                    const void* fs, const void* fn, void* fo, int stage, cudaStream_t st);
// Persistent batched kernel (hlb_persist.cu): 1D FP32 groups without a p_z
// axis, one launch per RK-3 step.  The work items of one stage: node chunks
// (kind 0: cells [a, b) of instance inst -> moment sums, factor lines, the
// wall densities of the walls they hold) and x-segments (kind 1: a = index
// into the group's work list), the node chunks of an instance before its
// segments.  The control words (head, abort, progress counters) are zeroed
// before every launch.
constexpr int kPersistNodeChunk = 512;   // cells per node item at most (one thread per cell)
struct PersistItem {
    int kind, inst, a, b;
};
struct PersistArgs {
    float* buf[3];            // the group's three state buffers
    int cur;                  // index of the current state buffer (S) at the step's start
    int nitems;               // work items per stage
    const PersistItem* items; // [nitems]
    int* head;                // work-queue counter
    int* abort;               // nonzero: a wait ran out; every CTA leaves
    unsigned* prog_node;      // [ninst] node items of the step completed per instance
    unsigned* prog_march;     // [ninst] segments of the step completed per instance
    const int* nchunk;        // [ninst] node items per instance and stage
    const int* nseg;          // [ninst] segments per instance and stage
};
bool persist_available(int QX2, int VY, int form, int Nmax);
cudaError_t prepare_persist(int adv, int QX2, int VY, int form, int* blocks_per_sm);
size_t persist_smem_bytes(int QX2, int VY, int form);
void launch_persist(int adv, int QX2, int VY, int form, const GroupDev& g, const Work* works, const PersistArgs& a,
                    int grid, cudaStream_t st);
void launch_broadcast(int precision, void* f, const void* gvec, long long nvalues, int V, cudaStream_t st);
// FP32 FMA throughput of the current device in TFLOP/s (FMA = 2 flop), scalar
// or packed f32x2 (hlb_kernels.cu)
cudaError_t measure_fp32_peak(int packed, double* tflops);
// The double-float exp(-z^2) and erf(z) of the factor-line prelude for n
// device values z (|z| <= 2.5), as doubles (hi + lo), synchronously.
cudaError_t launch_df_special(const double* z, int n, double* erf_out, double* exp_out);
// n, u, T, q of every node of the group (any output may be NULL).  Node j of
// member k goes to index gnode[k] + (j - node_start[k]) of the outputs when
// gnode (device, [ninst]) is given, else to node_base + j.
void launch_moments(int precision, const GroupDev& g, const void* fs, double* n, double* u, double* T,
                    double* q, int node_base, cudaStream_t st, const long long* gnode = nullptr);
void launch_residual(int precision, const GroupDev& g, const void* a, const void* b, double* out,
                     cudaStream_t st);
}  // namespace hlb
