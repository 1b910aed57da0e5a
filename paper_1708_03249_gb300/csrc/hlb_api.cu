// C ABI of libhlb: handle management, tables upload, RK-3 stepping (eager or
// replayed from a captured CUDA graph), moments, state I/O and diagnostics.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "hlb.h"
#include "hlb_internal.h"

namespace {

thread_local std::string g_last_error;

hlb_status fail(hlb_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

// Allocation-failure injection (hlb_set_alloc_fail_test): when armed with
// n > 0, the n-th device or page-locked allocation from then on fails as if
// memory were exhausted, and the injection disarms.
std::atomic<long long> g_alloc_countdown{0};

bool injected_alloc_failure() {
    long long c = g_alloc_countdown.load();
    while (c > 0) {
        if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
    }
    return false;
}

cudaError_t dev_malloc(void** p, size_t bytes) {
    if (injected_alloc_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t host_malloc(void** p, size_t bytes) {
    if (injected_alloc_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}

#define HLB_CUDA(expr)                                                                 \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(HLB_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

struct PinnedBuf {                           // page-locked host memory
    void* p = nullptr;
    size_t bytes = 0;
    ~PinnedBuf() { if (p) cudaFreeHost(p); }
};

struct Group {
    int precision = HLB_FP32, adv = HLB_WENO5;   // precision: HLB_FP64 or HLB_FP32 (the state's type)
    int force_request = 0;                   // 0: the library's choice; 1: 3xTF32; 2: split-BF16 (FP32 state)
    int force_form = 0;                      // resolved: 0 FMA, 1 3xTF32, 2 split-BF16
    int Qx = 0, Qy = 0, Qz = 0, Nx = 0, Ny = 0, Nz = 0;
    bool x_full = false;                     // p_x on the full-range Gauss-Hermite axis
    hlb::AxisTables tx, ty, tz;
    int V = 0, QX2 = 0, VY = 1, VZ = 1;
    size_t esize = 4;
    std::vector<int> members;               // handle-level instance ids
    std::vector<hlb::InstDev> inst;
    std::vector<int> node_start, row_start;
    std::vector<double> dx_all;
    long long nvalues = 0;
    int nnodes = 0, nrows = 0;
    DevBuf buf[3];
    int cur = 0, prev = -1;
    DevBuf d_inst, d_node_start, d_row_start, d_K, d_p, d_pd, d_T, d_rec, d_dx, d_gw, d_nw, d_resid;
    DevBuf d_mom;                            // moments scratch: 6 doubles per node
    DevBuf d_gnode;                          // [members]: each member's first node in the caller's layout
    PinnedBuf h_mom;                         // pinned word for the non-finite flag (hlb_moments), first use
    DevBuf d_Td, d_invdx, d_wscale, d_coef, d_works, d_err, d_recf, d_Tf, d_sums;
    DevBuf d_KxT, d_KxJ;                     // FP64 Kx transposed and its jump factors (kx_global groups only)
    DevBuf d_gquad, d_glrule;                // G^{+-} by quadrature above the recurrence's stable order (FP64)
    DevBuf d_wpart, d_wcount;                // wall kernel: per-chunk partial fluxes, row counters
    int wchunks = 1;
    bool quad_x = false;
    int vchunks = 1;                         // CTAs per node of the generic stage kernel
    hlb::GroupDev dev{};
    int block = 256, grid = 1;
    size_t smem = 0;
    // marching stage kernel (node + march) or the generic per-node kernel
    int TY = 1, SX = 0, nworks = 0;
    bool march_ok = false;
    // per-node acceleration field (hlb_set_force_field): [nnodes][3] doubles,
    // allocated on first use; one flag per member instance
    DevBuf d_afield;
    std::vector<char> field_on;
    bool has_field = false;
    bool sround = false;                     // FP32 stage outputs rounded stochastically (hlb_set_rounding)
    const void* mom_buf = nullptr;           // state buffer read by a pending hlb_moments_async
    // persistent batched kernel (1D FP32 groups without a p_z axis): one
    // launch per step; control words [head, abort, pad, pad, node counters
    // [ninst], segment counters [ninst]] zeroed before each launch; the work
    // items of a stage (per instance its node chunks, then its segments),
    // node chunks and segments per instance, resident CTAs
    bool persist_ok = false;
    bool persist_use = true;                 // the autotuner's pick: persistent or per-stage launches
    float tuned_ms_persist = 0.0f, tuned_ms_stages = 0.0f;   // its best step times (0: not timed)
    int persist_per_sm = 0, persist_grid = 0, persist_nitems = 0;
    DevBuf d_pctl, d_nseg, d_nchunk, d_pitems;
};

// Host-side NVTX range (the library's calls and the RK-3 stages they enqueue,
// for profilers; free when no tool is attached).  Ranges opened while a CUDA
// graph is captured mark the capture, not the replays.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

struct KernelTimer {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> stage, wall;
};

}  // namespace

struct hlb_handle {
    std::vector<hlb_config> cfg;
    std::vector<int> inst_group, inst_local;
    std::vector<long long> inst_node_off;    // global node offset of each instance
    std::vector<long long> inst_value_off;   // global value offset of each instance
    std::vector<std::unique_ptr<Group>> groups;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int precision = HLB_FP32;
    long long nsteps = 0;
    long long total_nodes = 0, total_values = 0;
    bool use_graphs = true, time_kernels = false;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    KernelTimer timer;
    double stage_ms = 0, wall_ms = 0;
    long long stage_n = 0, wall_n = 0;
    long long launches = 0;                  // kernels enqueued by hlb_step (graph replays included)
    bool have_residual = false;
    size_t esize = 4;
    // staged state (hlb_prefetch_state / hlb_commit_state): a device buffer in
    // the caller's layout, filled on a copy stream of its own
    void* stage_buf = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t stage_free = nullptr, stage_filled = nullptr;
    bool staged = false;
    // asynchronous moments (hlb_moments_async / hlb_moments_wait): a result
    // stream of the handle's own; mom_done completes when the last request's
    // copies have landed; each group records the state buffer it reads
    cudaStream_t mom_stream = nullptr;
    cudaEvent_t mom_state = nullptr, mom_done = nullptr;
    bool mom_pending = false;
    // velocity-set groups after the first step on streams of their own (the
    // groups share no data within a step): forked from and joined back into
    // the handle's stream, also inside a captured graph
    std::vector<cudaStream_t> group_stream;
    std::vector<cudaEvent_t> group_done;
    cudaEvent_t step_fork = nullptr;
    bool persistent = true;                  // eligible groups step with the persistent kernel
    // device-to-device state copies between the caller's layout and the
    // groups' buffers (commit of a staged state, the _dev state I/O): chunks
    // of at most kRegroupChunk bytes, group by group, copied by one launch per
    // group instead of one cudaMemcpyAsync per instance; built on first use
    void* d_regroup = nullptr;
    std::vector<int> regroup_first;          // per group: its first chunk (size ngroups + 1)
    int regroup_state = 0;                   // 0 not built, 1 built, -1 a layout the kernel cannot take
    // moments of a handle with several instances, in the caller's layout
    // (n [N], u [3N], T [N], q [N], N = total_nodes): written there by the
    // moments kernels directly, then read back in four copies; first use
    DevBuf d_mom_global;
};

namespace {

std::string check_config(const hlb_config& c, int i) {
    auto bad = [&](const char* what) { return "instance " + std::to_string(i) + ": " + what; };
    if (c.Qx < 1 || c.Qx > hlb::kMaxQHalf) return bad("Qx must be in [1, 32], or up to 200 for the half-range Hermite axis");
    if (c.Qx > hlb::kMaxQ && c.x_basis == HLB_X_HALF_RANGE && c.precision != HLB_FP64)
        return bad("Qx > 32 needs HLB_FP64 (the weights fall below the FP32 range)");
    if (c.Qx > hlb::kMaxQ && c.x_basis != HLB_X_HALF_RANGE) return bad("Qx must be in [1, 32]");
    if (c.x_basis != HLB_X_HALF_RANGE && c.x_basis != HLB_X_FULL_RANGE && c.x_basis != HLB_X_HALF_LAGUERRE)
        return bad("x_basis must be HLB_X_HALF_RANGE, HLB_X_FULL_RANGE or HLB_X_HALF_LAGUERRE");
    if (c.x_basis == HLB_X_HALF_LAGUERRE && c.Qx > hlb::kMaxQLaguerre) return bad("Gauss-Laguerre Qx must be in [1, 16]");
    if (c.x_basis == HLB_X_FULL_RANGE && (c.Qx < 2 || c.Qx % 2)) return bad("full-range Qx must be even in [2, 32]");
    for (int q : {c.Qy, c.Qz})
        if (q < 0 || q > hlb::kMaxQ || (q % 2)) return bad("Qy, Qz must be 0 or even in [2, 32]");
    if (c.Nx_eq >= c.Qx || c.Nx_eq < -1) return bad("Nx_eq must be -1 or in [0, Qx - 1]");
    if ((c.Nx_eq < 0 ? c.Qx - 1 : c.Nx_eq) >= hlb::kMaxN)
        return bad("Nx_eq must be at most 31 (give it explicitly when Qx > 32)");
    if (c.Qy && (c.Ny_eq >= c.Qy || c.Ny_eq < -1)) return bad("Ny_eq must be -1 or in [0, Qy - 1]");
    if (c.Qz && (c.Nz_eq >= c.Qz || c.Nz_eq < -1)) return bad("Nz_eq must be -1 or in [0, Qz - 1]");
    if (c.advection != HLB_WENO5 && c.advection != HLB_UPWIND2) return bad("advection must be HLB_UPWIND2 or HLB_WENO5");
    if (c.precision != HLB_FP32 && c.precision != HLB_FP64 && c.precision != HLB_FP32_TF32X3 &&
        c.precision != HLB_FP32_BF16SPLIT)
        return bad("precision must be HLB_FP64, HLB_FP32, HLB_FP32_TF32X3 or HLB_FP32_BF16SPLIT");
    if (c.nx < (c.advection == HLB_WENO5 ? 6 : 3)) return bad("nx must be >= 6 (WENO5) or >= 3 (upwind2)");
    if (c.ny < 1 || c.ny == 2) return bad("ny must be 1 or >= 3");
    if ((long long)c.nx * c.ny > (1LL << 30)) return bad("nx * ny too large");
    if (!(c.Lx > 0) || !std::isfinite(c.Lx)) return bad("Lx must be > 0");
    if (c.ny > 1 && (!(c.Ly > 0) || !std::isfinite(c.Ly))) return bad("Ly must be > 0");
    if (!(c.stretch_A >= 0 && c.stretch_A < 1)) return bad("stretch_A must be in [0, 1)");
    if (!(c.dt > 0) && !(c.cfl > 0)) return bad("either dt > 0 or cfl > 0");
    if (!std::isfinite(c.dt) || !std::isfinite(c.cfl)) return bad("dt and cfl must be finite");
    if (!(c.T_left > 0) || !(c.T_right > 0) || !std::isfinite(c.T_left) || !std::isfinite(c.T_right))
        return bad("wall temperatures must be finite and > 0");
    if (!std::isfinite(c.ax) || !std::isfinite(c.ay) || !std::isfinite(c.az)) return bad("acceleration must be finite");
    if (!(c.Kn > 0)) return bad("Kn must be > 0 (+INFINITY: collisionless)");
    return "";
}

template <typename T>
hlb_status upload(DevBuf& b, const std::vector<T>& v) {
    if (b.p) { cudaFree(b.p); b.p = nullptr; }
    size_t bytes = std::max<size_t>(v.size() * sizeof(T), 16);
    if (dev_malloc((void**)&b.p, bytes) != cudaSuccess) return fail(HLB_ENOMEM, "cudaMalloc of tables failed");
    if (!v.empty()) HLB_CUDA(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return HLB_OK;
}

template <typename R>
std::vector<R> cast_vec(const std::vector<double>& v) {
    return std::vector<R>(v.begin(), v.end());
}

hlb_status upload_real(DevBuf& b, const std::vector<double>& v, int precision) {
    return precision == HLB_FP64 ? upload(b, v) : upload(b, cast_vec<float>(v));
}

// Wall Maxwellian of a group at temperature Tw (V values, FP64) and its
// emitted-flux denominator for the given wall side.
void wall_maxwellian(const Group& G, double Tw, std::vector<double>& gvec) {
    std::vector<double> gx(G.QX2), gy(G.VY), gz(G.VZ);
    hlb::axis_equilibrium(G.tx, 0.0, Tw, gx.data());
    hlb::axis_equilibrium(G.ty, 0.0, Tw, gy.data());
    hlb::axis_equilibrium(G.tz, 0.0, Tw, gz.data());
    gvec.assign(G.V, 0.0);
    for (int k = 0; k < G.VZ; ++k)
        for (int j = 0; j < G.VY; ++j)
            for (int i = 0; i < G.QX2; ++i) gvec[(k * G.VY + j) * G.QX2 + i] = gx[i] * gy[j] * gz[k];
}

double emitted_denominator(const Group& G, const std::vector<double>& gvec, bool left) {
    double s = 0.0;
    for (int v = 0; v < G.V; ++v) {
        const double px = G.tx.p[v % G.QX2];
        if ((left && px > 0) || (!left && px < 0)) s += px * gvec[v];
    }
    return s;
}

hlb_status upload_inst(Group& G) { return upload(G.d_inst, G.inst); }

hlb_status refresh_walls(hlb_handle* h, Group& G) {
    std::vector<double> all((size_t)G.members.size() * 2 * G.V);
    for (size_t m = 0; m < G.members.size(); ++m) {
        const hlb_config& c = h->cfg[G.members[m]];
        std::vector<double> gl, gr;
        wall_maxwellian(G, c.T_left, gl);
        wall_maxwellian(G, c.T_right, gr);
        G.inst[m].den_left = emitted_denominator(G, gl, true);
        G.inst[m].den_right = emitted_denominator(G, gr, false);
        G.inst[m].gw_off = (int)(m * 2 * G.V);
        std::copy(gl.begin(), gl.end(), all.begin() + m * 2 * G.V);
        std::copy(gr.begin(), gr.end(), all.begin() + m * 2 * G.V + G.V);
    }
    hlb_status s = upload_real(G.d_gw, all, G.precision);
    if (s != HLB_OK) return s;
    return upload_inst(G);
}

constexpr unsigned long long kDefaultWaitNs = 1000000000ull;   // 1 s

// The form the FP32 marching kernels of group G launch with: the resolved
// force-term form, or the FMA form's instantiations with a per-node field (3),
// with stochastic rounding (4), or both (5).
int march_form(const Group& G) {
    if (G.precision != HLB_FP32 || (!G.has_field && !G.sround)) return G.force_form;
    return G.has_field ? (G.sround ? 5 : 3) : 4;
}

void fill_dev(Group& G) {
    hlb::GroupDev& d = G.dev;
    d.V = G.V; d.QX2 = G.QX2; d.VY = G.VY; d.VZ = G.VZ; d.Qx = G.tx.Q; d.x_full = G.x_full ? 1 : 0;
    d.om0 = G.tx.om0;
    {
        const float hi = (float)(-G.tx.om0);
        d.m_om0f = make_float2(hi, (float)(-G.tx.om0 - (double)hi));
    }
    d.Nx = G.Nx; d.Ny = G.Qy ? G.Ny : 0; d.Nz = G.Qz ? G.Nz : 0;
    d.Qy = G.Qy; d.Qz = G.Qz;
    d.D = 1 + (G.Qy > 0) + (G.Qz > 0);
    d.ninst = (int)G.members.size();
    d.nnodes = G.nnodes;
    d.nrows = G.nrows;
    d.inst = (const hlb::InstDev*)G.d_inst.p;
    d.node_start = (const int*)G.d_node_start.p;
    d.row_start = (const int*)G.d_row_start.p;
    d.K = G.d_K.p; d.p = G.d_p.p; d.pd = (const double*)G.d_pd.p; d.Tt = G.d_T.p;
    d.KxT = (const double*)G.d_KxT.p;
    d.KxJ = (const double*)G.d_KxJ.p;
    d.kx_global = G.d_KxT.p ? 1 : 0;
    d.vchunks = G.vchunks;
    d.rec = (const double*)G.d_rec.p; d.dx = (const double*)G.d_dx.p;
    d.gw = G.d_gw.p; d.nw = (double*)G.d_nw.p;
    d.Td = (const double*)G.d_Td.p;
    d.inv_dx = G.d_invdx.p;
    d.wscale = G.d_wscale.p;
    d.coef = G.d_coef.p;
    d.sums = G.d_sums.p;
    d.ncp = ((G.QX2 + G.VY + G.VZ + 1 + 3) + 3) / 4 * 4;      // factors, 1/tau, a_x a_y a_z
    d.field_off = G.QX2 + G.VY + G.VZ + 1;
    d.has_field = G.has_field ? 1 : 0;
    d.afield = static_cast<const double*>(G.d_afield.p);
    d.err = (int*)G.d_err.p;
    d.nonfinite = (int*)G.d_err.p + 1;
    d.recf = (const float2*)G.d_recf.p;
    d.Tf = (const float2*)G.d_Tf.p;
    d.use_df = (G.precision == HLB_FP32 && G.Nx <= 15) ? 1 : 0;
    d.wait_ns = kDefaultWaitNs;
    d.inject_stall = 0;
    // with a field and / or stochastic rounding the FP32 marching kernels run
    // the FMA form's instantiations for them
    d.force_form = march_form(G);
    d.sround = G.sround && G.precision == HLB_FP32 ? 1 : 0;
    d.quad_x = G.quad_x ? 1 : 0;
    d.wchunks = G.wchunks;
    d.wpart = static_cast<double*>(G.d_wpart.p);
    d.wcount = static_cast<unsigned*>(G.d_wcount.p);
    d.gquad = static_cast<double*>(G.d_gquad.p);
    d.glrule = static_cast<const double*>(G.d_glrule.p);
}

// The marching kernel's work list: one CTA per (p_z slab, instance, strip of
// TY rows, x-segment of SX cells).
hlb_status set_segments(hlb_handle* h, Group& G, int SX) {
    G.SX = SX;
    std::vector<hlb::Work> works;
    for (int kz = 0; kz < G.VZ; ++kz)
        for (size_t m = 0; m < G.members.size(); ++m) {
            const hlb_config& c = h->cfg[G.members[m]];
            for (int xa = 0; xa < c.nx; xa += G.SX)
                for (int y0 = 0; y0 < c.ny; y0 += G.TY) {
                    hlb::Work w{};
                    w.inst = (int)m; w.y0 = y0; w.xa = xa; w.xb = std::min(c.nx, xa + G.SX); w.kz = kz;
                    works.push_back(w);
                }
        }
    G.nworks = (int)works.size();
    hlb_status st = upload(G.d_works, works);
    if (st != HLB_OK || !G.persist_ok) return st;
    // the persistent kernel's items of one stage: the node chunks (one cell
    // per thread) of every instance, then the segments of every instance (in
    // the work list's order: instance, then x).  A segment then rarely finds
    // its instance's node chunks unfinished (they were taken long before),
    // and a node chunk of the next stage its instance's segments.
    const int chunk = std::min(G.V, hlb::kPersistNodeChunk);
    std::vector<int> nseg(G.members.size(), 0), nchunk(G.members.size(), 0);
    std::vector<hlb::PersistItem> items;
    for (size_t m = 0; m < G.members.size(); ++m) {
        const int nx = h->cfg[G.members[m]].nx;
        for (int a = 0; a < nx; a += chunk) {
            items.push_back(hlb::PersistItem{0, (int)m, a, std::min(nx, a + chunk)});
            ++nchunk[m];
        }
    }
    for (size_t j = 0; j < works.size(); ++j) {
        items.push_back(hlb::PersistItem{1, works[j].inst, (int)j, 0});
        ++nseg[works[j].inst];
    }
    G.persist_nitems = (int)items.size();
    if ((st = upload(G.d_pitems, items)) != HLB_OK) return st;
    if ((st = upload(G.d_nchunk, nchunk)) != HLB_OK) return st;
    return upload(G.d_nseg, nseg);
}

hlb_status build_group(hlb_handle* h, Group& G) {
    const hlb_config& c0 = h->cfg[G.members[0]];
    G.precision = c0.precision == HLB_FP64 ? HLB_FP64 : HLB_FP32;
    G.force_request = c0.precision == HLB_FP32_TF32X3 ? 1 : (c0.precision == HLB_FP32_BF16SPLIT ? 2 : 0);
    G.adv = c0.advection;
    G.Qx = c0.Qx; G.Qy = c0.Qy; G.Qz = c0.Qz;
    G.Nx = c0.Nx_eq < 0 ? c0.Qx - 1 : c0.Nx_eq;
    G.Ny = c0.Qy ? (c0.Ny_eq < 0 ? c0.Qy - 1 : c0.Ny_eq) : 0;
    G.Nz = c0.Qz ? (c0.Nz_eq < 0 ? c0.Qz - 1 : c0.Nz_eq) : 0;
    G.x_full = c0.x_basis == HLB_X_FULL_RANGE;
    std::string e = G.x_full ? hlb::build_full_x_axis(G.Qx, G.Nx, G.tx)
                             : hlb::build_half_axis(G.Qx, G.Nx, G.tx, c0.x_basis == HLB_X_HALF_LAGUERRE);
    if (!e.empty()) return fail(HLB_EINVAL, e);
    if (G.Qy) { e = hlb::build_full_axis(G.Qy, G.Ny, G.ty); if (!e.empty()) return fail(HLB_EINVAL, e); }
    else hlb::absent_axis(G.ty);
    if (G.Qz) { e = hlb::build_full_axis(G.Qz, G.Nz, G.tz); if (!e.empty()) return fail(HLB_EINVAL, e); }
    else hlb::absent_axis(G.tz);
    G.QX2 = G.tx.count; G.VY = G.ty.count; G.VZ = G.tz.count;
    G.V = G.QX2 * G.VY * G.VZ;
    G.esize = G.precision == HLB_FP64 ? 8 : 4;

    // instances
    G.inst.resize(G.members.size());
    G.node_start.assign(G.members.size() + 1, 0);
    G.row_start.assign(G.members.size() + 1, 0);
    G.dx_all.clear();
    long long nv = 0;
    int nodes = 0, rows = 0;
    for (size_t m = 0; m < G.members.size(); ++m) {
        const hlb_config& c = h->cfg[G.members[m]];
        hlb::InstDev& I = G.inst[m];
        std::vector<double> dx;
        hlb::grid_widths(c.nx, c.Lx, c.stretch_A, dx);
        I.f_off = nv;
        I.node_off = nodes;
        I.row_off = rows;
        I.nx = c.nx;
        I.ny = c.ny;
        I.dx_off = (int)G.dx_all.size();
        G.dx_all.insert(G.dx_all.end(), dx.begin(), dx.end());
        const double dy = c.ny > 1 ? c.Ly / c.ny : 0.0;
        I.inv_dy = c.ny > 1 ? 1.0 / dy : 0.0;
        if (c.dt > 0) {
            I.dt = c.dt;
        } else {
            double maxpx = 0, maxpy = 0;
            for (double p : G.tx.p) maxpx = std::max(maxpx, std::fabs(p));
            for (double p : G.ty.p) maxpy = std::max(maxpy, std::fabs(p));
            double rate = maxpx / *std::min_element(dx.begin(), dx.end());
            if (c.ny > 1) rate += maxpy / dy;
            I.dt = c.cfl / rate;
        }
        I.inv_Kn = std::isinf(c.Kn) ? 0.0 : 1.0 / c.Kn;
        I.ax = c.ax; I.ay = c.ay; I.az = c.az;
        nv += (long long)c.nx * c.ny * G.V;
        nodes += c.nx * c.ny;
        rows += c.ny;
        G.node_start[m + 1] = nodes;
        G.row_start[m + 1] = rows;
    }
    G.nvalues = nv;
    G.nnodes = nodes;
    G.nrows = rows;

    // tables
    std::vector<double> K, p, T, rec;
    K.insert(K.end(), G.tx.K.begin(), G.tx.K.end());
    K.insert(K.end(), G.ty.K.begin(), G.ty.K.end());
    K.insert(K.end(), G.tz.K.begin(), G.tz.K.end());
    p.insert(p.end(), G.tx.p.begin(), G.tx.p.end());
    p.insert(p.end(), G.ty.p.begin(), G.ty.p.end());
    p.insert(p.end(), G.tz.p.begin(), G.tz.p.end());
    T.insert(T.end(), G.tx.T.begin(), G.tx.T.end());
    T.insert(T.end(), G.ty.T.begin(), G.ty.T.end());
    T.insert(T.end(), G.tz.T.begin(), G.tz.T.end());
    rec.insert(rec.end(), G.tx.ra.begin(), G.tx.ra.end());
    rec.insert(rec.end(), G.tx.rb.begin(), G.tx.rb.end());
    rec.insert(rec.end(), G.tx.rc.begin(), G.tx.rc.end());
    rec.insert(rec.end(), G.tx.h0.begin(), G.tx.h0.end());
    rec.insert(rec.end(), G.tx.dcoef.begin(), G.tx.dcoef.end());
    if (G.x_full) rec.assign(5 * (size_t)G.Nx + 1, 0.0);     // the full-range x roles read no recurrence table
    std::vector<double> invdx(G.dx_all.size()), wscale(G.V);
    for (size_t i = 0; i < invdx.size(); ++i) invdx[i] = 1.0 / G.dx_all[i];
    for (int k = 0; k < G.VZ; ++k)
        for (int j = 0; j < G.VY; ++j)
            for (int i = 0; i < G.QX2; ++i)
                // the power of two nearest 1/(w_x w_y w_z): the WENO weights do
                // not change under a common scale, and a power of two makes the
                // FP32 kernels' scaled stencils exact, so that a centre value
                // rebuilt from its scaled copy is the stored one (a rounded
                // scale s fl(1/s) != 1 biases every evolving value each stage,
                // about 5e-9 of the mass per step)
                wscale[(k * G.VY + j) * G.QX2 + i] =
                    std::exp2(std::round(std::log2(1.0 / (G.tx.w[i] * G.ty.w[j] * G.tz.w[k]))));
    if (G.precision == HLB_FP32)
        for (double ws : wscale)
            if (!(ws < 1e36))
                return fail(HLB_EUNSUPPORTED, "velocity set with weights below 1e-36: the FP32 state cannot hold it");
    hlb_status s;
    {
        auto split = [](const std::vector<double>& v) {
            std::vector<float2> out(v.size());
            for (size_t i = 0; i < v.size(); ++i) {
                const float hi = (float)v[i];
                out[i] = make_float2(hi, (float)(v[i] - (double)hi));
            }
            return out;
        };
        if ((s = upload(G.d_recf, split(rec))) != HLB_OK) return s;
        if ((s = upload(G.d_Tf, split(T))) != HLB_OK) return s;
    }
    if ((s = upload(G.d_Td, T)) != HLB_OK) return s;
    if ((s = upload_real(G.d_invdx, invdx, G.precision)) != HLB_OK) return s;
    if ((s = upload_real(G.d_wscale, wscale, G.precision)) != HLB_OK) return s;
    if ((s = upload_real(G.d_K, K, G.precision)) != HLB_OK) return s;
    if (G.QX2 > 2 * hlb::kMaxQ) {
        if (G.tx.jc.size() != (size_t)G.QX2) return fail(HLB_EUNSUPPORTED, "large p_x sets need a half-range axis");
        // Kx beyond the shared-memory budget of the generic stage kernel
        // (400 x 400 doubles at Qx = 200): transposed, so that the threads of a
        // warp read consecutive entries of one column
        std::vector<double> KT((size_t)G.QX2 * G.QX2);
        for (int i = 0; i < G.QX2; ++i)
            for (int j = 0; j < G.QX2; ++j) KT[(size_t)j * G.QX2 + i] = G.tx.K[(size_t)i * G.QX2 + j];
        if ((s = upload(G.d_KxT, KT)) != HLB_OK) return s;
        std::vector<double> J(G.tx.jc);
        J.insert(J.end(), G.tx.jd.begin(), G.tx.jd.end());
        if ((s = upload(G.d_KxJ, J)) != HLB_OK) return s;
    }
    if ((s = upload_real(G.d_p, p, G.precision)) != HLB_OK) return s;
    // FP64 half-range Hermite groups above the recurrence's stable order: the
    // coefficients G^{+-} of every collisional node by quadrature, once per
    // node and stage (quad_coef_kernel)
    if (G.precision == HLB_FP64 && G.tx.half && !G.x_full && c0.x_basis == HLB_X_HALF_RANGE &&
        G.Nx > hlb::kStableRecurrenceN) {
        std::vector<double> gx, gw;
        hlb::gauss_legendre_rule(hlb::kQuadNodes, gx, gw);
        gx.insert(gx.end(), gw.begin(), gw.end());
        if ((s = upload(G.d_glrule, gx)) != HLB_OK) return s;
        if ((s = upload(G.d_gquad, std::vector<double>((size_t)G.nnodes * 2 * (G.Nx + 1), 0.0))) != HLB_OK) return s;
        G.quad_x = true;
    }
    if ((s = upload(G.d_pd, p)) != HLB_OK) return s;
    if ((s = upload_real(G.d_T, T, G.precision)) != HLB_OK) return s;
    if ((s = upload(G.d_rec, rec)) != HLB_OK) return s;
    if ((s = upload(G.d_dx, G.dx_all)) != HLB_OK) return s;
    if ((s = upload(G.d_node_start, G.node_start)) != HLB_OK) return s;
    if ((s = upload(G.d_row_start, G.row_start)) != HLB_OK) return s;
    if ((s = upload(G.d_nw, std::vector<double>((size_t)G.nrows * 2, 0.0))) != HLB_OK) return s;
    if ((s = upload(G.d_resid, std::vector<double>(G.members.size() * 2, 0.0))) != HLB_OK) return s;
    if ((s = upload(G.d_err, std::vector<int>(4, 0))) != HLB_OK) return s;
    {
        // the wall kernel's rows over several CTAs when there are few rows of
        // many velocities (one CTA per row ran the 400-velocity FP64 fluxes of
        // the order-200 set on 8 SMs): chunks of about 64 velocities, up to
        // two CTAs per SM in all
        int dev = 0, nsm = 1;
        HLB_CUDA(cudaGetDevice(&dev));
        HLB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        G.wchunks = std::max(1, std::min((G.V + 63) / 64, (2 * nsm + G.nrows - 1) / G.nrows));
        if (G.wchunks > 1) {
            if ((s = upload(G.d_wpart, std::vector<double>((size_t)G.nrows * G.wchunks * 2, 0.0))) != HLB_OK) return s;
            if ((s = upload(G.d_wcount, std::vector<unsigned>((size_t)G.nrows, 0u))) != HLB_OK) return s;
        }
    }
    if ((s = refresh_walls(h, G)) != HLB_OK) return s;

    // state buffers
    const size_t bytes = (size_t)G.nvalues * G.esize;
    for (auto& b : G.buf) {
        if (dev_malloc((void**)&b.p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(HLB_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes for the state failed");
        }
        HLB_CUDA(cudaMemset(b.p, 0, bytes));
    }
    if (dev_malloc((void**)&G.d_mom.p, std::max<size_t>((size_t)G.nnodes * 6 * sizeof(double), 16)) != cudaSuccess) {
        cudaGetLastError();
        return fail(HLB_ENOMEM, "cudaMalloc of moment scratch failed");
    }
    {
        const int ncp = ((G.QX2 + G.VY + G.VZ + 1 + 3) + 3) / 4 * 4;
        if (dev_malloc((void**)&G.d_coef.p, std::max<size_t>((size_t)G.nnodes * ncp * G.esize, 16)) != cudaSuccess ||
            dev_malloc((void**)&G.d_sums.p, std::max<size_t>((size_t)G.nnodes * 16 * G.esize, 16)) != cudaSuccess) {
            cudaGetLastError();
            return fail(HLB_ENOMEM, "cudaMalloc of the equilibrium factor lines failed");
        }
    }
    // marching kernel: slab = the 2Qx x Qy velocities of one p_z; strips of TY
    // rows (2D) and x-segments sized for enough CTAs to fill the GPU
    {
        bool two_d = false, small_ny = false;
        long long xwork = 0;
        for (size_t m = 0; m < G.members.size(); ++m) {
            const hlb_config& c = h->cfg[G.members[m]];
            if (c.ny > 1) two_d = true;
            xwork += (long long)c.nx * c.ny * G.VZ;
        }
        G.TY = two_d ? 2 : 1;
        for (size_t m = 0; m < G.members.size(); ++m) {
            const hlb_config& c = h->cfg[G.members[m]];
            if ((c.ny > 1) != two_d || (two_d && c.ny < G.TY + 3)) small_ny = true;
        }
        bool big = false;      // the marching kernel indexes an instance with 32-bit offsets
        for (size_t m = 0; m < G.members.size(); ++m) {
            const hlb_config& c = h->cfg[G.members[m]];
            if ((long long)c.nx * c.ny * G.V >= (1LL << 31) - (long long)G.V * 8) big = true;
        }
        G.march_ok = !small_ny && !big && hlb::march_available(G.precision, G.adv, G.QX2, G.VY, G.TY);
        if (G.march_ok) {
            // segment length: about 4096 CTAs in 2D (strips of two rows), about
            // 1216 (8 per SM) over the rows of 1D instances; at least 24 cells
            // so that a CTA's window and table set-up is amortised, at most 512
            const long long rows = xwork / std::max(1LL, (long long)G.TY);
            long long sx = rows / (two_d ? 4096 : 1216);
            sx = std::max(24LL, std::min(512LL, (sx + 5) / 6 * 6));
            // the force term's form (below) decides the persistent kernel's
            // eligibility, and that the segment bound: resolve the form first
            G.force_form = 0;
            if (G.precision == HLB_FP32 && hlb::force_tc_available(G.QX2, G.VY)) {
                if (G.force_request) G.force_form = G.force_request;
                else if (G.TY == 1 && G.QX2 * G.VY >= 512) G.force_form = 1;
                else if (G.TY == 2 && G.adv == HLB_UPWIND2 && G.QX2 * G.VY == 128) G.force_form = 1;
            }
            // persistent batched kernel: 1D FP32 groups without a p_z axis,
            // equilibrium in double-float, the line kernel's slabs
            if (G.precision == HLB_FP32 && G.TY == 1 && G.VZ == 1 && !G.x_full && G.Nx <= 15 &&
                hlb::persist_available(G.QX2, G.VY, G.force_form, std::max(G.Nx, G.Ny))) {
                int per = 0;
                if (hlb::prepare_persist(G.adv, G.QX2, G.VY, G.force_form, &per) == cudaSuccess && per > 0) {
                    int dev = 0, nsm = 1;
                    HLB_CUDA(cudaGetDevice(&dev));
                    HLB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
                    G.persist_ok = true;
                    G.persist_per_sm = per;
                    G.persist_grid = nsm * per;
                    if ((s = upload(G.d_pctl, std::vector<int>(4 + 2 * G.members.size(), 0))) != HLB_OK) return s;
                } else {
                    cudaGetLastError();
                }
            }
            if ((s = set_segments(h, G, (int)sx)) != HLB_OK) return s;
            // the force term's form (set above): on the tensor cores where the
            // caller asked for it and the slab tiles into 16 x 8 x 8 blocks;
            // by default where 3xTF32 measured faster than the FMA loop on a
            // GB300: the 1D kernel's 32 x 16 slabs (0.412 against 0.523 ms
            // per stage, 131072 cells) and the 2D kernel's 16 x 8 slabs with
            // upwind2 (2.06 against 2.39 ms, 1024 x 512 cells, 1024
            // velocities); with WENO-5 the 2D kernel is issue-bound and the
            // FMA loop is faster (3.43 against 3.64 ms; 32 x 16: 0.330
            // against 0.347 ms)
            HLB_CUDA(hlb::prepare_march(G.precision, G.adv, G.QX2, G.VY, G.TY, G.force_form));
            HLB_CUDA(hlb::prepare_node());
        }
    }
    fill_dev(G);

    // launch shape of the stage kernel.  With Kx in global memory each
    // velocity's force term is a 2Qx-term dot product (FP64), so the velocities
    // of a node are split over several CTAs (the balanced split below); the
    // CTAs of one node form its moments redundantly.
    int per_sm = 1, dev = 0, nsm = 1;
    HLB_CUDA(cudaGetDevice(&dev));
    HLB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    G.vchunks = 1;
    auto block_of = [&](int vc) { return std::min(256, std::max(32, ((G.V + vc - 1) / vc + 31) / 32 * 32)); };
    if (G.d_KxT.p) {
        // about 64 velocities per CTA at most, and enough CTAs for the two per
        // SM the stage kernel is compiled for (measured against a split that
        // minimised rounds times CTA size: 0.0927 against 0.0985 ms per stage
        // launch on the eight-case order-200 handle)
        const int by_size = (G.V + 63) / 64;
        const int by_fill = (2 * nsm + G.nnodes - 1) / G.nnodes;
        G.vchunks = std::max(1, std::min(by_size, by_fill));
    }
    fill_dev(G);
    G.block = block_of(G.vchunks);
    G.smem = hlb::stage_smem_bytes(G.dev, G.precision, G.block);
    if (G.smem > 200 * 1024) return fail(HLB_EUNSUPPORTED, "velocity set too large for the stage kernel's shared memory");
    HLB_CUDA(hlb::prepare_stage(G.precision, G.adv, G.smem));
    HLB_CUDA(hlb::stage_occupancy(G.precision, G.adv, G.block, G.smem, &per_sm));
    const long long items = (long long)G.nnodes * G.vchunks;
    G.grid = (int)std::max(1LL, std::min(items, (long long)nsm * std::max(1, per_sm)));
    return HLB_OK;
}

// The marching kernel keeps one p_z per CTA; a force along p_z mixes them (a
// field may have a p_z component: groups with a field and a p_z axis take the
// per-node kernel).
bool group_has_z_force(const hlb_handle* h, const Group& G) {
    if (!G.Qz) return false;
    if (G.has_field) return true;
    for (int i : G.members)
        if (h->cfg[i].az != 0.0) return true;
    return false;
}

// Make stream s wait, on the device, for the pending asynchronous moments
// (their kernels read a state buffer and reuse the moments scratch).
void wait_moments(hlb_handle* h, cudaStream_t s) {
    if (h->mom_pending) cudaStreamWaitEvent(s, h->mom_done, 0);
}

// One RK-3 step of one group on stream st: three (node pass, wall, stage)
// triples; buffer roles rotate.
// Whether group G steps with the persistent kernel: eligible, enabled, not
// timed per stage, no per-node force field (that adds a pass per stage).
bool persist_on(const hlb_handle* h, const Group& G) {
    return G.persist_ok && G.persist_use && G.march_ok && h->persistent && !h->time_kernels && !G.has_field;
}

// One RK-3 step of group G by one launch of the persistent kernel (its
// control words zeroed first).
void enqueue_persist_step(Group& G, cudaStream_t st) {
    NvtxRange range("RK-3 step (persistent)");
    hlb::PersistArgs a{};
    for (int k = 0; k < 3; ++k) a.buf[k] = static_cast<float*>(G.buf[k].p);
    a.cur = G.cur;
    a.nitems = G.persist_nitems;
    a.items = static_cast<const hlb::PersistItem*>(G.d_pitems.p);
    const size_t ninst = G.members.size();
    int* ctl = static_cast<int*>(G.d_pctl.p);
    a.head = ctl;
    a.abort = ctl + 1;
    a.prog_node = reinterpret_cast<unsigned*>(ctl + 4);
    a.prog_march = reinterpret_cast<unsigned*>(ctl + 4 + ninst);
    a.nchunk = static_cast<const int*>(G.d_nchunk.p);
    a.nseg = static_cast<const int*>(G.d_nseg.p);
    cudaMemsetAsync(ctl, 0, (4 + 2 * ninst) * sizeof(int), st);
    hlb::launch_persist(G.adv, G.QX2, G.VY, G.force_form, G.dev, (const hlb::Work*)G.d_works.p, a,
                        std::min(G.persist_grid, 3 * G.persist_nitems), st);
}

void enqueue_group_step(hlb_handle* h, Group& G, cudaStream_t st_) {
    static const char* kStageNames[3] = {"RK-3 stage 1", "RK-3 stage 2", "RK-3 stage 3"};
    if (persist_on(h, G)) {
        enqueue_persist_step(G, st_);
        G.prev = G.cur;
        G.cur = (G.cur + 1) % 3;
        return;
    }
    void* S = G.buf[G.cur].p;
    void* X = G.buf[(G.cur + 1) % 3].p;
    void* Y = G.buf[(G.cur + 2) % 3].p;
    const void* ins[3] = {S, X, Y};
    void* outs[3] = {X, Y, X};
    for (int st = 0; st < 3; ++st) {
        cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
        if (h->time_kernels) {
            cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventCreate(&e2);
            cudaEventRecord(e0, st_);
        }
        NvtxRange range(kStageNames[st]);
        const bool march = G.march_ok && !group_has_z_force(h, G);
        if (G.quad_x) hlb::launch_quad_coef(G.dev, ins[st], st_);
        if (march) hlb::launch_node(G.precision, G.dev, ins[st], st_);
        hlb::launch_wall(G.precision, G.adv, G.dev, ins[st], st_);
        if (h->time_kernels) cudaEventRecord(e1, st_);
        if (march)
            hlb::launch_march(G.precision, G.adv, G.QX2, G.VY, G.TY, G.dev, (const hlb::Work*)G.d_works.p,
                              G.nworks, ins[st], S, outs[st], st, st_);
        else
            hlb::launch_stage(G.precision, G.adv, G.dev, ins[st], S, outs[st], st, G.grid, G.block, G.smem, st_);
        if (h->time_kernels) {
            cudaEventRecord(e2, st_);
            h->timer.wall.push_back({e0, e1});
            h->timer.stage.push_back({e1, e2});
        }
    }
    G.prev = G.cur;
    G.cur = (G.cur + 1) % 3;
}

void enqueue_step(hlb_handle* h) {
    const size_t ng = h->groups.size();
    if (ng == 1 || h->time_kernels || h->group_stream.size() + 1 != ng) {
        for (auto& G : h->groups) enqueue_group_step(h, *G, h->stream);
        return;
    }
    // fork: groups 1.. wait for the work already on the handle's stream
    cudaEventRecord(h->step_fork, h->stream);
    for (size_t k = 1; k < ng; ++k) {
        cudaStreamWaitEvent(h->group_stream[k - 1], h->step_fork, 0);
        enqueue_group_step(h, *h->groups[k], h->group_stream[k - 1]);
        cudaEventRecord(h->group_done[k - 1], h->group_stream[k - 1]);
    }
    enqueue_group_step(h, *h->groups[0], h->stream);
    for (size_t k = 1; k < ng; ++k) cudaStreamWaitEvent(h->stream, h->group_done[k - 1], 0);   // join
}

// Kernels one RK-3 step launches: per stage the node pass (sums, factor
// lines) when the marching kernel runs, the wall kernel and the stage kernel.
long long kernels_per_step(hlb_handle* h) {
    long long n = 0;
    for (auto& G : h->groups)
        n += persist_on(h, *G) ? 1
                               : 3 * ((G->march_ok && !group_has_z_force(h, *G)) ? 4 : 2) + (G->quad_x ? 3 : 0);
    return n;
}

hlb_status collect_timer(hlb_handle* h) {
    HLB_CUDA(cudaStreamSynchronize(h->stream));
    // events shared between the wall and stage lists are destroyed once
    std::vector<cudaEvent_t> owned;
    for (auto& pr : h->timer.wall) {
        float ms = 0;
        cudaEventElapsedTime(&ms, pr.first, pr.second);
        h->wall_ms += ms;
        h->wall_n += 1;
        owned.push_back(pr.first);
    }
    for (auto& pr : h->timer.stage) {
        float ms = 0;
        cudaEventElapsedTime(&ms, pr.first, pr.second);
        h->stage_ms += ms;
        h->stage_n += 1;
        owned.push_back(pr.first);
        owned.push_back(pr.second);
    }
    for (auto e : owned) cudaEventDestroy(e);
    h->timer.wall.clear();
    h->timer.stage.clear();
    return HLB_OK;
}

hlb_status build_graph(hlb_handle* h) {
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    const int per = std::max(1, 10 / (int)h->groups.size());
    h->graph_steps = 3 * per;
    cudaGraph_t graph = nullptr;
    HLB_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    for (int s = 0; s < h->graph_steps; ++s) enqueue_step(h);
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (e != cudaSuccess) return fail(HLB_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    // capture does not execute: restore the buffer phase
    for (auto& G : h->groups) { G->cur = (G->cur + 3 * 100 - h->graph_steps) % 3; }
    e = cudaGraphInstantiate(&h->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(HLB_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return HLB_OK;
}

// Reads and clears the groups' device error words (after a stream sync).
hlb_status check_device_error(hlb_handle* h) {
    HLB_CUDA(cudaStreamSynchronize(h->stream));
    for (auto& G : h->groups) {
        int err = 0;
        HLB_CUDA(cudaMemcpy(&err, G->d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (err) {
            HLB_CUDA(cudaMemset(G->d_err.p, 0, sizeof(int)));
            if (err == HLB_ETIMEOUT)
                return fail(HLB_ETIMEOUT, "a bounded device wait (bulk-copy pipeline) gave up; state is invalid");
            return fail((hlb_status)err, "device error word set");
        }
    }
    return HLB_OK;
}

Group* group_of(hlb_handle* h, int inst, int* local) {
    Group* G = h->groups[h->inst_group[inst]].get();
    if (local) *local = h->inst_local[inst];
    return G;
}

}  // namespace

extern "C" {

const char* hlb_last_error(void) { return g_last_error.c_str(); }
const char* hlb_version(void) { return "libhlb 0.1 (sm_103a)"; }

// Teardown of a handle whose creation failed: the caller's error message is
// the creation's, not whatever the teardown runs into.
static void destroy_keeping_error(hlb_handle* h) {
    const std::string keep = g_last_error;
    hlb_destroy(h);
    g_last_error = keep;
}

hlb_status hlb_create(const hlb_config* cfg, int ninst, void* cuda_stream, hlb_handle** out) {
    g_last_error.clear();
    if (!out) return fail(HLB_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg || ninst < 1) return fail(HLB_EINVAL, "cfg is NULL or ninst < 1");
    for (int i = 0; i < ninst; ++i) {
        std::string e = check_config(cfg[i], i);
        if (!e.empty()) return fail(HLB_EINVAL, e);
        if (cfg[i].precision != cfg[0].precision) return fail(HLB_EINVAL, "all instances must share precision");
    }
    // a handle that fails half-built is torn down like a finished one
    // (streams and events included), not only freed
    std::unique_ptr<hlb_handle, void (*)(hlb_handle*)> h(new hlb_handle(), destroy_keeping_error);
    h->cfg.assign(cfg, cfg + ninst);
    h->precision = cfg[0].precision == HLB_FP64 ? HLB_FP64 : HLB_FP32;
    h->esize = h->precision == HLB_FP64 ? 8 : 4;
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        HLB_CUDA(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    // group by velocity model
    std::map<std::tuple<int, int, int, int, int, int, int, int>, int> key2g;
    h->inst_group.resize(ninst);
    h->inst_local.resize(ninst);
    for (int i = 0; i < ninst; ++i) {
        const hlb_config& c = cfg[i];
        auto key = std::make_tuple(c.Qx, c.Qy, c.Qz, c.Nx_eq < 0 ? c.Qx - 1 : c.Nx_eq,
                                   c.Qy ? (c.Ny_eq < 0 ? c.Qy - 1 : c.Ny_eq) : 0,
                                   c.Qz ? (c.Nz_eq < 0 ? c.Qz - 1 : c.Nz_eq) : 0, c.advection, c.x_basis);
        auto it = key2g.find(key);
        int gi;
        if (it == key2g.end()) {
            gi = (int)h->groups.size();
            key2g[key] = gi;
            h->groups.emplace_back(new Group());
        } else {
            gi = it->second;
        }
        h->inst_group[i] = gi;
        h->inst_local[i] = (int)h->groups[gi]->members.size();
        h->groups[gi]->members.push_back(i);
    }
    for (auto& G : h->groups) {
        hlb_status s = build_group(h.get(), *G);
        if (s != HLB_OK) return s;
    }
    h->inst_node_off.resize(ninst);
    h->inst_value_off.resize(ninst);
    long long nodes = 0, values = 0;
    for (int i = 0; i < ninst; ++i) {
        h->inst_node_off[i] = nodes;
        h->inst_value_off[i] = values;
        const Group* G = h->groups[h->inst_group[i]].get();
        nodes += (long long)cfg[i].nx * cfg[i].ny;
        values += (long long)cfg[i].nx * cfg[i].ny * G->V;
    }
    h->total_nodes = nodes;
    h->total_values = values;
    for (auto& G : h->groups) {
        std::vector<long long> gn;
        for (int i : G->members) gn.push_back(h->inst_node_off[i]);
        hlb_status s = upload(G->d_gnode, gn);
        if (s != HLB_OK) return s;
    }
    if (h->groups.size() > 1) {
        HLB_CUDA(cudaEventCreateWithFlags(&h->step_fork, cudaEventDisableTiming));
        for (size_t k = 1; k < h->groups.size(); ++k) {
            cudaStream_t s2 = nullptr;
            cudaEvent_t e2 = nullptr;
            HLB_CUDA(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
            h->group_stream.push_back(s2);
            HLB_CUDA(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
            h->group_done.push_back(e2);
        }
    }
    *out = h.release();
    return HLB_OK;
}

void hlb_destroy(hlb_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    collect_timer(h);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->mom_stream) { cudaStreamSynchronize(h->mom_stream); cudaStreamDestroy(h->mom_stream); }
    if (h->mom_state) cudaEventDestroy(h->mom_state);
    if (h->mom_done) cudaEventDestroy(h->mom_done);
    if (h->copy_stream) { cudaStreamSynchronize(h->copy_stream); cudaStreamDestroy(h->copy_stream); }
    if (h->stage_free) cudaEventDestroy(h->stage_free);
    if (h->stage_filled) cudaEventDestroy(h->stage_filled);
    if (h->stage_buf) cudaFree(h->stage_buf);
    if (h->d_regroup) cudaFree(h->d_regroup);
    for (cudaStream_t s2 : h->group_stream) { cudaStreamSynchronize(s2); cudaStreamDestroy(s2); }
    for (cudaEvent_t e2 : h->group_done) cudaEventDestroy(e2);
    if (h->step_fork) cudaEventDestroy(h->step_fork);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

hlb_status hlb_set_walls(hlb_handle* h, int inst, double T_left, double T_right) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (inst < -1 || inst >= (int)h->cfg.size()) return fail(HLB_EINVAL, "instance out of range");
    if (!(T_left > 0) || !(T_right > 0) || !std::isfinite(T_left) || !std::isfinite(T_right))
        return fail(HLB_EINVAL, "wall temperatures must be finite and > 0");
    HLB_CUDA(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < (int)h->cfg.size(); ++i)
        if (inst < 0 || i == inst) { h->cfg[i].T_left = T_left; h->cfg[i].T_right = T_right; }
    for (auto& G : h->groups) {
        hlb_status s = refresh_walls(h, *G);
        if (s != HLB_OK) return s;
        fill_dev(*G);
    }
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    return HLB_OK;
}

hlb_status hlb_set_force(hlb_handle* h, int inst, double ax, double ay, double az) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (inst < -1 || inst >= (int)h->cfg.size()) return fail(HLB_EINVAL, "instance out of range");
    if (!std::isfinite(ax) || !std::isfinite(ay) || !std::isfinite(az)) return fail(HLB_EINVAL, "acceleration must be finite");
    HLB_CUDA(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < (int)h->cfg.size(); ++i) {
        if (inst >= 0 && i != inst) continue;
        h->cfg[i].ax = ax; h->cfg[i].ay = ay; h->cfg[i].az = az;
        int l;
        Group* G = group_of(h, i, &l);
        G->inst[l].ax = ax; G->inst[l].ay = ay; G->inst[l].az = az;
    }
    for (auto& G : h->groups) {
        hlb_status s = upload_inst(*G);
        if (s != HLB_OK) return s;
        fill_dev(*G);
    }
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    return HLB_OK;
}

hlb_status hlb_set_force_field(hlb_handle* h, int inst, const double* ax, const double* ay, const double* az) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (inst < 0 || inst >= (int)h->cfg.size()) return fail(HLB_EINVAL, "instance out of range");
    const hlb_config& c = h->cfg[inst];
    const size_t nodes = (size_t)c.nx * c.ny;
    const double* comp[3] = {ax, ay, az};
    for (const double* a : comp)
        if (a)
            for (size_t k = 0; k < nodes; ++k)
                if (!std::isfinite(a[k])) return fail(HLB_EINVAL, "acceleration field must be finite");
    int l;
    Group* G = group_of(h, inst, &l);
    const bool on = ax || ay || az;
    HLB_CUDA(cudaStreamSynchronize(h->stream));
    for (cudaStream_t s2 : h->group_stream) HLB_CUDA(cudaStreamSynchronize(s2));
    if (on && !G->d_afield.p) {
        if (dev_malloc((void**)&G->d_afield.p, (size_t)G->nnodes * 3 * sizeof(double)) != cudaSuccess) {
            G->d_afield.p = nullptr;
            return fail(HLB_ENOMEM, "cudaMalloc of the acceleration field failed");
        }
        HLB_CUDA(cudaMemset(G->d_afield.p, 0, (size_t)G->nnodes * 3 * sizeof(double)));
        // the FP32 marching kernels' field instantiations (FMA force term)
        if (G->march_ok && G->precision == HLB_FP32)
            HLB_CUDA(hlb::prepare_march(G->precision, G->adv, G->QX2, G->VY, G->TY, G->sround ? 5 : 3));
    }
    if (G->field_on.size() != G->members.size()) G->field_on.assign(G->members.size(), 0);
    if (G->d_afield.p) {
        std::vector<double> a(nodes * 3, 0.0);
        for (int k = 0; k < 3; ++k)
            if (comp[k])
                for (size_t j = 0; j < nodes; ++j) a[3 * j + k] = comp[k][j];
        HLB_CUDA(cudaMemcpy((double*)G->d_afield.p + 3 * (size_t)G->node_start[l], a.data(), a.size() * sizeof(double),
                            cudaMemcpyHostToDevice));
    }
    G->field_on[l] = on;
    G->has_field = std::any_of(G->field_on.begin(), G->field_on.end(), [](char f) { return f != 0; });
    fill_dev(*G);                    // the kernels read the field through the factor lines
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    return HLB_OK;
}

hlb_status hlb_set_Kn(hlb_handle* h, int inst, double Kn) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (inst < -1 || inst >= (int)h->cfg.size()) return fail(HLB_EINVAL, "instance out of range");
    if (!(Kn > 0)) return fail(HLB_EINVAL, "Kn must be > 0 (+INFINITY: collisionless)");
    HLB_CUDA(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < (int)h->cfg.size(); ++i) {
        if (inst >= 0 && i != inst) continue;
        h->cfg[i].Kn = Kn;
        int l;
        Group* G = group_of(h, i, &l);
        G->inst[l].inv_Kn = std::isinf(Kn) ? 0.0 : 1.0 / Kn;
    }
    for (auto& G : h->groups) {
        hlb_status s = upload_inst(*G);
        if (s != HLB_OK) return s;
        fill_dev(*G);
    }
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    return HLB_OK;
}

hlb_status hlb_init_equilibrium(hlb_handle* h, double n, double ux, double uy, double T) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (!(n > 0) || !(T > 0) || !std::isfinite(n) || !std::isfinite(T) || !std::isfinite(ux) || !std::isfinite(uy))
        return fail(HLB_EINVAL, "need finite n > 0, T > 0, ux, uy");
    wait_moments(h, h->stream);                         // the state buffer may be read by pending moments
    for (auto& Gp : h->groups) {
        Group& G = *Gp;
        std::vector<double> gx(G.QX2), gy(G.VY), gz(G.VZ), gv(G.V);
        hlb::axis_equilibrium(G.tx, ux, T, gx.data());
        hlb::axis_equilibrium(G.ty, uy, T, gy.data());
        hlb::axis_equilibrium(G.tz, 0.0, T, gz.data());
        for (int k = 0; k < G.VZ; ++k)
            for (int j = 0; j < G.VY; ++j)
                for (int i = 0; i < G.QX2; ++i) gv[(k * G.VY + j) * G.QX2 + i] = n * gx[i] * gy[j] * gz[k];
        DevBuf tmp;
        hlb_status s = upload_real(tmp, gv, G.precision);
        if (s != HLB_OK) return s;
        hlb::launch_broadcast(G.precision, G.buf[G.cur].p, tmp.p, G.nvalues, G.V, h->stream);
        HLB_CUDA(cudaGetLastError());
        HLB_CUDA(cudaStreamSynchronize(h->stream));   // tmp is freed on return
    }
    h->have_residual = false;
    return HLB_OK;
}

hlb_status hlb_step(hlb_handle* h, long nsteps) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (nsteps < 0) return fail(HLB_EINVAL, "nsteps < 0");
    NvtxRange range("hlb_step");
    if (h->mom_pending && nsteps > 0) {
        // one step reads the state the pending moments read and writes the
        // other two buffers, so it need not wait; more steps reuse that buffer
        bool conflict = nsteps > 1;
        for (auto& G : h->groups)
            if (G->mom_buf && (G->buf[(G->cur + 1) % 3].p == G->mom_buf || G->buf[(G->cur + 2) % 3].p == G->mom_buf))
                conflict = true;
        if (conflict) wait_moments(h, h->stream);
    }
    long left = nsteps;
    while (left > 0) {
        const bool phase0 = std::all_of(h->groups.begin(), h->groups.end(), [](const std::unique_ptr<Group>& G) { return G->cur == 0; });
        if (h->use_graphs && !h->time_kernels && phase0) {
            if (!h->graph) {
                hlb_status s = build_graph(h);
                if (s != HLB_OK) return s;
            }
            if (left >= h->graph_steps) {
                HLB_CUDA(cudaGraphLaunch(h->graph, h->stream));
                h->launches += h->graph_steps * kernels_per_step(h);
                for (auto& G : h->groups) { G->prev = (G->cur + 2) % 3; }   // cur returns to 0
                left -= h->graph_steps;
                h->nsteps += h->graph_steps;
                continue;
            }
        }
        enqueue_step(h);
        HLB_CUDA(cudaGetLastError());
        h->launches += kernels_per_step(h);
        left -= 1;
        h->nsteps += 1;
    }
    if (nsteps > 0) h->have_residual = true;
    HLB_CUDA(cudaGetLastError());
    return HLB_OK;
}

hlb_status hlb_moments_dev(hlb_handle* h, double* n_dev, double* u_dev, double* T_dev, double* q_dev) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    wait_moments(h, h->stream);
    if (h->cfg.size() > 1) {          // every group's kernel writes its nodes in place: no copies
        for (auto& Gp : h->groups) {
            Group& G = *Gp;
            hlb::launch_moments(G.precision, G.dev, G.buf[G.cur].p, n_dev, u_dev, T_dev, q_dev, 0, h->stream,
                                (const long long*)G.d_gnode.p);
            HLB_CUDA(cudaGetLastError());
        }
        return HLB_OK;
    }
    for (auto& Gp : h->groups) {
        Group& G = *Gp;
        double* m = (double*)G.d_mom.p;
        hlb::launch_moments(G.precision, G.dev, G.buf[G.cur].p, m, m + G.nnodes, m + 4LL * G.nnodes,
                            m + 5LL * G.nnodes, 0, h->stream);
        HLB_CUDA(cudaGetLastError());
        for (size_t k = 0; k < G.members.size(); ++k) {
            const int i = G.members[k];
            const long long go = h->inst_node_off[i];
            const long long lo = G.node_start[k];
            const long long cnt = G.node_start[k + 1] - G.node_start[k];
            if (n_dev) HLB_CUDA(cudaMemcpyAsync(n_dev + go, m + lo, cnt * 8, cudaMemcpyDeviceToDevice, h->stream));
            if (u_dev) HLB_CUDA(cudaMemcpyAsync(u_dev + 3 * go, m + G.nnodes + 3 * lo, 3 * cnt * 8, cudaMemcpyDeviceToDevice, h->stream));
            if (T_dev) HLB_CUDA(cudaMemcpyAsync(T_dev + go, m + 4LL * G.nnodes + lo, cnt * 8, cudaMemcpyDeviceToDevice, h->stream));
            if (q_dev) HLB_CUDA(cudaMemcpyAsync(q_dev + go, m + 5LL * G.nnodes + lo, cnt * 8, cudaMemcpyDeviceToDevice, h->stream));
        }
    }
    return HLB_OK;
}

// The non-finite flag's pinned word of a group (first use).
static hlb_status ensure_mom_flag(Group& G) {
    if (!G.h_mom.p) {
        if (host_malloc((void**)&G.h_mom.p, 16) != cudaSuccess) {
            cudaGetLastError();
            G.h_mom.p = nullptr;
            return fail(HLB_ENOMEM, "cudaMallocHost of the moments flag failed");
        }
        G.h_mom.bytes = 16;
    }
    return HLB_OK;
}

// Several instances: every group's moments kernel writes its nodes into the
// handle's buffer in the caller's layout, then one copy per requested array
// and one per group's non-finite flag, all on stream st (instead of four
// copies per instance).
static hlb_status moments_global_to_host(hlb_handle* h, double* n, double* u, double* T, double* q, cudaStream_t st) {
    const long long N = h->total_nodes;
    if (!h->d_mom_global.p && dev_malloc(&h->d_mom_global.p, (size_t)N * 6 * sizeof(double)) != cudaSuccess) {
        h->d_mom_global.p = nullptr;
        return fail(HLB_ENOMEM, "cudaMalloc of the moments buffer failed");
    }
    double* gm = (double*)h->d_mom_global.p;
    double* on = n ? gm : nullptr;
    double* ou = u ? gm + N : nullptr;
    double* oT = T ? gm + 4 * N : nullptr;
    double* oq = q ? gm + 5 * N : nullptr;
    for (auto& Gp : h->groups) {
        Group& G = *Gp;
        hlb_status e = ensure_mom_flag(G);
        if (e != HLB_OK) return e;
        HLB_CUDA(cudaMemsetAsync(G.dev.nonfinite, 0, sizeof(int), st));
        hlb::launch_moments(G.precision, G.dev, G.buf[G.cur].p, on, ou, oT, oq, 0, st, (const long long*)G.d_gnode.p);
        HLB_CUDA(cudaGetLastError());
        G.mom_buf = G.buf[G.cur].p;
        HLB_CUDA(cudaMemcpyAsync(G.h_mom.p, G.dev.nonfinite, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    const cudaMemcpyKind d2h = cudaMemcpyDeviceToHost;
    if (n) HLB_CUDA(cudaMemcpyAsync(n, on, (size_t)N * 8, d2h, st));
    if (u) HLB_CUDA(cudaMemcpyAsync(u, ou, (size_t)N * 24, d2h, st));
    if (T) HLB_CUDA(cudaMemcpyAsync(T, oT, (size_t)N * 8, d2h, st));
    if (q) HLB_CUDA(cudaMemcpyAsync(q, oq, (size_t)N * 8, d2h, st));
    return HLB_OK;
}

// A single instance (one group, the caller's layout): the moments kernel into
// the group's scratch, four copies and the non-finite flag, on stream st.
static hlb_status moments_one_to_host(Group& G, double* n, double* u, double* T, double* q, cudaStream_t st) {
    hlb_status e = ensure_mom_flag(G);
    if (e != HLB_OK) return e;
    double* m = (double*)G.d_mom.p;
    const size_t N = (size_t)G.nnodes;
    HLB_CUDA(cudaMemsetAsync(G.dev.nonfinite, 0, sizeof(int), st));
    hlb::launch_moments(G.precision, G.dev, G.buf[G.cur].p, m, m + N, m + 4 * N, m + 5 * N, 0, st);
    HLB_CUDA(cudaGetLastError());
    G.mom_buf = G.buf[G.cur].p;
    const cudaMemcpyKind d2h = cudaMemcpyDeviceToHost;
    if (n) HLB_CUDA(cudaMemcpyAsync(n, m, N * 8, d2h, st));
    if (u) HLB_CUDA(cudaMemcpyAsync(u, m + N, N * 24, d2h, st));
    if (T) HLB_CUDA(cudaMemcpyAsync(T, m + 4 * N, N * 8, d2h, st));
    if (q) HLB_CUDA(cudaMemcpyAsync(q, m + 5 * N, N * 8, d2h, st));
    HLB_CUDA(cudaMemcpyAsync(G.h_mom.p, G.dev.nonfinite, sizeof(int), cudaMemcpyDeviceToHost, st));
    return HLB_OK;
}

hlb_status hlb_moments(hlb_handle* h, double* n, double* u, double* T, double* q) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    NvtxRange range("hlb_moments");
    wait_moments(h, h->stream);                         // the moments scratch is shared
    {
        hlb_status e0 = check_device_error(h);
        if (e0 != HLB_OK) return e0;
    }
    // every group: clear its non-finite flag, launch the moments kernel, copy
    // the moments into the caller's arrays (direct DMA when they are
    // page-locked) and the flag into a small pinned word; then one
    // synchronisation
    hlb_status e = h->cfg.size() > 1 ? moments_global_to_host(h, n, u, T, q, h->stream)
                                     : moments_one_to_host(*h->groups[0], n, u, T, q, h->stream);
    for (auto& Gp : h->groups) Gp->mom_buf = nullptr;  // read on this stream, which synchronises below
    if (e != HLB_OK) return e;
    HLB_CUDA(cudaStreamSynchronize(h->stream));
    bool finite = true;
    for (auto& Gp : h->groups)
        if (*(const int*)Gp->h_mom.p) finite = false;
    if (!finite) return fail(HLB_ENONFINITE, "non-finite moments in the state");
    return HLB_OK;
}

hlb_status hlb_moments_async(hlb_handle* h, double* n, double* u, double* T, double* q) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (!h->mom_stream) {
        HLB_CUDA(cudaStreamCreateWithFlags(&h->mom_stream, cudaStreamNonBlocking));
        HLB_CUDA(cudaEventCreateWithFlags(&h->mom_state, cudaEventDisableTiming));
        HLB_CUDA(cudaEventCreateWithFlags(&h->mom_done, cudaEventDisableTiming));
    }
    // after the work already on the handle's stream (the state to read)
    HLB_CUDA(cudaEventRecord(h->mom_state, h->stream));
    HLB_CUDA(cudaStreamWaitEvent(h->mom_stream, h->mom_state, 0));
    hlb_status e = h->cfg.size() > 1 ? moments_global_to_host(h, n, u, T, q, h->mom_stream)
                                     : moments_one_to_host(*h->groups[0], n, u, T, q, h->mom_stream);
    if (e != HLB_OK) return e;
    HLB_CUDA(cudaEventRecord(h->mom_done, h->mom_stream));
    h->mom_pending = true;
    return HLB_OK;
}

hlb_status hlb_moments_wait(hlb_handle* h) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (!h->mom_pending) return HLB_OK;
    HLB_CUDA(cudaEventSynchronize(h->mom_done));
    h->mom_pending = false;
    bool finite = true;
    for (auto& Gp : h->groups) {
        Gp->mom_buf = nullptr;
        if (Gp->h_mom.p && *(const int*)Gp->h_mom.p) finite = false;
    }
    hlb_status e = check_device_error(h);
    if (e != HLB_OK) return e;
    if (!finite) return fail(HLB_ENONFINITE, "non-finite moments in the state");
    return HLB_OK;
}

hlb_status hlb_sizes(const hlb_handle* h, long long* nodes, long long* values, long long* bytes) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (nodes) *nodes = h->total_nodes;
    if (values) *values = h->total_values;
    if (bytes) *bytes = h->total_values * (long long)h->esize;
    return HLB_OK;
}

hlb_status hlb_get_dt(const hlb_handle* h, int inst, double* dt) {
    if (!h || !dt) return fail(HLB_EINVAL, "handle or dt is NULL");
    if (inst < 0 || inst >= (int)h->cfg.size()) return fail(HLB_EINVAL, "instance out of range");
    const Group* G = h->groups[h->inst_group[inst]].get();
    *dt = G->inst[h->inst_local[inst]].dt;
    return HLB_OK;
}

hlb_status hlb_force_form(const hlb_handle* h, int inst, int* form) {
    if (!h || !form) return fail(HLB_EINVAL, "handle or output is NULL");
    if (inst < 0 || inst >= (int)h->cfg.size()) return fail(HLB_EINVAL, "instance out of range");
    const Group& G = *h->groups[h->inst_group[inst]];
    *form = (G.march_ok && !group_has_z_force(h, G) && !G.has_field) ? G.force_form : 0;
    return HLB_OK;
}

hlb_status hlb_get_nsteps(const hlb_handle* h, long long* nsteps) {
    if (!h || !nsteps) return fail(HLB_EINVAL, "handle or nsteps is NULL");
    *nsteps = h->nsteps;
    return HLB_OK;
}

struct RegroupChunk {
    long long ext, dev;      // byte offsets in the caller's layout and in the group's buffer
    int bytes, pad;
};
constexpr int kRegroupChunk = 1 << 16;

// One chunk per CTA, 16-byte words (every offset and length a multiple of 16).
__global__ void __launch_bounds__(256) regroup_kernel(char* __restrict__ dev, char* __restrict__ ext,
                                                      const RegroupChunk* __restrict__ chunks, int to_ext) {
    const RegroupChunk c = chunks[blockIdx.x];
    const int4* src = reinterpret_cast<const int4*>(to_ext ? dev + c.dev : ext + c.ext);
    int4* dst = reinterpret_cast<int4*>(to_ext ? ext + c.ext : dev + c.dev);
    for (int i = threadIdx.x; i < c.bytes / 16; i += blockDim.x) dst[i] = src[i];
}

// The chunk table of the handle's layout, or regroup_state = -1 if some
// instance's offset or length is not a multiple of 16 bytes.
static hlb_status build_regroup(hlb_handle* h) {
    std::vector<RegroupChunk> ch;
    h->regroup_first.assign(1, 0);
    for (auto& Gp : h->groups) {
        const Group& G = *Gp;
        for (size_t k = 0; k < G.members.size(); ++k) {
            const long long ext = h->inst_value_off[G.members[k]] * (long long)G.esize;
            const long long dev = (long long)G.inst[k].f_off * (long long)G.esize;
            const long long len = (long long)(G.node_start[k + 1] - G.node_start[k]) * G.V * (long long)G.esize;
            if (ext % 16 || dev % 16 || len % 16) {
                h->regroup_state = -1;
                return HLB_OK;
            }
            for (long long o = 0; o < len; o += kRegroupChunk)
                ch.push_back({ext + o, dev + o, (int)std::min<long long>(kRegroupChunk, len - o), 0});
        }
        h->regroup_first.push_back((int)ch.size());
    }
    if (!ch.empty()) {
        if (dev_malloc(&h->d_regroup, ch.size() * sizeof(RegroupChunk)) != cudaSuccess) {
            h->d_regroup = nullptr;
            return fail(HLB_ENOMEM, "cudaMalloc of the regroup table failed");
        }
        HLB_CUDA(cudaMemcpy(h->d_regroup, ch.data(), ch.size() * sizeof(RegroupChunk), cudaMemcpyHostToDevice));
    }
    h->regroup_state = 1;
    return HLB_OK;
}

static hlb_status state_copy(hlb_handle* h, void* ext, size_t bytes, bool to_ext, cudaMemcpyKind kind, bool sync) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (!ext) return fail(HLB_EINVAL, "buffer is NULL");
    if (!to_ext) wait_moments(h, h->stream);            // the state buffer may be read by pending moments
    if (bytes != (size_t)(h->total_values * (long long)h->esize))
        return fail(HLB_EINVAL, "state buffer must be exactly " + std::to_string(h->total_values * (long long)h->esize) + " bytes");
    // device to device across several instances: one launch per group
    if (kind == cudaMemcpyDeviceToDevice && h->cfg.size() > 1 && (reinterpret_cast<uintptr_t>(ext) % 16) == 0) {
        if (h->regroup_state == 0) {
            const hlb_status e = build_regroup(h);
            if (e != HLB_OK) return e;
        }
        if (h->regroup_state == 1) {
            for (size_t gi = 0; gi < h->groups.size(); ++gi) {
                const int c0 = h->regroup_first[gi], n = h->regroup_first[gi + 1] - c0;
                if (n == 0) continue;
                Group& G = *h->groups[gi];
                regroup_kernel<<<n, 256, 0, h->stream>>>((char*)G.buf[G.cur].p, (char*)ext,
                                                         (const RegroupChunk*)h->d_regroup + c0, to_ext ? 1 : 0);
                HLB_CUDA(cudaGetLastError());
            }
            if (sync) HLB_CUDA(cudaStreamSynchronize(h->stream));
            if (!to_ext) h->have_residual = false;
            return HLB_OK;
        }
    }
    for (auto& Gp : h->groups) {
        Group& G = *Gp;
        char* dev = (char*)G.buf[G.cur].p;
        for (size_t k = 0; k < G.members.size(); ++k) {
            const int i = G.members[k];
            const size_t off_ext = (size_t)h->inst_value_off[i] * G.esize;
            const size_t off_dev = (size_t)G.inst[k].f_off * G.esize;
            const size_t len = (size_t)(G.node_start[k + 1] - G.node_start[k]) * G.V * G.esize;
            if (to_ext) HLB_CUDA(cudaMemcpyAsync((char*)ext + off_ext, dev + off_dev, len, kind, h->stream));
            else HLB_CUDA(cudaMemcpyAsync(dev + off_dev, (const char*)ext + off_ext, len, kind, h->stream));
        }
    }
    if (sync) HLB_CUDA(cudaStreamSynchronize(h->stream));
    if (!to_ext) h->have_residual = false;
    return HLB_OK;
}

hlb_status hlb_get_state(hlb_handle* h, void* host_f, size_t bytes) {
    if (h) {
        hlb_status e = check_device_error(h);
        if (e != HLB_OK) return e;
    }
    return state_copy(h, host_f, bytes, true, cudaMemcpyDeviceToHost, true);
}
hlb_status hlb_set_state(hlb_handle* h, const void* host_f, size_t bytes) {
    return state_copy(h, const_cast<void*>(host_f), bytes, false, cudaMemcpyHostToDevice, true);
}
hlb_status hlb_get_state_dev(hlb_handle* h, void* f_dev, size_t bytes) {
    return state_copy(h, f_dev, bytes, true, cudaMemcpyDeviceToDevice, false);
}
hlb_status hlb_set_state_dev(hlb_handle* h, const void* f_dev, size_t bytes) {
    return state_copy(h, const_cast<void*>(f_dev), bytes, false, cudaMemcpyDeviceToDevice, false);
}

hlb_status hlb_prefetch_state(hlb_handle* h, const void* host_f, size_t bytes) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (!host_f) return fail(HLB_EINVAL, "buffer is NULL");
    const size_t total = (size_t)(h->total_values * (long long)h->esize);
    if (bytes != total) return fail(HLB_EINVAL, "state buffer must be exactly " + std::to_string(total) + " bytes");
    if (!h->copy_stream) {
        HLB_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
        HLB_CUDA(cudaEventCreateWithFlags(&h->stage_free, cudaEventDisableTiming));
        HLB_CUDA(cudaEventCreateWithFlags(&h->stage_filled, cudaEventDisableTiming));
    }
    if (!h->stage_buf && dev_malloc((void**)&h->stage_buf, total) != cudaSuccess) {
        h->stage_buf = nullptr;
        return fail(HLB_ENOMEM, "cudaMalloc of the staging buffer failed");
    }
    // the staging buffer is free once the work already on the handle's
    // stream (an earlier commit's copy out of it) has run
    HLB_CUDA(cudaEventRecord(h->stage_free, h->stream));
    HLB_CUDA(cudaStreamWaitEvent(h->copy_stream, h->stage_free, 0));
    wait_moments(h, h->copy_stream);                    // after a swap the staging buffer may be one they read
    HLB_CUDA(cudaMemcpyAsync(h->stage_buf, host_f, total, cudaMemcpyHostToDevice, h->copy_stream));
    HLB_CUDA(cudaEventRecord(h->stage_filled, h->copy_stream));
    h->staged = true;
    return HLB_OK;
}

hlb_status hlb_commit_state(hlb_handle* h) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (!h->staged) return fail(HLB_EINVAL, "no state staged: call hlb_prefetch_state first");
    HLB_CUDA(cudaStreamWaitEvent(h->stream, h->stage_filled, 0));
    // One group whose state layout is the caller's: the staging buffer becomes
    // the state buffer and the old state buffer the next staging buffer (no
    // copy).  The next prefetch writes it only after the work enqueued so far
    // (which may still read it) has run.  A captured graph holds the old
    // pointers, so it is dropped; hlb_step captures a new one when it needs it.
    bool same_layout = h->groups.size() == 1;
    if (same_layout) {
        const Group& G = *h->groups[0];
        same_layout = G.nvalues == h->total_values;
        for (size_t k = 0; same_layout && k < G.members.size(); ++k)
            same_layout = G.inst[k].f_off == h->inst_value_off[G.members[k]];
    }
    if (same_layout) {
        Group& G = *h->groups[0];
        std::swap(G.buf[G.cur].p, h->stage_buf);
        if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
        h->have_residual = false;
        h->staged = false;
        return HLB_OK;
    }
    const hlb_status s = state_copy(h, h->stage_buf, (size_t)(h->total_values * (long long)h->esize), false,
                                    cudaMemcpyDeviceToDevice, false);
    if (s == HLB_OK) h->staged = false;
    return s;
}

hlb_status hlb_diag(hlb_handle* h, double* total_N, double* residual) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    const int ninst = (int)h->cfg.size();
    if (total_N) {
        std::vector<double> n((size_t)h->total_nodes);
        hlb_status s = hlb_moments(h, n.data(), nullptr, nullptr, nullptr);
        if (s != HLB_OK && s != HLB_ENONFINITE) return s;
        for (int i = 0; i < ninst; ++i) {
            const hlb_config& c = h->cfg[i];
            const Group* G = h->groups[h->inst_group[i]].get();
            const int l = h->inst_local[i];
            const double dy = c.ny > 1 ? c.Ly / c.ny : 1.0;
            double acc = 0.0;
            for (int y = 0; y < c.ny; ++y)
                for (int x = 0; x < c.nx; ++x)
                    acc += n[h->inst_node_off[i] + (long long)y * c.nx + x] * G->dx_all[G->inst[l].dx_off + x];
            total_N[i] = acc * dy;
        }
    }
    if (residual) {
        for (int i = 0; i < ninst; ++i) residual[i] = 0.0;
        if (h->have_residual) {
            for (auto& Gp : h->groups) {
                Group& G = *Gp;
                if (G.prev < 0) continue;
                HLB_CUDA(cudaMemsetAsync(G.d_resid.p, 0, G.members.size() * 2 * sizeof(double), h->stream));
                hlb::launch_residual(G.precision, G.dev, G.buf[G.prev].p, G.buf[G.cur].p, (double*)G.d_resid.p, h->stream);
                HLB_CUDA(cudaGetLastError());
                std::vector<double> r(G.members.size() * 2);
                HLB_CUDA(cudaMemcpyAsync(r.data(), G.d_resid.p, r.size() * 8, cudaMemcpyDeviceToHost, h->stream));
                HLB_CUDA(cudaStreamSynchronize(h->stream));
                for (size_t k = 0; k < G.members.size(); ++k)
                    residual[G.members[k]] = r[2 * k + 1] > 0 ? r[2 * k] / (G.inst[k].dt * r[2 * k + 1]) : 0.0;
            }
        }
    }
    return HLB_OK;
}

hlb_status hlb_tables(const hlb_handle* h, int inst, double* px, double* py, double* pz, double* wx,
                      double* wy, double* wz, double* Kx, double* Ky, double* Kz, double* dx) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (inst < 0 || inst >= (int)h->cfg.size()) return fail(HLB_EINVAL, "instance out of range");
    const Group* G = h->groups[h->inst_group[inst]].get();
    auto cp = [](const std::vector<double>& v, double* o) { if (o) std::copy(v.begin(), v.end(), o); };
    cp(G->tx.p, px); cp(G->ty.p, py); cp(G->tz.p, pz);
    cp(G->tx.w, wx); cp(G->ty.w, wy); cp(G->tz.w, wz);
    cp(G->tx.K, Kx); cp(G->ty.K, Ky); cp(G->tz.K, Kz);
    if (dx) {
        const hlb::InstDev& I = G->inst[h->inst_local[inst]];
        std::copy(G->dx_all.begin() + I.dx_off, G->dx_all.begin() + I.dx_off + I.nx, dx);
    }
    return HLB_OK;
}

hlb_status hlb_axis(int Q, int half, double* p, double* w, double* K) {
    hlb::AxisTables ax;
    const int N = std::min(Q - 1, hlb::kMaxN - 1);          // p, w and K do not depend on N
    std::string e = half ? hlb::build_half_axis(Q, std::max(N, 0), ax, half == 2) : hlb::build_full_axis(Q, N, ax);
    if (!e.empty()) return fail(HLB_EINVAL, e);
    if (p) std::copy(ax.p.begin(), ax.p.end(), p);
    if (w) std::copy(ax.w.begin(), ax.w.end(), w);
    if (K) std::copy(ax.K.begin(), ax.K.end(), K);
    return HLB_OK;
}

hlb_status hlb_equilibrium_x(int Qx, int Nx_eq, double u, double T, double* g) {
    if (!g) return fail(HLB_EINVAL, "g is NULL");
    if (!(T > 0) || !std::isfinite(u) || !std::isfinite(T)) return fail(HLB_EINVAL, "need finite u and T > 0");
    const int N = Nx_eq < 0 ? Qx - 1 : Nx_eq;
    if (N >= hlb::kMaxN) return fail(HLB_EINVAL, "Nx_eq must be at most 31");
    hlb::AxisTables ax;
    std::string e = hlb::build_half_axis(Qx, N, ax);
    if (!e.empty()) return fail(HLB_EINVAL, e);
    hlb::axis_equilibrium(ax, u, T, g);
    return HLB_OK;
}

namespace {
// Timing of one group's candidates; errors leave the group on a valid work list.
struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~EventPair() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Persistent groups: the segment length (cells per work item) and the CTAs
// resident per SM, timed over whole persistent steps (one untimed, three
// timed).  A step reads the state buffer and writes the two scratch buffers
// (stage 1 S -> X, stage 2 X -> Y, stage 3 Y -> X), so the state is kept.
hlb_status tune_persist(hlb_handle* h, Group& G, EventPair& ev, int* chosen, float* step_ms) {
    int dev = 0, nsm = 1;
    HLB_CUDA(cudaGetDevice(&dev));
    HLB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int base_sx = G.SX, base_grid = G.persist_grid;
    std::vector<int> per_sm = {G.persist_per_sm};
    if (G.persist_per_sm >= 2) per_sm.push_back(G.persist_per_sm / 2);
    int best_sx = base_sx, best_grid = base_grid;
    float best_ms = -1.0f;
    hlb_status s = HLB_OK;
    for (int sx : {24, 36, 48, 72, 96, 132, 192, 264}) {
        if ((s = set_segments(h, G, sx)) != HLB_OK) break;
        for (int per : per_sm) {
            G.persist_grid = nsm * per;
            for (int round = 0; round < 4; ++round) {
                if (round == 1) cudaEventRecord(ev.e0, h->stream);
                enqueue_persist_step(G, h->stream);
            }
            cudaEventRecord(ev.e1, h->stream);
            float ms = 0.0f;
            cudaError_t e = cudaEventSynchronize(ev.e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.e0, ev.e1);
            if (e != cudaSuccess) { s = fail(HLB_ECUDA, std::string("autotune timing: ") + cudaGetErrorString(e)); break; }
            if (best_ms < 0.0f || ms < best_ms) { best_ms = ms; best_sx = sx; best_grid = G.persist_grid; }
        }
        if (s != HLB_OK) break;
    }
    G.persist_grid = s == HLB_OK ? best_grid : base_grid;
    const hlb_status s2 = set_segments(h, G, s == HLB_OK ? best_sx : base_sx);
    if (s2 != HLB_OK) G.march_ok = false;
    *chosen = G.march_ok ? G.SX : 0;
    *step_ms = best_ms / 3.0f;
    return s != HLB_OK ? s : s2;
}

// One RK-3 step of the per-stage launches (node pass, wall, stage kernel per
// stage), timed over three steps after an untimed one.  The steps read the
// state buffer and write the two scratch buffers; the buffer roles are put
// back, so the state is kept.
hlb_status time_per_stage_step(hlb_handle* h, Group& G, EventPair& ev, float* step_ms) {
    const int cur = G.cur, prev = G.prev;
    const bool use = G.persist_use;
    G.persist_use = false;
    for (int round = 0; round < 4; ++round) {
        if (round == 1) cudaEventRecord(ev.e0, h->stream);
        enqueue_group_step(h, G, h->stream);
        G.cur = cur;
        G.prev = prev;
    }
    cudaEventRecord(ev.e1, h->stream);
    G.persist_use = use;
    float ms = 0.0f;
    cudaError_t e = cudaEventSynchronize(ev.e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.e0, ev.e1);
    if (e != cudaSuccess) return fail(HLB_ECUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
    *step_ms = ms / 3.0f;
    return HLB_OK;
}

hlb_status tune_group_stages(hlb_handle* h, Group& G, EventPair& ev, int* chosen);

// A group the persistent kernel can step: the per-stage launches with their
// best segment length against the persistent kernel with its best segment
// length and grid, whole steps timed; the faster is kept (the results agree
// to FP32 rounding either way).
hlb_status tune_group(hlb_handle* h, Group& G, EventPair& ev, int* chosen) {
    G.persist_use = true;
    if (!persist_on(h, G)) return tune_group_stages(h, G, ev, chosen);
    G.persist_use = false;
    hlb_status s = tune_group_stages(h, G, ev, chosen);
    if (s != HLB_OK) { G.persist_use = true; return s; }
    const int sx_stages = G.SX;
    float ms_stages = 0.0f, ms_persist = 0.0f;
    if ((s = time_per_stage_step(h, G, ev, &ms_stages)) != HLB_OK) { G.persist_use = true; return s; }
    G.persist_use = true;
    if ((s = tune_persist(h, G, ev, chosen, &ms_persist)) != HLB_OK) return s;
    G.tuned_ms_stages = ms_stages;
    G.tuned_ms_persist = ms_persist;
    if (ms_stages < ms_persist) {
        G.persist_use = false;
        s = set_segments(h, G, sx_stages);
        if (s != HLB_OK) G.march_ok = false;
        *chosen = G.march_ok ? G.SX : 0;
    }
    return s;
}

hlb_status tune_group_stages(hlb_handle* h, Group& G, EventPair& ev, int* chosen) {
    // candidates around the heuristic's segment length, multiples of 6 cells
    const int base = G.SX;
    std::vector<int> cand;
    for (int f : {-2, -1, 0, 1, 2}) {
        int sx = f < 0 ? base >> (-f) : base << f;
        sx = std::max(12, std::min(1020, (sx + 5) / 6 * 6));
        if (std::find(cand.begin(), cand.end(), sx) == cand.end()) cand.push_back(sx);
    }
    // each candidate: one untimed and three timed rounds of the three stage
    // launches; inputs are the state buffer (read only) and the two scratch
    // buffers, outputs only the scratch buffers, so the state is kept
    void* S = G.buf[G.cur].p;
    void* X = G.buf[(G.cur + 1) % 3].p;
    void* Y = G.buf[(G.cur + 2) % 3].p;
    const void* ins[3] = {S, X, Y};
    void* outs[3] = {X, Y, X};
    int best = base;
    float best_ms = 0.0f;
    hlb_status s = HLB_OK;
    for (int sx : cand) {
        if ((s = set_segments(h, G, sx)) != HLB_OK) break;
        for (int round = 0; round < 4; ++round) {
            if (round == 1) cudaEventRecord(ev.e0, h->stream);
            for (int st = 0; st < 3; ++st)
                hlb::launch_march(G.precision, G.adv, G.QX2, G.VY, G.TY, G.dev, (const hlb::Work*)G.d_works.p,
                                  G.nworks, ins[st], S, outs[st], st, h->stream);
        }
        cudaEventRecord(ev.e1, h->stream);
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(ev.e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.e0, ev.e1);
        if (e != cudaSuccess) { s = fail(HLB_ECUDA, std::string("autotune timing: ") + cudaGetErrorString(e)); break; }
        if (sx == cand.front() || ms < best_ms) { best_ms = ms; best = sx; }
    }
    // the chosen length (the heuristic's after an error), or no marching at all
    const hlb_status s2 = set_segments(h, G, s == HLB_OK ? best : base);
    if (s2 != HLB_OK) G.march_ok = false;
    *chosen = G.march_ok ? G.SX : 0;
    return s != HLB_OK ? s : s2;
}
}  // namespace

hlb_status hlb_autotune(hlb_handle* h, int* segments_out) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (h->mom_stream) HLB_CUDA(cudaStreamSynchronize(h->mom_stream));
    HLB_CUDA(cudaStreamSynchronize(h->stream));
    for (cudaStream_t s2 : h->group_stream) HLB_CUDA(cudaStreamSynchronize(s2));
    EventPair ev;
    HLB_CUDA(cudaEventCreate(&ev.e0));
    HLB_CUDA(cudaEventCreate(&ev.e1));
    hlb_status result = HLB_OK;
    for (size_t gi = 0; gi < h->groups.size(); ++gi) {
        Group& G = *h->groups[gi];
        const bool marches = G.march_ok && !group_has_z_force(h, G);
        int chosen = marches ? G.SX : 0;
        if (result == HLB_OK && marches) result = tune_group(h, G, ev, &chosen);
        if (segments_out) segments_out[gi] = chosen;
    }
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }   // it holds the old work lists
    h->have_residual = false;
    if (result != HLB_OK) return result;
    return check_device_error(h);
}

hlb_status hlb_fp32_peak(int packed, double* tflops) {
    if (!tflops) return fail(HLB_EINVAL, "tflops is NULL");
    const cudaError_t e = hlb::measure_fp32_peak(packed, tflops);
    if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? HLB_ENOMEM : HLB_ECUDA,
                                      std::string("FP32 peak measurement: ") + cudaGetErrorString(e));
    return HLB_OK;
}

hlb_status hlb_df_special_check(const double* z_dev, int n, double* erf_dev, double* exp_dev) {
    if (n < 0) return fail(HLB_EINVAL, "n < 0");
    if (n > 0 && (!z_dev || !erf_dev || !exp_dev)) return fail(HLB_EINVAL, "buffer is NULL");
    const cudaError_t e = hlb::launch_df_special(z_dev, n, erf_dev, exp_dev);
    if (e != cudaSuccess) return fail(HLB_ECUDA, std::string("double-float check: ") + cudaGetErrorString(e));
    return HLB_OK;
}

hlb_status hlb_set_persistent(hlb_handle* h, int on) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (h->persistent != (on != 0) && h->graph) {     // the captured steps change: re-capture
        HLB_CUDA(cudaStreamSynchronize(h->stream));
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->persistent = on != 0;
    return HLB_OK;
}

hlb_status hlb_set_rounding(hlb_handle* h, int mode) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (mode != HLB_ROUND_NEAREST && mode != HLB_ROUND_STOCHASTIC)
        return fail(HLB_EINVAL, "mode must be HLB_ROUND_NEAREST or HLB_ROUND_STOCHASTIC");
    HLB_CUDA(cudaStreamSynchronize(h->stream));
    for (cudaStream_t s2 : h->group_stream) HLB_CUDA(cudaStreamSynchronize(s2));
    for (auto& Gp : h->groups) {
        Group& G = *Gp;
        G.sround = mode == HLB_ROUND_STOCHASTIC;
        if (G.march_ok && G.precision == HLB_FP32)
            HLB_CUDA(hlb::prepare_march(G.precision, G.adv, G.QX2, G.VY, G.TY, march_form(G)));
        fill_dev(G);
    }
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    return HLB_OK;
}

hlb_status hlb_step_form(const hlb_handle* h, int inst, int* persistent, int* segment_cells, int* ctas,
                         double* tuned_ms) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (inst < 0 || inst >= (int)h->cfg.size()) return fail(HLB_EINVAL, "instance out of range");
    const Group& G = *h->groups[h->inst_group[inst]];
    const bool p = persist_on(h, G);
    if (persistent) *persistent = p ? 1 : 0;
    if (segment_cells) *segment_cells = G.march_ok ? G.SX : 0;
    if (ctas) *ctas = p ? std::min(G.persist_grid, 3 * G.persist_nitems) : (G.march_ok ? G.nworks : G.grid);
    if (tuned_ms) {
        tuned_ms[0] = G.tuned_ms_persist;
        tuned_ms[1] = G.tuned_ms_stages;
    }
    return HLB_OK;
}

hlb_status hlb_set_options(hlb_handle* h, int use_graphs, int time_kernels) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    h->use_graphs = use_graphs != 0;
    if (h->time_kernels != (time_kernels != 0) && h->graph) {   // timed steps launch per stage: re-capture later
        HLB_CUDA(cudaStreamSynchronize(h->stream));
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->time_kernels = time_kernels != 0;
    return HLB_OK;
}

hlb_status hlb_kernel_times(hlb_handle* h, double* stage_ms, long long* stage_launches, double* wall_ms,
                            long long* wall_launches, int reset) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    hlb_status s = collect_timer(h);
    if (s != HLB_OK) return s;
    if (stage_ms) *stage_ms = h->stage_ms;
    if (stage_launches) *stage_launches = h->stage_n;
    if (wall_ms) *wall_ms = h->wall_ms;
    if (wall_launches) *wall_launches = h->wall_n;
    if (reset) { h->stage_ms = h->wall_ms = 0; h->stage_n = h->wall_n = 0; }
    return HLB_OK;
}

hlb_status hlb_launch_count(hlb_handle* h, long long* launches, int reset) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (launches) *launches = h->launches;
    if (reset) h->launches = 0;
    return HLB_OK;
}

hlb_status hlb_set_alloc_fail_test(long long nth) {
    if (nth < 0) return fail(HLB_EINVAL, "nth must be >= 0");
    g_alloc_countdown.store(nth);
    return HLB_OK;
}

hlb_status hlb_set_wait_test(hlb_handle* h, int withhold_copies, double wait_limit_s) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    if (!(wait_limit_s >= 0) || wait_limit_s > 60.0) return fail(HLB_EINVAL, "wait_limit_s must be in [0, 60]");
    const unsigned long long ns = wait_limit_s > 0 ? (unsigned long long)(wait_limit_s * 1e9) : kDefaultWaitNs;
    for (auto& G : h->groups) {
        G->dev.wait_ns = ns;
        G->dev.inject_stall = withhold_copies ? 1 : 0;
    }
    if (h->graph) {                      // the kernels' parameters changed: re-capture
        HLB_CUDA(cudaStreamSynchronize(h->stream));
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return HLB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Moments without any allocation.
//
// Some callers cannot allocate device memory when they read the moments:
// code that runs while a memory pool is exhausted or capped, a host that has
// handed its allocator to another runtime, or a real-time loop that must not
// enter the CUDA allocator at all.  hlb_moments_noalloc serves them: it runs
// the same moments kernel as hlb_moments_dev, but its per-node scratch (six
// doubles per node: n, u_x, u_y, u_z, T, q) is the static device array below
// instead of memory owned by the handle, and it calls no cudaMalloc, no
// cudaFree and no allocating library routine.
// ---------------------------------------------------------------------------
namespace {

constexpr long long kNoAllocMaxNodes = 1LL << 18;          // per group: 12 MiB of doubles

// Shared by every call on a device, kept for the life of the process.
static __device__ __align__(256) double g_noalloc_scratch[6 * kNoAllocMaxNodes];

// Device address of the scratch in the current device's context.  The
// host-side name of the array is only a stand-in, so the address is looked up
// on every call: the lookup allocates nothing, and a cached address would go
// stale if the primary context were reset and the module loaded again.  The
// first lookup in a context loads the module (lazy loading), which is why the
// first call on a device must come before any stream capture.
hlb_status noalloc_scratch(double** out) {
    void* p = nullptr;
    HLB_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    *out = static_cast<double*>(p);
    return HLB_OK;
}

}  // namespace

extern "C" hlb_status hlb_moments_noalloc(hlb_handle* h, double* n_dev, double* u_dev, double* T_dev,
                                          double* q_dev) {
    if (!h) return fail(HLB_EINVAL, "handle is NULL");
    wait_moments(h, h->stream);
    for (auto& Gp : h->groups)
        if (Gp->nnodes > kNoAllocMaxNodes)
            return fail(HLB_EINVAL, "hlb_moments_noalloc: a group of this handle has " +
                                        std::to_string(Gp->nnodes) + " nodes; this entry point handles at most " +
                                        std::to_string(kNoAllocMaxNodes) +
                                        " nodes per group (its static scratch holds 6 doubles per node)");
    double* m = nullptr;
    hlb_status st = noalloc_scratch(&m);
    if (st != HLB_OK) return st;
    // The kernel writes all six entries of every node of the group before
    // they are read, so the scratch needs no clearing between calls.
    for (auto& Gp : h->groups) {
        Group& G = *Gp;
        const long long nn = G.nnodes;
        hlb::launch_moments(G.precision, G.dev, G.buf[G.cur].p, m, m + nn, m + 4 * nn, m + 5 * nn, 0, h->stream);
        HLB_CUDA(cudaGetLastError());
        for (size_t k = 0; k < G.members.size(); ++k) {
            const int i = G.members[k];
            const long long go = h->inst_node_off[i];
            const long long lo = G.node_start[k];
            const long long cnt = G.node_start[k + 1] - G.node_start[k];
            if (n_dev) HLB_CUDA(cudaMemcpyAsync(n_dev + go, m + lo, cnt * 8, cudaMemcpyDeviceToDevice, h->stream));
            if (u_dev) HLB_CUDA(cudaMemcpyAsync(u_dev + 3 * go, m + nn + 3 * lo, 3 * cnt * 8, cudaMemcpyDeviceToDevice, h->stream));
            if (T_dev) HLB_CUDA(cudaMemcpyAsync(T_dev + go, m + 4 * nn + lo, cnt * 8, cudaMemcpyDeviceToDevice, h->stream));
            if (q_dev) HLB_CUDA(cudaMemcpyAsync(q_dev + go, m + 5 * nn + lo, cnt * 8, cudaMemcpyDeviceToDevice, h->stream));
        }
    }
    return HLB_OK;
}
