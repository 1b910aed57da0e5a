/*
 * hlb.h -- C ABI of libhlb, the GB300 (sm_103a) time step of the half-range
 * Gauss-Hermite lattice Boltzmann model with a force term
 * (Ambrus, Sofonea, Fournier, Blanco, arXiv:1708.03249).
 *
 * The library advances the discrete Boltzmann-BGK equation with an external
 * force (Eq. "eq:boltzk"; multi-D form Eq. "eq:boltz_multi_k", App. A)
 *     d_t f_k + p_k . grad f_k + a . (grad_p f)_k = -(f_k - feq_k)/tau
 * for a gas between two diffuse-reflecting walls at rest (Sec. V, Eq.
 * "eq:fwall"), walls at x = 0 and x = Lx, periodic in y.  Units: m = 1 and
 * p_0 = 1 (momenta equal velocities); a = F/m.
 *
 *  - momentum set (App. A): p_x on the half-range Gauss-Hermite quadrature
 *    of order Qx per half (2 Qx values, Sec. IV.B.1, Eq. "eq:hh_pk"; up to
 *    the Qx = 200 of the paper's HHLB(20;200) model in FP64; or, by
 *    hlb_config.x_basis, the half-range Gauss-Laguerre quadrature or the
 *    full-range Gauss-Hermite one of the HLB models); p_y and p_z on
 *    full-range Gauss-Hermite quadratures of even order Qy, Qz (Sec. IV.A.1;
 *    0 = axis absent);
 *  - force: (grad_p f)_k = sum_k' K_kk' f_k' per axis, with K^h of Eq.
 *    "eq:hh_Kk_hh" along p_x (the paper's main result: the distributional
 *    derivative across the p_x = 0 jump; K^L of Eq. "eq:hh_Kk_L" for the
 *    Laguerre set, K^H for the full-range one) and K^H of Eq. "eq:H_Kk" along
 *    p_y, p_z; the acceleration is uniform per instance, plus an optional
 *    per-node field (hlb_set_force_field);
 *  - collision: BGK towards feq = n g_x g_y g_z (Eqs. "eq:hh_gk", "eq:H_gk"),
 *    tau = Kn/n (Eq. "eq:tau");
 *  - advection: WENO-5 without epsilon (Sec. IV.C.2, Tab. "weno") or linear
 *    2nd-order upwind, on a uniform or tanh-stretched grid (Eq. "eq:x_eta");
 *  - walls: diffuse reflection with the emitted density fixed by zero net
 *    mass flux (Sec. IV.C.3, Eq. "eq:nplus_def");
 *  - time: the TVD RK-3 of Eq. "eq:rk3".
 *
 * Memory and ownership.  A handle owns all device memory (the state, two
 * stage buffers, tables) and enqueues on the CUDA stream given at creation
 * (or on a stream of its own).  Every pointer argument below is a HOST pointer owned by
 * the caller unless its name ends in _dev; a _dev pointer is device memory
 * owned by the caller, valid for the duration of the call.  The CUDA device
 * is the one current on the calling thread at hlb_create; later calls must
 * be made with that device current.
 *
 * State layout (the "logical state" of get/set_state): for each instance in
 * creation order, f[y][x][kz][jy][ix], ix fastest (2 Qx entries, the first Qx
 * for p_x = +z_k, the next Qx for p_x = -z_k; Qx entries split Qx/2 + Qx/2 the
 * same way for the full-range p_x set), then jy (max(Qy,1)), kz (max(Qz,1));
 * element type double for HLB_FP64 handles, float for HLB_FP32.
 *
 * Errors.  Every call returns an hlb_status; nothing aborts.  On failure
 * hlb_last_error() returns a message describing the most recent failing call
 * of the calling thread.  HLB_ECUDA is returned for any CUDA runtime error
 * (the message carries cudaGetErrorString); a handle whose call returned
 * HLB_ECUDA should be destroyed.  HLB_EINVAL is returned, before any device
 * work, for invalid arguments.
 */
#ifndef HLB_H
#define HLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hlb_handle hlb_handle;

typedef enum {
    HLB_OK = 0,
    HLB_EINVAL = 1,        /* invalid argument (checked on the host)           */
    HLB_ENOMEM = 2,        /* device or host allocation failed                 */
    HLB_ECUDA = 3,         /* a CUDA runtime call failed                       */
    HLB_ETIMEOUT = 4,      /* a bounded device wait gave up                    */
    HLB_ENONFINITE = 5,    /* NaN or Inf found in the moments                  */
    HLB_EUNSUPPORTED = 6   /* valid request this build does not implement      */
} hlb_status;

enum { HLB_UPWIND2 = 0, HLB_WENO5 = 1 };
/* Arithmetic (hlb_config.precision).  HLB_FP64: FP64 state and arithmetic.
 * The other three keep an FP32 state with FP32 bulk arithmetic (advection,
 * collision, RK-3), compensated FP32 moment sums and an FP64 wall balance;
 * they differ in the force term a . K f of App. A (Eqs. "eq:hh_Kk_hh",
 * "eq:H_Kk"), a small dense contraction along p_x and p_y:
 *  - HLB_FP32: the library picks the form per velocity set and scheme, the
 *    one measured faster on GB300 (FP32 FMAs; 3xTF32 for the 1D kernel's
 *    32 x 16 slabs and for the 2D kernel's 16 x 8 slabs with upwind2);
 *  - HLB_FP32_TF32X3: on the tensor cores as three TF32 products (hi/lo split
 *    of both operands) with FP32 accumulation;
 *  - HLB_FP32_BF16SPLIT: on the tensor cores with every operand split into
 *    three bf16 terms and the six leading products accumulated in FP32.
 * The tensor-core forms apply to the marching kernels' slabs with 2 Qx and
 * Qy multiples of 8 (16 x 8 and 32 x 16 values of (p_x, p_y)); other velocity
 * sets keep the FMA form (hlb_force_form reports the form in use).  All
 * three keep the moments within 1e-5 of the FP64 solution. */
enum { HLB_FP64 = 0, HLB_FP32 = 1, HLB_FP32_TF32X3 = 2, HLB_FP32_BF16SPLIT = 3 };
/* Quadrature along p_x: the half-range Hermite of Sec. IV.B (HHLB models,
 * 2 Qx values), the full-range Gauss-Hermite of Sec. IV.A (HLB models, Qx
 * values, Qx even), the model the paper compares against in Sec. V, or the
 * half-range Gauss-Laguerre of Sec. IV.B (2 Qx values, Qx <= 16; force matrix
 * Eq. "eq:hh_Kk_L", weights Eq. "eq:wk_half"). */
enum { HLB_X_HALF_RANGE = 0, HLB_X_FULL_RANGE = 1, HLB_X_HALF_LAGUERRE = 2 };

/* One channel instance.  Field order and types are part of the ABI. */
typedef struct {
    int Qx;              /* half-range order per half, 1..32 (2 Qx values of p_x); up to
                            200 on the half-range Hermite axis with HLB_FP64 (the
                            HHLB(20;200) model of Sec. V: weights down to 5e-221)    */
    int Qy, Qz;          /* full-range orders: 0 (axis absent) or even 2..32 (Sec. IV.A.1) */
    int Nx_eq, Ny_eq, Nz_eq; /* equilibrium orders N (0 <= N < Q, N <= 31); -1 => Q - 1    */
    int nx, ny;          /* cells: nx >= 6 (WENO5) or >= 3 (upwind2) between the walls;
                            ny >= 1 periodic cells in y (ny = 1: 1D channel)               */
    double Lx, Ly;       /* channel width (walls at x = 0, Lx) and periodic length in y   */
    double stretch_A;    /* 0: uniform; 0 < A < 1: tanh stretching, Eqs. "eq:x_eta","eq:etai" */
    int advection;       /* HLB_UPWIND2 or HLB_WENO5                                      */
    int precision;       /* HLB_FP64, HLB_FP32, HLB_FP32_TF32X3 or HLB_FP32_BF16SPLIT      */
    double cfl;          /* dt = cfl / (max|p_x|/min dx + [ny>1] max|p_y|/dy) if dt <= 0   */
    double dt;           /* explicit time step if > 0                                     */
    double T_left, T_right;  /* wall temperatures (> 0) at x = 0 and x = Lx               */
    double ax, ay, az;   /* acceleration a = F/m; gravity g along -x is ax = -g            */
    double Kn;           /* Knudsen number > 0; +INFINITY = collisionless (no BGK term)   */
    int x_basis;         /* HLB_X_HALF_RANGE (0, default), HLB_X_HALF_LAGUERRE (2), or
                            HLB_X_FULL_RANGE: then Qx is the even full-range order and
                            p_x holds Qx values, ordered +z_1 < ... < +z_{Qx/2}, then
                            -z_1, ..., -z_{Qx/2}                                        */
} hlb_config;

/* Create a handle for `ninst` independent instances (ninst >= 1).  Instances
 * that share (Qx, Qy, Qz, N*, advection) are advanced together by the same
 * kernels; mixed velocity sets form separate groups.  All instances of one
 * handle must share `precision`.  `cuda_stream` is a cudaStream_t on which
 * every later call enqueues its work; NULL makes the handle create (and
 * later destroy) its own non-blocking stream.  The state is zero until
 * hlb_init_equilibrium or hlb_set_state.
 * Errors: HLB_EINVAL (bad config: message names the instance and field),
 * HLB_ENOMEM, HLB_ECUDA. */
hlb_status hlb_create(const hlb_config* cfg, int ninst, void* cuda_stream, hlb_handle** out);

/* Free everything the handle owns (after synchronising its stream).  NULL is a no-op. */
void hlb_destroy(hlb_handle* h);

/* Per-instance parameters (inst = -1: all instances).  Wall temperatures
 * define the emitted Maxwellians g^w = g_x(0,T_w) g_y(0,T_w) g_z(0,T_w)
 * (Eq. "eq:fwall"); ax, ay, az the acceleration (App. A, Eq. "eq:Fnp_exp");
 * Kn the relaxation tau = Kn/n (Eq. "eq:tau").  Changing the walls or the
 * force after a step is allowed; the CFL time step is fixed at creation.
 * Errors: HLB_EINVAL. */
hlb_status hlb_set_walls(hlb_handle* h, int inst, double T_left, double T_right);
hlb_status hlb_set_force(hlb_handle* h, int inst, double ax, double ay, double az);
hlb_status hlb_set_Kn(hlb_handle* h, int inst, double Kn);

/* Per-node acceleration field of instance `inst` (0 <= inst < ninst), added
 * to its uniform acceleration: at node (y, x) the force term of App. A acts
 * with a = (ax_u + ax[y nx + x], ay_u + ay[...], az_u + az[...]), e.g. the
 * force -grad V / m of a potential V(x, y) (the conclusion, Sec. "sec:conc",
 * presents the force-term formalism for general forces; the paper's tests use
 * a constant one).  ax, ay, az: host arrays of nx * ny finite values in node
 * order (y-major), copied before the call returns; NULL is a zero component;
 * all three NULL removes the field.  The stage kernels apply it themselves:
 * the node pass writes each node's a into its equilibrium factor line, and
 * the FP32 marching kernels of a group with a field run a variant that scales
 * K_x f and K_y f per cell (FMA form of the force term; a group with a field
 * and a p_z axis takes the per-node stage kernel).  No extra launch.
 * Errors: HLB_EINVAL (instance, non-finite value), HLB_ENOMEM, HLB_ECUDA. */
hlb_status hlb_set_force_field(hlb_handle* h, int inst, const double* ax, const double* ay, const double* az);

/* State = n g_x(ux,T) g_y(uy,T) g_z(0,T) at every node of every instance
 * (App. A equilibrium), computed on the host in FP64 and broadcast on the
 * device.  Enqueued on the handle's stream.  Errors: HLB_EINVAL (n, T <= 0). */
hlb_status hlb_init_equilibrium(hlb_handle* h, double n, double ux, double uy, double T);

/* Enqueue `nsteps` RK-3 steps (Eq. "eq:rk3") on the handle's stream and
 * return without waiting.  Each step runs, per stage: the node pass (moment
 * sums, then n, u, T, 1/tau and the equilibrium factors per node, Eqs.
 * "eq:fmoms", "eq:hh_gk", "eq:H_gk"), the wall kernel (the emitted densities
 * n_w from the incident fluxes, FP64 balance) and the stage kernel (force,
 * BGK, advection, RK combination).  Groups with a force along p_z and Q_z > 0
 * run a fused per-node stage kernel instead of the first and last.  With
 * graphs enabled (default) the steps are replayed from a captured CUDA graph.
 * Errors: HLB_EINVAL (nsteps < 0), HLB_ECUDA. */
hlb_status hlb_step(hlb_handle* h, long nsteps);

/* Macroscopic moments of the current state (Eq. "eq:fmoms", App. A), in
 * FP64, for all nodes of all instances in state order.  n, T, q: one value
 * per node; u: 3 values per node (u_x, u_y, u_z).  T = sum |p-u|^2 f/(D n)
 * with D the number of momentum axes; q = q_x = sum (p_x-u_x)|p-u|^2 f/2.
 * Any output pointer may be NULL.  The values are copied from device memory
 * straight into the caller's arrays (page-locked arrays avoid a staging
 * copy): with several instances, each velocity-set group's moments kernel
 * writes its nodes into a device buffer in this layout (6 doubles per node,
 * allocated on first use), then one copy per requested array.  Synchronises
 * the handle's stream.  Errors: HLB_ECUDA, HLB_ETIMEOUT
 * (a bounded device wait ran out since the last check), HLB_ENOMEM,
 * HLB_ENONFINITE (a non-finite n or T; outputs are still written). */
hlb_status hlb_moments(hlb_handle* h, double* n, double* u, double* T, double* q);

/* Same as hlb_moments, but the outputs are device arrays (each may be NULL);
 * enqueued on the handle's stream, no synchronisation, no non-finite check.
 * With several instances every group's moments kernel writes its nodes in
 * place; with one, the kernel's scratch is copied. */
hlb_status hlb_moments_dev(hlb_handle* h, double* n_dev, double* u_dev, double* T_dev, double* q_dev);

/* Same outputs as hlb_moments_dev, for callers that cannot allocate device
 * memory at this point (an exhausted or capped memory pool, an allocator
 * owned by another runtime, a loop that must stay out of the allocator).  The
 * paper has no counterpart: this is a library service.  The call allocates
 * nothing: its scratch is a static device array of 6 x 2^18 doubles (12 MiB)
 * that every GPU which loads the library holds until the process exits.
 * Limits and behaviour:
 *  - each velocity-set group of the handle may have at most 262144 nodes;
 *    larger handles get HLB_EINVAL and nothing is launched;
 *  - every call looks the array's device address up (cudaGetSymbolAddress,
 *    which allocates nothing); the first lookup on a device loads the
 *    library's device code there, so make the first call on a device before
 *    any stream capture on that device;
 *  - every call shares the one array: calls that overlap on the GPU (other
 *    streams, other handles, other threads) race on it.  The array keeps the
 *    last call's contents; each call overwrites all entries it later reads.
 * Enqueued on the handle's stream; outputs are device arrays (NULL skips one). */
hlb_status hlb_moments_noalloc(hlb_handle* h, double* n_dev, double* u_dev, double* T_dev, double* q_dev);

/* Asynchronous hlb_moments: enqueues the moments of the current state and
 * their copies into the caller's host arrays (layout as hlb_moments) on a
 * result stream of the handle's own, after the work already enqueued on the
 * handle's stream, and returns at once; the next steps run meanwhile.  The
 * arrays should be page-locked (pageable memory makes the copies
 * synchronous) and must stay valid until hlb_moments_wait returns.  Later
 * calls that would overwrite the state buffer the moments read (a second
 * step, a graph replay, hlb_set_state, hlb_init_equilibrium, the upload of
 * hlb_prefetch_state into a swapped-out buffer) or reuse the moments scratch
 * wait for them on the device.  hlb_moments_wait blocks until the last
 * request has landed and reports non-finite moments (HLB_ENONFINITE) and
 * device errors like hlb_moments; with nothing pending it returns HLB_OK.
 * No counterpart in the paper (host I/O).  Errors: HLB_ENOMEM, HLB_ECUDA. */
hlb_status hlb_moments_async(hlb_handle* h, double* n, double* u, double* T, double* q);
hlb_status hlb_moments_wait(hlb_handle* h);

/* Number of nodes and of values in the state (all instances), and the bytes
 * of one state copy.  Any output pointer may be NULL. */
hlb_status hlb_sizes(const hlb_handle* h, long long* nodes, long long* values, long long* bytes);

/* Form of the force term in the stage kernel of instance `inst`'s velocity
 * set: 0 FP32 (or FP64) FMAs, 1 3xTF32 tensor-core products, 2 split-BF16
 * tensor-core products (see HLB_FP32_TF32X3 and HLB_FP32_BF16SPLIT).
 * Errors: HLB_EINVAL. */
hlb_status hlb_force_form(const hlb_handle* h, int inst, int* form);

/* Time step and step counter of instance `inst`. */
hlb_status hlb_get_dt(const hlb_handle* h, int inst, double* dt);
hlb_status hlb_get_nsteps(const hlb_handle* h, long long* nsteps);

/* Copy the state to / from a caller buffer of exactly hlb_sizes(...bytes)
 * bytes (layout in the header comment).  Host variants synchronise the
 * stream; _dev variants enqueue a device copy on the handle's stream: with
 * several instances and f_dev 16-byte aligned, one copy kernel per velocity-set
 * group (the first call also uploads a table of the instances' chunks), else
 * one cudaMemcpyAsync per instance.  Errors: HLB_EINVAL (size), HLB_ENOMEM
 * (the chunk table), HLB_ECUDA. */
hlb_status hlb_get_state(hlb_handle* h, void* host_f, size_t bytes);
hlb_status hlb_set_state(hlb_handle* h, const void* host_f, size_t bytes);
hlb_status hlb_get_state_dev(hlb_handle* h, void* f_dev, size_t bytes);
hlb_status hlb_set_state_dev(hlb_handle* h, const void* f_dev, size_t bytes);

/* Autotuner of the marching kernels' launch shape: for every velocity-set
 * group that runs them, times the three stage launches of one step for x-
 * segment lengths from a quarter to four times the built-in heuristic's (CUDA
 * events on the handle's stream, one untimed round, three timed) and keeps the
 * fastest; for groups on the persistent kernel, whole persistent steps for
 * segment lengths (cells per work item) of 24 to 264 cells times one or half
 * the resident CTAs per SM.  The state is only read (the launches write the two scratch
 * buffers), so the call may come at any time between steps; it synchronises
 * the handle's streams and drops the captured graph.  The results do not
 * depend on the segment length (every cell's update is computed the same way),
 * only the time does.  segments_out (may be NULL): one entry per group in
 * creation order, the chosen length in cells (0: the group does not march).
 * No counterpart in the paper.  Errors: HLB_ECUDA, HLB_ETIMEOUT. */
hlb_status hlb_autotune(hlb_handle* h, int* segments_out);

/* Staged state input, so that the upload of the next state overlaps the
 * steps still running (no counterpart in the paper: host I/O only).
 * hlb_prefetch_state enqueues a host-to-device copy of host_f (exactly
 * hlb_sizes(...bytes) bytes, layout as hlb_set_state) into a staging buffer
 * that the handle allocates on first use, on a copy stream of the handle's
 * own, after the work already enqueued on the handle's stream that reads the
 * staging buffer; it returns at once.  The copy overlaps compute only from
 * page-locked host memory.  host_f must stay valid and unchanged until the
 * copy has run, i.e. until the hlb_commit_state that consumes it has been
 * followed by a synchronisation of the handle's stream (hlb_moments, or the
 * caller's own).  A second prefetch before a commit replaces the first.
 * hlb_commit_state makes the handle's stream wait for that copy, then makes
 * the staging buffer the current state: for a single velocity set whose layout
 * is the caller's, by swapping the two buffers (no copy); otherwise by a
 * device-to-device copy as in hlb_set_state_dev.
 * Errors: HLB_EINVAL (size, NULL, commit with nothing staged), HLB_ENOMEM,
 * HLB_ECUDA. */
hlb_status hlb_prefetch_state(hlb_handle* h, const void* host_f, size_t bytes);
hlb_status hlb_commit_state(hlb_handle* h);

/* Diagnostics of the current state: the particle number per instance
 * N = int n dx dy (Eq. "eq:Ndef"; ninst values) and the last step's
 * residual max|f^{n+1} - f^n| / (dt max|f^{n+1}|) per instance (0 before the
 * first step).  Either pointer may be NULL.  Synchronises. */
hlb_status hlb_diag(hlb_handle* h, double* total_N, double* residual);

/* Host-side tables of instance `inst`'s velocity set, for inspection and
 * testing (no device work).  Any pointer may be NULL; sizes: px 2Qx, py
 * max(Qy,1), pz max(Qz,1), wx 2Qx, wy, wz likewise, Kx (2Qx)^2 row-major
 * [k][k'], Ky Qy^2, Kz Qz^2, x-cell widths nx. */
hlb_status hlb_tables(const hlb_handle* h, int inst, double* px, double* py, double* pz,
                      double* wx, double* wy, double* wz, double* Kx, double* Ky, double* Kz,
                      double* dx);

/* One momentum axis built on the host (no handle, no device work): half == 1
 * gives the half-range Hermite axis of order Q (2Q points, Eq. "eq:hh_pk",
 * K^h of Eq. "eq:hh_Kk_hh", Q <= 200), half == 2 the half-range Gauss-Laguerre axis
 * (2Q points, K^L of Eq. "eq:hh_Kk_L", Q <= 16), half == 0 the full-range
 * Gauss-Hermite axis of even order Q (Q points, K^H of Eq. "eq:H_Kk").  p and
 * w have the axis' point count, K its square (row-major [k][k']); any pointer
 * may be NULL. */
hlb_status hlb_axis(int Q, int half, double* p, double* w, double* K);

/* Equilibrium g_x(u, T) (2Qx values) of a velocity set, computed on the host
 * in FP64 as the library's wall Maxwellians and hlb_init_equilibrium are:
 * for Nx_eq <= 12 by the per-node recurrence the kernels use, above by
 * quadrature of the projection integrals (the recurrence's rounding grows
 * about threefold per order).  No handle needed.  Nx_eq (-1: Qx - 1) must be
 * at most 31; HLB_EINVAL otherwise. */
hlb_status hlb_equilibrium_x(int Qx, int Nx_eq, double u, double T, double* g);

/* Persistent batched kernel on (1, the default) or off (0).  Velocity-set
 * groups of 1D FP32 instances without a p_z axis (2 Qx x Qy slabs of 8 x 4,
 * 16 x 8, 32 x 16 with the default force-term form, or 32 x 1; equilibrium
 * orders up to 15) step with one persistent launch per RK-3 step: the CTAs
 * take work items from a queue in stage-major order, per instance first its
 * node chunks (moment sums, equilibrium factors, the emitted densities of the
 * walls they hold), then its x-segments (the marching update), and each item
 * waits on per-instance counters for what it reads (bounded: a wait that
 * runs out records HLB_ETIMEOUT and ends the launch).  Off, or with per-launch timing, or for a group with
 * a force field, those groups launch the node pass, the wall kernel and the
 * stage kernel per stage.  The results agree to FP32 rounding (the moment
 * sums are formed in another order).  Drops a captured graph (synchronises).
 * No counterpart in the paper.  Errors: HLB_EINVAL. */
hlb_status hlb_set_persistent(hlb_handle* h, int on);

/* Rounding of the FP32 stage outputs (each RK-3 stage's f, Eq. "eq:rk3"):
 * HLB_ROUND_NEAREST (the default) or HLB_ROUND_STOCHASTIC.  With round to
 * nearest, a stage drops an increment dt L below half a unit in the last
 * place of f, so near a steady state the FP32 state stops where |dt L| is
 * below that, short of L = 0 by about that over dt times the slowest
 * relaxation rate (with small time steps this can exceed 1e-5 of the
 * moments).  Stochastic rounding moves each output one unit in the last
 * place toward its exact value (out of TwoSum error terms of the stage's last
 * additions) with probability equal to the remainder's fraction of that
 * unit, so that its expectation is exact; the random number is a hash of the
 * value's address, the stage and the bits of the value and its error:
 * deterministic, run to run and inside a captured graph.  It costs a few
 * tens of instructions per node-velocity and stage, and the FP32 marching
 * kernels then take the FMA force term (not the tensor-core forms).  FP64
 * groups are unaffected.  Drops a captured graph (synchronises).  No
 * counterpart in the paper.  Errors: HLB_EINVAL, HLB_ECUDA. */
enum { HLB_ROUND_NEAREST = 0, HLB_ROUND_STOCHASTIC = 1 };
hlb_status hlb_set_rounding(hlb_handle* h, int mode);

/* How instance `inst`'s velocity-set group steps: persistent (1: the
 * persistent kernel, 0: per-stage launches), segment_cells (cells per work
 * item or CTA of the marching kernels; 0 if the group does not march), ctas
 * (the persistent grid, or the stage kernel's CTAs per launch) and
 * tuned_ms[2] (the RK-3 step times hlb_autotune measured for the group with
 * the persistent kernel and with the per-stage launches, each with its best
 * shape; 0 where it did not time them).  Any output may be NULL.
 * Errors: HLB_EINVAL. */
hlb_status hlb_step_form(const hlb_handle* h, int inst, int* persistent, int* segment_cells, int* ctas,
                         double* tuned_ms);

/* Enable (1) / disable (0) CUDA-graph replay in hlb_step, and per-launch
 * CUDA-event timing (timing forces eager launches).  hlb_kernel_times
 * returns the accumulated device time (ms) and counts of the timed intervals
 * since the last reset (reset != 0 clears them after reading): "stage" is
 * the stage kernel of each RK-3 stage alone, "wall" everything the stage
 * launches before it (the node pass, when the marching kernel runs, and the
 * wall kernel).  Synchronises. */
hlb_status hlb_set_options(hlb_handle* h, int use_graphs, int time_kernels);
hlb_status hlb_kernel_times(hlb_handle* h, double* stage_ms, long long* stage_launches,
                            double* wall_ms, long long* wall_launches, int reset);

/* Number of kernels hlb_step has enqueued (CUDA-graph replays counted by the
 * kernels they hold) since the handle was created or last reset (reset != 0
 * clears the count after reading).  Host-only; does not synchronise. */
hlb_status hlb_launch_count(hlb_handle* h, long long* launches, int reset);

/* Test hook of the bounded device waits (no counterpart in the paper).  Every
 * wait of the marching stage kernels on its bulk-copy pipeline gives up after
 * wait_limit_s seconds (0: the default, 1 s; at most 60), records
 * HLB_ETIMEOUT in the handle's device error word and ends its CTA's loop at
 * the next barrier.  withhold_copies != 0 makes every marching CTA skip the
 * copies of its second pipeline step, so that those waits run out: the next
 * hlb_moments / hlb_get_state / hlb_diag (total_N) returns HLB_ETIMEOUT and the state
 * is invalid (re-initialise it).  Steps that do not use the marching kernels
 * are unaffected.  Synchronises if a CUDA graph has to be re-captured. */
hlb_status hlb_set_wait_test(hlb_handle* h, int withhold_copies, double wait_limit_s);

/* Test hook: the double-float exp(-z^2) and erf(z) from which the FP32
 * groups' node pass starts the half-range recurrence (App. A; used for
 * equilibrium orders up to 10 and |z| = |u_x| / sqrt(2T) <= 2.5, FP64 erf and
 * exp otherwise), evaluated for n values z in device memory, the results as
 * doubles (hi + lo) into device arrays; synchronises the device.  No
 * counterpart in the paper.  Errors: HLB_EINVAL (n < 0, NULL), HLB_ECUDA. */
hlb_status hlb_df_special_check(const double* z_dev, int n, double* erf_dev, double* exp_dev);

/* Test hook of the out-of-memory paths (no counterpart in the paper; process
 * wide, no handle).  nth > 0 arms it: the nth device or page-locked
 * allocation the library makes from then on fails as if memory were
 * exhausted (the call that made it returns HLB_ENOMEM and frees what it had
 * allocated; a failed hlb_create leaves nothing behind), and the hook
 * disarms.  nth == 0 disarms it.  Errors: HLB_EINVAL (nth < 0). */
hlb_status hlb_set_alloc_fail_test(long long nth);

/* FP32 FMA throughput of the current device in TFLOP/s (an FMA counts two
 * flop), measured with independent dependent-FMA chains on every SM (scalar
 * fmaf for packed == 0, packed f32x2 FMAs otherwise), best of three timed
 * launches after a warm-up (about 0.1 s; allocates and frees a small device
 * buffer; synchronises the device).  The ALU roof of the FP32 stage kernels;
 * no counterpart in the paper.  Errors: HLB_EINVAL, HLB_ENOMEM, HLB_ECUDA. */
hlb_status hlb_fp32_peak(int packed, double* tflops);

/* Message of the calling thread's last failing call ("" if none). */
const char* hlb_last_error(void);

/* Library version string. */
const char* hlb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HLB_H */
