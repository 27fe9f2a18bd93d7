/*
 * ps.h -- C ABI of libps: the GPU time step of the penalized pseudo-spectral
 * Navier--Stokes solver (Truong, Engels, Kolomenskiy, Schneider, "A mass-spring
 * fluid-structure interaction solver: application to flexible revolving
 * wings", Sec. 4.1), its wing mask rasteriser, force/moment reductions and
 * discrete adjoint.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns a ps_status; PS_OK is 0. On failure the context keeps
 *   a message readable with ps_last_error(). The library never prints, never
 *   exits and never frees memory it did not allocate.
 * - Device pointers ("_dev") are caller-owned CUDA device memory on the
 *   device the context was created on, densely packed, in the layout stated
 *   at each call. Host pointers are plain host memory.
 * - Real-valued device arrays use the context's precision: float for
 *   PS_FP32, double for PS_FP64 ("real" below). Force, moment, diagnostics,
 *   node coordinates and frames are always double.
 * - Physical fields are C-order [ix][iy][iz] (z fastest) on the n x n x nz
 *   grid (ps_params.nz, n for a cubic grid), n^2 nz values per component,
 *   components stored one after another (3 n^2 nz for a vector).
 * - The context allocates NO device memory: the caller passes one workspace
 *   of ps_workspace_size() bytes (256-byte aligned) to ps_init and keeps it
 *   alive until ps_destroy.
 * - Work is enqueued on the CUDA stream given to ps_init and is
 *   asynchronous unless a call says it synchronises. Asynchronous CUDA
 *   errors surface as PS_ECUDA at the next synchronising call.
 * - Fault injection for tests: with the environment variable
 *   PS_FAULT_ALLOC set to "ctx" (ps_init), "ms" (ps_ms_create) or "all",
 *   those calls fail their host allocation and return PS_ENOMEM (before
 *   any CUDA call).
 */
#ifndef PS_H
#define PS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ps_ctx ps_ctx;

typedef enum {
    PS_OK = 0,
    PS_EINVAL = 1,        /* bad argument (null pointer, size, value)          */
    PS_ENOMEM = 2,        /* workspace too small                               */
    PS_ECUDA = 3,         /* a CUDA call or kernel failed                      */
    PS_ESTATE = 4,        /* call not valid in the context's current state     */
    PS_EUNSUPPORTED = 5,  /* grid size or option not built into this library   */
    PS_ENUMERIC = 6       /* a NaN or Inf was found by a diagnostic reduction  */
} ps_status;

enum { PS_FP32 = 0, PS_FP64 = 1 };
enum { PS_MASK_COS = 0, PS_MASK_TANH = 1 };
enum { PS_MEAN_FIXED = 0, PS_MEAN_FREE = 1 };

/*
 * Solver parameters (Sec. 4.1, Eq. penalized Navier--Stokes; the paper's
 * C_eta is eta here).
 *   n          points along x and y of the periodic n x n x nz grid on
 *              [0, L)^2 x [0, Lz); the library supports the sizes listed
 *              by ps_supported_n().
 *   nz         points along z: 0 or n (cubic box, Lz = L), or n/2 for
 *              n >= 32 (Lz = L/2: the 4 x 4 x 2 box with N x N x N/2 points
 *              of the paper's revolving-wing runs, Sec. 4.2). The spacing
 *              L/n is the same on every axis; z wavenumbers are 2 pi m/Lz
 *              and the 2/3 rule keeps 3|m_z| < nz. Other values return
 *              PS_EUNSUPPORTED.
 *   precision  PS_FP32: transforms, nonlinear term, projection and update in
 *              float, force/moment/diagnostic reductions in double;
 *              PS_FP64: everything in double.
 *   mask_profile  profile used by ps_set_mask_from_nodes: PS_MASK_COS is
 *              Sec. 4.1 Eq. (mask_function) (banded, chi = 0 beyond t_w + h);
 *              PS_MASK_TANH is chi = (1 - tanh((delta - t_w)/h))/2 at every
 *              grid point.
 *   mean_mode  PS_MEAN_FIXED: the k = 0 mode of the right-hand side is
 *              dropped (mean velocity fixed); PS_MEAN_FREE: kept.
 *   with_adjoint  1: the workspace also holds the adjoint state and scratch
 *              (six spectral state arrays and nine physical fields more).
 *   L, nu, eta, dt  box length, kinematic viscosity, penalization constant,
 *              time step (all > 0).
 *   tw, h      wing semi-thickness and smoothing semi-width of the mask.
 *   x0         reference point of the moment.
 *   keep_uw    1: the workspace also holds three z-spectral fields
 *              (3 n^2 Kzp complex, Kzp = (nz-1)/3 + 1 rounded up to 16 (FP32)
 *              or 8 (FP64) values) so that ps_pressure keeps u and omega of the
 *              state it evaluated; a ps_step right after it (nothing between
 *              that changes the velocity) then starts at its z pass and skips
 *              the x- and y-inverse passes. This is the staggered coupling's
 *              order (fluid step, pressure, solid, mask, fluid step).
 *              0: no extra memory, every step runs all passes.
 */
typedef struct {
    int32_t n;
    int32_t precision;
    int32_t mask_profile;
    int32_t mean_mode;
    int32_t with_adjoint;
    double L, nu, eta, dt;
    double tw, h;
    double x0[3];
    int32_t keep_uw;
    int32_t nz;
} ps_params;

/* Wing frame -> global frame (Sec. 4.1, Eq. relative_velocities):
 * R row-major 3x3 rotation (global = X_O + R x_wing), X_O origin,
 * V_O translational velocity, Omega angular velocity. */
typedef struct {
    double R[9];
    double X_O[3];
    double V_O[3];
    double Omega[3];
} ps_frame;

/* Writes up to `cap` supported grid sizes to `out` and the total count to
 * *count (out may be NULL to query the count). */
ps_status ps_supported_n(int32_t* out, int32_t cap, int32_t* count);

/* Bytes of device workspace a context with these parameters needs. */
ps_status ps_workspace_size(const ps_params* p, size_t* bytes);

/* Create a context on the current CUDA device. cuda_stream is a
 * cudaStream_t (NULL = legacy default stream). workspace_dev must hold
 * ps_workspace_size() bytes; the context zeroes it (velocity and mask start
 * at zero). Returns PS_EUNSUPPORTED for a grid size that is not built in. */
ps_status ps_init(const ps_params* p, void* cuda_stream, void* workspace_dev,
                  size_t workspace_bytes, ps_ctx** out);
ps_status ps_destroy(ps_ctx* ctx);

/* Velocity u (3 n^2 nz real, physical, caller device memory). ps_set_velocity
 * transforms it, truncates it by the 2/3 rule and projects it onto
 * divergence-free fields (mean kept); the Adams--Bashforth history restarts,
 * so the next step is an integrating-factor Euler step. ps_get_velocity
 * writes the current velocity back to physical space. */
ps_status ps_set_velocity(ps_ctx* ctx, const void* u_dev);
ps_status ps_get_velocity(ps_ctx* ctx, void* u_dev_out);

/* Dense mask chi (n^2 nz real in [0,1]) and solid velocity u_s (3 n^2 nz real),
 * caller device memory, copied into the workspace (Sec. 4.1: chi and u_s of
 * the penalization term). */
ps_status ps_set_mask(ps_ctx* ctx, const void* chi_dev, const void* us_dev);

/* Copy the current mask chi (n^2 nz real) and solid velocity u_s (3 n^2 nz real)
 * into caller device memory. */
ps_status ps_get_mask(ps_ctx* ctx, void* chi_dev_out, void* us_dev_out);

/* Rasterise chi and u_s from the wing's triangle mesh (Sec. 4.1,
 * Eq. mask_function, the bounding-box-limited distance to the triangles,
 * barycentric velocity on the closest triangle, Eq. relative_velocities).
 *   xw_dev, vw_dev  n_nodes x 3 double: wing-frame node positions/velocities
 *   tri_dev         n_tri x 3 int32 vertex indices (0-based)
 *   frame           host pointer, wing -> global frame
 * Ties in distance go to the smallest triangle index. Where chi = 0, u_s = 0
 * (PS_MASK_COS); with PS_MASK_TANH every point is evaluated. */
ps_status ps_set_mask_from_nodes(ps_ctx* ctx, const double* xw_dev, const double* vw_dev,
                                 int32_t n_nodes, const int32_t* tri_dev, int32_t n_tri,
                                 const ps_frame* frame);

/* Advance nsteps time steps (Sec. 4.1: u^n -> u^{n+1} with chi^n, u_s^n):
 * integrating-factor AB2, the first step after ps_set_velocity being
 * integrating-factor Euler. Asynchronous. */
ps_status ps_step(ps_ctx* ctx, int32_t nsteps);

/* Penalization force and moment on the solid, F = (dx^3/eta) sum chi (u - u_s),
 * M = (dx^3/eta) sum (x - x0) x chi (u - u_s), of the velocity at the start of
 * the last step taken (Sec. 4.2.2 defines lift and drag from this force).
 * Host outputs; synchronises the stream. */
ps_status ps_forces(ps_ctx* ctx, double F[3], double M[3]);
/* Spectral array sizes of the context: K kept x/y modes (x/y index c <->
 * mode c if c <= (n-1)/3, else c - K), Kz kept z modes, Kzp the padded kz
 * columns of every spectral array. Host outputs. */
ps_status ps_grid_info(const ps_ctx* ctx, int32_t* K, int32_t* Kz, int32_t* Kzp);

/* Slab decomposition of the step (the paper's solver runs MPI slabs,
 * Sec. 4.1; here one context per slab, on one or several GPUs). A slab
 * context runs its share of each pass:
 *   phase 0  x-inverse with the curl on its kept ky rows [ky0, ky1)
 *            (writes the x-pass array A, fields 0..5, those ky rows, all x);
 *   phase 1  y-inverse, z pass (n, forces) and y-forward on its x-planes
 *            [x0, x1) (reads A fields 0..5 at those x-planes, all ky rows;
 *            writes A fields 0..2 at those x-planes, all ky rows);
 *   phase 2  x-forward, projection and the integrating-factor AB2 update on
 *            its ky rows (reads A fields 0..2 at those ky rows, all x).
 * Between phases 0 and 1 every slab needs the other slabs' A rows for its
 * x-planes, between 1 and 2 their x-planes for its ky rows (the two
 * all-to-all exchanges of the sharded step); the caller moves those blocks
 * (ps_slab_buffer gives A). ps_forces of a slab context is its x-planes'
 * share of F and M; the step's force is the sum over the slabs. The state
 * (U, H) of a slab context is valid on its ky rows only; its mask is used
 * on its x-planes only, and ps_set_mask_from_nodes rasterises only them.
 * ps_slab_set: PS_EINVAL for empty or out-of-range bounds, or x-plane bounds
 * whose product with n is not a multiple of the z pass's lines per batch.
 * ps_slab_phase: asynchronous; phase 2 counts the step (the first is the
 * Euler start). ps_slab_buffer: A, 6 x [K][n][Kzp] complex in the context
 * precision, [field][ky][x][kz], owned by the context's workspace. */
ps_status ps_slab_set(ps_ctx* ctx, int32_t x0, int32_t x1, int32_t ky0, int32_t ky1);
ps_status ps_slab_phase(ps_ctx* ctx, int32_t phase);
ps_status ps_slab_buffer(ps_ctx* ctx, void** a_dev, size_t* bytes);

/* Device error flag. Every wait of a kernel on its asynchronous copies has
 * an iteration cap; a wait that gives up sets the context's device error
 * flag, lets the copies it started land, and ends the kernel early, so the
 * results of that launch are invalid. ps_forces then returns PS_ECUDA. The
 * flag is sticky: every later ps_forces fails too, until ps_clear_error
 * resets it (synchronises the stream). */
ps_status ps_clear_error(ps_ctx* ctx);
/* Test hook for the error path above (no counterpart in the paper): one
 * block waits, with an iteration cap of `cap` polls (>= 1), on an mbarrier
 * that expects 16 bytes of bulk copy that no copy delivers (none is
 * issued), gives up and sets the device error flag like a transform pass.
 * Nothing stays in flight. Synchronises. PS_EINVAL for cap < 1. */
ps_status ps_debug_wait_timeout(ps_ctx* ctx, int32_t cap);

/* Sponge term (Sec. 4.1, Eq. penalized Navier--Stokes: the vorticity
 * damping term), added to the nonlinear term of every following step:
 *   S = -(1/C_sp) curl^{-1}(chi_sp omega),  S_hat = -(1/C_sp) i k x s_hat / |k|^2,
 * s_hat the 2/3-truncated transform of chi_sp omega. (The paper prints the
 * term with 1/lap and a minus sign, which read literally amplifies; the
 * damping form its text describes is taken: for chi_sp = 1, S = -u/C_sp.)
 *   chi_sp_dev  n^2 nz array [x][y][z] in the context precision, caller-owned;
 *               read by every step while set, so it must stay valid and
 *               unchanged until the sponge is turned off. NULL turns it off.
 *   c_sp        C_sp > 0 (ignored when turning off).
 * With the sponge on, a step also transforms the three components of
 * chi_sp omega forward (the z pass's otherwise idle thread groups) and reads
 * six fields in the x-forward pass. PS_EINVAL for c_sp <= 0. */
ps_status ps_set_sponge(ps_ctx* ctx, const void* chi_sp_dev, double c_sp);

/* Static pressure p = Pi - (1/2)|u|^2 of the current state with the current
 * mask (Sec. 4.1: Pi = p + (1/2) u.u is the total pressure of the rotational
 * form; the fluid-solid coupling computes p^{n+1} from u^{n+1}). Pi is the
 * gradient part the Leray projection removes from the nonlinear and
 * penalization term N: Pi_hat = -i (k . N_hat)/|k|^2, mean zero.
 *   p_dev  caller-owned n^2 nz array [x][y][z] in the context precision.
 * Costs about one time step (the step's passes 1-4, then one inverse
 * field). Leaves the state and the forces of ps_forces unchanged; uses the
 * internal scratch arrays. With keep_uw the x and y passes it ran are not
 * repeated by the next ps_step (or a second ps_pressure) on the same state;
 * the results are the same bits either way. Asynchronous. PS_ESTATE without
 * a velocity. */
ps_status ps_pressure(ps_ctx* ctx, void* p_dev);

/* Pressure loads on the wing's mass points (Sec. 4.1, coupling paragraph):
 * p_v = p interpolated at node v (global position X_O + R x_v) with the
 * smoothed 4-point cosine delta (the 4-point cosine kernel convolved with
 * the unit box, five points per axis, periodic), and
 * F_v = -p_v sum over the triangles T containing v of (A_T/3) n_T, n_T the
 * unit normal (b - a) x (c - a)/|...| of T's vertex order, global frame.
 *   p_dev        n^2 nz pressure from ps_pressure (context precision)
 *   xw_dev, tri_dev, frame  as in ps_set_mask_from_nodes
 *   p_nodes_dev  n_nodes doubles out; f_nodes_dev n_nodes x 3 doubles out
 * All device pointers caller-owned; sums in double. Asynchronous. */
ps_status ps_pressure_loads(ps_ctx* ctx, const void* p_dev, const double* xw_dev, int32_t n_nodes,
                            const int32_t* tri_dev, int32_t n_tri, const ps_frame* frame,
                            double* p_nodes_dev, double* f_nodes_dev);

/* Kinetic energy (1/2) int |u|^2 dV and max_k |k . c_k| of the current state
 * (c_k the Fourier coefficients), in double. Host outputs; synchronises.
 * Returns PS_ENUMERIC (and still writes the values) if the state holds a
 * NaN or Inf. */
ps_status ps_diagnostics(ps_ctx* ctx, double* energy, double* max_div);

/* Checkpoint of the time-stepping state (spectral velocity, AB2 history,
 * step counter) to/from caller device memory of ps_state_size() bytes,
 * 16-byte aligned (PS_EINVAL for a null or unaligned buffer). Both calls
 * synchronise the stream. The mask and the sponge are not part of the state;
 * after a restore the next step runs all passes (keep_uw). */
ps_status ps_state_size(const ps_ctx* ctx, size_t* bytes);
ps_status ps_save_state(ps_ctx* ctx, void* buf_dev);
ps_status ps_restore_state(ps_ctx* ctx, const void* buf_dev);

/* Discrete adjoint (no counterpart in the paper: the exact transpose of the
 * step's operations) for objectives J = sum_n (a_n . F^n + b_n . M^n), F^n,
 * M^n the force and moment of step n (ps_forces). Needs with_adjoint = 1.
 * ps_adjoint_reset zeroes the adjoint state (before the last step of a
 * window is reversed). ps_adjoint_step reverses step n: the context must hold
 * the forward state u^n (use ps_restore_state / ps_step to get there) and the
 * mask chi^n, u_s^n of that step; dJdF = a_n, dJdM = b_n (host, 3 doubles
 * each); first = 1 if step n was the integrating-factor Euler start step.
 * It overwrites grad_chi_dev (n^2 nz real) and grad_us_dev (3 n^2 nz real) with
 * dJ/dchi^n and dJ/du_s^n and updates the adjoint state. Asynchronous. */
ps_status ps_adjoint_reset(ps_ctx* ctx);
ps_status ps_adjoint_step(ps_ctx* ctx, const double dJdF[3], const double dJdM[3], int32_t first,
                          void* grad_chi_dev, void* grad_us_dev);

/* Vector-Jacobian product of the last ps_set_mask_from_nodes call: given
 * dJ/dchi and dJ/du_s on the grid (caller device memory, context precision),
 * ADDS dJ/dx^(w) of the wing-frame node positions to grad_xw_dev (n_nodes x 3
 * double, caller device memory), holding each point's closest triangle fixed.
 * The node/triangle arrays of that call must still be alive. Asynchronous;
 * PS_ESTATE if the mask was set densely since. */
ps_status ps_mask_nodes_vjp(ps_ctx* ctx, const void* grad_chi_dev, const void* grad_us_dev,
                            double* grad_xw_dev);

/* Per-pass device timing with CUDA events on the context's stream.
 * ps_timing_enable(ctx, 1) resets the accumulators and records events around
 * each pass of every following ps_step (and around ps_set_mask_from_nodes)
 * for up to 256 steps; 0 stops recording. ps_timing_read synchronises and
 * writes, for each of *count passes (named by ps_timing_name(i)), the summed
 * milliseconds and the number of timed steps (a pass split into x slabs that
 * run on two streams counts the sum of its slab kernels' times, each measured
 * on its own stream, once per step). With ms or launches NULL or
 * cap too small it only sets *count. */
ps_status ps_timing_enable(ps_ctx* ctx, int32_t on);
ps_status ps_timing_read(ps_ctx* ctx, double* ms, int64_t* launches, int32_t cap, int32_t* count);
const char* ps_timing_name(int32_t i);

/* Penalization force and moment of caller-supplied physical fields, for
 * callers that must not allocate device memory after start-up: a real-time
 * loop (cudaMalloc can block and synchronise the device), a process whose
 * framework's memory pool already holds nearly all device memory (a fresh
 * cudaMalloc fails there), code under a no-dynamic-allocation rule. It needs
 * no ps_ctx and no workspace. The paper has no counterpart; it is the force
 * reduction of ps_step (F = (dx^3/eta) sum chi (u - u_s),
 * M = (dx^3/eta) sum (x - x0) x chi (u - u_s), x = (i, j, k) dx) offered alone.
 *   n, precision, L, eta, x0  grid size, PS_FP32/PS_FP64 (type of the real
 *              arrays), box length, penalization constant, moment point
 *              (host array of 3 doubles)
 *   u_dev (3*n^3), chi_dev (n^3), us_dev (3*n^3)  physical fields of a cubic
 *              n^3 grid, layout as
 *              everywhere in this header
 *   FM_dev     device output, 6 doubles: F then M
 *   cuda_stream  stream the work is enqueued on (asynchronous)
 * Scratch lives in a fixed 48 KiB array compiled into the library (one
 * partial per x-plane, 1024 planes): n > 1024 returns PS_EINVAL. Nothing is
 * allocated: no cudaMalloc, no cudaFree. The first call on each device looks
 * up the array's device address and caches it; after cudaDeviceReset that
 * address is stale and the call must not be used again. Calls share the
 * array: two calls that may overlap on the GPU (unordered streams) race.
 * It makes CUDA calls, so it must not be called from a stream callback or a
 * host function (cudaLaunchHostFunc). Returns PS_ECUDA, leaving the error in
 * place, if an error from earlier work is pending on entry, and PS_ECUDA if
 * one of its own launches fails. */
ps_status ps_penalization_force_noalloc(int32_t n, int32_t precision, double L, double eta,
                                        const double x0[3], const void* u_dev, const void* chi_dev,
                                        const void* us_dev, double* FM_dev, void* cuda_stream);

/* Text of the last error on this context ("" if none). */
const char* ps_last_error(const ps_ctx* ctx);


/* ------------------------------------------------------------------------
 * Mass-spring network of the wing (Sec. 2.1-2.2). Host code, host memory,
 * double precision; no CUDA call. Node arrays are n_nodes x 3, row-major.
 *
 * Springs (Eq. extension_spring, Eq. two_bending_angles): an extension
 * spring (i, j) stores k^e and its rest length |x0_j - x0_i|; a bending
 * spring (i, j, k) stores k^b and the rest angles theta^y_0, theta^z_0 of
 * x0, theta^y = atan2[(x_j-x_i)(y_k-y_j) - (x_k-x_j)(y_j-y_i),
 * (x_j-x_i)(x_k-x_j) + (y_j-y_i)(y_k-y_j)], theta^z the same with z for y.
 * Internal forces are minus the gradient of
 *   E = sum (1/2) k^e (l - l_0)^2 + sum (1/2) k^b [(dtheta^y)^2 + (dtheta^z)^2],
 * angle changes taken in (-pi, pi]. The extension force is the printed
 * one; the bending force is the gradient of the bending energy (the
 * printed bending force has no lever length; Eq. EI_k_relation, which sets
 * k^b = (EI/l_b) n(2n+1)/(2(n+1)), equates energies). Fixed nodes never
 * move; the others follow m dv/dt = F_int + F_ext (Eq. Newton_law).
 *
 * Moving frame: the network may be solved in a frame with origin
 * acceleration A_O, angular velocity Omega and angular acceleration
 * dOmega, all expressed in the frame's own axes; each free node then also
 * feels -m (A_O + dOmega x x + Omega x (Omega x x) + 2 Omega x v).
 * -------------------------------------------------------------------- */
typedef struct ps_ms ps_ms;

typedef struct {
    double A_O[3];
    double Omega[3];
    double dOmega[3];
} ps_ms_frame;

/* Build a network. mass (n_nodes, > 0), x0 (rest and initial positions),
 * v0 (initial velocities; NULL = 0), fixed (n_nodes flags; NULL = none),
 * ext_ij (n_ext x 2), ke (n_ext), bend_ijk (n_bend x 3), kb (n_bend).
 * Inputs are copied. The free nodes are ordered by reverse Cuthill--McKee
 * for a banded Newton matrix. PS_EINVAL for an out-of-range or repeated
 * index or a mass <= 0; PS_ENOMEM if allocation fails. */
ps_status ps_ms_create(int32_t n_nodes, const double* mass, const double* x0, const double* v0,
                       const unsigned char* fixed, int32_t n_ext, const int32_t* ext_ij, const double* ke,
                       int32_t n_bend, const int32_t* bend_ijk, const double* kb, ps_ms** out);
ps_status ps_ms_destroy(ps_ms* m);

/* Free-node count, the node bandwidth of the Newton matrix and how many
 * times a Newton matrix has been built and factored (outputs may be NULL). */
ps_status ps_ms_info(const ps_ms* m, int32_t* n_free, int32_t* bandwidth, int64_t* factorizations);

/* Internal spring forces at positions x (n_nodes x 3) into f_out. */
ps_status ps_ms_forces(const ps_ms* m, const double* x, double* f_out);

/* Current positions/velocities (either output may be NULL). */
ps_status ps_ms_state(const ps_ms* m, double* x_out, double* v_out);

/* Replace positions and velocities (v NULL = 0; fixed nodes get v = 0)
 * and forget the step history: the next step is backward Euler. */
ps_status ps_ms_set_state(ps_ms* m, const double* x, const double* v);

/* One time step of length dt (Eq. discretized_ODEs, variable-step BDF2,
 * xi = dt / previous dt; the first step after create/set_state/equilibrium
 * is backward Euler). f_ext (n_nodes x 3, NULL = 0) is the external force
 * held over the step; frame (NULL = inertial) adds the fictitious forces
 * at the new time level. Newton--Raphson on the positions (velocities
 * eliminated), starting from the current state. The factored Newton matrix
 * of an earlier iteration or step is reused while the iteration contracts
 * by at least 1/2 per iteration (for at most six iterations) and c dt
 * (c = (1+xi)/(1+2xi)) is within 20 % of the one it was built for;
 * otherwise it is rebuilt at the current iterate. Converged when the update (times rate/(1 - rate) once a rate is
 * known) is below tol * max(1, |x|) in L2. Returns the iterations in *iters_out
 * (may be NULL). PS_ENUMERIC, state unchanged, if Newton does not converge
 * in max_iter iterations or its matrix is singular. */
ps_status ps_ms_step(ps_ms* m, double dt, const double* f_ext, const ps_ms_frame* frame, double tol,
                     int32_t max_iter, int32_t* iters_out);

/* Static equilibrium F_int(x) + f_ext = 0 by Newton--Raphson with the load
 * raised in load_steps equal increments (each converged to tol as in
 * ps_ms_step). Sets the positions, zero velocities, clears the history.
 * PS_ENUMERIC (state unchanged) if a load increment does not converge. */
ps_status ps_ms_equilibrium(ps_ms* m, const double* f_ext, int32_t load_steps, double tol, int32_t max_iter,
                            int32_t* iters_out);

/* Checkpoint of the network's time-stepping state (positions, velocities,
 * the previous level of both and the previous step, for the BDF2 history)
 * to/from a caller host buffer of ps_ms_state_size() bytes. Saving makes
 * the next step rebuild its Newton matrix, as a restored network does, so a
 * run continued after ps_ms_save and one resumed by ps_ms_restore give the
 * same bits. ps_ms_restore returns PS_EINVAL for a buffer that is not a
 * state of a network with this node count (springs are not stored: restore
 * into a network built from the same inputs). */
ps_status ps_ms_state_size(const ps_ms* m, size_t* bytes);
ps_status ps_ms_save(ps_ms* m, void* buf);
ps_status ps_ms_restore(ps_ms* m, const void* buf);

/* Text of the last error on this network ("" if none). */
const char* ps_ms_last_error(const ps_ms* m);

#ifdef __cplusplus
}
#endif
#endif /* PS_H */
