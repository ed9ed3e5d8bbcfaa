/*
 * ps.h - C ABI of the GB300 (sm_103a) pseudospectral Navier-Stokes
 * right-hand side and its integrating-factor Runge-Kutta step.
 *
 * The method is the one of Rosenberg, Mininni, Reddy and Pouquet,
 * "GPU parallelization of a hybrid pseudospectral fluid turbulence framework
 * using CUDA" (arXiv:1808.01309), Sec. 2: incompressible Navier-Stokes
 * (Eq. mom with theta = 0, Eq. divv) on a periodic box, each velocity
 * component expanded in the discrete Fourier series of Eq. (fftsum), the
 * Galerkin ODEs for the coefficients advanced by an explicit Runge-Kutta
 * scheme of 2nd or 4th order, the nonlinear term formed in physical space
 * between a backward and a forward 3D transform, and the pressure acting as a
 * projection of that term onto divergence-free fields.  The same machinery
 * advances the MHD system (Eqs. uMHD, bMHD) and the Boussinesq system
 * (Eqs. mom, temp, divv), selected by ps_config.eq.
 *
 * Conventions fixed by this library (readings of the paper):
 *   - Forward transform: u_hat(k) = (1/(Nx Ny Nz)) sum_x u(x) exp(-i k.x);
 *     backward transform unnormalised.  x_i = Lx i/Nx; k = 2 pi (p/Lx, q/Ly, r/Lz).
 *   - Nonlinear term in rotational form u x omega, omega = curl u.
 *   - 2/3-rule dealiasing (cubic: |p| < Nx/3, |q| < Ny/3, |r| < Nz/3; spherical
 *     also requires (3p/Nx)^2 + (3q/Ny)^2 + (3r/Nz)^2 < 1; none keeps all but the
 *     Nyquist modes).  The state is the truncated Galerkin system: modes
 *     outside the mask are treated as zero on input and written as zero.
 *   - Leray projection P(k) = I - k k^T/|k|^2 of the nonlinear term plus the
 *     forcing; the k = 0 mode of the right-hand side is zero.
 *   - Runge-Kutta in Lawson (integrating factor) form with
 *     E = exp(-nu |k|^2 dt/2):
 *       RK4: k1 = R(u), k2 = R(E(u + dt/2 k1)), k3 = R(E u + dt/2 k2),
 *            k4 = R(E^2 u + dt E k3), u+ = E^2 u + dt/6 (E^2 k1 + 2E(k2+k3) + k4)
 *       RK2: k1 = R(u), k2 = R(E^2 (u + dt k1)), u+ = E^2 (u + dt/2 k1) + dt/2 k2
 *     where R = D P(F[u x omega] + f) is the right-hand side without viscosity.
 *
 * Data layout of every spectral vector field (state, right-hand side,
 * forcing): interleaved complex (float2 for PS_FP32, double2 for PS_FP64),
 * C order [component][kz 0..nz-1][ky 0..ny-1][kx 0..nx/2], kx fastest,
 * ky and kz in FFT order (0..n/2-1, -n/2..-1).  This is the layout of
 * torch.fft.rfftn / numpy.fft.rfftn of a real (nz, ny, nx) array per
 * component.  Components: 3 (u) for PS_HD, 6 (u, B) for PS_MHD, 4 (u, theta)
 * for PS_BOUSSINESQ.  Field bytes: ncomp * nz * ny * (nx/2+1) * (8 or 16).
 * Every device field must start on a multiple of its element size (8 bytes
 * in FP32, 16 in FP64; cudaMalloc and torch allocations are); a misaligned
 * pointer returns PS_ERR_INVALID_ARG before any launch.
 *
 * Ownership: the caller owns the state, right-hand-side and forcing buffers.
 * The plan owns its scratch (intermediate fields, twiddles, stage registers).
 * All calls are asynchronous on the plan's CUDA stream except those that
 * return host values (ps_diagnostics, ps_step_stats, ps_rk_step_host,
 * ps_plan_get_timing), which synchronise it.  A plan is used by one host
 * thread at a time.
 *
 * Errors: arguments are checked on the host before any launch.  On
 * PS_ERR_INVALID_ARG / PS_ERR_UNSUPPORTED nothing was launched and the plan
 * stays usable.  After PS_ERR_CUDA the plan must be destroyed.  No C++
 * exception crosses this interface.  ps_last_error() gives a message for the
 * last failure of the calling thread.
 */
#ifndef PS_H_
#define PS_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PS_OK = 0,
  PS_ERR_INVALID_ARG = 1,  /* bad pointer, size, aliasing or config value */
  PS_ERR_UNSUPPORTED = 2,  /* valid request this library does not implement */
  PS_ERR_OOM = 3,          /* device allocation failed */
  PS_ERR_CUDA = 4,         /* CUDA runtime or launch error */
  PS_ERR_NONFINITE = 5,    /* a diagnostic came out NaN or infinite */
  PS_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up */
} ps_status;

typedef enum { PS_FP32 = 0, PS_FP64 = 1 } ps_precision;
typedef enum { PS_HD = 0, PS_MHD = 1, PS_BOUSSINESQ = 2 } ps_equations;
typedef enum { PS_DEALIAS_CUBIC = 0, PS_DEALIAS_SPHERICAL = 1, PS_DEALIAS_NONE = 2 } ps_dealias;

typedef struct ps_plan ps_plan;

/* One solve (Sec. 2: grid and box may differ per axis).
 *   nx, ny, nz : powers of two in [8, 1024], or 48, 96, 192 (radix-3 lines)
 *   lx, ly, lz : box lengths, finite and > 0
 *   prec       : arithmetic and storage precision of all fields
 *   eq         : PS_HD, or PS_MHD (Eqs. uMHD, bMHD: the state then has six
 *                components u_x, u_y, u_z, B_x, B_y, B_z; the magnetic
 *                field advances with dB/dt = curl(u x B) - eta |k|^2 B,
 *                the curl taken in spectral space after the product; in
 *                PS_FP32 that multiplies the product's rounding by |k|, so
 *                the relative error of the induction term grows with the
 *                grid, about 2e-6 at 128^3 to 7e-6 at 512^3 for fields
 *                whose energy sits at low k; PS_FP64 keeps 1e-12), or
 *                PS_BOUSSINESQ (Eqs. mom, temp, divv: four components u_x,
 *                u_y, u_z, theta; du/dt = P(F[u x omega] + f - n_bv theta z)
 *                - nu |k|^2 u and dtheta/dt = -F[u . grad theta] + n_bv w
 *                - kappa |k|^2 theta, grad theta taken in spectral space
 *                before the backward transforms, the scalar integrated
 *                with the factor exp(-kappa |k|^2 dt/2))
 *   dealias    : truncation rule
 *   rk_order   : 2 or 4
 *   nu         : kinematic viscosity >= 0;  eta: magnetic diffusivity >= 0 (MHD)
 *   n_bv       : Brunt-Vaisala frequency (Boussinesq, finite, any sign)
 *   kappa      : scalar diffusivity >= 0 (Boussinesq)
 *   forcing    : device pointer to a constant-in-time forcing of the
 *                velocity (three components, state layout and precision), or
 *                NULL.  Its retained modes are copied at plan creation; later
 *                changes are not seen. */
typedef struct {
  int nx, ny, nz;
  double lx, ly, lz;
  ps_precision prec;
  ps_equations eq;
  ps_dealias dealias;
  int rk_order;
  double nu, eta;
  const void* forcing;
  double n_bv, kappa;
} ps_config;

/* Global diagnostics of the retained state, accumulated in FP64.
 *   energy    = 1/2 sum w |u_hat|^2   (w = 1 on kx = 0 and kx = nx/2, else 2)
 *   enstrophy = 1/2 sum w |omega_hat|^2,  helicity = sum w Re(u_hat* . omega_hat)
 *   max_div   = max |k . u_hat|,  max_u = max over grid points of |u(x)|
 *   cfl_dt    = cfl * min(lx/nx, ly/ny, lz/nz) / max_u
 *   spectrum  : caller-owned host array of capacity nshells (or NULL); shell
 *               K holds 1/2 sum w |u_hat|^2 over modes with floor(|k|+1/2) = K
 *   nshells   : in: capacity of spectrum; out: number of shells of this grid
 *   time      : t + dt of the last ps_rk_step on this plan (0 if none)
 *   MHD only (0 for HD): magnetic_energy = 1/2 sum w |B_hat|^2,
 *   cross_helicity = sum w Re(u_hat* . B_hat), magnetic_helicity =
 *   sum w Re(A_hat* . B_hat) with A_hat = i k x B_hat/|k|^2 (Coulomb gauge);
 *   the velocity entries above describe u only.
 *   Boussinesq only (0 otherwise): potential_energy = 1/2 sum w |theta_hat|^2. */
typedef struct {
  double energy, enstrophy, helicity, max_div, max_u, cfl_dt, time;
  double* spectrum;
  int nshells;
  double magnetic_energy, cross_helicity, magnetic_helicity;
  double potential_energy;
} ps_diag;

#define PS_NKINDS 7
/* Per-kernel-kind device time measured with CUDA events on the plan stream
 * while timing is enabled: 0 z-inverse, 1 y-inverse, 2 fused x pass,
 * 3 y-forward, 4 z-forward transform, 5 auxiliary, 6 per-mode update
 * (forcing, projection, closure, RHS or RK stage update). */
typedef struct {
  double ms[PS_NKINDS];
  long long launches[PS_NKINDS];
} ps_timing;

/* Create a plan: validates cfg, allocates scratch on the current device,
 * builds FP64-accurate twiddle tables and copies the forcing.  cuda_stream is
 * a cudaStream_t (NULL = legacy default stream).  Synchronises the stream. */
ps_status ps_plan_create(const ps_config* cfg, void* cuda_stream, ps_plan** out);

/* Free every plan-owned allocation.  NULL is accepted. */
ps_status ps_plan_destroy(ps_plan* plan);

/* Device bytes a plan with this config allocates (without forcing box). */
ps_status ps_plan_workspace_bytes(const ps_config* cfg, size_t* bytes);

/* Right-hand side of the Galerkin ODEs (Sec. 2):
 *   rhs_out = D P(F[u x omega] + f) - nu |k|^2 D u_hat
 * uhat and rhs_out are device buffers in the state layout; they must not
 * overlap.  t is the time of uhat (the forcing is constant; t is recorded
 * only).  Asynchronous. */
ps_status ps_rhs(ps_plan* plan, const void* uhat, void* rhs_out, double t);

/* One integrating-factor Runge-Kutta step of order cfg.rk_order, in place on
 * the device state uhat (Sec. 2, explicit RK of 2nd-4th order).  Also records,
 * for the state at the start of the step, its energy and max |u(x)|
 * (ps_step_stats).  dt must be finite.  Asynchronous. */
ps_status ps_rk_step(ps_plan* plan, void* uhat, double dt, double t);

/* nsteps calls of ps_rk_step on the device state uhat, replayed as one CUDA
 * graph: the first call for a given (uhat, dt, nsteps) captures the steps,
 * later calls with the same triple launch the captured graph on the plan
 * stream (for small grids, whose steps are bound by launch latency).  The
 * result equals nsteps calls of ps_rk_step bit for bit.  With per-kernel
 * timing on, the steps are launched one by one.  Asynchronous. */
ps_status ps_rk_steps(ps_plan* plan, void* uhat, double dt, double t, int nsteps);

/* Same as nsteps calls of ps_rk_step on a HOST buffer, then synchronises
 * (nsteps = 0 does nothing).  How the state moves (ps_plan_set_host_mode):
 *   PS_HOST_AUTO   : (default) for a page-locked buffer (cudaHostAlloc /
 *                    cudaHostRegister) only the retained cube of modes crosses
 *                    the host link, gathered and scattered by kernels through
 *                    the buffer's device mapping (NVLink-C2C on Grace
 *                    systems), while host threads of the calling process write
 *                    the zeros of the masked modes into the host buffer during
 *                    the steps; pageable memory takes PS_HOST_COPY;
 *   PS_HOST_CUBE_CE: as PS_HOST_AUTO with the zeros written by copy engines
 *                    (3D copies from a device buffer of zeros over the link);
 *   PS_HOST_COPY   : cudaMemcpyAsync of the whole state to a plan-owned device
 *                    buffer (allocated on the first call) and back;
 *   PS_HOST_SMCOPY : the whole state copied by a streaming kernel through the
 *                    device mapping, and back;
 *   PS_HOST_MAPPED : the passes use the page-locked buffer in place (the
 *                    first pass and every stage update read its retained
 *                    modes, the last stage writes it).
 * SMCOPY and MAPPED fail with PS_ERR_UNSUPPORTED on pageable memory.  The
 * modes outside the retained set are zero on return in every mode. */
enum { PS_HOST_AUTO = 0, PS_HOST_COPY = 1, PS_HOST_MAPPED = 2, PS_HOST_SMCOPY = 3, PS_HOST_CUBE_CE = 4 };
ps_status ps_rk_step_host(ps_plan* plan, void* uhat_host, double dt, double t, int nsteps);
ps_status ps_plan_set_host_mode(ps_plan* plan, int mode);

/* Energy (kinetic + magnetic for MHD, + potential 1/2 theta^2 for Boussinesq)
 * and max |u(x)| (FP64) of the state at
 * the start of the last ps_rk_step.  Synchronises the plan stream. */
ps_status ps_step_stats(ps_plan* plan, double* energy, double* max_u);

/* Diagnostics of the device state uhat (see ps_diag).  Runs the backward
 * transforms once for max |u(x)|.  Synchronises the plan stream.  Returns
 * PS_ERR_NONFINITE (with out filled) if a result is not finite. */
ps_status ps_diagnostics(ps_plan* plan, const void* uhat, double cfl, ps_diag* out);

/* Per-kernel CUDA-event timing (see ps_timing).  Enabling clears the totals;
 * ps_plan_get_timing synchronises, reports the totals since then and keeps
 * accumulating. */
ps_status ps_plan_set_timing(ps_plan* plan, int enable);
ps_status ps_plan_get_timing(ps_plan* plan, ps_timing* out);

/* Number of kernels this plan has launched since creation. */
ps_status ps_plan_launch_count(ps_plan* plan, long long* launches);

/* Test hook for the failure path of the bounded device waits (the paper has
 * no counterpart).  With polls > 0, every CTA of the x pass of the plan's
 * following right-hand sides waits for a copy that is never issued and gives
 * up after `polls` polls of its barrier (instead of the default 2^26): the
 * pass records PS_ERR_TIMEOUT in the plan's device error word, the update
 * kernel writes NaN into every retained output of that right-hand side, and
 * the next synchronising call (ps_step_stats, ps_diagnostics, ps_rk_step_host,
 * ...) returns PS_ERR_TIMEOUT once and clears the word.  No fault, trap or
 * hang is involved and the context stays usable.  polls = 0 (the default)
 * turns the hook off; polls outside [0, 2^20] returns PS_ERR_INVALID_ARG. */
ps_status ps_plan_set_wait_test(ps_plan* plan, int polls);

/* Tile shape of one column pass of the plan's right-hand sides (pass 0: the
 * z-inverse pass, 1: both y passes, 2: the z-forward pass; Sec. 2 describes
 * each 3D transform as 1D transforms along the axes, this only chooses how
 * the lines are tiled).  variant 0: the default (8 kx columns per CTA in
 * FP32); 1: half the columns per CTA and twice the lines; 2: the other radix
 * schedule (8 <-> 16 points per thread and line; not for lengths with a
 * factor 3).  Variants 1 and 2 exist for FP32 hydrodynamic plans whose
 * pass axis has 64, 96 or 128 points (PS_ERR_UNSUPPORTED otherwise).  All
 * variants compute the same transforms (results agree to rounding).  cols
 * and points (may be NULL) receive the chosen columns per CTA and points per
 * thread.  The ensemble tuner sets these per grid size. */
ps_status ps_plan_set_pass_shape(ps_plan* plan, int pass, int variant, int* cols, int* points);

/* Name of a kernel kind of ps_timing (0..PS_NKINDS-1), or "?". */
const char* ps_kind_name(int kind);

/* ---- Ensembles of independent solves ------------------------------------
 * Many independent solves of possibly different sizes and viscosities, each
 * with its own state, stepped together.  The paper's solver runs one field per
 * MPI task; this is the single-GPU way to keep a GB300 busy with many small
 * problems.  One plan per member; no data is shared between members. */
typedef struct ps_ensemble ps_ensemble;
#define PS_ENS_MAX_MEMBERS 1024
#define PS_ENS_MAX_SIZES 8

/* PS_ENS_SEQUENTIAL: member after member, every kernel launched separately on
 * the ensemble stream.  PS_ENS_GRAPH: all nsteps steps of all members as one
 * CUDA graph launch; each member's launch chain is a branch, branches run
 * concurrently (number of branches chosen by ps_ensemble_tune, default
 * min(members, 16)).  PS_ENS_PERSISTENT: all nsteps steps of all members in
 * ONE persistent kernel launch whose CTAs take (member, pass, tile) work items
 * from a device queue; a member's pass starts once the member's previous pass
 * is complete (device counters), so the passes of different members overlap.
 * The launch is captured in a CUDA graph with the reset of its counters.  It
 * needs members of one precision, the hydrodynamic system without a closure
 * and axis lengths in {32, 48, 64, 96, 128} (PS_ERR_UNSUPPORTED otherwise);
 * its bounded waits report through ps_ensemble_check; on 128-point x rows
 * it takes 8 points per thread where the other modes take 16 (results agree
 * to rounding there, bit for bit elsewhere at equal tile shapes).
 * PS_ENS_BATCHED:
 * members of one grid class (same grid, box, precision, dealiasing and RK
 * order) share one launch per pass (tiles of all members in one grid; the x
 * pass loops over (member, row group) pairs), in sub-batches of at most 32
 * members (the tuner picks the size) that run as concurrent branches of one
 * CUDA graph; same member restrictions as the persistent
 * launch, results bit for bit those of PS_ENS_GRAPH at the default tile
 * shapes.  PS_ENS_AUTO: the mode ps_ensemble_tune found fastest
 * (PS_ENS_GRAPH before tuning).  Graphs are captured on the first call with
 * given (states, dt, nsteps) and replayed by later identical calls (t does
 * not enter the right-hand side). */
typedef enum {
  PS_ENS_SEQUENTIAL = 0,
  PS_ENS_GRAPH = 1,
  PS_ENS_PERSISTENT = 2,
  PS_ENS_AUTO = 3,
  PS_ENS_BATCHED = 4
} ps_ens_mode;

/* Result of ps_ensemble_tune: concurrent branches, and per distinct grid
 * (first nsizes entries, n = nx of the grid) the x-pass rows per CTA chosen
 * (0 = the automatic maximum) and the tile shape chosen for each column pass
 * (see ps_plan_set_pass_shape); step_ms = graph time of one step of all
 * members with the chosen shapes.  The persistent launch's choices:
 * resident CTAs per SM (0 = as many as fit), member order (0 = as created,
 * 1 = largest grid first, 2 = largest first and staggered: member k starts
 * k mod 6 passes late, so that different passes run side by side) and
 * tiles per work item of the z-inverse,
 * y-inverse, x, y-forward, z-forward and update passes (in that order);
 * persistent_step_ms is its time of one step (-1: not supported by these
 * members).  best_mode is what PS_ENS_AUTO now runs (graph, persistent or
 * batched, whichever was fastest). */
typedef struct {
  int branches;
  int nsizes;
  int n[PS_ENS_MAX_SIZES];
  int xrpc[PS_ENS_MAX_SIZES];
  double step_ms;
  int pass_cols[PS_ENS_MAX_SIZES][3];    /* kx columns per CTA of the z-inverse, y and z-forward passes */
  int pass_points[PS_ENS_MAX_SIZES][3];  /* points per thread (radix schedule) of the same passes */
  double persistent_step_ms;
  int persistent_ctas_per_sm;
  int persistent_order;
  int persistent_tiles_per_item[6];
  double batched_step_ms;  /* PS_ENS_BATCHED, one step (-1: not supported by these members) */
  int batched_members_per_launch;  /* sub-batch size chosen for PS_ENS_BATCHED */
  int best_mode;
} ps_ens_tuning;

/* Create count (1..PS_ENS_MAX_MEMBERS) member plans from cfgs[i] (each as for
 * ps_plan_create) on the current device; cuda_stream is the ensemble stream. */
ps_status ps_ensemble_create(const ps_config* cfgs, int count, void* cuda_stream, ps_ensemble** out);
ps_status ps_ensemble_destroy(ps_ensemble* e);

/* nsteps IF-RK steps of every member, in place on uhats[i] (device state of
 * member i, layout of its config), starting at time t.  Asynchronous on the
 * ensemble stream.  The sequential, graph and batched modes give identical
 * results at equal tile shapes (the persistent launch: see above). */
ps_status ps_ensemble_rk_steps(ps_ensemble* e, void* const* uhats, double dt, double t, int nsteps,
                               ps_ens_mode mode);

/* Autotuner: times, on device copies of uhats (left unchanged), for each
 * distinct grid the x-pass rows per CTA and the tile shape (columns per CTA,
 * radix schedule) of each column pass, then the number of concurrent graph
 * branches, the persistent launch's knobs and the members per batched
 * launch; keeps the fastest of each, sets the mode PS_ENS_AUTO runs and
 * reports them.  Allocates temporary copies of the states.  Synchronises
 * the ensemble stream. */
ps_status ps_ensemble_tune(ps_ensemble* e, const void* const* uhats, double dt, ps_ens_tuning* out);

/* Synchronises the ensemble stream and reports whether a bounded device wait
 * gave up since the last check, in any mode: a dependency wait of the
 * persistent launch or an x-pass copy wait of a member (PS_ERR_TIMEOUT; the
 * affected states are then invalid: the stage updates write NaN once an
 * error word is set).  Clears the reports. */
ps_status ps_ensemble_check(ps_ensemble* e);

/* Test hook of the persistent launch's failure path: with polls > 0 one pass
 * instance waits for one tile more than its predecessor has, and every wait
 * gives up after `polls` polls; 0 restores normal operation. */
ps_status ps_ensemble_set_wait_test(ps_ensemble* e, unsigned polls);

/* ---- Learned LES closure: pointwise MLP on the BF16 tensor cores --------
 * A multilayer perceptron 5 -> 64 -> 64 -> 6 with GELU (tanh form) maps the
 * standardised gradient invariants of a resolved velocity to the subgrid
 * stress.  Parameters are one FP32 device vector of PS_MLP_NPARAM values:
 * W1[5][64] | b1[64] | W2[64][64] | b2[64] | W3[64][6] | b3[6], y = x W + b.
 * Products run on the tensor cores (mma, BF16 operands, FP32 accumulation);
 * biases, activations and sums stay FP32.  The paper has no closure; the
 * model follows the LES workload of this library. */
#define PS_MLP_NPARAM 4934

/* Y[count][6] = MLP(X[count][5]) (device FP32 buffers).  Asynchronous. */
ps_status ps_mlp_forward(const float* params, const float* X, float* Y, long long count, void* cuda_stream);

/* Mean-squared-error loss L = mean((MLP(X) - T)^2) over count samples and 6
 * outputs (*loss, device double) and dL/dparams (grad, device FP32, overwritten).
 * Asynchronous. */
ps_status ps_mlp_grad(const float* params, const float* X, const float* T, long long count, float* grad,
                      double* loss, void* cuda_stream);

/* Tensor-basis fit: loss L = mean over count samples and 6 components of
 * (sum_n y_n T_n(A/s_A) - T/s_tau)^2 with y = MLP(X), A[count][9] the
 * gradients of the samples and T_n the basis of ps_plan_set_closure; *loss
 * (device double) and dL/dparams (grad, overwritten).  Asynchronous. */
ps_status ps_mlp_grad_tb(const float* params, const float* X, const float* A, const float* T, long long count,
                         double s_A, double s_tau, float* grad, double* loss, void* cuda_stream);

/* Backpropagation only: grad += dL/dparams for given output deltas
 * dY[count][6] = dL/dy at the samples X[count][5] (device FP32; grad is
 * accumulated, not overwritten).  Asynchronous. */
ps_status ps_mlp_backward(const float* params, const float* X, const float* dY, long long count, float* grad,
                          void* cuda_stream);

/* One Adam update (bias-corrected, step >= 1) of params with the moment
 * buffers m, v (device FP32, PS_MLP_NPARAM each, zero before step 1). */
ps_status ps_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1,
                      float beta2, float eps, void* cuda_stream);

/* Attach a trained closure to an FP32 HD plan (cubic or no truncation):
 * afterwards ps_rhs and ps_rk_step add -div tau to the nonlinear term before
 * the projection (every RK stage), with the model stress
 *   tau = s_tau sum_{n=1..6} g_n T_n(S/s_A, R/s_A),
 *   g = MLP((lambda - mean)/std),
 * lambda the five invariants tr S^2, tr R^2, tr S^3, tr S R^2, tr S^2 R^2 of
 * the resolved velocity gradient A_ij = du_i/dx_j (S, R its symmetric and
 * antisymmetric parts) and T_1..T_6 the first six tensors of Pope's (1975)
 * integrity basis: S, SR - RS, S^2 - tr(S^2) I/3, R^2 - tr(R^2) I/3,
 * RS^2 - S^2 R, R^2 S + S R^2 - 2 tr(S R^2) I/3.
 *   params : device FP32 vector of PS_MLP_NPARAM values (copied), or NULL to
 *            detach the closure
 *   norm12 : host doubles mean[5], std[5], s_tau, s_A (std, s_tau, s_A > 0)
 * Grid sizes 16..512 (powers of two, 48, 96, 192).  Allocates the closure
 * scratch on first use (about 29 floats per grid point); synchronises the
 * plan stream.  PS_ERR_UNSUPPORTED for FP64, MHD or spherical truncation. */
ps_status ps_plan_set_closure(ps_plan* plan, const float* params, const double* norm12);

/* Force-matched training of the attached closure (ps_plan_set_closure gives
 * the normalisation; params here replaces the attached network):
 *   L = sum over the half spectrum of w |D P(-div tau(ubar)) - f|^2
 * (w = 1 on the kx = 0 plane, 2 elsewhere; by Parseval the grid mean of the
 * squared residual), with f a projected, band-limited subgrid force in the
 * state layout, e.g. the filtered DNS right-hand side minus the LES
 * right-hand side of the filtered state.  Adds L to *loss (device double) and
 * dL/dparams to grad (device FP32); accumulate = 0 zeroes both first.
 * Allocates 9 more floats per grid point on first use.  Asynchronous. */
ps_status ps_plan_closure_grad(ps_plan* plan, const float* params, const void* ubar, const void* force, float* grad,
                               double* loss, int accumulate);

/* Same for the energy-transfer loss L = sum_{K < nshells} (T(K) - t_exact[K])^2,
 * T(K) = sum over the kept modes of shell K = floor(|k| + 1/2) of
 * w Re(ubar* . D P(-div tau(ubar))): the energy the closure moves into each
 * shell, against t_exact (host, nshells <= 1024 doubles), e.g. the transfer
 * of the exact subgrid force.  Synchronises the plan stream. */
ps_status ps_plan_closure_grad_transfer(ps_plan* plan, const float* params, const void* ubar, const double* t_exact,
                                        int nshells, float* grad, double* loss, int accumulate);

/* Training data for the closure from one DNS state (FP32, n_dns^3, 2 pi box,
 * HD layout, device): with F the box filter |p|,|q|,|r| <= kc and ubar = F[u]
 * sampled on an n_les^3 grid (P = n_les^3 points, order z, y, x):
 *   X[P][5] : standardised invariants of grad ubar (raw if norm12 is NULL;
 *             only mean and std of norm12 are used)
 *   A[P][9] : grad ubar, A_ij at 3i+j (optional, NULL to skip)
 *   T[P][6] : subgrid stress F[u_i u_j] - F[ubar_i ubar_j], order 11, 22,
 *             33, 12, 13, 23 (the part of the filtered momentum flux that an
 *             LES truncated at kc does not form itself)
 * n_dns, n_les in {16, 32, 48, 64, 96, 128, 192, 256, 512}, n_les <= n_dns,
 * 1 <= kc <= ceil(n_les/3) - 1.  Allocates and frees its scratch (about 60
 * bytes per DNS point); synchronises the stream. */
ps_status ps_les_training_sample(int n_dns, const void* uhat_dns, int n_les, int kc, const double* norm12, float* X,
                                 float* A, float* T, void* cuda_stream);

/* Box filter of an FP32 HD state: uhat_les (n_les^3 layout, device) receives
 * the modes |p|, |q|, |r| <= kc of uhat_dns (n_dns^3) and zeros elsewhere.
 * Even sizes 8..1024, n_les <= n_dns, 0 <= kc < n_les/2, no aliasing of the
 * two buffers.  Asynchronous. */
ps_status ps_les_filter(int n_dns, const void* uhat_dns, int n_les, int kc, void* uhat_les, void* cuda_stream);

/* ---- Plain 3D transforms ----------------------------------------------------
 * The discrete Fourier sum of Eq. (fftsum) on an n^3 grid (2 pi box) for
 * nfields real FP32 fields, with the line transforms the passes are built
 * from but without pruning, masking or fusion (every mode is kept):
 *   ps_fft_r2c: spec[f](k) = (1/n^3) sum_x phys[f](x) exp(-i k.x)
 *   ps_fft_c2r: phys[f](x) = sum_k spec[f](k) exp(+i k.x) over the full
 *               Hermitian spectrum (the unnormalised backward sum)
 * spec: [nfields][n][n][n/2+1] complex64 in the state layout (device);
 * phys: [nfields][n][n][n] float32, x fastest (device); the input is not
 * modified.  n in {16, 32, 48, 64, 96, 128, 192, 256, 512}, 1 <= nfields
 * <= 16.  Allocate and free their scratch (twiddles; for c2r a copy of the
 * spectrum) and synchronise the stream. */
ps_status ps_fft_r2c(int n, int nfields, const float* phys, void* spec, void* cuda_stream);
ps_status ps_fft_c2r(int n, int nfields, const void* spec, float* phys, void* cuda_stream);

/* ---- Checkpoint and resume -----------------------------------------------
 * The paper returns the fields to the host to write restart files (Sec. 3)
 * and describes no format; this is one.  A checkpoint file is a 136-byte
 * little-endian header followed by the state exactly as in device memory
 * (the ABI layout above, ncomp * nz * ny * (nx/2+1) complex values):
 *   off   0: magic "PSCKPT" then the bytes 0x00 0x01   off   8: uint32 version (1)
 *   off  12: uint32 header bytes (136)
 *   off  16: int32 nx, ny, nz, prec, eq, dealias, rk_order, ncomp
 *   off  48: double lx, ly, lz, nu, eta, n_bv, kappa, t
 *   off 112: int64 step          off 120: uint64 payload bytes
 *   off 128: uint64 FNV-1a (64-bit) checksum of the payload
 * The forcing is not part of a checkpoint (it is the caller's, constant).
 *
 * ps_checkpoint_save: writes the device state uhat of the plan (after the
 *   work queued on the plan stream) with time t and step number `step` to
 *   `path` (through path + ".part", renamed when complete).  Synchronises.
 * ps_checkpoint_load: reads `path` into the device state uhat of a plan with
 *   the same grid, box, precision and equations (else PS_ERR_INVALID_ARG);
 *   the checksum is verified before uhat is touched (a corrupted or truncated
 *   file returns PS_ERR_INVALID_ARG and leaves uhat unchanged); t and step
 *   (optional) receive the saved values.  Synchronises.
 * ps_checkpoint_info: reads and checks the header only, filling cfg (forcing
 *   NULL), t and step (each optional); needs no GPU.
 * Continuing from a loaded checkpoint with the same plan configuration gives
 * the same states bit for bit as the uninterrupted run. */
ps_status ps_checkpoint_save(ps_plan* plan, const void* uhat, double t, long long step, const char* path);
ps_status ps_checkpoint_load(ps_plan* plan, void* uhat, double* t, long long* step, const char* path);
ps_status ps_checkpoint_info(const char* path, ps_config* cfg, double* t, long long* step);

/* Size of the static device array behind ps_rhs_noalloc: 32 MiB. */
#define PS_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* Right-hand side like ps_rhs, but without a plan and without allocating any
 * memory, for callers that cannot allocate: a program that has handed the
 * device to its own pool allocator, a plugin or callback that must keep the
 * memory footprint fixed, or code that cannot accept the synchronisation
 * cudaMalloc/cudaFree may cause.  The paper has no counterpart of this call.
 *   cfg         : as for ps_plan_create; the forcing buffer, if any, is read
 *                 by the kernels queued on cuda_stream, so it must stay valid
 *                 and unchanged until that work has completed, like uhat
 *   cuda_stream : cudaStream_t the kernels run on (NULL = legacy default)
 *   uhat, rhs_out, t : as for ps_rhs (device buffers, must not overlap)
 * Scratch: one file-scope __device__ array of PS_NOALLOC_SCRATCH_BYTES that
 * every GPU loading this library holds until exit (enough for a 64^3 grid in
 * FP32 or FP64, with forcing).  A grid needing more returns
 * PS_ERR_INVALID_ARG, with the sizes in ps_last_error(), before any launch.
 * Every call looks up the array's device address with the device current
 * (the first call on a device may also load the library's device code, so
 * make it before any stream capture).  All calls share the one array and
 * each overwrites it; the one word in it that must start at zero (the error
 * word of the x pass's bounded waits) is cleared by every call; calls whose
 * kernels overlap on the GPU race on it: serialise them (one stream, or
 * events).  Asynchronous: a bounded device wait that gives up cannot be
 * reported as a status here (there is no later synchronising call), so it
 * turns every retained mode of rhs_out into NaN instead. */
ps_status ps_rhs_noalloc(const ps_config* cfg, void* cuda_stream, const void* uhat, void* rhs_out, double t);

/* ---- Slab decomposition over several ranks ---------------------------------
 * The paper distributes each 3D transform as slabs and exchanges the data
 * once per transform with an all-to-all between the passes along the local
 * axes and the pass along the distributed axis (Sec. 2, slab decomposition;
 * Sec. 3.3, transpose and exchange).  A ps_slab runs the passes of one HD
 * right-hand side for one rank: its retained kx columns [kx_lo, kx_hi) of all
 * (ky, kz) in spectral space and its z planes [z_lo, z_hi) of all (y, x) in
 * physical space.  The caller moves the data between the three calls (two
 * all-to-alls: 6 fields after ps_slab_inverse, 3 after ps_slab_xpass), e.g.
 * with NCCL; paper_1808_01309_gb300/slab.py does this bookkeeping.
 *
 * Local layouts (interleaved complex as above; kxp and cxp from
 * ps_slab_info: ncx = kx_hi - kx_lo local columns, kxp = ncx rounded up to a
 * multiple of 16, cxp = (Kx + 1) rounded up likewise, rows = (z_hi - z_lo) ny):
 *   uhat_local, rhs_local, forcing : [3][nz][ny][ncx], FFT order in ky, kz
 *   out6 (ps_slab_inverse)         : [6][nz][ny][kxp]  u, omega after the
 *                                    backward z and y transforms
 *   xin  (ps_slab_xpass)           : [6][rows][cxp]    the same fields, full x
 *                                    rows of the local planes (kx < Kx + 1
 *                                    used, the rest ignored)
 *   xout (ps_slab_xpass)           : [3][rows][cxp]    forward x transform of
 *                                    u x omega, kx < Kx + 1 (the rest zero)
 *   yin  (ps_slab_forward)         : [3][nz][ny][kxp]  xout of every rank's
 *                                    planes for the local columns
 * rhs_local receives the right-hand side of ps_rhs restricted to the local
 * columns (zero at masked modes).  Every buffer is the caller's device
 * memory, 16-byte aligned (else PS_ERR_INVALID_ARG); the slab owns its
 * scratch.  Calls are asynchronous on the slab's stream; ps_slab_check
 * synchronises it and returns PS_ERR_TIMEOUT once if a bounded wait of the
 * x pass gave up.  cfg->forcing, if set, is the local forcing
 * [3][nz][ny][ncx], read (into the slab's copy) during ps_slab_create.
 * PS_ERR_UNSUPPORTED for other equation sets; PS_ERR_INVALID_ARG for ranges
 * outside 0 <= kx_lo < kx_hi <= Kx + 1, 0 <= z_lo < z_hi <= nz. */
typedef struct ps_slab ps_slab;
typedef struct {
  int ncx, kxp, cxp, rows;
} ps_slab_info;
ps_status ps_slab_create(const ps_config* cfg, int kx_lo, int kx_hi, int z_lo, int z_hi, void* cuda_stream,
                         ps_slab** out);
ps_status ps_slab_destroy(ps_slab* slab);
ps_status ps_slab_info_get(const ps_slab* slab, ps_slab_info* out);
ps_status ps_slab_inverse(ps_slab* slab, const void* uhat_local, void* out6);
ps_status ps_slab_xpass(ps_slab* slab, const void* xin, void* xout);
ps_status ps_slab_forward(ps_slab* slab, const void* yin, const void* uhat_local, void* rhs_local);
ps_status ps_slab_check(ps_slab* slab);

/* ---- Measurement ------------------------------------------------------------
 * Fused multiply-add rate of the current device in TFLOP/s (2 flops per FMA)
 * for prec (PS_FP32 or PS_FP64): eight independent FMA chains per thread, 8
 * CTAs of 256 threads per SM, best of five timed launches after one warm-up,
 * CUDA events on cuda_stream (NULL = legacy default).  The denominator of the
 * arithmetic roofline of the FP64 passes, which the GPU's FP64 rate bounds
 * rather than HBM (the paper has no counterpart).  Synchronises the stream;
 * allocates nothing and changes no device setting.  *tflops receives the
 * rate; PS_ERR_INVALID_ARG for a NULL pointer or an unknown precision. */
ps_status ps_probe_fma_tflops(ps_precision prec, void* cuda_stream, double* tflops);

const char* ps_status_string(ps_status s);
const char* ps_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PS_H_ */
