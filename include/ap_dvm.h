/* ap_dvm.h — C ABI of the GB300 (sm_103a) implementation of the
 * asymptotic-preserving IMEX Runge-Kutta scheme for the six-velocity (D2V6)
 * lattice-Boltzmann-type discrete velocity model in the low-Mach /
 * diffusive scaling (Dimarco, Klar, Koefler, Pareschi: "Asymptotic preserving
 * methods for the low Mach limit in discrete velocity models approximating
 * kinetic equations").
 *
 * The library advances the closed moment system of Sec. 2.1 (vector form of
 * Sec. 3) with Algorithm 1 of Sec. 3.1 and the finite-difference operators of
 * Sec. 3.2 on a periodic nx x ny grid of cell centres.
 *
 * Conventions for every call below:
 *  - All array pointers are DEVICE pointers unless the name starts with h_.
 *  - A "plane" is nx*ny values, row-major with x fastest: element (i, j) of
 *    cell centre ((i+1/2) Lx/nx, (j+1/2) Ly/ny) is at j*nx + i.
 *  - A "moment state" is 6 consecutive double planes in the order
 *    (u1, u2, theta, v1, v2, q) of Sec. 2.1 (rescaled moments).
 *  - "Populations" are 6 consecutive planes dF_1..dF_6, the deviations
 *    F_i - rho0/6 of the D2V6 populations (c_i = (cos(pi(i-1)/3),
 *    sin(pi(i-1)/3))), scaled so that dF = rho0 * mach * f with
 *    sum f = 2 eps theta, sum c f = u, sum (c1^2 - 1/2) f = -eps v1,
 *    sum c1 c2 f = eps v2, sum c1 (c2^2 - 1/4) f = eps^2 q.
 *  - The caller owns all device memory, including workspaces.  Apart from
 *    a CUDA graph it may instantiate (ap_dvm_set_graph_steps), the library
 *    allocates no device memory: it carves the workspaces it is given.
 *  - Calls that launch work are asynchronous on the handle's stream.
 *  - Errors: a status code is returned synchronously for argument errors;
 *    device-side conditions (non-finite state) are latched in a device flag
 *    read by ap_dvm_sync_status.  Nothing aborts or traps.
 */
#ifndef AP_DVM_H
#define AP_DVM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AP_DVM_OK = 0,
  AP_DVM_ERR_ARG = 1,          /* invalid argument (message in ap_dvm_last_error) */
  AP_DVM_ERR_TABLEAU = 2,      /* tableau is not a DIRK GSA IMEX tableau with a_11 >= 0, a_ii > 0 for i >= 2 */
  AP_DVM_ERR_WORKSPACE = 3,    /* workspace too small or misaligned */
  AP_DVM_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  AP_DVM_ERR_NONFINITE = 5,    /* a step produced a non-finite value (latched on the device) */
  AP_DVM_ERR_TIMEOUT = 6,      /* a bounded device wait (tile copy) expired; the kernel returned early */
  AP_DVM_ERR_UNSUPPORTED = 7   /* valid but not implemented configuration */
} ap_dvm_status;

enum { AP_DVM_D2V6 = 6 };                                        /* velocity set (Sec. 2.1) */
enum { AP_DVM_LF1_C2 = 0, AP_DVM_WENO3_C4 = 1, AP_DVM_WENO5_C4 = 2 }; /* spatial scheme (Sec. 3.2) */
enum { AP_DVM_FP64 = 0, AP_DVM_FP32_DEV = 1, AP_DVM_FP32_DEV_TH = 2 }; /* precision form */
#define AP_DVM_MAX_STAGES 4

/* Parameters of one solve.
 *  nx, ny      cells per direction, in [8, 4096].  Any size: an axis whose
 *              length is not a power of two takes its Helmholtz transforms
 *              by a mixed-radix FFT when the length factors into 2, 3, 5
 *              and 7, else by Bluestein's chirp-z identity with a
 *              power-of-two length M >= 2n - 1 (either way the transform
 *              occupies M values of shared memory); the stencil tiles at
 *              the high edges of the grid may be ragged.  Grids whose rows are not a multiple of
 *              16 bytes stage their tiles with plain loads instead of TMA.
 *  Lx, Ly      periodic domain [0,Lx) x [0,Ly), > 0 (the paper uses 2 pi).
 *  velocity_set  AP_DVM_D2V6 (the only set of Sec. 2.1).
 *  eps         Knudsen / scaling parameter epsilon >= 0 (eps = 0 is the exact
 *              incompressible limit; the FP32 form needs eps > 0).
 *  tau         BGK coefficient tau >= 0 (the limit viscosity is tau/4, Sec. 2.1);
 *              tau < 0 selects tau = 4 eps / mach (from eps = Ma/Re, Re = 4/tau).
 *  mach        storage amplitude A > 0 of the populations (dF = rho0 A f);
 *              a pure scale of the population view.
 *  rho0        reference density > 0.
 *  dt          time step > 0.
 *  s           number of stages, 2..AP_DVM_MAX_STAGES.
 *  A_ex, A_im  explicit (strictly lower) and implicit (lower) tableaux of
 *              Sec. 3.1, row-major with row stride AP_DVM_MAX_STAGES; the
 *              implicit tableau is of type CK/ARS (a_11 = 0: stage 1 is X^n)
 *              or of type A (a_11 > 0: stage 1 is computed by Algorithm 1
 *              with i = 1), with a_ii > 0 for i >= 2, and the pair globally
 *              stiffly accurate, so that the last stage is the new state.
 *  space_scheme  AP_DVM_LF1_C2, AP_DVM_WENO3_C4 or AP_DVM_WENO5_C4.
 *  precision   AP_DVM_FP64 (all in FP64) or AP_DVM_FP32_DEV (FP32 deviation
 *              populations and FP32 transport; FP64 moment sums, division by
 *              rho0*mach, and closed-form relaxation when eps <= 1e-4).
 *              AP_DVM_FP32_DEV_TH is AP_DVM_FP32_DEV with theta carried from
 *              step to step in its own FP32 plane beside the populations
 *              instead of being summed back from them: theta rides at O(eps)
 *              inside the populations, so summing it from FP32 populations
 *              costs ~6e-8/eps of its relative precision (the pressure error
 *              of AP_DVM_FP32_DEV); the populations are written as in
 *              AP_DVM_FP32_DEV.
 *  weno_eps    epsilon of the WENO weights (1e-6 by default); at least 1e-30
 *              (FP64) or 1e-9 (FP32 form), so that the products and
 *              reciprocals of the smoothness terms stay in range.
 */
typedef struct {
  int nx, ny;
  double Lx, Ly;
  int velocity_set;
  double eps, tau, mach, rho0, dt;
  int s;
  double A_ex[AP_DVM_MAX_STAGES * AP_DVM_MAX_STAGES];
  double A_im[AP_DVM_MAX_STAGES * AP_DVM_MAX_STAGES];
  int space_scheme;
  int precision;
  double weno_eps;
} ap_dvm_params;

typedef struct ap_dvm_handle ap_dvm_handle;

/* ---- single solve --------------------------------------------------------- */

/* Bytes of device workspace ap_dvm_create needs for *p (0 if *p is invalid). */
size_t ap_dvm_workspace_size(const ap_dvm_params* p);

/* Create a handle for one solve (Algorithm 1 on the grid of *p).
 *  d_workspace  device buffer of at least ap_dvm_workspace_size(p) bytes,
 *               256-byte aligned, owned by the caller for the handle's life.
 *  cuda_stream  cudaStream_t on which all work is enqueued (NULL = legacy default).
 *  out          receives the handle (host memory owned by the library; free
 *               with ap_dvm_destroy).
 * The state is zero until set with ap_dvm_set_state / _equilibrium / _populations. */
ap_dvm_status ap_dvm_create(const ap_dvm_params* p, void* d_workspace, size_t bytes, void* cuda_stream,
                            ap_dvm_handle** out);

/* ---- batches of uneven solves (one launch per kernel covers all of them) ---- */

/* Bytes of the batch tables for up to `capacity` instances whose sizes do not
 * exceed tmpl->nx, tmpl->ny.  tmpl fixes the scheme, precision and tableau. */
size_t ap_dvm_batch_workspace_size(const ap_dvm_params* tmpl, int capacity);
/* Bytes of device workspace of one instance attached to a batch. */
size_t ap_dvm_instance_workspace_size(const ap_dvm_params* p);
/* Create an empty batch. */
ap_dvm_status ap_dvm_batch_create(const ap_dvm_params* tmpl, int capacity, void* d_workspace, size_t bytes,
                                  void* cuda_stream, ap_dvm_handle** out);
/* Attach a solve to slot 0 <= slot < capacity with its own workspace of
 * ap_dvm_instance_workspace_size(p) bytes.  p must share the template's
 * scheme, precision and tableau; nx <= tmpl->nx, ny <= tmpl->ny, and its
 * transform lengths (n, or M for a size that is not a power of two) must not
 * exceed the template's longest (AP_DVM_ERR_ARG otherwise).  Must not be
 * called while the handle's stream is being captured. */
ap_dvm_status ap_dvm_attach(ap_dvm_handle* h, int slot, const ap_dvm_params* p, void* d_workspace, size_t bytes);
/* Remove a solve from the batch; its workspace may be reused once the stream
 * has passed this point. */
ap_dvm_status ap_dvm_detach(ap_dvm_handle* h, int slot);

/* ---- state (slot = 0 for a single solve) ----------------------------------- */

/* Set the moment state from 6 double planes (u1, u2, theta, v1, v2, q). */
ap_dvm_status ap_dvm_set_state(ap_dvm_handle* h, int slot, const double* d_moments6);
/* Set the state at equilibrium from a velocity and a pressure (3 double
 * planes): theta = p + |u|^2/2 (Sec. 3.1), v = F(u) = ((u2^2-u1^2)/2, u1 u2), q = 0. */
ap_dvm_status ap_dvm_set_equilibrium(ap_dvm_handle* h, int slot, const double* d_u1, const double* d_u2,
                                     const double* d_p);
/* Set the state from 6 population planes: double (FP64 form or FP32 form),
 * or float (is_float = 1, FP32 form only). */
ap_dvm_status ap_dvm_set_populations(ap_dvm_handle* h, int slot, const void* d_dF6, int is_float);
/* AP_DVM_FP32_DEV_TH only: overwrite the carried theta plane with d_theta
 * (one double plane, rounded once to FP32), e.g. after ap_dvm_set_populations,
 * which sums theta from the populations; with the populations read by
 * ap_dvm_get_populations (float) and theta by ap_dvm_get_state, the two calls
 * restore a solve bit for bit.  AP_DVM_ERR_ARG in the other forms. */
ap_dvm_status ap_dvm_set_theta(ap_dvm_handle* h, int slot, const double* d_theta);
/* Read the moment state into 6 double planes (the FP32 forms: the moments of the
 * populations in FP64, with the carried theta in AP_DVM_FP32_DEV_TH). */
ap_dvm_status ap_dvm_get_state(ap_dvm_handle* h, int slot, double* d_moments6);
/* Read the populations into 6 planes (double, or float when is_float = 1). */
ap_dvm_status ap_dvm_get_populations(ap_dvm_handle* h, int slot, void* d_dF6, int is_float);
/* Macroscopic outputs (4 double planes): density rho = rho0 (1 + 2 mach eps theta),
 * velocity u1, u2 and pressure p = theta - |u|^2/2 (Sec. 3.1, theta = p + |u|^2/2). */
ap_dvm_status ap_dvm_moments(ap_dvm_handle* h, int slot, double* d_rho, double* d_u1, double* d_u2, double* d_p);

/* Flow diagnostics of the state of slot (Sec. 4: the divergence history of
 * Figs. 2-3 and the vorticity of Tables 1-2), with the central difference D_0
 * of the solve's scheme (2nd order for AP_DVM_LF1_C2, 4th order otherwise):
 *   out3[0] = max |D_0 . u|,  out3[1] = (sum (D_0 . u)^2 dx dy)^(1/2),
 *   out3[2] = (1/2) sum omega^2 dx dy,  omega = D_0x u2 - D_0y u1.
 * d_vorticity (device, nullable) receives omega as nx*ny doubles.  out3 is a
 * host array of 3 doubles.  Synchronises the stream; the slot's right-hand-side
 * plane serves as scratch, so call it between steps, not while a graph of
 * steps is being captured. */
ap_dvm_status ap_dvm_diagnostics(ap_dvm_handle* h, int slot, double* d_vorticity, double* out3);

/* ---- time stepping ------------------------------------------------------------ */

/* Advance every attached solve by nsteps IMEX steps (Algorithm 1; the GSA
 * property makes the last stage the new state).  Asynchronous.  With
 * graph steps k > 0 (ap_dvm_set_graph_steps) the steps are replayed from a
 * CUDA graph of k steps. */
ap_dvm_status ap_dvm_step(ap_dvm_handle* h, int nsteps);
/* Advance the attached solves by different numbers of steps in one call: the
 * solve in slot k by steps_per_slot[k] steps (host array of capacity entries,
 * read for attached slots only, each in [0, nsteps]; else AP_DVM_ERR_ARG and
 * nothing runs).  The call runs nsteps steps at most, as ap_dvm_step does, in
 * segments between the counts at which solves drop out: a solve whose count is
 * reached sits out the remaining steps (it leaves the kernels' work lists and
 * its state stays as it is), so a short request does not shorten the others'
 * share of the call.  Each solve ends exactly where ap_dvm_step would leave it
 * after its own count of steps.  Asynchronous; the work lists are re-uploaded
 * at each change of the stepping set (stream-ordered copies), so the call may
 * not run inside a stream capture when the counts differ. */
ap_dvm_status ap_dvm_step_slots(ap_dvm_handle* h, int nsteps, const int* steps_per_slot);
/* Use a captured CUDA graph of k steps for ap_dvm_step (k = 0: direct launches). */
ap_dvm_status ap_dvm_set_graph_steps(ap_dvm_handle* h, int k);
/* Tile shape of the stencil kernels: 0 = 32x8, 1 = 32x4, 2 = 16x8, 3 = 8x8,
 * 4 = 64x4, 5 = 32x16, -1 = automatic.  Every attached grid must be at least the tile. */
ap_dvm_status ap_dvm_set_tile(ap_dvm_handle* h, int tile);
int ap_dvm_get_tile(const ap_dvm_handle* h);
/* Kernel launches enqueued by one ap_dvm_step(h, 1). */
int ap_dvm_launches_per_step(const ap_dvm_handle* h);

/* Per-kernel timing.  While enabled, ap_dvm_step launches directly (no graph)
 * and brackets every kernel with CUDA events on the handle's stream; enabling
 * or disabling resets the totals. */
ap_dvm_status ap_dvm_profile_enable(ap_dvm_handle* h, int enable);
/* Synchronise and read per-kernel totals since the last reset: up to max
 * entries of kernel name (static string), total milliseconds and launch
 * count.  Returns the number of kernel kinds (8: explicit, rhs, fft_rows_fwd,
 * fft_cols, fft_rows_inv, update, finish, stage1), or -1 on error. */
int ap_dvm_profile_read(ap_dvm_handle* h, const char** names, double* total_ms, long* launches, int max);

/* End-to-end call on HOST buffers: copy 6 moment planes h_in (double) to the
 * device, set the state of slot, run nsteps, and copy the moment state back
 * into h_out (6 double planes); synchronous.  Pinned host memory gives
 * asynchronous copies; d_stage must hold 6 planes of doubles. */
ap_dvm_status ap_dvm_run_host(ap_dvm_handle* h, int slot, const double* h_in, double* h_out, double* d_stage,
                              int nsteps);

/* Advance one small FP64 solve by nsteps IMEX steps without allocating or
 * being given any device memory beyond its state.  The paper has no
 * counterpart: this is a deployment variant of ap_dvm_create + ap_dvm_step
 * for callers that cannot call cudaMalloc or hand over a workspace, e.g.
 * code running under a host framework that owns every device allocation,
 * real-time loops that forbid allocation after start-up, or plugins loaded
 * into a process whose allocator they may not touch.
 *  p          parameters (FP64 form only; nx, ny powers of two <= 128 and
 *             the whole scratch of the solve <= 8 MiB: at 128 x 128, CK/ARS
 *             tableaux up to 4 stages, type-A tableaux up to 3).
 *  d_state6   device moment state, 6 double planes (u1, u2, theta, v1, v2, q):
 *             read at the start, overwritten with the state after nsteps.
 *  cuda_stream  stream for the copies and kernels.
 * Returns AP_DVM_ERR_ARG for invalid parameters or a grid beyond the limit
 * above, AP_DVM_ERR_UNSUPPORTED for the FP32 form or a size that is not a
 * power of two, AP_DVM_ERR_CUDA if a CUDA call fails, and, like
 * ap_dvm_sync_status, AP_DVM_ERR_TIMEOUT if a kernel gave up a bounded wait
 * for one of its tile copies (the state is then invalid) or
 * AP_DVM_ERR_NONFINITE if a step produced a non-finite value (d_state6 then
 * holds that state).  The scratch is one 8 MiB file-scope device array that
 * every GPU which loads this library holds until the process exits; the
 * first call on a device looks up that array's address.  Each call is
 * synchronous: it synchronises the stream after staging its small
 * descriptors from host memory, and again at the end to read the device
 * error flags, so it cannot be called while the stream is being captured
 * into a CUDA graph.  All calls share the one array and it keeps the last
 * call's contents: calls whose work overlaps on the GPU (other streams,
 * other host threads) race and give wrong results; serialise them. */
ap_dvm_status ap_dvm_step_noalloc(const ap_dvm_params* p, double* d_state6, int nsteps, void* cuda_stream);

/* Synchronise the stream and return AP_DVM_ERR_TIMEOUT if a kernel gave up a
 * bounded wait for one of its tile copies (2 s), else AP_DVM_ERR_NONFINITE if
 * any step since the last call produced a non-finite value; the flags are
 * then cleared. */
ap_dvm_status ap_dvm_sync_status(ap_dvm_handle* h);
/* Exercise the timeout path of the bounded device waits without a fault:
 * enqueue on the handle's stream one kernel that waits, with the same bounded
 * wait the stencil kernels use for their tile copies and a limit of wait_ns
 * nanoseconds (in [1e3, 1e10]), on an mbarrier that nothing completes.  The
 * wait expires, the kernel sets the handle's timeout flag and returns, so the
 * next ap_dvm_sync_status returns AP_DVM_ERR_TIMEOUT and the context stays
 * usable.  The paper has no counterpart: this checks the library's failure
 * detection.  Returns AP_DVM_ERR_ARG for a limit out of range. */
ap_dvm_status ap_dvm_check_wait_timeout(ap_dvm_handle* h, long long wait_ns);
/* Message of the last error on this handle (never NULL). */
const char* ap_dvm_last_error(const ap_dvm_handle* h);
/* Release the handle (host memory and graphs); device workspaces stay with the caller. */
void ap_dvm_destroy(ap_dvm_handle* h);

/* ---- measurement ---------------------------------------------------------------- */

/* Arithmetic peak of the current GPU for the roofline of the FP64 form (the
 * paper has no counterpart: it reports no hardware figures).  Launches a
 * kernel whose threads run only independent fused multiply-add chains
 * (FP64 for precision = AP_DVM_FP64, FP32 for AP_DVM_FP32_DEV), as many
 * resident 256-thread blocks as fit on every SM, `iters` x 128 FMAs per
 * thread, once to warm up and then `reps` times between CUDA events on
 * cuda_stream; synchronises.  Writes the rate (2 flops per FMA) to *tflops
 * and the mean launch time to *ms_per_launch.  Returns AP_DVM_ERR_ARG for
 * null outputs, iters < 1, reps < 1 or another precision, AP_DVM_ERR_CUDA if
 * a CUDA call fails. */
ap_dvm_status ap_dvm_fma_peak(int precision, int iters, int reps, void* cuda_stream, double* tflops,
                              double* ms_per_launch);

/* Self-check of the integer-pipe FP32 <-> FP64 conversions the FP32 forms use in place
 * of the conversion instructions (the moment sums of the close and the FP64
 * relaxations): for each of the n FP64 values at d_in (device), the narrowing to FP32
 * (nearest, ties to even) and the widening of that FP32 value back to FP64 are compared
 * with the instructions' results bit for bit (a NaN only as a NaN).  d_counts (device,
 * 2 unsigned, caller-owned) receives the numbers of mismatching narrowings and
 * widenings; it is zeroed first.  Asynchronous on cuda_stream.  Returns AP_DVM_ERR_ARG
 * for null pointers or n < 0, AP_DVM_ERR_CUDA if a launch fails. */
ap_dvm_status ap_dvm_check_conversions(const double* d_in, int n, unsigned* d_counts, void* cuda_stream);

/* Fill *p with defaults: 2 pi periodic square, D2V6, rho0 = 1, mach = 1e-2,
 * tau = 0.05, the second-order GSA tableau of Sec. 4.1 (c = 2.25), WENO5+C4,
 * FP64, weno_eps = 1e-6; nx, ny, eps and dt are set from the arguments. */
void ap_dvm_default_params(ap_dvm_params* p, int nx, int ny, double eps, double dt);

#ifdef __cplusplus
}
#endif
#endif /* AP_DVM_H */
