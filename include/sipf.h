/*
 * sipf.h — C ABI of the GB300 SIPF-PIC library (libsipf.so).
 *
 * The library advances the stochastic interacting particle-field method with
 * particle-in-cell acceleration (SIPF-PIC, Algorithm 4 of "A fast stochastic
 * interacting particle-field method for 3D parabolic-parabolic chemotaxis
 * systems", arXiv 2512.03452) for the Keller-Segel system
 *     rho_t = div(mu grad rho - chi rho grad c),  eps c_t = Lap c - k^2 c + rho
 * on the periodic box [-L/2, L/2)^3 (Sec. 2.2), on one CUDA GPU.
 *
 * Conventions shared by every entry point
 *   - Return value: SIPF_OK (0) or a negative SIPF_E* code; nothing throws.
 *     sipf_strerror() names a code, sipf_last_error() gives the message of the
 *     last failure on the calling thread.
 *   - Host buffers are owned by the caller; the library copies them and never
 *     keeps a caller pointer after the call returns.
 *   - A context owns all device memory it allocates and is not thread-safe.
 *     Its work is ordered on the CUDA stream given at sipf_init (NULL: the
 *     library creates one).  Entry points that return host data synchronise
 *     that stream; sipf_step / sipf_run only enqueue work.
 *   - Device-pointer entry points (suffix _dev) take caller-owned device
 *     memory, launch on the given stream and return without synchronising.
 *     Positions on the device are structure-of-arrays: x, y, z arrays of P
 *     elements, in the context's precision (float for 32, double for 64).
 *   - Grids are H^3 real arrays, row-major with the third axis fastest:
 *     node (i, j, k) at [(i*H + j)*H + k]; node index j in [-H/2, H/2) is
 *     stored at j mod H and sits at x = j*L/H.
 *   - Spectra are the r2c half layout H x H x (H/2+1) of interleaved complex
 *     numbers (re, im); index m on an axis stands for q = m (m < H/2) or
 *     q = m - H (m >= H/2).
 */
#ifndef SIPF_H
#define SIPF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define SIPF_OK 0
#define SIPF_EINVAL (-1)      /* bad argument or parameter                */
#define SIPF_ENOMEM (-2)      /* device or host allocation failed        */
#define SIPF_ECUDA (-3)       /* a CUDA call failed                       */
#define SIPF_ENONFINITE (-4)  /* a position or spectrum became non-finite */
#define SIPF_ETIMEOUT (-5)    /* a bounded device wait ran out            */
#define SIPF_ENODEV (-6)      /* no usable CUDA device                    */

/* ---- option values ------------------------------------------------------ */
#define SIPF_SPLIT_HALF 0     /* W^- , drift at X+W^-, W^+  (Algorithm 4)       */
#define SIPF_SPLIT_PLAIN 1    /* Euler-Maruyama, Eq. (rho_hat_update)            */
#define SIPF_DEPOSIT_ATOMIC 0 /* floating-point atomics (order-dependent rounding) */
#define SIPF_DEPOSIT_DETERMINISTIC 1 /* 64-bit fixed-point sums: bit-reproducible */
#define SIPF_PROP_IMPLICIT 0  /* implicit Euler, Eq. (alpha_hat_update)           */
#define SIPF_PROP_EXP 1       /* exponential propagator, Sec. 3.4                 */

/* Parameters of one run.  Names follow the problem statement (Sec. 2.2,
 * Eq. (system)) and Algorithm 4.  sipf_params_default() fills the defaults. */
typedef struct sipf_params {
  double chi;        /* chemotactic sensitivity, > 0 (>= 0 allowed)          */
  double mu;         /* diffusivity, > 0                                      */
  double eps;        /* relaxation rate of c, > 0                             */
  double k;          /* degradation rate, >= 0                                */
  double L;          /* box side; domain [-L/2, L/2)^3, periodic              */
  double mass;       /* M0; every particle carries M0/P (Eq. (def_rho_hat))   */
  double dt;         /* tau, > 0                                               */
  double T;          /* final time for sipf_run: N_T = ceil(T/tau)            */
  double H0;         /* Gaussian filter scale: < 0 auto ceil(8 H^(8/13) L^(5/13))
                        (Sec. 5.1), 0 off, > 0 as given                       */
  uint64_t seed;     /* key of the counter-based noise                        */
  int64_t P;         /* number of particles, 1 <= P <= 2^30                    */
  int32_t H;         /* modes / grid points per axis: power of 2 in [8, 256]   */
  int32_t precision; /* 32 (float state and kernels) or 64 (double)           */
  int32_t p2g_order; /* 4 (Gamma_4, default) or 2 (Gamma_2), Sec. 3.1         */
  int32_t g2p_order; /* 2 (Gamma_2, default) or 4 (Gamma_4)                   */
  int32_t splitting; /* SIPF_SPLIT_*                                           */
  int32_t deposit_mode; /* SIPF_DEPOSIT_*                                      */
  int32_t propagator;   /* SIPF_PROP_*                                         */
  int32_t resort_every; /* rebuild the tile-bin capacities every n steps (0: 16);
                           results do not depend on it                         */
} sipf_params;

/* FP64 diagnostics of the current state (Sec. 5). */
typedef struct sipf_diag {
  double mass;        /* sum of the deposited mass grid I rho-hat, accumulated in FP64 */
  double alpha0;      /* zero mode of c-hat, carried in FP64                          */
  double peak;        /* max over the grid of rho_num = F^-1(Phi F_H I rho-hat)       */
  double hf_frac;     /* share of sum |alpha_q|^2 in modes with ||q|| >= 4            */
  double m2;          /* (1/P) sum_p |X_p|^2                                            */
  double ring_radius; /* (1/P) sum_p sqrt(x1^2 + x2^2)  (R_num of Sec. 5.4)             */
  int64_t step;       /* n of the state the numbers describe                          */
} sipf_diag;

typedef struct sipf_ctx sipf_ctx;

/* Fill *p with the defaults: chi=mu=eps=k=1, L=1, mass=1, dt=1e-3, T=0,
 * H0=-1 (auto), seed=0, P=0 (must be set), H=64, precision=32,
 * p2g_order=4, g2p_order=2, splitting=HALF, deposit_mode=ATOMIC,
 * propagator=IMPLICIT, resort_every=0 (16).  Returns SIPF_EINVAL if p is NULL. */
int sipf_params_default(sipf_params* p);

/* Check a parameter set without touching the GPU.  SIPF_EINVAL names the
 * first offending field in sipf_last_error(). */
int sipf_validate(const sipf_params* p);

/* The Gaussian filter scale a context built from *p uses (host only, no GPU):
 * p->H0 when it is >= 0, else the automatic H0 = ceil(8 H^(8/13) L^(5/13)) of
 * Sec. 5.1, evaluated exactly where the value is an integer (H = L = 8 gives
 * 64).  *H0_out receives it.  SIPF_EINVAL for NULL pointers or parameters
 * sipf_validate rejects. */
int sipf_filter_scale(const sipf_params* p, double* H0_out);

/* Create a context: validate *p, allocate the state on the current CUDA
 * device, copy X0 (host, P x 3 row-major float64, i.e. x0 y0 z0 x1 ...;
 * points outside the box are wrapped into it), set alpha^(0) = 0 and deposit
 * X^(0) (initialisation of Algorithm 4).  stream: a cudaStream_t or NULL.
 * On success *out owns the context; release it with sipf_destroy. */
int sipf_init(const sipf_params* p, const double* X0, void* stream, sipf_ctx** out);

/* Advance nsteps >= 0 steps of Algorithm 4 (asynchronous on the context's
 * stream): per step, F_H of the deposited masses, the implicit update of
 * alpha (Eq. (alpha_hat_update)) with the filtered spectral gradient of
 * alpha^(n-1), three inverse transforms, the particle move (W^-, gather of
 * grad c at X + W^- with I*, drift, W^+, periodic wrap) with re-binning of
 * the particles by grid tile; the deposit of X^(n) is made when the grid is
 * next read (the next step's first kernel, or a density query). */
int sipf_step(sipf_ctx* ctx, int64_t nsteps);

/* Advance until n * dt >= T (N_T = ceil(T/dt) steps in total). */
int sipf_run(sipf_ctx* ctx);

/* Current step index n (number of steps taken since sipf_init). */
int64_t sipf_current_step(const sipf_ctx* ctx);

/* Copy X^(n) to host `out` (P x 3 row-major float64).  Synchronises. */
int sipf_positions(sipf_ctx* ctx, double* out);

/* Replace X^(n) by host `X` (P x 3 row-major float64; wrapped into the box)
 * and re-deposit it.  The step index and alpha are kept. */
int sipf_set_positions(sipf_ctx* ctx, const double* X);

/* Host<->device copies of X in the context's own precision and layout
 * (three arrays of P floats or doubles).  Asynchronous on the context's
 * stream when the host buffers are pinned; the caller keeps them alive and
 * unchanged until sipf_sync().  upload re-deposits the new positions.
 * download into page-locked buffers mapped into the device's address space
 * (cudaHostAlloc / cudaHostRegister memory) is written by a kernel directly;
 * other buffers are filled through staged copies. */
int sipf_upload_soa(sipf_ctx* ctx, const void* x, const void* y, const void* z);
int sipf_download_soa(sipf_ctx* ctx, void* x, void* y, void* z);

/* Write X^(n) in particle order into caller-owned device arrays x, y, z (P
 * elements each, float or double as the context's precision).  Internally the
 * particles are kept grouped by grid tile; this gathers them back by id.
 * Asynchronous on the context's stream. */
int sipf_positions_dev(sipf_ctx* ctx, void* x, void* y, void* z);

/* Density on the grid (host H^3 float64).  filtered = 0: I rho-hat / h^3,
 * the deposited mass per cell volume (Def. particle2grid); filtered = 1:
 * rho_num = F_H^-1(Phi F_H I rho-hat), rho-hat convolved with N(0,(L/H0)^2 I)
 * (Sec. 5.2).  Synchronises. */
int sipf_density(sipf_ctx* ctx, double* out, int filtered);

/* c-hat^(n) on the grid nodes, F_H^-1 alpha^(n) (host H^3 float64). */
int sipf_field(sipf_ctx* ctx, double* out);

/* alpha^(n) (host, H*H*(H/2+1) complex as 2 float64 each). */
int sipf_spectrum(sipf_ctx* ctx, double* out);

/* The gradient grids F_H^-1(2 pi i q/L Phi alpha^(n)) used by the next move
 * (host, 3 x H^3 float64: component-major). */
int sipf_gradient(sipf_ctx* ctx, double* out);

/* FP64 diagnostics of the current state.  Synchronises. */
int sipf_diagnostics(sipf_ctx* ctx, sipf_diag* out);

/* Device time of the steps taken while timing is on, per stage, from CUDA
 * events recorded on the context's stream around each stage of every step;
 * `kernels` counts the library kernels those steps launched. */
typedef struct sipf_timing {
  double forward_ms;     /* F_H of the deposit: rows r2c + middle-axis pass  */
  double spectral_ms;    /* x-axis pass fused with the update of alpha and G  */
  double inverse_ms;     /* middle-axis pass + rows c2r of the 3 gradients    */
  double move_ms;        /* move + re-bin kernel (noise, gather, push)        */
  double bookkeeping_ms; /* chunk lists and periodic capacity rebuilds        */
  double deposit_ms;     /* deposit of the new positions from their bins      */
  int64_t steps;
  int64_t kernels;
  int64_t overflow;      /* particle-steps spent in the overflow bin (deposited
                            with global reductions instead of a window)       */
} sipf_timing;

/* Start (enable != 0) or stop recording per-stage events; starting clears
 * the accumulated times. */
int sipf_timing_enable(sipf_ctx* ctx, int enable);

/* Synchronise and add up the recorded stage times. */
int sipf_timing_read(sipf_ctx* ctx, sipf_timing* out);

/* Kernels launched by the context since sipf_init (host-side count). */
int64_t sipf_kernel_launches(const sipf_ctx* ctx);

/* Wait for the context's stream and report the kernels' sticky error flags
 * since the last call (then cleared): SIPF_ENONFINITE for a non-finite
 * position, SIPF_ETIMEOUT for a bounded wait on a staging copy that ran out,
 * SIPF_ENOMEM if the overflow bin of the particle layout was full (a particle
 * was dropped). */
int sipf_sync(sipf_ctx* ctx);

/* Free everything the context owns.  NULL is a no-op. */
void sipf_destroy(sipf_ctx* ctx);

const char* sipf_strerror(int code);
const char* sipf_last_error(void);

/* ---- batched runs --------------------------------------------------------
 * Many independent runs of Algorithm 4 (an ensemble over seeds, chi, P, H,
 * ... as in the parameter studies of Sec. 5) advanced together: per step the
 * field solve is launched once per distinct grid size H (runs of equal H in
 * one launch of each FFT kernel) and every particle pass once for all runs,
 * whose work items are drawn from one shared counter.  Steps are recorded
 * in a CUDA graph of 32 steps and replayed.  Each run computes exactly what
 * a sipf_ctx with the same parameters and X0 computes (bit for bit in
 * deterministic deposit mode; up to the order of floating-point atomic
 * additions otherwise).
 */
typedef struct sipf_batch sipf_batch;

/* Create nruns runs: run r has parameters params[r] and initial positions
 * X0[r] (host, params[r].P x 3 row-major float64).  All runs must share
 * precision and deposit_mode, have H >= 32 and resort_every 0 or 16;
 * 1 <= nruns <= 4096.
 * stream: a cudaStream_t (not the legacy default stream, which cannot be
 * captured) or NULL for a stream the batch creates.  On failure nothing is
 * left allocated and *out is NULL; SIPF_EINVAL names the offending run. */
int sipf_batch_init(int32_t nruns, const sipf_params* params, const double* const* X0,
                    void* stream, sipf_batch** out);

/* Advance every run by nsteps >= 0 steps (asynchronous on the batch's
 * stream).  The step index n is shared by all runs and kept on the device. */
int sipf_batch_step(sipf_batch* b, int64_t nsteps);

/* Launch shapes chosen by sipf_batch_autotune, per distinct grid size H
 * (groups in order of first appearance) and for the particle passes. */
typedef struct sipf_batch_tuning {
  int32_t ngroups;
  int32_t H[4];
  int32_t cols_tile[4];           /* pencils per block of the y passes: 8, 16, 32   */
  int32_t xpass_tile[4];          /* pencils per block of the fused x pass: 4, 8, 16 */
  int32_t rows_blocks_per_sm[4];  /* blocks per SM shared by the row passes          */
  int32_t plane_kernels[4];       /* 1: both inner axes in one plane kernel per
                                     direction (one x-plane per block); 2: the same
                                     with each x-plane's columns spread over a
                                     cluster of 2 (H <= 128) or 4 (H = 256) blocks
                                     sharing rows through distributed shared
                                     memory (H >= 64); 0: separate pencil passes */
  int32_t plane_warps[4];         /* warps per block of the plane kernels: 8, 16, 32 */
  int32_t xpass_warps[4];         /* warps per block of the fused x pass: 8, 16      */
  int32_t inverse_all_components[4]; /* inverse plane kernel: 1 one block per x-plane for
                                     all three gradient components, writing whole
                                     nodes (H <= 64); 2 one block per (component,
                                     x-plane); 0 chosen by the number of blocks    */
  int32_t move_blocks_per_sm;     /* move + re-bin blocks per SM (0: occupancy limit) */
  int32_t deposit_blocks_per_sm;  /* deposit blocks per SM (0: occupancy limit)       */
  double field_ms[4];             /* best device ms per step of each group's field solve */
  double move_ms;                 /* best device ms per step: move, chunk lists, run prefix */
  double deposit_ms;              /* best device ms per step: deposit                   */
  int64_t steps_used;             /* steps the runs advanced while tuning               */
} sipf_batch_tuning;

/* Autotuner of the batch's tile and block shapes: coordinate descent over the
 * candidates above, each timed with CUDA events on steps_per_trial (>= 2)
 * real steps of the batch (the first step of a trial is not timed).  Shapes
 * do not change results, so the runs advance by out->steps_used steps (about
 * steps_per_trial x (18 per group + 9)).  Later steps use the chosen shapes;
 * out may be NULL.  Synchronises. */
int sipf_batch_autotune(sipf_batch* b, int32_t steps_per_trial, sipf_batch_tuning* out);

/* Apply a tuning (for example one saved from sipf_batch_autotune on the same
 * kind of batch): groups must list the batch's H values in the same order;
 * 0 in a shape field means the default.  SIPF_EINVAL for shapes the kernels
 * do not support (shared memory). */
int sipf_batch_set_tuning(sipf_batch* b, const sipf_batch_tuning* t);

/* enable = 0: issue every step's launches directly instead of replaying the
 * recorded 32-step graph (same results; for timing the graph's benefit). */
int sipf_batch_use_graph(sipf_batch* b, int enable);

/* Step index n of all runs; -1 for NULL. */
int64_t sipf_batch_current_step(const sipf_batch* b);

/* Library kernels launched since sipf_batch_init, counting every kernel of
 * a replayed graph (host-side count); -1 for NULL. */
int64_t sipf_batch_kernel_launches(const sipf_batch* b);

/* Per-run read-back, as sipf_positions / sipf_diagnostics / sipf_spectrum
 * for run `run` (0 <= run < nruns).  Synchronise. */
int sipf_batch_positions(sipf_batch* b, int32_t run, double* out);
int sipf_batch_diagnostics(sipf_batch* b, int32_t run, sipf_diag* out);
int sipf_batch_spectrum(sipf_batch* b, int32_t run, double* out);

/* Wait for the batch's stream; report the first run's sticky kernel error
 * flags as sipf_sync does. */
int sipf_batch_sync(sipf_batch* b);

/* Free every run and the batch.  NULL is a no-op. */
void sipf_batch_destroy(sipf_batch* b);

/* ---- adjoint -------------------------------------------------------------
 * Gradients of a scalar J(rho(T)) with respect to chi, mu and X^0 through
 * N = nsteps steps of Algorithm 4, the noise held fixed (the same Philox
 * counters as the forward), by reverse mode with hand-written transposes of
 * every operator of the step: the deposit I and the gather I* are each
 * other's transposes (<I rho, f> = <rho, I* f>, the relation stated after
 * Def. grid2particle in Sec. 3.1), the transpose of F_H is L^-3 F_H^-1,
 * pointwise spectral factors turn into their complex conjugates, and
 * particle positions enter through the derivatives of the weight
 * polynomials of Eqs. (2ord) and (4ord).  rho(T) is the deposited density
 * I rho-hat / h^3 of X^N (sipf_density with filtered = 0).
 * Memory: the forward keeps X^n (id order) and alpha^n every
 * checkpoint_every steps; the reverse sweep recomputes one segment at a time
 * and holds its X^{n-1} and gradient grids.  chi and mu > 0 may change
 * between forward calls; the other parameters are fixed at init.
 */
typedef struct sipf_adjoint sipf_adjoint;

/* Create the adjoint engine for parameters *p (p->chi and p->mu are the
 * first values; p->mu > 0), initial positions X0 (host P x 3 float64), N =
 * nsteps >= 1, checkpoint_every >= 1 (0: 20).  stream: cudaStream_t or NULL. */
int sipf_adjoint_init(const sipf_params* p, const double* X0, int64_t nsteps,
                      int32_t checkpoint_every, void* stream, sipf_adjoint** out);

/* Run the N forward steps from X0 (host P x 3 float64; NULL keeps the last
 * one) with the given chi and mu, keeping the checkpoints, and write rho(T)
 * (host H^3 float64) to rho_out unless NULL.  Synchronises. */
int sipf_adjoint_forward(sipf_adjoint* a, double chi, double mu, const double* X0,
                         double* rho_out);

/* Given rho_bar = dJ/drho(T) (host H^3 float64), write dJ/dchi, dJ/dmu and
 * dJ/dX^0 (host P x 3 float64); any output may be NULL.  Needs a preceding
 * sipf_adjoint_forward.  dJ/dchi and dJ/dmu are accumulated in FP64.
 * Synchronises. */
int sipf_adjoint_backward(sipf_adjoint* a, const double* rho_bar, double* grad_chi,
                          double* grad_mu, double* grad_X0);

/* Device time of the last forward and backward calls (CUDA events). */
int sipf_adjoint_timing(const sipf_adjoint* a, double* forward_ms, double* backward_ms);

/* Library kernels launched by the engine so far; -1 for NULL. */
int64_t sipf_adjoint_kernel_launches(const sipf_adjoint* a);

void sipf_adjoint_destroy(sipf_adjoint* a);

/* Measure this GPU's FP64 fused multiply-add throughput (GFLOP/s, 2 per FMA)
 * with a throughput-bound kernel of independent FMA chains on `stream`;
 * the FP64 form's arithmetic bound.  Synchronises. */
int sipf_measure_fp64_fma(void* stream, double* gflops);

/* ---- stateless operators on caller-owned device memory ------------------
 * precision: 32 or 64 (element type float / double of every real array).
 * All are asynchronous on `stream` (cudaStream_t or NULL for the default).
 */

/* Philox4x32-10 normals: z[j*P + p] for j = 0..5, particle index first+p,
 * counter (particle lo, particle hi, step, block), key (seed lo, seed hi),
 * Box-Muller on uniforms (x + 1/2) 2^-32.  (Algorithm 4 draws
 * W^-, W^+ ~ N(0, mu tau I) from z0..z2 and z3..z5.) */
int sipf_noise_dev(int precision, uint64_t seed, int64_t step, int64_t first,
                   int64_t P, void* z, void* stream);

/* Algorithm 2 without its FFT: grid (H^3, zeroed here first) receives
 * w * F_gamma(lambda(X_p)) at (floor(H X_p/L) + gamma) mod H for every
 * particle, order 2 (Gamma_2) or 4 (Gamma_4). */
int sipf_deposit_dev(int precision, const void* x, const void* y, const void* z,
                     int64_t P, int32_t H, double L, double w, int32_t order,
                     void* grid, void* stream);

/* Algorithm 3: out[c*P + p] = sum_gamma F_gamma(lambda(X_p)) f_c[...] for
 * ncomp component grids f (component c at f + c*H^3), order 2 or 4. */
int sipf_gather_dev(int precision, const void* x, const void* y, const void* z,
                    int64_t P, int32_t H, double L, const void* f, int32_t ncomp,
                    int32_t order, void* out, void* stream);

/* beta = F_H(grid) = L^-3 sum_j grid_j e^{-2 pi i q.j/H} (Sec. 3.1) into the
 * half spectrum `spec` (H*H*(H/2+1) complex values). */
int sipf_forward_ft_dev(int precision, int32_t H, double L, const void* grid,
                        void* spec, void* stream);

/* grid = F_H^-1(spec) = sum_q spec_q e^{+2 pi i q.j/H} (real part of the
 * Hermitian extension); `spec` is overwritten (used as work space). */
int sipf_inverse_ft_dev(int precision, int32_t H, void* spec, void* grid,
                        void* stream);

/* The inverse transform of sipf_inverse_ft_dev for callers that cannot
 * allocate device memory -- for example code running inside another
 * library's callback, a server with a fixed memory budget, or any path where
 * the implicit device synchronisation of cudaMalloc/cudaFree is not allowed.
 * The paper has no counterpart: this is a property of the library only.
 *   - Unlike sipf_inverse_ft_dev, `spec` is left unchanged: the transform runs
 *     in a work space built into the library (a static device array of
 *     64*64*33 complex doubles, about 2.1 MB, held on every GPU that loads the
 *     library until the process exits).  H*H*(H/2+1) complex values must fit
 *     in it: H <= 64 in either precision; larger H returns SIPF_EINVAL.
 *   - Nothing is allocated; the spectrum is copied device to device into the
 *     work space, then transformed as in sipf_inverse_ft_dev.
 *   - The first call on a device looks up the work space's device address
 *     (and uploads the twiddle table if no other entry point did); make that
 *     first call before any stream capture.
 *   - All calls share the one work space, which keeps the last call's
 *     contents.  Calls whose work overlaps on the GPU (different streams, or
 *     different host threads without ordering) race and give wrong results;
 *     order them on one stream. */
int sipf_inverse_ft_noalloc_dev(int precision, int32_t H, const void* spec, void* grid,
                                void* stream);

/* ---- 2D variant: the parabolic-elliptic system of Sec. 5.2 ---------------
 * The Keller-Segel system in two dimensions on [-L/2, L/2)^2 with an H x H
 * grid, H a power of two in [8, 256]: eps = 0 is the parabolic-elliptic
 * system of Sec. 5.2 ((|y|^2 + k^2) c-hat = F_H I rho-hat, the field of level
 * n-1 driving the move of step n; k = 0 leaves the zero mode at 0), eps > 0
 * the 2D parabolic-parabolic system with the implicit update of
 * Eq. (alpha_hat_update).  Deposit with the 12-node 2D analogue of Eq. (4ord)
 * (p2g_order 4) or the bilinear stencil, gather with the bilinear stencil
 * (g2p_order 2) or the 12-node one; noise W^- = s (z0, z1), W^+ = s (z2, z3)
 * from the first Philox block of particle p at step n (the 3D generator's
 * first four normals).  Fields of sipf_params as in 3D; deposit_mode must be
 * SIPF_DEPOSIT_ATOMIC and propagator SIPF_PROP_IMPLICIT.  Particles stay in
 * particle order (no bins).  Same conventions as the 3D context (owned device
 * memory, stream ordering, not thread-safe). */
typedef struct sipf2d_ctx sipf2d_ctx;

/* Create a 2D context: X0 host P x 2 row-major float64 (wrapped into the box);
 * the initial positions are deposited.  SIPF_EINVAL for parameters outside the
 * 2D ranges above, SIPF_ENONFINITE for a non-finite coordinate. */
int sipf2d_init(const sipf_params* p, const double* X0, void* stream, sipf2d_ctx** out);
/* Advance nsteps >= 0 steps (asynchronous on the context's stream). */
int sipf2d_step(sipf2d_ctx* ctx, int64_t nsteps);
/* Steps taken since sipf2d_init (-1 for NULL). */
int64_t sipf2d_current_step(const sipf2d_ctx* ctx);
/* Positions X^(n), host P x 2 row-major float64.  Synchronises. */
int sipf2d_positions(sipf2d_ctx* ctx, double* out);
/* The field spectrum of the last step, host H x (H/2+1) x 2 float64 (eps = 0:
 * c-hat of level n-1; eps > 0: alpha^(n)).  Synchronises. */
int sipf2d_spectrum(sipf2d_ctx* ctx, double* out);
/* Host H x H float64: the deposited density I rho-hat / h^2 of X^(n)
 * (filtered = 0) or rho_num = F_H^-1(Phi F_H I rho-hat) (filtered = 1). */
int sipf2d_density(sipf2d_ctx* ctx, double* out, int filtered);
/* FP64 diagnostics: mass (sum of the deposit grid), peak of rho_num, hf_frac
 * (share of the field spectrum's energy with ||q|| >= 4), m2 = (1/P) sum |X|^2
 * (Sec. 5.2), step; alpha0 and ring_radius are 0.  Synchronises. */
int sipf2d_diagnostics(sipf2d_ctx* ctx, sipf_diag* out);
/* Wait for the context's work; SIPF_ENONFINITE if a position became non-finite. */
int sipf2d_sync(sipf2d_ctx* ctx);
/* Release the context (NULL is ignored). */
void sipf2d_destroy(sipf2d_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SIPF_H */
