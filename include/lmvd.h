/* lmvd: one Runge-Kutta substage of the low-Mach, variable-density pseudospectral method of
 * Reuter, Oliver and Moser (arXiv:2206.09878) on one GB300 GPU.
 *
 * The state S = (z, Omega2, m2^d, <m1>, <m3>) of Sec. 4.4 (Eq. DNS_system) is advanced by
 * Algorithm 2: m^d from Eq. phi_poisson / md_recon, R_z and the BDF-like guess of
 * Eq. dzdt_guesses, k_f fixed-point applications of L (Eq. y_k, Sec. 4.3), m^c from
 * Eq. COM_fourier / CF_fourier / mc_recon / mc_mean, the right-hand sides of Eq. DNS_system,
 * and the segregated midpoint RK2 update (Sec. 3.3). The adjoints of a substage and of the start-up
 * (the differentiation path) and a double-float precision path for the transforms and products are
 * part of the same library.
 *
 * Conventions shared by every call
 * --------------------------------
 * Spectral arrays are complex128 (interleaved re, im), C-contiguous, layout [y][kz][kx]:
 *   y  : B-spline coefficient index, ny rows (ny + 1 for m2, whose space has one more function);
 *   kz : nz slots in FFT order (slot j is kz = j for j < nz/2, j - nz for j > nz/2);
 *   kx : nx/2 + 1 slots, kx = 0 .. nx/2.
 * Retained modes are |kx| < nx/2, |kz| < nz/2 (Eq. disc_f); the Nyquist slots kx = nx/2 and
 * kz = nz/2 must be zero. The kx = 0 column is Hermitian in kz (f(0,-kz) = conj f(0,kz)).
 * The plane means <m1>, <m3> are float64 vectors of ny B-spline coefficients.
 * y-basis: clamped B-splines on uniform breakpoints of [y0, y1] (Appendix C), order p for all
 * fields but m2 and order p + 1 for m2, collocated at Greville abscissae.
 * Boundaries at y0 and y1: no-slip walls or the paper's potential matching (lmvd_config.bc_mode);
 * dz/dy = 0 there in both.
 *
 * Pointers passed to set/get calls may be device memory or host memory (pinned host memory
 * gives asynchronous copies); they are read or written on the context's stream with
 * cudaMemcpyDefault and remain owned by the caller. The library owns only its own workspace.
 * Every call is asynchronous on the context's stream unless it says otherwise; a caller that
 * reads an output must synchronize that stream (or call lmvd_synchronize). Inputs written on another
 * stream must be ordered before the call by the caller (e.g. an event the context's stream waits on);
 * the Python binding's Context does this for the tensors it exchanges.
 *
 * Errors: every int-returning call returns LMVD_OK (0) or a negative LMVD_ERR_* code and never
 * traps the GPU. The first error is also latched in the context (lmvd_status).
 */
#ifndef LMVD_H
#define LMVD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LMVD_OK 0
#define LMVD_ERR_INVALID_ARG (-1)
#define LMVD_ERR_CUDA (-2)
#define LMVD_ERR_OOM (-3)
#define LMVD_ERR_NONFINITE (-4)
#define LMVD_ERR_UNSUPPORTED (-5)
#define LMVD_ERR_FP_DIVERGED (-6)
/* Only in the library built with index checks (liblmvd_check.so, -DLMVD_CHECK): a kernel found an index
 * outside the array it was about to access and skipped that access. Latched by lmvd_synchronize. */
#define LMVD_ERR_OUT_OF_BOUNDS (-7)

/* Problem definition, copied at lmvd_create (all host values).
 * nx, nz      : Fourier grid (even; 3*nx/2 and 3*nz/2 must have no prime factors other than 2, 3).
 * ny          : number of order-p B-splines in y (>= p + 4).
 * spline_order: p (4 .. 8).
 * lx, lz      : periods in x and z;  y0 < y1: the boundaries in y.
 * re, sc, fr  : Reynolds, Schmidt, Froude numbers: mu = 1/re, rho D_z = 1/(re sc), g = 1/fr^2 along -y.
 * rho_heavy, rho_light: densities of the pure fluids; EOS rho = rl rh / (rh - (rh - rl) z) (Sec. 5).
 * dt          : time step of one RK2 step (two substages).
 * kf          : fixed-point applications of L per substage (Sec. 3.2).
 * beta_n, beta_p: free parameters of the guesses of Eq. dzdt_guesses (paper: 0 and -4).
 * n_startup   : fixed-point iterations from dz/dt = 0 used by lmvd_set_state without history.
 * precision   : 0 = FP64 throughout; 1 = transforms and physical-space products in double-float
 *               arithmetic on the FP32 units (pairs of floats, 48-bit significand, error-free
 *               TwoSum/TwoProd compensation), while every spectral step (collocation, m^c and m2^d
 *               solves, RHS assembly, the RK update and the state) and the EOS (rho, 1/rho, f'(z))
 *               stay FP64.
 * bc_mode     : boundary rows at y0 and y1. 0 = no-slip walls: Omega2 = 0, m2^d = dm2^d/dy = 0,
 *               m2^c = 0, <m1> = <m3> = 0, dz/dy = 0, <m2^c>(y1) = 0.
 *               1 = the paper's potential matching (Sec. 4.5, Eq. bc_both, md_bc) for a domain
 *               truncated in y: the Robin rows k m2 -+ dm2/dy = 0 at y0 / y1 (Eq. bc_both multiplied
 *               by k) on m2^c and on m2^d, phi2 = 0 at y0 and y1 as the other two m2^d rows,
 *               Omega2 = 0, d<m1>/dy = d<m3>/dy = 0, dz/dy = 0, <m2^c>(y1) = 0. Both modes put the
 *               boundary rows first and last in each per-mode system and factor it without pivoting.
 * memory_layout: 0 = automatic (the full layout unless its workspace would take more than 85% of the
 *               free device memory), 1 = full, 2 = lean (6 instead of 10 physical work fields, the products
 *               of the RHS formed in three batches instead of one, a 2-field instead of 4-field transform
 *               intermediate: the same results in about 43 GB less at 768 x 769 x 768).
 */
typedef struct {
  int nx, ny, nz, spline_order;
  double lx, lz, y0, y1;
  double re, sc, fr, rho_heavy, rho_light;
  double dt;
  int kf;
  double beta_n, beta_p;
  int n_startup;
  int precision;
  int bc_mode;
  int memory_layout;
} lmvd_config;

typedef struct lmvd_ctx lmvd_ctx;

/* Fill *cfg with the defaults (p = 6, 2 pi periods, walls at -1 and +1, Re = 1000, Sc = Fr = 1,
 * density ratio 3, dt = 1e-3, kf = 4, beta_n = 0, beta_p = -4, n_startup = 20, precision = 0, bc_mode = 0,
 * memory_layout = 0) for
 * the given grid.
 * Returns LMVD_ERR_INVALID_ARG if cfg is NULL. */
int lmvd_default_config(lmvd_config* cfg, int nx, int ny, int nz);

/* Build the y-operators (Appendix C), factor the per-mode m^c and m2^d systems (Sec. 4.1-4.2),
 * plan the transforms and allocate all device workspace (one allocation) on the current device.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream) on which every later call runs.
 * *out receives a context owned by the caller until lmvd_destroy. Synchronous.
 * Errors: INVALID_ARG (NULL pointers, bad sizes), UNSUPPORTED (grid sizes the transforms do not
 * handle: 3nx/2 and 3nz/2 must have no prime factors but 2 and 3, 3nx/2 <= 1536, 3nz/2 <= 3072),
 * OOM (device allocation failed), CUDA (any other CUDA failure). */
int lmvd_create(const lmvd_config* cfg, void* cuda_stream, lmvd_ctx** out);

/* Release all device memory of the context. NULL is ignored. */
void lmvd_destroy(lmvd_ctx* ctx);

/* Load the state (Sec. 4.4: z, Omega2, m2^d -- held instead of phi2 = (d2/dy2 - k^2) m2^d -- and
 * the plane means). z_hat, omega2_hat: ny rows; m2d_hat: ny + 1 rows; mean_m1, mean_m3: ny doubles.
 * history: NULL, or a blob of lmvd_history_bytes() bytes from lmvd_get_state (restart).
 * With history == NULL the substage counter is reset to 0 and a start-up runs: n_startup
 * applications of the fixed point of Eq. dz_fixedpoint_stageone from dz/dt = 0, then the z history
 * of Eq. dzdt_guesses is back-filled with Taylor steps z - j dt/2 dz/dt, j = 1, 2, 3 (the paper
 * leaves start-up open). Nyquist slots and the k = 0 slot of Omega2 and m2^d are zeroed.
 * Asynchronous on the context's stream, except that with a history blob its substage counter is read
 * to the host in stream order (the stream is synchronised once).
 * Errors: INVALID_ARG (NULL ctx or state pointer, negative counter), CUDA. */
int lmvd_set_state(lmvd_ctx* ctx, const void* z_hat, const void* omega2_hat, const void* m2d_hat,
                   const double* mean_m1, const double* mean_m3, const void* history);

/* Copy the state out (same layouts as lmvd_set_state). Any pointer may be NULL to skip it.
 * history, if not NULL, receives lmvd_history_bytes() bytes: int64 substage counter, 8 bytes
 * padding, then z^{s-1}, z^{s-2}, z^{s-3}, (dz/dt)^{s-1}, RHS_Omega2^{s-1} (ny rows),
 * RHS_phi2^{s-1} (ny + 1 rows) as spectral arrays, then RHS_<m1>^{s-1}, RHS_<m3>^{s-1} (ny doubles
 * each). The RHS arrays hold values at collocation points. Asynchronous. Errors: INVALID_ARG, CUDA. */
int lmvd_get_state(lmvd_ctx* ctx, void* z_hat, void* omega2_hat, void* m2d_hat, double* mean_m1,
                   double* mean_m3, void* history);

/* Bytes of the history blob. 0 if ctx is NULL. */
size_t lmvd_history_bytes(const lmvd_ctx* ctx);

/* One substage s -> s + 1 of Algorithm 2 (steps 1-6): stage n for even s, stage ' (t_{n+1/2})
 * for odd s. Asynchronous; enqueues kernels only. Errors: INVALID_ARG, CUDA. */
int lmvd_advance_substage(lmvd_ctx* ctx);

/* nsteps RK2 steps = 2 * nsteps substages. Errors as lmvd_advance_substage. */
int lmvd_step(lmvd_ctx* ctx, int nsteps);

/* CUDA graphs for lmvd_advance_substage / lmvd_step (no paper counterpart: launch overhead of this
 * implementation). When on (the default), a substage is captured into a CUDA graph the first time its
 * launch pattern occurs and replayed afterwards; the pattern is the stage (n or '), the diagnostics flag
 * and which internal buffer holds which state and history field, so a run meets 10 patterns (the
 * z history cycles through five buffers, the other fields through two). Results are those of the
 * eager launches (same kernels, same arguments, same order). Substages run eagerly while per-launch
 * profiling is on, inside the adjoint's recording, on the legacy default stream (ctx created with a
 * NULL stream), while the caller is capturing the stream (the launches then go into the caller's
 * graph), or after a capture was refused. Off: eager launches, the graphs are released.
 * Errors: INVALID_ARG (NULL). */
int lmvd_graphs_enable(lmvd_ctx* ctx, int on);

/* Number of substage graphs the context holds (-1 if ctx is NULL). */
int lmvd_graph_count(const lmvd_ctx* ctx);

/* Intermediate fields of the last substage, for testing and diagnostics (B coefficients unless
 * stated): which = LMVD_FIELD_*. out: caller-owned host or device buffer of lmvd_field_bytes().
 * Errors: INVALID_ARG (unknown field, NULL), CUDA. */
#define LMVD_FIELD_RZ 0        /* R_z (Sec. 2.1)                                  ny rows   */
#define LMVD_FIELD_ZDOT 1      /* (dz/dt)^{s,k_f}                                 ny rows   */
#define LMVD_FIELD_RHO_T 2     /* f'(z) (dz/dt)^{s,k_f}                           ny rows   */
#define LMVD_FIELD_MC1 3       /* m1^c                                            ny rows   */
#define LMVD_FIELD_MC2 4       /* m2^c (order p + 1 space)                        ny+1 rows */
#define LMVD_FIELD_MC3 5       /* m3^c                                            ny rows   */
#define LMVD_FIELD_R_OMEGA2 6  /* RHS_Omega2 at the order-p Greville points       ny rows   */
#define LMVD_FIELD_R_PHI2 7    /* RHS_phi2 at the order-(p+1) Greville points     ny+1 rows */
#define LMVD_FIELD_R_MEANS 8   /* RHS_<m1>, RHS_<m3> at the Greville points: 2*ny doubles   */
int lmvd_get_field(lmvd_ctx* ctx, int which, void* out);
size_t lmvd_field_bytes(const lmvd_ctx* ctx, int which);

/* Fourier synthesis / analysis with the 3/2 rule (Eq. disc_f; Sec. 4.4: nonlinear terms are formed
 * on the physical grid), always in FP64, on the context's grid and stream, using its workspace.
 * spec: nfields consecutive spectral arrays [ny][nz][nx/2+1] complex128 holding values at the ny
 *       collocation points (not B-spline coefficients); Nyquist slots are ignored on input and
 *       written as zero on output.
 * phys: nfields consecutive physical arrays [ny][3nz/2][3nx/2] float64 on the padded grid
 *       x_i = i lx / (3nx/2), z_k = k lz / (3nz/2).
 * lmvd_inverse_transform: phys(x, z) = sum over retained (kx, kz) of spec exp(i (kx x + kz z)),
 *   the kx < 0 half by Hermitian symmetry (the kx = 0 column is taken as Hermitian).
 * lmvd_forward_transform: spec = retained coefficients of phys, scaled by 1 / ((3nx/2)(3nz/2)).
 * Both pointers must be device memory owned by the caller; spec of the inverse transform 16-byte aligned
 * (it is read by TMA tile copies; every complex128 element boundary is). Asynchronous.
 * Errors: INVALID_ARG (NULL pointer, nfields < 0, spec of the inverse not 16-byte aligned), CUDA. */
int lmvd_inverse_transform(lmvd_ctx* ctx, const void* spec, double* phys, int nfields);
int lmvd_forward_transform(lmvd_ctx* ctx, const double* phys, void* spec, int nfields);

/* Allocation-free inverse transform (the paper has no counterpart: this serves callers that may not
 * allocate device memory at all -- code running under an allocator owned by another framework, or
 * after a start-up phase that forbids new allocations -- and therefore cannot create a context).
 * Computes the same FP64 synthesis as lmvd_inverse_transform (same layouts) for an nx x ny x nz grid,
 * on cuda_stream (NULL = legacy default stream) of the current device, without any cudaMalloc: its
 * working memory is one static 32 MiB device array that every device loading the library holds until
 * the process exits. Its twiddle factors are computed on the device (sincospi) where a context rounds
 * long-double host values, so the two agree to rounding (relative max difference <= 1e-13 in the
 * tests), not bit for bit. Limits: the twiddle tables plus ny * (3nz/2) * (nx/2) * 16 bytes must fit in
 * the 32 MiB (e.g. 128 x 129 x 128 fits; 256 x 257 x 256 does not), and ny <= 65535 (one grid row of
 * CTAs per y-plane).
 * spec, phys: caller-owned device memory. The first call on a device sets itself up (looks up the
 * array's device address, raises the kernels' shared-memory limit); make that first call before any
 * stream capture. All calls on a device share the array and leave their contents in it; calls whose
 * GPU work overlaps (different streams or host threads) race, so order them on one stream.
 * Launch errors: a launch error left pending on the calling host thread by earlier, unrelated work is
 * cleared on entry (after the argument checks) and not reported; each of this call's launches is then
 * checked, and the first failure returns CUDA without launching the rest.
 * Errors: INVALID_ARG (NULL pointer, spec not 16-byte aligned, odd or too small nx/nz, ny < 1 or
 * ny > 65535, nfields < 0, grid too large for the static array), UNSUPPORTED (3nx/2 or 3nz/2 with prime factors other than 2 and 3, or
 * above the limits of lmvd_create), CUDA. */
int lmvd_inverse_transform_noalloc(int nx, int ny, int nz, const void* spec, double* phys, int nfields,
                                   void* cuda_stream);

/* Self-test of the precision path's conversions (precision = 1; no paper counterpart). The spectral
 * ends of its transforms split each FP64 value into a double-float pair and round pairs back, with
 * integer operations only; this runs the same device code on caller arrays:
 *   (hi[i], lo[i]) = split of x[i]: hi the top 24 significand bits of x (truncated), lo the rest rounded
 *     to a float, renormalised (|lo| <= ulp(hi) / 2, |hi + lo - x| <= 2^-48 |x| for |x| >= 2^-102;
 *     smaller magnitudes lose lo gradually and become signed zeros below 2^-126; |x| >= 2^128 gives a
 *     signed infinity, nan a nan);
 *   sum[i] = pair_hi[i] + pair_lo[i] rounded to a double (exact when representable; otherwise the
 *     bits of pair_lo below the double's last place rounded to nearest); inf and nan keep their value.
 * All arrays are caller-owned device memory of n entries; asynchronous on cuda_stream.
 * Errors: INVALID_ARG (NULL pointer with n > 0), CUDA. */
int lmvd_df64_convert(const double* x, float* hi, float* lo, const float* pair_hi, const float* pair_lo,
                      double* sum, size_t n, void* cuda_stream);

/* Adjoint of one substage (the differentiation path; the paper's method is differentiated, the paper
 * itself has no adjoint). Let x = (state, history) be the context's current state and history and
 * y = (state', history') what lmvd_advance_substage would produce from it. Given ybar, this computes
 * xbar = J(x)^T ybar, with the inner products sum Re(conj(a) b) over every stored complex entry and
 * sum a b over the real arrays. Every linear step is transposed exactly (transposed banded evaluations
 * and band solves, transforms G^T = (px pz) W F and F^T = G W^{-1} / (px pz) with W = 1 at kx = 0 and 2
 * at kx > 0); the products of Sec. 2.1, 4.3 and Eq. om / phi are differentiated at the fields of a
 * forward substage that this call runs first, so the context advances by one substage as a side effect.
 * state blobs (lmvd_state_bytes): z_hat | omega2_hat | m2d_hat | mean_m1 | mean_m3, packed in this order
 * in the layouts of lmvd_set_state; history blobs: as lmvd_get_state (the leading counter is ignored on
 * input and set to the substage index on output). Pointers: host or device memory, caller-owned.
 * Synchronous. Allocates the adjoint workspace on its first call (tape of the physical fields plus the
 * adjoint fields, about 45 spectral and 44 physical fields).
 * Errors: INVALID_ARG (NULL), UNSUPPORTED (precision 1 or kf > 15), OOM, CUDA. */
size_t lmvd_state_bytes(const lmvd_ctx* ctx);
int lmvd_adjoint_substage(lmvd_ctx* ctx, const void* state_bar_out, const void* history_bar_out,
                          void* state_bar_in, void* history_bar_in);

/* Adjoint of the start-up that lmvd_set_state runs when it is given no history (reading of the paper's
 * open start-up: n_startup applications of the fixed point from dz/dt = 0, then the history
 * z - j dt/2 dz/dt, j = 1, 2, 3, dz/dt_prev = dz/dt, RHS_prev = 0). Let x be the context's current state
 * (z, Omega2, m2^d, means; its history is not read) and y = (x, history) what lmvd_set_state(x, NULL)
 * produces. Given ybar (a state blob and a history blob, as for lmvd_adjoint_substage; the RHS_prev part
 * of the history blob is ignored because the start-up sets it to zero), this writes xbar = J(x)^T ybar
 * into state_bar_in (a state blob), with the inner products of lmvd_adjoint_substage. The call re-runs the
 * start-up from x, keeping dz/dt before each application (n_startup spectral fields, allocated on the
 * first call and kept), then differentiates each application from its stored iterate; afterwards the
 * context holds x with the start-up history, as after lmvd_set_state(x, NULL). Pointers: host or device
 * memory, caller-owned. Synchronous.
 * Errors: INVALID_ARG (NULL), UNSUPPORTED (precision 1 or kf > 15), OOM, CUDA. */
int lmvd_adjoint_startup(lmvd_ctx* ctx, const void* state_bar_out, const void* history_bar_out,
                         void* state_bar_in);

/* Device memory (bytes) the context holds: its workspace (state, history, work fields, transform
 * intermediate), the y-operators and their factors (the per-mode factors of the m^c and m2^d systems are
 * stored for the kz >= 0 half-plane: they depend on kz^2 only), the transform tables, and the adjoint
 * workspace once an adjoint call has allocated it. 0 if ctx is NULL. (No paper counterpart: the HBM footprint of this implementation.) */
size_t lmvd_device_bytes(const lmvd_ctx* ctx);

/* Substage counter s (0 after a start-up). -1 if ctx is NULL. */
int lmvd_substage_index(const lmvd_ctx* ctx);

/* Block until all work of the context's stream is done; returns the latched status or CUDA.
 * Failure detection: every substage checks its new state on the device (inf or nan anywhere in z,
 * Omega2, m2^d or the means sets a device status word, no host synchronisation); this call reads that
 * word and latches LMVD_ERR_NONFINITE if it is set. The z-passes of the transforms wait at most ~1 s for
 * their tile copies (TMA); a copy that did not complete sets another bit of the word, which this call
 * latches as LMVD_ERR_CUDA (the results of that transform are not valid). */
int lmvd_synchronize(lmvd_ctx* ctx);

/* First error latched in the context (LMVD_OK if none; a non-finite state is latched by the next
 * lmvd_synchronize). */
int lmvd_status(const lmvd_ctx* ctx);

/* Diagnostics of the fixed-point iteration and of mass conservation (observability; the paper discusses
 * convergence of the iteration in Sec. 3.1-3.2, Eq. y_k_delta, and instability when its iteration matrix
 * has spectral radius >= 1). When enabled, each substage records on the device, without host
 * synchronisation: the relative mass residual |rho_t + i k1 m1^c + i k3 m3^c + D* m2^c| / |rho_t| of its
 * final m^c (B-coefficient space, all modes) and, for each of its k_f fixed-point applications, the
 * relative change |dz/dt^{k+1} - dz/dt^k| / |dz/dt^{k+1}| (2-norms over all stored entries). If the last
 * change is >= 1/2, the iteration did not converge: a device status bit is set and the next
 * lmvd_synchronize latches LMVD_ERR_FP_DIVERGED. Enabling allocates a small record on the first call;
 * the cost is one extra copy and read of dz/dt per application. Off by default.
 * Errors: INVALID_ARG (NULL), OOM. */
int lmvd_diagnostics_enable(lmvd_ctx* ctx, int on);

/* Copies the record of the last substage (synchronous): out[0] = its substage index, out[1] = relative
 * mass residual, out[2 + k] = relative change of application k + 1 (k < k_f), then
 *   out[2 + k_f] = kinetic energy (1/2) integral of |m|^2 / rho dV of m = m^d + m^c at the substage's start
 *     (the state's m^d and the substage's final m^c; x-z means on the padded grid, the y-integral of the
 *     interpolant through the Greville values, times lx lz),
 *   out[3 + k_f] = max over the padded grid of |m| (same m),
 *   out[4 + k_f] = <m2^c> at y0 (the bottom value of the plane-mean curl-free momentum; Eq. mc_mean fixes
 *     it to zero at y1, so this is the net mass flux the mean density change implies, Sec. 4.2).
 * Writes min(n, 5 + k_f) values and returns 5 + k_f (the number available). The values are sums of
 * atomics, not bitwise reproducible. Errors: INVALID_ARG (NULL, n < 0, diagnostics never enabled), CUDA. */
int lmvd_diagnostics(lmvd_ctx* ctx, double* out, int n);

/* Kernel accounting (no paper counterpart: observability of this implementation).
 * Every kernel the context enqueues belongs to one of LMVD_KERNEL_CLASSES classes
 * (lmvd_kernel_class_name: fft_z_inverse, fft_x_inverse, fft_x_forward, fft_z_forward, eval_pass1,
 * eval, solve_collocation, solve_mc, rhs_combine, rhs_eval, rk_update, products, misc).
 * lmvd_profile_enable(ctx, on): synchronizes the stream, resets the per-class counters and, when on
 *   is non-zero, brackets every later launch with CUDA events recorded on the context's stream.
 * lmvd_profile_read(ctx, cls, out4): synchronizes the stream and writes, for class cls since the
 *   last enable: out4[0] total kernel milliseconds (CUDA events; 0 when profiling is off),
 *   out4[1] launches, out4[2] algorithmic flops, out4[3] algorithmic DRAM bytes (the minimum
 *   traffic of each launch: its inputs read once and its outputs written once).
 * lmvd_kernel_launches(ctx): kernels enqueued since lmvd_create, those of replayed graphs included
 *   (-1 if ctx is NULL).
 * Errors: INVALID_ARG (NULL ctx or out4, cls out of range), CUDA. */
#define LMVD_KERNEL_CLASSES 13
int lmvd_profile_enable(lmvd_ctx* ctx, int on);
int lmvd_profile_read(lmvd_ctx* ctx, int cls, double* out4);
const char* lmvd_kernel_class_name(int cls);
long long lmvd_kernel_launches(const lmvd_ctx* ctx);

/* Static description of an error code. */
const char* lmvd_strerror(int code);

/* Issue rate of one arithmetic operation on the current device (no paper counterpart: it measures the
 * denominators of the roofline fractions). op: 0 = FP64 FMA, 1 = FP64 add, 2 = FP64 multiply, 3 = FP32
 * FMA. Runs 8 independent chains per thread, 8 CTAs of 256 threads per SM, iters iterations, after one
 * shorter warm-up launch, on cuda_stream (NULL = legacy default stream), and writes the operations per
 * second (CUDA-event time) to *ops_per_second. Synchronous; allocates and frees a small output array.
 * Errors: INVALID_ARG (NULL output, iters < 1, op outside 0..3), OOM, CUDA. */
int lmvd_rate_probe(int op, int iters, double* ops_per_second, void* cuda_stream);

/* The bounded wait of the transforms' tile copies, on its own (no paper counterpart: it tests the failure
 * path of lmvd_synchronize's tile-copy bit without a fault). One CTA copies 128 bytes from src (device,
 * 16-byte aligned, at least 16 doubles) into shared memory while its mbarrier expects 128 + extra_bytes;
 * extra_bytes = 0 completes (and the copy is checked: bit 3 of *status if it differs), extra_bytes > 0
 * (a multiple of 16, at most 1024) never completes, and the CTA gives up after ~1 s of SM clock and sets
 * bit 2 of *status (device word, caller-owned, not cleared). Asynchronous on cuda_stream (NULL = legacy
 * default stream). Errors: INVALID_ARG (NULL or unaligned pointer, extra_bytes out of range), CUDA. */
int lmvd_tile_wait_probe(const double* src, int extra_bytes, unsigned* status, void* cuda_stream);

/* 1 if this library was built with the kernels' index checks (-DLMVD_CHECK, liblmvd_check.so), else 0
 * (no paper counterpart: the checked build is a testing aid). In the checked build every checked access
 * first tests its index against the extent of its array; a failed test skips the access and sets a
 * device word that lmvd_synchronize turns into LMVD_ERR_OUT_OF_BOUNDS. The checks never trap. */
int lmvd_checked_build(void);

#ifdef __cplusplus
}
#endif
#endif
