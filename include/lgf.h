/*
 * lgf.h -- C ABI of the GB300 (sm_103a) library for Landau gauge fixing of 4D
 * SU(3) lattice gauge fields by Fourier-accelerated steepest descent.
 *
 * Method (Cardoso, Silva, Oliveira, Bicudo, arXiv:1301.3460): Landau gauge is
 * the maximum over gauge transformations g of the functional (introduction)
 *     F_U[g] = 1/(N_d N_c V) sum_x sum_mu Re Tr[g(x) U_mu(x) g^dag(x+mu)],
 * reached by steepest descent with Fourier acceleration (introduction); the
 * paper's runs use alpha = 0.08 and stop at theta < 1e-15 (description of the
 * 32^4 comparison) and keep links as 12 reals (description of the GPU set-up).
 * One iteration on the current links U:
 *     M(x)     = sum_mu [U_mu(x-mu) - U_mu(x)]
 *     Delta(x) = (M - M^dag) - Tr(M - M^dag)/3
 *     theta    = 1/(N_c V) sum_x Tr[Delta Delta^dag],   F = F_U[1]
 *     stop if theta < tol (the test is made before an update)
 *     Delta~   = IFFT[ p2max/p2(k) FFT[Delta](k) ] / V,  k = 0 removed,
 *                p2(k) = sum_mu 4 sin^2(pi k_mu/L_mu)
 *     g(x)     = reunit(1 + alpha/2 Delta~(x))   (row Gram-Schmidt onto SU(3))
 *     U_mu(x) <- g(x) U_mu(x) g^dag(x+mu),  G(x) <- g(x) G(x)
 *
 * Conventions
 *   - Every function returns an lgf_status; none throws or aborts.
 *   - Lattice extents dims[4] = {Lx, Ly, Lz, Lt}; site s = x + Lx*(y + Ly*(z + Lz*t)).
 *   - Link arrays are complex128 [4][V][3][3] (mu, site, row, column), real and
 *     imaginary parts interleaved, row-major: 18 doubles per link.  Gauge
 *     transformations are [V][3][3] complex128.
 *   - Pointers are owned by the caller; the library copies in and out.  A flag
 *     on_device = 1 means the pointer is device memory of the current CUDA
 *     device, 0 means host memory (pinned or pageable).
 *   - The context owns all of its device memory and runs its work on the stream
 *     given by lgf_set_stream (default: the legacy default stream).  Calls on
 *     one context must not overlap; separate contexts are independent.
 *   - No CPU fallback exists: without a usable CUDA device lgf_create fails
 *     with LGF_ERR_CUDA.
 */
#ifndef LGF_H
#define LGF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lgf_ctx lgf_ctx;

typedef enum {
    LGF_OK = 0,
    LGF_ERR_ARG = 1,              /* null pointer, bad parameter value */
    LGF_ERR_CUDA = 2,             /* a CUDA call failed (no device, out of memory, launch error) */
    LGF_ERR_NOT_SU3 = 3,          /* input links are not in SU(3) to 1e-12 */
    LGF_ERR_UNSUPPORTED_DIMS = 4, /* an extent or the plane sizes are outside what the FFT kernels take */
    LGF_ERR_NOT_CONVERGED = 5,    /* max_iter updates applied before theta < tol */
    LGF_ERR_NAN = 6,              /* theta or F became NaN or infinite */
    LGF_ERR_TIMEOUT = 7,          /* the device loop hit its safety bound on body executions, or a
                                     kernel gave up waiting (about a second) for its own tensor copies */
    LGF_ERR_STATE = 8             /* call out of order (e.g. lgf_fix before lgf_set_links) */
} lgf_status;

/* creation flags */
#define LGF_FP64 0        /* every step in FP64 */
#define LGF_MIXED 1       /* FP32 Delta/FFT/update until theta < switch_tol, then FP64 (see lgf_set_switch_tol) */
#define LGF_NO_GAUGE 2    /* do not accumulate G (lgf_get_gauge then fails); FP64 mode only */
#define LGF_LINKS18 8     /* keep row 2 of each FP64 link in memory (18 reals) instead of rebuilding it on
                             every load (12 reals): the same values (row 2 is stored as the rebuild from
                             rows 0,1), 50% more link bytes, fewer FP64 operations per update */
#define LGF_LINKS8 16     /* keep each FP64 link in its 8-real form (u01, u02, u10 and the phases of u00 and
                             u20; the rest rebuilt from unitarity and det = 1 on every load): a third of the
                             12-real bytes, two sqrt, two sincos and a division more per load, two atan2 per
                             store.  Singular where |u00| = 1 and accurate to ~1e-15/(|u01|^2 + |u02|^2) near
                             it: lgf_set_links also rejects links it cannot hold to 1e-10 (LGF_ERR_NOT_SU3),
                             and the configuration generator (unit links) is not available (LGF_ERR_STATE).
                             Exclusive with LGF_LINKS18 */
#define LGF_PLAIN_SD 4    /* steepest descent without Fourier acceleration: g = reunit(1 + alpha/2 Delta);
                             the method whose critical slowing down the introduction cites (alpha < 0.125
                             for stability with this Delta normalisation) */

/*
 * lgf_create: allocate a context for a lattice of extents dims[4].
 * Each extent must be one of 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, and the
 * shared-memory FFT tiles (the four fields of one xy-plane with rows padded to
 * Lx + 1, and one z,t pencil one x-column wide with rows padded to Lz + 1 plus
 * its multipliers) must fit in 220 KiB in FP64: Ly*(Lx + 1) <= 3520 and
 * Lt*(3 Lz + 2) <= 28160 (e.g. 64x48, 96x32 or 128x24 planes, 96x96, 64x128 or
 * 128x64 pencils); and 24 V must fit a signed 32-bit offset (V <= 89,478,485
 * sites, e.g. 96^4); else LGF_ERR_UNSUPPORTED_DIMS.  Extents are checked before
 * any CUDA call.  flags: LGF_FP64 or
 * LGF_MIXED, optionally | LGF_NO_GAUGE, | LGF_PLAIN_SD, | LGF_LINKS18 or | LGF_LINKS8.  *out receives the
 * context.
 */
int lgf_create(const int dims[4], int flags, lgf_ctx** out);

/* Run all later work of ctx on this cudaStream_t (NULL = legacy default stream). */
int lgf_set_stream(lgf_ctx* ctx, void* cuda_stream);

/*
 * lgf_set_links: copy links U ([4][V][3][3] complex128, layout above) into the
 * context, keeping rows 0,1 of each link (row 2 is rebuilt as conj(row0 x row1),
 * the 12-real form).  Checks every link: max|U U^dag - 1| and |det U - 1| must
 * be below 1e-12, else LGF_ERR_NOT_SU3 (the context keeps no links then).
 * Resets the accumulated gauge transformation G to 1.
 */
int lgf_set_links(lgf_ctx* ctx, const double* U, int on_device);

/*
 * lgf_fix: iterate Fourier-accelerated steepest descent on the stored links
 * until theta < theta_tol (tested on the current links before each update) or
 * max_iter updates are applied.  alpha > 0 is the step (0.08 in the paper).
 * Outputs (each may be NULL): *iters = updates applied, *F and *theta of the
 * final links.  They are valid also when the call returns LGF_ERR_NOT_CONVERGED
 * or LGF_ERR_NAN.  In LGF_MIXED mode the FP32 phase runs while theta >=
 * switch_tol and FP32 keeps improving theta (lgf_set_switch_tol), its links
 * rebuilt from the input every few updates (lgf_set_fp32_refresh); then G is
 * reprojected onto SU(3) in FP64 and the links are rebuilt as
 * U = G U_in G^dag(x+mu) in FP64 before the FP64 phase.  Blocks until done.
 */
int lgf_fix(lgf_ctx* ctx, double alpha, double theta_tol, int max_iter, int* iters, double* F, double* theta);

/* lgf_get_links: write the current links as full matrices (row 2 rebuilt as
 * conj(row0 x row1) for the 12-real form, the whole matrix for the 8-real form). */
int lgf_get_links(lgf_ctx* ctx, double* U_out, int on_device);

/*
 * lgf_get_gauge: write the accumulated gauge transformation G ([V][3][3]
 * complex128), so that the current links equal G(x) U_in(x) G^dag(x+mu) up to
 * rounding.  LGF_ERR_STATE if the context was created with LGF_NO_GAUGE.
 */
int lgf_get_gauge(lgf_ctx* ctx, double* G_out, int on_device);

/*
 * lgf_get_history: copy (theta_n, F_n) of the last lgf_fix, n = 0..iters, as
 * 2*n doubles into theta_F (host memory), at most n_max pairs; *written gets the
 * number of pairs.  The device keeps the most recent 65536 pairs.
 */
int lgf_get_history(lgf_ctx* ctx, double* theta_F, int n_max, int* written);

/*
 * Snapshots of the stored links in the context's own layout (no conversion, no
 * check), for callers that return to earlier states many times, such as the
 * checkpointed derivative through K steps (the paper has no counterpart).
 * lgf_links_state_bytes: size of a snapshot.  lgf_save_links: copy the stored
 * links to dst (device memory of that size).  lgf_load_links: store a snapshot
 * that lgf_save_links wrote from a context of the same extents and flags, and
 * reset G to 1.  Both block until the copy is done.
 */
size_t lgf_links_state_bytes(const lgf_ctx* ctx);
int lgf_save_links(lgf_ctx* ctx, void* dst);
int lgf_load_links(lgf_ctx* ctx, const void* src);

/* lgf_stats: phase split of the last lgf_fix (iterations in the FP32 phase). */
int lgf_get_stats(lgf_ctx* ctx, int* iters_fp32, int* iters_fp64);

/*
 * lgf_set_loop_bound (fault injection for tests): cap each device-side loop of
 * later lgf_fix calls at max_body_runs executions of its body.  A loop ended by
 * the cap before its stop condition makes lgf_fix return LGF_ERR_TIMEOUT, the
 * status the safety bound (max_iter + 2 body runs) would give.  0 removes the
 * cap (the default).
 */
int lgf_set_loop_bound(lgf_ctx* ctx, int max_body_runs);

/*
 * Threshold on theta that ends the FP32 phase of LGF_MIXED (default 1e-6).
 * The FP32 phase also ends when FP32 arithmetic stops improving theta: 50
 * iterations without a new smallest theta once theta < 1e-12 (FP32's floor is
 * near 1e-14 on the lattices measured), 2000 iterations above that.  FP32
 * iterations track FP64 ones down to theta ~1e-13, so switch_tol = 1e-13 leaves
 * the FP64 finish only the error of the re-projection to remove; switch_tol = 0
 * runs the FP32 phase down to its floor.
 */
int lgf_set_switch_tol(lgf_ctx* ctx, double switch_tol);

/*
 * LGF_MIXED: every `every` FP32 updates (default 25; 0 = never) G is
 * re-orthonormalised and the FP32 links are rebuilt from the input links as
 * G(x) U_in(x) G^dag(x+mu), so that FP32 rounding does not accumulate along a
 * long FP32 phase: the drift would otherwise be left for the FP64 finish.
 */
int lgf_set_fp32_refresh(lgf_ctx* ctx, int every);

/*
 * LGF_MIXED: the form of the FP32 phase's update.  form = 0: the update writes
 * each new link's packed anti-Hermitian part and Re Tr, and a separate kernel
 * forms Delta from them (the FP64 phase's form).  form = 2 (default): as 0, with
 * the g builder (inverse x,y transform and FP64 Gram-Schmidt) and the update in
 * one persistent launch whose blocks take xy-planes from a queue, each update
 * waiting (bounded, on per-plane flags) for the g of the planes it reads, so
 * that building g (FP64 pipe) and updating links (HBM) run side by side on the
 * device; its results are bit-identical to form 0.  form = 1: one kernel
 * updates the links and forms Delta, theta and F of the new links, recomputing
 * the anti-Hermitian part of each link that enters a site from its neighbour's
 * old link (the links alternate between two FP32 buffers); it agrees with forms
 * 0 and 2 to FP32 rounding.  The setting only changes the kernels' work.  Other
 * values: LGF_ERR_ARG; form 2 outside a mixed context: LGF_ERR_STATE.
 */
int lgf_set_fp32_update(lgf_ctx* ctx, int form);

/*
 * LGF_MIXED: precision of the accelerator (forward 4D FFT of Delta, the
 * multiplier p2max/(p2(k) V), inverse FFT; the introduction's Fourier
 * acceleration) in the FP64 iterations.  64 (default): every step of an FP64
 * iteration in FP64.  32: Delta, theta, F, the Gram-Schmidt of g and the update
 * stay in FP64 (the fix still stops on the FP64 theta < theta_tol and keeps the
 * links on the input's gauge orbit in FP64), while Delta is rounded to FP32 for
 * the transforms, which run in the FP32 phase's kernels.  The accelerator only
 * preconditions the step: Delta~ = 0 exactly when Delta = 0, so its rounding
 * changes how fast theta falls (relative error ~1e-7 per mode), not where the
 * iteration stops.  With switch_tol above the first theta the FP32 phase is
 * empty and the whole fix runs in FP64 with the FP32 accelerator.  Needs a
 * mixed context without LGF_PLAIN_SD (LGF_ERR_STATE otherwise); other values:
 * LGF_ERR_ARG.  lgf_batch_set_accel_precision sets every lattice of a batch.
 */
int lgf_set_accel_precision(lgf_ctx* ctx, int precision);

/*
 * Stage entry points (same arithmetic as inside lgf_fix, exposed for checking
 * each step on its own).  All arrays are caller-owned, layouts as above.
 *
 * lgf_delta: Delta ([V][3][3] complex128, may be NULL), theta and F of the
 *   stored links, in FP64.
 * lgf_accelerate: Delta~ = IFFT[p2max/p2 FFT[Delta]]/V of a given traceless
 *   anti-Hermitian field Delta ([V][3][3]); Dt_out gets the full matrices.
 * lgf_build_g: g = reunit(1 + alpha/2 Dt) of a given Dt ([V][3][3]).
 */
int lgf_delta(lgf_ctx* ctx, double* Delta_out, int on_device, double* theta, double* F);
int lgf_accelerate(lgf_ctx* ctx, const double* Delta_in, double* Dt_out, int on_device);
int lgf_build_g(lgf_ctx* ctx, const double* Dt_in, double alpha, double* g_out, int on_device);

/*
 * The same three stages as the FP32 phase of LGF_MIXED computes them (its own
 * kernels; inputs and outputs in FP64, layouts as above), for checking that
 * phase stage by stage against the FP64 results to FP32 accuracy.  Need a
 * context created with LGF_MIXED, else LGF_ERR_STATE.
 *
 * lgf_delta32: the stored links rounded to FP32, then Delta (forward x,y
 *   transform and back, as the phase transforms it) with theta and F reduced in
 *   FP64.  Needs lgf_set_links first (LGF_ERR_STATE).  Overwrites the context's
 *   FP32 links, which lgf_fix rebuilds from the FP64 links on every call.
 * lgf_accelerate32: Delta~ of a given Delta with the FP32 transforms and FP32
 *   multipliers p2max/(p2 V).
 * lgf_build_g32: g = reunit(1 + alpha/2 Dt): the field rounded to FP32 and taken
 *   through the phase's forward and inverse x,y transforms, the Gram-Schmidt in
 *   FP64, g rounded to FP32 (row 2 rebuilt in FP32 from the rounded rows).
 */
int lgf_delta32(lgf_ctx* ctx, double* Delta_out, int on_device, double* theta, double* F);
int lgf_accelerate32(lgf_ctx* ctx, const double* Delta_in, double* Dt_out, int on_device);
int lgf_build_g32(lgf_ctx* ctx, const double* Dt_in, double alpha, double* g_out, int on_device);

/*
 * lgf_time_kernels (instrumentation): run n_iter iterations of the loop body on
 * the stored links, launching the kernels one by one on the context's stream
 * with CUDA events around each launch, and write to ms[4] the median over the
 * iterations of the duration (milliseconds) of (0) the Delta + x,y FFT kernel, (1) the z,t FFT +
 * accelerator kernel, (2) the inverse x,y FFT + g kernel, (3) the update
 * kernel.  precision 64 times the FP64 kernels; 32 the FP32 kernels of the
 * form lgf_set_fp32_update chose (mixed contexts only; they start from an FP32
 * copy of the stored links; with the fused update, (0) is the x,y FFT alone and
 * (3) the update fused with Delta).  The stored links advance by n_iter updates
 * (precision 64) or are left as they were (32).
 */
int lgf_time_kernels(lgf_ctx* ctx, double alpha, int n_iter, int precision, double* ms);

/*
 * lgf_autotune: choose the launch shapes of the shared-memory FFT kernels (block
 * sizes of the plane and pencil kernels, x-columns per z,t pencil and the z,t
 * kernel's form, see lgf_set_shape) for this lattice by
 * timing the candidates on the stored links; both precisions of a mixed
 * context.  The choice is cached for the process by extents and precision.
 * Needs lgf_set_links first (LGF_ERR_STATE otherwise).  Changes no result
 * beyond rounding.
 */
int lgf_autotune(lgf_ctx* ctx);

/*
 * lgf_set_shape / lgf_get_shape (instrumentation, no counterpart in the paper):
 * the launch shape of the FFT kernels of one precision (64: the FP64 kernels;
 * 32: the FP32 phase's, mixed contexts only, LGF_ERR_STATE otherwise).
 *   nt_xy, nt_zt  threads per block of the xy-plane kernels and of the z,t kernel
 *                 (multiples of 32; at most 128 in FP64, 256 in FP32)
 *   xw            x-columns per z,t pencil (a power of two dividing Lx)
 *   zt_form       0: the pencil-tiled z,t kernel (one block per pencil);
 *                 1: the persistent z,t kernel whose pencils are staged by tensor
 *                 copies (TMA) into two shared-memory buffers guarded by
 *                 mbarriers (FP32: xw >= 2; its grid fills the device)
 * lgf_set_shape returns LGF_ERR_ARG for a shape the kernels cannot run
 * (including a form-1 shape whose buffers exceed shared memory); it waits for the
 * context's stream and replaces the captured loop.  lgf_autotune overwrites it.
 * lgf_get_shape writes {nt_xy, nt_zt, xw, zt_form, grid of form 1} to shape_out[5].
 * Every shape gives the same results up to rounding.
 */
int lgf_set_shape(lgf_ctx* ctx, int precision, int nt_xy, int nt_zt, int xw, int zt_form);
int lgf_get_shape(lgf_ctx* ctx, int precision, int* shape_out);

/*
 * lgf_probe_fma (instrumentation, no counterpart in the paper): the FMA rate of
 * the current GPU in FP64 (precision 64) or FP32 (32), from one launch of 16
 * independent FMA chains of n_iter steps per thread over 8 blocks of 256 threads
 * per SM, timed with CUDA events after a short warm-up launch; *gflops counts
 * an FMA as two flops, *ms (may be NULL) is the launch time.  The FP64 rate is
 * the arithmetic ceiling of the FP64 iteration kernels.  Allocates a small
 * output buffer; blocks until done.
 */
int lgf_probe_fma(int precision, int n_iter, double* gflops, double* ms);

/*
 * lgf_check_conversions (instrumentation, no counterpart in the paper): the
 * integer-pipe conversions the FP32 phase's g builder uses, applied elementwise
 * on the device: f_out[i] = d_in[i] rounded to binary32 (to nearest, ties to
 * even), d_out[i] = f_in[i] widened to binary64 (exact).  All four are device
 * pointers to n elements, owned by the caller; the results must equal the
 * hardware conversions bit for bit.  n = 0 does nothing; n < 0 or a NULL pointer
 * with n > 0 gives LGF_ERR_ARG.  Blocks until done.
 */
int lgf_check_conversions(const double* d_in, float* f_out, const float* f_in, double* d_out, int n);

/*
 * Batched ensembles (no counterpart in the paper's single-lattice runs): n
 * lattices of possibly different extents, fixed together by one CUDA graph
 * launch in which every lattice's device-resident loop is an independent branch,
 * so lattices of uneven size and uneven convergence run concurrently and each
 * retires when it meets its stop condition.
 *
 * lgf_batch_create: dims = [n][4] extents (each as for lgf_create), flags as for
 *   lgf_create (LGF_MIXED recommended).  Allocates every lattice's state.
 * lgf_batch_set_links: links of lattice i (layout and checks as lgf_set_links).
 * lgf_batch_fix: the first call autotunes the FFT shapes of each distinct
 *   extent; then one graph launch runs all lattices to theta < theta_tol or
 *   max_iter.  Per-lattice outputs (arrays of n, each may be NULL): iters, F,
 *   theta, status (an lgf_status), t_retire_ms = time from the start of the
 *   launch to the lattice's retirement, measured on the GPU clock.  Returns
 *   LGF_OK if every lattice converged, else the first non-OK status.
 * lgf_batch_get_links / _get_gauge / _get_stats: as the single-lattice calls.
 */
typedef struct lgf_batch lgf_batch;
int lgf_batch_create(int n, const int* dims, int flags, lgf_batch** out);
int lgf_batch_set_stream(lgf_batch* b, void* cuda_stream);
int lgf_batch_set_switch_tol(lgf_batch* b, double switch_tol);  /* every lattice, as lgf_set_switch_tol */
int lgf_batch_set_accel_precision(lgf_batch* b, int precision);  /* every lattice, as lgf_set_accel_precision */
int lgf_batch_set_fp32_update(lgf_batch* b, int form);  /* every lattice, as lgf_set_fp32_update */
int lgf_batch_set_links(lgf_batch* b, int i, const double* U, int on_device);
int lgf_batch_fix(lgf_batch* b, double alpha, double theta_tol, int max_iter, int* iters, double* F, double* theta,
                  int* status, double* t_retire_ms);
int lgf_batch_get_links(lgf_batch* b, int i, double* U_out, int on_device);
int lgf_batch_get_gauge(lgf_batch* b, int i, double* G_out, int on_device);
int lgf_batch_get_stats(lgf_batch* b, int i, int* iters_fp32, int* iters_fp64);
void lgf_batch_destroy(lgf_batch* b);

/*
 * Derivatives (no counterpart in the paper, which only fixes the gauge): the
 * vector-Jacobian products of one Fourier-accelerated step and of the gluon
 * propagator at the smallest momenta, FP64, for differentiating gauge-fixed
 * observables with respect to the input links.  Gradients of a real loss L
 * follow G = dL/dRe U + i dL/dIm U, i.e. dL = Re sum conj(G) dU.  Arrays are
 * device pointers, complex128 [4][V][3][3] like the links.
 *
 * lgf_step_fwd: one Fourier-accelerated step: U_out = the links after one
 *   update of U_in (checked and stored as lgf_set_links does); the stored links
 *   are then U_out and G holds g of the step.
 * lgf_step_bwd: the stored links are the step's input U (rows 0,1 used, row 2
 *   rebuilt); gU_out is the cotangent of the step's output U' (all three rows,
 *   row 2 taken as its rebuild from rows 0,1); gU_in receives the cotangent of
 *   U (row 2 zero: the step does not read it).  alpha as in lgf_fix.
 * lgf_gluon_pmin: D = mean over the four momenta with one k_mu = 1 of
 *   D(p) = 2/((N_c^2-1)(N_d-1)V) sum_mu Tr[A~_mu(p) A~_mu(p)^dag],
 *   A_mu = (U - U^dag)/(2i) - trace/3, of the stored links; Dp[4] (may be NULL)
 *   gets the four values.
 * lgf_gluon_pmin_bwd: gU = gD * dD/dU of the stored links (row 2 zero).
 */
int lgf_step_fwd(lgf_ctx* ctx, double alpha, const double* U_in, double* U_out);
int lgf_step_bwd(lgf_ctx* ctx, double alpha, const double* gU_out, double* gU_in);
int lgf_gluon_pmin(lgf_ctx* ctx, double* D, double* Dp);
int lgf_gluon_pmin_bwd(lgf_ctx* ctx, double gD, double* gU);

/*
 * lgf_accelerate_noalloc: lgf_accelerate without a context, for callers that
 * cannot let a library allocate device memory (they have handed the GPU's
 * memory to an allocator of their own, such as a framework's caching pool or a
 * runtime's fixed arena).  The paper has no counterpart: this is an interface
 * variant, not a step of the method.
 *   dims      lattice extents as for lgf_create; additionally V <= 65536 sites
 *             (e.g. 16^4) and planes that fit the shared-memory tiles, else
 *             LGF_ERR_UNSUPPORTED_DIMS (use lgf_create + lgf_accelerate instead)
 *   Delta_in  device pointer, [V][3][3] complex128, traceless anti-Hermitian
 *   Dt_out    device pointer, [V][3][3] complex128, receives the result
 *   cuda_stream  the cudaStream_t to run on (NULL = legacy default stream)
 * The call allocates nothing: its scratch is a file-scope device array of about
 * 5 MiB that every GPU loading the library holds until the process exits.  Each
 * call looks up the array's device address on the current device; the first
 * call on a device (and the first after the array has moved, e.g. after
 * cudaDeviceReset) also sets kernel attributes.  All calls share the array and
 * it keeps the last call's
 * contents (what must start at zero is cleared on every call); calls whose work
 * overlaps on the GPU race on it.  Returns after the stream has finished.
 */
int lgf_accelerate_noalloc(const int dims[4], const double* Delta_in, double* Dt_out, void* cuda_stream);

/*
 * One lattice over several ranks (FP64): the counterpart of the paper's MPI
 * code, whose 4D FFT is distributed by transposes (description of the CPU
 * implementation).  Rank `rank` of `nranks` holds the t-slab t in [rank nt,
 * (rank+1) nt), nt = Lt/nranks, every array in the library's site order of an
 * Lx x Ly x Lz x nt lattice.  The library computes; the caller moves data between
 * ranks (NCCL, or copies between slabs of one process), through device buffers
 * of the slab (lgf_slab_buffer, all complex128):
 *   LGF_SLAB_A, LGF_SLAB_B  the four packed fields of the slab (4 V_slab
 *       values each) in all-to-all order: A is [j][4][nt][nz][Lx Ly], block j =
 *       the z-range [j nz, (j+1) nz) of this slab (nz = Lz/nranks); B is
 *       [i][4][nt][nz][Lx Ly], block i = rank i's t-range of this rank's z-range.
 *   LGF_SLAB_AH_SEND/RECV  [4][Lz Lx Ly]: the packed anti-Hermitian parts of the
 *       t-links of a slab's last plane, which enter the next slab's first plane.
 *   LGF_SLAB_G_SEND/RECV   [9][Lz Lx Ly]: g on a slab's first plane, which is
 *       g(x + t) of the previous slab's last plane.
 * One iteration, on every rank in this order (each call on the slab's stream):
 *   lgf_slab_pack_halo(AH_SEND); send it to rank+1's AH_RECV;
 *   lgf_slab_delta -> this slab's theta and F (normalised by the slab's sites;
 *     the lattice's are their means over ranks); stop here if theta < tol;
 *   all-to-all A -> B (block j of A to rank j, into block `rank` of its B);
 *   lgf_slab_accelerate; all-to-all B -> A (block i of B to rank i);
 *   lgf_slab_build_g(alpha); lgf_slab_pack_halo(G_SEND); send it to rank-1's G_RECV;
 *   lgf_slab_update.
 * Extents as for lgf_create, Lt and Lz multiples of nranks
 * (LGF_ERR_UNSUPPORTED_DIMS otherwise).  Links in and out are device pointers
 * to [4][V_slab][3][3] complex128 (the slab's sites), G to [V_slab][3][3];
 * lgf_slab_set_links checks SU(3) as lgf_set_links does and sets G = 1.
 * lgf_slab_delta blocks until its theta and F are known; the other calls return
 * with their work queued.  Calls before lgf_slab_set_links: LGF_ERR_STATE.
 */
typedef struct lgf_slab lgf_slab;
#define LGF_SLAB_A 0
#define LGF_SLAB_B 1
#define LGF_SLAB_AH_SEND 2
#define LGF_SLAB_AH_RECV 3
#define LGF_SLAB_G_SEND 4
#define LGF_SLAB_G_RECV 5
int lgf_slab_create(const int dims[4], int nranks, int rank, lgf_slab** out);
void lgf_slab_destroy(lgf_slab* slab);
int lgf_slab_set_stream(lgf_slab* slab, void* cuda_stream);
int lgf_slab_set_links(lgf_slab* slab, const double* U);
int lgf_slab_get_links(lgf_slab* slab, double* U_out);
int lgf_slab_get_gauge(lgf_slab* slab, double* G_out);
int lgf_slab_buffer(lgf_slab* slab, int which, void** ptr, size_t* bytes);
int lgf_slab_pack_halo(lgf_slab* slab, int which);
int lgf_slab_delta(lgf_slab* slab, double* theta, double* F);
int lgf_slab_accelerate(lgf_slab* slab);
int lgf_slab_build_g(lgf_slab* slab, double alpha);
int lgf_slab_update(lgf_slab* slab);

/*
 * Configurations to fix, made on the device (the paper fixes Wilson-action
 * configurations and does not say how it made them).  These calls change the
 * links stored in ctx in place, in FP64, and reset G to 1.
 *
 * lgf_set_unit_links: U_mu(x) = 1 (a cold start).
 * lgf_wilson_sweeps: n_heatbath times, one heat-bath sweep at coupling beta >= 0
 *   for the action beta sum_P (1 - Re Tr U_P / 3) followed by n_overrelax
 *   overrelaxation sweeps.  A sweep updates every link once: mu = 0..3, for
 *   each the sites with x+y+z+t even, then odd (links of one such class share
 *   no plaquette and are updated at once), each link through the SU(2)
 *   subgroups (0,1), (0,2), (1,2) in turn (heat bath: Kennedy-Pendleton for
 *   b = 2 beta k/3 >= 1.6, Creutz's method below; overrelaxation: the reflection
 *   that keeps the local action) and then reunitarised.  Heat-bath sweep i takes
 *   its random numbers from Philox4x32-10 with key = seed and sweep counter
 *   first_sweep + i (counter (mu V + s, sweep, 1024 subgroup + draw, 0)), so the
 *   result does not depend on the launch shape, and splitting a run into calls
 *   at any heat-bath sweep gives the same links.  n_heatbath = 0 runs
 *   n_overrelax overrelaxation sweeps alone.  Needs stored links
 *   (LGF_ERR_STATE); every extent must be even (LGF_ERR_UNSUPPORTED_DIMS).
 *   Blocks until done.
 * lgf_plaquette: *P = mean over all plaquettes of Re Tr U_P / 3 of the stored
 *   links, FP64, summed in a fixed order (the same value on every call).
 */
int lgf_set_unit_links(lgf_ctx* ctx);
int lgf_wilson_sweeps(lgf_ctx* ctx, double beta, unsigned long long seed, int first_sweep, int n_heatbath,
                      int n_overrelax);
int lgf_plaquette(lgf_ctx* ctx, double* P);

/*
 * lgf_set_generator_precision: 64 (default) or 32.  With 32 the staples, W, the
 * SU(2) draws and the rotation of each link in lgf_wilson_sweeps are FP32
 * (the links and their staples read from an FP32 copy of the links that the
 * sweeps keep current, uniforms from the top 24 bits of the same Philox words);
 * the links stay FP64 in memory, rows 0,1 of each re-orthonormalised in FP64
 * after its update.  A chain of its own, with the Wilson action's equilibrium up
 * to FP32 rounding, about 15x faster on GB300, where FP64 arithmetic runs at 1/64
 * of the FP32 rate (32^4: 1.30 against 19.6 ms per heat-bath sweep; the copy
 * takes 4 V x 48 bytes of device memory); the FP64 generator is the one that
 * matches the reference to rounding.
 */
int lgf_set_generator_precision(lgf_ctx* ctx, int bits);

/* Release all device memory of ctx.  NULL is a no-op. */
void lgf_destroy(lgf_ctx* ctx);

/* Static description of a status code. */
const char* lgf_strerror(int status);

/* Text of the last failed CUDA call on this thread (empty if none). */
const char* lgf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LGF_H */
