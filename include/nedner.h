/*
 * nedner.h -- C-ABI of the GB300 NEDNER-NUFFT reconstruction library.
 *
 * Schmid et al., "Non-Equispaced Grid Sampling in Photoacoustics with a
 * Non-Uniform FFT", arXiv:1510.01078.
 *
 * The library reconstructs the initial pressure p0(x, y, z) from pressure
 * time series recorded at M non-equispaced positions (x_m, y_m) of the plane
 * z = 0 through the discretised Fourier inversion formula (Sec. 2, Eq. exact
 * and Eq. disc_rec), evaluated with the three-step NEDNER algorithm of Sec. 3:
 *   (a) a 2-D NED-NUFFT over the sensor positions (Sec. 3.2, Eq. NED_NUFFT),
 *   (b) a 1-D NER-NUFFT at the non-equispaced temporal frequencies
 *       nu = sign(l) c Nt dt |k| (Sec. 3.1, Eq. NER_NUFFT),
 *   (c) the Jacobian factor 2 l / kappa of Eq. exact,
 *   (d) a uniform inverse 3-D FFT (Sec. 3, step 3).
 * Every stage runs in hand-written CUDA kernels for sm_103a, in FP32.
 *
 * Conventions shared by every entry point
 *   - Output grid: nx x ny x nz voxels of size dx x dy x dz; voxel (qx,qy,qz)
 *     is at x = (qx - nx/2) dx, y = (qy - ny/2) dy, z = qz dz.  X = nx dx,
 *     Y = ny dy, Z = nz dz.
 *   - The reconstruction R computes
 *       G[j,n]  = sum_m w_m g[m,n] exp(-2 pi i (jx x_m/X + jy y_m/Y))
 *       F[j,l]  = W s sum_n G[j,n] exp(-2 pi i nu[j,l] n / Nt)
 *       p0[q]   = Re (1/(nx ny nz)) sum_{j,l} F[j,l] exp(2 pi i (jx (qx-nx/2)/nx
 *                                     + jy (qy-ny/2)/ny + l qz/nz))
 *     over jx in {-nx/2..nx/2-1}, jy in {-ny/2..ny/2-1}, l in {-nz/2..nz/2-1},
 *     with w_m = h_m/(dx dy), W = 2|l/Z|/|k| (W(0,0) = 2, W(j!=0,0) = 0),
 *     s = c dt / dz.  With apply_weights = 0, w_m = 1 and W s = 1.
 *   - Array layouts (row-major, last index fastest):
 *       sensor_xy  host double [M][2]   positions in metres
 *       g          device float [M][Nt] time series, t_n = n dt, n fastest
 *       p0         device float [nz][ny][nx]
 *       dL_dxy     device float [M][2]
 *   - All device buffers belong to the caller; the plan owns its tables and
 *     its workspace.  Calls are asynchronous on the given CUDA stream
 *     (cudaStream_t passed as void*, NULL = legacy default stream); a status
 *     other than NEDNER_OK is returned synchronously for argument errors and
 *     launch failures.  There is no CPU fallback.
 *   - A plan may be used from one host thread at a time.
 */
#ifndef NEDNER_H_
#define NEDNER_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nedner_plan_s* nedner_plan_t;

typedef enum {
    NEDNER_OK = 0,
    NEDNER_EINVAL = 1,  /* bad argument: sizes not powers of two, NULL pointer, ... */
    NEDNER_ERANGE = 2,  /* a sensor outside the open aperture (-X/2, X/2) x (-Y/2, Y/2) */
    NEDNER_ENOMEM = 3,  /* host or device allocation failed, or workspace above the limit */
    NEDNER_ECUDA = 4,   /* a CUDA call failed (no device, launch error, ...) */
    NEDNER_ENAN = 5     /* non-finite values reached an output (see nedner_device_status) */
} nedner_status;

typedef struct {
    int nx, ny, nz;          /* voxels; each a power of two, 8 <= n <= 2048 */
    double dx, dy, dz;       /* voxel size (metres), > 0 */
} nedner_grid;

enum { NEDNER_WINDOW_KB = 0, NEDNER_WINDOW_GAUSS = 1 };

typedef struct {
    int kind;    /* NEDNER_WINDOW_KB (Kaiser-Bessel, Sec. 3.1) or NEDNER_WINDOW_GAUSS */
    int width;   /* taps per dimension, w = 2K of Eq. NER_NUFFT; even, 4 <= w <= 16 */
} nedner_window;

typedef struct {
    int apply_weights;            /* 1: h_m/(dx dy) and W s (the reconstruction R);
                                     0: both replaced by 1 */
    int band_mask;                /* 1: zero F where nu is outside [-Nt/2, Nt/2) */
    size_t max_workspace_bytes;   /* 0 = no limit; plan fails with ENOMEM above it.  Under a
                                     limit the transposed entry points work in shorter passes
                                     over the time samples where that lets the plan fit. */
    const double* sensor_w;       /* host [M] detector areas h_m (m^2), or NULL for X Y / M */
    int precision;                /* NEDNER_PRECISION_* (default FP32 NUFFT), see below */
    int ner_interp;               /* NEDNER_NER_* (default the NER-NUFFT), see below */
} nedner_opts;

/*
 * ner_interp selects how nedner_forward evaluates the non-equispaced range
 * sums F[j, l] = sum_n Ghat[j, n] exp(-2 pi i nu_l n / Nt) (stage b):
 *   NEDNER_NER_KB         the NER-NUFFT of Sec. 3.1 (centred, window
 *                         deconvolution, w-tap window interpolation on the
 *                         2 Nt grid);
 *   NEDNER_NER_LINEAR_S2  the comparison method of Sec. 5.1: each line
 *                         zero-padded at the end to 2 Nt, FFT'd, and the
 *                         spectrum interpolated linearly at 2 nu (FFT, c = 2);
 *   NEDNER_NER_LINEAR_S1  the same without padding (FFT, c = 1);
 *   NEDNER_NER_DIRECT     the direct sum over n (the "direct FT" of Sec. 5.1,
 *                         O(Nt) per value, FP32 with the phase re-anchored in
 *                         FP64 every 16 terms).
 * Plans with another value than NEDNER_NER_KB serve the comparison only: the
 * transposed entry points (nedner_adjoint, nedner_grad_positions) answer
 * NEDNER_EINVAL for them.
 */
enum { NEDNER_NER_KB = 0, NEDNER_NER_LINEAR_S2 = 1, NEDNER_NER_LINEAR_S1 = 2, NEDNER_NER_DIRECT = 3 };

/*
 * precision selects the arithmetic of stage (a) in nedner_forward,
 * nedner_forward_host and nedner_ned_stage (every other stage is FP32):
 *   NEDNER_PRECISION_FP32_NUFFT  the NED-NUFFT of Sec. 3.2 in FP32 (any sensor layout);
 *   NEDNER_PRECISION_BF16_GEMM   sensors on a tensor product x_m = xs[a], y_m = ys[b],
 *                                m = b * 128 + a, 128 x 128 of them, output grid
 *                                nx = ny = 256: the NED sum (Eq. NUDFT2 with a
 *                                separable exponent) evaluated exactly as two complex
 *                                GEMMs per time sample on the tensor cores, BF16
 *                                operands with a hi + lo split of every factor
 *                                (hi*hi + lo*hi + hi*lo) and FP32 accumulation;
 *   NEDNER_PRECISION_FP16_GEMM   the same GEMMs with FP16 hi + lo operands (11
 *                                significant bits per part), the data scaled by a
 *                                power of two on the device so that they fit FP16's
 *                                range (the scale is removed in FP32 afterwards).
 * The GEMM modes give NEDNER_EINVAL for other layouts.  The transposed entry
 * points (nedner_adjoint, nedner_grad_positions) always use the FP32 NUFFT.
 */
enum { NEDNER_PRECISION_FP32_NUFFT = 0, NEDNER_PRECISION_BF16_GEMM = 1, NEDNER_PRECISION_FP16_GEMM = 2 };

/*
 * Build a plan (host tables, device tables, device workspace).
 *   sensor_xy  host [M][2] metres, each strictly inside (-X/2, X/2) x (-Y/2, Y/2)
 *              (Sec. 2: x_m in (-X/2, X/2)^{d-1}), else NEDNER_ERANGE.  M >= 0.
 *   Nt, dt     number (power of two, 8 <= Nt <= 4096) and spacing (s) of time samples.
 *   c          sound speed (m/s), > 0.
 *   out_grid   output grid (see nedner_grid).
 *   window     interpolation window of both NUFFTs (Sec. 3.1-3.2).
 *   sigma      oversampling factor (the paper's c > 1); this build supports 2.0.
 *   opts       NULL for defaults {1, 0, 0, NULL, NEDNER_PRECISION_FP32_NUFFT, NEDNER_NER_KB}.
 *   stream     stream used for the table uploads (synchronised before return).
 *   out        receives the plan; untouched on error.
 * Returns NEDNER_OK, NEDNER_EINVAL, NEDNER_ERANGE, NEDNER_ENOMEM or NEDNER_ECUDA.
 */
nedner_status nedner_plan(const double* sensor_xy, int64_t M, int Nt, double dt, double c,
                          const nedner_grid* out_grid, nedner_window window, double sigma,
                          const nedner_opts* opts, void* stream, nedner_plan_t* out);

/*
 * Move the sensors (same M): rebuilds the per-sensor window taps and the
 * sensor-to-row tables (Sec. 3.2, the mu_{m,k} and Psi-hat of Eq. NED_NUFFT).
 * Areas h_m are kept.  Synchronous.  Same range rule as nedner_plan.
 */
nedner_status nedner_set_positions(nedner_plan_t plan, const double* sensor_xy);

/*
 * p0 = R g: the reconstruction of Eq. disc_rec by the NEDNER algorithm (Sec. 3).
 *   g   device float [M][Nt], read only, 16-byte aligned (NEDNER_EINVAL otherwise).
 *   p0  device float [nz][ny][nx], written (every element), 8-byte aligned.
 */
nedner_status nedner_forward(nedner_plan_t plan, const float* g, float* p0, void* stream);

/*
 * nedner_forward with host buffers: p0_host = R g_host, one call for the
 * upload of g, the reconstruction and the download of p0.  g is uploaded in
 * four contiguous parts (whole sensor rows) on four copy streams at once, and
 * p0 is downloaded in four blocks of depth planes, each as soon as the last
 * inverse FFT has written it.  Asynchronous with respect to the host on
 * `stream` (the stream's work completes when p0_host holds the result);
 * page-locked host memory is needed for the copies to run asynchronously.
 *   g_host   host float [M][Nt], read only;  p0_host  host float [nz][ny][nx], written.
 * The first call allocates the plan's device copies of g and p0 (M Nt + nx ny nz
 * floats), the copy streams and their events; later calls allocate nothing.
 */
nedner_status nedner_forward_host(nedner_plan_t plan, const float* g_host, float* p0_host, void* stream);

/*
 * g = R^T p0: the exact transpose of nedner_forward (same real-linear map,
 * transposed; spreading and interpolation of both NUFFTs swapped).
 *   p0  device float [nz][ny][nx], read only.
 *   g   device float [M][Nt], written.
 */
nedner_status nedner_adjoint(nedner_plan_t plan, const float* p0, float* g, void* stream);

/*
 * Sensor-position gradient of a loss L(p0) with p0 = R(x) g and h_m held fixed:
 *   dL_dxy[m][0] = dL/dx_m,  dL_dxy[m][1] = dL/dy_m   (units: 1/metre times L)
 * obtained by differentiating the NED exponent of Eq. disc_rec (derivative
 * window in the interpolation).
 *   g       device float [M][Nt], dL_dp0 device float [nz][ny][nx], read only.
 *   dL_dxy  device float [M][2], written.
 */
nedner_status nedner_grad_positions(nedner_plan_t plan, const float* g, const float* dL_dp0,
                                    float* dL_dxy, void* stream);

/*
 * Stage (a) alone, for inspection: the NED output G[j,n] (without the NER,
 * weight and inverse FFT) on the half lattice used internally,
 *   Ghat  device float2 [nx/2+1][ny+1][Nt],  Ghat[a][b][n] = G[(jx=a, jy=b-ny/2), n],
 * i.e. jx = 0..nx/2 and jy = -ny/2..ny/2 (both Nyquist rows included).
 * g as in nedner_forward; g and Ghat 16-byte aligned, else NEDNER_EINVAL.
 */
nedner_status nedner_ned_stage(nedner_plan_t plan, const float* g, void* Ghat, void* stream);

/*
 * nedner_forward with per-kernel timing, for measurement: records a CUDA event
 * around each of the forward kernels on `stream`, waits for the stream, and
 * writes each kernel's device time in milliseconds to stage_ms (host array of
 * NEDNER_FORWARD_KERNELS floats: NED spread, x-FFT, y-FFT, NER lines, y-IFFT,
 * x complex-to-real; where stage (a) runs per chunk of time samples its
 * three kernels' times are summed over the chunks; where the spread and
 * x-FFT are one kernel, or stage (a) is the tensor-core GEMMs, its time is the
 * first and the x-FFT's is 0).  Synchronous.  Same arguments and errors otherwise.
 */
#define NEDNER_FORWARD_KERNELS 6
nedner_status nedner_forward_profiled(nedner_plan_t plan, const float* g, float* p0, void* stream,
                                      float* stage_ms);

/*
 * nedner_adjoint and nedner_grad_positions with per-stage timing, for
 * measurement: CUDA events on `stream` between the launches; waits for the
 * stream and writes each stage's device time in milliseconds to stage_ms
 * (host array of NEDNER_TRANSPOSED_KERNELS floats): transposed x
 * complex-to-real, transposed y-IFFT, transposed NER, transposed y-FFT, the
 * transposed x-FFT and the transposed interpolation (gather; where the two
 * are one kernel its time is the gather's and the x-FFT's is 0), both summed
 * over their passes of time samples, and the per-sensor sum of the entries.
 * Synchronous.  Same arguments and errors as the unprofiled calls otherwise.
 */
#define NEDNER_TRANSPOSED_KERNELS 7
nedner_status nedner_adjoint_profiled(nedner_plan_t plan, const float* p0, float* g, void* stream,
                                      float* stage_ms);
nedner_status nedner_grad_positions_profiled(nedner_plan_t plan, const float* g, const float* dL_dp0,
                                             float* dL_dxy, void* stream, float* stage_ms);

/*
 * nedner_ned_stage without touching the plan's workspace and without any
 * device allocation: the same two kernels, with their intermediate array
 * ([nx/2+1][2 ny][Nt] complex64) in a fixed buffer of
 * NEDNER_STATIC_SCRATCH_BYTES that is part of the library's device image.
 * The paper has no counterpart to this entry point.
 *
 * Who needs it: callers that cannot call cudaMalloc at the moment they run
 * the stage -- code being recorded into a CUDA graph (allocation is not a
 * stream operation and breaks the capture), applications whose device memory
 * is handed out by their own pool or by another framework's allocator and is
 * exhausted by it, and pipelines that forbid allocation after start-up -- and
 * that want the NED stage of a plan whose own workspace is busy (for example
 * with nedner_forward on another stream).  The plan itself (tables) is built
 * beforehand and passed in; inputs and outputs are the caller's, as in
 * nedner_ned_stage.
 *
 *   Arguments: as nedner_ned_stage; g and Ghat 16-byte aligned, else
 *          NEDNER_EINVAL before anything is launched.  Plans built with the
 *          tensor-core precision modes are refused with NEDNER_EINVAL (their
 *          stage (a) needs the plan's own operand buffers; their geometry,
 *          128 x 128 sensors on a 256 x 256 grid, would not fit the limit).
 *   Limit: (nx/2+1) * 2 ny * Nt * 8 bytes must not exceed
 *          NEDNER_STATIC_SCRATCH_BYTES (16 MiB), else NEDNER_ENOMEM and
 *          nothing is launched.
 *   Memory: every GPU on which the library's device code is loaded holds the
 *          16 MiB buffer until the process exits.
 *   Set-up: the first call on a device looks up the buffer's device address
 *          (cudaGetSymbolAddress, with that device current) and caches it;
 *          make that first call before any stream capture.  Calls on a stream
 *          that is not being captured look the address up again, so after a
 *          cudaDeviceReset the next such call refreshes it; a call on a
 *          capturing stream with no cached address returns NEDNER_ECUDA.
 *   Sharing: all calls share the one buffer, which keeps the previous call's
 *          contents (the first kernel overwrites all of it before use, so no
 *          clearing is needed).  Calls that overlap on the GPU -- on several
 *          streams or from several host threads -- race and give wrong results.
 *   Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 */
#define NEDNER_STATIC_SCRATCH_BYTES (16u << 20)
nedner_status nedner_ned_stage_static(nedner_plan_t plan, const float* g, void* Ghat, void* stream);

/*
 * Device-side status of the plan's kernels since the previous call, read
 * back and cleared.  Waits for the device (synchronous).  *flags gets:
 *   NEDNER_STATUS_WAIT_TIMEOUT  a bounded wait of the tensor-core kernels
 *       (precision modes with GEMMs) ran out: those kernels bound every wait
 *       on an mbarrier (bulk copies, MMA completion), and when one runs out
 *       the kernel sets this flag and returns early, leaving its output
 *       incomplete, instead of hanging;
 *   NEDNER_STATUS_NONFINITE  an output kernel (the last stage of
 *       nedner_forward / nedner_forward_host, nedner_adjoint or
 *       nedner_grad_positions) wrote a NaN or an infinity.  Every input value
 *       reaches every output value through the transforms, so a non-finite
 *       value in g (or p0, dL_dp0) marks the whole result; so does overflow.
 * Returns NEDNER_ENAN when NEDNER_STATUS_NONFINITE is set, otherwise
 * NEDNER_OK; NEDNER_EINVAL for a null argument, NEDNER_ECUDA if the device
 * reports an error.  (Sec. 2 assumes finite data; the paper has no such check.)
 */
enum { NEDNER_STATUS_WAIT_TIMEOUT = 1, NEDNER_STATUS_NONFINITE = 2 };
nedner_status nedner_device_status(nedner_plan_t plan, int* flags);

/*
 * Test hook for the bounded waits of the tensor-core kernels: the pipeline
 * waits (operand ring, accumulator hand-over) give up after `polls` polls of
 * their mbarrier (0: at once) instead of the default 2^26; the waits that
 * drain a CTA's own copies and MMAs before it frees tensor memory keep the
 * default.  With a small limit a pipeline wait runs out, the kernels set
 * NEDNER_STATUS_WAIT_TIMEOUT and return with their output incomplete; pass
 * 1 << 26 to restore.  No effect on plans without the tensor-core stage.
 * Returns NEDNER_EINVAL for a null plan or negative polls.  No paper counterpart.
 */
nedner_status nedner_debug_set_wait_limit(nedner_plan_t plan, int polls);

/* Bytes of device workspace held by the plan. */
size_t nedner_workspace_bytes(nedner_plan_t plan);

/*
 * Data low-pass against spatial aliasing (Sec. 8): sensor m's time series
 * keeps the frequencies |f| <= f_cut,m = c / (2 dx_m), dx_m the distance
 * from sensor m to its nearest neighbour (the local sensor spacing; no
 * filtering for a lone sensor).  Ideal filter on the length-Nt DFT of each
 * series: bins k with |k| <= floor(f_cut,m Nt dt) are kept (the rest set to
 * zero), out = the inverse DFT.  The cut-off bins are computed on the host
 * from the plan's positions (nedner_plan, nedner_set_positions).
 *   g, out: device, M x Nt float32, sensor-major, t contiguous (caller
 *           owned; 4-byte aligned; out may equal g).
 * Returns NEDNER_EINVAL for a null plan or pointer or a misaligned buffer,
 * NEDNER_ECUDA on a launch failure.  Asynchronous on `stream`.
 */
nedner_status nedner_lowpass(nedner_plan_t plan, const float* g, float* out, void* stream);

/*
 * The low-pass's highest kept bin per sensor (host copy, M values written to
 * out while nout allows).  Returns 0, or -1 for a null plan (or a null out
 * with nout > 0).
 */
int nedner_lowpass_bins(nedner_plan_t plan, int* out, int64_t nout);

/*
 * Tenenbaum sharpness of B images (Appendix B): for image b (ny x nx, x
 * fastest) F[b] = (1 / (nx ny)) sum over the pixels whose 3 x 3
 * neighbourhood lies in the image of (S_x * U)^2 + (S_y * U)^2, S_x the
 * Sobel operator [-1 0 1; -2 0 2; -1 0 1] and S_y its transpose; summed in
 * FP64 in a fixed order (deterministic).
 *   U: device, B x ny x nx float32 (4-byte aligned); F: device, B doubles
 *   (8-byte aligned).  Caller owned.
 * Returns NEDNER_EINVAL for negative sizes, null or misaligned pointers.
 */
nedner_status nedner_tenenbaum(const float* U, int64_t B, int ny, int nx, double* F, void* stream);

/*
 * Maximum intensity projection of a volume (nz, ny, nx), x fastest, along
 * axis 0 (z: out is ny x nx), 1 (y: nz x nx) or 2 (x: nz x ny).  Device
 * float32 buffers, caller owned, 4-byte aligned.  Returns NEDNER_EINVAL for
 * non-positive sizes, a bad axis or null/misaligned pointers.
 */
nedner_status nedner_mip(const float* vol, int nz, int ny, int nx, int axis, float* out, void* stream);

/*
 * The two-dimensional variant (Sec. 7): sensors at x_m on the line z = 0,
 * an output image of nz x nx pixels (x fastest), the reconstruction
 *   p2[qz][qx] = Re (1/(nx nz)) sum_{jx, l} F[jx, l] exp(2 pi i (jx (qx - nx/2)/nx + l qz/nz)),
 *   F = W s sum_n G[jx, n] exp(-2 pi i nu n / Nt),  nu = sign(l) c Nt dt sqrt((jx/X)^2 + (l/Z)^2),
 *   G[jx, n] = sum_m (h_m / dx) g[m, n] exp(-2 pi i jx x_m / X),
 * i.e. Eq. disc_rec with one lateral axis (W, s and the readings as in the
 * 3-D plan).  The plan evaluates it on the 3-D path with every sensor at
 * y = 0 on a grid of 8 rows of dy = dx and sums the 3-D image over its rows
 * (exact: only the jy = 0 lines survive that sum); the adjoint copies the
 * image to every row and runs the 3-D adjoint.
 *   sensor_x   host [M] metres, strictly inside (-X/2, X/2), X = nx dx.
 *   opts       as for nedner_plan; sensor_w are lengths h_m (m), default X/M;
 *              precision must be NEDNER_PRECISION_FP32_NUFFT.
 *   g          device [M][Nt] f32 (16-byte aligned); p2 device [nz][nx] f32.
 * The plan owns a 3-D image buffer (nz x 8 x nx floats): calls on one plan
 * must not overlap.  Errors as for the 3-D entry points.
 */
typedef struct nedner2d_plan_s* nedner2d_plan_t;
nedner_status nedner2d_plan(const double* sensor_x, int64_t M, int Nt, double dt, double c, int nx, int nz,
                            double dx, double dz, nedner_window window, double sigma, const nedner_opts* opts,
                            void* stream, nedner2d_plan_t* out);
nedner_status nedner2d_set_positions(nedner2d_plan_t plan, const double* sensor_x);
nedner_status nedner2d_forward(nedner2d_plan_t plan, const float* g, float* p2, void* stream);
nedner_status nedner2d_adjoint(nedner2d_plan_t plan, const float* p2, float* g, void* stream);
nedner_status nedner2d_destroy(nedner2d_plan_t plan);

/*
 * The plan's passes over time, as chosen at nedner_plan for its geometry,
 * sensor count and workspace limit (host only, no device work).  Writes up
 * to nout values to out (host), in this order:
 *   [0] split:  1 if stage (a) runs as block spread + x-FFT + y-FFT kernels
 *               (and the transposed interpolation as transposed x-FFT +
 *               block gather), 0 for the fused spread and row gather;
 *   [1] tq:     time samples per chunk of the split stage (a);
 *   [2] tp_adj: time samples per pass of the adjoint's gather;
 *   [3] gsplit: 1 if the adjoint and gradient use the block gather;
 *   [4] tp_g:   time samples per pass of the gradient's block gather (0 if
 *               gsplit is 0: one pass over the whole record);
 *   [5] kernel launches of one nedner_forward, [6] of one nedner_adjoint,
 *       [7] of one nedner_grad_positions (this library's kernels only).
 * Returns the number of values available (8), or -1 for a null plan or out.
 * No paper counterpart.
 */
int nedner_plan_info(nedner_plan_t plan, int64_t* out, int nout);

/*
 * The work split a plan of this geometry uses (sigma = 2, window width w),
 * computed on the host without a device, so that the kernels' size
 * conditions can be checked for every geometry.  Writes up to nout values to
 * out, in this order: c1, c2f, c4, c5, groups1, threads1, per1, tpl1, ca,
 * per_adj, tpl_adj, threads_adj, lpc, threads3 (time samples, depth planes,
 * rows or lines per CTA, threads per CTA, values per thread and time samples
 * per lane of the stages), then the dynamic shared memory in bytes of the
 * spread, y-FFT, NER, y-IFFT, x complex-to-real and transposed gather
 * (adjoint, gradient) kernels; then split1 (1: stage (a) runs as block spread,
 * x-FFT and y-FFT per chunk of tq time samples), tq, the block spread's warps
 * per CTA, the x-FFT kernel's complex columns, threads and values per thread
 * per CTA, the shared memory of both, that of the transposed NER and the
 * depth frequencies of one line it holds at a time.
 * Returns the number of values (31), or -1 for
 * a geometry nedner_plan rejects or a null out.  No paper counterpart.
 */
int nedner_work_split(int nx, int ny, int nz, int Nt, int w, int64_t* out, int nout);

/* Free the plan (synchronises its device work first).  NULL is allowed. */
nedner_status nedner_destroy(nedner_plan_t plan);

/* Static string for a status code. */
const char* nedner_strerror(nedner_status status);

#ifdef __cplusplus
}
#endif

#endif /* NEDNER_H_ */
