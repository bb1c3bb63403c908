/*
 * ldbp.h -- C ABI of the GB300 (sm_103a) split-step / learned-DBP library.
 *
 * Method: Haeger & Pfister, "Physics-Based Deep Learning for Fiber-Optic
 * Communication Systems", arXiv:2010.14258.  Displayed equations are numbered
 * in order of appearance: Eq. (4) NLSE, (5) time-discretised NLSE,
 * (6) asymmetric split-step method (SSM), (7) parameterised model,
 * (8) symmetric SSM, (11) transmit signal, (12) receiver chain,
 * (14) effective SNR, (15) CD memory.
 *
 * Conventions shared by every entry point
 *  - Complex samples are interleaved complex64 (float re, float im), one
 *    waveform of n samples per row, rows contiguous: x[b * n + m].  Device
 *    pointers must be 8-byte aligned; 16-byte alignment enables the TMA
 *    bulk-copy path (otherwise plain loads are used).
 *  - Every waveform is periodic (circular): sample index m is taken mod n
 *    (Sec. IV-A: the symbol sequence is periodic; Sec. III-B: circular
 *    convolution).
 *  - The caller owns every device buffer and the stream.  `stream` is a
 *    cudaStream_t (NULL = legacy default stream).  All work is enqueued
 *    asynchronously on `stream`; nothing synchronises the device unless stated.
 *  - Return value: 0 on success, a negative LDBP_E* code otherwise; the
 *    message of the last failure on the calling thread is ldbp_last_error().
 *    No call aborts, throws or traps.  Errors detected on the device (a
 *    bounded wait that ran out) are reported by ldbp_device_status().
 *  - Gradients follow g = dl/dRe(z) + j dl/dIm(z) for a real loss l.
 */
#ifndef LDBP_H_
#define LDBP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LDBP_OK 0
#define LDBP_EINVAL (-1)      /* bad size, pointer, length or aliasing */
#define LDBP_ENOMEM (-2)      /* a library-owned table could not be allocated */
#define LDBP_ECUDA (-3)       /* a CUDA runtime call failed */
#define LDBP_ETIMEOUT (-4)    /* a bounded device wait ran out */
#define LDBP_EUNSUPPORTED (-5) /* valid request outside what this build supports */
#define LDBP_ENONFINITE (-6)  /* a NaN or infinite model / fiber parameter */

/* Largest number of LDBP steps per call and largest filter half-width K
 * (filter length T = 2K + 1 <= 33) of the fused LDBP kernels. */
#define LDBP_MAX_STEPS 64
#define LDBP_MAX_HALF_TAPS 16

/* Message of the last failed call on this thread ("" if none). */
const char* ldbp_last_error(void);

/* Library version (major * 10000 + minor * 100 + patch). */
int ldbp_version(void);

/* Reads and clears the device-side status word of the current device
 * (synchronises the device).  Returns LDBP_OK, LDBP_ETIMEOUT if a bounded
 * wait inside a kernel ran out since the last call, or LDBP_ECUDA. */
int ldbp_device_status(void);

/* ldbp_wait_probe -- exercises the bounded device wait of the library's
 * kernels (failure detection; the paper has no counterpart).  One block
 * initialises a shared-memory mbarrier that expects two arrivals, makes
 * `arrivals` of them (0, 1 or 2; no asynchronous copy is involved) and waits
 * for the phase with the same bounded wait the TMA and cluster-exchange
 * waits use, giving up after `limit` polls.  With fewer than two arrivals
 * the wait runs out: the kernel records LDBP_ETIMEOUT in the device status
 * word (read and cleared by ldbp_device_status) and returns; the context
 * stays usable.  Asynchronous on `stream`.
 * Errors: LDBP_EINVAL for arrivals outside 0..2 or limit outside
 * 1..2^20; LDBP_ECUDA if the launch fails. */
int ldbp_wait_probe(int32_t arrivals, int32_t limit, void* stream);

/*
 * ldbp_apply -- learned digital backpropagation, forward pass.
 *
 * Computes y = f_theta(x) of Eq. (7) with the symmetric-FIR linear steps of
 * Sec. III-B, for each of `batch` waveforms of n samples:
 *   u_0 = x;  for i = 0..M-1:
 *     v_m   = sum_{k=-K_i}^{K_i} h^(i)_|k| u_{(m-k) mod n}        (circular FIR)
 *     u_i+1 = v * exp(j c_i |v|^2)                                 (Kerr step)
 *   y = u_M.
 * All M steps run in one fused kernel: each thread block loads a time tile
 * plus the summed overlap-save halo H = sum_i K_i once (TMA bulk copy), keeps
 * it on chip for every step and writes its interior once.
 *
 *  taps   device, complex64 [M][taps_stride]: half-tap vector
 *         (h_0, h_1, ..., h_K) of step i at taps[i * taps_stride] (theta of
 *         Sec. III-B).  Entries beyond K_i are ignored.
 *  T      host, int32 [M]: filter length T_i = 2 K_i + 1 (odd, 1 <= T_i <= 33,
 *         T_i <= taps_stride * 2 - 1).  A pruned filter is passed with its
 *         current (shorter) length.
 *  c      host, float [M]: nonlinear coefficient of step i (c_i = -gamma
 *         L_eff(delta_i) for DBP; 0 makes a linear-only layer, Sec. III-C).
 *  M      number of steps, 1..LDBP_MAX_STEPS.
 *  x      device, complex64 [batch][n], read only.
 *  y      device, complex64 [batch][n]; must not overlap x.
 *  n      samples per waveform (>= 1); batch >= 1.
 *  ckpt   device, complex64 [M][batch][n], or NULL.  When given, ckpt[i]
 *         receives u_i (the input of step i); ldbp_backward consumes it.
 * Errors: LDBP_EINVAL for NULL x/y/taps/T/c, M out of range, an even or
 * out-of-range T_i, n < 1, batch < 1, overlapping x and y, or a halo sum too
 * large for one tile (2 H > 2048); LDBP_ENONFINITE for a NaN or infinite
 * c_i; LDBP_ECUDA if the launch fails.
 */
int ldbp_apply(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, int32_t M,
               const void* x, void* y, int64_t n, int32_t batch, void* ckpt, void* stream);

/*
 * ldbp_essm_apply -- learned enhanced SSM (filtered DBP, Sec. III-C,
 * Eqs. (9)-(10)): ldbp_apply whose nonlinear steps rotate by a filtered power,
 *   u_{i+1,j} = v_j exp(j c_i sum_{k=-kappa_i}^{kappa_i} eta^(i)_k |v_{j-k}|^2),
 *   v = A_i u_i (the symmetric circular FIR of ldbp_apply), indices mod n.
 * With kappa_i = 0 and eta^(i) = (1) this is ldbp_apply.
 *
 *  taps, taps_stride, T, c, M, x, y, n, batch   as for ldbp_apply, except
 *         T_i <= 2 * LDBP_ESSM_MAX_HALF_TAPS + 1.
 *  eta    device, float [M][eta_stride]: row i holds the real filter
 *         eta^(i)_{-kappa_i} .. eta^(i)_{kappa_i} (2 kappa_i + 1 values).
 *  kappa  host, int32 [M]: 0 <= kappa_i <= LDBP_ESSM_MAX_KAPPA.
 *  ckpt   device complex64 [M][batch][n] or NULL: receives u_i (the input of
 *         step i) for ldbp_essm_backward.
 * The tile halo is sum_i (K_i + kappa_i) per side.
 * Errors: LDBP_EINVAL (as ldbp_apply; kappa out of range; eta_stride too
 * small); LDBP_ENONFINITE for a NaN or infinite c_i; LDBP_ECUDA.
 */
#define LDBP_ESSM_MAX_KAPPA 24
#define LDBP_ESSM_MAX_HALF_TAPS 8
int ldbp_essm_apply(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, const float* eta,
                    int32_t eta_stride, const int32_t* kappa, int32_t M, const void* x, void* y, int64_t n,
                    int32_t batch, void* ckpt, void* stream);

/*
 * ldbp_essm_backward -- adjoint of ldbp_essm_apply.  Given g_y = dl/dRe(y) +
 * j dl/dIm(y), for i = M-1 .. 0 with v = A_i u_i, p = |v|^2,
 * phi = eta^(i) * p, w = v exp(j c_i phi) and g the gradient at w:
 *   a = -c_i Im(w conj(g)),  dl/dp_m = sum_k eta_k a_{m+k},
 *   g_v = exp(-j c_i phi) g + 2 (dl/dp) v,
 *   dl/deta^(i)_k = sum_{b,j} a_j p_{j-k},
 *   taps and g_u = A_i^H g_v as in ldbp_backward.
 *  ckpt   device complex64 [M][batch][n] from ldbp_essm_apply (ckpt != NULL)
 *  gtaps  device complex64 [M][taps_stride] (output); entries k > K_i are 0
 *  geta   device float [M][eta_stride] (output): dl/deta^(i)_k at
 *         index k + kappa_i; entries beyond 2 kappa_i are 0
 *  gx     device complex64 [batch][n] (output) or NULL
 *  workspace  >= ldbp_essm_backward_workspace() bytes, caller-owned
 * The per-block sums are reduced in a fixed order in FP64 (bitwise
 * reproducible).  Errors: as ldbp_essm_apply, plus LDBP_EINVAL for a short
 * workspace or gx aliasing gy / ckpt.
 */
int ldbp_essm_backward_workspace(int64_t n, int32_t batch, const int32_t* T, const int32_t* kappa, int32_t M,
                                 size_t* bytes);
int ldbp_essm_backward(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, const float* eta,
                       int32_t eta_stride, const int32_t* kappa, int32_t M, const void* ckpt, const void* gy,
                       void* gx, void* gtaps, float* geta, int64_t n, int32_t batch, void* workspace,
                       size_t workspace_bytes, void* stream);

/*
 * ldbp_apply_host -- ldbp_apply on waveforms in HOST memory (the receiver's
 * end-to-end call): the batch is cut into `chunks` groups of waveforms whose
 * host->device copy, LDBP pass (the computation of ldbp_apply, Eq. (7)) and
 * device->host copy overlap on library-owned streams (copy-in, two compute
 * streams, copy-out).  The call is
 * ordered after earlier work on `stream` and `stream` is made to wait for the
 * last copy; it returns after enqueueing (synchronise `stream` before reading
 * y_host).
 *
 *  taps, taps_stride, T, c, M, n, batch   as for ldbp_apply.
 *  x_host   host, complex64 [batch][n], read only.  Page-locked memory
 *           (cudaHostAlloc / cudaHostRegister) is needed for the copies to
 *           overlap; pageable memory works but serialises them.
 *  y_host   host, complex64 [batch][n]; must not overlap x_host.
 *  chunks   1..min(batch, 256); 12 is the fastest measured for 256 x 65536
 *           (copy-bound: 1.0 ms against 0.8 ms for the two copies alone).
 *  workspace  device, >= ldbp_apply_host_workspace(n, batch) bytes, 16-byte
 *           aligned, caller-owned: the device copies of x and y.
 * Errors: as ldbp_apply, plus LDBP_EINVAL for NULL host pointers, chunks out
 * of range or a short workspace; LDBP_ECUDA for a failed copy or launch.
 */
size_t ldbp_apply_host_workspace(int64_t n, int32_t batch);
int ldbp_apply_host(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, int32_t M,
                    const void* x_host, void* y_host, int64_t n, int32_t batch, int32_t chunks, void* workspace,
                    size_t workspace_bytes, void* stream);

/*
 * Ragged batches: many learned-DBP waveforms of different length n_w, step
 * count M_w and filter lengths in ONE persistent launch (the computation of
 * ldbp_apply per waveform).  Waveforms are packed back to back in x and y
 * (waveform w starts at sample offset sum_{v<w} n_v); the steps of all
 * waveforms are packed in taps [total_steps][taps_stride] (device), c
 * [total_steps] (device float) and T [total_steps] (host, at plan creation),
 * waveform w owning rows sum_{v<w} M_v .. + M_w - 1.
 *
 * ldbp_ragged_plan_create  builds the work list of (waveform, tile) items,
 *     longest first, in plan-owned device memory (allocates; synchronous).
 * ldbp_ragged_autotune     times candidate tile-length caps and blocks per SM
 *     on the given buffers (synchronous, writes y) and keeps the fastest.
 * ldbp_apply_ragged        resets the work counter and launches the
 *     persistent kernel on `stream`.  done_ns (device uint64 [count], zeroed
 *     by the caller) receives each waveform's completion time and start_ns
 *     (device uint64 [1], set to UINT64_MAX by the caller) the earliest block
 *     start, both from the GPU global timer; either may be NULL.
 * ldbp_ragged_graph_capture / _graph_launch  capture that launch (counter
 *     reset + kernel) for fixed buffers into a CUDA graph owned by the plan,
 *     and replay it on `stream`.
 * ldbp_ragged_info         total samples, total steps, work items, tile cap,
 *     blocks per SM of the plan.
 * ldbp_ragged_set_schedule pins the tile cap (even, 256..4096 output samples
 *     per tile) and the blocks per SM (1..the occupancy of the plan's
 *     K_max class), e.g. to replay a configuration the autotuner chose
 *     earlier; rebuilds the work list (allocates; synchronous) and drops a
 *     captured graph.
 * The plan is bound to the device current at creation.  Errors: LDBP_EINVAL
 * (NULL pointers, n < 1, M outside 1..LDBP_MAX_STEPS, T invalid, halo too
 * large, overlapping x / y, wrong device), LDBP_ECUDA.
 */
int ldbp_ragged_plan_create(void** plan, int32_t count, const int64_t* n, const int32_t* M, const int32_t* T,
                            int32_t taps_stride);
int ldbp_ragged_plan_destroy(void* plan);
int ldbp_ragged_info(const void* plan, int64_t* total_samples, int32_t* total_steps, int32_t* items,
                     int32_t* tile_cap, int32_t* blocks_per_sm);
int ldbp_ragged_autotune(void* plan, const void* taps, const float* c, const void* x, void* y, void* stream);
int ldbp_ragged_set_schedule(void* plan, int32_t tile_cap, int32_t blocks_per_sm);
int ldbp_apply_ragged(void* plan, const void* taps, const float* c, const void* x, void* y, uint64_t* done_ns,
                      uint64_t* start_ns, void* stream);
int ldbp_ragged_graph_capture(void* plan, const void* taps, const float* c, const void* x, void* y);
int ldbp_ragged_graph_launch(void* plan, void* stream);

/*
 * ldbp_backward -- adjoint of ldbp_apply (hand-written reverse sweep).
 *
 * Given g_y = dl/dRe(y) + j dl/dIm(y) of a real loss l at the output of
 * ldbp_apply, computes for i = M-1 .. 0 (Eq. (7) with the FIR of Sec. III-B):
 *   Kerr:  g_v = exp(-j c_i |v|^2) g_w - 2 c_i Im(w conj(g_w)) v,  v = A_i u_i, w = u_{i+1}
 *   taps:  dl/dh^(i)_0 = sum_{b,m} g_v conj(u_i[m]),
 *          dl/dh^(i)_k = sum_{b,m} g_v conj(u_i[m-k] + u_i[m+k])  (k = 1..K_i)
 *   FIR:   g_u = A_i^H g_v  (symmetric FIR with conjugated taps).
 * v is recomputed from the checkpoints u_i written by ldbp_apply (ckpt
 * != NULL there); the sweep is one fused kernel plus a deterministic
 * fixed-order reduction of the per-block tap sums (bitwise reproducible).
 *  taps, taps_stride, T, c, M  as in ldbp_apply (same values as the forward call)
 *  ckpt       device complex64 [M][batch][n] from ldbp_apply
 *  gy         device complex64 [batch][n]
 *  gx         device complex64 [batch][n] (output, dl/dx) or NULL
 *  gtaps      device complex64 [M][taps_stride] (output); entries k > K_i are 0
 *  workspace  device scratch of at least ldbp_backward_workspace() bytes,
 *             owned by the caller; its contents on entry are irrelevant
 * Errors: LDBP_EINVAL (as ldbp_apply; a too small workspace; gx aliasing gy
 * or ckpt; halo sum H + K_max too large for one tile), LDBP_ECUDA.
 */
int ldbp_backward(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, int32_t M,
                  const void* ckpt, const void* gy, void* gx, void* gtaps, int64_t n, int32_t batch, void* workspace,
                  size_t workspace_bytes, void* stream);

/*
 * ldbp_backward_c -- ldbp_backward that also returns the gradients of the
 * nonlinear coefficients (the learnable scaling of the nonlinear steps,
 * Remark 1: c_i = eta_i gamma L_eff(delta_i)):
 *   dl/dc_i = -sum_{b,m} |v_m|^2 Im(w_m conj(g_w,m)),   v = A_i u_i, w = u_{i+1}.
 *  gc   device float [M] (output), or NULL (then this is ldbp_backward).
 * Same workspace, ordering and errors as ldbp_backward; the sums are reduced
 * in the same fixed order (bitwise reproducible).
 */
int ldbp_backward_c(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, int32_t M,
                    const void* ckpt, const void* gy, void* gx, void* gtaps, float* gc, int64_t n, int32_t batch,
                    void* workspace, size_t workspace_bytes, void* stream);

/* Workspace bytes ldbp_backward needs for (n, batch, T[0..M)).  Host only. */
int ldbp_backward_workspace(int64_t n, int32_t batch, const int32_t* T, int32_t M, size_t* bytes);

/* Size of the device array ldbp_backward_static uses as scratch: 4 MiB. */
#define LDBP_STATIC_SCRATCH_BYTES ((size_t)4 << 20)

/*
 * ldbp_backward_static -- ldbp_backward without any device allocation.
 *
 * The paper has no counterpart: this entry point serves callers that cannot
 * call cudaMalloc, for example a host application that reserves all device
 * memory once at start-up, or a plug-in whose framework owns every device
 * allocation and forbids new ones while it runs.  It computes exactly what
 * ldbp_backward computes, with the same arguments minus the workspace: the
 * per-block tap sums go to a file-scope __device__ array of
 * LDBP_STATIC_SCRATCH_BYTES that is part of the library's device code, so
 * every GPU that loads the library holds those 4 MiB until the process exits.
 * The caller still provides ckpt, gy, gx and gtaps.
 *  - Problems whose workspace (ldbp_backward_workspace) exceeds
 *    LDBP_STATIC_SCRATCH_BYTES are rejected with LDBP_EINVAL and a message
 *    naming both sizes; nothing is launched.
 *  - The first call on a device looks up the array's device address with
 *    cudaGetSymbolAddress (with that device current) and caches it for the
 *    current CUDA context; make that first call before any stream capture.
 *    A device reset (cudaDeviceReset) destroys the context and the array may
 *    be loaded elsewhere in the next one: the next call sees the new context
 *    id and looks the address up again, so make it outside a capture too.
 *    No call allocates or frees memory.
 *  - Every call on a device shares the one array and it keeps the last call's
 *    contents; nothing in it needs clearing, because each call writes every
 *    element it later reads.  Calls whose executions overlap on the GPU (on
 *    different streams, or from several host threads) race on the array and
 *    must be serialised by the caller.
 * Errors: as ldbp_backward, plus LDBP_EUNSUPPORTED for a device index >= 64.
 */
int ldbp_backward_static(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, int32_t M,
                         const void* ckpt, const void* gy, void* gx, void* gtaps, int64_t n, int32_t batch,
                         void* stream);

/*
 * ldbp_adam_step -- one Adam update of the LDBP taps (Sec. IV-B; Table I:
 * learning rate 1e-3) with the pruning mask of Sec. IV-C.
 *
 * Treats taps [M][taps_stride] complex64 as real pairs and applies, per real
 * parameter, m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
 * theta <- theta - lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps).
 * Taps with k > K_i = (T_i - 1)/2 (pruned or unused) and their moments are
 * set to zero, so a filter shortened by the caller stays shortened.
 *  taps   device complex64 [M][taps_stride] (updated in place)
 *  gtaps  device complex64 [M][taps_stride] gradient (ldbp_backward)
 *  m, v   device float [M][taps_stride][2] moments (caller-owned, start at 0)
 *  T      host int32 [M] current filter lengths; step >= 1.
 * Errors: LDBP_EINVAL, LDBP_ECUDA.
 */
int ldbp_adam_step(void* taps, const void* gtaps, float* m, float* v, const int32_t* T, int32_t M,
                   int32_t taps_stride, int32_t step, float lr, float beta1, float beta2, float eps, void* stream);

/* Fiber parameters in the paper's units (Table I). */
typedef struct {
  double alpha_db_per_km;   /* power attenuation, dB/km (>= 0) */
  double beta2_ps2_per_km;  /* group-velocity dispersion, ps^2/km */
  double gamma_per_w_km;    /* Kerr nonlinearity, 1/(W km) */
} ldbp_fiber;

/* Link (Sec. IV-A): n_spans spans of span_km, each followed by an EDFA that
 * restores the launch power and (if ase != 0) adds white Gaussian ASE noise of
 * PSD (e^{alpha L_sp} - 1) h nu_s n_sp, n_sp = NF / (2 (1 - e^{-alpha L_sp})).
 * steps_per_span uniform split steps of delta = span_km / steps_per_span;
 * symmetric != 0 selects Eq. (8), otherwise Eq. (6).  The ASE realisation is
 * drawn by Philox4x32-10 with key (seed lo, seed hi) and counter words
 * (bin k / 2, waveform, span, counter lo) in the frequency domain. */
typedef struct {
  int32_t n_spans;
  double span_km;
  int32_t steps_per_span;
  int32_t symmetric;
  int32_t ase;
  double nf_db;
  double carrier_hz;
  uint64_t seed;
  uint64_t counter;
} ldbp_link;

/*
 * ssm_forward -- fiber channel by the split-step Fourier method.
 *
 * Propagates each waveform over the link: per span, steps_per_span steps of
 * the symmetric SSM (Eq. (8): A_{d/2} sigma_d A_{d/2}, with the Kerr rotation
 * x exp(j gamma l(d) |x|^2), l(d) = 2 sinh(alpha d / 2) / alpha, at the step
 * midpoint) or of the asymmetric SSM (Eq. (6), Kerr with L_eff(d) first, then
 * the lossy linear step A_d = e^{-alpha d/2} F^-1 diag(exp(j beta2/2 w_k^2 d)) F),
 * then the amplifier gain e^{alpha L_sp / 2} and the ASE noise.
 * omega_k = 2 pi fs kappa_k / n with kappa_k the fftfreq integers (Eq. (5)).
 *
 *  fiber, link   host structs (read during the call only).
 *  fs_hz         sampling rate of the waveform.
 *  x             device complex64 [batch][n] launch waveform in sqrt(W).
 *  y             device complex64 [batch][n]; may equal x (in place).
 *  n             a power of two in 512..131072, or three times a power of two
 *                in 1536..49152 (the 6 samples/symbol grids of the analog-rate
 *                simulation: clusters of 3, 6 or 12 blocks).
 * Execution: for most lengths and batches one kernel launch runs all steps,
 * each waveform held in the shared memory of a thread-block cluster.
 * Batches of 24 or more waveforms of n = 65536 and of 8 or more of n = 131072
 * run instead as two kernels per step (row and column transforms of the
 * n = N1 x 256 four-step split), in chunks of at most 64 MB of samples that
 * stay in the L2 cache across the steps.  Both give the same results to FP32
 * rounding.  The first call for a given (device, fiber, link, fs, n)
 * computes the FP64 spectral tables and uploads them into library-owned
 * device memory (cudaMalloc + synchronous copy), and the first run on the
 * two-kernel path adds transposed copies and twiddle tables; later calls
 * reuse them.
 * Errors: LDBP_EINVAL (NULL pointer, n not a supported length,
 * non-positive fs/span/steps/batch, negative alpha); LDBP_ENONFINITE (a NaN
 * or infinite fiber, link or fs value); LDBP_ECUDA.
 */
int ssm_forward(const ldbp_fiber* fiber, const ldbp_link* link, double fs_hz, const void* x, void* y, int64_t n,
                int32_t batch, void* stream);

/*
 * dbp_apply -- full-length frequency-domain digital backpropagation.
 *
 * Solves the propagation backwards (Sec. IV): spans in reverse order, the
 * amplifier gain undone, and steps_per_span steps of the SSM with
 * (beta2, gamma, alpha) -> (-beta2, -gamma, -alpha): symmetric != 0 gives
 * A^-1_{d/2} sigma_{-d} A^-1_{d/2} (the exact inverse of the symmetric
 * channel step), otherwise Eq. (6) order: linear step with full-length
 * dispersion filter, then Kerr rotation with -gamma L_eff(d).
 * link->ase, seed and counter are ignored.  Arguments and errors as
 * ssm_forward; y may equal x.
 */
int dbp_apply(const ldbp_fiber* fiber, const ldbp_link* link, double fs_hz, int32_t steps_per_span,
              int32_t symmetric, const void* x, void* y, int64_t n, int32_t batch, void* stream);

/*
 * ssm_cufft -- the same split-step programs as ssm_forward (dbp_steps_per_span
 * == 0) or dbp_apply (dbp_steps_per_span >= 1, dbp_symmetric) executed with
 * the cuFFT library: per step a batched C2C FFT, a spectral-multiply kernel,
 * an inverse FFT and a Kerr kernel.  Provided only as the library-FFT
 * comparison for the fused kernel; results agree with ssm_forward/dbp_apply
 * to FP32 rounding.  cuFFT allocates its own work area on the first call for
 * a given (stream, n, batch).  Arguments and errors as ssm_forward, except
 * that n may be any length in [2, 2^27] (e.g. the 6 samples/symbol grids of
 * the analog-rate simulation of Sec. IV-A, Table I).
 */
int ssm_cufft(const ldbp_fiber* fiber, const ldbp_link* link, double fs_hz, int32_t dbp_steps_per_span,
              int32_t dbp_symmetric, const void* x, void* y, int64_t n, int32_t batch, void* stream);

/*
 * ldbp_tx -- transmit waveform of Eq. (11), sampled at sps samples/symbol.
 *
 * x_b = sqrt(P_b sps) * iDFT( H_rrc . DFT(upsample(s_b)) ), with
 * H_rrc(f) = sqrt(sps RC(f / R_s)) the root-raised-cosine response of the
 * given roll-off (RC the raised-cosine spectrum) on the fftfreq grid; the
 * symbol sequence is periodic, so the waveform is circular.  For unit-energy
 * symbols the mean power is P_b.
 *  symbols  device complex64 [batch][nsym]
 *  power_w  device float [batch], launch power per waveform in W
 *  x        device complex64 [batch][nsym * sps] (output)
 * nsym * sps must be a power of two in [512, 131072]; 0 < rolloff <= 1.
 * Errors: LDBP_EINVAL, LDBP_ECUDA.
 */
int ldbp_tx(const void* symbols, const float* power_w, int32_t sps, double rolloff, void* x, int64_t nsym,
            int32_t batch, void* stream);

/*
 * ldbp_rx -- receiver chain of Eq. (12), loss and its gradient (Sec. IV-B).
 *
 * s_tilde_b = (M y_b) / sqrt(P_b sps): matched RRC filter (the ldbp_tx
 * response) and every sps-th sample from offset 0; phi_b = arg(s_b^H s_tilde_b)
 * (genie-aided phase correction); mse_b = ||s_tilde_b e^{-j phi_b} - s_b||^2 / nsym.
 * If grad != NULL it receives g = d l / d y with l = grad_scale / 2 * sum_b
 * ||s_hat_b - s_b||^2 (phi held constant, the matched filter being real and
 * even); grad_scale = 2 / (nsym * batch) gives the batch-mean MSE.
 *  y          device complex64 [batch][n], n = nsym * sps
 *  symbols    device complex64 [batch][nsym]
 *  power_w    device float [batch]
 *  stats      device double [batch][2] (output): mse_b and the mean |s_b|^2
 *  phi        device float [batch] (output)
 *  grad       device complex64 [batch][n] or NULL (output; may not alias y)
 *  workspace  device complex64 [batch][n] scratch owned by the caller
 * Errors: LDBP_EINVAL, LDBP_ECUDA.
 */
int ldbp_rx(const void* y, const void* symbols, const float* power_w, int32_t sps, double rolloff, int64_t nsym,
            int32_t batch, double* stats, float* phi, void* grad, float grad_scale, void* workspace, void* stream);

/*
 * ldbp_resample -- receiver front end of Sec. IV-A (Table I) and its inverse.
 *
 * The channel is simulated at rho_a samples/symbol (n_in = rho_a N_sym); the
 * received waveform passes an ideal brick-wall low-pass of total bandwidth
 * Delta B and is sampled at t = k / f_s (n_out = rho_d N_sym).  Both grids
 * span the same period N_sym / R_s, so DFT bin kappa (signed, fftfreq order)
 * is the same frequency on either, and
 *   y_b[m] = (1 / n_in) sum_{|kappa| < bandwidth n_c / 2} X_b[kappa] e^{j 2 pi kappa m / n_out},
 *   X_b = DFT(x_b) (unnormalised), n_c = min(n_in, n_out),
 * i.e. the low-passed waveform sampled at the output rate.  bandwidth is
 * Delta B relative to the coarser grid's sample rate; 1 is Table I's
 * Delta B = f_s.  The passband is open, so at bandwidth 1 the Nyquist bin is
 * rejected.  With n_out > n_in the same formula is band-limited interpolation
 * onto a finer grid (e.g. a DSP-rate transmit waveform onto the analog grid).
 *  x          device complex64 [batch][n_in], 16-byte aligned
 *  y          device complex64 [batch][n_out] (output), 16-byte aligned; it
 *             may equal x when n_in == n_out and must not overlap it otherwise
 *  n_in, n_out  one divides the other; the coarser one is a power of two in
 *             512..4096, the ratio r = n_fine / n_coarse is at most 8 and
 *             n_fine at most 16384 (e.g. 6144 -> 2048: 1024 symbols at
 *             rho_a = 6 and rho_d = 2, the paper's frame, Table I)
 *  bandwidth  in (0, 1]
 * One kernel launch, asynchronous on stream: a block per waveform reads it
 * once, runs r polyphase transforms of the coarse length (sampling down) or
 * r inverse ones (interpolation) in shared memory, and writes the output
 * once.  No workspace; the first call for a (device, n_coarse, r) uploads two
 * small constant tables (cudaMalloc + synchronous copy).
 * Errors: LDBP_EINVAL (NULL pointer, sizes, misalignment, overlap, bandwidth
 * out of range), LDBP_ENONFINITE (bandwidth NaN or infinite), LDBP_ECUDA.
 */
int ldbp_resample(const void* x, int64_t n_in, void* y, int64_t n_out, double bandwidth, int32_t batch,
                  void* stream);

/*
 * ldbp_ubench -- arithmetic ceilings of the current device (synchronous).
 *
 * Measures, on every SM, the throughput of one instruction class with eight
 * independent dependency chains per thread:
 *   kind 0: scalar FP32 fused multiply-add (lane operations/s),
 *   kind 1: packed FP32x2 fused multiply-add (lane FP32 operations/s, 2 per lane),
 *   kind 2: special-function sine (__sinf, operations/s),
 *   kind 3: packed and scalar FP32 FMA interleaved (lane FP32 operations/s).
 * These are the denominators the fused kernels' FP32 roofline is checked
 * against (the paper itself has no hardware figures).  Allocates a 1 KB
 * scratch buffer and synchronises the device.
 * Errors: LDBP_EINVAL for a NULL result pointer or an unknown kind; LDBP_ECUDA.
 */
int ldbp_ubench(int32_t kind, double* ops_per_second);

#ifdef __cplusplus
}
#endif

#endif /* LDBP_H_ */
