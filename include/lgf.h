/*
 * lgf -- Fourier-accelerated steepest-descent Landau gauge fixing of SU(3)
 * lattice gauge fields on one NVIDIA GB300 (sm_103a).
 *
 * Method: N. Cardoso, P. J. Silva, P. Bicudo, O. Oliveira, "Landau Gauge
 * Fixing on GPUs", arXiv:1206.0675.  Section 2 defines every quantity used
 * here: the gauge transformation (eq. 2), the functional F (eq. 3), the
 * Fourier-accelerated transform g(x) (Eq. (eq:gx)), the lattice divergence
 * Delta(x) and the stopping quantity theta; Algorithm 1 is the loop.
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice: extents[4] = {Lx, Ly, Lz, Lt}, periodic in all directions,
 *   V = Lx*Ly*Lz*Lt sites numbered s = x + Lx*(y + Ly*(z + Lz*t)).
 *   Directions mu = 0, 1, 2, 3 are x, y, z, t.
 * Link layout (user side, FP64): U[mu][t][z][y][x][row][col][re, im], i.e.
 *   4*V*18 doubles, each 3x3 complex matrix row-major with interleaved real
 *   and imaginary parts.  Site fields (g, G, Delta) use the same layout
 *   without the leading mu: V*18 doubles.
 * where: LGF_HOST means a host pointer (any host memory; pinned memory gives
 *   the fastest copies), LGF_DEVICE a device pointer on the handle's device.
 * Ownership: the caller owns every buffer it passes; the library copies in
 *   and out and never keeps a caller pointer beyond the call, except the
 *   history buffers registered with lgf_set_trace.  The library owns its
 *   device workspace (allocated in lgf_create, freed in lgf_destroy), taken
 *   from CUDA's stream-ordered allocator or from a caller-supplied allocator
 *   (lgf_create_with_allocator).
 * Streams: all device work of a handle runs on the stream given to
 *   lgf_create (NULL = the legacy default stream), except that lgf_set_links
 *   from host memory checks the copied pieces on a second, internal stream
 *   of the handle, which it joins to the first before returning.  lgf_step
 *   is asynchronous; every call that returns numbers to the host
 *   synchronises that stream.
 * Errors: every call returns an lgf_status and never aborts; no C++
 *   exception crosses this interface.  A CUDA error is sticky for the handle:
 *   afterwards only lgf_destroy and lgf_last_error are meaningful.
 * Threads: a handle may be used by one host thread at a time.
 *
 * Readings of the paper fixed by this library
 * -------------------------------------------
 *  - theta = (1/(3V)) sum_x Tr[Delta Delta^dagger] with the paper's Delta,
 *    which is built from U - U^dagger and so equals 2 Delta_A, Delta_A being
 *    the divergence of the traceless anti-Hermitian parts A_mu of the links.
 *  - The Fourier filter is K(k) = alpha * p2max / p2(k) with
 *    p2(k) = sum_mu 4 sin^2(pi k_mu / L_mu) and K(0) = 0.
 *  - g(x) = reunitarize(1 + F^-1[K F[Delta_A]](x)): the exponential expanded
 *    to first order, then Gram-Schmidt on rows 1-2 and row 3 = (a x b)^*.
 *  - Algorithm 1 iterates while theta >= tol; the iteration count is the
 *    number of link updates.
 */
#ifndef LGF_H
#define LGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lgf_ctx* lgf_handle;

typedef enum {
  LGF_OK = 0,
  LGF_E_ARG = 1,          /* bad argument, or input links not in SU(3) within 1e-10 */
  LGF_E_NOMEM = 2,        /* device or pinned host allocation failed */
  LGF_E_CUDA = 3,         /* a CUDA call failed; the handle is now unusable */
  LGF_E_STATE = 4,        /* call not valid in the handle's state (e.g. no links set) */
  LGF_E_NONFINITE = 5,    /* non-finite input links, F or theta */
  LGF_E_NOTCONV = 6,      /* lgf_fix reached max_iter with theta >= tol */
  LGF_E_TIMEOUT = 7,      /* a bounded device wait gave up */
  LGF_E_UNSUPPORTED = 8   /* extents or options the library does not handle */
} lgf_status;

typedef enum {
  LGF_FP64 = 0,   /* FP64 links, FFTs and updates throughout */
  LGF_FP32 = 1,   /* FP32 links, Delta and FFTs; FP64 reductions and reunitarisation */
  LGF_MIXED = 2   /* FP32 phase until theta < switch level, then FP64 rebuilt from the FP64 input */
} lgf_precision;

enum {
  LGF_STORE18 = 0,        /* keep all three rows of each link (18 reals) */
  LGF_STORE12 = 1 << 0,   /* keep rows 1-2 (12 reals), rebuild row 3 = (a x b)^* (Sec. 3.2) */
  LGF_TRACK_G = 1 << 1,   /* accumulate G(x) = g_k(x)...g_1(x) for lgf_get_transform */
  LGF_LEARNED = 1 << 2,   /* multiply the filter by the learned per-mode multiplier (lgf_load_preconditioner) */
  LGF_PLAIN_SD = 1 << 3,  /* plain steepest descent: filter K(k) = alpha (no Fourier acceleration) */
  LGF_EXACT_EXP = 1 << 4  /* g = reunitarize(exp(Delta')) instead of the first-order reunitarize(1 + Delta')
                             of Sec. 2 (the exponential of Eq. (eq:gx) evaluated exactly, in FP64) */
};

enum { LGF_HOST = 0, LGF_DEVICE = 1 };

/* Create a handle for one lattice.
 * extents: {Lx, Ly, Lz, Lt}; each must be 2^a 3^b with 2 <= L <= 128, and
 *   the (x,y) and (z,t) planes must fit the shared-memory FFT passes
 *   (all extents up to 96, and 128 in z and t, are accepted); otherwise
 *   LGF_E_UNSUPPORTED.
 * prec: LGF_FP64, LGF_FP32 or LGF_MIXED.  flags: LGF_STORE12, LGF_TRACK_G,
 *   LGF_PLAIN_SD, LGF_LEARNED, LGF_EXACT_EXP (LGF_MIXED always tracks G);
 *   any other bit gives LGF_E_ARG.
 * cuda_stream: a cudaStream_t or NULL.  out: receives the handle.
 * Allocates all device workspace up front, stream-ordered on cuda_stream
 * (cudaMallocAsync; LGF_E_NOMEM if it does not fit), and synchronises that
 * stream before returning. */
lgf_status lgf_create(const int32_t extents[4], lgf_precision prec, uint32_t flags, void* cuda_stream,
                      lgf_handle* out);

/* Device memory supplied by the caller (for example from the caching
 * allocator of the framework the library runs under).  alloc returns `bytes`
 * bytes of device memory on the handle's device, at least 256-byte aligned,
 * usable by work enqueued on cuda_stream, or NULL on failure; free returns a
 * buffer that alloc gave, with the same size and stream.  Both are called
 * only from the thread that calls the library, with ctx passed through. */
typedef struct {
  void* (*alloc)(size_t bytes, void* cuda_stream, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* cuda_stream, void* ctx);
  void* ctx;
} lgf_allocator;

/* lgf_create with every device buffer of the handle taken from the caller's
 * allocator instead of CUDA's stream-ordered allocator (which lgf_create
 * uses: cudaMallocAsync / cudaFreeAsync on the handle's stream).  The
 * buffers are requested in this call and in lgf_set_trace,
 * lgf_load_preconditioner and lgf_set_mode_log, and all returned by
 * lgf_destroy.  allocator may be NULL (same as lgf_create); a non-NULL
 * allocator needs both functions (else LGF_E_ARG).  LGF_E_NOMEM when alloc
 * returns NULL, LGF_E_ARG when it returns memory not 256-byte aligned. */
lgf_status lgf_create_with_allocator(const int32_t extents[4], lgf_precision prec, uint32_t flags,
                                     void* cuda_stream, const lgf_allocator* allocator, lgf_handle* out);

/* Free the handle and its device memory.  NULL is accepted. */
lgf_status lgf_destroy(lgf_handle h);

/* Copy links in (layout above) and make them the current configuration:
 * the U_mu(x) on which the gauge transformation of Sec. 2, eq. 2,
 * U_mu(x) -> g(x) U_mu(x) g^dag(x + mu^), acts.
 * Resets G = 1 and the iteration counter, and measures F and theta.
 * Links must be finite (else LGF_E_NONFINITE) and in SU(3):
 * max(|U U^dag - 1|, |det U - 1|) <= 1e-10 (else LGF_E_ARG).
 * Synchronises the handle's stream. */
lgf_status lgf_set_links(lgf_handle h, const double* U, int where);

/* Copy the current links out as FP64 18-real matrices (12-real storage is
 * expanded with row 3 = (a x b)^*).  Synchronises. */
lgf_status lgf_get_links(lgf_handle h, double* U, int where);

/* One body of Algorithm 1: 4D FFT of Delta, filter K(k) (alpha given here),
 * inverse FFT, g = reunitarize(1 + Delta'), U -> g U g^dag(x+mu), then the
 * measurement of Delta, F and theta.  Asynchronous (enqueued on the stream),
 * except with LGF_LEARNED, where it synchronises to redo a rejected step
 * with the plain filter, and for an LGF_MIXED handle in its FP32 phase,
 * where it synchronises to read theta: when theta of the current links is
 * below the switch level (lgf_set_switch_theta) the handle first switches to
 * FP64 exactly as lgf_fix does, so that every step below that level runs in
 * FP64. */
lgf_status lgf_step(lgf_handle h, double alpha);

/* F and theta of the current links (Sec. 2, eq. 3 and the theta formula).
 * Either pointer may be NULL.  Synchronises. */
lgf_status lgf_measure(lgf_handle h, double* F, double* theta);

/* Algorithm 1: iterate lgf_step while theta >= theta_tol, at most max_iter
 * updates, with the loop condition evaluated on the device (CUDA graph with
 * a WHILE node; no host round trip per iteration).  In LGF_MIXED mode the
 * FP32 phase runs while theta >= max(theta_tol, switch level, default 1e-9;
 * see lgf_set_switch_theta), then G is
 * projected to SU(3) in FP64, U = G U0 G^dag(x+mu) is rebuilt in FP64 from
 * the FP64 input U0, and the FP64 phase runs to theta_tol.
 * iters, F, theta (each may be NULL) receive the update count of this call
 * and the final measurement.  Returns LGF_E_NOTCONV when max_iter is hit,
 * LGF_E_NONFINITE when F or theta became non-finite.  Synchronises. */
lgf_status lgf_fix(lgf_handle h, double theta_tol, int32_t max_iter, double alpha, int32_t* iters, double* F,
                   double* theta);

/* Overrelaxation gauge fixing, the lower-memory alternative that Sec. 3.2
 * names beside the Fourier-accelerated method.  The paper gives no algorithm
 * for it; this is the published one it refers to: F of Sec. 2, eq. 3, is
 * maximised one site at a time over all sites of one checkerboard colour at
 * once, the SU(3) maximisation done in the SU(2) subgroups (0,1), (0,2),
 * (1,2) in turn (Cabibbo and Marinari, 1982), each SU(2) maximiser r replaced
 * by r^omega ~ 1 + omega (r - 1) projected back onto SU(2) (Mandula and
 * Ogilvie, 1990).  One sweep is the even colour (x + y + z + t even), then
 * the odd one; each colour applies the gauge transformation of Sec. 2, eq. 2,
 * with g = 1 on the other colour, so G (LGF_TRACK_G, lgf_get_transform)
 * accumulates it like the Fourier-accelerated steps.
 * Needs every extent even and a handle without LGF_LEARNED, else
 * LGF_E_UNSUPPORTED.  The site algebra runs in the link precision; the
 * F/theta measurement is the one of lgf_measure.  After overrelaxation
 * sweeps lgf_get_gauge gives LGF_E_STATE (no g of a single step describes
 * them).
 *
 * lgf_or_sweep: nsweeps >= 0 sweeps with 1 <= omega < 2 (else LGF_E_ARG),
 * then one measurement; the update counter advances by nsweeps.
 * Asynchronous, except that an LGF_MIXED handle in its FP32 phase reads
 * theta first and switches to FP64 below the switch level, as lgf_step does. */
lgf_status lgf_or_sweep(lgf_handle h, double omega, int32_t nsweeps);

/* lgf_or_fix: measure, then while theta >= theta_tol and fewer than
 * max_sweeps sweeps: check_every sweeps and a measurement, all on the device
 * (CUDA graph WHILE node).  The count may pass max_sweeps by less than
 * check_every.  LGF_MIXED runs the FP32 phase to the switch level, rebuilds
 * the FP64 links as lgf_fix does and continues in FP64.  sweeps, F, theta
 * (each may be NULL) receive the sweep count and the final measurement; the
 * trace (lgf_set_trace) holds entry i after i sweeps at the measured counts.
 * Returns LGF_E_NOTCONV when max_sweeps is reached, LGF_E_ARG unless
 * 1 <= omega < 2, check_every >= 1, max_sweeps >= 0 and theta_tol >= 0.
 * Synchronises. */
lgf_status lgf_or_fix(lgf_handle h, double theta_tol, int32_t max_sweeps, double omega, int32_t check_every,
                      int32_t* sweeps, double* F, double* theta);

/* Copy out the accumulated transform G(x) = g_k(x) ... g_1(x) (site layout,
 * FP64): the product of the gauge transformations of Sec. 2, eq. 2, applied
 * by the steps since lgf_set_links, so that the current links equal
 * G(x) U_in(x) G^dag(x+mu) for the links U_in given to lgf_set_links.
 * LGF_E_STATE unless the handle tracks G.  Synchronises. */
lgf_status lgf_get_transform(lgf_handle h, double* G, int where);

/* Copy out the gauge transformation g(x) of the last step (site layout,
 * FP64).  LGF_E_STATE before the first step.  Synchronises. */
lgf_status lgf_get_gauge(lgf_handle h, double* g, int where);

/* Copy out Delta_A(x), the divergence of the traceless anti-Hermitian parts
 * of the current links (site layout, FP64; the paper's Delta is twice this).
 * Synchronises. */
lgf_status lgf_get_divergence(lgf_handle h, double* D, int where);

/* Register host arrays that receive F and theta after every measurement of
 * the next lgf_fix (entry 0 = the measurement before the first update,
 * entry k = after update k), up to cap entries.  cap = 0 unregisters.
 * The arrays must stay valid until lgf_fix returns. */
lgf_status lgf_set_trace(lgf_handle h, double* F_hist, double* theta_hist, int32_t cap);

/* Trace flags, one int32 per measurement (lgf_set_trace_ex).  Entry k > 0
 * describes update k and the measurement after it; entry 0 the measurement
 * before the first update (LGF_TRACE_FP64 only). */
enum {
  LGF_TRACE_FP64 = 1,      /* the update and the measurement ran in FP64 (else FP32) */
  LGF_TRACE_LEARNED = 2,   /* the update's filter was multiplied by the learned table */
  LGF_TRACE_REDO = 4,      /* the update redid a rejected learned step with the plain filter */
  LGF_TRACE_REPAIRED = 8   /* the links were reunitarised before the update (lgf_set_defect_bound) */
};

/* lgf_set_trace with two more per-measurement arrays (either may be NULL):
 * flags_hist receives the LGF_TRACE_* bits, defect_hist the sampled link
 * unitarity defect of the measured links (see lgf_set_defect_bound). */
lgf_status lgf_set_trace_ex(lgf_handle h, double* F_hist, double* theta_hist, int32_t* flags_hist,
                            double* defect_hist, int32_t cap);

/* Guard against loss of unitarity (an addition; no step of the paper's
 * Algorithm 1 reunitarises the links, so rounding drift accumulates, and far
 * from the fixed point -- e.g. with alpha above its convergent range -- the
 * rebuild of row 3 from rows 1-2 compounds it until F overflows).  Every
 * measurement also forms, over one link in 64 (every sixteenth warp of
 * sites, one direction each, all four directions covered), the largest of
 * | |a|^2 - 1 |, | |b|^2 - 1 | and |<a, b>| over the stored rows a, b, in the
 * link precision.  When it exceeds the bound of the running phase, lgf_fix
 * stops the device loop, reunitarises every link by Gram-Schmidt (rows 1-2,
 * row 3 = (a x b)^*), re-measures and continues; the step after a repair is
 * flagged LGF_TRACE_REPAIRED.  A repair is not a gauge transformation: it
 * moves the links by about the defect, so G then reproduces them only to
 * that level.  Defaults: 1e-10 for FP64 phases (the input tolerance of
 * lgf_set_links, so valid inputs never trigger it) and 1e-4 for FP32
 * phases; 0 disables the check.  LGF_E_ARG for negative bounds.  lgf_fix
 * returns LGF_E_NONFINITE if the bound is passed again within one step of a
 * repair. */
lgf_status lgf_set_defect_bound(lgf_handle h, double bound_fp64, double bound_fp32);

/* The sampled link defect of the last measurement, and the number of
 * reunitarisations in the last lgf_fix (either pointer may be NULL).
 * Synchronises. */
lgf_status lgf_get_link_defect(lgf_handle h, double* defect, int32_t* repairs);

/* The library's own 4D DFT of nfields = 4 complex fields in place, in the
 * handle's precision: data[f][t][z][y][x][re, im] (FP64 on the user side).
 * sign = -1: f^(k) = sum_x f(x) e^{-2 pi i k.x/L};  sign = +1: the same sum
 * with e^{+...}, unnormalised.  Exposed so that the transform can be checked
 * against the defining sum.  Synchronises. */
lgf_status lgf_fft4(lgf_handle h, double* data, int32_t nfields, int32_t sign, int where);

/* Per-kernel timing of lgf_step.  enable != 0 starts recording CUDA events
 * on the handle's stream around each kernel of every subsequent lgf_step
 * (not inside lgf_fix's graph) and clears the accumulators; enable = 0
 * stops.  Synchronises. */
lgf_status lgf_set_timing(lgf_handle h, int32_t enable);

/* Mean device time in milliseconds per step of each stage of the lgf_step
 * calls since timing was enabled: ms[0] pass A (forward (x,y) DFT), ms[1]
 * pass B ((z,t) DFT, filter, inverse), ms[2] pass C (inverse (x,y) DFT and
 * g), ms[3] link update, ms[4] measurement; nkernels <= 5 entries are
 * written.  With LGF_FFT_1D4 or LGF_FFT_3D1D, ms[0] holds the forward
 * passes, ms[1] the pass carrying the filter and ms[2] the inverse passes
 * and g; in a fused FP32 phase (lgf_set_fused_update) ms[3] holds the fused
 * update + measurement and ms[4] is 0.  nsteps (may be NULL) receives the
 * number of steps averaged.  Synchronises. */
lgf_status lgf_get_timing(lgf_handle h, double* ms, int32_t nkernels, int32_t* nsteps);
/* (ms[5], with nkernels = 6: the learned extras -- undo of a rejected step,
 * its re-measurement and the network inference -- of LGF_LEARNED handles.) */

/* ---- learned per-mode multiplier (an addition; the paper has no learned part) ----
 *
 * With LGF_LEARNED every step multiplies the filter by m(k) in [0.25, 2],
 * predicted for each momentum class (modes with the same per-direction
 * p2_mu = 4 sin^2(pi k_mu / L_mu)) by a network 8 -> 64 -> 64 -> 64 -> 1
 * (ReLU hidden layers, m = softplus(z)) with BF16 weights and FP32
 * accumulation on the tensor cores.  Features of a mode:
 *   (p2_x/4, p2_y/4, p2_z/4, p2_t/4, -floor(2 log10 theta)/32, min(iter/10000, 1),
 *    clamp(log10(theta/theta_prev), -2, 1)/2, r_class)
 * where theta and iter are those of the links the step starts from,
 * theta_prev that of the links one step earlier (the seventh feature is 0 on
 * the first step), and r_class the contraction of the mode's class over the
 * last step whose two Fourier-space divergences are kept:
 *   r_obs = sum Re<D^_{k-1}, D^_{k-2}> / sum |D^_{k-2}|^2  (over the modes and
 *   packed fields of the class),  r_class = clamp(1 - (1 - r_obs) / m, -1, 1),
 * m being the multiplier that produced D^_{k-1} from D^_{k-2}, so that r_class
 * is the contraction the plain filter would have given (0 until two
 * divergences are kept).  The filter pass stores each step's Fourier-space
 * divergence (before the filter, FP32) for this purpose.  A step that lowers
 * F is undone and redone with the plain filter; theta (of the plain
 * definition) decides convergence.
 *
 * Parameter layout (8961 numbers, rows [out][in]):
 *   W1[64][8] @0, b1[64] @512, W2[64][64] @576, b2[64] @4672,
 *   W3[64][64] @4736, b3[64] @8832, w4[64] @8896, b4 @8960. */
#define LGF_MLP_NPARAM 8961

/* Load BF16 network parameters (n_w must be LGF_MLP_NPARAM) into the
 * handle; where = LGF_HOST or LGF_DEVICE.  Synchronises. */
lgf_status lgf_load_preconditioner(lgf_handle h, const uint16_t* bf16_w, size_t n_w, int where);

/* Level below which the learned multiplier is applied (not in the paper: a
 * setting of the learned filter).  A step of an LGF_LEARNED handle from
 * links with theta >= theta uses the plain filter of Eq. (eq:gx) (the
 * network still runs, and writes a table of ones); below it the learned
 * table.  Default +inf: every step.  0 gives the plain method exactly.
 * LGF_E_STATE on a handle without LGF_LEARNED, LGF_E_ARG for a negative or
 * NaN level.  Takes effect from the next step. */
lgf_status lgf_set_learned_theta(lgf_handle h, double theta);

/* Number of learned steps that were rejected (F did not increase) and redone
 * with the plain filter during the last lgf_fix. */
lgf_status lgf_get_fallbacks(lgf_handle h, int32_t* n);

/* Mode log (training data).  enable != 0 makes every subsequent lgf_step
 * also accumulate, for each theta bucket b and momentum class c, the sums
 *   Re<D^_{k+1}, D^_k>, |D^_k|^2, count, iteration fraction of step k,
 *   last-step contraction feature of step k, Re<D^_k, D^_{k-1}>, |D^_{k-1}|^2
 * over the modes of the class, D^ being the 4D Fourier transform of the
 * packed divergence (b = clamp(4 - 2 floor(2 log10 theta_k)/2, 0, 39)); the
 * last two only once D^_{k-1} is known.  Enabling clears the sums.
 * Synchronises. */
lgf_status lgf_set_mode_log(lgf_handle h, int32_t enable);

/* Copy the mode-log sums out: n must be 40 * nclass * 7 doubles, laid out
 * [b][c][7] with nclass = prod_mu (L_mu/2 + 1) and
 * c = ((f_t H_z + f_z) H_y + f_y) H_x + f_x, f_mu = min(k_mu, L_mu - k_mu),
 * H_mu = L_mu/2 + 1.  out is a host pointer.  Synchronises. */
lgf_status lgf_get_mode_log(lgf_handle h, double* out, int64_t n);

/* Network inference on the tensor cores for arbitrary feature rows
 * (device pointers): X[n][8] FP32 features, P[8961] BF16 parameters,
 * m[n] = softplus(z) FP32 out (unclamped).  Enqueued on cuda_stream. */
lgf_status lgf_mlp_eval(const uint16_t* P, const float* X, int64_t n, float* m, void* cuda_stream);

/* Loss L = (1/n) sum_i w_i (log m_i - y_i)^2 over all rows and its gradient
 * with respect to the FP32 parameters (device pointers: P[8961], X[n][8],
 * Y[n], W[n], grad[8961]); *loss on the host.  Synchronises. */
lgf_status lgf_mlp_loss_grad(const float* P, const float* X, const float* Y, const float* W, int64_t n, float* grad,
                             double* loss, void* cuda_stream);

/* Adam training of the FP32 parameters P (device, in place) on minibatches of
 * `batch` rows drawn by a counter-based hash of (seed, step, row): `steps`
 * updates with learning rate lr, moments in adam[2 * 8961] (device, zero for
 * a fresh start), t0 = number of updates done before (bias correction).
 * loss_hist (host, may be NULL) receives the minibatch loss of every
 * update.  Synchronises. */
lgf_status lgf_mlp_train(float* P, float* adam, const float* X, const float* Y, const float* W, int64_t n,
                         int32_t batch, int32_t steps, float lr, uint64_t seed, int32_t t0, double* loss_hist,
                         void* cuda_stream);

/* FP32 -> BF16 (round to nearest even) of the 8961 parameters (device). */
lgf_status lgf_mlp_to_bf16(const float* P, uint16_t* out, void* cuda_stream);

/* Theta below which an LGF_MIXED fix leaves the FP32 phase (default 1e-9;
 * accepted range [1e-10, 1e-6], so every iteration below 1e-10 is FP64). */
lgf_status lgf_set_switch_theta(lgf_handle h, double theta);

/* Decomposition of the 4D transform of every following step (Sec. 3.2
 * compares the three on cuFFT; here each is a set of shared-memory passes):
 *   LGF_FFT_2D2D (default): (x,y) pass; (z,t) pass with the filter; inverse
 *     (x,y) pass fused with g -- three passes over the divergence.
 *   LGF_FFT_1D4: one pass per direction and sign, the t pass carrying the
 *     filter, then a separate g kernel -- seven passes plus g.
 *   LGF_FFT_3D1D: an (x,y,z) pass per t plane, a t pass with the filter, the
 *     inverse (x,y,z) pass, then g -- three passes plus g; only where one
 *     field's (x,y,z) slab fits in shared memory (up to 16^3 in FP64, 24^3
 *     in FP32), else LGF_E_UNSUPPORTED.
 * All three give the same result up to rounding (the learned multiplier is
 * applied in the pass that carries the filter in each).  Synchronises. */
enum { LGF_FFT_2D2D = 0, LGF_FFT_1D4 = 1, LGF_FFT_3D1D = 2 };
lgf_status lgf_set_fft_decomposition(lgf_handle h, int32_t decomposition);

/* FP32 phase only: run the link update and the following measurement as one
 * kernel (enable != 0, the default for LGF_FP32 and LGF_MIXED handles) or as
 * two (enable = 0).  The fused kernel reads the links from one of two
 * buffers and writes the updated links to the other; it recomputes the
 * updated backward links U'_mu(x - mu^) in registers instead of reading them
 * back, so the links cross HBM once less per step.  The undo of a rejected
 * learned step works on whichever buffer holds the current links.  Results
 * are bit-identical either way.  No effect on FP64 phases.  Synchronises. */
lgf_status lgf_set_fused_update(lgf_handle h, int32_t enable);

/* Autotuner of a handle: times the transform and g of one step (CUDA events,
 * best of 3 after a warm-up) under every tile plan of the 2D + 2D passes
 * (fields per CTA of the (x,y) passes, x columns of the (z,t) pass, CTA
 * sizes) and under LGF_FFT_1D4 (with its tiles) and LGF_FFT_3D1D where it
 * fits, for each precision the handle runs in, and keeps the fastest
 * for the following steps.  report (may be NULL): receives a JSON object
 * {"fp64": {"chosen": i, "candidates": [{"decomposition", "fields_per_cta_xy",
 * "x_columns_zt", "threads", "ms"}, ...]}, "fp32": ...}; LGF_E_ARG if len is
 * too small (the choice is kept).  When the environment variable
 * LGF_AUTOTUNE_CACHE names a file, a choice recorded there for the same
 * lattice, precision, storage and device is applied without timing (report:
 * "cached": true, one candidate with "ms": null) and new choices are
 * appended to it, so that separate runs use the same plan.  Overwrites the
 * divergence workspace and g (lgf_get_gauge then fails until the next step)
 * and re-measures the current links.  Synchronises. */
lgf_status lgf_autotune(lgf_handle h, char* report, size_t len);

/* Phase of an LGF_MIXED handle: 32 while in the FP32 phase, 64 after the
 * switch (FP64 and FP32 handles report their fixed precision). */
lgf_status lgf_get_phase(lgf_handle h, int32_t* bits);

/* Largest lattice (sites) lgf_measure_static accepts. */
#define LGF_STATIC_MAX_SITES 16777216

/* Measurement of Delta_A, F and theta that allocates nothing.  The paper has
 * no counterpart: this exists for callers that must not allocate device
 * memory where they measure -- e.g. a host application whose device memory
 * is owned entirely by its own pool allocator, or monitoring code between
 * the steps of a time-critical loop, where cudaMalloc/cudaFree could fail or
 * synchronise the device.  The computation is the one lgf_measure and
 * lgf_get_divergence perform, without a handle.
 * extents: {Lx, Ly, Lz, Lt}, each 2^a 3^b in [2, 128], and at most
 *   LGF_STATIC_MAX_SITES sites in total (else LGF_E_UNSUPPORTED; nothing is
 *   launched).
 * U: device pointer, FP64 links in the user layout (4*V*18 doubles, read only).
 * D: device pointer to V*18 doubles receiving Delta_A in the site layout, or
 *   NULL to skip it.
 * F_theta: device pointer to 2 doubles receiving F and theta.
 * cuda_stream: a cudaStream_t or NULL; the work is enqueued there and the
 *   call returns without synchronising.
 * Scratch: a fixed 1 MB device array inside the library (one per device,
 *   held until the process exits) that every call on a device shares.  Calls
 *   whose kernels may overlap on the GPU (other streams, other host threads)
 *   race on it and must be serialised by the caller.  The first call on each
 *   device looks up the array's device address, so make that first call
 *   before any stream capture begins.  No cudaMalloc, cudaFree or other
 *   allocating routine is called.
 * Returns LGF_OK, LGF_E_ARG (NULL pointers), LGF_E_UNSUPPORTED or LGF_E_CUDA. */
lgf_status lgf_measure_static(const int32_t extents[4], const double* U, double* D, double* F_theta,
                              void* cuda_stream);

/* ---- batches of configurations (an addition; the paper fixes one at a time) ----
 *
 * Many configurations of possibly different lattice shapes fixed together,
 * FP64 with 18-real links and the plain filter.  Configurations of the same
 * shape share their kernel launches (one launch per step kernel per shape);
 * lgf_batch_fix runs the whole fix as ONE CUDA graph launch whose WHILE loop
 * continues while any configuration has theta >= tol and fewer than
 * max_iter updates; a configuration retires (stops being updated) as soon as
 * its own theta falls below tol.  Every kernel of a retired configuration
 * returns immediately; no kernel waits on another.  The FFT tile shapes of
 * each shape are chosen at creation by timing every candidate on the
 * configurations' buffers (cached per process, and in the file named by the
 * environment variable LGF_AUTOTUNE_CACHE when it is set). */
typedef struct lgf_batch_ctx* lgf_batch;

/* n configurations; extents: n*4 int32 ({Lx, Ly, Lz, Lt} of each, rules as
 * in lgf_create).  prec must be LGF_FP64 and flags 0 (else
 * LGF_E_UNSUPPORTED).  Allocates and autotunes.  Synchronises. */
lgf_status lgf_batch_create(int32_t n, const int32_t* extents, lgf_precision prec, uint32_t flags, void* cuda_stream,
                            lgf_batch* out);
lgf_status lgf_batch_destroy(lgf_batch b);

/* Links of configuration i (0 <= i < n) in the user layout of its own shape;
 * validated like lgf_set_links.  Synchronises. */
lgf_status lgf_batch_set_links(lgf_batch b, int32_t i, const double* U, int where);
lgf_status lgf_batch_get_links(lgf_batch b, int32_t i, double* U, int where);

/* Fix every configuration: iters, F, theta (each NULL or n entries) receive
 * the per-configuration update counts and final measurements.
 * LGF_E_NOTCONV if any configuration reached max_iter.  Synchronises. */
lgf_status lgf_batch_fix(lgf_batch b, double theta_tol, int32_t max_iter, double alpha, int32_t* iters, double* F,
                         double* theta);

/* JSON description of the shape classes and their autotuned FFT tiles. */
lgf_status lgf_batch_describe(lgf_batch b, char* buf, size_t len);
const char* lgf_batch_last_error(lgf_batch b);

/* Human-readable name of a status code (static string). */
const char* lgf_status_string(lgf_status s);

/* Text of the last error on the handle ("" if none; static for NULL). */
const char* lgf_last_error(lgf_handle h);

#ifdef __cplusplus
}
#endif

#endif /* LGF_H */
