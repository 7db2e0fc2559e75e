/*
 * gl.h - C ABI of libgl, a B300 (sm_103a) library that evaluates the
 * log-posterior of a strong gravitational lens model, and its gradient, for
 * a batch of parameter vectors per call.
 *
 * The model is the one the GIGA-Lens pipeline samples (Sec. 3 of the paper:
 * an elliptical power-law (EPL) mass with external shear, elliptical Sersic
 * lens light, elliptical Sersic source light, intensities as free parameters
 * ("forward" modelling), a supersampled pixel grid; the priors of Eq.
 * sim-dist, Sec. 4.2). Every multi-start MAP step, SVI draw and HMC leapfrog
 * of the pipeline (Sec. 3, Sec. 3.1) reduces to the calls below.
 *
 * Model definition (the paper defers the forward model to its predecessor;
 * these are the readings this library implements):
 *   grid      pixel (i, j) centre x = (j - (nx-1)/2) D, y = (i - (ny-1)/2) D
 *             (D = pixel_scale, arcsec); sub-pixel (k, l) of supersampling s
 *             at ((l + 1/2)/s - 1/2) D, ((k + 1/2)/s - 1/2) D from it.
 *   ellipticity (e1, e2) -> axis ratio q = (1-|e|)/(1+|e|), position angle
 *             atan2(e2, e1)/2 (major axis along +x for e1 > 0).
 *   EPL       deflection by the Tessore & Metcalf (2015) hypergeometric
 *             series, theta_E in the intermediate-axis convention
 *             (b = theta_E sqrt(q)); convergence (2-t)/2 (b/R)^t, t = gamma-1,
 *             R = sqrt(q^2 x'^2 + y'^2).
 *   shear     alpha = (g1 x + g2 y, g2 x - g1 y), centred on the origin.
 *   Sersic    I_e exp(-b_n ((R/R_e)^(1/n) - 1)), b_n = 1.9992 n - 0.3271,
 *             R = sqrt(q x'^2 + y'^2/q).  Radii are clamped below at 1e-6".
 *   source    evaluated at beta = theta - alpha_EPL - alpha_shear.
 *   image     m = PSF (*) [D^2 x mean of the s x s sub-pixel brightnesses],
 *             true convolution, "same" size, zero padding, PSF renormalised
 *             to unit sum.
 *   log p     -1/2 sum ((d - m)/sigma)^2 + log prior (normalised 1-D
 *             densities; |e| < emax discs restrict the support only).
 *
 * Parameter vector (row-major theta[B][P], P = 8 + 7 (n_lens_light +
 * n_source)), in the order of Eq. sim-dist:
 *   [theta_E, gamma, e1, e2, x, y]_EPL, [gamma1, gamma2]_shear,
 *   per lens-light component [R_e, n, e1, e2, x, y, I_e],
 *   per source component     [R_e, n, e1, e2, x, y, I_e].
 *
 * Domain. A row outside the model's domain (theta_E <= 0, gamma outside
 * (1, 3), any |e| >= 0.8, R_e <= 0, n < 0.2) or outside the prior's support
 * gets logp = -inf and a zero gradient. A row holding a NaN gets NaN for
 * logp and every gradient entry. Neither is an error: the call returns GL_OK.
 *
 * Conventions for every call:
 *   - Pointers documented "device" are CUDA device (or managed) pointers on
 *     the current device; "host" are ordinary host pointers.
 *   - Calls that take a stream enqueue work on it (a cudaStream_t passed as
 *     void*, NULL = the legacy default stream) and return without waiting.
 *   - The caller owns theta and every output buffer; the library never frees
 *     or keeps them. The library owns gl_system and gl_surrogate objects and
 *     their device copies.
 *   - Every call returns a status and never aborts. GL_EINVAL = rejected
 *     arguments (nothing was enqueued), GL_ENOMEM = a device allocation
 *     failed, GL_ECUDA = a CUDA call failed. gl_last_error() describes the
 *     last failure on the calling host thread.
 *   - One gl_system must not be used by two host threads at once, nor by two
 *     streams whose work overlaps (it owns one scratch arena).
 */
#ifndef GL_H
#define GL_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GL_OK = 0,
  GL_EINVAL = 1,
  GL_ENOMEM = 2,
  GL_ECUDA = 3,
  GL_ENOSURROGATE = 4,
  GL_ETIMEOUT = 5
} gl_status;

/* Which deflection the EPL uses:
 *   GL_DEFL_SERIES     the exact series at every sub-pixel;
 *   GL_DEFL_SURROGATE  the learned surrogate (gl_system_set_surrogate): per
 *                      row, F and its derivatives on 128 angles from the
 *                      network, interpolated (cubic Hermite) at every
 *                      sub-pixel; rows outside its training domain use the
 *                      exact series; the tables are built by a launch of their
 *                      own;
 *   GL_DEFL_TABLE      the same tables filled from the exact series summed in
 *                      FP64 (rows with |e| > 0.5 use the series): differs from
 *                      GL_DEFL_SERIES by the interpolation error only;
 *   GL_DEFL_TABLE32    the same, with the series at the table's nodes summed in
 *                      FP32 (the build takes a fraction of the FP64 one's time on
 *                      a GPU whose FP64 rate is 1/64 of its FP32 rate);
 *   GL_DEFL_SURROGATE_FUSED  the surrogate of GL_DEFL_SURROGATE with its results
 *                      bit for bit, but gl_logp_grad evaluates the network
 *                      inside each row's CTA of the gradient kernel (tensor
 *                      cores; the table never leaves shared memory) where two
 *                      such CTAs fit per SM; the other entry points, and
 *                      gl_logp_grad where they do not fit, build the tables in
 *                      a launch of their own. On the B300 the separate launch
 *                      is the faster of the two at the benchmark's sizes. */
typedef enum {
  GL_DEFL_SERIES = 0,
  GL_DEFL_SURROGATE = 1,
  GL_DEFL_TABLE = 2,
  GL_DEFL_TABLE32 = 3,
  GL_DEFL_SURROGATE_FUSED = 4
} gl_deflection;

/* Prior kinds (Eq. sim-dist, Sec. 4.2). */
typedef enum {
  GL_PRIOR_FLAT = 0,      /* no density; support [lo, hi] (may be infinite) */
  GL_PRIOR_UNIFORM = 1,   /* U(lo, hi), lo < hi finite                       */
  GL_PRIOR_NORMAL = 2,    /* N(a, b), b > 0                                  */
  GL_PRIOR_TRUNCNORM = 3, /* N(a, b) truncated to [lo, hi], renormalised     */
  GL_PRIOR_LOGNORMAL = 4  /* log x ~ N(a, b), x > 0                          */
} gl_prior_kind;

typedef struct {
  int kind; /* gl_prior_kind */
  float a, b, lo, hi;
} gl_prior;

/* Description of one lens system. All arrays are copied by gl_system_create
 * and may be freed by the caller afterwards. */
typedef struct {
  int ny, nx;          /* image size in pixels, 1..2048 each                 */
  float pixel_scale;   /* arcsec per pixel, > 0                              */
  int supersample;     /* s, 1..8                                            */
  const float* data;   /* observed image d [ny*nx], row-major (y = row)      */
  const float* sigma;  /* noise map [ny*nx], > 0 (+inf masks a pixel)       */
  const float* psf;    /* PSF [psf_ny*psf_nx], positive sum                  */
  int psf_ny, psf_nx;  /* odd, 1..21                                         */
  int n_lens_light;    /* Sersic lens-light components, 0..2                 */
  int n_source;        /* Sersic source components, 1..3                     */
  const gl_prior* prior; /* host [P]                                         */
  const float* emax;   /* host [1 + n_lens_light + n_source]: |e| < emax per
                          component (EPL first), 0 = no constraint; may be NULL */
  int inputs_on_device; /* nonzero: data, sigma and psf are device pointers  */
} gl_system_desc;

typedef struct gl_system gl_system;
typedef struct gl_surrogate gl_surrogate;

/* Creates a system: validates desc, copies data, sigma^-2 and the normalised
 * PSF to the current device. Synchronous. On error *out is NULL. */
gl_status gl_system_create(const gl_system_desc* desc, gl_system** out);

/* Frees a system and its device memory (waits for the device first). NULL is
 * accepted. */
gl_status gl_system_destroy(gl_system* sys);

/* P = 8 + 7 (n_lens_light + n_source); -1 for NULL. */
int gl_system_num_params(const gl_system* sys);

/* log p(theta_b | d) for b < B (Sec. 3: the quantity every MAP, SVI and HMC
 * step evaluates). theta: device [B][P]; logp: device [B]. B = 0 is a no-op.
 * GL_ENOSURROGATE if defl = GL_DEFL_SURROGATE and no surrogate is attached. */
gl_status gl_logp(gl_system* sys, const float* theta, int B, float* logp, gl_deflection defl,
                  void* stream);

/* log p and its gradient d log p / d theta (the autodiff call of Sec. 3).
 * grad: device [B][P]. */
gl_status gl_logp_grad(gl_system* sys, const float* theta, int B, float* logp, float* grad,
                       gl_deflection defl, void* stream);

/* The same with HOST buffers: copies theta in, evaluates, copies logp and grad
 * (grad may be NULL) back and waits for the stream. When every buffer passed is
 * page-locked host memory (cudaHostAlloc, cudaHostRegister, torch's
 * pin_memory) from its first to its last byte, the copies go directly between
 * those buffers and the device; otherwise they go through the system's own
 * pinned staging buffers (one host memcpy each way). Grows the system's
 * staging buffers on first use. */
gl_status gl_logp_grad_host(gl_system* sys, const float* theta_host, int B, float* logp_host,
                            float* grad_host, gl_deflection defl, void* stream);

/* ---------------------------------------------------------------------------
 * Uneven multi-system batches: many systems (different image sizes,
 * supersampling, component counts), each with its own rows, per call (the
 * batched structure of Sec. 3.1 over the simulated systems of Sec. 4.2). One
 * persistent launch per group of systems sharing (n_lens_light, n_source)
 * and launch shape evaluates all rows of the group; rows are taken heaviest
 * system first from a device work queue. The groups' launches run
 * concurrently on streams the plan owns (so one group's tail overlaps the
 * next group's start), forked from and joined back into the caller's stream:
 * the call stays stream-ordered for the caller.
 * ------------------------------------------------------------------------- */
typedef struct gl_multi gl_multi;

/* Shared-memory policies for the image buffers of a multi-system launch:
 *   0  all buffers in global scratch (occupancy set by registers alone);
 *   1  shared memory while the launch shape's full occupancy still fits
 *      (two CTAs of 256 threads or four of 128 per SM), the rest in global
 *      scratch;
 *   2  shared memory up to one CTA per SM.
 * Which is fastest depends on the size mix; the package's autotuner times them. */
enum { GL_MULTI_SMEM_GLOBAL = 0, GL_MULTI_SMEM_TWO_CTAS = 1, GL_MULTI_SMEM_ONE_CTA = 2 };

/* Plans a batch over n_sys systems (borrowed: they must outlive the plan and
 * live on the current device) with rows_per_sys[k] rows each. Allocates the
 * work lists and the per-CTA scratch. */
gl_status gl_multi_create(gl_system* const* systems, int n_sys, const int* rows_per_sys,
                          int smem_policy, gl_multi** out);

/* The same with a launch shape per system (the tile shape that the package's
 * autotuner picks per image class): threads_per_cta[k] in {128, 256} (CTAs
 * of 128 threads run four per SM, of 256 two, at 128 registers a thread) and
 * pixel_pairs[k] in {2, 3}, the pixel pairs each thread keeps in flight in
 * the forward binning (more independent work per thread for the latency of
 * the MUFU/FP32 chain). Either array may be NULL: 256 threads, 2 pairs. The
 * pixel pairs do not change results (each pixel sums its sub-pixels in the
 * same order); with 256 threads the results equal gl_logp_grad's bit for bit,
 * with 128 the chi^2 and gradient terms are summed in another order and agree
 * to FP32 reassociation. Other values: GL_EINVAL. */
gl_status gl_multi_create_ex(gl_system* const* systems, int n_sys, const int* rows_per_sys,
                             int smem_policy, const int* threads_per_cta,
                             const int* pixel_pairs, gl_multi** out);

/* log p and gradient of every row of every system: theta[k] device
 * [rows_k][P_k], logp[k] device [rows_k], grad[k] device [rows_k][P_k] (host
 * arrays of device pointers). Results equal gl_logp_grad per system with the
 * same deflection (bit for bit in the default launch shape). The work lists
 * are re-uploaded when a pointer changes. */
gl_status gl_multi_logp_grad(gl_multi* multi, const float* const* theta, float* const* logp,
                             float* const* grad, gl_deflection defl, void* stream);

/* Frees a plan (waits for the device). NULL is accepted. */
gl_status gl_multi_destroy(gl_multi* multi);

/* n_steps HMC leapfrog steps for B chains, in place (the integrator of the
 * pipeline's HMC stage, Sec. 3; Sec. 3.1 runs chains independently). Per step,
 * with diagonal inverse mass M^-1 and step size eps:
 *   p += eps/2 grad; theta += eps M^-1 p; (logp, grad) at theta; p += eps/2 grad.
 * theta, p, grad: device [B][P]; logp: device [B]; inv_mass: device [P].
 * On entry logp and grad must hold the values at theta (from gl_logp_grad or a
 * previous block); on return they hold the values at the new theta. A chain
 * whose log p is not finite is frozen (theta and p left as they are) and keeps
 * its -inf/NaN log p: divergent trajectories are flagged, not trapped.
 * The block runs as one CUDA graph launch on the stream: the library captures
 * it on a private stream the first time and again whenever a pointer, eps,
 * n_steps or B changes (re-capture costs about a millisecond). Do not call it
 * while the calling thread is capturing a stream. */
gl_status gl_leapfrog(gl_system* sys, float* theta, float* p, float* logp, float* grad,
                      const float* inv_mass, float eps, int n_steps, int B, void* stream);

/* Model image m (binned, PSF-convolved) for each row: img device [B][ny][nx].
 * Rows outside the model's domain or holding a NaN give NaN images; the prior
 * is not checked. */
gl_status gl_model_image(gl_system* sys, const float* theta, int B, float* img,
                         gl_deflection defl, void* stream);

/* Size of the fixed scratch array used by gl_logp_grad_noalloc, in floats
 * (64 MiB). */
#define GL_NOALLOC_SCRATCH_FLOATS (16u * 1024u * 1024u)

/* gl_logp_grad for callers that must not allocate device memory. The paper
 * has no counterpart: this is a deployment variant of the same computation.
 * It is meant for code that runs under a framework owning a fixed device
 * memory budget, or in a real-time loop that cannot take cudaMalloc's
 * implicit synchronisation; gl_logp_grad may call cudaMalloc to grow the
 * system's scratch, this call never allocates (no cudaMalloc, cudaFree or
 * allocating library routine).
 *   - Scratch: one file-scope device array of GL_NOALLOC_SCRATCH_FLOATS floats
 *     that every GPU loading the library holds until the process exits.
 *     Images whose two padded buffers fit in shared memory use none of it;
 *     larger ones need one slot per row (below), and a batch whose slots
 *     exceed the array is rejected with GL_EINVAL (gl_last_error() states the
 *     largest batch that fits).
 *   - The first call on each device looks up the array's device address (and
 *     may load the library's device code); make that first call before any
 *     stream capture. The address is kept for the life of the process, so the
 *     call must not be used after a cudaDeviceReset of that device.
 *   - Images whose padded buffer does not fit in shared memory take scratch
 *     per row: one padded buffer (Hp x Wp floats, Hp = ny + psf_ny - 1,
 *     Wp = nx + psf_nx - 1, rounded up to a multiple of 4) when that one
 *     buffer fits in shared memory but two do not, two buffers otherwise.
 *   - The caller's current CUDA device is the same on return.
 *   - Every call shares the one array, which keeps the last call's contents
 *     (the kernel writes every value it later reads): calls whose work
 *     overlaps on the GPU, from any system or stream, race on it.
 * Arguments, outputs and errors are those of gl_logp_grad with
 * defl = GL_DEFL_SERIES. */
gl_status gl_logp_grad_noalloc(gl_system* sys, const float* theta, int B, float* logp,
                               float* grad, void* stream);

/* ---------------------------------------------------------------------------
 * Learned EPL deflection surrogate (a learned replacement of the
 * hypergeometric series the deflection uses, Sec. 3 mass model).
 * A 4 -> 64 -> 64 -> 64 -> 64 -> 2 SiLU MLP with inputs (q, gamma,
 * log(R/theta_E), vphi): q the EPL axis ratio, vphi the angle of q x' + i y'
 * in [0, 2 pi). It predicts F = 2F1(1, t/2; 2 - t/2; -f e^{2 i vphi}) beyond
 * its first two series terms with the factor z^3 taken out, times 4:
 *   F = 1 + c1 z + c2 z^2 + z^3 y/4, z = -f e^{2 i vphi}, c1 = t/(4-t),
 *   c2 = c1 (2+t)/(6-t), y (complex) ~ 4 sum_{n>=3} c_n z^{n-3}.
 * BF16 weights and activations, FP32 accumulation (tensor cores), FP32
 * master weights. Parameter vector (FP32, gl_surrogate_num_params() floats):
 * W1[64][4], b1[64], W2[64][64], b2, W3, b3, W4, b4, W5[2][64], b5[2]
 * (W[out][in], row-major), acting on normalised inputs
 *   ((q-0.75)/0.25, (gamma-2)/0.3, log(R/theta_E)/2.3, (vphi-pi)/pi).
 * ------------------------------------------------------------------------- */
typedef struct {
  long long n_samples;    /* training tuples labelled by the exact series (e.g. 1e7) */
  int epochs;             /* passes over the tuples                              */
  int batch;              /* rows per step, a multiple of 128                    */
  float lr, lr_min;       /* Adam learning rate, cosine-decayed to lr_min        */
  unsigned long long seed_data, seed_init;
  float q_lo, q_hi;       /* q ~ U(q_lo, q_hi), 0 < q_lo < q_hi <= 1            */
  float gamma_lo, gamma_hi;  /* gamma ~ U(gamma_lo, gamma_hi) inside (1, 3)      */
  float r_lo, r_hi;       /* R/theta_E ~ logU(r_lo, r_hi)                         */
} gl_surrogate_train_desc;

/* Number of FP32 parameters of the surrogate MLP (12930). */
int gl_surrogate_num_params(void);

/* Generates the training tuples on the device, trains with Adam (on the
 * current device; synchronous) and returns the trained surrogate. final_loss
 * (may be NULL) receives the mean squared error of the last batch in the
 * scaled output units. The [q_lo, q_hi] x [gamma_lo, gamma_hi] box is the
 * surrogate's domain: rows outside it use the exact series. */
gl_status gl_surrogate_train(const gl_surrogate_train_desc* desc, gl_surrogate** out,
                             float* final_loss);

/* A surrogate from given parameters (host [gl_surrogate_num_params()]) with
 * the default domain q in [0.5, 1], gamma in [1.7, 2.3]. */
gl_status gl_surrogate_create(const float* params_host, gl_surrogate** out);

/* Copies the FP32 parameters to host memory. */
gl_status gl_surrogate_params(const gl_surrogate* sur, float* params_host);

/* F (Re, Im) for N raw inputs x: device [N][4] = (q, gamma, log(R/theta_E),
 * vphi) -> y: device [N][2]. x is read as float4 and must be 16-byte aligned,
 * y 8-byte aligned (else GL_EINVAL). */
gl_status gl_surrogate_infer(const gl_surrogate* sur, const float* x, int N, float* y,
                             void* stream);

/* The exact F = 2F1(1, t/2; 2 - t/2; -f e^{2 i vphi}) (Sec. 3 mass model,
 * the series of Tessore & Metcalf 2015), summed in FP64 on the device until
 * the terms fall below 1e-18, for N raw inputs x: device [N][4] = (q, gamma,
 * ignored, vphi) -> F: device [N][2] (Re, Im, rounded to FP32); the
 * reference the surrogate's deflection error is measured against. Tuples outside 0.01 <= q <= 1,
 * 1 < gamma < 3 (or not finite) give NaN. Asynchronous on stream; GL_EINVAL for N < 0, NULL
 * pointers with N > 0, or x not 16-byte / F not 8-byte aligned. */
gl_status gl_series_F(const float* x, int N, float* F, void* stream);

/* Mean squared training loss and its gradient w.r.t. the parameters for N
 * rows (N a multiple of 128): x device [N][4] raw inputs (16-byte aligned),
 * target device [N][2] (8-byte aligned) in the network's output units (y
 * above); loss_host and
 * grad_host [gl_surrogate_num_params()] receive the results. Synchronous. */
gl_status gl_surrogate_loss_grad(const gl_surrogate* sur, const float* x, const float* target,
                                 int N, float* loss_host, float* grad_host);

/* The tensor-core surrogate kernels (the per-row table build behind
 * GL_DEFL_SURROGATE, and the training step) bound every wait for a tensor-core
 * completion. A wait that runs out drains its outstanding commit (bounded
 * again), frees its tensor memory and fills its outputs with NaN; the call
 * reports GL_ETIMEOUT: gl_surrogate_train and gl_surrogate_loss_grad at
 * once (they are synchronous), a table build at the first GL_DEFL_SURROGATE
 * call on the same surrogate after the failed build has completed on its
 * stream (asynchronous, like CUDA's own errors); the rows it served have NaN
 * log p and gradient.
 *
 * Test hook (no counterpart in the paper): with on != 0 the tensor-core
 * kernels launched afterwards take that timeout path at their first wait as
 * if it had run out, without waiting (so no wait really runs out and every
 * commit is still drained before the tensor memory is freed); on = 0
 * restores normal operation. Process-wide, for every device the calling
 * thread's current device is; synchronous. Not for production use. */
gl_status gl_debug_force_wait_timeout(int on);

/* Save / load the parameters and domain to / from a flat binary file. */
gl_status gl_surrogate_save(const gl_surrogate* sur, const char* path);
gl_status gl_surrogate_load(const char* path, gl_surrogate** out);

/* Frees a surrogate (waits for the device). NULL is accepted. */
void gl_surrogate_destroy(gl_surrogate* sur);

/* Attaches a surrogate to a system (borrowed: it must outlive the system's
 * use of GL_DEFL_SURROGATE); NULL detaches. */
gl_status gl_system_set_surrogate(gl_system* sys, const gl_surrogate* sur);

/* ------------------------------------------------------------------------
 * Inference layer (Sec. 3): the MAP, SVI and HMC stages work on an
 * unconstrained vector u, mapped to the parameters by a bijection theta(u)
 * ("mapped into an unconstrained space via a bijective transformation",
 * Sec. 3.1). The paper defers the map to its earlier release; this library
 * takes one map per prior support:
 *   normal, or no finite bound  theta = u
 *   both bounds finite          theta = lo + (hi - lo) sigmoid(u)
 *   log-normal                  theta = exp(u)
 *   one finite bound            theta = lo + exp(u) / hi - exp(u)
 * (the bounds of a uniform, truncated-normal or flat prior)
 * and, for a component whose ellipticity is restricted to |e| < emax while
 * both e priors are unbounded, the radial map e = v emax tanh(|v|)/|v|.
 * log p~(u) = log p(theta(u)) + log|det d theta/d u|. All arrays below are
 * device arrays in row-major [B][P] (u, theta, gradients) or [B] (log p, log
 * |J|), unless marked host. Calls are asynchronous on the stream.
 * ------------------------------------------------------------------------ */

/* theta(u) and log|det d theta/d u| (logdetj may be NULL). */
gl_status gl_bijector_forward(gl_system* sys, const float* u, int B, float* theta,
                              float* logdetj, void* stream);

/* u(theta), the inverse map; theta must lie inside the support (rows outside
 * give NaN or infinite u). */
gl_status gl_bijector_inverse(gl_system* sys, const float* theta, int B, float* u, void* stream);

/* log p~(u) and its gradient d log p~/d u = J^T grad_theta log p + grad log|J|
 * (three launches: the map, the fused log p + gradient kernel, the
 * pull-back). Rows whose log p is -inf/NaN keep it, with a zero/NaN gradient. */
gl_status gl_logp_grad_unconstrained(gl_system* sys, const float* u, int B, float* logp,
                                     float* grad, gl_deflection defl, void* stream);

/* Multi-start MAP (Sec. 3.1: every particle descends independently): n_steps
 * of Adam (Kingma & Ba 2015) on each row of u, maximising log p~(u), in place.
 *   m, v     Adam moments [B][P]: zeros for a fresh start, or the state a
 *            previous call left (with t0 = the steps already taken);
 *   lr, beta1, beta2, eps   Adam's hyper-parameters (the step is
 *            lr m^/(sqrt(v^) + eps));
 *   logp     [B]: log p~ at the last point evaluated (before the last update).
 * Each step is one gradient evaluation and one fused pull-back + update
 * kernel; the n_steps run as one CUDA graph launch, captured on a private
 * stream and re-captured when a pointer, n_steps, B or the deflection changes
 * (t0 and the hyper-parameters are read from device memory). Do not call
 * while the calling thread is capturing a stream. */
gl_status gl_map_adam(gl_system* sys, float* u, float* m, float* v, int B, int n_steps, int t0,
                      float lr, float beta1, float beta2, float eps, float* logp,
                      gl_deflection defl, void* stream);

/* HMC sampler (the pipeline's sampling stage, Sec. 3): B independent chains
 * on log p~(u), each transition a leapfrog trajectory of n_leapfrog steps with
 * diagonal inverse mass M^-1 and a Metropolis-Hastings accept/reject.
 * Momenta and acceptance draws come from SplitMix64 (Steele et al. 2014) used
 * as a counter-based generator: draw j of chain b in transition n takes the
 * output for state seed + ((n B + b)(2P + 2) + j) * 0x9E3779B97F4A7C15, whose
 * top 24 bits k give the uniform (k + 1/2) 2^-24; momentum k is Box-Muller on
 * draws 2k (radius) and 2k + 1 (angle), scaled by sqrt(M); draw 2P is the
 * acceptance uniform a, and the chain moves when log a < min(0, H0 - H1),
 * H = -log p~ + p^T M^-1 p / 2 (a non-finite H1 rejects). Everything stays on
 * the device: one CUDA graph per transition, no host synchronisation. */
typedef struct gl_hmc gl_hmc;

typedef struct {
  int chains;                    /* B >= 1                                    */
  int n_leapfrog;                /* leapfrog steps per transition, >= 1       */
  float step_size;               /* initial step size eps > 0                 */
  float target_accept;           /* dual-averaging target, in (0, 1)          */
  unsigned long long seed;       /* generator seed                            */
  int deflection;                /* gl_deflection of the gradient evaluations */
} gl_hmc_desc;

/* Flags of gl_hmc_run. */
enum {
  GL_HMC_ADAPT_STEP = 1,      /* dual-averaging step size (Hoffman & Gelman 2014)
                                 on the mean acceptance probability over chains */
  GL_HMC_COLLECT_MOMENTS = 2  /* accumulate per-parameter mean and variance of u
                                 over chains and transitions (mass adaptation) */
};

/* Creates a sampler at u0 (device [B][P], copied); M^-1 starts at ones.
 * Evaluates log p~ and its gradient at u0 on the stream and waits for it.
 * The sampler uses the system (and its attached surrogate) until it is
 * destroyed: destroy it first. */
gl_status gl_hmc_create(gl_system* sys, const gl_hmc_desc* desc, const float* u0,
                        gl_hmc** out, void* stream);

/* Sets M^-1 (device [P], copied). */
gl_status gl_hmc_set_inv_mass(gl_hmc* hmc, const float* inv_mass, void* stream);

/* Runs n transitions. draws (device [n][B][P], or NULL) receives theta(u) of
 * every chain after each transition; accept (device [n], or NULL) the mean
 * acceptance probability of each transition. */
gl_status gl_hmc_run(gl_hmc* hmc, int n, int flags, float* draws, float* accept, void* stream);

/* Ends adaptation (Sec. 3.3): the step size becomes the dual-averaging
 * average; if set_inv_mass, M^-1 becomes the variances collected with
 * GL_HMC_COLLECT_MOMENTS (the Gaussian fitted to those burn-in samples), and
 * the collection is cleared. A later GL_HMC_ADAPT_STEP phase restarts the
 * dual averaging from the new step size (a second burn-in that retunes the
 * step to the new mass matrix). */
gl_status gl_hmc_end_adaptation(gl_hmc* hmc, int set_inv_mass, void* stream);

/* Current state: u [B][P], log p~ [B], inv_mass [P] (device, each may be NULL)
 * and the step size (host, may be NULL; this waits for the stream). */
gl_status gl_hmc_state(gl_hmc* hmc, float* u, float* logp, float* inv_mass,
                       float* step_size_host, void* stream);

/* Frees a sampler (waits for the device). NULL is accepted. */
gl_status gl_hmc_destroy(gl_hmc* hmc);

/* Stochastic variational inference (Sec. 3.1-3.2): n_steps of AdaBelief
 * (Zhuang et al. 2020) on a full-covariance Gaussian q(u; mu, L L^T), with
 * the score-function ELBO gradient (Eqs. elbo, elbo-grad) over n_samples draws
 * per step: u_i = mu + L z_i, z_i ~ N(0, I) from the generator above (draw j
 * of sample i in step n: state seed + ((n n_samples + i) 2P + j) * gamma),
 *   ELBO = mean_i w_i,  w_i = log q(u_i) - log p~(u_i),
 *   grad = mean_i w_i grad log q(u_i),  grad_mu log q = L^-T z,
 *   grad_L log q = tril(L^-T z z^T) - diag(1/L_ii).
 * The optimised vector is phi = (mu [P], then L row-major [P][P] with its
 * diagonal stored as log L_ii); opt is AdaBelief's state [2 (P + P P)] (m then
 * s; zeros for a fresh start) and t0 the steps already taken; elbo (device
 * [n_steps], or NULL) receives each step's ELBO estimate. Only log p~ is
 * evaluated (no gradient): the score-function estimator needs none. Samples
 * whose log p~ is not finite are left out of the means. One CUDA graph per
 * step, captured on a private stream (re-captured when a pointer, n_samples
 * or the deflection changes). */
gl_status gl_svi_adabelief(gl_system* sys, float* phi, float* opt, int n_samples, int n_steps,
                           int t0, float lr, float beta1, float beta2, float eps,
                           unsigned long long seed, float* elbo, gl_deflection defl,
                           void* stream);

/* gl_svi_adabelief with a choice of gradient estimator. GL_SVI_SCORE is the
 * score-function form above, as Eq. elbo-grad prints it. GL_SVI_PATHWISE is
 * the reparameterisation gradient that automatic differentiation of the
 * sampled ELBO gives (Sec. 3.2 says the gradient is taken that way): with
 * u_i = mu + L z_i, log q(u_i) does not depend on mu, so
 *   grad_mu = -mean_i g_i,  grad_L = -tril(mean_i g_i z_i^T) - diag(1/L_jj),
 * g_i = grad_u log p~(u_i) from the fused gradient kernel and the bijection's
 * pull-back. It costs a log p + gradient evaluation per draw instead of a
 * log p, and its variance is far lower: on narrow lensing posteriors the
 * score-function estimate is mostly noise. Both have the same expectation,
 * and both report the same ELBO estimate. Any other estimator value is
 * GL_EINVAL. */
#define GL_SVI_SCORE 0
#define GL_SVI_PATHWISE 1
gl_status gl_svi_adabelief_ex(gl_system* sys, float* phi, float* opt, int n_samples, int n_steps,
                              int t0, float lr, float beta1, float beta2, float eps,
                              unsigned long long seed, float* elbo, gl_deflection defl,
                              int estimator, void* stream);

/* "Backward" intensity modelling (Sec. 3: the light intensities solved by
 * linear inversion instead of sampled). The model image is linear in the
 * Sersic intensities, m = sum_k I_k M_k, so per row the intensities that
 * maximise the likelihood solve (M^T W M) I = M^T W d, W = diag(sigma^-2)
 * (compensated FP32 sums per thread, FP64 across threads, Cholesky in FP64).
 * The paper gives no formula; this
 * library takes:
 *   theta      [B][P]; its intensity entries (index 8 + 7c + 6 of light
 *              component c, lens lights first) are ignored;
 *   logp       [B]: the log-likelihood at the solved intensities plus the log
 *              prior of the other parameters (intensities carry no prior and
 *              may come out negative);
 *   grad       [B][P]: d logp / d theta of the other parameters, the ordinary
 *              gradient at the solved intensities (the likelihood's intensity
 *              derivative vanishes there), and 0 in the intensity entries;
 *   intensity  [B][n_lens_light + n_source] or NULL: the solved intensities.
 * A row whose normal matrix is singular (a component with no light in the
 * image) gets all intensities 0. Cost per row: n_lens_light + n_source image
 * renders and one fused log p + gradient evaluation. */
gl_status gl_logp_grad_backward(gl_system* sys, const float* theta, int B, float* logp,
                                float* grad, float* intensity, gl_deflection defl, void* stream);

/* Throughput of the pipes that bound the lens kernels, measured on the
 * current device in operations per SM per SM clock (the roofline's r_FP32
 * and r_MUFU): fp32 with scalar FMAs, fp32x2 with paired (two-lane) FMAs, an
 * FMA counting one operation per lane; mufu with ex2 / lg2 approximations.
 * One CTA per SM, independent dependency chains, clock64 timing; runs about
 * 10 ms on the device, synchronously. GL_EINVAL for NULL outputs. */
gl_status gl_unit_rates(double* fp32, double* fp32x2, double* mufu);

/* Last failure message on this host thread ("" if none). */
const char* gl_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GL_H */
