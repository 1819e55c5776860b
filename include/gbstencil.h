/*
 * gbstencil -- explicit finite-difference stencil sweeps on GB300 (sm_103a).
 *
 * C ABI of the library.  Every entry point is `extern "C"`, takes plain
 * pointers and sizes, returns a gbst_status (0 = OK, < 0 = error), never
 * aborts and never prints (unless the environment variable GBST_LOG=1).
 * After an error, stencil_last_error() returns a message for the calling
 * thread.
 *
 * What is computed (Bisbas et al., "A shared compilation stack for
 * distributed-memory parallelism in stencil DSLs", ASPLOS 2024):
 *  - Section 2: a grid point at step n+1 is a function of its neighbours at
 *    earlier steps; the halo is read-only and as wide as the stencil radius.
 *  - Section 5.1 (Devito heat listing): forward Euler for u_t = alpha Lap(u):
 *        u^{n+1} = u^n + a L(u^n),  a = alpha dt / h^2.
 *  - Section 6.1: heat diffusion and the isotropic acoustic wave equation,
 *    2D and 3D, space orders 2/4/8; the wave is second order in time:
 *        u^{n+1} = 2 u^n - u^{n-1} + kappa L(u^n),  kappa = c^2 dt^2 / h^2.
 *  - L(u)_p = sum over axes, sum over m=-r..r of w_|m| u_{p + m e_axis},
 *    r = space_order / 2, w the central second-derivative weights of accuracy
 *    space_order (or caller-supplied weights).
 *  - Section 4.2 (dmp.swap): in decomposition mode the domain is split into
 *    equal subdomains, each with its own halo; before every sweep each
 *    subdomain receives its neighbours' boundary slabs into its halo.
 *
 * Threading: handles are not thread-safe; distinct handles may be used from
 * distinct threads.  Ownership: the library owns all device memory it
 * allocates (through the optional allocator, else cudaMalloc) and frees it in
 * the matching destroy call; caller buffers are only read or written during
 * the call that receives them (asynchronously on the handle's stream where
 * stated).
 */
#ifndef GBSTENCIL_H
#define GBSTENCIL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBST_OK = 0,
    GBST_EINVAL = -1,     /* invalid argument (message says which) */
    GBST_ENOMEM = -2,     /* device or host allocation failed */
    GBST_ECUDA = -3,      /* a CUDA call failed; the handle is poisoned */
    GBST_ETIMEOUT = -4,   /* a bounded device-side wait expired; the handle is poisoned */
    GBST_EUNSTABLE = -5,  /* time step above the von Neumann limit, or NaN/Inf detected */
    GBST_ESTATE = -6,     /* call not valid in the handle's current state */
    GBST_ENOTSUP = -7     /* combination not supported by the library */
} gbst_status;

enum { GBST_HEAT = 0, GBST_WAVE = 1 };                    /* gbst_desc.eq */
enum { GBST_BC_ZERO = 0, GBST_BC_PERIODIC = 1 };          /* gbst_desc.bc */
enum { GBST_F32 = 0, GBST_BF16 = 1, GBST_F64 = 2 };       /* storage / transfer dtypes */
enum { GBST_U = 0, GBST_U_PREV = 1, GBST_VEL = 2 };       /* fields */
enum { GBST_RED_SUM = 0, GBST_RED_L2SQ = 1, GBST_RED_MAXABS = 2, GBST_RED_ENERGY = 3 };
enum { GBST_KERNEL_AUTO = 0, GBST_KERNEL_STREAM = 1, GBST_KERNEL_SIMPLE = 2 };

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns a device pointer of at least `bytes` bytes, 256-byte aligned, or NULL;
 * release frees it.  `stream` is the handle's cudaStream_t. */
typedef struct gbst_allocator {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*release)(void *ptr, size_t bytes, void *stream, void *ctx);
    void *ctx;
} gbst_allocator;

/* Problem description.  Zero-initialise, then set the fields you need. */
typedef struct gbst_desc {
    int ndim;              /* 2 or 3 */
    int64_t dims[3];       /* interior points; dims[0] = x (fastest); dims[2] ignored for 2D */
    int space_order;       /* 2, 4 or 8 (radius r = space_order/2) */
    int eq;                /* GBST_HEAT or GBST_WAVE */
    int bc;                /* GBST_BC_ZERO (Dirichlet ghosts, the paper's read-only halo)
                              or GBST_BC_PERIODIC (test mode, for closed forms) */
    int storage;           /* GBST_F32 or GBST_BF16 (fields stored in BF16, FP32 arithmetic) */
    double h;              /* grid spacing */
    double dt;             /* time step */
    double alpha;          /* heat: diffusivity, a = alpha dt / h^2 */
    const double *coeffs;  /* optional r+1 one-sided weights w_0..w_r; NULL = standard central.
                              Weights that are integers over a common denominator D <= 10^6
                              (the central ones: D = 1, 12, 5040 for orders 2, 4, 8) are
                              applied as those integers, exact in FP32, with 1/D in the
                              coefficient (heat: a / D; wave: the weighted sum times 1/D
                              before kappa), so the FP32 star of a constant is exactly 0 */
    int decomp[3];         /* subdomains per axis ({0,0,0} or {1,1,1} = none; e.g. {2,2,2}) */
    int allow_unstable;    /* 0: reject time steps above the von Neumann limit (GBST_EUNSTABLE) */
    int kernel;            /* GBST_KERNEL_AUTO / STREAM (TMA 2.5D) / SIMPLE (one thread per point) */
    int tile;              /* 0 = cached autotuned plan, else the default; k > 0 = kernel variant k-1 */
    int use_graph;         /* 0: direct launches; 1: capture the step loop as a CUDA graph */
    void *stream;          /* cudaStream_t for all work; NULL = legacy default stream */
    const gbst_allocator *allocator; /* NULL = cudaMalloc / cudaFree */
    int temporal_block;    /* heat, FP32, 3D, zero ghosts, space order 2 or 4 only:
                              0 = automatic (single steps by default; stencil_tune may pick
                              two-step blocking), 1 = off, 2 = two time steps per pass over
                              memory (overlapped temporal blocking; results are bit-identical to
                              single steps; afterwards GBST_U_PREV does not hold u^{n-1}).  With a
                              decomposition the ghost regions are 2r deep and every two-step
                              sweep is preceded by a three-phase exchange (x, y, then z faces
                              2r deep, the later phases spanning the earlier phases' ghosts, so
                              that the edge regions two steps reach are filled too) */
} gbst_desc;

typedef struct gbst_grid_s *gbst_handle;

/* Version of this ABI (major*10000 + minor*100 + patch). */
int gbst_version(void);

/* Message of the last failed call on this thread ("" if none).  Never NULL. */
const char *stencil_last_error(void);

/* Central second-derivative weights w_0..w_r of accuracy `space_order` (2..16,
 * even) written to out[0..r].  Defined by sum_m w_m m^k = 2[k==2], k <= 2r
 * (the standard finite-difference scheme; the paper, Section 6.1, names only
 * the orders).  Host only. */
gbst_status stencil_fd_weights(int space_order, double *out);

/* Create a grid: allocates the fields (interior + r-wide zero halo per axis,
 * x pitch padded to 128 bytes) on the current CUDA device, sets u = u_prev = 0,
 * kappa = 0.  `out` receives the handle.  Errors: EINVAL (bad desc), ENOMEM,
 * EUNSTABLE (heat with a*ndim*S > 2 and allow_unstable == 0). */
gbst_status stencil_create(const gbst_desc *desc, gbst_handle *out);

/* Copy a dense interior field in (x fastest, dims[0]*dims[1]*dims[2] values of
 * `src_dtype`; GBST_F32, GBST_F64 or GBST_BF16).  src_on_device selects a
 * device or host pointer (host memory may be pageable or pinned).  Values are
 * rounded to the storage type (round-to-nearest-even).  For GBST_VEL the values
 * are wave speeds c and the library stores kappa = c^2 dt^2 / h^2 (FP32); for
 * the wave, a VEL whose kappa exceeds the stability limit returns EUNSTABLE
 * unless allow_unstable.  Synchronous with respect to the caller's buffer. */
gbst_status stencil_set_field(gbst_handle h, int field, const void *src, int src_dtype,
                              int src_on_device);

/* Copy a dense interior field out (same layout rules; GBST_VEL returns kappa).
 * Synchronises the handle's stream and reports any deferred device error.
 * Host buffers move by the copy engines through a device staging buffer
 * (allocated from the handle's allocator for the duration of the copy). */
gbst_status stencil_get_field(gbst_handle h, int field, void *dst, int dst_dtype,
                              int dst_on_device);

/* Asynchronous forms of stencil_set_field / stencil_get_field for GBST_U and
 * GBST_U_PREV: the copy is enqueued on the handle's stream and the call returns
 * at once.  The buffer must be device memory or page-locked host memory (else
 * EINVAL), and must stay valid, and unmodified / unread by the caller, until
 * the stream reaches the copy (e.g. stencil_sync).  Host data in the storage
 * type of a grid (or batch member) without decomposition moves by one pitched
 * copy straight between the dense host array and the padded field; otherwise
 * through a staging buffer and a conversion kernel, the buffer released in
 * stream order, which needs a stream-ordered allocator (e.g. a framework's
 * caching allocator; with the default cudaMalloc / cudaFree the release
 * synchronises the device).  Device errors
 * surface at the next synchronising call.  No counterpart in the paper: lets a
 * caller overlap one grid's transfers with another grid's sweeps. */
gbst_status stencil_set_field_async(gbst_handle h, int field, const void *src, int src_dtype,
                                    int src_on_device);
gbst_status stencil_get_field_async(gbst_handle h, int field, void *dst, int dst_dtype,
                                    int dst_on_device);

/* Wave only: a Ricker point source at interior index idx = (i, j, k) (k ignored
 * in 2D).  At the end of step n the value amp * c_s^2 dt^2 * R(n dt) is added to
 * u^{n+1} at idx, R(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2).
 * f0 <= 0 removes the source. */
gbst_status stencil_set_source(gbst_handle h, const int64_t idx[3], double f0_hz, double t0_s,
                               double amp);

/* Advance nsteps time steps, asynchronously on the handle's stream.  Each step
 * is: [decomposition/periodic: halo swap kernel] + one sweep kernel (a two-step
 * plan: [the three-phase deep exchange] + one sweep per two steps).  Device
 * errors are reported by the next synchronising call. */
gbst_status stencil_run(gbst_handle h, int64_t nsteps);

/* Wait for the handle's stream; returns ETIMEOUT/ECUDA if a kernel failed. */
gbst_status stencil_sync(gbst_handle h);

/* Current step counter n (the field GBST_U holds u^n) and its setter (used to
 * resume from a checkpoint made with get_field of U and U_PREV). */
gbst_status stencil_get_step(gbst_handle h, int64_t *step);
gbst_status stencil_set_step(gbst_handle h, int64_t step);

/* FP64 reduction over the interior of the stored fields, synchronous:
 *   GBST_RED_SUM    sum_p u_p            (heat mass)
 *   GBST_RED_L2SQ   sum_p u_p^2
 *   GBST_RED_MAXABS max_p |u_p|
 *   GBST_RED_ENERGY wave only: E = sum_p (u_p - v_p)^2 / kappa_p + sum_p u_p (A v)_p,
 *                   u = u^n, v = u^{n-1}, A = -L (zero halo): the leapfrog discrete
 *                   energy, conserved by the source-free scheme.
 * Returns EUNSTABLE (with *out set) if the result is NaN or Inf. */
gbst_status stencil_reduce_f64(gbst_handle h, int kind, double *out);

/* Describe the execution plan chosen for the sweep kernel (NUL-terminated
 * text into buf of size len). */
gbst_status stencil_describe(gbst_handle h, char *buf, size_t len);

/* Destroy the handle and free its device memory (synchronises first). */
gbst_status stencil_destroy(gbst_handle h);

/* Device time of the last sweep kernel launches: the sum over the launches of
 * the last stencil_run call, measured with CUDA events on the handle's stream
 * when `profile` was enabled with stencil_set_profile.  ms receives the total,
 * launches the count.  Synchronises. */
gbst_status stencil_set_profile(gbst_handle h, int enable);
gbst_status stencil_last_kernel_time(gbst_handle h, double *ms, int64_t *launches);

/* ---- batches ---------------------------------------------------------------
 * A batch handle holds n independent grids advanced together: every sweep
 * launch (or, in persistent mode, the one launch of a whole run) covers the
 * tiles of all of them.  All members share ndim, space_order, eq, storage,
 * coefficients and kernel choice, have zero halos and no decomposition; each
 * has its own dims, h, dt and alpha (descs[i]), its own fields and source.
 * stream and allocator are taken from descs[0].  stencil_run, stencil_sync,
 * stencil_tune, stencil_set_plan, stencil_describe, stencil_destroy,
 * stencil_reduce_f64 (over all members) and the step counter apply to the whole
 * batch; the functions below address one member, 0 <= grid < n.
 * (Not in the paper: the batching of many small problems into one launch.) */
gbst_status stencil_batch_create(const gbst_desc *descs, int n, gbst_handle *out);
gbst_status stencil_batch_size(gbst_handle h, int *n);

/* A coupled system of nfields (2..4) FP32 fields on one 3D grid with zero
 * halos, advanced by fused multi-field sweeps (several stencils in one pass
 * over memory; a synthetic stand-in for the multi-stencil regions of the
 * paper's Section 6.2):
 *     u_k^{n+1} = u_k^n + sum_j A[k][j] L(u_j^n),   A = coupling (row-major).
 * desc: eq = GBST_HEAT, storage = GBST_F32, ndim = 3, bc = GBST_BC_ZERO, no
 * decomposition; alpha, dt and h are not used (A holds the coefficients).
 * The handle is a batch whose members are the fields: stencil_batch_set_field
 * / _get_field / _reduce_f64 with grid = k address field k (GBST_U); run,
 * sync, tune, set_plan, describe apply to the whole system.  EUNSTABLE unless
 * |I + lambda A|_2 <= 1 for every symbol value lambda in [-ndim S, 0] of the
 * stencil (the exact von Neumann condition for symmetric A) or
 * allow_unstable.  No temporal blocking, no persistent mode. */
gbst_status stencil_system_create(const gbst_desc *desc, int nfields, const double *coupling,
                                  gbst_handle *out);
gbst_status stencil_batch_set_field(gbst_handle h, int grid, int field, const void *src, int src_dtype,
                                    int src_on_device);
gbst_status stencil_batch_get_field(gbst_handle h, int grid, int field, void *dst, int dst_dtype,
                                    int dst_on_device);
gbst_status stencil_batch_set_source(gbst_handle h, int grid, const int64_t idx[3], double f0_hz, double t0_s,
                                     double amp);
gbst_status stencil_batch_reduce_f64(gbst_handle h, int grid, int kind, double *out);

/* Persistent mode (enable != 0): stencil_run(n) issues ONE cooperative launch
 * that performs all n steps, with a grid-wide barrier between steps (every
 * CTA resident; the barrier wait is bounded and reports GBST_ETIMEOUT at the
 * next synchronising call if it expires).  Requires the streaming kernel and
 * no halo exchanges (no decomposition, zero halos).  With use_graph the launch
 * is captured as a single graph node. */
gbst_status stencil_set_persistent(gbst_handle h, int enable);

/* Test hook: make every grid barrier of persistent launches wait for `extra`
 * arrivals that never come, so the bounded wait expires (0 restores normal use). */
gbst_status stencil_debug_barrier_extra(gbst_handle h, unsigned int extra);

/* ---- learned closure (not in the paper) ---------------------------------------
 * A 3-layer 3x3x3 convolutional network (4 -> 16 -> 16 -> 1, GELU, zero
 * padding) that corrects a 2x-coarsened acoustic-wave step: with u+ the plain
 * coarse step, u^n the current level and c_n = c / c_ref,
 *   x = s (u+, u^n, c_n^2 u+, c_n^2 u^n),  o = net(x),  u+ <- u+ + o / t
 * (s = in_scale; t = the output scale, closure_set_out_scale, default s).
 * BF16 weights and activations, FP32 accumulation on the tensor cores, FP32
 * master weights and Adam (beta 0.9/0.999, eps 1e-8).  cin is 4 (the inputs
 * above) or 8 (FP32 stencil features, closure_set_features); hidden is 16.  Parameters are a flat
 * FP32 vector in the order w1[16][cin][3][3][3], b1[16], w2[16][16][3][3][3],
 * b2[16], w3[1][16][3][3][3], b3[1] (zero after creation).  Device arrays are
 * dense FP32, x fastest, nx*ny*nz <= max_points.  All calls are ordered on
 * `stream`; loss_grad and the parameter copies synchronise it. */
typedef struct gbst_closure_s *gbst_closure;
gbst_status closure_create(int cin, int hidden, int64_t max_points, double in_scale, void *stream,
                           const gbst_allocator *allocator, gbst_closure *out);
gbst_status closure_destroy(gbst_closure c);
gbst_status closure_param_count(gbst_closure c, int64_t *n);
gbst_status closure_set_params(gbst_closure c, const float *host, int64_t n);
gbst_status closure_get_params(gbst_closure c, float *host, int64_t n);
/* correction = o / t for the given coarse fields (device). */
gbst_status closure_forward(gbst_closure c, const float *u_plus, const float *u_n, const float *c_norm,
                            int64_t nx, int64_t ny, int64_t nz, float *correction);
/* loss = mean (o - t (u_ref - u+))^2 and its gradient w.r.t. every parameter
 * (kept on the device; closure_get_grads copies it out). */
gbst_status closure_loss_grad(gbst_closure c, const float *u_plus, const float *u_n, const float *c_norm,
                              const float *u_ref, int64_t nx, int64_t ny, int64_t nz, double *loss);
gbst_status closure_get_grads(gbst_closure c, float *host, int64_t n);
/* One Adam update of the parameters with the last gradient. */
gbst_status closure_adam_step(gbst_closure c, double lr);
/* Output scale t (default in_scale): the loss compares o with t (u_ref - u+) and
 * the correction added to u+ is o / t, so the network works with O(1) targets
 * even when one-step corrections are small next to the field. */
gbst_status closure_set_out_scale(gbst_closure c, double out_scale);
/* Factor w > 0 on the loss and its gradient in later closure_loss_grad calls
 * (default 1), e.g. 1 / mean(target^2) to give every sample the same weight. */
gbst_status closure_set_loss_weight(gbst_closure c, double w);
/* freeze != 0: Adam leaves the three bias vectors unchanged (with zero biases a
 * zero field then gets a zero correction). */
gbst_status closure_freeze_biases(gbst_closure c, int freeze);
/* Convolution kernels: impl 0 (default) = tcgen05 MMAs with accumulators in
 * tensor memory, operands staged by TMA, the one-channel last layer in
 * tap-split form (the tensor cores contract channels and x taps per input row,
 * the CUDA cores add the nine y/z taps); impl 1 = the mma.sync kernels (kept
 * as an independent cross-check of the same arithmetic); impl 2 = tcgen05 for
 * the two hidden layers, the one-channel last layer on the CUDA cores; impl 3 =
 * tcgen05 with the last layer computed like the hidden ones (its single output
 * channel padded to the MMA's N).  A bounded wait that
 * expires in a tcgen05 kernel is reported as GBST_ETIMEOUT by the next
 * closure_loss_grad / closure_get_params / closure_get_grads. */
gbst_status closure_set_conv_impl(gbst_closure c, int impl);

/* Per-parameter mask of closure_adam_step (host array of n = parameter count
 * bytes, non-zero = the parameter trains; NULL: every parameter trains, the
 * default).  Combines with closure_freeze_biases.  A layer whose weights and
 * biases are all masked out gets no weight gradient from closure_loss_grad and
 * closure_backward (its entries of the gradient are left as they were, zero
 * unless accumulating); the data gradient still passes through it.  Synchronises
 * the stream. */
gbst_status closure_set_trainable(gbst_closure c, const unsigned char *mask, int64_t n);
/* Feature inputs (closures created with cin = 8; none of this is in the paper).
 * The network's 8 input channels are x_k = scales[k] f_k with, for u+ the plain
 * coarse step, u^n the current level and cn2 = c_n^2,
 *   f0 = u+, f1 = u^n, f2 = cn2 u+, f3 = cn2 u^n,
 *   f4 = cn2 sum_a delta_a^6 u^n          (delta^6 = (1, -6, 15, -20, 15, -6, 1) per axis),
 *   f5 = cn2 L(cn2 L u^n),  f6 = sum_a D_a(cn2) D_a(u^n),  f7 = (sum_a |D_a cn2|) L u^n,
 * L the central star of space_order (2, 4 or 8, default 4), D_a the central
 * difference, zero outside the grid; computed in FP32, then rounded to BF16.
 * f4 and f5 are, up to the constants kappa_ref / 90 and kappa_ref^2 / 12, the
 * leading one-step defects of the order-4 leapfrog scheme (its spatial
 * truncation and its dt^4 u_tttt / 12 term); f6, f7 couple the field to velocity
 * jumps.  Every channel vanishes with the field.  n must be 8. */
gbst_status closure_set_features(gbst_closure c, int space_order, const double *scales, int n);
/* The unscaled FP32 features f0..f7 of (u_plus, u_n, c_norm) into out, channel-major
 * (out + k * nx*ny*nz); device arrays; asynchronous on the closure's stream. */
gbst_status closure_feature_values(gbst_closure c, const float *u_plus, const float *u_n, const float *c_norm,
                                   int64_t nx, int64_t ny, int64_t nz, float *out);
/* The activation of the closure's hidden layers, y[i] = GELU(x[i]) = x[i] Phi(x[i])
 * for i < n, as the forward convolutions evaluate it (device arrays, FP32, y may
 * equal x; asynchronous on `stream`, a cudaStream_t or null).  Phi comes from the
 * erfc approximation of Abramowitz & Stegun 7.1.26; the result is within
 * 1.8e-7 max(1, |x|) of the exact GELU.  GBST_EINVAL for null arrays or n < 0. */
gbst_status closure_gelu(const float *x, float *y, int64_t n, void *stream);
/* Backward pass of one corrected step (closures with cin = 8), for training
 * through rollouts.  The corrected step is u^{n+1} = u+ + correction(u+, u^n).
 * Given grad_out = dLoss/du^{n+1} (dense device FP32), adds dLoss/d(parameters)
 * into the closure's gradient (zeroed first unless accumulate) and writes the
 * cotangents of the step's inputs: grad_up = dLoss/du+ (grad_out plus the path
 * through the network and its features) and grad_un = dLoss/du^n.  grad_up must
 * not alias grad_out.  Asynchronous on the closure's stream (a bounded wait that
 * expires is reported by the next closure_loss_grad / closure_get_params /
 * closure_get_grads). */
gbst_status closure_backward(gbst_closure c, const float *u_plus, const float *u_n, const float *c_norm,
                             int64_t nx, int64_t ny, int64_t nz, const float *grad_out, float *grad_up,
                             float *grad_un, int accumulate);
/* Transpose of one source-free leapfrog step (Section 6.1's scheme) on dense
 * FP32 device arrays [nz][ny][nx] (x fastest) with zero ghosts, used to train a
 * closure through whole coarse-grid rollouts.  The step maps (u^n, u^{n-1}) to
 * (u^{n+1}, u^n) with u^{n+1} = 2 u^n - u^{n-1} + kappa L u^n (L the central
 * star of space_order 2, 4 or 8, unit spacing; kappa per point).  Given the
 * cotangents lam_next of u^{n+1} and lam_cur of u^n it writes
 *     lam_cur  <- lam_cur + 2 lam_next + L(kappa lam_next)    (L is symmetric)
 *     lam_prev <- -lam_next                                    (if lam_prev != NULL)
 * FP32 arithmetic.  Asynchronous on `stream` (a cudaStream_t, NULL = legacy
 * default); the caller owns every array; lam_cur must not alias lam_next. */
gbst_status stencil_wave_adjoint_dense(int space_order, int64_t nx, int64_t ny, int64_t nz, const float *kappa,
                                       const float *lam_next, float *lam_cur, float *lam_prev, void *stream);

/* Attach a closure to a single (undecomposed) 3D wave grid: from then on every
 * step of stencil_run is the plain sweep followed by u^{n+1} += closure
 * correction (c_ref normalises the velocity, c_norm = c / c_ref).  NULL detaches. */
gbst_status stencil_attach_closure(gbst_handle h, gbst_closure c, double c_ref);

/* Gradient of a rollout loss of the closure attached to h (which must have
 * feature inputs, cin = 8), by backpropagation through the coarse time steps.
 * From the levels u^{n0} = u_cur and u^{n0-1} = u_prev (dense device FP32, the
 * grid's interior) at step index n0 = step0, the grid takes nsteps corrected
 * steps (sweep with its source, then u^{n+1} = u+ + correction) and
 *     loss = (1 / nsteps) sum_j |u^{n0+j+1} - refs[j]|^2 / |refs[j]|^2
 * (refs: a host array of nsteps dense device fields).  The parameters' gradient
 * of this loss replaces the closure's gradient (closure_get_grads, then
 * closure_adam_step); the backward pass uses closure_backward and the transpose
 * of the leapfrog step (stencil_wave_adjoint_dense).  The grid is left at step
 * n0 + nsteps.  Synchronises the grid's stream; *loss receives the loss.
 * Work buffers of 3 nsteps + 6 dense fields are allocated on the first call
 * (through the grid's allocator) and kept. */
gbst_status stencil_closure_rollout_grad(gbst_handle h, const float *u_cur, const float *u_prev, int64_t step0,
                                         const float *const *refs, int nsteps, double *loss);

/* Every stride-th interior point (0, stride, 2 stride, .. along each axis) of a
 * field into a dense FP32 device array of ceil(dims/stride) points (injection
 * restriction of a fine grid onto a 2x-coarser one when stride = 2). */
gbst_status stencil_get_field_strided(gbst_handle h, int field, float *dst_device, int stride);

/* Execution plan of the streaming sweep.  variant: index into the kernel
 * table (stencil_variant_count / stencil_variant_info; -1 = the default for
 * this grid); txt: 0, or the variant's own threads along x of a tile (the tile
 * shape is part of the variant; any other value is EINVAL); zchunks: chunks of
 * the streamed axis per tile column (0 = cost model); ctas: CTAs launched (0 =
 * all that are resident).  Synchronises; invalidates captured graphs. */
gbst_status stencil_set_plan(gbst_handle h, int variant, int txt, int zchunks, int ctas);

/* Work assignment of the streaming sweep's launches (the plan's work units
 * are (tile, z-range) pieces in list order).  dynamic = 0: unit i goes to CTA
 * i mod grid size; 1: every CTA draws its next unit from a global counter of
 * the handle, so that the units in flight stay a contiguous window of the list
 * (neighbouring tiles share their halo planes in L2, and the load balances
 * itself); -1: the library's default (dynamic).  Results do not depend on it:
 * each unit writes its own output points.  EINVAL for other values.
 * Synchronises; invalidates captured graphs.  The autotuner tries both. */
gbst_status stencil_set_schedule(gbst_handle h, int dynamic);

/* Overlap of the halo exchange with the sweep (decomposition mode, Section 4.2's
 * dmp.swap; and the periodic wrap): each step copies the faces on a second
 * stream while the work units whose boxes read no exchanged ghost cell sweep,
 * then sweeps the remaining units (communication-computation overlap, which
 * Section 4.2 lists as a limitation of its dmp design).  enable = 1 on, 0 off (copies, then one sweep), -1 the library's
 * default (off: on one device the copies are a small part of a step and the
 * split sweep costs more than it hides).  Single-step streaming plans only;
 * results are the same bits either way; with the overlap on, the autotuner
 * keeps to plans that can split.  EINVAL for other values.  Synchronises;
 * invalidates captured graphs. */
gbst_status stencil_set_overlap(gbst_handle h, int enable);

/* Autotuner: times every applicable (kernel variant, z-chunking)
 * on the handle's own fields with `reps` launches each (CUDA events on the
 * handle's stream), keeps the fastest and caches it per shape class -- in the
 * process, and appended to the file named by the environment variable
 * GBST_TUNE_CACHE, which stencil_create reads.  The fields are left unchanged.
 * report (optional, len bytes) receives a JSON summary of the candidates. */
gbst_status stencil_tune(gbst_handle h, int reps, char *report, size_t len);

/* Number of compiled streaming-kernel variants, and a JSON description of one. */
int stencil_variant_count(void);
gbst_status stencil_variant_info(int i, char *buf, size_t len);

/* FP64 reduction of a dense device array that allocates no device memory.
 * The paper has no counterpart; this serves callers that cannot allocate
 * device memory when they need the reduction -- applications whose device
 * memory is all owned by their own pool, and latency-critical loops that must
 * not call cudaMalloc/cudaFree because those can synchronise the device.
 *   x      device pointer to n values of dtype GBST_F32, GBST_F64 or GBST_BF16
 *   kind   GBST_RED_SUM, GBST_RED_L2SQ or GBST_RED_MAXABS (as stencil_reduce_f64)
 *   out    device pointer to one double, written asynchronously on `stream`
 *          (a cudaStream_t; NULL = legacy default stream); synchronise before reading
 * The per-block partial sums go to a fixed 128 KB array inside the library's
 * device image (16384 doubles, 256-byte aligned), which every GPU that loads the
 * library keeps until the process exits.  n may be at most 2^30 (16384 blocks of
 * 65536 values); larger n returns GBST_EINVAL.  The first call in each CUDA
 * context (the current device's primary context, unless the caller made another
 * one current) looks up the array's device address with that context current and
 * caches it for that context; make that first call outside any stream capture.
 * Errors are reported with the entry point's name; an error left pending by an
 * earlier, unrelated launch is cleared, not reported.  All calls share the one array and it keeps
 * the last call's contents; every call writes all the partials it reads, so no
 * clearing is needed, but calls that overlap on the GPU (different streams,
 * no ordering between them) race on it.  No cudaMalloc, cudaFree or allocating
 * library routine is called. */
gbst_status gbst_reduce_dense_f64_noalloc(const void *x, int dtype, int64_t n, int kind, double *out,
                                          void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GBSTENCIL_H */
