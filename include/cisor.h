/*
 * cisor.h -- C ABI of the GB300 (sm_103a) hot path of CISOR.
 *
 * CISOR (Ma, Mansour, Liu, Boufounos, Kamilov, "Accelerated Image
 * Reconstruction for Nonlinear Diffractive Imaging", arXiv:1708.01663)
 * estimates a permittivity contrast f from scattered fields
 *     y_t = H diag(u_t) f + e_t,     u_t = u_in,t + G diag(f) u_t      (Sec. II, Eqs. 2-3)
 * by relaxed FISTA (Sec. III-A, Eqs. 9-11) on D(f) + R(f) (Eqs. 6-8), with
 * the gradient of D from the adjoint-state formula of Prop. 1 (Eqs. 12-13).
 *
 * Conventions for every entry point:
 *  - complex arrays are interleaved complex64 (float re, float im), row-major
 *    with the x index fastest; N = n^dim pixels; fields are transmitter-major
 *    [T, N] ([T, n, n] in 2D, [T, n, n, n] in 3D).  For a vectorial geometry
 *    every field written [T, N] below is [T, 3, N] (E^(1), E^(2), E^(3)) and H
 *    is [M, 3N]; f, gradients and prox arrays stay [N];
 *  - array arguments may be device or host pointers: inputs are copied into
 *    the context's device buffers and results out of them with
 *    cudaMemcpyDefault (unified addressing); a call that writes host memory
 *    returns after the data is there;
 *  - the caller owns every array it passes; the context owns its tables
 *    (G spectrum, H, incident fields) and all workspace;
 *  - work is ordered after prior work on the stream given to cisor_create,
 *    and later work on that stream is ordered after it; host scalar outputs
 *    (D, solve info) synchronise that stream;
 *  - no C++ exception crosses this ABI; on error the status is returned and
 *    cisor_last_error() describes it (thread-local).  A CUDA error leaves the
 *    context unusable (destroy it).
 * Lengths are in any unit shared by delta, wavelength and the positions.
 */
#ifndef CISOR_H
#define CISOR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CISOR_OK = 0,
  CISOR_ERR_INVALID_ARG = 1,   /* bad size, null pointer, unsupported grid */
  CISOR_ERR_NOT_CONVERGED = 2, /* a field solve hit max_iter; outputs still written */
  CISOR_ERR_BREAKDOWN = 3,     /* a Krylov scalar vanished; outputs still written */
  CISOR_ERR_OOM = 4,           /* device allocation failed */
  CISOR_ERR_CUDA = 5           /* other CUDA error */
} cisor_status;
/* The sensing GEMMs (cisor_sense, cisor_sense_adjoint and every call that
 * forms y, w or the gradient) run on the tensor cores when T <= 128 and M and
 * the field length are even; their waits on the tensor cores are bounded.  A
 * wait that gives up leaves a flag that the context reads without
 * synchronising: the call that made it returns CISOR_ERR_CUDA if it had
 * already waited for its stream (host outputs), else the next call on the
 * context that does; the outputs since are invalid, the context stays usable. */

typedef struct cisor_ctx cisor_ctx;

/* Geometry of one imaging set-up (Sec. II and Appendix A, grid).
 * Pixel l = 1..n of each axis sits at (l - n/2 - 0.5) * delta.  Transmitters
 * are plane waves exp(j k_b d_t . r) (d_t = (cos a_t, sin a_t) in 2D, a unit
 * vector in 3D) or, with tx_kind = 1, unit point (3D) / line (2D) sources at
 * positions outside the grid, u_in,t(r) = g(|r - r_t|) with g of Eq. 1 (the
 * Fresnel set-ups of Sec. IV).  Receivers are points outside the grid. */
typedef struct {
  int dim;                  /* 2 or 3 (the scalar models of Eq. 1) */
  int n;                    /* grid side, 8 <= n <= 256 (2D) or 128 (3D); N = n^dim */
  double delta;             /* pixel size */
  double wavelength;        /* vacuum wavelength; k = 2 pi / wavelength */
  double eps_b;             /* background permittivity; k_b = k sqrt(eps_b) */
  int T;                    /* transmitters, 1 <= T <= 1024 */
  const double* tx_angles;  /* host; tx_kind 0: [T] angles, radians (2D) or [T, 3] unit directions (3D);
                               tx_kind 1: [T, dim] source positions, each outside the grid's bounding box */
  int M;                    /* receivers, 1 <= M */
  const double* rx_pos;     /* host [M, dim] receiver positions */
  int complex_f;            /* 0: f real (Im f is neither updated nor regularised); 1: complex f */
  int pad;                  /* FFT side P >= 2n - 1, a power of two <= 512 (2D) / 256 (3D); 0 = smallest such */
  int tx_kind;              /* 0: plane waves; 1: point / line sources */
  int vectorial;            /* 1: the 3D vectorial model of the appendix (dim 3, eps_b = 1, n <= 64):
                               fields are [T, 3, N] (E^(1), E^(2), E^(3)), tx_angles is [T, 6]
                               (unit direction, unit polarisation orthogonal to it), H is [M, 3N]
                               (z component at the receivers); 0: the scalar model */
} cisor_geometry;

/* Options of the field solves A u = u_in and A^H v = b (Eq. 13). */
typedef struct {
  double tol;     /* stop when the true relative residual ||b - A x|| / ||b|| <= tol */
  int max_iter;   /* BiCGSTAB iteration cap per transmitter */
  int x0_mode;    /* 0: cold start (u_in for A u = u_in, 0 for the adjoint); 1: x0 argument;
                     2: previous solution held by the context (cold if none) */
} cisor_solve_opts;

/* Per-call solve statistics (host struct, filled on return). */
typedef struct {
  int iters_max;        /* max BiCGSTAB iterations over transmitters (forward solve) */
  double iters_mean;
  double resid_max;     /* max true relative residual at exit */
  int n_not_converged;
  int adj_iters_max;    /* same for the adjoint solve (cisor_grad / cisor_step) */
  double adj_iters_mean;
  double adj_resid_max;
} cisor_solve_info;

/* Relaxed-FISTA state (Eqs. 9-11).  f and s are caller-owned [N] complex64
 * arrays; on entry f = f_{k-1}, s = s_k, t = t_k; on return f = f_k,
 * s = s_{k+1}, t = t_{k+1}, k incremented.  Start with f = s = f_0, t = 1, k = 1. */
typedef struct {
  void* f;
  void* s;
  double t;
  int k;
  double alpha;     /* relaxation, 0 <= alpha < 1 (0.96 in Sec. IV) */
  double gamma;     /* step size, 0 < gamma <= (1 - alpha^2) / (2 L) (Prop. 3) */
  double tau;       /* TV weight (Eq. 8) */
  int tv_iters;     /* FGP iterations of the prox */
  double lo, hi;    /* box C for Re f */
  double lo_im, hi_im; /* box C for Im f (complex_f only) */
  double D;         /* out: D(s_k) of Eq. 7 */
  int tv_kind;      /* 0: isotropic TV of Eq. 8 by FGP; 1: anisotropic TV by the parallel proximal
                       algorithm (cisor_tv_prox_aniso) */
} cisor_fista_state;

/* Build the tables of a geometry on the current CUDA device: the spectrum of
 * the circulant embedding of G (Eq. 3, FP64, then stored complex64), H (Eq. 2),
 * incident fields, and the solver workspace.  `stream` is a cudaStream_t
 * (NULL = legacy default stream).  On success *out owns all of it. */
cisor_status cisor_create(cisor_ctx** out, const cisor_geometry* geom, void* stream);

/* Free a context (NULL is a no-op). */
cisor_status cisor_destroy(cisor_ctx* ctx);

/* Grid size actually used: writes n, P, T, M, N (any pointer may be NULL). */
cisor_status cisor_sizes(const cisor_ctx* ctx, int* n, int* P, int* T, int* M, long long* N);

/* Copy out the unscaled spectrum ghat = FFT_P(c) of the circulant embedding
 * of G (Eq. 3 through Sec. III-A's FFT convolution): [P, P] complex64. */
cisor_status cisor_green_spectrum(cisor_ctx* ctx, void* ghat_out);

/* Copy out H (Eq. 2): [M, N] complex64. */
cisor_status cisor_sensing_matrix(cisor_ctx* ctx, void* H_out);

/* Copy out the incident fields u_in: [T, N] complex64. */
cisor_status cisor_incident(cisor_ctx* ctx, void* u_in_out);

/* y = A x (adjoint = 0) or y = A^H x (adjoint = 1) with A = I - G diag(f)
 * (Eq. 4), for nvec <= T vectors x, y: [nvec, N] complex64; f: [N]. */
cisor_status cisor_apply_A(cisor_ctx* ctx, const void* f, const void* x, void* y, int adjoint, int nvec);

/* Forward model (Eqs. 2-3, 13): solve A u_t = u_in,t for every transmitter,
 * then y_t = H diag(u_t) f.  u_in: [T, N] or NULL (the geometry's plane
 * waves); x0: [T, N] initial guesses (x0_mode 1) or NULL; u_out: [T, N] or
 * NULL; y_out: [T, M] or NULL.  The solution is kept for x0_mode 2. */
cisor_status cisor_forward(cisor_ctx* ctx, const void* f, const void* u_in, const void* x0, void* u_out,
                           void* y_out, const cisor_solve_opts* opts, cisor_solve_info* info);

/* Z = H diag(u_t) f for all transmitters (Eq. 5): u [T, N], Z_out [T, M]. */
cisor_status cisor_sense(cisor_ctx* ctx, const void* f, const void* u, void* Z_out);

/* z_t = H^H w_t and b_t = diag(f)^H z_t (right-hand side of Eq. 13):
 * w [T, M]; z_out, b_out [T, N] (either may be NULL). */
cisor_status cisor_sense_adjoint(cisor_ctx* ctx, const void* f, const void* w, void* z_out, void* b_out);

/* Data term and gradient (Eq. 7, Prop. 1): D = 1/2 sum_t ||H diag(u_t) f - y_t||^2
 * and g = sum_t conj(u_t) (H^H w_t + G^H v_t) with A u_t = u_in,t,
 * A^H v_t = diag(f)^H H^H w_t.  grad_out [N] complex64 receives g: its real
 * part is grad D for real f; for complex f, (Re g, Im g) are the partial
 * derivatives in (Re f, Im f).  y: [T, M]; D_out: host double (may be NULL). */
cisor_status cisor_grad(cisor_ctx* ctx, const void* f, const void* y, void* grad_out, double* D_out,
                        const cisor_solve_opts* opts, cisor_solve_info* info);

/* Forward half of cisor_grad, for reverse-mode use: solves A u_t = u_in,t
 * (Eq. 13), forms w_t = H diag(u_t) f - y_t and D (Eq. 7), and keeps f, u_t
 * and w_t in the context (the checkpoint the backward half needs; [N] and
 * [T, N] complex64).  D_out: host double (may be NULL). */
cisor_status cisor_data_term(cisor_ctx* ctx, const void* f, const void* y, double* D_out,
                             const cisor_solve_opts* opts, cisor_solve_info* info);

/* Backward half of cisor_grad (Prop. 1): from the f, u_t, w_t of the last
 * cisor_data_term on this context, solves A^H v_t = diag(f)^H H^H w_t and
 * writes g = sum_t conj(u_t) (H^H w_t + G^H v_t) to grad_out ([N] complex64).
 * Calls that only read f in between (cisor_apply_A, cisor_sense,
 * cisor_tv_prox, cisor_autotune, cisor_time_matvec) leave the checkpoint
 * intact.  CISOR_ERR_INVALID_ARG if no cisor_data_term preceded it, or if a
 * call that overwrites u_t or w_t came after it (cisor_forward, cisor_grad,
 * cisor_step, cisor_sense_adjoint, a batch solve on this context). */
cisor_status cisor_data_backward(cisor_ctx* ctx, void* grad_out, const cisor_solve_opts* opts,
                                 cisor_solve_info* info);

/* x = argmin_{x in C} 1/2 ||x - z||^2 + gamma_tau TV_iso(x) (prox of Eq. 8)
 * by `iters` FGP iterations (Beck-Teboulle, cited in Sec. III-A), dual cold
 * start; C is the box [lo, hi] for Re and, for complex_f, [lo_im, hi_im] for
 * Im (separable prox); for real f Im x = 0.  z, x: [N] complex64. */
cisor_status cisor_tv_prox(cisor_ctx* ctx, const void* z, void* x, double gamma_tau, int iters, double lo,
                           double hi, double lo_im, double hi_im);

/* As cisor_tv_prox for the anisotropic TV, sum_d sum_n |[D_d x]_n| (the
 * alternative Sec. III-A points to), by `iters` iterations of the parallel
 * Dykstra-like proximal algorithm over the 2 dim pair-difference pieces and
 * the box; dual-free, cold start. */
cisor_status cisor_tv_prox_aniso(cisor_ctx* ctx, const void* z, void* x, double gamma_tau, int iters, double lo,
                                 double hi, double lo_im, double hi_im);

/* One relaxed-FISTA iteration (Eqs. 9-11) on the state; y: [T, M] measurements.
 * Inner solves use opts (x0_mode 2 warm-starts from the previous step). */
cisor_status cisor_step(cisor_ctx* ctx, cisor_fista_state* st, const void* y, const cisor_solve_opts* opts,
                        cisor_solve_info* info);

/* Update half of cisor_step, for a gradient summed outside this context:
 * the transmitters split over several contexts (one per rank or GPU), each
 * running cisor_grad on its own transmitters, and the partial g and D summed
 * (D and g are sums over transmitters, Eq. 7 and Prop. 1).  From that sum:
 *   f_k     = prox_{gamma R}(s_k - gamma grad)    (Eq. 9; real f steps with Re grad)
 *   t_{k+1}, s_{k+1}                              (Eqs. 10-11)
 * grad: [N] complex64, Prop. 1's g summed over ALL transmitters; D: D(s_k)
 * summed likewise, stored in st->D.  State as in cisor_step.  Identical
 * inputs give identical outputs on every rank, so no broadcast follows. */
cisor_status cisor_step_update(cisor_ctx* ctx, cisor_fista_state* st, const void* grad, double D);

/* Number of CUDA kernels this context has launched since creation (kernels
 * inside replayed CUDA graphs included).  *count is a host long long. */
cisor_status cisor_launch_count(const cisor_ctx* ctx, long long* count);

/* Arithmetic resources of CUDA device `device`, for roofline figures:
 * *sm_count multiprocessors, *max_clock_khz their peak clock, *fp32_lanes
 * FP32 FMA lanes per multiprocessor (128 on compute capability 10.x and 12.x,
 * 64 on 9.0 and 8.0, else 0 = unknown), *cc compute capability x 10.  Any
 * output pointer may be NULL.  No GPU work is launched. */
cisor_status cisor_device_info(int device, int* sm_count, int* max_clock_khz, int* fp32_lanes, int* cc);

/* Self-test of the bounded waits of the tensor-core kernels (no counterpart
 * in the paper; a diagnostic): one CTA on the current device takes tensor
 * memory and waits at most `polls` (>= 1) polls on an mbarrier that it
 * completes itself (arrive = 1) or that nothing completes (arrive = 0), frees
 * the tensor memory and returns.  *completed (host) receives 1 if the wait
 * completed, 0 if it gave up.  Synchronous (legacy default stream). */
cisor_status cisor_tc_wait_selftest(int arrive, int polls, int* completed);

/* Time `reps` back-to-back batched matvecs y_t = A x_t (adjoint = 0) or
 * A^H x_t (adjoint = 1) over all T transmitters of the context's workspace
 * (the FFT-convolution kernels of the field solves, Eq. 4), with CUDA events
 * on the context's stream, after one untimed pass.  *ms_per_pass receives
 * the mean milliseconds of one pass.  f: [N] complex64, as in cisor_apply_A. */
cisor_status cisor_time_matvec(cisor_ctx* ctx, const void* f, int adjoint, int reps, double* ms_per_pass);

/* y = A x (adjoint = 0) or y = A^H x (adjoint = 1), A = I - G diag(f), for
 * nvec vectors, WITHOUT allocating device memory and without a context.  The
 * paper has no counterpart: this serves callers that cannot call cudaMalloc
 * (code inside a host framework that owns all device allocations, or code
 * that must not allocate while a CUDA graph is being captured).
 *   ghat_scaled: device [P, P] complex64, the Green spectrum divided by P*P
 *                (cisor_green_spectrum's output / (P*P));
 *   f: device [n*n]; x, y: device [nvec, n*n] complex64; 8 <= n <= 256;
 *   P a power of two in [64, 512] with P >= 2n - 1; stream: cudaStream_t of
 *   the current device (a stream of another device: CISOR_ERR_INVALID_ARG).
 * Scratch lives in one file-scope device array of 16 MiB that every GPU
 * loading the library holds until exit; calls needing more (16 bytes x 512
 * + 8 x nvec x n x P bytes) return CISOR_ERR_INVALID_ARG with a message.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and raises the convolution kernels' shared-memory
 * limit (cudaFuncSetAttribute), so make it before any stream capture.  Every call
 * shares the array: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  Each call rewrites
 * every scratch value it reads.  Asynchronous on `stream`. */
cisor_status cisor_apply_A_static(const void* ghat_scaled, const void* f, const void* x, void* y, int n, int P,
                                  int nvec, int adjoint, void* stream);

/* Autotuner of the FFT convolution's column-kernel shape and transmitter
 * chunk (cisor_set_tx_chunk): times the
 * three-stage (8 x 8 x 8 at P = 512) column kernel with 512- and 256-thread
 * CTAs (8 or 4 columns per CTA at P = 512) and, where it exists, the
 * two-stage kernel (shape code 16: one shared-memory exchange per transform;
 * 512 = 32 x 16 on 2D grids, 256 = 16 x 16 and 128 = 16 x 8 on 2D and 3D
 * grids; none at P = 64), on this context's sizes, `reps` batched matvecs
 * each with CUDA events, and keeps the fastest.  *cols_nt_out (may be NULL)
 * receives the chosen shape code (512, 256 or 16).  Results agree to FP32
 * rounding whichever shape runs. */
cisor_status cisor_autotune(cisor_ctx* ctx, int reps, int* cols_nt_out);

/* Split every FFT-convolution pass into consecutive launches of `tx_chunk`
 * transforms (transmitters; field components in the vectorial model), each
 * running the whole row / column / row chain before the next; 0 = all at
 * once.  The chunks share the start of the row-FFT intermediate, so a chunk
 * small enough for L2 keeps it there instead of writing it to HBM and reading
 * it back.  cisor_autotune measures chunks of about 16, 32 and 48 MB of
 * intermediate against no chunking and keeps the fastest (with the column
 * shape).  Results are identical whatever the chunk. */
cisor_status cisor_set_tx_chunk(cisor_ctx* ctx, int tx_chunk);

/* How a solve's BiCGSTAB iterations are driven.  device_loop = 1: the whole
 * solve is ONE CUDA-graph launch whose WHILE node repeats a captured chunk of
 * iterations until no transmitter is active (a device-side condition kernel
 * decides; the loop count is capped at max_iter / chunk + 2), so the host
 * waits once per solve.  device_loop = 0 (the default for a context): the host
 * replays a chunk graph and reads the active flags after every chunk; kernel
 * profilers list the kernels of such graphs, while they cannot look inside a
 * graph with conditional nodes (only the whole graph).  Results are identical
 * and so, measured, is the time at the benchmark sizes; where conditional
 * graph nodes are unavailable the library falls back to 0 by itself. */
cisor_status cisor_set_solve_loop(cisor_ctx* ctx, int device_loop);

/* The context's current column shape (512, 256 or 16) and transmitter chunk
 * (0 = none); either output may be NULL. */
cisor_status cisor_tuning(const cisor_ctx* ctx, int* cols_nt, int* tx_chunk);

/* Per-transmitter receiver mask (the Fresnel set-ups of Sec. IV record each
 * transmitter on a subset of the receivers): mask [T, M] bytes, non-zero =
 * active, host or device, copied into the context.  D (Eq. 7) and the
 * gradient (Prop. 1) then sum only active (t, m) pairs; inactive entries of y
 * are ignored.  mask = NULL restores all receivers. */
cisor_status cisor_set_rx_mask(cisor_ctx* ctx, const void* mask);

/* Set the column-kernel shape instead of measuring it, for reproducible
 * profiles: 512 or 256 (threads per CTA of the three-stage kernel) or 16 (the
 * two-stage kernel; P = 128 or 256, or P = 512 on a 2D grid;
 * CISOR_ERR_INVALID_ARG elsewhere).  Drops the captured solver graphs. */
cisor_status cisor_set_cols_cta(cisor_ctx* ctx, int cols_nt);

/* Per-transmitter BiCGSTAB iterations of the last forward (adjoint = 0) or
 * adjoint (adjoint = 1) solve on this context.  *count receives the number
 * of transmitters of that solve (0 if none ran); iters_out (host [count],
 * may be NULL to query the count) receives the iterations. */
cisor_status cisor_solve_iterations(const cisor_ctx* ctx, int adjoint, int* iters_out, int* count);

/* ---- Several problems of uneven size, solved together ----
 * A batch owns one context per geometry (grid side, transmitters and
 * receivers may all differ).  Its field solves advance every problem in ONE
 * CUDA-graph launch per chunk of BiCGSTAB iterations (fork to the problems'
 * streams, join back); the problems' other steps run concurrently on their
 * own streams.  Arrays are given per problem (arrays of pointers, host or
 * device).  x0_mode 0 (cold) or 2 (previous solution) only. */
typedef struct cisor_batch cisor_batch;

/* Create contexts for nprob geometries (1..256); autotune != 0 runs
 * cisor_autotune on each. */
cisor_status cisor_batch_create(cisor_batch** out, const cisor_geometry* geoms, int nprob, void* stream,
                                int autotune);
/* As cisor_set_solve_loop for a batch: device_loop = 1 (the batch default) runs each
 * solve of all problems as one graph launch with a device-side loop over
 * chunks of iterations of every problem; 0 replays a chunk graph per host
 * iteration. */
cisor_status cisor_batch_set_solve_loop(cisor_batch* batch, int device_loop);

cisor_status cisor_batch_destroy(cisor_batch* b);

/* The context of problem i (for table read-back or single-problem calls). */
cisor_status cisor_batch_context(cisor_batch* b, int i, cisor_ctx** ctx);

/* Forward solves of every problem (Eq. 13): f[i] [N_i], u_out[i] [T_i, N_i]
 * (u_out or any entry may be NULL); info: array of nprob (may be NULL). */
cisor_status cisor_batch_forward(cisor_batch* b, const void* const* f, void* const* u_out,
                                 const cisor_solve_opts* opts, cisor_solve_info* info);

/* D and gradient of every problem (Eq. 7, Prop. 1): y[i] [T_i, M_i],
 * grad_out[i] [N_i]; D_out: host array of nprob (may be NULL). */
cisor_status cisor_batch_grad(cisor_batch* b, const void* const* f, const void* const* y, void* const* grad_out,
                              double* D_out, const cisor_solve_opts* opts, cisor_solve_info* info);

/* ---- Learned warm start (not in the paper) ----
 * A Fourier neural operator predicts the scattered field u - u_in of the
 * field solve A u = u_in from (f, u_in) on 128 x 128 grids: 8 input channels
 * (Re f, Im f, Re u_in, Im u_in, the unit local propagation direction of
 * u_in from its phase gradient, x, y), 1x1 lifting to width 32, four Fourier
 * layers (16 x 32 retained modes, 1x1 skip, GELU), projection 32 -> 128 -> 2.
 * The network output e is the demodulated scattered field: u - u_in is
 * predicted as u_in * e (targets are conj(u_in) (u - u_in)).
 * Weights are FP32 masters with a BF16 copy that every kernel reads;
 * activations and accumulation are FP32.  The prediction only seeds x0 of the
 * solve (x0_mode 1), which still stops on the true residual.  Parameter
 * arrays are [cisor_fno_num_params] floats in the layout W0 [32x8], b0 [32],
 * per layer l: R_l [32 kx][16 ky][32 in][32 out] complex, W_l [32x32], b_l
 * [32]; then P1 [128x32], c1 [128], P2 [2x128], c2 [2].
 * Errors: the calls that run the network (forward, loss_grad, train_step,
 * warm_start) synchronise the network's stream before they return; if a
 * kernel's bounded wait on its tensor-core operations gave up, the call
 * returns CISOR_ERR_CUDA ("a wait on the tensor cores timed out") and its
 * outputs are invalid; the context stays usable. */
typedef struct cisor_fno cisor_fno;

/* Seeded random initialisation; max_batch (1..256) samples per call. */
cisor_status cisor_fno_create(cisor_fno** out, int max_batch, unsigned long long seed, void* stream);
cisor_status cisor_fno_destroy(cisor_fno* fno);
cisor_status cisor_fno_num_params(const cisor_fno* fno, long long* count);

/* Copy out the parameters: as_used = 1 gives the weights as the kernels read
 * them (BF16 values, biases FP32); 0 gives the FP32 masters. */
cisor_status cisor_fno_get_params(cisor_fno* fno, float* out, int as_used);

/* Replace the FP32 masters (and the BF16 copy); resets the Adam state. */
cisor_status cisor_fno_set_params(cisor_fno* fno, const float* in);

/* u_sc_out [B, 16384] = network output e(f, u_in) for B samples; f is [B, 16384]
 * (f_per_sample = 1) or one [16384] image shared by all samples (0);
 * u_in [B, 16384]; complex64. */
cisor_status cisor_fno_forward(cisor_fno* fno, const void* f, int f_per_sample, const void* u_in, int B,
                               void* u_sc_out);

/* Mean relative L2 loss against target [B, 16384] and, if grad_out is not
 * NULL, its gradient in every parameter (cisor_fno_num_params floats). */
cisor_status cisor_fno_loss_grad(cisor_fno* fno, const void* f, int f_per_sample, const void* u_in,
                                 const void* target, int B, double* loss, float* grad_out);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) at learning rate lr on the
 * loss above; *loss receives the loss before the step. */
cisor_status cisor_fno_train_step(cisor_fno* fno, const void* f, int f_per_sample, const void* u_in,
                                  const void* target, int B, double lr, double* loss);

/* x0_out [T, N] = u_in (1 + e(f, u_in)) for every transmitter of a context
 * with a 128 x 128 grid: the warm start for cisor_forward's x0 (x0_mode 1). */
cisor_status cisor_fno_warm_start(cisor_fno* fno, cisor_ctx* ctx, const void* f, void* x0_out);

/* Last error message of this thread ("" if none). */
const char* cisor_last_error(void);

/* Library version string. */
const char* cisor_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CISOR_H */
