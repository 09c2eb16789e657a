/*
 * smsm.h -- C ABI of the GB300-native SMS-MUSSELS reconstruction library.
 *
 * SMS-MUSSELS (Mani et al., arXiv 1901.01893) recovers the slice-unfolded,
 * per-shot k-space of a simultaneous-multislice (blipped-CAIPI) multi-shot
 * diffusion acquisition by minimising (Eq. 10)
 *
 *     || A(m) - y ||^2  +  lambda * sum_l || H_l(m) ||_*
 *
 * where A is the SENSE/CAIPI forward model of Fig. 1 and H_l is the block
 * Hankel matrix of slice l's shot k-spaces (Eqs. 8-9).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All array arguments are DEVICE pointers owned by the caller, C-contiguous,
 *    16-byte aligned, complex values interleaved (re, im).  complex64 = two
 *    float32, complex128 = two float64.  The x (readout, kx) index is fastest.
 *  - k-space is centred: index n has DC at n = N/2; the DFT is unitary.
 *  - L = mb (slices), Ns = shots, Nc = coils, N = nx = ny, r = filter,
 *    C = Ns*r*r (columns of H_l), P = (N-r+1)^2 (VALID patch origins).
 *  - Unknown x: [L][Ns][N][N] complex64, per-shot k-space of each slice.
 *    Data y: [Ns][Nc][N/Ns][N] complex64; shot i holds the lines
 *    n = m*Ns + i, m = 0..N/Ns-1 (Eq. 2, 0-based).
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream).  Only the report of smsm_reconstruct needs a sync, which
 *    that call performs itself when `report` is non-NULL.
 *  - Errors never abort: every call returns an smsm_status; smsm_last_error()
 *    returns a message for the calling thread's last failure.
 *  - A plan is not thread-safe: calls on one plan must be serialised by the
 *    caller (its workspace is shared by all its calls).
 */
#ifndef SMSM_H
#define SMSM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smsm_plan_s* smsm_plan_t;

typedef enum {
  SMSM_OK = 0,
  SMSM_ERR_ARG = 1,       /* bad size, NULL or misaligned pointer, unsupported shape */
  SMSM_ERR_CUDA = 2,      /* a CUDA runtime call failed (message has the CUDA error) */
  SMSM_ERR_NOMEM = 3,     /* device allocation failed while building the plan */
  SMSM_ERR_DIVERGED = 4,  /* a CG scalar became NaN/Inf (reported via smsm_report) */
  SMSM_ERR_NOT_PD = 5,    /* <p, N p> <= 0 in CG: system not positive definite */
  SMSM_ERR_TIMEOUT = 6,   /* reserved: a bounded device wait gave up */
  SMSM_ERR_STATE = 7,     /* call out of order, e.g. no coil maps set yet */
  SMSM_ERR_EIG_UNCONVERGED = 8 /* the Jacobi eigen step hit smsm_params.max_sweeps with a
                                  rotation still pending (reported via smsm_report; the
                                  solve ran on with the last rotations) */
} smsm_status;

typedef enum { SMSM_MODE_IRLS = 0, SMSM_MODE_NULLSPACE = 1 } smsm_mode;

/*
 * Plan options (all zero = defaults).
 * batch = D > 1 makes the plan solve D independent problems at once -- e.g.
 * the diffusion directions of one slice group, which share the geometry and
 * the coil maps.  Every per-problem array then gains a leading [D] dimension
 * (x: [D][L][Ns][N][N], y: [D][Ns][Nc][N/Ns][N], phase: [D][L][Ns][N][N],
 * G and W: [D][L][C][C]); coil maps stay [L][Nc][N][N].  Each problem keeps
 * its own CG scalars and eps schedule.
 */
typedef struct {
  int caipi_div;   /* CAIPI FOV shift is FOV/caipi_div per slice index; 0 -> mb (Eq. 1) */
  int batch;       /* D, number of problems per call; 0 -> 1 (at most 4096) */
  int flags;       /* SMSM_FLAG_* bits */
  int precision;   /* smsm_precision of the Hankel Gram (default FP32) */
  int boundary;    /* smsm_boundary of the Hankel lifting (default VALID) */
  int reserved[3];
} smsm_opts;

/*
 * Precision of the Hankel Gram, which runs on the tensor cores when C <= 144
 * (larger C: FP32 FMA; the BF16 split form needs C <= 144):
 *   FP32: every FP32 value split exactly into three BF16 pieces b1 + b2 + b3,
 *         six BF16 products b_i b_j' (i + j <= 4), FP32 accumulation: every
 *         product as accurate as an FP32 multiply;
 *   BF16_SPLIT: two pieces hi = bf16(x), lo = bf16(x - hi), three products
 *         hi hi' + hi lo' + lo hi' (~2^-16 relative per product).
 */
typedef enum { SMSM_PRECISION_FP32 = 0, SMSM_PRECISION_BF16_SPLIT = 1 } smsm_precision;

/* smsm_opts.boundary: which patch origins the Hankel lifting of Eq. 8 takes.
 *   VALID: k in [0, N-r]^2, the (N1-r+1)(N2-r+1) rows of Eq. 8;
 *   PERIODIC: every k in [0, N)^2 with indices taken mod N (k-space treated as
 *             periodic).  Then the Gram is block circular cross-correlation and the
 *             penalty is the image-domain multiplier alone (no border band). */
typedef enum { SMSM_BOUNDARY_VALID = 0, SMSM_BOUNDARY_PERIODIC = 1 } smsm_boundary;

/* smsm_opts.flags (same results up to rounding; for testing and comparison):
 *   GENERIC_KERNELS: the shape-generic kernels even where a specialised fast
 *                    path exists;
 *   PER_COIL_NORMAL: the column stage of A^H A loops over the coils with two
 *                    M-point transforms per coil instead of applying the
 *                    per-class coil correlations (which need N % caipi_div == 0);
 *   CLUSTER_EIG: the eigen step by one-sided block Jacobi on a cluster of eight
 *                CTAs per Gram (C = shots*filter^2 >= 65) even where the two-CTA
 *                two-sided solver fits.  C > 168 always takes the cluster solver
 *                (G of up to 320 x 320 does not fit one CTA's shared memory). */
#define SMSM_FLAG_GENERIC_KERNELS 1
#define SMSM_FLAG_PER_COIL_NORMAL 2
#define SMSM_FLAG_CLUSTER_EIG 4

/*
 * Solver parameters.  The paper minimises Eq. 10 with an augmented-Lagrangian
 * scheme whose listing is in another paper; this library minimises the same
 * cost by IRLS: at outer iteration k the nuclear norm is majorised with
 * W_l = (G_l + eps_k I)^(-1/2), G_l = H_l^H H_l, and cg_iters steps of CG solve
 *     (A^H A + lambda P_W) x = A^H y,   P_W(x)_l = H_l^*(H_l(x_l) W_l).
 * eps_1 = eps0_rel * max_l s_max(G_l); eps_k = max(eps_{k-1}/eta, eps_min_rel*eps_1).
 * NULLSPACE mode instead uses W_l = projector onto the C - rank smallest
 * eigenvectors of G_l (one rank for every slice).
 */
typedef struct {
  double lambda;      /* penalty weight in the normal equations (default 1e-2) */
  double eps0_rel;    /* default 1e-2 */
  double eta;         /* default 1.5 */
  double eps_min_rel; /* default 1e-2: eps_min = 1e-4 s_max, so the weights (s + eps)^(-1/2)
                         span at most a factor 100, the range the FP32 penalty represents */
  int outer_iters;    /* K, default 10, at most SMSM_MAX_OUTER */
  int cg_iters;       /* J, default 10 */
  int mode;           /* smsm_mode */
  int rank;           /* NULLSPACE rank, 0 < rank < C */
  int warm;           /* 1: x holds the starting point on entry; 0: start from A^H y */
  int max_sweeps;     /* cap on Jacobi sweeps of the eigen step, 0 -> 30 (at most 30);
                         reaching it with rotations pending sets SMSM_ERR_EIG_UNCONVERGED */
  int timing;         /* bitmask of (1 << smsm_stage): bracket those launches with CUDA
                         events inside the solve and report their device time */
  int eig_cold;       /* 1: restart the eigensolver from scratch every outer iteration
                         (default 0: start from the previous iteration's eigenvectors) */
  int lanes;          /* batch > 1: split the batch into this many sub-batches solved as
                         concurrent branches of the captured graph, started out of phase
                         so that one lane's (latency-bound) eigensolver runs while other
                         lanes' CG runs; 0 -> automatic (3 for a batch of at least 9, 2
                         from 4), at most SMSM_MAX_LANES and the batch.  Results do not
                         depend on it. */
  float eig_tol;      /* rotation threshold of the Jacobi eigen step, relative (a pair is rotated
                         while its coupling exceeds eig_tol times the geometric mean of its
                         diagonal terms); 0 -> 1e-6 for the two-CTA solver, 2e-6 for the
                         cluster solver (whose pair sums carry ~1e-7 relative rounding) */
  int reserved[2];
} smsm_params;

#define SMSM_MAX_LANES 4

#define SMSM_MAX_OUTER 128

/* Kernel classes of the solve, for smsm_params.timing and smsm_report.stage_ms. */
typedef enum {
  SMSM_STAGE_ADJOINT = 0,    /* b = A^H y (row FFT, column stage, row FFT) */
  SMSM_STAGE_GRAM = 1,       /* Hankel Gram partials + reduction */
  SMSM_STAGE_EIG = 2,        /* Jacobi sweeps on G */
  SMSM_STAGE_VAPPLY = 3,     /* Newton-Schulz re-orthonormalisation of V */
  SMSM_STAGE_WEIGHTS = 4,    /* eps schedule + W */
  SMSM_STAGE_FILTERS = 5,    /* filters from W + image-domain multipliers */
  SMSM_STAGE_ROWFFT_INV = 6, /* x-direction inverse FFT of the CG vector */
  SMSM_STAGE_COLUMN = 7,     /* fused column stage of (A^H A + lambda P_W) */
  SMSM_STAGE_ROWFFT_FWD = 8, /* x-direction forward FFT back to k-space */
  SMSM_STAGE_BAND = 9,       /* border-band correction of the penalty */
  SMSM_STAGE_CG = 10,        /* CG vector updates */
  SMSM_NUM_STAGES = 11
} smsm_stage;

/* Per-call report, filled after the call's work has finished (host memory).
 * With batch > 1, status is the first nonzero status over the problems and the
 * per-iteration arrays follow problem 0. */
typedef struct {
  int status;                           /* smsm_status of the device-side checks */
  int outer_done;                       /* outer iterations run */
  double eps[SMSM_MAX_OUTER];           /* eps_k (IRLS) */
  double rr_start[SMSM_MAX_OUTER];      /* ||r||^2 at the start of outer k's CG */
  double rr_end[SMSM_MAX_OUTER];        /* ||r||^2 after its cg_iters steps */
  int sweeps[SMSM_MAX_OUTER];           /* Jacobi sweeps used (max over slices) */
  float elapsed_ms;                     /* device time of the solve (CUDA events) */
  int graph_kernels;                    /* kernel launches in one solve (nodes of its graph) */
  float stage_ms[16];                   /* device time per smsm_stage (timed stages only; with
                                           several lanes, the launches of lane 0) */
  int stage_launches[16];               /* timed launches per smsm_stage */
  int lanes;                            /* concurrent lanes the batch was solved as */
  int lane0_batch;                      /* problems in lane 0 (each timed launch covers them) */
} smsm_report;

/* Fill *p with the defaults listed above. */
void smsm_default_params(smsm_params* p);

/*
 * Create a plan for one slice-group geometry (the problem statement around
 * Eq. 10: y of size N1 x N2/Ns x Nc x Ns, L simultaneously excited slices,
 * filter (phase-support) size r of Eq. 8).
 *   mb     L >= 1         shots  Ns >= 1, N % Ns == 0
 *   coils  Nc >= 1        nx, ny equal, even, of the form 2^a 3^b, 16..512
 *   filter r, 1 <= r <= N/2; C = Ns*r*r <= 320
 * Allocates all device workspace (caller's current device).  On failure *out
 * is NULL.
 */
smsm_status smsm_plan(smsm_plan_t* out, int mb, int shots, int coils, int nx, int ny, int filter,
                      const smsm_opts* opts /* nullable */);

/* Release the plan and its device memory (NULL is a no-op). */
smsm_status smsm_plan_destroy(smsm_plan_t plan);

/* Bytes of device memory the plan holds. */
size_t smsm_plan_workspace_bytes(smsm_plan_t plan);

/*
 * Set the coil sensitivities S (Fig. 1 step (ii)): sens is [L][Nc][N][N]
 * complex64, image domain.  The plan keeps its own copy (transposed for the
 * column kernels) and, where the CAIPI shift is a whole number of pixels, the
 * coil correlations of every aliasing class of A^H A derived from it, so
 * `sens` may be freed once the stream has passed this call.
 */
smsm_status smsm_plan_set_sens(smsm_plan_t plan, const void* sens, void* stream);

/*
 * y = A(x), Fig. 1 steps (i)-(v): inverse DFT, coil multiply, DFT, CAIPI phase
 * exp(-j 2 pi l (n - N/2)/caipi_div) and slice sum (Eqs. 1, 3), shot mask.
 *   phase == NULL: x is [L][Ns][N][N] per-shot k-space (the unknown of Eq. 10).
 *   phase != NULL: x is [L][1][N][N] shared k-space and phase [L][Ns][N][N]
 *                  complex64 is the image-domain shot phase phi_{l,i} (Eq. 4).
 *   y: [Ns][Nc][N/Ns][N] complex64 (overwritten).
 */
smsm_status smsm_forward(smsm_plan_t plan, const void* x, const void* phase, void* y, void* stream);

/* x = A^H(y), the adjoint of smsm_forward (same layouts; x overwritten). */
smsm_status smsm_adjoint(smsm_plan_t plan, const void* y, const void* phase, void* x, void* stream);

/*
 * G_l = H_l^H H_l for every slice (Eqs. 8-9): x is [L][Ns][N][N] complex64,
 * G is [L][C][C] complex128 (full Hermitian matrix, overwritten), with
 * G[(i,p),(i',q)] = sum_{k in [0,N-r]^2} conj(x_i[k+p]) x_i'[k+q],
 * column index (i,p) = i*r*r + py*r + px.  x must be 16-byte aligned (its image
 * rows are copied into shared memory by bulk copies); SMSM_ERR_ARG otherwise.
 */
smsm_status smsm_hankel_gram(smsm_plan_t plan, const void* x, void* G, void* stream);

/*
 * out = P_W(x): out_l = H_l^*(H_l(x_l) W_l), the annihilating-filter penalty
 * (the gradient of ||H_l(x) W^(1/2)||_F^2 up to a factor 2).  W is
 * [L][C][C] complex128, Hermitian (only that is assumed); x, out are
 * [L][Ns][N][N] complex64 and must not alias.
 */
smsm_status smsm_apply_filters(smsm_plan_t plan, const void* W, const void* x, void* out,
                               void* stream);

/*
 * The SMS-MUSSELS reconstruction (Eq. 10) by IRLS + CG (see smsm_params).
 *   y: [Ns][Nc][N/Ns][N] complex64 measured data.
 *   x: [L][Ns][N][N] complex64; input when params->warm, always the output.
 * The whole solve runs on the device (captured once per plan and parameter
 * set as a CUDA graph).  `report` (host, nullable) is filled after a stream
 * sync; without it the call does not block.
 */
smsm_status smsm_reconstruct(smsm_plan_t plan, const void* y, void* x, const smsm_params* params,
                             smsm_report* report, void* stream);

/*
 * Independent slice groups that may differ in geometry (MB, shots, coils, N,
 * filter; one plan each, coil maps set) reconstructed together in ONE graph launch
 * on `stream`: a graph holding, for every group, the copy of its y (and warm start)
 * in, its captured solve (as smsm_reconstruct, same params for all) as a child
 * graph and the copy of x out, the groups as independent branches, so the kernels
 * of small and large groups share the GPU.  The graph is built on the first call
 * with a given list of plans, buffers and params and reused while they stay the
 * same (a few such lists are kept; destroying a plan drops those holding it).  With
 * params->timing set, each group's solve is launched on its own stream instead,
 * forked from `stream` and joined back into it.  ys[k], xs[k] are laid out as for
 * smsm_reconstruct on plans[k]; a plan may appear only once, and every plan must
 * belong to the current device.  `reports`
 * (nullable) is an array of n, filled after a synchronisation of `stream`.
 */
smsm_status smsm_reconstruct_groups(int n, smsm_plan_t const* plans, const void* const* ys, void* const* xs,
                                    const smsm_params* params, smsm_report* reports, void* stream);

/*
 * SMS-SENSE, the comparison reconstruction of the paper's simulation and in-vivo
 * figures (Results): the k-space data of all shots are combined into one k-space per
 * slice (the shot-shared model of Eq. 4: phase phi_{l,i} [D][L][Ns][N][N] complex64,
 * image domain, or phase == NULL for no phase correction) and the slices are unfolded
 * by least squares: cg_iters steps of CG on A^H A x = A^H y from x = 0.
 *   y: [D][Ns][Nc][N/Ns][N] complex64; x: [D][L][1][N][N] complex64 (overwritten).
 * Runs on the stream without a graph; `report` (nullable) gets the status after a sync.
 */
smsm_status smsm_sense(smsm_plan_t plan, const void* y, const void* phase, void* x, int cg_iters,
                       smsm_report* report, void* stream);

/*
 * Centred unitary 2D DFT of `count` N x N complex64 images (Fig. 1 steps
 * (i)/(iii)): inverse != 0 selects F^-1.  in and out may alias.
 */
smsm_status smsm_fft2c(smsm_plan_t plan, const void* in, void* out, int count, int inverse,
                       void* stream);

/*
 * The Hankel Gram of smsm_hankel_gram without any device allocation and
 * without a plan (the paper has no counterpart: this is a service to callers
 * that may not allocate GPU memory -- a host framework that owns every device
 * allocation through its own pool, or a real-time path that must not block in
 * the allocator -- and so cannot call smsm_plan, which allocates).
 *   x: [mb][shots][n][n] complex64, G: [mb][C][C] complex128, C = shots*filter^2,
 *   same definition and layouts as smsm_hankel_gram; 1 <= shots <= 8,
 *   16 <= n <= 512, 1 <= filter <= min(12, n/2), C <= 320.
 * Scratch: one fixed 8 MiB array compiled into the library, held by every GPU
 * that loads the library's device code until exit (with lazy module loading,
 * from the first call of this entry point or the first launch of any of the
 * library's kernels on that GPU).  Geometries needing more than
 * ceil((n-filter+1)/16) * C^2 * 16 bytes > 8 MiB are rejected with
 * SMSM_ERR_ARG, as is C > 320.  All calls on a device share that array: calls
 * that overlap on the GPU race and must be serialised by the caller.  Nothing
 * in it needs clearing between calls.  Every call looks the array's address
 * up in the current context; the first call on a device may load the
 * library's device code, so make it once at set-up, before any stream capture
 * on that device.
 */
smsm_status smsm_hankel_gram_noalloc(const void* x, void* G, int mb, int shots, int n, int filter,
                                     void* stream);

/*
 * Autotuner (not in the paper).  Times, on the plan's own data y (layout of
 * smsm_reconstruct), the tensor-core Gram with each candidate number of split-K
 * blocks (one to six waves of CTAs over the GPU) and shortened solves (min(K, 6)
 * outer iterations of `params`, so that the cold first eigen step weighs about as
 * little as in the full solve) with 1..min(batch, SMSM_MAX_LANES) concurrent lanes,
 * keeps the fastest of each for this plan (the lanes apply when params->lanes is 0)
 * and remembers them for every later plan of the same shape (mb, shots, coils, N,
 * filter, batch, precision, boundary, flags, CAIPI shift) in this process.
 * Synchronises `stream`; `report` (host, nullable) receives what was timed.
 * Results do not depend on the choices up to the order of the Gram's partial sums.
 */
typedef struct {
  int gram_nG;              /* chosen split-K blocks (0: no tensor-core Gram) */
  int n_gram;               /* candidates timed */
  int gram_candidates[8];
  float gram_ms[8];         /* device time of one Gram launch per candidate */
  int lanes;                /* chosen lanes */
  float lane_ms[SMSM_MAX_LANES]; /* device time of the shortened solve per lane count */
} smsm_tune_report;

smsm_status smsm_autotune(smsm_plan_t plan, const void* y, const smsm_params* params, smsm_tune_report* report,
                          void* stream);

/* ------------------------------------------------------------------------
 * Learned warm start (not in the paper, which starts its iteration from the
 * data alone).  A complex CNN maps the aliased, zero-filled image of every
 * (slice, shot), a = F^-1(A^H y) ([n][B][H][W] complex64, B = L*Ns), to a
 * starting image x0 = a + f(a): f is `layers` complex 3x3 convolutions
 * (cross-correlation, zero padding) with channels B -> width -> ... -> B and
 * CReLU (ReLU of the real and of the imaginary part) between them.  The start
 * seeds the k-space of the IRLS solve of Eq. 10 and so its first Gram and
 * annihilating filters (Eq. 9).  Weights: FP32 master copies, every product
 * taken with the weight rounded to BF16, FP32 activations and accumulation.
 * Parameters are one complex64 vector: for each layer k, W_k [Cout][Cin][3][3]
 * then b_k [Cout].  Loss of a sample ||x0 - t||^2 / ||t||^2, averaged over the
 * batch; gradients are given as dL/dRe + i dL/dIm.  All pointers are device
 * pointers, 16-byte aligned, owned by the caller; calls are asynchronous on
 * `stream` except where a host `loss` is requested (then they synchronise).
 * ------------------------------------------------------------------------ */
typedef struct smsm_cnn_s* smsm_cnn_t;

/* Create a network for images of height x wdt with `channels` = B input and output
 * channels and `width` hidden ones; buffers for batches up to max_batch are held
 * (activations of every layer, for training).  Parameters start at zero: set them. */
smsm_status smsm_cnn_create(smsm_cnn_t* out, int channels, int width, int layers, int height, int wdt,
                            int max_batch);
smsm_status smsm_cnn_destroy(smsm_cnn_t cnn);
/* Number of complex parameters. */
size_t smsm_cnn_param_count(smsm_cnn_t cnn);
/* Copy params [count] complex64 in (also clears the optimiser's moments), or out. */
smsm_status smsm_cnn_set_params(smsm_cnn_t cnn, const void* params, void* stream);
smsm_status smsm_cnn_get_params(smsm_cnn_t cnn, void* params, void* stream);
/* x0 = a + f(a) for n samples (a and x0 distinct). */
smsm_status smsm_cnn_forward(smsm_cnn_t cnn, const void* a, void* x0, int n, void* stream);
/* Loss of the n samples (a, target t) and its gradient grad [count]; `loss` (host,
 * nullable) receives the mean loss after a synchronisation. */
smsm_status smsm_cnn_gradients(smsm_cnn_t cnn, const void* a, const void* t, int n, void* grad, double* loss,
                               void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step size lr) on the gradient of
 * the batch's loss. */
smsm_status smsm_cnn_train_step(smsm_cnn_t cnn, const void* a, const void* t, int n, float lr, double* loss,
                                void* stream);
/* The learned refinement of a k-space estimate for every problem of `plan`:
 * x_out = F(cnn(F^-1(x_in))), x_in and x_out [D][L][Ns][N][N] (the layout of x in
 * smsm_reconstruct; they may alias).  x_in is A^H y (smsm_adjoint) or an early iterate
 * of smsm_reconstruct; pass x_out to smsm_reconstruct with params->warm = 1.  Needs cnn
 * channels = L*Ns, an N x N image and max_batch >= D. */
smsm_status smsm_learned_start(smsm_plan_t plan, smsm_cnn_t cnn, const void* x_in, void* x_out, void* stream);

/*
 * Synchronise `stream` and report the plan's device error flag: SMSM_OK, or
 * SMSM_ERR_TIMEOUT when a kernel gave up a bounded wait (its outputs are then
 * unspecified).  smsm_reconstruct's report carries the same flag.
 */
smsm_status smsm_plan_device_status(smsm_plan_t plan, void* stream);

/* Message of the calling thread's last failed call ("" if none). */
const char* smsm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SMSM_H */
