/*
 * lbm.h -- C ABI of the GB300 slip-wall D2Q9 MRT lattice Boltzmann library
 * (liblbm.so).
 *
 * The library advances a 2-D lattice with the multiple-relaxation-time
 * lattice Boltzmann equation with Guo forcing (Sec. 2 of Wang et al.,
 * "Curved boundary conditions of the lattice Boltzmann method for simulating
 * microgaseous flows in the slip regime", Eqs. LBENS, LBEequi, LBEforce,
 * MomentPost) and applies the paper's local curved slip boundary scheme on
 * every boundary link (Sec. 3.A, Eq. EqNewBDSC), with the free parameter,
 * combination parameter and uniform tau_q of Sec. 3.B (Eqs. Eqexlva,
 * SliCoeffrtsr, NSliCoertstq, the clamp of l below -0.4).
 *
 * Conventions shared by every entry point:
 *   * D2Q9 velocities c_0..c_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),
 *     (-1,1),(-1,-1),(1,-1) (Eq. 3); lattice units, delta_x = delta_t = 1.
 *   * Node (x, y) has row-major index y*nx + x.  Host field arrays are
 *     nx*ny doubles in that order; population arrays are 9*nx*ny doubles,
 *     index (i*ny + y)*nx + x.
 *   * A boundary link (x, y, i, q, ubx, uby) names a fluid node x_f = (x, y)
 *     whose neighbour x_f - c_i is solid, so f_i(x_f) is unknown after
 *     streaming; q is the distance ratio gamma = |x_b - x_f| / |x_r - x_f| in
 *     (0, 1] of Fig. 1 and (ubx, uby) the wall velocity at x_b.
 *   * Every call returns an lbm_status code; no call aborts or exits.  On an
 *     error the handle's message (lbm_last_error) says what was wrong.
 *   * All device work runs on the stream given at creation (params.stream,
 *     a cudaStream_t; NULL = the legacy default stream).  Calls that return
 *     host data synchronise that stream; the others are asynchronous.
 *   * The handle owns its device memory; every input array is copied at
 *     creation, so the caller keeps ownership of its buffers.
 */
#ifndef LBM_H_
#define LBM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,    /* bad argument, link set or parameter (tau_q <= 1/2, ...) */
  LBM_ECUDA = 2,     /* a CUDA runtime call failed */
  LBM_EUNSTABLE = 3, /* a non-finite density or velocity was found */
  LBM_ETIMEOUT = 4,  /* a device-side wait hit its iteration limit */
  LBM_ENOMEM = 5,    /* device or host allocation failed */
  LBM_EIO = 6        /* a checkpoint file could not be written or read */
} lbm_status;

typedef enum {
  LBM_FP64 = 0, /* populations stored and collided in FP64 */
  LBM_FP32 = 1, /* populations stored as FP32 deviations f_i - w_i, FP32 arithmetic */
  LBM_BF16 = 2, /* deviations stored as BF16, FP32 arithmetic */
  LBM_FP16 = 3  /* deviations times storage_scale stored as FP16, FP32 arithmetic */
} lbm_precision;
/* BF16 and FP16 storage round every stored value stochastically (to one of
 * its two storage neighbours, with probabilities that make it exact on
 * average), so changes smaller than a storage unit are not lost step after
 * step.  The random bits are a counter-based hash of the node and the step
 * count: a run is reproducible, and a resumed or batched case takes the
 * same roundings as the uninterrupted lone case.  A value beyond the
 * largest finite 16-bit number saturates there; lbm_residual reports a
 * saturated value as non-finite (LBM_EUNSTABLE). */

typedef enum {
  LBM_L_PAPER = 0,        /* l from Eq. Eqexlva, set to 0 where it is below l_clamp */
  LBM_L_ZERO = 1,         /* l = 0 (the halfway DBB scheme when gamma = 1/2) */
  LBM_L_GAMMA = 2,        /* l = gamma      (alternatives compared in Sec. 4) */
  LBM_L_2GAMMA = 3,       /* l = 2 gamma */
  LBM_L_GAMMA2 = 4,       /* l = gamma^2 */
  LBM_L_GAMMA2_GAMMA = 5, /* l = gamma^2 + gamma */
  LBM_L_FIXED = 6         /* l = params.l_value for every link */
} lbm_l_mode;

typedef struct lbm_handle lbm_handle_t;

typedef struct {
  int32_t nx, ny;                 /* lattice size, both >= 1 */
  int32_t periodic_x, periodic_y; /* 1 = periodic; a non-periodic axis needs solid edge rows */
  double H;                       /* characteristic length in lattice units (Eq. tKnrela) */
  double ax, ay;                  /* body acceleration a, lattice units (Eq. LBEforce) */
} lbm_domain_t;

typedef struct {
  double sigma;   /* wall accommodation coefficient (Sec. 4), default 1 */
  double L1, L2;  /* slip coefficients of Eq. PhyscSlip; NaN = from sigma (Sec. 4) */
  double E;       /* constant of Eq. Eqexlva; NaN = min(-0.65, E_max - 0.1), E_max of Eq. EqECond */
  double l_clamp; /* l := 0 where Eq. Eqexlva gives l < l_clamp (Sec. 3.B), default -0.4 */
  double tau_rho, tau_j, tau_e, tau_eps; /* fixed relaxation times (Sec. 4): 1, 1, 1.1, 1.2 */
  double tau_s;   /* NaN = 1/2 + sqrt(6/pi) Kn H (Eq. tKnrela) */
  double tau_q;   /* NaN = Eq. NSliCoertstq */
  double r_value; /* NaN = Eq. SliCoeffrtsr with the l actually used; else r for every link */
  double l_value; /* used by LBM_L_FIXED */
  int32_t l_mode;       /* lbm_l_mode, default LBM_L_PAPER */
  int32_t diffuse_mode; /* Maxwell part of Eq. EqNewBDSC at 0 = the fluid velocity of x_f
                           (the reading under which Sec. 3.B holds, default), 1 = the wall
                           velocity u_b (the equation as printed) */
  int32_t precision;    /* lbm_precision, default LBM_FP32 */
  int32_t residual_every; /* steps between residual checks in lbm_run_to, default 100 */
  double storage_scale; /* LBM_FP16 only: deviations are stored times this power of two
                           (0 = 4096, which keeps |d| from 1.5e-8 to 16 in FP16's normal range) */
  int32_t collision;    /* 0 = MRT (default); 1 = BGK reading of Sec. 3.B: every relaxation
                           time equals tau_s and E solves Eq. NSliCoertstq for tau_q = tau_s
                           (tau_q, E and the fixed relaxation times given here are ignored) */
  void *stream;         /* cudaStream_t for all device work; NULL = legacy default stream */
  int32_t mass_mode;    /* LBM_FP32 only.  0 (default): the exact-mass step where a wall moves
                           (some link has a nonzero wall velocity) or the lattice has no
                           boundary links (periodic, often uniform flow); 1: always; -1: never.
                           The exact-mass step sums rho - 1 and j in twice the working
                           precision, rounds f'_1..f'_8 to FP32 stochastically (unbiased),
                           forms each boundary link's value (Eq. EqNewBDSC) in double-FP32
                           arithmetic (about 48 significant bits) and the rest population's
                           mass closure in twice the working precision, and keeps, per link
                           and per node, what FP32 storage dropped from them, adding it to the
                           next value: the stored mass then follows the exact trajectory
                           instead of drifting by roundings that repeat every step.  It costs
                           4 B per link and 8 B per fluid node of extra traffic per step and
                           about 2.5x the plain step's time. */
  int32_t residual_mode; /* 0 (default): lbm_residual's residual is the one-step change
                            ||u^n - u^(n-1)|| / ||u^n||.  1: the interval change
                            ||u^n - u^m|| / ((n - m) ||u^n||), u^m the velocity field at the
                            previous lbm_residual call (m its step count; the initial state,
                            lbm_set_f / lbm_set_fields or lbm_load start a new interval): the
                            mean change per step, which near a steady state does not floor at the
                            rounding noise that 16-bit or FP32 storage leaves in one step. */
} lbm_params_t;

typedef struct {
  int64_t n_nodes, n_fluid, n_links;
  int64_t steps;          /* time steps taken since creation (or the last lbm_set_f) */
  double tau_s, tau_q, E, E_max, L1, L2;
  int64_t n_clamped;      /* links whose l was set to 0 by the clamp */
  int64_t device_bytes;   /* device memory held by the handle */
  int32_t precision, pitch; /* storage precision; row pitch in elements of a dense lattice
                               (0: the single-case solver stores fluid nodes only) */
  int32_t exact_mass;     /* 1 if the step runs the exact-mass variant (see mass_mode) */
  int32_t reserved;
} lbm_info_t;

/* Fill *p with the defaults listed above (no side effects). */
void lbm_params_default(lbm_params_t *p);

/*
 * Create a solver for one case.  solid: nx*ny bytes, nonzero = solid.
 * Links: n_links entries in six parallel arrays (any order; duplicates,
 * links whose node is solid or whose neighbour x_f - c_i is fluid, gamma
 * outside (0, 1], and fluid nodes with an unknown direction that no link
 * covers are LBM_EINVAL).  Kn is the Knudsen number of Eq. tKnrela.  The
 * state starts at rest, f_i = w_i (rho = 1, u = 0).  The device copy keeps
 * the fluid nodes only (row-major, with per-node neighbour offsets), so its
 * size follows the fluid fraction, not nx*ny.  Limits of that layout, each
 * LBM_EINVAL: rows of at most 65535 nodes (nx <= 65535); 9 x fluid nodes +
 * links below 2^32; no 32 consecutive fluid nodes (row-major order) spread
 * over more than 16384 rows.  On success *out holds
 * the handle; on failure *out is NULL and the returned code says why
 * (lbm_last_error(NULL) gives the message of the last failed creation on
 * this thread).
 */
int lbm_create(const lbm_domain_t *dom, const uint8_t *solid, size_t n_links,
               const int32_t *link_x, const int32_t *link_y, const int32_t *link_dir,
               const double *link_q, const double *link_ubx, const double *link_uby,
               double Kn, const lbm_params_t *params, lbm_handle_t **out);

/* Advance n >= 0 time steps (collision, streaming, boundary links: Sec. 2,
 * Eq. EqNewBDSC).  Asynchronous on the handle's stream. */
int lbm_step(lbm_handle_t *h, int64_t n);

/*
 * Density and velocity (Eq. FluidMacr: rho = sum f, rho u = sum c f + rho a/2)
 * of every node, nx*ny doubles each; solid nodes get 0.  on_device = 0: host
 * pointers (the call synchronises); 1: device pointers on the handle's
 * device (asynchronous).  Any of the three pointers may be NULL.
 */
int lbm_fields(lbm_handle_t *h, double *rho, double *ux, double *uy, int on_device);

/*
 * Convergence and conservation monitor: residual = ||u^n - u^(n-1)||_2 /
 * ||u^n||_2 over fluid nodes (0 before the first step; with
 * params.residual_mode = 1 the interval change described there) and mass =
 * sum over fluid nodes of sum_i f_i, both accumulated in FP64.  Synchronises.
 * Returns LBM_EUNSTABLE (with the values still written) when a fluid node
 * has a non-finite density or velocity.
 */
int lbm_residual(lbm_handle_t *h, double *residual, double *mass);

/* Step in chunks of params.residual_every until the residual is below tol
 * or max_steps were taken; *steps_done and *residual report the outcome. */
int lbm_run_to(lbm_handle_t *h, double tol, int64_t max_steps, int64_t *steps_done,
               double *residual);

/* All populations f_i (not deviations) as 9*nx*ny host doubles, plane i at
 * i*nx*ny (get: the current state, solid nodes as the rest state w_i; set:
 * replaces the state and the previous-step state of every fluid node, so
 * the next residual is 0 until a step is taken; solid entries are
 * ignored).  Synchronise. */
int lbm_get_f(lbm_handle_t *h, double *f);
int lbm_set_f(lbm_handle_t *h, const double *f);

/* Warm start: replace the state by populations built from density and
 * velocity fields (nx*ny doubles each, the convention of lbm_fields; host
 * pointers, or device pointers with on_device = 1): at every fluid node the
 * equilibrium of Eq. LBEequi at u - a/2 (so that Eq. FluidMacr returns u)
 * plus the first-order Chapman-Enskog non-equilibrium part
 * -3 tau_s w_i rho (c_i c_i - I/3) : grad u, with grad u by central
 * differences over fluid neighbours (one-sided next to walls).  The previous
 * state is set equal to it (residual 0 until a step).  Synchronises. */
int lbm_set_fields(lbm_handle_t *h, const double *rho, const double *ux, const double *uy,
                   int on_device);

/* Per-link free parameter l and combination parameter r as used, in the
 * order the links were given at creation (n_links doubles each, host). */
int lbm_link_params(const lbm_handle_t *h, double *r, double *l);

int lbm_get_info(const lbm_handle_t *h, lbm_info_t *info);

/*
 * Host-only FP64 precompute of Sec. 3.B without creating a solver (no CUDA
 * call): tau_s (Eq. tKnrela), L1, L2, E, E_max, tau_q (Eq. NSliCoertstq)
 * into *info (the other info fields are zero), and for n links with
 * directions dir[] (1..8), distance ratios q[] and wall velocities
 * (ubx[], uby[]) the free parameter l[] (Eq. Eqexlva with the clamp) and
 * the combination parameter r[] (Eq. SliCoeffrtsr).  r and l may be NULL.
 * LBM_EINVAL (message via lbm_last_error(NULL)) for the same parameter
 * errors lbm_create reports.
 */
int lbm_precompute(double Kn, double H, const lbm_params_t *params, size_t n,
                   const int32_t *dir, const double *q, const double *ubx, const double *uby,
                   double *r, double *l, lbm_info_t *info);

/*
 * Residual and mass of a state the caller holds, with no device allocation.
 * The paper has no counterpart: this is a library facility for callers that
 * cannot allocate device memory where they monitor convergence (their
 * device memory belongs to another framework's pool, or an allocation there
 * would synchronise or fail).  Same quantities as lbm_residual.
 *   f_cur, f_prev: device arrays, 9*nx*ny doubles each, full populations f_i
 *                  in the layout of lbm_get_f (states at steps n and n-1).
 *   solid:         device array, nx*ny bytes, nonzero = solid (as lbm_create).
 *   ax, ay:        body acceleration (for the half-force velocity).
 *   stream:        cudaStream_t to run on (NULL = legacy default stream);
 *                  the call synchronises it.
 *   residual, mass: host outputs.
 * Scratch: a fixed device array in the library (16384 rows x 5 doubles,
 * 640 KiB), held by every GPU that loads the library until the process
 * exits; ny > 16384 is LBM_EINVAL.  Each call looks up that array's address
 * in the context current on the calling thread (the lookup allocates
 * nothing; it is repeated on every call so that a device reset or another
 * context never leaves a stale address).  The first call on a device may
 * load the library's device code there, so make it before any stream
 * capture.  All calls share the array and each call overwrites every part
 * of it that it reads, so calls whose work overlaps on the GPU (other
 * threads, other streams) race and must not be issued concurrently.
 * Errors: LBM_EINVAL, LBM_ECUDA, LBM_EUNSTABLE (a fluid node with a
 * non-finite density or velocity in either state; outputs still written);
 * the message is lbm_last_error(NULL).
 */
int lbm_residual_noalloc(const double *f_cur, const double *f_prev, const uint8_t *solid,
                         int32_t nx, int32_t ny, double ax, double ay, void *stream,
                         double *residual, double *mass);

/* ---------------------------------------------------------------------------
 * Batched solver: many independent cases of different sizes, geometries and
 * parameters advanced together.  Each case is what lbm_create takes; all of
 * them are stored in one precision.  A step is one launch over every active
 * case; every check_every steps a batched reduction computes each case's
 * residual (as lbm_residual) and retires converged cases on the device; the
 * steps and the reduction run as one captured CUDA graph.  Cases follow the
 * same per-node arithmetic as a lone case created with the same inputs.
 * ------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch_t;

typedef struct {
  lbm_domain_t dom;
  const uint8_t *solid;  /* nx*ny bytes, as lbm_create */
  size_t n_links;
  const int32_t *link_x, *link_y, *link_dir;
  const double *link_q, *link_ubx, *link_uby;
  double Kn;
  lbm_params_t params;   /* precision and stream are taken from the batch */
} lbm_case_t;

/* Copy and validate n_cases cases (errors name the case), lay them out on
 * the device (each case in the layout lbm_create uses, with its limits),
 * pick the step kernel's CTA width and L2 prefetch by timing each
 * candidate over 12 steps twice on the batch itself (cached per precision
 * and size class), start every case at rest.  stream: cudaStream_t or NULL
 * (the batch then makes its own, since graph capture needs a non-legacy
 * stream). */
int lbm_batch_create(const lbm_case_t *cases, int32_t n_cases, int32_t precision, void *stream,
                     lbm_batch_t **out);
/* Back to rest, every case active, step counts zero. */
int lbm_batch_reset(lbm_batch_t *b);
/* Advance all active cases, check_every (even, >= 2) steps at a time, until
 * every case has residual < tol or max_steps were taken.  A case's residual
 * follows its params.residual_mode: the one-step change, or (1) the change
 * over the check_every steps since the previous check divided by
 * check_every.  The batch advances
 * in whole rounds of check_every steps, so a max_steps that is not a
 * multiple of check_every is rounded up to the next multiple.  Outputs
 * (host, n_cases entries, may be NULL): the step count at which each case
 * met tol (negative if it became non-finite, 0 if still running) and its
 * last residual; *steps_total = steps taken by the batch.  Synchronises. */
int lbm_batch_run_to(lbm_batch_t *b, double tol, int64_t max_steps, int32_t check_every,
                     int64_t *steps_per_case, double *residual_per_case, int64_t *steps_total);
/* Warm start of case c from density / velocity fields (host, nx*ny
 * doubles each), as lbm_set_fields; call after lbm_batch_create or
 * lbm_batch_reset and before lbm_batch_run_to. */
int lbm_batch_set_fields(lbm_batch_t *b, int32_t c, const double *rho, const double *ux,
                         const double *uy);
/* Density and velocity of case c (host arrays of nx*ny doubles, may be NULL). */
int lbm_batch_fields(lbm_batch_t *b, int32_t c, double *rho, double *ux, double *uy);
/* Sizes of the batch (outputs may be NULL): lattice nodes and fluid nodes
 * of all cases, the step kernel's CTA width and its CTAs per step. */
int lbm_batch_info(const lbm_batch_t *b, int64_t *total_nodes, int64_t *total_fluid,
                   int32_t *cta_threads, int32_t *n_ctas);
/* Override the autotuner's launch shape (for comparisons): the step
 * kernel's CTA width (64, 128, or 256 for FP32 / FP64) and the L2 prefetch
 * of the chunks half the resident CTAs ahead (1) or none (0).  Takes
 * effect at the next lbm_batch_run_to (the CUDA graph is captured again).
 * LBM_EINVAL for another width or flag, or while the state is mid-graph. */
int lbm_batch_set_launch(lbm_batch_t *b, int32_t cta_threads, int32_t l2_prefetch);
void lbm_batch_destroy(lbm_batch_t *b);
/* Last error of the batch; with b = NULL, of the last failed lbm_batch_create. */
const char *lbm_batch_last_error(const lbm_batch_t *b);

/* ---------------------------------------------------------------------------
 * Warm-start network (the paper has none): a convolutional encoder-decoder
 * with `levels` levels and `base` channels at the top level, doubling per
 * level; per level two 3x3 convolutions with ReLU, 2x2 average pooling
 * down, nearest upsampling and concatenation with the encoder output up,
 * a 1x1 convolution to c_out outputs.  Inputs / outputs are NHWC FP32 device
 * arrays of H x W pixels.  precision: LBM_BF16 (activations and gradients
 * stored in BF16, every product accumulated in FP32; master weights and Adam
 * state FP32) or LBM_FP32.  Parameters are one FP32 vector, layer by layer
 * (encoder levels top-down, decoder levels bottom-up, head), each layer its
 * weights [kh][kw][ci][co] then its biases; lbm_net_create draws He-normal
 * weights from `seed` and zero biases.  Calls synchronise `stream`.
 * ------------------------------------------------------------------------- */
typedef struct lbm_net lbm_net_t;
int lbm_net_create(int32_t base, int32_t levels, int32_t c_in, int32_t c_out, int32_t precision,
                   int32_t max_batch, int32_t H, int32_t W, uint64_t seed, void *stream,
                   lbm_net_t **out);
int64_t lbm_net_num_params(const lbm_net_t *n);
int lbm_net_set_params(lbm_net_t *n, const float *params, int64_t count);  /* host; resets Adam */
int lbm_net_get_params(const lbm_net_t *n, float *params, int64_t count);  /* host */
/* y = net(x) for `batch` samples (device arrays). */
int lbm_net_forward(lbm_net_t *n, const float *x, int32_t batch, float *y);
/* Mean squared error of net(x) against t and its gradient with respect to
 * every parameter (host array of lbm_net_num_params floats, may be NULL). */
int lbm_net_gradients(lbm_net_t *n, const float *x, const float *t, int32_t batch, float *grads,
                      double *loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected) on that loss. */
int lbm_net_train_step(lbm_net_t *n, const float *x, const float *t, int32_t batch, float lr,
                       double *loss);
/* LBM_ETIMEOUT from a network call means a tensor-core kernel gave up
 * waiting on one of its barriers (a bounded wait) and returned early; the
 * network's activations and parameters are then unspecified.  Destroy the
 * network and create a new one; do not reuse it. */
void lbm_net_destroy(lbm_net_t *n);
const char *lbm_net_last_error(const lbm_net_t *n);

/*
 * Checkpoint and resume (the paper has no counterpart: a long solve can be
 * stopped and continued bit for bit).  lbm_save writes the solver state --
 * both lattices in their storage precision (the current one and the one of
 * the step before, which the residual compares against) and the step
 * count -- to the file `path` (created or truncated).  lbm_load reads such
 * a file into a handle created for the same case (same domain, solid mask,
 * links, Kn, parameters and precision: a fingerprint of these is stored in
 * the file and checked) and sets its step count; the following steps and
 * residuals are then those of the saved solver.  Both synchronise the
 * handle's stream.  The file holds a 64-byte header (magic "LBMSTAT1",
 * version, precision, nx, ny, fluid nodes, links, elements per lattice,
 * steps, fingerprint; native byte order) and then the two lattices.
 * Errors: LBM_EINVAL (null path, a file of another case, precision or
 * version), LBM_EIO (the file cannot be opened, written or read in full),
 * LBM_ECUDA, LBM_ENOMEM.
 */
int lbm_save(lbm_handle_t *h, const char *path);
int lbm_load(lbm_handle_t *h, const char *path);

/* ---------------------------------------------------------------------------
 * Three dimensions (D3Q19): the extension the paper names as future work
 * (Sec. 5).  The same collision (MRT in moment space with Guo forcing, Eqs.
 * LBEequi, LBEforce, MomentPost, on the D3Q19 moment basis of d'Humieres et
 * al. 2002), streaming and slip scheme per boundary link (Eq. EqNewBDSC with
 * the D3Q19 weights), with the parameters of Sec. 3.B from the paper's
 * two-dimensional analysis.  The paper gives no three-dimensional
 * derivation; carried out for a D3Q19 flow u_x(z) between walls normal to
 * z, the same analysis reaches the wall relation of Eq. u1u0Coeff exactly
 * when the third-order moments relax with tau_q, which they do here (the
 * fourth-order ones relax with tau_eps), so the slip law of Sec. 3.B holds
 * for 3-D flat channels; for curved 3-D walls it is an extrapolation.
 * Conventions:
 *   * D3Q19 velocities, in this order: (0,0,0); +x, -x, +y, -y, +z, -z; the
 *     diagonals of the xy, xz and yz planes, each as (+,+), (+,-), (-,+),
 *     (-,-) (e.g. 7 = (1,1,0), 12 = (1,0,-1), 18 = (0,-1,-1)).
 *   * Node (x, y, z) has index (z*ny + y)*nx + x; populations are 19*nx*ny*nz
 *     doubles, index q*nx*ny*nz + node.
 *   * A link (x, y, z, i, q, u_b) names a fluid node whose neighbour
 *     x - c_i is solid (or outside a non-periodic axis); every such
 *     (node, direction) needs exactly one link.  link_ub holds 3 doubles per
 *     link.
 *   * Storage LBM_FP64 or LBM_FP32 (deviations f_i - w_i); params as
 *     lbm_create takes them (collision must be MRT; residual_mode does not
 *     apply).  mass_mode as for lbm_create: by default FP32 takes the
 *     exact-mass step where a wall moves or the lattice has no boundary
 *     links (d - d_eq in double-FP32, stochastic rounding of f'_1..f'_18 to
 *     FP32, double-FP32 link values, per-link and per-node carries; about
 *     3.7x the plain step's time).  The lattice
 *     is dense (every node has slots).  Calls synchronise the handle's
 *     stream, except lbm3d_step.
 * ------------------------------------------------------------------------- */
typedef struct lbm3d lbm3d_t;

typedef struct {
  int32_t nx, ny, nz;
  int32_t periodic_x, periodic_y, periodic_z;
  double H;          /* characteristic length (Eq. tKnrela) */
  double ax, ay, az; /* body acceleration */
} lbm3d_domain_t;

int lbm3d_create(const lbm3d_domain_t *dom, const uint8_t *solid, size_t n_links,
                 const int32_t *link_x, const int32_t *link_y, const int32_t *link_z,
                 const int32_t *link_dir, const double *link_q, const double *link_ub, double Kn,
                 const lbm_params_t *params, lbm3d_t **out);
/* Advance n >= 0 time steps (asynchronous on the handle's stream). */
int lbm3d_step(lbm3d_t *h, int64_t n);
/* One-step residual ||u^n - u^(n-1)|| / ||u^n|| and mass over fluid nodes (FP64 sums). */
int lbm3d_residual(lbm3d_t *h, double *residual, double *mass);
/* All populations f_i as 19*nx*ny*nz host doubles (get: solid nodes as w_i;
 * set: replaces both states, steps restart at 0). */
int lbm3d_get_f(lbm3d_t *h, double *f);
int lbm3d_set_f(lbm3d_t *h, const double *f);
/* Density and velocity (Eq. FluidMacr) of every node, nx*ny*nz host doubles
 * each (solid nodes 0; any pointer may be NULL). */
int lbm3d_fields(lbm3d_t *h, double *rho, double *ux, double *uy, double *uz);
/* Per-link r and l as used, in the order the links were given. */
int lbm3d_link_params(const lbm3d_t *h, double *r, double *l);
/* The case's sizes and parameters as lbm_get_info reports them (pitch = nx;
 * exact_mass: 1 if the step runs the exact-mass variant). */
int lbm3d_get_info(const lbm3d_t *h, lbm_info_t *info);
void lbm3d_destroy(lbm3d_t *h);
/* Last error of the handle; with h = NULL, of the last failed lbm3d_create. */
const char *lbm3d_last_error(const lbm3d_t *h);

/* Release the handle and its device memory (waits for its stream).  NULL is a no-op. */
void lbm_destroy(lbm_handle_t *h);

/* Message of the handle's last error ("" if none); with h = NULL, the last
 * failed lbm_create (or handle-less call) on the calling thread. */
const char *lbm_last_error(const lbm_handle_t *h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H_ */
