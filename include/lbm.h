/*
 * lbm.h -- C ABI of the GB300 (sm_103a) pseudo-potential multiphase lattice
 * Boltzmann library (liblbm.so).
 *
 * The method is the Shan-Chen pseudo-potential LB model as analysed in
 * Peng, Ayala, Ayala & Wang, "Isotropy and spurious currents in pseudo-potential
 * multiphase lattice Boltzmann models" (arXiv:1906.11027):
 *   psi(rho) field potential, interaction force F (Eq. 1) on an isotropic force
 *   stencil of 4th..10th order (Sec. 2, Eq. 2) or the lattice itself (the paper's
 *   "consistent implementation", Sec. 3), Guo-forced BGK collision (Eqs. 3-4) or
 *   its moment-space (MRT) form, and periodic pull streaming (Eq. 3), on the
 *   D2Q9, D3Q19, D2Q13 and D2Q25 lattices (Table 1).
 *
 * Conventions shared by every call:
 *  - Return value: LBM_OK (0) or a negative LBM_E* code; lbm_strerror() names
 *    it and lbm_last_error() gives the text of the most recent failure on the
 *    calling thread.  Outputs are written only on success (except
 *    LBM_ENOTCONVERGED from the run-to-steady calls, which still fills them).
 *  - Units: lattice units, dt = dx = 1.  All scalars are double.
 *  - Host arrays are owned by the caller.  Device memory is owned by the
 *    library; it is taken from params.dev_alloc / dev_free when given (e.g. the
 *    PyTorch caching allocator), else from cudaMalloc / cudaFree.
 *  - Cell layout of every host field: x fastest, then y, then z
 *    (index = (z * ny + y) * nx + x).  Populations: [Q][cell] (SoA).
 *  - A context is bound to the device that was current at lbm_create and to
 *    one CUDA stream; it is not thread-safe.  Step calls are asynchronous and
 *    stream-ordered; calls that return host data synchronise the stream.
 *  - Velocity order inside each lattice: the rest vector first, then shells of
 *    increasing |c|^2; inside a shell, the vectors whose first non-zero
 *    component is positive in decreasing lexicographic order, each followed by
 *    its opposite (D2Q9: 0, +x, -x, +y, -y, (1,1), (-1,-1), (1,-1), (-1,1)).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define LBM_OK 0
#define LBM_EINVAL (-1)          /* bad size, tau <= 1/2, unknown enum, NULL pointer */
#define LBM_EUNSUPPORTED (-2)    /* valid but not provided (e.g. MRT on D2Q13) */
#define LBM_ENOMEM (-3)          /* the device allocator failed */
#define LBM_ECUDA (-4)           /* a CUDA runtime/driver call failed */
#define LBM_ENONFINITE (-5)      /* NaN/Inf in the fields, or a negative P-R sqrt argument */
#define LBM_ETIMEOUT (-6)        /* a bounded device wait ran out */
#define LBM_ENOTCONVERGED (-7)   /* run-to-steady reached max_steps */
#define LBM_EIO (-8)             /* checkpoint file could not be read or written */

/* ---- enums --------------------------------------------------------------- */
typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1, LBM_D2Q13 = 2, LBM_D2Q25 = 3 } lbm_lattice;

/* Force stencil by isotropy order (Sec. 2).  LBM_STENCIL_LATTICE uses the
 * lattice's own velocities and weights as the stencil (Sec. 3): order 4 for
 * D2Q9 and D3Q19, 6 for D2Q13, 8 for D2Q25.  2-D supports 4, 6, 8, 10; 3-D 4, 6. */
typedef enum { LBM_STENCIL_LATTICE = 0, LBM_ISO4 = 4, LBM_ISO6 = 6, LBM_ISO8 = 8, LBM_ISO10 = 10 } lbm_stencil;

/* psi(rho): 1 - exp(-rho), or the Peng-Robinson form of Sec. 3,
 * psi = sqrt(2 (p_EOS - c_s^2 rho) / (G c_s'^2)) with a = 2/49, b = 2/21, R = 1,
 * omega = 0.344 and T = T_over_Tc * T_c (T_c the critical point of the EOS). */
typedef enum { LBM_PSI_EXP = 0, LBM_PSI_PENG_ROBINSON = 1 } lbm_psi;

/* LBM_BGK and LBM_MRT use Guo's forcing (Eq. 4).  LBM_BGK_EDM is BGK with the
 * exact-difference forcing the paper's own runs use (Sec. 3):
 *   f* = f - (f - feq(rho, u'))/tau + feq(rho, u' + F/rho) - feq(rho, u'),
 *   u' = sum_b f_b c_b / rho; the reported velocity is u' + F/(2 rho) as with
 *   Guo's scheme.  It is provided for the 2-D lattices (D2Q9, D2Q13, D2Q25);
 *   other lattices return LBM_EUNSUPPORTED. */
typedef enum { LBM_BGK = 0, LBM_MRT = 1, LBM_BGK_EDM = 2 } lbm_collision;

/* Storage and arithmetic precision of the populations.  LBM_FP32_SHIFTED keeps
 * f - w_b rho_bar in float (rho_bar = mean density of the initial state);
 * reductions stay in double. */
typedef enum { LBM_FP64 = 0, LBM_FP32_SHIFTED = 1 } lbm_precision;

/* Kernel schedule of one time step.  Every schedule computes the same step:
 * bit-identical in FP64 and among the one-cell-per-thread FP32 schedules, within
 * FP32 round-off for the packed-pair FP32 ones (see lbm_schedule_report).
 * LBM_PATH_TWO_PASS: a psi kernel writes psi (with periodic ghosts) to its own
 * buffer, then the fused stream-collide-force kernel stages psi tiles plus the
 * stencil halo into shared memory by TMA.  LBM_PATH_ONE_PASS: one kernel
 * marches each tile along z (2-D: y), computing psi of the tile and its halo
 * one slab ahead into a shared-memory ring, so every population is read from
 * HBM once per step.  LBM_PATH_AUTO: the faster of the two, measured on the
 * first step (see lbm_schedule_report). */
typedef enum { LBM_PATH_AUTO = 0, LBM_PATH_TWO_PASS = 1, LBM_PATH_ONE_PASS = 2 } lbm_path;

/* ---- parameters ------------------------------------------------------------ */
typedef struct lbm_params {
    int nx, ny, nz;          /* periodic box; nz = 1 for 2-D lattices; each >= 8 */
    int lattice;             /* lbm_lattice */
    int stencil;             /* lbm_stencil */
    int psi;                 /* lbm_psi */
    double T_over_Tc;        /* Peng-Robinson only */
    double G;                /* interaction strength of Eq. 1 (G < 0 attracts; P-R needs G < 0) */
    double tau;              /* relaxation time, > 1/2 */
    int collision;           /* lbm_collision */
    double s_e, s_eps, s_q;  /* MRT rates of the energy, 4th-order and 3rd-order moments, in (0, 2) */
    int precision;           /* lbm_precision */
    int path;                /* lbm_path */
    void* stream;            /* cudaStream_t to run on; NULL: the library creates its own */
    void* (*dev_alloc)(size_t bytes, void* alloc_ctx);  /* NULL: cudaMalloc */
    void (*dev_free)(void* ptr, void* alloc_ctx);
    void* alloc_ctx;
    /* Wall (Sec. 3, Fig. 6), 2-D lattices, two-pass schedule: the rows
     * y < wall_rows are solid.  A solid node takes no collision and returns every
     * population the way it came, f*_b = f_{-b} (standard bounce-back); in Eq. 1
     * it carries psi(rho_w), the virtual wall density that sets the
     * wettability.  The box stays periodic, so the band is the floor of the fluid
     * and its ceiling; wall_rows must be at least the lattice's reach and the
     * force stencil's radius (LBM_EINVAL otherwise), and psi(rho_w) must exist
     * (Peng-Robinson: LBM_EINVAL if its argument is negative).  0 = no wall
     * (the default; rho_w then unused, default 1). */
    int wall_rows;
    double rho_w;
} lbm_params;

/* Observables of the current state (Sec. 3 measurements):
 * rho_l = rho at the centre node (nx/2, ny/2, nz/2); rho_g = rho at node 0
 * (with a wall: rho_l at (nx/2, wall_rows), the first fluid node above the wall
 * under the centre, rho_g at (0, ny - 1), the top fluid row; max_u, mean_u and
 * mom then run over the fluid nodes, and mass over every node, which is what
 * the scheme conserves);
 * dp = p(rho_l) - p(rho_g) with the bulk pressure p = c_s^2 rho + (G c_s'^2/2) psi^2
 * (= p_EOS for Peng-Robinson); max_u / mean_u = max and mean over cells of |u|,
 * u = (sum f c + F/2) / rho; mass = sum rho; mom = sum rho u; thickness =
 * number of nodes on the x line through the centre with
 * 1.05 rho_g <= rho <= 0.95 rho_l (the interface-thickness measure of Sec. 3,
 * meaningful for a flat interface normal to x); step = steps taken. */
typedef struct lbm_obs {
    double rho_l, rho_g, dp, max_u, mean_u, mass, mom[3], thickness;
    int64_t step;
} lbm_obs;

typedef struct lbm_ctx lbm_ctx;

/* ---- single domain ----------------------------------------------------------- */

/* Fills p with the defaults: 64x64 D2Q9, LBM_STENCIL_LATTICE, exp psi, G = -5,
 * tau = 1, BGK, s_e = 1.64, s_eps = 1.54, s_q = 1.9, FP64, auto path, no stream,
 * cudaMalloc. */
int lbm_params_default(lbm_params* p);

/* Validates p, builds the lattice/stencil tables, allocates the two population
 * buffers, the ghosted psi buffer and the reduction scratch on the current
 * device, and encodes the TMA descriptor of the psi buffer.  The populations
 * start at zero; call an lbm_init_* before stepping.  *out is set on success. */
int lbm_create(const lbm_params* p, lbm_ctx** out);

/* Synchronises the stream and frees everything the context owns. NULL is a no-op. */
int lbm_destroy(lbm_ctx* ctx);

/* Static droplet (Sec. 3): rho0 = (rl + rg)/2 - (rl - rg)/2 tanh(2 (r - R) / width),
 * r the periodic distance to the centre node (nx/2, ny/2, nz/2); populations
 * f = feq(rho0, u = 0) = w_b rho0.  Resets the step counter. */
int lbm_init_droplet(lbm_ctx* ctx, double rho_l, double rho_g, double R, double width);

/* Flat liquid slab normal to `axis` (0 = x, 1 = y, 2 = z) on [L/4, 3L/4): the same
 * tanh profile with r = |i - L/2| and R = L/4. */
int lbm_init_flat(lbm_ctx* ctx, double rho_l, double rho_g, double width, int axis);

/* f = w_b rho0 from a host density field of nx*ny*nz doubles. */
int lbm_init_from_rho(lbm_ctx* ctx, const double* rho_host);

/* Pre-collision populations f_b(x, n) in double, [Q][cell], to / from host
 * arrays of Q*nx*ny*nz doubles (the state the step of Eq. 3 acts on). */
int lbm_get_populations(lbm_ctx* ctx, double* f_host);
int lbm_set_populations(lbm_ctx* ctx, const double* f_host);

/* Advances n >= 0 time steps (Eq. 3), asynchronously on the context's stream. */
int lbm_step(lbm_ctx* ctx, int64_t n);

/* Like lbm_step, but without graph replay and with CUDA events recorded on the
 * context's stream around every kernel; synchronises at the end.  mean_ms
 * (capacity max_kernels) receives the mean duration of each kernel position of
 * one step, *nkernels their number; lbm_step_kernel_name() names position i. */
int lbm_step_timed(lbm_ctx* ctx, int64_t n, double* mean_ms, int max_kernels, int* nkernels);
const char* lbm_step_kernel_name(const lbm_ctx* ctx, int i);

/* Names the step schedule in use and the time per step of every candidate the
 * autotuner measured, as "chosen=NAME;NAME=ms;..." in buf (NUL-terminated,
 * truncated to len).  With LBM_PATH_AUTO / LBM_PATH_ONE_PASS the first
 * lbm_step (or this call) times each compiled variant (tile shape, chunk
 * length, register cap; and the two-pass schedule under AUTO) on the current
 * state, without advancing it, and keeps the fastest.  The variants compute the
 * same step; FP64 and one-cell-per-thread FP32 variants are bitwise alike, while
 * the packed-pair FP32 variants order their float operations differently and
 * agree within FP32 round-off. */
int lbm_schedule_report(lbm_ctx* ctx, char* buf, int len);

/* Pins the step schedule to the named candidate (a name lbm_schedule_report
 * lists, e.g. "two_pass"), skipping the autotuner.  LBM_EINVAL if the name is
 * not a candidate of this context's path. */
int lbm_set_schedule(lbm_ctx* ctx, const char* name);

/* Steps until the change of max|u| between checks taken every `check_every`
 * steps, divided by check_every, is below tol (FP32 storage adds the floor
 * 1e-6 max|u| / check_every for its round-off), or until max_steps.  Returns
 * LBM_ENOTCONVERGED at max_steps.  *steps_out (may be NULL) = steps taken. */
int lbm_run_to_steady(lbm_ctx* ctx, double tol, int64_t max_steps, int64_t check_every,
                      int64_t* steps_out);

/* Observables of the current state (see lbm_obs); synchronises.  Returns
 * LBM_ENONFINITE if any cell holds NaN/Inf or an invalid P-R argument. */
int lbm_observables(lbm_ctx* ctx, lbm_obs* out);

/* Density (nx*ny*nz) and velocity (3 per cell, xyz, u = (sum f c + F/2)/rho)
 * to host arrays; either may be NULL.  Synchronises. */
int lbm_get_fields(lbm_ctx* ctx, double* rho_host, double* u_host);

/* Device pointer and layout of the current population buffer, for callers
 * that time or inspect the kernels: *elem_bytes = 8 (FP64) or 4 (FP32
 * deviations), [Q][cell]. */
int lbm_device_state(lbm_ctx* ctx, const void** f_dev, int* Q, int64_t* ncells, int* elem_bytes);

/* Raw checkpoint: header (magic, version, parameters, step, rho_bar) followed by
 * the population buffer.  lbm_load needs a context created with the same
 * parameters and restores a bit-identical trajectory. */
int lbm_save(lbm_ctx* ctx, const char* path);
int lbm_load(lbm_ctx* ctx, const char* path);

/* Algorithmic HBM bytes of one lattice update for this context's lattice and
 * precision: 2 Q s_f + 2 s_psi (one read and one write of every population,
 * one write and one read of psi). */
double lbm_bytes_per_update(const lbm_ctx* ctx);

/* ---- batched sweep of independent 2-D domains --------------------------------- */

/* A batch advances n independent periodic D2Q9 domains (each with its own size,
 * G, tau and force-stencil order; exp psi, BGK, one precision for all) with one
 * persistent kernel per step over a work list of (domain, tile, row chunk)
 * items, inside a CUDA graph that also checks every domain for steady state;
 * converged domains retire from the work list (the parameter study of the
 * paper's Sec. 3, run as one job). */
typedef struct lbm_batch lbm_batch;

/* ps[d]: lattice = LBM_D2Q9, psi = LBM_PSI_EXP, collision = LBM_BGK, nx, ny >= 8,
 * nz = 1, stencil 0/4/6/8/10, G, tau; precision, stream and allocator are taken
 * from ps[0] (all precisions equal).  init[4d .. 4d+3] = rho_l, rho_g, R, width of
 * domain d's centred tanh droplet (as lbm_init_droplet). */
int lbm_batch_create(const lbm_params* ps, const double* init, int n, lbm_batch** out);
int lbm_batch_destroy(lbm_batch* b);

/* n steps of every active domain, without checks (asynchronous). */
int lbm_batch_step(lbm_batch* b, int64_t n);

/* Replays blocks of check_every (even) steps until every domain satisfies
 * |max|u|(t) - max|u|(t - K)| / K < tol (FP32 adds the floor 1e-6 max|u| / K) or
 * max_steps.  steps_per_domain[d] (may be NULL) = steps domain d took before it
 * retired; obs_per_domain[d] (may be NULL) = its observables (rho_l, rho_g, dp,
 * max_u, mean_u, mass, mom, step; thickness 0).  A domain whose fields become
 * non-finite (the BGK pseudo-potential model diverges for some strong-G, small-tau
 * pairs) retires at that check with max_u = +inf.  LBM_ENOTCONVERGED if domains
 * remain active at max_steps (outputs still filled). */
int lbm_batch_run_to_steady(lbm_batch* b, double tol, int64_t max_steps, int64_t check_every,
                            int64_t* steps_per_domain, lbm_obs* obs_per_domain);
int lbm_batch_observables(lbm_batch* b, lbm_obs* obs_per_domain);

/* Pre-collision populations of domain d in double, [9][ny][nx], from / to host
 * arrays (set_populations writes the buffer that holds the domain's state, e.g.
 * to continue in FP64 a domain converged in FP32). */
int lbm_batch_get_populations(lbm_batch* b, int d, double* f_host);
int lbm_batch_set_populations(lbm_batch* b, int d, const double* f_host);

/* Tile shape of the batch step kernel (cells per tile along x by rows per work
 * item): "tileTX_rowsZC" shapes gather populations per thread; "stagedTX_rowsZC"
 * shapes stage each row segment in shared memory with bulk copies (FP32 batches
 * whose every nx is a multiple of 4 only).  The first lbm_batch_step /
 * lbm_batch_run_to_steady (or this call) times every applicable shape for a few
 * steps on the batch's current state, restores the state, and keeps the
 * fastest; all shapes perform the same per-cell arithmetic, so results are
 * bitwise the same whichever is chosen.  The report is "chosen=NAME;NAME=ms;..."
 * in buf (NUL-terminated, truncated to len). */
int lbm_batch_schedule_report(lbm_batch* b, char* buf, int len);

/* Pins the tile shape to the named one, skipping the autotuner; LBM_EINVAL for
 * an unknown name or a staged shape the batch does not qualify for. */
int lbm_batch_set_schedule(lbm_batch* b, const char* name);

/* ---- learned warm start ------------------------------------------------------ */

/* A multilayer perceptron 5 -> 128 -> 128 -> 128 -> 128 -> 1 with SiLU activations
 * that maps scaled features (G, tau, stencil order, R, signed distance d to the
 * interface) to the steady density of a droplet, trained on steady profiles the
 * method itself produces; it only initialises the relaxation (the LB step decides
 * the result).  Weights are FP32 masters with BF16 copies; the GEMMs of training
 * and inference run on the tensor cores with FP32 accumulation.
 * Features (lbm_mlp_features): ((G + 4.9)/0.6, (tau - 0.8)/0.2, (order - 7)/3,
 * (min(10/R, 2) - 0.5)/0.4, d/24): the radius enters as a curvature (capped at
 * that of R = 5), and d spans |d| <= 24, the interface and the bulk on both
 * sides.  Parameter vector: W1 [5][128], b1, W2 [128][128], b2, W3,
 * b3, W4, b4, W5 [128][1], b5 (50,433 floats); z = h W + b. */
typedef struct lbm_mlp lbm_mlp;
int lbm_mlp_create(lbm_mlp** out, uint64_t seed);   /* He-uniform weights from SplitMix64(seed) */
int lbm_mlp_destroy(lbm_mlp* net);
int lbm_mlp_num_params(void);
int lbm_mlp_get_params(const lbm_mlp* net, float* params_out);
int lbm_mlp_set_params(lbm_mlp* net, const float* params);
/* raw: n x (G, tau, order, R, d) doubles -> out: n x 5 scaled floats */
int lbm_mlp_features(const double* raw, int64_t n, float* out);
/* y[i] = network(X[i]) for n scaled feature rows (host arrays) */
int lbm_mlp_predict(lbm_mlp* net, const float* X, int64_t n, float* y);
/* mean-squared-error loss of one batch and its gradient w.r.t. every parameter */
int lbm_mlp_loss_grad(lbm_mlp* net, const float* X, const float* y, int n, double* loss, float* grad_out);
/* Adam (lr, beta 0.9/0.999, eps 1e-8) over `epochs` passes of mini-batches of
 * `batch` rows (a SplitMix64 permutation per epoch); *final_loss = mean loss of
 * the last epoch. */
int lbm_mlp_train(lbm_mlp* net, const float* X, const float* y, int64_t n, int epochs, double lr, int batch,
                  double* final_loss);
int lbm_mlp_save(const lbm_mlp* net, const char* path);
int lbm_mlp_load(lbm_mlp** out, const char* path);

/* Warm start of a centred droplet (psi = 1 - exp(-rho) contexts): the density is
 * the network's profile for the context's G, tau and stencil order at radius
 * R_eff, R_eff chosen by bisection so that the total mass equals that of the
 * tanh droplet (rho_l, rho_g, R, width) of lbm_init_droplet, the remainder removed
 * by a uniform shift; populations f = w_b rho0.  On D3Q19 the network, which
 * holds 2-D profiles, is evaluated at radius R_eff/2, the 2-D droplet with the
 * same Laplace pressure jump (2 sigma/R in 3-D), and the profile is placed at
 * R_eff.  Falls back to the tanh droplet
 * (*used_fallback = 1) if the network gives a non-finite or non-positive
 * density, and for G > -4.65, where close to the critical coupling G_c = -4 the
 * steady state (droplet or none, and the current it carries) depends on the
 * initial state.  *R_eff_out (may
 * be NULL) = the radius used. */
int lbm_init_droplet_learned(lbm_ctx* ctx, lbm_mlp* net, double R, double rho_l, double rho_g, double width,
                             int* used_fallback, double* R_eff_out);

/* Mass and momentum totals of a population buffer, computed without allocating
 * anything.  The paper has no counterpart: this serves callers that cannot
 * allocate device memory at the moment they need the totals, such as an
 * application whose device memory is all reserved up front by another
 * framework's pool, or a service that must not call cudaMalloc on its
 * latency-critical path.
 *   f_dev     populations in the library's layout: [Q][cell], the
 *             post-collision buffer that lbm_device_state returns; double for
 *             LBM_FP64, float deviations from w_b rho_bar for LBM_FP32_SHIFTED
 *   lattice, precision, nx, ny, nz, rho_bar   describe that buffer (rho_bar is
 *             ignored for LBM_FP64; for a context's buffer it is the value
 *             lbm_reference_density returns)
 *   stream    cudaStream_t the kernels run on (NULL: the legacy default stream);
 *             the call synchronises it.  The caller orders it after the work
 *             that writes f_dev: a context steps on its own stream, which is a
 *             non-blocking stream when lbm_params.stream was NULL, so pass that
 *             stream or synchronise it first
 *   out_host  4 doubles: sum over every cell of rho, then of sum_b f_b c_b
 *             (x, y, z), the momentum before the half-force term.  With a wall
 *             the sums include the solid band (lbm_observables takes its
 *             momentum over the fluid nodes only; its mass also covers every
 *             cell)
 * The block partials live in one static device array of about 512 KiB that
 * every GPU loading the library keeps until exit, so at most 16,777,216 cells
 * are accepted (LBM_EINVAL beyond, with a message in lbm_last_error()).  The
 * first call on a device looks the array up with cudaGetSymbolAddress; make it
 * before any stream capture.  Every call shares the array: calls that overlap
 * on the GPU race and must be serialised by the caller. */
int lbm_moments_noalloc(const void* f_dev, int lattice, int precision, int nx, int ny, int nz,
                        double rho_bar, void* stream, double* out_host);

/* The reference density rho_bar of a context's FP32 deviation storage
 * (populations kept as f_b - w_b rho_bar): the mean density of the state the
 * context was last initialised or loaded from.  0 for LBM_FP64 contexts.  This
 * is the value to pass to lbm_moments_noalloc with lbm_device_state's buffer. */
int lbm_reference_density(lbm_ctx* ctx, double* rho_bar);

/* Failure-detection check (the paper has no counterpart).  Launches one block
 * whose thread waits, through the same time-bounded mbarrier wait that the
 * staged step kernels use, on a shared-memory barrier that nothing completes
 * and against which no copy is issued.  The wait gives up after about 2 s; the
 * kernel records the timeout in the context's device error word and returns
 * with nothing in flight, and the call reports the word exactly as a step's
 * readback would: LBM_ETIMEOUT is the expected result (any other code means
 * the wait or the reporting is broken).  The context stays usable afterwards.
 * Synchronises the context's stream. */
int lbm_diag_wait_timeout(lbm_ctx* ctx);

const char* lbm_strerror(int code);
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
