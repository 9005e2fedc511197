/*
 * lbm_ewod.h -- C ABI of the GB300 D2Q9 Shan-Chen electrowetting library.
 *
 * The library advances the lattice Boltzmann model of Li, Li, Chen & Fang,
 * "Lattice Boltzmann simulation of electrowetting-on-dielectric in a
 * rough-wall channel" (arXiv:0708.4182) on one GPU. One time step is one
 * fused CUDA kernel launch that performs, for every fluid node x:
 *
 *   streaming      f_a(x, t) = f*_a(x - e_a, t-1), periodic in x and y,
 *                  half-way bounce-back where x - e_a is solid  (left side of Eq. 1)
 *   moments        rho = sum_a f_a,  rho u = sum_a f_a e_a      (Eq. 2)
 *   pseudopotential psi = rho0 (1 - exp(-rho/rho0))              (text after Eq. 4)
 *   forces         F_sigma = -psi(x) sum_a G_a psi(x+e_a) e_a    (Eq. 5)
 *                  F_w     = -psi(x) sum_a W_a S(x+e_a) e_a      (Eq. 6)
 *                  f n on conductive (rho >= rho_c) fluid nodes of the
 *                  single layer next to a wall                  (Eq. 9 and the
 *                                                                 critical-density paragraph)
 *                  rho * body force (channel runs)
 *   velocity shift rho u' = rho u + tau (F_sigma + F_w + f + F_b) (Eq. 10)
 *   BGK collision  f*_a = f_a - (f_a - f_a^eq(rho, u'))/tau     (Eq. 1, Eq. 3)
 *
 * Readings of points the paper leaves open (see the parameter comments):
 * Green-function magnitudes (lbm_params.green), psi = 0 on solid nodes in
 * Eq. 5, the electric force as f per solid axis face of a conductive
 * wall-layer node, the body force as rho * (body_fx, body_fy), half-way
 * bounce-back walls, and observables with u = (sum_a f_a e_a + F/2)/rho.
 *
 * Conventions
 *  - Directions in the paper's order: e0 = (0,0); e1..e4 = (1,0), (0,1),
 *    (-1,0), (0,-1); e5..e8 = (1,1), (-1,1), (-1,-1), (1,-1).
 *  - Field arrays crossing the ABI are row-major, x fastest, dense (no
 *    padding): populations as double[9][ny][nx], (rho, ux, uy) as
 *    double[3][ny][nx], the solid mask as uint8_t[ny][nx] (1 = solid).
 *  - "on_device" = 1 means the pointer is CUDA device memory readable on
 *    the context's stream; 0 means ordinary host memory. All inputs are
 *    copied: the caller keeps ownership of every buffer it passes.
 *  - Nothing is thrown across the ABI. Every call returns an lbm_status;
 *    lbm_last_error() gives a message for the last failure on a context.
 *  - Work is enqueued on the context's CUDA stream. lbm_step returns as
 *    soon as the launches are enqueued; calls that hand data back to the
 *    host synchronise that stream.
 *  - A context is not thread-safe; use one context per thread.
 */
#ifndef LBM_EWOD_H
#define LBM_EWOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque; one per simulation domain */

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,   /* bad argument: null pointer, size, parameter range */
    LBM_ENOMEM = 2,   /* workspace too small, or host allocation failed */
    LBM_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
    LBM_ENAN = 4,     /* observables found non-finite density or velocity */
    LBM_ETIMEOUT = 5, /* a bounded device-side wait gave up */
    LBM_ESTATE = 6,   /* call out of order (e.g. step before geometry and field) */
    LBM_ENOTCONV = 7  /* lbm_run_to_steady reached max_steps before the criterion */
} lbm_status;

/* Green-function magnitudes for Eq. 4-6. LBM_GREEN_MC (the default) uses
 * Martys & Chen's convention, G on axis links (|e| = 1) and G/2 on diagonal
 * links (|e| = sqrt 2), for both G_a and W_a; with the paper's G = -0.52 this
 * gives liquid/vapor densities 2.805/0.0631 around rho_c = 1 and runs stably
 * at the paper's tau = 0.9. LBM_GREEN_PRINTED uses the weights as printed with
 * Eq. 4 (2G axis, G diagonal), which diverges at G = -0.52. */
enum { LBM_GREEN_MC = 0, LBM_GREEN_PRINTED = 1 };

/* Direction of the electric force f n of Eq. 9 at a wall-layer node.
 * LBM_NORMAL_FACES (the default): f per solid axis face, pointing into that
 * face, summed (a concave corner where two perpendicular faces meet gets f
 * along each). LBM_NORMAL_UNIT: the same sum of face directions scaled to
 * unit length (a concave corner gets f along the diagonal). The two differ
 * only where two perpendicular solid faces meet. */
enum { LBM_NORMAL_FACES = 0, LBM_NORMAL_UNIT = 1 };

/* Thread layout of the step kernel for the 32-bit storage forms (the 16-bit
 * forms have one layout and ignore the field). No counterpart in the paper:
 * both layouts compute the same update and store the same bits.
 * LBM_LAYOUT_PAIRS: each thread updates two neighbouring nodes with paired
 *                   FP32 instructions (fewer instructions per node; the
 *                   faster layout once the domain fills the GPU).
 * LBM_LAYOUT_SINGLE: one node per thread (twice the threads per CTA, which
 *                   hide more latency on small domains).
 * LBM_LAYOUT_AUTO (0, the default): pairs unless the domain (a batch: all
 *                   its domains together) gives no more than 3 CTAs per SM
 *                   at 4-row segments. A batch takes the first domain's
 *                   field. */
enum { LBM_LAYOUT_AUTO = 0, LBM_LAYOUT_PAIRS = 1, LBM_LAYOUT_SINGLE = 2 };

/* Population storage in device memory (arithmetic is FP32 in all forms).
 * LBM_FP32:     the post-collision populations f*_a, FP32 (36 B per node).
 * LBM_FP32_DEV: rho* = sum_a f*_a (FP32) and the deviations
 *               d_a = f*_a - w_a rho* from the node's weighted rest
 *               equilibrium, FP32 (36 B per node). Slow flows whose per-step
 *               change is below half an ulp of a plain FP32 population keep
 *               evolving in this form (plain FP32 stalls short of the steady
 *               state, e.g. 0.4% low in the flux of a channel driven by 1e-6).
 * LBM_FP16_DEV / LBM_BF16_DEV: as LBM_FP32_DEV with d_a in 16 bits (20 B per
 *               node, rounded to nearest; FP16 holds 2^12 d_a, so |d_a| must
 *               stay below 16); nx must be a multiple of 8. */
enum { LBM_FP32 = 0, LBM_FP32_DEV = 1, LBM_FP16_DEV = 2, LBM_BF16_DEV = 3 };

/* Field selectors for lbm_set_field / lbm_get_field (LBM_RHO_U_PHYS and
 * LBM_RHO: set only; LBM_UX_PROFILE: get only). */
enum { LBM_RHO_U = 0, LBM_POPS = 1, LBM_RHO_U_PHYS = 2, LBM_UX_PROFILE = 3, LBM_RHO = 4 };

typedef struct {
    int32_t nx, ny;    /* lattice size; x and y are periodic, walls come
                          from the solid mask */
    double tau;        /* BGK relaxation time (Eq. 1), > 0.5 */
    double G;          /* fluid-fluid strength (calligraphic G, Eq. 4); paper -0.52 */
    double G_wall;     /* fluid-wall strength w (Eq. 6); paper -0.14 */
    double rho0;       /* psi constant; paper 1.0 */
    double rho_c;      /* critical density: rho >= rho_c is conductive; paper 1.0 */
    double f_elec;     /* electric force f per wall-layer node (Eq. 9), >= 0 */
    double body_fx;    /* body-force acceleration; the paper drives its */
    double body_fy;    /*   channels with a rightward f_b                */
    int32_t green;     /* LBM_GREEN_MC or LBM_GREEN_PRINTED */
    int32_t storage;   /* LBM_FP32, LBM_FP32_DEV, LBM_FP16_DEV or LBM_BF16_DEV */
    int32_t obs_every; /* K > 0: every step whose index t is a multiple of K
                          also reduces the observables of state t, fused into
                          the step kernel (read with lbm_obs_latest); 0: off */
    int32_t tile_rows; /* rows per CTA segment of the step kernel (>= 4), 0 = auto */
    int32_t normal;    /* LBM_NORMAL_FACES or LBM_NORMAL_UNIT */
    int32_t layout;    /* LBM_LAYOUT_AUTO, LBM_LAYOUT_PAIRS or LBM_LAYOUT_SINGLE */
} lbm_params;

typedef struct {
    int64_t step;      /* time index t of the state these values describe */
    double mass;       /* sum of rho over fluid nodes */
    double flux_Q;     /* Eq. 11: (1/nx) * sum over fluid nodes of u_x */
    double mom_x;      /* sum of rho u over fluid nodes, u = (sum f e + F/2)/rho */
    double mom_y;
    double max_u;      /* max |u| over fluid nodes */
    double min_rho;    /* min rho over fluid nodes */
    int64_t nonfinite; /* fluid nodes whose rho or u is NaN/Inf (not in the sums) */
} lbm_obs;

/* Bytes of device workspace a context with these parameters needs (0 if the
 * parameters are invalid). The caller allocates it (e.g. as a torch tensor). */
size_t lbm_workspace_bytes(const lbm_params *params);

/* Create a context. d_workspace: device memory of at least
 * lbm_workspace_bytes(params) bytes, 256-byte aligned, owned by the caller
 * and kept alive until lbm_destroy. cuda_stream: the cudaStream_t all work is
 * enqueued on (NULL = legacy default stream). Errors: LBM_EINVAL for invalid
 * parameters or pointers, LBM_ENOMEM if bytes is too small. On success *out
 * receives the context; on failure *out is NULL. */
lbm_status lbm_create(const lbm_params *params, void *d_workspace, size_t bytes,
                      void *cuda_stream, lbm_ctx **out);

/* Set the solid mask S of Eq. 6 (uint8_t[ny][nx], nonzero = solid). Resets
 * the time index to 0 and invalidates the populations: lbm_set_field must
 * follow before lbm_step. */
lbm_status lbm_set_geometry(lbm_ctx *ctx, const uint8_t *solid, int on_device);

/* Set the state at the current time index.
 * LBM_RHO_U: data = double[3][ny][nx] (rho, ux, uy); every fluid node gets
 *            f_a = f_a^eq(rho, u) of Eq. 3. Values on solid nodes are ignored.
 * LBM_RHO_U_PHYS: data as for LBM_RHO_U, with u the physical velocity
 *            (sum_a f_a e_a + F/2)/rho that lbm_get_field(LBM_RHO_U) and the
 *            observables report: f_a = f_a^eq(rho, u - F/(2 rho)), F the
 *            total force (Eqs. 5 and 6, the electric force, the body force)
 *            of the given density field, in FP64. Reading the field back
 *            returns (rho, u) up to storage rounding, so a run restarted
 *            from a (rho, u) snapshot does not receive the momentum kick
 *            F/2 per node that LBM_RHO_U gives at interfaces.
 * LBM_RHO:   data = double[ny][nx], the density of a fluid at rest: every
 *            fluid node gets f_a = w_a rho (Eq. 3 at u = 0), the same state
 *            LBM_RHO_U gives with zero velocity, from a third of the data.
 * LBM_POPS:  data = double[9][ny][nx], the populations f_a(x, t) after
 *            streaming (the f of Eq. 2). Values on solid nodes are ignored.
 * Populations are rounded to the storage type. Needs lbm_set_geometry first
 * (LBM_ESTATE otherwise). */
lbm_status lbm_set_field(lbm_ctx *ctx, int which, const double *data, int on_device);

/* Set the state of a fluid at rest from an FP32 density rho = float[ny][nx]
 * (host or device memory, on_device as for lbm_set_field; values on solid
 * nodes are ignored). The state is the one LBM_RHO describes (f_a = w_a rho,
 * Eq. 3 at u = 0, after streaming) with FP32 arithmetic and weights: the
 * post-collision populations are f*_a(x) = w_a rho(s_a), s_a = x + e_a or, if
 * that node is solid, x (the half-way bounce-back); the deviation forms store
 * rho* = rho(x) + delta with delta = sum_a w_a (rho(s_a) - rho(x)) and
 * d_a = w_a ((rho(s_a) - rho(x)) - delta). One memory-bound kernel on half the
 * bytes of LBM_RHO's FP64 input; the populations differ from LBM_RHO's by
 * FP32 rounding. No counterpart in the paper (a set-up path). Needs
 * lbm_set_geometry first (LBM_ESTATE otherwise); LBM_EINVAL for NULL. */
lbm_status lbm_set_density_f32(lbm_ctx *ctx, const float *rho, int on_device);

/* Read the current state into out (layouts as for lbm_set_field).
 * LBM_RHO_U: rho and the velocity u = (sum_a f_a e_a + F/2)/rho, 0 on solids.
 * LBM_POPS:  post-streaming populations f_a(x, t), 0 on solids.
 * LBM_UX_PROFILE: double[ny], the mean velocity profile across the channel
 *            u_x(y) averaged over x, (1/nx) sum_x u_x(x, y), solid nodes
 *            counting 0 (the channel velocity profiles of the paper's
 *            rough-channel figures; summed over y it is Eq. 11's Q).
 * Synchronises the context's stream when out is host memory. */
lbm_status lbm_get_field(lbm_ctx *ctx, int which, double *out, int on_device);

/* Advance nsteps >= 0 time steps (asynchronous). Runs of 32 plain steps
 * with no fused-observables step among them are replayed as one CUDA graph
 * (built on first use, per context). LBM_ESTATE before geometry and field
 * are set. */
lbm_status lbm_step(lbm_ctx *ctx, int64_t nsteps);

/* Self-test of the device-side timeout path (no counterpart in the paper):
 * one kernel waits, with the step kernel's bounded mbarrier wait (2^18
 * polls), on an mbarrier phase that nothing completes. The wait gives up and
 * raises the context's error flag, and the call returns LBM_ETIMEOUT once the
 * stream has drained (about a second). The flag is cleared when read, so the
 * context stays usable. Any other status means the timeout path is broken. */
lbm_status lbm_selftest_timeout(lbm_ctx *ctx);

/* Observables of the current state (Eq. 11 and mass/momentum bookkeeping),
 * computed by an extra read-only pass; synchronises the stream. Returns
 * LBM_ENAN (with *out filled) if any fluid node is non-finite. */
lbm_status lbm_observables(lbm_ctx *ctx, lbm_obs *out);

/* Step until the flux of Eq. 11 is steady: every check_every steps compute
 * Q (an observables pass) and stop once |Q(t) - Q(t - check_every)| <=
 * rel_tol * |Q(t)|, or after max_steps more steps. *out receives the
 * observables of the last check (out->step is the time index reached).
 * Returns LBM_OK when the criterion was met, LBM_ENOTCONV when max_steps ran
 * out first (with *out filled), LBM_ENAN as lbm_observables, LBM_EINVAL for
 * check_every < 1 or rel_tol < 0. Synchronises the stream at every check. */
lbm_status lbm_run_to_steady(lbm_ctx *ctx, double rel_tol, int64_t check_every, int64_t max_steps,
                             lbm_obs *out);

/* The most recent observables fused into lbm_step (params.obs_every > 0):
 * those of the last state t < current time with t % obs_every == 0.
 * Synchronises the stream. LBM_ESTATE if none has been recorded yet;
 * LBM_ENAN as for lbm_observables. */
lbm_status lbm_obs_latest(lbm_ctx *ctx, lbm_obs *out);

/* As lbm_obs_latest without the synchronisation: enqueues the copy of that
 * record into *out (host memory) on the context's stream and returns. *out
 * is valid once the stream has passed this point (e.g. after an event
 * recorded next completes) and must stay allocated until then; page-locked
 * memory keeps the copy asynchronous (pageable memory makes it synchronous,
 * as for any CUDA copy). The caller checks out->nonfinite itself. Lets a
 * host loop read every step's result while the next step runs. LBM_ESTATE
 * if no record exists yet. */
lbm_status lbm_obs_latest_async(lbm_ctx *ctx, lbm_obs *out);

/* Current time index (steps taken since the last lbm_set_geometry). */
int64_t lbm_time(const lbm_ctx *ctx);

/* Message for the last error on ctx ("" if none); valid until the next call. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Static name of a status code. */
const char *lbm_status_string(int status);

/* Destroy a context. Frees only what the library allocated (host-side
 * bookkeeping); the caller's workspace is untouched. NULL is a no-op. */
void lbm_destroy(lbm_ctx *ctx);

/* ------------------------------------------------------------------------
 * Batches: many domains (different sizes, geometries and forces, one
 * storage form) advanced together, one persistent kernel launch per step.
 * Not in the paper, which runs its sweeps (over f and channel width) one
 * domain at a time; a batch runs such a sweep as one job.
 */
typedef struct lbm_batch lbm_batch;

/* Device workspace for count domains with parameters params[0..count-1]
 * (0 if any parameter set is invalid or the storage forms differ). */
size_t lbm_batch_workspace_bytes(const lbm_params *params, int32_t count);

/* Create a batch in the caller's workspace (256-byte aligned, owned by the
 * caller, kept alive until lbm_batch_destroy). Every domain gets an ordinary
 * context carved from it; fetch it with lbm_batch_domain and use the
 * single-domain calls (lbm_set_geometry, lbm_set_field, lbm_get_field,
 * lbm_observables, ...) on it. */
lbm_status lbm_batch_create(const lbm_params *params, int32_t count, void *d_workspace, size_t bytes,
                            void *cuda_stream, lbm_batch **out);

/* The context of domain i (owned by the batch; NULL if i is out of range). */
lbm_ctx *lbm_batch_domain(lbm_batch *b, int32_t i);

/* Advance every active domain by nsteps. Each step is one launch of a
 * persistent kernel whose CTAs walk a tile list (domain, strip, row segment)
 * covering all active domains; pairs of steps run as one CUDA graph. */
lbm_status lbm_batch_step(lbm_batch *b, int64_t nsteps);

/* Observables of every domain (one batched pass), out[count]. */
lbm_status lbm_batch_observables(lbm_batch *b, lbm_obs *out);

/* active[count]: nonzero = stepped by lbm_batch_step (all start active). */
lbm_status lbm_batch_set_active(lbm_batch *b, const uint8_t *active);

/* Row-segment height of the tiles (>= 4; 0 = each domain's own default). */
lbm_status lbm_batch_set_tile_rows(lbm_batch *b, int32_t rows);
int32_t lbm_batch_tile_rows(const lbm_batch *b);

/* Time candidates[0..n-1] as tile heights over `steps` steps each (after 2
 * warm-up steps) with CUDA events, keep the fastest (*chosen) and report
 * ms_per_step[n] (may be NULL). Advances every active domain by
 * n * (steps + 2) steps. */
lbm_status lbm_batch_autotune(lbm_batch *b, const int32_t *candidates, int32_t n, int32_t steps,
                              int32_t *chosen, double *ms_per_step);

/* Resident CTAs per SM of the persistent grid: 1 up to the most that fit
 * on one SM (shared memory and registers of the batch's step kernel, from
 * the CUDA occupancy query at creation; that maximum is the default).
 * LBM_EINVAL outside that range. */
lbm_status lbm_batch_set_ctas_per_sm(lbm_batch *b, int32_t ctas);
int32_t lbm_batch_ctas_per_sm(const lbm_batch *b);

/* Autotune over tile height x CTAs per SM: every pair (rows[i], ctas[j]) is
 * timed as in lbm_batch_autotune, ms_per_step[j * nrows + i] (may be NULL)
 * gets its time, and the fastest pair is kept (*chosen_rows, *chosen_ctas).
 * Advances every active domain by nrows * nctas * (steps + 2) steps. */
lbm_status lbm_batch_autotune_grid(lbm_batch *b, const int32_t *rows, int32_t nrows, const int32_t *ctas,
                                   int32_t nctas, int32_t steps, int32_t *chosen_rows, int32_t *chosen_ctas,
                                   double *ms_per_step);

/* Step the active domains until each one's flux is steady (criterion as in
 * lbm_run_to_steady, checked every check_every steps); a domain stops being
 * stepped once it is steady. steps_to_steady[count] gets each domain's time
 * index at convergence (-1 if inactive or not converged, -2 if it became
 * non-finite: such a domain is dropped and the others run on), out[count]
 * its last observables. LBM_ENAN if some domain became non-finite, else
 * LBM_ENOTCONV if some active domain did not converge within max_steps.
 * With an explicit tile height (lbm_batch_set_tile_rows or the autotuners),
 * the height is halved, down to 4 rows, whenever the domains still running
 * give fewer than two waves of tiles for the persistent grid (a tiling
 * change leaves every population bit for bit as it was). The caller's
 * active set and tile height are restored on return. */
lbm_status lbm_batch_run_to_steady(lbm_batch *b, double rel_tol, int64_t check_every, int64_t max_steps,
                                   int64_t *steps_to_steady, lbm_obs *out);

const char *lbm_batch_last_error(const lbm_batch *b);

/* Destroy the batch and its domain contexts (not the caller's workspace). */
void lbm_batch_destroy(lbm_batch *b);

/* Observables without a context and without any allocation. The paper has
 * no counterpart to this entry point: it exists for callers that cannot
 * allocate device memory at the moment they need the numbers. Examples are
 * a host process working inside a fixed device memory budget that is
 * already spent (an allocation there would fail or evict something else),
 * and monitoring or checkpoint tools that hold a state in their own buffers
 * and must not touch the allocator of the application they observe.
 *
 * Inputs (device memory, owned by the caller): d_pops, the post-streaming
 * populations as double[9][ny][nx] (the LBM_POPS layout of lbm_get_field);
 * d_solid, the mask as uint8_t[ny][nx]. params gives nx, ny and the model
 * parameters (tau, G, G_wall, rho0, rho_c, f_elec, body force, green; the
 * storage, obs_every and tile_rows fields are only validated). step is
 * copied into out->step. Output: *out, host memory, filled as
 * lbm_observables fills it (same per-node arithmetic, partial sums in a
 * different order). The call enqueues its work on cuda_stream and then
 * synchronises that stream.
 *
 * Scratch: a fixed 64 KB array in device memory that the library declares
 * statically (1024 per-CTA partial slots and one result record); every GPU
 * that loads the library holds it until the process exits. Domains of more
 * than 16,777,216 nodes (nx * ny) are rejected with LBM_EINVAL. The first
 * call in a device's context sets up: it looks up the array's device
 * address (once per context, normally once per device, with that device
 * current); make that first call before any stream capture begins on the
 * device. All calls share the array and each call overwrites what it
 * reads, so nothing needs clearing; calls that overlap on the GPU (other
 * streams, other host threads) race on it and must be serialised by the
 * caller. No cudaMalloc, cudaFree or allocating library routine is called.
 *
 * Returns LBM_EINVAL (bad parameters, null pointers, domain too large),
 * LBM_ECUDA, LBM_ENAN (with *out filled) or LBM_OK;
 * lbm_noalloc_last_error() gives the message of the calling thread's last
 * failure. */
lbm_status lbm_observables_noalloc(const lbm_params *params, const double *d_pops,
                                   const uint8_t *d_solid, int64_t step, void *cuda_stream,
                                   lbm_obs *out);

/* Message for the calling thread's last lbm_observables_noalloc failure. */
const char *lbm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_EWOD_H */
