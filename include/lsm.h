/*
 * lsm.h -- C ABI of liblsm.so: the analytic linac source model of Tian et al.,
 * "An analytic linear accelerator source model for Monte Carlo dose
 * calculations. II. Model utilization in a GPU-based Monte Carlo package and
 * automatic source commissioning" (arXiv:1503.01725), on one B300 GPU.
 *
 * Conventions
 *   - Every call returns lsm_status. LSM_ERR_ARG: an argument failed
 *     validation before any GPU work was queued (nothing was changed).
 *     LSM_ERR_CUDA: a CUDA runtime call failed; the message is available from
 *     lsm_last_error(). LSM_ERR_OVERFLOW / LSM_ERR_TIMEOUT: the GPU work ran to
 *     completion but a bounded resource (a particle queue, a step cap, a
 *     bounded wait) was exhausted; results are complete except for the counted
 *     events, which were handled as documented at the call. LSM_ERR_IO: a
 *     file could not be opened, read or written (the message names it).
 *   - Handles (lsm_psl, lsm_phantom, lsm_tally) are opaque, created and owned
 *     by the library, and must be released with the matching *_destroy. A
 *     handle lives on the device that was current when it was created.
 *   - Input arrays are owned by the caller and are only read during the call
 *     (host pointers are copied before the call returns).
 *   - lsm_mem says whether a pointer is host or device memory; device pointers
 *     may come from any allocator (e.g. PyTorch tensors).
 *   - lsm_stream is a cudaStream_t (NULL = legacy default stream). Calls that
 *     take a stream return once the work is queued, unless stated otherwise;
 *     results written to device memory are stream-ordered. Calls that write
 *     host memory synchronise the stream before returning.
 *   - Positions are in cm along a beam axis from the target (z = 0) towards
 *     the phantom; energies in MeV; angles in radians.
 */
#ifndef LSM_H
#define LSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LSM_OK = 0,
    LSM_ERR_ARG = 1,
    LSM_ERR_CUDA = 2,
    LSM_ERR_OVERFLOW = 3,
    LSM_ERR_TIMEOUT = 4,
    LSM_ERR_NOT_CONVERGED = 5,
    LSM_ERR_IO = 6
} lsm_status;

typedef enum { LSM_MEM_HOST = 0, LSM_MEM_DEVICE = 1 } lsm_mem;

typedef void *lsm_stream;              /* cudaStream_t */
typedef struct lsm_model lsm_model;
typedef struct lsm_psl lsm_psl;
typedef struct lsm_phantom lsm_phantom;
typedef struct lsm_tally lsm_tally;

/* Sub-source types (Sec. 2.1.3): 0 primary photon, 1 scatter photon, 2 electron. */
#define LSM_N_STYPE 3
/* Gaussian components of the scatter-photon direction model (Eq. 6, K = 3). */
#define LSM_K_MIX 3

/*
 * PSR model (Sec. 2.1.1; the model and its parameters come from part I of the
 * paper). A PSR is (sub-source s, energy bin e, ring R). Ring R covers radii
 * [R dr, (R+1) dr) on the phase-space plane at z = z_phsp; energy bin e of
 * sub-source s covers [e_lo[s] + e de[s], e_lo[s] + (e+1) de[s]).
 * All arrays are host memory, C order.
 *   w       [3][n_e][n_r]   PSR weights (>= 0, finite)
 *   sigma_s                 primary focal-spot Gaussian width (Eq. 4), cm
 *   mix_c   [n_e][n_r][3]   scatter mixture weights c_{i,k} (Eq. 6), >= 0, sum > 0
 *   mix_mu  [n_e][n_r][3]   mixture means mu_{i,k} of alpha
 *   mix_sa, mix_sb          mixture widths sigma_alpha, sigma_beta
 *   e_sa, e_sb [n_e][n_r]   electron direction widths (Eq. 7)
 * Validation: 1 <= n_e <= 64, 1 <= n_r <= 32, dr > 0, z_phsp > 0, de > 0,
 * sigma_s >= 0, |mu| + 5.8 sigma_alpha < pi/2 and 5.8 sigma_beta < pi/2 for
 * every component (the largest Gaussian deviate the sampler can draw is 5.77).
 */
typedef struct {
    int32_t n_e, n_r;
    double dr, z_phsp, sigma_s;
    double e_lo[3], de[3];
    const double *w, *mix_c, *mix_mu, *mix_sa, *mix_sb, *e_sa, *e_sb;
} lsm_psr_model;

/*
 * lsm_model_create -- the PSR model of Sec. 2.1.1 as a library handle: checks
 * `psr` against the ranges above and keeps its own host copy of every array
 * (the caller's arrays may be freed or changed afterwards without affecting
 * the handle). Plans are built from the handle (lsm_build_psl); a plan does
 * not refer to its model once the build call has returned, so the model may
 * be destroyed while plans built from it are still in use. A commissioned
 * model (Sec. 2.2.4: the PSR weights W_R scaled by x) is a new handle.
 * Errors: LSM_ERR_ARG (NULL pointers or a value out of range; *out = NULL).
 */
lsm_status lsm_model_create(const lsm_psr_model *psr, lsm_model **out);
void lsm_model_destroy(lsm_model *model);
/*
 * lsm_model_commission -- Sec. 2.2.4: the commissioned model, a new handle
 * whose PSR weights are W_R x_R. x (host, n_x values >= 0): either one factor
 * per PSR (n_x = 3 n_e n_r, in PSR order (s n_e + e) n_r + R), or the solution
 * of Eq. 8 over lsm_basis_matrix_units' columns (n_x = 2 n_e n_r + n_e: the
 * photon PSRs, then one factor per electron energy bin, applied to all rings
 * of that bin). Every other parameter is the model's.
 * Errors: LSM_ERR_ARG (NULL pointers, another n_x, a negative or non-finite x).
 */
lsm_status lsm_model_commission(const lsm_model *model, const double *x, int32_t n_x, lsm_model **out);
/* lsm_model_weights -- copy the model's PSR weights W_R to host memory w
 * (double [3][n_e][n_r]), e.g. the commissioned weights. */
lsm_status lsm_model_weights(const lsm_model *model, double *w);

/*
 * Beams of a plan (step S1). Jaw edges x1 < x2, y1 < y2 are given at the
 * isocentre plane z = sad; the Y and X jaws have their upper surfaces at
 * z_jaw_y and z_jaw_x (z_phsp < z_jaw < sad). jaws: host [n_beams][4]
 * (x1, x2, y1, y2). 1 <= n_beams <= 16.
 * gantry: NULL, or host [n_beams] gantry angles (radians, |angle| <= 4 pi).
 * With NULL, the beam frame is the phantom frame (every beam along +z, the
 * phantom's top face z0 facing the source). Otherwise beam b is turned about
 * the axis through iso (phantom coordinates, cm) parallel to y: a point q of
 * the beam frame (target at the origin, axis +z, isocentre at (0, 0, sad))
 * sits at iso + R_b (q - (0, 0, sad)), R_b (a, b, c) = (a cos g + c sin g, b,
 * -a sin g + c cos g), so the beam axis runs along (sin g, 0, cos g). A
 * particle then enters the phantom wherever its ray first meets the voxel box
 * (and is counted as missing it otherwise); the box must not reach the
 * phase-space plane of any beam.
 */
typedef struct {
    double sad, z_jaw_y, z_jaw_x;
    int32_t n_beams;
    const double *jaws;
    const double *gantry;
    double iso[3];
} lsm_beams;

/*
 * lsm_build_psl -- Sec. 2.1.1-2.1.3 (Eq. 1-3, Fig. 3), on the GPU in FP64.
 * Converts the PSR model to its PSL representation on a 2 n_r x 2 n_r grid of
 * pitch dr centred on the axis (steps 1-4 of Sec. 2.1.1, normalised per
 * (sub-source, energy bin) block), determines the sampling areas of every
 * beam (primary: jaw opening scaled to the plane; scatter and electrons: upper
 * jaw surfaces back-projected from the field centre on the isocentre plane,
 * X and Y separately, intersected), keeps the PSLs that overlap an area with
 * positive area, and integerises Eq. 3 (largest remainders, ties to the lower
 * loop index) so that the counts sum exactly to the requested histories.
 * Plan loop order: beam, sub-source, energy bin, PSL row (y), PSL column (x).
 *
 *   per_psr_hist == NULL: one plan of n_hist histories over the whole source.
 *   per_psr_hist != NULL (host, [3 n_e n_r]): batched basis runs for
 *     commissioning (Sec. 2.2.2) -- for every PSR k and beam b a run of
 *     per_psr_hist[k] histories drawn from PSR k's share of the PSL weights
 *     (the k-th term of the linear PSR -> PSL map); n_hist is ignored. Every
 *     particle of such a run carries PSR index k.
 * The plan is periodic: history g uses plan position g mod (plan size), so a
 * run of B passes is B statistically independent batches.
 * model: a handle from lsm_model_create (read only during the call).
 * Errors: LSM_ERR_ARG on a NULL model, invalid beams, n_hist < 1
 * (whole-source), an empty sampling area, or a plan larger than 2^31 entries.
 */
lsm_status lsm_build_psl(const lsm_model *model, const lsm_beams *beams, int64_t n_hist,
                         const int64_t *per_psr_hist, lsm_psl **out, lsm_stream stream);
/*
 * lsm_build_psl_async -- lsm_build_psl without waiting for the build: returns
 * once its kernels are queued on `stream`. The plan's results (entries, the
 * Eq. 3 denominator) are read on the first call that needs them on the host
 * (lsm_psl_info, lsm_psl_copy, lsm_sample, a synchronising lsm_run), which is
 * also where an empty sampling area is reported (LSM_ERR_ARG). Argument
 * errors are returned at once. Per-PSR plans are built synchronously.
 */
lsm_status lsm_build_psl_async(const lsm_model *model, const lsm_beams *beams, int64_t n_hist,
                               const int64_t *per_psr_hist, lsm_psl **out, lsm_stream stream);
/* Releases the plan; its device memory returns to the pool in the order of
 * the legacy default stream. Work using the plan on non-blocking streams must
 * have completed. */
void lsm_psl_destroy(lsm_psl *psl);

/* info: [n_xy, n_entries, plan size (histories per pass), per_psr flag];
 * denom: the Eq. 3 denominator (whole-source plans). Synchronises. */
lsm_status lsm_psl_info(const lsm_psl *psl, int64_t info[4], double *denom);
/*
 * Copy a plan table to host memory (synchronises). which:
 *   0 PSL weights   double [3][n_e][n_xy][n_xy]
 *   1 inclusion     uint8  [n_beams][2][n_xy][n_xy] (class 0 primary, 1 scatter+electron)
 *   2 areas         double [n_beams][2][4] (xa, xb, ya, yb on the phase-space plane)
 *   3 counts        int64  whole-source [n_beams][3][n_e][n_xy][n_xy];
 *                          per-PSR [3 n_e n_r][n_beams][n_xy][n_xy]
 *   4 entry starts  int64  [n_entries + 1] (exclusive prefix of the counts)
 *   5 entries       int32  [n_entries][6] (beam, stype, ebin, ix, iy, forced PSR or -1)
 *   6 entry scale   double [n_entries] per-PSR plans: (in-area weight of the
 *                          PSR for that beam) / per_psr_hist[k]; 0 otherwise
 */
lsm_status lsm_psl_copy(const lsm_psl *psl, int which, void *host_dst);

/*
 * Particles in structure-of-arrays form, all DEVICE pointers with capacity n.
 * Position (x, y, z) and direction (u, v, w) are where the particle crosses
 * the phantom surface plane (z = phantom z0); E kinetic energy.
 * hist: history id g. psr: PSR index (s n_e + e) n_r + R carried for the
 * basis tally; beam: beam index; type: 0 photon, 1 electron; status:
 * 0 accepted, 1 rejected by the jaws, 2 missed the phantom top face.
 * info (optional, may be NULL): int32 [n][4] = (stype | ebin << 8,
 * ring used for the direction model, mixture component or -1, plan entry).
 */
typedef struct {
    float *x, *y, *z, *u, *v, *w, *E;
    uint64_t *hist;
    uint16_t *psr;
    uint8_t *beam, *type, *status;
    int32_t *info;
} lsm_particles;

/*
 * lsm_sample -- steps S3-S5 on the GPU (Eq. 4-7): particles for histories
 * [hist_begin, hist_begin + n) of the plan, drawn from Philox4x32-10 with key
 * `seed` and counter (history, stream 0, draw index). Position uniform in the
 * PSL, energy uniform in the bin; primary direction from a Gaussian focal spot
 * (Eq. 4-5); scatter direction from the K=3 mixture of the ring that holds the
 * sampled radius (Eq. 6); electron direction from Eq. 7; rotation by the polar
 * angle of (x, y); straight flight to the jaw planes (rejection) and to the
 * phantom surface at z = z_surface. Every history produces one record.
 * Errors: LSM_ERR_ARG if n < 0 or a required pointer is NULL.
 */
lsm_status lsm_sample(const lsm_psl *psl, uint64_t seed, uint64_t hist_begin, int64_t n,
                      double z_surface, const lsm_particles *out, lsm_stream stream);

/*
 * Voxel phantom: nx * ny * nz voxels of dx * dy * dz cm, first voxel corner
 * at (x0, y0, z0); z0 is the phantom surface. rho: float32 density (g/cm^3,
 * 1e-4 <= rho <= 25), mat: uint8 material class (0 water-like, 1 bone), both
 * [nz][ny][nx] in `mem`. Creation also generates the interaction tables of the
 * stated transport model (Klein-Nishina Compton, photoelectric and pair cross
 * sections, Bethe collision stopping power; 1024 log-spaced energies from
 * 1 keV to 7 MeV) and the Woodcock majorant of this phantom.
 */
typedef struct {
    int32_t nx, ny, nz;
    double dx, dy, dz, x0, y0, z0;
    const float *rho;
    const uint8_t *mat;
    lsm_mem mem;
} lsm_phantom_desc;

lsm_status lsm_phantom_create(const lsm_phantom_desc *desc, lsm_phantom **out, lsm_stream stream);
/* The same phantom without waiting on the host for the input check: the
 * copies and set-up kernels are only queued on `stream`, so host code goes on
 * at once (the end-to-end path of a dose calculation). The check's verdict
 * stays on the device: runs on an invalid phantom transport nothing, and
 * lsm_dose and lsm_basis_matrix(_units) into host memory and
 * lsm_phantom_check report LSM_ERR_ARG for it.
 * rho/mat in pageable host memory are read before the call returns; in pinned
 * host or device memory they must stay unchanged until `stream` has passed the
 * call. Errors at the call: as lsm_phantom_create except the value check. */
lsm_status lsm_phantom_create_async(const lsm_phantom_desc *desc, lsm_phantom **out, lsm_stream stream);
/* The verdict of the phantom's input check (densities in [1e-4, 25], materials
 * in {0, 1}): LSM_OK or LSM_ERR_ARG. Synchronises `stream`, which must be
 * ordered after the creation. */
lsm_status lsm_phantom_check(const lsm_phantom *ph, lsm_stream stream);
/* Releases the phantom; its device memory returns to the device's memory
 * pool in the order of the legacy default stream (no device-wide wait). Work
 * using it on non-blocking streams must have completed. */
void lsm_phantom_destroy(lsm_phantom *ph);
/* Copy the interaction tables to host (synchronises): out float
 * [2 materials][1024][4] = (mu_compton, mu_photo, mu_pair in cm^2/g, S_col in
 * MeV cm^2/g), then [1024] majorant (1/cm), then [32][129] inverse
 * Klein-Nishina CDF v = (eta - 1) / (2k) at ln E = ln 0.05 + i (ln 7 - ln 0.05)/31
 * and u = j/128 (eta = E/E', k = E/mc^2); grid[2] = (ln E_min, d ln E) of the
 * 1024-point grid. */
lsm_status lsm_phantom_tables(const lsm_phantom *ph, float *out, double grid[2]);

/*
 * Tally. mode 0: energy per voxel. mode 1: basis tally of Sec. 2.2.2 -- a 2D
 * array [n_beams * n_rows][n_psr]; a deposit in voxel v goes to row
 * idx3d[v] - 1 of the particle's beam block, column = the particle's PSR,
 * and is dropped when idx3d[v] == 0. idx3d: uint16 [nz][ny][nx] in idx3d_mem.
 * Deposits accumulate in FP32 partials that are flushed into FP64 after every
 * sample/transport iteration; lsm_tally_end_batch folds the open FP64 batch
 * into the running sums S1 (sum of batch totals) and S2 (sum of squares).
 */
typedef struct {
    int32_t mode;
    const uint16_t *idx3d;
    lsm_mem idx3d_mem;
    int32_t n_rows, n_psr, n_beams;
} lsm_tally_desc;

lsm_status lsm_tally_create(const lsm_phantom *ph, const lsm_tally_desc *desc, lsm_tally **out,
                            lsm_stream stream);
/* Releases the tally (and its transport workspace) to the device's memory
 * pool in the order of the legacy default stream; its own graph stream is
 * drained first. Work using it on other non-blocking streams must have
 * completed. */
void lsm_tally_destroy(lsm_tally *t);
/* Zero every sum, counter and the energy ledger. */
lsm_status lsm_tally_reset(lsm_tally *t, lsm_stream stream);
/* Flush pending FP32 partials and fold the open batch into S1/S2. */
lsm_status lsm_tally_end_batch(lsm_tally *t, lsm_stream stream);
/* s1, s2: double [cells] in `mem` (either may be NULL); *n_batches = folded
 * batches. Synchronises when mem is HOST. */
lsm_status lsm_tally_read(lsm_tally *t, double *s1, double *s2, lsm_mem mem, int32_t *n_batches,
                          lsm_stream stream);
/* lsm_tally_load -- restore a checkpoint: S1, S2 (double [cells] in `mem`),
 * the folded batch count and, optionally, the ledger and statistics as
 * lsm_tally_ledger returns them (NULL: zero). The partial slices and the open
 * batch are cleared. Stream-ordered (host arrays are read before it returns).
 * Errors: LSM_ERR_ARG for a NULL tally or S1/S2, or n_batches < 0. */
lsm_status lsm_tally_load(lsm_tally *t, const double *s1, const double *s2, int32_t n_batches,
                          const double ledger[4], const int64_t stats[11], lsm_mem mem, lsm_stream stream);
/*
 * lsm_tally_history_ledger -- a test mode: attach (ledger != NULL) or detach
 * (NULL) a per-history energy ledger to a dose (mode 0) tally. While attached,
 * lsm_run on this tally adds, for each history g with 0 <= g - first_history <
 * n_hist (h = g - first_history), the energy of its source particle to
 * ledger[2h] and every deposited, escaped or jaw-rejected energy of the
 * particles it leads to (all generations) to ledger[2h + 1], so that
 * ledger[2h + 1] = ledger[2h] checks energy conservation history by history.
 * ledger: device memory, FP64 [n_hist][2], owned and zeroed by the caller,
 * 8-byte aligned; it must stay valid while attached. The run uses separate
 * kernel instances (graph replay off); other calls (lsm_transport,
 * lsm_pslfile_run) ignore the ledger. Errors: LSM_ERR_ARG for a NULL tally, a
 * basis tally, n_hist < 1, first_history < 0 or a misaligned buffer.
 */
lsm_status lsm_tally_history_ledger(lsm_tally *t, double *ledger, int64_t n_hist, int64_t first_history);

/* ledger (MeV): source, rejected, escaped (incl. missed), deposited.
 * stats: histories, accepted photons, accepted electrons, rejected, missed,
 * Woodcock flights, real photon interactions, electron steps, step-cap hits,
 * queue overflows, secondary electrons (those photon interactions put on the
 * electron queue: Compton, photoelectric and pair electrons at or above the
 * electron cutoff, electron_mode 1). Synchronises. */
lsm_status lsm_tally_ledger(lsm_tally *t, double ledger[4], int64_t stats[11], lsm_stream stream);

/*
 * Transport options (the stated simplification of the paper's engine; the
 * paper fixes only the cutoffs, electrons 200 keV and photons 50 keV,
 * Sec. 2.3). electron_mode 0 deposits electron energy where the electron is
 * created; 1 transports electrons by CSDA steps: step = min(s_geo, f_e E/S),
 * energy loss by the midpoint rule, deposit at the step midpoint, Highland
 * Gaussian deflection. s_geo <= 0 means half the smallest voxel side.
 * majorant_factor >= 1 inflates the Woodcock majorant (results unchanged in
 * expectation). chunk: histories per sample/transport iteration (the paper's
 * M); 0 = 2^23. Plans smaller than chunk run several whole batches per
 * iteration. max_steps: per-particle step cap (>= 1), after which the
 * remaining energy is deposited locally and counted. ctas_per_sm: CTAs per SM
 * of the persistent transport kernels (0 = as many as fit). use_graph != 0:
 * lsm_run captures its launch sequence into a CUDA graph on first use and
 * replays it for later runs with the same plan, phantom, tally and options
 * (the seed may change). A graph captured while the event timers are on
 * holds their events, which are read after every replay; turning the timers
 * on or off re-captures it. no_sync != 0: lsm_run returns once the run is
 * queued, without waiting for it: queue overflows stay counted in the tally
 * statistics (stats[9]) instead of being returned, and an empty plan from
 * lsm_build_psl_async runs no history and is reported by lsm_psl_info.
 * first_batch: index of the run's first batch; pass b of the run uses the
 * histories of batch first_batch + b, so a run of B batches equals runs of
 * B1 and B - B1 batches (the second with first_batch = B1) with the tally
 * saved and restored in between (lsm_tally_read / lsm_tally_ledger, then
 * lsm_tally_load): the checkpoint of a dose calculation is its tally sums,
 * its statistics and the next batch index.
 * e_queue_cap: capacity of the secondary-electron queue in particles (0 =
 * 4 chunk + 2^18, which no run of the stated physics fills); a smaller queue
 * bounds the workspace's memory, and electrons created once it is full are
 * deposited where they are created, counted in stats[9] and reported as
 * LSM_ERR_OVERFLOW (the energy balance still holds).
 * streams: 1 (0 = 1) or 2. With 2, when an iteration holds several whole
 * batches, its batches are split into two halves with their own particle
 * queues, sampled and transported on two CUDA streams (the second one owned
 * by the tally), so that one half's passes run on the SMs the other half's
 * passes leave idle while their queues drain; the halves tally into different
 * batch slots. Results are those of streams = 1 (the same histories).
 */
typedef struct {
    int32_t electron_mode;
    int32_t n_batches;
    double majorant_factor, f_e, s_geo;
    int32_t max_steps;
    int32_t chunk;
    int32_t ctas_per_sm;
    int32_t use_graph;
    int32_t no_sync;
    int64_t first_batch;
    int32_t e_queue_cap;
    int32_t streams;
} lsm_run_opts;

/*
 * lsm_transport -- transport the accepted particles (status 0) of `in`
 * (device SoA of n records, as written by lsm_sample with the same seed) and
 * every secondary they create, depositing into `tally`'s open batch. Each
 * particle draws from its own Philox stream (key = seed, counter = (history
 * lo, history hi, stream id, draw index)): primaries use stream id 1; a
 * particle created at an interaction takes as stream id MurmurHash3's fmix32
 * finaliser of its parent's stream id combined with the parent's draw counter
 * and the child's slot (pair event: electron 0, positron 1, annihilation
 * photons 2 and 3), ids below 2 shifted up by 2 (0 and 1 are reserved).
 * A photon draws one block per Woodcock flight (word 0 flight length, word 1
 * the collision: u mu_max above mu_total is virtual, below it selects Compton,
 * photoelectric or pair; words 2-3 a Compton event's eta and azimuth) and one
 * more per pair event; an electron draws half a block per deflection.
 * Errors: LSM_ERR_ARG on mismatched handles; LSM_ERR_OVERFLOW when the
 * secondary-electron queue filled up (the excess electrons were deposited at
 * their creation point and counted in stats[9]).
 */
lsm_status lsm_transport(const lsm_phantom *ph, const lsm_particles *in, int64_t n, uint64_t seed,
                         lsm_tally *tally, const lsm_run_opts *opts, lsm_stream stream);

/*
 * lsm_run -- the whole dose calculation of Sec. 2.1.3: n_batches passes over
 * the plan, each iterating [sample M histories -> transport photons (with
 * the annihilation photons of their pair events) -> transport electrons ->
 * flush] until the
 * plan is exhausted, then folding the batch (lsm_tally_end_batch). Histories
 * of pass b are g = b * plan size + h.
 * Errors: as lsm_transport.
 */
lsm_status lsm_run(const lsm_psl *psl, const lsm_phantom *ph, lsm_tally *tally, uint64_t seed,
                   const lsm_run_opts *opts, lsm_stream stream);

/*
 * Dose per source particle (MeV/g) and its batch standard deviation from a
 * mode-0 tally: dose = S1 / B * scale / (rho V), sigma from the batch spread,
 * where scale = (Eq. 3 denominator) / (plan size) converts per-history to
 * per-source-particle. dose, sigma: double [nvox] in mem (sigma may be NULL).
 */
lsm_status lsm_dose(const lsm_tally *t, const lsm_phantom *ph, double scale, double *dose,
                    double *sigma, lsm_mem mem, lsm_stream stream);

/*
 * Basis matrix A of Sec. 2.2.2 from a mode-1 tally over a per-PSR plan:
 * A[(b, row), k] = S1 / B * (entry scale of PSR k, beam b) / (rho V of the row's
 * voxel), i.e. the dose per source particle of the full model contributed by
 * PSR k. A: double [n_beams * n_rows][n_psr] in mem.
 */
lsm_status lsm_basis_matrix(const lsm_tally *t, const lsm_psl *psl, const lsm_phantom *ph,
                            const uint16_t *idx3d, lsm_mem idx3d_mem, double *A, lsm_mem mem,
                            lsm_stream stream);

/*
 * lsm_basis_matrix_units -- the basis matrix over the unknowns of Eq. 8
 * (Sec. 2.2.3): one column per photon PSR (primary and scatter, as
 * lsm_basis_matrix), then one column per electron energy bin e, the sum of the
 * n_r electron PSR columns of that bin (the "effective electron unit": the
 * electron PSRs are too weak to be commissioned one by one). A: double
 * [n_beams n_rows][2 n_e n_r + n_e] in `mem` (rows as lsm_basis_matrix). The
 * tally's PSR count must be 3 n_e n_r of the plan's model.
 * Errors: as lsm_basis_matrix.
 */
lsm_status lsm_basis_matrix_units(const lsm_tally *t, const lsm_psl *psl, const lsm_phantom *ph, double *A,
                                  lsm_mem mem, lsm_stream stream);

/*
 * lsm_commission -- Eq. 8: x = argmin_{x >= 0} ||A x - b||^2 in FP64 on the
 * GPU. A: double [m][n] row-major, b: double [m], both in `mem`; x: host
 * double [n] (also the starting point of the projected-gradient methods when
 * opts->use_x0 != 0). method 0: active set (Lawson & Hanson) with the
 * passive-set least squares solved by Cholesky of the normal equations;
 * method 1: gradient projection with Armijo's rule (Sec. 2.2.4), stopped when
 * the relative change of F falls below delta; method 2: gradient projection
 * with Barzilai-Borwein step lengths (alpha = d'd / (2 d'Gd) from the last
 * move d, G = A'A) and the exact minimiser of F along each projected step,
 * same stop (armijo_sigma and armijo_beta unused). Synchronises.
 * Errors: LSM_ERR_ARG for m < 1, 1 > n > 1024, a method other than 0-2 or NULL pointers;
 * LSM_ERR_NOT_CONVERGED when max_iter was reached (x holds the last iterate).
 */
typedef struct {
    int32_t method;
    int32_t max_iter;
    double delta;
    double armijo_sigma, armijo_beta;
    int32_t use_x0;
} lsm_nnls_opts;

typedef struct {
    int32_t iterations;
    int32_t converged;
    double objective;
    double kkt;            /* max violation of x >= 0, grad >= 0, x * grad = 0 */
} lsm_nnls_report;

lsm_status lsm_commission(const double *A, int32_t m, int32_t n, const double *b, lsm_mem mem,
                          const lsm_nnls_opts *opts, double *x, lsm_nnls_report *report,
                          lsm_stream stream);

/*
 * lsm_commission_static -- the same solve as lsm_commission, for callers that
 * must not allocate GPU memory while they run (for example a planning service
 * that reserves all of its device memory at start-up, or a host application
 * that owns the GPU memory and loads this library as a plugin; cudaMalloc and
 * cudaFree would also synchronise the whole device). The paper has no
 * counterpart: this is a deployment variant. Its scratch is one fixed device
 * array of about 1 MiB that every GPU loading the library holds until process
 * exit; it limits the problem to n <= 256 unknowns (larger n: LSM_ERR_ARG).
 * A (double [m][n], row-major), b (double [m]) and x (double [n]) are all
 * DEVICE pointers; x receives the solution (and is the projected-gradient
 * start when opts->use_x0 != 0, else it is set to 1). report is host memory
 * and may be NULL; A, b or x that is not device or managed memory returns
 * LSM_ERR_ARG (checked with cudaPointerGetAttributes). The first call on a
 * device looks up the array's device address (once per device, with that
 * device current) and keeps it for the life of the process: it assumes the
 * device's primary context is never reset (after cudaDeviceReset the array may
 * sit elsewhere; do not call this entry point again in that process). Make the
 * first call before any stream capture. Every call shares the one array, which keeps the
 * previous call's contents: calls that overlap on the GPU (other streams or
 * host threads) race and must be serialised by the caller. Calls no
 * cudaMalloc or cudaFree. Synchronises the stream before returning.
 */
lsm_status lsm_commission_static(const double *A, int32_t m, int32_t n, const double *b,
                                 const lsm_nnls_opts *opts, double *x, lsm_nnls_report *report,
                                 lsm_stream stream);

/*
 * Timers (the breakdown of Sec. 3.1 / Table 1: source initialisation, particle
 * generation, transport simulation). When enabled, the library records CUDA
 * events on the launching stream around each kernel group and accumulates
 * their elapsed device time:
 *   0 PSL build (T_src_init)       1 sampling (T_par_gen_tr)
 *   2 photon transport             3 (unused: annihilation photons are
 *                                    transported within timer 2)
 *   4 electron transport           5 tally flush and fold
 *   6 NNLS solve                   7 phantom set-up and tables
 *   8 denoiser 3x3x3 convolutions  9 denoiser pooling, upsampling, input
 *                                    packing and output head
 * lsm_timing_read synchronises the device, returns milliseconds and launch
 * counts per timer, and clears them when reset != 0. Disabled by default.
 */
/*
 * lsm_set_wait_limits -- bounds of the library's device-side waits, for
 * tests of the give-up paths and for hosts that want failures reported
 * sooner. Values < 0 keep the current setting.
 *   stage_polls: polls of the mbarrier on which a transport CTA waits for its
 *     interaction tables to arrive in shared memory (default 2^22). When they
 *     run out, the CTA reads the tables from global memory instead (the same
 *     values: results are unchanged), sets the run's fallback flag (see
 *     lsm_run_fallbacks) and, before it exits, waits for its copy to land.
 *     0 gives up at once.
 *   conv_wait_ns: the 3x3x3 convolution kernels' wait on each pipeline
 *     barrier (default 2e9 ns). When it runs out, the CTA stops, waits for its
 *     own copies and tensor-core operations in flight (a fixed 100 ms bound),
 *     releases its tensor memory and sets an error word that the next
 *     synchronising denoiser call returns as LSM_ERR_TIMEOUT.
 * Applies to launches queued after the call (captured graphs keep the
 * values they were captured with).
 */
lsm_status lsm_set_wait_limits(int64_t stage_polls, int64_t conv_wait_ns);
/* Number of transport CTAs that fell back to global-memory tables since the
 * last reset (synchronises the device); reset != 0 clears it. */
lsm_status lsm_run_fallbacks(int64_t *count, int reset);

#define LSM_N_TIMERS 10
lsm_status lsm_timing_enable(int on);
lsm_status lsm_timing_read(double ms[LSM_N_TIMERS], int64_t launches[LSM_N_TIMERS], int reset);

/* ------------------------------------------------------------------------
 * Dose denoiser. The paper stops at Monte Carlo dose (Sec. 2.3) and states
 * run times for a target statistical uncertainty (Sec. 3); the denoiser maps a
 * low-history dose and the phantom density to an estimate of the high-history
 * dose. Network: a four-level 3D U-Net with widths 16/32/64/128, 3x3x3
 * zero-padded convolutions with bias and ReLU, 2x2x2 max pooling, nearest 2x
 * upsampling, skip concatenation (skip channels first) and a 1x1x1 head added
 * to the input dose (residual). BF16 activations and weights, FP32
 * accumulation in tensor memory (tcgen05), FP32 output.
 *
 * Activation volumes (lsm_vol) are device BF16 arrays laid out
 * [n][(d+2)(h+2)(w+2)][c_total]: every volume carries a one-voxel zero halo,
 * voxel (z, y, x) of the interior at padded index ((z+1)(h+2) + y+1)(w+2) + x+1.
 * The halo must hold zeros; the kernels keep it so. A call uses channels
 * [c_offset, c_offset + c) of each voxel. c_total and c_offset are multiples of
 * 8; the base pointer is 16-byte aligned.
 * ------------------------------------------------------------------------ */
typedef struct {
    void *data;
    int32_t n, d, h, w;         /* volumes, interior size */
    int32_t c_total, c_offset, c;
} lsm_vol;

/* Bytes of a padded activation volume (n * (d+2)(h+2)(w+2) * c_total * 2). */
int64_t lsm_vol_bytes(int32_t n, int32_t d, int32_t h, int32_t w, int32_t c_total);

typedef struct lsm_conv3d lsm_conv3d;
/*
 * lsm_conv3d_create -- one 3x3x3 convolution layer. weight: host FP32
 * [c_out][3][3][3][c_in] indexed (dz, dy, dx) (cross-correlation: output
 * voxel (z,y,x) takes input (z+dz-1, y+dy-1, x+dx-1)); bias: host FP32
 * [c_out] (NULL = zero). Both are rounded to BF16 and packed into the
 * tensor-core operand layout on the device; the caller's arrays are not kept.
 * c_in and c_out in {16, 32, 64, 128}, relu 0/1.
 * Errors: LSM_ERR_ARG for other sizes or NULL weight.
 */
lsm_status lsm_conv3d_create(int32_t c_in, int32_t c_out, int32_t relu, const float *weight, const float *bias,
                             lsm_conv3d **out, lsm_stream stream);
void lsm_conv3d_destroy(lsm_conv3d *conv);
/*
 * lsm_conv3d_forward -- out[:, c_offset : c_offset + c_out] = act(conv(in) +
 * bias) over every interior voxel, written as BF16. Interior rows are written
 * whole (their two x-halo voxels as zero); the other halo voxels are read as
 * the zero padding and left unchanged, so both volumes must hold a zero halo.
 * in->c must equal c_in and out->c c_out; n, d, h, w must match.
 * Stream-ordered. ctas_per_sm: persistent CTAs per SM (0 = as many as fit).
 */
lsm_status lsm_conv3d_forward(const lsm_conv3d *conv, const lsm_vol *in, const lsm_vol *out, int32_t ctas_per_sm,
                              lsm_stream stream);
/* 2x2x2 max pooling (out = in / 2 in every dimension; in->c == out->c). */
lsm_status lsm_pool3d(const lsm_vol *in, const lsm_vol *out, lsm_stream stream);
/* Nearest 2x upsampling (out = 2 in in every dimension; in->c == out->c). */
lsm_status lsm_upsample3d(const lsm_vol *in, const lsm_vol *out, lsm_stream stream);

typedef struct lsm_unet lsm_unet;
/* Number of FP32 parameters of the network: per conv layer (14, in network
 * order) its weights [c_out][3][3][3][c_in] then its bias, then the head's 16
 * weights and its bias. */
int64_t lsm_unet_param_count(void);
/* lsm_unet_create -- the network from a host FP32 parameter vector of
 * lsm_unet_param_count() values (copied and packed; not kept). */
lsm_status lsm_unet_create(const float *params, int64_t n_params, lsm_unet **out, lsm_stream stream);
void lsm_unet_destroy(lsm_unet *net);
/*
 * lsm_unet_forward -- denoised dose of n volumes [n][d][h][w] (x fastest),
 * d, h, w multiples of 8. dose and rho: FP32 (dose in any unit, rho in
 * g/cm^3), out: FP32 in the unit of dose; all three host or device (mem).
 * The input is normalised by each volume's maximum dose, the network runs in
 * BF16 with FP32 accumulation, and out = dose + Dmax * head. Activation
 * buffers are allocated on the first call for a shape and reused.
 * Stream-ordered for device buffers; synchronises for host buffers.
 */
lsm_status lsm_unet_forward(lsm_unet *net, int32_t n, int32_t d, int32_t h, int32_t w, const float *dose,
                            const float *rho, float *out, lsm_mem mem, lsm_stream stream);
/* Copy the stored output of conv layer `layer` (0..13) of the last forward
 * call, interior voxels only, as BF16 [n][d_l][h_l][w_l][c_out] into dst
 * (host or device). */
lsm_status lsm_unet_activation(const lsm_unet *net, int32_t layer, void *dst, lsm_mem mem, lsm_stream stream);

/*
 * Training of the denoiser on pairs (low-history dose, density) -> high-history
 * dose: loss = mean over voxels of (out / Dmax - target / Dmax)^2 with Dmax
 * the input dose's maximum per volume. One call runs the forward pass, the
 * gradient of every parameter (BF16 activation gradients, FP32 parameter
 * gradients; data gradients on the tensor cores) and, when opts->lr > 0, one
 * Adam step (with bias correction and decoupled weight decay) on the FP32
 * master parameters, after which the BF16 operand images are repacked.
 * dose, rho, target: device FP32 [n][d][h][w]; d, h, w multiples of 8.
 * loss: host pointer (the call then synchronises and reports pipeline
 * timeouts) or NULL (stream-ordered). opts NULL: gradients only.
 */
typedef struct {
    double lr, beta1, beta2, eps, weight_decay;
} lsm_adam_opts;
lsm_status lsm_unet_train_step(lsm_unet *net, int32_t n, int32_t d, int32_t h, int32_t w, const float *dose,
                               const float *rho, const float *target, const lsm_adam_opts *opts, double *loss,
                               lsm_stream stream);
/* Current FP32 parameters (lsm_unet_param_count values, flat order of
 * lsm_unet_create) and the gradient of the last training step. */
lsm_status lsm_unet_params(const lsm_unet *net, float *dst, lsm_mem mem, lsm_stream stream);
lsm_status lsm_unet_grad(const lsm_unet *net, float *dst, lsm_mem mem, lsm_stream stream);
/*
 * lsm_unet_set_wgrad -- where lsm_unet_train_step computes the convolutions'
 * weight gradients: 1 (default) on the tensor cores (a tcgen05 GEMM over
 * voxels: M = (tap, input channel), N = output channels, BF16 operands from
 * channel-major copies of the layer input and output gradient, FP32
 * accumulation in tensor memory), 0 on the CUDA cores (FP32). Both read the
 * same BF16 activations and accumulate in FP32. Process-wide.
 * Errors: LSM_ERR_ARG for another value.
 */
lsm_status lsm_unet_set_wgrad(int tensor_cores);

/*
 * Judging a dose estimate against a reference (the denoiser's error against
 * plain high-history Monte Carlo). Arrays are FP32 [d][h][w] (x fastest),
 * host or device (mem); the results are returned on the host (synchronises).
 *
 * lsm_gamma -- global gamma index (Low, Harms, Mutic & Purdy, Med. Phys. 25,
 * 656, 1998): over reference voxels above threshold * max(ref), the fraction
 * with min over points r of |r - r_ref|^2/dta^2 + (eval(r) - ref)^2 /
 * (dose_crit * max(ref))^2 <= 1, eval interpolated trilinearly (edge values
 * continued outside), r on a grid of step step_mm within the DTA sphere.
 * voxel_mm: (z, y, x) voxel size. n_roi (optional): voxels evaluated.
 * pass_map (optional, same memory kind, d*h*w bytes): 0 outside the region,
 * 3 pass, 2 fail.
 */
lsm_status lsm_gamma(const float *eval, const float *ref, int32_t d, int32_t h, int32_t w, const double voxel_mm[3],
                     double dose_crit, double dta_mm, double threshold, double step_mm, lsm_mem mem,
                     double *pass_rate, int64_t *n_roi, unsigned char *pass_map, lsm_stream stream);
/*
 * lsm_dose_error -- RMS relative error of est against ref over voxels with
 * ref > level * max(ref); with sigma_ref (optional) the reference's own mean
 * relative variance is subtracted: sqrt(max(mean(((est-ref)/ref)^2) -
 * mean((sigma_ref/ref)^2), 0)).
 */
lsm_status lsm_dose_error(const float *est, const float *ref, const float *sigma_ref, int64_t n, double level,
                          lsm_mem mem, double *rms_rel, lsm_stream stream);

/*
 * lsm_curve_compare -- the dose comparison of the commissioning validation
 * (Sec. 3.2): a calculated curve against a measured one, both sampled at the
 * same n positions `pos` (ascending, cm; a depth-dose curve or a lateral
 * profile), over the points with lo <= pos < hi (lo <= |pos| < hi when
 * use_abs != 0):
 *   out[0] RMS (Eq. 10) = sqrt(mean((calc - meas)^2)) / dmax_m,
 *   out[1] Max (Eq. 11) = max |calc - meas| / dmax_m (fractions, not percent),
 *   out[2], out[3] mean and max distance to agreement (cm): at a measured
 *     point x, min |x - y| over y where the calculated curve, linear between
 *     its points and continued along its first and last segments beyond the
 *     end points, equals meas(x); points where it never does are left out,
 *   out[4] points compared, out[5] points left out of the DTA figures.
 * Arrays float32 in `mem`; synchronises. Errors: LSM_ERR_ARG for n < 2,
 * n > 2^20 or dmax_m <= 0.
 */
lsm_status lsm_curve_compare(const float *pos, const float *calc, const float *meas, int32_t n, double lo, double hi,
                             int32_t use_abs, double dmax_m, lsm_mem mem, double out[6], lsm_stream stream);

/*
 * lsm_l2_atomic_peak -- the ceiling for the tally updates of transport: the
 * rate of FP32 atomic adds whose result is unused, to pseudo-random cells of a
 * device array of n_cells floats (each thread walks a linear congruential
 * sequence and maps it to a cell), over a grid of 8 CTAs per SM. A device
 * buffer of n_cells floats is allocated and freed inside the call; two warm-up
 * launches, then `reps` launches of 256 x 256 atomics per thread timed with
 * CUDA events on `stream`. *atomics_per_s: atomic operations per second.
 * Synchronises. Errors: LSM_ERR_ARG for a NULL output, n_cells outside
 * [1, 2^31] or reps outside [1, 1000]; LSM_ERR_CUDA when allocation or a launch
 * fails.
 */
lsm_status lsm_l2_atomic_peak(int64_t n_cells, int32_t reps, double *atomics_per_s, lsm_stream stream);

/*
 * lsm_philox_blocks -- the random-number contract (Philox4x32-10, Salmon et
 * al., SC 2011) as the device evaluates it, for checking against other
 * implementations: out[4 i .. 4 i + 3] = the block at key (seed lo, seed hi)
 * and counter (g lo, g hi, stream_id, draw) for history g = first_history + i,
 * i < n. Stream id 0 is source sampling, 1 a primary's transport. out: n x 4
 * uint32 in `mem` (host: synchronises). Errors: LSM_ERR_ARG for a NULL output
 * or n outside [1, 2^28].
 */
lsm_status lsm_philox_blocks(uint64_t seed, uint64_t first_history, uint32_t stream_id, uint32_t draw, int64_t n,
                             uint32_t *out, lsm_mem mem, lsm_stream stream);

/*
 * PSL files -- the comparator source model of Table 1 (Sec. 3.1): particles
 * stored on disk grouped by phase-spacelet, read for a field, copied to the
 * GPU and translated there, instead of being sampled on the fly.
 *
 * File layout (little endian): a 4096-byte header
 *   char magic[8] = "LSMPSLF1"; uint32 version = 1; uint32 record_bytes = 32;
 *   int32 n_xy, n_e, n_r, 0; double dr, z_phsp, w_record, denom;
 *   int64 n_records, index_offset, data_offset; uint64 seed;
 * then at index_offset int64 start[3 n_xy n_xy + 1]: records of PSL cell
 * c = (stype * n_xy + iy) * n_xy + ix are [start[c], start[c+1]); then at
 * data_offset (a multiple of 4096) n_records records of 32 bytes:
 *   float x, y (cm, on the phase-space plane), u, v, w, E (MeV);
 *   uint32 psr | type << 16 (type 0 photon, 1 electron); uint32 stype | ebin << 8.
 * Every record stands for source weight w_record = denom / n_records.
 */
typedef struct {
    int64_t records;      /* records read (all passes) */
    int64_t bytes;        /* bytes read from the file */
    int64_t chunks;       /* chunks transported */
    double t_read_s;      /* time the reader thread spent in read calls */
    double t_copy_s;      /* host-to-device copy time (events on the copy stream) */
    double t_total_s;     /* wall time of the whole call */
    double dose_scale;    /* scale for lsm_dose: n_batches * w_record */
    int32_t cold;         /* the file's page cache was dropped before reading */
    int32_t pad;
} lsm_pslfile_stats;

/*
 * lsm_pslfile_write -- sample every history of `plan` (a whole-source,
 * single-beam plan, normally with the jaws wide open) at the phase-space
 * plane (lsm_sample with z_surface = z_phsp and key `seed`) and write them as
 * a PSL file at `path`, grouped by PSL cell. Synchronises. n_written
 * (optional) receives the record count. Errors: LSM_ERR_ARG for a per-PSR or
 * multi-beam plan or a plan above 2^28 histories; LSM_ERR_IO if the file
 * cannot be written.
 */
lsm_status lsm_pslfile_write(const lsm_psl *plan, uint64_t seed, const char *path, int64_t *n_written,
                             lsm_stream stream);

/*
 * lsm_pslfile_run -- dose from a PSL file for the field of `field` (a
 * whole-source single-beam plan on the file's PSL grid; only its inclusion
 * table and jaws are used). The records of the PSL cells that the field's
 * sampling areas include (primary cells for sub-source 0, scatter/electron
 * cells for 1 and 2) are read from disk by a reader thread into pinned
 * buffers, copied to the GPU on a copy stream, and for each chunk a kernel
 * applies the jaw test at the upper jaw surfaces, flies the particle to the
 * phantom surface and queues it for the same photon/electron transport as
 * lsm_run. Included record j of pass p is history p * N + j (N included
 * records per pass) and falls in batch slot j mod n_batches; every pass ends
 * by folding n_batches batches into the tally. Pass p > 0 reuses the same
 * records with new transport streams. opts->chunk: records per chunk (0 = 2^22).
 * cold != 0: drop the file's cached pages first (fdatasync + fadvise), so
 * that reads come from storage. stats (optional) as above.
 * Errors: LSM_ERR_ARG on a file/plan mismatch or bad counts; LSM_ERR_IO on
 * read errors; LSM_ERR_OVERFLOW as lsm_run.
 */
lsm_status lsm_pslfile_run(const char *path, const lsm_psl *field, const lsm_phantom *ph, lsm_tally *tally,
                           uint64_t seed, int32_t n_batches, int32_t n_passes, int32_t cold,
                           const lsm_run_opts *opts, lsm_pslfile_stats *stats, lsm_stream stream);

/* Library diagnostics. */
const char *lsm_last_error(void);
/* Kernels launched by this library in this process so far. */
int64_t lsm_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* LSM_H */
