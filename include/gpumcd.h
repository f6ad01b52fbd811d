/*
 * gpumcd.h - C ABI of the GB300 coupled photon-electron Monte Carlo dose engine.
 *
 * The engine follows GPUMCD (Hissoiny, Bouchard, Ozell, Despres): a voxelized
 * phantom of material ids and densities (§II.C.2), material cross-section and
 * stopping-power data (§II.C.2), a source of one particle type with a
 * monoenergetic energy or a spectrum and a beam geometry (§II.C.2, §II.D), a
 * number of histories (§II.D); the result is the dose per voxel and its
 * statistical uncertainty (§II.D, the Delta D estimator).
 *
 * Conventions, for every call:
 *  - every call returns a gpumcd_status; no call aborts, traps or exits;
 *  - input arrays are copied; the caller keeps ownership of everything it passes;
 *  - output arrays are caller-allocated;
 *  - pointers documented as "host" are ordinary CPU memory, pointers documented
 *    as "device" are CUDA device memory of the context's device (for example
 *    from torch), and `stream` is a cudaStream_t passed as void* (NULL means
 *    the context's own stream);
 *  - voxel arrays are ordered x fastest, then y, then z; the beam enters
 *    through the z = 0 face travelling along +z;
 *  - dose is in Gy per history (MeV/g x 1.602176634e-10);
 *  - energies in the ledgers are integers in units of 2^-26 MeV.
 * A context is not thread-safe: serialize calls on one context.
 */
#ifndef GPUMCD_H
#define GPUMCD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gpumcd_ctx gpumcd_ctx;
typedef int32_t gpumcd_status;

#define GPUMCD_OK 0
#define GPUMCD_ERR_INVALID_ARG (-1)    /* a pointer, size or value is out of range */
#define GPUMCD_ERR_OOM (-2)            /* device allocation failed */
#define GPUMCD_ERR_CUDA (-3)           /* a CUDA call failed (or no device) */
#define GPUMCD_ERR_QUEUE_OVERFLOW (-4) /* particle queues full: the run stopped, nothing was dropped silently */
#define GPUMCD_ERR_TIMEOUT (-5)        /* a bounded device wait gave up */
#define GPUMCD_ERR_NOT_FOUND (-6)      /* unknown phantom or plan id */
#define GPUMCD_ERR_BUDGET (-7)         /* the allocation would exceed the context's HBM budget */
#define GPUMCD_ERR_STATE (-8)          /* a call came in the wrong order (e.g. no materials loaded) */

#define GPUMCD_MAX_MATERIALS 4
#define GPUMCD_MAX_ELEMENTS 16
#define GPUMCD_MAX_PLANS_PER_RUN 64
#define GPUMCD_MAX_INFLIGHT 2        /* launch sequences gpumcd_submit keeps in flight at once */
#define GPUMCD_MAX_SPECTRUM_BINS 1024

#define GPUMCD_PHOTON 0
#define GPUMCD_ELECTRON 1
#define GPUMCD_BEAM_PENCIL 0
#define GPUMCD_BEAM_SQUARE 1
#define GPUMCD_BEAM_PHASE_SPACE 2 /* primaries listed by the caller, history h taking record h mod n */
/* Energy grouping of a polyenergetic source (gpumcd_source.energy_grouping):
 * particles of similar energy are started together, the divergence measure
 * §IV proposes for polyenergetic beams.  Warps claim primaries in chunks from
 * one cursor, so consecutive claims run side by side.  With
 * GPUMCD_ENERGY_GROUPED a spectrum or a phase space keeps its sample: each
 * history starts as it would ungrouped (the same energy draw, or the same
 * record h mod n of the list as given), so on the same kernel the tallies are
 * equal bit for bit, for any split of the histories into runs.  What changes
 * is the order of the claims: each launch first sorts its histories of the
 * plan by their primary's energy (a counting sort over the spectrum's bins,
 * or over 64 bins an octave of a record's energy, of at most 2^28 histories a
 * launch; the rest are claimed as numbered) and claims them in decreasing
 * order.  So the warps, and the whole grid at any moment, start histories of
 * similar energy, the longest first.  A monoenergetic beam is unchanged.  A
 * launch holding a grouped spectral plan runs the phase-space kernel, with
 * its restrictions. */
#define GPUMCD_ENERGY_UNGROUPED 0
#define GPUMCD_ENERGY_GROUPED 1

/* Energy unit of the ledgers and of the dose tally: 2^-26 MeV. */
#define GPUMCD_ENERGY_QUANTUM_MEV (1.0 / 67108864.0)

/* One material: element mass fractions and mean excitation energy
 * (§II.C.2 composition data).  Z, A (g/mol) and w (mass fraction) for
 * n_elements <= GPUMCD_MAX_ELEMENTS entries; the w need not be normalized. */
typedef struct {
    int32_t n_elements;
    int32_t Z[GPUMCD_MAX_ELEMENTS];
    double A[GPUMCD_MAX_ELEMENTS];
    double w[GPUMCD_MAX_ELEMENTS];
    double I_eV;
} gpumcd_material;

/* Transport cut-offs and thresholds in MeV (§II.A P_cut, §II.B E_c/K_cut) and
 * the step controls: estepe = largest fractional CSDA loss per step (the
 * e_s-max bound of §II.B.3); e_max = top of the table energy range (<= 20);
 * nudge_cm = distance added to the voxel-boundary distance of a step. */
typedef struct {
    double p_cut, e_abs, t_c, k_c, estepe, e_max, nudge_cm;
} gpumcd_physics;

/* Source (§II.C.2 initParticle): particle type, beam shape and energy.
 * A spectrum has n_spectrum bins with n_spectrum+1 increasing edges (host,
 * MeV) and n_spectrum non-negative weights (host); n_spectrum = 0 selects the
 * monoenergetic energy_mev.  Pencil beams enter at (center_cm[0],
 * center_cm[1], 0); square beams are uniform over a field_cm x field_cm square
 * centred there. */
typedef struct {
    int32_t particle;
    int32_t beam;
    double energy_mev;
    int32_t n_spectrum;
    const double *spectrum_edges;
    const double *spectrum_weights;
    double center_cm[2];
    double field_cm;
    /* GPUMCD_BEAM_PHASE_SPACE (the paper's outlook, §V): n_phase_space records
     * of 7 doubles, x, y, z (cm), ux, uy, uz (normalised on upload), E (MeV,
     * in (0, e_max]), all of `particle`; history h starts as record h mod n.
     * Host array, copied at gpumcd_plan_open; energy and spectrum are ignored.
     * A launch holding such a plan runs a separately compiled kernel (none of
     * the GPUMCD_LAUNCH_PROFILE, GPUMCD_LAUNCH_WARP_AGGREGATE,
     * GPUMCD_LAUNCH_KERMA flags nor a refill_period other than 1: else
     * GPUMCD_ERR_INVALID_ARG at run time). */
    int32_t n_phase_space;
    const double *phase_space;
    /* GPUMCD_ENERGY_UNGROUPED or GPUMCD_ENERGY_GROUPED (another value:
     * GPUMCD_ERR_INVALID_ARG at gpumcd_plan_open or gpumcd_simulate). */
    int32_t energy_grouping;
} gpumcd_source;

/* Launch tuning; 0 in a field keeps the current value.  See gpumcd_set_launch. */
typedef struct {
    uint32_t block_threads;   /* threads per CTA (multiple of 32, <= 1024) */
    uint32_t blocks_per_sm;   /* resident CTAs per SM of the persistent grid */
    uint32_t stack_capacity;  /* per-warp particle stack entries per type */
    uint32_t switch_high;     /* a warp switches type when the other stack holds this many (= stack_capacity: never) */
    uint32_t refill_low;      /* ...or when it fills fewer lanes than this and the other type has work */
    uint32_t chunk;           /* primaries or queued particles a warp claims at once */
    uint32_t overflow_capacity; /* global overflow queue entries per type */
    uint32_t flags;           /* GPUMCD_LAUNCH_* */
    uint32_t refill_period;   /* lane refill policy, the divergence-reduction ablation (below) */
} gpumcd_launch;

/* refill_period: 1 (the default) refills a warp's empty lanes at every pass,
 * the persistent "pool" of GPUMCD §II.C.3.  N >= 2 refills them only every
 * N-th pass of the warp or when all its lanes are empty, like the paper's
 * stream compaction after N steps.  GPUMCD_REFILL_WHEN_EMPTY refills only
 * an empty warp, so each set of 32 particles runs until its slowest one ends
 * (the paper's base configuration).  In the last two forms a warp also
 * considers a low-occupancy type switch only on refill passes.  Hard-event
 * passes and type switches by stack level stay on in every form.  The
 * tallies do not depend on the form.  A form other than 1 runs a separately
 * compiled kernel: it needs none of GPUMCD_LAUNCH_PROFILE,
 * GPUMCD_LAUNCH_WARP_AGGREGATE or GPUMCD_LAUNCH_KERMA (else GPUMCD_ERR_INVALID_ARG). */
#define GPUMCD_REFILL_WHEN_EMPTY 0xFFFFFFFFu

#define GPUMCD_LAUNCH_WARP_AGGREGATE 1u /* combine a warp's deposits to one voxel into one atomic */
#define GPUMCD_LAUNCH_PROFILE 2u        /* count clock cycles per event type (see gpumcd_debug_counters) */
/* The two flags above select separately compiled kernels: they cannot be combined with each
 * other, with GPUMCD_LAUNCH_KERMA or with a refill_period other than 1 (GPUMCD_ERR_INVALID_ARG). */
#define GPUMCD_LAUNCH_GRAPH 4u          /* replay a sequence's first launch from a captured CUDA graph */
/* Photon-only transport: every electron (a photon's secondary, or a primary) deposits its
 * kinetic energy in the voxel where it is created, and no electron is transported.  The
 * "photon-only fast mode" of the paper's outlook; the dose is then the kerma of the photon
 * field (kinetic energy released per mass), not the absorbed dose.  A separately compiled
 * kernel: it needs none of GPUMCD_LAUNCH_PROFILE, GPUMCD_LAUNCH_WARP_AGGREGATE or a
 * refill_period other than 1 (else GPUMCD_ERR_INVALID_ARG). */
#define GPUMCD_LAUNCH_KERMA 8u

/* Counters of one run.  The ledger satisfies, exactly,
 * e_deposited + e_escaped + e_rest == e_incident. */
typedef struct {
    uint64_t histories;
    uint64_t e_incident, e_deposited, e_escaped, e_rest;
    uint64_t n_photon_events, n_photon_real, n_compton, n_photo, n_pair;
    uint64_t n_electron_steps, n_hard_real, n_hard_fict, n_moller, n_brem;
    uint64_t n_photons, n_electrons, n_overflow;
    uint64_t n_spilled;        /* particles moved from warp stacks to the global overflow queue */
    uint64_t n_sampler_capped; /* rejection samplers stopped at their proposal cap (expected 0) */
    uint32_t n_launches, n_batches;
    double transport_ms; /* device time of the transport launches */
    double d_max_gy;     /* largest voxel dose */
    double s_thr;        /* mean sigma/D over voxels with D > threshold * D_max */
} gpumcd_run_stats;

/* Name of a status code; never NULL. */
const char *gpumcd_status_string(gpumcd_status status);

/* Creates a context on CUDA device `device`.  Device memory the context
 * allocates (phantoms, tallies, scratch) is limited to hbm_budget_bytes
 * (0 = no limit).  *out receives the context, or NULL on error. */
gpumcd_status gpumcd_init(gpumcd_ctx **out, int32_t device, uint64_t hbm_budget_bytes);

/* Frees every resource of the context; NULL is accepted. */
gpumcd_status gpumcd_destroy(gpumcd_ctx *ctx);

/* Loads n <= GPUMCD_MAX_MATERIALS materials (host array, copied) and the
 * transport parameters, and builds the cross-section, stopping-power and
 * multiple-scattering tables on the device in FP64 (stored FP32 on a log
 * energy grid, §II.C.2).  Phantoms and plans must be destroyed first if any
 * exist (GPUMCD_ERR_STATE). */
gpumcd_status gpumcd_load_materials(gpumcd_ctx *ctx, const gpumcd_material *materials, int32_t n,
                                    const gpumcd_physics *physics);

/* Copies a phantom (§II.C.2: composition ids and densities) to the device.
 * dims (host, 3 ints >= 1), voxel_cm (host, 3 doubles > 0), material_ids
 * (host, nx*ny*nz bytes, each < number of loaded materials) and densities
 * (host, nx*ny*nz floats in (0, 16) g/cm^3).  Densities are kept with a
 * resolution of 2^-24 g/cm^3.  *phantom_id receives a handle. */
gpumcd_status gpumcd_create_phantom(gpumcd_ctx *ctx, const int32_t dims[3], const double voxel_cm[3],
                                    const uint8_t *material_ids, const float *densities,
                                    int32_t *phantom_id);

/* As gpumcd_create_phantom with device arrays, enqueued on `stream`. */
gpumcd_status gpumcd_create_phantom_device(gpumcd_ctx *ctx, const int32_t dims[3],
                                           const double voxel_cm[3], const uint8_t *material_ids,
                                           const float *densities, void *stream,
                                           int32_t *phantom_id);

/* Frees a resident phantom's device memory.  GPUMCD_ERR_NOT_FOUND for an
 * unknown id, GPUMCD_ERR_STATE while a plan on it is still open. */
gpumcd_status gpumcd_destroy_phantom(gpumcd_ctx *ctx, int32_t phantom_id);

/* One dose calculation on a resident phantom (GPUMCD §II.C.2: the primaries
 * of initParticle, then the photon and electron transport of every history;
 * §II.D: the dose per voxel and its uncertainty by the Delta D estimator):
 * n_histories primaries of the source with random streams keyed by seed.  With target_rel_unc > 0 the run
 * continues in rounds of n_histories until s_thr (threshold 0.5 D_max) falls
 * to target_rel_unc or max(16 n_histories, 1e9) histories are done.
 * dose_out and sigma_out are host arrays of nx*ny*nz doubles (either may be
 * NULL); stats may be NULL. */
gpumcd_status gpumcd_simulate(gpumcd_ctx *ctx, int32_t phantom_id, const gpumcd_source *source,
                              uint64_t n_histories, uint64_t seed, double target_rel_unc,
                              double *dose_out, double *sigma_out, gpumcd_run_stats *stats);

/* As gpumcd_simulate with device outputs, enqueued on `stream` (the call
 * still waits for the run to finish before it returns). */
gpumcd_status gpumcd_simulate_device(gpumcd_ctx *ctx, int32_t phantom_id,
                                     const gpumcd_source *source, uint64_t n_histories,
                                     uint64_t seed, double target_rel_unc, double *dose_out,
                                     double *sigma_out, void *stream, gpumcd_run_stats *stats);

/* ---- plans: the batched and served forms ------------------------------- */

/* Opens a plan: a phantom, a source, a seed and a dose tally of n_batches
 * (power of two in [8, 64]; 0 = 32) batch copies kept on the device.  The
 * plan's histories are numbered from 0 and its tally accumulates over runs, so
 * the result after N histories does not depend on how the runs were split or
 * on what other plans shared them. */
gpumcd_status gpumcd_plan_open(gpumcd_ctx *ctx, int32_t phantom_id, const gpumcd_source *source,
                               uint64_t seed, uint32_t n_batches, int32_t *plan_id);

/* Frees a plan's tally and source data.  GPUMCD_ERR_NOT_FOUND for an unknown
 * id, GPUMCD_ERR_STATE while a submitted sequence holding it is in flight. */
gpumcd_status gpumcd_plan_close(gpumcd_ctx *ctx, int32_t plan_id);

/* Restarts a plan in place: zeroes its tally and ledger (on `stream`),
 * numbers its histories from 0 again and keys them with `seed`.  Nothing is
 * allocated or freed. */
gpumcd_status gpumcd_plan_reset(gpumcd_ctx *ctx, int32_t plan_id, uint64_t seed, void *stream);

/* One batched persistent launch (sequence): plan plan_ids[i] simulates its next
 * n_histories[i] histories, for n_plans <= GPUMCD_MAX_PLANS_PER_RUN distinct
 * plans (host arrays).  Enqueued on `stream`; returns once the launch sequence
 * has finished.  A set holding both electron and photon plans runs as two
 * sequences, the electron plans' then the photon plans' (one launch drawing
 * both kinds of primaries is slower); each plan's transport_ms is then its own
 * sequence's, and gpumcd_debug_counters reports the second.  The whole set is
 * validated before anything runs. */
gpumcd_status gpumcd_run(gpumcd_ctx *ctx, int32_t n_plans, const int32_t *plan_ids,
                         const uint64_t *n_histories, void *stream);

/* Asynchronous gpumcd_run, for continuous batching (a serving step of the
 * paper's history loop, §II.C, with no counterpart of its own there).  Enqueues
 * the sequence's first launch and returns a ticket at once.  Each of the
 * GPUMCD_MAX_INFLIGHT sequences has its own scratch and its own low-priority
 * stream.  That stream waits for the work already enqueued on the context's
 * stream; work the caller enqueued on other streams must be ordered by the
 * caller.
 *
 * Sequences in flight overlap on the device.  The CTAs of one fill the SMs
 * that the other's drain frees.  A plan may be in several sequences at once.
 * Its histories are numbered in submission order, and the tally is an integer
 * sum, so the result does not depend on the overlap.  While a plan is in a
 * sequence that has not finished, gpumcd_plan_result, _noalloc, _reset and
 * _close return GPUMCD_ERR_STATE.  A sequence that fails marks its plans
 * failed: their results return GPUMCD_ERR_STATE until gpumcd_plan_reset.
 * With all slots busy, the call returns GPUMCD_ERR_STATE. */
gpumcd_status gpumcd_submit(gpumcd_ctx *ctx, int32_t n_plans, const int32_t *plan_ids,
                            const uint64_t *n_histories, int32_t *ticket);

/* Without blocking: *done = 0 while the ticket's first launch runs.  Else it
 * finishes the sequence as gpumcd_wait does (including any relaunches over
 * the overflow queues), sets *done = 1 and returns the sequence's status.  A
 * ticket that is finished or unknown returns GPUMCD_ERR_NOT_FOUND. */
gpumcd_status gpumcd_poll(gpumcd_ctx *ctx, int32_t ticket, int32_t *done);

/* Blocks until the ticket's sequence has finished; returns its status. */
gpumcd_status gpumcd_wait(gpumcd_ctx *ctx, int32_t ticket);

/* FP64 fold of a plan's tally (§II.D): dose and sigma in Gy per history into
 * device arrays of nx*ny*nz doubles (either may be NULL), plus stats with
 * s_thr over voxels with dose > threshold_frac * D_max. */
gpumcd_status gpumcd_plan_result(gpumcd_ctx *ctx, int32_t plan_id, double threshold_frac,
                                 double *dose_out, double *sigma_out, void *stream,
                                 gpumcd_run_stats *stats);

/* gpumcd_plan_result with host outputs: dose_out and sigma_out are host arrays
 * of nx*ny*nz doubles (either may be NULL; pinned memory copies fastest).  The
 * fold runs on the context's stream into the context's scratch and both arrays
 * are copied back before the call returns.  Errors as gpumcd_plan_result. */
gpumcd_status gpumcd_plan_result_host(gpumcd_ctx *ctx, int32_t plan_id, double threshold_frac,
                                      double *dose_out, double *sigma_out, gpumcd_run_stats *stats);

/* Runs plans to a target uncertainty (§II.D: s, the mean of sigma/D over the
 * voxels with dose above threshold_frac x D_max; the "1% uncertainty" of a
 * dose calculation).  All n_plans <= GPUMCD_MAX_PLANS_PER_RUN distinct plans
 * (host array plan_ids) run together in rounds over the plans still above the
 * target, each round followed by their folds, all on `stream`.  In a round, a
 * plan given at least 2^23 histories runs in a launch of its own; the others
 * share one gpumcd_run (which saves a launch's fixed cost per plan, while
 * plans that share a launch share the SMs' caches).
 * In the first round plan i runs first_histories[i] more histories; after
 * each round a plan with N histories and uncertainty s > target is given
 * enough to reach max(1.05 N (s/target)^2, 1.1 N), since s falls as 1/sqrt(N).
 * Every round's count is a whole multiple of the plan's n_batches (equal
 * batches) and a plan stops at max_histories[i] in total.  A plan's schedule
 * depends on its own results only, so running plans together or one by one
 * gives the same histories and, bit for bit, the same tallies.  Outputs (host,
 * optional): histories_out[i] the plan's total histories, s_thr_out[i] its
 * final s (infinity if no dose), *rounds_out the rounds run,
 * *transport_ms_out the device time of their transport launches and
 * *sequences_out the launch sequences they took.  Plans continue
 * from the histories they hold.  Errors: GPUMCD_ERR_INVALID_ARG (target <= 0,
 * threshold outside [0, 1], first_histories[i] = 0, max_histories[i] below
 * first_histories[i] or above 2^32, a repeated id), GPUMCD_ERR_NOT_FOUND,
 * GPUMCD_ERR_STATE (a plan in flight or failed), or any error of gpumcd_run
 * or gpumcd_plan_result (the plans then hold the rounds that finished). */
gpumcd_status gpumcd_run_to_uncertainty(gpumcd_ctx *ctx, int32_t n_plans, const int32_t *plan_ids,
                                        const uint64_t *first_histories, const uint64_t *max_histories,
                                        double target_rel_unc, double threshold_frac, void *stream,
                                        uint64_t *histories_out, double *s_thr_out, uint32_t *rounds_out,
                                        double *transport_ms_out, uint32_t *sequences_out);

/* Histories of a plan's finished sequences. */
gpumcd_status gpumcd_plan_histories(gpumcd_ctx *ctx, int32_t plan_id, uint64_t *histories);

/* Device bytes the context currently holds, and its budget. */
gpumcd_status gpumcd_memory(gpumcd_ctx *ctx, uint64_t *used_bytes, uint64_t *budget_bytes);

/* ---- allocation-free result ---------------------------------------------- */

/* Largest phantom, in voxels, that gpumcd_plan_result_noalloc accepts. */
#define GPUMCD_NOALLOC_MAX_VOXELS 67108864

/* The paper has no counterpart to this call.
 *
 * The same dose and sigma as gpumcd_plan_result, bit for bit (it uses the same
 * per-voxel arithmetic), and the same stats (s_thr to about 1e-12 relative, as
 * it sums in another order), but the call allocates no memory at all.
 * It is meant for callers that cannot allocate device memory when they ask for
 * a result: a serving loop whose HBM budget is already committed in full to
 * resident phantoms and tallies, or a latency-bound loop in which a
 * cudaMalloc/cudaFree pair would stall the device.  dose_out and sigma_out
 * (device, nx*ny*nz doubles) are required here.
 *
 * Its reduction scratch is a fixed array of 128 KiB in the library's device
 * code, which every GPU that loads the library holds until the process exits.
 * That array bounds the phantom to GPUMCD_NOALLOC_MAX_VOXELS voxels; a larger
 * phantom returns GPUMCD_ERR_INVALID_ARG.  The first call on a device looks up
 * the array's device address (under a lock, so first calls from several host
 * threads are safe), so make that first call before any stream capture begins
 * on any thread.  Every call reuses the same array: calls whose work overlaps
 * on the GPU (other streams or other host threads) race, so serialize them.
 * The call is synchronous: it waits on `stream` for the fold and copies the
 * stats to the host before it returns.  A plan with no histories yet returns
 * GPUMCD_ERR_STATE. */
gpumcd_status gpumcd_plan_result_noalloc(gpumcd_ctx *ctx, int32_t plan_id, double threshold_frac,
                                         double *dose_out, double *sigma_out, void *stream,
                                         gpumcd_run_stats *stats);

/* ---- launch tuning ------------------------------------------------------ */

/* Sets the launch of later runs; fields left 0 keep their value.  A new
 * context starts at 1024 threads x 1 CTA per SM, stack_capacity 512,
 * switch_high 320, refill_low 16, chunk 32, overflow_capacity 2^20, flags 0.
 * Supported shapes have block_threads a multiple of 32, 1 <= blocks_per_sm
 * <= 4 and at most 1024 threads per SM (block_threads x blocks_per_sm):
 * shapes of up to 512 threads per SM run a kernel with 128 registers a
 * thread, up to 768 (at most 384 a CTA) one with 80, the others one with 64.
 * Also required:
 * 128 <= stack_capacity <= 65536, 32 <= switch_high <= stack_capacity,
 * refill_low <= 32, 1 <= chunk <= 4096 and 64 <= overflow_capacity <= 2^26.
 * Anything else returns GPUMCD_ERR_INVALID_ARG, and so does a call while a
 * submitted sequence is in flight (GPUMCD_ERR_STATE).  The launch changes the
 * speed of a run, never its result. */
gpumcd_status gpumcd_set_launch(gpumcd_ctx *ctx, const gpumcd_launch *launch);
/* Copies the context's current launch into *launch (host memory). */
gpumcd_status gpumcd_get_launch(gpumcd_ctx *ctx, gpumcd_launch *launch);

/* ---- diagnostics used by the tests ------------------------------------- */

/* Copies the device FP32 tables to host memory.  which = 0: photon tables
 * [material][mu_total, mu_compton, mu_photo][grid] in cm^2/g; 1: electron
 * tables [material][L_restricted, Sigma_hard, Sigma_brem, lambda1_inv][grid];
 * 2: the multiple-scattering ln(a) table; 3: the energy grids
 * [photon grid | electron grid] in MeV.  With out == NULL only *count is set. */
gpumcd_status gpumcd_get_tables(gpumcd_ctx *ctx, int32_t which, float *out, int32_t *count);

/* Runs one of the device samplers n times (host output of n floats):
 * kind 0 Klein-Nishina cos(theta) at photon energy p0; 1 Sauter cos(theta) at
 * kinetic energy p0; 2 Moller eps at T = p0; 3 bremsstrahlung k at T = p0 in
 * material `material`; 4 multiple-scattering mu at G1 = p0; 5 source energy
 * of the spectrum in `source`; 6 Klein-Nishina k'/k at p0. */
gpumcd_status gpumcd_debug_sample(gpumcd_ctx *ctx, int32_t kind, double p0, int32_t material,
                                  const gpumcd_source *source, uint64_t n, uint64_t seed,
                                  float *out);

/* Raw device counters of the last gpumcd_run launch sequence (host array of
 * *count entries; with out == NULL only *count is set): event counts, spills,
 * and with GPUMCD_LAUNCH_PROFILE the per-type cycle profile.  The order is
 * that of the library's counter list (photon events, real photon events,
 * Compton, photoelectric, pair, electron steps, real and fictitious hard
 * events, Moller, bremsstrahlung, photons, electrons, overflows, spilled
 * particles, capped samplers, then cycles[2], passes[2] and active lanes[2]
 * of the photon and electron warps' event passes, refill cycles, type
 * switches). */
gpumcd_status gpumcd_debug_counters(gpumcd_ctx *ctx, uint64_t *out, int32_t *count);

/* A phantom's majorant tables (GPUMCD §II.A mu_max, §II.B.3 electron
 * Woodcock) and per-material maximum densities, copied to host arrays:
 * majorants[0..511] = max over materials m of rho_max[m] * mu_m on the photon
 * grid (1/cm), majorants[512..1023] = the running maximum over the electron
 * grid of max_m rho_max[m] * Sigma_hard,m (1/cm); rho_max holds
 * GPUMCD_MAX_MATERIALS entries (g/cm^3, 0 for materials absent from the
 * phantom), each the largest density of that material after quantisation to
 * 2^-24 g/cm^3.  Photon flights sample with the photon majorant.  An electron
 * step samples its hard distance with its own voxel's rho * Sigma_hard at the
 * step's start energy, an exact majorant because the step stays in the voxel;
 * the electron half here is the phantom-wide bound of §II.B.3, kept for
 * diagnostics.  Errors: GPUMCD_ERR_NOT_FOUND for an unknown phantom. */
gpumcd_status gpumcd_debug_majorants(gpumcd_ctx *ctx, int32_t phantom, float *majorants, float *rho_max);

/* Philox4x32-10 on the device: for i < n, out[4i..4i+3] = Philox(counter
 * ctr[4i..4i+3], key) (host arrays).  With use_curand != 0 the same words come
 * from cuRAND's Philox4_32_10 device generator started at that counter. */
gpumcd_status gpumcd_debug_philox(gpumcd_ctx *ctx, const uint32_t *ctr, const uint32_t key[2],
                                  uint64_t n, int32_t use_curand, uint32_t *out);

#ifdef __cplusplus
}
#endif
#endif
