/*
 * pmc.h -- C ABI of the GB300 proton Monte Carlo engine.
 *
 * The engine implements the condensed-history proton transport method of
 * Wan Chan Tseung, Ma & Beltran (arXiv:1409.8336): transport through a
 * voxelised geometry with tabulated stopping power and CSDA range (Sec. II.A.2,
 * Eq. 1 and Eq. 2), Gaussian energy-loss straggling, Highland multiple
 * scattering scaled by 1.07 with a random hinge (Sec. II.A.2-3), coherent
 * nuclear elastic scattering with the Ranft angular distribution (Sec. II.A.5,
 * Eq. 3), non-elastic collisions handed to an intranuclear-cascade plus
 * evaporation event generator (Sec. II.A.4), and dose scoring in ten groups for
 * a per-voxel statistical error (Sec. II.B.2).
 *
 * Conventions for every entry point:
 *   - units are MeV, cm, g/cm^3; volumes are indexed x fastest:
 *     v = (iz * ny + iy) * nx + ix;
 *   - host arrays passed in are owned by the caller and copied during the call;
 *     device memory is owned by the context (allocated through the optional
 *     allocator in pmc_options, else cudaMalloc) and released by pmc_destroy;
 *   - the return value is PMC_OK (0) or a negative PMC_E_* code; the message of
 *     the last failure is available from pmc_last_error.  No C++ exception
 *     crosses this boundary.  A context is not thread safe.
 */
#ifndef PMC_H
#define PMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PMC_OK 0
#define PMC_E_INVALID (-1)        /* bad argument or call order */
#define PMC_E_OOM (-2)            /* device allocation failed */
#define PMC_E_QUEUE_OVERFLOW (-3) /* a particle queue was full: results incomplete */
#define PMC_E_TIMEOUT (-4)        /* a bounded device loop hit its limit */
#define PMC_E_CUDA (-5)           /* CUDA runtime error */

/* physics switches (pmc_options.physics_flags); 0 = full physics */
#define PMC_NO_STRAGGLING 1u
#define PMC_NO_MCS 2u
#define PMC_NO_ELASTIC 4u
#define PMC_NO_INELASTIC 8u
/* Moliere multiple scattering (Bethe's form of Moliere's theory: characteristic and
 * screening angles, B from B - ln B = ln(chi_c^2 / 1.167 chi_a^2) with the validity floor
 * B = 4.5, space angle from F0 + F1/B + F2/B^2) instead of the paper's Highland width
 * (Sec. II.A.2), at the step-start energy over the planned step. */
#define PMC_MOLIERE 16u
/* physics flag: Vavilov energy-loss straggling (the paper uses Bohr's Gaussian, Sec. II.A.2,
 * and prints no Vavilov formula).  Where kappa = xi / T_max <= 10 (xi = (K/2)(Z/A) rho s /
 * beta^2 over the step's path s, T_max the largest transfer to a free electron) the loss
 * fluctuation about the CSDA mean is drawn from Vavilov's distribution for the Bethe spectrum
 * of transfers, tabulated from its characteristic function (kappa clamped to [0.001, 10], the
 * quantile tails cut at 1e-4, each row centred so the mean loss stays the CSDA loss); above
 * 10, Bohr's Gaussian of the same variance. */
#define PMC_VAVILOV 32u

/* transport modes */
#define PMC_FULL_CASCADE 0        /* non-elastic events by cascade + evaporation */
#define PMC_SURROGATE 1           /* non-elastic events by the trained quantile network */

#define PMC_MAX_NUCLIDES 16
#define PMC_MAX_MATERIALS 16
#define PMC_MAX_NUC_PER_MAT 12
#define PMC_MAX_HU_BINS 16

typedef struct pmc_ctx pmc_ctx;

/* Optional device allocator (e.g. a framework's caching allocator).  `alloc`
 * and `free` are given together or not at all (pmc_create returns
 * PMC_E_INVALID for one without the other).  `alloc` must return memory of the
 * context's device aligned to 256 bytes, as cudaMalloc does (the kernels move
 * records and weights in 16-byte units and by bulk copies); a misaligned block
 * is handed back to `free` and the call that needed it fails with PMC_E_OOM. */
typedef void* (*pmc_alloc_fn)(size_t bytes, void* user);
typedef void (*pmc_free_fn)(void* ptr, void* user);

typedef struct {
    int device;               /* CUDA device ordinal */
    int n_batches;            /* statistical groups, 2..1024 (paper: 10, Sec. II.B.2) */
    unsigned physics_flags;   /* PMC_NO_* */
    int block_size;           /* transport block size; 0 = autotuned on first transport */
    int64_t chunk;            /* histories per sub-group (Sec. II.B.2); 0 = automatic */
    pmc_alloc_fn alloc;       /* NULL = cudaMalloc */
    pmc_free_fn free;
    void* alloc_user;
} pmc_options;

/* A target nuclide (Z, A), its molar mass (g/mol) and mean excitation energy (eV). */
typedef struct { int Z, A; double mass_u, I_eV; } pmc_nuclide;

/* A material: mass fractions w of nuclides nuc[0..n-1], nominal density, mean
 * excitation energy (0 = Bragg additivity), and whether it keeps its own
 * stopping-power table (air and titanium, Sec. II.A.2) instead of the scaled
 * water table of Eq. 1.  Material 0 is the reference water. */
typedef struct {
    int n;
    int nuc[PMC_MAX_NUC_PER_MAT];
    double w[PMC_MAX_NUC_PER_MAT];
    double rho;
    double I_eV;
    int own_table;
} pmc_material;

/* HU bin [lo, hi) -> material, density rho = rho_a + rho_b * HU (Sec. II.A.1). */
typedef struct { int lo, hi, material; double rho_a, rho_b; } pmc_hu_bin;

/* A Gaussian pencil-beam spot entering the phantom through its z = z0 face:
 * mean energy and spread, centre and widths (cm), direction, relative weight. */
typedef struct { double E, sigma_E, x, y, sigma_x, sigma_y, u, v, w, weight; } pmc_spot;

/* Energy ledger of the last transport, in units of 2^-24 MeV:
 * incident = deposited + escaped + binding (+ rounding of a few units per event).
 * The counts: histories, condensed-history steps, elastic and non-elastic nuclear
 * collisions, secondary protons queued, events without an allowed cascade
 * (transparent) and cascade attempts redrawn, queue_high_water (unused, 0),
 * generations (launch rounds: 2, the primaries and the drain of all later
 * generations), particles dropped for want of queue room, errors (step limit or
 * a bounded device wait that ran out), and the non-elastic events generated by
 * the learned stand-in (surrogate mode: the primaries' events; the few events of
 * later generations run the full cascade inside the drain). */
typedef struct {
    int64_t incident, deposited, escaped, binding;
    int64_t histories, steps, elastic, inelastic, secondaries, transparent, inc_retries;
    int64_t queue_high_water, generations, dropped, errors;
    int64_t surrogate_events;
} pmc_ledger;

/* Creates a context on opt->device (opt may be NULL for defaults). */
int pmc_create(pmc_ctx** out, const pmc_options* opt);
void pmc_destroy(pmc_ctx* ctx);
const char* pmc_last_error(const pmc_ctx* ctx);

/* Builds the physics tables (Sec. II.A.2, II.A.4-5) for the nuclides and
 * materials and uploads them.  n_hu may be 0 when the phantom is given by
 * material indices.  Errors: PMC_E_INVALID for counts beyond the PMC_MAX_*
 * limits, fractions that do not sum to 1 within 1e-6, or material 0 not a
 * scaled-table material. */
int pmc_load_materials(pmc_ctx* ctx, const pmc_nuclide* nuc, int n_nuc,
                       const pmc_material* mat, int n_mat,
                       const pmc_hu_bin* hu, int n_hu);

/* Uploads the voxel geometry (Sec. II.A.1): either hu (int16 HU, mapped by
 * the HU bins) or mat (uint8 material index) with rho (float density); the
 * other pointer(s) NULL.  Pointers are host memory. */
int pmc_load_phantom(pmc_ctx* ctx, int nx, int ny, int nz,
                     double dx, double dy, double dz, double x0, double y0, double z0,
                     const int16_t* hu, const uint8_t* mat, const float* rho);

/* Appends n spots; pmc_clear_spots removes them all. */
int pmc_add_spots(pmc_ctx* ctx, const pmc_spot* spots, int n);
int pmc_clear_spots(pmc_ctx* ctx);

/* Simulates n_histories primary protons, spread over the spots in proportion
 * to weight (largest remainder), with random numbers keyed by seed (Sec. II.B:
 * per sub-group, the phase space and transport of the primaries, the event stage
 * of their non-elastic collisions -- cascade and evaporation, or with mode
 * PMC_SURROGATE the learned stand-in -- then one drain launch that transports
 * every later generation and runs its events through the full cascade; one CUDA
 * graph per run shape).  History h scores into group h mod n_batches.  Tallies
 * are zeroed first; the call ends with the batch-statistics kernel, so dose and
 * error are ready on the device.  stream: a cudaStream_t or NULL (the context's
 * own stream).  The call blocks until the run has finished.  PMC_E_TIMEOUT when a
 * particle exceeded the step limit or a bounded device wait ran out (the run's
 * ledger is still readable); PMC_E_QUEUE_OVERFLOW when a queue was full. */
int pmc_transport(pmc_ctx* ctx, uint64_t n_histories, uint64_t seed, int mode, void* stream);

/* Dose (Gy) and its statistical standard error per voxel, to host arrays of
 * n_voxels doubles (either may be NULL). */
int pmc_read_dose(pmc_ctx* ctx, double* dose_gy, double* sigma_gy, size_t n_voxels);

/* Raw group tallies [n_voxels][n_batches] in units of 2^-24 MeV (host array). */
int pmc_read_tally(pmc_ctx* ctx, int64_t* tally, size_t n);

int pmc_read_ledger(pmc_ctx* ctx, pmc_ledger* out);

/* Per-history ledger for the first max_histories histories of the next
 * transports ([h][4]: incident, deposited, escaped, binding in 2^-24 MeV);
 * 0 disables it.  Read with pmc_read_history_ledger. */
int pmc_enable_history_ledger(pmc_ctx* ctx, uint64_t max_histories);
int pmc_read_history_ledger(pmc_ctx* ctx, int64_t* out, uint64_t n_histories);

/* Records up to cap protons leaving the grid in the next transports
 * ([i][8] floats: E, x, y, z, u, v, w, history); 0 disables it. */
int pmc_enable_escape_record(pmc_ctx* ctx, uint64_t cap);
int pmc_read_escape_record(pmc_ctx* ctx, float* out, uint64_t cap, uint64_t* n);

/* Debug deposit log: pins the fixed-point tally (Sec. II.B.3: dose tallies updated by
 * atomic operations; here 64-bit integers in units of 2^-24 MeV).  With the log enabled,
 * every deposit of the next transports (condensed-history steps, absorbed protons, elastic
 * recoils, cascade and evaporation fragments, residual nuclei) is also recorded as the
 * energies it was computed from: tally entry [voxel][group] received
 *   llrint(e[0] 2^24) - llrint(e[1] 2^24) - llrint(e[2] 2^24)   (round half to even),
 * so the integer sum of the log equals the tally bit for bit.  Meant for small runs
 * (<= about 1e3 histories: some 200 records per history).  The log runs the full cascade
 * with the paper's physics options only (Highland, Bohr, no LET): pmc_transport returns
 * PMC_E_INVALID otherwise.
 * pmc_enable_deposit_log: room for cap records on the device (32 bytes each); 0 frees it.
 * pmc_read_deposit_log: copies min(records, cap) records of the last transport to out and
 *   the number logged to *n; PMC_E_QUEUE_OVERFLOW when the log was too small (the records
 *   beyond its capacity are lost), PMC_E_INVALID when it is not enabled. */
typedef struct {
  int32_t voxel;             /* v = (iz * ny + iy) * nx + ix */
  int32_t group;             /* statistical group h mod n_batches */
  double e[3];               /* MeV: deposit = fix(e[0]) - fix(e[1]) - fix(e[2]) */
} pmc_deposit;
int pmc_enable_deposit_log(pmc_ctx* ctx, uint64_t cap);
int pmc_read_deposit_log(pmc_ctx* ctx, pmc_deposit* out, uint64_t cap, uint64_t* n);

/* Dose-averaged LET scored beside the dose (Sec. IV: LET_d computed together with
 * the physical dose).  Every energy loss q of a transported proton (the steps, and
 * the remainder of a proton absorbed below E_cut or within its residual range) is
 * weighted by L, the mean CSDA stopping power of the local medium over the path of
 * that loss (keV/um): the step's CSDA loss over its length, or E/R for an absorbed
 * proton.  Recoil nuclei and cascade fragments do not score (as in Sec. IV).
 * LET_d(v) = sum q L / sum q per voxel, in keV/um, with its standard error from the
 * group tallies by the ratio estimator:
 *   var = B/(B-1) sum_b (num_b - LET_d den_b)^2 / den^2.
 * pmc_enable_let: on != 0 scores LET in the next transports (two more int64
 *   [n_voxels][n_batches] tallies on the device); 0 frees them.
 * pmc_read_let: LET_d and its standard error per voxel (host arrays of n_voxels,
 *   either may be NULL; 0 where no proton lost energy).  PMC_E_INVALID unless the
 *   last transport scored LET on the current grid.
 * pmc_read_let_tally: raw group tallies [n_voxels][n_batches] (host arrays):
 *   num in 2^-24 MeV keV/um, den in 2^-24 MeV. */
int pmc_enable_let(pmc_ctx* ctx, int on);
int pmc_read_let(pmc_ctx* ctx, double* let_d, double* sigma, size_t n_voxels);
int pmc_read_let_tally(pmc_ctx* ctx, int64_t* num, int64_t* den, size_t n);

/* Sets the transport launch shape (block size, histories per sub-group)
 * chosen by the caller; 0 keeps the current value.  A non-zero block size
 * also switches the autotuner off. */
int pmc_set_launch(pmc_ctx* ctx, int block_size, int64_t chunk);

/* Autotuner of the launch shape (the paper sizes sub-groups as multiples of
 * the block size, Sec. II.B.2): times full transports of n_histories for
 * block sizes {128, 192, 256} x sub-group sizes {n, n/2 when n >= 2^17} and
 * keeps the fastest (written to *block_out, *chunk_out when not NULL).  It
 * runs on the first pmc_transport of a context created with block_size 0;
 * the trial runs overwrite the tallies. */
int pmc_autotune(pmc_ctx* ctx, uint64_t n_histories, uint64_t seed, int* block_out, int64_t* chunk_out);

/* Kernel timing: with on = 1 the run records CUDA events around every launch
 * group on the run's stream (inside the captured graph); with on = 2 around
 * the primary-transport groups only (the lightest: about 3 % of a step less
 * than on = 1 on the slab workload); 0 turns it off.  Other values are
 * PMC_E_INVALID.  A group is the kernels of one stage launched back to back:
 * phase space + transport for the primaries, cascade + evaporation, the
 * secondary drain's set-up + drain, the dose statistics.
 * pmc_read_profile returns, per kind (0 primary transport, 1 secondary
 * transport -- the drain, which also runs the secondaries' cascades --,
 * 2 cascade of the primaries' events, 3 dose statistics), for the last
 * transport: in ms[0..3] the summed milliseconds of its groups, in ms[4..7]
 * the span from the first group's start to the last group's end (groups of two
 * sub-groups may run concurrently), in launches[0..3] the number of groups and
 * in launches[4..7] the number of kernels they launched (launches has 8
 * entries), and the primary-transport step count in *primary_steps. */
int pmc_enable_profile(pmc_ctx* ctx, int on);
int pmc_read_profile(pmc_ctx* ctx, double* ms, int64_t* launches, int64_t* primary_steps);

/* Transport that allocates no device memory (the paper has no counterpart).
 * For callers that cannot call cudaMalloc during a dose calculation -- a
 * real-time loop that must not stall on the allocator, or an application that
 * gave its whole device memory to its own pool.  The call itself synchronises
 * its stream and blocks until the run is done, so it cannot be made from a CUDA
 * stream callback (no CUDA call is allowed there) or inside a stream capture.  It runs the full cascade (never the learned
 * stand-in), with the context's physics options, and produces the same tallies
 * as pmc_transport for the same seed; it does not score LET, the per-history
 * ledger, the escape record or the deposit log, and pmc_read_dose / pmc_read_let
 * keep returning the last allocating run's results (the caller's arrays hold
 * this run's).  All scratch (three particle queues, the residual nuclei
 * between cascade and evaporation, counters, the secondary drain's control block
 * and ready marks, spot table, seed) lives in one
 * static device array of PMC_NOALLOC_SCRATCH_BYTES that every GPU loading this
 * library holds until the process exits.  Inputs are the context's loaded
 * materials, phantom and spots; outputs are caller-owned device arrays: tally
 * [n_voxels][n_batches] int64 (units of 2^-24 MeV, zeroed by the call) and,
 * optionally (both or neither), dose_gy and sigma_gy [n_voxels].  At most
 * PMC_NOALLOC_MAX_SPOTS spots may receive histories; more is rejected with
 * PMC_E_INVALID.  All calls on a device share the array and it keeps the last
 * call's contents (each call clears what must start at zero); calls from
 * several host threads of one process are serialised per device by a lock, and
 * work of another process never shares it.  The first call on a device looks up
 * the array's device address (once per device, thread-safe).  Blocks until done;
 * pmc_read_ledger then reports this run. */
#define PMC_NOALLOC_CHUNK 65536          /* histories per sub-group */
#define PMC_NOALLOC_MAX_SPOTS 4096
#define PMC_NOALLOC_SCRATCH_BYTES                                                                  \
    (3ull * PMC_NOALLOC_CHUNK * 48ull + PMC_NOALLOC_CHUNK * 128ull + 1792ull + PMC_NOALLOC_CHUNK * 12ull + \
     PMC_NOALLOC_MAX_SPOTS * 56ull)
int pmc_transport_noalloc(pmc_ctx* ctx, uint64_t n_histories, uint64_t seed, int64_t* tally,
                          double* dose_gy, double* sigma_gy, void* stream);

/* ---- learned stand-in of the event generator (the paper has none) ----
 * A conditional quantile network (MLP 32-256-256-256-256-16, ReLU, BF16
 * tensor-core math with FP32 accumulation and FP32 master weights) that maps
 * (incident energy, target nuclide, a multiplicity token, ten uniforms) to
 * quantiles of a non-elastic event's summary: number of protons above E_cut,
 * energies and polar cosines of up to four of them, and the locally deposited
 * energy.  Trained with the pinball loss on events from the engine's own
 * cascade + evaporation kernel (Sec. II.A.4 method); used by pmc_transport
 * with PMC_SURROGATE in place of that kernel.  The targets are the loaded
 * nuclides with A >= 2, in load order (at most 6). */
#define PMC_SURROGATE_PARAMS 209936
#define PMC_SURROGATE_FEATURES 12   /* E, target slot, n_p, T/E[4], cos[4], local/E */

typedef struct {
    uint64_t n_events;   /* training events drawn from the cascade kernel (E uniform 10-250 MeV) */
    int epochs, batch;   /* batch: events per step (two network rows each) */
    double lr, weight_decay;
    uint64_t seed;
} pmc_train_opts;

typedef struct { double first_loss, last_loss; int64_t steps; } pmc_train_result;

/* n_events event summaries [n][PMC_SURROGATE_FEATURES] (host array), as used for training. */
int pmc_surrogate_dataset(pmc_ctx* ctx, uint64_t n_events, uint64_t seed, float* out);
/* Generates the data, trains with AdamW on the device, keeps the network in the context. */
int pmc_train_surrogate(pmc_ctx* ctx, const pmc_train_opts* opts, pmc_train_result* result);
/* Reads / sets the network's PMC_SURROGATE_PARAMS parameters (host arrays). */
int pmc_surrogate_params(pmc_ctx* ctx, float* params, size_t n);
int pmc_surrogate_load(pmc_ctx* ctx, const float* params, size_t n);
/* One forward + backward pass on given rows (host arrays): inputs x[rows][32],
 * targets y, levels tau and mask [rows][16]; returns the mean pinball loss,
 * the gradient [PMC_SURROGATE_PARAMS] and the outputs yhat [rows][16]. */
int pmc_surrogate_grad(pmc_ctx* ctx, const float* params, const float* x, const float* y, const float* tau,
                       const float* mask, int rows, float* loss, float* grad, float* yhat);
/* The loaded network on the tensor cores, as inside the transport's event stage: inputs
 * x[rows][32] -> outputs y[rows][16] (host arrays, 1 <= rows <= 1048576), BF16 weights and
 * activations with FP32 accumulation (the network is not part of the paper: it stands in
 * for Sec. II.A.4's event generator).  PMC_E_INVALID without a network or with bad
 * arguments, PMC_E_TIMEOUT if a device wait of the tensor-core pipeline timed out. */
int pmc_surrogate_infer(pmc_ctx* ctx, const float* x, int rows, float* y);

/* ---- non-elastic event generator -------------------------------------------
 * n non-elastic interactions of a proton of kinetic energy E (MeV) with the
 * loaded nuclide index `nuclide` (A >= 2): intranuclear cascade and evaporation
 * (Sec. II.A.4), the same device code and random streams (key seed, particle
 * pid0 + i for event i) as inside the transport.  The workload of Table I.
 * Synchronous on the context's stream; `out` receives the totals over the events
 * and the device time of the event kernel.  Energies in MeV. */
typedef struct {
    uint64_t events, transparent, retries;
    uint64_t count[6];                  /* emitted n, p, d, t, 3He, alpha */
    double energy[6];                   /* their summed kinetic energies */
    double residual_T, excitation_left, binding;   /* summed over the events */
    double ms;                          /* device time of the event kernel */
} pmc_event_yields;
int pmc_nonelastic_events(pmc_ctx* ctx, int nuclide, double E, uint64_t n, uint64_t seed, uint64_t pid0,
                          pmc_event_yields* out);

/* ---- multi-plan stream ---------------------------------------------------------
 * Many plans (phantom + spots + histories) through one device, several at a time.
 * A pool of n_slots concurrency slots, each an engine context with its own CUDA
 * streams, serves the plans in the order given: a plan is admitted when its device
 * footprint (pmc_plans_bytes) fits in the memory budget left by the plans running;
 * its slot uploads the phantom, transports (the same kernels, graph and random
 * streams as pmc_transport, so the dose is bit-identical to a pmc_transport of the
 * plan alone), copies dose and error out and releases the plan's buffers.  Kernels
 * of concurrently admitted plans share the SMs.  Allocation is stream-ordered from
 * one memory pool, so admitting or retiring a plan never synchronises the device.
 * The paper runs one plan at a time; this serves the batched multi-plan workload.
 *
 * pmc_plans_create: opt as for pmc_create (block_size 0 means 256: slots are not
 *   autotuned; opt->alloc is ignored); budget_bytes > 0.
 * pmc_plans_load_materials / pmc_plans_load_surrogate: as pmc_load_materials and
 *   pmc_surrogate_load, for every slot.
 * pmc_plans_bytes: the device footprint of a plan in `mode`.
 * pmc_plans_run: runs plans[0..n) (host arrays that must stay valid during the
 *   call) and fills results[n]; synchronous.  A plan whose footprint exceeds the
 *   budget is skipped with status PMC_E_OOM.  Returns PMC_OK when every plan
 *   succeeded, else the first failing plan's status. */
typedef struct pmc_plan_stream pmc_plan_stream;
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, x0, y0, z0;      /* cm, as pmc_load_phantom */
    const int16_t* hu;                  /* HU volume, or NULL with mat and rho */
    const uint8_t* mat;
    const float* rho;
    const pmc_spot* spots;
    int n_spots;
    uint64_t n_histories, seed;
    double* dose_gy;                    /* outputs: host arrays of nx*ny*nz, or NULL */
    double* sigma_gy;
} pmc_plan;
typedef struct {
    int status;                         /* PMC_OK or the plan's error */
    int slot;                           /* slot that ran it (-1: never admitted) */
    uint64_t device_bytes;              /* admitted footprint */
    double t_admit_ms, t_end_ms;        /* host clock from the start of pmc_plans_run */
    double gpu_ms;                      /* device time on its slot's stream, upload to dose */
    pmc_ledger ledger;
} pmc_plan_result;
int pmc_plans_create(pmc_plan_stream** out, const pmc_options* opt, int n_slots, uint64_t budget_bytes);
void pmc_plans_destroy(pmc_plan_stream* s);
const char* pmc_plans_last_error(const pmc_plan_stream* s);
int pmc_plans_load_materials(pmc_plan_stream* s, const pmc_nuclide* nuc, int n_nuc, const pmc_material* mat,
                             int n_mat, const pmc_hu_bin* hu, int n_hu);
int pmc_plans_load_surrogate(pmc_plan_stream* s, const float* params, size_t n);
int pmc_plans_bytes(const pmc_plan_stream* s, const pmc_plan* plan, int mode, uint64_t* bytes);
int pmc_plans_run(pmc_plan_stream* s, const pmc_plan* plans, int n, int mode, pmc_plan_result* results);

/* ---- 3-D gamma index -------------------------------------------------------
 * The dose-comparison metric of Sec. II.D (Low et al.), which the paper also
 * computes on the GPU.  For every reference voxel whose dose exceeds
 * threshold x max(ref):
 *   gamma^2 = min over evaluated voxels within search_mm of
 *             r^2 / dta_mm^2 + (eval - ref)^2 / tol^2,   tol = dose_pct/100 x max(ref)
 * (global dose criterion, on the grid, no interpolation; FP64).  Doses are
 * [nz][ny][nx], x fastest, in any unit (both grids the same); voxel sizes in cm.
 * search_mm <= 0 means 1.5 x dta_mm.  gamma[v] = sqrt(gamma^2) as float, -1 for
 * voxels not evaluated.  Pass: gamma^2 <= 1 + 1e-12.
 *
 * pmc_gamma_plan_bytes: device bytes of a plan for these voxel sizes and distance
 *   criteria (independent of the grid size).  PMC_E_INVALID if an argument is out
 *   of range or the search sphere holds more than PMC_GAMMA_MAX_OFFSETS voxels.
 * pmc_gamma_plan: writes the plan (the search sphere's offsets, sorted) into
 *   `plan`, caller-owned device memory, 256-byte aligned, plan_bytes long;
 *   asynchronous on `stream` (cudaStream_t; NULL = legacy default stream).
 * pmc_gamma_device: compares device-resident grids with a plan, asynchronous on
 *   `stream`; ref, eval and gamma (may be NULL) are caller-owned device pointers.
 *   When the stream reaches completion the plan's first 16 bytes hold two uint64:
 *   voxels evaluated and voxels passing.  Allocates nothing.  A plan serves one
 *   comparison at a time (order them on one stream).
 * pmc_gamma_index: the same from host arrays (gamma may be NULL), synchronous,
 *   with device memory of its own; pass_rate = passed / evaluated (NaN if none). */
#define PMC_GAMMA_MAX_OFFSETS 65536
int pmc_gamma_plan_bytes(double dx, double dy, double dz, double dta_mm, double search_mm, size_t* bytes);
int pmc_gamma_plan(double dx, double dy, double dz, double dta_mm, double search_mm, void* plan, size_t plan_bytes,
                   void* stream);
int pmc_gamma_device(void* plan, const double* ref, const double* eval, int nx, int ny, int nz, double dose_pct,
                     double threshold, float* gamma, void* stream);
int pmc_gamma_index(const double* ref, const double* eval, int nx, int ny, int nz, double dx, double dy, double dz,
                    double dose_pct, double dta_mm, double threshold, double search_mm, float* gamma,
                    double* pass_rate);

/* Device-side evaluation of single routines, for tests.
 * pmc_debug_philox: Philox4x32-10 of n counters ctr[n][4] under key[2]
 *   (Salmon et al., SC'11) into out[n][4].
 * pmc_debug_tables: range R (g/cm^2) and inverse E(R) of material m's table
 *   at n energies (Sec. II.A.2): r_out[i] = R(E[i]), e_out[i] = E(r_out[i]).
 * pmc_debug_inc: n non-elastic events of a proton of energy E on nuclide
 *   index `nuclide` (Sec. II.A.4) with pids pid0 + i, in the frame where the
 *   proton moves along +z.  summary[n][8] = n_products, Z_res, A_res, T_res,
 *   E*_left, binding, retries, transparent; products[n][cap][5] = species
 *   (0 n, 1 p, 2 d, 3 t, 4 He3, 5 alpha), T, direction.
 * pmc_debug_elastic: n elastic scatterings on nuclide index `nuclide` at
 *   energy E (Sec. II.A.5, Eq. 3) from uniforms u[n][3];
 *   out[n][5] = T1, cos1, T2, cos2, cos_cm. */
int pmc_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n);
int pmc_debug_tables(pmc_ctx* ctx, int material, const double* E, double* r_out, double* e_out, int n);
int pmc_debug_inc(pmc_ctx* ctx, int nuclide, double E, uint64_t seed, uint64_t pid0, int n,
                  double* summary, double* products, int cap);
int pmc_debug_elastic(pmc_ctx* ctx, int nuclide, double E, const double* u, double* out, int n);

/* The event stage on its own: n non-elastic events (proton of energy E[i] MeV on nuclide
 * nuclide[i], A >= 2, moving along +z, random streams keyed by seed and identity i) through
 * the cascade and evaporation kernels (mode PMC_FULL_CASCADE, Sec. II.A.4) or through the
 * learned stand-in's event kernel (PMC_SURROGATE; needs a trained or loaded network) -- the
 * same kernels the transport runs.  Emitted protons (those above E_cut, which the transport
 * would queue) go to protons [cap][3] as (event index, kinetic energy MeV, cosine to the
 * incident direction), their number to *n_protons; local[i] (n doubles, or NULL) receives the
 * energy event i deposits locally (MeV).  PMC_E_QUEUE_OVERFLOW when more than cap protons
 * were emitted (the first cap are copied). */
int pmc_debug_event_stage(pmc_ctx* ctx, int mode, const int* nuclide, const double* E, int n, uint64_t seed,
                          float* protons, uint64_t cap, uint64_t* n_protons, double* local);
/* pmc_debug_surrogate_waits: runs the tensor-core network on one 128-row tile with its MMAs
 * withheld and short mbarrier waits, so that every wait runs out: returns PMC_E_TIMEOUT
 * (the block stops, frees its tensor memory and reports), and the context stays usable.
 * PMC_E_INVALID without a loaded network. */
int pmc_debug_surrogate_waits(pmc_ctx* ctx);
/* pmc_debug_drain_waits: a full-cascade pmc_transport whose drain of the secondary
 * generations counts one item that never comes, so that it never sees its work finished and
 * every warp's bounded wait for more work runs out (after 4096 polls instead of ~1e6):
 * returns PMC_E_TIMEOUT with the run's real work done, and the context stays usable.
 * PMC_E_INVALID as pmc_transport. */
int pmc_debug_drain_waits(pmc_ctx* ctx, uint64_t n_histories, uint64_t seed);
/* pmc_debug_vavilov_table: the Vavilov straggling table the transport samples from, built on
 * the host (no device needed): quantiles of z = (loss - mean loss) / xi, [6 values of beta^2 in
 * [0, 0.5]][31 values of ln kappa in [ln 0.01, ln 10]][513 values of u in [1e-4, 1 - 1e-4]],
 * each row shifted to mean zero.  n must be 6 * 31 * 513; PMC_E_INVALID otherwise. */
int pmc_debug_vavilov_table(float* out, size_t n);

#ifdef __cplusplus
}
#endif
#endif /* PMC_H */
