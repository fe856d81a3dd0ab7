/*
 * mc.h -- C ABI of libmc, a GB300 (sm_103a) implementation of the parallel
 * checkerboard Metropolis algorithm and the parallel constrained Monte Carlo
 * algorithm for the classical Heisenberg model on a simple-cubic lattice,
 * after Lepadatu et al., arXiv:2103.03517.
 *
 * Model (Sec. 2, Eq. 2), reduced units (k_B = 1, mu_S = 1; the Zeeman field
 * H is an energy, H = mu0 mu_S H_a of Eq. 2):
 *   E_i = -J sum_{j in NN(i)} S_i.S_j - K_u (S_i.e_i)^2
 *         + K_c (Sx^2 Sy^2 + Sx^2 Sz^2 + Sy^2 Sz^2) - H.S_i
 * Acceptance (Eq. 1): a trial S' is accepted iff P < exp(-(E(S') - E(S))/T),
 * P uniform on [0, 1).
 *
 * Conventions for every entry point:
 *  - Return value is an mc_status: MC_OK (0), MC_PENDING (1) or a negative
 *    error code.  mc_last_error() returns a message for the last error of
 *    the calling thread.
 *  - Pointers named host_* or documented as host memory are read or written
 *    synchronously before the call returns; the library never keeps them.
 *  - The library owns all device memory of a lattice, from mc_create* until
 *    mc_destroy.  Handles are not thread safe: use one handle per thread.
 *    A server (mc_server_*) is internally synchronised.
 *  - mc_sweep, mc_constrained_sweep and mc_group_sweep are asynchronous on
 *    the lattice's CUDA stream; errors found on the device (MC_ERR_CONSTRAINT,
 *    MC_ERR_STATE) are reported by the next synchronising call (mc_measure,
 *    mc_samples, mc_profile, mc_get_spins, mc_sync, mc_save).
 *  - Site order of every host spin array is x + Lx (y + Ly z), three
 *    components per site (N x 3, row major); bcc / fcc / hcp lattices put
 *    the sub-lattice first: s + nsub (x + Lx (y + Ly z)).
 */
#ifndef MC_H
#define MC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_API __attribute__((visibility("default")))

typedef enum mc_status {
    MC_OK = 0,
    MC_PENDING = 1,
    MC_ERR_ARG = -1,        /* invalid argument (checked on the host)            */
    MC_ERR_NOMEM = -2,      /* device memory exhausted / job can never fit       */
    MC_ERR_CUDA = -3,       /* a CUDA call failed (message in mc_last_error)     */
    MC_ERR_TIMEOUT = -4,    /* a bounded device wait gave up (the wavefront and  */
                            /* resident kernels' waits, about one second each;   */
                            /* MC_WAVE_INJECT_TIMEOUT=1 or                       */
                            /* MC_RESIDENT_INJECT_TIMEOUT=1 in the environment   */
                            /* when a lattice is created makes its first wait    */
                            /* run out: a test hook)                             */
    MC_ERR_CONSTRAINT = -5, /* constrained run with M_L <= 0 (Table A2)          */
    MC_ERR_STATE = -6,      /* call not valid in the current state               */
    MC_ERR_IO = -7,         /* checkpoint file could not be read or written      */
    MC_ERR_CANCELLED = -8   /* the job was cancelled (mc_cancel)                  */
} mc_status;

typedef enum mc_precision { MC_FP32 = 0, MC_FP64 = 1 } mc_precision;

/* Boundary mode of one axis.  PERIODIC needs an even size (two-colouring).
 * OPEN drops bonds across the face.  PINNED is OPEN and, in addition, the
 * two end planes of that axis are never updated (fixed by the initial
 * state: e.g. a Bloch wall held by +z / -z end planes).  ANTIPERIODIC wraps
 * like PERIODIC (even size) but a bond across the face couples S_i to -S_j,
 * i.e. S(x + L) = -S(x): the wall setup of Sec. 3, which holds one wall. */
typedef enum mc_boundary { MC_PERIODIC = 0, MC_OPEN = 1, MC_PINNED = 2, MC_ANTIPERIODIC = 3 } mc_boundary;

/* Kernels of an FP32 lattice.  AUTO takes a row kernel for the colour
 * passes where the row layout applies (Lh = Lx/2 a power of two <= 64 or a
 * multiple of 64, Nc a multiple of 64) and the general kernel otherwise,
 * and walks the constrained pairs in site order (each pair led by the
 * member whose shuffled position is even); an all-periodic lattice with
 * Lx = 128 and no film tables whose rows fit the SMs' shared memory sweeps
 * resident when it runs alone (see RESIDENT).  GENERAL always takes the
 * general colour-pass kernel and the pairs in pair order.  ROW is AUTO
 * without the resident sweeps: the row kernels for every colour pass.
 * WAVE is ROW, except that on an all-periodic lattice with Lx = 128 and
 * Ly >= 16 (no film tables) the sweeps of each mc_sweep / mc_group_sweep
 * call run two at a time as single wavefront launches (red and black pass
 * fused, each spin read and written once per sweep; the lattice then holds
 * a second spin buffer, and an odd last sweep of a call runs as two row
 * passes).  RESIDENT is AUTO, named: an all-periodic lattice with Lx = 128
 * (no film tables) whose rows fit the SMs' shared memory (about 30 MB of
 * spins on 152 SMs, e.g. 128^3) sweeps, when it runs alone (mc_sweep, or a
 * group of that one lattice), held in shared memory: one cooperative launch
 * per run of up to 2048 unconstrained sweeps, one block per brick of rows,
 * the blocks waiting on their neighbours between colour passes and on all
 * blocks between sweeps (each wait bounded; a wait that runs out gives
 * MC_ERR_TIMEOUT).  A group made only of such lattices of at least 2^21
 * spins each (128^3 and larger) sweeps them resident one after another.
 * Constrained sweeps, calls of fewer than 3 sweeps and other groups take
 * the row kernels.  The colour passes of AUTO, GENERAL,
 * WAVE and RESIDENT agree up to FP32 rounding (the draws are keyed to the
 * same sites; the wavefront, resident and row kernels bit for bit) and the
 * two pair orders exactly; GENERAL, ROW, WAVE and RESIDENT exist to compare
 * them.  FP64 lattices always take the general kernel and pair order. */
typedef enum mc_kernel_path {
    MC_PATH_AUTO = 0, MC_PATH_GENERAL = 1, MC_PATH_ROW = 2, MC_PATH_WAVE = 3, MC_PATH_RESIDENT = 4
} mc_kernel_path;

/* Crystal structure (Sec. 2).  SC: the simple cubic lattice, sites at the
 * cells.  BCC / FCC: 2 / 4 simple cubic sub-lattices with basis (0,0,0),
 * (1/2,1/2,1/2) / (0,0,0), (1/2,1/2,0), (1/2,0,1/2), (0,1/2,1/2) of a cubic
 * cell; J couples nearest neighbours (8 / 12, other sub-lattices) and J2
 * next-nearest ones (6, the same sub-lattice one cell away).  HCP: 4 simple
 * tetragonal sub-lattices (0,0,0), (1/2,1/2,0), (1/2,1/6,1/2), (0,2/3,1/2)
 * of the orthohexagonal cell (a, sqrt(3) a, c), c/a = sqrt(8/3); J couples
 * the 12 nearest neighbours (two of them on the same sub-lattice, one cell
 * away along x); J2 must be 0.  dims count cells (even, all boundaries
 * PERIODIC).  Each sub-lattice is split red/black by cell parity and the
 * 2 nsub sub-sets are updated in turn: sub-lattice 0 red, 0 black, 1 red,
 * ...  Site order of spin arrays: i = s + nsub (x + Lx (y + Ly z)).
 * Constrained sweeps (Table A2) run one sub-set at a time as well, the pairs
 * shuffled within it, with the sub-lattice index in bits 4.. of the Philox
 * tag of its draws.  These lattices take no films, groups, serving,
 * profiles or autotuning (MC_ERR_ARG). */
typedef enum mc_lattice_type { MC_SC = 0, MC_BCC = 1, MC_FCC = 2, MC_HCP = 3 } mc_lattice_type;

typedef enum mc_init {
    MC_INIT_UNIFORM = 0, /* every spin along init_dir (default +z)             */
    MC_INIT_WALL = 1     /* +z for x < Lx/2, -z otherwise (Bloch wall start)    */
} mc_init;

typedef struct mc_lattice* mc_handle;
typedef struct mc_group* mc_group_handle;
typedef struct mc_server mc_server;

/* Full description of one lattice (mc_create_ex).  Zero-initialise and fill
 * what is needed; mc_desc_default() gives the documented defaults. */
typedef struct mc_desc {
    int dims[3];            /* Lx, Ly, Lz >= 1; Lx must be even                   */
    int boundary[3];        /* mc_boundary per axis                               */
    int precision;          /* mc_precision: FP32 spins (fixed-point sample sums, */
                            /* FP64 moments) or FP64                              */
    double J;               /* nearest-neighbour exchange                         */
    double K_u;             /* uniaxial anisotropy constant                       */
    double axis[3];         /* uniaxial easy axis (normalised by the library)     */
    double K_c;             /* cubic anisotropy constant (axes x, y, z)           */
    double H[3];            /* Zeeman field (energy units)                        */
    double T;               /* temperature, > 0                                   */
    uint64_t seed;          /* Philox key                                         */
    int theta0_deg;         /* initial cone half-angle, 1..180 (default 30)       */
    int adapt_in_measure;   /* 1: cone angle adapts in measurement sweeps too     */
    int init;               /* mc_init                                            */
    double init_dir[3];     /* direction for MC_INIT_UNIFORM (default +z)         */
    int ring_capacity;      /* per-sweep samples kept (default 4096)              */
    int sample_torque;      /* 1 (default): every sample also has the torque of  */
                            /* Sec. 3; 0: magnetisation and energies only, the   */
                            /* torque reads 0 (constrained samples always have it) */
    /* optional granular-film tables, host memory, copied at create:            */
    const uint8_t* bond_mask;   /* N entries or NULL; bit d set = bond present,   */
                                /* d = 0..5 for -x,+x,-y,+y,-z,+z; must be        */
                                /* symmetric (bond i->j iff j->i)                 */
    const int32_t* grain_id;    /* N entries or NULL: per-site easy axis index    */
    const double* grain_axis;   /* n_grains x 3 easy axes (normalised here)       */
    int n_grains;
    void* stream;           /* cudaStream_t to run on, or NULL for a library stream */
    int device;             /* CUDA device ordinal                                */
    int kernel_path;        /* mc_kernel_path (default MC_PATH_AUTO)              */
    int lattice;            /* mc_lattice_type (default MC_SC)                    */
    double J2;              /* bcc / fcc: next-nearest exchange (same sub-lattice) */
} mc_desc;

/* Ensemble averages over the measurement sweeps since the last reset
 * (Sec. 3).  Means are per sample; m is the normalised magnetisation of
 * one sample, energies and torques are per spin. */
typedef struct mc_observables {
    int64_t n_samples;
    int64_t sweeps_done;     /* sweeps run since create (both kinds)              */
    int theta_deg;           /* current cone half-angle                           */
    int error;               /* sticky device error (mc_status), 0 if none        */
    double accept_last;      /* acceptance rate of the last sweep                 */
    double m[3];             /* <m_a>                                             */
    double m2[3];            /* <m_a^2>                                           */
    double m_abs[3];         /* <|m_a|>                                           */
    double ml, ml2, ml4;     /* <|m|>, <|m|^2>, <|m|^4>                           */
    double e, e2;            /* <E/N>, <(E/N)^2>                                  */
    double e_parts[4];       /* <E_ex/N>, <E_u/N>, <E_c/N>, <E_Z/N>               */
    double torque[3];        /* <tau/N>, tau = sum_i S_i x (-dE_anis,Z/dS_i)      */
    double torque2[3];       /* <(tau_a/N)^2>                                     */
    double chi[4];           /* Eq. 6 in reduced units: N/T (<m_a^2> - <m_a>^2)   */
                             /* for a = l (|m|), x, y, z                          */
    double binder;           /* 1 - <|m|^4> / (3 <|m|^2>^2)                       */
} mc_observables;

/* One measurement sweep (the per-sweep time series). */
typedef struct mc_sample {
    int64_t sweep;           /* index of the sweep this sample closed             */
    int32_t theta_deg;       /* cone angle after this sweep's adaptation          */
    int32_t pad;
    int64_t accepted;        /* accepted single-spin moves (pairs count 2)        */
    double m[3];
    double e_parts[4];       /* per spin: exchange, uniaxial, cubic, Zeeman       */
    double torque[3];        /* per spin                                          */
} mc_sample;

/* ---------------------------------------------------------------- lattice */

/* Defaults: 16^3 periodic FP32, J = 1, all other couplings 0, axis z, T = 1,
 * seed 0, theta0 30, adapt_in_measure 1, uniform +z start, ring 4096,
 * torques sampled. */
MC_API void mc_desc_default(mc_desc* d);

/* Create a lattice (Eq. 2 parameters; Sec. 2).  dims: Lx, Ly, Lz, all
 * periodic; FP32 spins, fixed-point sample sums and FP64 moments; spins
 * start along +z.
 * Errors: MC_ERR_ARG (odd periodic size, T <= 0, |axis| = 0, ...),
 * MC_ERR_NOMEM, MC_ERR_CUDA.  *out is set only on MC_OK. */
MC_API int mc_create(const int dims[3], double J, double K_u, const double axis[3], double K_c,
                     const double H[3], double T, uint64_t seed, mc_handle* out);

/* Create a lattice from a full description (see mc_desc). */
MC_API int mc_create_ex(const mc_desc* d, mc_handle* out);

/* Free every device and host resource of the lattice.  NULL is ignored. */
MC_API int mc_destroy(mc_handle h);

/* Change T (> 0) or H for the following sweeps (Eq. 1, Eq. 2).  Ordered on
 * the lattice's stream after the sweeps already queued. */
MC_API int mc_set_temperature(mc_handle h, double T);
MC_API int mc_set_field(mc_handle h, const double H[3]);

/* Queue n_sweeps iterations of the parallel algorithm of Table A1: red pass,
 * black pass, then the cone angle moves one degree toward 50% acceptance.
 * measure != 0 takes one sample per sweep (fused into the black pass).
 * n_sweeps >= 0.  Asynchronous. */
MC_API int mc_sweep(mc_handle h, int n_sweeps, int measure);

/* Queue n_sweeps iterations of the parallel constrained algorithm of
 * Table A2 with the constraint direction e_C = (sin t cos p, sin t sin p,
 * cos t), t = theta_c_deg in [0, 180], p = phi_c_deg: M_L = sum S.e_C once
 * per iteration (exact, order-independent), shuffled same-colour pairs,
 * pair moves that keep the transverse magnetisation.  Not allowed with
 * pinned boundaries.  M_L <= 0 stops the run with MC_ERR_CONSTRAINT. */
MC_API int mc_constrained_sweep(mc_handle h, double theta_c_deg, double phi_c_deg, int n_sweeps,
                                int measure);

/* Wait for the lattice's queued work; returns the sticky device error. */
MC_API int mc_sync(mc_handle h);

/* Ensemble averages since the last mc_reset_stats (Sec. 3, Eq. 6).
 * Synchronises.  out: caller-owned. */
MC_API int mc_measure(mc_handle h, mc_observables* out);

/* Temperature scaling of the anisotropy by Eq. 4 (Sec. 3), from the mean
 * easy-axis anisotropy energy of the samples since the last mc_reset_stats
 * (standard sweeps, no constraint).  K_easy = mean anisotropy energy per
 * spin above its T = 0 value along the easy direction; K_0,hard = T = 0
 * energy per spin of the hard direction above the easy one.
 *   uniaxial (E_u = -K_u (S.e)^2, K_u > 0):  K_easy = <E_u/N> + K_u,
 *     K_0,hard = K_u,      out[0] = k_u = 1 - 3 K_easy / (2 K_0,hard);
 *   cubic (E_c = K_c q(S), K_c > 0: easy <100>, hard <111>, the long cube
 *     diagonal):  K_easy = <E_c/N>,  K_0,hard = K_c / 3,
 *                          out[1] = k_c = 1 - 5 K_easy / (3 K_0,hard).
 * Either is NaN when its constant is zero.  Synchronises.  out: caller-owned
 * double[2].  Errors: MC_ERR_ARG (null), MC_ERR_STATE (no samples). */
MC_API int mc_anisotropy_scaling(mc_handle h, double out[2]);

/* Slice-averaged profile <m_a(x)> = <(1/(Ly Lz)) sum_{y,z} S_a> for every
 * x-plane (Sec. 3, domain-wall profile), averaged over the profile samples
 * taken by mc_profile_sample.  axis: component a (0, 1, 2).  out: len >= Lx
 * doubles, caller-owned.  Synchronises. */
MC_API int mc_profile(mc_handle h, int component, double* out, int len);

/* Queue one profile sample of the current state (all three components). */
MC_API int mc_profile_sample(mc_handle h);

/* Queue one grain sample of a film lattice (one created with a grain table):
 * for every grain g, m_g = |sum_{i in g} S_i| / N_g, the magnetisation length
 * of the grain alone (Sec. 4: each grain contributes its own Bloch term to
 * Eq. 8, with weight N_g / N for columnar grains).  Asynchronous on the
 * lattice's stream.  Errors: MC_ERR_ARG (null handle, no grain table). */
MC_API int mc_grain_sample(mc_handle h);

/* <m_g> over the grain samples since create or the last mc_reset_stats, for
 * g = 0 .. n_grains - 1 (the ids of the grain table).  out: caller-owned,
 * len >= n_grains doubles; *n_samples (may be null) receives the number of
 * samples (0: out is all zero).  Synchronises.  Errors: MC_ERR_ARG (null
 * handle or out, no grain table, len too small). */
MC_API int mc_grain_magnetization(mc_handle h, double* out, int len, int64_t* n_samples);

/* Copy up to max of the most recent per-sweep samples (oldest first) into
 * out; *n receives the count.  Synchronises. */
MC_API int mc_samples(mc_handle h, mc_sample* out, int max, int* n);

/* Zero the accumulators, the sample ring, the profile sums and the grain
 * samples. */
MC_API int mc_reset_stats(mc_handle h);

/* Spins as FP64 host arrays of n = N sites (site order x + Lx(y + Ly z)).
 * mc_set_spins normalises nothing: pass unit vectors.  Synchronises. */
MC_API int mc_get_spins(mc_handle h, double* host_xyz, size_t n);
MC_API int mc_set_spins(mc_handle h, const double* host_xyz, size_t n);

/* Raw device-layout state (colour-split structure of arrays in the
 * lattice's precision): bytes = mc_state_bytes(h).  For fast transfer and
 * checkpointing; host memory, pinned or pageable. */
MC_API size_t mc_state_bytes(mc_handle h);
MC_API int mc_export_state(mc_handle h, void* host_buf, size_t bytes);
MC_API int mc_import_state(mc_handle h, const void* host_buf, size_t bytes);

/* Current cone angle and sweep counter (synchronises). */
MC_API int mc_get_theta(mc_handle h, int* theta_deg, int64_t* sweeps_done);

/* Checkpoint: description, counters, cone angle, accumulators, sample ring
 * and spins.  The generator is counter-based, so a resumed run is bit-exact
 * with an uninterrupted one.  mc_load creates a new handle (stream NULL). */
MC_API int mc_save(mc_handle h, const char* path);
MC_API int mc_load(const char* path, mc_handle* out);

/* ------------------------------------------------------------ batching */

/* A group advances many independent lattices (same precision, same device)
 * with one kernel launch per colour pass, replayed from a captured CUDA
 * graph.  The lattices keep their own state; mc_measure etc. work on each.
 * The group runs on the first lattice's stream.  The caller keeps the
 * handles alive until mc_group_destroy. */
MC_API int mc_group_create(const mc_handle* lattices, int n, mc_group_handle* out);
MC_API int mc_group_destroy(mc_group_handle g);

/* n_sweeps of Table A1 for every lattice of the group. */
MC_API int mc_group_sweep(mc_group_handle g, int n_sweeps, int measure);

/* n_sweeps of Table A2 for every lattice of the group; lattice i uses the
 * constraint direction (theta_c_deg[i], phi_c_deg[i]). */
MC_API int mc_group_constrained_sweep(mc_group_handle g, const double* theta_c_deg,
                                      const double* phi_c_deg, int n_sweeps, int measure);

/* Time the launches of the group: the next n_sweeps sweeps of Table A1
 * record CUDA events around every launch that moves spins (a colour pass,
 * which updates one colour of every lattice of its kernel, or a wavefront
 * launch, which sweeps its lattices once); *avg_ms receives the mean
 * duration of one launch and *launches the number timed.  Synchronises. */
MC_API int mc_group_time_passes(mc_group_handle g, int n_sweeps, int measure, double* avg_ms,
                                int* launches);

/* The same, by kind: avg_ms[0] / launches[0] for the wavefront launches
 * (one sweep of the lattices that take them), [1] for the colour passes of
 * the row and general kernels, [2] for the pair passes of Table A2, [3] for
 * the resident launches (MC_PATH_RESIDENT: each runs up to 2048 of the
 * n_sweeps sweeps, so a launch's time per sweep is avg_ms[3] times
 * launches[3] over n_sweeps).  With
 * constrained != 0 the sweeps are constrained sweeps about each lattice's
 * last constraint direction (MC_ERR_STATE before any constrained sweep of
 * the group).  A kind with no launch reads 0 ms.  Measurement support
 * around the paper's method; the paper has no counterpart.  Synchronises. */
MC_API int mc_group_time_kernels(mc_group_handle g, int n_sweeps, int measure, int constrained, double avg_ms[4],
                                 int launches[4]);

/* Ensemble averages of every lattice of the group (Sec. 3, Eq. 6), as
 * mc_measure gives them, read with one wait on the group stream instead of
 * one per lattice.  out: caller-owned array of n = the group's size, in the
 * order of the handles given to mc_group_create.  The first call allocates a
 * pinned host staging area of n device-state records, freed with the group.
 * Synchronises.  Errors: MC_ERR_ARG (null, n not the group's size),
 * MC_ERR_CUDA; the first member's sticky device error after every entry is
 * filled in. */
MC_API int mc_group_measure(mc_group_handle g, mc_observables* out, int n);

MC_API int mc_group_sync(mc_group_handle g);

/* ------------------------------------------------------------- autotuner */

/* Launch-shape autotuning of the batched sweeps (the block and tile shapes of
 * a persistent launch).  Candidates, in the order of the report's arrays:
 *   row:   FP32 row kernel, minimum resident blocks per SM (so registers per
 *          thread): all-periodic lattices {3, 2}, boundaries and films {2, 3};
 *          a lattice swept resident (MC_PATH_RESIDENT): threads per block
 *          {512, 640};
 *   field: constrained neighbour-field kernel, tiles per grid-stride step
 *          {4, 8, 2};
 *   pair:  constrained pair pass, the same {4, 8, 2}, then 4 tiles per step
 *          with more resident warps (site order: blocks of 128 threads, five
 *          per SM; pair order: one more block of 256 threads per SM).
 * what: MC_TUNE_SWEEP tunes the row kernel on sweeps of Table A1,
 * MC_TUNE_CONSTRAINED the field and pair kernels on sweeps of Table A2 (with
 * each lattice's present constraint direction; a lattice that has not run a
 * constrained sweep yet gets its packed copy here), both or-ed together.
 * Each candidate runs 1 + sweeps sweeps, the last `sweeps` timed with CUDA
 * events; knobs are tuned one after the other, each at the best choice of the
 * ones before.  Another candidate replaces a knob's first (its default) only if
 * it is more than 1% faster.  The lattices' spins and device state (theta, sweep counter,
 * accumulators) are saved first and restored after, so the chains continue as
 * if no tuning had run; the chosen shapes apply to later sweeps (captured
 * graphs are rebuilt).  Synchronises.  out (may be null) receives the choices
 * and the mean ms per sweep of every candidate tried (0 where not tried).
 * Errors: MC_ERR_ARG (null group, sweeps < 1, what empty), MC_ERR_NOMEM (no
 * room for the saved state), MC_ERR_CUDA. */
#define MC_TUNE_SWEEP 1
#define MC_TUNE_CONSTRAINED 2
typedef struct mc_tune_report {
    int row, field, pair;          /* chosen candidate of each knob */
    int pad;
    double row_ms[4], field_ms[4], pair_ms[4];
} mc_tune_report;
MC_API int mc_group_autotune(mc_group_handle g, int sweeps, int what, mc_tune_report* out);

/* The same for one lattice swept alone (mc_sweep, mc_constrained_sweep).
 * Crystal lattices (bcc, fcc, hcp) have no tunable shape: MC_ERR_ARG. */
MC_API int mc_autotune(mc_handle h, int sweeps, int what, mc_tune_report* out);

/* Set the group's launch shapes directly (candidate indices as in the
 * report: row 0..1, field 0..2, pair 0..3), e.g. from an earlier tuning.
 * No result depends on them.  Errors: MC_ERR_ARG (null group, index out of
 * range). */
MC_API int mc_group_set_shapes(mc_group_handle g, int row, int field, int pair);

/* ------------------------------------------------------------- serving */

typedef struct mc_server_desc {
    int device;
    size_t memory_budget;    /* bytes of device memory the server may hold; 0 =  */
                             /* 90% of free memory at create                      */
    int max_resident;        /* lattices resident at once (default 256)           */
    int max_epoch_sweeps;    /* sweeps per batched epoch (default 50)             */
} mc_server_desc;

typedef enum mc_job_kind { MC_JOB_SWEEP = 0, MC_JOB_CONSTRAINED = 1 } mc_job_kind;

typedef struct mc_job {
    mc_desc lattice;         /* film tables are copied at submit                  */
    int kind;                /* mc_job_kind                                       */
    double theta_c_deg, phi_c_deg;  /* constrained jobs                           */
    int n_equilibrate;       /* sweeps before measuring                           */
    int n_measure;           /* measurement sweeps                                */
} mc_job;

typedef struct mc_result {
    mc_observables obs;
    double t_submit, t_admit, t_finish;  /* seconds on the server's clock         */
    int status;              /* MC_OK or the job's error                          */
} mc_result;

MC_API int mc_server_create(const mc_server_desc* d, mc_server** out);
MC_API int mc_server_destroy(mc_server* s);

/* Queue a job; non-blocking.  MC_ERR_NOMEM if the job can never fit in the
 * server's memory budget, MC_ERR_ARG for an invalid description. */
MC_API int mc_submit(mc_server* s, const mc_job* job, uint64_t* job_id);

/* MC_PENDING while queued or running; MC_OK and *out once finished (the
 * result stays available); MC_ERR_ARG for an unknown id. */
MC_API int mc_poll(mc_server* s, uint64_t job_id, mc_result* out);

/* Cancel a job.  A queued job is dropped at once; a resident job is retired
 * at the end of the current epoch (its lattice destroyed, its memory
 * returned).  Its result then reads status MC_ERR_CANCELLED.  MC_ERR_STATE
 * if the job has already finished, MC_ERR_ARG for an unknown id. */
MC_API int mc_cancel(mc_server* s, uint64_t job_id);

/* Drop the record of a finished job (its result, its id), so that a server
 * fed an endless stream of requests keeps only the jobs still in flight.
 * Poll the result first: afterwards the id is unknown (MC_ERR_ARG).
 * MC_ERR_STATE while the job is queued or running.  Serving bookkeeping
 * around the paper's method; the paper has no counterpart. */
MC_API int mc_forget(mc_server* s, uint64_t job_id);

/* Current server clock (seconds), jobs queued / resident, bytes in use. */
MC_API int mc_server_stats(mc_server* s, double* now, int* queued, int* resident, size_t* bytes);

/* ------------------------------------------------------------ slabs */

/* One lattice split along z into slabs, for devices that each hold a part
 * (the domain decomposition behind the paper's multi-GPU projection, Sec. 2:
 * without dipolar coupling the parts exchange only their boundary planes).
 * A slab holds global planes [z0, z0 + nz) of the lattice described by d
 * (FP32, simple cubic, periodic in z, no film tables; x and y as in d) plus
 * one halo plane below and above: its spin arrays (mc_set_spins /
 * mc_get_spins) are Lx x Ly x (nz + 2) sites, local plane 0 = global plane
 * z0 - 1, plane nz + 1 = global plane z0 + nz (mod Lz).  The local lattice
 * must have the FP32 row layout (Lx/2 a power of two <= 64 or a multiple of
 * 64; Lx Ly (nz + 2) / 2 a multiple of 64), else MC_ERR_ARG.  Draws are keyed
 * by global site index and colour, the halo planes never move and are left
 * out of the sample, so a split chain equals the unsplit chain bit for bit.
 * A slab is not swept by mc_sweep or in a group (MC_ERR_STATE / MC_ERR_ARG),
 * nor saved by mc_save or profiled by mc_profile_sample (its planes include
 * the halo copies);
 * one sweep of Table A1 is, on every slab in turn:
 *   mc_slab_pass(colour 0); exchange colour 0's boundary planes;
 *   mc_slab_pass(colour 1, measure); exchange colour 1's boundary planes;
 *   mc_slab_export; sum the exported words over all slabs; mc_slab_close.
 * The caller moves planes and sums words between devices (e.g. with NCCL
 * send/recv and all-reduce on the device addresses these calls return);
 * mc_slab_sweep does it all for slabs on one device.  mc_measure and
 * mc_samples of every slab then give the whole lattice's observables. */
MC_API int mc_slab_create(const mc_desc* d, int z0, int nz, mc_handle* out);

/* The slab's planes: z0, nz and the lattice's Lz (any may be NULL).
 * MC_ERR_ARG if h is not a slab. */
MC_API int mc_slab_info(mc_handle h, int* z0, int* nz, int* Lz);

/* Queue one colour pass (colour 0 red, 1 black: the lattice's global
 * colours) over the slab's own planes; measure (black pass only) adds the
 * sample sums of the own planes.  Does not close the sweep. */
MC_API int mc_slab_pass(mc_handle h, int colour, int measure);

/* Device addresses of one plane of the given colour: ptrs[a] = component a
 * (a = 0, 1, 2), *count sites of that colour per plane (FP32 each).  which:
 * 0 the first own plane (sent to the slab below), 1 the last own plane
 * (sent above), 2 the lower halo plane (received from below), 3 the upper
 * halo plane (received from above).  Owned by the slab; valid until
 * mc_destroy. */
MC_API int mc_slab_plane(mc_handle h, int colour, int which, void* ptrs[3], size_t* count);

/* Queue the export of the sweep's counts: MC_SLAB_WORDS int64 words at the
 * device address *counts (accepted moves, movable sites, own sites, then
 * the fixed-point sample sums), cleared from the slab.  Sum them over all
 * slabs of the lattice, elementwise, in place, before mc_slab_close. */
#define MC_SLAB_WORDS 16
MC_API int mc_slab_export(mc_handle h, int64_t** counts);

/* Queue the end of the sweep from the summed words: the cone rule of Table
 * A1 with the total accepted count, the sample (measure != 0) with the total
 * sums, the sweep counter. */
MC_API int mc_slab_close(mc_handle h, int measure);

/* n_sweeps sweeps of the n slabs of one lattice held on one device and one
 * stream (slabs[0] starts at plane 0, each slab ends where the next begins,
 * the last ends at Lz): passes, halo copies (cudaMemcpyAsync device to
 * device), export, sum and close as above.  n <= 64. */
MC_API int mc_slab_sweep(const mc_handle* slabs, int n, int n_sweeps, int measure);

/* ------------------------------------------------------ no allocation */

/* FP32 sweeps of Table A1 on a lattice whose spin memory the caller owns,
 * for callers that cannot allocate device memory: code that runs while a
 * framework's memory pool owns the whole device, inside another library's
 * loop that forbids allocation (and the synchronisation cudaMalloc implies),
 * or in a process whose allocator is not the CUDA runtime's.  The paper has
 * no counterpart; this is a deployment variant of mc_sweep.
 *
 * The entry point allocates nothing: no cudaMalloc, no cudaFree, no stream,
 * no library routine that allocates.  The scratch the sweep kernels need
 * (lattice descriptor with its counters and sums, launch tables, cone table,
 * sample ring) is one static 32 KiB device array inside libmc, reserved on
 * every GPU that loads the library until the process exits.  Each call
 * looks up the array's device address in the current device's context (a
 * lookup that allocates nothing); the first call on a device also loads
 * libmc's kernels there, so make that first call before any stream
 * capture.  Every call rewrites the whole scratch
 * and clears its counters; calls that overlap on the GPU (on different
 * streams, or from different threads) race on it.
 *
 * spins     device memory, FP32, colour-split layout of mc_export_state:
 *           6 * stride floats, stride = N/2 rounded up to a multiple of 64,
 *           component a of colour c at spins[(3c + a) stride + q]; updated
 *           in place
 * dims...   a periodic lattice as for mc_create (every size even)
 * first_sweep  sweep counter of the chain (0 for a new chain; a continuing
 *           chain passes the previous first_sweep + n_sweeps)
 * theta_deg host in/out: cone half-angle (1..180) before and after
 * samples   NULL, or device memory for n_sweeps samples of 14 doubles each
 *           (sweep, theta, accepted, m[3], energies[4], torque[3], 0); with
 *           samples every sweep is a measurement sweep
 * stream    cudaStream_t (NULL = default stream); the call synchronises it
 *           before returning (to read theta back)
 * Errors: MC_ERR_ARG for invalid sizes or parameters, and for n_sweeps > 256
 * with samples (the scratch holds 256 samples per call); MC_ERR_CUDA. */
MC_API int mc_sweep_noalloc(float* spins, const int dims[3], double J, double K_u, const double axis[3],
                            double K_c, const double H[3], double T, uint64_t seed, int64_t first_sweep,
                            int n_sweeps, int* theta_deg, double* samples, void* stream);

/* -------------------------------------------------------------- misc */

MC_API const char* mc_last_error(void);
MC_API const char* mc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MC_H */
