/*
 * pic.h -- C ABI of the GB300 (sm_103a) library for the 1D electrostatic
 * electron Particle-in-Cell step of Markidis & Lapenta, "Development and
 * performance analysis of a UPC Particle-in-Cell code" (PGAS10).
 *
 * The method (Sec. 2): N electrons on a periodic line of length L cut into
 * NG cells of width dx = L/NG, nodes at the cell centres (g + 1/2) dx,
 * immobile neutralising ions of density rho_ion, charge-to-mass ratio qm < 0,
 * time step dt.  One step advances the state (x^n, v^{n-1/2}, E^n):
 *   gather   E_p = linear interpolation of E^n at x^n       (Sec. 2.3)
 *   kick     v^{n+1/2} = v^{n-1/2} + qm E_p dt              (Sec. 2.1, Eq. 3)
 *   drift    x^{n+1} = x^n + v^{n+1/2} dt, wrapped to [0,L) (Sec. 2.1, Eq. 2)
 *   deposit  linear weighting of x^{n+1} onto the nodes     (Sec. 2.3)
 *   solve    Phi_{g+1} - 2 Phi_g + Phi_{g-1} = -rho_g dx^2  (Sec. 2.2, Eq. 6)
 *   field    E_g = -(Phi_{g+1} - Phi_{g-1}) / (2 dx)        (Sec. 2.2, Eq. 7)
 *
 * Precision (PIC_FP32_FIXED, the default): positions and velocities are
 * float32; the deposit is exact integer arithmetic on 2^-24 fractions of a
 * particle (below), so the density is the same integer for any launch shape
 * or particle order; the field solve and all diagnostics are float64.
 *
 * Cell units.  In the float32 modes the device keeps each position as its
 * cell coordinate u = x NG / L in [0, NG) (node g at u = g + 1/2), so the box
 * is exactly [0, NG) and the drift is u += v (float)(dt NG/L).  Positions
 * cross the ABI in physical units and are converted on the device, each
 * conversion one rounding of a float64 product:
 *   in   u = (float)((double)x (NG/L)), a u rounding to NG is 0;
 *   out  x = (float)((double)u (L/NG)), at most the float below (float)L.
 * pic_get_cells / pic_set_cells exchange u itself (exact checkpoints).
 *
 * Fixed-point deposit (the library's exact form of the Sec. 2.3 weighting).
 * With float operations rounded to nearest:
 *   s = u - 0.5f, i = floorf(s), f = s - i, W = trunc(f * 2^24);
 *   rho_q[(i+1) mod NG] += W,  rho_q[i mod NG] += 2^24 - W.
 * The float64 density is rho_g = rho_ion - rho_ion (NG/N) rho_q[g] 2^-24.
 *
 * Ownership.  The caller owns all device memory: it allocates one workspace
 * of pic_workspace_size() bytes (any allocator; 256-byte alignment) and the
 * library carves every device array out of it.  The library allocates no
 * device memory.  It keeps a small host-side handle (pic_run) and CUDA graphs.
 * All work is enqueued on the caller's stream; calls return before the GPU
 * finishes, except those documented as synchronising.
 *
 * Errors.  Every int-returning call returns PIC_OK (0) or a negative code.
 * Kernels never trap: a particle with a non-finite or out-of-range position
 * sets a device error word, which the synchronising calls (pic_sync,
 * pic_diagnostics, pic_get_state, pic_get_field) report as PIC_EDEVICE.
 *
 * Threading.  Calls on one run are not thread-safe; different runs are.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_ABI_VERSION 1

/* Return codes. */
#define PIC_OK 0
#define PIC_EINVAL (-1)   /* bad argument or parameter                       */
#define PIC_ENOMEM (-2)   /* workspace too small / pool budget exhausted      */
#define PIC_ECUDA (-3)    /* a CUDA runtime call failed                       */
#define PIC_ETIMEOUT (-4) /* reserved: no call waits on the device with a
                             time limit (every device wait is a hardware
                             block or cluster barrier)                      */
#define PIC_EDEVICE (-5)  /* a kernel flagged bad particle data                */
#define PIC_ESTATE (-6)   /* call out of order (e.g. push before init)         */

/* Precision modes. */
#define PIC_FP32_FIXED 0  /* float32 push, int64 fixed-point deposit (default) */
#define PIC_FP32_ATOMIC 1 /* float32 push, float32 atomic deposit              */
#define PIC_FP64 2        /* float64 push, float64 atomic deposit              */

/* Deposit-kernel variants of the fused push (PIC_FP32_FIXED only); all give
 * the same integers.  The values 3, 4 and 7 are not variants (PIC_EINVAL). */
#define PIC_DEPOSIT_AUTO 0   /* chosen by the library                        */
#define PIC_DEPOSIT_ATOMIC 1 /* two shared-memory atomics per particle       */
#define PIC_DEPOSIT_MATCH 2  /* warp groups of equal cell (match + reduce)   */
#define PIC_DEPOSIT_QUAD 5         /* runs within a thread's 4 particles,
                                      two atomics per run                  */
#define PIC_DEPOSIT_PAIR 6         /* QUAD with two open runs per thread, so
                                      particles of two interleaved cells (two
                                      beams before a sort) still combine    */
#define PIC_DEPOSIT_QUAD8 8        /* QUAD over a thread's 8 consecutive
                                      particles, moved by 32-byte vector
                                      loads and stores (unroll: 8-particle
                                      groups per thread per iteration, 1, 2) */
#define PIC_DEPOSIT_PAIR8 9        /* PAIR over 8 consecutive particles, the
                                      same loads and stores as QUAD8        */

/* Field solvers (pic_params.field_solver).  Both solve the Eq. 6 system with
 * Phi_0 = 0 (the gauge the paper pins).
 *   EXACT  the converged solution, by exact prefix sums (default);
 *   CG     the paper's solver (Sec. 2.2, Sec. 3.3, Appendix A): matrix-free
 *          conjugate gradient from Phi = 0, a fixed number of iterations
 *          (the paper forces 150), float64, unconverged field included.
 *          Single runs only (the pool rejects it with PIC_EINVAL). */
/* Particle shapes (pic_params.shape): how charge goes to the grid and the
 * field comes back (Sec. 2.3 and Sec. 2), nodes at the cell centres.
 *   CIC  the two-cell linear weighting of Sec. 2.3 and the listing (default);
 *   NGP  nearest grid point: the cell the particle belongs to, floor(x NG/L)
 *        in float32, takes its whole charge and gives its field (Sec. 2: a
 *        cell's density is the count of its particles).  PIC_FP32_FIXED only; single
 *        runs only (the pool rejects it). */
#define PIC_SHAPE_CIC 0
#define PIC_SHAPE_NGP 1

#define PIC_SOLVER_EXACT 0
#define PIC_SOLVER_CG 1
#define PIC_CG_DEFAULT_ITERATIONS 150

#define PIC_NCELL_MAX 8192  /* largest NG (the per-block density tile)       */
#define PIC_NMODES 8        /* Fourier modes recorded per step               */

/* Parameters of one run (Sec. 2; names follow the paper's symbols). */
typedef struct pic_params {
    int64_t npart;         /* N, particles (>= 1)                             */
    int32_t ncell;         /* NG, cells (1 .. PIC_NCELL_MAX)                   */
    int32_t precision;     /* PIC_FP32_FIXED | PIC_FP32_ATOMIC | PIC_FP64      */
    double length;         /* L > 0                                           */
    double dt;             /* time step > 0                                   */
    double qm;             /* charge-to-mass ratio, < 0 (electrons: -1)        */
    double rho_ion;        /* ion background density > 0 (paper: 1)            */
    int32_t sort_interval; /* counting sort by cell every S steps (0 = never)  */
    int32_t history;       /* rows of the device diagnostics ring (>= 1)       */
    int32_t deposit_variant; /* PIC_DEPOSIT_*                                 */
    int32_t block_size;    /* threads per block of the fused push (0 = auto;
                              at most 512 in PIC_FP32_FIXED, else 1024)       */
    int32_t blocks_per_sm; /* resident blocks per SM of the fused push (0=auto)*/
    int32_t unroll;        /* float4 groups per thread per iteration of the
                              fused push: 1, 2, 4 (0 = auto)                 */
    int32_t field_solver;  /* PIC_SOLVER_EXACT | PIC_SOLVER_CG                 */
    int32_t cg_iterations; /* PIC_SOLVER_CG: iterations per solve, run to the
                              end whether converged or not (0 = 150, the
                              paper's fixed count; at most 100000)           */
    int32_t shape;         /* PIC_SHAPE_CIC | PIC_SHAPE_NGP                    */
    int32_t reserved;      /* must be 0                                       */
} pic_params;

/* One row of the per-step diagnostics (all float64 on the device). */
typedef struct pic_diag_row {
    int64_t step;          /* n                                               */
    double kinetic;        /* KE^n = (1/2) m sum_p v^{n-1/2} v^{n+1/2};  NaN
                              until the push of step n has run                 */
    double momentum;       /* m sum_p v^{n+1/2} (NaN likewise)                 */
    double field;          /* (1/2) dx sum_g (E^n_g)^2                          */
    double charge;         /* dx sum_g rho^n_g (0 for a neutral box)           */
    int64_t charge_q;      /* sum_g rho_q^n (= N 2^24 exactly in FIXED mode)    */
    double mode[PIC_NMODES]; /* 2 |(1/NG) sum_g E^n_g e^{-2 pi i m g/NG}|,
                                m = 1..8                                       */
} pic_diag_row;

typedef struct pic_run pic_run;

/* Library ABI version (PIC_ABI_VERSION). */
int pic_version(void);

/* Static text for a return code. */
const char *pic_strerror(int code);

/* Bytes of device workspace a run with parameters *p needs.
 * Returns PIC_EINVAL for invalid parameters. */
int pic_workspace_size(const pic_params *p, size_t *bytes);

/* Create a run on the current CUDA device.  workspace: caller-owned device
 * memory of at least pic_workspace_size() bytes, 256-byte aligned, kept alive
 * until pic_destroy.  stream: a cudaStream_t (NULL = legacy default stream).
 * Validates parameters (PIC_EINVAL), reads the device's SM count and picks the
 * launch shape.  Enqueues nothing. */
int pic_create(const pic_params *p, void *workspace, size_t workspace_bytes,
               void *stream, pic_run **out);

/* Release the host handle and its CUDA graphs (not the workspace). */
void pic_destroy(pic_run *run);

/* Load the initial state and make E^0 ready (Sec. 2, the initial set-up;
 * Appendix A).  x0, v0: host arrays of N values in the run's precision
 * (float for the FP32 modes, double for PIC_FP64); v0 is v^{-1/2}.  Positions
 * must lie in [0, L).  Copies them to the device, deposits rho^0, solves Phi^0
 * and E^0 and resets the step counter to 0.  Synchronises the stream (the host
 * arrays may be reused on return).  PIC_EINVAL for positions outside [0, L)
 * (checked on the device after the upload; the run then holds no usable
 * state, and calls other than pic_init / pic_set_state return PIC_ESTATE). */
int pic_init(pic_run *run, const void *x0, const void *v0);

/* Charge deposit (Sec. 2.3) of the current positions into the density
 * accumulator, which it zeroes first.  Asynchronous. */
int pic_deposit(pic_run *run);

/* Field solve (Sec. 2.2, Eqs. 6-7) of the accumulated density: rho, Phi
 * (Phi_0 = 0), E in float64 and the float32 copy used by the gather; records
 * field energy and modes for the current step and clears the accumulator.
 * Asynchronous. */
int pic_solve_field(pic_run *run);

/* Fused gather, kick, drift, wrap and deposit of x^{n+1} (Sec. 2.1 Eqs. 2-3,
 * Sec. 2.3) for all particles; rho_q then holds the fixed-point density of
 * x^{n+1}.  Follow it with pic_solve_field to finish the step.  Asynchronous. */
int pic_push(pic_run *run);

/* Counting sort of the particles by cell (stable: particles of one cell keep
 * their order).  Changes no physical quantity.  Asynchronous. */
int pic_sort(pic_run *run);

/* n whole steps: [sort if due] + push + solve, replayed from CUDA graphs.
 * A step n with n % S == 0 (S = sort_interval > 0, n > 0) sorts first.
 * Asynchronous. */
int pic_step_n(pic_run *run, int64_t n);

/* Wait for the stream, then report the device error word (PIC_EDEVICE). */
int pic_sync(pic_run *run);

/* The counting sort by cell of pic_sort, for callers that cannot allocate
 * device memory.  The paper has no counterpart; this is a service of the
 * library.  Some callers cannot hand the library a workspace: a framework
 * whose own caching allocator owns all of the device memory and takes no
 * outside allocations, a process held to a fixed memory reservation, or
 * latency-critical code that cannot pay for the device-wide synchronisation a
 * cudaMalloc brings.  This entry point allocates nothing: its scratch (cell
 * counts, offsets, cell bases, an error word) lives in one device array of
 * PIC_SORT_NOALLOC_SCRATCH bytes inside the library, which every GPU that
 * loads the library keeps until the process exits.
 * x, v: n float32 positions and velocities (device memory); x_out, v_out:
 * n float32 each (device memory), receiving the particles ordered by cell
 * trunc(x c), c = (float)(NG/L), clamped to [0, NG-1] (NaN to cell 0),
 * particles of one cell in their input order.  x must be 16-byte aligned
 * (its cells are counted in float4 groups; a tensor slice at an odd element
 * offset is not), v, x_out and v_out 4-byte aligned; neither output may
 * overlap the other output or an input.  Limits: 1 <= n <= 2^32 - 1,
 * 1 <= ncell <= PIC_NCELL_MAX, L finite and > 0.  Any violation returns
 * PIC_EINVAL from checks on the host, before anything is enqueued; larger n
 * only uses fewer, longer chunks to keep the tables inside the array.
 * Enqueued on `stream`, asynchronous; the call reports no device-side error
 * (its one device check, on the scatter's destination index, can fail only
 * if another writer changes x while the sort runs).  The first call on a
 * device looks up the array's device address with that device current: make
 * it before any stream capture.  That address belongs to the device's primary
 * context and does not survive cudaDeviceReset: do not call this entry point
 * again in a process after a reset.  Every call shares the array and leaves
 * its contents behind (each call rewrites its tables in full and clears the
 * error word first); calls whose work overlaps on the GPU race on it. */
#define PIC_SORT_NOALLOC_SCRATCH (4u << 20)
int pic_sort_noalloc(const float *x, const float *v, float *x_out, float *v_out, int64_t n,
                     int32_t ncell, double length, void *stream);

/* Copy the diagnostics rows of steps [first, first + count) (each must still
 * be in the history ring) to rows[] on the host.  Synchronises. */
int pic_diagnostics(pic_run *run, int64_t first, int32_t count,
                    pic_diag_row *rows);

/* Current step number n (host-side count of completed steps). */
int64_t pic_step_count(const pic_run *run);

/* Copy x^n, v^{n-1/2} (N values each, run precision) to host arrays, in the
 * current particle order; float32 positions are converted from cell units
 * (above) in the run's idle particle buffer.  Synchronises. */
int pic_get_state(pic_run *run, void *x, void *v);

/* Replace x, v with host arrays (a checkpoint restore) and set the step
 * counter to `step`; re-deposits and re-solves like pic_init. Synchronises. */
int pic_set_state(pic_run *run, const void *x, const void *v, int64_t step);

/* The float32 modes' state exactly as the device holds it: u^n (cell
 * coordinates, N float) and v^{n-1/2} (N float), in the current particle
 * order.  pic_set_cells restores such a state (u must lie in [0, NG), else
 * PIC_EINVAL as for pic_init) and sets the step counter; together they make
 * a checkpoint that continues bit for bit.  PIC_EINVAL for PIC_FP64 runs.
 * Synchronise. */
int pic_get_cells(pic_run *run, float *u, void *v);
int pic_set_cells(pic_run *run, const float *u, const void *v, int64_t step);

/* Copy the grid of the last solve to host arrays (any may be NULL):
 * rho[NG], phi[NG], E[NG] float64 and rho_q[NG] (the fixed-point sums that
 * solve consumed; FIXED mode only, else zeros).  Synchronises. */
int pic_get_field(pic_run *run, double *rho, double *phi, double *E,
                  int64_t *rho_q);

/* Phase-space histogram f(x, v) of the current particles (the (x, v)
 * snapshots of the Sec. 4 two-stream test, Fig. 1): counts[iv * nx + ix] (host,
 * nx * nv uint32) of the particles with ix = min(nx - 1, trunc(p * sx)) and
 * iv = floor((v - vmin) * (nv/(vmax - vmin))), the scale factors, the
 * difference and the products in float32, where p is the stored position:
 * the cell coordinate u with sx = nx/NG in the float32 modes, x with
 * sx = nx/L in PIC_FP64.  Particles with iv outside [0, nv) are not counted.
 * nx * nv <= PIC_PHASE_MAX_BINS, vmax > vmin, else PIC_EINVAL.  Synchronises. */
#define PIC_PHASE_MAX_BINS 16384
int pic_phase_space(pic_run *run, int32_t nx, int32_t nv, double vmin, double vmax,
                    uint32_t *counts);

/* Device pointers of the current particle arrays (they alternate after each
 * sort; positions in cell units in the float32 modes) and of the float32
 * field used by the gather. */
int pic_device_arrays(pic_run *run, void **x, void **v, void **E32);

/* The launch shape the run uses for its fused push (any pointer may be
 * NULL): grid, threads per block, deposit variant (15: the NGP shape's
 * kernel), float4 groups per thread per iteration. */
int pic_launch_shape(const pic_run *run, int32_t *grid, int32_t *block,
                     int32_t *variant, int32_t *unroll);

/* Device-side initial loading of a two-stream plasma (Sec. 2, the initial set-up;
 * Appendix A; the Sec. 4 beams).  Particle j of N:
 *   x = (j + 1/2) L/N - sum_m (eps_m/k_m) sin(k_m x0 + phase_m), k_m = 2 pi m/L,
 *       folded into [0, L), float32 (a value rounding to L is 0);
 *   v = s_j v0 + vth sqrt(-2 ln u1) cos(2 pi u2), s_j = +1 (j even) / -1 (odd),
 *   u1 = (top24(z_{2j+1}) + 1) 2^-24, u2 = top24(z_{2j+2}) 2^-24, z_k the k-th
 *   output of SplitMix64 seeded with `seed`. */
#define PIC_LOAD_MAX_MODES 8
typedef struct pic_loading {
    double v0;               /* beam speed (0: one Maxwellian)                 */
    double vth;              /* thermal spread                                 */
    uint64_t seed;           /* SplitMix64 seed                                */
    int32_t nmodes;          /* perturbed modes (0 .. PIC_LOAD_MAX_MODES)       */
    int32_t reserved;        /* must be 0                                      */
    int32_t mode[PIC_LOAD_MAX_MODES];   /* m >= 1                              */
    double eps[PIC_LOAD_MAX_MODES];     /* density amplitude of mode m         */
    double phase[PIC_LOAD_MAX_MODES];   /* phase of mode m                     */
} pic_loading;

/* Fill caller-owned device arrays x[n], v[n] (float32, 4-byte aligned) on
 * `stream`.  Asynchronous. */
int pic_load_two_stream(const pic_loading *ld, int64_t n, double length, void *x, void *v,
                        void *stream);

/* pic_init with the state generated on the device by pic_load_two_stream. */
int pic_init_loaded(pic_run *run, const pic_loading *ld);

/* Set the launch shape of the fused push (deposit variant, block size, unroll,
 * resident blocks per SM; 0 keeps the current value / picks the default).
 * Drops the captured graphs.  PIC_EINVAL for a shape the kernel cannot run. */
int pic_set_launch(pic_run *run, int32_t variant, int32_t block, int32_t unroll,
                   int32_t blocks_per_sm);

/* One timed candidate of pic_autotune. */
typedef struct pic_tune_entry {
    int32_t variant, block, unroll, grid;
    float ms;                 /* mean CUDA-event time of one fused push      */
} pic_tune_entry;

/* Autotune the fused push (PIC_FP32_FIXED): time every candidate shape
 * (deposit variant x block size x unroll) on a copy of the current particles
 * (the sort buffers and a scratch density accumulator; the run's state is
 * untouched), pushed with the current field: `reps` pushes of the copy as it
 * is, or, when the run sorts every S steps, min(S, 64) pushes of a freshly
 * sorted copy (one sort period); adopt the one with the smallest mean push
 * time.  The order of a sorting run settles after its first sorts (within a
 * cell, particles keep the order of the cells they came from, so of their
 * velocities), and the fastest shape changes with it: tune after those.
 * Writes up to
 * max_results entries to results (may be NULL) and their count to *nresults.
 * Synchronises.  PIC_ESTATE before pic_init or between pic_push and
 * pic_solve_field. */
int pic_autotune(pic_run *run, int32_t reps, pic_tune_entry *results,
                 int32_t max_results, int32_t *nresults);

/* ------------------------------------------------------------------------
 * One plasma on several GPUs, sharded by particles (the paper decomposes the
 * line over its threads and reduces the density and the solver's sums every
 * cycle, Sec. 3.1-3.3; here every rank keeps the whole grid).  Rank w holds
 * N_w of the N particles in its own run.  A step is, on every rank: [its own
 * sort when due] + pic_push + an all-reduce (sum, int64) of the NG density
 * sums pic_device_density points at + pic_solve_field.  The sums are exact
 * integers, so every rank solves the same density into the same field, and
 * the shards' particles are those of the whole run bit for bit.  The start:
 * pic_init of each rank's particles, then pic_deposit + the all-reduce +
 * pic_solve_field to make E^0 from the whole density.  The history rows'
 * kinetic energy and momentum are the rank's shares (sum them over the
 * ranks); the field rows are the whole plasma's.  pic_step_n cannot take
 * the all-reduce: step a shard with pic_push / pic_solve_field.
 * ------------------------------------------------------------------------ */

/* The run is one rank's shard of a plasma of npart_total particles
 * (npart <= npart_total <= 2^39): the density, the particle charge and mass
 * are normalised by npart_total.  PIC_FP32_FIXED only.  Drops the captured
 * graphs. */
int pic_set_shard(pic_run *run, int64_t npart_total);

/* Device pointer of the density accumulator: NG int64 fixed-point sums, the
 * deposit of the particles pushed since the last solve (PIC_FP32_FIXED). */
int pic_device_density(pic_run *run, void **rho_q);

/* Tune the sort interval S (PIC_FP32_FIXED): for each candidate in
 * intervals[count] (0 = never sort, else 1 .. 256; count <= 64), the mean
 * cost of a step's sort and push, modelled on a copy of the state with the
 * run's push shape: the sort of the state is timed, then the sorted copy is
 * pushed max(S) times with the current field, each push timed (t(k), k pushes
 * after a sort); cost(S) = (t_sort + sum_{k<S} t(k)) / S, cost(0) = the mean
 * of the last quarter of t(k).  ms_per_step[count] (may be NULL) receives the
 * costs, *best (may be NULL) the cheapest candidate; adopt != 0 sets the
 * run's sort interval to it (dropping the captured graphs).  The run's state
 * is untouched.  Synchronises.  PIC_ESTATE as for pic_autotune. */
int pic_tune_sort_interval(pic_run *run, const int32_t *intervals, int32_t count,
                           float *ms_per_step, int32_t *best, int32_t adopt);

/* ------------------------------------------------------------------------
 * Ensembles: many independent runs in one persistent launch (the batched and
 * served forms of the same step).  A pool owns a caller-provided device arena
 * and up to max_slots runs.  Every run's step is the step above, bit-identical
 * in particles and field to the same run on its own (pic_create ...).  Each
 * run needs pic_pool_run_bytes() of the arena; admission fails with
 * PIC_ENOMEM when the arena or the slots are full.  A run is advanced only by
 * pic_pool_advance, which launches one thread-block-cluster kernel for all
 * runs with steps left: each cluster takes runs from a queue, largest work
 * first, and keeps a run on chip through all of its steps of that launch.
 * A run with sort_interval S > 0 sorts its particles by cell before every
 * step n > 0 with n % S == 0, as the single run does (a stable counting sort
 * inside the cluster, into a second pair of particle buffers: 8 N more
 * arena bytes).
 * ------------------------------------------------------------------------ */

typedef struct pic_pool pic_pool;

typedef struct pic_pool_config {
    int32_t max_slots;     /* runs held at once (>= 1)                         */
    int32_t ncell_max;     /* largest NG admitted (<= PIC_NCELL_MAX)            */
    int32_t history;       /* diagnostics rows kept per run (>= 1)              */
    int32_t variant;       /* PIC_DEPOSIT_ATOMIC | _MATCH | _QUAD | _PAIR
                              (0 = MATCH); + 16: kernel built for two
                              512-thread blocks per SM (64 registers)
                              instead of one                                 */
    int32_t cluster;       /* blocks per cluster: 1, 2, 4, 8 (0 = 8)            */
    int32_t block;         /* threads per block: 128 .. 512 (0 = 256); the
                              shape needs ceil(ncell_max / cluster) <= block   */
} pic_pool_config;

/* Arena bytes one run with parameters *p takes in a pool with `history`
 * rows (twice the particle bytes when it sorts).  PIC_EINVAL for what no
 * pool admits: a precision other than PIC_FP32_FIXED, the CG solver, the
 * NGP shape, history < 1. */
int pic_pool_run_bytes(const pic_params *p, int32_t history, size_t *bytes);

/* Bytes at the start of the arena for the pool's own tables. */
int pic_pool_table_bytes(const pic_pool_config *cfg, size_t *bytes);

/* Create a pool over a caller-owned device arena (256-byte aligned; kept
 * alive until pic_pool_destroy).  Enqueues nothing. */
int pic_pool_create(const pic_pool_config *cfg, void *arena, size_t arena_bytes,
                    void *stream, pic_pool **out);
void pic_pool_destroy(pic_pool *pool);

/* Change the launch shape (variant, cluster, block) of later advances. */
int pic_pool_configure(pic_pool *pool, int32_t variant, int32_t cluster, int32_t block);

/* Admit a run: copy its initial state x0, v0 (host, N float32 each, positions
 * in [0, L)) into the arena and queue its set-up (deposit + solve of E^0,
 * done by the next advance).  It will be advanced for `steps` steps in total.
 * *slot receives its slot.  PIC_ENOMEM: no free slot or arena space;
 * PIC_EINVAL: bad parameters or positions. */
int pic_pool_admit(pic_pool *pool, const pic_params *p, const void *x0, const void *v0,
                   int64_t steps, int32_t *slot);

/* pic_pool_admit with the initial state generated on the device
 * (pic_load_two_stream) instead of copied from the host. */
int pic_pool_admit_loaded(pic_pool *pool, const pic_params *p, const pic_loading *ld,
                          int64_t steps, int32_t *slot);

/* Advance every admitted run by min(k, steps left) steps (set-up first for
 * newly admitted runs).  *active receives the number of runs that took part.
 * Asynchronous. */
int pic_pool_advance(pic_pool *pool, int64_t k, int32_t *active);

/* Slots whose runs have done all their steps (host bookkeeping; the results
 * are ready once the stream has reached the advance that finished them). */
int pic_pool_finished(const pic_pool *pool, int32_t *slots, int32_t max, int32_t *n);

/* Steps done by the run in `slot`. */
int pic_pool_step_count(const pic_pool *pool, int32_t slot, int64_t *step);

/* Results of a run (synchronise): state (positions converted from cell
 * units on the host, by the same two float64-rounded steps as pic_get_state),
 * the state in cell units as held on the device, field of its last step,
 * history. */
int pic_pool_get_state(pic_pool *pool, int32_t slot, void *x, void *v);
int pic_pool_get_cells(pic_pool *pool, int32_t slot, float *u, float *v);
int pic_pool_get_field(pic_pool *pool, int32_t slot, double *rho, double *phi, double *E,
                       int64_t *rho_q);
int pic_pool_diagnostics(pic_pool *pool, int32_t slot, int64_t first, int32_t count,
                         pic_diag_row *rows);

/* Free the run's arena space and slot. */
int pic_pool_release(pic_pool *pool, int32_t slot);

/* Wait for the stream and report the device error word. */
int pic_pool_sync(pic_pool *pool);

/* Arena bytes in use and free (largest free block). */
int pic_pool_usage(const pic_pool *pool, size_t *used, size_t *largest_free);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
