// pic_internal.cuh -- kernel argument blocks and launcher declarations shared
// by the translation units of libpic (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pic.h"

namespace pic {

// A named NVTX range over a call of the C ABI, so that a timeline tool shows
// each stage (push, solve, sort, step_n, pool advance, host copies) with its
// kernels and copies; without a tool attached the calls do nothing.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

constexpr unsigned kFull = 0xffffffffu;   // all lanes of a warp

// Fixed-point deposit: each particle adds exactly 2^24 to the density sum.
constexpr int kFixBits = 24;
constexpr uint32_t kFixOne = 1u << kFixBits;

// Bits of the device error word.
enum : uint32_t {
    kErrPosition = 1u,   // a position outside [0, L) or not finite
    kErrSortKey = 4u,    // a sort key outside the grid
    kErrInput = 8u,      // an uploaded position outside [0, L) (pic_init, pic_set_state)
};

// Float32 constants of the push, formed once on the host.  In the float32
// modes a position is kept as its cell coordinate u = x NG / L in [0, NG)
// (cell units: node g sits at u = g + 1/2), so the box end is the exact
// float NG and locating a particle needs no scale factor.
struct PushConsts {
    int ng;          // NG
    float ngf;       // (float)NG, exact: the box length in cell units
    float kdrift;    // (float)(dt NG / L): u advances by v kdrift per step
    float qmdt;      // (float)(qm * dt)
};

// Fused push + fixed-point deposit (or deposit alone when push == false).
struct PushArgs {
    float *x, *v;                 // N each (x: cell coordinates), 16-byte aligned
    long long n;                  // N
    const float *E32;             // field at the nodes, float32 [NG]
    unsigned long long *rho_q;    // fixed-point density accumulator [NG]
    double *partials;             // per-block [sum v_old v_new, sum v_new]
    unsigned int *err;            // device error word
    PushConsts c;
};

// Float64 push (PIC_FP64) and float32 push with float32 atomic deposit.
struct PushArgs64 {
    double *x, *v;
    long long n;
    const double *E64;
    double *rho_acc;              // sum of weights per node [NG]
    double *partials;
    unsigned int *err;
    int ng;
    double inv_dx, length, qmdt, dt;
};

struct PushArgsF32Atomic {
    float *x, *v;
    long long n;
    const float *E32;
    float *rho_acc;               // sum of float32 weights per node [NG]
    double *partials;
    unsigned int *err;
    PushConsts c;
};

// Per-block share of the step diagnostics, reduced by the solve's last block.
enum { kDiagFE = 0, kDiagKE, kDiagMom, kDiagCharge, kDiagModes,
       kDiagFields = kDiagModes + 2 * PIC_NMODES };
struct DiagPartial {
    double v[kDiagFields];         // field energy sum, KE and momentum sums,
                                   // charge, mode sums (re, im) x 8
    unsigned long long cq;         // fixed-point charge sum
};

// Field solve (fixed point: one cluster of up to 16 blocks; float modes and
// CG: one block).
struct SolveArgs {
    int mode;                     // PIC_FP32_FIXED / PIC_FP32_ATOMIC / PIC_FP64
    unsigned long long *rho_q;    // FIXED: accumulator (read, then zeroed)
    unsigned long long *rho_q_last; // FIXED: copy of the consumed sums
    float *rho_f32;               // FP32_ATOMIC accumulator
    double *rho_f64;              // FP64 accumulator
    double *rho, *phi, *E64;      // outputs [NG]
    float *E32;                   // output copy for the gather [NG]
    const double *partials;       // per-block sums of the push that ran
    int npartials;                // 0: no push ran since the last solve
    DiagPartial *dpart;           // [kSolveMaxBlocks]
    unsigned *counter;            // last-block ticket (0 between launches)
    pic_diag_row *hist;           // history ring
    int hist_len;
    long long *dstep;             // device step counter
    int ng;
    long long weight_total;       // N 2^24
    double rho_ion;
    double q_over_dx;             // Q0/dx = -rho_ion NG / N (float modes)
    double k_rho;                 // rho_ion / (N 2^24)
    double k_e;                   // (dx/2) k_rho / NG
    double k_phi;                 // -dx^2 k_rho / NG
    double k_mode;                // 2 / NG: mode amplitude of the mode sums
    double dx;
    double mass;                  // particle mass m = Q0/qm
    int solver;                   // PIC_SOLVER_EXACT / PIC_SOLVER_CG
    int cg_maxit;                 // CG: iterations per solve
};

// Counting sort by cell.
template <typename T>
struct SortArgs {
    const T *x, *v;               // source
    T *x_out, *v_out;             // destination
    long long n;
    int ng;
    T inv_dx;                     // NG / L in the particle precision
    int nchunk;                   // blocks of the count/scatter passes
    long long chunk;              // particles per block
    int nseg;                     // chunk segments of the column scan
    int seg_len;                  // chunks per segment
    unsigned int *hist;           // [nchunk][NG] counts, then offsets
    unsigned int *segtot;         // [nseg][NG] segment totals, then offsets
    unsigned int *base;           // [NG] first slot of each cell
    unsigned int *err;
};

// One run of a batched ensemble (device descriptor; host-built).
struct BatchRun {
    float *x, *v;                 // particles (cell coordinates u), 16-byte aligned
    float *xa, *va;               // the sort's destination (sort_interval > 0)
    int sort_interval;            // S: sort by cell before steps n % S == 0, n > 0
    long long n;                  // N
    PushConsts pc;                // ng, c = NG/L, L, qm dt, dt (float32)
    float *E32;                   // [NG] field of the current step (state)
    double *E64, *phi, *rho;      // [NG] written at the end of a launch
    unsigned long long *rho_q_last;  // [NG] idem
    pic_diag_row *hist;           // history ring of the run
    int hist_len;
    int steps;                    // steps to advance in this launch (0: idle)
    long long *step;              // device step counter of the run
    long long weight_total;       // N 2^24
    double k_rho, k_e, k_phi, dx, mass;
    double k_mode;                // 2 / NG: mode amplitude of the mode sums
};

struct BatchArgs {
    BatchRun *runs;
    const int *order;             // runs to process, largest first
    int nrun;                     // entries of order
    unsigned *next;               // work-queue ticket (0 at launch)
    unsigned *err;                // device error word
    int push;                     // 1: advance `steps`; 0: deposit + solve only
    int ng_max;                   // largest NG of the launch (tile size)
};

// Device-side initial loading (load.cu).
struct LoadArgs {
    float *x, *v;
    long long n;
    double length;
    float lengthf;
    float v0, vth;
    unsigned long long seed;
    int nmodes;
    float k[PIC_LOAD_MAX_MODES], amp[PIC_LOAD_MAX_MODES], phase[PIC_LOAD_MAX_MODES];
};
cudaError_t launch_load(const LoadArgs &a, int sms, cudaStream_t s);
int make_load_args(const pic_loading *ld, long long n, double length, float *x, float *v,
                   LoadArgs *out);

// Internal kernel choice of the fused push for the nearest-grid-point shape
// (not a public deposit variant: PIC_SHAPE_NGP selects it).
constexpr int kDepositNgp = 15;

// Phase-space histogram (phase.cu).
constexpr int kPhaseMaxBins = 16384;
template <typename T>
struct PhaseArgs {
    const T *x, *v;
    long long n;
    int nx, nv;
    float sx;             // nx / L
    float vmin, sv;       // nv / (vmax - vmin)
    unsigned *counts;     // [nv][nx]
};
template <typename T>
cudaError_t launch_phase(const PhaseArgs<T> &a, int sms, cudaStream_t s);

// Range check of uploaded positions: sets kErrInput unless every x is in
// [0, L) (phase.cu).
template <typename T>
cudaError_t launch_check_positions(const T *x, long long n, T length, unsigned *err, int sms,
                                   cudaStream_t s);

// Unit conversions of float32 positions (phase.cu), both rounded once from a
// float64 product:
//   to cells     u = (float)((double)x (NG/L)), a u that rounds to NG is 0;
//                sets kErrInput unless x is in [0, (float)L); in place.
//   to physical  x = (float)((double)u (L/NG)), at most the largest float
//                below (float)L.
// The host forms the same two products in pool_to_physical (ensemble.cu).
cudaError_t launch_to_cells(float *x, long long n, double to_cells, float ngf, float length32,
                            unsigned *err, int sms, cudaStream_t s);
cudaError_t launch_to_physical(const float *u, float *x, long long n, double to_phys,
                               float length32, int sms, cudaStream_t s);
// Cell coordinates read back from a caller: every u must lie in [0, NG).
cudaError_t launch_check_cells(const float *u, long long n, float ngf, unsigned *err, int sms,
                               cudaStream_t s);
float below(float v);            // the largest float below v (v > 0)

// Parameter checks shared by the single-run and the pool entry points.
int validate_params(const pic_params *p);

// Launchers (each returns the launch's cudaError_t).
cudaError_t launch_push_fixed(const PushArgs &a, int grid, int block,
                              int variant, int unroll, bool push, cudaStream_t s);
cudaError_t launch_push_f32_atomic(const PushArgsF32Atomic &a, int grid,
                                   int block, bool push, cudaStream_t s);
cudaError_t launch_push_f64(const PushArgs64 &a, int grid, int block,
                            bool push, cudaStream_t s);
size_t push_smem_bytes(int mode, int ng);
cudaError_t push_prepare_attributes(int mode, int ng);
int push_max_blocks_per_sm(int mode, int variant, int unroll, int block, int ng);

cudaError_t launch_solve(const SolveArgs &a, cudaStream_t s);
cudaError_t solve_prepare_attributes();
constexpr int kSolveThreads = 1024;
constexpr int kSolveMaxBlocks = 32;

cudaError_t launch_sort_f32(const SortArgs<float> &a, cudaStream_t s);
cudaError_t launch_sort_f64(const SortArgs<double> &a, cudaStream_t s);
cudaError_t sort_prepare_attributes(int ng);
constexpr int kSortThreads = 256;

cudaError_t launch_batch(const BatchArgs &a, int variant, int cluster, int block,
                         int nclusters, cudaStream_t s);
size_t batch_smem_bytes(int ng_max, int cluster, int block);
int batch_max_clusters(int variant, int cluster, int block, int ng_max);
cudaError_t batch_prepare_attributes();

}  // namespace pic
