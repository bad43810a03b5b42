// pic_api.cu -- the C ABI of include/pic.h: parameter checks, the workspace
// layout, the run handle, step sequencing and CUDA-graph replay.
//
// The caller owns every device byte (one workspace); this file only carves it.
// A step is [sort if due] + fused push/deposit + field solve, enqueued on the
// caller's stream.  pic_step_n replays whole sort periods from CUDA graphs
// (captured once per run on a private stream, launched on the caller's), so a
// period of S steps costs one graph launch instead of 2 S + 4 kernel launches.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "pic_internal.cuh"

using namespace pic;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxPushGrid = 4096;     // per-block partial sums kept
constexpr int kMaxSortChunks = 1024;
constexpr int kPlainBlock = 16;        // steps per graph when not sorting
constexpr int kDefaultHistory = 4096;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

bool is_variant(int v) {
    return v == PIC_DEPOSIT_ATOMIC || v == PIC_DEPOSIT_MATCH || v == PIC_DEPOSIT_QUAD ||
           v == PIC_DEPOSIT_PAIR || v == PIC_DEPOSIT_QUAD8 || v == PIC_DEPOSIT_PAIR8;
}

// particles a thread takes per group: 8 for the 32-byte variants, else 4
int group_width(int v) { return v == PIC_DEPOSIT_QUAD8 || v == PIC_DEPOSIT_PAIR8 ? 8 : 4; }

}  // namespace

int pic::validate_params(const pic_params *p) {
    if (!p) return PIC_EINVAL;
    if (p->npart < 1 || p->npart > (int64_t)0xFFFFFFFFll) return PIC_EINVAL;
    if (p->ncell < 1 || p->ncell > PIC_NCELL_MAX) return PIC_EINVAL;
    if (p->precision < PIC_FP32_FIXED || p->precision > PIC_FP64) return PIC_EINVAL;
    if (!finite_pos(p->length) || !finite_pos(p->dt) || !finite_pos(p->rho_ion)) return PIC_EINVAL;
    if (!std::isfinite(p->qm) || !(p->qm < 0.0)) return PIC_EINVAL;
    if (p->sort_interval < 0 || p->history < 0) return PIC_EINVAL;
    if (p->deposit_variant != PIC_DEPOSIT_AUTO && !is_variant(p->deposit_variant)) return PIC_EINVAL;
    if (p->block_size != 0 && (p->block_size < 32 || p->block_size > 1024 || p->block_size % 32)) return PIC_EINVAL;
    if (p->precision == PIC_FP32_FIXED && p->block_size > 512) return PIC_EINVAL;
    if (p->blocks_per_sm < 0 || p->blocks_per_sm > 32) return PIC_EINVAL;
    if (p->unroll != 0 && p->unroll != 1 && p->unroll != 2 && p->unroll != 4) return PIC_EINVAL;
    if (p->field_solver != PIC_SOLVER_EXACT && p->field_solver != PIC_SOLVER_CG) return PIC_EINVAL;
    if (p->cg_iterations < 0 || p->cg_iterations > 100000) return PIC_EINVAL;
    if (p->shape != PIC_SHAPE_CIC && p->shape != PIC_SHAPE_NGP) return PIC_EINVAL;
    if (p->shape == PIC_SHAPE_NGP && p->precision != PIC_FP32_FIXED) return PIC_EINVAL;
    if (p->reserved != 0) return PIC_EINVAL;
    return PIC_OK;
}

namespace {

struct Layout {
    size_t x[2], v[2];
    size_t rho_q, rho_q_last, rho_f32, rho_f64;
    size_t rho, phi, E64, E32;
    size_t partials, dpart, hist, dev, tune_rho, phase;
    size_t s_hist, s_segtot, s_base;
    size_t total;
    int hist_len;
    int nchunk, nseg, seg_len;
    long long chunk;
};

// Device scalars of a run.
struct DevScalars {
    long long step;
    unsigned err;
    unsigned counter;
};

// Chunks of the counting sort: 2048 particles (one scatter tile) or more
// each, at most kMaxSortChunks, and at most 32 MiB of per-chunk counts;
// segments of about sqrt(nchunk) chunks.
void sort_geometry(int64_t n, int ng, int *nchunk, long long *chunk, int *nseg, int *seg_len) {
    long long nc = (n + 2047) / 2048;
    const long long cap_tab = (32ll << 20) / (4ll * ng);
    if (nc > kMaxSortChunks) nc = kMaxSortChunks;
    if (nc > cap_tab) nc = cap_tab;
    if (nc < 1) nc = 1;
    long long ch = (n + nc - 1) / nc;
    ch = (ch + 3) & ~3ll;                   // chunks start on float4 groups
    nc = (n + ch - 1) / ch;
    int ns = 1;
    while ((long long)ns * ns < nc) ns++;   // nseg, seg_len <= 32 (nchunk <= 1024)
    *nchunk = (int)nc;
    *chunk = ch;
    *seg_len = (int)((nc + ns - 1) / ns);
    *nseg = (int)((nc + *seg_len - 1) / *seg_len);
}

void make_layout(const pic_params *p, Layout *L) {
    const size_t n = (size_t)p->npart, ng = (size_t)p->ncell;
    const size_t es = p->precision == PIC_FP64 ? 8 : 4;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    L->x[0] = take(n * es);
    L->v[0] = take(n * es);
    L->x[1] = take(n * es);
    L->v[1] = take(n * es);
    L->rho_q = take(ng * 8);
    L->rho_q_last = take(ng * 8);
    L->rho_f32 = take(ng * 4);
    L->rho_f64 = take(ng * 8);
    L->rho = take(ng * 8);
    L->phi = take(ng * 8);
    L->E64 = take(ng * 8);
    L->E32 = take(ng * 4);
    L->partials = take((size_t)kMaxPushGrid * 2 * 8);
    L->dpart = take((size_t)kSolveMaxBlocks * sizeof(DiagPartial));
    L->hist_len = p->history > 0 ? p->history : kDefaultHistory;
    L->hist = take((size_t)L->hist_len * sizeof(pic_diag_row));
    L->dev = take(sizeof(DevScalars));
    L->tune_rho = take(ng * 8);
    L->phase = take((size_t)kPhaseMaxBins * 4);
    sort_geometry(p->npart, p->ncell, &L->nchunk, &L->chunk, &L->nseg, &L->seg_len);
    L->s_hist = take((size_t)L->nchunk * ng * 4);
    L->s_segtot = take((size_t)L->nseg * ng * 4);
    L->s_base = take(ng * 4);
    L->total = off;
}

int cuda_fail(cudaError_t e) {
    if (e == cudaSuccess) return PIC_OK;
    std::fprintf(stderr, "libpic: CUDA error %d: %s\n", (int)e, cudaGetErrorString(e));
    return PIC_ECUDA;
}

#define PIC_CUDA(call)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_);    \
    } while (0)

}  // namespace

struct pic_run {
    pic_params p{};
    Layout lay{};
    int device = 0, sms = 0;
    cudaStream_t stream = nullptr;   // the caller's
    cudaStream_t cap = nullptr;      // private stream for graph capture
    cudaStream_t aux = nullptr;      // private stream: the second host copy of a load or read-back
    cudaEvent_t fork = nullptr, join = nullptr;
    unsigned char *ws = nullptr;
    int cur = 0;                     // which x/v buffer holds the state
    int grid = 0, block = 0, variant = 0, unroll = 1;
    int64_t step = 0;
    bool ready = false, pending_push = false;
    cudaGraphExec_t period[2] = {nullptr, nullptr};   // S steps from x parity 0/1
    cudaGraphExec_t plain = nullptr;                  // kPlainBlock steps, no sort
    PushConsts pc{};
    double dx = 0, mass = 0, q_over_dx = 0, k_rho = 0, k_e = 0, k_phi = 0;
    double to_cells = 0, to_phys = 0;  // NG/L and L/NG (float32 positions)
    int64_t npart_total = 0;           // particles of the whole plasma (a shard holds npart)
    float length32 = 0;                // (float)L: positions lie in [0, length32)

    template <typename T> T *at(size_t off) const { return reinterpret_cast<T *>(ws + off); }
    DevScalars *dev() const { return at<DevScalars>(lay.dev); }
    size_t elem() const { return p.precision == PIC_FP64 ? 8 : 4; }
    void *xs(int i) const { return ws + lay.x[i]; }
    void *vs(int i) const { return ws + lay.v[i]; }
};

namespace {

// Float64 constants of the solve for a plasma of n_total particles (Appendix
// A: Q0 = rho_init0 Lx / N, with the sign of qm; a shard holds n of them).
void set_solve_constants(pic_run *r, int64_t n_total) {
    const pic_params *p = &r->p;
    r->npart_total = n_total;
    r->dx = p->length / (double)p->ncell;
    const double q0 = (p->rho_ion * p->length / (double)n_total) * (p->qm / std::fabs(p->qm));
    r->q_over_dx = q0 / r->dx;
    r->mass = q0 / p->qm;
    r->k_rho = p->rho_ion / std::ldexp((double)n_total, kFixBits);
    r->k_e = 0.5 * r->dx * r->k_rho / (double)p->ncell;
    r->k_phi = -r->dx * r->dx * r->k_rho / (double)p->ncell;
}

void destroy_graphs(pic_run *r) {
    for (auto &g : r->period)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    if (r->plain) { cudaGraphExecDestroy(r->plain); r->plain = nullptr; }
}

cudaError_t enqueue_push(pic_run *r, cudaStream_t s, bool push) {
    const int c = r->cur;
    if (r->p.precision == PIC_FP32_FIXED) {
        PushArgs a;
        a.x = (float *)r->xs(c);
        a.v = (float *)r->vs(c);
        a.n = r->p.npart;
        a.E32 = r->at<float>(r->lay.E32);
        a.rho_q = r->at<unsigned long long>(r->lay.rho_q);
        a.partials = r->at<double>(r->lay.partials);
        a.err = &r->dev()->err;
        a.c = r->pc;
        return launch_push_fixed(a, r->grid, r->block, r->variant, r->unroll, push, s);
    } else if (r->p.precision == PIC_FP32_ATOMIC) {
        PushArgsF32Atomic a;
        a.x = (float *)r->xs(c);
        a.v = (float *)r->vs(c);
        a.n = r->p.npart;
        a.E32 = r->at<float>(r->lay.E32);
        a.rho_acc = r->at<float>(r->lay.rho_f32);
        a.partials = r->at<double>(r->lay.partials);
        a.err = &r->dev()->err;
        a.c = r->pc;
        return launch_push_f32_atomic(a, r->grid, r->block, push, s);
    } else {
        PushArgs64 a;
        a.x = (double *)r->xs(c);
        a.v = (double *)r->vs(c);
        a.n = r->p.npart;
        a.E64 = r->at<double>(r->lay.E64);
        a.rho_acc = r->at<double>(r->lay.rho_f64);
        a.partials = r->at<double>(r->lay.partials);
        a.err = &r->dev()->err;
        a.ng = r->p.ncell;
        a.inv_dx = (double)r->p.ncell / r->p.length;
        a.length = r->p.length;
        a.qmdt = r->p.qm * r->p.dt;
        a.dt = r->p.dt;
        return launch_push_f64(a, r->grid, r->block, push, s);
    }
}

cudaError_t enqueue_solve(pic_run *r, cudaStream_t s, bool after_push) {
    SolveArgs a;
    a.mode = r->p.precision;
    a.rho_q = r->at<unsigned long long>(r->lay.rho_q);
    a.rho_q_last = r->at<unsigned long long>(r->lay.rho_q_last);
    a.rho_f32 = r->at<float>(r->lay.rho_f32);
    a.rho_f64 = r->at<double>(r->lay.rho_f64);
    a.rho = r->at<double>(r->lay.rho);
    a.phi = r->at<double>(r->lay.phi);
    a.E64 = r->at<double>(r->lay.E64);
    a.E32 = r->at<float>(r->lay.E32);
    a.partials = r->at<double>(r->lay.partials);
    a.npartials = after_push ? r->grid : 0;
    a.dpart = r->at<DiagPartial>(r->lay.dpart);
    a.counter = &r->dev()->counter;
    a.hist = r->at<pic_diag_row>(r->lay.hist);
    a.hist_len = r->lay.hist_len;
    a.dstep = &r->dev()->step;
    a.ng = r->p.ncell;
    a.weight_total = (long long)r->npart_total << kFixBits;
    a.rho_ion = r->p.rho_ion;
    a.q_over_dx = r->q_over_dx;
    a.k_rho = r->k_rho;
    a.k_e = r->k_e;
    a.k_phi = r->k_phi;
    a.k_mode = 2.0 / (double)r->p.ncell;
    a.dx = r->dx;
    a.mass = r->mass;
    a.solver = r->p.field_solver;
    a.cg_maxit = r->p.cg_iterations ? r->p.cg_iterations : PIC_CG_DEFAULT_ITERATIONS;
    return launch_solve(a, s);
}

cudaError_t enqueue_sort(pic_run *r, cudaStream_t s) {
    const int c = r->cur;
    cudaError_t e;
    if (r->p.precision == PIC_FP64) {
        SortArgs<double> a;
        a.x = (const double *)r->xs(c); a.v = (const double *)r->vs(c);
        a.x_out = (double *)r->xs(1 - c); a.v_out = (double *)r->vs(1 - c);
        a.n = r->p.npart; a.ng = r->p.ncell;
        a.inv_dx = (double)r->p.ncell / r->p.length;
        a.nchunk = r->lay.nchunk; a.chunk = r->lay.chunk;
        a.nseg = r->lay.nseg; a.seg_len = r->lay.seg_len;
        a.hist = r->at<unsigned>(r->lay.s_hist);
        a.segtot = r->at<unsigned>(r->lay.s_segtot);
        a.base = r->at<unsigned>(r->lay.s_base);
        a.err = &r->dev()->err;
        e = launch_sort_f64(a, s);
    } else {
        SortArgs<float> a;
        a.x = (const float *)r->xs(c); a.v = (const float *)r->vs(c);
        a.x_out = (float *)r->xs(1 - c); a.v_out = (float *)r->vs(1 - c);
        a.n = r->p.npart; a.ng = r->p.ncell;
        a.inv_dx = 1.0f;                      // cell coordinates: the key is trunc(u)
        a.nchunk = r->lay.nchunk; a.chunk = r->lay.chunk;
        a.nseg = r->lay.nseg; a.seg_len = r->lay.seg_len;
        a.hist = r->at<unsigned>(r->lay.s_hist);
        a.segtot = r->at<unsigned>(r->lay.s_segtot);
        a.base = r->at<unsigned>(r->lay.s_base);
        a.err = &r->dev()->err;
        e = launch_sort_f32(a, s);
    }
    if (e == cudaSuccess) r->cur = 1 - c;
    return e;
}

// Sort buffer `from` into buffer 1-from (the run's current buffer is left as
// it is).
cudaError_t enqueue_sort_into(pic_run *r, int from, cudaStream_t s) {
    const int saved = r->cur;
    r->cur = from;
    cudaError_t e = enqueue_sort(r, s);
    r->cur = saved;
    return e;
}

// One step on stream s: [sort] + push + solve.
cudaError_t enqueue_step(pic_run *r, cudaStream_t s, bool sort) {
    cudaError_t e;
    if (sort && (e = enqueue_sort(r, s)) != cudaSuccess) return e;
    if ((e = enqueue_push(r, s, true)) != cudaSuccess) return e;
    return enqueue_solve(r, s, true);
}

// Capture `nsteps` steps (the first with a sort if `sort_first`) starting
// from x parity `parity` into an executable graph.
int capture(pic_run *r, int parity, bool sort_first, int nsteps, cudaGraphExec_t *out) {
    const int saved = r->cur;
    r->cur = parity;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(r->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { r->cur = saved; return cuda_fail(e); }
    cudaError_t le = cudaSuccess;
    for (int i = 0; i < nsteps && le == cudaSuccess; i++)
        le = enqueue_step(r, r->cap, sort_first && i == 0);
    e = cudaStreamEndCapture(r->cap, &g);
    r->cur = saved;
    if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(le); }
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e); }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return cuda_fail(e);
}

// Grid of the persistent push: SMs x resident blocks, no more blocks than
// there is work for, at most kMaxPushGrid (the partial-sum slots).
int push_grid(const pic_run *r, int variant, int block, int unroll, int bps_cap) {
    int bps = push_max_blocks_per_sm(r->p.precision, variant, unroll, block, r->p.ncell);
    if (bps < 1) return 0;
    if (bps_cap && bps_cap < bps) bps = bps_cap;
    long long want = (long long)r->sms * bps;
    const int gw = group_width(variant);
    const long long units = r->p.precision == PIC_FP32_FIXED ? (r->p.npart + gw - 1) / gw
                                                             : r->p.npart;
    const long long per_block = (long long)block * unroll;
    const long long need = (units + per_block - 1) / per_block;
    if (want > need) want = need;
    if (want > kMaxPushGrid) want = kMaxPushGrid;
    if (want < 1) want = 1;
    return (int)want;
}

// Work on the private stream after everything enqueued on the run's stream
// so far (fork), and the run's stream after that work (join).
cudaError_t fork_aux(pic_run *r) {
    cudaError_t e = cudaEventRecord(r->fork, r->stream);
    return e == cudaSuccess ? cudaStreamWaitEvent(r->aux, r->fork, 0) : e;
}

cudaError_t join_aux(pic_run *r) {
    cudaError_t e = cudaEventRecord(r->join, r->aux);
    return e == cudaSuccess ? cudaStreamWaitEvent(r->stream, r->join, 0) : e;
}

int read_error_word(pic_run *r) {
    unsigned err = 0;
    PIC_CUDA(cudaMemcpyAsync(&err, &r->dev()->err, sizeof(err), cudaMemcpyDeviceToHost, r->stream));
    PIC_CUDA(cudaStreamSynchronize(r->stream));
    if (err & kErrInput) return PIC_EINVAL;
    return err ? PIC_EDEVICE : PIC_OK;
}

// How the positions in buffer 0 are given.
enum class Units { kPhysical, kCells };

// With x, v in buffer 0: check (and, in the float32 modes, convert to cell
// coordinates) the positions, reset the run, deposit and solve: E^step ready.
int prepare_loaded(pic_run *r, int64_t step, Units units, bool aux_copy = false) {
    DevScalars ds{};
    ds.step = step;
    PIC_CUDA(cudaMemcpyAsync(r->dev(), &ds, sizeof(ds), cudaMemcpyHostToDevice, r->stream));
    if (r->p.precision == PIC_FP64)
        PIC_CUDA(launch_check_positions((const double *)r->xs(0), r->p.npart, r->p.length,
                                        &r->dev()->err, r->sms, r->stream));
    else if (units == Units::kPhysical)
        PIC_CUDA(launch_to_cells((float *)r->xs(0), r->p.npart, r->to_cells, r->pc.ngf,
                                 r->length32, &r->dev()->err, r->sms, r->stream));
    else
        PIC_CUDA(launch_check_cells((const float *)r->xs(0), r->p.npart, r->pc.ngf,
                                    &r->dev()->err, r->sms, r->stream));
    PIC_CUDA(cudaMemsetAsync(r->ws + r->lay.rho_q, 0, (size_t)r->p.ncell * 8, r->stream));
    PIC_CUDA(cudaMemsetAsync(r->ws + r->lay.rho_f32, 0, (size_t)r->p.ncell * 4, r->stream));
    PIC_CUDA(cudaMemsetAsync(r->ws + r->lay.rho_f64, 0, (size_t)r->p.ncell * 8, r->stream));
    PIC_CUDA(cudaMemsetAsync(r->ws + r->lay.hist, 0xFF, (size_t)r->lay.hist_len * sizeof(pic_diag_row), r->stream));
    PIC_CUDA(enqueue_push(r, r->stream, false));
    PIC_CUDA(enqueue_solve(r, r->stream, false));
    if (aux_copy) PIC_CUDA(join_aux(r));
    PIC_CUDA(cudaStreamSynchronize(r->stream));
    r->step = step;
    r->pending_push = false;
    const int rc = read_error_word(r);
    r->ready = rc == PIC_OK;       // a rejected upload leaves no usable state
    return rc;
}

// Upload a state, deposit it and solve: E^step ready.
// The positions are range-checked (and converted) on the device after the
// upload (a host loop over N positions cost more than the whole upload).
// The positions go up first; the velocities follow on the private stream
// while the positions are converted and deposited and the field is solved
// (none of which reads v), so that work hides under the second copy.
int load_state(pic_run *r, const void *x, const void *v, int64_t step, Units units) {
    if (!x || !v) return PIC_EINVAL;
    const size_t bytes = (size_t)r->p.npart * r->elem();
    r->ready = false;           // until the new state is loaded, checked and solved
    r->cur = 0;
    PIC_CUDA(cudaMemcpyAsync(r->xs(0), x, bytes, cudaMemcpyHostToDevice, r->stream));
    PIC_CUDA(fork_aux(r));
    PIC_CUDA(cudaMemcpyAsync(r->vs(0), v, bytes, cudaMemcpyHostToDevice, r->aux));
    return prepare_loaded(r, step, units, true);
}

}  // namespace

extern "C" {

int pic_version(void) { return PIC_ABI_VERSION; }

const char *pic_strerror(int code) {
    switch (code) {
        case PIC_OK: return "ok";
        case PIC_EINVAL: return "invalid argument";
        case PIC_ENOMEM: return "workspace too small or budget exhausted";
        case PIC_ECUDA: return "CUDA runtime error";
        case PIC_ETIMEOUT: return "device wait timed out";
        case PIC_EDEVICE: return "kernel flagged bad particle data";
        case PIC_ESTATE: return "call out of order";
        default: return "unknown error";
    }
}

int pic_workspace_size(const pic_params *p, size_t *bytes) {
    int rc = validate_params(p);
    if (rc) return rc;
    if (!bytes) return PIC_EINVAL;
    Layout L;
    make_layout(p, &L);
    *bytes = L.total;
    return PIC_OK;
}

int pic_create(const pic_params *p, void *workspace, size_t workspace_bytes,
               void *stream, pic_run **out) {
    if (!out) return PIC_EINVAL;
    *out = nullptr;
    int rc = validate_params(p);
    if (rc) return rc;
    if (!workspace || ((uintptr_t)workspace % kAlign)) return PIC_EINVAL;
    pic_run *r = new (std::nothrow) pic_run();
    if (!r) return PIC_ENOMEM;
    r->p = *p;
    make_layout(p, &r->lay);
    if (workspace_bytes < r->lay.total) { delete r; return PIC_ENOMEM; }
    r->ws = (unsigned char *)workspace;
    r->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&r->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&r->sms, cudaDevAttrMultiProcessorCount, r->device);
    if (e == cudaSuccess) e = push_prepare_attributes(p->precision, p->ncell);
    if (e == cudaSuccess) e = sort_prepare_attributes(p->ncell);
    if (e == cudaSuccess) e = solve_prepare_attributes();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&r->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&r->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->join, cudaEventDisableTiming);
    if (e != cudaSuccess) { pic_destroy(r); return cuda_fail(e); }

    // float32 constants of the push in cell units (u = x NG/L)
    r->pc.ng = p->ncell;
    r->pc.ngf = (float)p->ncell;
    r->pc.kdrift = (float)(p->dt * (double)p->ncell / p->length);
    r->pc.qmdt = (float)(p->qm * p->dt);
    r->to_cells = (double)p->ncell / p->length;
    r->to_phys = p->length / (double)p->ncell;
    r->length32 = (float)p->length;
    set_solve_constants(r, p->npart);

    // launch shape of the fused push
    r->variant = p->deposit_variant ? p->deposit_variant : PIC_DEPOSIT_QUAD;
    if (p->precision != PIC_FP32_FIXED) r->variant = PIC_DEPOSIT_ATOMIC;
    if (p->shape == PIC_SHAPE_NGP) r->variant = kDepositNgp;
    r->block = p->block_size ? p->block_size : (p->precision == PIC_FP32_FIXED ? 512 : 256);
    r->unroll = p->unroll ? p->unroll : 1;
    if (p->precision != PIC_FP32_FIXED) r->unroll = 1;
    r->grid = push_grid(r, r->variant, r->block, r->unroll, p->blocks_per_sm);
    if (r->grid < 1) { delete r; return PIC_EINVAL; }
    *out = r;
    return PIC_OK;
}

void pic_destroy(pic_run *run) {
    if (!run) return;
    destroy_graphs(run);
    if (run->cap) cudaStreamDestroy(run->cap);
    if (run->aux) cudaStreamDestroy(run->aux);
    if (run->fork) cudaEventDestroy(run->fork);
    if (run->join) cudaEventDestroy(run->join);
    delete run;
}

int pic_init(pic_run *run, const void *x0, const void *v0) {
    pic::TraceRange trace_("pic_init");
    if (!run) return PIC_EINVAL;
    return load_state(run, x0, v0, 0, Units::kPhysical);
}

int pic_init_loaded(pic_run *run, const pic_loading *ld) {
    pic::TraceRange trace_("pic_init_loaded");
    if (!run || !ld) return PIC_EINVAL;
    if (run->p.precision == PIC_FP64) return PIC_EINVAL;
    LoadArgs a;
    int rc = make_load_args(ld, run->p.npart, run->p.length, (float *)run->xs(0),
                            (float *)run->vs(0), &a);
    if (rc) return rc;
    run->ready = false;
    run->cur = 0;
    PIC_CUDA(launch_load(a, run->sms, run->stream));
    return prepare_loaded(run, 0, Units::kPhysical);
}

int pic_set_state(pic_run *run, const void *x, const void *v, int64_t step) {
    pic::TraceRange trace_("pic_set_state");
    if (!run || step < 0) return PIC_EINVAL;
    return load_state(run, x, v, step, Units::kPhysical);
}

int pic_set_cells(pic_run *run, const float *u, const void *v, int64_t step) {
    pic::TraceRange trace_("pic_set_cells");
    if (!run || step < 0) return PIC_EINVAL;
    if (run->p.precision == PIC_FP64) return PIC_EINVAL;
    return load_state(run, u, v, step, Units::kCells);
}

int pic_get_cells(pic_run *run, float *u, void *v) {
    pic::TraceRange trace_("pic_get_cells");
    if (!run) return PIC_EINVAL;
    if (run->p.precision == PIC_FP64) return PIC_EINVAL;
    if (!run->ready) return PIC_ESTATE;
    const size_t bytes = (size_t)run->p.npart * run->elem();
    if (u) PIC_CUDA(cudaMemcpyAsync(u, run->xs(run->cur), bytes, cudaMemcpyDeviceToHost, run->stream));
    if (v) PIC_CUDA(cudaMemcpyAsync(v, run->vs(run->cur), bytes, cudaMemcpyDeviceToHost, run->stream));
    PIC_CUDA(cudaStreamSynchronize(run->stream));
    return read_error_word(run);
}

int pic_deposit(pic_run *run) {
    pic::TraceRange trace_("pic_deposit");
    if (!run) return PIC_EINVAL;
    if (!run->ready) return PIC_ESTATE;
    const size_t ng = (size_t)run->p.ncell;
    PIC_CUDA(cudaMemsetAsync(run->ws + run->lay.rho_q, 0, ng * 8, run->stream));
    PIC_CUDA(cudaMemsetAsync(run->ws + run->lay.rho_f32, 0, ng * 4, run->stream));
    PIC_CUDA(cudaMemsetAsync(run->ws + run->lay.rho_f64, 0, ng * 8, run->stream));
    PIC_CUDA(enqueue_push(run, run->stream, false));
    return PIC_OK;
}

int pic_solve_field(pic_run *run) {
    pic::TraceRange trace_("pic_solve_field");
    if (!run) return PIC_EINVAL;
    if (!run->ready) return PIC_ESTATE;
    PIC_CUDA(enqueue_solve(run, run->stream, run->pending_push));
    if (run->pending_push) run->step++;
    run->pending_push = false;
    return PIC_OK;
}

int pic_push(pic_run *run) {
    pic::TraceRange trace_("pic_push");
    if (!run) return PIC_EINVAL;
    if (!run->ready || run->pending_push) return PIC_ESTATE;
    PIC_CUDA(enqueue_push(run, run->stream, true));
    run->pending_push = true;
    return PIC_OK;
}

int pic_sort(pic_run *run) {
    pic::TraceRange trace_("pic_sort");
    if (!run) return PIC_EINVAL;
    if (!run->ready) return PIC_ESTATE;
    PIC_CUDA(enqueue_sort(run, run->stream));
    return PIC_OK;
}

int pic_step_n(pic_run *run, int64_t n) {
    pic::TraceRange trace_("pic_step_n");
    if (!run || n < 0) return PIC_EINVAL;
    if (!run->ready || run->pending_push) return PIC_ESTATE;
    const int64_t S = run->p.sort_interval;
    while (n > 0) {
        const bool sort_due = S > 0 && run->step > 0 && run->step % S == 0;
        if (sort_due && n >= S) {
            cudaGraphExec_t &g = run->period[run->cur];
            if (!g) {
                int rc = capture(run, run->cur, true, (int)S, &g);
                if (rc) return rc;
            }
            PIC_CUDA(cudaGraphLaunch(g, run->stream));
            run->cur = 1 - run->cur;
            run->step += S;
            n -= S;
        } else if (S == 0 && n >= kPlainBlock) {
            if (!run->plain) {
                int rc = capture(run, run->cur, false, kPlainBlock, &run->plain);
                if (rc) return rc;
            }
            PIC_CUDA(cudaGraphLaunch(run->plain, run->stream));
            run->step += kPlainBlock;
            n -= kPlainBlock;
        } else {
            PIC_CUDA(enqueue_step(run, run->stream, sort_due));
            run->step += 1;
            n -= 1;
        }
    }
    return PIC_OK;
}

int pic_sync(pic_run *run) {
    if (!run) return PIC_EINVAL;
    PIC_CUDA(cudaStreamSynchronize(run->stream));
    return read_error_word(run);
}

int64_t pic_step_count(const pic_run *run) { return run ? run->step : -1; }

int pic_diagnostics(pic_run *run, int64_t first, int32_t count, pic_diag_row *rows) {
    pic::TraceRange trace_("pic_diagnostics");
    if (!run || !rows || count < 0 || first < 0) return PIC_EINVAL;
    if (!run->ready) return PIC_ESTATE;
    const int64_t H = run->lay.hist_len;
    const int64_t last = first + count - 1;
    if (count == 0) return PIC_OK;
    if (last > run->step || first < run->step - H + 1) return PIC_EINVAL;
    const pic_diag_row *hist = run->at<pic_diag_row>(run->lay.hist);
    int64_t done = 0;
    while (done < count) {
        const int64_t slot = (first + done) % H;
        int64_t len = count - done;
        if (slot + len > H) len = H - slot;
        PIC_CUDA(cudaMemcpyAsync(rows + done, hist + slot, (size_t)len * sizeof(pic_diag_row),
                                 cudaMemcpyDeviceToHost, run->stream));
        done += len;
    }
    PIC_CUDA(cudaStreamSynchronize(run->stream));
    return read_error_word(run);
}

int pic_get_state(pic_run *run, void *x, void *v) {
    pic::TraceRange trace_("pic_get_state");
    if (!run) return PIC_EINVAL;
    if (!run->ready) return PIC_ESTATE;
    const size_t bytes = (size_t)run->p.npart * run->elem();
    // the velocities go down on the private stream while the positions are
    // converted, then the positions follow
    if (v) {
        PIC_CUDA(fork_aux(run));
        PIC_CUDA(cudaMemcpyAsync(v, run->vs(run->cur), bytes, cudaMemcpyDeviceToHost, run->aux));
    }
    if (x) {
        const void *src = run->xs(run->cur);
        if (run->p.precision != PIC_FP64) {
            // physical positions into the idle particle buffer, then out
            float *tmp = (float *)run->xs(1 - run->cur);
            PIC_CUDA(launch_to_physical((const float *)src, tmp, run->p.npart, run->to_phys,
                                        run->length32, run->sms, run->stream));
            src = tmp;
        }
        PIC_CUDA(cudaMemcpyAsync(x, src, bytes, cudaMemcpyDeviceToHost, run->stream));
    }
    if (v) PIC_CUDA(join_aux(run));
    PIC_CUDA(cudaStreamSynchronize(run->stream));
    return read_error_word(run);
}

int pic_get_field(pic_run *run, double *rho, double *phi, double *E, int64_t *rho_q) {
    pic::TraceRange trace_("pic_get_field");
    if (!run) return PIC_EINVAL;
    if (!run->ready) return PIC_ESTATE;
    const size_t ng = (size_t)run->p.ncell;
    if (rho) PIC_CUDA(cudaMemcpyAsync(rho, run->ws + run->lay.rho, ng * 8, cudaMemcpyDeviceToHost, run->stream));
    if (phi) PIC_CUDA(cudaMemcpyAsync(phi, run->ws + run->lay.phi, ng * 8, cudaMemcpyDeviceToHost, run->stream));
    if (E) PIC_CUDA(cudaMemcpyAsync(E, run->ws + run->lay.E64, ng * 8, cudaMemcpyDeviceToHost, run->stream));
    if (rho_q) {
        if (run->p.precision == PIC_FP32_FIXED)
            PIC_CUDA(cudaMemcpyAsync(rho_q, run->ws + run->lay.rho_q_last, ng * 8, cudaMemcpyDeviceToHost, run->stream));
        else
            std::memset(rho_q, 0, ng * 8);
    }
    PIC_CUDA(cudaStreamSynchronize(run->stream));
    return read_error_word(run);
}

int pic_phase_space(pic_run *run, int32_t nx, int32_t nv, double vmin, double vmax,
                    uint32_t *counts) {
    pic::TraceRange trace_("pic_phase_space");
    if (!run || !counts || nx < 1 || nv < 1 || (long long)nx * nv > PIC_PHASE_MAX_BINS ||
        !(vmax > vmin) || !std::isfinite(vmin) || !std::isfinite(vmax))
        return PIC_EINVAL;
    if (!run->ready) return PIC_ESTATE;
    unsigned *d = run->at<unsigned>(run->lay.phase);
    const size_t bytes = (size_t)nx * nv * 4;
    PIC_CUDA(cudaMemsetAsync(d, 0, bytes, run->stream));
    // the bin rule on the stored positions: cell coordinates in the float32
    // modes (nx/NG), x in PIC_FP64 (nx/L)
    const float sx = (float)((double)nx / (run->p.precision == PIC_FP64 ? run->p.length
                                                                       : (double)run->p.ncell));
    const float sv = (float)((double)nv / (vmax - vmin));
    if (run->p.precision == PIC_FP64) {
        PhaseArgs<double> a{(const double *)run->xs(run->cur), (const double *)run->vs(run->cur),
                            run->p.npart, nx, nv, sx, (float)vmin, sv, d};
        PIC_CUDA(launch_phase(a, run->sms, run->stream));
    } else {
        PhaseArgs<float> a{(const float *)run->xs(run->cur), (const float *)run->vs(run->cur),
                           run->p.npart, nx, nv, sx, (float)vmin, sv, d};
        PIC_CUDA(launch_phase(a, run->sms, run->stream));
    }
    PIC_CUDA(cudaMemcpyAsync(counts, d, bytes, cudaMemcpyDeviceToHost, run->stream));
    PIC_CUDA(cudaStreamSynchronize(run->stream));
    return read_error_word(run);
}

int pic_device_arrays(pic_run *run, void **x, void **v, void **E32) {
    if (!run) return PIC_EINVAL;
    if (x) *x = run->xs(run->cur);
    if (v) *v = run->vs(run->cur);
    if (E32) *E32 = run->ws + run->lay.E32;
    return PIC_OK;
}

int pic_launch_shape(const pic_run *run, int32_t *grid, int32_t *block, int32_t *variant,
                     int32_t *unroll) {
    if (!run) return PIC_EINVAL;
    if (grid) *grid = run->grid;
    if (block) *block = run->block;
    if (variant) *variant = run->variant;
    if (unroll) *unroll = run->unroll;
    return PIC_OK;
}

int pic_set_launch(pic_run *run, int32_t variant, int32_t block, int32_t unroll,
                   int32_t blocks_per_sm) {
    if (!run) return PIC_EINVAL;
    if (run->pending_push) return PIC_ESTATE;
    const bool fixed = run->p.precision == PIC_FP32_FIXED;
    const bool ngp = run->p.shape == PIC_SHAPE_NGP;
    if (ngp && variant) return PIC_EINVAL;   // the shape fixes the deposit
    const int v = variant ? variant : run->variant;
    const int b = block ? block : run->block;
    const int u = unroll ? unroll : run->unroll;
    if (!ngp && (!is_variant(v) || (!fixed && v != PIC_DEPOSIT_ATOMIC)))
        return PIC_EINVAL;
    if (b < 32 || b % 32 || b > (fixed ? 512 : 1024)) return PIC_EINVAL;
    if ((u != 1 && u != 2 && u != 4) || (!fixed && u != 1)) return PIC_EINVAL;
    if (blocks_per_sm < 0 || blocks_per_sm > 32) return PIC_EINVAL;
    const int g = push_grid(run, v, b, u, blocks_per_sm);
    if (g < 1) return PIC_EINVAL;
    run->variant = v;
    run->block = b;
    run->unroll = u;
    run->grid = g;
    destroy_graphs(run);
    return PIC_OK;
}

int pic_autotune(pic_run *run, int32_t reps, pic_tune_entry *results,
                 int32_t max_results, int32_t *nresults) {
    pic::TraceRange trace_("pic_autotune");
    if (!run || reps < 1) return PIC_EINVAL;
    if (!run->ready || run->pending_push) return PIC_ESTATE;
    if (nresults) *nresults = 0;
    if (run->p.precision != PIC_FP32_FIXED) return PIC_OK;
    static const int variants[] = {PIC_DEPOSIT_ATOMIC, PIC_DEPOSIT_MATCH, PIC_DEPOSIT_QUAD,
                                   PIC_DEPOSIT_PAIR, PIC_DEPOSIT_QUAD8, PIC_DEPOSIT_PAIR8};
    static const int ngp_only[] = {kDepositNgp};
    static const int blocks[] = {128, 256, 512};
    static const int unrolls[] = {1, 2};
    const size_t bytes = (size_t)run->p.npart * run->elem();
    const int c = run->cur;
    cudaEvent_t ev[128];
    int made = 0;
    for (; made < 128; made++) {
        const cudaError_t ec = cudaEventCreate(&ev[made]);
        if (ec != cudaSuccess) {
            for (int i = 0; i < made; i++) cudaEventDestroy(ev[i]);
            return cuda_fail(ec);
        }
    }
    float best = 1e30f;
    int bv = run->variant, bb = run->block, bu = run->unroll, bg = run->grid, count = 0;
    int rc = PIC_OK;
    // A run that sorts every S steps spends each period drifting away from a
    // freshly sorted order (many lanes of a warp in one cell right after the
    // sort, spread apart later), so a candidate is timed over one period:
    // the copy is sorted, then pushed min(S, 64) times with the current
    // field, and the mean is minimised.  Without sorting, `reps` pushes of a
    // copy of the current order (which drifts as it is pushed).
    const int S = run->p.sort_interval;
    const int nrep = S > 0 ? (S < 64 ? S : 64) : (reps < 64 ? reps : 64);
    const bool ngp = run->p.shape == PIC_SHAPE_NGP;
    const int *vlist = ngp ? ngp_only : variants;
    const int nv = ngp ? 1 : (int)(sizeof(variants) / sizeof(variants[0]));
    for (int iv = 0; iv < nv; iv++)
        for (int b : blocks) {
            const int v = vlist[iv];
            for (int u : unrolls) {
                const int g = push_grid(run, v, b, u, run->p.blocks_per_sm);
                if (g < 1) continue;
                PushArgs a;
                a.x = (float *)run->xs(1 - c);
                a.v = (float *)run->vs(1 - c);
                a.n = run->p.npart;
                a.E32 = run->at<float>(run->lay.E32);
                a.rho_q = run->at<unsigned long long>(run->lay.tune_rho);
                a.partials = run->at<double>(run->lay.partials);
                a.err = &run->dev()->err;
                a.c = run->pc;
                cudaError_t e = cudaMemcpyAsync(a.x, run->xs(c), bytes, cudaMemcpyDeviceToDevice,
                                                run->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(a.v, run->vs(c), bytes, cudaMemcpyDeviceToDevice, run->stream);
                if (e == cudaSuccess) e = launch_push_fixed(a, g, b, v, u, true, run->stream);  // warm
                if (e == cudaSuccess && S > 0) e = enqueue_sort_into(run, c, run->stream);
                // the pushes go back to back, as in a run, and are read after
                for (int i = 0; i < nrep && e == cudaSuccess; i++) {
                    e = cudaEventRecord(ev[2 * i], run->stream);
                    if (e == cudaSuccess) e = launch_push_fixed(a, g, b, v, u, true, run->stream);
                    if (e == cudaSuccess) e = cudaEventRecord(ev[2 * i + 1], run->stream);
                }
                if (e == cudaSuccess) e = cudaStreamSynchronize(run->stream);
                float total = 0.0f;
                for (int i = 0; i < nrep && e == cudaSuccess; i++) {
                    float ms = 0.0f;
                    e = cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
                    total += ms;
                }
                if (e != cudaSuccess) { rc = cuda_fail(e); goto done; }
                const float med = total / (float)nrep;
                if (results && count < max_results) results[count] = pic_tune_entry{v, b, u, g, med};
                count++;
                if (med < best) { best = med; bv = v; bb = b; bu = u; bg = g; }
            }
        }
    run->variant = bv;
    run->block = bb;
    run->unroll = bu;
    run->grid = bg;
    destroy_graphs(run);
    if (nresults) *nresults = count < max_results || !results ? count : max_results;
done:
    for (int i = 0; i < made; i++) cudaEventDestroy(ev[i]);
    if (rc) return rc;
    PIC_CUDA(cudaMemsetAsync(run->ws + run->lay.tune_rho, 0, (size_t)run->p.ncell * 8, run->stream));
    return read_error_word(run);
}

int pic_set_shard(pic_run *run, int64_t npart_total) {
    if (!run) return PIC_EINVAL;
    if (run->p.precision != PIC_FP32_FIXED) return PIC_EINVAL;
    if (npart_total < run->p.npart || npart_total > ((int64_t)1 << 39)) return PIC_EINVAL;
    if (run->pending_push) return PIC_ESTATE;
    set_solve_constants(run, npart_total);
    destroy_graphs(run);
    return PIC_OK;
}

int pic_device_density(pic_run *run, void **rho_q) {
    if (!run || !rho_q) return PIC_EINVAL;
    if (run->p.precision != PIC_FP32_FIXED) return PIC_EINVAL;
    *rho_q = run->ws + run->lay.rho_q;
    return PIC_OK;
}

// Sort-interval tuner: the mean cost of a step's sort and push for each
// candidate S, modelled from measurements on a copy of the state.  The sort
// of the state into the idle buffer is timed, then the sorted copy is pushed
// kmax times with the current field (the particles drift apart as they do
// between sorts) and each push is timed: t(k), k pushes after a sort.  For
// S > 0 the cost is (t_sort + sum_{k<S} t(k)) / S; for S = 0 (never sort) it
// is the mean of the last quarter of t(k), the drifted state.  The run's own
// state is untouched (the copy's pushes deposit into the tuning density).
int pic_tune_sort_interval(pic_run *run, const int32_t *intervals, int32_t count,
                           float *ms_per_step, int32_t *best, int32_t adopt) {
    pic::TraceRange trace_("pic_tune_sort_interval");
    if (!run || !intervals || count < 1 || count > 64) return PIC_EINVAL;
    if (run->p.precision != PIC_FP32_FIXED) return PIC_EINVAL;
    int kmax = 8;
    for (int i = 0; i < count; i++) {
        if (intervals[i] < 0 || intervals[i] > 256) return PIC_EINVAL;
        if (intervals[i] > kmax) kmax = intervals[i];
    }
    if (!run->ready || run->pending_push) return PIC_ESTATE;
    const int c = run->cur;
    cudaEvent_t ev[2 * 257 + 2];
    const int nev = 2 * kmax + 2;
    int made = 0;
    int rc = PIC_OK;
    cudaError_t e = cudaSuccess;
    for (; made < nev && e == cudaSuccess; made++) e = cudaEventCreate(&ev[made]);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], run->stream);
    if (e == cudaSuccess) e = enqueue_sort_into(run, c, run->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], run->stream);
    PushArgs a;
    a.x = (float *)run->xs(1 - c);
    a.v = (float *)run->vs(1 - c);
    a.n = run->p.npart;
    a.E32 = run->at<float>(run->lay.E32);
    a.rho_q = run->at<unsigned long long>(run->lay.tune_rho);
    a.partials = run->at<double>(run->lay.partials);
    a.err = &run->dev()->err;
    a.c = run->pc;
    for (int k = 0; k < kmax && e == cudaSuccess; k++) {
        e = cudaEventRecord(ev[2 + 2 * k], run->stream);
        if (e == cudaSuccess)
            e = launch_push_fixed(a, run->grid, run->block, run->variant, run->unroll, true,
                                  run->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[3 + 2 * k], run->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(run->stream);
    float tsort = 0.0f, t[256];
    if (e == cudaSuccess) e = cudaEventElapsedTime(&tsort, ev[0], ev[1]);
    for (int k = 0; k < kmax && e == cudaSuccess; k++)
        e = cudaEventElapsedTime(&t[k], ev[2 + 2 * k], ev[3 + 2 * k]);
    if (e != cudaSuccess) rc = cuda_fail(e);
    for (int i = 0; i < made; i++) cudaEventDestroy(ev[i]);
    if (rc) return rc;
    float drift = 0.0f;
    const int q0 = kmax - kmax / 4;
    for (int k = q0; k < kmax; k++) drift += t[k];
    drift /= (float)(kmax - q0);
    int bi = 0;
    float bcost = 0.0f;
    for (int i = 0; i < count; i++) {
        const int S = intervals[i];
        float cost = drift;
        if (S > 0) {
            cost = tsort;
            for (int k = 0; k < S; k++) cost += t[k];
            cost /= (float)S;
        }
        if (ms_per_step) ms_per_step[i] = cost;
        if (i == 0 || cost < bcost) { bi = i; bcost = cost; }
    }
    if (best) *best = intervals[bi];
    if (adopt && run->p.sort_interval != intervals[bi]) {
        run->p.sort_interval = intervals[bi];
        destroy_graphs(run);
    }
    PIC_CUDA(cudaMemsetAsync(run->ws + run->lay.tune_rho, 0, (size_t)run->p.ncell * 8, run->stream));
    return read_error_word(run);
}

}  // extern "C"
