// ensemble.cu -- pools of independent runs advanced together by the batched
// cluster kernel (batch.cu): slot table, arena allocator, admission, the
// advance launches and result access.  The pool holds no device memory of
// its own: everything lives in the caller's arena.
//
// Arena layout: [descriptor table | order table | ticket + error word] then
// the runs, each a 256-byte-aligned block from a first-fit free list:
//   x[N], v[N] (float32), [x'[N], v'[N]: the sort's destination, when the run
//   sorts], E32[NG], E64[NG], phi[NG], rho[NG], rho_q_last[NG], history[H],
//   step counter.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "pic_internal.cuh"

using namespace pic;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct RunLayout {
    size_t x, v, xa, va, E32, E64, phi, rho, rq, hist, step, total;
};

RunLayout run_layout(const pic_params *p, int history) {
    RunLayout L;
    const size_t n = (size_t)p->npart, ng = (size_t)p->ncell;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b); return o; };
    L.x = take(4 * n);
    L.v = take(4 * n);
    L.xa = p->sort_interval > 0 ? take(4 * n) : 0;
    L.va = p->sort_interval > 0 ? take(4 * n) : 0;
    L.E32 = take(4 * ng);
    L.E64 = take(8 * ng);
    L.phi = take(8 * ng);
    L.rho = take(8 * ng);
    L.rq = take(8 * ng);
    L.hist = take((size_t)history * sizeof(pic_diag_row));
    L.step = take(8);
    L.total = off;
    return L;
}

struct TableLayout {
    size_t runs, order, scalars, total;
};

TableLayout table_layout(int max_slots) {
    TableLayout T;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b); return o; };
    T.runs = take((size_t)max_slots * sizeof(BatchRun));
    T.order = take((size_t)max_slots * sizeof(int));
    T.scalars = take(2 * sizeof(unsigned));
    T.total = off;
    return T;
}

int check_cfg(const pic_pool_config *c) {
    if (!c || c->max_slots < 1 || c->ncell_max < 1 || c->ncell_max > PIC_NCELL_MAX ||
        c->history < 1)
        return PIC_EINVAL;
    return PIC_OK;
}

// variant + 16 (two blocks per SM, 64 registers) is accepted too.
int check_shape(int code, int cluster, int block, int ncell_max) {
    const int variant = code & 15;
    if (code >> 4 > 1) return PIC_EINVAL;
    if (variant != PIC_DEPOSIT_ATOMIC && variant != PIC_DEPOSIT_MATCH && variant != PIC_DEPOSIT_QUAD &&
        variant != PIC_DEPOSIT_PAIR)
        return PIC_EINVAL;
    if (cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8) return PIC_EINVAL;
    if (block < 128 || block > 512 || block % 32) return PIC_EINVAL;
    const int P = (ncell_max + cluster - 1) / cluster;
    if (P > block) return PIC_EINVAL;   // one slice node per thread
    return PIC_OK;
}

int cuda_fail(cudaError_t e) {
    if (e == cudaSuccess) return PIC_OK;
    std::fprintf(stderr, "libpic: CUDA error %d: %s\n", (int)e, cudaGetErrorString(e));
    return PIC_ECUDA;
}

#define PIC_CUDA(call)                               \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

}  // namespace

struct pic_pool {
    pic_pool_config cfg{};
    cudaStream_t stream = nullptr;
    unsigned char *arena = nullptr;
    size_t arena_bytes = 0;
    TableLayout tab{};
    std::map<size_t, size_t> free_list;   // offset -> size
    size_t used = 0;
    struct Slot {
        bool used = false, needs_init = false;
        pic_params p{};
        size_t off = 0, size = 0;
        RunLayout lay{};
        BatchRun desc{};
        int64_t target = 0, done = 0;
        float *buf_x[2] = {nullptr, nullptr}, *buf_v[2] = {nullptr, nullptr};

        // The buffers holding the state after `done` steps: a sort precedes
        // every step n > 0 with n % S == 0, so floor((done - 1) / S) sorts
        // have run; each swaps the pair.
        void point_at_state() {
            const int S = p.sort_interval;
            const int cur = (S > 0 && done >= 1) ? (int)(((done - 1) / S) & 1) : 0;
            desc.x = buf_x[cur];
            desc.v = buf_v[cur];
            desc.xa = buf_x[1 - cur];
            desc.va = buf_v[1 - cur];
        }
    };
    std::vector<Slot> slots;
    std::vector<BatchRun> h_runs;
    std::vector<int> h_order;
    int variant = PIC_DEPOSIT_MATCH, cluster = 8, block = 256, nclusters = 1;
    int sms = 0;

    BatchRun *d_runs() const { return reinterpret_cast<BatchRun *>(arena + tab.runs); }
    int *d_order() const { return reinterpret_cast<int *>(arena + tab.order); }
    unsigned *d_next() const { return reinterpret_cast<unsigned *>(arena + tab.scalars); }
    unsigned *d_err() const { return d_next() + 1; }

    bool alloc(size_t bytes, size_t *off) {
        for (auto it = free_list.begin(); it != free_list.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t roff = it->first + bytes;
                free_list.erase(it);
                if (rest) free_list[roff] = rest;
                used += bytes;
                return true;
            }
        }
        return false;
    }

    void release(size_t off, size_t bytes) {
        used -= bytes;
        auto it = free_list.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_list.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_list.erase(nx);
        }
        if (it != free_list.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_list.erase(it);
            }
        }
    }
};

namespace {

int set_shape(pic_pool *pool, int variant, int cluster, int block) {
    int rc = check_shape(variant, cluster, block, pool->cfg.ncell_max);
    if (rc) return rc;
    const int nc = batch_max_clusters(variant, cluster, block, pool->cfg.ncell_max);
    if (nc < 1) return PIC_EINVAL;
    pool->variant = variant;
    pool->cluster = cluster;
    pool->block = block;
    pool->nclusters = nc;
    return PIC_OK;
}

// Upload the descriptors of `order` and launch one batched pass.
int launch(pic_pool *pool, const std::vector<int> &order, bool push) {
    if (order.empty()) return PIC_OK;
    for (size_t i = 0; i < order.size(); i++) pool->h_order[i] = order[i];
    for (int s : order) pool->h_runs[s] = pool->slots[s].desc;
    // the table is small; copy the whole of it
    PIC_CUDA(cudaMemcpyAsync(pool->d_runs(), pool->h_runs.data(),
                             pool->h_runs.size() * sizeof(BatchRun), cudaMemcpyHostToDevice,
                             pool->stream));
    PIC_CUDA(cudaMemcpyAsync(pool->d_order(), pool->h_order.data(), order.size() * sizeof(int),
                             cudaMemcpyHostToDevice, pool->stream));
    PIC_CUDA(cudaMemsetAsync(pool->d_next(), 0, sizeof(unsigned), pool->stream));
    BatchArgs a;
    a.runs = pool->d_runs();
    a.order = pool->d_order();
    a.nrun = (int)order.size();
    a.next = pool->d_next();
    a.err = pool->d_err();
    a.push = push ? 1 : 0;
    a.ng_max = pool->cfg.ncell_max;
    int nc = pool->nclusters;
    if (nc > (int)order.size()) nc = (int)order.size();
    PIC_CUDA(launch_batch(a, pool->variant, pool->cluster, pool->block, nc, pool->stream));
    // the copies above read pageable host memory: wait so the next launch
    // may rewrite the host tables
    PIC_CUDA(cudaStreamSynchronize(pool->stream));
    return PIC_OK;
}

bool slot_ok(const pic_pool *pool, int32_t slot) {
    return pool && slot >= 0 && slot < (int)pool->slots.size() && pool->slots[slot].used;
}

int read_error(pic_pool *pool) {
    unsigned err = 0;
    PIC_CUDA(cudaMemcpyAsync(&err, pool->d_err(), sizeof(err), cudaMemcpyDeviceToHost, pool->stream));
    PIC_CUDA(cudaStreamSynchronize(pool->stream));
    return err ? PIC_EDEVICE : PIC_OK;
}

}  // namespace

extern "C" {

int pic_pool_run_bytes(const pic_params *p, int32_t history, size_t *bytes) {
    if (!p || !bytes || history < 1) return PIC_EINVAL;
    int rc = validate_params(p);
    if (rc) return rc;
    if (p->precision != PIC_FP32_FIXED) return PIC_EINVAL;
    if (p->field_solver != PIC_SOLVER_EXACT || p->shape != PIC_SHAPE_CIC) return PIC_EINVAL;
    *bytes = run_layout(p, history).total;
    return PIC_OK;
}

int pic_pool_table_bytes(const pic_pool_config *cfg, size_t *bytes) {
    int rc = check_cfg(cfg);
    if (rc) return rc;
    if (!bytes) return PIC_EINVAL;
    *bytes = table_layout(cfg->max_slots).total;
    return PIC_OK;
}

int pic_pool_create(const pic_pool_config *cfg, void *arena, size_t arena_bytes, void *stream,
                    pic_pool **out) {
    if (!out) return PIC_EINVAL;
    *out = nullptr;
    int rc = check_cfg(cfg);
    if (rc) return rc;
    if (!arena || ((uintptr_t)arena % kAlign)) return PIC_EINVAL;
    const TableLayout T = table_layout(cfg->max_slots);
    if (arena_bytes < T.total) return PIC_ENOMEM;
    pic_pool *pool = new (std::nothrow) pic_pool();
    if (!pool) return PIC_ENOMEM;
    pool->cfg = *cfg;
    pool->arena = (unsigned char *)arena;
    pool->arena_bytes = arena_bytes;
    pool->stream = (cudaStream_t)stream;
    pool->tab = T;
    if (arena_bytes > T.total) pool->free_list[T.total] = arena_bytes - T.total;
    pool->slots.resize(cfg->max_slots);
    pool->h_runs.resize(cfg->max_slots);
    pool->h_order.resize(cfg->max_slots);
    std::memset(pool->h_runs.data(), 0, pool->h_runs.size() * sizeof(BatchRun));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&pool->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = batch_prepare_attributes();
    if (e != cudaSuccess) { delete pool; return cuda_fail(e); }
    rc = set_shape(pool, cfg->variant ? cfg->variant : PIC_DEPOSIT_MATCH,
                   cfg->cluster ? cfg->cluster : 8, cfg->block ? cfg->block : 256);
    if (rc) { delete pool; return rc; }
    e = cudaMemsetAsync(pool->arena + T.scalars, 0, 2 * sizeof(unsigned), pool->stream);
    if (e != cudaSuccess) { delete pool; return cuda_fail(e); }
    *out = pool;
    return PIC_OK;
}

void pic_pool_destroy(pic_pool *pool) { delete pool; }

int pic_pool_configure(pic_pool *pool, int32_t variant, int32_t cluster, int32_t block) {
    if (!pool) return PIC_EINVAL;
    return set_shape(pool, variant, cluster, block);
}

}  // extern "C"

namespace {

// Take a slot and arena space for a run; fill its descriptor; zero its
// counters.  The particles are written by the caller.
int admit_common(pic_pool *pool, const pic_params *p, int64_t steps, int32_t *slot) {
    int s = -1;
    for (int i = 0; i < (int)pool->slots.size(); i++)
        if (!pool->slots[i].used) { s = i; break; }
    if (s < 0) return PIC_ENOMEM;
    const RunLayout L = run_layout(p, pool->cfg.history);
    size_t off;
    if (!pool->alloc(L.total, &off)) return PIC_ENOMEM;
    pic_pool::Slot &sl = pool->slots[s];
    sl.used = true;
    sl.needs_init = true;
    sl.p = *p;
    sl.off = off;
    sl.size = L.total;
    sl.lay = L;
    sl.target = steps;
    sl.done = 0;
    unsigned char *base = pool->arena + off;
    BatchRun &d = sl.desc;
    sl.buf_x[0] = (float *)(base + L.x);
    sl.buf_v[0] = (float *)(base + L.v);
    sl.buf_x[1] = p->sort_interval > 0 ? (float *)(base + L.xa) : nullptr;
    sl.buf_v[1] = p->sort_interval > 0 ? (float *)(base + L.va) : nullptr;
    sl.point_at_state();
    d.sort_interval = p->sort_interval;
    d.n = p->npart;
    d.pc.ng = p->ncell;
    d.pc.ngf = (float)p->ncell;
    d.pc.kdrift = (float)(p->dt * (double)p->ncell / p->length);
    d.pc.qmdt = (float)(p->qm * p->dt);
    d.E32 = (float *)(base + L.E32);
    d.E64 = (double *)(base + L.E64);
    d.phi = (double *)(base + L.phi);
    d.rho = (double *)(base + L.rho);
    d.rho_q_last = (unsigned long long *)(base + L.rq);
    d.hist = (pic_diag_row *)(base + L.hist);
    d.hist_len = pool->cfg.history;
    d.steps = 0;
    d.step = (long long *)(base + L.step);
    d.weight_total = (long long)p->npart << kFixBits;
    d.dx = p->length / (double)p->ncell;
    const double q0 = (p->rho_ion * p->length / (double)p->npart) * (p->qm / std::fabs(p->qm));
    d.mass = q0 / p->qm;
    d.k_rho = p->rho_ion / std::ldexp((double)p->npart, kFixBits);
    d.k_e = 0.5 * d.dx * d.k_rho / (double)p->ncell;
    d.k_phi = -d.dx * d.dx * d.k_rho / (double)p->ncell;
    d.k_mode = 2.0 / (double)p->ncell;
    cudaError_t e = cudaMemsetAsync(d.step, 0, 8, pool->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.E32, 0, 4 * (size_t)p->ncell, pool->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d.hist, 0xFF, (size_t)pool->cfg.history * sizeof(pic_diag_row), pool->stream);
    if (e != cudaSuccess) {
        sl = pic_pool::Slot();
        pool->release(off, L.total);
        return cuda_fail(e);
    }
    *slot = s;
    return PIC_OK;
}

int check_admit(const pic_pool *pool, const pic_params *p) {
    int rc = validate_params(p);
    if (rc) return rc;
    if (p->precision != PIC_FP32_FIXED || p->ncell > pool->cfg.ncell_max) return PIC_EINVAL;
    if (p->field_solver != PIC_SOLVER_EXACT || p->shape != PIC_SHAPE_CIC) return PIC_EINVAL;
    return PIC_OK;
}

void drop_slot(pic_pool *pool, int s) {
    pic_pool::Slot &sl = pool->slots[s];
    pool->release(sl.off, sl.size);
    sl = pic_pool::Slot();
}

}  // namespace

extern "C" {

int pic_pool_admit(pic_pool *pool, const pic_params *p, const void *x0, const void *v0,
                   int64_t steps, int32_t *slot) {
    pic::TraceRange trace_("pic_pool_admit");
    if (!pool || !p || !x0 || !v0 || !slot || steps < 0) return PIC_EINVAL;
    *slot = -1;
    int rc = check_admit(pool, p);
    if (rc) return rc;
    const float Lf = (float)p->length;
    const float *xf = (const float *)x0;
    for (int64_t i = 0; i < p->npart; i++)
        if (!(xf[i] >= 0.0f && xf[i] < Lf)) return PIC_EINVAL;
    int32_t s;
    rc = admit_common(pool, p, steps, &s);
    if (rc) return rc;
    const BatchRun &d = pool->slots[s].desc;
    const size_t pb = (size_t)p->npart * 4;
    cudaError_t e = cudaMemcpyAsync(d.x, x0, pb, cudaMemcpyHostToDevice, pool->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.v, v0, pb, cudaMemcpyHostToDevice, pool->stream);
    if (e == cudaSuccess)
        e = launch_to_cells(d.x, p->npart, (double)p->ncell / p->length, (float)p->ncell, Lf,
                            pool->d_err(), pool->sms, pool->stream);
    if (e != cudaSuccess) { drop_slot(pool, s); return cuda_fail(e); }
    *slot = s;
    return PIC_OK;
}

int pic_pool_admit_loaded(pic_pool *pool, const pic_params *p, const pic_loading *ld,
                          int64_t steps, int32_t *slot) {
    pic::TraceRange trace_("pic_pool_admit_loaded");
    if (!pool || !p || !ld || !slot || steps < 0) return PIC_EINVAL;
    *slot = -1;
    int rc = check_admit(pool, p);
    if (rc) return rc;
    LoadArgs a;
    rc = make_load_args(ld, p->npart, p->length, (float *)pool->arena, (float *)pool->arena, &a);
    if (rc) return rc;
    int32_t s;
    rc = admit_common(pool, p, steps, &s);
    if (rc) return rc;
    a.x = pool->slots[s].desc.x;
    a.v = pool->slots[s].desc.v;
    cudaError_t e = launch_load(a, pool->sms, pool->stream);
    if (e == cudaSuccess)
        e = launch_to_cells(a.x, p->npart, (double)p->ncell / p->length, (float)p->ncell,
                            (float)p->length, pool->d_err(), pool->sms, pool->stream);
    if (e != cudaSuccess) { drop_slot(pool, s); return cuda_fail(e); }
    *slot = s;
    return PIC_OK;
}

int pic_pool_advance(pic_pool *pool, int64_t k, int32_t *active) {
    pic::TraceRange trace_("pic_pool_advance");
    if (!pool || k < 0) return PIC_EINVAL;
    if (active) *active = 0;
    std::vector<int> order;
    for (int i = 0; i < (int)pool->slots.size(); i++)
        if (pool->slots[i].used && pool->slots[i].needs_init) order.push_back(i);
    if (!order.empty()) {
        std::sort(order.begin(), order.end(), [&](int a, int b) {
            return pool->slots[a].p.npart > pool->slots[b].p.npart;
        });
        int rc = launch(pool, order, false);
        if (rc) return rc;
        for (int i : order) pool->slots[i].needs_init = false;
    }
    if (k == 0) return PIC_OK;
    order.clear();
    for (int i = 0; i < (int)pool->slots.size(); i++) {
        pic_pool::Slot &sl = pool->slots[i];
        if (!sl.used) continue;
        const int64_t left = sl.target - sl.done;
        const int64_t take = left < k ? left : k;
        // one launch advances at most INT_MAX steps (the descriptor's int)
        sl.desc.steps = (int)(take > INT_MAX ? INT_MAX : take);
        if (sl.desc.steps > 0) order.push_back(i);
    }
    // longest work first (particles x steps)
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        const double wa = (double)pool->slots[a].p.npart * pool->slots[a].desc.steps;
        const double wb = (double)pool->slots[b].p.npart * pool->slots[b].desc.steps;
        return wa > wb;
    });
    int rc = launch(pool, order, true);
    if (rc) return rc;
    for (int i : order) {
        pool->slots[i].done += pool->slots[i].desc.steps;
        pool->slots[i].point_at_state();
    }
    if (active) *active = (int32_t)order.size();
    return PIC_OK;
}

int pic_pool_finished(const pic_pool *pool, int32_t *slots, int32_t max, int32_t *n) {
    if (!pool || !n || max < 0) return PIC_EINVAL;
    int c = 0;
    for (int i = 0; i < (int)pool->slots.size(); i++) {
        const pic_pool::Slot &sl = pool->slots[i];
        if (sl.used && !sl.needs_init && sl.done >= sl.target) {
            if (slots && c < max) slots[c] = i;
            c++;
        }
    }
    *n = c;
    return PIC_OK;
}

int pic_pool_step_count(const pic_pool *pool, int32_t slot, int64_t *step) {
    if (!slot_ok(pool, slot) || !step) return PIC_EINVAL;
    *step = pool->slots[slot].done;
    return PIC_OK;
}

int pic_pool_get_cells(pic_pool *pool, int32_t slot, float *u, float *v) {
    pic::TraceRange trace_("pic_pool_get_cells");
    if (!slot_ok(pool, slot)) return PIC_EINVAL;
    const pic_pool::Slot &sl = pool->slots[slot];
    if (sl.needs_init) return PIC_ESTATE;
    const size_t pb = (size_t)sl.p.npart * 4;
    if (u) PIC_CUDA(cudaMemcpyAsync(u, sl.desc.x, pb, cudaMemcpyDeviceToHost, pool->stream));
    if (v) PIC_CUDA(cudaMemcpyAsync(v, sl.desc.v, pb, cudaMemcpyDeviceToHost, pool->stream));
    return read_error(pool);
}

int pic_pool_get_state(pic_pool *pool, int32_t slot, void *x, void *v) {
    pic::TraceRange trace_("pic_pool_get_state");
    int rc = pic_pool_get_cells(pool, slot, (float *)x, (float *)v);
    if (rc || !x) return rc;
    // cell coordinates to physical positions on the host, with the same two
    // float64-rounded steps as the device conversion of a single run
    const pic_pool::Slot &sl = pool->slots[slot];
    const double to_phys = sl.p.length / (double)sl.p.ncell;
    const float top = below((float)sl.p.length);
    float *xf = (float *)x;
    for (int64_t i = 0; i < sl.p.npart; i++) {
        const float xi = (float)((double)xf[i] * to_phys);
        xf[i] = xi > top ? top : xi;
    }
    return PIC_OK;
}

int pic_pool_get_field(pic_pool *pool, int32_t slot, double *rho, double *phi, double *E,
                       int64_t *rho_q) {
    pic::TraceRange trace_("pic_pool_get_field");
    if (!slot_ok(pool, slot)) return PIC_EINVAL;
    const pic_pool::Slot &sl = pool->slots[slot];
    if (sl.needs_init) return PIC_ESTATE;
    const size_t nb = (size_t)sl.p.ncell * 8;
    if (rho) PIC_CUDA(cudaMemcpyAsync(rho, sl.desc.rho, nb, cudaMemcpyDeviceToHost, pool->stream));
    if (phi) PIC_CUDA(cudaMemcpyAsync(phi, sl.desc.phi, nb, cudaMemcpyDeviceToHost, pool->stream));
    if (E) PIC_CUDA(cudaMemcpyAsync(E, sl.desc.E64, nb, cudaMemcpyDeviceToHost, pool->stream));
    if (rho_q)
        PIC_CUDA(cudaMemcpyAsync(rho_q, sl.desc.rho_q_last, nb, cudaMemcpyDeviceToHost, pool->stream));
    return read_error(pool);
}

int pic_pool_diagnostics(pic_pool *pool, int32_t slot, int64_t first, int32_t count,
                         pic_diag_row *rows) {
    pic::TraceRange trace_("pic_pool_diagnostics");
    if (!slot_ok(pool, slot) || !rows || count < 0 || first < 0) return PIC_EINVAL;
    const pic_pool::Slot &sl = pool->slots[slot];
    const int64_t H = pool->cfg.history;
    if (count == 0) return PIC_OK;
    if (first + count - 1 > sl.done || first < sl.done - H + 1) return PIC_EINVAL;
    int64_t got = 0;
    while (got < count) {
        const int64_t pos = (first + got) % H;
        int64_t len = count - got;
        if (pos + len > H) len = H - pos;
        PIC_CUDA(cudaMemcpyAsync(rows + got, sl.desc.hist + pos, (size_t)len * sizeof(pic_diag_row),
                                 cudaMemcpyDeviceToHost, pool->stream));
        got += len;
    }
    return read_error(pool);
}

int pic_pool_release(pic_pool *pool, int32_t slot) {
    if (!slot_ok(pool, slot)) return PIC_EINVAL;
    pic_pool::Slot &sl = pool->slots[slot];
    // the arena space may be reused by the next admission: its uploads are
    // stream-ordered after every launch already enqueued
    pool->release(sl.off, sl.size);
    sl = pic_pool::Slot();
    return PIC_OK;
}

int pic_pool_sync(pic_pool *pool) {
    if (!pool) return PIC_EINVAL;
    PIC_CUDA(cudaStreamSynchronize(pool->stream));
    return read_error(pool);
}

int pic_pool_usage(const pic_pool *pool, size_t *used, size_t *largest_free) {
    if (!pool) return PIC_EINVAL;
    if (used) *used = pool->used;
    if (largest_free) {
        size_t m = 0;
        for (auto &kv : pool->free_list) m = kv.second > m ? kv.second : m;
        *largest_free = m;
    }
    return PIC_OK;
}

}  // extern "C"
