// push.cu -- the fused particle kernel of one PIC step: field gather (Sec.
// 2.3), velocity update (Sec. 2.1, Eq. 3), position update and periodic wrap
// (Sec. 2.1, Eq. 2; Appendix A wrap), and the charge deposit of the new
// positions (Sec. 2.3).
//
// Design (GB300): one persistent grid of (SMs x resident blocks), each block
// streaming float4 groups of 4 particles (x and v are separate float32 arrays,
// 16 B loads and stores, streaming cache hints: the particle arrays are read
// and written once per step and do not fit in L2).  The block stages E in
// shared memory and accumulates a private density tile there; the tile is
// added to the global density with one 64-bit atomic per non-zero node when
// the block ends.  The deposit is exact integer arithmetic (2^-24 fractions
// of a particle), so the density is the same integer whatever the launch
// shape, the particle order or the deposit variant.
//
// Deposit variants (all give the same integers):
//   ATOMIC        two shared-memory atomics per particle;
//   MATCH         lanes of a warp whose particles share a left node are
//                 grouped by __match_any_sync; the group's weights are summed
//                 by __reduce_add_sync and its first lane does two atomics;
//   PACKED        one atomic per particle on a packed (count << 40 | sum W)
//                 word per left node, unpacked when the tile is flushed;
//   MATCH_PACKED  the two combined: one atomic per warp group;
//   QUAD          runs of equal left node among a thread's 4 particles are
//                 summed in registers, then two atomics per run;
//   PAIR          the same with two open runs, so that particles of two
//                 interleaved cells (the two beams before the first sort)
//                 still combine.
// The nearest-grid-point shape (PIC_SHAPE_NGP) uses the same loop with the
// NGP gather and a QUAD-style deposit of whole particles to the cell's node.
// The packed forms flush the tile to global memory before any node can hold
// 2^16 particles, so the 40-bit weight field never carries into the count.
// The unpacked tiles hold exact 64-bit sums in two 32-bit words (below).
#include "particle_ops.cuh"

namespace pic {
namespace {


// Add the block's tile to the global density and clear it (ghost nodes
// folded onto their periodic images).
template <bool PACKED>
__device__ __forceinline__ void flush_tile(const Tile &t, u64 *rho_q, int ng) {
    __syncthreads();
    const int top = PACKED ? ng : ng + 1;     // last used tile index
    for (int j = threadIdx.x; j <= top; j += blockDim.x) {
        const int left = j == 0 ? ng - 1 : j - 1;      // node of index j
        if (PACKED) {
            const u64 w = t.packed[j];
            if (w == 0) continue;
            t.packed[j] = 0;
            const u64 cnt = w >> kPackShift, sw = w & kPackMask;
            const u64 lw = cnt * kFixOne - sw;
            const int right = j == ng ? 0 : j;
            if (lw) atomicAdd(&rho_q[left], lw);
            if (sw) atomicAdd(&rho_q[right], sw);
        } else {
            const u64 w = ((u64)t.hi[j] << 32) | (u64)t.lo[j];
            if (w == 0) continue;
            t.lo[j] = 0u;
            t.hi[j] = 0u;
            atomicAdd(&rho_q[j == ng + 1 ? 0 : left], w);
        }
    }
    __syncthreads();
}

// Sum two per-thread values over the block in a fixed order; thread 0 gets it.
__device__ __forceinline__ void block_sum2(double &a, double &b, double *scratch) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(kFull, a, o);
        b += __shfl_down_sync(kFull, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = (blockDim.x + 31) >> 5;
    if (lane == 0) { scratch[2 * w] = a; scratch[2 * w + 1] = b; }
    __syncthreads();
    if (w == 0) {
        a = lane < nw ? scratch[2 * lane] : 0.0;
        b = lane < nw ? scratch[2 * lane + 1] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(kFull, a, o);
            b += __shfl_down_sync(kFull, b, o);
        }
    }
}

// One block-iteration covers U*blockDim consecutive float4 groups; thread t
// takes groups q0 + u*blockDim + t (coalesced for each u).  The next
// iteration's groups are loaded before the current ones are processed.
template <int VARIANT, bool PUSH, int U>
__global__ void __launch_bounds__(512) pic_push_fixed_kernel(PushArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[64];
    constexpr bool kPacked = VARIANT == PIC_DEPOSIT_PACKED || VARIANT == kMatchPacked;
    const PushConsts c = a.c;
    const int ng = c.ng;
    Tile tile;                                                       // 8 (ng + 2) B
    tile.packed = reinterpret_cast<u64 *>(smem_raw);
    tile.lo = reinterpret_cast<unsigned *>(smem_raw);
    tile.hi = tile.lo + ng + 2;
    float *sE = reinterpret_cast<float *>(smem_raw + 8 * (ng + 2));  // ng + 2
    const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31;
    for (int j = tid; j < ng + 2; j += bs) {
        tile.packed[j] = 0;
        if (PUSH) sE[j] = a.E32[j == 0 ? ng - 1 : (j == ng + 1 ? 0 : j - 1)];
    }
    __syncthreads();

    float ke = 0.0f, mom = 0.0f;
    const long long n4 = a.n >> 2;
    float4 *x4 = reinterpret_cast<float4 *>(a.x);
    float4 *v4 = reinterpret_cast<float4 *>(a.v);
    const long long span = (long long)bs * U;
    const long long stride = (long long)gridDim.x * span;
    const int flush_every = kPacked ? max(1, kPackLimit / (int)(4 * span)) : 0;
    int since_flush = 0;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 cx[U], cv[U];
    long long q0 = (long long)blockIdx.x * span;
#pragma unroll
    for (int u = 0; u < U; u++) {
        const long long q = q0 + u * bs + tid;
        cx[u] = q < n4 ? __ldcs(x4 + q) : zero4;
        cv[u] = (PUSH && q < n4) ? __ldcs(v4 + q) : zero4;
    }
    // The trip count is uniform over the block (q0 is), so the packed flush
    // may synchronise inside the loop and every warp is converged for match.
    for (; q0 < n4; q0 += stride) {
        float4 nx[U], nv[U];
        const long long q1 = q0 + stride;
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long q = q1 + u * bs + tid;
            nx[u] = q < n4 ? __ldcs(x4 + q) : zero4;
            nv[u] = (PUSH && q < n4) ? __ldcs(v4 + q) : zero4;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long q = q0 + u * bs + tid;
            const bool valid = q < n4;
            float4 xx = cx[u], vv = cv[u];
            if (PUSH && valid) {
                if (VARIANT == kDepositNgp) {
                    push_particle_ngp(xx.x, vv.x, sE, c, ke, mom);
                    push_particle_ngp(xx.y, vv.y, sE, c, ke, mom);
                    push_particle_ngp(xx.z, vv.z, sE, c, ke, mom);
                    push_particle_ngp(xx.w, vv.w, sE, c, ke, mom);
                } else {
                    push_particle(xx.x, vv.x, sE, c, ke, mom);
                    push_particle(xx.y, vv.y, sE, c, ke, mom);
                    push_particle(xx.z, vv.z, sE, c, ke, mom);
                    push_particle(xx.w, vv.w, sE, c, ke, mom);
                }
            }
            deposit4<VARIANT>(tile, xx, valid, c, a.err, lane);
            if (PUSH && valid) {
                __stcs(x4 + q, xx);
                __stcs(v4 + q, vv);
            }
        }
        if (kPacked && ++since_flush == flush_every) {
            flush_tile<true>(tile, a.rho_q, ng);
            since_flush = 0;
        }
#pragma unroll
        for (int u = 0; u < U; u++) { cx[u] = nx[u]; cv[u] = nv[u]; }
    }
    // The last N mod 4 particles: warp 0 of block 0, converged.
    if (blockIdx.x == 0 && tid < 32) {
        const long long i = n4 * 4 + lane;
        const bool valid = i < a.n;
        float xs = valid ? a.x[i] : 0.0f, vs = valid && PUSH ? a.v[i] : 0.0f;
        if (PUSH && valid) {
            if (VARIANT == kDepositNgp) push_particle_ngp(xs, vs, sE, c, ke, mom);
            else push_particle(xs, vs, sE, c, ke, mom);
        }
        deposit_one<VARIANT>(tile, xs, valid, c, a.err, lane);
        if (PUSH && valid) { a.x[i] = xs; a.v[i] = vs; }
    }
    if (PUSH) {
        double dke = ke, dmom = mom;
        __syncthreads();
        block_sum2(dke, dmom, red);
        if (tid == 0) {
            a.partials[2 * blockIdx.x] = dke;
            a.partials[2 * blockIdx.x + 1] = dmom;
        }
    }
    flush_tile<kPacked>(tile, a.rho_q, ng);
}

// ---- the fused push with bulk-copy tiles (PIC_DEPOSIT_QUAD_BULK) ----------
//
// The same per-particle work (QUAD deposit), with the particle arrays moved
// between HBM and shared memory by the Tensor Memory Accelerator's bulk copies
// instead of per-thread loads and stores.  A block walks tiles of 2048
// particles (one float4 of x and of v per thread), tile blockIdx.x + k grid.
// kBulkStages tiles are in flight: one thread issues the two bulk loads of a
// tile into a stage, with the stage's mbarrier counting the bytes; the block
// waits on the barrier, pushes and deposits in shared memory, writes the
// results back in place, and the same thread bulk-stores the stage to HBM.
// A stage is refilled one tile later, once its store has read it
// (cp.async.bulk.wait_group.read 1), so the issuing thread rarely waits.
// Every wait is bounded by a clock budget: a barrier that never completes sets
// kErrTimeout and the block stops.  The last n mod 2048 particles go through
// the per-thread path in block 0.
constexpr int kBulkThreads = 512;
constexpr int kBulkTile = kBulkThreads * 4;            // particles per tile
constexpr unsigned kBulkBytes = kBulkTile * 4;         // bytes per array per tile
constexpr int kBulkStages = 3;
constexpr long long kBulkSpinCycles = 2000000000ll;    // ~1 s at 2 GHz

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}

// false when the phase of `parity` did not complete within the clock budget
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kBulkSpinCycles) return false;
    return true;
}

__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, unsigned bytes,
                                          unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_store(void *dst, const void *src_smem, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_1() {
    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The two bulk loads of tile t into stage buffer st (x then v), counted by bar.
__device__ __forceinline__ void load_tile(const PushArgs &a, float *st, long long t,
                                          unsigned long long *bar) {
    mbar_expect_tx(bar, 2 * kBulkBytes);
    bulk_load(st, a.x + t * kBulkTile, kBulkBytes, bar);
    bulk_load(st + kBulkTile, a.v + t * kBulkTile, kBulkBytes, bar);
}

__global__ void __launch_bounds__(kBulkThreads) pic_push_bulk_kernel(PushArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[kBulkStages];
    __shared__ double red[64];
    const PushConsts c = a.c;
    const int ng = c.ng;
    float *stage = reinterpret_cast<float *>(smem_raw);   // kBulkStages x (x tile, v tile)
    float *sE = stage + (size_t)kBulkStages * 2 * kBulkTile;
    Tile tile;
    tile.lo = reinterpret_cast<unsigned *>(sE + ng + 2);
    tile.hi = tile.lo + ng + 2;
    tile.packed = nullptr;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int j = tid; j < ng + 2; j += kBulkThreads) {
        tile.lo[j] = 0u;
        tile.hi[j] = 0u;
        sE[j] = a.E32[j == 0 ? ng - 1 : (j == ng + 1 ? 0 : j - 1)];
    }
    if (tid == 0) {
        for (int s = 0; s < kBulkStages; s++) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const long long ntiles = a.n / kBulkTile;
    const long long G = gridDim.x;
    if (tid == 0)
        for (int s = 0; s < kBulkStages; s++) {
            const long long t = blockIdx.x + s * G;
            if (t < ntiles) load_tile(a, stage + (size_t)s * 2 * kBulkTile, t, &full[s]);
        }
    float ke = 0.0f, mom = 0.0f;
    bool failed = false;
    long long k = 0;
    for (;; k++) {
        const long long t = blockIdx.x + k * G;
        if (t >= ntiles) break;
        const int s = (int)(k % kBulkStages);
        float *st = stage + (size_t)s * 2 * kBulkTile;
        const bool arrived = mbar_wait(&full[s], (unsigned)((k / kBulkStages) & 1));
        if (__syncthreads_or(!arrived)) { failed = true; break; }
        float4 *x4 = reinterpret_cast<float4 *>(st);
        float4 *v4 = reinterpret_cast<float4 *>(st + kBulkTile);
        float4 xx = x4[tid], vv = v4[tid];
        push_particle(xx.x, vv.x, sE, c, ke, mom);
        push_particle(xx.y, vv.y, sE, c, ke, mom);
        push_particle(xx.z, vv.z, sE, c, ke, mom);
        push_particle(xx.w, vv.w, sE, c, ke, mom);
        deposit4<PIC_DEPOSIT_QUAD>(tile, xx, true, c, a.err, lane);
        x4[tid] = xx;
        v4[tid] = vv;
        fence_proxy_async();            // the results, visible to the bulk store
        __syncthreads();
        if (tid == 0) {
            bulk_store(a.x + t * kBulkTile, st, kBulkBytes);
            bulk_store(a.v + t * kBulkTile, st + kBulkTile, kBulkBytes);
            bulk_commit();
            if (k >= 1) {
                // the stage of tile k-1: its store (the older group) has read it
                bulk_wait_read_1();
                const long long tn = blockIdx.x + (k - 1 + kBulkStages) * G;
                const int sp = (int)((k - 1) % kBulkStages);
                if (tn < ntiles) load_tile(a, stage + (size_t)sp * 2 * kBulkTile, tn, &full[sp]);
            }
        }
    }
    if (tid == 0) {
        bulk_wait_all();
        if (failed) {
            atomicOr(a.err, kErrTimeout);
            // let the loads still in flight land before the block's memory
            // goes: tiles k .. k+S-1 after the prologue, k .. k+S-2 later
            const long long kend = k + (k == 0 ? kBulkStages : kBulkStages - 1);
            for (long long kk = k; kk < kend; kk++) {
                const long long t = blockIdx.x + kk * G;
                if (t >= ntiles) break;
                mbar_wait(&full[kk % kBulkStages], (unsigned)((kk / kBulkStages) & 1));
            }
        }
    }
    // the last n mod kBulkTile particles: block 0, four per thread
    if (blockIdx.x == 0 && !failed) {
        const long long i0 = ntiles * kBulkTile + (long long)tid * 4;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const long long i = i0 + j;
            const bool valid = i < a.n;
            float xs = valid ? a.x[i] : 0.0f, vs = valid ? a.v[i] : 0.0f;
            if (valid) push_particle(xs, vs, sE, c, ke, mom);
            deposit_one<PIC_DEPOSIT_QUAD>(tile, xs, valid, c, a.err, lane);
            if (valid) { a.x[i] = xs; a.v[i] = vs; }
        }
    }
    double dke = ke, dmom = mom;
    __syncthreads();
    block_sum2(dke, dmom, red);
    if (tid == 0) {
        a.partials[2 * blockIdx.x] = dke;
        a.partials[2 * blockIdx.x + 1] = dmom;
    }
    flush_tile<false>(tile, a.rho_q, ng);
}

// ---- float32 push with float32 atomic deposit (precision study) -------------

template <bool PUSH>
__global__ void __launch_bounds__(1024) pic_push_f32atomic_kernel(PushArgsF32Atomic a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[64];
    const PushConsts c = a.c;
    const int ng = c.ng;
    float *sRho = reinterpret_cast<float *>(smem_raw);   // ng + 2, ghost-padded
    float *sE = sRho + ng + 2;                            // ng + 2, ghost-padded
    const int tid = threadIdx.x, bs = blockDim.x;
    for (int j = tid; j < ng + 2; j += bs) {
        sRho[j] = 0.0f;
        if (PUSH) sE[j] = a.E32[j == 0 ? ng - 1 : (j == ng + 1 ? 0 : j - 1)];
    }
    __syncthreads();
    float ke = 0.0f, mom = 0.0f;
    const long long stride = (long long)gridDim.x * bs;
    for (long long i = (long long)blockIdx.x * bs + tid; i < a.n; i += stride) {
        float x = a.x[i], v = PUSH ? a.v[i] : 0.0f;
        if (PUSH) push_particle(x, v, sE, c, ke, mom);
        const Loc l = locate(x, c.inv_dx);
        if (l.j <= (unsigned)ng) {
            atomicAdd(&sRho[l.j], 1.0f - l.f);
            atomicAdd(&sRho[l.j + 1], l.f);
        } else {
            atomicOr(a.err, kErrPosition);
        }
        if (PUSH) { a.x[i] = x; a.v[i] = v; }
    }
    if (PUSH) {
        double dke = ke, dmom = mom;
        __syncthreads();
        block_sum2(dke, dmom, red);
        if (tid == 0) {
            a.partials[2 * blockIdx.x] = dke;
            a.partials[2 * blockIdx.x + 1] = dmom;
        }
    }
    __syncthreads();
    for (int j = tid; j < ng + 2; j += bs) {
        const float t = sRho[j];
        if (t == 0.0f) continue;
        const int node = j == 0 ? ng - 1 : (j == ng + 1 ? 0 : j - 1);
        atomicAdd(&a.rho_acc[node], t);
    }
}

// ---- float64 push with float64 atomic deposit (precision study) ------------

template <bool PUSH>
__global__ void __launch_bounds__(1024) pic_push_f64_kernel(PushArgs64 a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[64];
    double *sRho = reinterpret_cast<double *>(smem_raw);
    double *sE = sRho + a.ng;
    const int tid = threadIdx.x, bs = blockDim.x, ng = a.ng;
    for (int g = tid; g < ng; g += bs) {
        sRho[g] = 0.0;
        if (PUSH) sE[g] = a.E64[g];
    }
    __syncthreads();
    double ke = 0.0, mom = 0.0;
    const long long stride = (long long)gridDim.x * bs;
    const int lane = tid & 31;
    // the trip count is uniform over a warp (base is), so every lane takes
    // part in the deposit's shuffles
    for (long long base = (long long)blockIdx.x * bs + (tid & ~31); base < a.n; base += stride) {
        const long long i = base + lane;
        const bool valid = i < a.n;
        double x = valid ? a.x[i] : 0.0;
        double s = x * a.inv_dx - 0.5;
        double fl = floor(s);
        bool ok = valid && fl >= -1.0 && fl <= (double)(ng - 1);
        if (PUSH && valid) {
            double v = a.v[i];
            int j = ok ? (int)fl : 0;
            int il = j < 0 ? j + ng : j, ir = j + 1 >= ng ? j + 1 - ng : j + 1;
            double f = s - fl;
            double ep = ok ? (1.0 - f) * sE[il] + f * sE[ir] : 0.0;
            double vn = v + a.qmdt * ep;
            ke += v * vn;
            mom += vn;
            x = x + vn * a.dt;
            if (x < 0.0) x += a.length;
            else if (x >= a.length) x -= a.length;
            if (x >= a.length) x = 0.0;
            a.x[i] = x;
            a.v[i] = vn;
            s = x * a.inv_dx - 0.5;
            fl = floor(s);
            ok = fl >= -1.0 && fl <= (double)(ng - 1);
        }
        // Deposit.  Lanes with equal left node in a row (particles in
        // lattice or sorted order share nodes) first add their weights in a
        // segmented shuffle sum, and the segment's first lane does the two
        // adds; a float64 add on shared memory is a compare-and-swap loop,
        // which lanes hitting one node would otherwise serialise.
        const int j = ok ? (int)fl : 0;
        const int il = j < 0 ? j + ng : j, ir = j + 1 >= ng ? j + 1 - ng : j + 1;
        const double f = s - fl;
        const unsigned key = ok ? (unsigned)il : 0xffffffffu;
        const unsigned kprev = __shfl_up_sync(kFull, key, 1);
        const bool head = ok && (lane == 0 || kprev != key);
        const unsigned heads = __ballot_sync(kFull, head || !ok);
        const unsigned above = lane == 31 ? 0u : heads & (0xffffffffu << (lane + 1));
        const int end = above ? __ffs(above) - 1 : 32;       // this lane's segment ends before
        double sl = ok ? 1.0 - f : 0.0, sr = ok ? f : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double tl = __shfl_down_sync(kFull, sl, o);
            const double tr = __shfl_down_sync(kFull, sr, o);
            if (lane + o < end) {
                sl += tl;
                sr += tr;
            }
        }
        if (head) {
            atomicAdd(&sRho[il], sl);
            atomicAdd(&sRho[ir], sr);
        }
        if (valid && !ok) atomicOr(a.err, kErrPosition);
    }
    if (PUSH) {
        __syncthreads();
        block_sum2(ke, mom, red);
        if (tid == 0) {
            a.partials[2 * blockIdx.x] = ke;
            a.partials[2 * blockIdx.x + 1] = mom;
        }
    }
    __syncthreads();
    for (int g = tid; g < ng; g += bs)
        if (sRho[g] != 0.0) atomicAdd(&a.rho_acc[g], sRho[g]);
}

using FixedKernel = void (*)(PushArgs);

template <int V>
FixedKernel pick_unroll(bool push, int unroll) {
    if (!push) return &pic_push_fixed_kernel<V, false, 1>;
    switch (unroll) {
        case 1: return &pic_push_fixed_kernel<V, true, 1>;
        case 2: return &pic_push_fixed_kernel<V, true, 2>;
        case 4: return &pic_push_fixed_kernel<V, true, 4>;
        default: return nullptr;
    }
}

FixedKernel pick_fixed(int variant, bool push, int unroll) {
    switch (variant) {
        case PIC_DEPOSIT_ATOMIC: return pick_unroll<PIC_DEPOSIT_ATOMIC>(push, unroll);
        case PIC_DEPOSIT_MATCH: return pick_unroll<PIC_DEPOSIT_MATCH>(push, unroll);
        case PIC_DEPOSIT_PACKED: return pick_unroll<PIC_DEPOSIT_PACKED>(push, unroll);
        case kMatchPacked: return pick_unroll<kMatchPacked>(push, unroll);
        case PIC_DEPOSIT_QUAD: return pick_unroll<PIC_DEPOSIT_QUAD>(push, unroll);
        case PIC_DEPOSIT_PAIR: return pick_unroll<PIC_DEPOSIT_PAIR>(push, unroll);
        case PIC_DEPOSIT_QUAD_BULK:
            // the deposit-only pass has nothing to stream back: QUAD's kernel
            if (!push) return pick_unroll<PIC_DEPOSIT_QUAD>(false, 1);
            return unroll == 1 ? &pic_push_bulk_kernel : nullptr;
        case kDepositNgp: return pick_unroll<kDepositNgp>(push, unroll);
        default: return nullptr;
    }
}

}  // namespace

size_t push_smem_bytes(int mode, int ng) {
    if (mode == PIC_FP64) return (size_t)ng * 16;
    if (mode == PIC_FP32_ATOMIC) return (size_t)(ng + 2) * 8;
    return (size_t)(ng + 2) * 12;
}

// Shared memory of a fused fixed-point push launch (the bulk kernel adds its
// tile stages).
size_t fixed_smem_bytes(int variant, bool push, int ng) {
    const size_t base = push_smem_bytes(PIC_FP32_FIXED, ng);
    if (variant == PIC_DEPOSIT_QUAD_BULK && push)
        return base + (size_t)kBulkStages * 2 * kBulkBytes;
    return base;
}

cudaError_t push_prepare_attributes(int mode, int ng) {
    const int bytes = (int)push_smem_bytes(mode, PIC_NCELL_MAX);
    (void)ng;
    cudaError_t e = cudaSuccess;
    if (mode == PIC_FP32_FIXED) {
        const int unrolls[3] = {1, 2, 4};
        const int fixed_variants[] = {PIC_DEPOSIT_ATOMIC, PIC_DEPOSIT_MATCH, PIC_DEPOSIT_PACKED,
                                      PIC_DEPOSIT_MATCH_PACKED, PIC_DEPOSIT_QUAD, PIC_DEPOSIT_PAIR,
                                      PIC_DEPOSIT_QUAD_BULK, kDepositNgp};
        for (int v : fixed_variants)
            for (int p = 0; p < 2; p++)
                for (int u : unrolls) {
                    FixedKernel k = pick_fixed(v, p != 0, u);
                    if (!k) continue;
                    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)fixed_smem_bytes(v, p != 0, PIC_NCELL_MAX));
                    if (e != cudaSuccess) return e;
                }
    } else if (mode == PIC_FP32_ATOMIC) {
        e = cudaFuncSetAttribute(&pic_push_f32atomic_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(&pic_push_f32atomic_kernel<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    } else {
        e = cudaFuncSetAttribute(&pic_push_f64_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(&pic_push_f64_kernel<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    }
    return e;
}

int push_max_blocks_per_sm(int mode, int variant, int unroll, int block, int ng) {
    int nb = 0;
    const size_t smem = push_smem_bytes(mode, ng);
    cudaError_t e;
    if (mode == PIC_FP32_FIXED) {
        FixedKernel k = pick_fixed(variant, true, unroll);
        if (!k || (variant == PIC_DEPOSIT_QUAD_BULK && block != kBulkThreads)) return 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block,
                                                          fixed_smem_bytes(variant, true, ng));
    }
    else if (mode == PIC_FP32_ATOMIC)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, &pic_push_f32atomic_kernel<true>, block, smem);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, &pic_push_f64_kernel<true>, block, smem);
    return e == cudaSuccess ? nb : 0;
}

cudaError_t launch_push_fixed(const PushArgs &a, int grid, int block, int variant,
                              int unroll, bool push, cudaStream_t s) {
    FixedKernel k = pick_fixed(variant, push, unroll);
    if (!k) return cudaErrorInvalidValue;
    k<<<grid, block, fixed_smem_bytes(variant, push, a.c.ng), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_push_f32_atomic(const PushArgsF32Atomic &a, int grid, int block,
                                   bool push, cudaStream_t s) {
    const size_t smem = push_smem_bytes(PIC_FP32_ATOMIC, a.c.ng);
    if (push) pic_push_f32atomic_kernel<true><<<grid, block, smem, s>>>(a);
    else pic_push_f32atomic_kernel<false><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_push_f64(const PushArgs64 &a, int grid, int block, bool push,
                            cudaStream_t s) {
    const size_t smem = push_smem_bytes(PIC_FP64, a.ng);
    if (push) pic_push_f64_kernel<true><<<grid, block, smem, s>>>(a);
    else pic_push_f64_kernel<false><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pic
