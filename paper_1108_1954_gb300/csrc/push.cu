// push.cu -- the fused particle kernel of one PIC step: field gather (Sec.
// 2.3), velocity update (Sec. 2.1, Eq. 3), position update and periodic wrap
// (Sec. 2.1, Eq. 2; Appendix A wrap), and the charge deposit of the new
// positions (Sec. 2.3).
//
// Design (GB300): one persistent grid of (SMs x resident blocks), each block
// streaming float4 groups of 4 particles (the cell coordinates u = x NG/L and
// the velocities v are separate float32 arrays,
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
//   QUAD          runs of equal left node among a thread's 4 particles are
//                 summed in registers, then two atomics per run;
//   PAIR          the same with two open runs, so that particles of two
//                 interleaved cells (the two beams before the first sort)
//                 still combine.
// The nearest-grid-point shape (PIC_SHAPE_NGP) uses the same loop with the
// NGP gather and a QUAD-style deposit of whole particles to the cell's node.
// The tiles hold exact 64-bit sums in two 32-bit words (particle_ops.cuh).
#include "particle_ops.cuh"

namespace pic {
namespace {


// Add the block's tile to the global density and clear it (ghost nodes
// folded onto their periodic images).
__device__ __forceinline__ void flush_tile(const Tile &t, u64 *rho_q, int ng) {
    __syncthreads();
    for (int j = threadIdx.x; j <= ng + 1; j += blockDim.x) {
        const u64 w = ((u64)t.hi[j] << 32) | (u64)t.lo[j];
        if (w == 0) continue;
        t.lo[j] = 0u;
        t.hi[j] = 0u;
        atomicAdd(&rho_q[j == 0 ? ng - 1 : (j == ng + 1 ? 0 : j - 1)], w);
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
    const PushConsts c = a.c;
    const int ng = c.ng;
    Tile tile;                                                       // 8 (ng + 2) B
    tile.lo = reinterpret_cast<unsigned *>(smem_raw);
    tile.hi = tile.lo + ng + 2;
    float *sE = reinterpret_cast<float *>(smem_raw + 8 * (ng + 2));  // ng + 2
    const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31;
    for (int j = tid; j < ng + 2; j += bs) {
        tile.lo[j] = 0u;
        tile.hi[j] = 0u;
        if (PUSH) sE[j] = a.E32[j == 0 ? ng - 1 : (j == ng + 1 ? 0 : j - 1)];
    }
    __syncthreads();

    float ke = 0.0f, mom = 0.0f;
    const long long n4 = a.n >> 2;
    float4 *x4 = reinterpret_cast<float4 *>(a.x);
    float4 *v4 = reinterpret_cast<float4 *>(a.v);
    const long long span = (long long)bs * U;
    const long long stride = (long long)gridDim.x * span;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 cx[U], cv[U];
    long long q0 = (long long)blockIdx.x * span;
#pragma unroll
    for (int u = 0; u < U; u++) {
        const long long q = q0 + u * bs + tid;
        cx[u] = q < n4 ? __ldcs(x4 + q) : zero4;
        cv[u] = (PUSH && q < n4) ? __ldcs(v4 + q) : zero4;
    }
    // The trip count is uniform over the block (q0 is), so every warp is
    // converged for the MATCH variant's warp votes.
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
    flush_tile(tile, a.rho_q, ng);
}

// ---- the fused push on 8-particle groups (QUAD8, PAIR8) ---------------------
//
// The same step, each thread taking 8 consecutive particles per group: one
// 32-byte vector load (and store) per array, lanes of a warp on consecutive
// groups (1 KB per warp and array, coalesced), and the deposit's runs of
// equal cell merged over all 8 particles, which halves the shared-memory
// atomics where neighbours share a cell (a sorted state, cold beams).
template <int VARIANT, bool PUSH, int U>
__global__ void __launch_bounds__(512) pic_push_oct_kernel(PushArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[64];
    const PushConsts c = a.c;
    const int ng = c.ng;
    Tile tile;                                                       // 8 (ng + 2) B
    tile.lo = reinterpret_cast<unsigned *>(smem_raw);
    tile.hi = tile.lo + ng + 2;
    float *sE = reinterpret_cast<float *>(smem_raw + 8 * (ng + 2));  // ng + 2
    const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31;
    for (int j = tid; j < ng + 2; j += bs) {
        tile.lo[j] = 0u;
        tile.hi[j] = 0u;
        if (PUSH) sE[j] = a.E32[j == 0 ? ng - 1 : (j == ng + 1 ? 0 : j - 1)];
    }
    __syncthreads();

    float ke = 0.0f, mom = 0.0f;
    const long long n8 = a.n >> 3;
    const long long span = (long long)bs * U;
    const long long stride = (long long)gridDim.x * span;
    F8 zero8;
#pragma unroll
    for (int k = 0; k < 8; k++) zero8.v[k] = 0.0f;
    // no loads ahead: a group's 16 values per thread are its registers'
    // worth, and three resident blocks hide the load latency instead
    for (long long q0 = (long long)blockIdx.x * span; q0 < n8; q0 += stride) {
        F8 cx[U], cv[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long q = q0 + u * bs + tid;
            cx[u] = q < n8 ? ld8(a.x + 8 * q) : zero8;
            cv[u] = (PUSH && q < n8) ? ld8(a.v + 8 * q) : zero8;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long q = q0 + u * bs + tid;
            const bool valid = q < n8;
            F8 xx = cx[u], vv = cv[u];
            if (PUSH && valid) {
#pragma unroll
                for (int k = 0; k < 8; k++) push_particle(xx.v[k], vv.v[k], sE, c, ke, mom);
            }
            deposit_group<VARIANT, 8>(tile, xx.v, valid, c, a.err, lane);
            if (PUSH && valid) {
                st8(a.x + 8 * q, xx);
                st8(a.v + 8 * q, vv);
            }
        }
    }
    // The last N mod 8 particles: warp 0 of block 0, converged.
    if (blockIdx.x == 0 && tid < 32) {
        const long long i = n8 * 8 + lane;
        const bool valid = i < a.n;
        float xs = valid ? a.x[i] : 0.0f, vs = valid && PUSH ? a.v[i] : 0.0f;
        if (PUSH && valid) push_particle(xs, vs, sE, c, ke, mom);
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
    flush_tile(tile, a.rho_q, ng);
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
        const Loc l = locate(x);
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

template <int V>
FixedKernel pick_oct(bool push, int unroll) {
    if (!push) return &pic_push_oct_kernel<V, false, 1>;
    switch (unroll) {
        case 1: return &pic_push_oct_kernel<V, true, 1>;
        case 2: return &pic_push_oct_kernel<V, true, 2>;
        default: return nullptr;
    }
}

FixedKernel pick_fixed(int variant, bool push, int unroll) {
    switch (variant) {
        case PIC_DEPOSIT_QUAD8: return pick_oct<PIC_DEPOSIT_QUAD8>(push, unroll);
        case PIC_DEPOSIT_PAIR8: return pick_oct<PIC_DEPOSIT_PAIR8>(push, unroll);
        case PIC_DEPOSIT_ATOMIC: return pick_unroll<PIC_DEPOSIT_ATOMIC>(push, unroll);
        case PIC_DEPOSIT_MATCH: return pick_unroll<PIC_DEPOSIT_MATCH>(push, unroll);
        case PIC_DEPOSIT_QUAD: return pick_unroll<PIC_DEPOSIT_QUAD>(push, unroll);
        case PIC_DEPOSIT_PAIR: return pick_unroll<PIC_DEPOSIT_PAIR>(push, unroll);
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

// Shared memory of a fused fixed-point push launch.
size_t fixed_smem_bytes(int ng) { return push_smem_bytes(PIC_FP32_FIXED, ng); }

cudaError_t push_prepare_attributes(int mode, int ng) {
    const int bytes = (int)push_smem_bytes(mode, PIC_NCELL_MAX);
    (void)ng;
    cudaError_t e = cudaSuccess;
    if (mode == PIC_FP32_FIXED) {
        const int unrolls[3] = {1, 2, 4};
        const int fixed_variants[] = {PIC_DEPOSIT_ATOMIC, PIC_DEPOSIT_MATCH, PIC_DEPOSIT_QUAD,
                                      PIC_DEPOSIT_PAIR, PIC_DEPOSIT_QUAD8, PIC_DEPOSIT_PAIR8,
                                      kDepositNgp};
        for (int v : fixed_variants)
            for (int p = 0; p < 2; p++)
                for (int u : unrolls) {
                    FixedKernel k = pick_fixed(v, p != 0, u);
                    if (!k) continue;
                    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)fixed_smem_bytes(PIC_NCELL_MAX));
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
        if (!k) return 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, fixed_smem_bytes(ng));
    }
    else if (mode == PIC_FP32_ATOMIC)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, &pic_push_f32atomic_kernel<true>, block, smem);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, &pic_push_f64_kernel<true>, block, smem);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();     // do not leave the error for a later launch check
        return 0;
    }
    return nb;
}

cudaError_t launch_push_fixed(const PushArgs &a, int grid, int block, int variant,
                              int unroll, bool push, cudaStream_t s) {
    FixedKernel k = pick_fixed(variant, push, unroll);
    if (!k) return cudaErrorInvalidValue;
    k<<<grid, block, fixed_smem_bytes(a.c.ng), s>>>(a);
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
