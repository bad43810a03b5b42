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
//   MATCH_PACKED  the two combined: one atomic per warp group.
// The packed forms flush the tile to global memory before any node can hold
// 2^16 particles, so the 40-bit weight field never carries into the count.
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMatchPacked = PIC_DEPOSIT_MATCH_PACKED;
constexpr unsigned long long kPackShift = 40;
constexpr unsigned long long kPackMask = (1ull << kPackShift) - 1ull;
// particles a block may pack into one node between flushes
constexpr int kPackLimit = 65535 - 32;

using u64 = unsigned long long;

// Left/right node and fraction of a float32 position, by the fixed-point
// recipe: s = x*c - 1/2, i = floor(s), f = s - i, each one float operation
// rounded to nearest (no contraction).  ok is false for a position that is not
// finite or lies outside the grid.
struct NodePair {
    int il, ir;
    float f;
    bool ok;
};

__device__ __forceinline__ NodePair locate(float x, const PushConsts &c) {
    NodePair p;
    const float u = __fmul_rn(x, c.inv_dx);
    const float s = __fsub_rn(u, 0.5f);
    const float fl = floorf(s);
    p.f = __fsub_rn(s, fl);
    p.ok = (fl >= -1.0f) && (fl <= (float)(c.ng - 1));
    const int i = p.ok ? (int)fl : 0;
    p.il = (i < 0) ? i + c.ng : i;
    p.ir = (i + 1 >= c.ng) ? i + 1 - c.ng : i + 1;
    return p;
}

// The right node's share W = trunc(f * 2^24) of a particle's 2^24.
__device__ __forceinline__ unsigned fixed_weight(float f) {
    return __float2uint_rz(__fmul_rn(f, 16777216.0f));
}

// Gather E at x (linear weights of the two nearest nodes), kick, drift, wrap.
__device__ __forceinline__ void push_particle(float &x, float &v, const float *sE,
                                              const PushConsts &c, float &ke,
                                              float &mom) {
    const NodePair p = locate(x, c);
    const float e0 = sE[p.il], e1 = sE[p.ir];
    const float ep = p.ok ? fmaf(p.f, e1 - e0, e0) : 0.0f;
    const float vn = fmaf(c.qmdt, ep, v);
    ke = fmaf(v, vn, ke);
    mom += vn;
    float xn = fmaf(vn, c.dt, x);
    if (xn < 0.0f) xn += c.length;
    else if (xn >= c.length) xn -= c.length;
    if (xn >= c.length) xn = 0.0f;  // x + L rounded up to L: the point 0
    x = xn;
    v = vn;
}

// Deposit one particle (valid lanes only; all 32 lanes of the warp call this
// together for the MATCH variants).
template <int VARIANT>
__device__ __forceinline__ void deposit(u64 *sRho, float x, bool valid,
                                        const PushConsts &c, unsigned *err,
                                        int lane) {
    const NodePair p = locate(x, c);
    const bool good = valid && p.ok;
    if (valid && !p.ok) atomicOr(err, kErrPosition);
    const unsigned W = good ? fixed_weight(p.f) : 0u;
    if (VARIANT == PIC_DEPOSIT_ATOMIC) {
        if (good) {
            atomicAdd(&sRho[p.il], (u64)(kFixOne - W));
            atomicAdd(&sRho[p.ir], (u64)W);
        }
    } else if (VARIANT == PIC_DEPOSIT_PACKED) {
        if (good) atomicAdd(&sRho[p.il], (1ull << kPackShift) | (u64)W);
    } else {
        const unsigned key = good ? (unsigned)p.il : 0xffffffffu;
        const unsigned peers = __match_any_sync(kFull, key);
        const unsigned wsum = __reduce_add_sync(peers, W);
        if (good && lane == __ffs(peers) - 1) {
            const u64 cnt = (u64)__popc(peers);
            if (VARIANT == PIC_DEPOSIT_MATCH) {
                atomicAdd(&sRho[p.il], cnt * kFixOne - (u64)wsum);
                atomicAdd(&sRho[p.ir], (u64)wsum);
            } else {
                atomicAdd(&sRho[p.il], (cnt << kPackShift) + (u64)wsum);
            }
        }
    }
}

// Add the block's tile to the global density and clear it.
template <bool PACKED>
__device__ __forceinline__ void flush_tile(u64 *sRho, u64 *rho_q, int ng) {
    __syncthreads();
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const u64 t = sRho[g];
        if (t == 0) continue;
        sRho[g] = 0;
        if (PACKED) {
            const u64 cnt = t >> kPackShift, sw = t & kPackMask;
            const u64 left = cnt * kFixOne - sw;
            if (left) atomicAdd(&rho_q[g], left);
            if (sw) atomicAdd(&rho_q[g + 1 == ng ? 0 : g + 1], sw);
        } else {
            atomicAdd(&rho_q[g], t);
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

template <int VARIANT, bool PUSH>
__global__ void __launch_bounds__(1024) pic_push_fixed_kernel(PushArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[64];
    constexpr bool kPacked = VARIANT == PIC_DEPOSIT_PACKED || VARIANT == kMatchPacked;
    const PushConsts c = a.c;
    u64 *sRho = reinterpret_cast<u64 *>(smem_raw);
    float *sE = reinterpret_cast<float *>(sRho + c.ng);
    const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31;
    for (int g = tid; g < c.ng; g += bs) {
        sRho[g] = 0;
        if (PUSH) sE[g] = a.E32[g];
    }
    __syncthreads();

    float ke = 0.0f, mom = 0.0f;
    const long long n4 = a.n >> 2;
    float4 *x4 = reinterpret_cast<float4 *>(a.x);
    float4 *v4 = reinterpret_cast<float4 *>(a.v);
    const long long stride = (long long)gridDim.x * bs;
    const int flush_every = kPacked ? max(1, kPackLimit / (4 * bs)) : 0;
    int since_flush = 0;
    // The trip count is uniform over the block (q0 is), so the packed flush
    // may synchronise inside the loop and every warp is converged for match.
    for (long long q0 = (long long)blockIdx.x * bs; q0 < n4; q0 += stride) {
        const long long q = q0 + tid;
        const bool valid = q < n4;
        float4 xx = make_float4(0.f, 0.f, 0.f, 0.f), vv = xx;
        if (valid) {
            xx = __ldcs(x4 + q);
            if (PUSH) vv = __ldcs(v4 + q);
        }
        if (PUSH && valid) {
            push_particle(xx.x, vv.x, sE, c, ke, mom);
            push_particle(xx.y, vv.y, sE, c, ke, mom);
            push_particle(xx.z, vv.z, sE, c, ke, mom);
            push_particle(xx.w, vv.w, sE, c, ke, mom);
        }
        deposit<VARIANT>(sRho, xx.x, valid, c, a.err, lane);
        deposit<VARIANT>(sRho, xx.y, valid, c, a.err, lane);
        deposit<VARIANT>(sRho, xx.z, valid, c, a.err, lane);
        deposit<VARIANT>(sRho, xx.w, valid, c, a.err, lane);
        if (PUSH && valid) {
            __stcs(x4 + q, xx);
            __stcs(v4 + q, vv);
        }
        if (kPacked && ++since_flush == flush_every) {
            flush_tile<true>(sRho, a.rho_q, c.ng);
            since_flush = 0;
        }
    }
    // The last N mod 4 particles: warp 0 of block 0, converged.
    if (blockIdx.x == 0 && tid < 32) {
        const long long i = n4 * 4 + lane;
        const bool valid = i < a.n;
        float xs = valid ? a.x[i] : 0.0f, vs = valid && PUSH ? a.v[i] : 0.0f;
        if (PUSH && valid) push_particle(xs, vs, sE, c, ke, mom);
        deposit<VARIANT>(sRho, xs, valid, c, a.err, lane);
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
    flush_tile<kPacked>(sRho, a.rho_q, c.ng);
}

// ---- float32 push with float32 atomic deposit (precision study) -------------

template <bool PUSH>
__global__ void __launch_bounds__(1024) pic_push_f32atomic_kernel(PushArgsF32Atomic a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[64];
    const PushConsts c = a.c;
    float *sRho = reinterpret_cast<float *>(smem_raw);
    float *sE = sRho + c.ng;
    const int tid = threadIdx.x, bs = blockDim.x;
    for (int g = tid; g < c.ng; g += bs) {
        sRho[g] = 0.0f;
        if (PUSH) sE[g] = a.E32[g];
    }
    __syncthreads();
    float ke = 0.0f, mom = 0.0f;
    const long long stride = (long long)gridDim.x * bs;
    for (long long i = (long long)blockIdx.x * bs + tid; i < a.n; i += stride) {
        float x = a.x[i], v = PUSH ? a.v[i] : 0.0f;
        if (PUSH) push_particle(x, v, sE, c, ke, mom);
        const NodePair p = locate(x, c);
        if (p.ok) {
            atomicAdd(&sRho[p.il], 1.0f - p.f);
            atomicAdd(&sRho[p.ir], p.f);
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
    for (int g = tid; g < c.ng; g += bs)
        if (sRho[g] != 0.0f) atomicAdd(&a.rho_acc[g], sRho[g]);
}

// ---- float64 push with float64 atomic deposit (precision study) ------------

template <bool PUSH>
__global__ void __launch_bounds__(1024) pic_push_f64_kernel(PushArgs64 a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
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
    for (long long i = (long long)blockIdx.x * bs + tid; i < a.n; i += stride) {
        double x = a.x[i];
        double s = x * a.inv_dx - 0.5;
        double fl = floor(s);
        bool ok = fl >= -1.0 && fl <= (double)(ng - 1);
        if (PUSH) {
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
        if (ok) {
            int j = (int)fl;
            int il = j < 0 ? j + ng : j, ir = j + 1 >= ng ? j + 1 - ng : j + 1;
            double f = s - fl;
            atomicAdd(&sRho[il], 1.0 - f);
            atomicAdd(&sRho[ir], f);
        } else {
            atomicOr(a.err, kErrPosition);
        }
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

FixedKernel pick_fixed(int variant, bool push) {
    switch (variant) {
        case PIC_DEPOSIT_ATOMIC:
            return push ? &pic_push_fixed_kernel<PIC_DEPOSIT_ATOMIC, true>
                        : &pic_push_fixed_kernel<PIC_DEPOSIT_ATOMIC, false>;
        case PIC_DEPOSIT_MATCH:
            return push ? &pic_push_fixed_kernel<PIC_DEPOSIT_MATCH, true>
                        : &pic_push_fixed_kernel<PIC_DEPOSIT_MATCH, false>;
        case PIC_DEPOSIT_PACKED:
            return push ? &pic_push_fixed_kernel<PIC_DEPOSIT_PACKED, true>
                        : &pic_push_fixed_kernel<PIC_DEPOSIT_PACKED, false>;
        case kMatchPacked:
            return push ? &pic_push_fixed_kernel<kMatchPacked, true>
                        : &pic_push_fixed_kernel<kMatchPacked, false>;
        default:
            return nullptr;
    }
}

}  // namespace

size_t push_smem_bytes(int mode, int ng) {
    if (mode == PIC_FP64) return (size_t)ng * 16;
    if (mode == PIC_FP32_ATOMIC) return (size_t)ng * 8;
    return (size_t)ng * 12;
}

cudaError_t push_prepare_attributes(int mode, int ng) {
    const int bytes = (int)push_smem_bytes(mode, PIC_NCELL_MAX);
    (void)ng;
    cudaError_t e = cudaSuccess;
    if (mode == PIC_FP32_FIXED) {
        for (int v = PIC_DEPOSIT_ATOMIC; v <= kMatchPacked; v++)
            for (int p = 0; p < 2; p++) {
                e = cudaFuncSetAttribute(pick_fixed(v, p != 0),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
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

int push_max_blocks_per_sm(int mode, int variant, int block, int ng) {
    int nb = 0;
    const size_t smem = push_smem_bytes(mode, ng);
    cudaError_t e;
    if (mode == PIC_FP32_FIXED)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pick_fixed(variant, true), block, smem);
    else if (mode == PIC_FP32_ATOMIC)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, &pic_push_f32atomic_kernel<true>, block, smem);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, &pic_push_f64_kernel<true>, block, smem);
    return e == cudaSuccess ? nb : 0;
}

cudaError_t launch_push_fixed(const PushArgs &a, int grid, int block, int variant,
                              bool push, cudaStream_t s) {
    FixedKernel k = pick_fixed(variant, push);
    if (!k) return cudaErrorInvalidValue;
    k<<<grid, block, push_smem_bytes(PIC_FP32_FIXED, a.c.ng), s>>>(a);
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
