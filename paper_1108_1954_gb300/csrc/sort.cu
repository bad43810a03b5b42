// sort.cu -- periodic counting sort of the particles by cell.
//
// Not a step of the paper's method: it reorders the particle arrays so that
// the particles a warp handles share few cells, which makes the fused push's
// field reads broadcasts and lets its deposit aggregate equal nodes before the
// shared-memory atomics.  It changes no physical quantity.
//
// Five passes, all deterministic and stable (particles of one cell keep their
// relative order):
//   count    block b counts the cells of its contiguous chunk -> hist[b][g]
//   colscan  per (segment of chunks, cell): exclusive prefix over the chunks
//            of the segment, in place, and the segment total
//   segscan  per cell: exclusive prefix over the segments, in place, and the
//            cell total
//   base     exclusive prefix of the cell totals over the cells -> base[g]
//   scatter  block b walks its chunk in order, 512 particles at a time
//            (64 consecutive per warp); the warps take their slots from the
//            per-cell cursors one after the other, so the order within a
//            cell is the original order.
// The destination index is bounds-checked; a violation sets the device error
// word instead of writing.
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr unsigned kNoKey = 0xffffffffu;

template <typename T>
__device__ __forceinline__ unsigned cell_key(T x, T inv_dx, int ng) {
    T u = x * inv_dx;
    u = u > (T)0 ? u : (T)0;                  // also maps NaN to 0
    const T top = (T)(ng - 1);
    u = u < top ? u : top;
    return (unsigned)u;
}

template <typename T>
__global__ void __launch_bounds__(kSortThreads) sort_count_kernel(SortArgs<T> a) {
    extern __shared__ unsigned sh_count[];
    const int ng = a.ng;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) sh_count[g] = 0u;
    __syncthreads();
    const long long start = (long long)blockIdx.x * a.chunk;
    const long long end = min(a.n, start + a.chunk);
    if (sizeof(T) == 4 && (a.chunk & 3) == 0) {
        // float4 groups (the chunk starts on a group): equal cells among a
        // group's 4 particles are counted with one atomic, K groups in flight
        constexpr int K = 4;
        const float4 *x4 = reinterpret_cast<const float4 *>(a.x);
        const long long q0 = start >> 2, q1 = end >> 2;
        for (long long qb = q0; qb < q1; qb += K * blockDim.x) {
            float4 xv[K];
#pragma unroll
            for (int k = 0; k < K; k++) {
                const long long q = qb + k * blockDim.x + threadIdx.x;
                xv[k] = q < q1 ? __ldcs(x4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < K; k++) {
                const long long q = qb + k * blockDim.x + threadIdx.x;
                if (q >= q1) continue;
                const float xs[4] = {xv[k].x, xv[k].y, xv[k].z, xv[k].w};
                unsigned key = cell_key((T)xs[0], a.inv_dx, ng), run = 1u;
#pragma unroll
                for (int j = 1; j < 4; j++) {
                    const unsigned kj = cell_key((T)xs[j], a.inv_dx, ng);
                    if (kj == key) {
                        run++;
                    } else {
                        atomicAdd(&sh_count[key], run);
                        key = kj;
                        run = 1u;
                    }
                }
                atomicAdd(&sh_count[key], run);
            }
        }
        // the chunk's last n mod 4 particles
        const long long i = (q1 << 2) + threadIdx.x;
        if (i < end) atomicAdd(&sh_count[cell_key(a.x[i], a.inv_dx, ng)], 1u);
    } else {
        constexpr int K = 8;   // loads in flight per thread
        for (long long i0 = start; i0 < end; i0 += K * blockDim.x) {
            T xv[K];
#pragma unroll
            for (int k = 0; k < K; k++) {
                const long long i = i0 + k * blockDim.x + threadIdx.x;
                xv[k] = i < end ? __ldcs(a.x + i) : (T)0;
            }
#pragma unroll
            for (int k = 0; k < K; k++) {
                const long long i = i0 + k * blockDim.x + threadIdx.x;
                if (i < end) atomicAdd(&sh_count[cell_key(xv[k], a.inv_dx, ng)], 1u);
            }
        }
    }
    __syncthreads();
    unsigned *row = a.hist + (size_t)blockIdx.x * ng;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) row[g] = sh_count[g];
}

// Exclusive prefix, in place, of the column p[0], p[stride], ... p[(len-1)
// stride]; returns the column total.  Loads are issued 16 at a time.
__device__ __forceinline__ unsigned column_scan(unsigned *p, size_t stride, int len) {
    constexpr int kB = 16;
    unsigned run = 0;
    for (int k0 = 0; k0 < len; k0 += kB) {
        unsigned c[kB];
#pragma unroll
        for (int k = 0; k < kB; k++) c[k] = k0 + k < len ? p[(size_t)(k0 + k) * stride] : 0u;
#pragma unroll
        for (int k = 0; k < kB; k++) {
            if (k0 + k < len) p[(size_t)(k0 + k) * stride] = run;
            run += c[k];
        }
    }
    return run;
}

template <typename T>
__global__ void __launch_bounds__(256) sort_colscan_kernel(SortArgs<T> a) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.ng) return;
    const int seg = blockIdx.y;
    const int b0 = seg * a.seg_len, b1 = min(a.nchunk, b0 + a.seg_len);
    a.segtot[(size_t)seg * a.ng + g] = column_scan(a.hist + (size_t)b0 * a.ng + g, a.ng, b1 - b0);
}

// Per cell: exclusive prefix of the segment totals over the segments (in
// place) and the cell total (into base).  One thread per cell.
template <typename T>
__global__ void __launch_bounds__(256) sort_segscan_kernel(SortArgs<T> a) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.ng) return;
    a.base[g] = column_scan(a.segtot + g, a.ng, a.nseg);
}

// Exclusive prefix of the cell totals over the cells -> first slot of each
// cell.  One block; each thread scans a contiguous run of cells.
template <typename T>
__global__ void __launch_bounds__(512) sort_base_kernel(SortArgs<T> a) {
    __shared__ unsigned wt[32];
    const int ng = a.ng, T_ = blockDim.x, t = threadIdx.x;
    const int k = (ng + T_ - 1) / T_;
    const int g0 = t * k;
    unsigned local = 0;
    for (int j = 0; j < k; j++) {
        const int g = g0 + j;
        if (g < ng) local += a.base[g];
    }
    const int lane = t & 31, w = t >> 5;
    unsigned inc = local;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) wt[w] = inc;
    __syncthreads();
    unsigned off = 0;
    for (int i = 0; i < w; i++) off += wt[i];
    unsigned run = off + inc - local;
    for (int j = 0; j < k; j++) {
        const int g = g0 + j;
        if (g >= ng) break;
        const unsigned c = a.base[g];
        a.base[g] = run;
        run += c;
    }
}

// Scatter: block b walks its chunk in order, 256 particles at a time (one
// per thread, with the loads four iterations ahead).  Lanes of
// one cell within a warp are ranked by __match_any_sync; the warps take their
// slots from the chunk's per-cell cursors one after the other (a barrier per
// warp), so the order within a cell is the original order.  Measured on
// GB300 against tile-wise variants (eight groups per warp turn, per-warp
// window histograms, one warp per chunk, a shared-memory radix sort of each
// 2048-particle tile with coalesced writes), this plain form was the fastest
// over the config-2 run: the others either lowered the number of resident
// blocks whose turns interleave, or spent ~175 instructions per particle.
// The scatter walks its chunk in rounds of kSub x 256 particles: warp w owns
// the round's particles [32 kSub w, 32 kSub (w + 1)) as kSub steps of 32
// (lane l takes particle 32 j + l of step j).  Lanes of one cell in a step are
// ranked by __match_any_sync; in its turn a warp's leaders take their slots
// from the per-cell cursors, step after step; the warps take their turns in
// order, so a cell's particles keep their order in the chunk.  One round of
// turns (a block barrier per warp) serves kSub x 256 particles; the next
// round's particles are loaded a round ahead.  Measured on GB300 (2^25
// particles after two sorts): kSub = 2, 30 registers, 134-147 us against 179
// us for one step per turn; kSub = 3, 4 and 8 take more registers and fewer
// blocks per SM and were slower (185, 147-152 and 199 us).
constexpr int kSub = 2;

template <typename T>
__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(SortArgs<T> a) {
    extern __shared__ unsigned cursor[];
    const int ng = a.ng;
    const int seg = blockIdx.x / a.seg_len;
    const unsigned *row = a.hist + (size_t)blockIdx.x * ng;
    const unsigned *srow = a.segtot + (size_t)seg * ng;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) cursor[g] = a.base[g] + srow[g] + row[g];
    __syncthreads();
    const long long start = (long long)blockIdx.x * a.chunk;
    const long long end = min(a.n, start + a.chunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const long long round = (long long)kSub * blockDim.x;
    // this lane's particle of step j in the round beginning at r0
    const long long own = (long long)warp * (kSub * 32) + lane;
    auto ldx = [&](long long i) { return i < end ? __ldcs(a.x + i) : (T)0; };
    auto ldv = [&](long long i) { return i < end ? __ldcs(a.v + i) : (T)0; };
    T nx[kSub], nv[kSub];
#pragma unroll
    for (int j = 0; j < kSub; j++) {
        nx[j] = ldx(start + own + 32 * j);
        nv[j] = ldv(start + own + 32 * j);
    }
    for (long long r0 = start; r0 < end; r0 += round) {
        T x[kSub], v[kSub];
#pragma unroll
        for (int j = 0; j < kSub; j++) {
            x[j] = nx[j];
            v[j] = nv[j];
            nx[j] = ldx(r0 + round + own + 32 * j);      // the next round, a round ahead
            nv[j] = ldv(r0 + round + own + 32 * j);
        }
        unsigned key[kSub], peers[kSub], base[kSub];
        int leader[kSub];
#pragma unroll
        for (int j = 0; j < kSub; j++) {
            const bool valid = r0 + own + 32 * j < end;
            key[j] = valid ? cell_key(x[j], a.inv_dx, ng) : kNoKey;
            peers[j] = __match_any_sync(kFull, key[j]);
            leader[j] = __ffs(peers[j]) - 1;
            base[j] = 0u;
        }
        for (int w = 0; w < nwarp; w++) {
            if (w == warp) {
#pragma unroll
                for (int j = 0; j < kSub; j++) {
                    if (key[j] != kNoKey && lane == leader[j]) {
                        base[j] = cursor[key[j]];
                        cursor[key[j]] = base[j] + (unsigned)__popc(peers[j]);
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < kSub; j++) {
            const unsigned b = __shfl_sync(kFull, base[j], leader[j]);
            if (key[j] != kNoKey) {
                const unsigned long long dst = (unsigned long long)b + __popc(peers[j] & lt);
                if (dst < (unsigned long long)a.n) {
                    a.x_out[dst] = x[j];
                    a.v_out[dst] = v[j];
                } else {
                    atomicOr(a.err, kErrSortKey);
                }
            }
        }
    }
}

template <typename T>
cudaError_t launch_sort_t(const SortArgs<T> &a, cudaStream_t s) {
    const size_t smem = (size_t)a.ng * sizeof(unsigned);
    sort_count_kernel<T><<<a.nchunk, kSortThreads, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 cg((a.ng + 255) / 256, a.nseg);
    sort_colscan_kernel<T><<<cg, 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    sort_segscan_kernel<T><<<(a.ng + 255) / 256, 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    sort_base_kernel<T><<<1, 512, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    sort_scatter_kernel<T><<<a.nchunk, kSortThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t sort_prepare_attributes(int ng) {
    (void)ng;
    const int bytes = PIC_NCELL_MAX * (int)sizeof(unsigned);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(&sort_count_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    if ((e = cudaFuncSetAttribute(&sort_scatter_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    if ((e = cudaFuncSetAttribute(&sort_count_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    return cudaFuncSetAttribute(&sort_scatter_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_sort_f32(const SortArgs<float> &a, cudaStream_t s) { return launch_sort_t(a, s); }
cudaError_t launch_sort_f64(const SortArgs<double> &a, cudaStream_t s) { return launch_sort_t(a, s); }

}  // namespace pic
