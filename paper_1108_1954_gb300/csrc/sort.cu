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
//   scatter  block b walks its chunk in order, 256 particles at a time; the
//            warps take their slots from the per-cell cursor one after the
//            other, so the order within a cell is the original order.
// The destination index is bounds-checked; a violation sets the device error
// word instead of writing.
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr unsigned kNoKey = 0xffffffffu;
constexpr int kMaxSegLen = 32;   // chunks per segment and segments (<= 32 each)

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
    __syncthreads();
    unsigned *row = a.hist + (size_t)blockIdx.x * ng;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) row[g] = sh_count[g];
}

template <typename T>
__global__ void __launch_bounds__(256) sort_colscan_kernel(SortArgs<T> a) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.ng) return;
    const int seg = blockIdx.y;
    const int b0 = seg * a.seg_len, b1 = min(a.nchunk, b0 + a.seg_len);
    unsigned c[kMaxSegLen];
#pragma unroll
    for (int k = 0; k < kMaxSegLen; k++)
        c[k] = b0 + k < b1 ? a.hist[(size_t)(b0 + k) * a.ng + g] : 0u;
    unsigned run = 0;
#pragma unroll
    for (int k = 0; k < kMaxSegLen; k++) {
        if (b0 + k < b1) a.hist[(size_t)(b0 + k) * a.ng + g] = run;
        run += c[k];
    }
    a.segtot[(size_t)seg * a.ng + g] = run;
}

// Per cell: exclusive prefix of the segment totals over the segments (in
// place) and the cell total (into base).  One thread per cell.
template <typename T>
__global__ void __launch_bounds__(256) sort_segscan_kernel(SortArgs<T> a) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.ng) return;
    const int ng = a.ng;
    unsigned c[kMaxSegLen];
#pragma unroll
    for (int s = 0; s < kMaxSegLen; s++) c[s] = s < a.nseg ? a.segtot[(size_t)s * ng + g] : 0u;
    unsigned run = 0;
#pragma unroll
    for (int s = 0; s < kMaxSegLen; s++) {
        if (s < a.nseg) a.segtot[(size_t)s * ng + g] = run;
        run += c[s];
    }
    a.base[g] = run;
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
    T nx = start + threadIdx.x < end ? __ldcs(a.x + start + threadIdx.x) : (T)0;
    T nv = start + threadIdx.x < end ? __ldcs(a.v + start + threadIdx.x) : (T)0;
    for (long long i0 = start; i0 < end; i0 += blockDim.x) {
        const long long i = i0 + threadIdx.x;
        const bool valid = i < end;
        const T x = nx, v = nv;
        const long long inext = i + blockDim.x;
        nx = inext < end ? __ldcs(a.x + inext) : (T)0;
        nv = inext < end ? __ldcs(a.v + inext) : (T)0;
        const unsigned key = valid ? cell_key(x, a.inv_dx, ng) : kNoKey;
        const unsigned peers = __match_any_sync(kFull, key);
        const int leader = __ffs(peers) - 1;
        unsigned base = 0;
        for (int w = 0; w < nwarp; w++) {
            if (w == warp && valid && lane == leader) {
                base = cursor[key];
                cursor[key] = base + (unsigned)__popc(peers);
            }
            __syncthreads();
        }
        base = __shfl_sync(kFull, base, leader);
        if (valid) {
            const unsigned long long dst = (unsigned long long)base + __popc(peers & lt);
            if (dst < (unsigned long long)a.n) {
                a.x_out[dst] = x;
                a.v_out[dst] = v;
            } else {
                atomicOr(a.err, kErrSortKey);
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
