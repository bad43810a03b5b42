// field_ops.cuh -- 128-bit integer helpers of the exact field solve, shared by
// the single-run solve (field.cu) and the batched cluster kernel (batch.cu).
#pragma once

#include <cooperative_groups.h>

#include "pic_internal.cuh"

namespace pic {

typedef __int128 i128;

__device__ __forceinline__ i128 shfl_up_i128(i128 v, int o) {
    long long lo = (long long)(unsigned long long)v;
    long long hi = (long long)(v >> 64);
    lo = __shfl_up_sync(kFull, lo, o);
    hi = __shfl_up_sync(kFull, hi, o);
    return (i128)(((unsigned __int128)(unsigned long long)hi << 64) |
                  (unsigned long long)lo);
}

__device__ __forceinline__ i128 shfl_down_i128(i128 v, int o) {
    long long lo = (long long)(unsigned long long)v;
    long long hi = (long long)(v >> 64);
    lo = __shfl_down_sync(kFull, lo, o);
    hi = __shfl_down_sync(kFull, hi, o);
    return (i128)(((unsigned __int128)(unsigned long long)hi << 64) |
                  (unsigned long long)lo);
}

__device__ __forceinline__ double i128_to_f64(i128 v) {
    const long long hi = (long long)(v >> 64);
    const unsigned long long lo = (unsigned long long)v;
    if ((hi == 0 && (long long)lo >= 0) || (hi == -1 && (long long)lo < 0))
        return (double)(long long)lo;
    return fma((double)hi, 0x1p64, (double)lo);
}


// Inclusive scans of two i128 values per thread over the block, in one
// pass with one barrier.  The warp totals go through shared memory as
// 64-bit halves (w64: 4 x 32 words), so every shared access is 8 bytes.  No
// trailing barrier: a caller that writes w64 again must synchronise first.
struct I128Pair {
    i128 a, b;
};
__device__ __forceinline__ I128Pair block_inclusive_scan2_i128(i128 a, i128 b,
                                                               unsigned long long *w64) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const i128 ta = shfl_up_i128(a, o), tb = shfl_up_i128(b, o);
        if (lane >= o) {
            a += ta;
            b += tb;
        }
    }
    if (lane == 31) {
        w64[w] = (unsigned long long)a;
        w64[32 + w] = (unsigned long long)(a >> 64);
        w64[64 + w] = (unsigned long long)b;
        w64[96 + w] = (unsigned long long)(b >> 64);
    }
    __syncthreads();
    i128 oa = 0, ob = 0;
    for (int i = 0; i < w; i++) {
        oa += (i128)(((unsigned __int128)w64[32 + i] << 64) | w64[i]);
        ob += (i128)(((unsigned __int128)w64[96 + i] << 64) | w64[64 + i]);
    }
    I128Pair r;
    r.a = a + oa;
    r.b = b + ob;
    return r;
}

// Sum of three i128 values over the block (all threads get the sums).
static __device__ void block_sum3_i128(i128 &a, i128 &b, i128 &c, i128 *sh /*[96]*/) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        a += shfl_down_i128(a, o);
        b += shfl_down_i128(b, o);
        c += shfl_down_i128(c, o);
    }
    if (lane == 0) { sh[w] = a; sh[32 + w] = b; sh[64 + w] = c; }
    __syncthreads();
    a = 0; b = 0; c = 0;
    for (int i = 0; i < nw; i++) { a += sh[i]; b += sh[32 + i]; c += sh[64 + i]; }
    __syncthreads();
}

// Block sum of K values per thread, fixed order; result valid in thread 0
// (in fact in every lane of warp 0).  Warp sums by shuffles; the cross-warp
// sum of each value by warp 0: for float64 (a slow pipe on GB300, so the
// dependent chain matters) a butterfly over the warp sums, one value at a
// time; for float32 lane i adds value i over the warps.
// Sums of 16 float32 values over the 32 lanes of a warp by recursive
// halving: at offset o = 16, 8, 4, 2 a lane keeps the half of its values
// that bit o of its lane index selects, adds the partner's (lane ^ o) copy
// of that half, and sends it the other half; a last exchange at offset 1
// completes the sums.  Lanes 2i and 2i+1 return the warp sum of value i.
// 16 shuffles instead of the 80 of 16 separate trees; the order of the
// additions is fixed.
__device__ __forceinline__ float warp_sum16_halving(const float (&v)[16], int lane) {
    float h8[8], h4[4], h2[2];
    const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4, b2 = lane & 2;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const float send = b16 ? v[i] : v[i + 8];
        const float keep = b16 ? v[i + 8] : v[i];
        h8[i] = keep + __shfl_xor_sync(kFull, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float send = b8 ? h8[i] : h8[i + 4];
        const float keep = b8 ? h8[i + 4] : h8[i];
        h4[i] = keep + __shfl_xor_sync(kFull, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float send = b4 ? h4[i] : h4[i + 2];
        const float keep = b4 ? h4[i + 2] : h4[i];
        h2[i] = keep + __shfl_xor_sync(kFull, send, 4);
    }
    const float send = b2 ? h2[0] : h2[1];
    const float keep = b2 ? h2[1] : h2[0];
    const float h1 = keep + __shfl_xor_sync(kFull, send, 2);
    return h1 + __shfl_xor_sync(kFull, h1, 1);
}

template <int K, typename T>
static __device__ void block_sum_t(T (&v)[K], T *sh /*[32*K]*/) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < K; i++)
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(kFull, v[i], o);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < K; i++) sh[w * K + i] = v[i];
    __syncthreads();
    if (w == 0) {
        static_assert(K <= 32, "one lane per value");
        if (sizeof(T) == 8) {
#pragma unroll
            for (int i = 0; i < K; i++) {
                T s = lane < nw ? sh[lane * K + i] : (T)0;
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
                v[i] = s;
            }
        } else {
            T s = 0;
            if (lane < K)
                for (int j = 0; j < nw; j++) s += sh[j * K + lane];
#pragma unroll
            for (int i = 0; i < K; i++) v[i] = __shfl_sync(kFull, s, i);
        }
    }
    __syncthreads();
}

// Sums of K float64 values per thread over a block (warp trees, then warp 0
// over the warp sums), valid in lane 0 of warp 0.  The adds run in the
// predicated lanes only (31 lane-adds per warp and value instead of 160):
// GB300 issues float64 at 2 lanes per clock per SM, so the full butterfly
// of block_sum_t costs more than the rest of a small solve.
template <int K>
__device__ __forceinline__ void block_sum_f64k(double (&v)[K], double *slot /*[32*K]*/) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < K; i++) {
            const double u = __shfl_down_sync(kFull, v[i], o);
            if (lane < o) v[i] += u;
        }
    }
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < K; i++) slot[w * K + i] = v[i];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int i = 0; i < K; i++) v[i] = lane < nw ? slot[lane * K + i] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            if (o >= nw) continue;            // warp-uniform: only the levels nw needs
#pragma unroll
            for (int i = 0; i < K; i++) {
                const double u = __shfl_down_sync(kFull, v[i], o);
                if (lane < o) v[i] += u;
            }
        }
    }
}

__device__ __forceinline__ double block_sum_f64(double v, double *slot /*[32]*/) {
    double a[1] = {v};
    block_sum_f64k<1>(a, slot);
    return a[0];
}

// Per-node diagnostics contribution of node g with field E (float64) and its
// float32 copy: field energy sum and the mode sums (float32 twiddles).
struct NodeDiag {
    double fe;
    float re[PIC_NMODES], im[PIC_NMODES];
};

__device__ __forceinline__ void node_diag_reset(NodeDiag &d) {
    d.fe = 0.0;
#pragma unroll
    for (int m = 0; m < PIC_NMODES; m++) { d.re[m] = 0.f; d.im[m] = 0.f; }
}

// The mode sums of node g: E32 e^{-i m theta}, theta = 2 pi g / NG, for
// m = 1..8, by one sincospi and the rotation e^{-i m theta} =
// e^{-i (m-1) theta} e^{-i theta} (float32; a diagnostic).
__device__ __forceinline__ void node_diag(NodeDiag &d, int g, int ng, double E, float E32) {
    d.fe = fma(E, E, d.fe);
    float s1, c1;
    sincospif(2.0f * (float)g / (float)ng, &s1, &c1);
    float cm = c1, sm = s1;            // cos(m theta), sin(m theta)
#pragma unroll
    for (int m = 0; m < PIC_NMODES; m++) {
        d.re[m] = fmaf(E32, cm, d.re[m]);
        d.im[m] = fmaf(-E32, sm, d.im[m]);
        const float cn = cm * c1 - sm * s1;
        const float sn = sm * c1 + cm * s1;
        cm = cn;
        sm = sn;
    }
}

// The cluster's diagnostics summed over its blocks, in one block (its
// threads read the other blocks' shared memory).  T holds a block's slice
// diagnostics: diag[kDiagFields], the push sums kv[2] and the integer charge
// cq.  Value f (f < kDiagFields: diag[f]; kDiagFields, +1: kv; kDiagFields + 2:
// cq) takes 8 lanes; lane k adds blocks KMAXC/8 k ... KMAXC/8 (k+1) - 1, then a
// fixed xor butterfly over the 8 lanes.  All remote reads are in flight
// together and the float64 sum is three levels deep.  The trip count depends
// on the block size only, so every lane takes part in the shuffles (the block
// size is a multiple of 32).
template <int KMAXC, class T>
__device__ __forceinline__ void cluster_diag_sums(cooperative_groups::cluster_group &cl, T &mine,
                                                  double *tot, unsigned long long *tot_cq) {
    static_assert(KMAXC == 8 || KMAXC == 16, "8 lanes per value");
    constexpr int kPer = KMAXC / 8;
    constexpr int kSlots = (kDiagFields + 3) * 8;
    const int C = (int)cl.num_blocks(), t = threadIdx.x;
    for (int base = 0; base < kSlots; base += (int)blockDim.x) {
        const int u = base + t, f = u >> 3, k = u & 7;
        const bool isq = f == kDiagFields + 2;
        const bool act = f < kDiagFields + 3;
        const int fd = act && !isq ? f : 0;
        double sv = 0.0;
        unsigned long long sq = 0ull;
#pragma unroll
        for (int h = 0; h < kPer; h++) {
            const int b = kPer * k + h;
            const T *pe = cl.map_shared_rank(&mine, b < C ? b : 0);
            const bool use = act && b < C;
            sv += (use && !isq) ? (fd < kDiagFields ? pe->diag[fd] : pe->kv[fd - kDiagFields]) : 0.0;
            sq += (use && isq) ? pe->cq : 0ull;
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            sv += __shfl_xor_sync(kFull, sv, o);
            sq += __shfl_xor_sync(kFull, sq, o);
        }
        if (act && k == 0) {
            if (isq) *tot_cq = sq;
            else tot[f] = sv;
        }
    }
}

}  // namespace pic
