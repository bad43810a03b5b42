// field_ops.cuh -- 128-bit integer helpers of the exact field solve, shared by
// the single-run solve (field.cu) and the batched cluster kernel (batch.cu).
#pragma once

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

__device__ __forceinline__ void node_diag(NodeDiag &d, int g, int ng, double E, float E32) {
    d.fe = fma(E, E, d.fe);
#pragma unroll
    for (int m = 1; m <= PIC_NMODES; m++) {
        const int ph = (int)(((long long)m * g) % ng);
        float sn, cs;
        sincospif(2.0f * (float)ph / (float)ng, &sn, &cs);
        d.re[m - 1] = fmaf(E32, cs, d.re[m - 1]);
        d.im[m - 1] = fmaf(-E32, sn, d.im[m - 1]);
    }
}

}  // namespace pic
