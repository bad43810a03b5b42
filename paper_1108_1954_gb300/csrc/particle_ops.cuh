// particle_ops.cuh -- the per-particle arithmetic of the PIC step, shared by
// the single-run fused push (push.cu) and the batched cluster kernel
// (batch.cu), so that a run gives bit-identical particles in either.
//   locate         cell of a position by the fixed-point recipe
//   fixed_weight   the right node's share trunc(f * 2^24)
//   push_particle  gather (Sec. 2.3), kick (Eq. 3), drift (Eq. 2), wrap
#pragma once

#include "pic_internal.cuh"

namespace pic {

// Cell location of a float32 position by the fixed-point recipe:
//   s = x*c - 1/2, fl = floor(s), f = s - fl   (float ops, round to nearest)
// floor(s) is formed as (s + 1.5*2^23 rounded down) - 1.5*2^23, which equals
// floorf(s) exactly for |s| < 2^22 (NG <= 8192; checked for every float in
// [-1, 8193]) and runs on the FMA pipe instead of the conversion unit; the
// rounded-down sum's bit pattern is 0x4B400000 + fl, which gives the node index
// without a float-to-int conversion.
// j = fl + 1 is the index of the left node in the ghost-padded tiles (node -1,
// the periodic image of NG-1, is j = 0); a valid position has j in [0, NG].
// A NaN, infinite or far-out-of-range position fails that one unsigned test.
struct Loc {
    unsigned j;
    float f;
};

constexpr float kMagic = 12582912.0f;          // 1.5 * 2^23
constexpr int kMagicBitsMinus1 = 0x4B400000 - 1;

__device__ __forceinline__ Loc locate(float x, float inv_dx) {
    Loc l;
    const float s = __fsub_rn(__fmul_rn(x, inv_dx), 0.5f);
    const float t = __fadd_rd(s, kMagic);
    const float fl = __fsub_rn(t, kMagic);
    l.f = __fsub_rn(s, fl);
    l.j = (unsigned)(__float_as_int(t) - kMagicBitsMinus1);
    return l;
}

// The right node's share W = trunc(f * 2^24) of a particle's 2^24.
__device__ __forceinline__ unsigned fixed_weight(float f) {
    return __float2uint_rz(__fmul_rn(f, 16777216.0f));
}

// Gather (left and right node), kick, drift, wrap.
// sE[j] = E_{(j-1) mod NG} for j = 0..NG+1 (ghost-padded).
__device__ __forceinline__ void push_particle(float &x, float &v, const float *sE,
                                              const PushConsts &c, float &ke,
                                              float &mom) {
    const Loc l = locate(x, c.inv_dx);
    const bool ok = l.j <= (unsigned)c.ng;
    const unsigned j = ok ? l.j : 0u;
    const float e0 = sE[j], e1 = sE[j + 1];
    const float ep = ok ? fmaf(l.f, e1 - e0, e0) : 0.0f;
    const float vn = fmaf(c.qmdt, ep, v);
    ke = fmaf(v, vn, ke);
    mom += vn;
    float xn = fmaf(vn, c.dt, x);
    xn = xn < 0.0f ? xn + c.length : xn;
    xn = xn >= c.length ? xn - c.length : xn;
    xn = xn >= c.length ? 0.0f : xn;   // x + L rounded up to L: the point 0
    x = xn;
    v = vn;
}

}  // namespace pic
