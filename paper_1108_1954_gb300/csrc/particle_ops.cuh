// particle_ops.cuh -- the per-particle arithmetic of the PIC step, shared by
// the single-run fused push (push.cu) and the batched cluster kernel
// (batch.cu), so that a run gives bit-identical particles in either.
//   locate         cell of a position by the fixed-point recipe
//   fixed_weight   the right node's share trunc(f * 2^24)
//   push_particle  gather (Sec. 2.3), kick (Eq. 3), drift (Eq. 2), wrap
#pragma once

#include "pic_internal.cuh"

namespace pic {

using u64 = unsigned long long;

// 8 consecutive float32 values moved by one 32-byte vector load or store
// (the QUAD8 and PAIR8 variants; the address 32-byte aligned).  .cs:
// streamed (the single run's arrays pass once per step); .cg: cached in L2
// only (the batched kernel's runs).
struct F8 {
    float v[8];
};

template <bool CG = false>
__device__ __forceinline__ F8 ld8(const float *p) {
    F8 r;
    if (CG)
        asm volatile("ld.global.cg.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]),
                       "=f"(r.v[5]), "=f"(r.v[6]), "=f"(r.v[7])
                     : "l"(p));
    else
        asm volatile("ld.global.cs.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]),
                       "=f"(r.v[5]), "=f"(r.v[6]), "=f"(r.v[7])
                     : "l"(p));
    return r;
}

template <bool CG = false>
__device__ __forceinline__ void st8(float *p, const F8 &r) {
    if (CG)
        asm volatile("st.global.cg.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p),
                     "f"(r.v[0]), "f"(r.v[1]), "f"(r.v[2]), "f"(r.v[3]), "f"(r.v[4]),
                     "f"(r.v[5]), "f"(r.v[6]), "f"(r.v[7])
                     : "memory");
    else
        asm volatile("st.global.cs.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p),
                     "f"(r.v[0]), "f"(r.v[1]), "f"(r.v[2]), "f"(r.v[3]), "f"(r.v[4]),
                     "f"(r.v[5]), "f"(r.v[6]), "f"(r.v[7])
                     : "memory");
}

// Cell location of a float32 cell coordinate u (the fixed-point recipe):
//   s = u - 1/2, fl = floor(s), f = s - fl   (float ops, round to nearest)
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

__device__ __forceinline__ Loc locate(float u) {
    Loc l;
    const float s = __fsub_rn(u, 0.5f);
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

// Kick (Eq. 3), drift (Eq. 2, in cell units: u advances by v dt NG/L) and
// the periodic wrap to [0, NG) of one particle, given the field ep at the
// particle; accumulates v_old v_new and v_new.
__device__ __forceinline__ void kick_drift_wrap(float &u, float &v, float ep, const PushConsts &c,
                                                float &ke, float &mom) {
    const float vn = fmaf(c.qmdt, ep, v);
    ke = fmaf(v, vn, ke);
    mom += vn;
    float un = fmaf(vn, c.kdrift, u);
    un = un < 0.0f ? un + c.ngf : un;
    un = un >= c.ngf ? un - c.ngf : un;
    un = un >= c.ngf ? 0.0f : un;      // u + NG rounded up to NG: the point 0
    u = un;
    v = vn;
}

// Gather (left and right node), kick, drift, wrap.
// sE[j] = E_{(j-1) mod NG} for j = 0..NG+1 (ghost-padded).
__device__ __forceinline__ void push_particle(float &u, float &v, const float *sE,
                                              const PushConsts &c, float &ke,
                                              float &mom) {
    const Loc l = locate(u);
    const bool ok = l.j <= (unsigned)c.ng;
    const unsigned j = ok ? l.j : 0u;
    const float e0 = sE[j], e1 = sE[j + 1];
    const float ep = ok ? fmaf(l.f, e1 - e0, e0) : 0.0f;
    kick_drift_wrap(u, v, ep, c, ke, mom);
}

// Nearest-grid-point weighting (PIC_SHAPE_NGP; Sec. 2: a grid point's density
// counts the particles of its cell, and a particle feels its cell's field):
// with nodes at the cell centres the cell of u is floor(u), formed by the
// same rounded-down magic sum as locate (exact on [-1, 8193]).  Returns the
// ghost-padded tile index j = cell + 1; a valid position has j - 1 in
// [0, NG] (one unsigned test).
__device__ __forceinline__ unsigned locate_ngp(float u) {
    const float t = __fadd_rd(u, kMagic);
    return (unsigned)(__float_as_int(t) - kMagicBitsMinus1);
}

__device__ __forceinline__ void push_particle_ngp(float &u, float &v, const float *sE,
                                                  const PushConsts &c, float &ke,
                                                  float &mom) {
    const unsigned j = locate_ngp(u);
    const bool ok = j - 1u <= (unsigned)c.ng;
    const float ep = ok ? sE[j] : 0.0f;
    kick_drift_wrap(u, v, ep, c, ke, mom);
}

// Shared-memory density tiles.  GB300 has no single-instruction 64-bit
// integer add on shared memory (it runs as a compare-and-swap loop, which
// serialises badly when the lanes of a warp hit one node), so a tile keeps
// each node's 64-bit sum as two 32-bit words: a 32-bit fetch-add on the low
// word, and +1 on the high word from the one add that wraps it.  The tile is
// ghost-padded: index j is node (j-1) mod NG, j = 0..NG+1.
struct Tile {
    unsigned *lo, *hi;      // 32-bit halves of the node sums
};

__device__ __forceinline__ void tile_add(const Tile &t, unsigned j, unsigned val) {
    const unsigned old = atomicAdd(&t.lo[j], val);
    if (old + val < old) atomicAdd(&t.hi[j], 1u);
}

// Deposit one particle (all 32 lanes of the warp call this together for the
// MATCH variants).
template <int VARIANT>
__device__ __forceinline__ void deposit_one(const Tile &t, float x, bool valid,
                                            const PushConsts &c, unsigned *err, int lane) {
    if (VARIANT == kDepositNgp) {
        const unsigned j = locate_ngp(x);
        const bool ok = valid && j - 1u <= (unsigned)c.ng;
        if (valid && !ok) atomicOr(err, kErrPosition);
        if (ok) tile_add(t, j, kFixOne);
        return;
    }
    const Loc l = locate(x);
    const bool ok = valid && l.j <= (unsigned)c.ng;
    if (valid && !ok) atomicOr(err, kErrPosition);
    const unsigned W = ok ? fixed_weight(l.f) : 0u;
    if (VARIANT == PIC_DEPOSIT_ATOMIC || VARIANT == PIC_DEPOSIT_QUAD ||
        VARIANT == PIC_DEPOSIT_PAIR || VARIANT == PIC_DEPOSIT_QUAD8 ||
        VARIANT == PIC_DEPOSIT_PAIR8) {
        if (ok) {
            tile_add(t, l.j, kFixOne - W);
            tile_add(t, l.j + 1, W);
        }
    } else {
        const unsigned key = ok ? l.j : 0xffffffffu;
        const unsigned peers = __match_any_sync(kFull, key);
        const unsigned wsum = __reduce_add_sync(peers, W);
        if (ok && lane == __ffs(peers) - 1) {
            const unsigned cnt = (unsigned)__popc(peers);
            // cnt * 2^24 - wsum <= 2^29: fits the 32-bit add
            tile_add(t, l.j, (cnt << kFixBits) - wsum);
            tile_add(t, l.j + 1, wsum);
        }
    }
}

// Deposit a thread's W consecutive particles (W = 4: a float4 group; W = 8:
// the 32-byte groups of the QUAD8 / PAIR8 variants), valid per lane.
template <int VARIANT, int W>
__device__ __forceinline__ void deposit_group(const Tile &t, const float (&xs)[W], bool valid,
                                              const PushConsts &c, unsigned *err, int lane) {
    if (VARIANT == kDepositNgp) {
        // runs of equal cell among the W particles: count * 2^24 per run
        unsigned key = 0xffffffffu, cnt = 0;
        bool bad = false;
#pragma unroll
        for (int k = 0; k < W; k++) {
            const unsigned j = locate_ngp(xs[k]);
            const bool ok = valid && j - 1u <= (unsigned)c.ng;
            bad |= valid && !ok;
            if (ok && j == key) {
                cnt += kFixOne;
            } else if (ok) {
                if (key != 0xffffffffu) tile_add(t, key, cnt);
                key = j;
                cnt = kFixOne;
            }
        }
        if (key != 0xffffffffu) tile_add(t, key, cnt);
        if (bad) atomicOr(err, kErrPosition);
    } else if (VARIANT == PIC_DEPOSIT_PAIR || VARIANT == PIC_DEPOSIT_PAIR8) {
        // two open runs (key, left, right); a third key closes run a
        unsigned ka = 0xffffffffu, la = 0, ra = 0, kb = 0xffffffffu, lb = 0, rb = 0;
        bool bad = false;
#pragma unroll
        for (int k = 0; k < W; k++) {
            const Loc l = locate(xs[k]);
            const bool ok = valid && l.j <= (unsigned)c.ng;
            bad |= valid && !ok;
            const unsigned Wk = fixed_weight(l.f);
            if (!ok) continue;
            if (l.j == ka) {
                la += kFixOne - Wk;
                ra += Wk;
            } else if (l.j == kb) {
                lb += kFixOne - Wk;
                rb += Wk;
            } else if (ka == 0xffffffffu) {
                ka = l.j; la = kFixOne - Wk; ra = Wk;
            } else if (kb == 0xffffffffu) {
                kb = l.j; lb = kFixOne - Wk; rb = Wk;
            } else {
                tile_add(t, ka, la);
                tile_add(t, ka + 1, ra);
                ka = l.j; la = kFixOne - Wk; ra = Wk;
            }
        }
        if (ka != 0xffffffffu) { tile_add(t, ka, la); tile_add(t, ka + 1, ra); }
        if (kb != 0xffffffffu) { tile_add(t, kb, lb); tile_add(t, kb + 1, rb); }
        if (bad) atomicOr(err, kErrPosition);
    } else if (VARIANT == PIC_DEPOSIT_QUAD || VARIANT == PIC_DEPOSIT_QUAD8) {
        // consecutive particles of the group with equal left node are summed
        // in registers first (at most W 2^24 <= 2^27 per word), then added once
        unsigned key = 0xffffffffu, left = 0, right = 0;
        bool bad = false;
#pragma unroll
        for (int k = 0; k < W; k++) {
            const Loc l = locate(xs[k]);
            const bool ok = valid && l.j <= (unsigned)c.ng;
            bad |= valid && !ok;
            const unsigned Wk = fixed_weight(l.f);
            if (ok && l.j == key) {
                left += kFixOne - Wk;
                right += Wk;
            } else if (ok) {
                if (key != 0xffffffffu) {
                    tile_add(t, key, left);
                    tile_add(t, key + 1, right);
                }
                key = l.j;
                left = kFixOne - Wk;
                right = Wk;
            }
        }
        if (key != 0xffffffffu) {
            tile_add(t, key, left);
            tile_add(t, key + 1, right);
        }
        if (bad) atomicOr(err, kErrPosition);
    } else {
#pragma unroll
        for (int k = 0; k < W; k++) deposit_one<VARIANT>(t, xs[k], valid, c, err, lane);
    }
}

// Deposit the 4 particles of a float4 group (valid per lane).
template <int VARIANT>
__device__ __forceinline__ void deposit4(const Tile &t, const float4 &xx, bool valid,
                                         const PushConsts &c, unsigned *err, int lane) {
    const float xs[4] = {xx.x, xx.y, xx.z, xx.w};
    deposit_group<VARIANT, 4>(t, xs, valid, c, err, lane);
}

}  // namespace pic
