// field.cu -- the field solve that closes a PIC step (Sec. 2.2) and the
// step's diagnostics.
//
// Poisson (Eq. 6) in flux form.  With D_{g+1/2} = Phi_{g+1} - Phi_g, Eq. 6 is
// D_{g+1/2} - D_{g-1/2} = -rho_g dx^2, so D_{g+1/2} = C - dx^2 S_g with the
// prefix sum S_g = sum_{k<=g} rho_k.  A periodic Phi needs sum_g D = 0, which
// fixes C = dx^2 mean(S); Phi_0 = 0 (the gauge the paper's CG pins) and
// Phi_g = sum_{k<g} D_{k+1/2}.  The field of Eq. 7 needs only D:
//   E_g = -(Phi_{g+1} - Phi_{g-1})/(2 dx) = -(D_{g+1/2} + D_{g-1/2})/(2 dx)
//       = (dx/2) (S_g + S_{g-1} - 2 mean(S)),   S_{-1} = S_{NG-1}.
// For a neutral box this is the exact solution of the linear system the
// paper's CG iterates on (with 2 global reductions per iteration).
//
// Fixed-point mode: exact integer prefix sums.  The density is
//   rho_g = K (N 2^24 - NG rho_q[g]) = K R_g,   K = rho_ion / (N 2^24),
// with R_g an integer and sum_g R_g = 0 exactly when every particle deposited.
// All prefix sums are taken on R in 128-bit integers, exactly:
//   P_g = sum_{k<=g} R_k,  M_g = NG P_g - sum_k P_k  ( = NG (S_g - mean S)/K ),
//   E_g   = (dx/2)(K/NG) (M_g + M_{g-1}),          M_{-1} = M_{NG-1}
//   Phi_g = -dx^2 (K/NG) sum_{k<g} M_k,
// and float64 arithmetic appears only in the final conversion of each value,
// so E is within an ulp or two of the exactly rounded solution.  GB300 runs
// float64 at a small fraction of its float32 rate; this keeps the solve cheap.
// The nodes are split over the blocks of one thread-block cluster (one node
// per thread); the blocks exchange their slice sums through distributed
// shared memory, and block 0 reduces the diagnostics and writes the history
// rows.
//
// Float modes (precision study): one block (one warp per 32 nodes, at most
// kSolveThreads threads), float64 prefix scans of rho; the block then reduces
// the diagnostics, writes the history rows, clears the density accumulator
// and advances the step counter (finalize).  The paper's CG solver
// (PIC_SOLVER_CG) runs on a thread-block cluster (below).
//
// Diagnostics: field energy (1/2) dx sum E^2 in float64; mode amplitudes
// from the float32 field with float32 twiddles, summed per block in float32
// and over blocks in float64; kinetic energy and momentum from the push's
// per-block float64 sums, reduced in a fixed order.
#include <math.h>

#include <cooperative_groups.h>

#include "field_ops.cuh"

namespace cg = cooperative_groups;

namespace pic {
namespace {

constexpr int kClusterSolveThreads = 512;   // most nodes per block (one per thread)
// nodes per block of the exact solve: its per-node float64 conversions and
// diagnostics are the critical path, so spread them over up to 16 SMs
constexpr int kSolveNodesPerBlock = 256;
constexpr int kMaxSolveCluster = 16;        // blocks per cluster (16: non-portable)

// The block's share of the diagnostics, written to a.dpart[blockIdx.x]; the
// push's per-block sums are split over the solve blocks.
__device__ void write_block_partials(const SolveArgs &a, NodeDiag &d, double charge,
                                     unsigned long long cq) {
    __shared__ float shf[32 * 2 * PIC_NMODES];
    __shared__ double shd[32 * 3];
    double kv[3] = {d.fe, 0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.npartials;
         i += gridDim.x * blockDim.x) {
        kv[1] += a.partials[2 * i];
        kv[2] += a.partials[2 * i + 1];
    }
    float md[2 * PIC_NMODES];
#pragma unroll
    for (int m = 0; m < PIC_NMODES; m++) { md[2 * m] = d.re[m]; md[2 * m + 1] = d.im[m]; }
    block_sum_t<3, double>(kv, shd);
    block_sum_t<2 * PIC_NMODES, float>(md, shf);
    if (threadIdx.x == 0) {
        DiagPartial &p = a.dpart[blockIdx.x];
        p.v[kDiagFE] = kv[0];
        p.v[kDiagKE] = kv[1];
        p.v[kDiagMom] = kv[2];
        p.v[kDiagCharge] = charge;
        p.cq = cq;
        for (int m = 0; m < 2 * PIC_NMODES; m++) p.v[kDiagModes + m] = (double)md[m];
    }
}

// Last block: reduce the per-block partials in a fixed order, write the
// history rows, clear the accumulator, advance the step counter.  Field f of
// the partials is summed over the blocks by thread f.
__device__ void finalize(const SolveArgs &a, long long step) {
    __shared__ unsigned ticket;
    __shared__ double tot[kDiagFields];
    __shared__ unsigned long long tot_cq;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(a.counter, 1u);
    __syncthreads();
    if (ticket != gridDim.x - 1) return;
    __threadfence();
    // the accumulator is no longer read by any block
    const int ng = a.ng;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        if (a.mode == PIC_FP32_FIXED) a.rho_q[g] = 0ull;
        else if (a.mode == PIC_FP32_ATOMIC) a.rho_f32[g] = 0.0f;
        else a.rho_f64[g] = 0.0;
    }
    // all the partials' loads in flight at once, summed in block order
    const int f = threadIdx.x;
    const int nb = (int)gridDim.x;
    if (f < kDiagFields) {
        double part[kSolveMaxBlocks];
#pragma unroll
        for (int b = 0; b < kSolveMaxBlocks; b++) part[b] = b < nb ? __ldcg(&a.dpart[b].v[f]) : 0.0;
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < kSolveMaxBlocks; b++) acc += part[b];
        tot[f] = acc;
    } else if (f == kDiagFields) {
        unsigned long long part[kSolveMaxBlocks];
#pragma unroll
        for (int b = 0; b < kSolveMaxBlocks; b++) part[b] = b < nb ? __ldcg(&a.dpart[b].cq) : 0ull;
        unsigned long long acc = 0;
#pragma unroll
        for (int b = 0; b < kSolveMaxBlocks; b++) acc += part[b];
        tot_cq = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long n = step;
        if (a.npartials > 0) {
            pic_diag_row *row = &a.hist[n % a.hist_len];
            row->kinetic = 0.5 * a.mass * tot[kDiagKE];
            row->momentum = a.mass * tot[kDiagMom];
            n = step + 1;
            *a.dstep = n;
        }
        pic_diag_row *row = &a.hist[n % a.hist_len];
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        row->step = n;
        row->kinetic = qnan;
        row->momentum = qnan;
        row->field = 0.5 * a.dx * tot[kDiagFE];
        row->charge = tot[kDiagCharge];
        row->charge_q = (long long)tot_cq;
        *a.counter = 0u;
    }
    // the mode amplitudes one lane each (warp 1 when there is one)
    const int mt = blockDim.x >= 64 ? (int)threadIdx.x - 32 : (int)threadIdx.x;
    if (mt >= 0 && mt < PIC_NMODES) {
        const long long n = a.npartials > 0 ? step + 1 : step;
        const double re = tot[kDiagModes + 2 * mt], im = tot[kDiagModes + 2 * mt + 1];
        a.hist[n % a.hist_len].mode[mt] = sqrt(re * re + im * im) * a.k_mode;
    }
}

// ---- the cluster solves' common parts -------------------------------------

// Sum over the cluster of the blocks' values *pub (each published by its
// block before the caller's cluster barrier), the same fixed tree over the
// ranks in every warp of every block: every thread gets the same total.
__device__ __forceinline__ double cluster_total(cg::cluster_group &cl, const double *pub, int C) {
    const int lane = threadIdx.x & 31;
    double p = lane < C ? *cl.map_shared_rank(pub, lane) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (o >= C) continue;                 // uniform: only the levels C needs
        const double u = __shfl_down_sync(kFull, p, o);
        if (lane < o) p += u;
    }
    return __shfl_sync(kFull, p, 0);
}

// The part of a block's shared memory that block 0 reads for the diagnostics.
struct ClusterDiag {
    double kv[2];                 // the block's share of the push sums
    double diag[kDiagFields];     // slice diagnostics
    unsigned long long cq;        // slice sum of rho_q
};

// The block's share of the push's per-block sums, summed by warp 0 alone
// (a few dozen values; float64 adds are scarce); valid in lane 0 of warp 0.
// Issued first in the solves, so the loads overlap the rest.
__device__ __forceinline__ void push_sums_share(const SolveArgs &a, int C, int r, double (&kv)[2]) {
    kv[0] = 0.0;
    kv[1] = 0.0;
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    for (int i = r * 32 + lane; i < a.npartials; i += C * 32) {
        kv[0] += a.partials[2 * i];
        kv[1] += a.partials[2 * i + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double u0 = __shfl_down_sync(kFull, kv[0], o);
        const double u1 = __shfl_down_sync(kFull, kv[1], o);
        if (lane < o) { kv[0] += u0; kv[1] += u1; }
    }
}

// Diagnostics of a cluster solve: block sums of the nodes' contributions,
// then block 0 sums the blocks in rank order (after a cluster barrier) and
// writes the history rows (scalars by thread 0, mode m by thread m); a last
// cluster barrier keeps every block's shared memory alive until block 0 has
// read it.  charge: this block's share of the charge diagnostic.
__device__ void cluster_finish(const SolveArgs &a, cg::cluster_group &cl, ClusterDiag &cd,
                               const double (&kv)[2], const NodeDiag &d, double charge,
                               unsigned long long q, long long step) {
    __shared__ __align__(16) double shd[32];
    __shared__ __align__(16) float shf[2 * PIC_NMODES][32];       // [value][warp]
    __shared__ __align__(16) unsigned long long cqw[32];
    const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
    // The block's sums of the field energy (float64), the mode sums (float32)
    // and the integer charge with one barrier: warp sums by shuffles (the 16
    // mode sums by recursive halving), then warp 0 across the warps -- the
    // field energy by the predicated float64 tree, each mode sum by one lane
    // in warp order.
    double fe = d.fe;
    unsigned long long cqb = q;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_down_sync(kFull, fe, o);
        if (lane < o) fe += u;
        cqb += __shfl_down_sync(kFull, cqb, o);
    }
    float md[2 * PIC_NMODES];
#pragma unroll
    for (int m = 0; m < PIC_NMODES; m++) { md[2 * m] = d.re[m]; md[2 * m + 1] = d.im[m]; }
    static_assert(2 * PIC_NMODES == 16, "16 mode sums per warp");
    const float msum = warp_sum16_halving(md, lane);   // value lane/2 in lanes 2i, 2i+1
    if ((lane & 1) == 0) shf[lane >> 1][w] = msum;
    if (lane == 0) {
        shd[w] = fe;
        cqw[w] = cqb;
    }
    __syncthreads();
    if (w == 0) {
        double sf = lane < nw ? shd[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            if (o >= nw) continue;                // warp-uniform
            const double u = __shfl_down_sync(kFull, sf, o);
            if (lane < o) sf += u;
        }
        if (lane < 2 * PIC_NMODES) {
            float sm = 0.0f;
            for (int j = 0; j < nw; j++) sm += shf[lane][j];
            cd.diag[kDiagModes + lane] = (double)sm;
        }
        if (lane == 0) {
            unsigned long long sc = 0;
            for (int j = 0; j < nw; j++) sc += cqw[j];
            cd.cq = sc;
            cd.kv[0] = kv[0];
            cd.kv[1] = kv[1];
            cd.diag[kDiagFE] = sf;
            cd.diag[kDiagKE] = 0.0;
            cd.diag[kDiagMom] = 0.0;
            cd.diag[kDiagCharge] = charge;
        }
    }
    cl.sync();
    if (r == 0) {
        __shared__ double tot[kDiagFields + 2];
        __shared__ unsigned long long tot_cq;
        cluster_diag_sums<kMaxSolveCluster>(cl, cd, tot, &tot_cq);
        __syncthreads();
        const long long n = a.npartials > 0 ? step + 1 : step;
        pic_diag_row *row = &a.hist[n % a.hist_len];
        if (t == 0) {
            if (a.npartials > 0) {
                pic_diag_row *prev = &a.hist[step % a.hist_len];
                prev->kinetic = 0.5 * a.mass * tot[kDiagFields];
                prev->momentum = a.mass * tot[kDiagFields + 1];
                *a.dstep = n;
            }
            const double qnan = __longlong_as_double(0x7ff8000000000000ll);
            row->step = n;
            row->kinetic = qnan;
            row->momentum = qnan;
            row->field = 0.5 * a.dx * tot[kDiagFE];
            row->charge = tot[kDiagCharge];
            row->charge_q = (long long)tot_cq;
        }
        // the amplitudes on warp 1 (when there is one), beside thread 0's row
        const int mt = blockDim.x >= 64 ? t - 32 : t;
        if (mt >= 0 && mt < PIC_NMODES) {
            const double re = tot[kDiagModes + 2 * mt], im = tot[kDiagModes + 2 * mt + 1];
            row->mode[mt] = sqrt(re * re + im * im) * a.k_mode;
        }
    }
    cl.sync();
}

// ---- fixed-point solve on one thread-block cluster --------------------------
//
// The same exact integer solve with the nodes split into C <= 16 slices of
// ceil(NG/C) nodes: one slice per block of a cluster, one node per thread.
// Each block reads (and clears) only its own slice of the accumulator, takes
// one block pass of two inclusive scans over its slice, of R_k and of k R_k
// (I and J below, over b0 <= k <= g), and publishes its slice sums sum_k R_k
// and sum_k k R_k (the scans' warp totals, summed) in shared memory.  After a
// cluster barrier every block forms, from all slices' sums (one remote read
// per lane of warp 0; integer sums, so the order does not matter),
//   A0 = sum_{k<b0} R_k,  B = sum_{k<b0} k R_k,
//   SR = sum_k R_k,       SP = NG SR - sum_k k R_k,
// and solves its slice: P_g = A0 + I, M_g = NG P_g - SP,
// M_{g-1} = NG (P_g - R_g) - SP (M_{-1} = NG SR - SP), and
// sum_{k<g} P_k = g P_g - (B + J); then the diagnostics (cluster_finish).
// Three cluster barriers, no global atomics.
struct SliceSums {
    i128 s0, s1;                  // slice sums of R and k R
};

__global__ void __launch_bounds__(kClusterSolveThreads) pic_solve_cluster_kernel(SolveArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ SliceSums ex;
    __shared__ ClusterDiag cd;
    __shared__ i128 pre[4];
    __shared__ __align__(16) unsigned long long scan64[4 * 32];
    const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
    const int ng = a.ng, t = threadIdx.x;
    const long long step = *a.dstep;
    const long long ntot = a.weight_total;
    const int per = (ng + C - 1) / C;
    const int b0 = r * per;
    const int b1 = min(ng, b0 + per);
    const int g = b0 + t;
    const bool mine = g < b1;
    unsigned long long q = 0ull;
    if (mine) {
        q = __ldcg(&a.rho_q[g]);
        a.rho_q[g] = 0ull;            // read by this thread only
        a.rho_q_last[g] = q;
    }
    double kv[2];
    push_sums_share(a, C, r, kv);
    const i128 R = mine ? (i128)ntot - (i128)ng * (i128)q : (i128)0;
    // one pass of the slice's inclusive scans of R_k and k R_k
    const I128Pair sc = block_inclusive_scan2_i128(R, R * (i128)g, scan64);
    if (t == 0) {
        i128 S0 = 0, S1 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            S0 += (i128)(((unsigned __int128)scan64[32 + w] << 64) | scan64[w]);
            S1 += (i128)(((unsigned __int128)scan64[96 + w] << 64) | scan64[64 + w]);
        }
        ex.s0 = S0;
        ex.s1 = S1;
    }
    cl.sync();                                                        // #1

    if (t < 32) {
        i128 v0 = 0, v1 = 0;
        if (t < C) {
            const SliceSums *pe = cl.map_shared_rank(&ex, t);
            v0 = pe->s0;
            v1 = pe->s1;
        }
        i128 a0 = t < r ? v0 : (i128)0, bb = t < r ? v1 : (i128)0;
        // lanes C.. hold zeros: kMaxSolveCluster lanes carry the sums
        for (int o = kMaxSolveCluster / 2; o > 0; o >>= 1) {
            a0 += shfl_down_i128(a0, o);
            bb += shfl_down_i128(bb, o);
            v0 += shfl_down_i128(v0, o);
            v1 += shfl_down_i128(v1, o);
        }
        if (t == 0) { pre[0] = a0; pre[1] = bb; pre[2] = v0; pre[3] = v1; }
    }
    __syncthreads();
    const i128 A0 = pre[0], B = pre[1], SR = pre[2], SS1 = pre[3];
    const i128 SP = (i128)ng * SR - SS1;          // sum_k (NG-k) R_k
    const i128 P = A0 + sc.a;                                          // P_g
    const i128 M = (i128)ng * P - SP;                                  // M_g
    // M_{g-1} = NG P_{g-1} - SP with P_{g-1} = P_g - R_g; M_{-1} = M_{NG-1}
    const i128 Mprev = g == 0 ? (i128)ng * SR - SP : (i128)ng * (P - R) - SP;
    NodeDiag d;
    node_diag_reset(d);
    if (mine) {
        // sum_{k<g} P_k = sum_{j<g} (g - j) R_j = g P_g - sum_{j<=g} j R_j
        const i128 sumP = (i128)g * P - (B + sc.b);
        const i128 sumM = (i128)ng * sumP - (i128)g * SP;                // sum_{k<g} M_k
        const double E = a.k_e * i128_to_f64(M + Mprev);
        const float E32 = (float)E;
        a.rho[g] = a.k_rho * i128_to_f64(R);
        a.E64[g] = E;
        a.E32[g] = E32;
        a.phi[g] = a.k_phi * i128_to_f64(sumM);
        node_diag(d, g, ng, E, E32);
    }
    const double charge = r == 0 ? a.dx * a.k_rho * i128_to_f64(SR) : 0.0;
    cluster_finish(a, cl, cd, kv, d, charge, q, step);                // #2, #3
}

// ---- CG: the paper's field solver, on one thread-block cluster ------------
//
// Sec. 2.2 / Sec. 3.3 / Appendix A: the matrix-free conjugate gradient on the
// Eq. 6 system with Phi_0 = 0 pinned (row 0 the identity) and the last row
// taking Phi_NG = 0, from x = 0 with r = v = -rho dx^2 (r_0 = v_0 = 0),
// c = r.r; while the initial |r| > 1e-16, exactly maxit iterations of
//   z = A v, t = c / (z.v), x += t v, r -= t z, d = r.r, v = (d/c) v + r, c = d
// (the paper forces 150 and keeps the unconverged field).  Where the next
// step would divide by zero (z.v == 0, t not finite, d == 0) it stops early.
// Then Phi = x and E by Eq. 7 with periodic neighbours.  For a neutral box
// the converged x is the periodic solution in the Phi_0 = 0 gauge.
//
// The nodes are split over the blocks of one cluster, one node per thread,
// C = ceil(NG/32) <= 16 blocks: float64 issue (2 lanes per clock per SM on
// GB300) rather than threads bounds an iteration, so the nodes are spread
// over as many SMs as a cluster holds.  Float64 throughout.  Per iteration two cluster-wide
// sums (z.v and r.r): block sums, published in shared memory, then every
// warp adds the C block sums in the same fixed tree, so every thread of every
// block holds the same scalars.  The two neighbour values of v that A v needs
// from other blocks are not exchanged after the update: each block publishes
// its boundary v (before the update) and r (after it) with r.r, and the
// neighbour forms beta v + r itself -- the same operation on the same numbers
// as the owner.  So an iteration has two cluster barriers.  A published value
// is read after the barrier that follows its write and rewritten only after
// the next barrier, which every reader passes after reading it.  Divisions
// are done by one lane per warp (float64 division is a long sequence).
struct CgExchange {
    double zv, rr;                // block sums
    double v0, v1, r0, r1;        // v (before the update) and r (after) at the
                                  // slice's first and last node
    double x0, x1;                // Phi at the slice's first and last node
    i128 sr;                      // fixed point: slice sum of R
};

__device__ __forceinline__ double warp_div(double num, double den) {
    double q = 0.0;
    if ((threadIdx.x & 31) == 0) q = num / den;
    return __shfl_sync(kFull, q, 0);
}

__global__ void __launch_bounds__(kClusterSolveThreads) pic_solve_cg_kernel(SolveArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double sv[kClusterSolveThreads + 2];   // v of the slice, ghost-padded
    __shared__ CgExchange ex;
    __shared__ ClusterDiag cd;
    __shared__ double slot[32];
    __shared__ i128 sh[96];
    const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
    const int ng = a.ng, t = threadIdx.x;
    const long long step = *a.dstep;
    const double dx = a.dx;
    const int per = (ng + C - 1) / C;
    const int b0 = r * per;
    const int cnt = min(ng, b0 + per) - b0;
    const int g = b0 + t;
    const bool mine = t < cnt;
    double kv[2];
    push_sums_share(a, C, r, kv);
    double rh = 0.0;
    unsigned long long q = 0ull;
    i128 R = 0;
    if (mine) {
        if (a.mode == PIC_FP32_FIXED) {
            q = __ldcg(&a.rho_q[g]);
            a.rho_q[g] = 0ull;
            a.rho_q_last[g] = q;
            R = (i128)a.weight_total - (i128)ng * (i128)q;
            rh = a.k_rho * i128_to_f64(R);
        } else if (a.mode == PIC_FP32_ATOMIC) {
            const float acc = a.rho_f32[g];
            a.rho_f32[g] = 0.0f;
            rh = a.rho_ion + a.q_over_dx * (double)acc;
        } else {
            const double acc = a.rho_f64[g];
            a.rho_f64[g] = 0.0;
            rh = a.rho_ion + a.q_over_dx * acc;
        }
        a.rho[g] = rh;
    }
    if (a.mode == PIC_FP32_FIXED) {
        i128 z1 = 0, z2 = 0, sr = R;
        block_sum3_i128(sr, z1, z2, sh);
        if (t == 0) ex.sr = sr;
    }
    double xg = 0.0;
    double rg = (mine && g >= 1) ? (-rh * dx) * dx : 0.0;
    double vg = rg;
    if (mine) sv[t + 1] = vg;
    if (t == 0) ex.v0 = vg;
    if (t == cnt - 1) ex.v1 = vg;
    {
        const double s = block_sum_f64(rg * rg, slot);
        if (t == 0) ex.rr = s;
    }
    cl.sync();
    double c = cluster_total(cl, &ex.rr, C);
    // the neighbours' boundary v (v = r at the start)
    if (t == 0 && r > 0) sv[0] = cl.map_shared_rank(&ex, r - 1)->v1;
    if (t == cnt - 1 && r < C - 1) sv[cnt + 1] = cl.map_shared_rank(&ex, r + 1)->v0;
    __syncthreads();
    if (sqrt(c) > 1e-16 && ng > 1) {
        for (int it = 0; it < a.cg_maxit; it++) {
            double z = 0.0;
            if (mine) {
                const double vl = sv[t], vc = sv[t + 1], vr = sv[t + 2];
                z = g == 0 ? vc : (g == ng - 1 ? vl - 2.0 * vc : (vl - 2.0 * vc) + vr);
            }
            {
                const double s = block_sum_f64(z * vg, slot);
                if (t == 0) ex.zv = s;
            }
            cl.sync();                                                // S1
            const double dotzv = cluster_total(cl, &ex.zv, C);
            if (!(dotzv != 0.0)) break;
            const double tk = warp_div(c, dotzv);
            if (!isfinite(tk)) break;
            if (mine) {
                xg = fma(tk, vg, xg);
                rg = fma(-tk, z, rg);
            }
            if (t == 0) { ex.v0 = vg; ex.r0 = rg; }
            if (t == cnt - 1) { ex.v1 = vg; ex.r1 = rg; }
            {
                const double s = block_sum_f64(rg * rg, slot);
                if (t == 0) ex.rr = s;
            }
            cl.sync();                                                // S2
            const double d = cluster_total(cl, &ex.rr, C);
            if (!(d > 0.0)) break;
            const double beta = warp_div(d, c);
            if (mine) {
                vg = fma(beta, vg, rg);
                sv[t + 1] = vg;
            }
            if (t == 0 && r > 0) {
                const CgExchange *pl = cl.map_shared_rank(&ex, r - 1);
                sv[0] = fma(beta, pl->v1, pl->r1);
            }
            if (t == cnt - 1 && r < C - 1) {
                const CgExchange *pr = cl.map_shared_rank(&ex, r + 1);
                sv[cnt + 1] = fma(beta, pr->v0, pr->r0);
            }
            c = d;
            __syncthreads();
        }
    }
    // Phi = x; E by Eq. 7 with periodic neighbours (across the blocks)
    __syncthreads();
    if (mine) sv[t + 1] = xg;
    if (t == 0) ex.x0 = xg;
    if (t == cnt - 1) ex.x1 = xg;
    cl.sync();
    if (t == 0) sv[0] = cl.map_shared_rank(&ex, r > 0 ? r - 1 : C - 1)->x1;
    if (t == cnt - 1) sv[cnt + 1] = cl.map_shared_rank(&ex, r < C - 1 ? r + 1 : 0)->x0;
    __syncthreads();
    NodeDiag dg;
    node_diag_reset(dg);
    double pcharge = 0.0;
    if (mine) {
        const double E = -(sv[t + 2] - sv[t]) / (2.0 * dx);
        const float E32 = (float)E;
        a.phi[g] = xg;
        a.E64[g] = E;
        a.E32[g] = E32;
        node_diag(dg, g, ng, E, E32);
        pcharge = rh;
    }
    double charge;
    if (a.mode == PIC_FP32_FIXED) {
        i128 sr = 0;
        if (r == 0)
            for (int b = 0; b < C; b++) sr += cl.map_shared_rank(&ex, b)->sr;
        charge = r == 0 ? dx * a.k_rho * i128_to_f64(sr) : 0.0;
    } else {
        charge = dx * block_sum_f64(pcharge, slot);
    }
    cluster_finish(a, cl, cd, kv, dg, charge, q, step);
}

// ---- float modes: one block, float64 prefix scans ---------------------------

constexpr int kMaxPerThread = (PIC_NCELL_MAX + kSolveThreads - 1) / kSolveThreads;

__device__ double block_exclusive_scan_f64(double val, double *warp_tot, double &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double inc = val;
    for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < nw; i++) {
        if (i < w) off += warp_tot[i];
        tot += warp_tot[i];
    }
    __syncthreads();
    total = tot;
    return off + inc - val;
}

__global__ void __launch_bounds__(kSolveThreads) pic_solve_float_kernel(SolveArgs a) {
    __shared__ double wt[32];
    __shared__ double last_of_warp[32];
    const int ng = a.ng, T = blockDim.x, t = threadIdx.x;
    const int k = (ng + T - 1) / T;
    const int g0 = t * k;
    const long long step = *a.dstep;
    double r[kMaxPerThread], S[kMaxPerThread];
    double lsum = 0.0;
#pragma unroll
    for (int j = 0; j < kMaxPerThread; j++) {
        const int g = g0 + j;
        double rho = 0.0;
        if (j < k && g < ng) {
            const double acc = (a.mode == PIC_FP32_ATOMIC) ? (double)a.rho_f32[g] : a.rho_f64[g];
            rho = a.rho_ion + a.q_over_dx * acc;
            a.rho[g] = rho;
        }
        r[j] = rho;
        lsum += rho;
    }
    double total_rho;
    double run = block_exclusive_scan_f64(lsum, wt, total_rho);
    double ssum = 0.0;
#pragma unroll
    for (int j = 0; j < kMaxPerThread; j++) {
        run += r[j];
        S[j] = run;
        if (j < k && g0 + j < ng) ssum += run;
    }
    double stot;
    block_exclusive_scan_f64(ssum, wt, stot);
    const double Sbar = stot / (double)ng;
    // S_{g0-1}: previous thread's last S; S_{-1} = S_{NG-1} = total
    double prev_last = __shfl_up_sync(kFull, S[kMaxPerThread - 1], 1);
    const int lane = t & 31, w = t >> 5;
    if (lane == 31) last_of_warp[w] = S[kMaxPerThread - 1];
    __syncthreads();
    if (lane == 0) prev_last = (w == 0) ? total_rho : last_of_warp[w - 1];
    double dsum = 0.0;
#pragma unroll
    for (int j = 0; j < kMaxPerThread; j++)
        if (j < k && g0 + j < ng) dsum += S[j] - Sbar;
    double dtot;
    double doff = block_exclusive_scan_f64(dsum, wt, dtot);
    const double half_dx = 0.5 * a.dx, dx2 = a.dx * a.dx;
    NodeDiag d;
    node_diag_reset(d);
    double sprev = prev_last, charge = 0.0;
#pragma unroll
    for (int j = 0; j < kMaxPerThread; j++) {
        const int g = g0 + j;
        if (j < k && g < ng) {
            const double E = half_dx * ((S[j] - Sbar) + (sprev - Sbar));
            const float E32 = (float)E;
            a.E64[g] = E;
            a.E32[g] = E32;
            a.phi[g] = -dx2 * doff;
            doff += S[j] - Sbar;
            charge += r[j];
            node_diag(d, g, ng, E, E32);
        }
        sprev = S[j];
    }
    double ch[1] = {charge};
    block_sum_t<1, double>(ch, wt);
    write_block_partials(a, d, a.dx * ch[0], 0ull);
    finalize(a, step);
}

}  // namespace


// Cluster shape of the solves: C = ceil(NG / per_block) blocks (at most 16),
// ceil(NG / C) nodes each, rounded up to whole warps.  The exact solve takes
// up to 256 nodes per block, the CG 32 (both are float64-bound on GB300).
void solve_cluster_shape(int ng, int per_block, int *C, int *threads) {
    int c = (ng + per_block - 1) / per_block;
    c = c < 1 ? 1 : (c > kMaxSolveCluster ? kMaxSolveCluster : c);
    const int per = (ng + c - 1) / c;
    *C = c;
    *threads = ((per + 31) / 32) * 32;
}

cudaError_t solve_prepare_attributes() {
    cudaError_t e = cudaFuncSetAttribute(&pic_solve_cluster_kernel,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(&pic_solve_cg_kernel,
                                cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

cudaError_t launch_solve(const SolveArgs &a, cudaStream_t s) {
    if (a.solver == PIC_SOLVER_CG || a.mode == PIC_FP32_FIXED) {
        int C = 1, threads = 32;
        solve_cluster_shape(a.ng, a.solver == PIC_SOLVER_CG ? 32 : kSolveNodesPerBlock, &C,
                            &threads);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        cfg.gridDim = dim3((unsigned)C, 1, 1);
        cfg.blockDim = dim3((unsigned)threads, 1, 1);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (a.solver == PIC_SOLVER_CG) return cudaLaunchKernelEx(&cfg, pic_solve_cg_kernel, a);
        return cudaLaunchKernelEx(&cfg, pic_solve_cluster_kernel, a);
    }
    // one block, one warp per 32 nodes up to kSolveThreads (the float64
    // scans cost per warp, not per node)
    const int threads = a.ng >= kSolveThreads ? kSolveThreads : ((a.ng + 31) / 32) * 32;
    pic_solve_float_kernel<<<1, threads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pic
