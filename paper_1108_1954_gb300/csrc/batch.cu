// batch.cu -- many independent PIC runs advanced in one persistent launch.
//
// The launch is a grid of thread-block clusters (C blocks each, one or more
// clusters per GPC).  A cluster takes the next run from a work queue (an
// atomic ticket over the runs ordered largest first, so the longest runs
// start first) and advances it through all its steps on chip; then it takes
// the next run.  Nothing on the data path crosses a cluster: no grid-wide
// barrier, no global atomics.  Per step, with the run's NG nodes split into C
// slices of P = ceil(NG/C) nodes and its particles into C contiguous parts:
//
//   A  each block pushes its particles (gather from its own copy of E in
//      shared memory, kick, drift, wrap) and deposits them into its own
//      fixed-point tile -- the same device code as the single-run push;
//      cluster barrier;
//   B  each block sums the C tiles over its node slice through distributed
//      shared memory, forms R_g = N 2^24 - NG rho_q[g], scans R and g R over
//      its slice and takes the slice sums from the scan's warp totals;
//      cluster barrier; from all slices' sums it has the prefixes the exact
//      integer solve needs (as in field.cu) and computes E (Eq. 7 via the
//      flux form of Eq. 6) for its slice in 128-bit integers, float64 at the
//      last conversion; cluster barrier;
//   C  each block copies the other slices of E into its own shared copy
//      (one node of each peer per thread, no division by the slice size);
//      block 0 sums the slice diagnostics over the blocks and writes the
//      step's history rows just before the next step's first barrier.
// A run with a sort interval S > 0 first sorts its particles by cell before
// every step n > 0 with n % S == 0 (the steps at which the single run sorts):
// a stable counting sort inside the cluster (cluster_sort below), from the
// run's buffers into its second pair, which then holds the state.
//
// A slice has at most one node per thread (ceil(NG/C) <= block, checked by
// the pool), so the integer solve of a slice is one block-wide scan.
//
// Every shared word a block reads from a peer was written before a cluster
// barrier that the reader has passed, and is next overwritten (or its block
// exits) only after a later barrier the reader must also reach, so three
// barriers per step suffice.  The particles and E of a run are bit-identical to the single-run
// path (the same operations on the same numbers; the density is an exact
// integer).  The diagnostics sum in a different order and agree to rounding.
#include <cooperative_groups.h>

#include "field_ops.cuh"
#include "particle_ops.cuh"

namespace cg = cooperative_groups;

namespace pic {
namespace {

constexpr int kU = 1;                   // float4 groups per thread per iteration (one: fewer spills in the 64-register build)
constexpr int kMaxCluster = 8;          // blocks per cluster (portable limit)

// The part of a block's shared memory its peers read.
struct Exchange {
    i128 s0, s1;                  // slice sums of R and g R
    double kv[2];                 // push sums (v_old v_new, v_new)
    double diag[kDiagFields];     // slice diagnostics
    unsigned long long cq;        // slice sum of rho_q
    unsigned sort_total;          // the sort: particles in the block's cell slice
    int ticket;                   // block 0: the run being processed
};

// Extra words of each tile array beyond NG + 2: the sort keeps a table of
// C x ceil(NG/C) <= NG + C - 1 words in one of them.
constexpr int kTilePad = kMaxCluster + 8;

// The sort key of a cell coordinate: trunc(u) clamped to [0, NG-1] (NaN to
// 0), the key of the single run's counting sort (sort.cu).
__device__ __forceinline__ unsigned sort_key(float u, int ng) {
    u = u > 0.0f ? u : 0.0f;
    const float top = (float)(ng - 1);
    u = u < top ? u : top;
    return (unsigned)u;
}

// Stable counting sort of one run's particles by cell, in one cluster.
// Block r owns the contiguous particle chunk [c0, c1) (the chunks in rank
// order cover the run) and the cell slice [b0, b1) of at most one cell per
// thread.  Four cluster barriers:
//   count    each block counts the cells of its chunk into tile.lo;
//   #1       the owner of cell g reads the C blocks' counts of g and forms
//            the per-block exclusive prefixes and the cell total; a block
//            scan over its slice gives the slice-local bases and the slice
//            total, published in ex.sort_total;
//   #2       every owner adds the totals of the slices before its own and
//            writes its table T[r'][g - b0] = first slot of block r' in cell
//            g into tile.hi;
//   #3       every block reads its first slot of every cell from the owners'
//            tables into tile.lo and scatters its chunk in order, 256
//            particles at a time (lanes of one cell ranked by match, warps
//            taking their slots one after the other), into xa, va;
//   #4       the scattered particles are visible to the whole cluster.
// The order within a cell is the input order, so the result is the unique
// stable order by cell: the single run's sort, bit for bit.
__device__ void cluster_sort(const BatchArgs &a, cg::cluster_group &cl, Exchange &ex,
                             const Tile &tile, const float *X, const float *V, float *XA,
                             float *VA, long long n, int ng, long long c0, long long c1,
                             int b0, int b1, int P) {
    __shared__ unsigned wsum[32];
    const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
    const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nwarp = bs >> 5;
    // count (the tile is empty at the start of a step)
    for (long long i = c0 + tid; i < c1; i += bs) atomicAdd(&tile.lo[sort_key(X[i], ng)], 1u);
    cl.sync();                                                        // #1
    const int g = b0 + tid;
    const bool mine = g < b1;
    unsigned cnt[kMaxCluster];
#pragma unroll
    for (int b = 0; b < kMaxCluster; b++)
        cnt[b] = (mine && b < C) ? cl.map_shared_rank(tile.lo, b)[g] : 0u;
    unsigned tot = 0;
#pragma unroll
    for (int b = 0; b < kMaxCluster; b++) tot += cnt[b];
    // block-wide exclusive scan of the cell totals over the slice
    unsigned inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    unsigned woff = 0, stot = 0;
    for (int w = 0; w < nwarp; w++) {
        if (w < warp) woff += wsum[w];
        stot += wsum[w];
    }
    const unsigned local = woff + inc - tot;          // slots before g within the slice
    if (tid == 0) ex.sort_total = stot;
    cl.sync();                                                        // #2
    unsigned before = 0;                               // particles in slices < r
    if (tid < 32) {
        unsigned t = (tid < r) ? cl.map_shared_rank(&ex.sort_total, tid)[0] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(kFull, t, o);
        if (tid == 0) wsum[0] = t;
    }
    __syncthreads();
    before = wsum[0];
    if (mine) {
        unsigned slot = before + local;
#pragma unroll
        for (int b = 0; b < kMaxCluster; b++) {
            if (b < C) tile.hi[b * P + tid] = slot;
            slot += cnt[b];
        }
    }
    cl.sync();                                                        // #3
    // this block's first slot of every cell, from the cell's owner
    for (int h = tid; h < ng; h += bs) {
        const int o = h / P;
        tile.lo[h] = cl.map_shared_rank(tile.hi, o)[r * P + (h - o * P)];
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (long long i0 = c0; i0 < c1; i0 += bs) {
        const long long i = i0 + tid;
        const bool valid = i < c1;
        const float x = valid ? X[i] : 0.0f, v = valid ? V[i] : 0.0f;
        const unsigned key = valid ? sort_key(x, ng) : 0xffffffffu;
        const unsigned peers = __match_any_sync(kFull, key);
        const int leader = __ffs(peers) - 1;
        unsigned base = 0;
        for (int w = 0; w < nwarp; w++) {
            if (w == warp && valid && lane == leader) {
                base = tile.lo[key];
                tile.lo[key] = base + (unsigned)__popc(peers);
            }
            __syncthreads();
        }
        base = __shfl_sync(kFull, base, leader);
        if (valid) {
            const unsigned long long dst = (unsigned long long)base + __popc(peers & lt);
            if (dst < (unsigned long long)n) {
                XA[dst] = x;
                VA[dst] = v;
            } else {
                atomicOr(a.err, kErrSortKey);
            }
        }
    }
    cl.sync();                                                        // #4
    // the tile empty again for the push (hi held the table: C P words)
    for (int j = tid; j < ng + kTilePad; j += bs) {
        tile.lo[j] = 0u;
        tile.hi[j] = 0u;
    }
    __syncthreads();
}

template <int VARIANT>
__device__ void run_steps(const BatchArgs &a, const BatchRun &R, cg::cluster_group &cl,
                          Exchange &ex, Tile &tile, float *sE, double *shd,
                          float *shf) {
    __shared__ i128 pre[4];
    __shared__ __align__(16) unsigned long long scan64[4 * 32];
    const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
    const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31;
    const PushConsts c = R.pc;
    const int ng = c.ng;
    const bool push = a.push != 0;
    const int steps = push ? R.steps : 1;
    const long long step0 = *R.step;
    const long long ntot = R.weight_total;

    // E of the current step, ghost-padded; empty tile
    for (int j = tid; j < ng + 2; j += bs) {
        sE[j] = R.E32[j == 0 ? ng - 1 : (j == ng + 1 ? 0 : j - 1)];
        tile.lo[j] = 0u;
        tile.hi[j] = 0u;
    }
    __syncthreads();

    const int P = (ng + C - 1) / C;
    const int b0 = min(ng, r * P), b1 = min(ng, b0 + P);
    const long long n4 = R.n >> 2;
    const long long qlo = n4 * r / C, qhi = n4 * (r + 1) / C;
    // the state's buffers and the sort's destination; they swap after a sort
    float *X = R.x, *V = R.v, *XA = R.xa, *VA = R.va;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    // Block 0: the history rows of step s from the blocks' slice
    // diagnostics (cluster_diag_sums); thread 0 writes the scalars and warp 1
    // the mode amplitudes.  Called for step s just before the next step's first
    // cluster barrier (where block 0 would wait for its peers anyway), or
    // after the last step: the peers rewrite their slice diagnostics only
    // after that barrier, and stay resident until block 0 has passed it.
    __shared__ double tot[kDiagFields + 2];
    __shared__ unsigned long long cqt;
    auto write_rows = [&](int s) {
        cluster_diag_sums<kMaxCluster>(cl, ex, tot, &cqt);
        __syncthreads();                          // block 0 only
        const long long n = push ? step0 + s + 1 : step0 + s;
        pic_diag_row *row = &R.hist[n % R.hist_len];
        if (tid == 0) {
            if (push) {
                pic_diag_row *prev = &R.hist[(step0 + s) % R.hist_len];
                prev->kinetic = 0.5 * R.mass * tot[kDiagFields];
                prev->momentum = R.mass * tot[kDiagFields + 1];
            }
            const double qnan = __longlong_as_double(0x7ff8000000000000ll);
            row->step = n;
            row->kinetic = qnan;
            row->momentum = qnan;
            row->field = 0.5 * R.dx * tot[kDiagFE];
            row->charge = tot[kDiagCharge];
            row->charge_q = (long long)cqt;
        }
        const int mt = bs >= 64 ? tid - 32 : tid;
        if (mt >= 0 && mt < PIC_NMODES) {
            const double re = tot[kDiagModes + 2 * mt], im = tot[kDiagModes + 2 * mt + 1];
            row->mode[mt] = sqrt(re * re + im * im) * R.k_mode;
        }
        __syncthreads();                          // tot and cqt free again
    };

    for (int s = 0; s < steps; s++) {
        const bool last = s == steps - 1;
        const long long nabs = step0 + s;
        if (push && R.sort_interval > 0 && nabs > 0 && nabs % R.sort_interval == 0) {
            // the sort touches only the tiles and ex.sort_total: the slice
            // diagnostics of step s-1 that block 0 reads below stay as they
            // are until this step's barrier #2
            cluster_sort(a, cl, ex, tile, X, V, XA, VA, R.n, ng, 4 * qlo,
                         r == C - 1 ? R.n : 4 * qhi, b0, b1, P);
            float *t = X; X = XA; XA = t;
            t = V; V = VA; VA = t;
        }
        float4 *x4 = reinterpret_cast<float4 *>(X);
        float4 *v4 = reinterpret_cast<float4 *>(V);
        // ---- A: push + deposit into the own tile; kU float4 groups per
        // thread per iteration, the next iteration's loads issued first
        float ke = 0.0f, mom = 0.0f;
        {
            const long long span = (long long)bs * kU;
            float4 cx[kU], cv[kU];
#pragma unroll
            for (int u = 0; u < kU; u++) {
                const long long q = qlo + u * bs + tid;
                cx[u] = q < qhi ? __ldcg(x4 + q) : zero4;
                cv[u] = (push && q < qhi) ? __ldcg(v4 + q) : zero4;
            }
            for (long long q0 = qlo; q0 < qhi; q0 += span) {
                float4 nx[kU], nv[kU];
#pragma unroll
                for (int u = 0; u < kU; u++) {
                    const long long q = q0 + span + u * bs + tid;
                    nx[u] = q < qhi ? __ldcg(x4 + q) : zero4;
                    nv[u] = (push && q < qhi) ? __ldcg(v4 + q) : zero4;
                }
#pragma unroll
                for (int u = 0; u < kU; u++) {
                    const long long q = q0 + u * bs + tid;
                    const bool valid = q < qhi;
                    float4 xx = cx[u], vv = cv[u];
                    if (push && valid) {
                        push_particle(xx.x, vv.x, sE, c, ke, mom);
                        push_particle(xx.y, vv.y, sE, c, ke, mom);
                        push_particle(xx.z, vv.z, sE, c, ke, mom);
                        push_particle(xx.w, vv.w, sE, c, ke, mom);
                    }
                    deposit4<VARIANT>(tile, xx, valid, c, a.err, lane);
                    if (push && valid) {
                        __stcg(x4 + q, xx);
                        __stcg(v4 + q, vv);
                    }
                }
#pragma unroll
                for (int u = 0; u < kU; u++) { cx[u] = nx[u]; cv[u] = nv[u]; }
            }
        }
        if (r == 0 && tid < 32) {                 // the last N mod 4 particles
            const long long i = n4 * 4 + lane;
            const bool valid = i < R.n;
            float xs = valid ? X[i] : 0.0f, vs = valid && push ? V[i] : 0.0f;
            if (push && valid) push_particle(xs, vs, sE, c, ke, mom);
            deposit_one<VARIANT>(tile, xs, valid, c, a.err, lane);
            if (push && valid) { X[i] = xs; V[i] = vs; }
        }
        if (r == 0 && s > 0) write_rows(s - 1);     // the previous step's rows
        cl.sync();                                                    // #1

        // ---- B: node slice sums over the cluster's tiles
        // one node per thread: g = b0 + tid (the pool keeps ceil(NG/C) <= block)
        const int g = b0 + tid;
        const bool mine = g < b1;
        // the C blocks' words for this node, all remote loads issued together
        unsigned long long rq = 0;
        if (mine) {
            unsigned lo[kMaxCluster], hi[kMaxCluster];
#pragma unroll
            for (int b = 0; b < kMaxCluster; b++) {
                lo[b] = b < C ? cl.map_shared_rank(tile.lo, b)[g + 1] : 0u;
                hi[b] = b < C ? cl.map_shared_rank(tile.hi, b)[g + 1] : 0u;
            }
#pragma unroll
            for (int b = 0; b < kMaxCluster; b++)
                rq += ((unsigned long long)hi[b] << 32) | lo[b];
            // the ghost words: index 0 (node -1) folds onto node NG-1, index
            // NG+1 (node NG) onto node 0
            // (both for NG = 1), the blocks' words read together
            for (int side = 0; side < 2; side++) {
                const bool fold = side == 0 ? g == ng - 1 : g == 0;
                if (!fold) continue;
                const int jg = side == 0 ? 0 : ng + 1;
                unsigned glo[kMaxCluster], ghi[kMaxCluster];
#pragma unroll
                for (int b = 0; b < kMaxCluster; b++) {
                    glo[b] = b < C ? cl.map_shared_rank(tile.lo, b)[jg] : 0u;
                    ghi[b] = b < C ? cl.map_shared_rank(tile.hi, b)[jg] : 0u;
                }
#pragma unroll
                for (int b = 0; b < kMaxCluster; b++)
                    rq += ((unsigned long long)ghi[b] << 32) | glo[b];
            }
        }
        const i128 Rg = mine ? (i128)ntot - (i128)ng * (i128)rq : (i128)0;
        // one pass of the slice's inclusive scans of R_k and k R_k (the
        // slice alone: no peer's words), and the slice sums from their warp
        // totals
        const I128Pair sc = block_inclusive_scan2_i128(Rg, Rg * (i128)g, scan64);
        if (tid == 0) {
            i128 S0 = 0, S1 = 0;
            for (int w = 0; w < (bs >> 5); w++) {
                S0 += (i128)(((unsigned __int128)scan64[32 + w] << 64) | scan64[w]);
                S1 += (i128)(((unsigned __int128)scan64[96 + w] << 64) | scan64[64 + w]);
            }
            ex.s0 = S0;
            ex.s1 = S1;
        }
        cl.sync();                                                    // #2

        // prefixes from the slice sums of all blocks: one remote read per
        // lane of warp 0 (integer sums, so the order does not matter)
        if (tid < 32) {
            i128 v0 = 0, v1 = 0;
            if (tid < C) {
                const Exchange *pe = cl.map_shared_rank(&ex, tid);
                v0 = pe->s0;
                v1 = pe->s1;
            }
            i128 a0 = tid < r ? v0 : (i128)0, bb = tid < r ? v1 : (i128)0;
            // lanes C.. hold zeros: kMaxCluster lanes carry the sums
            for (int o = kMaxCluster / 2; o > 0; o >>= 1) {
                a0 += shfl_down_i128(a0, o);
                bb += shfl_down_i128(bb, o);
                v0 += shfl_down_i128(v0, o);
                v1 += shfl_down_i128(v1, o);
            }
            if (tid == 0) { pre[0] = a0; pre[1] = bb; pre[2] = v0; pre[3] = v1; }
        }
        __syncthreads();
        const i128 A0 = pre[0], B = pre[1], SR = pre[2], SS1 = pre[3];
        const i128 SP = (i128)ng * SR - SS1;          // sum_k (NG-k) R_k
        const i128 Pg = A0 + sc.a;                                          // P_g
        const i128 M = (i128)ng * Pg - SP;                                  // M_g
        // M_{g-1} = NG P_{g-1} - SP with P_{g-1} = P_g - R_g; M_{-1} = M_{NG-1}
        const i128 Mprev = g == 0 ? (i128)ng * SR - SP : (i128)ng * (Pg - Rg) - SP;
        NodeDiag d;
        node_diag_reset(d);
        if (mine) {
            const double E = R.k_e * i128_to_f64(M + Mprev);
            const float E32 = (float)E;
            sE[g + 1] = E32;
            if (g == ng - 1) sE[0] = E32;
            if (g == 0) sE[ng + 1] = E32;
            if (last) {
                // sum_{k<g} P_k = sum_{j<g} (g - j) R_j = g P_g - sum_{j<=g} j R_j
                const i128 sumP = (i128)g * Pg - (B + sc.b);
                const i128 sumM = (i128)ng * sumP - (i128)g * SP;         // sum_{k<g} M_k
                R.E64[g] = E;
                R.E32[g] = E32;
                R.phi[g] = R.k_phi * i128_to_f64(sumM);
                R.rho[g] = R.k_rho * i128_to_f64(Rg);
                R.rho_q_last[g] = rq;
            }
            node_diag(d, g, ng, E, E32);
        }
        // the block's sums of the field energy (float64), the push sums and
        // the mode sums (float32 within a warp) and the integer charge, with
        // one barrier.  Warp sums by shuffles: the field energy by the
        // predicated float64 tree, the mode sums by recursive halving.  Then,
        // beside each other, warp 0 adds the mode sums over the warps (one
        // lane per value, warp order) and warp 1 the other values (one lane
        // each, float64, warp order).  GB300's float64 pipe takes 2 lanes per
        // clock, so the float64 work stays at one tree per warp.
        {
            double fe = d.fe;
            float k0 = ke, k1 = mom;
            unsigned long long cqb = rq;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double u = __shfl_down_sync(kFull, fe, o);
                if (lane < o) fe += u;
                k0 += __shfl_down_sync(kFull, k0, o);
                k1 += __shfl_down_sync(kFull, k1, o);
                cqb += __shfl_down_sync(kFull, cqb, o);
            }
            float md[2 * PIC_NMODES];
#pragma unroll
            for (int m = 0; m < PIC_NMODES; m++) { md[2 * m] = d.re[m]; md[2 * m + 1] = d.im[m]; }
            static_assert(2 * PIC_NMODES == 16, "16 mode sums per warp");
            const float msum = warp_sum16_halving(md, lane);   // value lane/2
            const int w = tid >> 5, nw = bs >> 5;
            __shared__ unsigned long long cqw[32];
            if ((lane & 1) == 0) shf[(lane >> 1) * 32 + w] = msum;
            if (lane == 0) {
                shd[w] = fe;
                shd[32 + w] = (double)k0;
                shd[64 + w] = (double)k1;
                cqw[w] = cqb;
            }
            __syncthreads();
            const int wo = nw > 1 ? 1 : 0;        // the warp of the other values
            if (w == 0 && lane < 2 * PIC_NMODES) {
                float sm = 0.0f;
                for (int j = 0; j < nw; j++) sm += shf[lane * 32 + j];
                ex.diag[kDiagModes + lane] = (double)sm;
            }
            if (w == wo && lane < 3) {
                double sd = 0.0;
                for (int j = 0; j < nw; j++) sd += shd[lane * 32 + j];
                if (lane == 0) ex.diag[kDiagFE] = sd;
                else ex.kv[lane - 1] = sd;
            }
            if (w == wo && lane == 3) {
                unsigned long long t = 0;
                for (int j = 0; j < nw; j++) t += cqw[j];
                ex.cq = t;
                ex.diag[kDiagKE] = 0.0;
                ex.diag[kDiagMom] = 0.0;
                ex.diag[kDiagCharge] = r == 0 ? R.dx * R.k_rho * i128_to_f64(SR) : 0.0;
            }
        }
        cl.sync();                                                    // #3

        // ---- C: the other slices of E into the own copy: thread t takes
        // node o P + t of every peer o (a slice has at most one node per
        // thread), all remote loads in flight together; then the tile is
        // cleared for the next step
        {
            float e[kMaxCluster];
#pragma unroll
            for (int o = 0; o < kMaxCluster; o++) {
                const int go = o * P + tid;
                e[o] = (o < C && o != r && tid < P && go < ng) ? cl.map_shared_rank(sE, o)[go + 1]
                                                                : 0.0f;
            }
#pragma unroll
            for (int o = 0; o < kMaxCluster; o++) {
                const int go = o * P + tid;
                if (o < C && o != r && tid < P && go < ng) {
                    sE[go + 1] = e[o];
                    if (go == ng - 1) sE[0] = e[o];
                    if (go == 0) sE[ng + 1] = e[o];
                }
            }
            for (int j = tid; j < ng + 2; j += bs) {
                tile.lo[j] = 0u;
                tile.hi[j] = 0u;
            }
        }
        __syncthreads();                          // sE and the tile complete
    }
    if (r == 0) write_rows(steps - 1);
    if (r == 0 && tid == 0 && push) *R.step = step0 + steps;
}

// MINB = 1: up to 128 registers, no spills; MINB = 2: 64 registers, two
// 512-thread blocks per SM (twice the warps), spills in the per-step solve.
template <int VARIANT, int MINB>
__global__ void __launch_bounds__(512, MINB) pic_batch_kernel(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Exchange ex;
    __shared__ __align__(16) double shd[32 * 3];
    __shared__ __align__(16) float shf[32 * 2 * PIC_NMODES];
    cg::cluster_group cl = cg::this_cluster();
    const int ngm = a.ng_max;
    Tile tile;
    tile.lo = reinterpret_cast<unsigned *>(smem_raw);
    tile.hi = tile.lo + ngm + kTilePad;
    float *sE = reinterpret_cast<float *>(tile.hi + ngm + kTilePad);
    for (;;) {
        if (cl.block_rank() == 0 && threadIdx.x == 0) ex.ticket = (int)atomicAdd(a.next, 1u);
        cl.sync();
        const int ticket = *cl.map_shared_rank(&ex.ticket, 0);
        // every block has read block 0's ticket before block 0 may overwrite
        // it or exit (a block's shared memory must not be read after it exits)
        cl.sync();
        if (ticket >= a.nrun) break;
        const BatchRun R = a.runs[a.order[ticket]];
        if (!(a.push && R.steps == 0))
            run_steps<VARIANT>(a, R, cl, ex, tile, sE, shd, shf);
        cl.sync();
    }
}

using BatchKernel = void (*)(BatchArgs);

template <int MINB>
BatchKernel pick_batch_minb(int variant) {
    switch (variant) {
        case PIC_DEPOSIT_ATOMIC: return &pic_batch_kernel<PIC_DEPOSIT_ATOMIC, MINB>;
        case PIC_DEPOSIT_MATCH: return &pic_batch_kernel<PIC_DEPOSIT_MATCH, MINB>;
        case PIC_DEPOSIT_QUAD: return &pic_batch_kernel<PIC_DEPOSIT_QUAD, MINB>;
        case PIC_DEPOSIT_PAIR: return &pic_batch_kernel<PIC_DEPOSIT_PAIR, MINB>;
        default: return nullptr;
    }
}

// variant + 16 * (minb - 1) selects the instantiation
BatchKernel pick_batch(int code) {
    const int variant = code & 15, minb = code >> 4 ? 2 : 1;
    return minb == 2 ? pick_batch_minb<2>(variant) : pick_batch_minb<1>(variant);
}

}  // namespace

size_t batch_smem_bytes(int ng_max, int cluster, int block) {
    (void)cluster;
    (void)block;
    return (size_t)(ng_max + kTilePad) * 8 + (size_t)(ng_max + 2) * 4;
}

cudaError_t batch_prepare_attributes() {
    const int bytes = (int)batch_smem_bytes(PIC_NCELL_MAX, 8, 512);
    const int vs[4] = {PIC_DEPOSIT_ATOMIC, PIC_DEPOSIT_MATCH, PIC_DEPOSIT_QUAD, PIC_DEPOSIT_PAIR};
    for (int v : vs)
        for (int m = 0; m < 2; m++) {
            cudaError_t e = cudaFuncSetAttribute(pick_batch(v + 16 * m),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

static void batch_config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr, int cluster,
                         int block, int nclusters, size_t smem, cudaStream_t s) {
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3((unsigned)(cluster * nclusters));
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
}

int batch_max_clusters(int variant, int cluster, int block, int ng_max) {
    BatchKernel k = pick_batch(variant);
    if (!k) return 0;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    batch_config(cfg, attr, cluster, block, 1, batch_smem_bytes(ng_max, cluster, block), nullptr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_batch(const BatchArgs &a, int variant, int cluster, int block,
                         int nclusters, cudaStream_t s) {
    BatchKernel k = pick_batch(variant);
    if (!k) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    batch_config(cfg, attr, cluster, block, nclusters,
                 batch_smem_bytes(a.ng_max, cluster, block), s);
    return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace pic
