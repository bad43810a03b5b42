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
// The nodes are split over up to 32 blocks; each block forms the global sums
// it needs (sum_k P_k and the prefixes up to its first node) as weighted
// integer reductions over the whole grid, then converts its own nodes.  The
// last block to finish (an atomic ticket, no waiting) reduces the per-block
// diagnostics in a fixed order, writes the history rows, clears the density
// accumulator and advances the step counter.
//
// Float modes (precision study): one block, float64 prefix scans of rho.
//
// Diagnostics: field energy (1/2) dx sum E^2 in float64; mode amplitudes
// from the float32 field with float32 twiddles, summed per block in float32
// and over blocks in float64; kinetic energy and momentum from the push's
// per-block float64 sums, reduced in a fixed order.
#include <math.h>

#include "field_ops.cuh"

namespace pic {
namespace {

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
        for (int m = 0; m < PIC_NMODES; m++) {
            const double re = tot[kDiagModes + 2 * m], im = tot[kDiagModes + 2 * m + 1];
            row->mode[m] = 2.0 * sqrt(re * re + im * im) / (double)ng;
        }
        *a.counter = 0u;
    }
}

// ---- fixed-point solve: exact integer prefix sums --------------------------

__global__ void __launch_bounds__(256) pic_solve_fixed_kernel(SolveArgs a) {
    __shared__ i128 sh[96];
    const int ng = a.ng, T = blockDim.x, t = threadIdx.x;
    const long long step = *a.dstep;
    const long long ntot = a.weight_total;   // N 2^24
    const int per = (ng + gridDim.x - 1) / gridDim.x;   // nodes per block (<= T)
    const int b0 = blockIdx.x * per;
    const int b1 = min(ng, b0 + per);

    // (a) global weighted sums of R over the whole grid:
    //   A0 = sum_{k<b0} R_k, A1 = sum_{k<b0} (b0-k) R_k   (prefixes to b0)
    //   SP = sum_k (NG-k) R_k = sum_g P_g,  also sum_k R_k (= P_{NG-1}).
    i128 A0 = 0, A1 = 0, SP = 0, SR = 0;
    {
        constexpr int kBatch = 8;   // loads in flight per thread
        for (int k0 = t; k0 < ng; k0 += kBatch * T) {
            unsigned long long q[kBatch];
#pragma unroll
            for (int i = 0; i < kBatch; i++) {
                const int k = k0 + i * T;
                q[i] = k < ng ? __ldcg(&a.rho_q[k]) : 0ull;
            }
#pragma unroll
            for (int i = 0; i < kBatch; i++) {
                const int k = k0 + i * T;
                if (k < ng) {
                    const i128 R = (i128)ntot - (i128)ng * (i128)q[i];
                    SP += R * (long long)(ng - k);
                    SR += R;
                    const bool before = k < b0;
                    A0 += before ? R : (i128)0;
                    A1 += before ? R * (long long)(b0 - k) : (i128)0;
                }
            }
        }
    }
    block_sum3_i128(A0, A1, SP, sh);
    {
        i128 z1 = 0, z2 = 0;
        block_sum3_i128(SR, z1, z2, sh);
    }

    // (b) the block's nodes: one per thread
    const int g = b0 + t;
    const bool mine = g < b1;
    const unsigned long long q = mine ? a.rho_q[g] : 0ull;
    const i128 R = mine ? (i128)ntot - (i128)ng * (i128)q : (i128)0;
    i128 tot;
    const i128 P = A0 + block_inclusive_scan_i128(R, sh, tot);  // P_g
    const i128 M = (i128)ng * P - SP;                          // M_g
    // M_{g-1}: previous thread, or for the block's first node the prefix to b0
    i128 Mprev = shfl_up_i128(M, 1);
    __shared__ i128 wlast[32];
    if ((t & 31) == 31) wlast[t >> 5] = M;
    __syncthreads();
    if ((t & 31) == 0) {
        if (t == 0) {
            // M_{b0-1} = NG P_{b0-1} - SP with P_{b0-1} = A0; b0 = 0 wraps to
            // M_{NG-1} = NG SR - SP
            Mprev = (b0 == 0) ? (i128)ng * SR - SP : (i128)ng * A0 - SP;
        } else {
            Mprev = wlast[(t >> 5) - 1];
        }
    }
    // sum_{k<g} M_k = NG sum_{k<g} P_k - g SP, with
    // sum_{k<g} P_k = (sum_{k<b0} P_k) + exclusive block prefix of P
    //               = (b0 A0 - A1 + A0... ) computed as below.
    // sum_{k<b0} P_k = sum_{k<b0} sum_{j<=k} R_j = sum_{j<b0} (b0 - j) R_j = A1.
    i128 ptot;
    const i128 Pexcl = block_inclusive_scan_i128(mine ? P : (i128)0, sh, ptot) - (mine ? P : (i128)0);
    const i128 sumM = (i128)ng * (A1 + Pexcl) - (i128)g * SP;

    NodeDiag d;
    node_diag_reset(d);
    if (mine) {
        const double rho = a.k_rho * i128_to_f64(R);
        const double E = a.k_e * i128_to_f64(M + Mprev);
        const double phi = a.k_phi * i128_to_f64(sumM);
        const float E32 = (float)E;
        a.rho[g] = rho;
        a.E64[g] = E;
        a.E32[g] = E32;
        a.phi[g] = phi;
        a.rho_q_last[g] = q;
        node_diag(d, g, ng, E, E32);
    }
    // charge of the block's nodes, exactly: dx K sum R (block 0 reports all)
    const double charge = (blockIdx.x == 0) ? a.dx * a.k_rho * i128_to_f64(SR) : 0.0;
    unsigned long long cq = q;
    for (int o = 16; o > 0; o >>= 1) cq += __shfl_down_sync(kFull, cq, o);
    __shared__ unsigned long long cqw[32];
    if ((t & 31) == 0) cqw[t >> 5] = cq;
    __syncthreads();
    cq = 0;
    for (int i = 0; i < (T >> 5); i++) cq += cqw[i];
    write_block_partials(a, d, charge, cq);
    finalize(a, step);
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

int solve_blocks(int mode, int ng) {
    if (mode != PIC_FP32_FIXED) return 1;
    int nb = (ng + kSolveThreads - 1) / kSolveThreads;   // at least NG/T nodes each
    const int want = (ng + 255) / 256;                   // about 256 nodes per block
    if (want > nb) nb = want;
    return nb < kSolveMaxBlocks ? nb : kSolveMaxBlocks;
}

cudaError_t launch_solve(const SolveArgs &a, cudaStream_t s) {
    if (a.mode == PIC_FP32_FIXED) {
        const int nb = solve_blocks(a.mode, a.ng);
        const int per = (a.ng + nb - 1) / nb;
        const int threads = ((per + 31) / 32) * 32;
        pic_solve_fixed_kernel<<<nb, threads < 32 ? 32 : threads, 0, s>>>(a);
    } else {
        pic_solve_float_kernel<<<1, kSolveThreads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace pic
