// load.cu -- initial particle loading on the device (Sec. 2: "the particles
// positions and velocities are sampled according to the particle distribution
// of the specific problem"; the Appendix A set-up; the two-stream set-up of
// Sec. 4).
//
// Particle j of N:
//   x0 = (j + 1/2) L / N                       lattice ("quiet start")
//   x  = x0 - sum_m (eps_m / k_m) sin(k_m x0 + phase_m),  k_m = 2 pi m / L
//        (a density perturbation sum_m eps_m cos(k_m x + phase_m)), folded
//        into [0, L) and rounded to float32 (a value that rounds to L is 0)
//   v  = s_j v0 + vth g_j,  s_j = +1 for even j, -1 for odd j
//   g_j = sqrt(-2 ln u1) cos(2 pi u2)          Box-Muller
// with u1 = (hi24(z_{2j+1}) + 1) 2^-24 in (0, 1], u2 = hi24(z_{2j+2}) 2^-24 in
// [0, 1), z_k the k-th output of SplitMix64 seeded with `seed` (Steele, Lea &
// Flood, OOPSLA 2014): state_k = seed + k * 0x9E3779B97F4A7C15, output =
// the SplitMix64 finaliser of state_k; hi24 = the top 24 bits.
// The lattice and the fold are float64; the perturbation and the velocity
// float32.
#include <math.h>
#include <cmath>

#include "pic_internal.cuh"

namespace pic {
namespace {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed,
                                                         unsigned long long k) {
    unsigned long long z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256) pic_load_kernel(LoadArgs a) {
    // x0 in float64; perturbation, Box-Muller and v in float32
    const long long stride = (long long)gridDim.x * blockDim.x;
    const double dxp = a.length / (double)a.n;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += stride) {
        const double x0 = ((double)j + 0.5) * dxp;
        const float x0f = (float)x0;
        float disp = 0.0f;
        for (int m = 0; m < a.nmodes; m++)
            disp = fmaf(a.amp[m], sinf(fmaf(a.k[m], x0f, a.phase[m])), disp);
        double x = x0 - (double)disp;
        if (x < 0.0) x += a.length;
        else if (x >= a.length) x -= a.length;
        float xf = (float)x;
        if (!(xf < a.lengthf)) xf = 0.0f;
        if (xf < 0.0f) xf = 0.0f;
        const unsigned long long z1 = splitmix64(a.seed, 2ull * (unsigned long long)j + 1ull);
        const unsigned long long z2 = splitmix64(a.seed, 2ull * (unsigned long long)j + 2ull);
        const float u1 = (float)((z1 >> 40) + 1ull) * 0x1p-24f;
        const float u2 = (float)(z2 >> 40) * 0x1p-24f;
        const float g = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
        const float s = (j & 1) ? -1.0f : 1.0f;
        a.x[j] = xf;
        a.v[j] = fmaf(a.vth, g, s * a.v0);
    }
}

}  // namespace

int make_load_args(const pic_loading *ld, long long n, double length, float *x, float *v,
                   LoadArgs *out) {
    if (!ld || n < 1 || !(length > 0.0) || !x || !v) return PIC_EINVAL;
    if (ld->nmodes < 0 || ld->nmodes > PIC_LOAD_MAX_MODES || ld->reserved != 0) return PIC_EINVAL;
    if (!(ld->vth >= 0.0) || !std::isfinite(ld->v0) || !std::isfinite(ld->vth)) return PIC_EINVAL;
    LoadArgs a;
    a.x = x;
    a.v = v;
    a.n = n;
    a.length = length;
    a.lengthf = (float)length;
    a.v0 = (float)ld->v0;
    a.vth = (float)ld->vth;
    a.seed = ld->seed;
    a.nmodes = ld->nmodes;
    const double two_pi = 6.283185307179586476925286766559;
    for (int m = 0; m < PIC_LOAD_MAX_MODES; m++) { a.k[m] = 0.f; a.amp[m] = 0.f; a.phase[m] = 0.f; }
    for (int m = 0; m < ld->nmodes; m++) {
        if (ld->mode[m] < 1 || !std::isfinite(ld->eps[m]) || !std::isfinite(ld->phase[m])) return PIC_EINVAL;
        const double k = two_pi * ld->mode[m] / length;
        a.k[m] = (float)k;
        a.amp[m] = (float)(ld->eps[m] / k);
        a.phase[m] = (float)ld->phase[m];
    }
    *out = a;
    return PIC_OK;
}

cudaError_t launch_load(const LoadArgs &a, int sms, cudaStream_t s) {
    long long blocks = (a.n + 255) / 256;
    const long long cap = (long long)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    pic_load_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pic

extern "C" int pic_load_two_stream(const pic_loading *ld, int64_t n, double length, void *x,
                                   void *v, void *stream) {
    pic::LoadArgs a;
    int rc = pic::make_load_args(ld, n, length, (float *)x, (float *)v, &a);
    if (rc) return rc;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PIC_ECUDA;
    return pic::launch_load(a, sms, (cudaStream_t)stream) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}
