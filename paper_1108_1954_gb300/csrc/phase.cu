// phase.cu -- phase-space histogram f(x, v) of the particles (the (x, v)
// snapshots of the Sec. 4 verification test, Fig. 1), on the device; the
// range check of uploaded positions and the unit conversions of float32
// positions between physical units and cell units.
//
// Bin rule (float32, as stated in include/pic.h): ix = min(nx - 1,
// trunc(p * sx)), iv = floor((v - vmin) * (nv / (vmax - vmin))), where p is
// the stored position (the cell coordinate in the float32 modes, sx =
// nx / NG; x in PIC_FP64, sx = nx / L); a particle with iv outside [0, nv)
// is not counted.  Each block counts into a
// shared-memory copy of the grid (32-bit atomics) and adds it to the global
// counts once.
#include <cmath>

#include "pic_internal.cuh"

namespace pic {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) pic_phase_kernel(PhaseArgs<T> a) {
    extern __shared__ unsigned sh[];
    const int cells = a.nx * a.nv;
    for (int i = threadIdx.x; i < cells; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += stride) {
        const float x = (float)a.x[p], v = (float)a.v[p];
        const float fx = x * a.sx;
        const float fv = floorf((v - a.vmin) * a.sv);
        if (!(fx >= 0.0f) || !(fv >= 0.0f) || !(fv < (float)a.nv)) continue;
        int ix = (int)fx;
        ix = ix < a.nx ? ix : a.nx - 1;
        atomicAdd(&sh[(int)fv * a.nx + ix], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cells; i += blockDim.x)
        if (sh[i]) atomicAdd(&a.counts[i], sh[i]);
}

}  // namespace

template <typename T>
cudaError_t launch_phase(const PhaseArgs<T> &a, int sms, cudaStream_t s) {
    long long blocks = (a.n + 255) / 256;
    if (blocks > (long long)sms * 4) blocks = (long long)sms * 4;
    if (blocks < 1) blocks = 1;
    const size_t smem = (size_t)a.nx * a.nv * sizeof(unsigned);
    cudaError_t e = cudaFuncSetAttribute(&pic_phase_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kPhaseMaxBins * sizeof(unsigned)));
    if (e != cudaSuccess) return e;
    pic_phase_kernel<T><<<(unsigned)blocks, 256, smem, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_phase<float>(const PhaseArgs<float> &, int, cudaStream_t);
template cudaError_t launch_phase<double>(const PhaseArgs<double> &, int, cudaStream_t);

// Uploaded positions must lie in [0, L) (NaN fails); one flag per block.
namespace {
template <typename T>
__global__ void __launch_bounds__(256) check_positions_kernel(const T *x, long long n, T length,
                                                              unsigned *err) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const T xi = __ldcs(x + i);
        bad |= !(xi >= (T)0 && xi < length);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrInput);
}
}  // namespace

template <typename T>
cudaError_t launch_check_positions(const T *x, long long n, T length, unsigned *err, int sms,
                                   cudaStream_t s) {
    long long blocks = (n + 255) / 256;
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    if (blocks < 1) blocks = 1;
    check_positions_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(x, n, length, err);
    return cudaGetLastError();
}

template cudaError_t launch_check_positions<float>(const float *, long long, float, unsigned *, int,
                                                   cudaStream_t);
template cudaError_t launch_check_positions<double>(const double *, long long, double, unsigned *,
                                                    int, cudaStream_t);

// ---- float32 positions: physical units <-> cell units -----------------------
namespace {

__global__ void __launch_bounds__(256) to_cells_kernel(float *x, long long n, double to_cells,
                                                       float ngf, float length32, unsigned *err) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float xi = x[i];
        bad |= !(xi >= 0.0f && xi < length32);
        float u = (float)((double)xi * to_cells);
        u = u >= ngf ? 0.0f : u;          // a position rounding up to the box end
        x[i] = u;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrInput);
}

__global__ void __launch_bounds__(256) to_physical_kernel(const float *u, float *x, long long n,
                                                          double to_phys, float top) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float xi = (float)((double)u[i] * to_phys);
        x[i] = xi > top ? top : xi;
    }
}

__global__ void __launch_bounds__(256) check_cells_kernel(const float *u, long long n, float ngf,
                                                          unsigned *err) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float ui = u[i];
        bad |= !(ui >= 0.0f && ui < ngf);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrInput);
}

unsigned grid_for(long long n, int sms) {
    long long blocks = (n + 255) / 256;
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    if (blocks < 1) blocks = 1;
    return (unsigned)blocks;
}

}  // namespace

float below(float v) { return std::nextafter(v, 0.0f); }

cudaError_t launch_to_cells(float *x, long long n, double to_cells, float ngf, float length32,
                            unsigned *err, int sms, cudaStream_t s) {
    to_cells_kernel<<<grid_for(n, sms), 256, 0, s>>>(x, n, to_cells, ngf, length32, err);
    return cudaGetLastError();
}

cudaError_t launch_to_physical(const float *u, float *x, long long n, double to_phys,
                               float length32, int sms, cudaStream_t s) {
    to_physical_kernel<<<grid_for(n, sms), 256, 0, s>>>(u, x, n, to_phys, below(length32));
    return cudaGetLastError();
}

cudaError_t launch_check_cells(const float *u, long long n, float ngf, unsigned *err, int sms,
                               cudaStream_t s) {
    check_cells_kernel<<<grid_for(n, sms), 256, 0, s>>>(u, n, ngf, err);
    return cudaGetLastError();
}

}  // namespace pic
