// sort_noalloc.cu -- the counting sort by cell for callers that cannot
// allocate device memory.
//
// Some callers cannot hand this library a workspace: frameworks whose own
// caching allocator owns all of the device memory and accepts no outside
// allocations, processes held to a fixed memory reservation, and
// latency-critical code that cannot afford the device-wide synchronisation a
// cudaMalloc implies.  For them pic_sort_noalloc runs the same four sort
// kernels as pic_sort (sort.cu), with their scratch (the per-chunk cell
// counts, the segment offsets, the cell bases and the error word) in one
// file-scope device array of kSortNoAllocScratch bytes.  Every GPU that loads
// the library keeps that array until the process exits.
//
// In host code the array's name stands for a host-side shadow, not a device
// address; the device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) on the first call made on
// it, and reused.  That first call should therefore come before any stream
// capture.  The cached address belongs to the device's primary context: it
// does not survive cudaDeviceReset (or anything else that destroys that
// context), after which this entry point must not be called again in the
// process.  Every call shares the array and leaves its contents behind; the
// counts, offsets and bases are rewritten in full by each call before they
// are read, and the error word is cleared at the start of each call.  Calls
// whose work overlaps on the GPU (on different streams) race on the array.
//
// Every argument is checked on the host before anything is enqueued: the
// count pass reads x as float4 groups, so x must be 16-byte aligned (a tensor
// slice at an odd element offset is not); v, x_out and v_out must be 4-byte
// aligned; neither output may overlap the other output or an input.  The
// scatter's bounds check on the destination index can only fail if x changes
// between the count and the scatter pass (another writer racing on it); the
// call returns before the kernels run, so such a failure is not reported.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "pic_internal.cuh"

namespace {

constexpr size_t kScratchBytes = PIC_SORT_NOALLOC_SCRATCH;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device (looked up once).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p % a) == 0; }

// true when the byte ranges [a, a + bytes) and [b, b + bytes) share a byte
bool overlap(const void *a, const void *b, size_t bytes) {
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + bytes && pb < pa + bytes;
}

// Scratch bytes of a sort with nchunk chunks and nseg segments.
size_t scratch_need(int nchunk, int nseg, int ng) {
    return align256(256) + align256((size_t)nchunk * ng * 4) + align256((size_t)nseg * ng * 4) +
           align256((size_t)ng * 4);
}

void geometry(long long n, int nchunk_max, int *nchunk, long long *chunk, int *nseg,
              int *seg_len) {
    long long nc = (n + 2047) / 2048;
    if (nc < 1) nc = 1;
    if (nc > nchunk_max) nc = nchunk_max;
    long long ch = (n + nc - 1) / nc;
    ch = (ch + 3) & ~3ll;                   // chunks start on float4 groups
    nc = (n + ch - 1) / ch;
    int ns = 1;
    while ((long long)ns * ns < nc) ns++;
    *nchunk = (int)nc;
    *chunk = ch;
    *seg_len = (int)((nc + ns - 1) / ns);
    *nseg = (int)((nc + *seg_len - 1) / *seg_len);
}

}  // namespace

extern "C" int pic_sort_noalloc(const float *x, const float *v, float *x_out, float *v_out,
                                int64_t n, int32_t ncell, double length, void *stream) {
    pic::TraceRange trace_("pic_sort_noalloc");
    if (!x || !v || !x_out || !v_out) return PIC_EINVAL;
    if (n < 1 || n > (int64_t)0xFFFFFFFFll || ncell < 1 || ncell > PIC_NCELL_MAX) return PIC_EINVAL;
    if (!(length > 0.0) || !std::isfinite(length)) return PIC_EINVAL;
    if (!aligned(x, 16) || !aligned(v, 4) || !aligned(x_out, 4) || !aligned(v_out, 4))
        return PIC_EINVAL;
    const size_t bytes = (size_t)n * sizeof(float);
    if (overlap(x_out, v_out, bytes) || overlap(x_out, x, bytes) || overlap(x_out, v, bytes) ||
        overlap(v_out, x, bytes) || overlap(v_out, v, bytes))
        return PIC_EINVAL;
    // the most chunks whose tables fit the scratch array (at most 1024)
    int nchunk = 0, nseg = 0, seg_len = 0;
    long long chunk = 0;
    int cap = 1024;
    for (;;) {
        geometry(n, cap, &nchunk, &chunk, &nseg, &seg_len);
        if (scratch_need(nchunk, nseg, ncell) <= kScratchBytes) break;
        if (cap == 1) return PIC_ENOMEM;   // the tables of one chunk do not fit
        cap = cap / 2 > 0 ? cap / 2 : 1;
    }
    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return PIC_ECUDA;
    unsigned char *p = (unsigned char *)base;
    cudaStream_t s = (cudaStream_t)stream;
    pic::SortArgs<float> a;
    a.x = x;
    a.v = v;
    a.x_out = x_out;
    a.v_out = v_out;
    a.n = n;
    a.ng = ncell;
    a.inv_dx = (float)((double)ncell / length);
    a.nchunk = nchunk;
    a.chunk = chunk;
    a.nseg = nseg;
    a.seg_len = seg_len;
    a.err = (unsigned *)p;
    size_t off = align256(256);
    a.hist = (unsigned *)(p + off);
    off += align256((size_t)nchunk * ncell * 4);
    a.segtot = (unsigned *)(p + off);
    off += align256((size_t)nseg * ncell * 4);
    a.base = (unsigned *)(p + off);
    if (cudaMemsetAsync(a.err, 0, sizeof(unsigned), s) != cudaSuccess) return PIC_ECUDA;
    return pic::launch_sort_f32(a, s) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}
