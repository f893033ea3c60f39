// FP64 sums of squares with no device allocation, for callers that cannot
// call cudaMalloc.
//
// Who needs it: a caller whose device memory is all reserved up front (for
// example by a caching allocator such as PyTorch's, which holds freed memory
// for itself), or code on a latency-critical path where a cudaMalloc /
// cudaFree would stall it (cudaFree synchronises the device).  Such callers
// pass their own input and output buffers; the per-block partial sums live in
// the file-scope array below instead of an allocated scratch buffer.
//
// The array is g_partials: 2 x 16384 doubles (256 KiB), reserved on every
// GPU that loads this library until the process exits.  It bounds the input
// to 16384 blocks x 16384 elements = 2^28 elements.
#include <mutex>

#include "plan_impl.h"
#include "stencil.h"

namespace stencil {
namespace {

constexpr int NA_THREADS = 256;
constexpr int64_t NA_PER_BLOCK = (int64_t)NA_THREADS * 64;      // elements per block
constexpr int NA_MAX_BLOCKS = 16384;
constexpr int64_t NA_MAX_ELEMS = NA_PER_BLOCK * NA_MAX_BLOCKS;  // 2^28
constexpr int NA_MAX_DEVICES = 64;

// Per-block partials {sum (a-b)^2, sum b^2}.  Every block overwrites its own
// two slots before the final kernel reads them, so nothing has to be cleared
// between calls; calls that overlap on the GPU (other streams) race on it.
static __device__ __align__(256) double g_partials[2 * NA_MAX_BLOCKS];

std::mutex g_setup_mutex;
double *g_partials_addr[NA_MAX_DEVICES] = {};

__device__ __forceinline__ void na_block_sum2(double v0, double v1, double *dst)
{
    __shared__ double red[2][NA_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, o);
        v1 += __shfl_down_sync(0xffffffffu, v1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = v0;
        red[1][threadIdx.x >> 5] = v1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) {
            s0 += red[0][w];
            s1 += red[1][w];
        }
        dst[0] = s0;
        dst[1] = s1;
    }
}

// Block k sums dense elements [k * NA_PER_BLOCK, (k+1) * NA_PER_BLOCK); a is
// read through its row pitch, b is dense.
__global__ void __launch_bounds__(NA_THREADS)
    sqdiff_static_partials(const float *a, int64_t pitch, const double *b, int nx, int ny, int64_t n,
                           double *partials)
{
    const int64_t begin = (int64_t)blockIdx.x * NA_PER_BLOCK;
    const int64_t end = min(n, begin + NA_PER_BLOCK);
    double d2 = 0.0, r2 = 0.0;
    // (row, x) of this thread's first element by one division; each stride
    // of NA_THREADS elements then moves it by (dq rows, dr columns)
    const int64_t i0 = begin + threadIdx.x;
    int64_t row = i0 / nx;
    int x = (int)(i0 - row * nx);
    const int dq = NA_THREADS / nx, dr = NA_THREADS % nx;
    for (int64_t i = i0; i < end; i += NA_THREADS) {
        const double av = (double)a[row * pitch + x];
        const double bv = b[i];
        const double d = av - bv;
        d2 += d * d;
        r2 += bv * bv;
        x += dr;
        row += dq;
        if (x >= nx) {
            x -= nx;
            ++row;
        }
    }
    (void)ny;
    na_block_sum2(d2, r2, partials + 2 * blockIdx.x);
}

__global__ void __launch_bounds__(NA_THREADS)
    sqdiff_static_final(const double *partials, int nblocks, double *out)
{
    double d2 = 0.0, r2 = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += NA_THREADS) {
        d2 += partials[2 * k];
        r2 += partials[2 * k + 1];
    }
    na_block_sum2(d2, r2, out);
}

// Device address of g_partials on the current device, looked up once per
// device (host code cannot use the symbol itself as a device pointer).
int partials_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(STENCIL_ENODEV, "no CUDA device: %s", cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= NA_MAX_DEVICES) return fail(STENCIL_EUNSUPPORTED, "device index %d too large", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress(g_partials)");
        g_partials_addr[dev] = static_cast<double *>(p);
    }
    *out = g_partials_addr[dev];
    return STENCIL_OK;
}

}  // namespace
}  // namespace stencil

using namespace stencil;

extern "C" int stencil_sqdiff_noalloc(const float *a, int64_t a_pitch, const double *b, int32_t nx, int32_t ny,
                                      int32_t nz, double *out, void *stream)
{
    if (!a || !b || !out) return fail(STENCIL_EINVAL, "null argument");
    if (nx < 1 || ny < 1 || nz < 1) return fail(STENCIL_EINVAL, "dims must be >= 1");
    if (a_pitch < nx) return fail(STENCIL_EINVAL, "a_pitch must be >= nx");
    const int64_t n = (int64_t)nx * ny * nz;
    if (n > NA_MAX_ELEMS)
        return fail(STENCIL_EINVAL, "%lld elements exceed the static scratch capacity of %lld (2^28)",
                    (long long)n, (long long)NA_MAX_ELEMS);
    double *partials = nullptr;
    int rc = partials_address(&partials);
    if (rc) return rc;
    const int nblocks = (int)((n + NA_PER_BLOCK - 1) / NA_PER_BLOCK);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    sqdiff_static_partials<<<nblocks, NA_THREADS, 0, s>>>(a, a_pitch, b, nx, ny, n, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e, "sqdiff_static_partials launch");
    sqdiff_static_final<<<1, NA_THREADS, 0, s>>>(partials, nblocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e, "sqdiff_static_final launch");
    return STENCIL_OK;
}
