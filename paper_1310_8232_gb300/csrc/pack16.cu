// FP32 <-> FP16 / BF16 with one power-of-two scale per z plane: the state
// transfer of plans that store u^n and d^n = u^n - u^{n-1} in 16 bits.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace stencil {
namespace {

// Smallest power of two s >= 2^-126 with b / s <= 2^15 (1 for b == 0); the
// same rule the sweep uses for its output planes.
__device__ __forceinline__ float pack_scale(float b)
{
    if (!(b > 0.0f)) return 1.0f;
    if (!isfinite(b)) return ldexpf(1.0f, 127);
    int e;
    frexpf(b, &e);
    return ldexpf(1.0f, max(e - 15, -126));
}

// the value packed at q: src[q], or src[q] - sub[q] (the difference of two
// FP32 fields, rounded once to FP32)
__device__ __forceinline__ float packed_value(const float *src, const float *sub, int64_t q)
{
    return sub ? src[q] - sub[q] : src[q];
}

// one block per plane: max |v| over the plane's nx x ny points
__global__ void plane_amax_kernel(const float *src, const float *sub, int nx, int ny, int64_t pitch, float *scale,
                                  unsigned *amax)
{
    const int z = blockIdx.x;
    const int64_t base = (int64_t)z * pitch * ny;
    unsigned m = 0;
    for (int64_t i = threadIdx.x; i < (int64_t)nx * ny; i += blockDim.x) {
        const int64_t y = i / nx;
        const int x = (int)(i - y * nx);
        m = max(m, __float_as_uint(fabsf(packed_value(src, sub, base + y * pitch + x))));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    __shared__ unsigned wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned b = 0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) b = max(b, wm[w]);
        amax[z] = b;
        scale[z] = pack_scale(__uint_as_float(b));
    }
}

template <typename E>
__device__ __forceinline__ E to_e(float v);
template <>
__device__ __forceinline__ __half to_e<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_e<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ float from_e(__half v) { return __half2float(v); }
__device__ __forceinline__ float from_e(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename E>
__global__ void pack_kernel(const float *src, const float *sub, E *dst, int nx, int ny, int nz, int64_t pitch,
                            const float *scale)
{
    const int64_t rows = (int64_t)ny * nz;
    const int64_t total = rows * nx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / nx;
        const int x = (int)(i - row * nx);
        const int z = (int)(row / ny);
        const int64_t q = row * pitch + x;
        dst[q] = to_e<E>(packed_value(src, sub, q) / scale[z]);   // exact division by a power of two
    }
}

template <typename E>
__global__ void unpack_kernel(const E *src, float *dst, int nx, int ny, int nz, int64_t pitch, const float *scale)
{
    const int64_t rows = (int64_t)ny * nz;
    const int64_t total = rows * nx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / nx;
        const int x = (int)(i - row * nx);
        const int z = (int)(row / ny);
        const int64_t q = row * pitch + x;
        dst[q] = from_e(src[q]) * scale[z];
    }
}

// u^{n-1} = u^n - d^n from the two 16-bit fields and their scales
template <typename E>
__global__ void unpack_prev_kernel(const E *u, const E *d, float *dst, int nx, int ny, int nz, int64_t pitch,
                                   const float *scale_u, const float *scale_d)
{
    const int64_t rows = (int64_t)ny * nz;
    const int64_t total = rows * nx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / nx;
        const int x = (int)(i - row * nx);
        const int z = (int)(row / ny);
        const int64_t q = row * pitch + x;
        dst[q] = from_e(u[q]) * scale_u[z] - from_e(d[q]) * scale_d[z];
    }
}

}  // namespace

cudaError_t launch_pack16(int storage, const float *src, const float *sub, void *dst, int nx, int ny, int nz,
                          int64_t pitch, float *scale, unsigned *amax, cudaStream_t s)
{
    plane_amax_kernel<<<nz, 256, 0, s>>>(src, sub, nx, ny, pitch, scale, amax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (storage == 1)
        pack_kernel<__half><<<1216, 256, 0, s>>>(src, sub, static_cast<__half *>(dst), nx, ny, nz, pitch, scale);
    else if (storage == 2)
        pack_kernel<__nv_bfloat16>
            <<<1216, 256, 0, s>>>(src, sub, static_cast<__nv_bfloat16 *>(dst), nx, ny, nz, pitch, scale);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_unpack16_prev(int storage, const void *u, const void *d, float *dst, int nx, int ny, int nz,
                                 int64_t pitch, const float *scale_u, const float *scale_d, cudaStream_t s)
{
    if (storage == 1)
        unpack_prev_kernel<__half><<<1216, 256, 0, s>>>(static_cast<const __half *>(u), static_cast<const __half *>(d),
                                                        dst, nx, ny, nz, pitch, scale_u, scale_d);
    else if (storage == 2)
        unpack_prev_kernel<__nv_bfloat16><<<1216, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(u),
                                                               static_cast<const __nv_bfloat16 *>(d), dst, nx, ny,
                                                               nz, pitch, scale_u, scale_d);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_unpack16(int storage, const void *src, float *dst, int nx, int ny, int nz, int64_t pitch,
                            const float *scale, cudaStream_t s)
{
    if (storage == 1)
        unpack_kernel<__half>
            <<<1216, 256, 0, s>>>(static_cast<const __half *>(src), dst, nx, ny, nz, pitch, scale);
    else if (storage == 2)
        unpack_kernel<__nv_bfloat16>
            <<<1216, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(src), dst, nx, ny, nz, pitch, scale);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace stencil
