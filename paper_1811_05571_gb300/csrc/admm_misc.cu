// Small device helpers of the setup path: complex128 -> complex64 packing into
// the padded layout, a finite-value check, and in-place scaling.
#include "admm_internal.h"

namespace admm {
namespace {

__global__ void pack_c128_kernel(const double2* __restrict__ src, int64_t m, int64_t n,
                                 float2* __restrict__ dst, int64_t ld) {
    const int64_t total = m * n;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = e / n, c = e - r * n;
        const double2 x = src[e];
        dst[r * ld + c] = make_float2(static_cast<float>(x.x), static_cast<float>(x.y));
    }
}

__global__ void finite_kernel(const float2* __restrict__ x, int64_t count, int* flag) {
    bool bad = false;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < count;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float2 v = x[e];
        if (!isfinite(v.x) || !isfinite(v.y)) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}

__global__ void scale_kernel(float2* x, int64_t count, float alpha) {
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < count;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float2 v = x[e];
        x[e] = make_float2(v.x * alpha, v.y * alpha);
    }
}

int grid_for(int64_t count) {
    int64_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    return static_cast<int>(blocks);
}

}  // namespace

cudaError_t launch_pack_c128(const double2* src, int64_t m, int64_t n, float2* dst, int64_t ld,
                             cudaStream_t s) {
    pack_c128_kernel<<<grid_for(m * n), 256, 0, s>>>(src, m, n, dst, ld);
    return cudaGetLastError();
}

cudaError_t launch_finite_check(const float2* x, int64_t count, int* flag, cudaStream_t s) {
    finite_kernel<<<grid_for(count), 256, 0, s>>>(x, count, flag);
    return cudaGetLastError();
}

cudaError_t launch_scale(float2* x, int64_t count, float alpha, cudaStream_t s) {
    scale_kernel<<<grid_for(count), 256, 0, s>>>(x, count, alpha);
    return cudaGetLastError();
}

}  // namespace admm
