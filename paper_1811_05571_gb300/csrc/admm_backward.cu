// Products of the single-scene reverse sweep (admm_backward): H sigma_bar by
// rows, K^{-1} w_bar, and H^H r_bar by columns, for every block, over the
// complex64 H or its FP16 copy (the matrix the recorded forward streamed).
// The elementwise steps of the sweep are the batched path's with one scene.
#include <cuda_fp16.h>

#include "admm_internal.h"

namespace admm {
namespace {

constexpr int kRowWarps = 8;

template <bool F16>
__device__ __forceinline__ float2 h_at(const ProdArgs& a, int r, int c) {
    if (F16) {
        const float2 v = __half22float2(static_cast<const __half2*>(a.H16)[static_cast<size_t>(r) * a.ld + c]);
        return v;   // times the group scale of row r, applied by the caller
    }
    return a.H[static_cast<size_t>(r) * a.ld + c];
}

// one warp per (block, row): out[p][r] = sum_c H[r0 + r][c0 + c] x[p][c]
template <bool F16>
__global__ void rows_kernel(ProdArgs a, const float2* __restrict__ x, float2* __restrict__ out) {
    const int p = blockIdx.x;
    const int i = p / a.N, j = p - (p / a.N) * a.N;
    const int r0 = a.row_off[i], mi = a.row_off[i + 1] - r0;
    const int c0 = a.col_off[j], nj = a.col_off[j + 1] - c0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.y * kRowWarps + warp;
    if (r >= mi) return;
    const float2* xp = x + static_cast<size_t>(p) * a.npitch;
    float2 acc = make_float2(0.f, 0.f);
    for (int c = lane; c < nj; c += 32) {
        const float2 h = h_at<F16>(a, r0 + r, c0 + c), z = xp[c];
        acc.x = fmaf(h.x, z.x, fmaf(-h.y, z.y, acc.x));
        acc.y = fmaf(h.x, z.y, fmaf(h.y, z.x, acc.y));
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) {
        const float sc = F16 ? a.scales[(r0 + r) >> 6] : 1.0f;
        out[static_cast<size_t>(p) * a.mpitch + r] = make_float2(acc.x * sc, acc.y * sc);
    }
}

// one thread per (block, column): out[p][c] = sum_r conj(H[r0 + r][c0 + c]) s_r y[p][r]
template <bool F16>
__global__ void cols_kernel(ProdArgs a, const float2* __restrict__ y, float2* __restrict__ out) {
    extern __shared__ float2 ys[];
    const int p = blockIdx.x;
    const int i = p / a.N, j = p - (p / a.N) * a.N;
    const int r0 = a.row_off[i], mi = a.row_off[i + 1] - r0;
    const int c0 = a.col_off[j], nj = a.col_off[j + 1] - c0;
    for (int r = threadIdx.x; r < mi; r += blockDim.x) {
        float2 v = y[static_cast<size_t>(p) * a.mpitch + r];
        if (F16) {
            const float sc = a.scales[(r0 + r) >> 6];
            v = make_float2(v.x * sc, v.y * sc);
        }
        ys[r] = v;
    }
    __syncthreads();
    const int c = blockIdx.y * blockDim.x + threadIdx.x;
    if (c >= nj) return;
    float2 acc = make_float2(0.f, 0.f);
    for (int r = 0; r < mi; ++r) {
        const float2 h = h_at<F16>(a, r0 + r, c0 + c), w = ys[r];
        acc.x = fmaf(h.x, w.x, fmaf(h.y, w.y, acc.x));
        acc.y = fmaf(h.x, w.y, fmaf(-h.y, w.x, acc.y));
    }
    out[static_cast<size_t>(p) * a.npitch + c] = acc;
}

// one warp per (block, row): out[p][r] = sum_t Kinv_p[r][t] y[p][t]
__global__ void factor_kernel(ProdArgs a, const float2* __restrict__ y, float2* __restrict__ out) {
    const int p = blockIdx.x;
    const int i = p / a.N;
    const int mi = a.row_off[i + 1] - a.row_off[i];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.y * kRowWarps + warp;
    if (r >= mi) return;
    const float2* K = a.kinv + a.kinv_off[p] + static_cast<size_t>(r) * a.kinv_pitch[p];
    const float2* yp = y + static_cast<size_t>(p) * a.mpitch;
    float2 acc = make_float2(0.f, 0.f);
    for (int t = lane; t < mi; t += 32) {
        const float2 k = K[t], v = yp[t];
        acc.x = fmaf(k.x, v.x, fmaf(-k.y, v.y, acc.x));
        acc.y = fmaf(k.x, v.y, fmaf(k.y, v.x, acc.y));
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) out[static_cast<size_t>(p) * a.mpitch + r] = acc;
}

}  // namespace

cudaError_t launch_bw_rows(const ProdArgs& a, bool f16, const float2* x, float2* out, cudaStream_t s) {
    const dim3 grid(a.M * a.N, (a.mimax + kRowWarps - 1) / kRowWarps);
    if (f16) rows_kernel<true><<<grid, 32 * kRowWarps, 0, s>>>(a, x, out);
    else rows_kernel<false><<<grid, 32 * kRowWarps, 0, s>>>(a, x, out);
    return cudaGetLastError();
}

cudaError_t launch_bw_cols(const ProdArgs& a, bool f16, const float2* y, float2* out, cudaStream_t s) {
    const dim3 grid(a.M * a.N, (a.njmax + 255) / 256);
    const size_t smem = static_cast<size_t>(a.mimax) * sizeof(float2);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f16 ? reinterpret_cast<const void*>(cols_kernel<true>)
                                                 : reinterpret_cast<const void*>(cols_kernel<false>),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    if (f16) cols_kernel<true><<<grid, 256, smem, s>>>(a, y, out);
    else cols_kernel<false><<<grid, 256, smem, s>>>(a, y, out);
    return cudaGetLastError();
}

cudaError_t launch_bw_factor(const ProdArgs& a, const float2* y, float2* out, cudaStream_t s) {
    const dim3 grid(a.M * a.N, (a.mimax + kRowWarps - 1) / kRowWarps);
    factor_kernel<<<grid, 32 * kRowWarps, 0, s>>>(a, y, out);
    return cudaGetLastError();
}

}  // namespace admm
