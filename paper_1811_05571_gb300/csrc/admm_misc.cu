// Small device helpers of the setup path: complex128 -> complex64 packing into
// the padded layout, a finite-value check, and in-place scaling.
#include <algorithm>

#include <cuda_fp16.h>

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

// max(|Re|, |Im|) of each 64-row group of H (as float bits: non-negative floats order like ints)
__global__ void group_absmax_kernel(const float2* __restrict__ H, int64_t m, int64_t ld,
                                    unsigned* __restrict__ gmax_bits) {
    const int64_t groups = (m + 63) / 64;
    for (int64_t g = blockIdx.y; g < groups; g += gridDim.y) {
        const int64_t r0 = g * 64, r1 = min(m, r0 + 64);
        float mx = 0.f;
        for (int64_t r = r0; r < r1; ++r)
            for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < ld;
                 c += static_cast<int64_t>(gridDim.x) * blockDim.x) {
                const float2 v = H[r * ld + c];
                mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
            }
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) atomicMax(gmax_bits + g, __float_as_uint(mx));
    }
}

// scale of a group: 2^(q - 14) where max = f 2^q, f in [0.5, 1) (so |H / scale| <= 2^14);
// H16 = H / scale rounded to FP16; optionally the dequantised H16 * scale in FP32
__global__ void quantize_kernel(const float2* __restrict__ H, int64_t m, int64_t ld,
                                const unsigned* __restrict__ gmax_bits, __half2* __restrict__ H16,
                                float* __restrict__ scales, float2* __restrict__ Hdeq) {
    const int64_t total = m * ld;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = e / ld;
        const float mx = __uint_as_float(gmax_bits[r >> 6]);
        int q = 0;
        frexpf(mx, &q);
        const float scale = mx > 0.f ? ldexpf(1.0f, q - 14) : 1.0f;
        if (e % ld == 0 && (r & 63) == 0) scales[r >> 6] = scale;
        const float2 v = H[e];
        const __half2 hv = __floats2half2_rn(v.x / scale, v.y / scale);
        H16[e] = hv;
        if (Hdeq) {
            const float2 f = __half22float2(hv);
            Hdeq[e] = make_float2(f.x * scale, f.y * scale);
        }
    }
}

// FP32 copy of the dequantised FP16 matrix (to rebuild its factors)
__global__ void dequantize_kernel(const __half2* __restrict__ H16, int64_t m, int64_t ld,
                                  const float* __restrict__ scales, float2* __restrict__ Hdeq) {
    const int64_t total = m * ld;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float scale = scales[(e / ld) >> 6];
        const float2 f = __half22float2(H16[e]);
        Hdeq[e] = make_float2(f.x * scale, f.y * scale);
    }
}

// ---- sharded iteration (Section IV: the blocks of one problem on several ranks)

__global__ void shard_ghat_sum_kernel(const float2* __restrict__ ghat, int N, int64_t m, float2* __restrict__ out) {
    for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < m;
         r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float2 t = make_float2(0.f, 0.f);
        for (int q = 0; q < N; ++q) {
            const float2 x = ghat[q * m + r];
            t.x += x.x;
            t.y += x.y;
        }
        out[r] = t;
    }
}

__global__ void shard_geff_kernel(const float2* __restrict__ g0, const float2* __restrict__ tg,
                                  const float2* __restrict__ tl, int64_t m, float2* __restrict__ g) {
    for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < m;
         r += static_cast<int64_t>(gridDim.x) * blockDim.x)
        g[r] = make_float2(g0[r].x - tg[r].x + tl[r].x, g0[r].y - tg[r].y + tl[r].y);
}

// v = S_kappa(sum / M_total) (Eq. softhresholding, the complex sign a/|a|),
// s_i += u_i - v for the local replicas, and the residual partials in FP64
__global__ void shard_vstep_kernel(float2* __restrict__ v, float2* __restrict__ s, const float2* __restrict__ u,
                                   const float2* __restrict__ sum, int64_t n, int64_t ld, int M, float inv_Mtot,
                                   float kappa, double* __restrict__ rec) {
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < n;
         c += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float2 a = make_float2(sum[c].x * inv_Mtot, sum[c].y * inv_Mtot);
        const float mag = hypotf(a.x, a.y);
        float2 vn = make_float2(0.f, 0.f);
        if (mag > kappa) {
            const float sc = 1.0f - kappa / mag;
            vn = make_float2(a.x * sc, a.y * sc);
        }
        const float2 vo = v[c];
        v[c] = vn;
        acc[1] += static_cast<double>((vn.x - vo.x) * (vn.x - vo.x) + (vn.y - vo.y) * (vn.y - vo.y));
        acc[3] += static_cast<double>(vn.x * vn.x + vn.y * vn.y);
        for (int i = 0; i < M; ++i) {
            const float2 uu = u[i * ld + c];
            float2 ss = s[i * ld + c];
            ss = make_float2((ss.x + uu.x) - vn.x, (ss.y + uu.y) - vn.y);
            s[i * ld + c] = ss;
            acc[0] += static_cast<double>((uu.x - vn.x) * (uu.x - vn.x) + (uu.y - vn.y) * (uu.y - vn.y));
            acc[2] += static_cast<double>(uu.x * uu.x + uu.y * uu.y);
            acc[4] += static_cast<double>(ss.x * ss.x + ss.y * ss.y);
        }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double x = acc[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(rec + q, x);
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

cudaError_t launch_quantize_f16(const float2* H, int64_t m, int64_t ld, unsigned* gmax_bits,
                                void* H16, float* scales, float2* Hdeq, cudaStream_t s) {
    const int64_t groups = (m + 63) / 64;
    cudaError_t e = cudaMemsetAsync(gmax_bits, 0, groups * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const int chunks = static_cast<int>(std::min<int64_t>(64, (ld + 255) / 256));
    const unsigned gy = static_cast<unsigned>(std::min<int64_t>(groups, 65535));
    group_absmax_kernel<<<dim3(chunks, gy), 256, 0, s>>>(H, m, ld, gmax_bits);
    quantize_kernel<<<grid_for(m * ld), 256, 0, s>>>(H, m, ld, gmax_bits, static_cast<__half2*>(H16),
                                                    scales, Hdeq);
    return cudaGetLastError();
}

cudaError_t launch_dequantize_f16(const void* H16, int64_t m, int64_t ld, const float* scales,
                                  float2* Hdeq, cudaStream_t s) {
    dequantize_kernel<<<grid_for(m * ld), 256, 0, s>>>(static_cast<const __half2*>(H16), m, ld, scales, Hdeq);
    return cudaGetLastError();
}

cudaError_t launch_shard_ghat_sum(const float2* ghat, int N, int64_t m, float2* out, cudaStream_t s) {
    shard_ghat_sum_kernel<<<grid_for(m), 256, 0, s>>>(ghat, N, m, out);
    return cudaGetLastError();
}

cudaError_t launch_shard_geff(const float2* g0, const float2* t_glob, const float2* t_loc, int64_t m, float2* g,
                              cudaStream_t s) {
    shard_geff_kernel<<<grid_for(m), 256, 0, s>>>(g0, t_glob, t_loc, m, g);
    return cudaGetLastError();
}

cudaError_t launch_shard_vstep(float2* v, float2* s, const float2* u, const float2* sum, int64_t n, int64_t ld, int M,
                               float inv_Mtot, float kappa, double* rec, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(rec, 0, 5 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    shard_vstep_kernel<<<std::min(grid_for(n), 1024), 256, 0, st>>>(v, s, u, sum, n, ld, M, inv_Mtot, kappa, rec);
    return cudaGetLastError();
}

cudaError_t launch_scale(float2* x, int64_t count, float alpha, cudaStream_t s) {
    scale_kernel<<<grid_for(count), 256, 0, s>>>(x, count, alpha);
    return cudaGetLastError();
}

}  // namespace admm
