// Batched shared-H norm-1 ADMM: B scenes (measurement vectors) solved with
// one sensing matrix, every product over H and over the cached factors run as
// a GEMM on the 5th-generation tensor cores (tcgen05.mma, FP16 operands, FP32
// accumulation in tensor memory).
//
// Complex products as real GEMMs.  H is held in the FP16 storage format (one
// power-of-two scale per 64-row group), interleaved (re, im) along K, so a
// complex row of H is a real row of twice the length.  A complex operand x of
// the right-hand side is split into x_hi + x_lo (both FP16, after a
// power-of-two scale per scene and block) and laid out as four real columns
// per scene,
//     (re_hi, -im_hi), (im_hi, re_hi), (re_lo, -im_lo), (im_lo, re_lo)
// over the (re, im) pairs of K, so that the four FP32 accumulator columns of a
// scene hold Re and Im of H x_hi and of H x_lo; their sums times the scales
// give H x to about 2^-22 of the scene's largest entry.  The factor products
// K^{-1} r use the same layout with K^{-1} itself split into hi + lo halves
// along K (three of the four partial products).
#include <algorithm>

#include <cuda_fp16.h>

#include "admm_batch.h"
#include "ptx.cuh"

namespace admm {
namespace batch {
namespace {

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
    return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// power-of-two scale 2^(q-14) for a block whose largest |component| is mx = f 2^q
__device__ __forceinline__ float pow2_scale(float mx) {
    if (!(mx > 0.f)) return 1.0f;
    int q = 0;
    frexpf(mx, &q);
    return ldexpf(1.0f, q - 14);
}

__device__ __forceinline__ float block_max(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        float x = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
        if (threadIdx.x == 0) red[32] = x;
    }
    __syncthreads();
    return red[32];
}

// ---------------------------------------------------------------------------
// the GEMM: D (128 x 256 tile, FP32 in TMEM) = A (128 x K) * B (256 x K)^T,
// both K-major FP16 tiles staged by TMA with 128-byte swizzling
// ---------------------------------------------------------------------------

constexpr int kTileM = 128, kTileN = 256, kTileK = 64;   // K in FP16 elements (128 bytes)
constexpr int kStages = 4;
constexpr int kABytes = kTileM * kTileK * 2;
constexpr int kBBytes = kTileN * kTileK * 2;
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kTmemCols = 512;       // two 256-column accumulators
constexpr int kChunk = 4;            // K blocks (256 elements of K) accumulated in TMEM per chunk
constexpr int kEpiWarps = 4;

// instruction descriptor: D FP32 (bits 4-5 = 1), A and B FP16 (bits 7-9, 10-12
// = 0), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at 24-28
constexpr uint32_t kIdesc = (1u << 4) | (uint32_t(kTileN >> 3) << 17) | (uint32_t(kTileM >> 4) << 24);

__device__ bool wait_bounded(uint64_t* bar, uint32_t parity, int* fail, const GemmArgs& a) {
    if (*reinterpret_cast<volatile int*>(fail)) return false;
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer_ns() - t0 > a.timeout_ns) {
            raise_status(a.status, ADMM_ETIMEOUT);
            *reinterpret_cast<volatile int*>(fail) = 1;
            return false;
        }
    }
    return true;
}

// wait that ignores earlier failures (for completions that must be observed
// before shared or tensor memory is reused or released)
__device__ bool wait_always(uint64_t* bar, uint32_t parity, const GemmArgs& a) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_timer_ns() - t0 > a.timeout_ns) {
            raise_status(a.status, ADMM_ETIMEOUT);
            return false;
        }
    return true;
}

// The tensor cores' FP32 accumulation loses more than the FP16 operand split
// over long K, so each CTA accumulates chunks of kChunk K blocks in one of two
// TMEM accumulators and the epilogue warps add every chunk into FP32 registers
// (hi and lo columns of a scene combined first: two values per scene).
__global__ void __launch_bounds__(kGemmThreads, 1)
    bgemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ GemmArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = align1024(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    uint64_t* acc_full = empty + kStages;   // [2]: chunk accumulated (MMA -> epilogue)
    uint64_t* acc_free = acc_full + 2;      // [2]: chunk read (epilogue -> MMA)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_free + 2);
    int* fail = reinterpret_cast<int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x / a.mtiles, mt = blockIdx.x - p * a.mtiles;
    const int nt = blockIdx.y, split = blockIdx.z;
    const int kbp = a.kb_prob[p];
    const int kb0 = split * a.kb_per_split;
    const int nk = max(min(kbp, kb0 + a.kb_per_split) - kb0, 0);
    const int nchunks = (nk + kChunk - 1) / kChunk;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_free[s], kEpiWarps);
        }
        *fail = 0;
        fence_mbarrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: one A tile and one B tile per stage
        prefetch_tensormap(&tmA);
        prefetch_tensormap(&tmB);
        const int ax = a.a_x0[p], ay = a.a_y0[p] + mt * kTileM, az = a.a_z[p];
        int issued = 0;
        for (int kb = 0; kb < nk; ++kb) {
            const int slot = kb % kStages;
            if (!wait_bounded(&empty[slot], ((kb / kStages) & 1) ^ 1, fail, a)) break;
            unsigned char* st = smem + slot * kStageBytes;
            mbar_arrive_expect_tx(&full[slot], kStageBytes);
            tma_load_3d(st, &tmA, ax + (kb0 + kb) * kTileK, ay, az, &full[slot]);
            tma_load_3d(st + kABytes, &tmB, (kb0 + kb) * kTileK, nt * kTileN, p, &full[slot]);
            ++issued;
        }
        // copies still in flight land before the CTA can exit
        for (int kb = max(issued - kStages, 0); kb < issued; ++kb)
            wait_always(&full[kb % kStages], (kb / kStages) & 1, a);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: four K=16 steps per 64-wide stage (32 bytes each)
        int kb = 0;
        for (int c = 0; c < nchunks; ++c) {
            const int buf = c & 1;
            // the epilogue has read the accumulator's previous chunk
            if (!wait_bounded(&acc_free[buf], ((c >> 1) & 1) ^ 1, fail, a)) break;
            tc_fence_after();
            const uint32_t d = tmem + buf * kTileN;
            const int kb_end = min(nk, kb + kChunk);
            bool ok = true;
            for (int first = kb; kb < kb_end; ++kb) {
                const int slot = kb % kStages;
                if (!wait_bounded(&full[slot], (kb / kStages) & 1, fail, a)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const unsigned char* st = smem + slot * kStageBytes;
                const uint64_t ad = umma_desc_k128(st), bd = umma_desc_k128(st + kABytes);
#pragma unroll
                for (int k = 0; k < kTileK / 16; ++k)
                    umma_f16(d, ad + 2 * k, bd + 2 * k, kIdesc, (kb > first || k > 0) ? 1u : 0u);
                umma_commit(&empty[slot]);
            }
            umma_commit(&acc_full[buf]);   // also marks every earlier MMA complete
            if (!ok) break;
        }
    } else if (warp >= 2) {
        // epilogue: TMEM lane quarter (warp % 4); per chunk, 8 loads of 32 columns
        // (8 scenes each) added into two FP32 registers per scene
        const int q = warp & 3;
        const int row = mt * kTileM + q * 32 + lane;
        const bool row_ok = row < a.rows[p];
        float acc[2 * (kTileN / 4)];
#pragma unroll
        for (int e = 0; e < 2 * (kTileN / 4); ++e) acc[e] = 0.f;
        bool ok = true;
        for (int c = 0; c < nchunks && ok; ++c) {
            const int buf = c & 1;
            ok = wait_always(&acc_full[buf], (c >> 1) & 1, a) && !*reinterpret_cast<volatile int*>(fail);
            tc_fence_after();
            if (ok) {
#pragma unroll
                for (int cc = 0; cc < kTileN / 32; ++cc) {
                    uint32_t r[32];
                    tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + buf * kTileN + cc * 32, r);
                    tmem_ld_wait();
#pragma unroll
                    for (int s = 0; s < 8; ++s) {
                        acc[2 * (cc * 8 + s)] += __uint_as_float(r[4 * s]) + __uint_as_float(r[4 * s + 2]);
                        acc[2 * (cc * 8 + s) + 1] += __uint_as_float(r[4 * s + 1]) + __uint_as_float(r[4 * s + 3]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_free[buf]);
        }
        float rs = 1.0f;
        if (a.row_scale && row_ok) rs = a.row_scale[(a.rs_off[p] + row) >> a.rs_shift];
#pragma unroll
        for (int s = 0; s < kTileN / 4; ++s) {
            const int b = nt * (kTileN / 4) + s;
            if (!row_ok || b >= a.B) continue;
            const float sc = rs * a.col_scale[p * a.B + b];
            const float re = ok ? acc[2 * s] : 0.f, im = ok ? acc[2 * s + 1] : 0.f;
            a.out[((static_cast<size_t>(split) * a.nprob + p) * a.B + b) * a.out_pitch + row] =
                make_float2(re * sc, im * sc);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// operand packing and the elementwise steps of the iteration
// ---------------------------------------------------------------------------

// B operand of problem p, scene b: x - y (times the H row scales when given),
// divided by a power of two per (p, b), split into FP16 hi + lo, four packed
// rows; one CTA per (p, b)
__global__ void pack_kernel(PackArgs a) {
    __shared__ float red[33];
    const int p = blockIdx.x, b = blockIdx.y;
    const int L = a.len[p];
    const float2* x = a.x + a.x_off[p] + static_cast<long long>(b) * a.x_bs;
    const float2* y = a.y ? a.y + a.y_off[p] + static_cast<long long>(b) * a.y_bs : nullptr;
    const int r0 = a.rs ? a.rs_row[p] : 0;
    auto value = [&](int e) {
        float2 v = x[e];
        if (y) {
            const float2 w = y[e];
            v = make_float2(v.x - w.x, v.y - w.y);
        }
        if (a.rs) {
            const float h = a.rs[(r0 + e) >> 6];
            v = make_float2(v.x * h, v.y * h);
        }
        return v;
    };
    float mx = 0.f;
    for (int e = threadIdx.x; e < L; e += blockDim.x) {
        const float2 v = value(e);
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    mx = block_max(mx, red);
    const float sc = pow2_scale(mx), inv = 1.0f / sc;
    if (threadIdx.x == 0) a.scale[p * a.B + b] = sc;
    const size_t row = a.row2;
    __half2* base = static_cast<__half2*>(a.dst) + (static_cast<size_t>(p) * 4 * a.B + 4 * b) * row;
    for (int e = threadIdx.x; e < L; e += blockDim.x) {
        const float2 v = value(e);
        const float xr = v.x * inv, xi = v.y * inv;
        const __half hr = __float2half_rn(xr), hi = __float2half_rn(xi);
        const __half lr = __float2half_rn(xr - __half2float(hr));
        const __half li = __float2half_rn(xi - __half2float(hi));
        __half2 c0, c1, c2, c3;
        if (!a.adjoint) {
            // A holds (re, im) of H: Re = re*xr - im*xi, Im = re*xi + im*xr
            c0 = __halves2half2(hr, __hneg(hi));
            c1 = __halves2half2(hi, hr);
            c2 = __halves2half2(lr, __hneg(li));
            c3 = __halves2half2(li, lr);
        } else {
            // A holds (re, im) of H^T: conj(h) x = (re*xr + im*xi) + i (re*xi - im*xr)
            c0 = __halves2half2(hr, hi);
            c1 = __halves2half2(hi, __hneg(hr));
            c2 = __halves2half2(lr, li);
            c3 = __halves2half2(li, __hneg(lr));
        }
        base[e] = c0;
        base[row + e] = c1;
        base[2 * row + e] = c2;
        base[3 * row + e] = c3;
        if (a.second >= 0) {
            base[a.second + e] = c0;
            base[row + a.second + e] = c1;
        }
    }
}

// R_p = Gt_j - sum of the split-K partials of H_ij z_j^i (rows of block i)
__global__ void residual_r_kernel(StepArgs a) {
    const size_t total = static_cast<size_t>(a.P) * a.B * a.mpitch;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(e % a.mpitch);
        const size_t pb = e / a.mpitch;
        const int b = static_cast<int>(pb % a.B), p = static_cast<int>(pb / a.B);
        const int i = p / a.N, j = p - (p / a.N) * a.N;
        const int r0 = a.row_off[i], mi = a.row_off[i + 1] - r0;
        if (r >= mi) continue;
        float2 acc = make_float2(0.f, 0.f);
        for (int sp = 0; sp < a.splits; ++sp) {
            const float2 x = a.Ppart[(static_cast<size_t>(sp) * a.P * a.B + pb) * a.mpitch + r];
            acc.x += x.x;
            acc.y += x.y;
        }
        const float2 g = a.Gt[(static_cast<size_t>(j) * a.B + b) * a.m + r0 + r];
        a.R[e] = make_float2(g.x - acc.x, g.y - acc.y);
    }
}

// Ghat_ij = Gt_ij - rho W_ij (H_ij u_j^i of this iterate, the exchanged estimated data)
__global__ void ghat_kernel(StepArgs a) {
    const size_t total = static_cast<size_t>(a.P) * a.B * a.mpitch;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(e % a.mpitch);
        const size_t pb = e / a.mpitch;
        const int b = static_cast<int>(pb % a.B), p = static_cast<int>(pb / a.B);
        const int i = p / a.N, j = p - (p / a.N) * a.N;
        const int r0 = a.row_off[i], mi = a.row_off[i + 1] - r0;
        if (r >= mi) continue;
        const size_t gi = (static_cast<size_t>(j) * a.B + b) * a.m + r0 + r;
        const float2 g = a.Gt[gi], w = a.W[e];
        a.Ghat[gi] = make_float2(g.x - a.rho * w.x, g.y - a.rho * w.y);
    }
}

// out[b][e] = sum over splits and over the blocks meeting index e of part[sp][p][b][e - off[k]]:
// by rows (forward: e in row block k = i, p = i N + q) or by columns (adjoint: k = j, p = q N + j)
__global__ void sum_blocks_kernel(const float2* __restrict__ part, int splits, int P, int B, int pitch,
                                  const int* __restrict__ off, int nblk, int N, int by_rows,
                                  float2* __restrict__ out, int out_len) {
    const size_t total = static_cast<size_t>(B) * out_len;
    const int others = P / nblk;
    for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int b = static_cast<int>(t / out_len), e = static_cast<int>(t % out_len);
        int k = 0;
        while (off[k + 1] <= e) ++k;
        float2 acc = make_float2(0.f, 0.f);
        for (int o = 0; o < others; ++o) {
            const int p = by_rows ? k * N + o : o * N + k;
            for (int sp = 0; sp < splits; ++sp) {
                const float2 x = part[((static_cast<size_t>(sp) * P + p) * B + b) * pitch + e - off[k]];
                acc.x += x.x;
                acc.y += x.y;
            }
        }
        out[t] = acc;
    }
}

__device__ __forceinline__ float2 soft(float2 x, float kappa) {
    const float mag = hypotf(x.x, x.y);
    if (!(mag > kappa)) return make_float2(0.f, 0.f);
    const float f = 1.0f - kappa / mag;
    return make_float2(x.x * f, x.y * f);
}

// v_j = S_kappa(v_j + mean_i sigma_j^i), s_j^i <- v_old + sigma_j^i - v_new (the
// u-step u = z + sigma and s += u - v combined); per-scene residual terms
__global__ void update_kernel(StepArgs a) {
    const int b = blockIdx.y;
    const float kappa = a.kappa[b];
    double rp = 0.0, rd = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.n; c += gridDim.x * blockDim.x) {
        int j = 0;
        while (a.col_off[j + 1] <= c) ++j;
        const int cl = c - a.col_off[j];
        float2* vp = a.V + static_cast<size_t>(b) * a.n + c;
        const float2 vo = *vp;
        float2 mean = make_float2(0.f, 0.f);
        for (int i = 0; i < a.M; ++i) {
            const float2 sg = a.Sig[(static_cast<size_t>(i * a.N + j) * a.B + b) * a.npitch + cl];
            mean.x += sg.x;
            mean.y += sg.y;
        }
        const float2 vn = soft(make_float2(vo.x + mean.x * a.inv_M, vo.y + mean.y * a.inv_M), kappa);
        *vp = vn;
        for (int i = 0; i < a.M; ++i) {
            const float2 sg = a.Sig[(static_cast<size_t>(i * a.N + j) * a.B + b) * a.npitch + cl];
            float2* sp = a.S + (static_cast<size_t>(i) * a.B + b) * a.n + c;
            const float2 so = *sp;
            // u = v_old - s + sigma; s_new = s + u - v_new
            const float2 u = make_float2(vo.x - so.x + sg.x, vo.y - so.y + sg.y);
            *sp = make_float2(so.x + u.x - vn.x, so.y + u.y - vn.y);
            const float dx = u.x - vn.x, dy = u.y - vn.y;
            rp += static_cast<double>(dx) * dx + static_cast<double>(dy) * dy;
        }
        const float ex = vn.x - vo.x, ey = vn.y - vo.y;
        rd += static_cast<double>(ex) * ex + static_cast<double>(ey) * ey;
    }
    for (int o = 16; o > 0; o >>= 1) {
        rp += __shfl_xor_sync(0xffffffffu, rp, o);
        rd += __shfl_xor_sync(0xffffffffu, rd, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(a.res + 2 * b, rp);
        atomicAdd(a.res + 2 * b + 1, rd);
    }
}

// Gt_j = g - sum_{q != j} Ghat_q (previous iterate), for the column splits
__global__ void gtilde_kernel(StepArgs a) {
    const size_t total = static_cast<size_t>(a.B) * a.m;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float2 g = a.G[e];
        float2 sum = make_float2(0.f, 0.f);
        for (int q = 0; q < a.N; ++q) {
            const float2 x = a.Ghat[q * total + e];
            sum.x += x.x;
            sum.y += x.y;
        }
        for (int j = 0; j < a.N; ++j) {
            const float2 x = a.Ghat[j * total + e];
            a.Gt[j * total + e] = make_float2(g.x - (sum.x - x.x), g.y - (sum.y - x.y));
        }
    }
}

// H16 (m x ld, (re, im) FP16) -> H16T (ld x m): the adjoint GEMM's K-major A operand
__global__ void transpose_h16_kernel(const __half2* __restrict__ H16, int m, int ld, __half2* __restrict__ HT) {
    __shared__ __half2 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        tile[y][threadIdx.x] = (r < m && c < ld) ? H16[static_cast<size_t>(r) * ld + c] : __half2();
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (c < ld && r < m) HT[static_cast<size_t>(c) * m + r] = tile[threadIdx.x][y];
    }
}

// K^{-1} of block p (complex64, m_i x kp) -> Kpack[p][row][4 m_imax]: hi half over
// K [0, 2 m_imax), lo half over [2 m_imax, 4 m_imax), one power-of-two scale per row
__global__ void pack_kinv_kernel(const float2* __restrict__ kinv, const long long* __restrict__ koff,
                                 const int* __restrict__ kpitch, const int* __restrict__ row_off, int N,
                                 int mimax, int kk, __half2* __restrict__ Kpack, float* __restrict__ kscale) {
    __shared__ float red[33];
    const int p = blockIdx.x, r = blockIdx.y;
    const int i = p / N;
    const int mi = row_off[i + 1] - row_off[i];
    if (r >= mi) return;
    const float2* K = kinv + koff[p] + static_cast<size_t>(r) * kpitch[p];
    float mx = 0.f;
    for (int t = threadIdx.x; t < mi; t += blockDim.x) mx = fmaxf(mx, fmaxf(fabsf(K[t].x), fabsf(K[t].y)));
    mx = block_max(mx, red);
    const float sc = pow2_scale(mx), inv = 1.0f / sc;
    if (threadIdx.x == 0) kscale[p * mimax + r] = sc;
    __half2* dst = Kpack + (static_cast<size_t>(p) * mimax + r) * (kk / 2);
    for (int t = threadIdx.x; t < mi; t += blockDim.x) {
        const float xr = K[t].x * inv, xi = K[t].y * inv;
        const __half hr = __float2half_rn(xr), hi = __float2half_rn(xi);
        dst[t] = __halves2half2(hr, hi);
        dst[mimax + t] = __halves2half2(__float2half_rn(xr - __half2float(hr)),
                                        __float2half_rn(xi - __half2float(hi)));
    }
}

}  // namespace

cudaError_t prepare_gemm() {
    return cudaFuncSetAttribute(bgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
}

cudaError_t launch_gemm(const CUtensorMap& A, const CUtensorMap& B, const GemmArgs& a, cudaStream_t s) {
    dim3 grid(static_cast<unsigned>(a.nprob * a.mtiles), static_cast<unsigned>(a.ntiles),
              static_cast<unsigned>(a.splits));
    bgemm_kernel<<<grid, kGemmThreads, kGemmSmem, s>>>(A, B, a);
    return cudaGetLastError();
}

cudaError_t launch_pack(const PackArgs& a, int nprob, cudaStream_t s) {
    pack_kernel<<<dim3(nprob, a.B), 256, 0, s>>>(a);
    return cudaGetLastError();
}

static int grid_of(size_t total) {
    return static_cast<int>(std::max<size_t>(1, std::min<size_t>(8192, (total + 255) / 256)));
}

cudaError_t launch_residual_r(const StepArgs& a, cudaStream_t s) {
    residual_r_kernel<<<grid_of(static_cast<size_t>(a.P) * a.B * a.mpitch), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ghat(const StepArgs& a, cudaStream_t s) {
    ghat_kernel<<<grid_of(static_cast<size_t>(a.P) * a.B * a.mpitch), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sum_blocks(const float2* part, int splits, int P, int B, int pitch, const int* off, int nblk,
                              int N, int by_rows, float2* out, int out_len, cudaStream_t s) {
    sum_blocks_kernel<<<grid_of(static_cast<size_t>(B) * out_len), 256, 0, s>>>(part, splits, P, B, pitch, off,
                                                                                 nblk, N, by_rows, out, out_len);
    return cudaGetLastError();
}

cudaError_t launch_update(const StepArgs& a, cudaStream_t s) {
    const int gx = std::max(1, std::min(64, (a.n + 255) / 256));
    update_kernel<<<dim3(gx, a.B), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gtilde(const StepArgs& a, cudaStream_t s) {
    const size_t total = static_cast<size_t>(a.B) * a.m;
    const int blocks = static_cast<int>(std::min<size_t>(4096, (total + 255) / 256));
    gtilde_kernel<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_transpose_h16(const void* H16, int m, int ld, void* HT, cudaStream_t s) {
    dim3 grid((ld + 31) / 32, (m + 31) / 32);
    transpose_h16_kernel<<<grid, dim3(32, 8), 0, s>>>(static_cast<const __half2*>(H16), m, ld,
                                                     static_cast<__half2*>(HT));
    return cudaGetLastError();
}

cudaError_t launch_pack_kinv(const float2* kinv, const long long* koff, const int* kpitch, const int* row_off,
                             int P, int N, int mimax, int kk, void* Kpack, float* kscale, cudaStream_t s) {
    pack_kinv_kernel<<<dim3(P, mimax), 256, 0, s>>>(kinv, koff, kpitch, row_off, N, mimax, kk,
                                                    static_cast<__half2*>(Kpack), kscale);
    return cudaGetLastError();
}

}  // namespace batch
}  // namespace admm
