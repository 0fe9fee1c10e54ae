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

// One output tile: problem p, row tile mt, column tile nt, K split `split`
struct Tile {
    int p, mt, nt, split, kb0, nk;
};

__device__ __forceinline__ Tile tile_of(const GemmArgs& a, int t) {
    Tile x;
    x.nt = t % a.ntiles;
    int r = t / a.ntiles;
    x.mt = r % a.mtiles;
    r /= a.mtiles;
    x.p = r % a.nprob;
    x.split = r / a.nprob;
    x.kb0 = x.split * a.kb_per_split;
    x.nk = max(min(a.kb_prob[x.p], x.kb0 + a.kb_per_split) - x.kb0, 0);
    return x;
}

// Persistent GEMM: each CTA walks tiles t = blockIdx.x, + gridDim.x, ... (tiles
// that share an A tile are adjacent).  The tensor cores' FP32 accumulation
// loses more than the FP16 operand split over long K, so each tile is
// accumulated in chunks of kChunk K blocks in one of two TMEM accumulators and
// the epilogue warps add every chunk into FP32 registers (hi and lo columns of
// a scene combined first: two values per scene).  Stage and chunk counters run
// on across tiles, so the epilogue of one tile overlaps the MMAs of the next.
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
    const int ntile = a.nprob * a.mtiles * a.ntiles * a.splits;

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
        int g = 0;   // stages issued
        bool ok = true;
        for (int t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
            const Tile x = tile_of(a, t);
            const int ax = a.a_x0[x.p], ay = a.a_y0[x.p] + x.mt * kTileM, az = a.a_z[x.p];
            for (int kb = 0; kb < x.nk; ++kb, ++g) {
                const int slot = g % kStages;
                if (!wait_bounded(&empty[slot], ((g / kStages) & 1) ^ 1, fail, a)) {
                    ok = false;
                    break;
                }
                unsigned char* st = smem + slot * kStageBytes;
                mbar_arrive_expect_tx(&full[slot], kStageBytes);
                tma_load_3d(st, &tmA, ax + (x.kb0 + kb) * kTileK, ay, az, &full[slot]);
                tma_load_3d(st + kABytes, &tmB, (x.kb0 + kb) * kTileK, x.nt * kTileN, x.p, &full[slot]);
            }
        }
        // copies still in flight land before the CTA can exit
        for (int q = max(g - kStages, 0); q < g; ++q) wait_always(&full[q % kStages], (q / kStages) & 1, a);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: four K=16 steps per 64-wide stage (32 bytes each)
        int g = 0, gc = 0;   // stages consumed, chunks started
        bool ok = true;
        for (int t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
            const Tile x = tile_of(a, t);
            for (int kb = 0; kb < x.nk && ok; ++gc) {
                const int buf = gc & 1;
                // the epilogue has read this accumulator's previous chunk
                if (!wait_bounded(&acc_free[buf], ((gc >> 1) & 1) ^ 1, fail, a)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + buf * kTileN;
                const int kb_end = min(x.nk, kb + kChunk);
                for (const int first = kb; kb < kb_end; ++kb, ++g) {
                    const int slot = g % kStages;
                    if (!wait_bounded(&full[slot], (g / kStages) & 1, fail, a)) {
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
            }
        }
        // every MMA issued has completed before TMEM can be released, also when
        // the epilogue stopped early after a failure
        if (gc > 0) wait_always(&acc_full[(gc - 1) & 1], ((gc - 1) >> 1) & 1, a);
    } else if (warp >= 2) {
        // epilogue: TMEM lane quarter (warp % 4); per chunk, 8 loads of 32 columns
        // (8 scenes each) added into two FP32 registers per scene
        const int q = warp & 3;
        int gc = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
            const Tile x = tile_of(a, t);
            const int nchunks = (x.nk + kChunk - 1) / kChunk;
            float acc[2 * (kTileN / 4)];
#pragma unroll
            for (int e = 0; e < 2 * (kTileN / 4); ++e) acc[e] = 0.f;
            for (int c = 0; c < nchunks && ok; ++c, ++gc) {
                const int buf = gc & 1;
                ok = wait_always(&acc_full[buf], (gc >> 1) & 1, a) && !*reinterpret_cast<volatile int*>(fail);
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
                            acc[2 * (cc * 8 + s) + 1] +=
                                __uint_as_float(r[4 * s + 1]) + __uint_as_float(r[4 * s + 3]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_free[buf]);
            }
            if (!ok) break;
            const int row = x.mt * kTileM + q * 32 + lane;
            const bool row_ok = row < a.rows[x.p];
            float rs = 1.0f;
            if (a.row_scale && row_ok) rs = a.row_scale[(a.rs_off[x.p] + row) >> a.rs_shift];
#pragma unroll
            for (int s = 0; s < kTileN / 4; ++s) {
                const int b = x.nt * (kTileN / 4) + s;
                if (!row_ok || b >= a.B) continue;
                const float sc = rs * a.col_scale[x.p * a.B + b];
                a.out[((static_cast<size_t>(x.split) * a.nprob + x.p) * a.B + b) * a.out_pitch + row] =
                    make_float2(acc[2 * s] * sc, acc[2 * s + 1] * sc);
            }
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
    if (a.vmax) {
        mx = __uint_as_float(a.vmax[p * a.B + b]);
    } else {
        for (int e = threadIdx.x; e < L; e += blockDim.x) {
            const float2 v = value(e);
            mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
        mx = block_max(mx, red);
    }
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
        if (a.rec_w) {
            const int k = *a.rec_k;
            if (k < a.rec_cap) a.rec_w[static_cast<size_t>(k) * total + e] = w;
        }
    }
}

// next recording slot (one thread, last in the iteration)
__global__ void rec_advance_kernel(int* k) { *k += 1; }

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
// u-step u = z + sigma and s += u - v combined); per-scene residual terms, and
// the largest |component| of the next z_j^i = v_new - s_new^i per (block, scene),
// so that the next packing of z takes one pass
constexpr int kUpdRegs = 16;     // replicas whose sigma and z maximum stay in registers
constexpr int kUpdThreads = 256;

// one CTA per (tile of kUpdCols columns inside one column block, scene); the
// first MR replicas are kept in registers (loops unrolled to MR, guarded by M)
template <int MR>
__global__ void __launch_bounds__(kUpdThreads, MR <= 2 ? 4 : (MR <= 4 ? 3 : 2)) update_kernel(StepArgs a) {
    __shared__ float zred[MR][kUpdThreads / 32];
    const int b = blockIdx.y;
    int j = 0;
    while (a.upd_tile_off[j + 1] <= static_cast<int>(blockIdx.x)) ++j;
    const int c_beg = a.col_off[j] + (blockIdx.x - a.upd_tile_off[j]) * kUpdCols;
    const int c_end = min(a.col_off[j + 1], c_beg + kUpdCols);
    const int cb = c_beg - a.col_off[j];
    const float kappa = a.kappa[b];
    float rp = 0.f, rd = 0.f;   // a few terms per thread; FP64 from the warp sums on
    float zm[MR];
#pragma unroll
    for (int i = 0; i < MR; ++i) zm[i] = 0.f;
    for (int c = c_beg + threadIdx.x; c < c_end; c += kUpdThreads) {
        const int cl = cb + (c - c_beg);
        float2* vp = a.V + static_cast<size_t>(b) * a.n + c;
        const float2 vo = *vp;
        const float2* sgp = a.Sig + (static_cast<size_t>(j) * a.B + b) * a.npitch + cl;
        const size_t sg_i = static_cast<size_t>(a.N) * a.B * a.npitch;   // next replica
        float2 sg[MR];
        float2 mean = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < MR; ++i) {
            sg[i] = i < a.M ? sgp[i * sg_i] : make_float2(0.f, 0.f);
            mean.x += sg[i].x;
            mean.y += sg[i].y;
        }
        for (int i = MR; i < a.M; ++i) {
            const float2 x = sgp[i * sg_i];
            mean.x += x.x;
            mean.y += x.y;
        }
        const float2 av = make_float2(vo.x + mean.x * a.inv_M, vo.y + mean.y * a.inv_M);
        const float2 vn = soft(av, kappa);
        *vp = vn;
        if (a.rec_a) {
            const int k = *a.rec_k;
            if (k < a.rec_cap) a.rec_a[(static_cast<size_t>(k) * a.B + b) * a.n + c] = av;
        }
        float2* spb = a.S + static_cast<size_t>(b) * a.n + c;
        const size_t s_i = static_cast<size_t>(a.B) * a.n;
        auto step = [&](float2 x, float2 so, float2* sp) {
            // u = v_old - s + sigma; s_new = s + u - v_new
            const float2 u = make_float2(vo.x - so.x + x.x, vo.y - so.y + x.y);
            const float2 sn = make_float2(so.x + u.x - vn.x, so.y + u.y - vn.y);
            *sp = sn;
            const float dx = u.x - vn.x, dy = u.y - vn.y;
            rp = fmaf(dx, dx, fmaf(dy, dy, rp));
            // largest component of the next z = v_new - s_new
            return fmaxf(fabsf(vn.x - sn.x), fabsf(vn.y - sn.y));
        };
        // all duals of the register replicas loaded before any is stored
        float2 so[MR];
#pragma unroll
        for (int i = 0; i < MR; ++i) so[i] = i < a.M ? spb[i * s_i] : make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < MR; ++i)
            if (i < a.M) zm[i] = fmaxf(zm[i], step(sg[i], so[i], spb + i * s_i));
        for (int i = MR; i < a.M; ++i)
            atomicMax(a.zmax + (i * a.N + j) * a.B + b,
                      __float_as_uint(step(sgp[i * sg_i], spb[i * s_i], spb + i * s_i)));
        const float ex = vn.x - vo.x, ey = vn.y - vo.y;
        rd = fmaf(ex, ex, fmaf(ey, ey, rd));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mreg = min(a.M, MR);
#pragma unroll
    for (int i = 0; i < MR; ++i) {
        float x = zm[i];
        for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
        if (lane == 0) zred[i][warp] = x;
    }
    double dp = rp, dd = rd;
    for (int o = 16; o > 0; o >>= 1) {
        dp += __shfl_xor_sync(0xffffffffu, dp, o);
        dd += __shfl_xor_sync(0xffffffffu, dd, o);
    }
    if (lane == 0) {
        atomicAdd(a.res + 2 * b, dp);
        atomicAdd(a.res + 2 * b + 1, dd);
    }
    __syncthreads();
    if (threadIdx.x < mreg) {
        float x = 0.f;
        for (int w = 0; w < kUpdThreads / 32; ++w) x = fmaxf(x, zred[threadIdx.x][w]);
        atomicMax(a.zmax + (threadIdx.x * a.N + j) * a.B + b, __float_as_uint(x));
    }
}

// ---------------------------------------------------------------------------
// reverse sweep of one recorded iteration (the adjoint of the iteration above;
// complex adjoints x_bar = dL/dRe x + i dL/dIm x)
// ---------------------------------------------------------------------------

__device__ __forceinline__ double block_sum_d(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    return t;
}

// t = v_bar - sum_i s_bar_i (all that reaches v' = S(a)); a_bar = S'(a)^T t;
// kappa_bar -= Re(conj(a_hat) t); sigma_bar_ij = s_bar_j^i + a_bar_j / M (into Sig);
// v_bar <- sum_i s_bar_i + a_bar (the z_bar terms are added after the adjoint product)
__global__ void bw_soft_kernel(StepArgs a) {
    __shared__ double red[8];
    const int b = blockIdx.y;
    int j = 0;
    while (a.upd_tile_off[j + 1] <= static_cast<int>(blockIdx.x)) ++j;
    const int c_beg = a.col_off[j] + (blockIdx.x - a.upd_tile_off[j]) * kUpdCols;
    const int c_end = min(a.col_off[j + 1], c_beg + kUpdCols);
    const float kappa = a.kappa[b];
    const float2* ak = a.rec_a + static_cast<size_t>(a.bk) * a.B * a.n;
    float kb = 0.f;
    for (int c = c_beg + threadIdx.x; c < c_end; c += blockDim.x) {
        const int cl = c - a.col_off[j];
        const size_t vi = static_cast<size_t>(b) * a.n + c;
        float2 ssum = make_float2(0.f, 0.f);
        for (int i = 0; i < a.M; ++i) {
            const float2 x = a.Sb[static_cast<size_t>(i) * a.B * a.n + vi];
            ssum.x += x.x;
            ssum.y += x.y;
        }
        const float2 vb = a.Vb[vi];
        const float2 t = make_float2(vb.x - ssum.x, vb.y - ssum.y);
        const float2 av = ak[vi];
        const float mag = hypotf(av.x, av.y);
        float2 abar = make_float2(0.f, 0.f);
        if (mag > kappa) {
            const float hx = av.x / mag, hy = av.y / mag;
            const float proj = hx * t.x + hy * t.y;   // Re(conj(a_hat) t)
            const float f = kappa / mag;
            abar = make_float2(t.x - f * (t.x - hx * proj), t.y - f * (t.y - hy * proj));
            kb -= proj;
        }
        a.Vb[vi] = make_float2(ssum.x + abar.x, ssum.y + abar.y);
        for (int i = 0; i < a.M; ++i) {
            const float2 x = a.Sb[static_cast<size_t>(i) * a.B * a.n + vi];
            float2* sg = const_cast<float2*>(a.Sig) + (static_cast<size_t>(i * a.N + j) * a.B + b) * a.npitch + cl;
            *sg = make_float2(x.x + abar.x * a.inv_M, x.y + abar.y * a.inv_M);
        }
    }
    const double tot = block_sum_d(kb, red);
    if (threadIdx.x == 0) atomicAdd(a.kbar + b, tot);
}

// w_bar = H sigma_bar (split partials) - rho ghat_bar (into R); rho_bar -= Re(w^H ghat_bar)
__global__ void bw_wbar_kernel(StepArgs a) {
    __shared__ double red[8];
    const int b = blockIdx.y, p = blockIdx.x;
    const int i = p / a.N, j = p - (p / a.N) * a.N;
    const int r0 = a.row_off[i], mi = a.row_off[i + 1] - r0;
    const size_t pb = static_cast<size_t>(p) * a.B + b;
    const float2* wk = a.rec_w + (static_cast<size_t>(a.bk) * a.P * a.B + pb) * a.mpitch;
    double acc = 0.0;
    for (int r = threadIdx.x; r < mi; r += blockDim.x) {
        float2 hs = make_float2(0.f, 0.f);
        for (int sp = 0; sp < a.splits; ++sp) {
            const float2 x = a.Ppart[(static_cast<size_t>(sp) * a.P * a.B + pb) * a.mpitch + r];
            hs.x += x.x;
            hs.y += x.y;
        }
        const float2 gb = a.Ghb[(static_cast<size_t>(j) * a.B + b) * a.m + r0 + r];
        a.R[pb * a.mpitch + r] = make_float2(hs.x - a.rho * gb.x, hs.y - a.rho * gb.y);
        const float2 w = wk[r];
        acc -= static_cast<double>(w.x) * gb.x + static_cast<double>(w.y) * gb.y;
    }
    const double tot = block_sum_d(acc, red);
    if (threadIdx.x == 0) atomicAdd(a.rbar + b, tot);
}

// r_bar = K^{-1} w_bar (in W); rho_bar -= Re(w^H r_bar); gt_bar = ghat_bar + r_bar (into Gt)
__global__ void bw_rbar_kernel(StepArgs a) {
    __shared__ double red[8];
    const int b = blockIdx.y, p = blockIdx.x;
    const int i = p / a.N, j = p - (p / a.N) * a.N;
    const int r0 = a.row_off[i], mi = a.row_off[i + 1] - r0;
    const size_t pb = static_cast<size_t>(p) * a.B + b;
    const float2* wk = a.rec_w + (static_cast<size_t>(a.bk) * a.P * a.B + pb) * a.mpitch;
    double acc = 0.0;
    for (int r = threadIdx.x; r < mi; r += blockDim.x) {
        const float2 rb = a.W[pb * a.mpitch + r];
        const float2 w = wk[r];
        acc -= static_cast<double>(w.x) * rb.x + static_cast<double>(w.y) * rb.y;
        const size_t gi = (static_cast<size_t>(j) * a.B + b) * a.m + r0 + r;
        const float2 gb = a.Ghb[gi];
        a.Gt[gi] = make_float2(gb.x + rb.x, gb.y + rb.y);
    }
    const double tot = block_sum_d(acc, red);
    if (threadIdx.x == 0) atomicAdd(a.rbar + b, tot);
}

// z_bar_ij = -H_ij^H r_bar_ij (Sig holds H^H r_bar): v_bar += sum_i z_bar, s_bar_i = -z_bar
__global__ void bw_state_kernel(StepArgs a) {
    const int b = blockIdx.y;
    int j = 0;
    while (a.upd_tile_off[j + 1] <= static_cast<int>(blockIdx.x)) ++j;
    const int c_beg = a.col_off[j] + (blockIdx.x - a.upd_tile_off[j]) * kUpdCols;
    const int c_end = min(a.col_off[j + 1], c_beg + kUpdCols);
    for (int c = c_beg + threadIdx.x; c < c_end; c += blockDim.x) {
        const int cl = c - a.col_off[j];
        const size_t vi = static_cast<size_t>(b) * a.n + c;
        float2 vb = a.Vb[vi];
        for (int i = 0; i < a.M; ++i) {
            const float2 x = a.Sig[(static_cast<size_t>(i * a.N + j) * a.B + b) * a.npitch + cl];
            vb.x -= x.x;
            vb.y -= x.y;
            a.Sb[static_cast<size_t>(i) * a.B * a.n + vi] = x;
        }
        a.Vb[vi] = vb;
    }
}

// gt_ij = g_i - sum_{q != j} ghat_iq: g_bar_i += sum_j gt_bar_ij, ghat_bar_iq = -sum_{j != q} gt_bar_ij
__global__ void bw_gtilde_kernel(StepArgs a) {
    const size_t total = static_cast<size_t>(a.B) * a.m;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        float2 tot = make_float2(0.f, 0.f);
        for (int j = 0; j < a.N; ++j) {
            const float2 x = a.Gt[j * total + e];
            tot.x += x.x;
            tot.y += x.y;
        }
        float2 g = a.dG[e];
        a.dG[e] = make_float2(g.x + tot.x, g.y + tot.y);
        for (int q = 0; q < a.N; ++q) {
            const float2 x = a.Gt[q * total + e];
            a.Ghb[q * total + e] = make_float2(x.x - tot.x, x.y - tot.y);
        }
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

static int grid_of(size_t total) {
    return static_cast<int>(std::max<size_t>(1, std::min<size_t>(8192, (total + 255) / 256)));
}

cudaError_t prepare_gemm() {
    return cudaFuncSetAttribute(bgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
}

cudaError_t launch_gemm(const CUtensorMap& A, const CUtensorMap& B, const GemmArgs& a, cudaStream_t s) {
    const int tiles = a.nprob * a.mtiles * a.ntiles * a.splits;
    const int grid = std::max(1, std::min(tiles, a.ctas));
    bgemm_kernel<<<grid, kGemmThreads, kGemmSmem, s>>>(A, B, a);
    return cudaGetLastError();
}

cudaError_t launch_pack(const PackArgs& a, int nprob, cudaStream_t s) {
    pack_kernel<<<dim3(nprob, a.B), 256, 0, s>>>(a);
    return cudaGetLastError();
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
    const dim3 grid(a.upd_tiles, a.B);
    if (a.M <= 1) update_kernel<1><<<grid, kUpdThreads, 0, s>>>(a);
    else if (a.M <= 2) update_kernel<2><<<grid, kUpdThreads, 0, s>>>(a);
    else if (a.M <= 4) update_kernel<4><<<grid, kUpdThreads, 0, s>>>(a);
    else if (a.M <= 8) update_kernel<8><<<grid, kUpdThreads, 0, s>>>(a);
    else update_kernel<kUpdRegs><<<grid, kUpdThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rec_advance(const StepArgs& a, cudaStream_t s) {
    rec_advance_kernel<<<1, 1, 0, s>>>(a.rec_k);
    return cudaGetLastError();
}

cudaError_t launch_bw_soft(const StepArgs& a, cudaStream_t s) {
    bw_soft_kernel<<<dim3(a.upd_tiles, a.B), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bw_wbar(const StepArgs& a, cudaStream_t s) {
    bw_wbar_kernel<<<dim3(a.P, a.B), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bw_rbar(const StepArgs& a, cudaStream_t s) {
    bw_rbar_kernel<<<dim3(a.P, a.B), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bw_state(const StepArgs& a, cudaStream_t s) {
    bw_state_kernel<<<dim3(a.upd_tiles, a.B), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bw_gtilde(const StepArgs& a, cudaStream_t s) {
    const size_t total = static_cast<size_t>(a.B) * a.m;
    bw_gtilde_kernel<<<grid_of(total), 256, 0, s>>>(a);
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
