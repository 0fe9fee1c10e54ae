// Direct branch of the block update for blocks with at least as many rows as
// columns (Section III-B: when N_m > N_p / N the original inversion is the
// cheaper one).  Block b = (i, j) keeps the n_j x n_j factor
//     L_b = (H_b^H H_b + rho I)^{-1}
// and one iteration is
//     q_b    = H_b^H gt_b + rho (v_j - s_j^i)          column pass over H_b
//     u_b    = L_b q_b                                 factor pass
//     a_j    = mean_i (u_j^i + s_j^i), v_j = S_kappa(a_j), s_j^i += u_j^i - v_j
//     ghat_b = H_b u_b                                 row pass (N > 1)
// (Eq. x_solution_columns and g_columns; for one column block gt_b = g_i, so
// H_i^H g_i is computed once per data vector and the iteration never reads H).
//
// Kernels hand results to each other through global memory only.  Inside a
// kernel the step that needs every CTA's result (the sum of the column-pass
// partials, the consensus update of a column chunk, the residual record) is
// done by whichever CTA increments the step's counter last; that CTA also
// resets the counter.  No CTA waits for another.
#include "admm_internal.h"
#include "ptx.cuh"

namespace admm {
namespace {

__device__ __forceinline__ float2 ldcg2(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ void stcg2(float2* p, float2 v) { __stcg(p, v); }
__device__ __forceinline__ float sq2(float2 a) { return a.x * a.x + a.y * a.y; }

// complex soft-threshold of Eq. (softhresholding)
__device__ __forceinline__ float2 shrink(float2 a, float kappa) {
    const float mag = hypotf(a.x, a.y);
    if (mag > kappa) {
        const float sc = 1.0f - kappa / mag;
        return make_float2(a.x * sc, a.y * sc);
    }
    return make_float2(0.0f, 0.0f);
}

__device__ __forceinline__ bool stopped(const DirectArgs& a) {
    return a.check_stop && ld_volatile(a.stop_flag) != 0;
}

// ---- column pass: partial[s][b][c] = sum over the rows of split s of
// conj(H_b[r][c]) gt_b[r]; the last of the S splits of a column tile adds them
__global__ void __launch_bounds__(kDirThreads) dir_cols_kernel(const DirectArgs a, int mode) {
    extern __shared__ float2 gts[];
    __shared__ int last;
    if (mode == 0 && stopped(a)) return;
    const int sidx = blockIdx.x % a.S;
    const int tile = blockIdx.x / a.S;
    const int cc = tile % a.ccn, p = tile / a.ccn;
    const int i = p / a.N, j = p - i * a.N;
    const int r0 = a.row_off[i], mi = a.row_off[i + 1] - r0;
    const int c0 = a.col_off[j], nj = a.col_off[j + 1] - c0;
    const int rb = static_cast<int>(static_cast<long long>(mi) * sidx / a.S);
    const int nr = static_cast<int>(static_cast<long long>(mi) * (sidx + 1) / a.S) - rb;
    const size_t Nm = static_cast<size_t>(a.N) * a.m;
    const float2* gh = a.ghat + static_cast<size_t>(__ldcg(a.k_done) & 1) * Nm;
    // gt_b = g_i - sum_{q != j} ghat_iq over the split's rows
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        const int row = r0 + rb + r;
        float2 x = a.g[row];
        if (mode == 0)
            for (int q = 0; q < a.N; ++q)
                if (q != j) {
                    const float2 e = ldcg2(gh + static_cast<size_t>(q) * a.m + row);
                    x.x -= e.x;
                    x.y -= e.y;
                }
        gts[r] = x;
    }
    __syncthreads();
    const int c = cc * kDirColTile + threadIdx.x;
    float2 acc = make_float2(0.f, 0.f);
    if (c < nj) {
        const float2* hp = a.H + static_cast<size_t>(r0 + rb) * a.ld + c0 + c;
        int r = 0;
        for (; r + 8 <= nr; r += 8) {
            float2 h[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) h[q] = __ldg(hp + static_cast<size_t>(r + q) * a.ld);
#pragma unroll
            for (int q = 0; q < 8; ++q) cfma_conj(acc, h[q], gts[r + q]);
        }
        for (; r < nr; ++r) cfma_conj(acc, __ldg(hp + static_cast<size_t>(r) * a.ld), gts[r]);
        stcg2(a.part + (static_cast<size_t>(sidx) * a.P + p) * a.npitch + c, acc);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(a.cnt_cols + tile, 1u) == static_cast<unsigned>(a.S - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (c < nj) {
        float2 sum = make_float2(0.f, 0.f);
        const float2* pp = a.part + static_cast<size_t>(p) * a.npitch + c;
        const size_t step = static_cast<size_t>(a.P) * a.npitch;
        int q = 0;
        for (; q + 4 <= a.S; q += 4) {
            float2 x[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) x[t] = ldcg2(pp + (q + t) * step);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                sum.x += x[t].x;
                sum.y += x[t].y;
            }
        }
        for (; q < a.S; ++q) {
            const float2 x = ldcg2(pp + q * step);
            sum.x += x.x;
            sum.y += x.y;
        }
        if (mode == 0) {
            const float2 vv = ldcg2(a.v + c0 + c), ss = ldcg2(a.s + static_cast<size_t>(i) * a.ld + c0 + c);
            sum.x += a.rho * (vv.x - ss.x);
            sum.y += a.rho * (vv.y - ss.y);
            stcg2(a.Q + static_cast<size_t>(p) * a.npitch + c, sum);
        } else {
            stcg2(a.C + static_cast<size_t>(p) * a.npitch + c, sum);
        }
    }
    if (threadIdx.x == 0) a.cnt_cols[tile] = 0u;
}

// ---- one column block: q_i = C_i + rho (v - s_i) ---------------------------
__global__ void __launch_bounds__(kDirThreads) dir_q_kernel(const DirectArgs a) {
    if (stopped(a)) return;
    const long long total = static_cast<long long>(a.M) * a.n;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e / a.n), c = static_cast<int>(e - static_cast<long long>(i) * a.n);
        const float2 cv = a.C[static_cast<size_t>(i) * a.npitch + c];
        const float2 vv = ldcg2(a.v + c), ss = ldcg2(a.s + static_cast<size_t>(i) * a.ld + c);
        stcg2(a.Q + static_cast<size_t>(i) * a.npitch + c,
              make_float2(cv.x + a.rho * (vv.x - ss.x), cv.y + a.rho * (vv.y - ss.y)));
    }
}

// ---- factor pass + update ----------------------------------------------------
// CTA (b, chunk): u_b[row0 .. row0 + 32) = L_b[rows] q_b, four rows per warp.
// The last of the M CTAs holding chunk `chunk` of column block j updates v_j,
// s_j^i over those 32 columns and writes the chunk's residual partials; the
// last chunk of all writes the iteration's residual record.
__global__ void __launch_bounds__(kDirThreads) dir_factor_kernel(const DirectArgs a) {
    extern __shared__ float4 qs4[];
    __shared__ int last;
    if (stopped(a)) return;
    const int chunk_in = blockIdx.x % a.fcn, p = blockIdx.x / a.fcn;
    const int i = p / a.N, j = p - i * a.N;
    const int c0 = a.col_off[j], nj = a.col_off[j + 1] - c0;
    const int row0 = chunk_in * kDirChunk;
    if (row0 >= nj) return;   // whole CTA: this chunk does not exist for the block
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int npairs = (nj + 1) >> 1;
    const float4* q4 = reinterpret_cast<const float4*>(a.Q + static_cast<size_t>(p) * a.npitch);
    for (int e = tid; e < npairs; e += blockDim.x) qs4[e] = __ldcg(q4 + e);
    __syncthreads();
    {
        const float2* Lp = a.L + a.L_off[p];
        const int pitch = a.L_pitch[p];
        const int rbase = row0 + warp * 4;
        const float4* lr[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int rq = min(rbase + q, nj - 1);   // clamped rows are computed and dropped
            lr[q] = reinterpret_cast<const float4*>(Lp + static_cast<size_t>(rq) * pitch);
        }
        float2 acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
        int e = lane;
        for (; e + 32 < npairs; e += 64) {
            const float4 x0 = qs4[e], x1 = qs4[e + 32];
            float4 l0[4], l1[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                l0[q] = __ldg(lr[q] + e);
                l1[q] = __ldg(lr[q] + e + 32);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                cfma(acc[q], make_float2(l0[q].x, l0[q].y), make_float2(x0.x, x0.y));
                cfma(acc[q], make_float2(l0[q].z, l0[q].w), make_float2(x0.z, x0.w));
                cfma(acc[q], make_float2(l1[q].x, l1[q].y), make_float2(x1.x, x1.y));
                cfma(acc[q], make_float2(l1[q].z, l1[q].w), make_float2(x1.z, x1.w));
            }
        }
        for (; e < npairs; e += 32) {
            const float4 x0 = qs4[e];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 l = __ldg(lr[q] + e);
                cfma(acc[q], make_float2(l.x, l.y), make_float2(x0.x, x0.y));
                cfma(acc[q], make_float2(l.z, l.w), make_float2(x0.z, x0.w));
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = warp_sum(acc[q]);
        if (lane == 0) {
            float2* up = a.u + static_cast<size_t>(i) * a.ld + c0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (rbase + q < nj) stcg2(up + rbase + q, acc[q]);
        }
    }
    __threadfence();
    __syncthreads();
    const int chunk = a.chunk_off[j] + chunk_in;
    if (tid == 0) last = atomicAdd(a.cnt_upd + chunk, 1u) == static_cast<unsigned>(a.M - 1);
    __syncthreads();
    if (!last || warp != 0) return;
    __threadfence();
    // consensus update of columns c0 + row0 + lane
    float d[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const int cl = row0 + lane;
    if (cl < nj) {
        const int col = c0 + cl;
        const float2 vv = ldcg2(a.v + col);
        float2 sum = make_float2(0.f, 0.f);
        for (int r = 0; r < a.M; ++r) {
            const float2 uu = ldcg2(a.u + static_cast<size_t>(r) * a.ld + col);
            const float2 ss = ldcg2(a.s + static_cast<size_t>(r) * a.ld + col);
            sum.x += uu.x + ss.x;
            sum.y += uu.y + ss.y;
        }
        const float2 av = make_float2(sum.x * a.inv_M, sum.y * a.inv_M);
        const float2 vn = shrink(av, a.kappa);
        d[1] = sq2(make_float2(vn.x - vv.x, vn.y - vv.y));
        d[3] = sq2(vn);
        for (int r = 0; r < a.M; ++r) {
            float2* sp = a.s + static_cast<size_t>(r) * a.ld + col;
            const float2 uu = ldcg2(a.u + static_cast<size_t>(r) * a.ld + col);
            const float2 ss = ldcg2(sp);
            const float2 sn = make_float2(ss.x + uu.x - vn.x, ss.y + uu.y - vn.y);
            d[0] += sq2(make_float2(uu.x - vn.x, uu.y - vn.y));
            d[2] += sq2(uu);
            d[4] += sq2(sn);
            stcg2(sp, sn);
        }
        stcg2(a.v + col, vn);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q)
        for (int o = 16; o > 0; o >>= 1) d[q] += __shfl_xor_sync(0xffffffffu, d[q], o);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) __stcg(a.res_chunk + static_cast<size_t>(chunk) * 5 + q, static_cast<double>(d[q]));
        a.cnt_upd[chunk] = 0u;
        __threadfence();
        last = atomicAdd(a.cnt_glob, 1u) == static_cast<unsigned>(a.nchunks - 1);
    }
    __syncwarp();
    if (!__shfl_sync(0xffffffffu, last, 0)) return;
    __threadfence();
    // residual record of the iteration (the same five norms as the persistent kernel)
    double acc[5] = {0, 0, 0, 0, 0};
    for (int c = lane; c < a.nchunks; c += 32) {
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[q] += __ldcg(a.res_chunk + static_cast<size_t>(c) * 5 + q);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = warp_sum_d(acc[q]);
    if (lane == 0) {
        a.cnt_glob[0] = 0u;
        const long long k = __ldcg(a.k_done);
        const double Md = static_cast<double>(a.M);
        double rec[5];
        rec[0] = acc[0];
        rec[1] = a.rho_d * a.rho_d * Md * acc[1];
        rec[2] = acc[2];
        rec[3] = Md * acc[3];
        rec[4] = acc[4];
        double* dst = a.hist + static_cast<size_t>(k % a.hist_cap) * 5;
#pragma unroll
        for (int q = 0; q < 5; ++q) dst[q] = rec[q];
        const bool bad = !isfinite(rec[0] + rec[1] + rec[2] + rec[3] + rec[4]);
        if (bad) raise_status(a.status, ADMM_EDIVERGED);
        if (a.check_stop && !bad) {
            const double pp = static_cast<double>(a.M) * static_cast<double>(a.n);
            const double eps_pri = sqrt(pp) * a.eps_abs + a.eps_rel * fmax(sqrt(rec[2]), sqrt(rec[3]));
            const double eps_dual = sqrt(pp) * a.eps_abs + a.eps_rel * a.rho_d * sqrt(rec[4]);
            if (sqrt(rec[0]) <= eps_pri && sqrt(rec[1]) <= eps_dual) {
                // the row pass of this iteration still runs (it completes the
                // estimated data of the final state); it raises stop_flag
                if (a.N == 1) *reinterpret_cast<volatile int*>(a.stop_flag) = 1;
                else *reinterpret_cast<volatile int*>(a.stop_pending) = 1;
            }
        }
        __threadfence();
        *reinterpret_cast<volatile long long*>(a.k_done) = k + 1;
    }
}

// ---- row pass: ghat_b = H_b u_b, eight rows per warp --------------------------
__global__ void __launch_bounds__(kDirThreads) dir_rows_kernel(const DirectArgs a) {
    extern __shared__ float2 us[];
    __shared__ int last;
    if (stopped(a)) return;
    const int bt = blockIdx.x % a.rtn, p = blockIdx.x / a.rtn;
    const int i = p / a.N, j = p - i * a.N;
    const int r0 = a.row_off[i], mi = a.row_off[i + 1] - r0;
    const int c0 = a.col_off[j], nj = a.col_off[j + 1] - c0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rt0 = bt * kDirRowTile;
    if (rt0 < mi) {
        const float2* up = a.u + static_cast<size_t>(i) * a.ld + c0;
        for (int c = tid; c < nj; c += blockDim.x) us[c] = ldcg2(up + c);
        __syncthreads();
        // after this iteration's update the device count is k + 1: its slot
        const size_t Nm = static_cast<size_t>(a.N) * a.m;
        float2* out = a.ghat + static_cast<size_t>(__ldcg(a.k_done) & 1) * Nm + static_cast<size_t>(j) * a.m + r0;
        const int rw = rt0 + warp * 8;
        if (rw < mi) {
            const float2* hr[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                hr[q] = a.H + static_cast<size_t>(r0 + min(rw + q, mi - 1)) * a.ld + c0;
            float2 acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
            for (int c = lane; c < nj; c += 32) {
                const float2 x = us[c];
                float2 h[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) h[q] = __ldg(hr[q] + c);
#pragma unroll
                for (int q = 0; q < 8; ++q) cfma(acc[q], h[q], x);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = warp_sum(acc[q]);
            if (lane < 8) {
                float2 mine = acc[0];
#pragma unroll
                for (int q = 1; q < 8; ++q)
                    if (lane == q) mine = acc[q];
                if (rw + lane < mi) stcg2(out + rw + lane, mine);
            }
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        last = atomicAdd(a.cnt_glob + 1, 1u) == gridDim.x - 1;
        if (last) {
            a.cnt_glob[1] = 0u;
            __threadfence();
            if (ld_volatile(a.stop_pending)) {
                *reinterpret_cast<volatile int*>(a.stop_pending) = 0;
                *reinterpret_cast<volatile int*>(a.stop_flag) = 1;
            }
        }
    }
}

// ---- HT = H^H, 32 x 32 tiles through shared memory ---------------------------
__global__ void conj_transpose_kernel(const float2* __restrict__ H, int64_t m, int64_t n, int64_t ld,
                                      float2* __restrict__ HT, int64_t ldT) {
    __shared__ float2 t[32][33];
    const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 32, c0 = static_cast<int64_t>(blockIdx.x) * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int k = ty; k < 32; k += 8) {
        const int64_t r = r0 + k, c = c0 + tx;
        t[k][tx] = (r < m && c < n) ? H[r * ld + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int64_t c = c0 + k, r = r0 + tx;
        if (c < n && r < m) {
            const float2 x = t[tx][k];
            HT[c * ldT + r] = make_float2(x.x, -x.y);
        }
    }
}

}  // namespace

cudaError_t prepare_direct(int smem_optin) {
    const int lim = std::min(smem_optin, kDirMaxCols * 8);
    cudaError_t e = cudaFuncSetAttribute(dir_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(dir_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    return e;
}

cudaError_t launch_dir_cols(const DirectArgs& a, int mode, cudaStream_t s) {
    const int rows = (a.mimax + a.S - 1) / a.S + 1;
    const size_t smem = static_cast<size_t>(rows) * sizeof(float2);
    dir_cols_kernel<<<a.P * a.ccn * a.S, kDirThreads, smem, s>>>(a, mode);
    return cudaGetLastError();
}

cudaError_t launch_dir_q(const DirectArgs& a, cudaStream_t s) {
    const long long total = static_cast<long long>(a.M) * a.n;
    const int blocks = static_cast<int>(std::min<long long>((total + kDirThreads - 1) / kDirThreads, 4096));
    dir_q_kernel<<<blocks, kDirThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dir_factor(const DirectArgs& a, cudaStream_t s) {
    const size_t smem = static_cast<size_t>((a.njmax + 1) / 2) * sizeof(float4);
    dir_factor_kernel<<<a.P * a.fcn, kDirThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dir_rows(const DirectArgs& a, cudaStream_t s) {
    const size_t smem = static_cast<size_t>(a.njmax) * sizeof(float2);
    dir_rows_kernel<<<a.P * a.rtn, kDirThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_conj_transpose(const float2* H, int64_t m, int64_t n, int64_t ld, float2* HT, int64_t ldT,
                                  cudaStream_t s) {
    const dim3 grid(static_cast<unsigned>((n + 31) / 32), static_cast<unsigned>((m + 31) / 32));
    conj_transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(H, m, n, ld, HT, ldT);
    return cudaGetLastError();
}

}  // namespace admm
