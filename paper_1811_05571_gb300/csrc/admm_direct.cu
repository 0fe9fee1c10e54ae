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
// resets the counter.  No CTA waits for another; the only waits are those
// between the producer lane and the consumer warps of one CTA of the streamed
// factor pass and of the tile pass (mbarriers, each bounded by the handle's
// timeout).
#include "admm_internal.h"
#include "ptx.cuh"

namespace admm {
namespace {

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

// Sum over the 32 lanes of x[0..7], leaving the sum of x[q] in lanes whose
// bits 4..2 spell q (lane >> 2 == q): three exchange steps halve the values a
// lane carries, two plain steps finish; 18 shuffles for eight complex values.
__device__ __forceinline__ float2 lanes_sum8(const float2 (&x)[8], int lane) {
    float2 y4[4];
    const bool b16 = lane & 16;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 keep = b16 ? x[q + 4] : x[q], send = b16 ? x[q] : x[q + 4];
        y4[q] = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, send.x, 16),
                            keep.y + __shfl_xor_sync(0xffffffffu, send.y, 16));
    }
    float2 y2[2];
    const bool b8 = lane & 8;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float2 keep = b8 ? y4[q + 2] : y4[q], send = b8 ? y4[q] : y4[q + 2];
        y2[q] = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, send.x, 8),
                            keep.y + __shfl_xor_sync(0xffffffffu, send.y, 8));
    }
    const bool b4 = lane & 4;
    const float2 keep = b4 ? y2[1] : y2[0], send = b4 ? y2[0] : y2[1];
    float2 y = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, send.x, 4),
                           keep.y + __shfl_xor_sync(0xffffffffu, send.y, 4));
    y.x += __shfl_xor_sync(0xffffffffu, y.x, 2);
    y.y += __shfl_xor_sync(0xffffffffu, y.y, 2);
    y.x += __shfl_xor_sync(0xffffffffu, y.x, 1);
    y.y += __shfl_xor_sync(0xffffffffu, y.y, 1);
    // lane bits: 16 -> q bit 2, 8 -> q bit 1, 4 -> q bit 0
    return y;
}

__device__ __forceinline__ bool stopped(const DirectArgs& a) {
    return a.check_stop && ld_volatile(a.stop_flag) != 0;
}

// ---- column pass: partial[s][b][c] = sum over the rows of split s of
// conj(H_b[r][c]) gt_b[r]; the last of the S splits of a column tile adds them.
// A tile is kDirColPairs column pairs from the block's first column rounded
// down to even (16-byte loads; columns outside the block are dropped).  Lane
// l of every warp owns pairs l, l + 32, l + 64, l + 96 of the tile; warp w
// takes rows w, w + 8, ... of the split, four at a time (16 loads in flight
// per lane), and the eight warps' sums meet in shared memory.
__global__ void __launch_bounds__(kDirColThreads, 2) dir_cols_kernel(const DirectArgs a, int mode) {
    extern __shared__ float2 dsm[];
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
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float2* gts = dsm;                                  // rows of the split
    float2* red = dsm + ((a.mimax + a.S - 1) / a.S + 1); // 8 warps x 2 kDirColPairs
    const size_t Nm = static_cast<size_t>(a.N) * a.m;
    const float2* gh = a.ghat + static_cast<size_t>(__ldcg(a.k_done) & 1) * Nm;
    // gt_b = g_i - sum_{q != j} ghat_iq over the split's rows
    for (int r = tid; r < nr; r += blockDim.x) {
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
    const int cb = (c0 & ~1) + cc * 2 * kDirColPairs;  // first column of the tile (even)
    const int cend = c0 + nj;
    float2 acc[4][2];
#pragma unroll
    for (int t = 0; t < 4; ++t) acc[t][0] = acc[t][1] = make_float2(0.f, 0.f);
    // pairs that hold a column of the block; the others load nothing
    bool live[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) live[t] = cb + 2 * (lane + 32 * t) < cend;
    const size_t step = static_cast<size_t>(a.ld) / 2;   // float4 per row
    const float4* hp = reinterpret_cast<const float4*>(a.H + static_cast<size_t>(r0 + rb) * a.ld + cb) + lane;
    int r = warp;
    for (; r + 24 < nr; r += 32) {
        float4 h[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int t = 0; t < 4; ++t)
                h[q][t] = live[t] ? __ldg(hp + (r + 8 * q) * step + 32 * t) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 x = gts[r + 8 * q];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                cfma_conj(acc[t][0], make_float2(h[q][t].x, h[q][t].y), x);
                cfma_conj(acc[t][1], make_float2(h[q][t].z, h[q][t].w), x);
            }
        }
    }
    for (; r < nr; r += 8) {
        const float2 x = gts[r];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float4 h = live[t] ? __ldg(hp + r * step + 32 * t) : make_float4(0.f, 0.f, 0.f, 0.f);
            cfma_conj(acc[t][0], make_float2(h.x, h.y), x);
            cfma_conj(acc[t][1], make_float2(h.z, h.w), x);
        }
    }
    // cross-warp sum: column c = 2 * pair + half of the tile
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int pr = lane + 32 * t;
        red[warp * 2 * kDirColPairs + 2 * pr] = acc[t][0];
        red[warp * 2 * kDirColPairs + 2 * pr + 1] = acc[t][1];
    }
    __syncthreads();
    float2* pp = a.part + (static_cast<size_t>(sidx) * a.P + p) * a.npitch;
    for (int c = tid; c < 2 * kDirColPairs; c += blockDim.x) {
        const int e = cb + c - c0;
        if (e < 0 || e >= nj) continue;
        float2 sum = red[c];
#pragma unroll
        for (int w = 1; w < kDirColThreads / 32; ++w) {
            const float2 x = red[w * 2 * kDirColPairs + c];
            sum.x += x.x;
            sum.y += x.y;
        }
        stcg2(pp + e, sum);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(a.cnt_cols + tile, 1u) == static_cast<unsigned>(a.S - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    const size_t sstep = static_cast<size_t>(a.P) * a.npitch;
    for (int c = tid; c < 2 * kDirColPairs; c += blockDim.x) {
        const int e = cb + c - c0;
        if (e < 0 || e >= nj) continue;
        float2 sum = make_float2(0.f, 0.f);
        const float2* ps = a.part + static_cast<size_t>(p) * a.npitch + e;
        int q = 0;
        for (; q + 4 <= a.S; q += 4) {
            float2 x[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) x[t] = ldcg2(ps + (q + t) * sstep);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                sum.x += x[t].x;
                sum.y += x[t].y;
            }
        }
        for (; q < a.S; ++q) {
            const float2 x = ldcg2(ps + q * sstep);
            sum.x += x.x;
            sum.y += x.y;
        }
        if (mode == 0) {
            const float2 vv = ldcg2(a.v + c0 + e), ss = ldcg2(a.s + static_cast<size_t>(i) * a.ld + c0 + e);
            sum.x += a.rho * (vv.x - ss.x);
            sum.y += a.rho * (vv.y - ss.y);
            stcg2(a.Q + static_cast<size_t>(p) * a.npitch + e, sum);
        } else {
            stcg2(a.C + static_cast<size_t>(p) * a.npitch + e, sum);
        }
    }
    if (tid == 0) a.cnt_cols[tile] = 0u;
}

// ---- one column block: q_i = C_i + rho (v - s_i) into the slot of the current
// iteration (later iterations get theirs from the update) ---------------------
__global__ void __launch_bounds__(kDirFacThreads) dir_q_kernel(const DirectArgs a) {
    if (stopped(a)) return;
    const long long total = static_cast<long long>(a.M) * a.n;
    float2* Q = a.Q + static_cast<size_t>(__ldcg(a.k_done) & 1) * a.P * a.npitch;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e / a.n), c = static_cast<int>(e - static_cast<long long>(i) * a.n);
        const float2 cv = a.C[static_cast<size_t>(i) * a.npitch + c];
        const float2 vv = ldcg2(a.v + c), ss = ldcg2(a.s + static_cast<size_t>(i) * a.ld + c);
        stcg2(Q + static_cast<size_t>(i) * a.npitch + c,
              make_float2(cv.x + a.rho * (vv.x - ss.x), cv.y + a.rho * (vv.y - ss.y)));
    }
}

__device__ void finish_record(const DirectArgs& a, long long k, int lane);

// Consensus update of update chunk `chunk` (entries row0 .. row0 + 16 of
// column block j), run by the warp that completed the chunk: v_j, s_j^i over
// those columns (with one column block also the next iteration's q_i there),
// the chunk's residual partials, and, by the warp that completes the last
// chunk of all, the iteration's residual record.
__device__ void update_chunk(const DirectArgs& a, int j, int c0, int nj, int row0, int chunk, long long k,
                             int lane) {
    __threadfence();
    float d[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const int cl = row0 + lane;
    if (lane < kDirChunk && cl < nj) {
        // replicas eight at a time, every load of a group issued before its use
        const int col = c0 + cl;
        const float2 vv = ldcg2(a.v + col);
        float2 sum = make_float2(0.f, 0.f);
        for (int rg = 0; rg < a.M; rg += 8) {
            float2 uu[8], ss[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const bool in = rg + q < a.M;
                const size_t o = static_cast<size_t>(rg + q) * a.ld + col;
                uu[q] = in ? ldcg2(a.u + o) : make_float2(0.f, 0.f);
                ss[q] = in ? ldcg2(a.s + o) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                sum.x += uu[q].x + ss[q].x;
                sum.y += uu[q].y + ss[q].y;
            }
        }
        const float2 av = make_float2(sum.x * a.inv_M, sum.y * a.inv_M);
        const float2 vn = shrink(av, a.kappa);
        d[1] = sq2(make_float2(vn.x - vv.x, vn.y - vv.y));
        d[3] = sq2(vn);
        float2* qn = a.Q + (a.N == 1 ? static_cast<size_t>((k + 1) & 1) * a.P * a.npitch : 0);
        for (int rg = 0; rg < a.M; rg += 8) {
            float2 uu[8], ss[8], cv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const bool in = rg + q < a.M;
                const size_t o = static_cast<size_t>(rg + q) * a.ld + col;
                uu[q] = in ? ldcg2(a.u + o) : make_float2(0.f, 0.f);
                ss[q] = in ? ldcg2(a.s + o) : make_float2(0.f, 0.f);
                cv[q] = (in && a.N == 1) ? ldcg2(a.C + static_cast<size_t>(rg + q) * a.npitch + col)
                                         : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (rg + q >= a.M) continue;
                const float2 sn = make_float2(ss[q].x + uu[q].x - vn.x, ss[q].y + uu[q].y - vn.y);
                d[0] += sq2(make_float2(uu[q].x - vn.x, uu[q].y - vn.y));
                d[2] += sq2(uu[q]);
                d[4] += sq2(sn);
                stcg2(a.s + static_cast<size_t>(rg + q) * a.ld + col, sn);
                if (a.N == 1)   // q_i of the next iteration: H_i^H g_i + rho (v - s_i)
                    stcg2(qn + static_cast<size_t>(rg + q) * a.npitch + col,
                          make_float2(cv[q].x + a.rho * (vn.x - sn.x), cv[q].y + a.rho * (vn.y - sn.y)));
            }
        }
        stcg2(a.v + col, vn);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q)
        for (int o = 16; o > 0; o >>= 1) d[q] += __shfl_xor_sync(0xffffffffu, d[q], o);
    int fin = 0;
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) __stcg(a.res_chunk + static_cast<size_t>(chunk) * 5 + q, static_cast<double>(d[q]));
        a.cnt_upd[chunk] = 0u;
        __threadfence();
        fin = atomicAdd(a.cnt_glob, 1u) == static_cast<unsigned>(a.nchunks - 1);
    }
    if (!__shfl_sync(0xffffffffu, fin, 0)) return;
    finish_record(a, k, lane);
}

// Residual record of iteration k from the update chunks' partials (the same
// five norms as the persistent kernel), by the warp that finished the last
// chunk; with the stopping test, the stop flags; then the device iteration
// count.
__device__ void finish_record(const DirectArgs& a, long long k, int lane) {
    __threadfence();
    double acc[5] = {0, 0, 0, 0, 0};
    for (int c = lane; c < a.nchunks; c += 32) {
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[q] += __ldcg(a.res_chunk + static_cast<size_t>(c) * 5 + q);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = warp_sum_d(acc[q]);
    if (lane == 0) {
        a.cnt_glob[0] = 0u;
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
        // (the next kernel reads the count after this one ends)
        *reinterpret_cast<volatile long long*>(a.k_done) = k + 1;
    }
}

// ---- factor pass + update ----------------------------------------------------
// The factor rows of all blocks, concatenated, are cut into one contiguous
// range per warp (two CTAs of eight warps per SM, one wave).  A warp takes its
// rows up to four at a time (never across a block or an update chunk), with
// four 16-byte loads per row in flight per lane, and q_b through the
// read-only cache.  Each update chunk counts the rows done for it over the M
// replicas; the warp whose rows complete it runs update_chunk.
__global__ void __launch_bounds__(kDirFacThreads, 2) dir_factor_kernel(const DirectArgs a) {
    if (stopped(a)) return;
    const int lane = threadIdx.x & 31;
    const int wpc = blockDim.x >> 5;
    const long long W = static_cast<long long>(gridDim.x) * wpc;
    const long long gw = static_cast<long long>(blockIdx.x) * wpc + (threadIdx.x >> 5);
    int r = static_cast<int>(gw * a.frows / W);
    const int rend = static_cast<int>((gw + 1) * a.frows / W);
    if (r >= rend) return;
    const long long k = __ldcg(a.k_done);
    const size_t qslot = a.N == 1 ? static_cast<size_t>(k & 1) * a.P * a.npitch : 0;
    int p = 0;
    while (a.F_off[p + 1] <= r) ++p;
    while (r < rend) {
        while (a.F_off[p + 1] <= r) ++p;
        const int i = p / a.N, j = p - i * a.N;
        const int c0 = a.col_off[j], nj = a.col_off[j + 1] - c0;
        const int row = r - a.F_off[p];
        const int row0 = row - row % kDirChunk;
        const int cend = min(row0 + kDirChunk, nj);
        const int g = min(min(4, cend - row), rend - r);
        const int npairs = (nj + 1) >> 1;
        const float4* q4 = reinterpret_cast<const float4*>(a.Q + qslot + static_cast<size_t>(p) * a.npitch);
        const float2* Lp = a.L + a.L_off[p];
        const int pitch = a.L_pitch[p];
        const float4* lr[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)   // rows past the group repeat its last row and are dropped
            lr[q] = reinterpret_cast<const float4*>(Lp + static_cast<size_t>(row + min(q, g - 1)) * pitch);
        float2 acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
        int e = lane;
        for (; e + 96 < npairs; e += 128) {
            float4 x[4], l[4][4];
#pragma unroll
            for (int t = 0; t < 4; ++t) x[t] = __ldg(q4 + e + 32 * t);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int t = 0; t < 4; ++t) l[q][t] = __ldg(lr[q] + e + 32 * t);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    cfma(acc[q], make_float2(l[q][t].x, l[q][t].y), make_float2(x[t].x, x[t].y));
                    cfma(acc[q], make_float2(l[q][t].z, l[q][t].w), make_float2(x[t].z, x[t].w));
                }
        }
        for (; e < npairs; e += 32) {
            const float4 x = __ldg(q4 + e);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 l = __ldg(lr[q] + e);
                cfma(acc[q], make_float2(l.x, l.y), make_float2(x.x, x.y));
                cfma(acc[q], make_float2(l.z, l.w), make_float2(x.z, x.w));
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = warp_sum(acc[q]);
        int last = 0;
        const int chunk = a.chunk_off[j] + row0 / kDirChunk;
        if (lane == 0) {
            float2* up = a.u + static_cast<size_t>(i) * a.ld + c0 + row;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < g) stcg2(up + q, acc[q]);
            __threadfence();
            const unsigned need = static_cast<unsigned>(a.M * (cend - row0));
            last = atomicAdd(a.cnt_upd + chunk, static_cast<unsigned>(g)) + g == need;
        }
        if (__shfl_sync(0xffffffffu, last, 0)) update_chunk(a, j, c0, nj, row0, chunk, k, lane);
        r += g;
    }
}

// ---- Hermitian factor pass + update -------------------------------------------
// L_b is Hermitian, so only its lower triangle is kept, in kDirTile x kDirTile
// tiles (diagonal tiles whole), about half the bytes of the full factor.
// Tile (I, J) adds L_IJ q_J to the rows of panel I and, below the diagonal,
// L_IJ^H q_I to the rows of panel J:
//     u_I = sum_{J <= I} L_IJ q_J + sum_{I' > I} L_I'I^H q_I'.
// Each tile's two sums are written out and added per row in a fixed order,
// so the result does not depend on which warp took which tile.

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start before its predecessor in the stream completes;
// pdl_wait blocks until the predecessor has completed and its writes are
// visible (a no-op without such a predecessor), pdl_trigger lets the
// successor start once every CTA of this grid has triggered or exited.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// a slot's piece number, published by the producer before it arms the slot
__device__ __forceinline__ void st_release_shared(int* p, int v) {
    asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_shared(const int* p) {
    int v;
    asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}

// Consumer wait for piece e in `slot`.  Different warps consume a slot's
// successive uses, so a warp may reach its use while the slot is still two
// phases behind, where a parity test alone would pass on the older phase:
// first the producer's piece number for the slot must be e (the slot's phase
// is then e's, running or complete), then the phase's parity.  Both waits are
// bounded.
__device__ __forceinline__ bool herm_wait_piece(const int* meta, uint64_t* full, int slot, long long e,
                                                const DirectArgs& a) {
    if (ld_acquire_shared(meta + slot) != static_cast<int>(e)) {
        const long long t0 = global_timer_ns();
        while (ld_acquire_shared(meta + slot) != static_cast<int>(e)) {
            if (global_timer_ns() - t0 > a.timeout_ns) {
                raise_status(a.status, ADMM_ETIMEOUT);
                return false;
            }
            __nanosleep(64);
        }
    }
    return mbar_wait_bounded(&full[slot], static_cast<uint32_t>((e / kHermSlots) & 1), a.status, a.timeout_ns);
}

constexpr int kHermPieces = kDirTile / kHermPieceRows;          // pieces per tile
constexpr int kHermUpdThreads = 256;                             // the update kernel's CTA
constexpr int kHermPieceBytes = kHermPieceRows * kDirTile * 8;  // 8 KB
constexpr int kHermCopyBytes = kHermPieceBytes < 8192 ? kHermPieceBytes : 8192;   // bytes per bulk copy
static_assert(kHermPieceBytes % kHermCopyBytes == 0, "whole copies per piece");
static_assert(kHermSlots % kHermPieces == 0, "a tile's pieces sit in consecutive slots");

__global__ void __launch_bounds__((kHermWarps + 1) * 32, 1) dir_herm_tile_kernel(const DirectArgs a) {
    extern __shared__ __align__(128) unsigned char hsm[];
    uint64_t* full = reinterpret_cast<uint64_t*>(hsm + static_cast<size_t>(kHermSlots) * kHermPieceBytes);
    uint64_t* empty = full + kHermSlots;
    int* meta = reinterpret_cast<int*>(empty + kHermSlots);   // piece number of each slot's current use
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x, c = blockIdx.x;
    const int ntile = c < a.ntiles ? (a.ntiles - 1 - c) / G + 1 : 0;   // this CTA's tiles
    if (ntile == 0) return;
    __shared__ int skip;
    if (threadIdx.x == 0) {
        // the previous update may still run (programmatic launch): the flag
        // read here can be stale, so the consumers read it again after their wait
        skip = stopped(a) ? 1 : 0;
        for (int q = 0; q < kHermSlots; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
            meta[q] = -1;
        }
        fence_mbarrier_init();
    }
    __syncthreads();
    if (skip) return;
    if (warp == kHermWarps) {
        // producer: piece e = kHermPieces i + h of the CTA's stream into slot e % kHermSlots.
        // The tiles change only at a factorisation, never inside an iteration,
        // so the producer streams while the previous update still runs.
        if (lane != 0) return;
        const uint64_t pol = policy_evict_first();   // every tile is read once per iteration
        long long e = 0;
        bool ok = true;
        auto tile_src = [&](int i) {
            return reinterpret_cast<const unsigned char*>(
                a.Lt + (static_cast<size_t>(c) + static_cast<size_t>(i) * G) * kDirTile * kDirTile);
        };
        for (int i = 0; i < ntile && ok; ++i) {
            const unsigned char* src = tile_src(i);
            for (int h = 0; h < kHermPieces; ++h, ++e) {
                const int slot = static_cast<int>(e % kHermSlots);
                const uint32_t use = static_cast<uint32_t>(e / kHermSlots);
                if (use > 0 && !mbar_wait_bounded(&empty[slot], (use - 1) & 1u, a.status, a.timeout_ns)) {
                    ok = false;
                    break;
                }
                st_release_shared(meta + slot, static_cast<int>(e));
                mbar_arrive_expect_tx(&full[slot], static_cast<uint32_t>(kHermPieceBytes));
                unsigned char* dst = hsm + static_cast<size_t>(slot) * kHermPieceBytes;
                const unsigned char* sp = src + static_cast<size_t>(h) * kHermPieceBytes;
#pragma unroll
                for (int o = 0; o < kHermPieceBytes; o += kHermCopyBytes)
                    bulk_load_hint(dst + o, sp + o, kHermCopyBytes, &full[slot], pol);
            }
        }
        // every copy into this CTA's shared memory lands before the CTA ends
        // (earlier pieces' slots were consumed and reused)
        for (long long q = e - 1; q >= 0 && q >= e - kHermSlots; --q)
            mbar_wait_bounded(&full[q % kHermSlots], static_cast<uint32_t>((q / kHermSlots) & 1), a.status,
                              a.timeout_ns);
        return;
    }
    // consumers: q_b, the iteration count and the tile sums' buffers belong to
    // the previous kernel until it completes; then the update may launch
    pdl_wait();
    pdl_trigger();
    long long k;
    if (a.defer_record) {
        k = __ldcg(a.dctl);
        if (c == 0 && warp == 0) {
            // the record of the previous iteration (its partials are in), and
            // the iteration number for the update
            if (lane == 0) a.dctl[1] = k;
            if (__ldcg(a.dctl + 2) != 0) {
                finish_record(a, k - 1, lane);
                if (lane == 0) a.dctl[2] = 0;
            }
        }
    } else {
        k = __ldcg(a.k_done);
    }
    const bool live = !stopped(a);   // stopped by the previous update: release the pieces unread
    const size_t qslot = a.N == 1 ? static_cast<size_t>(k & 1) * a.P * a.npitch : 0;
    // the warp's next tile and its q pairs, fetched one tile ahead, and the
    // table entry of the tile after it two tiles ahead (the q loads depend on it)
    auto entry = [&](int i) {
        return i < ntile ? __ldg(a.T_seq + c + static_cast<long long>(i) * G) : make_int4(0, 0, 0, 0);
    };
    int4 tn = entry(warp), tn2 = entry(warp + kHermWarps);
    float4 nqJ = make_float4(0.f, 0.f, 0.f, 0.f), nqI = nqJ;
    auto fetch = [&]() {
        const float2* qb = a.Q + qslot + static_cast<size_t>(tn.y) * a.npitch;
        nqJ = __ldg(reinterpret_cast<const float4*>(qb + tn.w * kDirTile) + lane);
        nqI = __ldg(reinterpret_cast<const float4*>(qb + tn.z * kDirTile) + lane);
    };
    if (warp < ntile) fetch();
    for (int i = warp; i < ntile; i += kHermWarps) {
        const int t = tn.x, I = tn.z, J = tn.w;
        const float4 qJ = nqJ, qI = nqI;
        tn = tn2;
        tn2 = entry(i + 2 * kHermWarps);
        if (i + kHermWarps < ntile) fetch();
        const bool diag = I == J;
        float2 c0 = make_float2(0.f, 0.f), c1 = make_float2(0.f, 0.f);
        bool ok = true;
        for (int h = 0; h < kHermPieces; ++h) {
            const long long e = static_cast<long long>(i) * kHermPieces + h;
            const int slot = static_cast<int>(e % kHermSlots);
            if (!herm_wait_piece(meta, full, slot, e, a)) {
                ok = false;
                break;
            }
            if (!live) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
                continue;
            }
            const float4* T4 = reinterpret_cast<const float4*>(hsm + static_cast<size_t>(slot) * kHermPieceBytes);
#pragma unroll
            for (int gg = 0; gg < kHermPieceRows / 8; ++gg) {
                float4 l[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) l[q] = T4[(8 * gg + q) * (kDirTile / 2) + lane];
                float2 racc[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    racc[q] = make_float2(0.f, 0.f);
                    cfma(racc[q], make_float2(l[q].x, l[q].y), make_float2(qJ.x, qJ.y));
                    cfma(racc[q], make_float2(l[q].z, l[q].w), make_float2(qJ.z, qJ.w));
                }
                const int row0 = h * kHermPieceRows + 8 * gg;   // tile row of l[0]
                const float2 rs = lanes_sum8(racc, lane);
                if ((lane & 3) == 0) stcg2(a.RP + static_cast<size_t>(t) * kDirTile + row0 + (lane >> 2), rs);
                if (!diag) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        // q_I of tile row row0 + q, held by lane (row0 + q) / 2
                        const int src = (row0 >> 1) + (q >> 1);
                        const float2 qi = make_float2(__shfl_sync(0xffffffffu, (q & 1) ? qI.z : qI.x, src),
                                                      __shfl_sync(0xffffffffu, (q & 1) ? qI.w : qI.y, src));
                        cfma_conj(c0, make_float2(l[q].x, l[q].y), qi);
                        cfma_conj(c1, make_float2(l[q].z, l[q].w), qi);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
        }
        if (!ok) break;
        if (live && !diag)   // the tile's column sums
            __stcg(reinterpret_cast<float4*>(a.CP + static_cast<size_t>(t) * kDirTile) + lane,
                   make_float4(c0.x, c0.y, c1.x, c1.y));
    }
}

// ---- panel sums + update (after the tile pass) ---------------------------------
// One CTA per update chunk (kDirChunk columns of column block j), eight
// warps.  Warp w takes the replicas i = w, w + 8, ...: the chunk's rows of
// u_b, each the sum of its NT tile sums in tile order (lanes 0-15 the first
// half of the tiles, 16-31 the second, sixteen loads in flight, then the two
// halves added), kept in shared memory with s_i and, with one column block,
// H_i^H g_i.  Then v over the chunk (warp 0, replicas in order), the duals
// and the next q per replica, and the chunk's residual partials (warps in
// order).  With several column blocks the CTA that adds the last chunk writes
// the iteration's record; with one (defer_record) the next tile pass or the
// record kernel writes it.  Shared memory: 3 M kDirChunk + kDirChunk complex
// values.
__global__ void __launch_bounds__(kHermUpdThreads) dir_herm_update_kernel(const DirectArgs a) {
    extern __shared__ float2 hred[];
    // launched once every tile CTA has seen the previous update complete, so
    // v, s and H_i^H g_i are current here (and, unless the record is deferred
    // to the tile pass, the stop flag); the next tile pass may start
    // streaming right away
    if (!a.defer_record && stopped(a)) return;
    pdl_trigger();
    constexpr int kWarps = kHermUpdThreads / 32;
    float2* us = hred;                                  // M x kDirChunk: u
    float2* ss = us + a.M * kDirChunk;                  // s before the update
    float2* cs = ss + a.M * kDirChunk;                  // H_i^H g_i (one column block)
    float2* vs = cs + a.M * kDirChunk;                  // kDirChunk: the new v
    __shared__ float dred[kWarps][5];
    __shared__ int last;
    const int chunk = blockIdx.x;
    int j = 0;
    while (a.chunk_off[j + 1] <= chunk) ++j;
    const int c0 = a.col_off[j], nj = a.col_off[j + 1] - c0;
    const int row0 = (chunk - a.chunk_off[j]) * kDirChunk;   // the chunk's first column in the block
    const int X = row0 / kDirTile, rr = row0 - X * kDirTile;
    const int NT = (nj + kDirTile - 1) / kDirTile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = lane & (kDirChunk - 1), half = lane >> 4;
    const bool inb = row0 + r < nj;
    const int col = c0 + row0 + r;
    const int hK = (NT + 1) >> 1;
    const int kb = half ? hK : 0, ke = half ? NT : hK;
    // v, s_i and H_i^H g_i of the chunk before the tile pass ends
    const float2 vv = (warp == 0 && half == 0 && inb) ? ldcg2(a.v + col) : make_float2(0.f, 0.f);
    for (int i = warp; i < a.M; i += kWarps)
        if (half == 0) {
            float2 sv = make_float2(0.f, 0.f), cv = sv;
            if (inb) {
                sv = ldcg2(a.s + static_cast<size_t>(i) * a.ld + col);
                if (a.N == 1) cv = ldcg2(a.C + static_cast<size_t>(i) * a.npitch + col);
            }
            ss[i * kDirChunk + r] = sv;
            cs[i * kDirChunk + r] = cv;
        }
    // the first replica's tile offset (constant) before the wait
    long long tb = warp < a.M ? __ldg(a.T_off + warp * a.N + j) : 0;
    pdl_wait();   // the tile sums (and a deferred record, with its stop flag)
    if (a.defer_record && stopped(a)) return;
    const long long k = a.defer_record ? __ldcg(a.dctl + 1) : __ldcg(a.k_done);
    for (int i = warp; i < a.M; i += kWarps) {
        if (i != warp) tb = __ldg(a.T_off + i * a.N + j);
        // the contributions to row row0 + r: tiles (X, kk) for kk <= X (row
        // sums), tiles (kk, X) for kk > X (column sums)
        float2 acc = make_float2(0.f, 0.f);
        for (int k0 = kb; k0 < ke; k0 += 16) {
            float2 x[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int kk = k0 + q;
                const float2* src = kk <= X ? a.RP + (tb + X * (X + 1) / 2 + kk) * kDirTile
                                            : a.CP + (tb + static_cast<long long>(kk) * (kk + 1) / 2 + X) * kDirTile;
                x[q] = kk < ke ? ldcg2(src + rr + r) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                acc.x += x[q].x;
                acc.y += x[q].y;
            }
        }
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 16);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 16);
        if (half == 0) {
            us[i * kDirChunk + r] = acc;
            if (inb) stcg2(a.u + static_cast<size_t>(i) * a.ld + col, acc);
        }
    }
    __syncthreads();
    float d[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (warp == 0 && half == 0 && inb) {
        float2 sum = make_float2(0.f, 0.f);
        for (int i = 0; i < a.M; ++i) {
            sum.x += us[i * kDirChunk + r].x + ss[i * kDirChunk + r].x;
            sum.y += us[i * kDirChunk + r].y + ss[i * kDirChunk + r].y;
        }
        const float2 vn = shrink(make_float2(sum.x * a.inv_M, sum.y * a.inv_M), a.kappa);
        d[1] = sq2(make_float2(vn.x - vv.x, vn.y - vv.y));
        d[3] = sq2(vn);
        vs[r] = vn;
        stcg2(a.v + col, vn);
    }
    __syncthreads();
    if (half == 0 && inb) {
        const float2 vn = vs[r];
        float2* qn = a.Q + (a.N == 1 ? static_cast<size_t>((k + 1) & 1) * a.P * a.npitch : 0);
        for (int i = warp; i < a.M; i += kWarps) {
            const float2 uu = us[i * kDirChunk + r], so = ss[i * kDirChunk + r];
            const float2 sn = make_float2(so.x + uu.x - vn.x, so.y + uu.y - vn.y);
            d[0] += sq2(make_float2(uu.x - vn.x, uu.y - vn.y));
            d[2] += sq2(uu);
            d[4] += sq2(sn);
            stcg2(a.s + static_cast<size_t>(i) * a.ld + col, sn);
            if (a.N == 1) {   // q_i of the next iteration: H_i^H g_i + rho (v - s_i)
                const float2 cv = cs[i * kDirChunk + r];
                stcg2(qn + static_cast<size_t>(i) * a.npitch + col,
                      make_float2(cv.x + a.rho * (vn.x - sn.x), cv.y + a.rho * (vn.y - sn.y)));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        for (int o = 8; o > 0; o >>= 1) d[q] += __shfl_xor_sync(0xffffffffu, d[q], o);
        if (lane == 0) dred[warp][q] = d[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            double t = 0.0;
            for (int w = 0; w < kWarps; ++w) t += static_cast<double>(dred[w][q]);
            __stcg(a.res_chunk + static_cast<size_t>(chunk) * 5 + q, t);
        }
        if (a.defer_record) {
            // every CTA writes the same values; the next tile pass reads them
            // after this grid ends
            a.dctl[0] = k + 1;
            a.dctl[2] = 1;
            last = 0;
        } else {
            __threadfence();
            last = atomicAdd(a.cnt_glob, 1u) == static_cast<unsigned>(a.nchunks - 1);
        }
    }
    __syncthreads();
    if (last && warp == 0) finish_record(a, k, lane);
}

// the record left pending by the last update of a launch sequence
__global__ void dir_record_kernel(const DirectArgs a) {
    if (__ldcg(a.dctl + 2) == 0) return;
    finish_record(a, __ldcg(a.dctl) - 1, threadIdx.x & 31);
    if (threadIdx.x == 0) a.dctl[2] = 0;
}

// the tiles of the pass, in its order, from the full factors (setup, after
// every factorisation); the parts of a tile past n_j are zero
__global__ void pack_herm_kernel(const float2* __restrict__ L, const long long* __restrict__ L_off,
                                 const int* __restrict__ L_pitch, const int* __restrict__ col_off, int N,
                                 const int4* __restrict__ T_seq, long long ntiles, float2* __restrict__ Lt) {
    const long long total = ntiles * kDirTile * kDirTile;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long pos = e / (kDirTile * kDirTile);
        const int w = static_cast<int>(e - pos * kDirTile * kDirTile);
        const int4 tq = T_seq[pos];
        const int p = tq.y, j = p % N;
        const int nj = col_off[j + 1] - col_off[j];
        const int r = tq.z * kDirTile + w / kDirTile, cc = tq.w * kDirTile + w % kDirTile;
        Lt[e] = (r < nj && cc < nj) ? L[L_off[p] + static_cast<long long>(r) * L_pitch[p] + cc]
                                    : make_float2(0.f, 0.f);
    }
}

// ---- streamed factor pass + update -------------------------------------------
// The same work as dir_factor_kernel for blocks up to kDirBulkMaxCols wide.
// Work items are the update chunks of every block (16 factor rows of block p,
// contiguous in memory), handed out by a global counter: one producer lane per
// CTA takes an item (fetching the next one while it streams the current), and
// streams it in stages of up to four rows with one 1-D bulk copy per row into
// a ring of shared-memory slots, each slot carrying its stage's description;
// a slot with no rows ends the CTA's work.  Every consumer warp takes one
// eighth of the columns of all rows of a stage (its segment of q_b stays in
// registers while the block lasts); the warp that adds its partial sums last
// (a shared-memory counter per slot, no barrier) sums the eight in warp order,
// writes u and adds the rows to the CTA's table of chunks in shared memory.
// After the last stage the table's counts go to the global chunk counters and
// the warps that complete a chunk run its update, so no stage waits for a
// global atomic or an update.  The last CTA to run out of items resets the
// item counter.  Every wait is bounded (ADMM_ETIMEOUT), and the producer waits
// for all its copies before the CTA ends.
__global__ void __launch_bounds__((kDirBulkWarps + 1) * 32, 1) dir_factor_stream_kernel(const DirectArgs a) {
    extern __shared__ __align__(128) unsigned char fsm[];
    if (stopped(a)) return;
    const int NS = a.fac_ns;
    unsigned char* ring = fsm;
    uint64_t* full = reinterpret_cast<uint64_t*>(fsm + static_cast<size_t>(NS) * a.fac_stage);
    uint64_t* empty = full + NS;
    float2* red = reinterpret_cast<float2*>(empty + NS);                  // NS x kDirBulkWarps x 4
    int* red_cnt = reinterpret_cast<int*>(red + NS * kDirBulkWarps * 4);  // NS
    int* tab_chunk = red_cnt + NS;                                        // kDirDeferred chunks of this CTA
    int* tab_cnt = tab_chunk + kDirDeferred;                              // rows counted for each
    int* meta = tab_cnt + kDirDeferred;                                   // NS x 4: p, row, g, table index
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < NS; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], kDirBulkWarps);
            red_cnt[q] = 0;
        }
        for (int q = 0; q < kDirDeferred; ++q) tab_cnt[q] = 0;
        fence_mbarrier_init();
    }
    __syncthreads();
    const long long k = __ldcg(a.k_done);
    unsigned* items = a.cnt_glob + 2;   // [0] next item, [1] CTAs out of items
    if (warp == kDirBulkWarps) {
        if (lane != 0) return;
        int issued = 0, slot = 0, p = 0, nitem = 0;
        uint32_t ph = 0;
        bool ok = true;
        int it = static_cast<int>(atomicAdd(items, 1u));
        while (ok && it < a.fitems) {
            const int nxt = static_cast<int>(atomicAdd(items, 1u));   // fetched while this item streams
            while (a.I_off[p + 1] <= it) ++p;
            const int j = p % a.N;
            const int nj = a.col_off[j + 1] - a.col_off[j];
            const int pitch = a.L_pitch[p];
            const uint32_t rbytes = static_cast<uint32_t>(pitch) * sizeof(float2);
            const int row_end = min((it - a.I_off[p] + 1) * kDirChunk, nj);
            for (int row = (it - a.I_off[p]) * kDirChunk; row < row_end;) {
                const int g = min(4, row_end - row);
                if (!mbar_wait_bounded(&empty[slot], ph ^ 1u, a.status, a.timeout_ns)) {
                    ok = false;
                    break;
                }
                int* m = meta + slot * 4;
                m[0] = p;
                m[1] = row;
                m[2] = g;
                m[3] = nitem;
                mbar_arrive_expect_tx(&full[slot], rbytes * g);
                // the stage's rows are contiguous: copies of at most 4 KB each
                const unsigned char* src = reinterpret_cast<const unsigned char*>(
                    a.L + a.L_off[p] + static_cast<size_t>(row) * pitch);
                unsigned char* dst = ring + static_cast<size_t>(slot) * a.fac_stage;
                const uint32_t total = rbytes * g;
                for (uint32_t off = 0; off < total; off += 4096u)
                    bulk_load(dst + off, src + off, min(4096u, total - off), &full[slot]);
                ++issued;
                if (++slot == NS) {
                    slot = 0;
                    ph ^= 1u;
                }
                row += g;
            }
            ++nitem;
            it = nxt;
        }
        // the last CTA out of items resets the item counter for the next launch
        if (atomicAdd(items + 1, 1u) == gridDim.x - 1) {
            items[0] = 0u;
            items[1] = 0u;
        }
        // every copy into this CTA's shared memory lands before the closing slot
        // (which completes one more phase of its slot) and before the CTA ends
        for (int q = 0; q < NS && q < issued; ++q) {
            const int lastq = q + ((issued - 1 - q) / NS) * NS;
            mbar_wait_bounded(&full[q], static_cast<uint32_t>((lastq / NS) & 1), a.status, a.timeout_ns);
        }
        // closing slot: no rows, no copy
        if (ok && mbar_wait_bounded(&empty[slot], ph ^ 1u, a.status, a.timeout_ns)) {
            int* m = meta + slot * 4;
            m[0] = p;
            m[1] = 0;
            m[2] = 0;
            m[3] = nitem;
            mbar_arrive(&full[slot]);
        }
        return;
    }
    const size_t qslot = a.N == 1 ? static_cast<size_t>(k & 1) * a.P * a.npitch : 0;
    int slot = 0, qp = -1, nlc = 0;
    uint32_t ph = 0;
    float2 qre[8], qim[8];
    for (;;) {
        if (!mbar_wait_bounded(&full[slot], ph, a.status, a.timeout_ns)) break;
        const int* m = meta + slot * 4;
        const int p = m[0], row = m[1], g = m[2], lc = m[3];
        if (g == 0) break;   // closing slot
        nlc = lc + 1;
        const int i = p / a.N, j = p - i * a.N;
        const int c0 = a.col_off[j], nj = a.col_off[j + 1] - c0;
        const int row0 = row - row % kDirChunk;
        const int cend = min(row0 + kDirChunk, nj);
        const int chunk = a.chunk_off[j] + row0 / kDirChunk;
        const int pitch = a.L_pitch[p];
        const int npairs = (nj + 1) >> 1;
        const int seg = (npairs + kDirBulkWarps - 1) / kDirBulkWarps;
        const int e_beg = warp * seg, e_end = min(npairs, e_beg + seg);
        const float4* l4 = reinterpret_cast<const float4*>(ring + static_cast<size_t>(slot) * a.fac_stage);
        if (p != qp) {
            // this warp's segment of q_b, kept in registers while the block lasts,
            // as (re, re) and (im, im) pairs for the paired FMAs
            const float4* q4 = reinterpret_cast<const float4*>(a.Q + qslot + static_cast<size_t>(p) * a.npitch);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int e = e_beg + lane + 32 * t;
                const float4 x = e < e_end ? __ldg(q4 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
                qre[2 * t] = make_float2(x.x, x.x);
                qim[2 * t] = make_float2(x.y, x.y);
                qre[2 * t + 1] = make_float2(x.z, x.z);
                qim[2 * t + 1] = make_float2(x.w, x.w);
            }
            qp = p;
        }
        const int rstep = pitch / 2;   // float4 per factor row
        // row q: A = sum (L.re q.re, L.im q.re), B = sum (L.re q.im, L.im q.im);
        // L q = (A.x - B.y, A.y + B.x)
        float2 A[4], Bv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) A[q] = Bv[q] = make_float2(0.f, 0.f);
        float4 l[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int e = e_beg + lane + 32 * t;
                l[q][t] = (q < g && e < e_end) ? l4[q * rstep + e] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float2 lo = make_float2(l[q][t].x, l[q][t].y), hi = make_float2(l[q][t].z, l[q][t].w);
                A[q] = __ffma2_rn(lo, qre[2 * t], A[q]);
                Bv[q] = __ffma2_rn(lo, qim[2 * t], Bv[q]);
                A[q] = __ffma2_rn(hi, qre[2 * t + 1], A[q]);
                Bv[q] = __ffma2_rn(hi, qim[2 * t + 1], Bv[q]);
            }
        float2 acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = make_float2(A[q].x - Bv[q].y, A[q].y + Bv[q].x);
        // lane sums of the four rows: two halving exchanges, then three plain
        // steps; row q's sum ends in the lanes whose bits 4..3 spell q
        {
            const bool b16 = lane & 16, b8 = lane & 8;
            float2 h2[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float2 keep = b16 ? acc[q + 2] : acc[q], send = b16 ? acc[q] : acc[q + 2];
                h2[q] = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, send.x, 16),
                                    keep.y + __shfl_xor_sync(0xffffffffu, send.y, 16));
            }
            const float2 keep = b8 ? h2[1] : h2[0], send = b8 ? h2[0] : h2[1];
            float2 y = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, send.x, 8),
                                   keep.y + __shfl_xor_sync(0xffffffffu, send.y, 8));
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                y.x += __shfl_xor_sync(0xffffffffu, y.x, o);
                y.y += __shfl_xor_sync(0xffffffffu, y.y, o);
            }
            acc[0] = y;   // row 2 * b16 + b8
        }
        float2* rs = red + static_cast<size_t>(slot) * kDirBulkWarps * 4;
        int last = 0;
        if ((lane & 7) == 0) rs[warp * 4 + (lane >> 3)] = acc[0];   // lanes 0, 8, 16, 24: rows 0..3
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            last = atomicAdd(&red_cnt[slot], 1) == kDirBulkWarps - 1;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        int now = 0;   // the chunk table is full: count this stage's rows at once
        if (last) {
            __threadfence_block();
            if (lane < g) {
                float2 t = make_float2(0.f, 0.f);
                for (int w = 0; w < kDirBulkWarps; ++w) {
                    const volatile float* x = reinterpret_cast<volatile float*>(&rs[w * 4 + lane]);
                    t.x += x[0];
                    t.y += x[1];
                }
                stcg2(a.u + static_cast<size_t>(i) * a.ld + c0 + row + lane, t);
            }
            if (lane == 0) {
                red_cnt[slot] = 0;
                if (lc < kDirDeferred) {
                    tab_chunk[lc] = chunk;
                    atomicAdd(&tab_cnt[lc], g);
                } else {
                    now = 1;
                }
            }
            now = __shfl_sync(0xffffffffu, now, 0);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        if (now) {
            __threadfence();
            int done = 0;
            if (lane == 0)
                done = atomicAdd(a.cnt_upd + chunk, static_cast<unsigned>(g)) + g ==
                       static_cast<unsigned>(a.M * (cend - row0));
            if (__shfl_sync(0xffffffffu, done, 0)) update_chunk(a, j, c0, nj, row0, chunk, k, lane);
        }
        if (++slot == NS) {
            slot = 0;
            ph ^= 1u;
        }
    }
    // the chunks counted in the table: one global count each, then the updates
    // (every consumer warp reaches this barrier, also after a failed wait)
    __threadfence();
    asm volatile("bar.sync 1, %0;" ::"r"(kDirBulkWarps * 32) : "memory");
    nlc = min(nlc, kDirDeferred);
    for (int e = warp; e < nlc; e += kDirBulkWarps) {
        const int chunk = tab_chunk[e], cnt = tab_cnt[e];
        if (cnt == 0) continue;
        int j = 0;
        while (a.chunk_off[j + 1] <= chunk) ++j;
        const int c0 = a.col_off[j], nj = a.col_off[j + 1] - c0;
        const int row0 = (chunk - a.chunk_off[j]) * kDirChunk;
        int done = 0;
        if (lane == 0)
            done = atomicAdd(a.cnt_upd + chunk, static_cast<unsigned>(cnt)) + cnt ==
                   static_cast<unsigned>(a.M * (min(row0 + kDirChunk, nj) - row0));
        if (__shfl_sync(0xffffffffu, done, 0)) update_chunk(a, j, c0, nj, row0, chunk, k, lane);
    }
}

// ---- row pass: ghat_b = H_b u_b -----------------------------------------------
// The rows of H of all blocks, concatenated, are cut into one contiguous range
// per warp (two CTAs of eight warps per SM, one wave).  A warp takes its rows
// up to eight at a time within one block, reading 16-byte column pairs from the
// block's first column rounded down to even; u_b comes through the read-only
// cache with the halves outside the block zeroed.
__global__ void __launch_bounds__(kDirRowThreads, 2) dir_rows_kernel(const DirectArgs a) {
    __shared__ int last;
    if (!stopped(a)) {
        const int lane = threadIdx.x & 31;
        const int wpc = blockDim.x >> 5;
        const long long W = static_cast<long long>(gridDim.x) * wpc;
        const long long gw = static_cast<long long>(blockIdx.x) * wpc + (threadIdx.x >> 5);
        int x = static_cast<int>(gw * a.hrows / W);
        const int xend = static_cast<int>((gw + 1) * a.hrows / W);
        // after this iteration's update the device count is k + 1: its slot
        const size_t Nm = static_cast<size_t>(a.N) * a.m;
        float2* outb = a.ghat + static_cast<size_t>(__ldcg(a.k_done) & 1) * Nm;
        int p = 0;
        while (x < xend) {
            while (a.R_off[p + 1] <= x) ++p;
            const int i = p / a.N, j = p - i * a.N;
            const int r0 = a.row_off[i], mi = a.row_off[i + 1] - r0;
            const int c0 = a.col_off[j], nj = a.col_off[j + 1] - c0;
            const int row = x - a.R_off[p];
            const int g = min(min(8, mi - row), xend - x);
            const int cb = c0 & ~1;
            const int npairs = (c0 + nj - cb + 1) >> 1;
            const float4* u4 = reinterpret_cast<const float4*>(a.u + static_cast<size_t>(i) * a.ld + cb);
            const float4* hr[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                hr[q] = reinterpret_cast<const float4*>(a.H + static_cast<size_t>(r0 + row + min(q, g - 1)) * a.ld + cb);
            float2 acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
            for (int e = lane; e < npairs; e += 64) {
                const bool two = e + 32 < npairs;
                float4 u[2];
                u[0] = __ldg(u4 + e);
                u[1] = two ? __ldg(u4 + e + 32) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int col = cb + 2 * (e + 32 * t);
                    if (col < c0) u[t].x = u[t].y = 0.f;
                    if (col + 1 >= c0 + nj) u[t].z = u[t].w = 0.f;
                }
                float4 h[2][8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    h[0][q] = __ldg(hr[q] + e);
                    h[1][q] = two ? __ldg(hr[q] + e + 32) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int t = 0; t < 2; ++t)
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        cfma(acc[q], make_float2(h[t][q].x, h[t][q].y), make_float2(u[t].x, u[t].y));
                        cfma(acc[q], make_float2(h[t][q].z, h[t][q].w), make_float2(u[t].z, u[t].w));
                    }
            }
            const float2 tot = lanes_sum8(acc, lane);
            const int q = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
            if ((lane & 3) == 0 && q < g) stcg2(outb + static_cast<size_t>(j) * a.m + r0 + row + q, tot);
            x += g;
        }
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
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
    const int cols = (kDirColRows + 1 + (kDirColThreads / 32) * 2 * kDirColPairs) * 8;
    cudaError_t e =
        cudaFuncSetAttribute(dir_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, std::min(smem_optin, cols));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(dir_factor_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
    return e;
}

size_t stream_smem(int ns, int stage) {
    return static_cast<size_t>(ns) * stage + 2 * ns * sizeof(uint64_t) + ns * kDirBulkWarps * 4 * sizeof(float2) +
           ns * sizeof(int) + 2 * kDirDeferred * sizeof(int) + ns * 4 * sizeof(int);
}

cudaError_t direct_stream_per_sm(int smem, int* per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, dir_factor_stream_kernel, (kDirBulkWarps + 1) * 32,
                                                         static_cast<size_t>(smem));
}

cudaError_t launch_dir_cols(const DirectArgs& a, int mode, cudaStream_t s) {
    const int rows = (a.mimax + a.S - 1) / a.S + 1;
    const size_t smem = (static_cast<size_t>(rows) + (kDirColThreads / 32) * 2 * kDirColPairs) * sizeof(float2);
    dir_cols_kernel<<<a.P * a.ccn * a.S, kDirColThreads, smem, s>>>(a, mode);
    return cudaGetLastError();
}

cudaError_t launch_dir_q(const DirectArgs& a, cudaStream_t s) {
    const long long total = static_cast<long long>(a.M) * a.n;
    const int blocks = static_cast<int>(std::min<long long>((total + kDirFacThreads - 1) / kDirFacThreads, 4096));
    dir_q_kernel<<<blocks, kDirFacThreads, 0, s>>>(a);
    return cudaGetLastError();
}

size_t herm_smem_bytes() {
    return static_cast<size_t>(kHermSlots) * kHermPieceBytes + kHermSlots * (2 * sizeof(uint64_t) + sizeof(int));
}

size_t herm_update_smem(int M) { return (static_cast<size_t>(3) * M * kDirChunk + kDirChunk) * sizeof(float2); }

cudaError_t herm_per_sm(int* per_sm) {
    const int smem = static_cast<int>(herm_smem_bytes());
    cudaError_t e = cudaFuncSetAttribute(dir_herm_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(dir_herm_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(herm_update_smem(kDirHermMaxRowBlocks)));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, dir_herm_tile_kernel, (kHermWarps + 1) * 32, smem);
}

cudaError_t launch_pack_herm(const float2* L, const long long* L_off, const int* L_pitch, const int* col_off,
                             int N, const int4* T_seq, long long ntiles, float2* Lt, cudaStream_t s) {
    const long long total = ntiles * kDirTile * kDirTile;
    const int blocks = static_cast<int>(std::min<long long>((total + 255) / 256, 8192));
    pack_herm_kernel<<<blocks, 256, 0, s>>>(L, L_off, L_pitch, col_off, N, T_seq, ntiles, Lt);
    return cudaGetLastError();
}

cudaError_t launch_dir_factor(const DirectArgs& a, cudaStream_t s) {
    if (a.fac_herm) {
        // both with programmatic stream serialization: each may start while
        // its predecessor finishes (the kernels wait where they need to)
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(a.herm_ctas);
        cfg.blockDim = dim3((kHermWarps + 1) * 32);
        cfg.dynamicSmemBytes = herm_smem_bytes();
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, dir_herm_tile_kernel, a);
        if (e != cudaSuccess) return e;
        cfg.gridDim = dim3(a.nchunks);
        cfg.blockDim = dim3(kHermUpdThreads);
        cfg.dynamicSmemBytes = herm_update_smem(a.M);
        e = cudaLaunchKernelEx(&cfg, dir_herm_update_kernel, a);
        if (e != cudaSuccess) return e;
    } else if (a.fac_stream) {
        const size_t smem = stream_smem(a.fac_ns, a.fac_stage);
        dir_factor_stream_kernel<<<a.fac_ctas, (kDirBulkWarps + 1) * 32, smem, s>>>(a);
    } else {
        dir_factor_kernel<<<a.ctas, kDirFacThreads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_dir_record(const DirectArgs& a, cudaStream_t s) {
    dir_record_kernel<<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dir_rows(const DirectArgs& a, cudaStream_t s) {
    dir_rows_kernel<<<a.ctas, kDirRowThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_conj_transpose(const float2* H, int64_t m, int64_t n, int64_t ld, float2* HT, int64_t ldT,
                                  cudaStream_t s) {
    const dim3 grid(static_cast<unsigned>((n + 31) / 32), static_cast<unsigned>((m + 31) / 32));
    conj_transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(H, m, n, ld, HT, ldT);
    return cudaGetLastError();
}

}  // namespace admm
