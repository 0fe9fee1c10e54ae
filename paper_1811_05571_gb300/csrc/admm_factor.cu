// One-time factor cache of the inversion lemma (Eq. inversion_lemma,
// inversion_lemma2, inversion_lemma3): for every block b = (i, j)
//     K_b = rho I + H_b H_b^H          (m_i x m_i, Gram of the block rows)
//     K_b = L_b L_b^H                   (FP64 Cholesky, 32 x 32 tiles)
//     K_b^{-1} = L_b^{-H} L_b^{-1}      (FP64 triangular inverse + product)
// stored as complex64 with a row pitch padded to a multiple of 4.  The Gram
// products read complex64 H, multiply in FP32 and accumulate 32-term chunks
// into FP64.  Every block is padded to T*32 rows with an identity tail, so
// all tile kernels see square, full tiles.
#include <cmath>

#include "admm_internal.h"
#include "ptx.cuh"

namespace admm {
namespace {

__device__ __forceinline__ double2 dsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// a * conj(b)
__device__ __forceinline__ void dfma_nc(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.y, b.x, acc.y);
    acc.y = fma(-a.x, b.y, acc.y);
}
// a * b
__device__ __forceinline__ void dfma_nn(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// conj(a) * b
__device__ __forceinline__ void dfma_cn(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

struct BlockGeom {
    int r0, mi, c0, nj;
    size_t base;  // offset of the block's (T*32)^2 workspace
};

__device__ __forceinline__ BlockGeom geom(const FactorArgs& f, int b) {
    const int i = b / f.N, j = b - (b / f.N) * f.N;
    BlockGeom g;
    g.r0 = f.row_off[i];
    g.mi = f.row_off[i + 1] - g.r0;
    g.c0 = f.col_off[j];
    g.nj = f.col_off[j + 1] - g.c0;
    const size_t S = static_cast<size_t>(f.T) * kTile;
    g.base = static_cast<size_t>(b) * S * S;
    return g;
}

// lower-triangular tile pair index -> (row tile, column tile), row >= column
__device__ __forceinline__ void tri_pair(int idx, int& r, int& c) {
    r = static_cast<int>((sqrtf(8.0f * idx + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= idx) ++r;
    while (r * (r + 1) / 2 > idx) --r;
    c = idx - r * (r + 1) / 2;
}

// ---- Gram: A_b = rho I + H_b H_b^H (lower tiles), identity padding ----------
constexpr int kKC = 32;

__global__ void __launch_bounds__(256) gram_kernel(const FactorArgs f) {
    __shared__ float2 As[kTile][kKC + 1];
    __shared__ float2 Bs[kTile][kKC + 1];
    const int b = blockIdx.y;
    int tr, tc;
    tri_pair(blockIdx.x, tr, tc);
    const BlockGeom g = geom(f, b);
    const int tid = threadIdx.x;
    const int x = tid >> 3, y0 = tid & 7;
    const size_t S = static_cast<size_t>(f.T) * kTile;
    double2 accd[4];
    for (int q = 0; q < 4; ++q) accd[q] = make_double2(0.0, 0.0);
    const bool rows_live = tr * kTile < g.mi && tc * kTile < g.mi;
    if (rows_live) {
        for (int k0 = 0; k0 < g.nj; k0 += kKC) {
            for (int e = tid; e < kTile * kKC; e += 256) {
                const int rr = e / kKC, kk = e - rr * kKC;
                const int ra = tr * kTile + rr, rb = tc * kTile + rr, col = k0 + kk;
                const bool okc = col < g.nj;
                As[rr][kk] = (okc && ra < g.mi)
                                 ? f.H[static_cast<size_t>(g.r0 + ra) * f.ld + g.c0 + col]
                                 : make_float2(0.f, 0.f);
                Bs[rr][kk] = (okc && rb < g.mi)
                                 ? f.H[static_cast<size_t>(g.r0 + rb) * f.ld + g.c0 + col]
                                 : make_float2(0.f, 0.f);
            }
            __syncthreads();
            float2 acc[4];
            for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
#pragma unroll 8
            for (int kk = 0; kk < kKC; ++kk) {
                const float2 av = As[x][kk];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 bv = Bs[y0 + 8 * q][kk];
                    // a * conj(b)
                    acc[q].x = fmaf(av.x, bv.x, acc[q].x);
                    acc[q].x = fmaf(av.y, bv.y, acc[q].x);
                    acc[q].y = fmaf(av.y, bv.x, acc[q].y);
                    acc[q].y = fmaf(-av.x, bv.y, acc[q].y);
                }
            }
            for (int q = 0; q < 4; ++q) {
                accd[q].x += static_cast<double>(acc[q].x);
                accd[q].y += static_cast<double>(acc[q].y);
            }
            __syncthreads();
        }
    }
    for (int q = 0; q < 4; ++q) {
        const int y = y0 + 8 * q;
        const int gr = tr * kTile + x, gc = tc * kTile + y;
        double2 val = accd[q];
        if (gr >= g.mi || gc >= g.mi) val = make_double2(gr == gc ? 1.0 : 0.0, 0.0);
        else if (gr == gc) val.x += f.rho;
        f.A[g.base + static_cast<size_t>(gr) * S + gc] = val;
    }
}

// ---- Cholesky of the diagonal tile k (one warp per block) -------------------
__global__ void __launch_bounds__(32) potrf_diag_kernel(const FactorArgs f, int k) {
    __shared__ double2 T[kTile][kTile + 1];
    const int b = blockIdx.x;
    const BlockGeom g = geom(f, b);
    const size_t S = static_cast<size_t>(f.T) * kTile;
    double2* A = f.A + g.base + static_cast<size_t>(k) * kTile * S + static_cast<size_t>(k) * kTile;
    const int t = threadIdx.x;
    for (int c = 0; c < kTile; ++c) T[t][c] = A[static_cast<size_t>(t) * S + c];
    __syncwarp();
    for (int j = 0; j < kTile; ++j) {
        double d = T[j][j].x;
        if (!(d > 0.0) || !isfinite(d)) {
            if (t == 0) raise_status(f.status, ADMM_ENOTPD);
            d = 1.0;
        }
        const double l = sqrt(d);
        __syncwarp();
        if (t == j) T[j][j] = make_double2(l, 0.0);
        if (t > j) T[t][j] = make_double2(T[t][j].x / l, T[t][j].y / l);
        __syncwarp();
        if (t > j) {
            const double2 ltj = T[t][j];
            for (int c = j + 1; c <= t; ++c) {
                const double2 lcj = T[c][j];
                double2 v = T[t][c];
                // v -= l_tj * conj(l_cj)
                v.x -= ltj.x * lcj.x + ltj.y * lcj.y;
                v.y -= ltj.y * lcj.x - ltj.x * lcj.y;
                T[t][c] = v;
            }
        }
        __syncwarp();
    }
    for (int c = 0; c < kTile; ++c)
        A[static_cast<size_t>(t) * S + c] = c <= t ? T[t][c] : make_double2(0.0, 0.0);
}

// ---- panel: L_rk = A_rk L_kk^{-H} for r > k (one warp per tile) --------------
__global__ void __launch_bounds__(32) trsm_panel_kernel(const FactorArgs f, int k) {
    __shared__ double2 L[kTile][kTile + 1];
    __shared__ double2 X[kTile][kTile + 1];
    const int r = k + 1 + blockIdx.x;
    const int b = blockIdx.y;
    const BlockGeom g = geom(f, b);
    const size_t S = static_cast<size_t>(f.T) * kTile;
    const double2* Lkk = f.A + g.base + static_cast<size_t>(k) * kTile * S + static_cast<size_t>(k) * kTile;
    double2* Ark = f.A + g.base + static_cast<size_t>(r) * kTile * S + static_cast<size_t>(k) * kTile;
    const int t = threadIdx.x;
    for (int c = 0; c < kTile; ++c) {
        L[t][c] = Lkk[static_cast<size_t>(t) * S + c];
        X[t][c] = Ark[static_cast<size_t>(t) * S + c];
    }
    __syncwarp();
    // row t of X solves x L^H = a:  x_c = (a_c - sum_{q<c} x_q conj(L_cq)) / L_cc
    for (int c = 0; c < kTile; ++c) {
        double2 v = X[t][c];
        for (int q = 0; q < c; ++q) {
            const double2 xq = X[t][q], lcq = L[c][q];
            v.x -= xq.x * lcq.x + xq.y * lcq.y;
            v.y -= xq.y * lcq.x - xq.x * lcq.y;
        }
        const double d = L[c][c].x;
        X[t][c] = make_double2(v.x / d, v.y / d);
    }
    __syncwarp();
    for (int c = 0; c < kTile; ++c) Ark[static_cast<size_t>(t) * S + c] = X[t][c];
}

// ---- trailing update: A_rc -= L_rk L_ck^H for k < c <= r --------------------
__global__ void __launch_bounds__(256) update_kernel(const FactorArgs f, int k) {
    __shared__ double2 Lr[kTile][kTile + 1];
    __shared__ double2 Lc[kTile][kTile + 1];
    int rr, cc;
    tri_pair(blockIdx.x, rr, cc);
    const int r = k + 1 + rr, c = k + 1 + cc;
    const int b = blockIdx.y;
    const BlockGeom g = geom(f, b);
    const size_t S = static_cast<size_t>(f.T) * kTile;
    const double2* Lrk = f.A + g.base + static_cast<size_t>(r) * kTile * S + static_cast<size_t>(k) * kTile;
    const double2* Lck = f.A + g.base + static_cast<size_t>(c) * kTile * S + static_cast<size_t>(k) * kTile;
    double2* Arc = f.A + g.base + static_cast<size_t>(r) * kTile * S + static_cast<size_t>(c) * kTile;
    const int tid = threadIdx.x;
    for (int e = tid; e < kTile * kTile; e += 256) {
        const int x = e / kTile, y = e - x * kTile;
        Lr[x][y] = Lrk[static_cast<size_t>(x) * S + y];
        Lc[x][y] = Lck[static_cast<size_t>(x) * S + y];
    }
    __syncthreads();
    const int x = tid >> 3, y0 = tid & 7;
    double2 acc[4];
    for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int t = 0; t < kTile; ++t) {
        const double2 a = Lr[x][t];
#pragma unroll
        for (int q = 0; q < 4; ++q) dfma_nc(acc[q], a, Lc[y0 + 8 * q][t]);
    }
    for (int q = 0; q < 4; ++q) {
        double2* p = Arc + static_cast<size_t>(x) * S + y0 + 8 * q;
        *p = dsub(*p, acc[q]);
    }
}

// ---- W_rr = L_rr^{-1} (one warp per diagonal tile) ---------------------------
__global__ void __launch_bounds__(32) trtri_diag_kernel(const FactorArgs f) {
    __shared__ double2 L[kTile][kTile + 1];
    __shared__ double2 X[kTile][kTile + 1];
    const int r = blockIdx.x;
    const int b = blockIdx.y;
    const BlockGeom g = geom(f, b);
    const size_t S = static_cast<size_t>(f.T) * kTile;
    const size_t off = g.base + static_cast<size_t>(r) * kTile * S + static_cast<size_t>(r) * kTile;
    const int t = threadIdx.x;
    for (int c = 0; c < kTile; ++c) L[t][c] = f.A[off + static_cast<size_t>(t) * S + c];
    __syncwarp();
    // column t of X: L x = e_t
    for (int i = 0; i < kTile; ++i) {
        double2 v = make_double2(i == t ? 1.0 : 0.0, 0.0);
        if (i < t) {
            X[i][t] = make_double2(0.0, 0.0);
            continue;
        }
        for (int q = t; q < i; ++q) {
            const double2 liq = L[i][q], xq = X[q][t];
            v.x -= liq.x * xq.x - liq.y * xq.y;
            v.y -= liq.x * xq.y + liq.y * xq.x;
        }
        const double d = L[i][i].x;
        X[i][t] = make_double2(v.x / d, v.y / d);
    }
    __syncwarp();
    for (int c = 0; c < kTile; ++c) f.W[off + static_cast<size_t>(t) * S + c] = X[t][c];
}

// ---- W_rc = -W_rr sum_{q=c}^{r-1} L_rq W_qc  for r = c + d ----------------------
__global__ void __launch_bounds__(256) trtri_off_kernel(const FactorArgs f, int d) {
    __shared__ double2 P[kTile][kTile + 1];
    __shared__ double2 Q[kTile][kTile + 1];
    const int c = blockIdx.x, r = c + d;
    const int b = blockIdx.y;
    const BlockGeom g = geom(f, b);
    const size_t S = static_cast<size_t>(f.T) * kTile;
    const int tid = threadIdx.x;
    const int x = tid >> 3, y0 = tid & 7;
    double2 acc[4];
    for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int qt = c; qt < r; ++qt) {
        const double2* Lrq = f.A + g.base + static_cast<size_t>(r) * kTile * S + static_cast<size_t>(qt) * kTile;
        const double2* Wqc = f.W + g.base + static_cast<size_t>(qt) * kTile * S + static_cast<size_t>(c) * kTile;
        for (int e = tid; e < kTile * kTile; e += 256) {
            const int u = e / kTile, v = e - u * kTile;
            P[u][v] = Lrq[static_cast<size_t>(u) * S + v];
            Q[u][v] = Wqc[static_cast<size_t>(u) * S + v];
        }
        __syncthreads();
        for (int t = 0; t < kTile; ++t) {
            const double2 a = P[x][t];
#pragma unroll
            for (int q = 0; q < 4; ++q) dfma_nn(acc[q], a, Q[t][y0 + 8 * q]);
        }
        __syncthreads();
    }
    // acc holds the sum; P <- W_rr, Q <- sum, then W_rc = -W_rr * sum
    const double2* Wrr = f.W + g.base + static_cast<size_t>(r) * kTile * S + static_cast<size_t>(r) * kTile;
    for (int q = 0; q < 4; ++q) Q[x][y0 + 8 * q] = acc[q];
    for (int e = tid; e < kTile * kTile; e += 256) {
        const int u = e / kTile, v = e - u * kTile;
        P[u][v] = Wrr[static_cast<size_t>(u) * S + v];
    }
    __syncthreads();
    double2* Wrc = f.W + g.base + static_cast<size_t>(r) * kTile * S + static_cast<size_t>(c) * kTile;
    for (int q = 0; q < 4; ++q) {
        const int y = y0 + 8 * q;
        double2 o = make_double2(0.0, 0.0);
        for (int t = 0; t < kTile; ++t) dfma_nn(o, P[x][t], Q[t][y]);
        Wrc[static_cast<size_t>(x) * S + y] = make_double2(-o.x, -o.y);
    }
}

// ---- K^{-1}_{ab} = sum_{q >= a} W_qa^H W_qb  (a >= b), complex64 output ----------
__global__ void __launch_bounds__(256) kinv_kernel(const FactorArgs f) {
    __shared__ double2 P[kTile][kTile + 1];
    __shared__ double2 Q[kTile][kTile + 1];
    int ta, tb;
    tri_pair(blockIdx.x, ta, tb);
    const int b = blockIdx.y;
    const BlockGeom g = geom(f, b);
    const size_t S = static_cast<size_t>(f.T) * kTile;
    const int tid = threadIdx.x;
    const int x = tid >> 3, y0 = tid & 7;
    if (ta * kTile >= g.mi) return;
    double2 acc[4];
    for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int qt = ta; qt < f.T; ++qt) {
        const double2* Wqa = f.W + g.base + static_cast<size_t>(qt) * kTile * S + static_cast<size_t>(ta) * kTile;
        const double2* Wqb = f.W + g.base + static_cast<size_t>(qt) * kTile * S + static_cast<size_t>(tb) * kTile;
        for (int e = tid; e < kTile * kTile; e += 256) {
            const int u = e / kTile, v = e - u * kTile;
            P[u][v] = Wqa[static_cast<size_t>(u) * S + v];
            Q[u][v] = Wqb[static_cast<size_t>(u) * S + v];
        }
        __syncthreads();
        for (int t = 0; t < kTile; ++t) {
            const double2 a = P[t][x];
#pragma unroll
            for (int q = 0; q < 4; ++q) dfma_cn(acc[q], a, Q[t][y0 + 8 * q]);
        }
        __syncthreads();
    }
    const int kp = f.kinv_pitch[b];
    float2* K = f.kinv + f.kinv_off[b];
    for (int q = 0; q < 4; ++q) {
        const int gr = ta * kTile + x, gc = tb * kTile + y0 + 8 * q;
        if (gr >= g.mi || gc >= g.mi) continue;
        const float2 val = make_float2(static_cast<float>(acc[q].x), static_cast<float>(acc[q].y));
        K[static_cast<size_t>(gr) * kp + gc] = val;
        if (ta != tb) K[static_cast<size_t>(gc) * kp + gr] = make_float2(val.x, -val.y);
    }
}

}  // namespace

cudaError_t launch_gram(const FactorArgs& f, cudaStream_t s) {
    const int nb = f.M * f.N;
    const int tiles = f.T * (f.T + 1) / 2;
    gram_kernel<<<dim3(tiles, nb), 256, 0, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_cholesky_inverse(const FactorArgs& f, cudaStream_t s) {
    const int nb = f.M * f.N;
    for (int k = 0; k < f.T; ++k) {
        potrf_diag_kernel<<<nb, 32, 0, s>>>(f, k);
        const int rest = f.T - k - 1;
        if (rest > 0) {
            trsm_panel_kernel<<<dim3(rest, nb), 32, 0, s>>>(f, k);
            update_kernel<<<dim3(rest * (rest + 1) / 2, nb), 256, 0, s>>>(f, k);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    trtri_diag_kernel<<<dim3(f.T, nb), 32, 0, s>>>(f);
    for (int d = 1; d < f.T; ++d) trtri_off_kernel<<<dim3(f.T - d, nb), 256, 0, s>>>(f, d);
    kinv_kernel<<<dim3(f.T * (f.T + 1) / 2, nb), 256, 0, s>>>(f);
    return cudaGetLastError();
}

}  // namespace admm
