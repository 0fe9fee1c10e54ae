// Internal interface of the batched shared-H path (admm_batch_kernels.cu,
// admm_batch_host.cu).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "admm_internal.h"

namespace admm {
namespace batch {

constexpr int kGemmThreads = 192;   // warp 0 TMA, warp 1 TMEM + MMA, warps 2-5 epilogue
constexpr int kGemmSmem = 4 * (128 * 64 * 2 + 256 * 64 * 2) + 1024 + 256;
constexpr int kTileRows = 128;      // GEMM tile rows (A rows)
constexpr int kTileCols = 256;      // GEMM tile columns (4 packed columns per scene: 64 scenes)
constexpr int kTileK = 64;          // FP16 elements of K per pipeline stage

// One grouped GEMM launch: problem p multiplies rows [a_y0[p], +rows[p]) of A
// (K offset a_x0[p], 3-D coordinate a_z[p]) with the packed B operand of
// problem p, and writes complex results out[split][p][b][row] scaled by
// row_scale[(rs_off[p] + row) >> rs_shift] * col_scale[p * B + b].
struct GemmArgs {
    int nprob, mtiles, ntiles, splits, kb_per_split;
    int ctas;                // persistent CTAs (one per SM)
    const int* a_x0;
    const int* a_y0;
    const int* a_z;
    const int* rows;
    const int* kb_prob;      // K blocks of 64 per problem
    const float* row_scale;  // may be null
    const int* rs_off;
    int rs_shift;
    const float* col_scale;
    float2* out;
    int out_pitch;
    int B;
    int* status;
    long long timeout_ns;
};

// Packing of complex vectors into the B operand of the GEMM: for problem p and
// scene b the vector x - y (y optional) of len[p] entries starting at
// x_off[p] + b * x_bs (and y_off[p] + b * y_bs), optionally times
// rs[(rs_row[p] + e) >> 6], is scaled by a power of two per (p, b) and split
// into FP16 hi + lo columns.
struct PackArgs {
    const float2* x;
    const long long* x_off;
    long long x_bs;
    const float2* y;
    const long long* y_off;
    long long y_bs;
    const float* rs;
    const int* rs_row;
    const int* len;
    int B;
    void* dst;             // [p][4B][row2] __half2
    int row2;              // __half2 per packed row (K / 2)
    int adjoint;           // 0: (re,-im),(im,re) form; 1: (re,im),(im,-re) form
    int second;            // __half2 offset of the (hi, hi, 0, 0) copy, or -1
    float* scale;          // [p * B + b]
    const unsigned* vmax;  // when set: [p * B + b] largest |component| of the vector (float
                           // bits), known beforehand, so packing takes one pass
};

// Elementwise steps of the batched iteration.
struct StepArgs {
    int m, n, M, N, P, B, splits, mpitch, npitch;
    const int* row_off;
    const int* col_off;
    float2* V;       // B x n
    float2* S;       // M x B x n
    const float2* G; // B x m
    float2* Gt;      // N x B x m
    float2* Ghat;    // N x B x m
    float2* R;       // P x B x mpitch
    const float2* Ppart;  // splits x P x B x mpitch
    const float2* W; // P x B x mpitch
    const float2* Sig;    // P x B x npitch
    const float* kappa;   // per scene
    float rho, inv_M;
    double* res;     // 2 per scene: ||r_p||^2, ||r_d||^2 / (rho^2 M)
    unsigned* zmax;  // [p * B + b] largest |component| of the next z_j^i (float bits)
    const int* upd_tile_off;  // N + 1: first update tile of each column block
    int upd_tiles;            // update tiles (kUpdCols columns, inside one block)
    // recording for the adjoint (null when off): iteration k writes its
    // shrinkage arguments a (B x n) and factor solutions w (P x B x mpitch)
    // into slot *rec_k, while *rec_k < rec_cap
    float2* rec_a;
    float2* rec_w;
    int* rec_k;
    int rec_cap;
    // reverse sweep
    float2* Vb;          // B x n: adjoint of v
    float2* Sb;          // M x B x n: adjoint of s
    float2* Ghb;         // N x B x m: adjoint of the estimated data
    float2* dG;          // B x m: gradient of g
    double* kbar;        // per scene: adjoint of kappa
    double* rbar;        // per scene: adjoint of rho (direct terms)
    int bk;              // iteration whose records the sweep reads
};

constexpr int kUpdCols = 1024;   // columns per update CTA

cudaError_t prepare_gemm();
cudaError_t launch_gemm(const CUtensorMap& A, const CUtensorMap& B, const GemmArgs& a, cudaStream_t s);
cudaError_t launch_pack(const PackArgs& a, int nprob, cudaStream_t s);
cudaError_t launch_residual_r(const StepArgs& a, cudaStream_t s);
cudaError_t launch_ghat(const StepArgs& a, cudaStream_t s);
cudaError_t launch_update(const StepArgs& a, cudaStream_t s);
cudaError_t launch_gtilde(const StepArgs& a, cudaStream_t s);
cudaError_t launch_rec_advance(const StepArgs& a, cudaStream_t s);
cudaError_t launch_bw_soft(const StepArgs& a, cudaStream_t s);
cudaError_t launch_bw_wbar(const StepArgs& a, cudaStream_t s);
cudaError_t launch_bw_rbar(const StepArgs& a, cudaStream_t s);
cudaError_t launch_bw_state(const StepArgs& a, cudaStream_t s);
cudaError_t launch_bw_gtilde(const StepArgs& a, cudaStream_t s);
cudaError_t launch_sum_blocks(const float2* part, int splits, int P, int B, int pitch, const int* off, int nblk,
                              int N, int by_rows, float2* out, int out_len, cudaStream_t s);
cudaError_t launch_transpose_h16(const void* H16, int m, int ld, void* HT, cudaStream_t s);
cudaError_t launch_pack_kinv(const float2* kinv, const long long* koff, const int* kpitch, const int* row_off,
                             int P, int N, int mimax, int kk, void* Kpack, float* kscale, cudaStream_t s);

}  // namespace batch
}  // namespace admm
