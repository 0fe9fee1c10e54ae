// Internal declarations shared by the host API (admm_api.cu), the iteration
// kernel (admm_iterate.cu) and the factor kernels (admm_factor.cu).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>
#include <vector>

#include "../../include/admm.h"

namespace admm {

constexpr int kConsumerWarps = 8;
constexpr int kConsumerThreads = kConsumerWarps * 32;
constexpr int kIterThreads = kConsumerThreads + 32;  // + one TMA producer warp
constexpr int kMaxBlocksPerSlab = 4;                 // column blocks one CTA slab may touch
constexpr int kMaxBlocks = 256;                      // row_blocks * col_blocks
constexpr int kTile = 32;                            // FP64 factor tile edge

// Host-side plan of the persistent iteration kernel.
struct Plan {
    int P = 0;            // CTAs
    int ld = 0;           // padded row pitch (complex elements), multiple of 32
    int wmax = 0;         // widest slab (columns, even)
    int npmax = 0;        // widest slab in column pairs
    int chunks = 0;       // per-lane 32-pair chunks (template width)
    int groups = 1;       // column groups of consumer warps per CTA (2: each takes half the slab)
    int nsub = 0;         // TMA boxes per slab row
    int wbox = 0;         // TMA box width (columns, even, <= 256)
    int R = 0;            // rows per stage (fixed by the chunk count)
    int nstages = 0;
    int stage_bytes = 0;  // bytes landed per stage (all boxes)
    int stage_stride = 0; // ring slot stride (128-byte multiple)
    int sub_bytes = 0;    // bytes per box
    int njs = 0;          // most column blocks touched by one slab
    int mimax = 0;        // tallest row block
    int kpmax = 0;        // padded pitch of the tallest factor
    // shared-memory layout (byte offsets into dynamic smem)
    int off_ring = 0, off_full = 0, off_empty = 0, off_ws = 0, off_rs = 0, off_gs = 0, off_red = 0,
        off_sigma = 0, off_misc = 0, smem = 0;
    bool aligned = false; // slabs aligned to column blocks (one block per slab)
    int red_lanes = 32;   // lanes summing the partials of one (block, row) in phase B
    bool ws_all = false;  // the whole w (m x njs) fits in shared memory
    int ws_rows = 0;      // rows of the shared w staging buffer
    int R16 = 0;          // FP16 stream: rows per stage
    int nstages16 = 0;    // FP16 stream: pipeline depth
    int stage_stride16 = 0;  // FP16 stream: ring slot size
    int ring_bytes = 0;   // shared memory of the ring (either mode's slots fit)
    int wbox16 = 0;       // FP16 stream: TMA box width (columns, multiple of 4)
    int nsub16 = 0;       // FP16 stream: boxes per slab row
    int npitch = 0;       // pair pitch of the per-pair shared buffers
    bool sigma_global = false;  // H_i^H w_i sums kept in the u buffer (wide slabs, many row blocks)
    bool red_single = false;    // one cross-warp reduction buffer instead of two
    std::vector<int> cta_beg;   // P slab starts (even)
    std::vector<int> cta_end;   // P slab ends (even)
    std::vector<int> cta_own0;  // P first owned column
    std::vector<int> cta_own1;  // P one past the last owned column
    std::vector<int> cta_jlo;   // P
    std::vector<int> cta_nj;    // P
    std::vector<int> j_cta_lo;  // N
    std::vector<int> j_cta_hi;  // N
    std::vector<int> solve_lo;  // P+1 split of the N*m factor-apply rows
};

// Returns ADMM_OK, ADMM_EINVAL or ADMM_EUNSUPPORTED; fills `plan`.  Multi-problem
// launches pass force_chunks (their shared instance) and max_groups = 1.
int make_plan(int64_t m, int64_t n, int M, int N, const std::vector<int>& row_off,
              const std::vector<int>& col_off, int num_sms, int smem_limit, Plan& plan,
              const char** why, int force_chunks = 0, int max_groups = 2);

void balanced_offsets(int64_t total, int parts, std::vector<int>& off);

// Message returned by admm_last_error(NULL) (calls that have no handle).
void set_handle_free_error(const char* msg);

// Device buffers of a single-scene handle that the batched path reuses: the
// FP16 copy of H, its group scales, the factors of the matrix it encodes and
// the block tables.  ADMM_EINVAL until the FP16 copy exists.
struct HandleView {
    const float2* H;
    const void* H16;
    const float* scales;
    const float2* kinv16;
    const long long* kinv_off;
    const int* kinv_pitch;
    const int* row_off;
    const int* col_off;
    int ld;
    int* status;
    const float2* kinv;
};
int view_handle(const admm_t* h, HandleView* v);

// SIMT products of the single-scene reverse sweep (admm_backward.cu): for block
// p = i N + j of the complex64 (f16 = false) or FP16 (group scales) H,
//   rows:   out[p][r] = sum_c H[r0_i + r][c0_j + c] x[p][c]              (x pitch xp)
//   cols:   out[p][c] = sum_r conj(H[r0_i + r][c0_j + c]) s_r y[p][r]    (s_r: FP16 row scale or 1)
//   factor: out[p][r] = sum_t Kinv_p[r][t] y[p][t]
struct ProdArgs {
    int M, N, ld, mimax, njmax, mpitch, npitch;
    const int* row_off;
    const int* col_off;
    const float2* H;
    const void* H16;
    const float* scales;
    const float2* kinv;
    const long long* kinv_off;
    const int* kinv_pitch;
};
cudaError_t launch_bw_rows(const ProdArgs& a, bool f16, const float2* x, float2* out, cudaStream_t s);
cudaError_t launch_bw_cols(const ProdArgs& a, bool f16, const float2* y, float2* out, cudaStream_t s);
cudaError_t launch_bw_factor(const ProdArgs& a, const float2* y, float2* out, cudaStream_t s);

// Arguments of the persistent iteration kernel (passed by value).
struct IterArgs {
    int m, n, ld, M, N, P;
    int R, nstages, stage_bytes, stage_stride, sub_bytes, nsub, wbox;
    int elem_bytes;       // bytes of one complex element of the streamed H (8 complex64, 4 FP16)
    int npitch;           // pair pitch of the per-pair shared buffers (red, sigma)
    int mimax, kpmax;
    int off_ring, off_full, off_empty, off_ws, off_rs, off_gs, off_red, off_sigma, off_misc;
    int red_lanes, ws_all, ws_rows, sigma_global, red_single;
    int pgroups;          // column groups per CTA (1 or 2): partial products per row = P * pgroups
    int chunks;           // the plan's chunk count (the kernel instance of a one-launch group)
    float rho, kappa, inv_M;
    double rho_d;
    const int* row_off;
    const int* col_off;
    const int* cta_col;   // slab starts
    const int* cta_end;   // slab ends
    const int* cta_own0;
    const int* cta_own1;
    const int* cta_jlo;
    const int* cta_nj;
    const int* j_cta_lo;
    const int* j_cta_hi;
    const int* solve_lo;
    float2* v;
    float2* s;
    float2* u;
    const float2* g;
    float2* ghat;         // two N x m buffers; iteration k reads buffer k & 1, writes the other
    float2* gt;           // N x m estimated-data-corrected g of the current iteration
    float2* r;            // N x m residuals r_b
    float2* w;
    float2* part;
    const float2* kinv;
    const long long* kinv_off;
    const int* kinv_pitch;
    double* res_part;
    double* hist;
    long long* k_done;
    unsigned* bar;
    int* status;
    int* stop_flag;
    long long k0;
    int hist_cap;
    int iters;
    int check_stop;
    double eps_abs, eps_rel;
    long long timeout_ns;
    int bar_extra;
    const float* scales;  // FP16 stream: one scale per 64-row group (null for complex64 H)
    long long* trace;     // optional phase timestamps (2 CTAs x trace_iters x 8)
    int trace_iters;
    int keep_stages;      // last stages of each pass keep the normal L2 priority (0 = no L2 hints)
    int prefetch_stages;  // stages after a pass's L2-resident head prefetched into L2 before it starts
    // recording for the adjoint (null when off): iteration k0 + it writes its
    // shrinkage arguments a (ld) and factor solutions w ([i N + j][rec_pitch])
    // into slot k0 + it while that is < rec_cap
    float2* rec_a;
    float2* rec_w;
    int rec_cap;
    int rec_pitch;
    int pending_prev;     // the previous launch's last residual record is still to be summed
    // sharded iteration (null otherwise): the epilogue writes u and, per column,
    // the sum over this handle's replicas of u_i + s_i here, and leaves v and s
    float2* shard_sum;
};

// The problems of a multi-problem launch, passed as kernel parameters (so the
// tensor maps and arguments sit in the parameter space, as for one problem).
constexpr int kMaxGroupWave = 48;
struct GroupParams {
    CUtensorMap tmap[kMaxGroupWave];
    IterArgs a[kMaxGroupWave];
    int count;
};

// Cooperative launch of `ctas` CTAs running several problems (the kernel
// instance with `chunks` chunks, complex64 or FP16 H, `smem` bytes of dynamic
// shared memory for the largest problem layout); CTA b runs local CTA
// cta_local[b] of problem cta_prob[b].
cudaError_t launch_group(const GroupParams& gp, const int* cta_prob, const int* cta_local, int ctas, int chunks,
                         bool f16, int smem, cudaStream_t stream);
// Every wave of a group in one cooperative launch of `ctas` CTAs: cta_map holds
// waves x ctas problem indices into gp (-1 idle) and then waves x ctas local
// CTA indices.
cudaError_t launch_waves(const GroupParams& gp, const int* cta_map, int waves, int ctas, int chunks, bool f16,
                         int smem, cudaStream_t stream);
// the kernel of launch_waves, and its shared-memory opt-in (outside any capture)
void* waves_kernel(int chunks, bool f16);
cudaError_t prepare_waves(int chunks, bool f16, int smem);
bool group_stage_geometry_ok(const IterArgs& a, int chunks, bool f16);

// Sum the per-CTA residual partials of iteration kabs into the history ring.
cudaError_t launch_finalize(const IterArgs& a, long long kabs, cudaStream_t stream);

// Rows of H per pipeline stage of the kernel instance with `chunks` chunks
// (complex64 or FP16 storage).
int rows_per_stage(int chunks, bool f16 = false);

// Launch the persistent cooperative iteration kernel for `a.iters` iterations.
// `f16` selects the instance that streams FP16 H (4-byte complex elements).
cudaError_t launch_iterate(const CUtensorMap& tmap, const IterArgs& a, int chunks, int smem,
                           cudaStream_t stream, bool f16 = false);
// Opt the kernel instances into `smem` bytes of dynamic shared memory.
cudaError_t prepare_iterate(int chunks, int smem, int groups = 1);
int max_coresident_iterate(int chunks, int smem, int* per_sm, int groups = 1);

// ---- setup kernels (admm_factor.cu) ------------------------------------------

struct FactorArgs {
    int m, ld, M, N;
    int T;                   // factor tiles per edge (ceil(mimax / 32))
    const int* row_off;
    const int* col_off;
    const float2* H;         // packed H (m x ld)
    double2* A;              // per block (T*32)^2, FP64: K_b, then L_b
    double2* W;              // per block (T*32)^2, FP64: L_b^{-1}
    float2* kinv;            // packed complex64 K_b^{-1}
    const long long* kinv_off;
    const int* kinv_pitch;
    double rho;
    int* status;
};

cudaError_t launch_gram(const FactorArgs& f, cudaStream_t s);
cudaError_t launch_cholesky_inverse(const FactorArgs& f, cudaStream_t s);

// ---- direct branch (admm_direct.cu) -------------------------------------------
// Blocks with m_b >= n_b solved with the n_b x n_b factor of Section III-B,
// L_b = (H_b^H H_b + rho I)^{-1}:
//     q_b = H_b^H gt_b + rho z_b      (column pass over H_b; for one column
//                                      block gt_b = g_i and H_b^H g_i is cached)
//     u_b = L_b q_b                   (factor pass)
//     v, s update                     (the last CTA of every column chunk)
//     ghat_b = H_b u_b                (row pass; only with col_blocks > 1)
// Every cross-CTA step is a last-arriver reduction on an atomic counter: no
// CTA waits for another, and a launch sequence is stable under graph capture
// (the estimated-data slot is taken from the device iteration count).

constexpr int kDirColThreads = 256;  // column pass: eight warps splitting the rows
constexpr int kDirColPairs = 128;    // column pairs per column-pass CTA (four per lane)
constexpr int kDirColRows = 4096;    // most rows per column-pass split (gt_b staged in shared memory)
constexpr int kDirFacThreads = 256;  // factor pass: eight warps, up to four rows at a time each
constexpr int kDirChunk = 16;        // entries of u_b per update chunk
constexpr int kDirRowThreads = 256;  // row pass: eight warps, up to eight rows at a time each
constexpr int kDirBulkWarps = 8;     // streamed factor pass: consumer warps (an eighth of the columns each)
constexpr int kDirDeferred = 32;     // update chunks a streamed factor CTA counts in shared memory
constexpr int kDirBulkMinCols = 1024;  // blocks the streamed factor pass takes: 1024 to 2048 columns
constexpr int kDirBulkMaxCols = 2048;  // (8 to 16 KB rows; narrower factors are latency-bound and
                                       // measured faster with the plain-load pass)
constexpr int kDirMaxCols = 12288;   // widest block of the direct branch (u_b staged in shared memory)
constexpr int kDirTile = 64;         // Hermitian factor pass: 64 x 64 tiles of each factor's lower triangle
constexpr int kDirHermMinCols = 256; // blocks this wide and wider keep their factors as such tiles
constexpr int kDirHermAutoCols = 1024;  // ... and use them by default from this width on (narrower
                                        // blocks have too few tiles to fill the GPU)
constexpr int kHermWarps = 8;        // tile pass: consumer warps per CTA (and a producer), one CTA per SM
constexpr int kHermSlots = 24;       // slots of the CTA's ring of tile pieces
constexpr int kHermPieceRows = 16;   // tile rows per piece (8 KB)
constexpr int kDirHermMaxRowBlocks = 512;   // the tile pass's update keeps 3 M x 16 values in shared memory

struct DirectArgs {
    int m, n, ld, M, N, P;
    int npitch;               // complex entries per block vector (Q, C, partial rows); multiple of 4
    int njmax, mimax;
    const int* row_off;
    const int* col_off;
    const float2* H;          // m x ld
    const float2* g;          // m
    float2* v;                // ld
    float2* s;                // M x ld
    float2* u;                // M x ld: u_j^i at u + i * ld + col_off[j]
    float2* ghat;             // 2 x N x m, slot (iteration count) & 1
    const float2* L;          // factors, block p = i * N + j at L + L_off[p], row pitch L_pitch[p]
    const long long* L_off;
    const int* L_pitch;
    float2* C;                // P x npitch: H_i^H g_i (one column block)
    float2* Q;                // q_b, P x npitch; with one column block two slots by
                              // iteration parity (the update writes the next q)
    float2* part;             // S x P x npitch: column-pass partial sums
    int S;                    // row splits of the column pass
    int ccn;                  // column tiles per block in the column pass
    int ctas;                 // CTAs of the factor and row passes (two per SM)
    int frows;                // factor rows of all blocks (sum of n_j over the blocks)
    int hrows;                // rows of H of all blocks (sum of m_i over the blocks)
    int fac_stream;           // factor pass: 1 = bulk copies into a shared-memory ring
    int fac_ctas;             // CTAs of the streamed factor pass
    int fac_ns;               // its ring stages
    int fac_stage;            // its stage bytes (four factor rows of the widest block)
    long long timeout_ns;     // bound of every wait of the streamed factor pass
    int fitems;               // work items of the streamed factor pass (update chunks of all blocks)
    const int* I_off;         // P + 1: first item of block p
    const int* F_off;         // P + 1: first factor row of block p in the concatenation
    const int* R_off;         // P + 1: first H row of block p in the concatenation
    unsigned* cnt_cols;       // P x ccn
    unsigned* cnt_upd;        // nchunks
    unsigned* cnt_glob;       // [0] update chunks finished, [1] row-pass CTAs finished,
                              // [2] next streamed factor item, [3] CTAs out of items
    const int* chunk_off;     // N + 1: first update chunk of each column block
    int nchunks;
    double* res_chunk;        // nchunks x 5
    double* hist;
    int hist_cap;
    long long* k_done;
    int* status;
    int* stop_flag;           // set once the stopping test passed (with check_stop)
    int* stop_pending;        // set by the update, turned into stop_flag after the row pass
    // Hermitian factor pass: the lower triangle of every L_b in kDirTile x kDirTile
    // tiles (diagonal tiles whole).  Block p's tile (I, J), J <= I, has the
    // index T_off[p] + I (I + 1) / 2 + J; Lt holds the tiles in the order of the
    // pass, T_seq[s] = {index, p, I, J} of the tile at position s.
    int fac_herm;
    const float2* Lt;         // ntiles x kDirTile x kDirTile, row-major tiles
    const int4* T_seq;        // ntiles
    const long long* T_off;   // P + 1
    float2* RP;               // ntiles x kDirTile, by index: row sums L_IJ q_J
    float2* CP;               // ntiles x kDirTile, by index: column sums L_IJ^H q_I (J < I)
    int ntiles;
    int herm_ctas;            // CTAs of the tile pass (one per SM)
    // One column block: the record of iteration k is written by the next tile
    // pass (or by the record kernel that ends a launch sequence), not by the
    // update's last CTA.  dctl[0]: iterations updated (written by the update,
    // read by the tile pass), dctl[1]: the iteration the tile pass summed
    // (written by the tile pass, read by the update), dctl[2]: a record is
    // pending.  No kernel reads a counter its own grid writes.
    int defer_record;
    long long* dctl;
    int check_stop;
    double eps_abs, eps_rel;
    float rho, kappa, inv_M;
    double rho_d;
};

// column pass: mode 0 writes Q = H^H gt + rho z, mode 1 writes C = H^H g (no z)
cudaError_t launch_dir_cols(const DirectArgs& a, int mode, cudaStream_t s);
// Q[slot of the device iteration count] = C + rho z (one column block)
cudaError_t launch_dir_q(const DirectArgs& a, cudaStream_t s);
cudaError_t launch_dir_factor(const DirectArgs& a, cudaStream_t s);
// the pending record of the last iteration (defer_record), one warp
cudaError_t launch_dir_record(const DirectArgs& a, cudaStream_t s);
cudaError_t launch_dir_rows(const DirectArgs& a, cudaStream_t s);
// the tiles of the tile pass from the full factors (the parts of a tile past n_j zero)
cudaError_t launch_pack_herm(const float2* L, const long long* L_off, const int* L_pitch, const int* col_off,
                             int N, const int4* T_seq, long long ntiles, float2* Lt, cudaStream_t s);
// the tile pass: its shared memory, and its resident CTAs per SM (after opting
// in to that shared memory)
size_t herm_smem_bytes();
cudaError_t herm_per_sm(int* per_sm);
cudaError_t prepare_direct(int smem_optin);
// shared memory of the streamed factor pass with `ns` stages of `stage` bytes,
// and its resident CTAs per SM with `smem` bytes
size_t stream_smem(int ns, int stage);
cudaError_t direct_stream_per_sm(int smem, int* per_sm);
// HT (n x ldT) = H^H of the m x ld matrix H
cudaError_t launch_conj_transpose(const float2* H, int64_t m, int64_t n, int64_t ld, float2* HT, int64_t ldT,
                                  cudaStream_t s);

// ---- small kernels (admm_misc.cu) ---------------------------------------------

cudaError_t launch_pack_c128(const double2* src, int64_t m, int64_t n, float2* dst, int64_t ld,
                             cudaStream_t s);
cudaError_t launch_finite_check(const float2* x, int64_t count, int* flag, cudaStream_t s);
// sharded iteration: out[r] = sum_q ghat[q * m + r] over the N column blocks;
// g[r] = g0[r] - t_glob[r] + t_loc[r];  v = S_kappa(sum / M_total), s_i += u_i - v
// for the M local replicas, with the FP64 residual partials (sum ||u_i - v||^2,
// ||v - v_old||^2, sum ||u_i||^2, ||v||^2, sum ||s_i||^2) added into rec[5]
cudaError_t launch_shard_ghat_sum(const float2* ghat, int N, int64_t m, float2* out, cudaStream_t s);
cudaError_t launch_shard_geff(const float2* g0, const float2* t_glob, const float2* t_loc, int64_t m, float2* g,
                              cudaStream_t s);
cudaError_t launch_shard_vstep(float2* v, float2* s, const float2* u, const float2* sum, int64_t n, int64_t ld, int M,
                               float inv_Mtot, float kappa, double* rec, cudaStream_t st);
cudaError_t launch_scale(float2* x, int64_t count, float alpha, cudaStream_t s);
// FP16 copy of H with one power-of-two scale per 64-row group (and, when Hdeq
// is not null, the dequantised matrix in FP32); gmax_bits holds ceil(m/64) words.
cudaError_t launch_quantize_f16(const float2* H, int64_t m, int64_t ld, unsigned* gmax_bits,
                                void* H16, float* scales, float2* Hdeq, cudaStream_t s);
cudaError_t launch_dequantize_f16(const void* H16, int64_t m, int64_t ld, const float* scales,
                                  float2* Hdeq, cudaStream_t s);

}  // namespace admm
