// Host side of libadmm.so: argument checks, the block partitioner, the launch
// plan of the persistent iteration kernel, device memory, the factor cache
// and the C ABI declared in include/admm.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "admm_batch.h"
#include "admm_internal.h"

using admm::Plan;

namespace {

thread_local std::string g_setup_error;

int round_up(int64_t x, int64_t q) { return static_cast<int>((x + q - 1) / q * q); }

}  // namespace

// device buffers and launch geometry of the direct form
struct DirectState {
    float2 *C = nullptr, *Q = nullptr, *part = nullptr;
    unsigned* cnt = nullptr;       // column tiles, update chunks, two global counters
    int* ints = nullptr;           // chunk_off (N + 1), L_pitch (P), F_off, R_off, I_off (P + 1 each)
    long long* L_off = nullptr;    // P
    double* res_chunk = nullptr;
    int* stop_pending = nullptr;
    int npitch = 0, njmax = 0, S = 1, ccn = 1, ctas = 1, frows = 0, hrows = 0, nchunks = 0, ncnt = 0;
    int fac_stream = 0, fac_ctas = 0, fac_ns = 0, fac_stage = 0, fitems = 0;   // streamed factor pass
    // the tile pass over the lower triangles (blocks of kDirHermMinCols columns and more)
    int herm = 0;                  // the tiles exist
    int pass = 0;                  // ADMM_OPT_DIR_FACTOR_PASS: 0 auto, 1 full rows, 2 tiles
    float2 *Lt = nullptr, *RP = nullptr, *CP = nullptr;
    long long* T_off = nullptr;    // P + 1
    int4* T_seq = nullptr;         // ntiles: the pass order, {index, p, I, J}
    long long* dctl = nullptr;     // 4: the deferred record's counters (one column block)
    long long ntiles = 0;
    int herm_ctas = 0;
    int64_t bytes = 0;
    bool c_valid = false;          // C = H_i^H g_i matches g (one column block)
    bool q_valid = false;          // Q of the current iteration matches C, v, s and rho
    cudaStream_t cap = nullptr;    // capture stream of the iteration graphs
    cudaGraphExec_t g1 = nullptr, g16 = nullptr;   // one and sixteen iterations
    double key[7] = {0, 0, 0, 0, 0, 0, 0};
    const void* key_hist = nullptr;
    bool key_set = false;
};

struct admm_problem {
    int device = 0;
    int num_sms = 0;
    int smem_optin = 0;
    int64_t m = 0, n = 0;
    int M = 1, N = 1;
    double lambda = 0.0, rho = 1.0;
    std::vector<int> row_off, col_off;
    Plan plan;
    // device memory owned by the handle
    float2 *H = nullptr, *g = nullptr, *v = nullptr, *s = nullptr, *u = nullptr;
    float2 *ghat = nullptr, *gt = nullptr, *r = nullptr, *w = nullptr, *part = nullptr;  // ghat: 2 x N x m
    float2* kinv = nullptr;
    long long* kinv_off_d = nullptr;
    int* ints_d = nullptr;  // all int tables in one allocation
    int *row_off_d = nullptr, *col_off_d = nullptr, *cta_col_d = nullptr, *cta_end_d = nullptr,
        *cta_own0_d = nullptr, *cta_own1_d = nullptr, *cta_jlo_d = nullptr,
        *cta_nj_d = nullptr, *j_cta_lo_d = nullptr, *j_cta_hi_d = nullptr, *solve_lo_d = nullptr,
        *kinv_pitch_d = nullptr;
    double *res_part = nullptr, *hist = nullptr;
    long long* k_done = nullptr;
    unsigned* bar = nullptr;
    int* status = nullptr;
    int* stop_flag = nullptr;
    CUtensorMap tmap;
    // FP16 copy of H (ADMM_OPT_H_FP16): one complex element in 4 bytes, a
    // power-of-two scale per 64-row group, and the factors of the matrix it encodes
    void* H16 = nullptr;
    float* scales = nullptr;
    unsigned* gmax = nullptr;
    float2* kinv16 = nullptr;
    CUtensorMap tmap16;
    int use_f16 = 0;     // the iteration kernel streams H16
    // recording of the forward for admm_backward, and the reverse-sweep buffers
    float2 *rec_a = nullptr, *rec_w = nullptr;
    int rec_cap = 0, rec_pitch = 0, rec_f16 = 0;
    bool rec_valid = false;   // every iteration since the reset was recorded, inputs unchanged
    float2 *bVb = nullptr, *bSb = nullptr, *bGhb = nullptr, *bGt = nullptr, *bdG = nullptr, *bSig = nullptr,
           *bP = nullptr, *bR = nullptr, *bW = nullptr;
    double *bkbar = nullptr, *brbar = nullptr;
    float* bkappa = nullptr;
    int* bupd = nullptr;
    int bupd_tiles = 0, bnpitch = 0;
    std::vector<long long> kinv_off;
    std::vector<int> kinv_pitch;
    int64_t kinv_elems = 0;
    int64_t state_bytes = 0;
    long long timeout_ns = 5000000000LL;
    int hist_cap = 4096;
    int bar_extra = 0;
    long long* trace = nullptr;  // phase timestamps, 2 x trace_iters x 8
    int trace_iters = 0;
    int64_t k = 0;       // iterations completed (host mirror)
    int pending = 0;     // the last launch's final residual record has not been summed yet
    int64_t l2_keep_bytes = 52LL << 20;  // H bytes per pass kept for the reversed next pass
    int64_t l2_prefetch_bytes = 0;       // H bytes prefetched into L2 ahead of each pass
    int form = ADMM_FORM_LEMMA;          // factor form of every block
    DirectState dir;
    int broken = 0;      // sticky error that blocks further iterations
    double gram_ms = 0.0, factor_ms = 0.0;
    // sharded iteration (admm_shard_*): replicas of all ranks, the data vector
    // as given, the exchanged sums and the residual partials
    int sh_Mtot = 0;     // 0: not sharded
    float2 *sh_g0 = nullptr, *sh_tloc = nullptr, *sh_tglob = nullptr, *sh_sum = nullptr;
    double* sh_rec = nullptr;
    std::string err;
};

namespace {

int fail(admm_t* h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_setup_error = buf;
    return code;
}

int cuda_fail(admm_t* h, cudaError_t e, const char* what) {
    if (h) h->broken = 1;
    return fail(h, ADMM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(h, call)                                         \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

void free_all(admm_t* h) {
    void* ptrs[] = {h->H, h->g, h->v, h->s, h->u, h->ghat, h->gt, h->r, h->w, h->part, h->kinv,
                    h->kinv_off_d, h->ints_d, h->res_part, h->hist, h->k_done, h->bar, h->status,
                    h->stop_flag, h->trace, h->H16, h->scales, h->gmax, h->kinv16, h->rec_a, h->rec_w,
                    h->bVb, h->bSb, h->bGhb, h->bGt, h->bdG, h->bSig, h->bP, h->bR, h->bW, h->bkbar,
                    h->brbar, h->bkappa, h->bupd, h->sh_g0, h->sh_tloc, h->sh_tglob, h->sh_sum, h->sh_rec};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    DirectState& d = h->dir;
    void* dptrs[] = {d.C, d.Q, d.part, d.cnt, d.ints, d.L_off, d.res_chunk, d.stop_pending,
                     d.Lt, d.RP, d.CP, d.T_off, d.T_seq, d.dctl};
    for (void* p : dptrs)
        if (p) cudaFree(p);
    if (d.g1) cudaGraphExecDestroy(d.g1);
    if (d.g16) cudaGraphExecDestroy(d.g16);
    if (d.cap) cudaStreamDestroy(d.cap);
}

}  // namespace

// ---------------------------------------------------------------------------
// partitioner and plan (host only)
// ---------------------------------------------------------------------------

namespace admm {

void set_handle_free_error(const char* msg) { g_setup_error = msg ? msg : ""; }

void balanced_offsets(int64_t total, int parts, std::vector<int>& off) {
    off.assign(parts + 1, 0);
    const int64_t base = total / parts, extra = total % parts;
    int64_t pos = 0;
    for (int p = 0; p < parts; ++p) {
        off[p] = static_cast<int>(pos);
        pos += base + (p < extra ? 1 : 0);
    }
    off[parts] = static_cast<int>(pos);
}

int make_plan(int64_t m, int64_t n, int M, int N, const std::vector<int>& row_off,
              const std::vector<int>& col_off, int num_sms, int smem_limit, Plan& pl,
              const char** why, int force_chunks, int max_groups) {
    *why = "";
    if (num_sms < 1 || smem_limit < 16384) {
        *why = "bad device limits";
        return ADMM_EINVAL;
    }
    pl = Plan();
    pl.ld = round_up(n, 32);
    const int ld = pl.ld;
    const int P0 = static_cast<int>(std::min<int64_t>(num_sms, std::max<int64_t>(1, ld / 64)));
    // column range of block j with the padding columns given to the last block
    auto blk_lo = [&](int j) { return col_off[j]; };
    auto blk_hi = [&](int j) { return j == N - 1 ? ld : col_off[j + 1]; };
    pl.aligned = N <= P0;
    if (pl.aligned) {
        // CTAs per column block in proportion to its width (largest remainders),
        // at least one each and never more than the block's 16-byte pairs
        std::vector<int> cnt(N, 1), pairs(N);
        std::vector<double> frac(N);
        int used = 0;
        for (int j = 0; j < N; ++j) {
            const int a = blk_lo(j) & ~1, b = (blk_hi(j) + 1) & ~1;
            pairs[j] = (b - a) / 2;
            const double quota = static_cast<double>(P0) * (blk_hi(j) - blk_lo(j)) / ld;
            cnt[j] = std::max(1, std::min(pairs[j], static_cast<int>(std::floor(quota))));
            frac[j] = quota - std::floor(quota);
            used += cnt[j];
        }
        while (used < P0) {
            int best = -1;
            for (int j = 0; j < N; ++j)
                if (cnt[j] < pairs[j] && (best < 0 || frac[j] > frac[best])) best = j;
            if (best < 0) break;
            ++cnt[best];
            frac[best] -= 1.0;
            ++used;
        }
        while (used > P0) {
            int best = -1;
            for (int j = 0; j < N; ++j)
                if (cnt[j] > 1 && (best < 0 || cnt[j] > cnt[best])) best = j;
            --cnt[best];
            --used;
        }
        pl.P = used;
        for (int j = 0; j < N; ++j) {
            const int a = blk_lo(j) & ~1;
            std::vector<int> off;
            balanced_offsets(pairs[j], cnt[j], off);
            for (int q = 0; q < cnt[j]; ++q) {
                const int beg = a + 2 * off[q], end = a + 2 * off[q + 1];
                pl.cta_beg.push_back(beg);
                pl.cta_end.push_back(end);
                pl.cta_own0.push_back(q == 0 ? blk_lo(j) : beg);
                pl.cta_own1.push_back(q == cnt[j] - 1 ? blk_hi(j) : end);
                pl.cta_jlo.push_back(j);
                pl.cta_nj.push_back(1);
            }
        }
    } else {
        // more column blocks than CTAs: balanced slabs, each meeting several blocks
        pl.P = P0;
        std::vector<int> poff;
        balanced_offsets(ld / 2, pl.P, poff);
        auto block_of_col = [&](int c) {
            int j = static_cast<int>(std::upper_bound(col_off.begin(), col_off.end(), c) - col_off.begin()) - 1;
            return std::min(std::max(j, 0), N - 1);
        };
        for (int c = 0; c < pl.P; ++c) {
            const int beg = 2 * poff[c], end = 2 * poff[c + 1];
            const int jlo = block_of_col(beg), jhi = block_of_col(end - 1);
            pl.cta_beg.push_back(beg);
            pl.cta_end.push_back(end);
            pl.cta_own0.push_back(beg);
            pl.cta_own1.push_back(end);
            pl.cta_jlo.push_back(jlo);
            pl.cta_nj.push_back(jhi - jlo + 1);
        }
    }
    pl.j_cta_lo.assign(N, pl.P);
    pl.j_cta_hi.assign(N, -1);
    pl.njs = 1;
    pl.wmax = 0;
    for (int c = 0; c < pl.P; ++c) {
        pl.wmax = std::max(pl.wmax, pl.cta_end[c] - pl.cta_beg[c]);
        pl.njs = std::max(pl.njs, pl.cta_nj[c]);
        for (int j = pl.cta_jlo[c]; j < pl.cta_jlo[c] + pl.cta_nj[c]; ++j) {
            // a CTA contributes to block j only through columns it owns
            if (std::max(pl.cta_own0[c], blk_lo(j)) >= std::min(pl.cta_own1[c], blk_hi(j))) continue;
            pl.j_cta_lo[j] = std::min(pl.j_cta_lo[j], c);
            pl.j_cta_hi[j] = std::max(pl.j_cta_hi[j], c);
        }
    }
    if (pl.njs > kMaxBlocksPerSlab) {
        *why = "a CTA column slab would touch more than 4 column blocks (column blocks too narrow)";
        return ADMM_EUNSUPPORTED;
    }
    // slabs of more than 256 pairs: two column groups of consumer warps, each
    // with half the slab (8 chunks per lane instead of 16); not in
    // multi-problem launches, which share one single-group kernel instance
    pl.npmax = pl.wmax / 2;
    pl.groups = (max_groups >= 2 && pl.npmax > 256) ? 2 : 1;
    int most = 1;
    for (int j = 0; j < N; ++j) {
        if (pl.j_cta_hi[j] < pl.j_cta_lo[j]) {
            *why = "internal: column block without a slab";
            return ADMM_EINVAL;
        }
        most = std::max(most, pl.j_cta_hi[j] - pl.j_cta_lo[j] + 1);
    }
    // phase B lane groups: the widest group that still covers every (block, row)
    // in one round over all warps, but no narrower than 16 partials per lane
    {
        const int64_t items = static_cast<int64_t>(N) * m;
        const int64_t warps = static_cast<int64_t>(pl.P) * kConsumerWarps;
        int need_groups = 1;
        while (need_groups < 32 && static_cast<int64_t>(need_groups) * warps < items) need_groups *= 2;
        const int l_round = 32 / need_groups;
        int l_regs = 1;
        while (l_regs < 32 && l_regs * 16 < most * pl.groups) l_regs *= 2;
        pl.red_lanes = std::max(l_regs, l_round);
    }
    const int need = (((pl.npmax + pl.groups - 1) / pl.groups) + 31) / 32;
    int ch = 1;
    while (ch < need) ch *= 2;
    while (ch < force_chunks) ch *= 2;   // a multi-problem launch shares one kernel instance
    if (ch > 16) {
        *why = "column slab wider than 1024 pairs per CTA";
        return ADMM_EUNSUPPORTED;
    }
    pl.chunks = ch;
    pl.nsub = (pl.wmax + 255) / 256;
    pl.wbox = round_up((pl.wmax + pl.nsub - 1) / pl.nsub, 2);
    const int npitch = pl.wbox * pl.nsub / 2;   // pair pitch of the per-pair buffers
    pl.npitch = npitch;
    // FP16 stream: the box starts at the slab start rounded down to 4 columns
    // (16 bytes of 4-byte elements), so it covers up to 2 columns more
    pl.nsub16 = (pl.wmax + 2 + 255) / 256;
    pl.wbox16 = round_up((pl.wmax + 2 + pl.nsub16 - 1) / pl.nsub16, 4);
    if (pl.wbox16 > 256) {
        ++pl.nsub16;
        pl.wbox16 = round_up((pl.wmax + 2 + pl.nsub16 - 1) / pl.nsub16, 4);
    }
    pl.mimax = 0;
    for (int i = 0; i < M; ++i) pl.mimax = std::max(pl.mimax, row_off[i + 1] - row_off[i]);
    pl.kpmax = round_up(pl.mimax, 4);
    pl.ws_all = static_cast<int64_t>(m) * pl.njs * 8 <= 48 * 1024;
    pl.ws_rows = pl.ws_all ? static_cast<int>(m) : pl.mimax;
    // shared memory: fixed regions, then the deepest ring that fits
    const int ws = pl.njs * pl.ws_rows * 8;
    const int rs = pl.kpmax * 8;   // r_b, and the same again for gt_b
    const int wg = kConsumerWarps / pl.groups;   // warps summed per pair in the second pass
    pl.red_single = 2 * wg * npitch * 16 > 64 * 1024;
    pl.sigma_global = static_cast<int64_t>(M) * npitch * 16 > 32 * 1024;
    const int red = (pl.red_single ? 1 : 2) * wg * npitch * 16;
    const int sigma = pl.sigma_global ? 0 : M * npitch * 16;
    const int misc = 1024;
    const int fixed = round_up(ws, 128) + 2 * round_up(rs, 128) + round_up(red, 128) +
                      round_up(sigma, 128) + misc + 256 + 1024;
    pl.R = rows_per_stage(pl.chunks);
    pl.R16 = rows_per_stage(pl.chunks, true);
    pl.sub_bytes = pl.R * pl.wbox * 8;
    pl.stage_bytes = pl.sub_bytes * pl.nsub;
    // one ring region, cut into slots of either mode's stage size
    pl.stage_stride = round_up(pl.stage_bytes, 128);
    pl.stage_stride16 = round_up(pl.R16 * pl.wbox16 * 4 * pl.nsub16, 128);
    pl.nstages = std::min(8, (smem_limit - fixed) / pl.stage_stride);
    pl.nstages16 = std::min(8, (smem_limit - fixed) / pl.stage_stride16);
    if (pl.nstages < 2 || pl.nstages16 < 2) {
        *why = "shared memory too small for two pipeline stages";
        return ADMM_EUNSUPPORTED;
    }
    pl.ring_bytes = std::max(pl.stage_stride * pl.nstages, pl.stage_stride16 * pl.nstages16);
    int off = 0;
    pl.off_ring = off;
    off += pl.ring_bytes;
    off = round_up(off, 128);
    pl.off_full = off;
    off += 8 * 8;
    pl.off_empty = off;
    off += 8 * 8;
    off = round_up(off, 128);
    pl.off_ws = off;
    off += round_up(ws, 128);
    pl.off_rs = off;
    off += round_up(rs, 128);
    pl.off_gs = off;
    off += round_up(rs, 128);
    pl.off_red = off;
    off += round_up(red, 128);
    pl.off_sigma = off;
    off += round_up(sigma, 128);
    pl.off_misc = off;
    off += misc;
    pl.smem = off;
    if (pl.smem > smem_limit) {
        *why = "shared memory plan exceeds the device limit";
        return ADMM_EUNSUPPORTED;
    }
    // factor-apply rows (N * m of them) split evenly over the CTAs
    balanced_offsets(static_cast<int64_t>(N) * m, pl.P, pl.solve_lo);
    return ADMM_OK;
}

int view_handle(const admm_t* h, HandleView* v) {
    if (!h || !v) return ADMM_EINVAL;
    v->H = h->H;
    v->H16 = h->H16;
    v->kinv = h->kinv;
    v->scales = h->scales;
    v->kinv16 = h->kinv16;
    v->kinv_off = h->kinv_off_d;
    v->kinv_pitch = h->kinv_pitch_d;
    v->row_off = h->row_off_d;
    v->col_off = h->col_off_d;
    v->ld = h->plan.ld;
    v->status = h->status;
    return ADMM_OK;
}

}  // namespace admm

// ---------------------------------------------------------------------------
// setup helpers
// ---------------------------------------------------------------------------

namespace {

int validate(int64_t m, int64_t n, int M, int N, double lambda, double rho, int dtype) {
    if (m < 1 || n < 1) return fail(nullptr, ADMM_EINVAL, "m and n must be >= 1 (got %lld x %lld)",
                                     (long long)m, (long long)n);
    if (m > (1LL << 24) || n > (1LL << 28))
        return fail(nullptr, ADMM_EUNSUPPORTED, "m must be <= 2^24 and n <= 2^28");
    if (M < 1 || M > m || N < 1 || N > n)
        return fail(nullptr, ADMM_EINVAL, "need 1 <= row_blocks <= m and 1 <= col_blocks <= n");
    if (static_cast<int64_t>(M) * N > admm::kMaxBlocks)
        return fail(nullptr, ADMM_EINVAL, "row_blocks * col_blocks must be <= %d", admm::kMaxBlocks);
    if (static_cast<int64_t>(N) * m >= (1LL << 31))
        return fail(nullptr, ADMM_EUNSUPPORTED, "col_blocks * m must be < 2^31");
    if (!(lambda >= 0.0) || !std::isfinite(lambda))
        return fail(nullptr, ADMM_EINVAL, "lambda must be finite and >= 0");
    if (!(rho > 0.0) || !std::isfinite(rho))
        return fail(nullptr, ADMM_EINVAL, "rho must be finite and > 0");
    if (dtype != ADMM_C64 && dtype != ADMM_C128)
        return fail(nullptr, ADMM_EINVAL, "h_dtype must be ADMM_C64 or ADMM_C128");
    return ADMM_OK;
}

int copy_vector_in(admm_t* h, float2* dst, const void* src, int64_t count, int dtype,
                   cudaStream_t st) {
    if (dtype == ADMM_C64) {
        CK(h, cudaMemcpyAsync(dst, src, count * sizeof(float2), cudaMemcpyDefault, st));
        return ADMM_OK;
    }
    double2* tmp = nullptr;
    CK(h, dalloc(&tmp, count));
    cudaError_t e = cudaMemcpyAsync(tmp, src, count * sizeof(double2), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = admm::launch_pack_c128(tmp, 1, count, dst, count, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy complex128 vector");
    return ADMM_OK;
}

// Gram products and FP64 Cholesky inverse of every block of the factor
// problem f (f.A, f.W are allocated here); `dim` is the largest factor edge.
int run_factor(admm_t* h, cudaStream_t st, admm::FactorArgs f, int dim, float2* kinv, bool timed) {
    const int T = (dim + admm::kTile - 1) / admm::kTile;
    const size_t S = static_cast<size_t>(T) * admm::kTile;
    const int nb = f.M * f.N;
    double2 *A = nullptr, *W = nullptr;
    if (dalloc(&A, S * S * nb) != cudaSuccess || dalloc(&W, S * S * nb) != cudaSuccess) {
        if (A) cudaFree(A);
        return fail(h, ADMM_ENOMEM, "cannot allocate %.1f MB of FP64 factor workspace",
                    2.0 * S * S * nb * 16 / 1e6);
    }
    f.T = T;
    f.A = A;
    f.W = W;
    f.kinv = kinv;
    f.rho = h->rho;
    f.status = h->status;
    cudaEvent_t e0, e1, e2;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    cudaError_t err = cudaMemsetAsync(kinv, 0, h->kinv_elems * sizeof(float2), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(h->status, 0, sizeof(int), st);
    if (err == cudaSuccess) err = cudaEventRecord(e0, st);
    if (err == cudaSuccess) err = admm::launch_gram(f, st);
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = admm::launch_cholesky_inverse(f, st);
    if (err == cudaSuccess) err = cudaEventRecord(e2, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    float t01 = 0.f, t12 = 0.f;
    if (err == cudaSuccess) {
        cudaEventElapsedTime(&t01, e0, e1);
        cudaEventElapsedTime(&t12, e1, e2);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    cudaFree(A);
    cudaFree(W);
    if (err != cudaSuccess) return cuda_fail(h, err, "factor kernels");
    if (timed) {
        h->gram_ms = t01;
        h->factor_ms = t12;
    }
    int st_code = 0;
    CK(h, cudaMemcpy(&st_code, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st_code == ADMM_ENOTPD)
        return fail(h, ADMM_ENOTPD, "a block factor is not positive definite in FP64");
    if (st_code != 0) return fail(h, st_code, "factor kernels raised status %d", st_code);
    return ADMM_OK;
}

// Factors of the handle's form from the complex64 matrix H (m x ld):
//  lemma:  K_b^{-1} = (rho I + H_b H_b^H)^{-1}, m_i x m_i;
//  direct: L_b = (H_b^H H_b + rho I)^{-1}, n_j x n_j, the same Gram and
//          inverse taken over the blocks of H^H (block (j, i) of H^H is H_b^H).
int build_factors(admm_t* h, cudaStream_t st, const float2* H, float2* kinv, bool timed) {
    admm::FactorArgs f;
    std::memset(&f, 0, sizeof f);
    if (h->form != ADMM_FORM_DIRECT) {
        f.m = static_cast<int>(h->m);
        f.ld = h->plan.ld;
        f.M = h->M;
        f.N = h->N;
        f.row_off = h->row_off_d;
        f.col_off = h->col_off_d;
        f.H = H;
        f.kinv_off = h->kinv_off_d;
        f.kinv_pitch = h->kinv_pitch_d;
        return run_factor(h, st, f, h->plan.mimax, kinv, timed);
    }
    const int64_t ldT = round_up(h->m, 32);
    float2* HT = nullptr;
    if (dalloc(&HT, static_cast<size_t>(ldT) * h->n) != cudaSuccess)
        return fail(h, ADMM_ENOMEM, "no room for the conjugate transpose of H (%.1f MB)", ldT * h->n * 8 / 1e6);
    cudaError_t e = cudaMemsetAsync(HT, 0, static_cast<size_t>(ldT) * h->n * sizeof(float2), st);
    if (e == cudaSuccess) e = admm::launch_conj_transpose(H, h->m, h->n, h->plan.ld, HT, ldT, st);
    if (e != cudaSuccess) {
        cudaFree(HT);
        return cuda_fail(h, e, "conjugate transpose of H");
    }
    f.m = static_cast<int>(h->n);
    f.ld = static_cast<int>(ldT);
    f.M = h->N;
    f.N = h->M;
    f.row_off = h->col_off_d;
    f.col_off = h->row_off_d;
    f.H = HT;
    f.kinv_off = h->kinv_off_d;      // indexed by the H^H block (j, i)
    f.kinv_pitch = h->kinv_pitch_d;
    const int code = run_factor(h, st, f, h->dir.njmax, kinv, timed);
    cudaFree(HT);
    return code;
}

// factors of the matrix the FP16 copy encodes (dequantised into a scratch copy)
int build_factors_f16(admm_t* h, cudaStream_t st) {
    const size_t elems = static_cast<size_t>(h->plan.ld) * h->m;
    float2* Hdeq = nullptr;
    if (dalloc(&Hdeq, elems) != cudaSuccess)
        return fail(h, ADMM_ENOMEM, "cannot allocate %.1f MB to dequantise the FP16 copy of H", elems * 8 / 1e6);
    cudaError_t e = admm::launch_dequantize_f16(h->H16, h->m, h->plan.ld, h->scales, Hdeq, st);
    int code = ADMM_OK;
    if (e != cudaSuccess) code = cuda_fail(h, e, "dequantise H");
    else code = build_factors(h, st, Hdeq, h->kinv16, false);
    cudaStreamSynchronize(st);
    cudaFree(Hdeq);
    return code;
}

int encode_tensor_map(admm_t* h) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(h, ADMM_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const Plan& pl = h->plan;
    // complex64 H: one 8-byte element per complex entry; FP16 H: one 4-byte element
    const bool f16 = h->H16 != nullptr;
    for (int f = 0; f < (f16 ? 2 : 1); ++f) {
        const size_t eb = f ? 4 : 8;
        cuuint64_t dims[2] = {static_cast<cuuint64_t>(pl.ld), static_cast<cuuint64_t>(h->m)};
        cuuint64_t strides[1] = {static_cast<cuuint64_t>(pl.ld) * eb};
        cuuint32_t box[2] = {static_cast<cuuint32_t>(f ? pl.wbox16 : pl.wbox),
                             static_cast<cuuint32_t>(f ? pl.R16 : pl.R)};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = encode(f ? &h->tmap16 : &h->tmap,
                            f ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                            f ? h->H16 : static_cast<void*>(h->H), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(h, ADMM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    return ADMM_OK;
}

// quantise H to the FP16 copy and factor the matrix it encodes (once per handle)
int enable_f16(admm_t* h) {
    if (h->H16) return ADMM_OK;
    const Plan& pl = h->plan;
    const size_t elems = static_cast<size_t>(pl.ld) * h->m;
    const int64_t groups = (h->m + 63) / 64;
    if (cudaMalloc(&h->H16, elems * 4) != cudaSuccess || dalloc(&h->scales, groups) != cudaSuccess ||
        dalloc(&h->gmax, groups) != cudaSuccess || dalloc(&h->kinv16, h->kinv_elems) != cudaSuccess) {
        void* ptrs[] = {h->H16, h->scales, h->gmax, h->kinv16};
        for (void* p : ptrs)
            if (p) cudaFree(p);
        h->H16 = nullptr;
        h->scales = nullptr;
        h->gmax = nullptr;
        h->kinv16 = nullptr;
        return fail(h, ADMM_ENOMEM, "cannot allocate %.1f MB for the FP16 copy of H", elems * 4 / 1e6);
    }
    cudaStream_t st = nullptr;
    CK(h, cudaDeviceSynchronize());
    CK(h, admm::launch_quantize_f16(h->H, h->m, pl.ld, h->gmax, h->H16, h->scales, nullptr, st));
    int code = build_factors_f16(h, st);
    if (code == ADMM_OK) code = encode_tensor_map(h);
    if (code) {
        void* ptrs[] = {h->H16, h->scales, h->gmax, h->kinv16};
        for (void* p : ptrs)
            if (p) cudaFree(p);
        h->H16 = nullptr;
        h->scales = nullptr;
        h->gmax = nullptr;
        h->kinv16 = nullptr;
        return code;
    }
    CK(h, cudaDeviceSynchronize());
    return ADMM_OK;
}

int zero_state(admm_t* h, cudaStream_t st) {
    const size_t ld = h->plan.ld;
    CK(h, cudaMemsetAsync(h->v, 0, ld * sizeof(float2), st));
    CK(h, cudaMemsetAsync(h->s, 0, ld * h->M * sizeof(float2), st));
    CK(h, cudaMemsetAsync(h->u, 0, ld * h->M * sizeof(float2), st));
    CK(h, cudaMemsetAsync(h->ghat, 0, 2 * static_cast<size_t>(h->N) * h->m * sizeof(float2), st));
    CK(h, cudaMemsetAsync(h->bar, 0, 2 * sizeof(unsigned), st));
    CK(h, cudaMemsetAsync(h->status, 0, sizeof(int), st));
    CK(h, cudaMemsetAsync(h->stop_flag, 0, sizeof(int), st));
    CK(h, cudaMemsetAsync(h->k_done, 0, sizeof(long long), st));
    CK(h, cudaMemsetAsync(h->hist, 0, static_cast<size_t>(h->hist_cap) * 5 * sizeof(double), st));
    h->dir.q_valid = false;
    if (h->sh_g0) CK(h, cudaMemcpyAsync(h->g, h->sh_g0, h->m * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    if (h->form == ADMM_FORM_DIRECT) {
        CK(h, cudaMemsetAsync(h->dir.cnt, 0, static_cast<size_t>(h->dir.ncnt) * sizeof(unsigned), st));
        CK(h, cudaMemsetAsync(h->dir.stop_pending, 0, sizeof(int), st));
    }
    h->k = 0;
    h->broken = 0;
    h->pending = 0;
    h->rec_valid = h->rec_cap > 0;
    h->rec_f16 = h->use_f16;
    return ADMM_OK;
}

// buffers of the direct form; off / pitch locate the factor of block p = i * N + j
int alloc_direct(admm_t* h, const std::vector<long long>& off, const std::vector<int>& pitch, int njmax) {
    DirectState& d = h->dir;
    const int P = h->M * h->N;
    const int mimax = h->plan.mimax;
    d.njmax = njmax;
    d.herm = njmax >= admm::kDirHermMinCols && h->M <= admm::kDirHermMaxRowBlocks ? 1 : 0;
    d.npitch = d.herm ? round_up(njmax, admm::kDirTile) : round_up(njmax, 4);   // tiles read whole q panels
    // column tiles: pairs from each block's first column rounded down to even
    int pairs = 1;
    for (int j = 0; j < h->N; ++j) {
        const int c0 = h->col_off[j], c1 = h->col_off[j + 1];
        pairs = std::max(pairs, (c1 - (c0 & ~1) + 1) / 2);
    }
    d.ccn = (pairs + admm::kDirColPairs - 1) / admm::kDirColPairs;
    d.ctas = 2 * h->num_sms;   // factor and row passes: one wave of two CTAs per SM
    // factor pass streamed through shared memory for blocks of 1024 to 2048
    // columns (a stage of four rows fits three times): a ring of up to eight
    // stages, as many CTAs per SM (up to four) as its registers and shared
    // memory hold
    d.fac_stream = 0;
    if (njmax >= admm::kDirBulkMinCols && njmax <= admm::kDirBulkMaxCols) {
        const int stage = round_up(static_cast<int64_t>(4) * round_up(njmax, 4) * 8, 128);
        int ns = 8;
        while (ns >= 2 && admm::stream_smem(ns, stage) > static_cast<size_t>(h->smem_optin)) --ns;
        int per_sm = 0;
        if (ns >= 2 && admm::prepare_direct(h->smem_optin) == cudaSuccess &&
            admm::direct_stream_per_sm(static_cast<int>(admm::stream_smem(ns, stage)), &per_sm) == cudaSuccess &&
            per_sm >= 1) {
            d.fac_stream = 1;
            d.fac_ns = ns;
            d.fac_stage = stage;
            d.fac_ctas = h->num_sms * std::min(4, per_sm);
        }
    }
    // row splits of the column pass: at most one wave at two CTAs per SM, at
    // least 32 rows per split where the blocks allow, at most kDirColRows (the
    // staged gt_b)
    int S = (2 * h->num_sms) / (P * d.ccn);
    S = std::min(S, std::max(1, mimax / 32));
    S = std::max(S, (mimax + admm::kDirColRows - 1) / admm::kDirColRows);
    d.S = std::max(S, 1);
    std::vector<int> ints(h->N + 1, 0);
    for (int j = 0; j < h->N; ++j)
        ints[j + 1] = ints[j] + (h->col_off[j + 1] - h->col_off[j] + admm::kDirChunk - 1) / admm::kDirChunk;
    d.nchunks = ints[h->N];
    ints.insert(ints.end(), pitch.begin(), pitch.end());
    // factor rows and H rows of the blocks in order p = i * N + j, concatenated
    std::vector<int> foff(P + 1, 0), roff(P + 1, 0);
    for (int q = 0; q < P; ++q) {
        const int i = q / h->N, j = q % h->N;
        foff[q + 1] = foff[q] + (h->col_off[j + 1] - h->col_off[j]);
        roff[q + 1] = roff[q] + (h->row_off[i + 1] - h->row_off[i]);
    }
    d.frows = foff[P];
    d.hrows = roff[P];
    ints.insert(ints.end(), foff.begin(), foff.end());
    ints.insert(ints.end(), roff.begin(), roff.end());
    // items of the streamed factor pass: the update chunks of each block
    std::vector<int> ioff(P + 1, 0);
    for (int q = 0; q < P; ++q) {
        const int j = q % h->N;
        ioff[q + 1] = ioff[q] + (h->col_off[j + 1] - h->col_off[j] + admm::kDirChunk - 1) / admm::kDirChunk;
    }
    d.fitems = ioff[P];
    ints.insert(ints.end(), ioff.begin(), ioff.end());
    d.ncnt = P * d.ccn + d.nchunks + 4;
    const size_t vec = static_cast<size_t>(P) * d.npitch;
    // the column pass writes partials in both uses (q_b every iteration with
    // several column blocks, C = H_i^H g_i once per data vector with one)
    const size_t nc = h->N == 1 ? vec : 1, np = static_cast<size_t>(d.S) * vec;
    const size_t nq = h->N == 1 ? 2 * vec : vec;   // one column block: a slot per iteration parity
    bool ok = dalloc(&d.C, nc) == cudaSuccess && dalloc(&d.Q, nq) == cudaSuccess &&
              dalloc(&d.part, np) == cudaSuccess && dalloc(&d.cnt, d.ncnt) == cudaSuccess &&
              dalloc(&d.ints, ints.size()) == cudaSuccess && dalloc(&d.L_off, off.size()) == cudaSuccess &&
              dalloc(&d.res_chunk, static_cast<size_t>(d.nchunks) * 5) == cudaSuccess &&
              dalloc(&d.stop_pending, 1) == cudaSuccess;
    if (ok && d.herm) {
        // block p's tiles (I, J), J <= I, indexed from T_off[p]
        std::vector<long long> toff(P + 1, 0);
        std::vector<int> nt(P, 0);
        for (int q = 0; q < P; ++q) {
            const int j = q % h->N;
            nt[q] = (h->col_off[j + 1] - h->col_off[j] + admm::kDirTile - 1) / admm::kDirTile;
            toff[q + 1] = toff[q] + static_cast<long long>(nt[q]) * (nt[q] + 1) / 2;
        }
        d.ntiles = toff[P];
        // the pass order: tile column J, then block, then tile row I
        std::vector<int4> seq;
        seq.reserve(static_cast<size_t>(d.ntiles));
        const int ntmax = *std::max_element(nt.begin(), nt.end());
        for (int J = 0; J < ntmax; ++J)
            for (int q = 0; q < P; ++q)
                for (int I = J; I < nt[q]; ++I)
                    seq.push_back(make_int4(static_cast<int>(toff[q] + static_cast<long long>(I) * (I + 1) / 2 + J),
                                            q, I, J));
        const size_t tile = static_cast<size_t>(admm::kDirTile) * admm::kDirTile;
        ok = dalloc(&d.Lt, static_cast<size_t>(d.ntiles) * tile) == cudaSuccess &&
             dalloc(&d.RP, static_cast<size_t>(d.ntiles) * admm::kDirTile) == cudaSuccess &&
             dalloc(&d.CP, static_cast<size_t>(d.ntiles) * admm::kDirTile) == cudaSuccess &&
             dalloc(&d.T_off, toff.size()) == cudaSuccess && dalloc(&d.T_seq, seq.size()) == cudaSuccess &&
             dalloc(&d.dctl, 4) == cudaSuccess;
        int per_sm = 0;
        if (ok && (admm::herm_per_sm(&per_sm) != cudaSuccess || per_sm < 1)) {
            cudaGetLastError();
            d.herm = 0;   // no tile pass on this device: the full-row passes remain
        }
        d.herm_ctas = h->num_sms * std::max(per_sm, 1);
        if (ok && d.herm) {
            CK(h, cudaMemcpy(d.T_off, toff.data(), toff.size() * sizeof(long long), cudaMemcpyHostToDevice));
            CK(h, cudaMemcpy(d.T_seq, seq.data(), seq.size() * sizeof(int4), cudaMemcpyHostToDevice));
            CK(h, cudaMemset(d.dctl, 0, 4 * sizeof(long long)));
        }
    }
    if (!ok) return ADMM_ENOMEM;
    // Q and C padding entries stay zero (the factor pass reads whole pairs)
    CK(h, cudaMemset(d.C, 0, nc * sizeof(float2)));
    CK(h, cudaMemset(d.Q, 0, nq * sizeof(float2)));
    CK(h, cudaMemset(d.cnt, 0, static_cast<size_t>(d.ncnt) * sizeof(unsigned)));
    CK(h, cudaMemset(d.stop_pending, 0, sizeof(int)));
    CK(h, cudaMemcpy(d.ints, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(d.L_off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice));
    d.bytes = static_cast<int64_t>((nc + nq + np) * sizeof(float2) + d.nchunks * 5 * sizeof(double));
    if (d.herm) d.bytes += static_cast<int64_t>(d.ntiles) * (admm::kDirTile * admm::kDirTile + 2 * admm::kDirTile) * 8;
    return ADMM_OK;
}

// the tile pass reads the factor's lower triangle: (re)pack it after every factorisation
int pack_direct_tiles(admm_t* h, cudaStream_t st) {
    const DirectState& d = h->dir;
    if (h->form != ADMM_FORM_DIRECT || !d.herm) return ADMM_OK;
    CK(h, admm::launch_pack_herm(h->kinv, d.L_off, d.ints + (h->N + 1), h->col_off_d, h->N, d.T_seq, d.ntiles, d.Lt,
                                 st));
    return ADMM_OK;
}

// the tile pass runs for this handle (forced, or by default on blocks of kDirHermAutoCols columns and more)
bool uses_tiles(const DirectState& d) {
    return d.herm && (d.pass == 2 || (d.pass == 0 && d.njmax >= admm::kDirHermAutoCols));
}

admm::DirectArgs direct_args(admm_t* h, int check_stop, double eps_abs, double eps_rel) {
    const DirectState& d = h->dir;
    admm::DirectArgs a;
    std::memset(&a, 0, sizeof a);
    a.m = static_cast<int>(h->m);
    a.n = static_cast<int>(h->n);
    a.ld = h->plan.ld;
    a.M = h->M;
    a.N = h->N;
    a.P = h->M * h->N;
    a.npitch = d.npitch;
    a.njmax = d.njmax;
    a.mimax = h->plan.mimax;
    a.row_off = h->row_off_d;
    a.col_off = h->col_off_d;
    a.H = h->H;
    a.g = h->g;
    a.v = h->v;
    a.s = h->s;
    a.u = h->u;
    a.ghat = h->ghat;
    a.L = h->kinv;
    a.L_off = d.L_off;
    a.L_pitch = d.ints + (h->N + 1);
    a.C = d.C;
    a.Q = d.Q;
    a.part = d.part;
    a.S = d.S;
    a.ccn = d.ccn;
    a.ctas = d.ctas;
    a.fac_stream = d.fac_stream;
    a.fac_ctas = d.fac_ctas;
    a.fac_ns = d.fac_ns;
    a.fac_stage = d.fac_stage;
    a.fac_herm = uses_tiles(d) ? 1 : 0;
    a.Lt = d.Lt;
    a.T_seq = d.T_seq;
    a.T_off = d.T_off;
    a.RP = d.RP;
    a.CP = d.CP;
    a.ntiles = static_cast<int>(d.ntiles);
    a.herm_ctas = d.herm_ctas;
    a.defer_record = a.fac_herm && h->N == 1 ? 1 : 0;
    a.dctl = d.dctl;
    a.timeout_ns = h->timeout_ns;
    a.frows = d.frows;
    a.hrows = d.hrows;
    a.F_off = d.ints + (h->N + 1) + a.P;
    a.R_off = d.ints + (h->N + 1) + a.P + (a.P + 1);
    a.I_off = d.ints + (h->N + 1) + a.P + 2 * (a.P + 1);
    a.fitems = d.fitems;
    a.cnt_cols = d.cnt;
    a.cnt_upd = d.cnt + a.P * d.ccn;
    a.cnt_glob = d.cnt + a.P * d.ccn + d.nchunks;
    a.chunk_off = d.ints;
    a.nchunks = d.nchunks;
    a.res_chunk = d.res_chunk;
    a.hist = h->hist;
    a.hist_cap = h->hist_cap;
    a.k_done = h->k_done;
    a.status = h->status;
    a.stop_flag = h->stop_flag;
    a.stop_pending = d.stop_pending;
    a.check_stop = check_stop;
    a.eps_abs = eps_abs;
    a.eps_rel = eps_rel;
    a.rho = static_cast<float>(h->rho);
    a.rho_d = h->rho;
    a.kappa = static_cast<float>(h->lambda / (h->M * h->rho));
    a.inv_M = 1.0f / static_cast<float>(h->M);
    return a;
}

void drop_direct_graphs(DirectState& d) {
    if (d.g1) cudaGraphExecDestroy(d.g1);
    if (d.g16) cudaGraphExecDestroy(d.g16);
    d.g1 = d.g16 = nullptr;
}

// `iters` iterations of the direct form: per iteration the column pass, the
// factor pass with the update and the row pass; with one column block the
// factor pass alone (its update writes the next iteration's q).  Launched as captured graphs of
// one and sixteen iterations, re-captured when a scalar argument changes.
int run_direct(admm_t* h, int iters, int check_stop, double eps_abs, double eps_rel, cudaStream_t st) {
    DirectState& d = h->dir;
    const admm::DirectArgs a = direct_args(h, check_stop, eps_abs, eps_rel);
    if (h->N == 1) {
        // one column block: C once per data vector, q of the current
        // iteration once per state change (each update writes the next q)
        if (!d.c_valid) {
            CK(h, admm::launch_dir_cols(a, 1, st));
            d.c_valid = true;
            d.q_valid = false;
        }
        if (!d.q_valid) {
            CK(h, admm::launch_dir_q(a, st));
            d.q_valid = true;
        }
    }
    if (a.defer_record) {
        // the tile pass counts from the recorded iterations, nothing pending
        CK(h, cudaMemcpyAsync(d.dctl, h->k_done, sizeof(long long), cudaMemcpyDeviceToDevice, st));
        CK(h, cudaMemsetAsync(d.dctl + 2, 0, sizeof(long long), st));
    }
    const double key[7] = {h->rho, h->lambda, static_cast<double>(check_stop), eps_abs, eps_rel,
                           static_cast<double>(h->hist_cap), static_cast<double>(h->timeout_ns)};
    if (!d.key_set || std::memcmp(key, d.key, sizeof key) != 0 || d.key_hist != h->hist) {
        drop_direct_graphs(d);
        std::memcpy(d.key, key, sizeof key);
        d.key_hist = h->hist;
        d.key_set = true;
    }
    auto capture = [&](int count, cudaGraphExec_t* out) -> cudaError_t {
        cudaError_t e = cudaStreamBeginCapture(d.cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        for (int q = 0; q < count && e == cudaSuccess; ++q) {
            if (h->N == 1) {
                e = admm::launch_dir_factor(a, d.cap);
            } else {
                e = admm::launch_dir_cols(a, 0, d.cap);
                if (e == cudaSuccess) e = admm::launch_dir_factor(a, d.cap);
                if (e == cudaSuccess) e = admm::launch_dir_rows(a, d.cap);
            }
        }
        if (e == cudaSuccess && a.defer_record) e = admm::launch_dir_record(a, d.cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(d.cap, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        return e;
    };
    int left = iters;
    if (left >= 16) {
        if (!d.g16) CK(h, capture(16, &d.g16));
        for (; left >= 16; left -= 16) CK(h, cudaGraphLaunch(d.g16, st));
    }
    if (left > 0) {
        if (!d.g1) CK(h, capture(1, &d.g1));
        for (; left > 0; --left) CK(h, cudaGraphLaunch(d.g1, st));
    }
    h->k += iters;
    h->pending = 0;   // the direct form writes each record inside the iteration
    return ADMM_OK;
}


// device tables and scratch that depend on the launch plan
struct PlanBuffers {
    const int *cta_col, *cta_end, *own0, *own1, *jlo, *nj, *j_lo, *j_hi, *solve_lo;
    float2* part;
    double* res_part;
    unsigned* bar;
};

PlanBuffers handle_buffers(admm_t* h) {
    return PlanBuffers{h->cta_col_d, h->cta_end_d, h->cta_own0_d, h->cta_own1_d,
                       h->cta_jlo_d, h->cta_nj_d, h->j_cta_lo_d, h->j_cta_hi_d, h->solve_lo_d, h->part,
                       h->res_part, h->bar};
}

// kernel arguments of `iters` iterations of h under plan pl
void fill_args(admm_t* h, const Plan& pl, const PlanBuffers& b, int iters, int check_stop, double eps_abs,
               double eps_rel, admm::IterArgs& a) {
    std::memset(&a, 0, sizeof a);
    a.m = static_cast<int>(h->m);
    a.n = static_cast<int>(h->n);
    a.ld = pl.ld;
    a.M = h->M;
    a.N = h->N;
    a.P = pl.P;
    const bool f16 = h->use_f16 != 0;
    a.R = f16 ? pl.R16 : pl.R;
    a.nstages = f16 ? pl.nstages16 : pl.nstages;
    a.stage_stride = f16 ? pl.stage_stride16 : pl.stage_stride;
    a.nsub = f16 ? pl.nsub16 : pl.nsub;
    a.wbox = f16 ? pl.wbox16 : pl.wbox;
    a.elem_bytes = f16 ? 4 : 8;
    a.sub_bytes = a.R * a.wbox * a.elem_bytes;
    a.stage_bytes = a.sub_bytes * a.nsub;
    a.npitch = pl.npitch;
    a.mimax = pl.mimax;
    a.kpmax = pl.kpmax;
    a.off_ring = pl.off_ring;
    a.off_full = pl.off_full;
    a.off_empty = pl.off_empty;
    a.off_ws = pl.off_ws;
    a.off_rs = pl.off_rs;
    a.off_gs = pl.off_gs;
    a.off_red = pl.off_red;
    a.off_sigma = pl.off_sigma;
    a.off_misc = pl.off_misc;
    a.red_lanes = pl.red_lanes;
    a.ws_all = pl.ws_all ? 1 : 0;
    a.ws_rows = pl.ws_rows;
    a.sigma_global = pl.sigma_global ? 1 : 0;
    a.red_single = pl.red_single ? 1 : 0;
    a.pgroups = pl.groups;
    a.chunks = pl.chunks;
    a.rho = static_cast<float>(h->rho);
    a.rho_d = h->rho;
    a.kappa = static_cast<float>(h->lambda / (h->M * h->rho));
    a.inv_M = 1.0f / static_cast<float>(h->M);
    a.row_off = h->row_off_d;
    a.col_off = h->col_off_d;
    a.cta_col = b.cta_col;
    a.cta_end = b.cta_end;
    a.cta_own0 = b.own0;
    a.cta_own1 = b.own1;
    a.cta_jlo = b.jlo;
    a.cta_nj = b.nj;
    a.j_cta_lo = b.j_lo;
    a.j_cta_hi = b.j_hi;
    a.solve_lo = b.solve_lo;
    a.v = h->v;
    a.s = h->s;
    a.u = h->u;
    a.g = h->g;
    a.ghat = h->ghat;
    a.gt = h->gt;
    a.r = h->r;
    a.w = h->w;
    a.part = b.part;
    a.kinv = f16 ? h->kinv16 : h->kinv;
    a.scales = f16 ? h->scales : nullptr;
    a.kinv_off = h->kinv_off_d;
    a.kinv_pitch = h->kinv_pitch_d;
    a.res_part = b.res_part;
    a.hist = h->hist;
    a.k_done = h->k_done;
    a.bar = b.bar;
    a.status = h->status;
    a.stop_flag = h->stop_flag;
    a.k0 = h->k;
    a.hist_cap = h->hist_cap;
    a.iters = iters;
    a.check_stop = check_stop;
    a.eps_abs = eps_abs;
    a.eps_rel = eps_rel;
    a.timeout_ns = h->timeout_ns;
    a.bar_extra = h->bar_extra;
    a.trace = h->trace;
    a.trace_iters = h->trace_iters;
    {
        const int64_t per_stage = f16 ? static_cast<int64_t>(pl.R16) * pl.ld * 4 : static_cast<int64_t>(pl.R) * pl.ld * 8;
        a.keep_stages = static_cast<int>(std::max<int64_t>(0, h->l2_keep_bytes / std::max<int64_t>(per_stage, 1)));
        a.prefetch_stages = static_cast<int>(h->l2_prefetch_bytes / std::max<int64_t>(per_stage, 1));
    }
    a.pending_prev = h->pending && h->k > 0 ? 1 : 0;
    if (h->rec_cap > 0) {
        if (h->use_f16 != h->rec_f16 || h->k + iters > h->rec_cap) h->rec_valid = false;
        a.rec_a = h->rec_a;
        a.rec_w = h->rec_w;
        a.rec_cap = h->rec_cap;
        a.rec_pitch = h->rec_pitch;
    }
}

int run_kernel(admm_t* h, int iters, int check_stop, double eps_abs, double eps_rel,
               cudaStream_t st) {
    const Plan& pl = h->plan;
    admm::IterArgs a;
    fill_args(h, pl, handle_buffers(h), iters, check_stop, eps_abs, eps_rel, a);
    const bool f16 = h->use_f16 != 0;
    cudaError_t e = admm::launch_iterate(f16 ? h->tmap16 : h->tmap, a, pl.chunks, pl.smem, st, f16);
    if (e != cudaSuccess) return cuda_fail(h, e, "cooperative launch of the iteration kernel");
    h->k += iters;
    h->pending = 1;   // this launch's last record is summed by the next launch or a sync call
    return ADMM_OK;
}

int device_status(admm_t* h, cudaStream_t st) {
    CK(h, cudaStreamSynchronize(st));
    long long kd0 = 0;
    CK(h, cudaMemcpy(&kd0, h->k_done, sizeof(long long), cudaMemcpyDeviceToHost));
    if (h->pending && kd0 > 0) {
        // sum the last launch's final residual record (its kernel ends without a grid barrier)
        admm::IterArgs a;
        std::memset(&a, 0, sizeof a);
        a.M = h->M;
        a.n = static_cast<int>(h->n);
        a.P = h->plan.P;
        a.rho_d = h->rho;
        a.res_part = h->res_part;
        a.hist = h->hist;
        a.hist_cap = h->hist_cap;
        a.status = h->status;
        CK(h, admm::launch_finalize(a, kd0 - 1, st));
        CK(h, cudaStreamSynchronize(st));
    }
    h->pending = 0;
    int code = 0;
    long long kd = 0;
    CK(h, cudaMemcpy(&code, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(&kd, h->k_done, sizeof(long long), cudaMemcpyDeviceToHost));
    h->k = kd;
    if (code == ADMM_ETIMEOUT) {
        h->broken = 1;
        return fail(h, code, "a bounded in-kernel wait expired (state undefined; call admm_reset)");
    }
    if (code == ADMM_EDIVERGED) return fail(h, code, "the iterates became NaN or Inf");
    if (code != 0) return fail(h, code, "device status %d", code);
    return ADMM_OK;
}

void free_record(admm_t* h) {
    void* ptrs[] = {h->rec_a, h->rec_w, h->bVb, h->bSb, h->bGhb, h->bGt, h->bdG, h->bSig, h->bP, h->bR,
                    h->bW, h->bkbar, h->brbar, h->bkappa, h->bupd};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    h->rec_a = h->rec_w = h->bVb = h->bSb = h->bGhb = h->bGt = h->bdG = h->bSig = h->bP = h->bR = h->bW = nullptr;
    h->bkbar = h->brbar = nullptr;
    h->bkappa = nullptr;
    h->bupd = nullptr;
    h->rec_cap = 0;
    h->rec_valid = false;
}

// record the next `value` iterations (and allocate the reverse sweep's buffers); resets the state
int set_record(admm_t* h, int64_t value) {
    if (value < 0 || value > (1 << 20)) return fail(h, ADMM_EINVAL, "record length out of range");
    CK(h, cudaDeviceSynchronize());
    free_record(h);
    if (value > 0) {
        const Plan& pl = h->plan;
        int mimax = 0, njmax = 0;
        for (int i = 0; i < h->M; ++i) mimax = std::max(mimax, h->row_off[i + 1] - h->row_off[i]);
        for (int j = 0; j < h->N; ++j) njmax = std::max(njmax, h->col_off[j + 1] - h->col_off[j]);
        h->rec_pitch = round_up(mimax, 32);
        h->bnpitch = round_up(njmax, 32);
        const size_t P = static_cast<size_t>(h->M) * h->N, ld = pl.ld, m = h->m;
        std::vector<int> uto(h->N + 1, 0);
        for (int j = 0; j < h->N; ++j)
            uto[j + 1] = uto[j] + (h->col_off[j + 1] - h->col_off[j] + admm::batch::kUpdCols - 1) / admm::batch::kUpdCols;
        h->bupd_tiles = uto[h->N];
        const bool ok = dalloc(&h->rec_a, static_cast<size_t>(value) * ld) == cudaSuccess &&
                        dalloc(&h->rec_w, static_cast<size_t>(value) * P * h->rec_pitch) == cudaSuccess &&
                        dalloc(&h->bVb, ld) == cudaSuccess && dalloc(&h->bSb, ld * h->M) == cudaSuccess &&
                        dalloc(&h->bGhb, m * h->N) == cudaSuccess && dalloc(&h->bGt, m * h->N) == cudaSuccess &&
                        dalloc(&h->bdG, m) == cudaSuccess && dalloc(&h->bSig, P * h->bnpitch) == cudaSuccess &&
                        dalloc(&h->bP, P * h->rec_pitch) == cudaSuccess && dalloc(&h->bR, P * h->rec_pitch) == cudaSuccess &&
                        dalloc(&h->bW, P * h->rec_pitch) == cudaSuccess && dalloc(&h->bkbar, 1) == cudaSuccess &&
                        dalloc(&h->brbar, 1) == cudaSuccess && dalloc(&h->bkappa, 1) == cudaSuccess &&
                        dalloc(&h->bupd, uto.size()) == cudaSuccess;
        if (!ok) {
            free_record(h);
            return fail(h, ADMM_ENOMEM, "no room to record %lld iterations", static_cast<long long>(value));
        }
        CK(h, cudaMemset(h->rec_a, 0, static_cast<size_t>(value) * ld * sizeof(float2)));
        CK(h, cudaMemcpy(h->bupd, uto.data(), uto.size() * sizeof(int), cudaMemcpyHostToDevice));
        h->rec_cap = static_cast<int>(value);
    }
    const int code = zero_state(h, nullptr);
    if (code) return code;
    CK(h, cudaDeviceSynchronize());
    return ADMM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

int admm_abi_version(void) { return ADMM_ABI_VERSION; }

const char* admm_strerror(int status) {
    switch (status) {
        case ADMM_OK: return "ok";
        case ADMM_EINVAL: return "invalid argument";
        case ADMM_ENOMEM: return "device allocation failed";
        case ADMM_ECUDA: return "CUDA error";
        case ADMM_ENOTPD: return "factor not positive definite";
        case ADMM_ENONFINITE: return "non-finite input";
        case ADMM_ETIMEOUT: return "bounded in-kernel wait expired";
        case ADMM_EUNSUPPORTED: return "unsupported problem shape";
        case ADMM_EDIVERGED: return "iterates diverged";
        default: return "unknown status";
    }
}

const char* admm_last_error(const admm_t* h) {
    return h ? h->err.c_str() : g_setup_error.c_str();
}

int admm_partition(int64_t total, int32_t parts, int64_t* offsets) {
    if (!offsets || parts < 1 || total < parts) return ADMM_EINVAL;
    const int64_t base = total / parts, extra = total % parts;
    int64_t pos = 0;
    for (int p = 0; p < parts; ++p) {
        offsets[p] = pos;
        pos += base + (p < extra ? 1 : 0);
    }
    offsets[parts] = pos;
    return ADMM_OK;
}

int admm_comm_elements(int64_t m, int64_t n, int32_t row_blocks, int32_t col_blocks, double* out) {
    if (!out || m < 1 || n < 1 || row_blocks < 1 || col_blocks < 1) return ADMM_EINVAL;
    const double Nm = static_cast<double>(m), Np = static_cast<double>(n);
    const double M = row_blocks, N = col_blocks;
    out[0] = 2 * Np;
    out[1] = N * Nm;
    out[2] = N * Nm / M + 2 * Np / N;
    return ADMM_OK;
}

int admm_plan(int64_t m, int64_t n, int32_t row_blocks, int32_t col_blocks, int32_t num_sms,
              int32_t smem_limit, admm_plan_t* out, int32_t* cta_cols) {
    if (!out) return ADMM_EINVAL;
    int code = validate(m, n, row_blocks, col_blocks, 0.0, 1.0, ADMM_C64);
    if (code) return code;
    std::vector<int> ro, co;
    admm::balanced_offsets(m, row_blocks, ro);
    admm::balanced_offsets(n, col_blocks, co);
    Plan pl;
    const char* why = "";
    code = admm::make_plan(m, n, row_blocks, col_blocks, ro, co, num_sms, smem_limit, pl, &why);
    if (code) return fail(nullptr, code, "%s", why);
    out->ctas = pl.P;
    out->slab_cols = pl.wmax;
    out->chunks = pl.chunks;
    out->box_cols = pl.wbox;
    out->boxes_per_row = pl.nsub;
    out->rows_per_stage = pl.R;
    out->stages = pl.nstages;
    out->smem_bytes = pl.smem;
    out->max_blocks_per_slab = pl.njs;
    out->ld = pl.ld;
    out->groups = pl.groups;
    out->reserved = 0;
    if (cta_cols) {
        for (int c = 0; c < pl.P; ++c) {
            cta_cols[4 * c] = pl.cta_beg[c];
            cta_cols[4 * c + 1] = pl.cta_end[c];
            cta_cols[4 * c + 2] = pl.cta_own0[c];
            cta_cols[4 * c + 3] = pl.cta_own1[c];
        }
    }
    return ADMM_OK;
}

int admm_setup(admm_t** out, const void* H, const void* g, int64_t m, int64_t n,
               int32_t row_blocks, int32_t col_blocks, double lambda, double rho,
               int32_t h_dtype, void* stream) {
    return admm_setup_form(out, H, g, m, n, row_blocks, col_blocks, lambda, rho, h_dtype, ADMM_FORM_LEMMA,
                           stream);
}

int admm_setup_form(admm_t** out, const void* H, const void* g, int64_t m, int64_t n,
                    int32_t row_blocks, int32_t col_blocks, double lambda, double rho,
                    int32_t h_dtype, int32_t form, void* stream) {
    if (!out) return fail(nullptr, ADMM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!H || !g) return fail(nullptr, ADMM_EINVAL, "H and g must not be NULL");
    int code = validate(m, n, row_blocks, col_blocks, lambda, rho, h_dtype);
    if (code) return code;
    if (form != ADMM_FORM_LEMMA && form != ADMM_FORM_DIRECT && form != ADMM_FORM_AUTO)
        return fail(nullptr, ADMM_EINVAL, "form must be ADMM_FORM_LEMMA, ADMM_FORM_DIRECT or ADMM_FORM_AUTO");
    std::vector<int> ro, co;
    admm::balanced_offsets(m, row_blocks, ro);
    admm::balanced_offsets(n, col_blocks, co);
    int mimin = static_cast<int>(m), mimax = 0, njmax = 0;
    for (int i = 0; i < row_blocks; ++i) {
        mimin = std::min(mimin, ro[i + 1] - ro[i]);
        mimax = std::max(mimax, ro[i + 1] - ro[i]);
    }
    for (int j = 0; j < col_blocks; ++j) njmax = std::max(njmax, co[j + 1] - co[j]);
    if (form == ADMM_FORM_AUTO)   // Section III-B: the lemma only when blocks have fewer rows than columns
        form = (mimin >= njmax && njmax <= admm::kDirMaxCols) ? ADMM_FORM_DIRECT : ADMM_FORM_LEMMA;
    if (form == ADMM_FORM_DIRECT && njmax > admm::kDirMaxCols)
        return fail(nullptr, ADMM_EUNSUPPORTED, "the direct form takes column blocks of at most %d columns",
                    admm::kDirMaxCols);
    const bool direct = form == ADMM_FORM_DIRECT;

    admm_t* h = new admm_t();
    h->m = m;
    h->n = n;
    h->M = row_blocks;
    h->N = col_blocks;
    h->lambda = lambda;
    h->rho = rho;
    h->row_off = ro;
    h->col_off = co;
    h->form = form;
    cudaStream_t st = as_stream(stream);
    auto bail = [&](int c) {
        g_setup_error = h->err;
        free_all(h);
        delete h;
        return c;
    };
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaGetDevice"));
    int coop = 0;
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    const int P = row_blocks * col_blocks;
    if (!direct) {
        if (!coop) return bail(fail(h, ADMM_EUNSUPPORTED, "device has no cooperative launch"));
        const char* why = "";
        code = admm::make_plan(m, n, row_blocks, col_blocks, ro, co, h->num_sms, h->smem_optin, h->plan, &why);
        if (code) return bail(fail(h, code, "%s", why));
    } else {
        // no persistent kernel: the plan only carries the pitch and the block sizes
        h->plan = Plan();
        h->plan.ld = round_up(n, 32);
        h->plan.P = 1;
        h->plan.mimax = mimax;
        h->plan.kpmax = round_up(mimax, 4);
    }
    const Plan& pl = h->plan;

    // factor layout.  lemma: block b = (i, j) holds m_i x kp_i complex64,
    // kp_i = m_i rounded up to 4.  direct: n_j x kp_j, stored in the order of
    // the blocks of H^H (b' = j * M + i), which the factor kernels index
    h->kinv_off.resize(P);
    h->kinv_pitch.resize(P);
    std::vector<long long> dir_off(P);
    std::vector<int> dir_pitch(P);
    int64_t kel = 0;
    if (!direct) {
        for (int i = 0; i < row_blocks; ++i)
            for (int j = 0; j < col_blocks; ++j) {
                const int mi = ro[i + 1] - ro[i];
                const int kp = round_up(mi, 4);
                h->kinv_off[i * col_blocks + j] = kel;
                h->kinv_pitch[i * col_blocks + j] = kp;
                kel += static_cast<int64_t>(mi) * kp;
            }
    } else {
        for (int i = 0; i < row_blocks; ++i)
            for (int j = 0; j < col_blocks; ++j) {
                const int nj = co[j + 1] - co[j];
                const int kp = round_up(nj, 4);
                dir_off[i * col_blocks + j] = kel;
                dir_pitch[i * col_blocks + j] = kp;
                h->kinv_off[j * row_blocks + i] = kel;
                h->kinv_pitch[j * row_blocks + i] = kp;
                kel += static_cast<int64_t>(nj) * kp;
            }
    }
    h->kinv_elems = kel;

    const size_t ld = pl.ld;
    const size_t Nm = static_cast<size_t>(col_blocks) * m;
    const size_t scratch = direct ? 1 : Nm;   // gt, r, w and the partials of the persistent kernel
    bool ok = dalloc(&h->H, ld * m) == cudaSuccess && dalloc(&h->g, m) == cudaSuccess &&
              dalloc(&h->v, ld) == cudaSuccess && dalloc(&h->s, ld * row_blocks) == cudaSuccess &&
              dalloc(&h->u, ld * row_blocks) == cudaSuccess && dalloc(&h->ghat, 2 * Nm) == cudaSuccess &&
              dalloc(&h->gt, scratch) == cudaSuccess && dalloc(&h->r, scratch) == cudaSuccess &&
              dalloc(&h->w, scratch) == cudaSuccess && dalloc(&h->part, scratch * pl.P * pl.groups) == cudaSuccess &&
              dalloc(&h->kinv, kel) == cudaSuccess &&
              dalloc(&h->kinv_off_d, h->kinv_off.size()) == cudaSuccess &&
              dalloc(&h->res_part, static_cast<size_t>(pl.P) * 8) == cudaSuccess &&
              dalloc(&h->hist, static_cast<size_t>(h->hist_cap) * 5) == cudaSuccess &&
              dalloc(&h->k_done, 1) == cudaSuccess && dalloc(&h->bar, 2) == cudaSuccess &&
              dalloc(&h->status, 1) == cudaSuccess && dalloc(&h->stop_flag, 1) == cudaSuccess;
    // int tables in one allocation
    std::vector<int> ints;
    auto put = [&](const std::vector<int>& x) {
        const size_t at = ints.size();
        ints.insert(ints.end(), x.begin(), x.end());
        return at;
    };
    const size_t o_row = put(ro), o_col = put(co), o_cta = put(pl.cta_beg), o_end = put(pl.cta_end),
                 o_own0 = put(pl.cta_own0), o_own1 = put(pl.cta_own1), o_jlo = put(pl.cta_jlo),
                 o_nj = put(pl.cta_nj), o_jl = put(pl.j_cta_lo), o_jh = put(pl.j_cta_hi),
                 o_sl = put(pl.solve_lo), o_kp = put(h->kinv_pitch);
    ok = ok && dalloc(&h->ints_d, ints.size()) == cudaSuccess;
    if (ok && direct) ok = alloc_direct(h, dir_off, dir_pitch, njmax) == ADMM_OK;
    if (!ok) return bail(fail(h, ADMM_ENOMEM, "device allocation failed (%.1f MB for H, %.1f MB of factors)",
                              ld * m * 8 / 1e6, kel * 8 / 1e6));
    h->row_off_d = h->ints_d + o_row;
    h->col_off_d = h->ints_d + o_col;
    h->cta_col_d = h->ints_d + o_cta;
    h->cta_end_d = h->ints_d + o_end;
    h->cta_own0_d = h->ints_d + o_own0;
    h->cta_own1_d = h->ints_d + o_own1;
    h->cta_jlo_d = h->ints_d + o_jlo;
    h->cta_nj_d = h->ints_d + o_nj;
    h->j_cta_lo_d = h->ints_d + o_jl;
    h->j_cta_hi_d = h->ints_d + o_jh;
    h->solve_lo_d = h->ints_d + o_sl;
    h->kinv_pitch_d = h->ints_d + o_kp;
    h->state_bytes = static_cast<int64_t>((ld * (1 + 2 * row_blocks) + 2 * Nm + 3 * scratch + scratch * pl.P) *
                                          sizeof(float2)) + h->dir.bytes;

#define SETUP_CK(call)                                             \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return bail(cuda_fail(h, e_, #call)); \
    } while (0)

    SETUP_CK(cudaMemcpyAsync(h->ints_d, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    SETUP_CK(cudaMemcpyAsync(h->kinv_off_d, h->kinv_off.data(), h->kinv_off.size() * sizeof(long long),
                             cudaMemcpyHostToDevice, st));
    // H into the padded layout (zero padding columns)
    SETUP_CK(cudaMemsetAsync(h->H, 0, ld * m * sizeof(float2), st));
    if (h_dtype == ADMM_C64) {
        SETUP_CK(cudaMemcpy2DAsync(h->H, ld * sizeof(float2), H, n * sizeof(float2), n * sizeof(float2), m,
                                   cudaMemcpyDefault, st));
    } else {
        double2* tmp = nullptr;
        if (dalloc(&tmp, static_cast<size_t>(m) * n) != cudaSuccess)
            return bail(fail(h, ADMM_ENOMEM, "no room for the complex128 staging copy of H"));
        cudaError_t e2 = cudaMemcpyAsync(tmp, H, static_cast<size_t>(m) * n * sizeof(double2), cudaMemcpyDefault, st);
        if (e2 == cudaSuccess) e2 = admm::launch_pack_c128(tmp, m, n, h->H, ld, st);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
        cudaFree(tmp);
        if (e2 != cudaSuccess) return bail(cuda_fail(h, e2, "pack complex128 H"));
    }
    code = copy_vector_in(h, h->g, g, m, h_dtype, st);
    if (code) return bail(code);
    // non-finite inputs
    SETUP_CK(cudaMemsetAsync(h->status, 0, sizeof(int), st));
    SETUP_CK(admm::launch_finite_check(h->H, static_cast<int64_t>(ld) * m, h->status, st));
    SETUP_CK(admm::launch_finite_check(h->g, m, h->status, st));
    int flag = 0;
    SETUP_CK(cudaStreamSynchronize(st));
    SETUP_CK(cudaMemcpy(&flag, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return bail(fail(h, ADMM_ENONFINITE, "H or g holds NaN or Inf"));
    code = build_factors(h, st, h->H, h->kinv, true);
    if (code == ADMM_OK && direct) code = pack_direct_tiles(h, st);
    if (code) return bail(code);
    if (!direct) {
        code = encode_tensor_map(h);
        if (code) return bail(code);
        // opt into the device maximum: several handles share one kernel instance
        SETUP_CK(admm::prepare_iterate(pl.chunks, h->smem_optin, pl.groups));
        int per_sm = 0;
        admm::max_coresident_iterate(pl.chunks, pl.smem, &per_sm, pl.groups);
        if (per_sm * h->num_sms < pl.P)
            return bail(fail(h, ADMM_EUNSUPPORTED, "iteration kernel cannot keep %d CTAs resident", pl.P));
    } else {
        SETUP_CK(admm::prepare_direct(h->smem_optin));
        SETUP_CK(cudaStreamCreateWithFlags(&h->dir.cap, cudaStreamNonBlocking));
    }
    code = zero_state(h, st);
    if (code) return bail(code);
    SETUP_CK(cudaStreamSynchronize(st));
#undef SETUP_CK
    *out = h;
    return ADMM_OK;
}

int admm_iterate(admm_t* h, int32_t iters, void* stream) {
    if (!h || iters < 0) return h ? fail(h, ADMM_EINVAL, "iters must be >= 0") : ADMM_EINVAL;
    if (h->broken) return fail(h, ADMM_ECUDA, "handle is in an error state; call admm_reset");
    if (iters == 0) return ADMM_OK;
    if (h->form == ADMM_FORM_DIRECT) return run_direct(h, iters, 0, 0.0, 0.0, as_stream(stream));
    return run_kernel(h, iters, 0, 0.0, 0.0, as_stream(stream));
}

int admm_solve(admm_t* h, int32_t max_iter, double eps_abs, double eps_rel, int32_t* iters_done,
               void* stream) {
    if (!h || max_iter < 0 || !(eps_abs >= 0.0) || !(eps_rel >= 0.0))
        return h ? fail(h, ADMM_EINVAL, "bad solve arguments") : ADMM_EINVAL;
    if (h->broken) return fail(h, ADMM_ECUDA, "handle is in an error state; call admm_reset");
    const int64_t k0 = h->k;
    if (iters_done) *iters_done = 0;
    if (max_iter == 0) return ADMM_OK;
    cudaStream_t st = as_stream(stream);
    if (h->form == ADMM_FORM_DIRECT) {
        // batches of 64 iterations; the kernels of iterations after the
        // stopping test passed return at once
        CK(h, cudaMemsetAsync(h->stop_flag, 0, sizeof(int), st));
        CK(h, cudaMemsetAsync(h->dir.stop_pending, 0, sizeof(int), st));
        for (int left = max_iter; left > 0;) {
            const int batch = std::min(left, 64);
            const int c = run_direct(h, batch, 1, eps_abs, eps_rel, st);
            if (c) return c;
            left -= batch;
            int stop = 0;
            CK(h, cudaMemcpyAsync(&stop, h->stop_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(h, cudaStreamSynchronize(st));
            if (stop) break;
        }
        const int c = device_status(h, st);
        if (iters_done) *iters_done = static_cast<int32_t>(h->k - k0);
        return c;
    }
    int code = run_kernel(h, max_iter, 1, eps_abs, eps_rel, st);
    if (code) return code;
    {
        // a solve that stopped early already summed the record of its last iteration
        CK(h, cudaStreamSynchronize(st));
        long long kd = 0;
        CK(h, cudaMemcpy(&kd, h->k_done, sizeof(long long), cudaMemcpyDeviceToHost));
        if (kd - k0 < max_iter) h->pending = 0;
    }
    code = device_status(h, st);
    if (iters_done) *iters_done = static_cast<int32_t>(h->k - k0);
    return code;
}

int admm_get_v(admm_t* h, void* v, void* stream) {
    if (!h || !v) return h ? fail(h, ADMM_EINVAL, "v is NULL") : ADMM_EINVAL;
    CK(h, cudaMemcpyAsync(v, h->v, h->n * sizeof(float2), cudaMemcpyDefault, as_stream(stream)));
    return ADMM_OK;
}

int admm_get_u(admm_t* h, void* u, void* stream) {
    if (!h || !u) return h ? fail(h, ADMM_EINVAL, "u is NULL") : ADMM_EINVAL;
    CK(h, cudaMemcpy2DAsync(u, h->n * sizeof(float2), h->u, h->plan.ld * sizeof(float2),
                            h->n * sizeof(float2), h->M, cudaMemcpyDefault, as_stream(stream)));
    return ADMM_OK;
}

int admm_get_residuals(admm_t* h, double* out, int32_t cap, int32_t* count, void* stream) {
    if (!h || !out || !count || cap < 0) return h ? fail(h, ADMM_EINVAL, "bad arguments") : ADMM_EINVAL;
    *count = 0;
    const int code = device_status(h, as_stream(stream));
    const int64_t avail = std::min<int64_t>(h->k, h->hist_cap);
    const int64_t want = std::min<int64_t>(avail, cap);
    std::vector<double> ring(static_cast<size_t>(h->hist_cap) * 5);
    CK(h, cudaMemcpy(ring.data(), h->hist, ring.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int64_t q = 0; q < want; ++q) {
        const int64_t it = h->k - want + q;
        const size_t slot = static_cast<size_t>(it % h->hist_cap);
        std::memcpy(out + q * 5, ring.data() + slot * 5, 5 * sizeof(double));
    }
    *count = static_cast<int32_t>(want);
    return code;
}

int admm_set_g(admm_t* h, const void* g, int32_t h_dtype, void* stream) {
    if (!h || !g) return h ? fail(h, ADMM_EINVAL, "g is NULL") : ADMM_EINVAL;
    if (h_dtype != ADMM_C64 && h_dtype != ADMM_C128) return fail(h, ADMM_EINVAL, "bad dtype");
    if (h->k > 0) h->rec_valid = false;
    h->dir.c_valid = false;
    h->dir.q_valid = false;
    const int code = copy_vector_in(h, h->g, g, h->m, h_dtype, as_stream(stream));
    if (code == ADMM_OK && h->sh_g0)
        CK(h, cudaMemcpyAsync(h->sh_g0, h->g, h->m * sizeof(float2), cudaMemcpyDeviceToDevice, as_stream(stream)));
    return code;
}

int admm_set_lambda(admm_t* h, double lambda) {
    if (!h) return ADMM_EINVAL;
    if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(h, ADMM_EINVAL, "lambda must be finite and >= 0");
    h->lambda = lambda;
    if (h->k > 0) h->rec_valid = false;
    return ADMM_OK;
}

int admm_set_rho(admm_t* h, double rho, void* stream) {
    if (!h) return ADMM_EINVAL;
    if (!(rho > 0.0) || !std::isfinite(rho)) return fail(h, ADMM_EINVAL, "rho must be finite and > 0");
    cudaStream_t st = as_stream(stream);
    const double old = h->rho;
    h->rho = rho;
    int code = build_factors(h, st, h->H, h->kinv, true);
    if (code == ADMM_OK && h->H16) code = build_factors_f16(h, st);
    if (code == ADMM_OK) code = pack_direct_tiles(h, st);
    if (code) {
        h->rho = old;
        build_factors(h, st, h->H, h->kinv, true);
        if (h->H16) build_factors_f16(h, st);
        pack_direct_tiles(h, st);
        return code;
    }
    h->rec_valid = false;
    h->dir.q_valid = false;
    CK(h, admm::launch_scale(h->s, static_cast<int64_t>(h->plan.ld) * h->M, static_cast<float>(old / rho), st));
    CK(h, cudaStreamSynchronize(st));
    return ADMM_OK;
}

int admm_reset(admm_t* h, void* stream) {
    if (!h) return ADMM_EINVAL;
    cudaStream_t st = as_stream(stream);
    const int code = zero_state(h, st);
    if (code) return code;
    CK(h, cudaStreamSynchronize(st));
    return ADMM_OK;
}

int admm_get_state(admm_t* h, int64_t* k, void* v, void* s, void* ghat, void* stream) {
    if (!h) return ADMM_EINVAL;
    cudaStream_t st = as_stream(stream);
    const int code = device_status(h, st);
    if (code == ADMM_ETIMEOUT || code == ADMM_ECUDA) return code;
    if (k) *k = h->k;
    if (v) CK(h, cudaMemcpyAsync(v, h->v, h->n * sizeof(float2), cudaMemcpyDefault, st));
    if (s)
        CK(h, cudaMemcpy2DAsync(s, h->n * sizeof(float2), h->s, h->plan.ld * sizeof(float2),
                                h->n * sizeof(float2), h->M, cudaMemcpyDefault, st));
    if (ghat)
        CK(h, cudaMemcpyAsync(ghat, h->ghat + static_cast<size_t>(h->k & 1) * h->N * h->m,
                              static_cast<size_t>(h->N) * h->m * sizeof(float2), cudaMemcpyDefault, st));
    CK(h, cudaStreamSynchronize(st));
    return code;
}

int admm_set_state(admm_t* h, int64_t k, const void* v, const void* s, const void* ghat, void* stream) {
    if (!h || !v || !s || k < 0) return h ? fail(h, ADMM_EINVAL, "v and s are required, k >= 0") : ADMM_EINVAL;
    if (!ghat && h->N > 1) return fail(h, ADMM_EINVAL, "ghat is required when col_blocks > 1");
    cudaStream_t st = as_stream(stream);
    CK(h, cudaStreamSynchronize(st));
    CK(h, cudaMemcpyAsync(h->v, v, h->n * sizeof(float2), cudaMemcpyDefault, st));
    CK(h, cudaMemcpy2DAsync(h->s, h->plan.ld * sizeof(float2), s, h->n * sizeof(float2),
                            h->n * sizeof(float2), h->M, cudaMemcpyDefault, st));
    float2* cur = h->ghat + static_cast<size_t>(k & 1) * h->N * h->m;
    if (ghat)
        CK(h, cudaMemcpyAsync(cur, ghat, static_cast<size_t>(h->N) * h->m * sizeof(float2),
                              cudaMemcpyDefault, st));
    else
        CK(h, cudaMemsetAsync(cur, 0, static_cast<size_t>(h->N) * h->m * sizeof(float2), st));
    CK(h, cudaMemcpyAsync(h->k_done, &k, sizeof(long long), cudaMemcpyHostToDevice, st));
    CK(h, cudaStreamSynchronize(st));
    h->k = k;
    h->pending = 0;   // the restored state has no residual record of its own
    h->rec_valid = false;
    h->dir.q_valid = false;
    return ADMM_OK;
}

int admm_get_info(const admm_t* h, admm_info_t* info) {
    if (!h || !info) return ADMM_EINVAL;
    const Plan& pl = h->plan;
    info->m = h->m;
    info->n = h->n;
    info->ld = pl.ld;
    info->row_blocks = h->M;
    info->col_blocks = h->N;
    info->lambda = h->lambda;
    info->rho = h->rho;
    info->kappa = h->lambda / (h->M * h->rho);
    info->iterations = h->k;
    info->ctas = pl.P;
    info->rows_per_stage = h->use_f16 ? pl.R16 : pl.R;
    info->stages = h->use_f16 ? pl.nstages16 : pl.nstages;
    info->slab_cols = pl.wmax;
    info->smem_bytes = pl.smem;
    info->num_sms = h->num_sms;
    info->h_bytes = h->m * h->n * static_cast<int64_t>(sizeof(float2));
    info->factor_bytes = h->kinv_elems * static_cast<int64_t>(sizeof(float2));
    info->state_bytes = h->state_bytes;
    info->setup_gram_ms = h->gram_ms;
    info->setup_factor_ms = h->factor_ms;
    info->h_fp16 = h->use_f16;
    info->h16_ready = h->H16 ? 1 : 0;
    info->h16_bytes = h->H16 ? h->m * h->n * 4 : 0;
    info->l2_keep_bytes = h->l2_keep_bytes;
    info->factor_form = h->form;
    info->reserved = 0;
    if (h->form == ADMM_FORM_DIRECT) {
        // the factor pass: streamed (a ring of stages of four factor rows) or plain loads
        const DirectState& d = h->dir;
        info->ctas = d.fac_stream ? d.fac_ctas : d.ctas;
        info->rows_per_stage = d.fac_stream ? 4 : 0;
        info->stages = d.fac_stream ? d.fac_ns : 0;
        info->slab_cols = 0;
        info->smem_bytes = d.fac_stream ? static_cast<int32_t>(admm::stream_smem(d.fac_ns, d.fac_stage)) : 0;
        if (uses_tiles(d)) {
            // the tile pass: the lower-triangle tiles through a ring of 16-row pieces
            info->ctas = d.herm_ctas;
            info->rows_per_stage = admm::kDirTile;
            info->stages = admm::kHermSlots;
            info->smem_bytes = static_cast<int32_t>(admm::herm_smem_bytes());
            info->factor_bytes = d.ntiles * admm::kDirTile * admm::kDirTile * static_cast<int64_t>(sizeof(float2));
        }
    }
    return ADMM_OK;
}

int admm_set_option(admm_t* h, int32_t option, int64_t value) {
    if (!h) return ADMM_EINVAL;
    if (h->form == ADMM_FORM_DIRECT && value != 0 &&
        (option == ADMM_OPT_H_FP16 || option == ADMM_OPT_RECORD_ITERS || option == ADMM_OPT_TRACE_ITERS ||
         option == ADMM_OPT_BARRIER_EXTRA))
        return fail(h, ADMM_EUNSUPPORTED, "option %d needs the lemma form (the persistent kernel)", option);
    switch (option) {
        case ADMM_OPT_TIMEOUT_NS:
            if (value < 1000) return fail(h, ADMM_EINVAL, "timeout must be >= 1000 ns");
            h->timeout_ns = value;
            return ADMM_OK;
        case ADMM_OPT_HIST_CAP: {
            if (value < 1 || value > (1 << 24)) return fail(h, ADMM_EINVAL, "history capacity out of range");
            double* nh = nullptr;
            CK(h, dalloc(&nh, static_cast<size_t>(value) * 5));
            CK(h, cudaDeviceSynchronize());
            cudaFree(h->hist);
            h->hist = nh;
            h->hist_cap = static_cast<int>(value);
            CK(h, cudaMemset(h->hist, 0, static_cast<size_t>(value) * 5 * sizeof(double)));
            return ADMM_OK;
        }
        case ADMM_OPT_TRACE_ITERS: {
            if (value < 0 || value > (1 << 20)) return fail(h, ADMM_EINVAL, "trace length out of range");
            CK(h, cudaDeviceSynchronize());
            if (h->trace) cudaFree(h->trace);
            h->trace = nullptr;
            h->trace_iters = 0;
            if (value > 0) {
                CK(h, dalloc(&h->trace, static_cast<size_t>(value) * 16));
                CK(h, cudaMemset(h->trace, 0, static_cast<size_t>(value) * 16 * sizeof(long long)));
                h->trace_iters = static_cast<int>(value);
            }
            return ADMM_OK;
        }
        case ADMM_OPT_L2_KEEP_BYTES:
            if (value < 0) return fail(h, ADMM_EINVAL, "L2 keep bytes must be >= 0");
            h->l2_keep_bytes = value;
            return ADMM_OK;
        case ADMM_OPT_H_FP16: {
            if (value != 0 && value != 1) return fail(h, ADMM_EINVAL, "ADMM_OPT_H_FP16 takes 0 or 1");
            if (value == 1) {
                const int code = enable_f16(h);
                if (code) return code;
            }
            h->use_f16 = static_cast<int>(value);
            return ADMM_OK;
        }
        case ADMM_OPT_RECORD_ITERS:
            return set_record(h, value);
        case ADMM_OPT_L2_PREFETCH_BYTES:
            if (value < 0) return fail(h, ADMM_EINVAL, "L2 prefetch bytes must be >= 0");
            h->l2_prefetch_bytes = value;
            return ADMM_OK;
        case ADMM_OPT_DIR_FACTOR_PASS:
            if (value < 0 || value > 2) return fail(h, ADMM_EINVAL, "ADMM_OPT_DIR_FACTOR_PASS takes 0, 1 or 2");
            if (h->form != ADMM_FORM_DIRECT) return ADMM_OK;   // the lemma form has no factor pass
            if (value == 2 && !h->dir.herm)
                return fail(h, ADMM_EUNSUPPORTED,
                            "the tile pass needs blocks of %d columns or more and at most %d row blocks",
                            admm::kDirHermMinCols, admm::kDirHermMaxRowBlocks);
            if (h->dir.pass != static_cast<int>(value)) {
                CK(h, cudaStreamSynchronize(h->dir.cap));
                drop_direct_graphs(h->dir);
                h->dir.pass = static_cast<int>(value);
            }
            return ADMM_OK;
        case ADMM_OPT_BARRIER_EXTRA:
            if (value < 0 || value > 1024) return fail(h, ADMM_EINVAL, "barrier extra out of range");
            h->bar_extra = static_cast<int>(value);
            return ADMM_OK;
        default:
            return fail(h, ADMM_EINVAL, "unknown option %d", option);
    }
}

int admm_tune(admm_t* h, void* stream) {
    if (!h) return ADMM_EINVAL;
    if (h->broken) return fail(h, ADMM_ECUDA, "handle is in an error state; call admm_reset");
    if (h->form == ADMM_FORM_DIRECT) return ADMM_OK;   // nothing to tune: no L2 policy in the direct form
    cudaStream_t st = as_stream(stream);
    const int64_t mib = 1LL << 20;
    const int64_t cand[] = {0, 16 * mib, 32 * mib, 44 * mib, 52 * mib, 64 * mib, 80 * mib, 96 * mib};
    const int64_t hb = h->m * h->plan.ld * (h->use_f16 ? 4 : 8);
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    int64_t best = h->l2_keep_bytes;
    float best_ms = 1e30f;
    int code = ADMM_OK;
    for (int64_t keep : cand) {
        if (keep > hb) break;
        h->l2_keep_bytes = keep;
        for (int r = 0; r < 2 && code == ADMM_OK; ++r) code = run_kernel(h, 1, 0, 0.0, 0.0, st);
        cudaEventRecord(e0, st);
        for (int r = 0; r < 5 && code == ADMM_OK; ++r) code = run_kernel(h, 1, 0, 0.0, 0.0, st);
        cudaEventRecord(e1, st);
        if (code) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = keep;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->l2_keep_bytes = best;
    if (code) return code;
    code = device_status(h, st);
    if (code) return code;
    code = zero_state(h, st);
    if (code) return code;
    CK(h, cudaStreamSynchronize(st));
    return ADMM_OK;
}

int admm_get_trace(admm_t* h, int64_t* out, int32_t cap, int32_t* count, void* stream) {
    if (!h || !out || !count || cap < 0) return h ? fail(h, ADMM_EINVAL, "bad arguments") : ADMM_EINVAL;
    *count = 0;
    if (!h->trace) return fail(h, ADMM_EINVAL, "tracing is off (ADMM_OPT_TRACE_ITERS)");
    CK(h, cudaStreamSynchronize(as_stream(stream)));
    const int n = std::min(cap, h->trace_iters);
    std::vector<long long> buf(static_cast<size_t>(h->trace_iters) * 16);
    CK(h, cudaMemcpy(buf.data(), h->trace, buf.size() * sizeof(long long), cudaMemcpyDeviceToHost));
    for (int sel = 0; sel < 2; ++sel)
        for (int it = 0; it < n; ++it)
            for (int q = 0; q < 8; ++q)
                out[(static_cast<size_t>(sel) * n + it) * 8 + q] =
                    buf[(static_cast<size_t>(sel) * h->trace_iters + it) * 8 + q];
    *count = n;
    return ADMM_OK;
}

int admm_backward(admm_t* h, const void* grad_v, void* grad_g, double* grad_lambda, double* grad_rho,
                  void* stream) {
    if (!h || !grad_v || !grad_g || !grad_lambda || !grad_rho)
        return h ? fail(h, ADMM_EINVAL, "NULL argument") : ADMM_EINVAL;
    if (h->form == ADMM_FORM_DIRECT) return fail(h, ADMM_EUNSUPPORTED, "the reverse sweep needs the lemma form");
    cudaStream_t st = as_stream(stream);
    int code = device_status(h, st);
    if (code) return code;
    if (!h->rec_cap || !h->rec_valid || h->k < 1 || h->k > h->rec_cap)
        return fail(h, ADMM_EINVAL, "no recorded iterations: set ADMM_OPT_RECORD_ITERS, then iterate at most that "
                                    "many times from the reset state without changing g, lambda, rho or the mode");
    const Plan& pl = h->plan;
    const size_t ld = pl.ld, m = h->m, P = static_cast<size_t>(h->M) * h->N;
    int mimax = 0, njmax = 0;
    for (int i = 0; i < h->M; ++i) mimax = std::max(mimax, h->row_off[i + 1] - h->row_off[i]);
    for (int j = 0; j < h->N; ++j) njmax = std::max(njmax, h->col_off[j + 1] - h->col_off[j]);
    const float kappa = static_cast<float>(h->lambda / (h->M * h->rho));
    CK(h, cudaMemsetAsync(h->bVb, 0, ld * sizeof(float2), st));
    CK(h, cudaMemcpyAsync(h->bVb, grad_v, h->n * sizeof(float2), cudaMemcpyDefault, st));
    CK(h, cudaMemsetAsync(h->bSb, 0, ld * h->M * sizeof(float2), st));
    CK(h, cudaMemsetAsync(h->bGhb, 0, m * h->N * sizeof(float2), st));
    CK(h, cudaMemsetAsync(h->bdG, 0, m * sizeof(float2), st));
    CK(h, cudaMemsetAsync(h->bkbar, 0, sizeof(double), st));
    CK(h, cudaMemsetAsync(h->brbar, 0, sizeof(double), st));
    CK(h, cudaMemcpyAsync(h->bkappa, &kappa, sizeof(float), cudaMemcpyHostToDevice, st));
    admm::batch::StepArgs sa;
    std::memset(&sa, 0, sizeof sa);
    sa.m = static_cast<int>(m);
    sa.n = static_cast<int>(ld);   // row pitch of v, s and the records
    sa.M = h->M;
    sa.N = h->N;
    sa.P = static_cast<int>(P);
    sa.B = 1;
    sa.splits = 1;
    sa.mpitch = h->rec_pitch;
    sa.npitch = h->bnpitch;
    sa.row_off = h->row_off_d;
    sa.col_off = h->col_off_d;
    sa.Gt = h->bGt;
    sa.R = h->bR;
    sa.Ppart = h->bP;
    sa.W = h->bW;
    sa.Sig = h->bSig;
    sa.kappa = h->bkappa;
    sa.rho = static_cast<float>(h->rho);
    sa.inv_M = 1.0f / h->M;
    sa.upd_tile_off = h->bupd;
    sa.upd_tiles = h->bupd_tiles;
    sa.rec_a = h->rec_a;
    sa.rec_w = h->rec_w;
    sa.rec_cap = h->rec_cap;
    sa.Vb = h->bVb;
    sa.Sb = h->bSb;
    sa.Ghb = h->bGhb;
    sa.dG = h->bdG;
    sa.kbar = h->bkbar;
    sa.rbar = h->brbar;
    admm::ProdArgs pa;
    pa.M = h->M;
    pa.N = h->N;
    pa.ld = pl.ld;
    pa.mimax = mimax;
    pa.njmax = njmax;
    pa.mpitch = h->rec_pitch;
    pa.npitch = h->bnpitch;
    pa.row_off = h->row_off_d;
    pa.col_off = h->col_off_d;
    pa.H = h->H;
    pa.H16 = h->H16;
    pa.scales = h->scales;
    pa.kinv = h->rec_f16 ? h->kinv16 : h->kinv;
    pa.kinv_off = h->kinv_off_d;
    pa.kinv_pitch = h->kinv_pitch_d;
    const bool f16 = h->rec_f16 != 0;
    for (int64_t k = h->k - 1; k >= 0; --k) {
        sa.bk = static_cast<int>(k);
        CK(h, admm::batch::launch_bw_soft(sa, st));
        CK(h, admm::launch_bw_rows(pa, f16, h->bSig, h->bP, st));
        CK(h, admm::batch::launch_bw_wbar(sa, st));
        CK(h, admm::launch_bw_factor(pa, h->bR, h->bW, st));
        CK(h, admm::batch::launch_bw_rbar(sa, st));
        CK(h, admm::launch_bw_cols(pa, f16, h->bW, h->bSig, st));
        CK(h, admm::batch::launch_bw_state(sa, st));
        CK(h, admm::batch::launch_bw_gtilde(sa, st));
    }
    CK(h, cudaMemcpyAsync(grad_g, h->bdG, m * sizeof(float2), cudaMemcpyDefault, st));
    double kb = 0.0, rb = 0.0;
    CK(h, cudaMemcpyAsync(&kb, h->bkbar, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(h, cudaMemcpyAsync(&rb, h->brbar, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    const double Md = h->M;
    *grad_lambda = kb / (Md * h->rho);
    *grad_rho = rb - kb * h->lambda / (Md * h->rho * h->rho);
    return device_status(h, st);
}

int admm_status(admm_t* h, void* stream) {
    if (!h) return ADMM_EINVAL;
    return device_status(h, as_stream(stream));
}

// ---------------------------------------------------------------------------
// sharded iteration: this handle holds some of the blocks of a larger split
// (Section IV); the caller exchanges the sums between ranks
// ---------------------------------------------------------------------------

int admm_shard_enable(admm_t* h, int32_t row_blocks_total, void* stream) {
    if (!h) return ADMM_EINVAL;
    if (h->form == ADMM_FORM_DIRECT)
        return fail(h, ADMM_EUNSUPPORTED, "the sharded iteration runs the lemma form only");
    if (row_blocks_total < h->M) return fail(h, ADMM_EINVAL, "row_blocks_total must be >= the handle's row blocks");
    cudaStream_t st = as_stream(stream);
    if (!h->sh_g0) {
        const size_t ld = h->plan.ld;
        if (dalloc(&h->sh_g0, h->m) != cudaSuccess || dalloc(&h->sh_tloc, h->m) != cudaSuccess ||
            dalloc(&h->sh_tglob, h->m) != cudaSuccess || dalloc(&h->sh_sum, ld) != cudaSuccess ||
            dalloc(&h->sh_rec, 5) != cudaSuccess)
            return fail(h, ADMM_ENOMEM, "no room for the sharded-iteration buffers");
        CK(h, cudaMemcpyAsync(h->sh_g0, h->g, h->m * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        CK(h, cudaMemsetAsync(h->sh_sum, 0, ld * sizeof(float2), st));
        CK(h, cudaMemsetAsync(h->sh_tloc, 0, h->m * sizeof(float2), st));
    }
    h->sh_Mtot = row_blocks_total;
    CK(h, cudaStreamSynchronize(st));
    return ADMM_OK;
}

int admm_shard_ghat_sum(admm_t* h, void* t_local, void* stream) {
    if (!h || !t_local) return h ? fail(h, ADMM_EINVAL, "t_local is NULL") : ADMM_EINVAL;
    if (!h->sh_Mtot) return fail(h, ADMM_EINVAL, "admm_shard_enable first");
    cudaStream_t st = as_stream(stream);
    const float2* cur = h->ghat + static_cast<size_t>(h->k & 1) * h->N * h->m;
    CK(h, admm::launch_shard_ghat_sum(cur, h->N, h->m, h->sh_tloc, st));
    CK(h, cudaMemcpyAsync(t_local, h->sh_tloc, h->m * sizeof(float2), cudaMemcpyDefault, st));
    return ADMM_OK;
}

int admm_shard_set_exchange(admm_t* h, const void* t_global, void* stream) {
    if (!h || !t_global) return h ? fail(h, ADMM_EINVAL, "t_global is NULL") : ADMM_EINVAL;
    if (!h->sh_Mtot) return fail(h, ADMM_EINVAL, "admm_shard_enable first");
    cudaStream_t st = as_stream(stream);
    CK(h, cudaMemcpyAsync(h->sh_tglob, t_global, h->m * sizeof(float2), cudaMemcpyDefault, st));
    CK(h, admm::launch_shard_geff(h->sh_g0, h->sh_tglob, h->sh_tloc, h->m, h->g, st));
    return ADMM_OK;
}

int admm_shard_ustep(admm_t* h, void* sum_out, void* stream) {
    if (!h || !sum_out) return h ? fail(h, ADMM_EINVAL, "sum_out is NULL") : ADMM_EINVAL;
    if (!h->sh_Mtot) return fail(h, ADMM_EINVAL, "admm_shard_enable first");
    if (h->broken) return fail(h, ADMM_ECUDA, "handle is in an error state; call admm_reset");
    cudaStream_t st = as_stream(stream);
    if (h->pending) {
        const int code = device_status(h, st);
        if (code) return code;
    }
    const Plan& pl = h->plan;
    admm::IterArgs a;
    fill_args(h, pl, handle_buffers(h), 1, 0, 0.0, 0.0, a);
    a.shard_sum = h->sh_sum;
    a.pending_prev = 0;
    a.rec_a = nullptr;
    a.rec_w = nullptr;
    a.rec_cap = 0;
    a.trace = nullptr;
    const bool f16 = h->use_f16 != 0;
    cudaError_t e = admm::launch_iterate(f16 ? h->tmap16 : h->tmap, a, pl.chunks, pl.smem, st, f16);
    if (e != cudaSuccess) return cuda_fail(h, e, "cooperative launch of the sharded u-step");
    h->k += 1;
    h->pending = 0;
    h->rec_valid = false;
    CK(h, cudaMemcpyAsync(sum_out, h->sh_sum, h->n * sizeof(float2), cudaMemcpyDefault, st));
    return ADMM_OK;
}

int admm_shard_vstep(admm_t* h, const void* sum_global, double* rec, void* stream) {
    if (!h || !sum_global || !rec) return h ? fail(h, ADMM_EINVAL, "NULL argument") : ADMM_EINVAL;
    if (!h->sh_Mtot) return fail(h, ADMM_EINVAL, "admm_shard_enable first");
    cudaStream_t st = as_stream(stream);
    CK(h, cudaMemcpyAsync(h->sh_sum, sum_global, h->n * sizeof(float2), cudaMemcpyDefault, st));
    const double Mt = h->sh_Mtot;
    CK(h, admm::launch_shard_vstep(h->v, h->s, h->u, h->sh_sum, h->n, h->plan.ld, h->M,
                                   static_cast<float>(1.0 / Mt), static_cast<float>(h->lambda / (Mt * h->rho)),
                                   h->sh_rec, st));
    CK(h, cudaMemcpyAsync(rec, h->sh_rec, 5 * sizeof(double), cudaMemcpyDefault, st));
    CK(h, cudaStreamSynchronize(st));
    int code = 0;
    CK(h, cudaMemcpy(&code, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (code) {
        if (code == ADMM_ETIMEOUT) h->broken = 1;
        return fail(h, code, "device status raised during the sharded iteration");
    }
    if (!std::isfinite(rec[0] + rec[1] + rec[2] + rec[3] + rec[4]))
        return fail(h, ADMM_EDIVERGED, "the iterates became NaN or Inf");
    return ADMM_OK;
}

void admm_destroy(admm_t* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    free_all(h);
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// several problems in one persistent launch
// ---------------------------------------------------------------------------

struct admm_group {
    struct Prob {
        admm_t* h = nullptr;
        Plan pl;
        int* tabs = nullptr;
        float2* part = nullptr;
        double* res_part = nullptr;
        unsigned* bar = nullptr;
        CUtensorMap tmap, tmap16;
        int o_beg = 0, o_end = 0, o_own0 = 0, o_own1 = 0, o_jlo = 0, o_nj = 0, o_jl = 0, o_jh = 0, o_sl = 0;
    };
    struct Wave {
        std::vector<int> probs;
        int ctas = 0, chunks = 1, smem = 0;
        int* cta_map = nullptr;   // [ctas] problem index in the wave, then [ctas] local CTA index
    };
    std::vector<Prob> probs;
    std::vector<Wave> waves;
    // all waves in one cooperative launch (up to kMaxGroupWave problems): per
    // wave and CTA the problem (-1 idle), then per wave and CTA the local CTA
    int* all_map = nullptr;
    int all_ctas = 0, all_chunks = 1, all_smem = 0;
    bool one_launch = false;
    // that launch captured once into a CUDA graph (one kernel node); each call
    // updates the node's arguments and replays it
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node = nullptr;
    int graph_f16 = -1;    // H mode the graph was captured with (-1: none)
    bool graph_failed = false;
    std::string err;
};

namespace {

thread_local std::string g_group_error;

int gfail(admm_group_t* g, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (g) g->err = buf;
    else g_group_error = buf;
    return code;
}

void free_group(admm_group_t* g) {
    for (auto& p : g->probs) {
        void* ptrs[] = {p.tabs, p.part, p.res_part, p.bar};
        for (void* q : ptrs)
            if (q) cudaFree(q);
    }
    for (auto& w : g->waves)
        if (w.cta_map) cudaFree(w.cta_map);
    if (g->all_map) cudaFree(g->all_map);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
}

// tensor map of h's H (f16: its FP16 copy) with the box of plan pl
int encode_for(admm_t* h, const Plan& pl, bool f16, CUtensorMap* map) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return ADMM_ECUDA;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const size_t eb = f16 ? 4 : 8;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(pl.ld), static_cast<cuuint64_t>(h->m)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(pl.ld) * eb};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(f16 ? pl.wbox16 : pl.wbox), static_cast<cuuint32_t>(f16 ? pl.R16 : pl.R)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                        f16 ? h->H16 : static_cast<void*>(h->H), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? ADMM_OK : ADMM_ECUDA;
}

}  // namespace

extern "C" {

const char* admm_group_last_error(const admm_group_t* g) { return g ? g->err.c_str() : g_group_error.c_str(); }

int admm_group_setup(admm_group_t** out, admm_t* const* handles, int32_t count, void* stream) {
    (void)stream;
    if (!out || !handles || count < 1) return gfail(nullptr, ADMM_EINVAL, "need out, handles and count >= 1");
    *out = nullptr;
    for (int q = 0; q < count; ++q) {
        if (!handles[q]) return gfail(nullptr, ADMM_EINVAL, "handle %d is NULL", q);
        if (handles[q]->form == ADMM_FORM_DIRECT)
            return gfail(nullptr, ADMM_EUNSUPPORTED, "handle %d has the direct form (no persistent kernel)", q);
    }
    const int sms = handles[0]->num_sms, limit = handles[0]->smem_optin;
    admm_group_t* g = new admm_group_t();
    auto bail = [&](int c) {
        g_group_error = g->err;
        free_group(g);
        delete g;
        return c;
    };
    // smallest CTA count each problem runs well with (slabs of at most 512
    // columns: the 4-chunk kernel instance, which keeps its accumulators in
    // registers), and its work per iteration
    std::vector<int> pmin(count), pmax(count);
    std::vector<double> work(count);
    for (int q = 0; q < count; ++q) {
        admm_t* h = handles[q];
        const int ld = h->plan.ld;
        pmax[q] = std::max(1, std::min(sms, ld / 64));
        pmin[q] = 0;
        for (int P = std::min(pmax[q], std::max(1, (ld + 511) / 512)); P <= pmax[q]; ++P) {
            Plan pl;
            const char* why = "";
            if (admm::make_plan(h->m, h->n, h->M, h->N, h->row_off, h->col_off, P, limit, pl, &why, 0, 1) == ADMM_OK &&
                pl.P == P) {
                pmin[q] = P;
                break;
            }
        }
        if (!pmin[q]) return bail(gfail(g, ADMM_EUNSUPPORTED, "problem %d has no plan on fewer than %d CTAs", q, sms));
        work[q] = static_cast<double>(h->m) * ld + 1.0 * h->kinv_elems;
    }
    // waves: a problem whose two passes over H take several times the fixed
    // per-iteration cost (grid barriers, reductions: about 15 us) on the whole
    // GPU runs alone with every CTA it can use (sharing its wave with small
    // problems measured slower); the others, by decreasing work, go first fit
    // into shared waves at their minimum CTA counts
    g->probs.resize(count);
    std::vector<int> order(count);
    for (int q = 0; q < count; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
    std::vector<int> used;
    const double solo_work = 2.0e7;   // complex entries of H (and factors): about 45 us per iteration
    for (int q : order) {
        if (work[q] >= solo_work) {
            g->waves.emplace_back();
            g->waves.back().probs.push_back(q);
            pmin[q] = pmax[q];
            used.push_back(sms);
            continue;
        }
        size_t w = 0;
        while (w < g->waves.size() &&
               (used[w] + pmin[q] > sms || g->waves[w].probs.size() >= static_cast<size_t>(admm::kMaxGroupWave)))
            ++w;
        if (w == g->waves.size()) {
            g->waves.emplace_back();
            used.push_back(0);
        }
        g->waves[w].probs.push_back(q);
        used[w] += pmin[q];
    }
    // with every problem in one launch, all share one kernel instance: the
    // largest chunk count any problem's plan needs
    const bool one_launch = count <= admm::kMaxGroupWave;
    std::vector<std::vector<int>> wave_P(g->waves.size());
    int ch_all = 1;
    for (size_t wi = 0; wi < g->waves.size(); ++wi) {
        auto& w = g->waves[wi];
        // CTAs in proportion to the work, within [pmin, pmax], at most one per SM in total
        double tot = 0.0;
        for (int q : w.probs) tot += work[q];
        std::vector<int> P(w.probs.size());
        int sum = 0;
        for (size_t t = 0; t < w.probs.size(); ++t) {
            const int q = w.probs[t];
            P[t] = std::max(pmin[q], std::min(pmax[q], static_cast<int>(sms * work[q] / tot)));
            sum += P[t];
        }
        while (sum > sms) {
            int best = -1;
            for (size_t t = 0; t < P.size(); ++t)
                if (P[t] > pmin[w.probs[t]] && (best < 0 || P[t] * work[w.probs[best]] > P[best] * work[w.probs[t]]))
                    best = static_cast<int>(t);
            if (best < 0) break;
            --P[best];
            --sum;
        }
        // plans: first per problem, then all with the largest chunk count (one kernel instance)
        int ch = 1;
        for (size_t t = 0; t < P.size(); ++t) {
            admm_t* h = handles[w.probs[t]];
            Plan pl;
            const char* why = "";
            int code = admm::make_plan(h->m, h->n, h->M, h->N, h->row_off, h->col_off, P[t], limit, pl, &why, 0, 1);
            // the planner may settle on fewer CTAs than offered; try fewer offers until one fits
            while (code != ADMM_OK && P[t] > pmin[w.probs[t]]) {
                --P[t];
                code = admm::make_plan(h->m, h->n, h->M, h->N, h->row_off, h->col_off, P[t], limit, pl, &why, 0, 1);
            }
            if (code) return bail(gfail(g, code, "problem %d: %s", w.probs[t], why));
            ch = std::max(ch, pl.chunks);
        }
        w.chunks = ch;
        ch_all = std::max(ch_all, ch);
        wave_P[wi] = P;
    }
    // with one launch every problem keeps its own chunk count (the kernel
    // switches per problem)
    const bool own_chunks = one_launch;
    for (size_t wi = 0; wi < g->waves.size(); ++wi) {
        auto& w = g->waves[wi];
        std::vector<int>& P = wave_P[wi];
        const int ch = own_chunks ? 0 : w.chunks;
        w.ctas = 0;
        w.smem = 0;
        std::vector<int> cta_map;
        std::vector<int> cprob, clocal;
        for (size_t t = 0; t < P.size(); ++t) {
            const int q = w.probs[t];
            admm_t* h = handles[q];
            admm_group_t::Prob& pr = g->probs[q];
            pr.h = h;
            const char* why = "";
            int code = admm::make_plan(h->m, h->n, h->M, h->N, h->row_off, h->col_off, P[t], limit, pr.pl, &why, ch, 1);
            if (code) return bail(gfail(g, code, "problem %d with %d chunks: %s", q, ch, why));
            if (!own_chunks && pr.pl.chunks != w.chunks)
                return bail(gfail(g, ADMM_EUNSUPPORTED, "problem %d: %d chunks in a wave of %d", q, pr.pl.chunks, w.chunks));
            w.smem = std::max(w.smem, pr.pl.smem);
            for (int c = 0; c < pr.pl.P; ++c) {
                cprob.push_back(static_cast<int>(t));
                clocal.push_back(c);
            }
            w.ctas += pr.pl.P;
            // the plan's tables and scratch
            std::vector<int> it;
            auto put = [&](const std::vector<int>& x) {
                const size_t at = it.size();
                it.insert(it.end(), x.begin(), x.end());
                return static_cast<int>(at);
            };
            pr.o_beg = put(pr.pl.cta_beg);
            pr.o_end = put(pr.pl.cta_end);
            pr.o_own0 = put(pr.pl.cta_own0);
            pr.o_own1 = put(pr.pl.cta_own1);
            pr.o_jlo = put(pr.pl.cta_jlo);
            pr.o_nj = put(pr.pl.cta_nj);
            pr.o_jl = put(pr.pl.j_cta_lo);
            pr.o_jh = put(pr.pl.j_cta_hi);
            pr.o_sl = put(pr.pl.solve_lo);
            const size_t Nm = static_cast<size_t>(h->N) * h->m;
            if (dalloc(&pr.tabs, it.size()) != cudaSuccess || dalloc(&pr.part, Nm * pr.pl.P) != cudaSuccess ||
                dalloc(&pr.res_part, static_cast<size_t>(pr.pl.P) * 8) != cudaSuccess ||
                dalloc(&pr.bar, 2) != cudaSuccess)
                return bail(gfail(g, ADMM_ENOMEM, "device allocation failed for problem %d", q));
            if (cudaMemcpy(pr.tabs, it.data(), it.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemset(pr.bar, 0, 2 * sizeof(unsigned)) != cudaSuccess)
                return bail(gfail(g, ADMM_ECUDA, "copy of the plan tables failed"));
            if (encode_for(h, pr.pl, false, &pr.tmap) != ADMM_OK ||
                (h->H16 && encode_for(h, pr.pl, true, &pr.tmap16) != ADMM_OK))
                return bail(gfail(g, ADMM_ECUDA, "cuTensorMapEncodeTiled failed for problem %d", q));
        }
        if (w.ctas > sms) return bail(gfail(g, ADMM_EUNSUPPORTED, "a wave needs %d CTAs on %d SMs", w.ctas, sms));
        cta_map = cprob;
        cta_map.insert(cta_map.end(), clocal.begin(), clocal.end());
        if (dalloc(&w.cta_map, cta_map.size()) != cudaSuccess ||
            cudaMemcpy(w.cta_map, cta_map.data(), cta_map.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(gfail(g, ADMM_ENOMEM, "device allocation failed for a wave"));
    }
    if (own_chunks) {
        const int W = static_cast<int>(g->waves.size());
        int C = 0, smem = 0;
        for (const auto& w : g->waves) {
            C = std::max(C, w.ctas);
            smem = std::max(smem, w.smem);
        }
        std::vector<int> map(2 * static_cast<size_t>(W) * C, -1);
        for (int wi = 0; wi < W; ++wi) {
            int b = 0;
            for (int q : g->waves[wi].probs)
                for (int c = 0; c < g->probs[q].pl.P; ++c, ++b) {
                    map[static_cast<size_t>(wi) * C + b] = q;
                    map[static_cast<size_t>(W + wi) * C + b] = c;
                }
        }
        if (dalloc(&g->all_map, map.size()) != cudaSuccess ||
            cudaMemcpy(g->all_map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(gfail(g, ADMM_ENOMEM, "device allocation failed for the launch map"));
        g->all_ctas = C;
        g->all_chunks = ch_all;
        g->all_smem = smem;
        g->one_launch = true;
    }
    *out = g;
    return ADMM_OK;
}

namespace {

// the last residual record of each problem's launch, from its group plan's partials
int finalize_group_records(admm_group_t* g, const std::vector<int>& probs, int iters, cudaStream_t st) {
    for (int q : probs) {
        admm_group_t::Prob& pr = g->probs[q];
        admm_t* h = pr.h;
        h->k += iters;
        admm::IterArgs a;
        std::memset(&a, 0, sizeof a);
        a.M = h->M;
        a.n = static_cast<int>(h->n);
        a.P = pr.pl.P;
        a.rho_d = h->rho;
        a.res_part = pr.res_part;
        a.hist = h->hist;
        a.hist_cap = h->hist_cap;
        a.status = h->status;
        const cudaError_t e = admm::launch_finalize(a, h->k - 1, st);
        if (e != cudaSuccess) return gfail(g, ADMM_ECUDA, "finalize failed: %s", cudaGetErrorString(e));
        h->pending = 0;
    }
    return ADMM_OK;
}

// arguments of problem q of the group for a launch of `iters` iterations
int group_args(admm_group_t* g, int q, int iters, bool f16, int chunks, cudaStream_t st, admm::IterArgs& a,
               CUtensorMap& map) {
    admm_group_t::Prob& pr = g->probs[q];
    admm_t* h = pr.h;
    if (h->broken) return gfail(g, ADMM_ECUDA, "problem %d is in an error state", q);
    if ((h->use_f16 != 0) != f16) return gfail(g, ADMM_EINVAL, "the problems of a group launch must share the H mode");
    if (h->pending) {
        const int code = device_status(h, st);
        if (code) return gfail(g, code, "problem %d: %s", q, h->err.c_str());
    }
    const int* T = pr.tabs;
    PlanBuffers b{T + pr.o_beg, T + pr.o_end, T + pr.o_own0, T + pr.o_own1, T + pr.o_jlo, T + pr.o_nj,
                  T + pr.o_jl, T + pr.o_jh, T + pr.o_sl, pr.part, pr.res_part, pr.bar};
    fill_args(h, pr.pl, b, iters, 0, 0.0, 0.0, a);
    a.trace = nullptr;
    map = f16 ? pr.tmap16 : pr.tmap;
    if (!admm::group_stage_geometry_ok(a, chunks, f16))
        return gfail(g, ADMM_EUNSUPPORTED, "inconsistent stage geometry for problem %d", q);
    return ADMM_OK;
}

}  // namespace

int admm_group_iterate(admm_group_t* g, int32_t iters, void* stream) {
    if (!g || iters < 0) return g ? gfail(g, ADMM_EINVAL, "iters must be >= 0") : ADMM_EINVAL;
    if (iters == 0) return ADMM_OK;
    cudaStream_t st = as_stream(stream);
    if (g->one_launch) {
        const bool f16 = g->probs[0].h->use_f16 != 0;
        std::vector<admm::GroupParams> gpv(1);   // ~30 KB: on the heap
        admm::GroupParams& gp = gpv[0];
        std::memset(&gp, 0, sizeof gp);
        const int count = static_cast<int>(g->probs.size());
        gp.count = count;
        std::vector<int> all(count);
        for (int q = 0; q < count; ++q) {
            all[q] = q;
            const int code = group_args(g, q, iters, f16, g->probs[q].pl.chunks, st, gp.a[q], gp.tmap[q]);
            if (code) return code;
            // a CTA that reaches a later wave's problem early waits at its first
            // grid barrier while the earlier waves finish
            gp.a[q].timeout_ns += 10000000000LL;
        }
        const int W = static_cast<int>(g->waves.size());
        cudaError_t e = admm::prepare_waves(g->all_chunks, f16, g->all_smem);
        if (e != cudaSuccess) return gfail(g, ADMM_ECUDA, "group launch setup failed: %s", cudaGetErrorString(e));
        if (g->graph_f16 != (f16 ? 1 : 0) && !g->graph_failed) {
            // capture the cooperative launch once (per H mode) into a graph
            if (g->exec) cudaGraphExecDestroy(g->exec);
            if (g->graph) cudaGraphDestroy(g->graph);
            g->exec = nullptr;
            g->graph = nullptr;
            g->graph_f16 = -1;
            cudaStream_t cap = nullptr;
            cudaError_t c = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
            if (c == cudaSuccess) c = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (c == cudaSuccess) {
                const cudaError_t c2 = admm::launch_waves(gp, g->all_map, W, g->all_ctas, g->all_chunks, f16,
                                                          g->all_smem, cap);
                c = cudaStreamEndCapture(cap, &g->graph);
                if (c2 != cudaSuccess) c = c2;
            }
            size_t nodes = 1;
            if (c == cudaSuccess) c = cudaGraphGetNodes(g->graph, &g->node, &nodes);
            if (c == cudaSuccess && nodes != 1) c = cudaErrorInvalidValue;
            if (c == cudaSuccess) c = cudaGraphInstantiate(&g->exec, g->graph, 0);
            if (cap) cudaStreamDestroy(cap);
            if (c == cudaSuccess) {
                g->graph_f16 = f16 ? 1 : 0;
            } else {
                // no graph: launch directly from now on
                cudaGetLastError();
                if (g->exec) cudaGraphExecDestroy(g->exec);
                if (g->graph) cudaGraphDestroy(g->graph);
                g->exec = nullptr;
                g->graph = nullptr;
                g->graph_failed = true;
            }
        }
        if (g->exec) {
            // this call's arguments (iteration counts, history slots) into the captured node
            cudaKernelNodeParams kp;
            std::memset(&kp, 0, sizeof kp);
            const int* map = g->all_map;
            int waves = W;
            void* args[] = {&gp, const_cast<int**>(&map), &waves};
            kp.func = admm::waves_kernel(g->all_chunks, f16);
            kp.gridDim = dim3(g->all_ctas);
            kp.blockDim = dim3(admm::kIterThreads);
            kp.sharedMemBytes = static_cast<unsigned>(g->all_smem);
            kp.kernelParams = args;
            e = cudaGraphExecKernelNodeSetParams(g->exec, g->node, &kp);
            if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, st);
        } else {
            e = admm::launch_waves(gp, g->all_map, W, g->all_ctas, g->all_chunks, f16, g->all_smem, st);
        }
        if (e != cudaSuccess) return gfail(g, ADMM_ECUDA, "group launch failed: %s", cudaGetErrorString(e));
        return finalize_group_records(g, all, iters, st);
    }
    for (auto& w : g->waves) {
        const bool f16 = g->probs[w.probs[0]].h->use_f16 != 0;
        std::vector<admm::GroupParams> gpv(1);   // ~30 KB: on the heap
        admm::GroupParams& gp = gpv[0];
        std::memset(&gp, 0, sizeof gp);
        gp.count = static_cast<int>(w.probs.size());
        for (size_t t = 0; t < w.probs.size(); ++t) {
            admm_group_t::Prob& pr = g->probs[w.probs[t]];
            admm_t* h = pr.h;
            if (h->broken) return gfail(g, ADMM_ECUDA, "problem %d is in an error state", w.probs[t]);
            if ((h->use_f16 != 0) != f16) return gfail(g, ADMM_EINVAL, "the problems of a wave must share the H mode");
            if (h->pending) {
                const int code = device_status(h, st);
                if (code) return gfail(g, code, "problem %d: %s", w.probs[t], h->err.c_str());
            }
            const int* T = pr.tabs;
            PlanBuffers b{T + pr.o_beg, T + pr.o_end, T + pr.o_own0, T + pr.o_own1, T + pr.o_jlo, T + pr.o_nj,
                          T + pr.o_jl, T + pr.o_jh, T + pr.o_sl, pr.part, pr.res_part, pr.bar};
            fill_args(h, pr.pl, b, iters, 0, 0.0, 0.0, gp.a[t]);
            gp.a[t].trace = nullptr;
            gp.tmap[t] = f16 ? pr.tmap16 : pr.tmap;
            if (!admm::group_stage_geometry_ok(gp.a[t], w.chunks, f16))
                return gfail(g, ADMM_EUNSUPPORTED, "inconsistent stage geometry for problem %d", w.probs[t]);
        }
        cudaError_t e = admm::launch_group(gp, w.cta_map, w.cta_map + w.ctas, w.ctas, w.chunks, f16, w.smem, st);
        if (e != cudaSuccess) return gfail(g, ADMM_ECUDA, "group launch failed: %s", cudaGetErrorString(e));
        for (size_t t = 0; t < w.probs.size(); ++t) {
            admm_group_t::Prob& pr = g->probs[w.probs[t]];
            admm_t* h = pr.h;
            h->k += iters;
            // the launch's last residual record, from this plan's partials
            admm::IterArgs a;
            std::memset(&a, 0, sizeof a);
            a.M = h->M;
            a.n = static_cast<int>(h->n);
            a.P = pr.pl.P;
            a.rho_d = h->rho;
            a.res_part = pr.res_part;
            a.hist = h->hist;
            a.hist_cap = h->hist_cap;
            a.status = h->status;
            e = admm::launch_finalize(a, h->k - 1, st);
            if (e != cudaSuccess) return gfail(g, ADMM_ECUDA, "finalize failed: %s", cudaGetErrorString(e));
            h->pending = 0;
        }
    }
    return ADMM_OK;
}

int admm_group_info(const admm_group_t* g, int32_t* waves, int32_t* ctas, int32_t cap) {
    if (!g || !waves) return ADMM_EINVAL;
    *waves = static_cast<int32_t>(g->waves.size());
    if (ctas)
        for (int q = 0; q < cap && q < static_cast<int>(g->probs.size()); ++q) ctas[q] = g->probs[q].pl.P;
    return ADMM_OK;
}

int admm_group_launches(const admm_group_t* g) {
    if (!g) return -1;
    return g->one_launch ? 1 : static_cast<int>(g->waves.size());
}

int admm_group_uses_graph(const admm_group_t* g) {
    if (!g) return -1;
    return g->exec ? 1 : 0;
}

void admm_group_destroy(admm_group_t* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    free_group(g);
    delete g;
}

}  // extern "C"
