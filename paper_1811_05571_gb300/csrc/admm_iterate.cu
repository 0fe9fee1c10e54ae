// Persistent cooperative kernel running whole ADMM iterations of the three
// splits of Sections III-A..C on one GPU.
//
// Per iteration (block b = (i, j), row block i, column block j):
//   A  r_b = gt_b - H_b z_b,  z_b = v_j - s_j^i        (first pass over H)
//   B  sum the per-CTA partial products, form gt_b = g_i - sum_{q!=j} ghat_iq
//   C  w_b = K_b^{-1} r_b  (cached factor, K_b = rho I + H_b H_b^H);
//      ghat_b = gt_b - rho w_b
//   D  u_b = z_b + H_b^H w_b                           (second pass over H),
//      v_j = S_kappa(mean_i u_j^i + mean_i s_j^i), s_j^i += u_j^i - v_j,
//      squared residual norms (FP32 per thread, FP64 across threads and CTAs).
// A-D is the paper's u-step (Eq. x_solution, x_solution_columns,
// x_solution_rows_columns) rewritten with the inversion lemma: with
// w = K^{-1}(gt - H z),  (H^H H + rho I)^{-1}(H^H gt + rho z) = z + H^H w
// and H u = gt - rho w, so the estimated data of Eq. (g_columns) and
// (g_rows_columns) costs no extra pass over H.
//
// Work layout: CTA c owns the column slab [cta_col[c], cta_col[c+1]) of H and
// the columns [cta_own0[c], cta_own1[c]) of every state vector for the whole
// launch.  Slabs are aligned to column blocks whenever there are no more
// column blocks than CTAs, so a slab meets one block; at an odd block
// boundary the 16-byte pair holding it is read by both neighbours and each
// masks the column it does not own.  A producer warp streams the slab row
// band by row band into a shared-memory ring with 2-D TMA tile loads
// (mbarrier completion); eight consumer warps each cover whole slab rows
// (16-byte complex pairs per lane) with paired FP32 FMAs.  Pass A walks rows
// upwards, pass D downwards, so the rows the previous pass read last are still
// in L2.  Only the m-length products cross CTAs, through three grid barriers
// per iteration whose waits are bounded by %globaltimer.
#include <cuda_fp16.h>

#include "admm_internal.h"
#include "ptx.cuh"

namespace admm {
namespace {

struct Misc {
    int stop;           // consumers -> producer: issue nothing more
    int issued;         // stages issued by the producer
    int producer_done;  // producer finished
    int bar_ok;         // broadcast of the last grid barrier's outcome
    int failed;         // a local bounded wait expired
    int pad[3];
    double red[kConsumerWarps][8];
};

__device__ __forceinline__ void csync() { named_sync<kConsumerThreads>(1); }

__device__ __forceinline__ float4 operator-(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float4 operator+(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float4 scale4(float4 a, float s) {
    return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}
__device__ __forceinline__ float4 lds128(const unsigned char* p) {
    return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float sq(float2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float2 shfl2(float2 v, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// Complex soft-threshold S_kappa(a) of Eq. (softhresholding): a - kappa a/|a|
// for |a| > kappa, else 0.
__device__ __forceinline__ float2 soft_threshold(float2 a, float kappa) {
    const float mag = hypotf(a.x, a.y);
    if (mag > kappa) {
        const float sc = 1.0f - kappa / mag;
        return make_float2(a.x * sc, a.y * sc);
    }
    return make_float2(0.0f, 0.0f);
}

// Sum of x[(lane >> 2) & 7] over the 32 lanes, left in every lane whose
// (lane >> 2) selects that value: 18 shuffles for eight values.
__device__ __forceinline__ float2 butterfly8(const float2 (&x)[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float2 y[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 keep = b4 ? x[q + 4] : x[q];
        const float2 send = b4 ? x[q] : x[q + 4];
        y[q] = keep + shfl2(send, 16);
    }
    float2 z[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float2 keep = b3 ? y[q + 2] : y[q];
        const float2 send = b3 ? y[q] : y[q + 2];
        z[q] = keep + shfl2(send, 8);
    }
    float2 w = (b2 ? z[1] : z[0]) + shfl2(b2 ? z[0] : z[1], 4);
    w = w + shfl2(w, 2);
    w = w + shfl2(w, 1);
    return w;
}

// Sense-reversing grid barrier over the consumer warps of every CTA.  The
// arrival counter is reset by the last arriver; waits are bounded.
__device__ bool grid_barrier(const IterArgs& a, Misc* misc) {
    csync();
    if (threadIdx.x == 0) {
        unsigned* count = a.bar;
        unsigned* gen = a.bar + 1;
        const unsigned expected = static_cast<unsigned>(a.P + a.bar_extra);
        const unsigned g0 = ld_acquire_gpu(gen);
        __threadfence();
        const unsigned prev = atomicAdd(count, 1u);
        if (prev + 1u == expected) {
            atomicExch(count, 0u);
            __threadfence();
            st_release_gpu(gen, g0 + 1u);
        } else {
            // tight spin (the CTA's other warps wait in bar.sync); the clock
            // and the status word are checked every 64 polls
            const long long t0 = global_timer_ns();
            for (unsigned polls = 1; ld_acquire_gpu(gen) == g0; ++polls) {
                if ((polls & 63u) == 0) {
                    if (ld_volatile(a.status) != 0) break;
                    if (global_timer_ns() - t0 > a.timeout_ns) {
                        raise_status(a.status, ADMM_ETIMEOUT);
                        break;
                    }
                }
            }
        }
        __threadfence();
        *reinterpret_cast<volatile int*>(&misc->bar_ok) =
            (ld_volatile(a.status) == 0 && !misc->failed) ? 1 : 0;
    }
    csync();
    return *reinterpret_cast<volatile int*>(&misc->bar_ok) != 0;
}

// ---------------------------------------------------------------------------
// producer warp (one lane)
// ---------------------------------------------------------------------------

__device__ bool producer_wait(uint64_t* bar, uint32_t parity, const IterArgs& a, Misc* misc) {
    const long long t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*reinterpret_cast<volatile int*>(&misc->stop)) return false;
        if (global_timer_ns() - t0 > a.timeout_ns) {
            raise_status(a.status, ADMM_ETIMEOUT);
            return false;
        }
    }
    return *reinterpret_cast<volatile int*>(&misc->stop) == 0;
}

// first row of stage `pos` of a pass (pass 0: blocks and rows ascending,
// pass 1: both descending); -1 past the end
__device__ int stage_row(const IterArgs& a, int pass, int pos) {
    for (int bi = 0; bi < a.M; ++bi) {
        const int i = pass == 0 ? bi : a.M - 1 - bi;
        const int r0 = a.row_off[i], r1 = a.row_off[i + 1];
        const int nb = (r1 - r0 + a.R - 1) / a.R;
        if (pos < nb) return r0 + (pass == 0 ? pos : nb - 1 - pos) * a.R;
        pos -= nb;
    }
    return -1;
}

__device__ void producer(const CUtensorMap* tmap, const IterArgs& a, uint64_t* full,
                         uint64_t* empty, Misc* misc, unsigned char* ring, int c_beg_slab) {
    prefetch_tensormap(tmap);
    // 4-byte elements: start at a multiple of 4 columns (x * 4 bytes a multiple of 16)
    const int c_beg = a.elem_bytes == 4 ? (c_beg_slab & ~3) : c_beg_slab;
    // The last keep_stages stages of every pass keep the normal L2 priority:
    // the next pass walks the rows in the opposite order and finds them in
    // L2.  All other stages are streamed evict_first so they do not displace
    // them, and once read the kept lines age out like any other line.
    const uint64_t pol_first = policy_evict_first();
    int per_pass = 0;
    for (int i = 0; i < a.M; ++i) per_pass += (a.row_off[i + 1] - a.row_off[i] + a.R - 1) / a.R;
    int stage = 0, slot = 0;   // stages issued; ring slot of the next one
    uint32_t pphase = 0;        // fill parity of that slot
    bool ok = true;
    for (int it = 0; it < a.iters && ok; ++it) {
        for (int pass = 0; pass < 2 && ok; ++pass) {
            int pos = 0;
            for (int bi = 0; bi < a.M && ok; ++bi) {
                const int i = pass == 0 ? bi : a.M - 1 - bi;
                const int r0 = a.row_off[i], r1 = a.row_off[i + 1];
                const int nb = (r1 - r0 + a.R - 1) / a.R;
                for (int bb = 0; bb < nb; ++bb, ++pos) {
                    const int b = pass == 0 ? bb : nb - 1 - bb;
                    const int y = r0 + b * a.R;
                    if (pos == 0 && a.prefetch_stages > 0) {
                        // while the consumers finish the previous pass and wait at
                        // the grid barriers, pull into L2 the rows this pass reads
                        // right after its L2-resident head (the kept tail of the
                        // previous pass) and after the stages the ring holds
                        const int q0 = max(a.keep_stages, a.nstages);
                        for (int q = q0; q < q0 + a.prefetch_stages; ++q) {
                            const int yq = stage_row(a, pass, q);
                            if (yq < 0) break;
                            for (int sb = 0; sb < a.nsub; ++sb) tma_prefetch_2d(tmap, c_beg + sb * a.wbox, yq);
                        }
                    }
                    const uint32_t parity = pphase ^ 1u;
                    if (!producer_wait(&empty[slot], parity, a, misc)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[slot], static_cast<uint32_t>(a.stage_bytes));
                    unsigned char* dst = ring + static_cast<size_t>(slot) * a.stage_stride;
                    const bool keep = a.keep_stages <= 0 || pos >= per_pass - a.keep_stages;
                    for (int sb = 0; sb < a.nsub; ++sb) {
                        if (keep)
                            tma_load_2d(dst + static_cast<size_t>(sb) * a.sub_bytes, tmap,
                                        c_beg + sb * a.wbox, y, &full[slot]);
                        else
                            tma_load_2d_hint(dst + static_cast<size_t>(sb) * a.sub_bytes, tmap,
                                             c_beg + sb * a.wbox, y, &full[slot], pol_first);
                    }
                    ++stage;
                    if (++slot == a.nstages) {
                        slot = 0;
                        pphase ^= 1u;
                    }
                    *reinterpret_cast<volatile int*>(&misc->issued) = stage;
                }
            }
        }
    }
    __threadfence_block();
    *reinterpret_cast<volatile int*>(&misc->producer_done) = 1;
}

// Record of iteration kabs (absolute index): FP64 sums of the per-CTA residual
// partials, written to the history ring; optional stopping test.  One warp.
__device__ void finalize_record(const IterArgs& a, long long kabs, int lane, bool check) {
    double acc[5] = {0, 0, 0, 0, 0};
    for (int c = lane; c < a.P; c += 32) {
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[q] += __ldcg(a.res_part + static_cast<size_t>(c) * 8 + q);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = warp_sum_d(acc[q]);
    if (lane == 0) {
        const double Md = static_cast<double>(a.M);
        double rec[5];
        rec[0] = acc[0];
        rec[1] = a.rho_d * a.rho_d * Md * acc[1];
        rec[2] = acc[2];
        rec[3] = Md * acc[3];
        rec[4] = acc[4];
        double* dst = a.hist + static_cast<size_t>(kabs % a.hist_cap) * 5;
#pragma unroll
        for (int q = 0; q < 5; ++q) dst[q] = rec[q];
        const bool bad = !isfinite(rec[0] + rec[1] + rec[2] + rec[3] + rec[4]);
        if (bad) raise_status(a.status, ADMM_EDIVERGED);
        if (check) {
            const double p = static_cast<double>(a.M) * static_cast<double>(a.n);
            const double eps_pri = sqrt(p) * a.eps_abs + a.eps_rel * fmax(sqrt(rec[2]), sqrt(rec[3]));
            const double eps_dual = sqrt(p) * a.eps_abs + a.eps_rel * a.rho_d * sqrt(rec[4]);
            const int stop = (!bad && sqrt(rec[0]) <= eps_pri && sqrt(rec[1]) <= eps_dual) ? 1 : 0;
            __stcg(a.stop_flag, stop);
        }
    }
}

// ---------------------------------------------------------------------------
// consumer warps
// ---------------------------------------------------------------------------

// rows of H per pipeline stage for a slab of CH 32-pair chunks (about 32 KB of
// complex64; FP16 stages take twice the rows, up to 64, to keep the bytes per
// stage: fewer, larger stages beat a deeper ring of small ones)
template <int CH, bool F16>
struct RowsOf {
    static constexpr int base = CH >= 8 ? 8 : 64 / CH;
    static constexpr int value = F16 ? (2 * base < 64 ? 2 * base : 64) : base;
};

// G column groups: the consumer warps split into G groups of kConsumerWarps/G
// warps; group q covers the q-th of G contiguous shares of the slab's pairs
// (so a lane holds CH chunks of a share instead of the whole slab), and the
// warps of a group take the rows of every stage in turn.  Each group's row
// sums of the first pass are separate partial products (P * G per row).
template <int CH, bool F16, int G>
struct Consumer {
    static constexpr int kWG = kConsumerWarps / G;    // warps per column group
    static constexpr int kR = RowsOf<CH, F16>::value;  // rows per stage
    static constexpr int kRPW = kR / kWG;             // rows per warp per stage
    static constexpr int kWin = 8 / kRPW;             // stages per 8-row reduction window
    static constexpr bool kPrefetch = CH <= 4;        // keep v and the next s_i in registers
    static_assert(kConsumerWarps % G == 0 && kR % kWG == 0 && kRPW <= 8 && 8 % kRPW == 0,
                  "rows per stage must split evenly over the warps of a group");

    const IterArgs& a;
    unsigned char* smem;
    Misc* misc;
    uint64_t* full;
    uint64_t* empty;
    const unsigned char* ring;
    int tid, warp, lane, cta;
    int grp, wg, pg0;     // column group, warp within it, first pair of its share
    int c_beg, npairs, jlo, nj, own0, own1, npmax;
    uint32_t valid;       // bit k: pair lane + 32k lies in this slab
    uint32_t owned;       // bit 2k+h: column h of pair lane + 32k is owned by this CTA
    uint64_t jl;          // 4 bits per chunk: block of column 0 (bits 0-1), column 1 (bits 2-3)
    int soff[CH];         // byte offset of pair lane + 32k inside a stage, row 0 (pairs outside
                          // the slab read pair 0: finite data, multiplied by a zero z)
    int slot;             // ring slot of the next stage
    uint32_t phase;       // parity of that slot's current fill

    __device__ Consumer(const IterArgs& args, unsigned char* sm, Misc* mi, uint64_t* f,
                        uint64_t* e, const unsigned char* rg, int cta_index)
        : a(args), smem(sm), misc(mi), full(f), empty(e), ring(rg) {
        tid = threadIdx.x;
        warp = tid >> 5;
        lane = tid & 31;
        cta = cta_index;
        grp = warp / kWG;
        wg = warp - grp * kWG;
        c_beg = a.cta_col[cta];
        npairs = (a.cta_end[cta] - c_beg) >> 1;
        const int share = (npairs + G - 1) / G;
        pg0 = min(npairs, grp * share);
        const int pg1 = min(npairs, pg0 + share);
        jlo = a.cta_jlo[cta];
        nj = a.cta_nj[cta];
        own0 = a.cta_own0[cta];
        own1 = a.cta_own1[cta];
        npmax = a.npitch;
        slot = 0;
        phase = 0;
        valid = 0;
        owned = 0;
        jl = 0;
        // columns of the stage box start at the slab start (FP16: rounded down to 4)
        const int shift = F16 ? (c_beg & 3) : 0;
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int p = pg0 + lane + 32 * k;
            const int rel = p < pg1 ? 2 * p + shift : shift;
            const int sb = rel / a.wbox;
            soff[k] = sb * a.sub_bytes + (rel - sb * a.wbox) * (F16 ? 4 : 8);
            if (p < pg1) {
                valid |= 1u << k;
                const int c0 = c_beg + 2 * p;
                uint64_t bits = 0;
                for (int h = 0; h < 2; ++h) {
                    if (c0 + h >= own0 && c0 + h < own1) owned |= 1u << (2 * k + h);
                    if (nj > 1) {
                        int j = jlo;
                        while (j + 1 < a.N && a.col_off[j + 1] <= c0 + h) ++j;
                        bits |= static_cast<uint64_t>(min(max(j - jlo, 0), 3)) << (2 * h);
                    }
                }
                jl |= bits << (4 * k);
            }
        }
    }

    __device__ __forceinline__ bool is_valid(int k) const { return (valid >> k) & 1u; }
    __device__ __forceinline__ bool is_owned(int k, int h) const { return (owned >> (2 * k + h)) & 1u; }
    __device__ __forceinline__ int jl_of(int k, int h) const {
        return static_cast<int>((jl >> (4 * k + 2 * h)) & 3u);
    }
    __device__ __forceinline__ int col_of(int k) const { return c_beg + 2 * (pg0 + lane + 32 * k); }
    // partial-product slot of this CTA's column group, and their count per row
    __device__ __forceinline__ int part_slot() const { return cta * G + grp; }
    __device__ __forceinline__ size_t part_pitch() const { return static_cast<size_t>(a.P) * G; }

    // one 16-byte complex pair of H (FP16 storage: 8 bytes, converted to FP32)
    __device__ __forceinline__ float4 load_pair(const unsigned char* rowp, int k) const {
        if (F16) {
            const uint2 raw = *reinterpret_cast<const uint2*>(rowp + soff[k]);
            const float2 c0 = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
            const float2 c1 = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
            return make_float4(c0.x, c0.y, c1.x, c1.y);
        }
        return lds128(rowp + soff[k]);
    }
    __device__ __forceinline__ float row_scale(int row) const {
        return F16 ? __ldg(a.scales + (row >> 6)) : 1.0f;
    }

    __device__ __forceinline__ void stamp(int it, int q) {
        if (a.trace && it < a.trace_iters && tid == 0 && (cta == 0 || cta == a.P - 1)) {
            const int sel = cta == 0 ? 0 : 1;
            a.trace[(static_cast<size_t>(sel) * a.trace_iters + it) * 8 + q] = global_timer_ns();
        }
    }

    // wait for the next stage; after a local failure, waits are skipped so that
    // every warp still reaches the same named barriers
    __device__ __forceinline__ const unsigned char* acquire_stage() {
        if (!*reinterpret_cast<volatile int*>(&misc->failed)) {
            if (!mbar_wait_bounded(&full[slot], phase, a.status, a.timeout_ns))
                *reinterpret_cast<volatile int*>(&misc->failed) = 1;
        }
        return ring + static_cast<size_t>(slot) * a.stage_stride;
    }
    __device__ __forceinline__ void release_stage() {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        if (++slot == a.nstages) {
            slot = 0;
            phase ^= 1u;
        }
    }

    // z_i for the lane's pairs, zero in columns this CTA does not own
    __device__ __forceinline__ float4 z_of(int k, float4 vv, float4 ss) const {
        float4 z = vv - ss;
        if (!is_owned(k, 0)) z.x = z.y = 0.f;
        if (!is_owned(k, 1)) z.z = z.w = 0.f;
        return z;
    }

    // ---- pass A (one column block per slab) --------------------------------
    __device__ void pass_up_single() {
        const int rowpitch = a.wbox * (F16 ? 4 : 8);
        float4 vreg[kPrefetch ? CH : 1], snext[kPrefetch ? CH : 1];
        if (kPrefetch) {
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                const int c = col_of(k);
                vreg[k] = is_valid(k) ? *reinterpret_cast<const float4*>(a.v + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                snext[k] = is_valid(k) ? *reinterpret_cast<const float4*>(a.s + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        for (int i = 0; i < a.M; ++i) {
            const int r0 = a.row_off[i], r1 = a.row_off[i + 1];
            // (z.re, z.re) and (z.im, z.im) for both columns of every pair
            float2 zr0[CH], zi0[CH], zr1[CH], zi1[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                if (is_valid(k)) {
                    if (kPrefetch) {
                        z = z_of(k, vreg[k], snext[k]);
                    } else {
                        const int c = col_of(k);
                        z = z_of(k, *reinterpret_cast<const float4*>(a.v + c),
                                 *reinterpret_cast<const float4*>(a.s + static_cast<size_t>(i) * a.ld + c));
                    }
                }
                zr0[k] = make_float2(z.x, z.x);
                zi0[k] = make_float2(z.y, z.y);
                zr1[k] = make_float2(z.z, z.z);
                zi1[k] = make_float2(z.w, z.w);
            }
            if (kPrefetch && i + 1 < a.M) {
#pragma unroll
                for (int k = 0; k < CH; ++k)
                    if (is_valid(k))
                        snext[k] = *reinterpret_cast<const float4*>(
                            a.s + static_cast<size_t>(i + 1) * a.ld + col_of(k));
            }
            const int nb = (r1 - r0 + kR - 1) / kR;
            for (int b0 = 0; b0 < nb; b0 += kWin) {
                float2 accA[8], accB[8];
#pragma unroll
                for (int v = 0; v < 8; ++v) accA[v] = accB[v] = make_float2(0.f, 0.f);
#pragma unroll
                for (int wi = 0; wi < kWin; ++wi) {
                    if (b0 + wi < nb) {
                        const unsigned char* buf = acquire_stage();
#pragma unroll
                        for (int q = 0; q < kRPW; ++q) {
                            const int v = wi * kRPW + q;
                            const unsigned char* rowp = buf + (wg + kWG * q) * rowpitch;
#pragma unroll
                            for (int k = 0; k < CH; ++k) {
                                // pairs outside the slab have z = 0
                                const float4 h = load_pair(rowp, k);
                                accA[v] = fma2(lo2(h), zr0[k], accA[v]);
                                accB[v] = fma2(lo2(h), zi0[k], accB[v]);
                                accA[v] = fma2(hi2(h), zr1[k], accA[v]);
                                accB[v] = fma2(hi2(h), zi1[k], accB[v]);
                            }
                        }
                        release_stage();
                    }
                }
                // h z = (sum h.re z.re - h.im z.im, sum h.im z.re + h.re z.im)
                float2 val[8];
#pragma unroll
                for (int v = 0; v < 8; ++v)
                    val[v] = make_float2(accA[v].x - accB[v].y, accA[v].y + accB[v].x);
                float2 sum = butterfly8(val, lane);
                const int v = lane >> 2;
                const int wi = v / kRPW, q = v - wi * kRPW;
                const int row = r0 + (b0 + wi) * kR + wg + kWG * q;
                if (F16) {
                    const float sc = row_scale(min(row, a.m - 1));
                    sum = make_float2(sum.x * sc, sum.y * sc);
                }
                if ((lane & 3) == 0 && b0 + wi < nb && row < r1)
                    stcg2(a.part + (static_cast<size_t>(jlo) * a.m + row) * part_pitch() + part_slot(), sum);
            }
        }
    }

    // ---- pass A (slab meeting several column blocks) -------------------------
    __device__ void pass_up_multi() {
        const int rowpitch = a.wbox * (F16 ? 4 : 8);
        for (int i = 0; i < a.M; ++i) {
            const int r0 = a.row_off[i], r1 = a.row_off[i + 1];
            float4 z[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                z[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (is_valid(k)) {
                    const int c = col_of(k);
                    z[k] = z_of(k, *reinterpret_cast<const float4*>(a.v + c),
                                *reinterpret_cast<const float4*>(a.s + static_cast<size_t>(i) * a.ld + c));
                }
            }
            const int nb = (r1 - r0 + kR - 1) / kR;
            for (int b = 0; b < nb; ++b) {
                const int y = r0 + b * kR;
                const unsigned char* buf = acquire_stage();
#pragma unroll
                for (int q = 0; q < kRPW; ++q) {
                    const int row = y + wg + kWG * q;
                    const unsigned char* rowp = buf + (wg + kWG * q) * rowpitch;
                    for (int jj = 0; jj < nj; ++jj) {
                        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k < CH; ++k) {
                            // pairs outside the slab have z = 0
                            const float2 z0 = jl_of(k, 0) == jj ? lo2(z[k]) : make_float2(0.f, 0.f);
                            const float2 z1 = jl_of(k, 1) == jj ? hi2(z[k]) : make_float2(0.f, 0.f);
                            const float4 h = load_pair(rowp, k);
                            cfma(acc, lo2(h), z0);
                            cfma(acc, hi2(h), z1);
                        }
                        acc = warp_sum(acc);
                        if (F16) {
                            const float sc = row_scale(min(row, a.m - 1));
                            acc = make_float2(acc.x * sc, acc.y * sc);
                        }
                        if (lane == 0 && row < r1)
                            stcg2(a.part + (static_cast<size_t>(jlo + jj) * a.m + row) * part_pitch() + part_slot(),
                                  acc);
                    }
                }
                release_stage();
            }
        }
    }

    // ---- phase B: r = gt - sum of partials; gt = g_i - sum_{q != j} ghat ----
    // Groups of red_lanes lanes sum the partials of one (column block, row).
    // The last CTA also sums the residual record of the previous iteration.
    __device__ void reduce_partials(int it) {
        if (cta == a.P - 1 && warp == 0) {
            if (it > 0) finalize_record(a, a.k0 + it - 1, lane, a.check_stop != 0);
            else if (a.pending_prev) finalize_record(a, a.k0 - 1, lane, false);
        }
        const size_t Nm = static_cast<size_t>(a.N) * a.m;
        const float2* ghat_cur = a.ghat + ((a.k0 + it) & 1) * Nm;
        const int L = a.red_lanes;
        const int groups = 32 / L;
        const int g = lane / L, gl = lane - (lane / L) * L;
        const int total = a.N * a.m;
        const int stride = a.P * kConsumerWarps * groups;
        for (int base = (cta * kConsumerWarps + warp) * groups; base < total; base += stride) {
            const int idx = base + g;
            float2 acc = make_float2(0.f, 0.f);
            int j = 0, row = 0;
            if (idx < total) {
                j = idx / a.m;
                row = idx - j * a.m;
                // every column group of the CTAs meeting block j left one partial
                const int lo = a.j_cta_lo[j] * G, hi = a.j_cta_hi[j] * G + G - 1;
                const float2* pp = a.part + static_cast<size_t>(idx) * part_pitch();
                // up to 16 loads per lane issued before any is summed
                for (int c0 = lo + gl; c0 <= hi; c0 += 16 * L) {
                    float2 x[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int c = c0 + u * L;
                        x[u] = c <= hi ? ldcg2(pp + c) : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < 16; ++u) acc = acc + x[u];
                }
            }
            for (int o = L >> 1; o >= 1; o >>= 1) acc = acc + shfl2(acc, o);
            if (idx < total && gl == 0) {
                float2 gtl = __ldg(a.g + row);
                for (int q = 0; q < a.N; ++q) {
                    if (q == j) continue;
                    const float2 gh = ldcg2(ghat_cur + static_cast<size_t>(q) * a.m + row);
                    gtl.x -= gh.x;
                    gtl.y -= gh.y;
                }
                stcg2(a.gt + idx, gtl);
                stcg2(a.r + idx, make_float2(gtl.x - acc.x, gtl.y - acc.y));
            }
        }
    }

    // ---- phase C: w_b = K_b^{-1} r_b, ghat_b = gt_b - rho w_b into the next
    // estimated-data buffer.  Two factor rows per warp, sixteen 16-byte loads
    // in flight per lane, factors streamed L2 evict_first.
    __device__ void apply_factors(int it) {
        float2* rS = reinterpret_cast<float2*>(smem + a.off_rs);
        const size_t Nm = static_cast<size_t>(a.N) * a.m;
        float2* ghat_nxt = a.ghat + ((a.k0 + it + 1) & 1) * Nm;
        const uint64_t pol = policy_evict_first();
        int idx = a.solve_lo[cta];
        const int end = a.solve_lo[cta + 1];
        while (idx < end) {
            const int j = idx / a.m;
            const int row = idx - j * a.m;
            int i = 0;
            while (a.row_off[i + 1] <= row) ++i;
            const int r0 = a.row_off[i], r1 = a.row_off[i + 1], mi = r1 - r0;
            const int seg_end = min(end, j * a.m + r1);
            const int b = i * a.N + j;
            const int kp = a.kinv_pitch[b];
            const float2* K = a.kinv + a.kinv_off[b];
            csync();
            for (int k = tid; k < kp; k += kConsumerThreads)
                rS[k] = k < mi ? ldcg2(a.r + static_cast<size_t>(j) * a.m + r0 + k) : make_float2(0.f, 0.f);
            csync();
            const float4* r4 = reinterpret_cast<const float4*>(rS);
            const int kp2 = kp >> 1;
            for (int q = idx + warp; q < seg_end; q += 2 * kConsumerWarps) {
                const int qb = q + kConsumerWarps;
                const bool has_b = qb < seg_end;
                const int rla = q - j * a.m - r0;
                const int rlb = has_b ? qb - j * a.m - r0 : rla;
                const float4* Ka = reinterpret_cast<const float4*>(K + static_cast<size_t>(rla) * kp);
                const float4* Kb = reinterpret_cast<const float4*>(K + static_cast<size_t>(rlb) * kp);
                float2 aa = make_float2(0.f, 0.f), ab = make_float2(0.f, 0.f);
                for (int t0 = 0; t0 < kp2; t0 += 256) {
                    float4 ka[8], kb[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int t = t0 + lane + 32 * u;
                        ka[u] = t < kp2 ? ldg_hint(Ka + t, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
                        kb[u] = (has_b && t < kp2) ? ldg_hint(Kb + t, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int t = t0 + lane + 32 * u;
                        if (t < kp2) {
                            const float4 x = r4[t];
                            cfma(aa, lo2(ka[u]), lo2(x));
                            cfma(aa, hi2(ka[u]), hi2(x));
                            cfma(ab, lo2(kb[u]), lo2(x));
                            cfma(ab, hi2(kb[u]), hi2(x));
                        }
                    }
                }
                aa = warp_sum(aa);
                ab = warp_sum(ab);
                if (lane == 0) {
                    stcg2(a.w + q, aa);
                    const float2 ga = ldcg2(a.gt + q);
                    stcg2(ghat_nxt + q, make_float2(ga.x - a.rho * aa.x, ga.y - a.rho * aa.y));
                    if (has_b) {
                        stcg2(a.w + qb, ab);
                        const float2 gb = ldcg2(a.gt + qb);
                        stcg2(ghat_nxt + qb, make_float2(gb.x - a.rho * ab.x, gb.y - a.rho * ab.y));
                    }
                    if (a.rec_w) {
                        const long long slot = a.k0 + it;
                        if (slot < a.rec_cap) {
                            float2* rw = a.rec_w + (static_cast<size_t>(slot) * a.M * a.N + i * a.N + j) * a.rec_pitch;
                            rw[rla] = aa;
                            if (has_b) rw[rlb] = ab;
                        }
                    }
                }
            }
            idx = seg_end;
        }
    }

    // ---- pass D: sigma_i = H_i^H w_i per slab column --------------------------
    __device__ void stage_w(int r0, int rows, int row_base_in_ws) {
        float2* wS = reinterpret_cast<float2*>(smem + a.off_ws);
        const int wpitch = a.ws_rows;
        // FP16 stream: fold the row scale of H into w (H_i^H w = sum conj(h16) (scale w))
        for (int jj = 0; jj < nj; ++jj)
            for (int k = tid; k < rows; k += kConsumerThreads) {
                float2 wv = ldcg2(a.w + static_cast<size_t>(jlo + jj) * a.m + r0 + k);
                if (F16) {
                    const float sc = row_scale(r0 + k);
                    wv = make_float2(wv.x * sc, wv.y * sc);
                }
                wS[jj * wpitch + row_base_in_ws + k] = wv;
            }
    }

    template <bool MULTI>
    __device__ void pass_down() {
        const int rowpitch = a.wbox * (F16 ? 4 : 8);
        const float2* wS = reinterpret_cast<const float2*>(smem + a.off_ws);
        float4* red = reinterpret_cast<float4*>(smem + a.off_red);
        float4* sigma = reinterpret_cast<float4*>(smem + a.off_sigma);
        const int wpitch = a.ws_rows;
        if (a.ws_all) {
            stage_w(0, a.m, 0);
            csync();
        }
        for (int bi = 0; bi < a.M; ++bi) {
            const int i = a.M - 1 - bi;
            const int r0 = a.row_off[i], r1 = a.row_off[i + 1], mi = r1 - r0;
            const int wbase = a.ws_all ? r0 : 0;   // row r of block i sits at wS[r - r0 + wbase]
            if (!a.ws_all) {
                stage_w(r0, mi, 0);
                csync();
            }
            // per pair: conj(h) w as (h.re w.re, h.im w.re) and (h.re w.im, h.im w.im)
            float2 aA0[CH], aB0[CH], aA1[CH], aB1[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) aA0[k] = aB0[k] = aA1[k] = aB1[k] = make_float2(0.f, 0.f);
            const int nb = (mi + kR - 1) / kR;
            for (int b = nb - 1; b >= 0; --b) {
                const int y = r0 + b * kR;
                const unsigned char* buf = acquire_stage();
#pragma unroll
                for (int q = 0; q < kRPW; ++q) {
                    const int rl = wg + kWG * q;
                    const bool ok = y + rl < r1;
                    const unsigned char* rowp = buf + rl * rowpitch;
                    if (!MULTI) {
                        const float2 wv = ok ? wS[y + rl - r0 + wbase] : make_float2(0.f, 0.f);
                        const float2 wre = make_float2(wv.x, wv.x), wim = make_float2(wv.y, wv.y);
#pragma unroll
                        for (int k = 0; k < CH; ++k) {
                            // sums of pairs outside the slab are never stored
                            const float4 h = load_pair(rowp, k);
                            aA0[k] = fma2(lo2(h), wre, aA0[k]);
                            aB0[k] = fma2(lo2(h), wim, aB0[k]);
                            aA1[k] = fma2(hi2(h), wre, aA1[k]);
                            aB1[k] = fma2(hi2(h), wim, aB1[k]);
                        }
                    } else {
                        float2 wv[kMaxBlocksPerSlab];
#pragma unroll
                        for (int jj = 0; jj < kMaxBlocksPerSlab; ++jj)
                            wv[jj] = (ok && jj < nj) ? wS[jj * wpitch + y + rl - r0 + wbase]
                                                     : make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k < CH; ++k) {
                            const float4 h = load_pair(rowp, k);
                            const float2 w0 = wv[jl_of(k, 0)], w1 = wv[jl_of(k, 1)];
                            aA0[k] = fma2(lo2(h), make_float2(w0.x, w0.x), aA0[k]);
                            aB0[k] = fma2(lo2(h), make_float2(w0.y, w0.y), aB0[k]);
                            aA1[k] = fma2(hi2(h), make_float2(w1.x, w1.x), aA1[k]);
                            aB1[k] = fma2(hi2(h), make_float2(w1.y, w1.y), aB1[k]);
                        }
                    }
                }
                release_stage();
            }
            // conj(h) w = (h.re w.re + h.im w.im, h.re w.im - h.im w.re); sum over warps
            // a group's warps sum through kWG rows of npmax pairs (the groups' pairs are disjoint)
            float4* rb = red + static_cast<size_t>(a.red_single ? 0 : (bi & 1)) * kWG * npmax;
            if (a.red_single) csync();   // the previous replica's sums have been read
#pragma unroll
            for (int k = 0; k < CH; ++k)
                if (is_valid(k))
                    rb[wg * npmax + pg0 + lane + 32 * k] =
                        make_float4(aA0[k].x + aB0[k].y, aB0[k].x - aA0[k].y,
                                    aA1[k].x + aB1[k].y, aB1[k].x - aA1[k].y);
            csync();
            for (int p = tid; p < npairs; p += kConsumerThreads) {
                float4 s = rb[p];
#pragma unroll
                for (int wq = 1; wq < kWG; ++wq) s = s + rb[wq * npmax + p];
                if (a.sigma_global) {
                    // an edge pair's other column belongs to the neighbouring CTA
                    const int c = c_beg + 2 * p;
                    const bool o0 = c >= own0 && c < own1, o1 = c + 1 >= own0 && c + 1 < own1;
                    float2* up = reinterpret_cast<float2*>(a.u + static_cast<size_t>(i) * a.ld + c);
                    if (o0 && o1) {
                        *reinterpret_cast<float4*>(up) = s;
                    } else {
                        if (o0) up[0] = lo2(s);
                        if (o1) up[1] = hi2(s);
                    }
                } else
                    sigma[static_cast<size_t>(i) * npmax + p] = s;
            }
        }
        csync();
    }

    // H_i^H w_i of pair p (same thread wrote it in pass_down)
    __device__ __forceinline__ float4 sigma_of(int i, int p) const {
        if (a.sigma_global)
            return *reinterpret_cast<const float4*>(a.u + static_cast<size_t>(i) * a.ld + c_beg + 2 * p);
        return reinterpret_cast<const float4*>(smem + a.off_sigma)[static_cast<size_t>(i) * npmax + p];
    }

    // ---- epilogue: u_i = z_i + sigma_i, v = S(mean u + mean s), s += u - v ----
    // ---- sharded epilogue: u_i = z_i + sigma_i and the sum over this handle's
    // replicas of u_i + s_i (the v and s update waits for the other ranks' sums)
    __device__ void shard_sums() {
        for (int p = tid; p < npairs; p += kConsumerThreads) {
            const int c = c_beg + 2 * p;
            const bool o0 = c >= own0 && c < own1, o1 = c + 1 >= own0 && c + 1 < own1;
            const float4 vv = *reinterpret_cast<const float4*>(a.v + c);
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int i = 0; i < a.M; ++i) {
                const float4 ss = *reinterpret_cast<const float4*>(a.s + static_cast<size_t>(i) * a.ld + c);
                const float4 uu = (vv - ss) + sigma_of(i, p);
                acc = acc + (uu + ss);
                float2* up = reinterpret_cast<float2*>(a.u + static_cast<size_t>(i) * a.ld + c);
                if (o0) up[0] = lo2(uu);
                if (o1) up[1] = hi2(uu);
            }
            float2* sp = reinterpret_cast<float2*>(a.shard_sum + c);
            if (o0) sp[0] = lo2(acc);
            if (o1) sp[1] = hi2(acc);
        }
    }

    __device__ void update_state(long long rec_slot) {
        if (a.shard_sum) {
            shard_sums();
            return;
        }
        float rp = 0.f, rdv = 0.f, u2 = 0.f, v2 = 0.f, s2 = 0.f;
        for (int p = tid; p < npairs; p += kConsumerThreads) {
            const int c = c_beg + 2 * p;
            const bool o0 = c >= own0 && c < own1, o1 = c + 1 >= own0 && c + 1 < own1;
            const float4 vv = *reinterpret_cast<const float4*>(a.v + c);
            float4 us = make_float4(0.f, 0.f, 0.f, 0.f), sb = us;
            for (int i = 0; i < a.M; ++i) {
                const float4 ss = *reinterpret_cast<const float4*>(a.s + static_cast<size_t>(i) * a.ld + c);
                us = us + ((vv - ss) + sigma_of(i, p));
                sb = sb + ss;
            }
            const float4 av = scale4(us + sb, a.inv_M);
            if (a.rec_a && rec_slot < a.rec_cap) {
                float2* ra = a.rec_a + static_cast<size_t>(rec_slot) * a.ld + c;
                if (o0 && o1) {
                    *reinterpret_cast<float4*>(ra) = av;
                } else {
                    if (o0) ra[0] = lo2(av);
                    if (o1) ra[1] = hi2(av);
                }
            }
            const float2 vn0 = soft_threshold(lo2(av), a.kappa);
            const float2 vn1 = soft_threshold(hi2(av), a.kappa);
            const float4 vn = make_float4(vn0.x, vn0.y, vn1.x, vn1.y);
            const float m0 = o0 ? 1.f : 0.f, m1 = o1 ? 1.f : 0.f;
            rdv += m0 * sq(make_float2(vn.x - vv.x, vn.y - vv.y)) + m1 * sq(make_float2(vn.z - vv.z, vn.w - vv.w));
            v2 += m0 * sq(vn0) + m1 * sq(vn1);
            for (int i = 0; i < a.M; ++i) {
                float4* sp = reinterpret_cast<float4*>(a.s + static_cast<size_t>(i) * a.ld + c);
                float4* up = reinterpret_cast<float4*>(a.u + static_cast<size_t>(i) * a.ld + c);
                const float4 ss = *sp;
                const float4 uu = (vv - ss) + sigma_of(i, p);
                const float4 sn = (ss + uu) - vn;
                rp += m0 * sq(make_float2(uu.x - vn.x, uu.y - vn.y)) + m1 * sq(make_float2(uu.z - vn.z, uu.w - vn.w));
                u2 += m0 * sq(lo2(uu)) + m1 * sq(hi2(uu));
                s2 += m0 * sq(lo2(sn)) + m1 * sq(hi2(sn));
                if (o0 && o1) {
                    *sp = sn;
                    *up = uu;
                } else {
                    float2* sp2 = reinterpret_cast<float2*>(sp);
                    float2* up2 = reinterpret_cast<float2*>(up);
                    if (o0) { sp2[0] = lo2(sn); up2[0] = lo2(uu); }
                    if (o1) { sp2[1] = hi2(sn); up2[1] = hi2(uu); }
                }
            }
            if (o0 && o1) {
                *reinterpret_cast<float4*>(a.v + c) = vn;
            } else {
                float2* vp = reinterpret_cast<float2*>(a.v + c);
                if (o0) vp[0] = vn0;
                if (o1) vp[1] = vn1;
            }
        }
        // FP32 within a warp (a few hundred positive terms), FP64 from the warp sums on
        float d[5] = {rp, rdv, u2, v2, s2};
#pragma unroll
        for (int q = 0; q < 5; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d[q] += __shfl_xor_sync(0xffffffffu, d[q], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 5; ++q) misc->red[warp][q] = static_cast<double>(d[q]);
        }
        csync();
        if (tid < 5) {
            double t = 0.0;
            for (int wq = 0; wq < kConsumerWarps; ++wq) t += misc->red[wq][tid];
            __stcg(a.res_part + static_cast<size_t>(cta) * 8 + tid, t);
        }
    }

    // wait until no TMA copy into this CTA's shared memory is in flight
    __device__ void drain() {
        csync();
        if (tid != 0) return;
        *reinterpret_cast<volatile int*>(&misc->stop) = 1;
        __threadfence_block();
        const long long t0 = global_timer_ns();
        while (*reinterpret_cast<volatile int*>(&misc->producer_done) == 0) {
            if (global_timer_ns() - t0 > a.timeout_ns) {
                raise_status(a.status, ADMM_ETIMEOUT);
                break;
            }
        }
        const int issued = *reinterpret_cast<volatile int*>(&misc->issued);
        for (int slot = 0; slot < a.nstages && slot < issued; ++slot) {
            const int last = slot + ((issued - 1 - slot) / a.nstages) * a.nstages;
            mbar_wait_bounded(&full[slot], (last / a.nstages) & 1, a.status, a.timeout_ns);
        }
    }

    __device__ void run() {
        const bool multi = nj > 1;
        int completed = 0;
        for (int it = 0; it < a.iters; ++it) {
            stamp(it, 0);
            if (multi) pass_up_multi(); else pass_up_single();
            stamp(it, 1);
            if (!grid_barrier(a, misc)) break;
            stamp(it, 2);
            reduce_partials(it);
            stamp(it, 3);
            if (!grid_barrier(a, misc)) break;
            stamp(it, 4);
            apply_factors(it);
            stamp(it, 5);
            if (!grid_barrier(a, misc)) break;
            stamp(it, 6);
            // the record of iteration it-1 was tested in phase B; stopping here
            // leaves v, s and the current estimated data of iteration it-1
            if (a.check_stop && it > 0 && __ldcg(a.stop_flag) != 0) break;
            if (multi) pass_down<true>(); else pass_down<false>();
            update_state(a.k0 + it);
            stamp(it, 7);
            completed = it + 1;
        }
        if (cta == 0 && tid == 0) a.k_done[0] = a.k0 + completed;
        drain();
    }
};

// One CTA of a problem's persistent iteration: local CTA index `cta` of a.P.
template <int CH, bool F16, int G>
__device__ __forceinline__ void iterate_body(const CUtensorMap* tmap, const IterArgs& a, int cta,
                                             unsigned char* smem) {
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.off_full);
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + a.off_empty);
    Misc* misc = reinterpret_cast<Misc*>(smem + a.off_misc);
    unsigned char* ring = smem + a.off_ring;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.nstages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        misc->stop = 0;
        misc->issued = 0;
        misc->producer_done = 0;
        misc->bar_ok = 1;
        misc->failed = 0;
        fence_mbarrier_init();
    }
    __syncthreads();
    if (warp == kConsumerWarps) {
        if ((threadIdx.x & 31) == 0)
            producer(tmap, a, full, empty, misc, ring, a.cta_col[cta]);
    } else {
        Consumer<CH, F16, G> c(a, smem, misc, full, empty, ring, cta);
        c.run();
    }
    // every copy has landed (the consumers drained the ring): the barriers can
    // be set up again for the CTA's next problem
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.nstages; ++s) {
            mbar_inval(&full[s]);
            mbar_inval(&empty[s]);
        }
    }
    __syncthreads();
}

template <int CH, bool F16, int G>
__global__ void __launch_bounds__(kIterThreads, 1)
    iterate_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ IterArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    iterate_body<CH, F16, G>(&tmap, a, blockIdx.x, smem);
}

// Several problems in one cooperative launch: CTA b runs local CTA cta_local[b]
// of problem cta_prob[b]; arguments and tensor maps are kernel parameters.
static_assert(sizeof(GroupParams) <= 32000, "group parameters exceed the kernel parameter space");

template <int CH, bool F16>
__global__ void __launch_bounds__(kIterThreads, 1)
    iterate_group_kernel(const __grid_constant__ GroupParams gp, const int* __restrict__ cta_prob,
                         const int* __restrict__ cta_local) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int p = cta_prob[blockIdx.x];
    iterate_body<CH, F16, 1>(&gp.tmap[p], gp.a[p], cta_local[blockIdx.x], smem);
}

// All waves of a group in one cooperative launch: in wave w, CTA b runs local
// CTA cta_map[W C + w C + b] of problem cta_map[w C + b] (-1: idle in that wave).
// A CTA that finishes its wave-w problem early goes on to its wave-(w+1)
// problem, whose grid barriers wait for that problem's other CTAs.  Each
// problem runs the body of its own chunk count (a.chunks).
template <bool F16>
__global__ void __launch_bounds__(kIterThreads, 1)
    iterate_waves_kernel(const __grid_constant__ GroupParams gp, const int* __restrict__ cta_map, int waves) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int C = gridDim.x;
    for (int w = 0; w < waves; ++w) {
        const int p = cta_map[w * C + blockIdx.x];
        if (p < 0) continue;
        const int local = cta_map[(waves + w) * C + blockIdx.x];
        switch (gp.a[p].chunks) {
            case 1: iterate_body<1, F16, 1>(&gp.tmap[p], gp.a[p], local, smem); break;
            case 2: iterate_body<2, F16, 1>(&gp.tmap[p], gp.a[p], local, smem); break;
            case 4: iterate_body<4, F16, 1>(&gp.tmap[p], gp.a[p], local, smem); break;
            case 8: iterate_body<8, F16, 1>(&gp.tmap[p], gp.a[p], local, smem); break;
            default: iterate_body<16, F16, 1>(&gp.tmap[p], gp.a[p], local, smem); break;
        }
    }
}

__global__ void __launch_bounds__(32) finalize_kernel(const __grid_constant__ IterArgs a, long long kabs) {
    finalize_record(a, kabs, threadIdx.x & 31, false);
}

template <int CH, bool F16, int G>
void* kernel_fn() {
    return reinterpret_cast<void*>(&iterate_kernel<CH, F16, G>);
}

// kernel instances: one column group with 1-16 chunks per lane, or two column
// groups of 8 chunks (slabs of more than 256 pairs)
template <bool F16>
void* pick_t(int chunks, int groups) {
    if (groups == 2) return chunks == 8 ? kernel_fn<8, F16, 2>() : nullptr;
    if (groups != 1) return nullptr;
    switch (chunks) {
        case 1: return kernel_fn<1, F16, 1>();
        case 2: return kernel_fn<2, F16, 1>();
        case 4: return kernel_fn<4, F16, 1>();
        case 8: return kernel_fn<8, F16, 1>();
        case 16: return kernel_fn<16, F16, 1>();
        default: return nullptr;
    }
}

void* pick(int chunks, bool f16 = false, int groups = 1) {
    return f16 ? pick_t<true>(chunks, groups) : pick_t<false>(chunks, groups);
}

template <int CH, bool F16>
void* group_fn() {
    return reinterpret_cast<void*>(&iterate_group_kernel<CH, F16>);
}

template <bool F16>
void* pick_group_t(int chunks) {
    switch (chunks) {
        case 1: return group_fn<1, F16>();
        case 2: return group_fn<2, F16>();
        case 4: return group_fn<4, F16>();
        case 8: return group_fn<8, F16>();
        case 16: return group_fn<16, F16>();
        default: return nullptr;
    }
}

void* pick_group(int chunks, bool f16) { return f16 ? pick_group_t<true>(chunks) : pick_group_t<false>(chunks); }

// the one-launch kernel runs problems of 1 to 16 chunks
template <bool F16>
void* pick_waves_t(int chunks) {
    if (chunks < 1 || chunks > 16) return nullptr;
    return reinterpret_cast<void*>(&iterate_waves_kernel<F16>);
}

}  // namespace

int rows_per_stage(int chunks, bool f16) {
    switch (chunks) {
        case 1: return f16 ? RowsOf<1, true>::value : RowsOf<1, false>::value;
        case 2: return f16 ? RowsOf<2, true>::value : RowsOf<2, false>::value;
        case 4: return f16 ? RowsOf<4, true>::value : RowsOf<4, false>::value;
        case 8: return f16 ? RowsOf<8, true>::value : RowsOf<8, false>::value;
        case 16: return f16 ? RowsOf<16, true>::value : RowsOf<16, false>::value;
        default: return 0;
    }
}

cudaError_t prepare_iterate(int chunks, int smem, int groups) {
    for (int f = 0; f < 2; ++f) {
        void* fn = pick(chunks, f == 1, groups);
        if (!fn) return cudaErrorInvalidValue;
        const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int max_coresident_iterate(int chunks, int smem, int* per_sm, int groups) {
    void* fn = pick(chunks, false, groups);
    if (!fn) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, kIterThreads, smem) != cudaSuccess)
        return 0;
    if (per_sm) *per_sm = blocks;
    return blocks;
}

cudaError_t launch_finalize(const IterArgs& a, long long kabs, cudaStream_t stream) {
    finalize_kernel<<<1, 32, 0, stream>>>(a, kabs);
    return cudaGetLastError();
}

// The mbarrier byte counts must equal what the TMA boxes deliver, and the ring
// slots must hold them: a mismatch would leave copies in flight when the CTAs
// exit, so the launch is refused instead.
bool stage_geometry_ok(const IterArgs& a, int chunks, bool f16) {
    const int eb = f16 ? 4 : 8;
    return (a.pgroups == 1 || (a.pgroups == 2 && chunks == 8)) && a.elem_bytes == eb && a.R == rows_per_stage(chunks, f16) && a.wbox >= 2 && a.wbox <= 256 &&
           (a.wbox * eb) % 16 == 0 && a.nsub >= 1 && a.sub_bytes == a.R * a.wbox * eb &&
           a.stage_bytes == a.sub_bytes * a.nsub && a.stage_bytes <= a.stage_stride &&
           a.nstages >= 2 && a.nstages <= 8 && (!f16 || a.scales != nullptr);
}

cudaError_t launch_iterate(const CUtensorMap& tmap, const IterArgs& a, int chunks, int smem,
                           cudaStream_t stream, bool f16) {
    if (!stage_geometry_ok(a, chunks, f16)) return cudaErrorInvalidValue;
    void* fn = pick(chunks, f16, a.pgroups);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {const_cast<CUtensorMap*>(&tmap), const_cast<IterArgs*>(&a)};
    return cudaLaunchCooperativeKernel(fn, dim3(a.P), dim3(kIterThreads), args,
                                       static_cast<size_t>(smem), stream);
}

cudaError_t launch_group(const GroupParams& gp, const int* cta_prob, const int* cta_local, int ctas, int chunks,
                         bool f16, int smem, cudaStream_t stream) {
    void* fn = pick_group(chunks, f16);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void* args[] = {const_cast<GroupParams*>(&gp), const_cast<int**>(&cta_prob), const_cast<int**>(&cta_local)};
    return cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(kIterThreads), args, static_cast<size_t>(smem), stream);
}

void* waves_kernel(int chunks, bool f16) { return f16 ? pick_waves_t<true>(chunks) : pick_waves_t<false>(chunks); }

cudaError_t prepare_waves(int chunks, bool f16, int smem) {
    void* fn = waves_kernel(chunks, f16);
    if (!fn) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_waves(const GroupParams& gp, const int* cta_map, int waves, int ctas, int chunks, bool f16,
                         int smem, cudaStream_t stream) {
    void* fn = waves_kernel(chunks, f16);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {const_cast<GroupParams*>(&gp), const_cast<int**>(&cta_map), &waves};
    return cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(kIterThreads), args, static_cast<size_t>(smem), stream);
}

bool group_stage_geometry_ok(const IterArgs& a, int chunks, bool f16) {
    return a.pgroups == 1 && stage_geometry_ok(a, chunks, f16);
}

}  // namespace admm

