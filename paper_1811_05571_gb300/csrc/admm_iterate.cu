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
//      FP64 partial squared residual norms.
// A-D is the paper's u-step (Eq. x_solution, x_solution_columns,
// x_solution_rows_columns) rewritten with the inversion lemma: with
// w = K^{-1}(gt - H z),  (H^H H + rho I)^{-1}(H^H gt + rho z) = z + H^H w
// and H u = gt - rho w, so the estimated data of Eq. (g_columns) and
// (g_rows_columns) costs no extra pass over H.
//
// Work layout: CTA c owns the column slab [cta_col[c], cta_col[c+1]) of H and
// of every state vector for the whole launch.  A producer warp streams that
// slab row band by row band into a shared-memory ring with 2-D TMA tile
// loads (mbarrier completion); eight consumer warps each cover whole slab rows
// (16-byte complex pairs per lane).  Pass A walks rows upwards, pass D
// downwards, so the rows the previous pass read last are still in L2.  Only
// the m-length products cross CTAs, through three grid barriers per
// iteration whose waits are bounded by %globaltimer.
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
__device__ __forceinline__ float4 scale4(float4 a, float s) {
    return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}
__device__ __forceinline__ float4 lds128(const unsigned char* p) {
    return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ double norm2(float2 a) {
    return static_cast<double>(a.x) * a.x + static_cast<double>(a.y) * a.y;
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
            const long long t0 = global_timer_ns();
            while (ld_acquire_gpu(gen) == g0) {
                if (ld_volatile(a.status) != 0) break;
                if (global_timer_ns() - t0 > a.timeout_ns) {
                    raise_status(a.status, ADMM_ETIMEOUT);
                    break;
                }
                __nanosleep(64);
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

__device__ void producer(const CUtensorMap* tmap, const IterArgs& a, uint64_t* full,
                         uint64_t* empty, Misc* misc, unsigned char* ring, int c_beg) {
    prefetch_tensormap(tmap);
    int stage = 0;
    bool ok = true;
    for (int it = 0; it < a.iters && ok; ++it) {
        for (int pass = 0; pass < 2 && ok; ++pass) {
            for (int bi = 0; bi < a.M && ok; ++bi) {
                const int i = pass == 0 ? bi : a.M - 1 - bi;
                const int r0 = a.row_off[i], r1 = a.row_off[i + 1];
                const int nb = (r1 - r0 + a.R - 1) / a.R;
                for (int bb = 0; bb < nb; ++bb) {
                    const int b = pass == 0 ? bb : nb - 1 - bb;
                    const int y = r0 + b * a.R;
                    const int slot = stage % a.nstages;
                    const uint32_t parity = ((stage / a.nstages) & 1) ^ 1;
                    if (!producer_wait(&empty[slot], parity, a, misc)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[slot], static_cast<uint32_t>(a.stage_bytes));
                    unsigned char* dst = ring + static_cast<size_t>(slot) * a.stage_stride;
                    for (int sb = 0; sb < a.nsub; ++sb)
                        tma_load_2d(dst + static_cast<size_t>(sb) * a.sub_bytes, tmap,
                                    c_beg + sb * a.wbox, y, &full[slot]);
                    ++stage;
                    *reinterpret_cast<volatile int*>(&misc->issued) = stage;
                }
            }
        }
    }
    __threadfence_block();
    *reinterpret_cast<volatile int*>(&misc->producer_done) = 1;
}

// ---------------------------------------------------------------------------
// consumer warps
// ---------------------------------------------------------------------------

template <int CH>
struct Consumer {
    const IterArgs& a;
    unsigned char* smem;
    Misc* misc;
    uint64_t* full;
    uint64_t* empty;
    const unsigned char* ring;
    int tid, warp, lane, cta;
    int c_beg, npairs, jlo, nj;
    uint32_t valid;       // bit k: pair lane + 32k lies in this slab
    uint64_t jl;          // 4 bits per chunk: jl of column 0 (bits 0-1), column 1 (bits 2-3)
    int soff[CH];         // byte offset of pair lane + 32k inside a stage, row 0
    int stage;            // stages consumed

    __device__ Consumer(const IterArgs& args, unsigned char* sm, Misc* mi, uint64_t* f,
                        uint64_t* e, const unsigned char* rg)
        : a(args), smem(sm), misc(mi), full(f), empty(e), ring(rg) {
        tid = threadIdx.x;
        warp = tid >> 5;
        lane = tid & 31;
        cta = blockIdx.x;
        c_beg = a.cta_col[cta];
        npairs = (a.cta_col[cta + 1] - c_beg) >> 1;
        jlo = a.cta_jlo[cta];
        nj = a.cta_nj[cta];
        stage = 0;
        valid = 0;
        jl = 0;
        const int ppb = a.wbox >> 1;
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int p = lane + 32 * k;
            const int sb = p / ppb;
            soff[k] = sb * a.sub_bytes + (p - sb * ppb) * 16;
            if (p < npairs) {
                valid |= 1u << k;
                const int c0 = c_beg + 2 * p;
                uint64_t bits = 0;
                for (int h = 0; h < 2; ++h) {
                    int j = jlo;
                    while (j + 1 < a.N && a.col_off[j + 1] <= c0 + h) ++j;
                    bits |= static_cast<uint64_t>(j - jlo) << (2 * h);
                }
                jl |= bits << (4 * k);
            }
        }
    }

    __device__ __forceinline__ bool is_valid(int k) const { return (valid >> k) & 1u; }
    __device__ __forceinline__ int jl_of(int k, int h) const {
        return static_cast<int>((jl >> (4 * k + 2 * h)) & 3u);
    }
    __device__ __forceinline__ int col_of(int k) const { return c_beg + 2 * (lane + 32 * k); }

    // wait for the next stage; after a local failure, waits are skipped so that
    // every warp still reaches the same named barriers
    __device__ __forceinline__ const unsigned char* acquire_stage(int& slot) {
        slot = stage % a.nstages;
        const uint32_t parity = (stage / a.nstages) & 1;
        if (!*reinterpret_cast<volatile int*>(&misc->failed)) {
            if (!mbar_wait_bounded(&full[slot], parity, a.status, a.timeout_ns))
                *reinterpret_cast<volatile int*>(&misc->failed) = 1;
        }
        return ring + static_cast<size_t>(slot) * a.stage_stride;
    }
    __device__ __forceinline__ void release_stage(int slot) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        ++stage;
    }

    // ---- pass A: partial products of H_b z_b per (row, column block) ------
    template <bool MULTI>
    __device__ void pass_rows_up() {
        const int rowpitch = a.wbox * 8;
        for (int i = 0; i < a.M; ++i) {
            const int r0 = a.row_off[i], r1 = a.row_off[i + 1];
            float4 z[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                if (is_valid(k)) {
                    const int c = col_of(k);
                    const float4 vv = *reinterpret_cast<const float4*>(a.v + c);
                    const float4 ss =
                        *reinterpret_cast<const float4*>(a.s + static_cast<size_t>(i) * a.ld + c);
                    z[k] = vv - ss;
                } else {
                    z[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            const int nb = (r1 - r0 + a.R - 1) / a.R;
            for (int b = 0; b < nb; ++b) {
                const int y = r0 + b * a.R;
                int slot;
                const unsigned char* buf = acquire_stage(slot);
                for (int t = warp; t < a.R; t += 2 * kConsumerWarps) {
                    const int ra = t, rb = t + kConsumerWarps;
                    const bool in_b = rb < a.R;
                    const bool oka = y + ra < r1, okb = in_b && (y + rb < r1);
                    if (!MULTI) {
                        float2 sa = make_float2(0.f, 0.f), sbv = make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k < CH; ++k) {
                            if (is_valid(k)) {
                                const float4 ha = lds128(buf + soff[k] + ra * rowpitch);
                                cfma(sa, make_float2(ha.x, ha.y), make_float2(z[k].x, z[k].y));
                                cfma(sa, make_float2(ha.z, ha.w), make_float2(z[k].z, z[k].w));
                                if (in_b) {
                                    const float4 hb = lds128(buf + soff[k] + rb * rowpitch);
                                    cfma(sbv, make_float2(hb.x, hb.y), make_float2(z[k].x, z[k].y));
                                    cfma(sbv, make_float2(hb.z, hb.w), make_float2(z[k].z, z[k].w));
                                }
                            }
                        }
                        sa = warp_sum(sa);
                        sbv = warp_sum(sbv);
                        if (lane == 0) {
                            const size_t base = static_cast<size_t>(jlo) * a.m;
                            if (oka)
                                stcg2(a.part + (base + y + ra) * a.P + cta, sa);
                            if (okb)
                                stcg2(a.part + (base + y + rb) * a.P + cta, sbv);
                        }
                    } else {
                        for (int jj = 0; jj < nj; ++jj) {
                            float2 sa = make_float2(0.f, 0.f), sbv = make_float2(0.f, 0.f);
#pragma unroll
                            for (int k = 0; k < CH; ++k) {
                                if (is_valid(k)) {
                                    const bool m0 = jl_of(k, 0) == jj, m1 = jl_of(k, 1) == jj;
                                    const float2 z0 = m0 ? make_float2(z[k].x, z[k].y)
                                                         : make_float2(0.f, 0.f);
                                    const float2 z1 = m1 ? make_float2(z[k].z, z[k].w)
                                                         : make_float2(0.f, 0.f);
                                    const float4 ha = lds128(buf + soff[k] + ra * rowpitch);
                                    cfma(sa, make_float2(ha.x, ha.y), z0);
                                    cfma(sa, make_float2(ha.z, ha.w), z1);
                                    if (in_b) {
                                        const float4 hb = lds128(buf + soff[k] + rb * rowpitch);
                                        cfma(sbv, make_float2(hb.x, hb.y), z0);
                                        cfma(sbv, make_float2(hb.z, hb.w), z1);
                                    }
                                }
                            }
                            sa = warp_sum(sa);
                            sbv = warp_sum(sbv);
                            if (lane == 0) {
                                const size_t base = static_cast<size_t>(jlo + jj) * a.m;
                                if (oka) stcg2(a.part + (base + y + ra) * a.P + cta, sa);
                                if (okb) stcg2(a.part + (base + y + rb) * a.P + cta, sbv);
                            }
                        }
                    }
                }
                release_stage(slot);
            }
        }
    }

    // ---- record of iteration k: FP64 sums over the CTAs, stopping test ------
    __device__ void finalize(int k) {
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
            double* dst = a.hist + static_cast<size_t>((a.k0 + k) % a.hist_cap) * 5;
#pragma unroll
            for (int q = 0; q < 5; ++q) dst[q] = rec[q];
            const bool bad = !isfinite(rec[0] + rec[1] + rec[2] + rec[3] + rec[4]);
            if (bad) raise_status(a.status, ADMM_EDIVERGED);
            if (a.check_stop) {
                const double p = static_cast<double>(a.M) * static_cast<double>(a.n);
                const double eps_pri =
                    sqrt(p) * a.eps_abs + a.eps_rel * fmax(sqrt(rec[2]), sqrt(rec[3]));
                const double eps_dual = sqrt(p) * a.eps_abs + a.eps_rel * a.rho_d * sqrt(rec[4]);
                const int stop = (!bad && sqrt(rec[0]) <= eps_pri && sqrt(rec[1]) <= eps_dual) ? 1 : 0;
                __stcg(a.stop_flag, stop);
            }
        }
    }

    // ---- phase B: r = gt - sum of partials; gt = g_i - sum_{q != j} ghat ----
    __device__ void reduce_partials(int it) {
        if (it > 0 && cta == 0 && warp == 0) finalize(it - 1);
        const int nw = a.P * kConsumerWarps;
        const int total = a.N * a.m;
        for (int idx = cta * kConsumerWarps + warp; idx < total; idx += nw) {
            const int j = idx / a.m;
            const int row = idx - j * a.m;
            const int lo = a.j_cta_lo[j], hi = a.j_cta_hi[j];
            const float2* pp = a.part + static_cast<size_t>(idx) * a.P;
            float2 acc = make_float2(0.f, 0.f);
            for (int c = lo + lane; c <= hi; c += 32) {
                const float2 x = ldcg2(pp + c);
                acc.x += x.x;
                acc.y += x.y;
            }
            acc = warp_sum(acc);
            if (lane == 0) {
                float2 gtl = __ldg(a.g + row);
                for (int q = 0; q < a.N; ++q) {
                    if (q == j) continue;
                    const float2 gh = ldcg2(a.ghat + static_cast<size_t>(q) * a.m + row);
                    gtl.x -= gh.x;
                    gtl.y -= gh.y;
                }
                stcg2(a.gt + idx, gtl);
                stcg2(a.r + idx, make_float2(gtl.x - acc.x, gtl.y - acc.y));
            }
        }
    }

    // ---- phase C: w_b = K_b^{-1} r_b, ghat_b = gt_b - rho w_b ----------------
    __device__ void apply_factors() {
        float2* rS = reinterpret_cast<float2*>(smem + a.off_rs);
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
                rS[k] = k < mi ? ldcg2(a.r + static_cast<size_t>(j) * a.m + r0 + k)
                               : make_float2(0.f, 0.f);
            csync();
            const float4* r4 = reinterpret_cast<const float4*>(rS);
            const int kp2 = kp >> 1;
            for (int q = idx + warp; q < seg_end; q += kConsumerWarps) {
                const int rl = q - j * a.m - r0;
                const float4* Kr = reinterpret_cast<const float4*>(K + static_cast<size_t>(rl) * kp);
                float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
                int t = lane;
                for (; t + 32 < kp2; t += 64) {
                    const float4 k0 = __ldg(Kr + t), k1 = __ldg(Kr + t + 32);
                    const float4 x0 = r4[t], x1 = r4[t + 32];
                    cfma(acc0, make_float2(k0.x, k0.y), make_float2(x0.x, x0.y));
                    cfma(acc0, make_float2(k0.z, k0.w), make_float2(x0.z, x0.w));
                    cfma(acc1, make_float2(k1.x, k1.y), make_float2(x1.x, x1.y));
                    cfma(acc1, make_float2(k1.z, k1.w), make_float2(x1.z, x1.w));
                }
                if (t < kp2) {
                    const float4 k0 = __ldg(Kr + t);
                    const float4 x0 = r4[t];
                    cfma(acc0, make_float2(k0.x, k0.y), make_float2(x0.x, x0.y));
                    cfma(acc0, make_float2(k0.z, k0.w), make_float2(x0.z, x0.w));
                }
                float2 acc = make_float2(acc0.x + acc1.x, acc0.y + acc1.y);
                acc = warp_sum(acc);
                if (lane == 0) {
                    stcg2(a.w + q, acc);
                    const float2 gtl = ldcg2(a.gt + q);
                    stcg2(a.ghat + q, make_float2(gtl.x - a.rho * acc.x, gtl.y - a.rho * acc.y));
                }
            }
            idx = seg_end;
        }
    }

    // ---- pass D: u = z + H^H w, then averaging, shrinkage, dual update ------
    template <bool MULTI>
    __device__ void pass_rows_down_and_update() {
        const int rowpitch = a.wbox * 8;
        float4* usum = reinterpret_cast<float4*>(smem + a.off_usum);
        float2* wS = reinterpret_cast<float2*>(smem + a.off_ws);
        float4* red = reinterpret_cast<float4*>(smem + a.off_red);
        const int npmax = a.wbox * a.nsub / 2;
        for (int p = tid; p < npairs; p += kConsumerThreads) usum[p] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int bi = 0; bi < a.M; ++bi) {
            const int i = a.M - 1 - bi;
            const int r0 = a.row_off[i], r1 = a.row_off[i + 1], mi = r1 - r0;
            for (int jj = 0; jj < nj; ++jj)
                for (int k = tid; k < mi; k += kConsumerThreads)
                    wS[jj * a.mimax + k] =
                        ldcg2(a.w + static_cast<size_t>(jlo + jj) * a.m + r0 + k);
            csync();
            float4 acc[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            const int nb = (mi + a.R - 1) / a.R;
            for (int b = nb - 1; b >= 0; --b) {
                const int y = r0 + b * a.R;
                int slot;
                const unsigned char* buf = acquire_stage(slot);
                for (int t = warp; t < a.R; t += 2 * kConsumerWarps) {
                    const int ra = t, rb = t + kConsumerWarps;
                    const bool in_b = rb < a.R;
                    const bool oka = y + ra < r1, okb = in_b && (y + rb < r1);
                    if (!MULTI) {
                        const float2 wa = oka ? wS[y + ra - r0] : make_float2(0.f, 0.f);
                        const float2 wb = okb ? wS[y + rb - r0] : make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k < CH; ++k) {
                            if (is_valid(k)) {
                                const float4 ha = lds128(buf + soff[k] + ra * rowpitch);
                                float2 c0 = make_float2(acc[k].x, acc[k].y);
                                float2 c1 = make_float2(acc[k].z, acc[k].w);
                                cfma_conj(c0, make_float2(ha.x, ha.y), wa);
                                cfma_conj(c1, make_float2(ha.z, ha.w), wa);
                                if (in_b) {
                                    const float4 hb = lds128(buf + soff[k] + rb * rowpitch);
                                    cfma_conj(c0, make_float2(hb.x, hb.y), wb);
                                    cfma_conj(c1, make_float2(hb.z, hb.w), wb);
                                }
                                acc[k] = make_float4(c0.x, c0.y, c1.x, c1.y);
                            }
                        }
                    } else {
                        float2 wa[kMaxBlocksPerSlab], wb[kMaxBlocksPerSlab];
#pragma unroll
                        for (int jj = 0; jj < kMaxBlocksPerSlab; ++jj) {
                            const bool use = jj < nj;
                            wa[jj] = (use && oka) ? wS[jj * a.mimax + y + ra - r0] : make_float2(0.f, 0.f);
                            wb[jj] = (use && okb) ? wS[jj * a.mimax + y + rb - r0] : make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int k = 0; k < CH; ++k) {
                            if (is_valid(k)) {
                                const int j0 = jl_of(k, 0), j1 = jl_of(k, 1);
                                const float4 ha = lds128(buf + soff[k] + ra * rowpitch);
                                float2 c0 = make_float2(acc[k].x, acc[k].y);
                                float2 c1 = make_float2(acc[k].z, acc[k].w);
                                cfma_conj(c0, make_float2(ha.x, ha.y), wa[j0]);
                                cfma_conj(c1, make_float2(ha.z, ha.w), wa[j1]);
                                if (in_b) {
                                    const float4 hb = lds128(buf + soff[k] + rb * rowpitch);
                                    cfma_conj(c0, make_float2(hb.x, hb.y), wb[j0]);
                                    cfma_conj(c1, make_float2(hb.z, hb.w), wb[j1]);
                                }
                                acc[k] = make_float4(c0.x, c0.y, c1.x, c1.y);
                            }
                        }
                    }
                }
                release_stage(slot);
            }
            // cross-warp sum of the replica's products, then u_i = z_i + H_i^H w_i
#pragma unroll
            for (int k = 0; k < CH; ++k)
                if (is_valid(k)) red[warp * npmax + lane + 32 * k] = acc[k];
            csync();
            for (int p = tid; p < npairs; p += kConsumerThreads) {
                float4 sum = red[p];
#pragma unroll
                for (int wq = 1; wq < kConsumerWarps; ++wq) sum = sum + red[wq * npmax + p];
                const int c = c_beg + 2 * p;
                const float4 vv = *reinterpret_cast<const float4*>(a.v + c);
                const float4 ss =
                    *reinterpret_cast<const float4*>(a.s + static_cast<size_t>(i) * a.ld + c);
                const float4 uu = (vv - ss) + sum;
                *reinterpret_cast<float4*>(a.u + static_cast<size_t>(i) * a.ld + c) = uu;
                usum[p] = usum[p] + uu;
            }
        }
        // v = S_kappa(mean u + mean s), s += u - v, FP64 residual partials
        double rp = 0.0, rdv = 0.0, u2 = 0.0, v2 = 0.0, s2 = 0.0;
        for (int p = tid; p < npairs; p += kConsumerThreads) {
            const int c = c_beg + 2 * p;
            const float4 ub = scale4(usum[p], a.inv_M);
            float4 sb = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int i = 0; i < a.M; ++i)
                sb = sb + *reinterpret_cast<const float4*>(a.s + static_cast<size_t>(i) * a.ld + c);
            sb = scale4(sb, a.inv_M);
            const float4 av = ub + sb;
            const float2 vn0 = soft_threshold(make_float2(av.x, av.y), a.kappa);
            const float2 vn1 = soft_threshold(make_float2(av.z, av.w), a.kappa);
            const float4 vn = make_float4(vn0.x, vn0.y, vn1.x, vn1.y);
            const float4 vo = *reinterpret_cast<const float4*>(a.v + c);
            rdv += norm2(make_float2(vn.x - vo.x, vn.y - vo.y)) + norm2(make_float2(vn.z - vo.z, vn.w - vo.w));
            v2 += norm2(vn0) + norm2(vn1);
            for (int i = 0; i < a.M; ++i) {
                float4* sp = reinterpret_cast<float4*>(a.s + static_cast<size_t>(i) * a.ld + c);
                const float4 ss = *sp;
                const float4 uu = *reinterpret_cast<const float4*>(a.u + static_cast<size_t>(i) * a.ld + c);
                const float4 sn = (ss + uu) - vn;
                *sp = sn;
                rp += norm2(make_float2(uu.x - vn.x, uu.y - vn.y)) + norm2(make_float2(uu.z - vn.z, uu.w - vn.w));
                u2 += norm2(make_float2(uu.x, uu.y)) + norm2(make_float2(uu.z, uu.w));
                s2 += norm2(make_float2(sn.x, sn.y)) + norm2(make_float2(sn.z, sn.w));
            }
            *reinterpret_cast<float4*>(a.v + c) = vn;
        }
        rp = warp_sum_d(rp);
        rdv = warp_sum_d(rdv);
        u2 = warp_sum_d(u2);
        v2 = warp_sum_d(v2);
        s2 = warp_sum_d(s2);
        if (lane == 0) {
            misc->red[warp][0] = rp;
            misc->red[warp][1] = rdv;
            misc->red[warp][2] = u2;
            misc->red[warp][3] = v2;
            misc->red[warp][4] = s2;
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
        bool ok = true, stopped = false;
        for (int it = 0; it < a.iters; ++it) {
            if (multi) pass_rows_up<true>(); else pass_rows_up<false>();
            if (!(ok = grid_barrier(a, misc))) break;
            reduce_partials(it);
            if (!(ok = grid_barrier(a, misc))) break;
            if (a.check_stop && it > 0 && __ldcg(a.stop_flag) != 0) {
                stopped = true;
                completed = it;
                break;
            }
            apply_factors();
            if (!(ok = grid_barrier(a, misc))) break;
            if (multi) pass_rows_down_and_update<true>(); else pass_rows_down_and_update<false>();
            completed = it + 1;
        }
        if (ok && !stopped) {
            ok = grid_barrier(a, misc);
            if (ok && cta == 0 && warp == 0) finalize(a.iters - 1);
        }
        if (cta == 0 && tid == 0) a.k_done[0] = a.k0 + completed;
        drain();
    }
};

template <int CH>
__global__ void __launch_bounds__(kIterThreads, 1)
    iterate_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ IterArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
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
            producer(&tmap, a, full, empty, misc, ring, a.cta_col[blockIdx.x]);
        return;
    }
    Consumer<CH> c(a, smem, misc, full, empty, ring);
    c.run();
}

template <int CH>
void* kernel_fn() {
    return reinterpret_cast<void*>(&iterate_kernel<CH>);
}

void* pick(int chunks) {
    switch (chunks) {
        case 1: return kernel_fn<1>();
        case 2: return kernel_fn<2>();
        case 4: return kernel_fn<4>();
        case 8: return kernel_fn<8>();
        case 16: return kernel_fn<16>();
        default: return nullptr;
    }
}

}  // namespace

cudaError_t prepare_iterate(int chunks, int smem) {
    void* fn = pick(chunks);
    if (!fn) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

int max_coresident_iterate(int chunks, int smem, int* per_sm) {
    void* fn = pick(chunks);
    if (!fn) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, kIterThreads, smem) != cudaSuccess)
        return 0;
    if (per_sm) *per_sm = blocks;
    return blocks;
}

cudaError_t launch_iterate(const CUtensorMap& tmap, const IterArgs& a, int chunks, int smem,
                           cudaStream_t stream) {
    void* fn = pick(chunks);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {const_cast<CUtensorMap*>(&tmap), const_cast<IterArgs*>(&a)};
    return cudaLaunchCooperativeKernel(fn, dim3(a.P), dim3(kIterThreads), args,
                                       static_cast<size_t>(smem), stream);
}

}  // namespace admm
