// Host side of the batched shared-H path: setup (FP16 copy of H and of its
// transpose, packed factors, tensor maps), the per-iteration kernel sequence
// captured once into a CUDA graph, and the admm_batch_* C ABI.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "admm_batch.h"

using namespace admm::batch;

namespace {

thread_local std::string g_batch_error;

constexpr int kTuneMaxSplits = 32;

int round_up(int64_t x, int64_t q) { return static_cast<int>((x + q - 1) / q * q); }

}  // namespace

struct admm_batch {
    admm_t* inner = nullptr;   // single-scene handle: H, its FP16 copy and the factors
    admm::HandleView hv{};
    int m = 0, n = 0, M = 1, N = 1, P = 1, B = 1, ld = 0;
    int mimax = 0, njmax = 0, mpitch = 0, npitch = 0, kz = 0, kr = 0, kw = 0, splits1 = 1;
    double rho = 1.0;
    std::vector<double> lam;
    std::vector<int> ro, co;
    // device memory
    void *H16T = nullptr, *Kpack = nullptr, *Zpack = nullptr, *Rpack = nullptr, *Wpack = nullptr;
    float* kscale = nullptr;
    float2 *V = nullptr, *S = nullptr, *G = nullptr, *Gt = nullptr, *Ghat = nullptr, *R = nullptr,
           *Ppart = nullptr, *W = nullptr, *Sig = nullptr, *X = nullptr, *Y = nullptr;
    float *zscale = nullptr, *rscale = nullptr, *wscale = nullptr, *kappa = nullptr;
    unsigned* zmax = nullptr;   // largest |component| of the next z per (block, scene)
    // recording for the adjoint and the reverse-sweep buffers
    float2 *rec_a = nullptr, *rec_w = nullptr, *Vb = nullptr, *Sb = nullptr, *Ghb = nullptr, *dG = nullptr;
    int* rec_k = nullptr;
    double *kbar = nullptr, *rbar = nullptr;
    int rec_cap = 0;
    int max_splits = 1;         // K splits the partial-product buffer holds (autotuner range)
    bool rec_valid = false;     // every iteration since the last reset was recorded
    PackArgs psb{};             // packing of sigma_bar for the forward product
    double* res = nullptr;
    int* itab = nullptr;
    long long* ltab = nullptr;
    int* status = nullptr;
    CUtensorMap mapH, mapHT, mapK, mapZ, mapR, mapW;
    GemmArgs g1{}, gk{}, g2{};
    PackArgs pz{}, pr{}, pw{}, px{}, py{};
    StepArgs st{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long timeout_ns = 5000000000LL;
    int64_t k = 0;
    int broken = 0;
    std::string err;
};

namespace {

int bfail(admm_batch_t* h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_batch_error = buf;
    return code;
}

#define BCK(h, call)                                                                      \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            if (h) (h)->broken = 1;                                                       \
            return bfail(h, ADMM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));          \
        }                                                                                 \
    } while (0)

template <typename T>
cudaError_t dalloc0(T** p, size_t count) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) e = cudaMemset(*p, 0, std::max<size_t>(count, 1) * sizeof(T));
    return e;
}

void free_batch(admm_batch_t* h) {
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    void* ptrs[] = {h->H16T, h->Kpack, h->Zpack, h->Rpack, h->Wpack, h->kscale, h->V, h->S, h->G, h->Gt,
                    h->Ghat, h->R, h->Ppart, h->W, h->Sig, h->X, h->Y, h->zscale, h->rscale, h->wscale,
                    h->kappa, h->res, h->itab, h->ltab, h->status, h->zmax, h->rec_a, h->rec_w,
                    h->Vb, h->Sb, h->Ghb, h->dG, h->rec_k, h->kbar, h->rbar};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->inner) admm_destroy(h->inner);
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3-D FP16 tensor map {inner (K), rows, planes}, box {64, box_rows, 1}, 128-byte swizzle
int encode3(admm_batch_t* h, CUtensorMap* map, const void* base, int64_t inner, int64_t rows, int64_t planes,
            int box_rows) {
    auto enc = encoder();
    if (!enc) return bfail(h, ADMM_ECUDA, "cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(rows),
                          static_cast<cuuint64_t>(planes)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(inner) * 2, static_cast<cuuint64_t>(inner * rows) * 2};
    cuuint32_t box[3] = {static_cast<cuuint32_t>(kTileK), static_cast<cuuint32_t>(box_rows), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return bfail(h, ADMM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
    return ADMM_OK;
}

// one iteration: every launch on stream s (captured into the graph)
cudaError_t enqueue_iteration(admm_batch_t* h, cudaStream_t s) {
    cudaError_t e = launch_gtilde(h->st, s);
    if (e == cudaSuccess) e = launch_pack(h->pz, h->P, s);
    if (e == cudaSuccess) e = launch_gemm(h->mapH, h->mapZ, h->g1, s);
    if (e == cudaSuccess) e = launch_residual_r(h->st, s);
    if (e == cudaSuccess) e = launch_pack(h->pr, h->P, s);
    if (e == cudaSuccess) e = launch_gemm(h->mapK, h->mapR, h->gk, s);
    if (e == cudaSuccess) e = launch_ghat(h->st, s);
    if (e == cudaSuccess) e = launch_pack(h->pw, h->P, s);
    if (e == cudaSuccess) e = launch_gemm(h->mapHT, h->mapW, h->g2, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->res, 0, 2 * sizeof(double) * h->B, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->zmax, 0, sizeof(unsigned) * h->P * h->B, s);
    if (e == cudaSuccess) e = launch_update(h->st, s);
    if (e == cudaSuccess && h->st.rec_a) e = launch_rec_advance(h->st, s);
    return e;
}

// one recorded iteration in reverse (st.bk selects the records)
cudaError_t enqueue_backward(admm_batch_t* h, const StepArgs& st, cudaStream_t s) {
    cudaError_t e = launch_bw_soft(st, s);
    if (e == cudaSuccess) e = launch_pack(h->psb, h->P, s);
    if (e == cudaSuccess) e = launch_gemm(h->mapH, h->mapZ, h->g1, s);
    if (e == cudaSuccess) e = launch_bw_wbar(st, s);
    if (e == cudaSuccess) e = launch_pack(h->pr, h->P, s);
    if (e == cudaSuccess) e = launch_gemm(h->mapK, h->mapR, h->gk, s);
    if (e == cudaSuccess) e = launch_bw_rbar(st, s);
    if (e == cudaSuccess) e = launch_pack(h->pw, h->P, s);
    if (e == cudaSuccess) e = launch_gemm(h->mapHT, h->mapW, h->g2, s);
    if (e == cudaSuccess) e = launch_bw_state(st, s);
    if (e == cudaSuccess) e = launch_bw_gtilde(st, s);
    return e;
}

int check_status(admm_batch_t* h, cudaStream_t s) {
    BCK(h, cudaStreamSynchronize(s));
    int code = 0;
    BCK(h, cudaMemcpy(&code, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (code == ADMM_ETIMEOUT) {
        h->broken = 1;
        return bfail(h, code, "a bounded in-kernel wait expired");
    }
    if (code) return bfail(h, code, "device status %d", code);
    return ADMM_OK;
}

}  // namespace

extern "C" {

int admm_batch_setup(admm_batch_t** out, const void* H, int64_t m, int64_t n, int32_t row_blocks,
                     int32_t col_blocks, int32_t batch, const double* lambda, double rho, int32_t h_dtype,
                     void* stream) {
    if (!out) return bfail(nullptr, ADMM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!H || !lambda) return bfail(nullptr, ADMM_EINVAL, "H and lambda must not be NULL");
    if (batch < 1 || batch > 4096) return bfail(nullptr, ADMM_EINVAL, "batch must be in [1, 4096]");
    for (int b = 0; b < batch; ++b)
        if (!(lambda[b] >= 0.0) || !std::isfinite(lambda[b]))
            return bfail(nullptr, ADMM_EINVAL, "lambda[%d] must be finite and >= 0", b);
    if (m < 4 || n < 4 || m % 4 || m > (1 << 20) || n > (1 << 24))
        return bfail(nullptr, ADMM_EUNSUPPORTED, "the batched path needs m a multiple of 4, m <= 2^20, n <= 2^24");
    std::vector<int> ro, co;
    if (row_blocks < 1 || col_blocks < 1 || row_blocks > m || col_blocks > n)
        return bfail(nullptr, ADMM_EINVAL, "bad row_blocks / col_blocks");
    admm::balanced_offsets(m, row_blocks, ro);
    admm::balanced_offsets(n, col_blocks, co);
    for (int i = 0; i <= row_blocks; ++i)
        if (ro[i] % 4) return bfail(nullptr, ADMM_EUNSUPPORTED, "row blocks must start at multiples of 4");
    for (int j = 0; j <= col_blocks; ++j)
        if (co[j] % 4 && j < col_blocks)
            return bfail(nullptr, ADMM_EUNSUPPORTED, "column blocks must start at multiples of 4");
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    admm_batch_t* h = new admm_batch_t();
    auto bail = [&](int c) {
        g_batch_error = h->err.empty() ? g_batch_error : h->err;
        free_batch(h);
        delete h;
        return c;
    };
    h->m = static_cast<int>(m);
    h->n = static_cast<int>(n);
    h->M = row_blocks;
    h->N = col_blocks;
    h->P = row_blocks * col_blocks;
    h->B = batch;
    h->rho = rho;
    h->lam.assign(lambda, lambda + batch);
    h->ro = ro;
    h->co = co;
    // the single-scene handle builds H, its FP16 copy and the factors of the encoded matrix
    std::vector<float2> gz(static_cast<size_t>(m), make_float2(0.f, 0.f));
    int code = admm_setup(&h->inner, H, gz.data(), m, n, row_blocks, col_blocks, 0.0, rho, h_dtype, stream);
    if (code) {
        h->err = admm_last_error(nullptr);
        return bail(code);
    }
    code = admm_set_option(h->inner, ADMM_OPT_H_FP16, 1);
    if (code) {
        h->err = admm_last_error(h->inner);
        return bail(code);
    }
    admm::view_handle(h->inner, &h->hv);
    if (!h->hv.H16) return bail(bfail(h, ADMM_ECUDA, "the FP16 copy of H is missing"));
    h->ld = h->hv.ld;
    for (int i = 0; i < row_blocks; ++i) h->mimax = std::max(h->mimax, ro[i + 1] - ro[i]);
    for (int j = 0; j < col_blocks; ++j) h->njmax = std::max(h->njmax, co[j + 1] - co[j]);
    h->mpitch = round_up(h->mimax, 32);
    h->npitch = round_up(h->njmax, 32);
    h->kz = round_up(2 * h->njmax, kTileK);
    h->kr = round_up(4 * h->mimax, kTileK);
    h->kw = round_up(2 * h->mimax, kTileK);
    const int P = h->P, Bn = batch;
    const int ntiles = (4 * Bn + kTileCols - 1) / kTileCols;
    const int mt1 = (h->mimax + kTileRows - 1) / kTileRows;
    const int mt2 = (h->njmax + kTileRows - 1) / kTileRows;
    // split K of the forward product so that about two CTAs per SM are in flight
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int kb1 = h->kz / kTileK;
    h->splits1 = std::max(1, std::min(kb1 / 8, (2 * sms + P * mt1 * ntiles - 1) / (P * mt1 * ntiles)));
    h->max_splits = std::max(h->splits1, std::max(1, std::min(kTuneMaxSplits, kb1 / 4)));
    const size_t mp = h->mpitch, np = h->npitch;
    bool ok = cudaMalloc(&h->H16T, static_cast<size_t>(h->ld) * m * 4) == cudaSuccess &&
              dalloc0(reinterpret_cast<unsigned short**>(&h->Kpack), static_cast<size_t>(P) * h->mimax * h->kr) ==
                  cudaSuccess &&
              dalloc0(&h->kscale, static_cast<size_t>(P) * h->mimax) == cudaSuccess &&
              dalloc0(reinterpret_cast<unsigned short**>(&h->Zpack), static_cast<size_t>(P) * 4 * Bn * h->kz) ==
                  cudaSuccess &&
              dalloc0(reinterpret_cast<unsigned short**>(&h->Rpack), static_cast<size_t>(P) * 4 * Bn * h->kr) ==
                  cudaSuccess &&
              dalloc0(reinterpret_cast<unsigned short**>(&h->Wpack), static_cast<size_t>(P) * 4 * Bn * h->kw) ==
                  cudaSuccess &&
              dalloc0(&h->V, static_cast<size_t>(Bn) * n) == cudaSuccess &&
              dalloc0(&h->S, static_cast<size_t>(row_blocks) * Bn * n) == cudaSuccess &&
              dalloc0(&h->G, static_cast<size_t>(Bn) * m) == cudaSuccess &&
              dalloc0(&h->Gt, static_cast<size_t>(col_blocks) * Bn * m) == cudaSuccess &&
              dalloc0(&h->Ghat, static_cast<size_t>(col_blocks) * Bn * m) == cudaSuccess &&
              dalloc0(&h->R, static_cast<size_t>(P) * Bn * mp) == cudaSuccess &&
              dalloc0(&h->Ppart, static_cast<size_t>(h->max_splits) * P * Bn * mp) == cudaSuccess &&
              dalloc0(&h->W, static_cast<size_t>(P) * Bn * mp) == cudaSuccess &&
              dalloc0(&h->Sig, static_cast<size_t>(P) * Bn * np) == cudaSuccess &&
              dalloc0(&h->zscale, static_cast<size_t>(P) * Bn) == cudaSuccess &&
              dalloc0(&h->rscale, static_cast<size_t>(P) * Bn) == cudaSuccess &&
              dalloc0(&h->wscale, static_cast<size_t>(P) * Bn) == cudaSuccess &&
              dalloc0(&h->kappa, static_cast<size_t>(Bn)) == cudaSuccess &&
              dalloc0(&h->zmax, static_cast<size_t>(P) * Bn) == cudaSuccess &&
              dalloc0(&h->res, static_cast<size_t>(2) * Bn) == cudaSuccess &&
              dalloc0(&h->status, 1) == cudaSuccess;
    if (!ok) return bail(bfail(h, ADMM_ENOMEM, "device allocation failed for the batched path"));
    // tables: per problem p = i N + j
    std::vector<int> it;
    auto put = [&](const std::vector<int>& x) {
        const size_t at = it.size();
        it.insert(it.end(), x.begin(), x.end());
        return at;
    };
    std::vector<int> a1x(P), a1y(P), zero(P, 0), rows1(P), kb1p(P), rsr(P), a2x(P), a2y(P), rows2(P), kb2p(P),
        kkp(P), ksoff(P), pz(P), lenz(P), lenr(P), kidx(P);
    std::vector<long long> xz(P), yz(P), xr(P), xy(P), xs(P);
    for (int i = 0; i < row_blocks; ++i)
        for (int j = 0; j < col_blocks; ++j) {
            const int p = i * col_blocks + j;
            const int mi = ro[i + 1] - ro[i], nj = co[j + 1] - co[j];
            a1x[p] = 2 * co[j];
            a1y[p] = ro[i];
            rows1[p] = mi;
            kb1p[p] = (2 * nj + kTileK - 1) / kTileK;
            rsr[p] = ro[i];
            a2x[p] = 2 * ro[i];
            a2y[p] = co[j];
            rows2[p] = nj;
            kb2p[p] = (2 * mi + kTileK - 1) / kTileK;
            kkp[p] = h->kr / kTileK;
            ksoff[p] = p * h->mimax;
            pz[p] = p;
            lenz[p] = nj;
            lenr[p] = mi;
            xz[p] = co[j];
            yz[p] = static_cast<long long>(i) * Bn * n + co[j];
            xr[p] = static_cast<long long>(p) * Bn * mp;
            xy[p] = ro[i];
            xs[p] = static_cast<long long>(p) * Bn * np;
        }
    std::vector<int> uto(col_blocks + 1, 0);
    for (int j = 0; j < col_blocks; ++j) uto[j + 1] = uto[j] + (co[j + 1] - co[j] + kUpdCols - 1) / kUpdCols;
    const size_t o_uto = put(uto);
    const size_t o_a1x = put(a1x), o_a1y = put(a1y), o_zero = put(zero), o_rows1 = put(rows1), o_kb1 = put(kb1p),
                 o_rsr = put(rsr), o_a2x = put(a2x), o_a2y = put(a2y), o_rows2 = put(rows2), o_kb2 = put(kb2p),
                 o_kk = put(kkp), o_ksoff = put(ksoff), o_pz = put(pz), o_lenz = put(lenz), o_lenr = put(lenr),
                 o_ro = put(ro), o_co = put(co);
    std::vector<long long> lt;
    auto lput = [&](const std::vector<long long>& x) {
        const size_t at = lt.size();
        lt.insert(lt.end(), x.begin(), x.end());
        return at;
    };
    const size_t o_xz = lput(xz), o_yz = lput(yz), o_xr = lput(xr), o_xy = lput(xy), o_xs = lput(xs);
    if (dalloc0(&h->itab, it.size()) != cudaSuccess || dalloc0(&h->ltab, lt.size()) != cudaSuccess)
        return bail(bfail(h, ADMM_ENOMEM, "device allocation failed for the batched tables"));
    if (cudaMemcpy(h->itab, it.data(), it.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->ltab, lt.data(), lt.size() * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(bfail(h, ADMM_ECUDA, "copy of the batched tables failed"));
    const int* T = h->itab;
    const long long* LT = h->ltab;
    std::vector<float> kap(Bn);
    for (int b = 0; b < Bn; ++b) kap[b] = static_cast<float>(h->lam[b] / (row_blocks * rho));
    if (cudaMemcpy(h->kappa, kap.data(), Bn * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(bfail(h, ADMM_ECUDA, "copy of kappa failed"));

    // H^T in FP16 and the packed factors
    if (launch_transpose_h16(h->hv.H16, h->m, h->ld, h->H16T, st) != cudaSuccess ||
        launch_pack_kinv(h->hv.kinv16, h->hv.kinv_off, h->hv.kinv_pitch, h->hv.row_off, P, col_blocks, h->mimax,
                         h->kr, h->Kpack, h->kscale, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return bail(bfail(h, ADMM_ECUDA, "transpose / factor packing failed"));
    // tensor maps
    if ((code = encode3(h, &h->mapH, h->hv.H16, 2LL * h->ld, m, 1, kTileRows)) ||
        (code = encode3(h, &h->mapHT, h->H16T, 2LL * m, h->ld, 1, kTileRows)) ||
        (code = encode3(h, &h->mapK, h->Kpack, h->kr, h->mimax, P, kTileRows)) ||
        (code = encode3(h, &h->mapZ, h->Zpack, h->kz, 4LL * Bn, P, kTileCols)) ||
        (code = encode3(h, &h->mapR, h->Rpack, h->kr, 4LL * Bn, P, kTileCols)) ||
        (code = encode3(h, &h->mapW, h->Wpack, h->kw, 4LL * Bn, P, kTileCols)))
        return bail(code);
    if (prepare_gemm() != cudaSuccess) return bail(bfail(h, ADMM_ECUDA, "GEMM shared-memory opt-in failed"));

    // forward product H_ij z_j^i
    GemmArgs& g1 = h->g1;
    g1.nprob = P;
    g1.mtiles = mt1;
    g1.ntiles = ntiles;
    g1.splits = h->splits1;
    g1.kb_per_split = (kb1 + h->splits1 - 1) / h->splits1;
    g1.a_x0 = T + o_a1x;
    g1.a_y0 = T + o_a1y;
    g1.a_z = T + o_zero;
    g1.rows = T + o_rows1;
    g1.kb_prob = T + o_kb1;
    g1.row_scale = h->hv.scales;
    g1.rs_off = T + o_rsr;
    g1.rs_shift = 6;
    g1.col_scale = h->zscale;
    g1.out = h->Ppart;
    g1.out_pitch = h->mpitch;
    g1.B = Bn;
    g1.status = h->status;
    g1.ctas = sms;
    g1.timeout_ns = h->timeout_ns;
    // factor product K_ij^{-1} r_ij
    GemmArgs& gk = h->gk;
    gk = g1;
    gk.mtiles = mt1;
    gk.splits = 1;
    gk.kb_per_split = h->kr / kTileK;
    gk.a_x0 = T + o_zero;
    gk.a_y0 = T + o_zero;
    gk.a_z = T + o_pz;
    gk.kb_prob = T + o_kk;
    gk.row_scale = h->kscale;
    gk.rs_off = T + o_ksoff;
    gk.rs_shift = 0;
    gk.col_scale = h->rscale;
    gk.out = h->W;
    // adjoint product H_ij^H w_ij
    GemmArgs& g2 = h->g2;
    g2 = g1;
    g2.mtiles = mt2;
    g2.splits = 1;
    g2.kb_per_split = h->kw / kTileK;
    g2.a_x0 = T + o_a2x;
    g2.a_y0 = T + o_a2y;
    g2.a_z = T + o_zero;
    g2.rows = T + o_rows2;
    g2.kb_prob = T + o_kb2;
    g2.row_scale = nullptr;
    g2.col_scale = h->wscale;
    g2.out = h->Sig;
    g2.out_pitch = h->npitch;
    // packing
    PackArgs& pz_ = h->pz;
    pz_.x = h->V;
    pz_.x_off = LT + o_xz;
    pz_.x_bs = n;
    pz_.y = h->S;
    pz_.y_off = LT + o_yz;
    pz_.y_bs = n;
    pz_.rs = nullptr;
    pz_.rs_row = T + o_rsr;
    pz_.len = T + o_lenz;
    pz_.B = Bn;
    pz_.dst = h->Zpack;
    pz_.row2 = h->kz / 2;
    pz_.adjoint = 0;
    pz_.second = -1;
    pz_.scale = h->zscale;
    pz_.vmax = h->zmax;
    PackArgs& pr_ = h->pr;
    pr_ = pz_;
    pr_.vmax = nullptr;
    pr_.x = h->R;
    pr_.x_off = LT + o_xr;
    pr_.x_bs = mp;
    pr_.y = nullptr;
    pr_.len = T + o_lenr;
    pr_.dst = h->Rpack;
    pr_.row2 = h->kr / 2;
    pr_.second = h->mimax;
    pr_.scale = h->rscale;
    PackArgs& pw_ = h->pw;
    pw_ = pr_;
    pw_.x = h->W;
    pw_.rs = h->hv.scales;
    pw_.dst = h->Wpack;
    pw_.row2 = h->kw / 2;
    pw_.adjoint = 1;
    pw_.second = -1;
    pw_.scale = h->wscale;
    // forward / adjoint of the public products: X (B x n) and Y (B x m) scratch
    PackArgs& px_ = h->px;
    px_ = pz_;
    px_.y = nullptr;
    px_.vmax = nullptr;
    PackArgs& py_ = h->py;
    py_ = pw_;
    py_.x_off = LT + o_xy;
    py_.x_bs = m;
    PackArgs& psb_ = h->psb;
    psb_ = pz_;
    psb_.x = h->Sig;
    psb_.x_off = LT + o_xs;
    psb_.x_bs = np;
    psb_.y = nullptr;
    psb_.vmax = nullptr;
    // elementwise steps
    StepArgs& s_ = h->st;
    s_.m = h->m;
    s_.n = h->n;
    s_.M = row_blocks;
    s_.N = col_blocks;
    s_.P = P;
    s_.B = Bn;
    s_.splits = h->splits1;
    s_.mpitch = h->mpitch;
    s_.npitch = h->npitch;
    s_.row_off = T + o_ro;
    s_.col_off = T + o_co;
    s_.V = h->V;
    s_.S = h->S;
    s_.G = h->G;
    s_.Gt = h->Gt;
    s_.Ghat = h->Ghat;
    s_.R = h->R;
    s_.Ppart = h->Ppart;
    s_.W = h->W;
    s_.Sig = h->Sig;
    s_.kappa = h->kappa;
    s_.rho = static_cast<float>(rho);
    s_.inv_M = 1.0f / row_blocks;
    s_.res = h->res;
    s_.zmax = h->zmax;
    s_.upd_tile_off = T + o_uto;
    s_.upd_tiles = uto[col_blocks];
    *out = h;
    return ADMM_OK;
}

const char* admm_batch_last_error(const admm_batch_t* h) { return h ? h->err.c_str() : g_batch_error.c_str(); }

int admm_batch_set_g(admm_batch_t* h, const void* G, void* stream) {
    if (!h || !G) return h ? bfail(h, ADMM_EINVAL, "G is NULL") : ADMM_EINVAL;
    BCK(h, cudaMemcpyAsync(h->G, G, static_cast<size_t>(h->B) * h->m * sizeof(float2), cudaMemcpyDefault,
                           static_cast<cudaStream_t>(stream)));
    BCK(h, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return ADMM_OK;
}

int admm_batch_reset(admm_batch_t* h, void* stream) {
    if (!h) return ADMM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BCK(h, cudaMemsetAsync(h->V, 0, static_cast<size_t>(h->B) * h->n * sizeof(float2), s));
    BCK(h, cudaMemsetAsync(h->S, 0, static_cast<size_t>(h->M) * h->B * h->n * sizeof(float2), s));
    BCK(h, cudaMemsetAsync(h->Ghat, 0, static_cast<size_t>(h->N) * h->B * h->m * sizeof(float2), s));
    BCK(h, cudaMemsetAsync(h->zmax, 0, static_cast<size_t>(h->P) * h->B * sizeof(unsigned), s));
    BCK(h, cudaMemsetAsync(h->status, 0, sizeof(int), s));
    if (h->rec_k) BCK(h, cudaMemsetAsync(h->rec_k, 0, sizeof(int), s));
    h->rec_valid = h->rec_cap > 0;
    BCK(h, cudaStreamSynchronize(s));
    h->k = 0;
    h->broken = 0;
    return ADMM_OK;
}

int admm_batch_iterate(admm_batch_t* h, int32_t iters, void* stream) {
    if (!h || iters < 0) return h ? bfail(h, ADMM_EINVAL, "iters must be >= 0") : ADMM_EINVAL;
    if (h->broken) return bfail(h, ADMM_ECUDA, "handle is in an error state; call admm_batch_reset");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!h->exec) {
        // capture one iteration on a private stream, then replay it on the caller's
        cudaStream_t cap;
        BCK(h, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t e2 = enqueue_iteration(h, cap);
            e = cudaStreamEndCapture(cap, &h->graph);
            if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->exec, h->graph, 0);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            h->broken = 1;
            return bfail(h, ADMM_ECUDA, "capture of the batched iteration failed: %s", cudaGetErrorString(e));
        }
    }
    for (int it = 0; it < iters; ++it) BCK(h, cudaGraphLaunch(h->exec, s));
    h->k += iters;
    if (h->k > h->rec_cap) h->rec_valid = false;
    return ADMM_OK;
}

int admm_batch_tune(admm_batch_t* h, void* stream) {
    if (!h) return ADMM_EINVAL;
    if (h->broken) return bfail(h, ADMM_ECUDA, "handle is in an error state; call admm_batch_reset");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // candidates: powers of two up to the buffer's capacity, each with at least 4 K blocks per split
    const int kb1 = h->kz / kTileK;
    cudaEvent_t e0, e1;
    BCK(h, cudaEventCreate(&e0));
    BCK(h, cudaEventCreate(&e1));
    int best = h->splits1;
    float best_ms = 1e30f;
    // the packed operand of the current state is what the timed products read
    BCK(h, launch_pack(h->pz, h->P, s));
    for (int sp = 1; sp <= h->max_splits; sp *= 2) {
        if (kb1 / sp < 4 && sp > 1) break;
        GemmArgs g = h->g1;
        g.splits = sp;
        g.kb_per_split = (kb1 + sp - 1) / sp;
        cudaError_t e = launch_gemm(h->mapH, h->mapZ, g, s);   // warm
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_gemm(h->mapH, h->mapZ, g, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            h->broken = 1;
            return bfail(h, ADMM_ECUDA, "tuning launch failed: %s", cudaGetErrorString(e));
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = sp;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->splits1 = best;
    h->g1.splits = best;
    h->g1.kb_per_split = (kb1 + best - 1) / best;
    h->st.splits = best;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
    return check_status(h, s);
}

int admm_batch_set_lambda(admm_batch_t* h, const double* lambda) {
    if (!h || !lambda) return h ? bfail(h, ADMM_EINVAL, "lambda is NULL") : ADMM_EINVAL;
    for (int b = 0; b < h->B; ++b)
        if (!(lambda[b] >= 0.0) || !std::isfinite(lambda[b]))
            return bfail(h, ADMM_EINVAL, "lambda[%d] must be finite and >= 0", b);
    std::vector<float> kap(h->B);
    for (int b = 0; b < h->B; ++b) kap[b] = static_cast<float>(lambda[b] / (h->M * h->rho));
    BCK(h, cudaDeviceSynchronize());
    BCK(h, cudaMemcpy(h->kappa, kap.data(), h->B * sizeof(float), cudaMemcpyHostToDevice));
    h->lam.assign(lambda, lambda + h->B);
    h->rec_valid = false;
    return ADMM_OK;
}

int admm_batch_set_rho(admm_batch_t* h, double rho, void* stream) {
    if (!h) return ADMM_EINVAL;
    if (!(rho > 0.0) || !std::isfinite(rho)) return bfail(h, ADMM_EINVAL, "rho must be finite and > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BCK(h, cudaDeviceSynchronize());
    int code = admm_set_rho(h->inner, rho, stream);
    if (code) return bfail(h, code, "refactorisation failed: %s", admm_last_error(h->inner));
    if (admm::view_handle(h->inner, &h->hv) != ADMM_OK) return bfail(h, ADMM_EINVAL, "inner handle view failed");
    const int P = h->M * h->N;
    BCK(h, launch_pack_kinv(h->hv.kinv16, h->hv.kinv_off, h->hv.kinv_pitch, h->hv.row_off, P, h->N, h->mimax,
                            h->kr, h->Kpack, h->kscale, st));
    const double old = h->rho;
    h->rho = rho;
    h->st.rho = static_cast<float>(rho);
    std::vector<float> kap(h->B);
    for (int b = 0; b < h->B; ++b) kap[b] = static_cast<float>(h->lam[b] / (h->M * rho));
    BCK(h, cudaMemcpyAsync(h->kappa, kap.data(), h->B * sizeof(float), cudaMemcpyHostToDevice, st));
    // the unscaled duals rho s are kept: s <- s rho_old / rho_new
    BCK(h, admm::launch_scale(h->S, static_cast<int64_t>(h->M) * h->B * h->n, static_cast<float>(old / rho), st));
    BCK(h, cudaStreamSynchronize(st));
    h->rec_valid = false;
    // the captured iteration carries rho as a kernel argument: capture it again
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
    return check_status(h, st);
}

int admm_batch_record(admm_batch_t* h, int32_t iters) {
    if (!h || iters < 0 || iters > (1 << 20)) return h ? bfail(h, ADMM_EINVAL, "bad record length") : ADMM_EINVAL;
    BCK(h, cudaDeviceSynchronize());
    void* old[] = {h->rec_a, h->rec_w, h->Vb, h->Sb, h->Ghb, h->dG, h->rec_k, h->kbar, h->rbar};
    for (void* p : old)
        if (p) cudaFree(p);
    h->rec_a = h->rec_w = h->Vb = h->Sb = h->Ghb = h->dG = nullptr;
    h->rec_k = nullptr;
    h->kbar = h->rbar = nullptr;
    h->rec_cap = 0;
    h->rec_valid = false;
    if (iters > 0) {
        const size_t Bn = h->B;
        if (dalloc0(&h->rec_a, static_cast<size_t>(iters) * Bn * h->n) != cudaSuccess ||
            dalloc0(&h->rec_w, static_cast<size_t>(iters) * h->P * Bn * h->mpitch) != cudaSuccess ||
            dalloc0(&h->Vb, Bn * h->n) != cudaSuccess || dalloc0(&h->Sb, static_cast<size_t>(h->M) * Bn * h->n) != cudaSuccess ||
            dalloc0(&h->Ghb, static_cast<size_t>(h->N) * Bn * h->m) != cudaSuccess ||
            dalloc0(&h->dG, Bn * h->m) != cudaSuccess || dalloc0(&h->rec_k, 1) != cudaSuccess ||
            dalloc0(&h->kbar, Bn) != cudaSuccess || dalloc0(&h->rbar, Bn) != cudaSuccess)
            return bfail(h, ADMM_ENOMEM, "no room to record %d iterations", iters);
        h->rec_cap = iters;
    }
    StepArgs& st = h->st;
    st.rec_a = h->rec_a;
    st.rec_w = h->rec_w;
    st.rec_k = h->rec_k;
    st.rec_cap = h->rec_cap;
    st.Vb = h->Vb;
    st.Sb = h->Sb;
    st.Ghb = h->Ghb;
    st.dG = h->dG;
    st.kbar = h->kbar;
    st.rbar = h->rbar;
    // the iteration graph is captured again with (or without) the recording launches
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
    return admm_batch_reset(h, nullptr);
}

int admm_batch_backward(admm_batch_t* h, const void* dV, void* dG, double* dlambda, double* drho, void* stream) {
    if (!h || !dV || !dG || !dlambda || !drho) return h ? bfail(h, ADMM_EINVAL, "NULL argument") : ADMM_EINVAL;
    if (!h->rec_cap || !h->rec_valid || h->k < 1)
        return bfail(h, ADMM_EINVAL, "no recorded iterations: admm_batch_record, then iterate at most the "
                                     "recorded count from the reset state");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t Bn = h->B;
    BCK(h, cudaMemcpyAsync(h->Vb, dV, Bn * h->n * sizeof(float2), cudaMemcpyDefault, s));
    BCK(h, cudaMemsetAsync(h->Sb, 0, static_cast<size_t>(h->M) * Bn * h->n * sizeof(float2), s));
    BCK(h, cudaMemsetAsync(h->Ghb, 0, static_cast<size_t>(h->N) * Bn * h->m * sizeof(float2), s));
    BCK(h, cudaMemsetAsync(h->dG, 0, Bn * h->m * sizeof(float2), s));
    BCK(h, cudaMemsetAsync(h->kbar, 0, Bn * sizeof(double), s));
    BCK(h, cudaMemsetAsync(h->rbar, 0, Bn * sizeof(double), s));
    StepArgs st = h->st;
    for (int64_t k = h->k - 1; k >= 0; --k) {
        st.bk = static_cast<int>(k);
        BCK(h, enqueue_backward(h, st, s));
    }
    BCK(h, cudaMemcpyAsync(dG, h->dG, Bn * h->m * sizeof(float2), cudaMemcpyDefault, s));
    std::vector<double> kb(Bn), rb(Bn);
    BCK(h, cudaMemcpyAsync(kb.data(), h->kbar, Bn * sizeof(double), cudaMemcpyDeviceToHost, s));
    BCK(h, cudaMemcpyAsync(rb.data(), h->rbar, Bn * sizeof(double), cudaMemcpyDeviceToHost, s));
    const int code = check_status(h, s);
    const double M = h->M, rho = h->rho;
    for (size_t b = 0; b < Bn; ++b) {
        dlambda[b] = kb[b] / (M * rho);
        drho[b] = rb[b] - kb[b] * h->lam[b] / (M * rho * rho);
    }
    return code;
}

int admm_batch_status(admm_batch_t* h, void* stream) {
    if (!h) return ADMM_EINVAL;
    return check_status(h, static_cast<cudaStream_t>(stream));
}

int admm_batch_get_v(admm_batch_t* h, void* V, void* stream) {
    if (!h || !V) return h ? bfail(h, ADMM_EINVAL, "V is NULL") : ADMM_EINVAL;
    BCK(h, cudaMemcpyAsync(V, h->V, static_cast<size_t>(h->B) * h->n * sizeof(float2), cudaMemcpyDefault,
                           static_cast<cudaStream_t>(stream)));
    return ADMM_OK;
}

int admm_batch_get_residuals(admm_batch_t* h, double* out, void* stream) {
    if (!h || !out) return h ? bfail(h, ADMM_EINVAL, "out is NULL") : ADMM_EINVAL;
    const int code = check_status(h, static_cast<cudaStream_t>(stream));
    std::vector<double> r(2 * static_cast<size_t>(h->B));
    BCK(h, cudaMemcpy(r.data(), h->res, r.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int b = 0; b < h->B; ++b) {
        out[2 * b] = r[2 * b];
        out[2 * b + 1] = h->rho * h->rho * h->M * r[2 * b + 1];
    }
    return code;
}

int admm_batch_forward(admm_batch_t* h, const void* X, void* Y, void* stream) {
    if (!h || !X || !Y) return h ? bfail(h, ADMM_EINVAL, "X and Y must not be NULL") : ADMM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!h->X) {
        if (dalloc0(&h->X, static_cast<size_t>(h->B) * h->n) != cudaSuccess ||
            dalloc0(&h->Y, static_cast<size_t>(h->B) * h->m) != cudaSuccess)
            return bfail(h, ADMM_ENOMEM, "no room for the product buffers");
    }
    BCK(h, cudaMemcpyAsync(h->X, X, static_cast<size_t>(h->B) * h->n * sizeof(float2), cudaMemcpyDefault, s));
    PackArgs px = h->px;
    px.x = h->X;
    BCK(h, launch_pack(px, h->P, s));
    BCK(h, launch_gemm(h->mapH, h->mapZ, h->g1, s));
    BCK(h, launch_sum_blocks(h->Ppart, h->splits1, h->P, h->B, h->mpitch, h->st.row_off, h->M, h->N, 1, h->Y,
                             h->m, s));
    BCK(h, cudaMemcpyAsync(Y, h->Y, static_cast<size_t>(h->B) * h->m * sizeof(float2), cudaMemcpyDefault, s));
    return check_status(h, s);
}

int admm_batch_adjoint(admm_batch_t* h, const void* Y, void* X, void* stream) {
    if (!h || !X || !Y) return h ? bfail(h, ADMM_EINVAL, "X and Y must not be NULL") : ADMM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!h->X) {
        if (dalloc0(&h->X, static_cast<size_t>(h->B) * h->n) != cudaSuccess ||
            dalloc0(&h->Y, static_cast<size_t>(h->B) * h->m) != cudaSuccess)
            return bfail(h, ADMM_ENOMEM, "no room for the product buffers");
    }
    BCK(h, cudaMemcpyAsync(h->Y, Y, static_cast<size_t>(h->B) * h->m * sizeof(float2), cudaMemcpyDefault, s));
    PackArgs py = h->py;
    py.x = h->Y;
    BCK(h, launch_pack(py, h->P, s));
    BCK(h, launch_gemm(h->mapHT, h->mapW, h->g2, s));
    BCK(h, launch_sum_blocks(h->Sig, 1, h->P, h->B, h->npitch, h->st.col_off, h->N, h->N, 0, h->X, h->n, s));
    BCK(h, cudaMemcpyAsync(X, h->X, static_cast<size_t>(h->B) * h->n * sizeof(float2), cudaMemcpyDefault, s));
    return check_status(h, s);
}

int admm_batch_get_info(const admm_batch_t* h, admm_batch_info_t* info) {
    if (!h || !info) return ADMM_EINVAL;
    info->m = h->m;
    info->n = h->n;
    info->batch = h->B;
    info->row_blocks = h->M;
    info->col_blocks = h->N;
    info->iterations = h->k;
    info->splits = h->splits1;
    // tensor-core FLOPs of one iteration as issued (padding included): 2 * rows * cols * K per GEMM
    const double cols = 256.0 * ((4.0 * h->B + 255) / 256);
    const int mt1 = (h->mimax + 127) / 128, mt2 = (h->njmax + 127) / 128;
    double fl = 0.0;
    for (int p = 0; p < h->P; ++p) {
        const int i = p / h->N, j = p % h->N;
        const int mi = h->ro[i + 1] - h->ro[i], nj = h->co[j + 1] - h->co[j];
        fl += 2.0 * mt1 * 128 * cols * 64.0 * ((2 * nj + 63) / 64);   // H z
        fl += 2.0 * mt1 * 128 * cols * h->kr;                          // K^{-1} r
        fl += 2.0 * mt2 * 128 * cols * 64.0 * ((2 * mi + 63) / 64);   // H^H w
    }
    info->tensor_flops = fl;
    // complex products of the method (8 real flops per complex MAC), all scenes
    double useful = 0.0;
    for (int i = 0; i < h->M; ++i)
        for (int j = 0; j < h->N; ++j) {
            const double mi = h->ro[i + 1] - h->ro[i], nj = h->co[j + 1] - h->co[j];
            useful += 8.0 * h->B * (2 * mi * nj + mi * mi);
        }
    info->method_flops = useful;
    // state bytes per iteration: V read + written, S read + written, Sigma written + read,
    // packed z written + read (16 bytes per complex entry), G / Gt / Ghat / R / W (m-length, small)
    const double Bn = h->B, n = h->n, M = h->M, P = h->P;
    info->state_bytes = Bn * n * 8 * (2 + 2 * M) + Bn * h->npitch * 8.0 * 2 * P + Bn * h->kz * 2.0 * 4 * 2 * P +
                        Bn * h->m * 8.0 * (2 + 4 * h->N) + Bn * h->mpitch * 8.0 * P * (2 * h->splits1 + 4);
    return ADMM_OK;
}

void admm_batch_destroy(admm_batch_t* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    free_batch(h);
    delete h;
}

}  // extern "C"
