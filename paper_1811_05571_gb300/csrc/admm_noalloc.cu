// Allocation-free small-problem solve: the same factor kernels and persistent
// iteration kernel as admm_setup + admm_iterate, with every piece of working
// memory carved out of one file-scope device array instead of cudaMalloc.
//
// Who needs this: code that may not allocate device memory itself -- a
// framework whose own pool allocator owns all of the GPU's memory, or a
// real-time loop that must not pay (or risk failing) an allocation.  They
// pass their own input and output buffers; the library's scratch is reserved
// once per device when the library loads.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include <cudaTypedefs.h>

#include "admm_internal.h"

namespace {

constexpr size_t kScratchBytes = static_cast<size_t>(8) << 20;   // 8 MiB per device
constexpr int kMaxDevices = 64;

// Device-side working memory of admm_solve_small_noalloc.  Host code must not
// use this name as a pointer: it is a host stand-in, so its device address is
// taken with cudaGetSymbolAddress (per device) before any kernel sees it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_scratch_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ADMM_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ADMM_ECUDA;
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return ADMM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct Carve {
    size_t used = 0;
    size_t take(size_t bytes) {
        const size_t at = used;
        used = align256(used + bytes);
        return at;
    }
};

// failures are described through admm_last_error(NULL)
int noalloc_fail(int code, const char* msg) {
    admm::set_handle_free_error(msg);
    return code;
}

// H, g and v_out are used in place by the kernels, so each must be device
// memory this device can address (cudaMalloc'd on it, or managed memory).
bool on_this_device(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // clear the error an unregistered host pointer may leave
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// the driver's tensor-map encoder, looked up once for every thread
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn_ptr = nullptr;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess && fn)
            fn_ptr = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return fn_ptr;
}

}  // namespace

extern "C" {

int admm_solve_small_noalloc(const void* H, const void* g, int64_t m, int64_t n, int32_t row_blocks,
                             int32_t col_blocks, double lambda, double rho, int32_t iters,
                             void* v_out, void* stream) {
    if (!H || !g || !v_out) return noalloc_fail(ADMM_EINVAL, "H, g and v_out must not be NULL");
    if (m < 1 || m > (1 << 20)) return noalloc_fail(ADMM_EINVAL, "need 1 <= m <= 2^20");
    if (n < 32 || n > (1 << 24) || n % 32 != 0)
        return noalloc_fail(ADMM_EINVAL, "need n a multiple of 32 in [32, 2^24]");
    if (reinterpret_cast<uintptr_t>(H) % 16 != 0)
        return noalloc_fail(ADMM_EINVAL, "H must be 16-byte aligned");
    if (row_blocks < 1 || row_blocks > m || col_blocks < 1 || col_blocks > n ||
        static_cast<int64_t>(row_blocks) * col_blocks > admm::kMaxBlocks)
        return noalloc_fail(ADMM_EINVAL, "bad row_blocks / col_blocks");
    if (!(lambda >= 0.0) || !std::isfinite(lambda) || !(rho > 0.0) || !std::isfinite(rho) || iters < 0)
        return noalloc_fail(ADMM_EINVAL, "need finite lambda >= 0, finite rho > 0, iters >= 0");
    {
        int cur = 0;
        if (cudaGetDevice(&cur) != cudaSuccess) return noalloc_fail(ADMM_ECUDA, "cudaGetDevice failed");
        if (!on_this_device(H, cur) || !on_this_device(g, cur) || !on_this_device(v_out, cur))
            return noalloc_fail(ADMM_EINVAL, "H, g and v_out must be device memory of the current device");
    }
    std::vector<int> ro, co;
    admm::balanced_offsets(m, row_blocks, ro);
    admm::balanced_offsets(n, col_blocks, co);

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, smem_optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_fail(ADMM_ECUDA, "cudaGetDevice failed");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    admm::Plan pl;
    const char* why = "";
    int code = admm::make_plan(m, n, row_blocks, col_blocks, ro, co, sms, smem_optin, pl, &why);
    if (code) return noalloc_fail(code, why);
    if (pl.ld != n) return noalloc_fail(ADMM_EINVAL, "n must be a multiple of 32");

    // carve the scratch: factors, FP64 factor workspace, state, products, flags
    const int M = row_blocks, N = col_blocks, nb = M * N;
    const int T = (pl.mimax + admm::kTile - 1) / admm::kTile;
    const size_t S = static_cast<size_t>(T) * admm::kTile;
    std::vector<long long> kinv_off(nb);
    std::vector<int> kinv_pitch(nb);
    size_t kel = 0;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < N; ++j) {
            const int mi = ro[i + 1] - ro[i];
            const int kp = (mi + 3) / 4 * 4;
            kinv_off[i * N + j] = static_cast<long long>(kel);
            kinv_pitch[i * N + j] = kp;
            kel += static_cast<size_t>(mi) * kp;
        }
    std::vector<int> ints;
    auto put = [&](const std::vector<int>& x) {
        const size_t at = ints.size();
        ints.insert(ints.end(), x.begin(), x.end());
        return at;
    };
    const size_t o_row = put(ro), o_col = put(co), o_beg = put(pl.cta_beg), o_end = put(pl.cta_end),
                 o_own0 = put(pl.cta_own0), o_own1 = put(pl.cta_own1), o_jlo = put(pl.cta_jlo),
                 o_nj = put(pl.cta_nj), o_jl = put(pl.j_cta_lo), o_jh = put(pl.j_cta_hi),
                 o_sl = put(pl.solve_lo), o_kp = put(kinv_pitch);
    const size_t ld = pl.ld;
    const size_t Nm = static_cast<size_t>(N) * m;
    Carve cv;
    const size_t x_A = cv.take(S * S * nb * sizeof(double2));
    const size_t x_W = cv.take(S * S * nb * sizeof(double2));
    const size_t x_kinv = cv.take(kel * sizeof(float2));
    const size_t x_koff = cv.take(nb * sizeof(long long));
    const size_t x_ints = cv.take(ints.size() * sizeof(int));
    const size_t x_v = cv.take(ld * sizeof(float2));
    const size_t x_s = cv.take(ld * M * sizeof(float2));
    const size_t x_u = cv.take(ld * M * sizeof(float2));
    const size_t x_ghat = cv.take(2 * Nm * sizeof(float2));
    const size_t x_gt = cv.take(Nm * sizeof(float2));
    const size_t x_r = cv.take(Nm * sizeof(float2));
    const size_t x_w = cv.take(Nm * sizeof(float2));
    const size_t x_part = cv.take(Nm * pl.P * pl.groups * sizeof(float2));
    const size_t x_res = cv.take(static_cast<size_t>(pl.P) * 8 * sizeof(double));
    const size_t x_hist = cv.take(5 * sizeof(double));
    const size_t x_kdone = cv.take(sizeof(long long));
    const size_t x_bar = cv.take(2 * sizeof(unsigned));
    const size_t x_status = cv.take(sizeof(int));
    const size_t x_stop = cv.take(sizeof(int));
    if (cv.used > kScratchBytes)
        return noalloc_fail(ADMM_EINVAL, "problem needs more than the 8 MiB allocation-free scratch");

    unsigned char* base = nullptr;
    if (scratch_for_current_device(&base) != ADMM_OK)
        return noalloc_fail(ADMM_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
    auto at = [&](size_t off) { return base + off; };
    float2* kinv = reinterpret_cast<float2*>(at(x_kinv));
    long long* koff_d = reinterpret_cast<long long*>(at(x_koff));
    int* ints_d = reinterpret_cast<int*>(at(x_ints));
    float2* v = reinterpret_cast<float2*>(at(x_v));
    float2* s = reinterpret_cast<float2*>(at(x_s));
    float2* u = reinterpret_cast<float2*>(at(x_u));
    float2* ghat = reinterpret_cast<float2*>(at(x_ghat));
    int* status = reinterpret_cast<int*>(at(x_status));

#define NA_CK(call)                                                        \
    do {                                                                   \
        if ((call) != cudaSuccess) return noalloc_fail(ADMM_ECUDA, #call); \
    } while (0)

    // tables, then everything that must start at zero (the array keeps the
    // previous call's contents)
    NA_CK(cudaMemcpyAsync(ints_d, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(koff_d, kinv_off.data(), nb * sizeof(long long), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemsetAsync(kinv, 0, kel * sizeof(float2), st));
    NA_CK(cudaMemsetAsync(at(x_v), 0, x_part - x_v, st));          // v, s, u, ghat, gt, r, w
    NA_CK(cudaMemsetAsync(at(x_hist), 0, cv.used - x_hist, st));   // history, counters, flags

    // non-finite inputs: checked before any factor or iteration kernel runs
    {
        int flag = 0;
        NA_CK(admm::launch_finite_check(static_cast<const float2*>(H), m * n, status, st));
        NA_CK(admm::launch_finite_check(static_cast<const float2*>(g), m, status, st));
        NA_CK(cudaMemcpyAsync(&flag, status, sizeof(int), cudaMemcpyDeviceToHost, st));
        NA_CK(cudaStreamSynchronize(st));
        if (flag) return noalloc_fail(ADMM_ENONFINITE, "H or g holds NaN or Inf");
    }

    admm::FactorArgs f;
    f.m = static_cast<int>(m);
    f.ld = static_cast<int>(ld);
    f.M = M;
    f.N = N;
    f.T = T;
    f.row_off = ints_d + o_row;
    f.col_off = ints_d + o_col;
    f.H = static_cast<const float2*>(H);
    f.A = reinterpret_cast<double2*>(at(x_A));
    f.W = reinterpret_cast<double2*>(at(x_W));
    f.kinv = kinv;
    f.kinv_off = koff_d;
    f.kinv_pitch = ints_d + o_kp;
    f.rho = rho;
    f.status = status;
    NA_CK(admm::launch_gram(f, st));
    NA_CK(admm::launch_cholesky_inverse(f, st));

    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return noalloc_fail(ADMM_ECUDA, "cuTensorMapEncodeTiled is not available");
    CUtensorMap tmap;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(ld), static_cast<cuuint64_t>(m)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * sizeof(float2)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(pl.wbox), static_cast<cuuint32_t>(pl.R)};
    cuuint32_t estr[2] = {1, 1};
    if (encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(H), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return noalloc_fail(ADMM_ECUDA, "cuTensorMapEncodeTiled failed");

    if (iters > 0) {
        NA_CK(admm::prepare_iterate(pl.chunks, smem_optin, pl.groups));
        admm::IterArgs a;
        std::memset(&a, 0, sizeof a);
        a.m = static_cast<int>(m);
        a.n = static_cast<int>(n);
        a.ld = pl.ld;
        a.M = M;
        a.N = N;
        a.P = pl.P;
        a.R = pl.R;
        a.nstages = pl.nstages;
        a.stage_bytes = pl.stage_bytes;
        a.stage_stride = pl.stage_stride;
        a.sub_bytes = pl.sub_bytes;
        a.nsub = pl.nsub;
        a.wbox = pl.wbox;
        a.elem_bytes = 8;
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
        a.rho = static_cast<float>(rho);
        a.rho_d = rho;
        a.kappa = static_cast<float>(lambda / (M * rho));
        a.inv_M = 1.0f / static_cast<float>(M);
        a.row_off = ints_d + o_row;
        a.col_off = ints_d + o_col;
        a.cta_col = ints_d + o_beg;
        a.cta_end = ints_d + o_end;
        a.cta_own0 = ints_d + o_own0;
        a.cta_own1 = ints_d + o_own1;
        a.cta_jlo = ints_d + o_jlo;
        a.cta_nj = ints_d + o_nj;
        a.j_cta_lo = ints_d + o_jl;
        a.j_cta_hi = ints_d + o_jh;
        a.solve_lo = ints_d + o_sl;
        a.v = v;
        a.s = s;
        a.u = u;
        a.g = static_cast<const float2*>(g);
        a.ghat = ghat;
        a.gt = reinterpret_cast<float2*>(at(x_gt));
        a.r = reinterpret_cast<float2*>(at(x_r));
        a.w = reinterpret_cast<float2*>(at(x_w));
        a.part = reinterpret_cast<float2*>(at(x_part));
        a.kinv = kinv;
        a.kinv_off = koff_d;
        a.kinv_pitch = ints_d + o_kp;
        a.res_part = reinterpret_cast<double*>(at(x_res));
        a.hist = reinterpret_cast<double*>(at(x_hist));
        a.k_done = reinterpret_cast<long long*>(at(x_kdone));
        a.bar = reinterpret_cast<unsigned*>(at(x_bar));
        a.status = status;
        a.stop_flag = reinterpret_cast<int*>(at(x_stop));
        a.k0 = 0;
        a.hist_cap = 1;
        a.iters = iters;
        a.timeout_ns = 5000000000LL;
        a.keep_stages = static_cast<int>((52LL << 20) / (static_cast<long long>(pl.R) * pl.ld * 8));
        a.pending_prev = 0;
        NA_CK(admm::launch_iterate(tmap, a, pl.chunks, pl.smem, st));
    }
    NA_CK(cudaMemcpyAsync(v_out, v, static_cast<size_t>(n) * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    int dev_status = 0;
    NA_CK(cudaMemcpyAsync(&dev_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
    if (dev_status == ADMM_ENOTPD) return noalloc_fail(ADMM_ENOTPD, "a factor was not positive definite");
    if (dev_status != 0) return noalloc_fail(dev_status, "device status raised during the solve");
    return ADMM_OK;
}

}  // extern "C"
