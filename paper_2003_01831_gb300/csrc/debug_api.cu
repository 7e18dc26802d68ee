// Diagnostic entry points (include/afqmc_debug.h): one tensor-core building block per
// call, host arrays in and out, for isolated parity tests.
#include <cmath>
#include <string>
#include <vector>

#include "../../include/afqmc_debug.h"
#include "kernels_fp64.cuh"
#include "kernels_tc.cuh"
#include "state.cuh"
#include "tc_ptx.cuh"

namespace afqmc {
namespace {

__global__ void split_kernel(const double* src, bf16* hi, bf16* lo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) tc::split_bf16(src[i], hi[i], lo[i]);
}

// Failure detection without a fault: one warp waits for a barrier phase that only completes
// when `release` is set (thread 0 arrives first), by the tensor-core kernels' bounded wait
// (mbarrier try_wait polled against a clock64 budget) with a budget of `limit` cycles.  A
// wait that runs out records FLAG_TIMEOUT and the kernel returns.
__global__ void wait_probe_kernel(long long limit, int release, unsigned* flags) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (release && threadIdx.x == 0) tc::mbar_arrive(&bar);
    const long long t0 = clock64();
    bool ok = true;
    while (!tc::mbar_try_wait(&bar, 0)) {
        if (clock64() - t0 > limit) {
            ok = false;
            break;
        }
    }
    if (!ok) atomicOr(flags, FLAG_TIMEOUT);
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

// Upload n = rows * K values; plain split, or row-scaled split when sc is given.
int upload_split(const double* h, int64_t rows, int64_t K, DevBuf& d64, DevBuf& hi, DevBuf& lo, DevBuf* sc,
                 DevBuf* rnd = nullptr) {
    const int64_t n = rows * K;
    if (cudaMalloc(&d64.p, n * 8) != cudaSuccess || cudaMalloc(&hi.p, n * 2) != cudaSuccess ||
        cudaMalloc(&lo.p, n * 2) != cudaSuccess || (sc && cudaMalloc(&sc->p, rows * 4) != cudaSuccess) ||
        (rnd && cudaMalloc(&rnd->p, n * 2) != cudaSuccess))
        return fail(AFQMC_ERR_OOM, "debug: allocation");
    AFQMC_CUDA_TRY(cudaMemcpy(d64.p, h, n * 8, cudaMemcpyHostToDevice));
    if (sc) {
        split_rows(static_cast<double*>(d64.p), K, rows, K, static_cast<bf16*>(hi.p), static_cast<bf16*>(lo.p),
                   static_cast<float*>(sc->p), 0, rnd ? static_cast<bf16*>(rnd->p) : nullptr);
    } else {
        split_kernel<<<(unsigned)((n + 255) / 256), 256>>>(static_cast<double*>(d64.p), static_cast<bf16*>(hi.p),
                                                           static_cast<bf16*>(lo.p), n);
    }
    return AFQMC_OK;
}

__global__ void f32_to_f64(const float* s, double* d, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = s[i];
}

}  // namespace
}  // namespace afqmc

using namespace afqmc;

extern "C" int afqmc_debug_split_gemm(const double* A, const double* B, int nbatch, int rows, int cols, int K, int BN,
                                      int exact, double* C) {
    if (!A || !B || !C || nbatch < 1 || rows < 1 || cols < 1 || K < 8 || K % 8)
        return fail(AFQMC_ERR_BADARG, "debug_split_gemm: bad arguments");
    const int64_t na = (int64_t)nbatch * rows * K, nb = (int64_t)nbatch * cols * K, nc = (int64_t)nbatch * rows * cols;
    DevBuf a64, ahi, alo, b64, bhi, blo, c32, c64, flags, asc, bsc;
    AFQMC_TRY(upload_split(A, na / K, K, a64, ahi, alo, exact ? &asc : nullptr));
    AFQMC_TRY(upload_split(B, nb / K, K, b64, bhi, blo, exact ? &bsc : nullptr));
    if (cudaMalloc(&c32.p, nc * 4) != cudaSuccess || cudaMalloc(&c64.p, nc * 8) != cudaSuccess ||
        cudaMalloc(&flags.p, 4) != cudaSuccess)
        return fail(AFQMC_ERR_OOM, "debug: allocation");
    cudaMemset(flags.p, 0, 4);
    cudaMemset(c32.p, 0, nc * 4);
    SplitMat sa, sb;
    sa.hi = static_cast<bf16*>(ahi.p); sa.lo = static_cast<bf16*>(alo.p);
    sa.K = K; sa.rows = rows; sa.batch = nbatch; sa.row_stride = K; sa.batch_stride = (int64_t)rows * K;
    sa.scale = exact ? static_cast<float*>(asc.p) : nullptr;
    sb.hi = static_cast<bf16*>(bhi.p); sb.lo = static_cast<bf16*>(blo.p);
    sb.K = K; sb.rows = cols; sb.batch = nbatch; sb.row_stride = K; sb.batch_stride = (int64_t)cols * K;
    sb.scale = exact ? static_cast<float*>(bsc.p) : nullptr;
    EpiParams e;
    e.kind = EPI_F32;
    e.rows_valid = rows; e.cols_valid = cols; e.ld = cols; e.ob = (int64_t)rows * cols;
    e.out_f32 = static_cast<float*>(c32.p);
    BatchMap bm;
    if (nbatch > 1) bm = BatchMap{1, nbatch};
    AFQMC_TRY(tc_gemm(sa, bm, sb, bm, rows, cols, K, nbatch, e, BN, exact != 0, static_cast<unsigned*>(flags.p), 0));
    f32_to_f64<<<(unsigned)((nc + 255) / 256), 256>>>(static_cast<float*>(c32.p), static_cast<double*>(c64.p), nc);
    AFQMC_CUDA_TRY(cudaDeviceSynchronize());
    unsigned fl = 0;
    AFQMC_CUDA_TRY(cudaMemcpy(&fl, flags.p, 4, cudaMemcpyDeviceToHost));
    if (fl & FLAG_TIMEOUT) return fail(AFQMC_ERR_TIMEOUT, "debug_split_gemm: device wait timed out");
    AFQMC_CUDA_TRY(cudaMemcpy(C, c64.p, nc * 8, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

extern "C" int afqmc_debug_energy(const double* Lt, const double* ThetaT, int Np, int Nchol, int nws, int M, int terms,
                                  double* t, double* X) {
    if (!Lt || !ThetaT || !t || !X || Nchol < 1 || nws < 1 || M < 64)
        return fail(AFQMC_ERR_BADARG, "debug_energy: bad arguments");
    const int64_t na = (int64_t)Nchol * Np * M, nb = (int64_t)nws * 2 * Np * M;
    if (terms < 3 || terms > 7) return fail(AFQMC_ERR_BADARG, "debug_energy: terms must be 3 to 7");
    const bool rounded = terms >= 5, single = terms >= 6;
    DevBuf a64, ahi, alo, arn, b64, bhi, blo, brn, dt, dx, flags, asc, bsc, sg;
    AFQMC_TRY(upload_split(Lt, na / M, M, a64, ahi, alo, &asc, rounded ? &arn : nullptr));
    AFQMC_TRY(upload_split(ThetaT, nb / M, M, b64, bhi, blo, &bsc, single ? &brn : nullptr));
    const int64_t no = (int64_t)nws * Nchol;
    const int G = 128 / Np, ng = (Nchol + G - 1) / G;
    if (cudaMalloc(&dt.p, no * 16) != cudaSuccess || cudaMalloc(&dx.p, no * 16) != cudaSuccess ||
        cudaMalloc(&flags.p, 4) != cudaSuccess || (single && cudaMalloc(&sg.p, (size_t)ng) != cudaSuccess))
        return fail(AFQMC_ERR_OOM, "debug: allocation");
    cudaMemset(flags.p, 0, 4);
    if (single) {   // 6: the odd pair tiles (n-groups 4 p + 2, 4 p + 3) single; 7: every tile
        std::vector<uint8_t> hs((size_t)ng);
        for (int g = 0; g < ng; ++g) hs[(size_t)g] = terms == 7 ? 1 : (uint8_t)((g / 2) % 2);
        AFQMC_CUDA_TRY(cudaMemcpy(sg.p, hs.data(), (size_t)ng, cudaMemcpyHostToDevice));
    }
    SplitMat sa, sb;
    sa.hi = static_cast<bf16*>(ahi.p); sa.lo = static_cast<bf16*>(alo.p);
    sa.K = M; sa.rows = (int64_t)Nchol * Np; sa.row_stride = M; sa.scale = static_cast<float*>(asc.p);
    sb.hi = static_cast<bf16*>(bhi.p); sb.lo = static_cast<bf16*>(blo.p);
    sb.K = M; sb.rows = (int64_t)nws * 2 * Np; sb.row_stride = M; sb.scale = static_cast<float*>(bsc.p);
    AFQMC_TRY(tc_energy(sa, sb, Np, Nchol, nws, M, static_cast<cplx*>(dt.p), static_cast<cplx*>(dx.p),
                        rounded ? kEnergyRounded : terms, nullptr, static_cast<bf16*>(arn.p),
                        static_cast<unsigned*>(flags.p), 0, single ? static_cast<uint8_t*>(sg.p) : nullptr,
                        static_cast<bf16*>(brn.p)));
    AFQMC_CUDA_TRY(cudaDeviceSynchronize());
    unsigned fl = 0;
    AFQMC_CUDA_TRY(cudaMemcpy(&fl, flags.p, 4, cudaMemcpyDeviceToHost));
    if (fl & FLAG_TIMEOUT) return fail(AFQMC_ERR_TIMEOUT, "debug_energy: device wait timed out");
    AFQMC_CUDA_TRY(cudaMemcpy(t, dt.p, no * 16, cudaMemcpyDeviceToHost));
    AFQMC_CUDA_TRY(cudaMemcpy(X, dx.p, no * 16, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

extern "C" int afqmc_debug_mixed_terms(afqmc_wk_debug_t wk, double* ST, double* Sinv, double* ThetaT, double* t,
                                       double* X, double* E1) {
    if (!wk) return fail(AFQMC_ERR_BADARG, "debug_mixed_terms: NULL handle");
    return tc_debug_terms(wk, ST, Sinv, ThetaT, t, X, E1);
}

extern "C" int afqmc_debug_inverse(const double* S, int N, int count, int variant, int with_inverse, double* Sout,
                                   double* logdet, float* ms) {
    if (!S || !logdet || N < 1 || count < 1 || variant < 0 || variant > 3 || (with_inverse && !Sout))
        return fail(AFQMC_ERR_BADARG, "debug_inverse: bad arguments");
    const int64_t n = (int64_t)count * N * N;
    DevBuf ds, dl, flags;
    if (cudaMalloc(&ds.p, n * 16) != cudaSuccess || cudaMalloc(&dl.p, (int64_t)count * 16) != cudaSuccess ||
        cudaMalloc(&flags.p, 4) != cudaSuccess)
        return fail(AFQMC_ERR_OOM, "debug: allocation");
    AFQMC_CUDA_TRY(cudaMemcpy(ds.p, S, n * 16, cudaMemcpyHostToDevice));
    cudaMemset(flags.p, 0, 4);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    LaunchPolicy saved = launch_policy();
    launch_policy().gj_variant = variant;
    cudaEventRecord(e0, 0);
    batched_inverse_logdet(static_cast<cplx*>(ds.p), (int64_t)N * N, N, count, static_cast<cplx*>(dl.p),
                           with_inverse != 0, static_cast<unsigned*>(flags.p), 0);
    cudaEventRecord(e1, 0);
    launch_policy() = saved;
    const cudaError_t le = cudaGetLastError();
    const cudaError_t se = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    AFQMC_CUDA_TRY(le);
    AFQMC_CUDA_TRY(se);
    if (ms) *ms = t;
    unsigned fl = 0;
    AFQMC_CUDA_TRY(cudaMemcpy(&fl, flags.p, 4, cudaMemcpyDeviceToHost));
    AFQMC_CUDA_TRY(cudaMemcpy(logdet, dl.p, (int64_t)count * 16, cudaMemcpyDeviceToHost));
    if (with_inverse) AFQMC_CUDA_TRY(cudaMemcpy(Sout, ds.p, n * 16, cudaMemcpyDeviceToHost));
    if (fl & FLAG_SINGULAR) return fail(AFQMC_ERR_SINGULAR, "debug_inverse: singular matrix");
    if (fl & FLAG_NONFINITE) return fail(AFQMC_ERR_NONFINITE, "debug_inverse: non-finite matrix");
    return AFQMC_OK;
}

extern "C" int afqmc_debug_select_energy_groups(const double* norms, int nch, int G, double eta,
                                                unsigned char* flags) {
    if (!norms || !flags || nch < 1 || G < 1 || !(eta >= 0.0 && eta < 1.0))
        return fail(AFQMC_ERR_BADARG, "debug_select_energy_groups: bad arguments");
    for (int n = 0; n < nch; ++n)
        if (!(norms[n] >= 0.0) || !std::isfinite(norms[n]))
            return fail(AFQMC_ERR_BADARG, "debug_select_energy_groups: norms must be finite and >= 0");
    select_lolo_groups(norms, nch, G, eta, flags);
    return AFQMC_OK;
}

extern "C" int afqmc_debug_select_single_groups(const double* sqnorms, int nch, int G, double eta,
                                                unsigned char* flags) {
    if (!sqnorms || !flags || nch < 1 || G < 1 || !(eta >= 0.0 && eta < 1.0))
        return fail(AFQMC_ERR_BADARG, "debug_select_single_groups: bad arguments");
    for (int n = 0; n < nch; ++n)
        if (!(sqnorms[n] >= 0.0) || !std::isfinite(sqnorms[n]))
            return fail(AFQMC_ERR_BADARG, "debug_select_single_groups: squared norms must be finite and >= 0");
    select_single_groups(sqnorms, nch, G, eta, flags);
    return AFQMC_OK;
}

extern "C" int afqmc_debug_set_energy_window(int ws_super) {
    if (ws_super < 0) return fail(AFQMC_ERR_BADARG, "debug_set_energy_window: negative window");
    launch_policy().energy_ws_super = ws_super;
    return AFQMC_OK;
}

extern "C" int afqmc_debug_energy_products(afqmc_wk_debug_t wk, double* mean) {
    if (!wk || !mean) return fail(AFQMC_ERR_BADARG, "debug_energy_products: NULL argument");
    return tc_energy_products(wk, mean);
}

extern "C" int afqmc_debug_set_launch_policy(int grid_cap, int bn_max, int energy_bk) {
    if (grid_cap < 0 || (bn_max != 0 && bn_max != 128 && bn_max != 256) ||
        (energy_bk != 0 && energy_bk != 16 && energy_bk != 32))
        return fail(AFQMC_ERR_BADARG, "debug_set_launch_policy: bad knob value");
    LaunchPolicy& p = launch_policy();
    p.grid_cap = grid_cap;
    p.bn_max = bn_max == 0 ? 256 : bn_max;
    p.energy_bk = energy_bk;
    return AFQMC_OK;
}

extern "C" int afqmc_debug_set_batch_padding(int granule) {
    if (granule != 8 && granule != 32) return fail(AFQMC_ERR_BADARG, "debug_set_batch_padding: granule must be 8 or 32");
    launch_policy().batch_n_granule = granule;
    return AFQMC_OK;
}

extern "C" int afqmc_debug_set_energy_variant(int pair) {
    if (pair != 0 && pair != 1) return fail(AFQMC_ERR_BADARG, "debug_set_energy_variant: pair must be 0 or 1");
    launch_policy().energy_pair = pair;
    return AFQMC_OK;
}

extern "C" int afqmc_debug_wait_probe(long long limit_cycles, int release, unsigned* status, float* ms) {
    if (!status) return fail(AFQMC_ERR_BADARG, "debug_wait_probe: status is NULL");
    if (limit_cycles < 1 || limit_cycles > tc::kTimeoutCycles)
        return fail(AFQMC_ERR_BADARG, "debug_wait_probe: limit outside 1 .. the production bound");
    DevBuf flags;
    if (cudaMalloc(&flags.p, sizeof(unsigned)) != cudaSuccess) return fail(AFQMC_ERR_OOM, "debug_wait_probe: flags");
    AFQMC_CUDA_TRY(cudaMemset(flags.p, 0, sizeof(unsigned)));
    cudaEvent_t e0, e1;
    AFQMC_CUDA_TRY(cudaEventCreate(&e0));
    AFQMC_CUDA_TRY(cudaEventCreate(&e1));
    cudaEventRecord(e0);
    count_launch();
    wait_probe_kernel<<<1, 32>>>(limit_cycles, release, static_cast<unsigned*>(flags.p));
    cudaEventRecord(e1);
    const cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(AFQMC_ERR_CUDA, std::string("debug_wait_probe: ") + cudaGetErrorString(e));
    AFQMC_CUDA_TRY(cudaMemcpy(status, flags.p, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (ms) *ms = t;
    return AFQMC_OK;
}
