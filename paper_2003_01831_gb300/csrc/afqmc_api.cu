// C-ABI front end of the AFQMC library: argument validation, host/device pointer
// handling, handle lifetime, set-up of the rotated Cholesky tensor, one-body
// propagator and trial energy, and the step loop.  The operations are those of
// Sec. V (Eqs. (1), (3)) and the phaseless algorithm it cites; see include/afqmc.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "state.cuh"

namespace afqmc {

namespace {
thread_local std::string g_last_error;

__global__ void cplx_real_part_kernel(const cplx* s, double* d, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = s[i].re;
}

// out[b][c][r] = in[b][r][c] for `nb` matrices of rows x cols
template <typename T>
__global__ void batched_transpose_kernel(const T* in, T* out, int nb, int rows, int cols) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)rows * cols;
    if (i >= per * nb) return;
    const int64_t b = i / per, e = i % per;
    const int r = (int)(e / cols), c = (int)(e % cols);
    out[b * per + (int64_t)c * rows + r] = in[i];
}

// flag = 1 when the two arrays differ anywhere (exact comparison)
__global__ void differ_kernel(const cplx* a, const cplx* b, int64_t n, unsigned* flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (a[i].re != b[i].re || a[i].im != b[i].im)) atomicOr(flag, 1u);
}

__global__ void max_abs_imag_kernel(const cplx* p, int64_t n, unsigned* flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && p[i].im != 0.0) atomicOr(flag, 1u);
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

void set_error(int code, const std::string& msg) {
    (void)code;
    g_last_error = msg;
}

LaunchPolicy& launch_policy() {
    static thread_local LaunchPolicy p;
    return p;
}

cudaError_t raise_dyn_smem(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> set;   // (device, kernel) -> limit set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = set[{dev, func}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

bool stream_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

int fail(int code, const std::string& msg) {
    set_error(code, msg);
    return code;
}

// true if p is device (or managed) memory
bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int copy_in(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (bytes == 0) return AFQMC_OK;
    AFQMC_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
    return AFQMC_OK;
}

// Copy device data to a caller pointer; synchronise if the destination is host memory.
int copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st, bool* needs_sync) {
    if (!dst || bytes == 0) return AFQMC_OK;
    AFQMC_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
    if (!is_device_ptr(dst)) *needs_sync = true;
    return AFQMC_OK;
}

int read_flags(unsigned* dflags, cudaStream_t st, unsigned* out) {
    unsigned h = 0;
    AFQMC_CUDA_TRY(cudaMemcpyAsync(&h, dflags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
    *out = h;
    return AFQMC_OK;
}

int flags_to_error(unsigned f, const char* where) {
    if (f & FLAG_TIMEOUT) return fail(AFQMC_ERR_TIMEOUT, std::string(where) + ": a bounded device wait gave up");
    if (f & FLAG_NONFINITE) return fail(AFQMC_ERR_NONFINITE, std::string(where) + ": NaN/Inf in input or result");
    if (f & FLAG_SINGULAR) return fail(AFQMC_ERR_SINGULAR, std::string(where) + ": singular overlap matrix");
    return AFQMC_OK;
}

}  // namespace afqmc

using namespace afqmc;

extern "C" {

void afqmc_default_opts(afqmc_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = AFQMC_PREC_FP64;
    o->k_taylor = 6;
    o->k_qr = 5;
    o->weight_mode = AFQMC_WEIGHT_PHASELESS;
    o->fb_cap = 1.0;
}

const char* afqmc_last_error(void) { return afqmc::g_last_error.c_str(); }

int afqmc_create_hamiltonian(const double* h, const double* L, double E0, int M, int Nchol, void* stream,
                             afqmc_ham_t* out) {
    if (!out) return fail(AFQMC_ERR_BADARG, "create_hamiltonian: out is NULL");
    *out = nullptr;
    if (!h || !L) return fail(AFQMC_ERR_BADARG, "create_hamiltonian: h or L is NULL");
    if (M < 1 || M > 1024 || Nchol < 1) return fail(AFQMC_ERR_SHAPE, "create_hamiltonian: need 1 <= M <= 1024, Nchol >= 1");
    if (!isfinite(E0)) return fail(AFQMC_ERR_NONFINITE, "create_hamiltonian: E0 not finite");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    afqmc_ham* H = new afqmc_ham();
    AFQMC_CUDA_TRY(cudaGetDevice(&H->device));
    H->M = M;
    H->Nchol = Nchol;
    H->E0 = E0;
    const size_t mm = (size_t)M * M;
    auto cleanup = [&](int rc) {
        if (H->h) cudaFree(H->h);
        if (H->L) cudaFree(H->L);
        if (H->hp) cudaFree(H->hp);
        if (H->flags) cudaFree(H->flags);
        delete H;
        return rc;
    };
    if (cudaMalloc(&H->h, mm * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&H->L, mm * Nchol * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&H->hp, mm * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&H->flags, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(AFQMC_ERR_OOM, "create_hamiltonian: device allocation failed"));
    }
    int rc = copy_in(H->h, h, mm * sizeof(double), st);
    if (rc == AFQMC_OK) rc = copy_in(H->L, L, mm * Nchol * sizeof(double), st);
    if (rc != AFQMC_OK) return cleanup(rc);
    cudaMemsetAsync(H->flags, 0, sizeof(unsigned), st);
    check_finite(H->h, (int64_t)mm, H->flags, st);
    check_finite(H->L, (int64_t)mm * Nchol, H->flags, st);
    check_symmetric(H->L, M, Nchol, H->flags, st);
    unsigned f = 0;
    rc = read_flags(H->flags, st, &f);
    if (rc != AFQMC_OK) return cleanup(rc);
    if (f & FLAG_NONFINITE) return cleanup(fail(AFQMC_ERR_NONFINITE, "create_hamiltonian: NaN/Inf in h or L"));
    if (f & 8u) return cleanup(fail(AFQMC_ERR_UNSUPPORTED, "create_hamiltonian: each L_n must be symmetric"));
    build_hprime(H->h, H->L, M, Nchol, H->hp, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cleanup(fail(AFQMC_ERR_CUDA, std::string("create_hamiltonian: ") + cudaGetErrorString(e)));
    *out = H;
    return AFQMC_OK;
}

int afqmc_create_hamiltonian_complex(const double* h, const double* L, double E0, int M, int Nchol, void* stream,
                                     afqmc_ham_t* out) {
    if (!out) return fail(AFQMC_ERR_BADARG, "create_hamiltonian_complex: out is NULL");
    *out = nullptr;
    if (!h || !L) return fail(AFQMC_ERR_BADARG, "create_hamiltonian_complex: h or L is NULL");
    if (M < 1 || M > 1024 || Nchol < 1 || Nchol > (1 << 29))
        return fail(AFQMC_ERR_SHAPE, "create_hamiltonian_complex: need 1 <= M <= 1024, Nchol >= 1");
    if (!isfinite(E0)) return fail(AFQMC_ERR_NONFINITE, "create_hamiltonian_complex: E0 not finite");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    afqmc_ham* H = new afqmc_ham();
    AFQMC_CUDA_TRY(cudaGetDevice(&H->device));
    const int Nv = 2 * Nchol;   // Hermitian split: two vectors per input vector
    H->M = M;
    H->Nchol = Nv;
    H->E0 = E0;
    H->cplx_L = true;
    const size_t mm = (size_t)M * M;
    cplx* Lin = nullptr;
    auto cleanup = [&](int rc) {
        if (Lin) cudaFree(Lin);
        if (H->h) cudaFree(H->h);
        if (H->L) cudaFree(H->L);
        if (H->hp) cudaFree(H->hp);
        if (H->flags) cudaFree(H->flags);
        delete H;
        return rc;
    };
    if (cudaMalloc(&H->h, mm * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&Lin, mm * Nchol * sizeof(cplx)) != cudaSuccess ||
        cudaMalloc(&H->L, mm * Nv * sizeof(cplx)) != cudaSuccess ||
        cudaMalloc(&H->hp, mm * sizeof(cplx)) != cudaSuccess ||
        cudaMalloc(&H->flags, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(AFQMC_ERR_OOM, "create_hamiltonian_complex: device allocation failed"));
    }
    int rc = copy_in(H->h, h, mm * sizeof(double), st);
    if (rc == AFQMC_OK) rc = copy_in(Lin, L, mm * Nchol * sizeof(cplx), st);
    if (rc != AFQMC_OK) return cleanup(rc);
    cudaMemsetAsync(H->flags, 0, sizeof(unsigned), st);
    check_finite(H->h, (int64_t)mm, H->flags, st);
    check_finite(reinterpret_cast<const double*>(Lin), 2 * (int64_t)mm * Nchol, H->flags, st);
    unsigned f = 0;
    rc = read_flags(H->flags, st, &f);
    if (rc != AFQMC_OK) return cleanup(rc);
    if (f & FLAG_NONFINITE) return cleanup(fail(AFQMC_ERR_NONFINITE, "create_hamiltonian_complex: NaN/Inf in h or L"));
    hermitian_split(Lin, M, Nchol, reinterpret_cast<cplx*>(H->L), st);
    build_hprime_hermitian(H->h, reinterpret_cast<const cplx*>(H->L), M, Nv, reinterpret_cast<cplx*>(H->hp), st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cleanup(fail(AFQMC_ERR_CUDA, std::string("create_hamiltonian_complex: ") + cudaGetErrorString(e)));
    cudaFree(Lin);
    Lin = nullptr;
    *out = H;
    return AFQMC_OK;
}

int afqmc_create_hamiltonian_thc(const double* h, const double* X, const double* Mk, double E0, int M, int Nmu,
                                 void* stream, afqmc_ham_t* out) {
    if (!out) return fail(AFQMC_ERR_BADARG, "create_hamiltonian_thc: out is NULL");
    *out = nullptr;
    if (!h || !X || !Mk) return fail(AFQMC_ERR_BADARG, "create_hamiltonian_thc: h, X or Mk is NULL");
    if (M < 1 || M > 1024 || Nmu < 1 || Nmu > 8192)
        return fail(AFQMC_ERR_SHAPE, "create_hamiltonian_thc: need 1 <= M <= 1024, 1 <= Nmu <= 8192");
    if (!isfinite(E0)) return fail(AFQMC_ERR_NONFINITE, "create_hamiltonian_thc: E0 not finite");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    afqmc_ham* H = new afqmc_ham();
    AFQMC_CUDA_TRY(cudaGetDevice(&H->device));
    H->M = M;
    H->E0 = E0;
    H->Nmu = Nmu;
    const size_t mm = (size_t)M * M, mq = (size_t)M * Nmu, qq = (size_t)Nmu * Nmu;
    double* work = nullptr;   // factor scratch, then real Nmu x Nmu products
    cplx* cw = nullptr;       // complex GEMM outputs (Nmu x Nmu, then M x Nmu and M x M)
    auto cleanup = [&](int rc) {
        void* ps[] = {H->h, H->hp, H->X, H->Mk, H->U, H->flags, work, cw};
        for (void* q : ps)
            if (q) cudaFree(q);
        delete H;
        return rc;
    };
    if (cudaMalloc(&H->h, mm * sizeof(double)) != cudaSuccess || cudaMalloc(&H->hp, mm * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&H->X, mq * sizeof(double)) != cudaSuccess || cudaMalloc(&H->Mk, qq * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&H->U, qq * sizeof(double)) != cudaSuccess || cudaMalloc(&H->flags, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&work, (qq + 3 * (size_t)Nmu) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&cw, std::max(qq, std::max(mq, mm)) * sizeof(cplx)) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(AFQMC_ERR_OOM, "create_hamiltonian_thc: device allocation failed"));
    }
    int rc = copy_in(H->h, h, mm * sizeof(double), st);
    if (rc == AFQMC_OK) rc = copy_in(H->X, X, mq * sizeof(double), st);
    if (rc == AFQMC_OK) rc = copy_in(H->Mk, Mk, qq * sizeof(double), st);
    if (rc != AFQMC_OK) return cleanup(rc);
    cudaMemsetAsync(H->flags, 0, sizeof(unsigned), st);
    check_finite(H->h, (int64_t)mm, H->flags, st);
    check_finite(H->X, (int64_t)mq, H->flags, st);
    check_finite(H->Mk, (int64_t)qq, H->flags, st);
    check_symmetric(H->Mk, Nmu, 1, H->flags, st);
    unsigned f = 0;
    rc = read_flags(H->flags, st, &f);
    if (rc != AFQMC_OK) return cleanup(rc);
    if (f & FLAG_NONFINITE) return cleanup(fail(AFQMC_ERR_NONFINITE, "create_hamiltonian_thc: NaN/Inf in h, X or Mk"));
    if (f & 8u) return cleanup(fail(AFQMC_ERR_BADARG, "create_hamiltonian_thc: the kernel Mk must be symmetric"));
    // M = U U^T: the modified (diagonally pivoted) Cholesky of the kernel
    int rank = 0;
    rc = thc_pivoted_cholesky(H->Mk, Nmu, 1e-12, work, H->U, &rank, st);
    if (rc != AFQMC_OK) return cleanup(rc);
    if (rank < 1) return cleanup(fail(AFQMC_ERR_BADARG, "create_hamiltonian_thc: the kernel has no positive direction"));
    H->Nchol = rank;
    // h' = h - 1/2 X [(X^T X) o (U U^T)] X^T
    double* P = work;   // [Nmu][Nmu] real
    {
        GemmArgs g;   // cw = U U^T
        g.m = Nmu; g.n = Nmu; g.k = rank;
        g.A.ptr = H->U; g.A.real = true; g.A.ld = rank;
        g.B.ptr = H->U; g.B.real = true; g.B.op = OP_T; g.B.ld = rank;
        g.C = cw; g.ldc = Nmu;
        zgemm(g, st);
        real_part(cw, P, (int64_t)qq, st);                // P = U U^T
        GemmArgs x;   // cw = X^T X
        x.m = Nmu; x.n = Nmu; x.k = M;
        x.A.ptr = H->X; x.A.real = true; x.A.op = OP_T; x.A.ld = Nmu;
        x.B.ptr = H->X; x.B.real = true; x.B.ld = Nmu;
        x.C = cw; x.ldc = Nmu;
        zgemm(x, st);
        real_part_times(cw, P, P, (int64_t)qq, st);       // P = (X^T X) o (U U^T)
        GemmArgs g1;   // cw = X P   [M][Nmu]
        g1.m = M; g1.n = Nmu; g1.k = Nmu;
        g1.A.ptr = H->X; g1.A.real = true; g1.A.ld = Nmu;
        g1.B.ptr = P; g1.B.real = true; g1.B.ld = Nmu;
        g1.C = cw; g1.ldc = Nmu;
        zgemm(g1, st);
    }
    cplx* R = nullptr;
    if (cudaMallocAsync(&R, mm * sizeof(cplx), st) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(AFQMC_ERR_OOM, "create_hamiltonian_thc: workspace"));
    }
    {
        GemmArgs g2;   // R = (X P) X^T   [M][M]
        g2.m = M; g2.n = M; g2.k = Nmu;
        g2.A.ptr = cw; g2.A.ld = Nmu;
        g2.B.ptr = H->X; g2.B.real = true; g2.B.op = OP_T; g2.B.ld = Nmu;
        g2.C = R; g2.ldc = M;
        zgemm(g2, st);
    }
    hprime_from(H->h, R, H->hp, (int64_t)mm, st);
    cudaFreeAsync(R, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(work);
    cudaFree(cw);
    work = nullptr;
    cw = nullptr;
    if (e != cudaSuccess) return cleanup(fail(AFQMC_ERR_CUDA, std::string("create_hamiltonian_thc: ") + cudaGetErrorString(e)));
    *out = H;
    return AFQMC_OK;
}

int afqmc_hamiltonian_info(afqmc_ham_t H, int* M, int* Nchol, int* Nmu) {
    if (!H) return fail(AFQMC_ERR_BADARG, "hamiltonian_info: NULL handle");
    if (M) *M = H->M;
    if (Nchol) *Nchol = H->Nchol;
    if (Nmu) *Nmu = H->Nmu;
    return AFQMC_OK;
}

int afqmc_destroy_hamiltonian(afqmc_ham_t H) {
    if (!H) return fail(AFQMC_ERR_BADARG, "destroy_hamiltonian: NULL handle");
    if (H->live_walker_sets > 0) return fail(AFQMC_ERR_BADARG, "destroy_hamiltonian: walker sets still use it");
    cudaFree(H->h);
    cudaFree(H->L);
    cudaFree(H->hp);
    cudaFree(H->X);
    cudaFree(H->Mk);
    cudaFree(H->U);
    cudaFree(H->flags);
    delete H;
    return AFQMC_OK;
}

static void free_walkers(afqmc_walkers* wk) {
    bp_close(wk);
    fp64_free(wk);
    tc_free(wk);
    void* ps[] = {wk->weight, wk->logS_old, wk->logS_new, wk->E_L, wk->xbar, wk->coef,
                  wk->accept, wk->x, wk->emix, wk->esum, wk->flags};
    for (void* p : ps)
        if (p) cudaFree(p);
    if (wk->ev0) cudaEventDestroy(wk->ev0);
    if (wk->ev1) cudaEventDestroy(wk->ev1);
    delete wk;
}

}  // extern "C"

// Walker set on a trial of ND determinants (coef: their complex coefficients, or NULL for one
// determinant); Psi_up / Psi_dn hold the determinants one after another.
static int init_walkers_impl(afqmc_ham_t ham, int ND, const double* Psi_up, const double* Psi_dn, const double* coef,
                             int Nup, int Ndn, int W, const double* Phi0, double tau, const afqmc_opts* opts,
                             void* stream, afqmc_wk_t* out) {
    if (!out) return fail(AFQMC_ERR_BADARG, "init_walkers: out is NULL");
    *out = nullptr;
    if (!ham || !Psi_up || !Psi_dn) return fail(AFQMC_ERR_BADARG, "init_walkers: NULL handle or trial");
    if (ND < 1 || ND > kMaxDets) return fail(AFQMC_ERR_SHAPE, "init_walkers: need 1 <= ND <= 1024 determinants");
    std::vector<cplx> c_host(ND, cplx{1.0, 0.0});
    int ref = 0;   // walkers start at the determinant with the largest |c_I| (lowest index on ties)
    if (coef) {
        AFQMC_CUDA_TRY(cudaMemcpy(c_host.data(), coef, sizeof(cplx) * ND, cudaMemcpyDefault));
        bool any = false;
        for (int I = 0; I < ND; ++I) {
            if (!isfinite(c_host[I].re) || !isfinite(c_host[I].im))
                return fail(AFQMC_ERR_NONFINITE, "init_walkers: non-finite determinant coefficient");
            any = any || c_host[I].re != 0.0 || c_host[I].im != 0.0;
            if (hypot(c_host[I].re, c_host[I].im) > hypot(c_host[ref].re, c_host[ref].im)) ref = I;
        }
        if (!any) return fail(AFQMC_ERR_BADARG, "init_walkers: every determinant coefficient is zero");
    }
    afqmc_opts o;
    afqmc_default_opts(&o);
    if (opts) o = *opts;
    const int M = ham->M;
    if (Nup < 1 || Ndn < 1 || Nup > std::min(M, 128) || Ndn > std::min(M, 128) || W < 1)
        return fail(AFQMC_ERR_SHAPE, "init_walkers: need 1 <= Nup, Ndn <= min(M, 128) and W >= 1");
    if (!(tau > 0.0) || !isfinite(tau)) return fail(AFQMC_ERR_BADARG, "init_walkers: tau must be > 0");
    if (o.k_taylor < 1 || o.k_taylor > 32 || o.k_qr < 0 ||
        (o.weight_mode != AFQMC_WEIGHT_PHASELESS && o.weight_mode != AFQMC_WEIGHT_FREE &&
         o.weight_mode != AFQMC_WEIGHT_LOCAL) ||
        (o.precision != AFQMC_PREC_FP64 && o.precision != AFQMC_PREC_BF16X3) || !isfinite(o.fb_cap))
        return fail(AFQMC_ERR_BADARG, "init_walkers: invalid option value");
    for (int r : o.reserved)
        if (r != 0) return fail(AFQMC_ERR_BADARG, "init_walkers: reserved options must be zero");
    if (o.walker_offset < 0) return fail(AFQMC_ERR_BADARG, "init_walkers: walker_offset must be >= 0");
    if (o.energy_terms < 0 || o.energy_terms > 4)
        return fail(AFQMC_ERR_BADARG, "init_walkers: energy_terms must be 0, 1, 2, 3 or 4");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    AFQMC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != ham->device) return fail(AFQMC_ERR_BADARG, "init_walkers: current device differs from the Hamiltonian's");

    afqmc_walkers* wk = new afqmc_walkers();
    wk->ham = ham;
    wk->device = dev;
    wk->M = M;
    wk->Nchol = ham->Nchol;
    wk->N[0] = Nup;
    wk->N[1] = Ndn;
    wk->W = W;
    wk->ND = ND;
    wk->tau = tau;
    wk->opts = o;
    const int nch = ham->Nchol;
    auto bail = [&](int rc) {
        free_walkers(wk);
        return rc;
    };
    auto al = [&](void** p, size_t bytes) -> int {
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            return fail(AFQMC_ERR_OOM, "init_walkers: device allocation failed");
        }
        return AFQMC_OK;
    };
    int rc = AFQMC_OK;
    rc = rc ? rc : al((void**)&wk->weight, sizeof(cplx) * W);
    rc = rc ? rc : al((void**)&wk->logS_old, sizeof(cplx) * W);
    rc = rc ? rc : al((void**)&wk->logS_new, sizeof(cplx) * W);
    rc = rc ? rc : al((void**)&wk->E_L, sizeof(cplx) * W);
    rc = rc ? rc : al((void**)&wk->xbar, sizeof(cplx) * W * nch);
    rc = rc ? rc : al((void**)&wk->coef, sizeof(cplx) * W * nch);
    rc = rc ? rc : al((void**)&wk->accept, sizeof(int) * W);
    rc = rc ? rc : al((void**)&wk->x, sizeof(double) * W * nch);
    rc = rc ? rc : al((void**)&wk->emix, sizeof(cplx) * 64);
    rc = rc ? rc : al((void**)&wk->esum, sizeof(cplx) * 2 * 64);
    rc = rc ? rc : al((void**)&wk->flags, 2 * sizeof(unsigned));
    if (rc) return bail(rc);
    wk->x_cap = 1;
    wk->emix_cap = 64;
    rc = fp64_alloc(wk);
    if (rc) return bail(rc);
    cudaEventCreate(&wk->ev0);
    cudaEventCreate(&wk->ev1);

    Fp64Buffers& f = wk->f;
    const double* psis[2] = {Psi_up, Psi_dn};
    // flags[0]: latched status bits; flags[1]: scratch word (imaginary part of the trial)
    cudaMemsetAsync(wk->flags, 0, 2 * sizeof(unsigned), st);
    for (int s = 0; s < 2; ++s) {
        const int64_t n = (int64_t)ND * M * wk->N[s];
        rc = copy_in(f.Psi[s], psis[s], sizeof(cplx) * n, st);
        if (rc) return bail(rc);
        check_finite(reinterpret_cast<const double*>(f.Psi[s]), 2 * n, wk->flags, st);
        count_launch();
        max_abs_imag_kernel<<<nblk(n), 256, 0, st>>>(f.Psi[s], n, wk->flags + 1);
    }
    unsigned* dspin = nullptr;   // BF16X3 forms one trial operand for both spins: Psi_up == Psi_dn
    if (o.precision == AFQMC_PREC_BF16X3 && Nup == Ndn) {
        if (cudaMallocAsync(&dspin, sizeof(unsigned), st) != cudaSuccess) return bail(fail(AFQMC_ERR_OOM, "init_walkers: workspace"));
        cudaMemsetAsync(dspin, 0, sizeof(unsigned), st);
        const int64_t n = (int64_t)ND * M * Nup;
        count_launch();
        differ_kernel<<<nblk(n), 256, 0, st>>>(f.Psi[0], f.Psi[1], n, dspin);
    }
    if (ND > 1) {   // conj(c_I), the factors of <psi_T| = sum_I conj(c_I) <D_I|
        for (cplx& c : c_host) c.im = -c.im;
        rc = copy_in(f.msd_cc, c_host.data(), sizeof(cplx) * ND, st);
        if (rc) return bail(rc);
    }
    {
        unsigned fl[3] = {0, 0, 0};
        AFQMC_CUDA_TRY(cudaMemcpyAsync(fl, wk->flags, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        if (dspin) AFQMC_CUDA_TRY(cudaMemcpyAsync(fl + 2, dspin, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
        if (dspin) cudaFree(dspin);
        if (fl[0] & FLAG_NONFINITE) return bail(fail(AFQMC_ERR_NONFINITE, "init_walkers: NaN/Inf in the trial"));
        wk->trial_real = fl[1] == 0;
        wk->Lt_real = wk->trial_real && !ham->cplx_L;
        wk->spin_same = dspin != nullptr && fl[2] == 0;
    }
    if (o.precision == AFQMC_PREC_BF16X3 && ham->cplx_L)
        return bail(fail(AFQMC_ERR_UNSUPPORTED, "init_walkers: BF16X3 needs real Cholesky vectors"));
    if (ham->Nmu > 0 && (o.precision == AFQMC_PREC_BF16X3 || ND > 1))
        return bail(fail(AFQMC_ERR_UNSUPPORTED, "init_walkers: a THC Hamiltonian runs on the FP64 path with one determinant"));
    if (o.precision == AFQMC_PREC_BF16X3 && ND > 1)
        return bail(fail(AFQMC_ERR_UNSUPPORTED, "init_walkers: BF16X3 needs a single-determinant trial"));
    if (o.precision == AFQMC_PREC_BF16X3) {
        if (!wk->trial_real || Nup != Ndn || !wk->spin_same || M % 64 != 0 || nch % 8 != 0)
            return bail(fail(AFQMC_ERR_UNSUPPORTED,
                             "init_walkers: BF16X3 needs a real trial with Psi_up == Psi_dn, M % 64 == 0, "
                             "Nchol % 8 == 0"));
    }
    // rotated Cholesky tensor (THC: the half-rotated orbital values Psi^+ X), its transpose,
    // rotated one-body matrix, per determinant
    for (int s = 0; s < 2 && ham->Nmu > 0; ++s) {
        GemmArgs g;   // Yt = Psi^+ X   [N][Nmu]
        g.m = wk->N[s]; g.n = ham->Nmu; g.k = M;
        g.A.ptr = f.Psi[s]; g.A.op = OP_C; g.A.ld = wk->N[s];
        g.B.ptr = ham->X; g.B.real = true; g.B.ld = ham->Nmu;
        g.C = f.Yt[s]; g.ldc = ham->Nmu;
        zgemm(g, st);
        GemmArgs gh;  // ht = Psi^+ h   [N][M]
        gh.m = wk->N[s]; gh.n = M; gh.k = M;
        gh.A.ptr = f.Psi[s]; gh.A.op = OP_C; gh.A.ld = wk->N[s];
        gh.B.ptr = ham->h; gh.B.real = true; gh.B.ld = M;
        gh.C = f.ht[s]; gh.ldc = M;
        zgemm(gh, st);
    }
    for (int s = 0; s < 2 && ham->Nmu == 0; ++s) {
        const int N = wk->N[s];
        const int64_t mn = (int64_t)M * N, tot = (int64_t)nch * N * M;
        cplx* tmp = nullptr;
        if (cudaMallocAsync(&tmp, sizeof(cplx) * (size_t)tot, st) != cudaSuccess)
            return bail(fail(AFQMC_ERR_OOM, "init_walkers: workspace"));
        for (int I = 0; I < ND; ++I) {
            const cplx* Psi = f.Psi[s] + I * mn;
            GemmArgs g;   // tmp[n] = Psi^+ L_n   [N][M]
            g.m = N; g.n = M; g.k = M; g.nb1 = nch;
            g.A.ptr = Psi; g.A.op = OP_C; g.A.ld = N;
            g.B.ptr = ham->L; g.B.real = !ham->cplx_L; g.B.ld = M; g.B.s1 = (int64_t)M * M;
            g.C = tmp; g.ldc = M; g.sc1 = (int64_t)N * M;
            zgemm(g, st);
            if (wk->Lt_real) {
                double* Lr = static_cast<double*>(f.Lt[s]) + I * tot;
                count_launch();
                cplx_real_part_kernel<<<nblk(tot), 256, 0, st>>>(tmp, Lr, tot);
                count_launch();
                batched_transpose_kernel<double><<<nblk(tot), 256, 0, st>>>(
                    Lr, static_cast<double*>(f.LtT[s]) + I * tot, nch, N, M);
            } else {
                cudaMemcpyAsync(static_cast<cplx*>(f.Lt[s]) + I * tot, tmp, sizeof(cplx) * tot,
                                cudaMemcpyDeviceToDevice, st);
                count_launch();
                batched_transpose_kernel<cplx><<<nblk(tot), 256, 0, st>>>(
                    tmp, static_cast<cplx*>(f.LtT[s]) + I * tot, nch, N, M);
            }
            GemmArgs gh;  // ht = Psi^+ h   [N][M]
            gh.m = N; gh.n = M; gh.k = M;
            gh.A.ptr = Psi; gh.A.op = OP_C; gh.A.ld = N;
            gh.B.ptr = ham->h; gh.B.real = true; gh.B.ld = M;
            gh.C = f.ht[s] + I * mn; gh.ldc = M;
            zgemm(gh, st);
        }
        cudaFreeAsync(tmp, st);
    }
    rc = ham->cplx_L ? expm_complex(reinterpret_cast<const cplx*>(ham->hp), -0.5 * tau, M,
                                    reinterpret_cast<cplx*>(f.Bh), st)
                     : expm_real(ham->hp, -0.5 * tau, M, f.Bh, st);
    if (rc) return bail(rc);
    // trial energy E_T: the trial's energy shift (its variational energy unless two determinants
    // of an expansion are exactly orthogonal; those pairs are left out).  One determinant: its local energy with
    // walker 0 placed at it.  ND determinants: with walker 0 at each D_J in turn, the local
    // energies E_IJ and log-overlaps log S_IJ of every D_I, then
    // sum_IJ conj(c_I) c_J S_IJ E_IJ / sum_IJ conj(c_I) c_J S_IJ.
    fill_cplx(wk->weight, W, cplx{1.0, 0.0}, st);
    cplx et;
    if (ND == 1) {
        for (int s = 0; s < 2; ++s)
            cudaMemcpyAsync(f.Phi[s], f.Psi[s], sizeof(cplx) * M * wk->N[s], cudaMemcpyDeviceToDevice, st);
        rc = fp64_measure(wk, true, st, 1);
        if (rc) return bail(rc);
        AFQMC_CUDA_TRY(cudaMemcpyAsync(&et, wk->E_L, sizeof(cplx), cudaMemcpyDeviceToHost, st));
    } else {
        cplx *EIJ = nullptr, *LIJ = nullptr, *d_et = nullptr;
        if (cudaMallocAsync(&EIJ, sizeof(cplx) * ND * ND, st) != cudaSuccess ||
            cudaMallocAsync(&LIJ, sizeof(cplx) * ND * ND, st) != cudaSuccess ||
            cudaMallocAsync(&d_et, sizeof(cplx), st) != cudaSuccess)
            return bail(fail(AFQMC_ERR_OOM, "init_walkers: workspace"));
        for (int J = 0; J < ND; ++J) {
            for (int s = 0; s < 2; ++s)
                cudaMemcpyAsync(f.Phi[s], f.Psi[s] + (int64_t)J * M * wk->N[s], sizeof(cplx) * M * wk->N[s],
                                cudaMemcpyDeviceToDevice, st);
            rc = fp64_measure(wk, true, st, 1);
            if (rc) return bail(rc);
            // column J of [ND][ND] from the first entries of the [ND][W] per-determinant arrays
            AFQMC_CUDA_TRY(cudaMemcpy2DAsync(EIJ + J, sizeof(cplx) * ND, f.msd_E, sizeof(cplx) * W, sizeof(cplx), ND,
                                             cudaMemcpyDeviceToDevice, st));
            AFQMC_CUDA_TRY(cudaMemcpy2DAsync(LIJ + J, sizeof(cplx) * ND, f.msd_ls, sizeof(cplx) * W, sizeof(cplx), ND,
                                             cudaMemcpyDeviceToDevice, st));
        }
        msd_variational_energy(f.msd_cc, EIJ, LIJ, ND, d_et, st);
        AFQMC_CUDA_TRY(cudaMemcpyAsync(&et, d_et, sizeof(cplx), cudaMemcpyDeviceToHost, st));
        cudaFreeAsync(EIJ, st);
        cudaFreeAsync(LIJ, st);
        cudaFreeAsync(d_et, st);
    }
    AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
    wk->E_T = et.re;
    // walkers
    if (Phi0) {
        const size_t per = (size_t)M * (Nup + Ndn) * sizeof(cplx);
        for (int s = 0; s < 2; ++s) {
            const size_t off = (s == 0 ? 0 : (size_t)M * Nup * sizeof(cplx));
            cudaError_t e = cudaMemcpy2DAsync(f.Phi[s], (size_t)M * wk->N[s] * sizeof(cplx),
                                              reinterpret_cast<const char*>(Phi0) + off, per,
                                              (size_t)M * wk->N[s] * sizeof(cplx), W, cudaMemcpyDefault, st);
            if (e != cudaSuccess) return bail(fail(AFQMC_ERR_CUDA, std::string("init_walkers: ") + cudaGetErrorString(e)));
            check_finite(reinterpret_cast<const double*>(f.Phi[s]), 2LL * W * M * wk->N[s], wk->flags, st);
        }
    } else {
        for (int s = 0; s < 2; ++s)
            replicate(f.Phi[s], f.Psi[s] + (int64_t)ref * M * wk->N[s], (int64_t)M * wk->N[s], W,
                      (int64_t)M * wk->N[s], st);
    }
    cudaMemsetAsync(wk->flags, 0, sizeof(unsigned), st);
    if (o.precision == AFQMC_PREC_BF16X3) {
        rc = tc_alloc(wk, st);
        if (rc) return bail(rc);
    }
    // check the walkers' overlaps with the trial once (several determinants: the combined one)
    if (ND == 1) {
        for (int s = 0; s < 2; ++s) {
            const int N = wk->N[s];
            GemmArgs g;
            g.m = N; g.n = N; g.k = M; g.nb1 = W;
            g.A.ptr = f.Psi[s]; g.A.op = OP_C; g.A.ld = N;
            g.B.ptr = f.Phi[s]; g.B.ld = N; g.B.s1 = (int64_t)M * N;
            g.C = f.S[s]; g.ldc = N; g.sc1 = (int64_t)N * N;
            zgemm(g, st);
            batched_inverse_logdet(f.S[s], (int64_t)N * N, N, W, f.ld[s], false, wk->flags, st);
        }
    } else {
        rc = fp64_measure(wk, false, st);
        if (rc) return bail(rc);
    }
    unsigned fl = 0;
    rc = read_flags(wk->flags, st, &fl);
    if (rc) return bail(rc);
    rc = flags_to_error(fl, "init_walkers");
    if (rc) return bail(rc);
    if (!isfinite(wk->E_T)) return bail(fail(AFQMC_ERR_NONFINITE, "init_walkers: trial energy not finite"));
    ham->live_walker_sets++;
    *out = wk;
    return AFQMC_OK;
}

extern "C" {

int afqmc_init_walkers(afqmc_ham_t ham, const double* Psi_up, const double* Psi_dn, int Nup, int Ndn, int W,
                       const double* Phi0, double tau, const afqmc_opts* opts, void* stream, afqmc_wk_t* out) {
    return init_walkers_impl(ham, 1, Psi_up, Psi_dn, nullptr, Nup, Ndn, W, Phi0, tau, opts, stream, out);
}

int afqmc_init_walkers_msd(afqmc_ham_t ham, int ND, const double* D_up, const double* D_dn, const double* c,
                           int Nup, int Ndn, int W, const double* Phi0, double tau, const afqmc_opts* opts,
                           void* stream, afqmc_wk_t* out) {
    if (!c) {
        if (out) *out = nullptr;
        return fail(AFQMC_ERR_BADARG, "init_walkers_msd: NULL coefficients");
    }
    return init_walkers_impl(ham, ND, D_up, D_dn, c, Nup, Ndn, W, Phi0, tau, opts, stream, out);
}

int afqmc_destroy_walkers(afqmc_wk_t wk) {
    if (!wk) return fail(AFQMC_ERR_BADARG, "destroy_walkers: NULL handle");
    wk->ham->live_walker_sets--;
    cudaDeviceSynchronize();
    free_walkers(wk);
    return AFQMC_OK;
}

static int ensure_x(afqmc_walkers* wk, int steps) {
    if (steps <= wk->x_cap) return AFQMC_OK;
    cudaFree(wk->x);
    wk->x = nullptr;
    if (cudaMalloc(&wk->x, sizeof(double) * (size_t)steps * wk->W * wk->Nchol) != cudaSuccess) {
        cudaGetLastError();
        wk->x_cap = 0;
        return fail(AFQMC_ERR_OOM, "step: field buffer");
    }
    wk->x_cap = steps;
    return AFQMC_OK;
}

static int ensure_emix(afqmc_walkers* wk, int n) {
    if (n <= wk->emix_cap) return AFQMC_OK;
    cudaFree(wk->emix);
    cudaFree(wk->esum);
    wk->emix = nullptr;
    wk->esum = nullptr;
    if (cudaMalloc(&wk->emix, sizeof(cplx) * n) != cudaSuccess || cudaMalloc(&wk->esum, sizeof(cplx) * 2 * n) != cudaSuccess) {
        cudaGetLastError();
        wk->emix_cap = 0;
        return fail(AFQMC_ERR_OOM, "step: trace buffer");
    }
    wk->emix_cap = n;
    return AFQMC_OK;
}

int afqmc_step(afqmc_wk_t wk, int nsteps, const double* x, uint64_t seed, int measure_every, double* E_mix_trace,
               void* stream) {
    if (!wk) return fail(AFQMC_ERR_BADARG, "step: NULL handle");
    if (nsteps < 0 || measure_every < 0) return fail(AFQMC_ERR_BADARG, "step: negative nsteps or measure_every");
    if (nsteps == 0) return AFQMC_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t per_step = (int64_t)wk->W * wk->Nchol;
    const bool x_dev = x && is_device_ptr(x);
    // caller fields: device pointers are used in place, host fields are staged per step
    if (x && !x_dev) AFQMC_TRY(ensure_x(wk, 1));
    if (!x) AFQMC_TRY(ensure_x(wk, 1));
    const int nmeas = measure_every > 0 ? (nsteps + measure_every - 1) / measure_every : 0;
    AFQMC_TRY(ensure_emix(wk, std::max(nmeas, 1)));
    wk->nmeas_last = 0;
    const bool tc = wk->opts.precision == AFQMC_PREC_BF16X3;
    wk->ev_valid = false;
    const long long launches0 = launch_count();
    // local-energy weights need E_L of every pre-step walker
    const bool local = wk->opts.weight_mode == AFQMC_WEIGHT_LOCAL;
    for (int s = 0; s < nsteps; ++s) {
        const bool meas = measure_every > 0 && s % measure_every == 0;
        AFQMC_TRY(tc ? tc_measure(wk, meas || local, st) : fp64_measure(wk, meas || local, st));
        if (meas)
            mixed_energy(wk->weight, wk->E_L, wk->W, wk->emix + s / measure_every, st,
                         wk->esum + 2 * (s / measure_every));
        const double* xs;
        if (x_dev) {
            xs = x + (int64_t)s * per_step;
        } else if (x) {
            AFQMC_TRY(copy_in(wk->x, x + (int64_t)s * per_step, sizeof(double) * per_step, st));
            xs = wk->x;
        } else {
            philox_fields(seed, wk->step, wk->W, wk->Nchol, wk->x, st, wk->opts.walker_offset);
            xs = wk->x;
        }
        AFQMC_TRY(tc ? tc_propagate_and_weight(wk, xs, st) : fp64_propagate_and_weight(wk, xs, st));
        bp_record(wk, st);
        wk->step++;
        if (wk->opts.k_qr > 0 && wk->step % wk->opts.k_qr == 0) AFQMC_TRY(tc ? tc_qr(wk, st) : fp64_qr(wk, st));
    }
    wk->kernels_per_step = (int)((launch_count() - launches0) / nsteps);
    wk->nmeas_last = nmeas;
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return fail(AFQMC_ERR_CUDA, std::string("step: launch failed: ") + cudaGetErrorString(le));
    bool sync = false;
    if (E_mix_trace && nmeas > 0) AFQMC_TRY(copy_out(E_mix_trace, wk->emix, sizeof(cplx) * nmeas, st, &sync));
    unsigned fl = 0;
    AFQMC_TRY(read_flags(wk->flags, st, &fl));
    return flags_to_error(fl, "step");
}

int afqmc_population_control(afqmc_wk_t wk, double xi, int* idx, void* stream) {
    if (!wk) return fail(AFQMC_ERR_BADARG, "population_control: NULL handle");
    if (!(xi >= 0.0 && xi < 1.0)) return fail(AFQMC_ERR_BADARG, "population_control: xi must lie in [0, 1)");
    if (wk->opts.weight_mode == AFQMC_WEIGHT_FREE)
        return fail(AFQMC_ERR_BADARG, "population_control: needs real (phaseless or local-energy) weights");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool tc = wk->opts.precision == AFQMC_PREC_BF16X3;
    const int W = wk->W, M = wk->M;
    struct Scratch {
        void* p[4] = {nullptr, nullptr, nullptr, nullptr};
        ~Scratch() {
            for (void* q : p)
                if (q) cudaFree(q);
        }
    } sc;
    if (cudaMalloc(&sc.p[0], sizeof(int) * W) != cudaSuccess || cudaMalloc(&sc.p[1], sizeof(double)) != cudaSuccess ||
        cudaMalloc(&sc.p[2], sizeof(cplx) * (size_t)W * std::max<size_t>((size_t)M * std::max(wk->N[0], wk->N[1]),
                                                                          (size_t)wk->Nchol)) != cudaSuccess ||
        cudaMalloc(&sc.p[3], sizeof(cplx) * W) != cudaSuccess) {
        cudaGetLastError();
        return fail(AFQMC_ERR_OOM, "population_control: scratch");
    }
    int* d_idx = static_cast<int*>(sc.p[0]);
    double* d_total = static_cast<double*>(sc.p[1]);
    cplx* tmp = static_cast<cplx*>(sc.p[2]);
    comb_indices(wk->weight, W, xi, d_idx, d_total, st);
    double total = 0.0;
    AFQMC_CUDA_TRY(cudaMemcpyAsync(&total, d_total, sizeof(double), cudaMemcpyDeviceToHost, st));
    AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(total > 0.0) || !isfinite(total)) return fail(AFQMC_ERR_BADARG, "population_control: no live walker");
    if (tc) AFQMC_TRY(tc_sync_walkers_to_fp64(wk, st));
    for (int s = 0; s < 2; ++s) {
        const int64_t per = (int64_t)M * wk->N[s];
        gather_rows(wk->f.Phi[s], per, d_idx, W, tmp, st);
        AFQMC_CUDA_TRY(cudaMemcpyAsync(wk->f.Phi[s], tmp, sizeof(cplx) * per * W, cudaMemcpyDeviceToDevice, st));
    }
    cplx* ltmp = static_cast<cplx*>(sc.p[3]);
    gather_rows(wk->logS_old, 1, d_idx, W, ltmp, st);
    AFQMC_CUDA_TRY(cudaMemcpyAsync(wk->logS_old, ltmp, sizeof(cplx) * W, cudaMemcpyDeviceToDevice, st));
    equal_weights(wk->weight, W, d_total, st);
    AFQMC_TRY(bp_follow_comb(wk, d_idx, tmp, st));
    if (tc) AFQMC_TRY(tc_sync_walkers_from_fp64(wk, st));
    if (idx) AFQMC_CUDA_TRY(cudaMemcpyAsync(idx, d_idx, sizeof(int) * W, cudaMemcpyDefault, st));
    AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
    unsigned fl = 0;
    AFQMC_TRY(read_flags(wk->flags, st, &fl));
    return flags_to_error(fl, "population_control");
}

int afqmc_comb_indices(const double* w, int W, double xi, int* idx, double* total, void* stream) {
    if (!w || !idx) return fail(AFQMC_ERR_BADARG, "comb_indices: NULL pointer");
    if (W < 1) return fail(AFQMC_ERR_SHAPE, "comb_indices: need W >= 1");
    if (!(xi >= 0.0 && xi < 1.0)) return fail(AFQMC_ERR_BADARG, "comb_indices: xi must lie in [0, 1)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    struct Scratch {
        void* p[4] = {nullptr, nullptr, nullptr, nullptr};
        ~Scratch() {
            for (void* q : p)
                if (q) cudaFree(q);
        }
    } sc;
    if (cudaMalloc(&sc.p[0], sizeof(double) * W) != cudaSuccess || cudaMalloc(&sc.p[1], sizeof(cplx) * W) != cudaSuccess ||
        cudaMalloc(&sc.p[2], sizeof(int) * W) != cudaSuccess || cudaMalloc(&sc.p[3], sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(AFQMC_ERR_OOM, "comb_indices: scratch");
    }
    double* dw = static_cast<double*>(sc.p[0]);
    cplx* wc = static_cast<cplx*>(sc.p[1]);
    int* d_idx = static_cast<int*>(sc.p[2]);
    double* d_total = static_cast<double*>(sc.p[3]);
    AFQMC_TRY(copy_in(dw, w, sizeof(double) * W, st));
    real_to_cplx(dw, wc, W, st);
    comb_indices(wc, W, xi, d_idx, d_total, st);
    double tot = 0.0;
    AFQMC_CUDA_TRY(cudaMemcpyAsync(&tot, d_total, sizeof(double), cudaMemcpyDeviceToHost, st));
    AFQMC_CUDA_TRY(cudaMemcpyAsync(idx, d_idx, sizeof(int) * W, cudaMemcpyDefault, st));
    AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(tot > 0.0) || !isfinite(tot)) return fail(AFQMC_ERR_BADARG, "comb_indices: weights must sum to a positive number");
    if (total) AFQMC_TRY(copy_in(total, &tot, sizeof(double), st));
    AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
    return AFQMC_OK;
}

int afqmc_energy(afqmc_wk_t wk, double* E_L, double* w, double* logS, double* E_mix, void* stream) {
    if (!wk) return fail(AFQMC_ERR_BADARG, "energy: NULL handle");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool tc = wk->opts.precision == AFQMC_PREC_BF16X3;
    if (tc) AFQMC_TRY(tc_sync_walkers_to_fp64(wk, st));
    AFQMC_TRY(tc ? tc_measure(wk, true, st) : fp64_measure(wk, true, st));
    mixed_energy(wk->weight, wk->E_L, wk->W, wk->emix, st, wk->esum);
    wk->nmeas_last = 1;
    bool sync = false;
    const int W = wk->W;
    AFQMC_TRY(copy_out(E_L, wk->E_L, sizeof(cplx) * W, st, &sync));
    AFQMC_TRY(copy_out(logS, wk->logS_old, sizeof(cplx) * W, st, &sync));
    AFQMC_TRY(copy_out(E_mix, wk->emix, sizeof(cplx), st, &sync));
    if (w) {
        if (wk->opts.weight_mode == AFQMC_WEIGHT_FREE) {
            AFQMC_TRY(copy_out(w, wk->weight, sizeof(cplx) * W, st, &sync));
        } else {
            // real parts: strided copy
            AFQMC_CUDA_TRY(cudaMemcpy2DAsync(w, sizeof(double), wk->weight, sizeof(cplx), sizeof(double), W,
                                             cudaMemcpyDefault, st));
        }
    }
    unsigned fl = 0;
    AFQMC_TRY(read_flags(wk->flags, st, &fl));
    return flags_to_error(fl, "energy");
}

int afqmc_mixed_sums(afqmc_wk_t wk, int nmeas, double* sums, void* stream) {
    if (!wk || !sums) return fail(AFQMC_ERR_BADARG, "mixed_sums: NULL handle or pointer");
    if (nmeas != wk->nmeas_last || nmeas < 1)
        return fail(AFQMC_ERR_BADARG, "mixed_sums: nmeas must equal the measurements of the last step/energy call (" +
                                          std::to_string(wk->nmeas_last) + ")");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bool sync = false;
    AFQMC_TRY(copy_out(sums, wk->esum, sizeof(cplx) * 2 * (size_t)nmeas, st, &sync));
    if (sync) AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
    return AFQMC_OK;
}

int afqmc_get_walkers(afqmc_wk_t wk, double* Phi, double* w, int64_t* step, void* stream) {
    if (!wk) return fail(AFQMC_ERR_BADARG, "get_walkers: NULL handle");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (wk->opts.precision == AFQMC_PREC_BF16X3) AFQMC_TRY(tc_sync_walkers_to_fp64(wk, st));
    const int M = wk->M, W = wk->W;
    const size_t per = (size_t)M * (wk->N[0] + wk->N[1]) * sizeof(cplx);
    if (Phi) {
        for (int s = 0; s < 2; ++s) {
            const size_t off = s == 0 ? 0 : (size_t)M * wk->N[0] * sizeof(cplx);
            AFQMC_CUDA_TRY(cudaMemcpy2DAsync(reinterpret_cast<char*>(Phi) + off, per, wk->f.Phi[s],
                                             (size_t)M * wk->N[s] * sizeof(cplx), (size_t)M * wk->N[s] * sizeof(cplx),
                                             W, cudaMemcpyDefault, st));
        }
    }
    if (w) {
        if (wk->opts.weight_mode == AFQMC_WEIGHT_FREE)
            AFQMC_CUDA_TRY(cudaMemcpyAsync(w, wk->weight, sizeof(cplx) * W, cudaMemcpyDefault, st));
        else
            AFQMC_CUDA_TRY(cudaMemcpy2DAsync(w, sizeof(double), wk->weight, sizeof(cplx), sizeof(double), W,
                                             cudaMemcpyDefault, st));
    }
    if (step) *step = wk->step;
    AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
    return AFQMC_OK;
}

int afqmc_set_walkers(afqmc_wk_t wk, const double* Phi, const double* w, int64_t step, void* stream) {
    if (!wk) return fail(AFQMC_ERR_BADARG, "set_walkers: NULL handle");
    if (step < 0) return fail(AFQMC_ERR_BADARG, "set_walkers: negative step");
    bp_close(wk);   // the window's walkers and history no longer describe these walkers
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int M = wk->M, W = wk->W;
    const size_t per = (size_t)M * (wk->N[0] + wk->N[1]) * sizeof(cplx);
    if (Phi) {
        for (int s = 0; s < 2; ++s) {
            const size_t off = s == 0 ? 0 : (size_t)M * wk->N[0] * sizeof(cplx);
            AFQMC_CUDA_TRY(cudaMemcpy2DAsync(wk->f.Phi[s], (size_t)M * wk->N[s] * sizeof(cplx),
                                             reinterpret_cast<const char*>(Phi) + off, per,
                                             (size_t)M * wk->N[s] * sizeof(cplx), W, cudaMemcpyDefault, st));
        }
    }
    if (w) {
        if (wk->opts.weight_mode == AFQMC_WEIGHT_FREE) {
            AFQMC_CUDA_TRY(cudaMemcpyAsync(wk->weight, w, sizeof(cplx) * W, cudaMemcpyDefault, st));
        } else {
            fill_cplx(wk->weight, W, cplx{0.0, 0.0}, st);
            AFQMC_CUDA_TRY(cudaMemcpy2DAsync(wk->weight, sizeof(cplx), w, sizeof(double), sizeof(double), W,
                                             cudaMemcpyDefault, st));
        }
    }
    wk->step = step;
    if (wk->opts.precision == AFQMC_PREC_BF16X3) AFQMC_TRY(tc_sync_walkers_from_fp64(wk, st));
    AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
    return AFQMC_OK;
}

int afqmc_philox_fields(uint64_t seed, int64_t step, int W, int Nchol, double* x, void* stream) {
    if (!x || W < 1 || Nchol < 1 || step < 0) return fail(AFQMC_ERR_BADARG, "philox_fields: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (is_device_ptr(x)) {
        philox_fields(seed, step, W, Nchol, x, st);
        AFQMC_CUDA_TRY(cudaGetLastError());
        return AFQMC_OK;
    }
    double* d = nullptr;
    AFQMC_CUDA_TRY(cudaMallocAsync(&d, sizeof(double) * (size_t)W * Nchol, st));
    philox_fields(seed, step, W, Nchol, d, st);
    AFQMC_CUDA_TRY(cudaMemcpyAsync(x, d, sizeof(double) * (size_t)W * Nchol, cudaMemcpyDeviceToHost, st));
    cudaFreeAsync(d, st);
    AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
    return AFQMC_OK;
}

int afqmc_energy_backward(afqmc_wk_t wk, const double* dE, const double* dlogS, double* dPsi_up, double* dPsi_dn,
                          double* dL, void* stream) {
    if (!wk) return fail(AFQMC_ERR_BADARG, "energy_backward: NULL handle");
    if (wk->ham->cplx_L) return fail(AFQMC_ERR_UNSUPPORTED, "energy_backward: needs real Cholesky vectors");
    if (wk->ham->Nmu > 0) return fail(AFQMC_ERR_UNSUPPORTED, "energy_backward: needs Cholesky vectors (not THC)");
    if (wk->ND > 1) return fail(AFQMC_ERR_UNSUPPORTED, "energy_backward: needs a single-determinant trial");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return fp64_backward(wk, reinterpret_cast<const cplx*>(dE), reinterpret_cast<const cplx*>(dlogS),
                         reinterpret_cast<cplx*>(dPsi_up), reinterpret_cast<cplx*>(dPsi_dn), dL, st);
}

int afqmc_last_step_stats(afqmc_wk_t wk, double* energy_kernel_ms, int* kernels_per_step) {
    if (!wk) return fail(AFQMC_ERR_BADARG, "last_step_stats: NULL handle");
    if (energy_kernel_ms) {
        *energy_kernel_ms = -1.0;
        if (wk->ev_valid) {
            float ms = 0.f;
            if (cudaEventSynchronize(wk->ev1) == cudaSuccess && cudaEventElapsedTime(&ms, wk->ev0, wk->ev1) == cudaSuccess)
                *energy_kernel_ms = ms;
            else
                cudaGetLastError();
        }
    }
    if (kernels_per_step) *kernels_per_step = wk->kernels_per_step;
    return AFQMC_OK;
}

}  // extern "C"
