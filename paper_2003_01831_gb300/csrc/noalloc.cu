// Allocation-free log-overlap entry point (afqmc_log_overlap_noalloc, include/afqmc.h).
//
// Some callers cannot allocate device memory at the point where they need this quantity:
// a service that reserved the whole device for its own memory pool (any cudaMalloc there
// may fail at run time), or a latency-critical loop that must not hit the allocator, which
// can synchronise the device.  This file therefore keeps its scratch in one file-scope
// device array of fixed size that every GPU loading the library holds until the process
// exits, and the entry point takes only caller-owned inputs and outputs.
//
// The scratch holds the overlap matrices S_s = Psi_s^+ Phi_s of every walker and spin, the
// per-spin log-determinants and a status word.  Every call reuses the same array and leaves
// its contents behind; calls whose device work overlaps (two streams, or two host threads on
// the same device) race on it and must be serialised by the caller.
#include <cuda.h>

#include <mutex>
#include <string>

#include "kernels_fp64.cuh"

namespace afqmc {

bool is_device_ptr(const void* p);

namespace {

// Bytes of scratch per device (the stated maximum of the entry point).
constexpr size_t kScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};   // context the address belongs to

// Unique id of the calling thread's current context (cuCtxGetId through the runtime's driver
// entry point), or 0 when it cannot be read.  A device's primary context that was reset
// (cudaDeviceReset, or another library in the process) comes back with a new id, and the
// scratch array then lives at a new address.
unsigned long long current_context_id() {
    typedef CUresult (*GetCtxFn)(CUcontext*);
    typedef CUresult (*GetIdFn)(CUcontext, unsigned long long*);
    static GetCtxFn get_ctx = nullptr;
    static GetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_ctx = reinterpret_cast<GetCtxFn>(p);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetIdFn>(p);
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_ctx || !get_id || get_ctx(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// logS[w] = ld0[w] + ld1[w] with the phase wrapped to (-pi, pi]
__global__ void noalloc_sum_kernel(const cplx* ld0, const cplx* ld1, int W, cplx* out) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const cplx s = ld0[w] + ld1[w];
    out[w] = cplx{s.re, atan2(sin(s.im), cos(s.im))};
}

// Device address of this device's scratch, looked up once per device (with that device
// current, which is the caller's current device), and again if the device's context has
// changed since (a reset context places the array elsewhere).
int scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(AFQMC_ERR_CUDA, std::string("log_overlap_noalloc: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(AFQMC_ERR_UNSUPPORTED, "log_overlap_noalloc: device index too large");
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev] || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(AFQMC_ERR_CUDA, std::string("log_overlap_noalloc: cudaGetSymbolAddress failed: ") +
                                            cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return AFQMC_OK;
}

}  // namespace
}  // namespace afqmc

using namespace afqmc;

extern "C" int afqmc_log_overlap_noalloc(const double* Psi_up, const double* Psi_dn, int Nup, int Ndn, int M, int W,
                                         const double* Phi, double* logS, void* stream) {
    if (!Psi_up || !Psi_dn || !Phi || !logS) return fail(AFQMC_ERR_BADARG, "log_overlap_noalloc: NULL pointer");
    if (M < 1 || Nup < 1 || Ndn < 1 || Nup > M || Ndn > M || W < 1)
        return fail(AFQMC_ERR_SHAPE, "log_overlap_noalloc: need 1 <= Nup, Ndn <= M and W >= 1");
    if (!is_device_ptr(Psi_up) || !is_device_ptr(Psi_dn) || !is_device_ptr(Phi) || !is_device_ptr(logS))
        return fail(AFQMC_ERR_BADARG, "log_overlap_noalloc: all pointers must be device memory");
    // scratch layout: [status word, 256 B] [S_up W*Nup*Nup] [S_dn W*Ndn*Ndn] [ld_up W] [ld_dn W]
    const size_t need = 256 + sizeof(cplx) * ((size_t)W * Nup * Nup + (size_t)W * Ndn * Ndn + 2 * (size_t)W);
    if (need > kScratchBytes)
        return fail(AFQMC_ERR_SHAPE, "log_overlap_noalloc: W*(Nup^2 + Ndn^2 + 2)*16 + 256 bytes exceeds the " +
                                         std::to_string(kScratchBytes >> 20) + " MiB scratch; use afqmc_energy");
    unsigned char* base = nullptr;
    AFQMC_TRY(scratch_for_current_device(&base));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned* flags = reinterpret_cast<unsigned*>(base);
    cplx* S[2];
    S[0] = reinterpret_cast<cplx*>(base + 256);
    S[1] = S[0] + (size_t)W * Nup * Nup;
    cplx* ld[2];
    ld[0] = S[1] + (size_t)W * Ndn * Ndn;
    ld[1] = ld[0] + W;
    AFQMC_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(unsigned), st));   // the status must start clear
    const int N[2] = {Nup, Ndn};
    const cplx* Psi[2] = {reinterpret_cast<const cplx*>(Psi_up), reinterpret_cast<const cplx*>(Psi_dn)};
    const int64_t per = (int64_t)M * (Nup + Ndn);
    for (int s = 0; s < 2; ++s) {
        GemmArgs g;   // S_s[w] = Psi_s^+ Phi_s[w]; walker w's spin-s block starts at w*per (+ M*Nup for down)
        g.m = N[s]; g.n = N[s]; g.k = M; g.nb1 = W;
        g.A.ptr = Psi[s]; g.A.op = OP_C; g.A.ld = N[s];
        g.B.ptr = reinterpret_cast<const cplx*>(Phi) + (s == 0 ? 0 : (int64_t)M * Nup);
        g.B.ld = N[s]; g.B.s1 = per;
        g.C = S[s]; g.ldc = N[s]; g.sc1 = (int64_t)N[s] * N[s];
        zgemm(g, st);
        batched_inverse_logdet(S[s], (int64_t)N[s] * N[s], N[s], W, ld[s], false, flags, st);
    }
    count_launch();
    noalloc_sum_kernel<<<(W + 255) / 256, 256, 0, st>>>(ld[0], ld[1], W, reinterpret_cast<cplx*>(logS));
    AFQMC_CUDA_TRY(cudaGetLastError());
    unsigned h = 0;
    AFQMC_CUDA_TRY(cudaMemcpyAsync(&h, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
    if (h & FLAG_NONFINITE) return fail(AFQMC_ERR_NONFINITE, "log_overlap_noalloc: NaN/Inf in the walkers or trial");
    if (h & FLAG_SINGULAR) return fail(AFQMC_ERR_SINGULAR, "log_overlap_noalloc: singular overlap matrix");
    return AFQMC_OK;
}
