// Shared device/host helpers of the AFQMC library (complex FP64 arithmetic,
// error plumbing, launch declarations).  Internal to the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/afqmc.h"

namespace afqmc {

// ---------------------------------------------------------------- complex FP64
struct cplx {
    double re, im;
};

__host__ __device__ __forceinline__ cplx mk(double r, double i) { return cplx{r, i}; }
__host__ __device__ __forceinline__ cplx operator+(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ cplx operator-(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cplx operator*(cplx a, cplx b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cplx operator*(double s, cplx a) { return {s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ cplx conjg(cplx a) { return {a.re, -a.im}; }
__host__ __device__ __forceinline__ double abs1(cplx a) { return fabs(a.re) + fabs(a.im); }
// a += b * c  (complex fused multiply-add on FP64 pipes)
__host__ __device__ __forceinline__ void cfma(cplx& a, cplx b, cplx c) {
    a.re = fma(b.re, c.re, fma(-b.im, c.im, a.re));
    a.im = fma(b.re, c.im, fma(b.im, c.re, a.im));
}
__host__ __device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    // Smith's algorithm for a / b
    if (fabs(b.re) >= fabs(b.im)) {
        double r = b.im / b.re, d = b.re + b.im * r;
        return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    } else {
        double r = b.re / b.im, d = b.im + b.re * r;
        return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
    }
}

// ---------------------------------------------------------------- error state
struct Status {
    int code = AFQMC_OK;
    std::string msg;
};
void set_error(int code, const std::string& msg);
int fail(int code, const std::string& msg);  // sets and returns code

// Number of kernels this library has launched (diagnostics: kernels per step).
void count_launch();
long long launch_count();

// Launch-shape knobs of the persistent tensor-core kernels, read when a kernel is launched
// (or captured into a graph) on the calling thread.  Defaults: one CTA per SM, the widest
// tile a call site allows.  The batch autotuner sets them around each candidate capture.
struct LaunchPolicy {
    int grid_cap = 0;    // > 0: at most this many CTAs per persistent launch
    int bn_max = 256;    // 128: narrow every plain GEMM tile to 128 columns
    int energy_bk = 0;   // K chunk of the fused energy kernel: 16 or 32 (default)
    int energy_ws_super = 0;   // walker-spin groups per L2 window of the energy kernel (0: default)
    int gj_variant = 0;        // batched inverse: 0 auto, 1 shared-memory kernel, 2 register kernel
    int energy_pair = 1;       // fused energy kernel: 1 CTA pairs (cta_group::2, default), 0 one CTA per tile
    int batch_n_granule = 8;   // batches pad N to a multiple of 8 (default), or 32: N' in {32, 64, 128}
};
LaunchPolicy& launch_policy();

// true while `st` is being captured into a CUDA graph (timing events are then skipped)
bool stream_capturing(cudaStream_t st);

// Raises `func`'s dynamic shared-memory limit on the current device to at least `bytes`, never
// lowering it: launches of one kernel with different sizes can sit in one captured graph (a
// batch of uneven systems), and every node needs the limit to cover its own size whenever it
// is launched.
cudaError_t raise_dyn_smem(const void* func, size_t bytes);
template <typename F>
cudaError_t raise_dyn_smem(F* func, size_t bytes) {
    return raise_dyn_smem(reinterpret_cast<const void*>(func), bytes);
}

#define AFQMC_CUDA_TRY(expr)                                                                   \
    do {                                                                                        \
        cudaError_t _e = (expr);                                                                \
        if (_e != cudaSuccess)                                                                  \
            return ::afqmc::fail(AFQMC_ERR_CUDA, std::string(#expr " failed: ") +              \
                                                     cudaGetErrorString(_e));                   \
    } while (0)

#define AFQMC_TRY(expr)                \
    do {                               \
        int _rc = (expr);              \
        if (_rc != AFQMC_OK) return _rc; \
    } while (0)

// ---------------------------------------------------------------- device flags
// Bits of the per-walker-set device status word (latched, read by the host).
enum : unsigned {
    FLAG_NONFINITE = 1u,
    FLAG_SINGULAR = 2u,
    FLAG_TIMEOUT = 4u,
};

}  // namespace afqmc
