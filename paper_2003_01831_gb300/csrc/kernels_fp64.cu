// FP64 (DFMA) kernels of the AFQMC walker step: batched complex GEMM, Gauss-Jordan
// inverse / log-det, trace epilogue, local energy and force bias, Philox fields,
// phaseless weights, Gram-Schmidt re-orthonormalisation, estimator reduction.
//
// The formulas follow the phaseless algorithm the paper cites in Sec. V (Zhang &
// Krakauer 2003; Motta & Zhang 2018) for the Hamiltonian of Sec. V, Eq. (1) with
// the Cholesky factorisation of Eq. (3).  All reductions run in a fixed order for
// a fixed launch shape, so results are bitwise reproducible run to run.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "ffc.cuh"
#include "kernels_fp64.cuh"

namespace afqmc {

namespace {

constexpr int kThreads = 256;

// Fixed-order block reduction of a complex value (all threads get the result).
__device__ cplx block_sum(cplx v, cplx* sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) sh[t] = sh[t] + sh[t + s];
        __syncthreads();
    }
    cplx r = sh[0];
    __syncthreads();
    return r;
}

__device__ double block_sum_d(double v, double* sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) sh[t] += sh[t + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ bool finite_c(cplx a) { return isfinite(a.re) && isfinite(a.im); }

// ------------------------------------------------------------------ batched GEMM
template <bool R>
struct Elem {
    using T = cplx;
};
template <>
struct Elem<true> {
    using T = double;
};

__device__ __forceinline__ void load_elem(double& dst, const void* base, int64_t idx, bool conj) {
    dst = static_cast<const double*>(base)[idx];
}
__device__ __forceinline__ void load_elem(cplx& dst, const void* base, int64_t idx, bool conj) {
    const double2 v = static_cast<const double2*>(base)[idx];
    dst.re = v.x;
    dst.im = conj ? -v.y : v.y;
}
__device__ __forceinline__ void zero_elem(double& d) { d = 0.0; }
__device__ __forceinline__ void zero_elem(cplx& d) { d = cplx{0.0, 0.0}; }

__device__ __forceinline__ void mac(cplx& acc, double a, double b) { acc.re = fma(a, b, acc.re); }
__device__ __forceinline__ void mac(cplx& acc, double a, cplx b) {
    acc.re = fma(a, b.re, acc.re);
    acc.im = fma(a, b.im, acc.im);
}
__device__ __forceinline__ void mac(cplx& acc, cplx a, double b) {
    acc.re = fma(a.re, b, acc.re);
    acc.im = fma(a.im, b, acc.im);
}
__device__ __forceinline__ void mac(cplx& acc, cplx a, cplx b) { cfma(acc, a, b); }

// Tiles of TS x TS outputs (TS = 64: 4 x 4 per thread; TS = 32: 2 x 2 per thread, for the small
// blocks of few-electron systems, e.g. the 32 x 32 T_n = Ltilde_n Theta blocks), K in steps of
// 512 / TS, so each operand tile holds 512 elements either way.
template <bool AR, bool BR, int TS>
__global__ void __launch_bounds__(kThreads) zgemm_kernel(GemmArgs g) {
    constexpr int BM = TS, BN = TS, BK = 512 / TS, R = TS / 16;
    using TA = typename Elem<AR>::T;
    using TB = typename Elem<BR>::T;
    __shared__ TA As[BK][BM + 1];
    __shared__ TB Bs[BK][BN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int64_t nbatch = (int64_t)g.nb0 * g.nb1 * g.nb2;
    for (int64_t b = blockIdx.z; b < nbatch; b += gridDim.z) {
        const int64_t b0 = b / ((int64_t)g.nb1 * g.nb2);
        const int64_t r12 = b % ((int64_t)g.nb1 * g.nb2);
        const int64_t b1 = r12 / g.nb2, b2 = r12 % g.nb2;
        const int64_t offA = b0 * g.A.s0 + b1 * g.A.s1 + b2 * g.A.s2;
        const int64_t offB = b0 * g.B.s0 + b1 * g.B.s1 + b2 * g.B.s2;
        cplx acc[R][R];
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
            for (int j = 0; j < R; ++j) acc[i][j] = cplx{0.0, 0.0};

        for (int k0 = 0; k0 < g.k; k0 += BK) {
            for (int e = threadIdx.x; e < BM * BK; e += kThreads) {
                int r, kk;
                if (g.A.op == OP_N) { r = e / BK; kk = e % BK; }
                else { kk = e / BM; r = e % BM; }
                const int gr = m0 + r, gk = k0 + kk;
                TA v;
                zero_elem(v);
                if (gr < g.m && gk < g.k) {
                    const int64_t idx = offA + (g.A.op == OP_N ? (int64_t)gr * g.A.ld + gk
                                                                : (int64_t)gk * g.A.ld + gr);
                    load_elem(v, g.A.ptr, idx, g.A.op == OP_C);
                }
                As[kk][r] = v;
            }
            for (int e = threadIdx.x; e < BN * BK; e += kThreads) {
                int c, kk;
                if (g.B.op == OP_N) { kk = e / BN; c = e % BN; }
                else { c = e / BK; kk = e % BK; }
                const int gc = n0 + c, gk = k0 + kk;
                TB v;
                zero_elem(v);
                if (gc < g.n && gk < g.k) {
                    const int64_t idx = offB + (g.B.op == OP_N ? (int64_t)gk * g.B.ld + gc
                                                                : (int64_t)gc * g.B.ld + gk);
                    load_elem(v, g.B.ptr, idx, g.B.op == OP_C);
                }
                Bs[kk][c] = v;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                TA a[R];
                TB bv[R];
#pragma unroll
                for (int i = 0; i < R; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < R; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < R; ++i)
#pragma unroll
                    for (int j = 0; j < R; ++j) mac(acc[i][j], a[i], bv[j]);
            }
            __syncthreads();
        }
        const bool use_beta = (g.beta.re != 0.0 || g.beta.im != 0.0);
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = m0 + ty + 16 * i;
            if (r >= g.m) continue;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const int c = n0 + tx + 16 * j;
                if (c >= g.n) continue;
                cplx v = g.alpha * acc[i][j];
                cplx* cp = g.C + b0 * g.sc0 + b1 * g.sc1 + b2 * g.sc2 + (int64_t)r * g.ldc + c;
                if (use_beta) v = v + g.beta * (*cp);
                *cp = v;
                if (g.D) {
                    cplx* dp = g.D + b0 * g.sd0 + b1 * g.sd1 + b2 * g.sd2 + (int64_t)r * g.ldd + c;
                    *dp = *dp + v;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ Gauss-Jordan
constexpr int kGJU = 8;   // element updates in flight per thread
__global__ void __launch_bounds__(kThreads)
    gj_kernel(cplx* Sbase, int64_t stride, int N, cplx* logdet, int with_inverse, unsigned* flags) {
    extern __shared__ unsigned char smem_raw[];
    cplx* prow = reinterpret_cast<cplx*>(smem_raw);  // N (scaled pivot row)
    cplx* pcol = prow + N;                           // N (pivot column)
    int* perm = reinterpret_cast<int*>(pcol + N);    // N
    __shared__ double red_v[kThreads];
    __shared__ int red_i[kThreads];
    __shared__ int s_piv;
    __shared__ int s_singular;
    cplx* A = Sbase + (int64_t)blockIdx.x * stride;
    const int t = threadIdx.x;
    double logabs = 0.0, phase = 0.0;  // meaningful in thread 0
    if (t == 0) s_singular = 0;
    __syncthreads();
    for (int k = 0; k < N; ++k) {
        // pivot: max |re|+|im| over rows k..N-1 of column k, lowest index on ties
        // (warp shuffles, then one pass over the per-warp winners)
        double best = -1.0;
        int bi = N;
        for (int i = k + t; i < N; i += kThreads) {
            const double v = abs1(A[(int64_t)i * N + k]);
            if (v > best || (v != v && best == best)) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            if (v2 > best || (v2 == best && i2 < bi) || (v2 != v2 && best == best)) { best = v2; bi = i2; }
        }
        if ((t & 31) == 0) {
            red_v[t >> 5] = best;
            red_i[t >> 5] = bi;
        }
        __syncthreads();
        if (t == 0) {
            double bv = red_v[0];
            int bidx = red_i[0];
            for (int q = 1; q < kThreads / 32; ++q) {
                const double v2 = red_v[q];
                const int i2 = red_i[q];
                if (v2 > bv || (v2 == bv && i2 < bidx) || (v2 != v2 && bv == bv)) { bv = v2; bidx = i2; }
            }
            s_piv = bidx;
            if (!(bv > 0.0)) s_singular = (bv != bv) ? 2 : 1;
            perm[k] = bidx;
        }
        __syncthreads();
        if (s_singular) break;
        const int p = s_piv;
        if (p != k) {
            for (int j = t; j < N; j += kThreads) {
                const cplx a = A[(int64_t)k * N + j];
                A[(int64_t)k * N + j] = A[(int64_t)p * N + j];
                A[(int64_t)p * N + j] = a;
            }
            __syncthreads();
        }
        const cplx piv = A[(int64_t)k * N + k];
        const cplx inv = cdiv(cplx{1.0, 0.0}, piv);
        if (t == 0) {
            logabs += log(hypot(piv.re, piv.im));
            phase += atan2(piv.im, piv.re) + (p != k ? M_PI : 0.0);
        }
        for (int j = t; j < N; j += kThreads) {
            prow[j] = A[(int64_t)k * N + j] * inv;
            pcol[j] = A[(int64_t)j * N + k];
        }
        __syncthreads();
        // Element updates, kGJU per thread in flight: all loads are issued before any
        // arithmetic, so a thread waits on the memory system once per batch, not per element.
        if (with_inverse) {
            const int64_t NN = (int64_t)N * N;
            for (int64_t e0 = t; e0 < NN; e0 += (int64_t)kThreads * kGJU) {
                cplx v[kGJU];
#pragma unroll
                for (int u = 0; u < kGJU; ++u) {
                    const int64_t e = e0 + (int64_t)u * kThreads;
                    if (e < NN) v[u] = A[e];
                }
#pragma unroll
                for (int u = 0; u < kGJU; ++u) {
                    const int64_t e = e0 + (int64_t)u * kThreads;
                    if (e >= NN) continue;
                    const int i = (int)(e / N), j = (int)(e % N);
                    if (i == k) v[u] = (j == k) ? inv : prow[j];
                    else if (j == k) v[u] = cplx{0.0, 0.0} - pcol[i] * inv;
                    else cfma(v[u], cplx{0.0, 0.0} - pcol[i], prow[j]);
                    A[e] = v[u];
                }
            }
        } else {
            const int nr = N - k - 1;
            const int64_t nn = (int64_t)nr * nr;
            for (int64_t e0 = t; e0 < nn; e0 += (int64_t)kThreads * kGJU) {
                cplx v[kGJU];
#pragma unroll
                for (int u = 0; u < kGJU; ++u) {
                    const int64_t e = e0 + (int64_t)u * kThreads;
                    if (e < nn) v[u] = A[(int64_t)(k + 1 + e / nr) * N + k + 1 + e % nr];
                }
#pragma unroll
                for (int u = 0; u < kGJU; ++u) {
                    const int64_t e = e0 + (int64_t)u * kThreads;
                    if (e >= nn) continue;
                    const int i = k + 1 + (int)(e / nr), j = k + 1 + (int)(e % nr);
                    cfma(v[u], cplx{0.0, 0.0} - pcol[i], prow[j]);
                    A[(int64_t)i * N + j] = v[u];
                }
            }
        }
        __syncthreads();
    }
    if (s_singular) {
        if (t == 0) {
            logdet[blockIdx.x] = cplx{-INFINITY, 0.0};
            atomicOr(flags, s_singular == 2 ? FLAG_NONFINITE : FLAG_SINGULAR);
        }
        return;
    }
    if (with_inverse) {
        for (int k = N - 1; k >= 0; --k) {
            const int p = perm[k];
            if (p != k) {
                for (int i = t; i < N; i += kThreads) {
                    const cplx a = A[(int64_t)i * N + k];
                    A[(int64_t)i * N + k] = A[(int64_t)i * N + p];
                    A[(int64_t)i * N + p] = a;
                }
            }
            __syncthreads();
        }
    }
    if (t == 0) logdet[blockIdx.x] = cplx{logabs, atan2(sin(phase), cos(phase))};
}

// ------------------------------------------------------- Gauss-Jordan in shared memory
// The same elimination (pivot max |re|+|im|, lowest index on ties; physical row swaps; the
// in-place inverse with its column permutation undone at the end) with the matrix held on
// chip: one CTA for N <= kGJSmemOne, else a cluster of two CTAs that own alternate columns
// (column j lives in CTA j % 2 at local column j / 2) and exchange the pivot column and the
// pivot index through distributed shared memory, two cluster barriers per elimination step.
// FP64 throughput, not memory latency, then bounds the elimination.
constexpr int kGJSmemOne = 96;      // largest N done by one CTA (N^2 complex in shared memory)
constexpr int kGJSmemMax = 128;     // largest N done by the two-CTA cluster
constexpr int kGJT = 512;           // threads per CTA
// local columns per lane: COLS = ceil(H / 32) <= 3 (template parameter)

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
    uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p)), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_peer_f64(uint32_t addr, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void st_peer_s32(uint32_t addr, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

template <int C>
__device__ __forceinline__ void gj_sync() {
    if (C == 1) __syncthreads();
    else cluster_sync_all();
}

template <int C, int COLS>
__global__ void __launch_bounds__(kGJT)
    gj_smem_kernel(cplx* Sbase, int64_t stride, int N, cplx* logdet, int with_inverse, unsigned* flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = (N + C - 1) / C;                   // local columns
    cplx* A = reinterpret_cast<cplx*>(smem_raw);     // [N][H]
    cplx* pcol = A + (size_t)N * H;                  // pivot column (before this step's swap)
    cplx* prow = pcol + N;                           // scaled pivot row, local columns
    int* perm = reinterpret_cast<int*>(prow + H);    // pivot row of every step
    int* pos = perm + N;                             // final column of each stored column
    __shared__ double red_v[kGJT / 32];
    __shared__ int red_i[kGJT / 32];
    __shared__ int s_piv;
    __shared__ int s_singular;
    constexpr int R = COLS <= 2 ? 4 : 2;               // rows per warp in flight
    const int rank = C == 1 ? 0 : (int)cluster_rank();
    const int64_t mat = C == 1 ? blockIdx.x : blockIdx.x / C;
    cplx* G = Sbase + mat * stride;
    const int t = threadIdx.x;
    const int NH = N * H;
    // load my columns: global column j = c*C + rank
    for (int e = t; e < NH; e += kGJT) {
        const int i = e / H, c = e % H, j = c * C + rank;
        A[e] = j < N ? G[(int64_t)i * N + j] : cplx{0.0, 0.0};
    }
    if (t == 0) s_singular = 0;
    double logabs = 0.0, phase = 0.0;   // thread 0 of rank 0
    gj_sync<C>();
    for (int k = 0; k < N; ++k) {
        const int owner = k % C, lk = k / C;
        if (rank == owner) {
            double best = -1.0;
            int bi = N;
            for (int i = k + t; i < N; i += kGJT) {
                const double v = abs1(A[i * H + lk]);
                if (v > best || (v != v && best == best)) { best = v; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
                const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
                if (v2 > best || (v2 == best && i2 < bi) || (v2 != v2 && best == best)) { best = v2; bi = i2; }
            }
            if ((t & 31) == 0) { red_v[t >> 5] = best; red_i[t >> 5] = bi; }
            // the pivot column (pre-swap) to both CTAs
            for (int i = t; i < N; i += kGJT) {
                const cplx v = A[i * H + lk];
                pcol[i] = v;
                if (C > 1) {
                    const uint32_t a = peer_addr(&pcol[i], (uint32_t)(owner ^ 1));
                    st_peer_f64(a, v.re);
                    st_peer_f64(a + 8, v.im);
                }
            }
            __syncthreads();
            if (t == 0) {
                double bv = red_v[0];
                int bidx = red_i[0];
                for (int q = 1; q < kGJT / 32; ++q) {
                    const double v2 = red_v[q];
                    const int i2 = red_i[q];
                    if (v2 > bv || (v2 == bv && i2 < bidx) || (v2 != v2 && bv == bv)) { bv = v2; bidx = i2; }
                }
                const int sing = (bv > 0.0) ? 0 : ((bv != bv) ? 2 : 1);
                s_piv = bidx;
                s_singular = sing;
                if (C > 1) {
                    st_peer_s32(peer_addr(&s_piv, (uint32_t)(owner ^ 1)), bidx);
                    st_peer_s32(peer_addr(&s_singular, (uint32_t)(owner ^ 1)), sing);
                }
            }
        }
        gj_sync<C>();
        if (s_singular) break;
        const int p = s_piv;
        if (p != k) {
            for (int c = t; c < H; c += kGJT) {
                const cplx a = A[k * H + c];
                A[k * H + c] = A[p * H + c];
                A[p * H + c] = a;
            }
        }
        __syncthreads();
        if (t == 0) {
            perm[k] = p;
            if (p != k) {
                const cplx a = pcol[k];
                pcol[k] = pcol[p];
                pcol[p] = a;
            }
        }
        __syncthreads();
        const cplx piv = pcol[k];
        const cplx inv = cdiv(cplx{1.0, 0.0}, piv);
        if (t == 0 && rank == 0) {
            logabs += log(hypot(piv.re, piv.im));
            phase += atan2(piv.im, piv.re) + (p != k ? M_PI : 0.0);
        }
        for (int c = t; c < H; c += kGJT) prow[c] = A[k * H + c] * inv;
        __syncthreads();
        // Rank-1 update: warps over rows, lanes over (at most COLS) local columns, so the
        // multiplier pcol[i] is one broadcast per row and the pivot row sits in registers.
        // Padding columns (j >= N) hold zeros and stay zero.
        const int warp = t >> 5, lane = t & 31;
        const bool own_k = rank == owner;
        // R rows per warp at a time: all their loads are issued before any arithmetic, so
        // a lane has R * COLS independent updates in flight.
        if (with_inverse) {
            cplx pr[COLS];
#pragma unroll
            for (int u = 0; u < COLS; ++u) pr[u] = (lane + 32 * u < H) ? prow[lane + 32 * u] : cplx{0.0, 0.0};
            for (int i0 = warp; i0 < N; i0 += R * (kGJT / 32)) {
                cplx m[R], a[R][COLS];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = i0 + r * (kGJT / 32);
                    const bool live = i < N && i != k;
                    m[r] = live ? cplx{0.0, 0.0} - pcol[i] : cplx{0.0, 0.0};
#pragma unroll
                    for (int u = 0; u < COLS; ++u) {
                        const int c = lane + 32 * u;
                        if (live && c < H) a[r][u] = A[i * H + c];
                    }
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = i0 + r * (kGJT / 32);
                    if (i >= N || i == k) continue;
#pragma unroll
                    for (int u = 0; u < COLS; ++u) {
                        const int c = lane + 32 * u;
                        if (c >= H) continue;
                        if (own_k && c == lk) a[r][u] = m[r] * inv;   // column k of the inverse
                        else cfma(a[r][u], m[r], pr[u]);
                        A[i * H + c] = a[r][u];
                    }
                }
            }
            for (int c = t; c < H; c += kGJT) A[k * H + c] = (own_k && c == lk) ? inv : prow[c];
        } else {
            // trailing block only: rows i > k, columns j > k
            const int c0 = (k + 1 - rank + C - 1) / C;   // first local column with j > k
            cplx pr[COLS];
#pragma unroll
            for (int u = 0; u < COLS; ++u) {
                const int c = c0 + lane + 32 * u;
                pr[u] = c < H ? prow[c] : cplx{0.0, 0.0};
            }
            for (int i0 = k + 1 + warp; i0 < N; i0 += R * (kGJT / 32)) {
                cplx m[R], a[R][COLS];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = i0 + r * (kGJT / 32);
                    m[r] = i < N ? cplx{0.0, 0.0} - pcol[i] : cplx{0.0, 0.0};
#pragma unroll
                    for (int u = 0; u < COLS; ++u) {
                        const int c = c0 + lane + 32 * u;
                        if (i < N && c < H) a[r][u] = A[i * H + c];
                    }
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = i0 + r * (kGJT / 32);
                    if (i >= N) continue;
#pragma unroll
                    for (int u = 0; u < COLS; ++u) {
                        const int c = c0 + lane + 32 * u;
                        if (c >= H) continue;
                        cfma(a[r][u], m[r], pr[u]);
                        A[i * H + c] = a[r][u];
                    }
                }
            }
        }
        gj_sync<C>();
    }
    if (s_singular) {
        if (t == 0 && rank == 0) {
            logdet[mat] = cplx{-INFINITY, 0.0};
            atomicOr(flags, s_singular == 2 ? FLAG_NONFINITE : FLAG_SINGULAR);
        }
        if (C > 1) cluster_sync_all();   // keep the peer's shared memory alive until both are done
        return;
    }
    if (with_inverse) {
        // undo the pivoting on the columns: for k = N-1..0 swap columns k and perm[k]
        if (t == 0) {
            for (int j = 0; j < N; ++j) pos[j] = j;    // pos: stored column -> final column, via idx
            int* idx = pos;                             // idx[j] = stored column at final position j
            for (int k = N - 1; k >= 0; --k) {
                const int q = perm[k];
                const int a = idx[k];
                idx[k] = idx[q];
                idx[q] = a;
            }
        }
        __syncthreads();
        // pos currently holds idx; write stored column s = idx[j] to final column j
        for (int e = t; e < N * N; e += kGJT) {
            const int i = e / N, j = e % N;
            const int sc = pos[j];
            if (sc % C != rank) continue;
            G[(int64_t)i * N + j] = A[i * H + sc / C];
        }
    }
    if (t == 0 && rank == 0) logdet[mat] = cplx{logabs, atan2(sin(phase), cos(phase))};
    if (C > 1) cluster_sync_all();
}

// ------------------------------------------------------- Gauss-Jordan in registers
// The inverse and log-determinant of an N x N complex matrix, 32 < N <= 128, held entirely in
// registers: one CTA for N <= 64, else a cluster of two CTAs (the two halves of a 128 x 128
// complex matrix fill two register files).  CTA r owns the 64 consecutive columns
// [64 r, 64 r + 64); warp w of it owns four of them, and lane l holds rows l, l + 32, ... (RQ of
// them), so the thread's block is a[RQ][4].  Pivoting is implicit: step k picks, among the rows
// not pivoted yet, the one with the largest |re| + |im| in column k (lowest row on ties), scales
// it and eliminates column k from every other row, in place, so that after N steps the stored
// array X satisfies X[p_k][j] = inverse[k][p_j] for the pivot rows p_k.  det = sign(p) prod(pivot).
// The warp owning column k+1 updates that column first, searches its pivot and publishes the
// column and the pivot row (to both CTAs' shared memory) before finishing its own update, so one
// cluster barrier per step orders the steps and the search is off the critical path.  The
// pivot row reaches the other lanes of each warp by shuffles; the column k multipliers are
// read from shared memory.  FP64 throughput bounds the elimination.
constexpr int kGJRegCols = 64;      // columns per CTA
constexpr int kGJRegThreads = 512;  // 16 warps x 4 columns

// Element arithmetic of the register Gauss-Jordan kernel.  NumD: FP64 complex.  NumFF: each of
// re, im a float pair hi + lo (~2^-44 relative, the TwoProduct / TwoSum error-free transforms on
// the fp32 pipe, which is ~64x GB300's FP64 pipe); pivot reciprocals, the read-out and the
// log-determinant are FP64 either way.
struct NumD {
    using T = cplx;
    __device__ static T from(cplx v) { return v; }
    __device__ static cplx to(const T& v) { return v; }
    __device__ static double mag(const T& v) { return abs1(v); }
    __device__ static T mul(const T& a, const T& b) { return a * b; }
    __device__ static void upd(T& a, const T& m, const T& p) { cfma(a, cplx{-m.re, -m.im}, p); }   // a -= m p
    __device__ static T negmul(const T& m, const T& b) { const cplx w = m * b; return cplx{-w.re, -w.im}; }
    __device__ static T shfl(const T& v, int src) {
        return cplx{__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
    }
    __device__ static void st_peer(uint32_t ad, const T& v) {
        st_peer_f64(ad, v.re);
        st_peer_f64(ad + 8, v.im);
    }
};
struct NumFF {
    using T = ffc;
    __device__ static T from(cplx v) {
        const float rh = (float)v.re, ih = (float)v.im;
        return ffc{rh, (float)(v.re - (double)rh), ih, (float)(v.im - (double)ih)};
    }
    __device__ static cplx to(const T& v) { return cplx{(double)v.rh + (double)v.rl, (double)v.ih + (double)v.il}; }
    __device__ static double mag(const T& v) { return (double)(fabsf(v.rh) + fabsf(v.ih)); }
    __device__ static T mul(const T& a, const T& b) {
        T r{0.f, 0.f, 0.f, 0.f};
        ff_fma(r.rh, r.rl, a.rh, a.rl, b.rh, b.rl);
        ff_fma(r.rh, r.rl, -a.ih, -a.il, b.ih, b.il);
        ff_fma(r.ih, r.il, a.rh, a.rl, b.ih, b.il);
        ff_fma(r.ih, r.il, a.ih, a.il, b.rh, b.rl);
        return r;
    }
    __device__ static void upd(T& a, const T& m, const T& p) {   // a -= m p
        ff_fma(a.rh, a.rl, -m.rh, -m.rl, p.rh, p.rl);
        ff_fma(a.rh, a.rl, m.ih, m.il, p.ih, p.il);
        ff_fma(a.ih, a.il, -m.rh, -m.rl, p.ih, p.il);
        ff_fma(a.ih, a.il, -m.ih, -m.il, p.rh, p.rl);
    }
    __device__ static T negmul(const T& m, const T& b) {
        const T w = mul(m, b);
        return ffc{-w.rh, -w.rl, -w.ih, -w.il};
    }
    __device__ static T shfl(const T& v, int src) {
        return ffc{__shfl_sync(0xffffffffu, v.rh, src), __shfl_sync(0xffffffffu, v.rl, src),
                   __shfl_sync(0xffffffffu, v.ih, src), __shfl_sync(0xffffffffu, v.il, src)};
    }
    __device__ static void st_peer(uint32_t ad, const T& v) {
        asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(ad), "f"(v.rh), "f"(v.rl), "f"(v.ih),
                     "f"(v.il)
                     : "memory");
    }
};

// 1 / z with one FP64 division: z is first scaled by an exact power of two so that its larger
// component lies in [1, 2), which keeps |z|^2 away from overflow and underflow.
__device__ __forceinline__ cplx crecip(cplx z) {
    int e = 0;
    frexp(fmax(fabs(z.re), fabs(z.im)), &e);
    const double xr = ldexp(z.re, 1 - e), xi = ldexp(z.im, 1 - e);
    const double r = 1.0 / fma(xr, xr, xi * xi);
    return cplx{ldexp(xr * r, 1 - e), ldexp(-xi * r, 1 - e)};
}

template <class T, int RQ>
__device__ __forceinline__ T sel_q(const T (&v)[RQ][4], int q, int u) {
    T r = v[0][u];
#pragma unroll
    for (int i = 1; i < RQ; ++i)
        if (q == i) r = v[i][u];
    return r;
}
template <class T, int RQ>
__device__ __forceinline__ T sel_u(const T (&v)[RQ][4], int q, int u) {
    T r = v[q][0];
#pragma unroll
    for (int i = 1; i < 4; ++i)
        if (u == i) r = v[q][i];
    return r;
}

// Pivot search over column k (local sub-column uk of the calling warp) and publication of the
// column (pre-elimination values), the pivot row (or -1 singular / -2 non-finite) and the
// pivot's reciprocal (FP64 Smith division, once here instead of in every thread).
template <class Num, int C, int RQ>
__device__ __forceinline__ void gj_reg_publish(const typename Num::T (&a)[RQ][4], int uk, unsigned used, int N,
                                               int lane, int owner_rank, typename Num::T* colbuf, int* pbuf,
                                               typename Num::T* invbuf, cplx* pivbuf) {
    using T = typename Num::T;
    double best = -1.0;
    int bi = N;
    T col[RQ];
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
        col[q] = sel_u<T, RQ>(a, q, uk);
        const int i = lane + 32 * q;
        if (i < N && !((used >> q) & 1u)) {
            const double v = Num::mag(col[q]);
            if (v > best || (v != v && best == best)) { best = v; bi = i; }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        if (v2 > best || (v2 == best && i2 < bi) || (v2 != v2 && best == best)) { best = v2; bi = i2; }
    }
    // a zero column is singular; a NaN or infinite pivot magnitude is non-finite
    const int code = (best > 0.0 && best <= DBL_MAX) ? bi : (best == 0.0 ? -1 : -2);
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
        const int i = lane + 32 * q;
        colbuf[i] = col[q];
        if (C > 1) Num::st_peer(peer_addr(&colbuf[i], (uint32_t)(owner_rank ^ 1)), col[q]);
    }
    // the pivot value from the lane that holds row bi
    const int bl = code >= 0 ? (code & 31) : 0, bq = code >= 0 ? (code >> 5) : 0;
    T pv = col[0];
#pragma unroll
    for (int q = 1; q < RQ; ++q)
        if (bq == q) pv = col[q];
    pv = Num::shfl(pv, bl);
    if (lane == 0) {
        const cplx pc = Num::to(pv);
        const T inv = Num::from(code >= 0 ? crecip(pc) : cplx{0.0, 0.0});
        *pbuf = code;
        *invbuf = inv;
        *pivbuf = pc;
        if (C > 1) {
            st_peer_s32(peer_addr(pbuf, (uint32_t)(owner_rank ^ 1)), code);
            Num::st_peer(peer_addr(invbuf, (uint32_t)(owner_rank ^ 1)), inv);
            NumD::st_peer(peer_addr(pivbuf, (uint32_t)(owner_rank ^ 1)), pc);
        }
    }
}

template <class Num, int C, int RQ>
__global__ void __launch_bounds__(kGJRegThreads, 1)
    gj_reg_kernel(cplx* Sbase, int64_t stride, int N, cplx* logdet, unsigned* flags) {
    using T = typename Num::T;
    constexpr int NR = 32 * RQ;
    __shared__ T colbuf[2][NR];
    __shared__ int pbuf[2];
    __shared__ T invbuf[2];
    __shared__ cplx pivbuf[2];
    __shared__ int perm[NR];
    __shared__ int pinv[NR];
    __shared__ cplx pivs[NR];
    const int rank = C == 1 ? 0 : (int)cluster_rank();
    const int64_t mat = C == 1 ? blockIdx.x : blockIdx.x / C;
    cplx* G = Sbase + mat * stride;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = rank * kGJRegCols + warp * 4;   // first global column of this thread
    T a[RQ][4];
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
        const int i = lane + 32 * q;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = c0 + u;
            a[q][u] = Num::from((i < N && j < N) ? G[(int64_t)i * N + j] : cplx{0.0, 0.0});
        }
    }
    unsigned used = 0;   // bit q: row lane + 32 q is a pivot row already
    auto owns = [&](int k) { return k < N && (k >> 6) == rank && ((k & 63) >> 2) == warp; };
    if (owns(0)) gj_reg_publish<Num, C, RQ>(a, 0, used, N, lane, rank, colbuf[0], &pbuf[0], &invbuf[0], &pivbuf[0]);
    gj_sync<C>();
    int singular = 0;
    for (int k = 0; k < N; ++k) {
        const int b = k & 1;
        const int p = pbuf[b];
        if (p < 0) { singular = p; break; }
        const T inv = invbuf[b];
        if (threadIdx.x == 0) { perm[k] = p; pivs[k] = pivbuf[b]; }
        const int pl = p & 31, pq = p >> 5;
        // the warp's four pivot-row entries: gathered from lane pl, each scaled by one lane
        // (lane u % 4 scales entry u), then shared again
        T rp[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) rp[u] = Num::shfl(sel_q<T, RQ>(a, pq, u), pl);
        T mine = rp[0];
#pragma unroll
        for (int u = 1; u < 4; ++u)
            if ((lane & 3) == u) mine = rp[u];
        mine = Num::mul(mine, inv);
        T prow[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) prow[u] = Num::shfl(mine, u);
        if (lane == pl) used |= 1u << pq;
        const bool ownk = owns(k);
        const int uk = k & 3;
        const bool own1 = owns(k + 1);
        const int u1 = (k + 1) & 3;
        // one element: a -= m prow, or prow in the pivot row; column k of the inverse (-m / piv,
        // 1 / piv in the pivot row) is written afterwards by its owner warp alone
        auto upd = [&](int q, int u, const T& m) {
            T v = a[q][u];
            Num::upd(v, m, prow[u]);
            a[q][u] = lane + 32 * q == p ? prow[u] : v;
        };
        if (own1) {   // look-ahead: column k+1 first, then its pivot search and publication
#pragma unroll
            for (int q = 0; q < RQ; ++q) {
                const T m = colbuf[b][lane + 32 * q];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (u == u1) upd(q, u, m);
            }
            gj_reg_publish<Num, C, RQ>(a, u1, used, N, lane, rank, colbuf[b ^ 1], &pbuf[b ^ 1], &invbuf[b ^ 1],
                                       &pivbuf[b ^ 1]);
        }
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
            const T m = colbuf[b][lane + 32 * q];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (!(own1 && u == u1)) upd(q, u, m);
        }
        if (ownk) {   // warp-uniform: column k of the inverse
#pragma unroll
            for (int q = 0; q < RQ; ++q) {
                const T val = lane + 32 * q == p ? inv : Num::negmul(colbuf[b][lane + 32 * q], inv);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (u == uk) a[q][u] = val;
            }
        }
        gj_sync<C>();
    }
    if (singular) {
        if (threadIdx.x == 0 && rank == 0) {
            logdet[mat] = cplx{-INFINITY, 0.0};
            atomicOr(flags, singular == -2 ? FLAG_NONFINITE : FLAG_SINGULAR);
        }
        if (C > 1) cluster_sync_all();   // keep shared memory alive until the peer is done
        return;
    }
    __syncthreads();
    if (threadIdx.x < N) pinv[perm[threadIdx.x]] = threadIdx.x;
    if (rank == 0 && warp == 0) {
        // log|det| and arg det: sums over the pivots in a fixed order, plus pi for an odd
        // pivot permutation (N - number of cycles transpositions)
        double la = 0.0, ph = 0.0;
        for (int k = lane; k < N; k += 32) {
            la += log(hypot(pivs[k].re, pivs[k].im));
            ph += atan2(pivs[k].im, pivs[k].re);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            la += __shfl_xor_sync(0xffffffffu, la, o);
            ph += __shfl_xor_sync(0xffffffffu, ph, o);
        }
        if (lane == 0) {
            unsigned seen[4] = {0u, 0u, 0u, 0u};
            int cycles = 0;
            for (int s0 = 0; s0 < N; ++s0) {
                if ((seen[s0 >> 5] >> (s0 & 31)) & 1u) continue;
                ++cycles;
                for (int x = s0; !((seen[x >> 5] >> (x & 31)) & 1u); x = perm[x]) seen[x >> 5] |= 1u << (x & 31);
            }
            if ((N - cycles) & 1) ph += M_PI;
            logdet[mat] = cplx{la, atan2(sin(ph), cos(ph))};
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
        const int i = lane + 32 * q;
        if (i >= N) continue;
        const int64_t orow = (int64_t)pinv[i] * N;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = c0 + u;
            if (j < N) G[orow + perm[j]] = Num::to(a[q][u]);
        }
    }
    if (C > 1) cluster_sync_all();
}

// ------------------------------------------------------------------ traces of T
__global__ void __launch_bounds__(kThreads)
    trace_kernel(const cplx* T, int W, int N, int n0, cplx* t_out, cplx* X_out, int64_t ldo) {
    __shared__ cplx sh[kThreads];
    const int w = blockIdx.x, c = blockIdx.y;
    const cplx* Tm = T + ((int64_t)c * W + w) * N * N;
    cplx tr{0.0, 0.0}, x{0.0, 0.0};
    for (int64_t e = threadIdx.x; e < (int64_t)N * N; e += kThreads) {
        const int a = (int)(e / N), b = (int)(e % N);
        const cplx tab = Tm[e];
        cfma(x, tab, Tm[(int64_t)b * N + a]);
        if (a == b) tr = tr + tab;
    }
    tr = block_sum(tr, sh);
    x = block_sum(x, sh);
    if (threadIdx.x == 0) {
        t_out[(int64_t)w * ldo + n0 + c] = tr;
        X_out[(int64_t)w * ldo + n0 + c] = x;
    }
}

// ------------------------------------------------------------------ local energy
__global__ void __launch_bounds__(kThreads) local_energy_kernel(LocalEnergyArgs a) {
    __shared__ cplx sh[kThreads];
    const int w = blockIdx.x;
    cplx e1{0.0, 0.0};
    for (int s = 0; s < 2; ++s) {
        const int Ns = s == 0 ? a.Nup : a.Ndn;
        const cplx* Th = a.Theta[s] + (int64_t)w * a.M * Ns;
        const cplx* ht = a.ht[s] + (a.wper > 0 ? (int64_t)(w / a.wper) * a.ht_stride[s] : 0);
        for (int64_t e = threadIdx.x; e < (int64_t)a.M * Ns; e += kThreads) {
            const int k = (int)(e / Ns), b = (int)(e % Ns);
            cfma(e1, ht[(int64_t)b * a.M + k], Th[e]);
        }
    }
    const double sq = sqrt(a.tau);
    cplx e2{0.0, 0.0};
    const bool energy = a.X[0] != nullptr || a.exch[0] != nullptr;
    for (int n = threadIdx.x; n < a.Nchol; n += kThreads) {
        const int64_t i = (int64_t)w * a.Nchol + n;
        const cplx ts = a.t[0][i] + a.t[1][i];
        if (energy) {
            cfma(e2, ts, ts);
            if (a.X[0]) e2 = e2 - a.X[0][i] - a.X[1][i];
        }
        cplx xb{sq * ts.im, -sq * ts.re};  // -i sqrt(tau) ts
        if (a.fb_cap > 0.0) {
            const double mag = hypot(xb.re, xb.im);
            if (mag > a.fb_cap) xb = (a.fb_cap / mag) * xb;
        }
        if (a.xbar) a.xbar[i] = xb;
    }
    if (energy) {
        e1 = block_sum(e1, sh);
        e2 = block_sum(e2, sh);
        if (threadIdx.x == 0) {
            if (a.exch[0]) e2 = e2 - a.exch[0][w] - a.exch[1][w];
            const cplx E = cplx{a.E0 + e1.re + 0.5 * e2.re, e1.im + 0.5 * e2.im};
            a.E_L[w] = E;
            if (!finite_c(E)) atomicOr(a.flags, FLAG_NONFINITE);
        }
    }
}

// ------------------------------------------------------------------ Philox4x32-10
__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                             uint32_t k0, uint32_t k1) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
}

// params (optional, device): {seed, step} read at run time (graph replays), the key being
// params[0] + seed; otherwise seed and step as given.
__global__ void philox_kernel(uint64_t seed, int64_t step, const int64_t* params, int W, int w0, int Nchol,
                              double* x) {
    const int nq = (Nchol + 3) / 4;
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)W * nq) return;
    if (params) {
        seed += (uint64_t)params[0];
        step = params[1];
    }
    const int w = (int)(id / nq), q = (int)(id % nq);
    uint32_t c0 = (uint32_t)q, c1 = (uint32_t)(w0 + w), c2 = (uint32_t)step, c3 = 0u;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        philox_round(c0, c1, c2, c3, k0, k1);
    }
    const double inv = 2.3283064365386963e-10;  // 2^-32
    const uint32_t o[4] = {c0, c1, c2, c3};
    double* xr = x + (int64_t)w * Nchol;
    for (int p = 0; p < 2; ++p) {
        const double u1 = ((double)o[2 * p] + 0.5) * inv;
        const double u2 = ((double)o[2 * p + 1] + 0.5) * inv;
        const double r = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        const int n = 4 * q + 2 * p;
        if (n < Nchol) xr[n] = r * cs;
        if (n + 1 < Nchol) xr[n + 1] = r * sn;
    }
}

// ------------------------------------------------------------------ small kernels
__global__ void hs_coeff_kernel(const double* x, const cplx* xbar, const cplx* weight, int W, int Nchol,
                                cplx* c, unsigned* flags) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)W * Nchol) return;
    const int w = (int)(id / Nchol);
    const double xv = x[id];
    if (!isfinite(xv)) atomicOr(flags, FLAG_NONFINITE);
    const bool alive = weight[w].re != 0.0 || weight[w].im != 0.0;
    c[id] = alive ? cplx{xv - xbar[id].re, -xbar[id].im} : cplx{0.0, 0.0};
}

__global__ void __launch_bounds__(kThreads) weight_kernel(WeightArgs a) {
    __shared__ cplx sh[kThreads];
    const int w = blockIdx.x;
    cplx s{0.0, 0.0};
    for (int n = threadIdx.x; n < a.Nchol; n += kThreads) {
        const int64_t i = (int64_t)w * a.Nchol + n;
        const cplx xb = a.xbar[i];
        // x xbar - xbar^2 / 2
        s = s + a.x[i] * xb;
        cfma(s, cplx{-0.5, 0.0} * xb, xb);
    }
    s = block_sum(s, sh);
    if (threadIdx.x != 0) return;
    const cplx w0 = a.weight[w];
    const bool alive = w0.re != 0.0 || w0.im != 0.0;
    if (!alive) { a.accept[w] = 0; return; }
    const cplx ln = a.logS_new[w];
    if (!finite_c(ln)) { a.accept[w] = 0; a.weight[w] = cplx{0.0, 0.0}; return; }
    const cplx dl = ln - a.logS_old[w];
    const cplx ex = cplx{dl.re + s.re + a.tau * (a.E_T - a.E0), dl.im + s.im};
    if (a.mode == AFQMC_WEIGHT_FREE) {
        const double m = exp(ex.re);
        a.weight[w] = w0 * cplx{m * cos(ex.im), m * sin(ex.im)};
    } else if (a.mode == AFQMC_WEIGHT_LOCAL) {
        // exp(-tau (E_b - E_T)), E_b the pre-step Re E_L bounded to E_T +- ebound
        const double el = a.E_L[w].re;
        if (!(el == el)) { a.accept[w] = 0; a.weight[w] = cplx{0.0, 0.0}; return; }
        const double eb = fmin(fmax(el, a.E_T - a.ebound), a.E_T + a.ebound);
        const double c = cos(dl.im);
        a.weight[w] = cplx{w0.re * exp(-a.tau * (eb - a.E_T)) * (c > 0.0 ? c : 0.0), 0.0};
    } else {
        const double c = cos(dl.im);
        a.weight[w] = cplx{w0.re * exp(ex.re) * (c > 0.0 ? c : 0.0), 0.0};
    }
    a.accept[w] = 1;
}

__global__ void commit_kernel(cplx* Phi, const cplx* Phi_new, const int* accept, int W, int64_t per) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)W * per) return;
    if (accept[id / per]) Phi[id] = Phi_new[id];
}

__global__ void __launch_bounds__(kThreads)
    qr_kernel(cplx* Phi, int64_t stride, int M, int N, const cplx* weight) {
    extern __shared__ unsigned char smem_raw[];
    cplx* v = reinterpret_cast<cplx*>(smem_raw);  // M
    cplx* r = v + M;                              // N
    __shared__ double shd[kThreads];
    const int w = blockIdx.x;
    if (weight[w].re == 0.0 && weight[w].im == 0.0) return;
    cplx* Q = Phi + (int64_t)w * stride;
    const int t = threadIdx.x;
    for (int j = 0; j < N; ++j) {
        for (int k = t; k < M; k += kThreads) v[k] = Q[(int64_t)k * N + j];
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = t; i < j; i += kThreads) {
                cplx acc{0.0, 0.0};
                for (int k = 0; k < M; ++k) cfma(acc, conjg(Q[(int64_t)k * N + i]), v[k]);
                r[i] = acc;
            }
            __syncthreads();
            for (int k = t; k < M; k += kThreads) {
                cplx acc = v[k];
                for (int i = 0; i < j; ++i) cfma(acc, cplx{0.0, 0.0} - Q[(int64_t)k * N + i], r[i]);
                v[k] = acc;
            }
            __syncthreads();
        }
        double nrm = 0.0;
        for (int k = t; k < M; k += kThreads) nrm += v[k].re * v[k].re + v[k].im * v[k].im;
        nrm = block_sum_d(nrm, shd);
        const double inv = 1.0 / sqrt(nrm);
        for (int k = t; k < M; k += kThreads) Q[(int64_t)k * N + j] = inv * v[k];
        __syncthreads();
    }
}

// E_mix = sum_w w E_L / sum_w w (fixed-order FP64); with `sums` also the two partial sums, from
// which processes holding parts of one population combine their E_mix.
__global__ void __launch_bounds__(kThreads) emix_kernel(const cplx* weight, const cplx* E_L, int W, cplx* out,
                                                        cplx* sums) {
    __shared__ cplx sh[kThreads];
    cplx num{0.0, 0.0}, den{0.0, 0.0};
    for (int w = threadIdx.x; w < W; w += kThreads) {
        cfma(num, weight[w], E_L[w]);
        den = den + weight[w];
    }
    num = block_sum(num, sh);
    den = block_sum(den, sh);
    if (threadIdx.x == 0) {
        out[0] = cdiv(num, den);
        if (sums) {
            sums[0] = num;
            sums[1] = den;
        }
    }
}

__global__ void fill_kernel(cplx* p, int64_t n, cplx v) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) p[id] = v;
}

__global__ void replicate_kernel(cplx* dst, const cplx* src, int64_t n, int copies, int64_t dst_stride) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n * copies) return;
    const int c = (int)(id / n);
    const int64_t e = id % n;
    dst[c * dst_stride + e] = src[e];
}

__global__ void r2c_kernel(const double* s, cplx* d, int64_t n) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) d[id] = cplx{s[id], 0.0};
}

__global__ void finite_kernel(const double* p, int64_t n, unsigned* flags) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n && !isfinite(p[id])) atomicOr(flags, FLAG_NONFINITE);
}

__global__ void sym_kernel(const double* L, int M, int Nchol, unsigned* flags) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)Nchol * M * M) return;
    const int n = (int)(id / ((int64_t)M * M));
    const int64_t e = id % ((int64_t)M * M);
    const int i = (int)(e / M), k = (int)(e % M);
    if (k <= i) return;
    const double a = L[id], b = L[(int64_t)n * M * M + (int64_t)k * M + i];
    if (fabs(a - b) > 1e-10 * fmax(1.0, fabs(a))) atomicOr(flags, 8u);
}

__global__ void hprime_reduce_kernel(const double* h, const cplx* parts, int nparts, int M, double* hp) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)M * M) return;
    double acc = 0.0;
    for (int p = 0; p < nparts; ++p) acc += parts[(int64_t)p * M * M + id].re;
    hp[id] = h[id] - 0.5 * acc;
}

// Hermitian split of general complex Cholesky vectors (Sec. V, Eq. (3) with complex L_n):
// V[2n] = (L_n + L_n^+)/2, V[2n+1] = (L_n - L_n^+)/(2i).  Both are Hermitian and
// sum_m V_m (x) V_m is the two-body operator of sum_n L_n (x) L_n^+ up to the exchange of the
// two electrons, which the antisymmetric fermion pair cannot see.
__global__ void herm_split_kernel(const cplx* L, int M, int Nchol, cplx* V) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t mm = (int64_t)M * M;
    if (id >= (int64_t)Nchol * mm) return;
    const int64_t n = id / mm, e = id % mm;
    const int i = (int)(e / M), k = (int)(e % M);
    const cplx a = L[id];
    const cplx b = conjg(L[n * mm + (int64_t)k * M + i]);   // (L_n^+)_ik
    const cplx d = a - b;
    V[2 * n * mm + e] = 0.5 * (a + b);
    V[(2 * n + 1) * mm + e] = cplx{0.5 * d.im, -0.5 * d.re};   // d / (2i)
}

__global__ void hprime_reduce_c_kernel(const double* h, const cplx* parts, int nparts, int M, cplx* hp) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)M * M) return;
    cplx acc{0.0, 0.0};
    for (int p = 0; p < nparts; ++p) acc = acc + parts[(int64_t)p * M * M + id];
    hp[id] = cplx{h[id] - 0.5 * acc.re, -0.5 * acc.im};
}

__device__ __forceinline__ cplx clog(cplx z) { return cplx{log(hypot(z.re, z.im)), atan2(z.im, z.re)}; }
__device__ __forceinline__ cplx cexp(cplx z) {
    const double r = exp(z.re);
    return cplx{r * cos(z.im), r * sin(z.im)};
}
__device__ __forceinline__ bool usable(cplx c, cplx l) {
    return (c.re != 0.0 || c.im != 0.0) && isfinite(l.re) && isfinite(l.im);
}

__global__ void __launch_bounds__(kThreads) msd_combine_kernel(MsdArgs a) {
    __shared__ cplx u[kMaxDets];
    __shared__ cplx sh[kThreads];
    const int w = blockIdx.x;
    if (w == 0 && threadIdx.x == 0 && a.inv_flags && (*a.inv_flags & FLAG_NONFINITE))
        atomicOr(a.flags, FLAG_NONFINITE);
    if (threadIdx.x == 0) {
        double m = -INFINITY;
        for (int I = 0; I < a.ND; ++I) {
            const cplx l = a.ls[(int64_t)I * a.ldw + w];
            if (usable(a.cc[I], l)) m = fmax(m, (clog(a.cc[I]) + l).re);
        }
        cplx Z{0.0, 0.0};
        for (int I = 0; I < a.ND; ++I) {
            const cplx l = a.ls[(int64_t)I * a.ldw + w];
            u[I] = usable(a.cc[I], l) ? cexp(clog(a.cc[I]) + l - cplx{m, 0.0}) : cplx{0.0, 0.0};
            Z = Z + u[I];
        }
        if (Z.re == 0.0 && Z.im == 0.0) {
            atomicOr(a.flags, FLAG_SINGULAR);
            a.logS[w] = cplx{-INFINITY, 0.0};
        } else {
            const cplx lz = clog(Z);
            a.logS[w] = cplx{m + lz.re, lz.im};
            for (int I = 0; I < a.ND; ++I) u[I] = cdiv(u[I], Z);
        }
    }
    __syncthreads();
    if (a.E) {
        cplx e{0.0, 0.0};
        for (int I = threadIdx.x; I < a.ND; I += kThreads)
            if (u[I].re != 0.0 || u[I].im != 0.0) e = e + u[I] * a.E[(int64_t)I * a.ldw + w];
        e = block_sum(e, sh);
        if (threadIdx.x == 0) {
            a.E_L[w] = e;
            if (!finite_c(e)) atomicOr(a.flags, FLAG_NONFINITE);
        }
    }
    if (a.t) {
        const double sq = sqrt(a.tau);
        for (int n = threadIdx.x; n < a.Nchol; n += kThreads) {
            cplx ts{0.0, 0.0};
            for (int I = 0; I < a.ND; ++I)
                if (u[I].re != 0.0 || u[I].im != 0.0) ts = ts + u[I] * a.t[((int64_t)I * a.ldw + w) * a.Nchol + n];
            cplx xb{sq * ts.im, -sq * ts.re};  // -i sqrt(tau) t
            if (a.fb_cap > 0.0) {
                const double mag = hypot(xb.re, xb.im);
                if (mag > a.fb_cap) xb = (a.fb_cap / mag) * xb;
            }
            a.xbar[(int64_t)w * a.Nchol + n] = xb;
        }
    }
}

__global__ void msd_variational_kernel(const cplx* cc, const cplx* E, const cplx* L, int ND, cplx* out) {
    double m = -INFINITY;
    for (int I = 0; I < ND; ++I)
        for (int J = 0; J < ND; ++J) {
            const cplx l = L[(int64_t)I * ND + J];
            if (usable(cc[I], l) && (cc[J].re != 0.0 || cc[J].im != 0.0))
                m = fmax(m, (clog(cc[I]) + clog(conjg(cc[J])) + l).re);
        }
    cplx num{0.0, 0.0}, den{0.0, 0.0};
    for (int I = 0; I < ND; ++I)
        for (int J = 0; J < ND; ++J) {
            const cplx l = L[(int64_t)I * ND + J];
            if (!usable(cc[I], l) || (cc[J].re == 0.0 && cc[J].im == 0.0)) continue;
            const cplx f = cexp(clog(cc[I]) + clog(conjg(cc[J])) + l - cplx{m, 0.0});
            num = num + f * E[(int64_t)I * ND + J];
            den = den + f;
        }
    *out = cdiv(num, den);
}

__global__ void cplx_add_kernel(const cplx* a, const cplx* b, cplx* d, int64_t n) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) d[id] = a[id] + b[id];
}

__global__ void c2r_scale_kernel(const cplx* s, double* d, int64_t n) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) d[id] = s[id].re;
}

__global__ void add_identity_kernel(cplx* A, int M, double s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) A[(int64_t)i * M + i].re += s;
}

inline unsigned blocks_for(int64_t n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ================================================================== launchers
// 32 x 32 tiles when they cover the output with at most 60% of the 64 x 64 tiles' area
// (small blocks of few-electron systems), 64 x 64 otherwise.
void zgemm(const GemmArgs& g, cudaStream_t st) {
    if (g.m <= 0 || g.n <= 0) return;
    const int64_t nbatch = (int64_t)g.nb0 * g.nb1 * g.nb2;
    const int64_t a64 = (int64_t)((g.m + 63) / 64) * ((g.n + 63) / 64) * 4096;
    const int64_t a32 = (int64_t)((g.m + 31) / 32) * ((g.n + 31) / 32) * 1024;
    const bool small = 10 * a32 <= 6 * a64;
    const int ts = small ? 32 : 64;
    dim3 grid((g.n + ts - 1) / ts, (g.m + ts - 1) / ts, (unsigned)std::min<int64_t>(nbatch, 65535));
    count_launch();
    auto go = [&](auto k32, auto k64) {
        if (small) k32<<<grid, kThreads, 0, st>>>(g);
        else k64<<<grid, kThreads, 0, st>>>(g);
    };
    if (g.A.real && g.B.real) go(zgemm_kernel<true, true, 32>, zgemm_kernel<true, true, 64>);
    else if (g.A.real) go(zgemm_kernel<true, false, 32>, zgemm_kernel<true, false, 64>);
    else if (g.B.real) go(zgemm_kernel<false, true, 32>, zgemm_kernel<false, true, 64>);
    else go(zgemm_kernel<false, false, 32>, zgemm_kernel<false, false, 64>);
}

void batched_inverse_logdet(cplx* S, int64_t stride, int N, int count, cplx* logdet, bool with_inverse,
                            unsigned* flags, cudaStream_t st, bool float_float) {
    if (count <= 0) return;
    const int variant = launch_policy().gj_variant;   // 0 auto, 1 shared memory, 2 registers, 3 float-float
    if (with_inverse && N > 32 && N <= 2 * kGJRegCols && variant != 1) {
        const bool ff = variant == 3 || (variant == 0 && float_float);
        count_launch();
        if (N <= kGJRegCols) {
            if (ff) gj_reg_kernel<NumFF, 1, 2><<<count, kGJRegThreads, 0, st>>>(S, stride, N, logdet, flags);
            else gj_reg_kernel<NumD, 1, 2><<<count, kGJRegThreads, 0, st>>>(S, stride, N, logdet, flags);
            return;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)count * 2);
        cfg.blockDim = dim3(kGJRegThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (ff) cudaLaunchKernelEx(&cfg, gj_reg_kernel<NumFF, 2, 4>, S, stride, N, logdet, flags);
        else cudaLaunchKernelEx(&cfg, gj_reg_kernel<NumD, 2, 4>, S, stride, N, logdet, flags);
        return;
    }
    if (N <= kGJSmemMax) {
        const int C = N <= kGJSmemOne ? 1 : 2;
        const int H = (N + C - 1) / C;
        const int cols = (H + 31) / 32;
        const size_t sm = (size_t)N * H * sizeof(cplx) + (size_t)(N + H) * sizeof(cplx) + 2 * N * sizeof(int);
        const int wi = with_inverse ? 1 : 0;
        count_launch();
        if (C == 1) {
            auto launch1 = [&](auto kern) {
                raise_dyn_smem(kern, sm);
                kern<<<count, kGJT, sm, st>>>(S, stride, N, logdet, wi, flags);
            };
            if (cols == 1) launch1(gj_smem_kernel<1, 1>);
            else if (cols == 2) launch1(gj_smem_kernel<1, 2>);
            else launch1(gj_smem_kernel<1, 3>);
        } else {
            raise_dyn_smem(gj_smem_kernel<2, 2>, sm);
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)count * 2);
            cfg.blockDim = dim3(kGJT);
            cfg.dynamicSmemBytes = sm;
            cfg.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 2;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            cudaLaunchKernelEx(&cfg, gj_smem_kernel<2, 2>, S, stride, N, logdet, wi, flags);   // H <= 64
        }
        return;
    }
    const size_t sm = (size_t)N * (2 * sizeof(cplx) + sizeof(int));
    count_launch();
    gj_kernel<<<count, kThreads, sm, st>>>(S, stride, N, logdet, with_inverse ? 1 : 0, flags);
}

void trace_terms(const cplx* T, int nc, int W, int N, int n0, cplx* t_out, cplx* X_out, int64_t ldo,
                 cudaStream_t st) {
    dim3 grid(W, nc);
    count_launch();
    trace_kernel<<<grid, kThreads, 0, st>>>(T, W, N, n0, t_out, X_out, ldo);
}

void msd_combine(const MsdArgs& a, cudaStream_t st) {
    count_launch();
    msd_combine_kernel<<<a.W, kThreads, 0, st>>>(a);
}

void msd_variational_energy(const cplx* cc, const cplx* E, const cplx* logS, int ND, cplx* out, cudaStream_t st) {
    count_launch();
    msd_variational_kernel<<<1, 1, 0, st>>>(cc, E, logS, ND, out);
}

void cplx_add(const cplx* a, const cplx* b, cplx* dst, int64_t n, cudaStream_t st) {
    count_launch();
    cplx_add_kernel<<<blocks_for(n), kThreads, 0, st>>>(a, b, dst, n);
}

void local_energy_forcebias(const LocalEnergyArgs& a, cudaStream_t st) {
    count_launch();
    local_energy_kernel<<<a.W, kThreads, 0, st>>>(a);
}

void philox_fields(uint64_t seed, int64_t step, int W, int Nchol, double* x, cudaStream_t st, int w0) {
    const int64_t n = (int64_t)W * ((Nchol + 3) / 4);
    count_launch();
    philox_kernel<<<blocks_for(n), kThreads, 0, st>>>(seed, step, nullptr, W, w0, Nchol, x);
}

void philox_fields_dev(const int64_t* params, uint64_t seed_add, int W, int Nchol, double* x, cudaStream_t st,
                       int w0) {
    const int64_t n = (int64_t)W * ((Nchol + 3) / 4);
    count_launch();
    philox_kernel<<<blocks_for(n), kThreads, 0, st>>>(seed_add, 0, params, W, w0, Nchol, x);
}

void hs_coefficients(const double* x, const cplx* xbar, const cplx* weight, int W, int Nchol, cplx* c,
                     unsigned* flags, cudaStream_t st) {
    count_launch();
    hs_coeff_kernel<<<blocks_for((int64_t)W * Nchol), kThreads, 0, st>>>(x, xbar, weight, W, Nchol, c, flags);
}

// Comb population control on one thread: the running sums must be formed left to right in
// FP64 so that every slot falls in the same interval as in any other implementation of the same
// definition.  Slot k sits at (k + xi) total / W (no fused multiply-add can form here).
__global__ void comb_kernel(const cplx* weight, int W, double xi, int* idx, double* total_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double total = 0.0;
    int last = W - 1;
    bool any = false;
    for (int j = 0; j < W; ++j) {
        total += weight[j].re;
        if (weight[j].re > 0.0) { last = j; any = true; }
    }
    if (!any) last = W - 1;
    *total_out = total;
    int j = 0;
    double c = weight[0].re;
    for (int k = 0; k < W; ++k) {
        const double u = ((double)k + xi) * total / (double)W;
        while (j < last && !(c > u)) c += weight[++j].re;
        idx[k] = j;
    }
}
__global__ void gather_rows_kernel(const cplx* src, int64_t per, const int* idx, int W, cplx* dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)W * per) return;
    const int64_t w = i / per, e = i % per;
    dst[i] = src[(int64_t)idx[w] * per + e];
}
__global__ void equal_weights_kernel(cplx* weight, int W, const double* total) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < W) weight[w] = cplx{*total / (double)W, 0.0};
}

void comb_indices(const cplx* weight, int W, double xi, int* idx, double* total, cudaStream_t st) {
    count_launch();
    comb_kernel<<<1, 32, 0, st>>>(weight, W, xi, idx, total);
}
void gather_rows(const cplx* src, int64_t per, const int* idx, int W, cplx* dst, cudaStream_t st) {
    const int64_t n = (int64_t)W * per;
    if (n <= 0) return;
    count_launch();
    gather_rows_kernel<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(src, per, idx, W, dst);
}
void equal_weights(cplx* weight, int W, const double* total, cudaStream_t st) {
    count_launch();
    equal_weights_kernel<<<(W + kThreads - 1) / kThreads, kThreads, 0, st>>>(weight, W, total);
}

void weight_update(const WeightArgs& a, cudaStream_t st) {
    count_launch();
    weight_kernel<<<a.W, kThreads, 0, st>>>(a);
}

void commit_walkers(cplx* Phi, const cplx* Phi_new, const int* accept, int W, int64_t per, cudaStream_t st) {
    count_launch();
    commit_kernel<<<blocks_for((int64_t)W * per), kThreads, 0, st>>>(Phi, Phi_new, accept, W, per);
}

void qr_reorthonormalise(cplx* Phi, int64_t stride, int M, int N, int W, const cplx* weight,
                         cudaStream_t st) {
    const size_t sm = (size_t)(M + N) * sizeof(cplx);
    count_launch();
    qr_kernel<<<W, kThreads, sm, st>>>(Phi, stride, M, N, weight);
}

void mixed_energy(const cplx* weight, const cplx* E_L, int W, cplx* out, cudaStream_t st, cplx* sums) {
    count_launch();
    emix_kernel<<<1, kThreads, 0, st>>>(weight, E_L, W, out, sums);
}

void fill_cplx(cplx* p, int64_t n, cplx v, cudaStream_t st) {
    if (n > 0) count_launch();
    if (n > 0) fill_kernel<<<blocks_for(n), kThreads, 0, st>>>(p, n, v);
}

void replicate(cplx* dst, const cplx* src, int64_t n, int copies, int64_t dst_stride, cudaStream_t st) {
    count_launch();
    replicate_kernel<<<blocks_for(n * copies), kThreads, 0, st>>>(dst, src, n, copies, dst_stride);
}

void real_to_cplx(const double* src, cplx* dst, int64_t n, cudaStream_t st) {
    count_launch();
    r2c_kernel<<<blocks_for(n), kThreads, 0, st>>>(src, dst, n);
}

void check_finite(const double* p, int64_t n, unsigned* flags, cudaStream_t st) {
    if (n > 0) count_launch();
    if (n > 0) finite_kernel<<<blocks_for(n), kThreads, 0, st>>>(p, n, flags);
}

void check_symmetric(const double* L, int M, int Nchol, unsigned* flags, cudaStream_t st) {
    const int64_t n = (int64_t)Nchol * M * M;
    count_launch();
    sym_kernel<<<blocks_for(n), kThreads, 0, st>>>(L, M, Nchol, flags);
}

namespace {

// sum_n L_n L_n^+ for symmetric (real) or Hermitian (complex) L_n, in `parts` partial sums:
// for such L_n it equals X^+ X with X[(n, k)][i] = L[n][k][i], a contiguous [Nchol*M][M]
// matrix.  The K = Nchol*M reduction is split into `parts` GEMMs (fixed split, reduced in a
// fixed order by the caller's kernel) to fill the GPU.  Returns the workspace, or NULL.
cplx* gram_of_cholesky(const void* L, bool real, int M, int Nchol, int parts, cudaStream_t st) {
    const int per = (Nchol + parts - 1) / parts;  // Cholesky vectors per part
    cplx* buf = nullptr;
    if (cudaMallocAsync(&buf, sizeof(cplx) * (size_t)parts * M * M, st) != cudaSuccess) {
        fail(AFQMC_ERR_OOM, "hprime workspace");
        return nullptr;
    }
    fill_cplx(buf, (int64_t)parts * M * M, cplx{0.0, 0.0}, st);
    for (int p = 0; p < parts; ++p) {
        const int n0 = p * per, n1 = std::min(Nchol, n0 + per);
        if (n1 <= n0) continue;
        GemmArgs g;
        g.m = g.n = M;
        g.k = (n1 - n0) * M;
        const void* X = real ? (const void*)(static_cast<const double*>(L) + (int64_t)n0 * M * M)
                             : (const void*)(static_cast<const cplx*>(L) + (int64_t)n0 * M * M);
        g.A.ptr = X; g.A.real = real; g.A.op = real ? OP_T : OP_C; g.A.ld = M;
        g.B.ptr = X; g.B.real = real; g.B.op = OP_N; g.B.ld = M;
        g.C = buf + (int64_t)p * M * M; g.ldc = M;
        zgemm(g, st);
    }
    return buf;
}

}  // namespace

void build_hprime(const double* h, const double* L, int M, int Nchol, double* hp, cudaStream_t st) {
    const int parts = std::min(Nchol, 16);
    cplx* buf = gram_of_cholesky(L, true, M, Nchol, parts, st);
    if (!buf) return;
    count_launch();
    hprime_reduce_kernel<<<blocks_for((int64_t)M * M), kThreads, 0, st>>>(h, buf, parts, M, hp);
    cudaFreeAsync(buf, st);
}

void build_hprime_hermitian(const double* h, const cplx* V, int M, int Nv, cplx* hp, cudaStream_t st) {
    const int parts = std::min(Nv, 16);
    cplx* buf = gram_of_cholesky(V, false, M, Nv, parts, st);
    if (!buf) return;
    count_launch();
    hprime_reduce_c_kernel<<<blocks_for((int64_t)M * M), kThreads, 0, st>>>(h, buf, parts, M, hp);
    cudaFreeAsync(buf, st);
}

void hermitian_split(const cplx* L, int M, int Nchol, cplx* V, cudaStream_t st) {
    const int64_t n = (int64_t)Nchol * M * M;
    count_launch();
    herm_split_kernel<<<blocks_for(n), kThreads, 0, st>>>(L, M, Nchol, V);
}

namespace {

// ||X||_1 (largest column sum of |x|) of a device M x M matrix, read on the host.
int norm1_on_host(const void* X, bool real, int M, cudaStream_t st, double* nrm) {
    const size_t n = (size_t)M * M;
    std::vector<cplx> hX(real ? 0 : n);
    std::vector<double> hR(real ? n : 0);
    cudaError_t e = real ? cudaMemcpyAsync(hR.data(), X, sizeof(double) * n, cudaMemcpyDefault, st)
                         : cudaMemcpyAsync(hX.data(), X, sizeof(cplx) * n, cudaMemcpyDefault, st);
    if (e != cudaSuccess) return fail(AFQMC_ERR_CUDA, "expm copy");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(AFQMC_ERR_CUDA, "expm sync");
    *nrm = 0.0;
    for (int j = 0; j < M; ++j) {
        double c = 0.0;
        for (int i = 0; i < M; ++i)
            c += real ? fabs(hR[(size_t)i * M + j]) : hypot(hX[(size_t)i * M + j].re, hX[(size_t)i * M + j].im);
        *nrm = std::max(*nrm, c);
    }
    return AFQMC_OK;
}

// E = exp(s Y) for a complex device matrix Y with ||Y||_1 = nrm:
// (T_q(s Y / 2^j))^(2^j), Taylor order 18 by Horner, j squarings so that ||s Y / 2^j||_1 <= 1/4
// (truncation error below 1e-20 relative).  E must not alias Y.
int expm_taylor_squaring(const cplx* Y, double nrm, double s, int M, cplx* E, cudaStream_t st) {
    nrm *= fabs(s);
    int sq = 0;
    while (nrm > 0.25 && sq < 60) { nrm *= 0.5; ++sq; }
    const double sc = s / ldexp(1.0, sq);
    cplx* Tm = nullptr;
    cplx* E0 = E;
    if (cudaMallocAsync(&Tm, sizeof(cplx) * M * M, st) != cudaSuccess) return fail(AFQMC_ERR_OOM, "expm workspace");
    // E = I
    fill_cplx(E, (int64_t)M * M, cplx{0.0, 0.0}, st);
    count_launch();
    add_identity_kernel<<<blocks_for(M), kThreads, 0, st>>>(E, M, 1.0);
    const int order = 18;
    for (int k = order; k >= 1; --k) {
        // E <- I + (sc / k) Y E
        GemmArgs g;
        g.m = g.n = g.k = M;
        g.A.ptr = Y; g.A.ld = M;
        g.B.ptr = E; g.B.ld = M;
        g.alpha = cplx{sc / k, 0.0};
        g.C = Tm; g.ldc = M;
        zgemm(g, st);
        count_launch();
        add_identity_kernel<<<blocks_for(M), kThreads, 0, st>>>(Tm, M, 1.0);
        std::swap(E, Tm);
    }
    for (int q = 0; q < sq; ++q) {
        GemmArgs g;
        g.m = g.n = g.k = M;
        g.A.ptr = E; g.A.ld = M;
        g.B.ptr = E; g.B.ld = M;
        g.C = Tm; g.ldc = M;
        zgemm(g, st);
        std::swap(E, Tm);
    }
    if (E != E0) {   // the result sits in the workspace: move it to the caller's buffer
        cudaMemcpyAsync(E0, E, sizeof(cplx) * M * M, cudaMemcpyDeviceToDevice, st);
        Tm = E;
    }
    cudaFreeAsync(Tm, st);
    return AFQMC_OK;
}

}  // namespace

int expm_real(const double* X, double s, int M, double* out, cudaStream_t st) {
    double nrm = 0.0;
    AFQMC_TRY(norm1_on_host(X, true, M, st, &nrm));
    cplx *Y = nullptr, *E = nullptr;
    const size_t bytes = sizeof(cplx) * M * M;
    if (cudaMallocAsync(&Y, bytes, st) != cudaSuccess || cudaMallocAsync(&E, bytes, st) != cudaSuccess)
        return fail(AFQMC_ERR_OOM, "expm workspace");
    real_to_cplx(X, Y, (int64_t)M * M, st);
    const int rc = expm_taylor_squaring(Y, nrm, s, M, E, st);
    if (rc == AFQMC_OK) {
        count_launch();
        c2r_scale_kernel<<<blocks_for((int64_t)M * M), kThreads, 0, st>>>(E, out, (int64_t)M * M);
    }
    cudaFreeAsync(Y, st);
    cudaFreeAsync(E, st);
    return rc;
}

int expm_complex(const cplx* X, double s, int M, cplx* out, cudaStream_t st) {
    double nrm = 0.0;
    AFQMC_TRY(norm1_on_host(X, false, M, st, &nrm));
    return expm_taylor_squaring(X, nrm, s, M, out, st);
}

}  // namespace afqmc
