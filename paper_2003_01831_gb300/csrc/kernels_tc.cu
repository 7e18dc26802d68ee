// tcgen05 + TMA split-precision GEMM engine for sm_103a.
//
// Every dense contraction of the mixed-precision walker step (overlap Psi^+ Phi, Green's
// function Phi S^-1, the Cholesky energy contraction Ltilde_n Theta, the HS potential
// sum_n c_n L_n, the Taylor terms A^k Phi and the one-body factors B Phi; Sec. V and the
// phaseless algorithm it cites) is a real GEMM C = A B^T on K-major bf16 operands stored as
// (hi, lo) pairs: x ~= hi + lo, C ~= Ahi Bhi + Ahi Blo + Alo Bhi, accumulated in fp32 in
// tensor memory.  Complex products are split into real GEMMs by the operand layouts
// (planar or "doubled" [[Re, -Im], [Im, Re]] operands) chosen by the step driver.
//
// The tensor cores round their fp32 accumulation toward zero, which biases long sums by a
// few 1e-6 relative.  The precision-critical contractions (overlap, Green's function,
// energy) therefore use row-scaled fp16 operands whose hi parts are integers with row 2-norm
// <= 2^11: the hi*hi products then sum exactly in one TMEM accumulator, and only the small
// remainder terms hi*lo + lo*hi + lo*lo (second accumulator) see the rounding ("exact" mode,
// kind::f16 with f16 inputs, four products).
//
// Kernel structure (one CTA per SM, persistent over output tiles):
//   warp 0      TMA producer: 64-wide K chunks of A (128 rows) and B (BN rows), hi and lo,
//               into a ring of shared-memory stages (128-byte swizzle).
//   warp 1      allocates tensor memory and issues tcgen05.mma (M=128, N=BN, K=16), three
//               per 16-wide K slice, into one of two TMEM accumulators.
//   warps 2..5  epilogue: tcgen05.ld 32 lanes x 32 columns at a time and write the tile.
// Every wait is bounded; on timeout the kernel sets FLAG_TIMEOUT, drains what it issued,
// frees tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>
#include <mutex>

#include "kernels_tc.cuh"
#include "tc_ptx.cuh"

namespace afqmc {

using namespace tc;

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;  // bf16 elements per K chunk (128 bytes)
constexpr int kGemmThreads = 192;

template <int BN>
struct Cfg {
    static constexpr int kStages = BN == 256 ? 2 : 3;
    static constexpr int kABytes = kBM * kBK * 2;  // one plane
    static constexpr int kBBytes = BN * kBK * 2;
    static constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;
};

// TMEM layout: NBUF accumulator buffers of (EXACT ? 2 : 1) x BN fp32 columns.
template <int BN, bool EXACT, int NBUF>
struct Tmem {
    static constexpr int kBufCols = EXACT ? 2 * BN : BN;
    static constexpr int kCols = NBUF * kBufCols;
    static_assert(kCols <= 512, "TMEM has 512 columns");
};

struct TileShape {
    int64_t rows, cols, K;
    int nbatch;
    int rt, ct;      // row / column tiles per batch
    int nk;          // K chunks
    int64_t tiles;
    BatchMap am, bm;
    const float* a_scale;  // [batch][a_rows] or null
    const float* b_scale;  // [batch][b_rows] or null
    int64_t a_rows, b_rows;
};

struct SharedCtl {
    uint64_t full[8];
    uint64_t empty[8];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t done;
    uint32_t tmem_base;
    int abort;
    double red[8][4];   // energy epilogue: per-warp (t.re, t.im, X.re, X.im)
};

__device__ __forceinline__ bool wait_drain(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kTimeoutCycles) return false;
    return true;
}

// --------------------------------------------------------------------------- epilogues
__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Writes 32 consecutive output columns [c0, c0+32) of row r (per batch b).
__device__ void epilogue_row(const EpiParams& e, int b, int64_t r, int64_t c0, const float (&v)[32]) {
    if (r >= e.rows_valid) return;
    const int ncol = (int)(e.cols_valid - c0 < 32 ? e.cols_valid - c0 : 32);
    if (ncol <= 0) return;
    const bool full = ncol == 32;
    switch (e.kind) {
        case EPI_F32: {
            float* o = e.out_f32 + b * e.ob + r * e.ld + c0;
            if (full && aligned16(o)) {
#pragma unroll
                for (int g = 0; g < 8; ++g)
                    reinterpret_cast<float4*>(o)[g] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < ncol) o[j] = v[j];
            }
            break;
        }
        default:
            break;
    }
}

// Epilogue of the three-slice GEMM: 32 consecutive columns [c0, c0+32) of row r, each value a
// float-float pair vh + vl.
__device__ __forceinline__ void st32f(float* o, const float (&v)[32]) {
    if (aligned16(o)) {
#pragma unroll
        for (int g = 0; g < 8; ++g)
            reinterpret_cast<float4*>(o)[g] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
    } else {
        for (int j = 0; j < 32; ++j) o[j] = v[j];
    }
}
__device__ void epilogue_row3(const EpiParams& e, int b, int64_t r, int64_t c0, const float (&vh)[32],
                              const float (&vl)[32]) {
    if (r >= e.rows_valid) return;
    const int ncol = (int)(e.cols_valid - c0 < 32 ? e.cols_valid - c0 : 32);
    if (ncol <= 0) return;
    const bool full = ncol == 32;
    switch (e.kind) {
        case EPI3_F64: {
            double* o = e.out_f64 + b * e.ob + r * e.ld + c0;
            if (full && aligned16(o)) {
#pragma unroll
                for (int g = 0; g < 16; ++g)
                    reinterpret_cast<double2*>(o)[g] =
                        make_double2((double)vh[2 * g] + (double)vl[2 * g], (double)vh[2 * g + 1] + (double)vl[2 * g + 1]);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < ncol) o[j] = (double)vh[j] + (double)vl[j];
            }
            break;
        }
        case EPI3_FF: {
            const int64_t off = b * e.ob + r * e.ld + c0;
            if (full) {
                st32f(e.out_f32 + off, vh);
                st32f(e.out_lo32 + off, vl);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < ncol) {
                        e.out_f32[off + j] = vh[j];
                        e.out_lo32[off + j] = vl[j];
                    }
            }
            break;
        }
        case EPI3_HSPOT_FF: {
            // row r = 2 w + c (coefficient re/im), column = i*M + k  ->  [w][i][c*M + k]
            const int64_t w = r >> 1, c = r & 1;
            const int64_t i0 = c0 / e.M, k0 = c0 % e.M;
            if (full && k0 + 32 <= e.M) {
                const int64_t off = (w * e.M + i0) * (2 * e.M) + c * e.M + k0;
                st32f(e.out_f32 + off, vh);
                st32f(e.out_lo32 + off, vl);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < ncol) {
                        const int64_t col = c0 + j, i = col / e.M, k = col % e.M;
                        const int64_t off = (w * e.M + i) * (2 * e.M) + c * e.M + k;
                        e.out_f32[off] = vh[j];
                        e.out_lo32[off] = vl[j];
                    }
            }
            break;
        }
        default:
            break;
    }
}

__device__ __forceinline__ void tile_coords(const TileShape& s, int64_t t, int& b, int& rt, int& ct) {
    const int64_t per = (int64_t)s.rt * s.ct;
    b = (int)(t / per);
    const int64_t rem = t % per;
    ct = (int)(rem / s.rt);
    rt = (int)(rem % s.rt);
}

// --------------------------------------------------------------------------- mainloop roles
template <int BN>
__device__ __forceinline__ uint8_t* stage_ptr(uint8_t* base, int st) {
    return base + (size_t)st * Cfg<BN>::kStageBytes;
}

template <int BN, typename TileFn>
__device__ void producer_loop(uint8_t* sbase, SharedCtl* ctl, const CUtensorMap* tAh, const CUtensorMap* tAl,
                              const CUtensorMap* tBh, const CUtensorMap* tBl, int64_t ntiles, int nk, TileFn coords,
                              bool three_d) {
    using C = Cfg<BN>;
    int64_t g = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int ay, az, by, bz;
        coords(t, ay, az, by, bz);
        for (int kb = 0; kb < nk; ++kb, ++g) {
            const int st = (int)(g % C::kStages);
            const uint32_t ph = (uint32_t)((g / C::kStages) & 1);
            if (!mbar_wait(&ctl->empty[st], ph ^ 1u, &ctl->abort)) { ok = false; break; }
            uint8_t* s = stage_ptr<BN>(sbase, st);
            mbar_arrive_expect_tx(&ctl->full[st], C::kStageBytes);
            const int x = kb * kBK;
            if (three_d) {
                tma_load_3d(s, tAh, &ctl->full[st], x, ay, az);
                tma_load_3d(s + C::kABytes, tAl, &ctl->full[st], x, ay, az);
                tma_load_3d(s + 2 * C::kABytes, tBh, &ctl->full[st], x, by, bz);
                tma_load_3d(s + 2 * C::kABytes + C::kBBytes, tBl, &ctl->full[st], x, by, bz);
            } else {
                tma_load_2d(s, tAh, &ctl->full[st], x, ay);
                tma_load_2d(s + C::kABytes, tAl, &ctl->full[st], x, ay);
                tma_load_2d(s + 2 * C::kABytes, tBh, &ctl->full[st], x, by);
                tma_load_2d(s + 2 * C::kABytes + C::kBBytes, tBl, &ctl->full[st], x, by);
            }
        }
    }
    if (!ok) {
        // drain: wait (bounded) for the copies of the last stages still in flight
        const int64_t first = g > C::kStages ? g - C::kStages : 0;
        for (int64_t j = first; j < g; ++j)
            wait_drain(&ctl->full[j % C::kStages], (uint32_t)((j / C::kStages) & 1));
    }
}

// Issues the MMAs of every tile of this CTA.  EXACT: hi*hi into accumulator 1 (exact for
// row-scaled operands), hi*lo + lo*hi + lo*lo into accumulator 2; else hi*hi + hi*lo + lo*hi
// into one accumulator.
template <int BN, bool EXACT, int NBUF>
__device__ void mma_loop(uint8_t* sbase, SharedCtl* ctl, int64_t ntiles, int nk) {
    using C = Cfg<BN>;
    using T = Tmem<BN, EXACT, NBUF>;
    constexpr uint32_t idesc = idesc_bf16(kBM, BN, EXACT);   // exact mode: fp16 planes
    const uint32_t tmem = ctl->tmem_base;
    int64_t g = 0;
    int it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
        const int buf = it % NBUF;
        const uint32_t u = (uint32_t)(it / NBUF);
        if (!mbar_wait(&ctl->tempty[buf], (u & 1u) ^ 1u, &ctl->abort)) break;
        tc_fence_after();
        const uint32_t d1 = tmem + (uint32_t)(buf * T::kBufCols);
        const uint32_t d2 = EXACT ? d1 + BN : d1;
        for (int kb = 0; kb < nk; ++kb, ++g) {
            const int st = (int)(g % C::kStages);
            const uint32_t ph = (uint32_t)((g / C::kStages) & 1);
            if (!mbar_wait(&ctl->full[st], ph, &ctl->abort)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sa = smem_u32(stage_ptr<BN>(sbase, st));
            const uint32_t sal = sa + C::kABytes;
            const uint32_t sb = sa + 2 * C::kABytes;
            const uint32_t sbl = sb + C::kBBytes;
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
                const uint32_t off = kk * 32;
                const uint64_t ah = desc_sw128(sa + off), al = desc_sw128(sal + off);
                const uint64_t bh = desc_sw128(sb + off), bl = desc_sw128(sbl + off);
                const uint32_t first = (kb | kk) != 0 ? 1u : 0u;
                mma_bf16(d1, ah, bh, idesc, first);
                mma_bf16(d2, ah, bl, idesc, EXACT ? first : 1u);
                mma_bf16(d2, al, bh, idesc, 1u);
                if (EXACT) mma_bf16(d2, al, bl, idesc, 1u);
            }
            mma_commit(&ctl->empty[st]);
        }
        if (!ok) break;
        mma_commit(&ctl->tfull[buf]);
    }
    // make sure nothing this thread issued is still running before TMEM is released
    mma_commit(&ctl->done);
    wait_drain(&ctl->done, 0);
}

// Epilogue-warp wait: lane 0 polls, the warp follows.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_flag) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    return ok != 0;
}

// 32 columns of an accumulator pair: v = acc1 (+ acc2); both loads issued before one wait.
template <bool EXACT>
__device__ __forceinline__ void load_acc32(uint32_t taddr1, uint32_t taddr2, float (&v)[32]) {
    uint32_t a[32], b[32];
    tmem_ld32_nw(taddr1, a);
    if (EXACT) tmem_ld32_nw(taddr2, b);
    tmem_ld_wait();
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = EXACT ? __uint_as_float(a[q]) + __uint_as_float(b[q]) : __uint_as_float(a[q]);
}

template <int BN, bool EXACT, int NBUF>
__device__ void setup_ctl(SharedCtl* ctl, int warp) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < Cfg<BN>::kStages; ++i) {
            mbar_init(&ctl->full[i], 1);
            mbar_init(&ctl->empty[i], 1);
        }
        for (int i = 0; i < NBUF; ++i) {
            mbar_init(&ctl->tfull[i], 1);
            mbar_init(&ctl->tempty[i], 128);
        }
        mbar_init(&ctl->done, 1);
        ctl->abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&ctl->tmem_base, Tmem<BN, EXACT, NBUF>::kCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

template <int BN, bool EXACT, int NBUF>
__device__ void teardown(SharedCtl* ctl, int warp, unsigned* flags) {
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(ctl->tmem_base, Tmem<BN, EXACT, NBUF>::kCols);
    }
    if (threadIdx.x == 0 && ctl->abort) atomicOr(flags, FLAG_TIMEOUT);
}

// --------------------------------------------------------------------------- generic GEMM
template <int BN, bool EXACT>
__global__ void __launch_bounds__(kGemmThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                   const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl, TileShape sh,
                   EpiParams epi, unsigned* flags) {
    using C = Cfg<BN>;
    constexpr int NBUF = 2;
    using T = Tmem<BN, EXACT, NBUF>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sbase = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    SharedCtl* ctl = reinterpret_cast<SharedCtl*>(sbase + C::kStages * C::kStageBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&tAh);
        tma_prefetch_desc(&tAl);
        tma_prefetch_desc(&tBh);
        tma_prefetch_desc(&tBl);
    }
    setup_ctl<BN, EXACT, NBUF>(ctl, warp);

    const bool three_d = sh.am.mod != (1 << 30) || sh.nbatch > 1;
    if (warp == 0) {
        if (lane == 0) {
            auto coords = [&](int64_t t, int& ay, int& az, int& by, int& bz) {
                int b, rt, ct;
                tile_coords(sh, t, b, rt, ct);
                ay = rt * kBM;
                az = (b / sh.am.div) % sh.am.mod;
                by = ct * BN;
                bz = (b / sh.bm.div) % sh.bm.mod;
            };
            producer_loop<BN>(sbase, ctl, &tAh, &tAl, &tBh, &tBl, sh.tiles, sh.nk, coords, three_d);
        }
    } else if (warp == 1) {
        if (lane == 0) mma_loop<BN, EXACT, NBUF>(sbase, ctl, sh.tiles, sh.nk);
    } else {
        const int g4 = warp & 3;
        const uint32_t lane_base = (uint32_t)(g4 * 32) << 16;
        int it = 0;
        for (int64_t t = blockIdx.x; t < sh.tiles; t += gridDim.x, ++it) {
            const int buf = it % NBUF;
            const uint32_t u = (uint32_t)(it / NBUF);
            if (!warp_wait(&ctl->tfull[buf], u & 1u, &ctl->abort)) break;
            tc_fence_after();
            int b, rt, ct;
            tile_coords(sh, t, b, rt, ct);
            const int64_t r = (int64_t)rt * kBM + g4 * 32 + lane;
            const int az = three_d ? (b / sh.am.div) % sh.am.mod : 0;
            const int bz = three_d ? (b / sh.bm.div) % sh.bm.mod : 0;
            const float sa = (sh.a_scale && r < sh.a_rows) ? sh.a_scale[(int64_t)az * sh.a_rows + r] : 1.0f;
            const uint32_t tb = ctl->tmem_base + lane_base + (uint32_t)(buf * T::kBufCols);
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                float v[32];
                load_acc32<EXACT>(tb + c * 32, tb + BN + c * 32, v);
                const int64_t c0 = (int64_t)ct * BN + c * 32;
                if (sh.a_scale || sh.b_scale) {
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int64_t col = c0 + q;
                        const float sb = (sh.b_scale && col < sh.b_rows) ? sh.b_scale[(int64_t)bz * sh.b_rows + col] : 1.0f;
                        v[q] *= sa * sb;
                    }
                }
                epilogue_row(epi, b, r, c0, v);
            }
            tc_fence_before();
            mbar_arrive(&ctl->tempty[buf]);
        }
    }
    teardown<BN, EXACT, NBUF>(ctl, warp, flags);
}

// --------------------------------------------------------------------------- energy kernel
// Tiles: (n-group of G = 128/Np Cholesky vectors) x (group of G walker-spin pairs).
// Accumulator columns of one ws: [re b = 0..Np) [im b = 0..Np).  Exact mode, one TMEM
// buffer (accumulator 1 in columns 0..255, accumulator 2 in 256..511).  EnergyShape,
// EnergySys and EnergyWork are in kernels_tc.cuh.

// Tile t -> (row group ng of nrow, walker-spin group wg): windows of ws_super walker-spin
// groups, each sweeping every row group.
__device__ __forceinline__ void energy_tile_rows(const EnergyShape& s, int64_t t, int nrow, int& ng, int& wg) {
    const int64_t per_super = (int64_t)s.ws_super * nrow;
    const int64_t sup = t / per_super;
    const int64_t rem = t % per_super;
    const int64_t first = sup * s.ws_super;
    const int width = (int)(s.ws_groups - first < s.ws_super ? s.ws_groups - first : s.ws_super);
    ng = (int)(rem / width);
    wg = (int)(first + rem % width);
}
__device__ __forceinline__ void energy_tile(const EnergyShape& s, int64_t t, int& ng, int& wg) {
    energy_tile_rows(s, t, s.n_groups, ng, wg);
}
// A pair tile (n-groups 2 ngp and 2 ngp + 1) forms the single product r*r' when every one of its
// n-groups is flagged single (the CTA-pair kernels; the one-CTA kernel never does).
__device__ __forceinline__ bool energy_pair_single(const EnergyShape& es, int ngp) {
    if (!es.single_group) return false;
    bool one = es.single_group[2 * ngp] != 0;
    if (2 * ngp + 1 < es.n_groups) one = one && es.single_group[2 * ngp + 1] != 0;
    return one;
}
template <int n>
__device__ __forceinline__ void zero_regs(uint32_t (&u)[n]) {
#pragma unroll
    for (int i = 0; i < n; ++i) u[i] = 0u;
}

// Energy kernel pipeline: K chunks of BK = 16 (32-byte swizzle, six 24 KB stages) or 32
// (64-byte swizzle, three 48 KB stages) in 144 KB of shared memory, one TMEM buffer
// (accumulator 1 in columns 0..255, accumulator 2 in 256..511).  The operands come from L2
// (~1-2 us under load), so the ring holds as many stages as the shared memory left by the
// epilogue allows: the epilogue keeps the real part of its rows of T in registers and stages
// only one plane (128 x 128 fp32, 66 KB) in shared memory (see the epilogue).  With the
// walker-spin window below, the wider chunks (half the barrier round trips per flop) are
// faster.
constexpr int kEStageRing = 144 * 1024;
// One stage: AP planes of the Ltilde rows (hi, lo and, for the rounded products, r) of 128
// rows each, then the hi and lo planes of BR Theta rows (256 for one CTA per tile, 128 per CTA
// of a pair), each K chunk of BK columns.
template <int BK, int AP, int BR>
struct EStage {
    static constexpr int kABytes = kBM * BK * 2;       // per A plane
    static constexpr int kBBytes = BR * BK * 2;        // per B plane
    static constexpr int kBOff = AP * kABytes;         // first B plane
    static constexpr int kStageBytes = AP * kABytes + 2 * kBBytes;
    static constexpr int kStages = kEStageRing / kStageBytes < 8 ? kEStageRing / kStageBytes : 8;
    static_assert(kStages >= 2, "stage ring");
};
constexpr int kEBKDefault = 32;
// Walker-spin groups per L2 window: the window's Theta pairs (512 KB per group at M = 512) stay
// in L2 while the L~ pairs stream through it once per window; the 152 CTAs then share ~19 L~
// n-groups and 8 Theta groups at a time.
constexpr int kEWsSuperDefault = 8;
constexpr int kEPitch = 129;                     // plane tile row pitch (floats): conflict-free
constexpr int kETileFloats = 128 * kEPitch;      // rows and columns

template <int BK>
__device__ __forceinline__ uint64_t edesc(uint32_t saddr) {
    return BK == 16 ? desc_sw32(saddr) : desc_sw64(saddr);
}


template <int BK, int AP>
__device__ void energy_producer(uint8_t* sbase, SharedCtl* ctl, const CUtensorMap* tAh, const CUtensorMap* tAl,
                                const CUtensorMap* tAr, const CUtensorMap* tBh, const CUtensorMap* tBl,
                                const EnergyShape& es) {
    using C = EStage<BK, AP, 256>;
    int64_t g = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < es.tiles && ok; t += gridDim.x) {
        int ng, wg;
        energy_tile(es, t, ng, wg);
        for (int kb = 0; kb < es.nk; ++kb, ++g) {
            const int st = (int)(g % C::kStages);
            const uint32_t ph = (uint32_t)((g / C::kStages) & 1);
            if (!mbar_wait(&ctl->empty[st], ph ^ 1u, &ctl->abort)) { ok = false; break; }
            uint8_t* s = sbase + (size_t)st * C::kStageBytes;
            mbar_arrive_expect_tx(&ctl->full[st], C::kStageBytes);
            const int x = kb * BK;
            const int ya = ng * es.G * es.Np, yb = wg * 2 * es.G * es.Np;   // 128 and 256 rows per group at Np | 128
            tma_load_2d(s, tAh, &ctl->full[st], x, ya);
            tma_load_2d(s + C::kABytes, tAl, &ctl->full[st], x, ya);
            if (AP == 3) tma_load_2d(s + 2 * C::kABytes, tAr, &ctl->full[st], x, ya);
            tma_load_2d(s + C::kBOff, tBh, &ctl->full[st], x, yb);
            tma_load_2d(s + C::kBOff + C::kBBytes, tBl, &ctl->full[st], x, yb);
        }
    }
    if (!ok) {
        const int64_t first = g > C::kStages ? g - C::kStages : 0;
        for (int64_t j = first; j < g; ++j) wait_drain(&ctl->full[j % C::kStages], (uint32_t)((j / C::kStages) & 1));
    }
}

// The split products of one K slice of 16.  AP = 3 (rounded products): D1 += hi*hi,
// D2 += r*lo + lo*hi, where r = fp16(y) is the row-scaled Ltilde value rounded to fp16: its bits
// beyond the integer hi carry the leading part of lo, so r*lo + lo*hi holds hi*lo + lo*hi and
// all of lo*lo but the Ltilde rounding error times lo (three products, the accuracy of four).
// AP = 2: D1 += hi*hi, D2 += hi*lo + lo*hi (+ lo*lo when `lolo`).
template <int AP, typename Mma>
__device__ __forceinline__ void energy_products(Mma mma, uint32_t d1, uint32_t d2, uint64_t ah, uint64_t al,
                                                uint64_t ar, uint64_t bh, uint64_t bl, uint32_t acc, bool lolo) {
    if (AP == 3) {
        mma(d1, ah, bh, acc);
        mma(d2, ar, bl, acc);
        mma(d2, al, bh, 1u);
    } else {
        mma(d1, ah, bh, acc);
        mma(d2, ah, bl, acc);
        mma(d2, al, bh, 1u);
        if (lolo) mma(d2, al, bl, 1u);
    }
}

// One stage of a CTA-pair energy tile (mp: Ltilde hi, lo, r and Theta hi, lo, r' tensor maps).
// Three or two products: K chunk kb of the Ltilde planes and of Theta's hi and lo.  Single
// product (rounded planes only): K chunks 2 kb and 2 kb + 1 of r (A slots 0 and 1) and r'
// (B slots 0 and 1), so a stage still carries two MMAs of K = 16 per chunk of 32 and the ring
// covers twice the K range.
template <int BK, int AP>
__device__ __forceinline__ void energy_stage_load_pair(uint8_t* s, SharedCtl* ctl, int st, const CUtensorMap* const* mp,
                                                       int kb, int ya, int yb, bool single, uint32_t rank) {
    using C = EStage<BK, AP, 128>;
    const uint32_t fb = mapa_shared(&ctl->full[st], 0);
    if (AP == 3 && single) {
        if (rank == 0) mbar_arrive_expect_tx(&ctl->full[st], 4 * (C::kABytes + C::kBBytes));   // both CTAs' bytes
        const int x0 = 2 * kb * BK;
        tma_load_2d_pair(s, mp[2], fb, x0, ya);
        tma_load_2d_pair(s + C::kABytes, mp[2], fb, x0 + BK, ya);
        tma_load_2d_pair(s + C::kBOff, mp[5], fb, x0, yb);
        tma_load_2d_pair(s + C::kBOff + C::kBBytes, mp[5], fb, x0 + BK, yb);
        return;
    }
    if (rank == 0) mbar_arrive_expect_tx(&ctl->full[st], 2 * C::kStageBytes);   // both CTAs' bytes
    const int x = kb * BK;
    tma_load_2d_pair(s, mp[0], fb, x, ya);
    tma_load_2d_pair(s + C::kABytes, mp[1], fb, x, ya);
    if (AP == 3) tma_load_2d_pair(s + 2 * C::kABytes, mp[2], fb, x, ya);
    tma_load_2d_pair(s + C::kBOff, mp[3], fb, x, yb);
    tma_load_2d_pair(s + C::kBOff + C::kBBytes, mp[4], fb, x, yb);
}

// The MMAs of one such stage (rank 0 of the pair), accumulating from the tile's first stage.
template <int BK, int AP>
__device__ __forceinline__ void energy_stage_mma_pair(uint32_t sa, uint32_t d1, uint32_t d2, int kb, bool single,
                                                      bool lolo) {
    using C = EStage<BK, AP, 128>;
    constexpr uint32_t idesc = idesc_bf16(256, 256, true);   // fp16 planes, M = 256 over the pair, N = 256
    const uint32_t sb = sa + C::kBOff;
    if (AP == 3 && single) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                mma_f16_pair(d1, edesc<BK>(sa + c * C::kABytes + kk * 32), edesc<BK>(sb + c * C::kBBytes + kk * 32),
                             idesc, (kb | c | kk) != 0 ? 1u : 0u);
        return;
    }
    const uint32_t sal = sa + C::kABytes, sar = sa + 2 * C::kABytes, sbl = sb + C::kBBytes;
#pragma unroll
    for (int kk = 0; kk < BK / 16; ++kk) {
        const uint32_t off = kk * 32;
        energy_products<AP>([&](uint32_t d, uint64_t a, uint64_t b, uint32_t c) { mma_f16_pair(d, a, b, idesc, c); },
                            d1, d2, edesc<BK>(sa + off), edesc<BK>(sal + off), edesc<BK>(sar + off),
                            edesc<BK>(sb + off), edesc<BK>(sbl + off), (kb | kk) != 0 ? 1u : 0u, lolo);
    }
}

template <int BK, int AP>
__device__ void energy_mma(uint8_t* sbase, SharedCtl* ctl, const EnergyShape& es) {
    using C = EStage<BK, AP, 256>;
    constexpr uint32_t idesc = idesc_bf16(kBM, 256, true);   // fp16 planes, M=128, N=256
    const uint32_t d1 = ctl->tmem_base, d2 = d1 + 256;
    int64_t g = 0;
    int it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < es.tiles && ok; t += gridDim.x, ++it) {
        int ng, wg;
        energy_tile(es, t, ng, wg);
        const bool lolo = es.lolo_group ? es.lolo_group[ng] != 0 : es.lolo != 0;
        if (!mbar_wait(&ctl->tempty[0], ((uint32_t)it & 1u) ^ 1u, &ctl->abort)) break;
        tc_fence_after();
        for (int kb = 0; kb < es.nk; ++kb, ++g) {
            const int st = (int)(g % C::kStages);
            const uint32_t ph = (uint32_t)((g / C::kStages) & 1);
            if (!mbar_wait(&ctl->full[st], ph, &ctl->abort)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sa = smem_u32(sbase + (size_t)st * C::kStageBytes);
            const uint32_t sal = sa + C::kABytes, sar = sa + 2 * C::kABytes;
            const uint32_t sb = sa + C::kBOff, sbl = sb + C::kBBytes;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint32_t off = kk * 32;
                energy_products<AP>([&](uint32_t d, uint64_t a, uint64_t b, uint32_t c) { mma_bf16(d, a, b, idesc, c); },
                                    d1, d2, edesc<BK>(sa + off), edesc<BK>(sal + off), edesc<BK>(sar + off),
                                    edesc<BK>(sb + off), edesc<BK>(sbl + off), (kb | kk) != 0 ? 1u : 0u, lolo);
            }
            mma_commit(&ctl->empty[st]);
        }
        if (!ok) break;
        mma_commit(&ctl->tfull[0]);
    }
    mma_commit(&ctl->done);
    wait_drain(&ctl->done, 0);
}

// Energy CTA: warp 0 = TMA producer, warp 1 = TMEM allocator + MMA issuer, warps 2..17 = epilogue
// (four warps per TMEM lane quadrant; warp w drains lanes 32 (w % 4) .. + 31 and quarter
// h = (w - 2) / 4 of the walker-spin columns, and forms the traces of those rows and columns).
constexpr int kEThreads = 576;
constexpr int kEEpi = 512;
__device__ __forceinline__ void ebar() { asm volatile("bar.sync 2, 512;" ::: "memory"); }
__device__ __forceinline__ int ebar_and(int pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 2, 512, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(pred)
        : "memory");
    return r;
}

// Epilogue of one tile of the energy kernels (warps 2..17 of a CTA): n-group ng of this CTA's
// accumulator rows, walker-spin group wg, the CTA's it-th tile (accumulator barrier phase).
// release() is called by lane 0 of each warp once the warp's tensor-memory reads are complete.
// Returns false when a wait gave up (all sixteen warps then leave together).
template <int Np, typename Release>
__device__ __forceinline__ bool energy_epilogue_tile(const EnergyShape& es, SharedCtl* ctl, float* plane,
                                                     float* colscale, double* ered, int ng, int wg, int it, bool d2,
                                                     Release release) {
    constexpr int Q = Np / 32;     // TMEM quadrants per n-block
    constexpr int G = 128 / Np;    // n-blocks (rows) and walker-spins (columns) per tile
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Epilogue.  The tile's accumulator columns are, per walker-spin j of the tile, Np real
    // columns then Np imaginary ones.  Compact column cc = j Np + b (b < Np) names element b
    // of walker-spin j; this thread owns row `row` and the 32 compact columns
    // [32 h, 32 h + 32), all in one walker-spin j.  Per (n-block, walker-spin) block, with
    // T = Tr + i Ti:
    //   t = Tr_aa + i Ti_aa,
    //   X = sum_ab T_ab T_ba = sum Tr_ab Tr_ba - sum Ti_ab Ti_ba + 2 i sum Tr_ab Ti_ba
    // (sum Ti_ab Tr_ba = sum Tr_ab Ti_ba by relabelling).  The drain writes Ti to the plane
    // tile and keeps the thread's Tr in registers; the TiTi and TrTi sums read the plane;
    // then Tr replaces it for the TrTr sum.  Partner reads T_ba run along a row of the plane
    // (lanes = consecutive a), own-row reads down a column (pitch 129): both conflict-free.
    const int q = warp & 3;                // TMEM lane quadrant: rows 32 q .. 32 q + 31
    const int h = (warp - 2) >> 2;         // compact columns [32 h, 32 h + 32)
    const int row = q * 32 + lane;         // tile row = (n-block i_blk, a)
    const int i_blk = row / Np, a = row % Np;
    const int et = threadIdx.x - 64;       // 0..511
    const uint32_t tq = ctl->tmem_base + ((uint32_t)(q * 32) << 16);
    const int cc0 = h * 32;                      // first compact column of this thread
    const int j = cc0 / Np, b0 = cc0 % Np;       // its walker-spin and first element
    const int col_re = j * 2 * Np + b0, col_im = col_re + Np;
    float* own = plane + row * kEPitch;                      // this row of the plane
    const float* pbase = plane + (i_blk * Np + b0) * kEPitch + j * Np + a;   // T_(b0+k) a
    const int cd = j * Np + a;                               // compact column of T_aa
    const bool diag = cd >= cc0 && cd < cc0 + 32;
    if (et < 256) {
        const int64_t brow = (int64_t)wg * 256 + et;
        colscale[et] = brow < (int64_t)es.nws * 2 * Np ? es.b_scale[brow] : 0.0f;
    }
    const int64_t arow = (int64_t)ng * 128 + row;
    const float sa = arow < (int64_t)es.Nchol * Np ? es.a_scale[arow] : 0.0f;
    ebar();
    // Drain.  Each warp waits for the tile, moves its Im columns of both accumulators
    // (scaled to true units) into the plane, loads its Re columns and releases tensor
    // memory at once (one arrival per warp), so the next tile's MMAs overlap the Re
    // scaling and everything after it.  If any warp's wait gave up, all sixteen leave
    // together after the release.
    const bool got = warp_wait(&ctl->tfull[0], (uint32_t)it & 1u, &ctl->abort);
    tc_fence_after();
    float tr[32];
    {
        uint32_t u1[32], u2[32];
        tmem_ld32_nw(tq + col_im, u1);
        if (d2) tmem_ld32_nw(tq + 256 + col_im, u2);
        else zero_regs(u2);   // a single-product tile leaves accumulator 2 unwritten
        tmem_ld_wait();
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const float4 cs = *reinterpret_cast<const float4*>(colscale + col_im + 4 * g);
            own[cc0 + 4 * g + 0] = (__uint_as_float(u1[4 * g + 0]) + __uint_as_float(u2[4 * g + 0])) * (sa * cs.x);
            own[cc0 + 4 * g + 1] = (__uint_as_float(u1[4 * g + 1]) + __uint_as_float(u2[4 * g + 1])) * (sa * cs.y);
            own[cc0 + 4 * g + 2] = (__uint_as_float(u1[4 * g + 2]) + __uint_as_float(u2[4 * g + 2])) * (sa * cs.z);
            own[cc0 + 4 * g + 3] = (__uint_as_float(u1[4 * g + 3]) + __uint_as_float(u2[4 * g + 3])) * (sa * cs.w);
        }
    }
    {
        uint32_t u1[32], u2[32];
        tmem_ld32_nw(tq + col_re, u1);
        if (d2) tmem_ld32_nw(tq + 256 + col_re, u2);
        else zero_regs(u2);
        tmem_ld_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0 && got) release();   // tensor memory free
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const float4 cs = *reinterpret_cast<const float4*>(colscale + col_re + 4 * g);
            tr[4 * g + 0] = (__uint_as_float(u1[4 * g + 0]) + __uint_as_float(u2[4 * g + 0])) * (sa * cs.x);
            tr[4 * g + 1] = (__uint_as_float(u1[4 * g + 1]) + __uint_as_float(u2[4 * g + 1])) * (sa * cs.y);
            tr[4 * g + 2] = (__uint_as_float(u1[4 * g + 2]) + __uint_as_float(u2[4 * g + 2])) * (sa * cs.z);
            tr[4 * g + 3] = (__uint_as_float(u1[4 * g + 3]) + __uint_as_float(u2[4 * g + 3])) * (sa * cs.w);
        }
    }
    if (!ebar_and(got ? 1 : 0)) return false;   // all sixteen warps leave together
    ebar();                                    // Ti plane complete
    // TiTi and TrTi sums over this thread's b, and the diagonal Ti_aa
    float sii = 0.f, sri = 0.f;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const float p = pbase[k * kEPitch];    // Ti[b0 + k][a] of walker-spin j
        sii = fmaf(own[cc0 + k], p, sii);
        sri = fmaf(tr[k], p, sri);
    }
    const float dim_ = diag ? own[cd] : 0.f;
    ebar();                                    // every read of the Ti plane done
#pragma unroll
    for (int k = 0; k < 32; ++k) own[cc0 + k] = tr[k];
    ebar();                                    // Tr plane complete
    // TrTr sum continues the -TiTi one, so Re X is accumulated in one register
    float srr = -sii;
#pragma unroll
    for (int k = 0; k < 32; ++k) srr = fmaf(tr[k], pbase[k * kEPitch], srr);
    const float dre = diag ? own[cd] : 0.f;
    float v0 = dre, v1 = dim_, v2 = srr, v3 = 2.0f * sri;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
        v3 += __shfl_xor_sync(0xffffffffu, v3, o);
    }
    // partial sums in fp32: the final reduction runs on one thread per output, and a chain of
    // FP64 adds there (GB300's FP64 pipe is 1/64 of the fp32 one) cost a third of a
    // single-product tile's epilogue
    float* eredf = reinterpret_cast<float*>(ered);
    if (lane < 16) {   // eredf[h][q][jj][v] for every walker-spin slot (zeros but j)
        const int jj = lane >> 2, v = lane & 3;
        const float val = jj != j ? 0.f : (v == 0 ? v0 : (v == 1 ? v1 : (v == 2 ? v2 : v3)));
        eredf[((h * 4 + q) * 4 + jj) * 4 + v] = val;
    }
    ebar();
    // one thread per (n-block, walker-spin) output: sum over the n-block's quadrants and
    // the four column quarters, in a fixed order
    if (et < G * G) {
        const int ib = et / G, jo = et % G;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        for (int hh = 0; hh < 4; ++hh)
            for (int qq = ib * Q; qq < (ib + 1) * Q; ++qq) {
                const float4 e = *reinterpret_cast<const float4*>(eredf + ((hh * 4 + qq) * 4 + jo) * 4);
                s0 += e.x;
                s1 += e.y;
                s2 += e.z;
                s3 += e.w;
            }
        const int n = ng * G + ib;
        const int ws = wg * G + jo;
        if (n < es.Nchol && ws < es.nws) {
            es.t_out[(int64_t)ws * es.Nchol + n] = cplx{(double)s0, (double)s1};
            es.X_out[(int64_t)ws * es.Nchol + n] = cplx{(double)s2, (double)s3};
        }
    }
    ebar();   // ered, colscale and the plane are read before the next tile rewrites them
    return true;
}

// Epilogue of one tile for any Np that is a multiple of 8 up to 128 (es.Np at run time; the
// batch pads each system's N to such an Np).  The tile holds G = floor(128 / Np) n-blocks (rows
// [0, G Np)) and G walker-spins (compact columns [0, G Np)); rows and compact columns beyond
// G Np are padding.  The thread owns row `row` and compact columns [32 h, 32 h + 32) as four
// chunks of 8: chunk c = 4 h + k holds compact columns 8 c .. 8 c + 7, all of walker-spin
// 8 c / Np since Np is a multiple of 8, read from tensor memory eight columns at a time.  The
// drain, the plane staging and the three sums are the fixed-Np epilogue's; the sums are kept
// per chunk, parked in the plane once it is free (Re t, Im t, Re X, Im X per row and chunk),
// and one warp reduces each (n-block, walker-spin) output over its Np rows and Np / 8 chunks
// in a fixed order.
template <typename Release>
__device__ __forceinline__ bool energy_epilogue_tile_gen(const EnergyShape& es, SharedCtl* ctl, float* plane,
                                                         float* colscale, int ng, int wg, int it, bool d2,
                                                         Release release) {
    const int Np = es.Np, G = es.G, GN = G * Np;
    // x / Np and x / G by multiply and shift (exact for the x < 256 used here)
    const uint32_t np_inv = es.np_inv, g_inv = es.g_inv;
    auto divn = [&](int x) { return (int)(((uint32_t)x * np_inv) >> 16); };
    auto divg = [&](int x) { return (int)(((uint32_t)x * g_inv) >> 16); };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3;                // TMEM lane quadrant: rows 32 q .. 32 q + 31
    const int h = (warp - 2) >> 2;         // compact columns [32 h, 32 h + 32)
    const int row = q * 32 + lane;
    const bool rok = row < GN;
    const int i_blk = divn(row), a = row - i_blk * Np;
    const int et = threadIdx.x - 64;       // 0..511
    const uint32_t tq = ctl->tmem_base + ((uint32_t)(q * 32) << 16);
    float* own = plane + row * kEPitch;
    if (et < 256) {
        const int64_t brow = (int64_t)wg * 2 * GN + et;
        colscale[et] = et < 2 * GN && brow < (int64_t)es.nws * 2 * Np ? es.b_scale[brow] : 0.0f;
    }
    const int64_t arow = (int64_t)ng * GN + row;
    const float sa = rok && arow < (int64_t)es.Nchol * Np ? es.a_scale[arow] : 0.0f;
    // chunk k: first compact column ccol(k) and the TMEM column tcol(k) of its real part; both
    // are warp-uniform, so are the chunk conditions below
    // (a padding chunk reads column 0 instead, in range, and its values are never used)
    auto ccol = [&](int k) { return 32 * h + 8 * k; };
    auto tcol = [&](int k) { return ccol(k) < GN ? ccol(k) + divn(ccol(k)) * Np : 0; };   // j 2 Np + b0
    auto icol = [&](int k) { return ccol(k) < GN ? tcol(k) + Np : 0; };
    ebar();
    const bool got = warp_wait(&ctl->tfull[0], (uint32_t)it & 1u, &ctl->abort);
    tc_fence_after();
    // Im of both accumulators, scaled to true units, into the plane: the loads of all four
    // chunks in flight at once, one wait
    {
        uint32_t u[4][2][8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            tmem_ld8_nw(tq + icol(k), u[k][0]);
            if (d2) tmem_ld8_nw(tq + 256 + icol(k), u[k][1]);
            else zero_regs(u[k][1]);
        }
        tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (ccol(k) < GN) {
                const int c0 = icol(k);
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    own[ccol(k) + e] =
                        (__uint_as_float(u[k][0][e]) + __uint_as_float(u[k][1][e])) * (sa * colscale[c0 + e]);
            }
    }
    // Re into registers, two chunks per wait (register budget); tensor memory is then free
    float tr[32];
#pragma unroll
    for (int k2 = 0; k2 < 4; k2 += 2) {
        uint32_t u[2][2][8];
#pragma unroll
        for (int k = k2; k < k2 + 2; ++k) {
            tmem_ld8_nw(tq + tcol(k), u[k - k2][0]);
            if (d2) tmem_ld8_nw(tq + 256 + tcol(k), u[k - k2][1]);
            else zero_regs(u[k - k2][1]);
        }
        tmem_ld_wait();
#pragma unroll
        for (int k = k2; k < k2 + 2; ++k) {
            const int c0 = tcol(k);
#pragma unroll
            for (int e = 0; e < 8; ++e)
                tr[8 * k + e] = ccol(k) < GN ? (__uint_as_float(u[k - k2][0][e]) + __uint_as_float(u[k - k2][1][e])) *
                                                   (sa * colscale[c0 + e])
                                             : 0.f;
        }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0 && got) release();
    if (!ebar_and(got ? 1 : 0)) return false;   // all sixteen warps leave together
    ebar();                                    // Ti plane complete
    // per chunk: TiTi and TrTi sums over its b, and the diagonal Ti_aa if the chunk holds it
    float sii[4], sri[4], dim_[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        sii[k] = 0.f;
        sri[k] = 0.f;
        dim_[k] = 0.f;
        if (rok && ccol(k) < GN) {
            const int j = divn(ccol(k)), b0 = ccol(k) - j * Np;
            const float* pb = plane + (i_blk * Np + b0) * kEPitch + j * Np + a;   // Ti[b0 + e][a]
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float pv = pb[e * kEPitch];
                sii[k] = fmaf(own[ccol(k) + e], pv, sii[k]);
                sri[k] = fmaf(tr[8 * k + e], pv, sri[k]);
            }
            const int cd = j * Np + a;
            if (cd >= ccol(k) && cd < ccol(k) + 8) dim_[k] = own[cd];
        }
    }
    ebar();                                    // every read of the Ti plane done
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (ccol(k) < GN) {
#pragma unroll
            for (int e = 0; e < 8; ++e) own[ccol(k) + e] = tr[8 * k + e];
        }
    ebar();                                    // Tr plane complete
    float srr[4], dre[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        srr[k] = -sii[k];
        dre[k] = 0.f;
        if (rok && ccol(k) < GN) {
            const int j = divn(ccol(k)), b0 = ccol(k) - j * Np;
            const float* pb = plane + (i_blk * Np + b0) * kEPitch + j * Np + a;
#pragma unroll
            for (int e = 0; e < 8; ++e) srr[k] = fmaf(tr[8 * k + e], pb[e * kEPitch], srr[k]);
            const int cd = j * Np + a;
            if (cd >= ccol(k) && cd < ccol(k) + 8) dre[k] = own[cd];
        }
    }
    ebar();                                    // every read of the Tr plane done
    // partial sums part[(c * 4 + v) * 128 + row]: the 32 lanes of a warp (consecutive rows) write
    // consecutive words, free of bank conflicts
    float* part = plane;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool v = rok && ccol(k) < GN;
        float* pc = part + (4 * h + k) * 4 * 128 + row;
        pc[0] = v ? dre[k] : 0.f;
        pc[128] = v ? dim_[k] : 0.f;
        pc[256] = v ? srr[k] : 0.f;
        pc[384] = v ? 2.0f * sri[k] : 0.f;
    }
    ebar();
    // one warp per (n-block, walker-spin) output: lane l adds rows l, l + 32, ... of the n-block
    // over the output's Np / 8 chunks in order, then a fixed shuffle tree, in fp32 (at most Np^2
    // products, the order of the fixed-Np epilogue's fp32 sums; GB300's FP64 pipe is 1/64 of the
    // fp32 one, so double adds in every lane would dominate the tile)
    const int nck = Np / 8;
    for (int o = warp - 2; o < G * G; o += kEEpi / 32) {
        const int ib = divg(o), jo = o - ib * G;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        for (int c = jo * nck; c < (jo + 1) * nck; ++c) {
            const float* pc = part + c * 4 * 128 + ib * Np;
            for (int r = lane; r < Np; r += 32) {
                s0 += pc[r];
                s1 += pc[128 + r];
                s2 += pc[256 + r];
                s3 += pc[384 + r];
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, off);
            s1 += __shfl_xor_sync(0xffffffffu, s1, off);
            s2 += __shfl_xor_sync(0xffffffffu, s2, off);
            s3 += __shfl_xor_sync(0xffffffffu, s3, off);
        }
        const int n = ng * G + ib;
        const int ws = wg * G + jo;
        if (lane == 0 && n < es.Nchol && ws < es.nws) {
            es.t_out[(int64_t)ws * es.Nchol + n] = cplx{s0, s1};
            es.X_out[(int64_t)ws * es.Nchol + n] = cplx{s2, s3};
        }
    }
    ebar();   // colscale and the partial sums are read before the next tile rewrites them
    return true;
}

// Epilogue of the single-system energy kernels: tile_of(t, ng, wg, d2) names the tile of persistent
// iteration t and whether its second accumulator was written (false for a single-product tile).
template <int Np, typename TileOf, typename Release>
__device__ void energy_epilogue(const EnergyShape& es, SharedCtl* ctl, float* plane, float* colscale, double* ered,
                                int64_t t_first, int64_t t_end, int64_t t_step, TileOf tile_of, Release release) {
    int it = 0;
    for (int64_t t = t_first; t < t_end; t += t_step, ++it) {
        int ng, wg;
        bool d2;
        tile_of(t, ng, wg, d2);
        bool ok;
        if constexpr (Np == 0) ok = energy_epilogue_tile_gen(es, ctl, plane, colscale, ng, wg, it, d2, release);
        else ok = energy_epilogue_tile<Np>(es, ctl, plane, colscale, ered, ng, wg, it, d2, release);
        if (!ok) break;
    }
}

template <int Np, int BK, int AP>
__global__ void __launch_bounds__(kEThreads, 1)
    tc_energy_kernel(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                     const __grid_constant__ CUtensorMap tAr, const __grid_constant__ CUtensorMap tBh,
                     const __grid_constant__ CUtensorMap tBl, EnergyShape es, unsigned* flags) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sbase = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    using C = EStage<BK, AP, 256>;
    float* plane = reinterpret_cast<float*>(sbase + C::kStages * C::kStageBytes);
    // 256 column scales of the tile; partial traces (fp32) at ered: [((h * 4 + q) * 4 + j) * 4 + v]
    float* colscale = plane + kETileFloats;       // 128 x 129 floats: 16-byte aligned
    double* ered = reinterpret_cast<double*>(colscale + 256);
    SharedCtl* ctl = reinterpret_cast<SharedCtl*>(ered + 256);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&tAh);
        tma_prefetch_desc(&tAl);
        if (AP == 3) tma_prefetch_desc(&tAr);
        tma_prefetch_desc(&tBh);
        tma_prefetch_desc(&tBl);
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < C::kStages; ++i) {
            mbar_init(&ctl->full[i], 1);
            mbar_init(&ctl->empty[i], 1);
        }
        mbar_init(&ctl->tfull[0], 1);
        mbar_init(&ctl->tempty[0], kEEpi / 32);   // one arrival per epilogue warp
        mbar_init(&ctl->done, 1);
        ctl->abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&ctl->tmem_base, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 0) {
        if (lane == 0) energy_producer<BK, AP>(sbase, ctl, &tAh, &tAl, &tAr, &tBh, &tBl, es);
    } else if (warp == 1) {
        if (lane == 0) energy_mma<BK, AP>(sbase, ctl, es);
    } else {
        energy_epilogue<Np>(
            es, ctl, plane, colscale, ered, blockIdx.x, es.tiles, gridDim.x,
            [&](int64_t t, int& ng, int& wg, bool& d2) {
                energy_tile(es, t, ng, wg);
                d2 = true;
            },
            [&]() { mbar_arrive(&ctl->tempty[0]); });
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(ctl->tmem_base, 512);
    }
    if (threadIdx.x == 0 && ctl->abort) atomicOr(flags, FLAG_TIMEOUT);
}

// ---------------------------------------------------------------- energy kernel, CTA pairs
// The same contraction on pairs of SMs (cta_group::2): a cluster of two CTAs computes the tiles
// of two n-groups (rank r: n-group 2 p + r) against one walker-spin group with one M = 256 MMA
// per K slice, issued by rank 0.  Each CTA stages its own 128 rows of Ltilde and half of the
// tile's 256 Theta rows (rank r: rows 128 r .. 128 r + 127), so a stage holds 128 + 128 rows
// per SM instead of 128 + 256: two thirds of the operand bytes per MMA of the one-CTA kernel,
// and four stages in the same ring.  Each CTA's tensor memory receives its own n-group's
// 128 x 256 accumulators, so the epilogue is the one-CTA kernel's.
// Synchronisation: rank 0's full[] barriers count both CTAs' TMA bytes (rank 0 posts the
// expected total); rank 0's MMA commits arrive on both CTAs' empty[] and tfull barriers
// (multicast); every epilogue warp of both CTAs arrives on rank 0's tempty.
template <int BK, int AP>
__device__ void energy_producer2(uint8_t* sbase, SharedCtl* ctl, const CUtensorMap* tAh, const CUtensorMap* tAl,
                                 const CUtensorMap* tAr, const CUtensorMap* tBh, const CUtensorMap* tBl,
                                 const CUtensorMap* tBr, const EnergyShape& es, uint32_t rank) {
    using C = EStage<BK, AP, 128>;
    const CUtensorMap* const mp[6] = {tAh, tAl, tAr, tBh, tBl, tBr};
    int64_t g = 0;
    bool ok = true;
    for (int64_t t = cluster_id_x(); t < es.tiles2 && ok; t += ncluster_x()) {
        int ngp, wg;
        energy_tile_rows(es, t, es.n_pairs, ngp, wg);
        const int ng = 2 * ngp + (int)rank;
        const bool single = energy_pair_single(es, ngp);
        const int nst = single ? es.nk / 2 : es.nk;   // es.nk is even (M % 64 == 0)
        const int ya = ng * es.G * es.Np, yb = wg * 2 * es.G * es.Np + (int)rank * 128;
        for (int kb = 0; kb < nst; ++kb, ++g) {
            const int st = (int)(g % C::kStages);
            const uint32_t ph = (uint32_t)((g / C::kStages) & 1);
            if (!mbar_wait(&ctl->empty[st], ph ^ 1u, &ctl->abort)) { ok = false; break; }
            energy_stage_load_pair<BK, AP>(sbase + (size_t)st * C::kStageBytes, ctl, st, mp, kb, ya, yb, single, rank);
        }
    }
    if (!ok) {
        if (rank == 0) {
            const int64_t first = g > C::kStages ? g - C::kStages : 0;
            for (int64_t j = first; j < g; ++j)
                wait_drain(&ctl->full[j % C::kStages], (uint32_t)((j / C::kStages) & 1));
        } else {
            // the peer cannot wait on rank 0's barriers: give its copies in flight time to land
            const long long t0 = clock64();
            while (clock64() - t0 < (1LL << 22)) {
            }
        }
    }
}

template <int BK, int AP>
__device__ void energy_mma2(uint8_t* sbase, SharedCtl* ctl, const EnergyShape& es) {
    using C = EStage<BK, AP, 128>;
    const uint32_t d1 = ctl->tmem_base, d2 = d1 + 256;
    int64_t g = 0;
    int it = 0;
    bool ok = true;
    for (int64_t t = cluster_id_x(); t < es.tiles2 && ok; t += ncluster_x(), ++it) {
        int ngp, wg;
        energy_tile_rows(es, t, es.n_pairs, ngp, wg);
        bool lolo = es.lolo != 0;
        if (es.lolo_group) {
            lolo = es.lolo_group[2 * ngp] != 0;
            if (2 * ngp + 1 < es.n_groups) lolo = lolo || es.lolo_group[2 * ngp + 1] != 0;
        }
        const bool single = energy_pair_single(es, ngp);
        const int nst = single ? es.nk / 2 : es.nk;
        if (!mbar_wait(&ctl->tempty[0], ((uint32_t)it & 1u) ^ 1u, &ctl->abort)) break;
        tc_fence_after();
        for (int kb = 0; kb < nst; ++kb, ++g) {
            const int st = (int)(g % C::kStages);
            const uint32_t ph = (uint32_t)((g / C::kStages) & 1);
            if (!mbar_wait(&ctl->full[st], ph, &ctl->abort)) { ok = false; break; }
            tc_fence_after();
            energy_stage_mma_pair<BK, AP>(smem_u32(sbase + (size_t)st * C::kStageBytes), d1, d2, kb, single, lolo);
            mma_commit_pair(&ctl->empty[st], 3);   // the stage is free in both CTAs
        }
        if (!ok) break;
        mma_commit_pair(&ctl->tfull[0], 3);        // both CTAs' accumulators are complete
    }
    mma_commit_pair(&ctl->done, 1);
    wait_drain(&ctl->done, 0);
}

template <int Np, int BK, int AP>
__global__ void __launch_bounds__(kEThreads, 1)
    tc_energy_pair_kernel(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                          const __grid_constant__ CUtensorMap tAr, const __grid_constant__ CUtensorMap tBh,
                          const __grid_constant__ CUtensorMap tBl, const __grid_constant__ CUtensorMap tBr,
                          EnergyShape es, unsigned* flags) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sbase = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    using C = EStage<BK, AP, 128>;
    float* plane = reinterpret_cast<float*>(sbase + C::kStages * C::kStageBytes);
    float* colscale = plane + kETileFloats;
    double* ered = reinterpret_cast<double*>(colscale + 256);
    SharedCtl* ctl = reinterpret_cast<SharedCtl*>(ered + 256);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&tAh);
        tma_prefetch_desc(&tAl);
        if (AP == 3) tma_prefetch_desc(&tAr);
        tma_prefetch_desc(&tBh);
        tma_prefetch_desc(&tBl);
        if (AP == 3 && es.single_group) tma_prefetch_desc(&tBr);
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < C::kStages; ++i) {
            mbar_init(&ctl->full[i], 1);
            mbar_init(&ctl->empty[i], 1);
        }
        mbar_init(&ctl->tfull[0], 1);
        mbar_init(&ctl->tempty[0], 2 * (kEEpi / 32));   // one arrival per epilogue warp of both CTAs
        mbar_init(&ctl->done, 1);
        ctl->abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    cluster_sync();   // both CTAs' barriers exist before any copy or arrival reaches them
    if (warp == 1) {
        tmem_alloc_pair(&ctl->tmem_base, 512);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    cluster_sync();   // tensor memory allocated in both CTAs before the first MMA

    if (warp == 0) {
        if (lane == 0) energy_producer2<BK, AP>(sbase, ctl, &tAh, &tAl, &tAr, &tBh, &tBl, &tBr, es, rank);
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) energy_mma2<BK, AP>(sbase, ctl, es);
    } else {
        const uint32_t tempty0 = mapa_shared(&ctl->tempty[0], 0);
        energy_epilogue<Np>(
            es, ctl, plane, colscale, ered, cluster_id_x(), es.tiles2, ncluster_x(),
            [&](int64_t t, int& ng, int& wg, bool& d2) {
                int ngp;
                energy_tile_rows(es, t, es.n_pairs, ngp, wg);
                ng = 2 * ngp + (int)rank;
                d2 = !energy_pair_single(es, ngp);
            },
            [&]() { mbar_arrive_cluster(tempty0); });
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();   // both CTAs are done with tensor memory and each other's shared memory
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(ctl->tmem_base, 512);
    }
    if (threadIdx.x == 0 && ctl->abort) atomicOr(flags, FLAG_TIMEOUT);
}

// ---------------------------------------------------------------- energy kernel, many systems
// One persistent launch for the energy contractions of several independent systems (a batch of
// uneven problems): a work list of pair tiles (system, n-group pair, walker-spin group) over
// every system, each system with its own operands (tensor maps kept in global memory), K,
// Np and outputs.  Per tile the arithmetic, and its order, are the single-system CTA-pair
// kernel's; only the tile's source changes.
template <int BK, int AP>
__device__ void energy_producer_multi(uint8_t* sbase, SharedCtl* ctl, const EnergySys* sys, const EnergyWork* work,
                                      int64_t nwork, uint32_t rank) {
    using C = EStage<BK, AP, 128>;
    int64_t g = 0;
    bool ok = true;
    for (int64_t t = cluster_id_x(); t < nwork && ok; t += ncluster_x()) {
        const EnergyWork w = work[t];
        const EnergySys* S = sys + w.sys;
        const bool single = energy_pair_single(S->es, w.ngp);
        const int nst = single ? S->es.nk / 2 : S->es.nk;
        const int ng = 2 * w.ngp + (int)rank;
        const CUtensorMap* const mp[6] = {&S->map[0], &S->map[1], &S->map[2], &S->map[3], &S->map[4], &S->map[5]};
        const int ya = ng * S->es.G * S->es.Np, yb = w.wg * 2 * S->es.G * S->es.Np + (int)rank * 128;
        for (int kb = 0; kb < nst; ++kb, ++g) {
            const int st = (int)(g % C::kStages);
            const uint32_t ph = (uint32_t)((g / C::kStages) & 1);
            if (!mbar_wait(&ctl->empty[st], ph ^ 1u, &ctl->abort)) { ok = false; break; }
            energy_stage_load_pair<BK, AP>(sbase + (size_t)st * C::kStageBytes, ctl, st, mp, kb, ya, yb, single, rank);
        }
    }
    if (!ok) {
        if (rank == 0) {
            const int64_t first = g > C::kStages ? g - C::kStages : 0;
            for (int64_t j = first; j < g; ++j)
                wait_drain(&ctl->full[j % C::kStages], (uint32_t)((j / C::kStages) & 1));
        } else {
            const long long t0 = clock64();
            while (clock64() - t0 < (1LL << 22)) {
            }
        }
    }
}

template <int BK, int AP>
__device__ void energy_mma_multi(uint8_t* sbase, SharedCtl* ctl, const EnergySys* sys, const EnergyWork* work,
                                 int64_t nwork) {
    using C = EStage<BK, AP, 128>;
    const uint32_t d1 = ctl->tmem_base, d2 = d1 + 256;
    int64_t g = 0;
    int it = 0;
    bool ok = true;
    for (int64_t t = cluster_id_x(); t < nwork && ok; t += ncluster_x(), ++it) {
        const EnergyWork w = work[t];
        const EnergyShape& es = sys[w.sys].es;
        bool lolo = es.lolo != 0;
        if (es.lolo_group) {
            lolo = es.lolo_group[2 * w.ngp] != 0;
            if (2 * w.ngp + 1 < es.n_groups) lolo = lolo || es.lolo_group[2 * w.ngp + 1] != 0;
        }
        const bool single = energy_pair_single(es, w.ngp);
        const int nst = single ? es.nk / 2 : es.nk;
        if (!mbar_wait(&ctl->tempty[0], ((uint32_t)it & 1u) ^ 1u, &ctl->abort)) break;
        tc_fence_after();
        for (int kb = 0; kb < nst; ++kb, ++g) {
            const int st = (int)(g % C::kStages);
            const uint32_t ph = (uint32_t)((g / C::kStages) & 1);
            if (!mbar_wait(&ctl->full[st], ph, &ctl->abort)) { ok = false; break; }
            tc_fence_after();
            energy_stage_mma_pair<BK, AP>(smem_u32(sbase + (size_t)st * C::kStageBytes), d1, d2, kb, single, lolo);
            mma_commit_pair(&ctl->empty[st], 3);
        }
        if (!ok) break;
        mma_commit_pair(&ctl->tfull[0], 3);
    }
    mma_commit_pair(&ctl->done, 1);
    wait_drain(&ctl->done, 0);
}

template <int BK, int AP>
__global__ void __launch_bounds__(kEThreads, 1)
    tc_energy_multi_kernel(const EnergySys* __restrict__ sys, const EnergyWork* __restrict__ work, int64_t nwork,
                           unsigned* flags) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sbase = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    using C = EStage<BK, AP, 128>;
    float* plane = reinterpret_cast<float*>(sbase + C::kStages * C::kStageBytes);
    float* colscale = plane + kETileFloats;
    double* ered = reinterpret_cast<double*>(colscale + 256);
    SharedCtl* ctl = reinterpret_cast<SharedCtl*>(ered + 256);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    if (threadIdx.x == 0) {
        for (int i = 0; i < C::kStages; ++i) {
            mbar_init(&ctl->full[i], 1);
            mbar_init(&ctl->empty[i], 1);
        }
        mbar_init(&ctl->tfull[0], 1);
        mbar_init(&ctl->tempty[0], 2 * (kEEpi / 32));
        mbar_init(&ctl->done, 1);
        ctl->abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    cluster_sync();
    if (warp == 1) {
        tmem_alloc_pair(&ctl->tmem_base, 512);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    cluster_sync();

    if (warp == 0) {
        if (lane == 0) energy_producer_multi<BK, AP>(sbase, ctl, sys, work, nwork, rank);
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) energy_mma_multi<BK, AP>(sbase, ctl, sys, work, nwork);
    } else {
        const uint32_t tempty0 = mapa_shared(&ctl->tempty[0], 0);
        auto release = [&]() { mbar_arrive_cluster(tempty0); };
        int it = 0;
        for (int64_t t = cluster_id_x(); t < nwork; t += ncluster_x(), ++it) {
            const EnergyWork w = work[t];
            const EnergyShape& es = sys[w.sys].es;
            const int ng = 2 * w.ngp + (int)rank;
            const bool d2 = !energy_pair_single(es, w.ngp);
            bool ok;
            switch (es.Np) {
                case 32: ok = energy_epilogue_tile<32>(es, ctl, plane, colscale, ered, ng, w.wg, it, d2, release); break;
                case 64: ok = energy_epilogue_tile<64>(es, ctl, plane, colscale, ered, ng, w.wg, it, d2, release); break;
                case 128:
                    ok = energy_epilogue_tile<128>(es, ctl, plane, colscale, ered, ng, w.wg, it, d2, release);
                    break;
                default: ok = energy_epilogue_tile_gen(es, ctl, plane, colscale, ng, w.wg, it, d2, release); break;
            }
            if (!ok) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(ctl->tmem_base, 512);
    }
    if (threadIdx.x == 0 && ctl->abort) atomicOr(flags, FLAG_TIMEOUT);
}

// --------------------------------------------------------------------------- row split
// One warp per row: scale = 2^(e-11) with ||x||_2 < 2^e, hi = rint(x/scale) (|hi| <= 2048, an
// integer, exact in fp16), lo = fp16(x/scale - hi).  ||hi||_2 <= 2^11 + sqrt(K)/2, so by
// Cauchy-Schwarz every partial sum of hi_A . hi_B is an integer below 2^23: exact in fp32.
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
// four halves at an 8-byte aligned address
__device__ __forceinline__ void store4h(__half* p, const __half (&h)[4]) {
    uint2 u;
    u.x = (uint32_t)__half_as_ushort(h[0]) | ((uint32_t)__half_as_ushort(h[1]) << 16);
    u.y = (uint32_t)__half_as_ushort(h[2]) | ((uint32_t)__half_as_ushort(h[3]) << 16);
    *reinterpret_cast<uint2*>(p) = u;
}

// With `rnd` set, also r = fp16(x/scale) (the rounded plane of the energy contraction's
// three rounded products).
template <typename Src>
__global__ void __launch_bounds__(256) split_rows_kernel(const Src* src, int64_t src_stride, int64_t rows, int64_t K,
                                                         __half* hi, __half* lo, float* scale, __half* rnd) {
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const Src* x = src + r * src_stride;
    // four consecutive values per lane when rows allow 16-byte (float) / 32-byte (double) loads
    const bool vec = (K & 3) == 0 && (reinterpret_cast<uintptr_t>(x) & (4 * sizeof(Src) - 1)) == 0;
    double ss = 0.0;
    if (vec) {
        for (int64_t k = 4 * lane; k < K; k += 128) {
            double v[4];
            load4(x + k, v);
            ss += v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
        }
    } else {
        for (int64_t k = lane; k < K; k += 32) ss += (double)x[k] * (double)x[k];
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const double nrm = sqrt(ss);
    int e = 0;
    if (nrm > 0.0) frexp(nrm, &e);        // nrm < 2^e
    const double inv = nrm > 0.0 ? ldexp(1.0, 11 - e) : 0.0;
    if (lane == 0) scale[r] = nrm > 0.0 ? (float)ldexp(1.0, e - 11) : 1.0f;
    if (vec) {
        for (int64_t k = 4 * lane; k < K; k += 128) {
            double v[4];
            load4(x + k, v);
            __half h[4], l[4], rr[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const double y = v[q] * inv;   // |y| < 2048
                const double s1 = rint(y);
                h[q] = __double2half(s1);
                l[q] = __double2half(y - s1);
                rr[q] = __double2half(y);
            }
            store4h(hi + r * K + k, h);
            store4h(lo + r * K + k, l);
            if (rnd) store4h(rnd + r * K + k, rr);
        }
    } else {
        for (int64_t k = lane; k < K; k += 32) {
            const double y = (double)x[k] * inv;
            const double s1 = rint(y);
            hi[r * K + k] = __double2half(s1);
            lo[r * K + k] = __double2half(y - s1);
            if (rnd) rnd[r * K + k] = __double2half(y);
        }
    }
}

// fp32 rows: the same split in single precision (FMA/ALU pipes; the FP64 pipe is narrow).  The
// row norm is summed in fp32 and raised by 2^-10 before the exponent is taken, so
// ||x||_2 < 2^e still holds (rows at most 2^-10 below a power of two get the next scale up);
// y = x / scale is exact (a power of two), rint(y) and y - rint(y) are exact in fp32.
__global__ void __launch_bounds__(256) split_rows_f32_kernel(const float* src, int64_t src_stride, int64_t rows,
                                                             int64_t K, __half* hi, __half* lo, float* scale,
                                                             __half* rnd) {
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const float* x = src + r * src_stride;
    const bool vec = (K & 3) == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
    float ss = 0.f;
    if (vec) {
        for (int64_t k = 4 * lane; k < K; k += 128) {
            const float4 a = *reinterpret_cast<const float4*>(x + k);
            ss = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, ss))));
        }
    } else {
        for (int64_t k = lane; k < K; k += 32) ss = fmaf(x[k], x[k], ss);
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const float nrm = sqrtf(ss) * (1.0f + 0x1p-10f);
    int e = 0;
    if (nrm > 0.f) frexpf(nrm, &e);
    const float inv = nrm > 0.f ? ldexpf(1.0f, 11 - e) : 0.f;
    if (lane == 0) scale[r] = nrm > 0.f ? ldexpf(1.0f, e - 11) : 1.0f;
    if (vec) {
        for (int64_t k = 4 * lane; k < K; k += 128) {
            const float4 a = *reinterpret_cast<const float4*>(x + k);
            const float v[4] = {a.x, a.y, a.z, a.w};
            __half h[4], l[4], rr[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float y = v[q] * inv, s1 = rintf(y);
                h[q] = __float2half_rn(s1);
                l[q] = __float2half_rn(y - s1);
                rr[q] = __float2half_rn(y);
            }
            store4h(hi + r * K + k, h);
            store4h(lo + r * K + k, l);
            if (rnd) store4h(rnd + r * K + k, rr);
        }
    } else {
        for (int64_t k = lane; k < K; k += 32) {
            const float y = x[k] * inv, s1 = rintf(y);
            hi[r * K + k] = __float2half_rn(s1);
            lo[r * K + k] = __float2half_rn(y - s1);
            if (rnd) rnd[r * K + k] = __float2half_rn(y);
        }
    }
}

// --------------------------------------------------------------------------- three-slice overlap
// S = Psi^T Phi to ~1e-9 (the overlap's log-determinant sets the phaseless weights, whose
// relative errors multiply the spread of the local energies in E_mix).  Rows are split into
// three fp16 slices with the row scale s = 2^(e-11) of the two-slice mode:
//   y = x / s,  h = rint(y) (|h| <= 2048),  m = rint((y - h) 2^7) (|m| <= 64),
//   l = fp16((y - h) 2^7 - m),  x = s (h + 2^-7 (m + l)).
// Products x_a x_b = s_a s_b [h h' + 2^-7 (h m' + m h') + 2^-7 (h l' + l h') + 2^-14 m m' + ...];
// the four kept groups go to four TMEM accumulators.  For K <= 1024 the partial sums of h h',
// h m' + m h' and m m' are integers below 2^24 (Cauchy-Schwarz), hence exact in fp32; the
// l terms are 2^-7 smaller and only rounded.  The dropped 2^-14 (m l' + l m' + l l') terms are
// ~1e-9 of |x_a||x_b|.
constexpr double kS3 = 1.0 / 128.0;

constexpr int kG3ABytes = kBM * kBK * 2;          // one plane, 128 rows x 64
constexpr int kG3BBytes = 128 * kBK * 2;          // B tile: 128 rows
constexpr int kG3StageBytes = 3 * (kG3ABytes + kG3BBytes);   // 96 KB
constexpr int kG3Stages = 2;

__global__ void __launch_bounds__(kGemmThreads, 1)
    tc_gemm3_kernel(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
                    const __grid_constant__ CUtensorMap tA2, const __grid_constant__ CUtensorMap tB0,
                    const __grid_constant__ CUtensorMap tB1, const __grid_constant__ CUtensorMap tB2, TileShape sh,
                    EpiParams epi, unsigned* flags) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sbase = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    SharedCtl* ctl = reinterpret_cast<SharedCtl*>(sbase + kG3Stages * kG3StageBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool three_d = sh.am.mod != (1 << 30) || sh.nbatch > 1;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kG3Stages; ++i) {
            mbar_init(&ctl->full[i], 1);
            mbar_init(&ctl->empty[i], 1);
        }
        mbar_init(&ctl->tfull[0], 1);
        mbar_init(&ctl->tempty[0], 128);
        mbar_init(&ctl->done, 1);
        ctl->abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&ctl->tmem_base, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        if (lane == 0) {
            const CUtensorMap* A[3] = {&tA0, &tA1, &tA2};
            const CUtensorMap* B[3] = {&tB0, &tB1, &tB2};
            int64_t g = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < sh.tiles && ok; t += gridDim.x) {
                int b, rt, ct;
                tile_coords(sh, t, b, rt, ct);
                const int az = three_d ? (b / sh.am.div) % sh.am.mod : 0;
                const int bz = three_d ? (b / sh.bm.div) % sh.bm.mod : 0;
                for (int kb = 0; kb < sh.nk; ++kb, ++g) {
                    const int st = (int)(g % kG3Stages);
                    const uint32_t ph = (uint32_t)((g / kG3Stages) & 1);
                    if (!mbar_wait(&ctl->empty[st], ph ^ 1u, &ctl->abort)) { ok = false; break; }
                    uint8_t* sp = sbase + (size_t)st * kG3StageBytes;
                    mbar_arrive_expect_tx(&ctl->full[st], kG3StageBytes);
                    const int x = kb * kBK;
                    for (int q = 0; q < 3; ++q) {
                        if (three_d) {
                            tma_load_3d(sp + q * kG3ABytes, A[q], &ctl->full[st], x, rt * kBM, az);
                            tma_load_3d(sp + 3 * kG3ABytes + q * kG3BBytes, B[q], &ctl->full[st], x, ct * 128, bz);
                        } else {
                            tma_load_2d(sp + q * kG3ABytes, A[q], &ctl->full[st], x, rt * kBM);
                            tma_load_2d(sp + 3 * kG3ABytes + q * kG3BBytes, B[q], &ctl->full[st], x, ct * 128);
                        }
                    }
                }
            }
            if (!ok) {
                const int64_t first = g > kG3Stages ? g - kG3Stages : 0;
                for (int64_t j = first; j < g; ++j)
                    wait_drain(&ctl->full[j % kG3Stages], (uint32_t)((j / kG3Stages) & 1));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(kBM, 128, true);
            const uint32_t d1 = ctl->tmem_base, d2 = d1 + 128, d3 = d1 + 256, d4 = d1 + 384;
            int64_t g = 0;
            int it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < sh.tiles && ok; t += gridDim.x, ++it) {
                if (!mbar_wait(&ctl->tempty[0], ((uint32_t)it & 1u) ^ 1u, &ctl->abort)) break;
                tc_fence_after();
                for (int kb = 0; kb < sh.nk; ++kb, ++g) {
                    const int st = (int)(g % kG3Stages);
                    const uint32_t ph = (uint32_t)((g / kG3Stages) & 1);
                    if (!mbar_wait(&ctl->full[st], ph, &ctl->abort)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(sbase + (size_t)st * kG3StageBytes);
                    const uint32_t sb = sa + 3 * kG3ABytes;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint32_t off = kk * 32;
                        const uint64_t ah = desc_sw128(sa + off), am = desc_sw128(sa + kG3ABytes + off),
                                       al = desc_sw128(sa + 2 * kG3ABytes + off);
                        const uint64_t bh = desc_sw128(sb + off), bm = desc_sw128(sb + kG3BBytes + off),
                                       bl = desc_sw128(sb + 2 * kG3BBytes + off);
                        const uint32_t acc = (kb | kk) != 0 ? 1u : 0u;
                        mma_bf16(d1, ah, bh, idesc, acc);
                        mma_bf16(d2, ah, bm, idesc, acc);
                        mma_bf16(d2, am, bh, idesc, 1u);
                        mma_bf16(d3, ah, bl, idesc, acc);
                        mma_bf16(d3, al, bh, idesc, 1u);
                        mma_bf16(d4, am, bm, idesc, acc);
                    }
                    mma_commit(&ctl->empty[st]);
                }
                if (!ok) break;
                mma_commit(&ctl->tfull[0]);
            }
            mma_commit(&ctl->done);
            wait_drain(&ctl->done, 0);
        }
    } else {
        const int g4 = warp & 3;
        const uint32_t tb = ctl->tmem_base + ((uint32_t)(g4 * 32) << 16);
        int it = 0;
        for (int64_t t = blockIdx.x; t < sh.tiles; t += gridDim.x, ++it) {
            if (!warp_wait(&ctl->tfull[0], (uint32_t)it & 1u, &ctl->abort)) break;
            tc_fence_after();
            int b, rt, ct;
            tile_coords(sh, t, b, rt, ct);
            const int az = three_d ? (b / sh.am.div) % sh.am.mod : 0;
            const int bz = three_d ? (b / sh.bm.div) % sh.bm.mod : 0;
            const int64_t r = (int64_t)rt * kBM + g4 * 32 + lane;
            const float sa = r < sh.a_rows ? sh.a_scale[(int64_t)az * sh.a_rows + r] : 0.0f;
            // value = sa sb (acc1 + 2^-7 (acc2 + acc3) + 2^-14 acc4) as the float-float pair
            // hi = sa sb acc1 (an integer times powers of two: exact), lo = sa sb (the rest);
            // the row and column scales are powers of two, so both products are exact
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                uint32_t a1[32], a2[32];
                float vh[32], vl[32];
                tmem_ld32_nw(tb + 128 + c * 32, a1);   // acc2
                tmem_ld32_nw(tb + 256 + c * 32, a2);   // acc3
                tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 32; ++q) vl[q] = __uint_as_float(a1[q]) + __uint_as_float(a2[q]);
                tmem_ld32_nw(tb + c * 32, a1);         // acc1
                tmem_ld32_nw(tb + 384 + c * 32, a2);   // acc4
                tmem_ld_wait();
                const int64_t c0 = (int64_t)ct * 128 + c * 32;
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int64_t col = c0 + q;
                    const float sc = col < sh.b_rows ? sa * sh.b_scale[(int64_t)bz * sh.b_rows + col] : 0.0f;
                    vl[q] = fmaf((float)kS3, vl[q], (float)(kS3 * kS3) * __uint_as_float(a2[q])) * sc;
                    vh[q] = __uint_as_float(a1[q]) * sc;
                }
                epilogue_row3(epi, b, r, c0, vh, vl);
            }
            tc_fence_before();
            mbar_arrive(&ctl->tempty[0]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(ctl->tmem_base, 512);
    }
    if (threadIdx.x == 0 && ctl->abort) atomicOr(flags, FLAG_TIMEOUT);
}

// Row scale 2^(e-11) from a float sum of squares, raised by 2^-10 so ||x||_2 < 2^e holds.
__device__ __forceinline__ void row_scale(float ss, float& inv, float& sc) {
    const float nrm = sqrtf(ss) * (1.0f + 0x1p-10f);
    int e = 0;
    if (nrm > 0.f) frexpf(nrm, &e);
    inv = nrm > 0.f ? ldexpf(1.0f, 11 - e) : 0.f;
    sc = nrm > 0.f ? ldexpf(1.0f, e - 11) : 1.0f;
}

// Three slices of FP64 rows (same slicing as split3_rows_ff_kernel).  One warp per row: pass 1
// finds the row's largest exponent and its sum of squares relative to it (fp32, rescaled as
// the maximum grows, then merged across lanes), which fixes the row scale 2^(e-11) with
// ||x||_2 < 2^e; pass 2 forms y = x 2^(11-e) as a float pair and slices it.
__global__ void __launch_bounds__(256) split3_rows_kernel(const double* src, int64_t rows, int64_t K, __half* h,
                                                          __half* m, __half* l, float* scale) {
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const double* x = src + r * K;
    int emax = 0;          // largest biased exponent met (0: none)
    float ss = 0.f;        // sum of squares in units of 2^(2 (emax - 1023))
    bool bad = false;
    for (int64_t k = lane; k < K; k += 32) {
        const uint32_t bh = (uint32_t)((unsigned long long)__double_as_longlong(x[k]) >> 32);
        const int E = (int)((bh >> 20) & 0x7ffu);
        if (E == 0x7ff) bad = true;
        if (E == 0 || E == 0x7ff) continue;
        if (E > emax) {
            const int d = 2 * (emax - E);   // rescale the sum to the new maximum
            ss = (emax == 0 || d < -126) ? 0.f : ss * __uint_as_float((uint32_t)(d + 127) << 23);
            emax = E;
        }
        const int d = E - emax;             // <= 0
        const float v = d < -60 ? 0.f : __uint_as_float(0x3f800000u | ((bh & 0xfffffu) << 3)) *
                                            __uint_as_float((uint32_t)(d + 127) << 23);
        ss = fmaf(v, v, ss);
    }
    int wmax = emax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    {
        const int d = 2 * (emax - wmax);
        ss = (emax == 0 || d < -126) ? 0.f : ss * __uint_as_float((uint32_t)(d + 127) << 23);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    bad = __any_sync(0xffffffffu, bad);
    // ||x|| < 2^(en) 2^(wmax - 1023); the 2^-10 margin covers the truncated mantissas and the
    // fp32 sum
    int kexp = 0;
    float sc = 1.0f;
    if (wmax > 0 && ss > 0.f) {
        int en = 0;
        frexpf(sqrtf(ss) * (1.0f + 0x1p-10f), &en);
        const int e = en + wmax - 1023;
        kexp = 11 - e;
        sc = ldexpf(1.0f, e - 11);
    }
    if (bad) sc = __int_as_float(0x7fc00000);
    if (lane == 0) scale[r] = sc;
    const bool zero = !(wmax > 0 && ss > 0.f);
    for (int64_t k = lane; k < K; k += 32) {
        float yh = 0.f, yl = 0.f;
        if (!zero) dbl_scaled_ff(x[k], kexp, yh, yl);
        if (bad) yh = __int_as_float(0x7fc00000);
        slice3(yh, yl, h[r * K + k], m[r * K + k], l[r * K + k]);
    }
}

__global__ void __launch_bounds__(256) split3_rows_ff_kernel(const float* xh, const float* xl, int64_t rows, int64_t K,
                                                             __half* h, __half* m, __half* l, float* scale) {
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const float* a = xh + r * K;
    const float* b = xl + r * K;
    float ss = 0.f;
    for (int64_t k = lane; k < K; k += 32) ss = fmaf(a[k], a[k], ss);
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    float inv, sc;
    row_scale(ss, inv, sc);
    if (lane == 0) scale[r] = sc;
    for (int64_t k = lane; k < K; k += 32) slice3(a[k] * inv, b[k] * inv, h[r * K + k], m[r * K + k], l[r * K + k]);
}

// Float-float helpers: exact product error and sum error (FMA-based).
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
    ph = ah * bh;
    pl = fmaf(ah, bh, -ph) + (ah * bl + al * bh);
}
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl, float& sh, float& sl) {
    sh = ah + bh;
    const float v = sh - ah;
    sl = ((ah - (sh - v)) + (bh - v)) + (al + bl);
}

// One warp per (ws, j): P = i s C (or P = Pacc when C is null), Pacc += P, doubled three-slice
// split of P when `split`.
__global__ void __launch_bounds__(256) taylor_step_ff_kernel(const float* Ch, const float* Cl, float s_hi, float s_lo,
                                                             float* Ph, float* Pl, int64_t WS, int N, int M, int split,
                                                             __half* h, __half* m, __half* l, float* scale) {
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);   // (ws, j)
    const int lane = threadIdx.x & 31;
    if (r >= WS * N) return;
    const int64_t ws = r / N;
    const int j = (int)(r % N);
    const int64_t row0 = ws * 2 * N + j, row1 = row0 + N;   // re, im rows
    float ss = 0.f;
    // pass 1: P, Pacc update, row norm (P is recomputed in pass 2: M values do not fit registers)
    for (int k = lane; k < M; k += 32) {
        float prh, prl, pih, pil;
        if (Ch) {
            ff_mul(-Ch[row1 * M + k], -Cl[row1 * M + k], s_hi, s_lo, prh, prl);   // Re P = -s Im C
            ff_mul(Ch[row0 * M + k], Cl[row0 * M + k], s_hi, s_lo, pih, pil);     // Im P =  s Re C
            float ah, al;
            ff_add(Ph[row0 * M + k], Pl[row0 * M + k], prh, prl, ah, al);
            Ph[row0 * M + k] = ah;
            Pl[row0 * M + k] = al;
            ff_add(Ph[row1 * M + k], Pl[row1 * M + k], pih, pil, ah, al);
            Ph[row1 * M + k] = ah;
            Pl[row1 * M + k] = al;
        } else {
            prh = Ph[row0 * M + k];
            pih = Ph[row1 * M + k];
        }
        ss = fmaf(prh, prh, fmaf(pih, pih, ss));
    }
    if (!split) return;
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    float inv, sc;
    row_scale(ss, inv, sc);
    if (lane == 0) { scale[row0] = sc; scale[row1] = sc; }
    const int64_t K2 = 2LL * M;
    for (int k = lane; k < M; k += 32) {
        float prh, prl, pih, pil;
        if (Ch) {
            ff_mul(-Ch[row1 * M + k], -Cl[row1 * M + k], s_hi, s_lo, prh, prl);
            ff_mul(Ch[row0 * M + k], Cl[row0 * M + k], s_hi, s_lo, pih, pil);
        } else {
            prh = Ph[row0 * M + k]; prl = Pl[row0 * M + k];
            pih = Ph[row1 * M + k]; pil = Pl[row1 * M + k];
        }
        __half Hr, Mr, Lr, Hi, Mi, Li;
        slice3(prh * inv, prl * inv, Hr, Mr, Lr);
        slice3(pih * inv, pil * inv, Hi, Mi, Li);
        h[row0 * K2 + k] = Hr;  m[row0 * K2 + k] = Mr;  l[row0 * K2 + k] = Lr;                     // Re
        h[row0 * K2 + M + k] = __hneg(Hi);  m[row0 * K2 + M + k] = __hneg(Mi);  l[row0 * K2 + M + k] = __hneg(Li);
        h[row1 * K2 + k] = Hi;  m[row1 * K2 + k] = Mi;  l[row1 * K2 + k] = Li;                     // Im
        h[row1 * K2 + M + k] = Hr;  m[row1 * K2 + M + k] = Mr;  l[row1 * K2 + M + k] = Lr;          // Re
    }
}

// --------------------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2-D or 3-D map over [batch][rows][K] bf16 with box {64, box_rows, 1} and 128-byte swizzle.
int make_map(CUtensorMap* m, const bf16* base, int64_t K, int64_t rows, int64_t batch, int64_t row_stride,
             int64_t batch_stride, int box_rows, bool three_d, bool fp16 = false, int swizzle = 128) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return fail(AFQMC_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (row_stride * 2) % 16 || (batch_stride * 2) % 16)
        return fail(AFQMC_ERR_SHAPE, "tensor map: base/stride not 16-byte aligned");
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)std::max<int64_t>(batch, 1)};
    cuuint64_t strides[2] = {(cuuint64_t)(row_stride * 2), (cuuint64_t)(std::max<int64_t>(batch_stride, row_stride) * 2)};
    cuuint32_t box[3] = {(cuuint32_t)(swizzle / 2), (cuuint32_t)box_rows, 1};   // one swizzle row of 16-bit values
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, three_d ? 3 : 2, const_cast<bf16*>(base), dims, strides,
                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swizzle == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                  : (swizzle == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B),
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(AFQMC_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return AFQMC_OK;
}

template <int BN>
size_t gemm_smem() {
    return 1024 + (size_t)Cfg<BN>::kStages * Cfg<BN>::kStageBytes + sizeof(SharedCtl);
}

template <int BK, int AP, int BR>
size_t energy_smem() {
    using C = EStage<BK, AP, BR>;
    return 1024 + (size_t)C::kStages * C::kStageBytes + (size_t)kETileFloats * 4 + 256 * 4 + 256 * 8 +
           sizeof(SharedCtl);
}

int g_num_sms = 0;

template <int BN, bool EXACT>
int launch_gemm(const CUtensorMap* m, const TileShape& sh, const EpiParams& epi, unsigned* flags, cudaStream_t st) {
    const size_t sm = gemm_smem<BN>();
    raise_dyn_smem(tc_gemm_kernel<BN, EXACT>, sm);
    const int cap = launch_policy().grid_cap > 0 ? std::min(launch_policy().grid_cap, tc_num_sms()) : tc_num_sms();
    const int grid = (int)std::min<int64_t>(sh.tiles, cap);
    count_launch();
    tc_gemm_kernel<BN, EXACT><<<grid, kGemmThreads, sm, st>>>(m[0], m[1], m[2], m[3], sh, epi, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AFQMC_ERR_CUDA, std::string("tc_gemm launch: ") + cudaGetErrorString(e));
    return AFQMC_OK;
}

template <int Np, int BK, int AP>
int launch_energy(const CUtensorMap* m, const EnergyShape& es, unsigned* flags, cudaStream_t st) {
    const size_t sm = energy_smem<BK, AP, 256>();
    raise_dyn_smem(tc_energy_kernel<Np, BK, AP>, sm);
    const int cap = launch_policy().grid_cap > 0 ? std::min(launch_policy().grid_cap, tc_num_sms()) : tc_num_sms();
    const int grid = (int)std::min<int64_t>(es.tiles, cap);
    count_launch();
    tc_energy_kernel<Np, BK, AP><<<grid, kEThreads, sm, st>>>(m[0], m[1], m[2], m[3], m[4], es, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AFQMC_ERR_CUDA, std::string("tc_energy launch: ") + cudaGetErrorString(e));
    return AFQMC_OK;
}

}  // namespace

template <int Np, int BK, int AP>
int launch_energy_pair(const CUtensorMap* m, const EnergyShape& es, unsigned* flags, cudaStream_t st) {
    auto kern = tc_energy_pair_kernel<Np, BK, AP>;
    const size_t sm = energy_smem<BK, AP, 128>();
    raise_dyn_smem(kern, sm);
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kEThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)(2 * (tc_num_sms() / 2)));
    int pairs = 0;   // CTA pairs that fit on the GPU at once (one CTA per SM)
    if (cudaOccupancyMaxActiveClusters(&pairs, kern, &cfg) != cudaSuccess || pairs < 1) {
        cudaGetLastError();
        pairs = tc_num_sms() / 2;
    }
    if (launch_policy().grid_cap > 0) pairs = std::max(1, std::min(pairs, launch_policy().grid_cap / 2));
    cfg.gridDim = dim3((unsigned)(2 * std::min<int64_t>(es.tiles2, pairs)));
    count_launch();
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, m[0], m[1], m[2], m[3], m[4], m[5], es, flags);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AFQMC_ERR_CUDA, std::string("tc_energy (CTA pairs) launch: ") + cudaGetErrorString(e));
    return AFQMC_OK;
}

int tc_num_sms() {
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

int tc_gemm(const SplitMat& A, BatchMap amap, const SplitMat& B, BatchMap bmap, int64_t rows, int64_t cols,
            int64_t K, int nbatch, const EpiParams& epi, int BN, bool exact, unsigned* flags, cudaStream_t st) {
    if (rows <= 0 || cols <= 0 || K <= 0 || nbatch <= 0) return AFQMC_OK;
    if (BN != 128 && BN != 256) return fail(AFQMC_ERR_BADARG, "tc_gemm: BN must be 128 or 256");
    if (!exact && BN == 256 && launch_policy().bn_max < 256) BN = 128;   // epilogues are per 32 columns
    if (exact && (BN != 128 || !A.scale || !B.scale))
        return fail(AFQMC_ERR_BADARG, "tc_gemm: exact mode needs BN = 128 and row-scaled operands");
    const bool three_d = nbatch > 1 || amap.mod != (1 << 30);
    CUtensorMap m[4];
    AFQMC_TRY(make_map(&m[0], A.hi, A.K, A.rows, A.batch, A.row_stride, A.batch_stride, kBM, three_d, exact));
    AFQMC_TRY(make_map(&m[1], A.lo, A.K, A.rows, A.batch, A.row_stride, A.batch_stride, kBM, three_d, exact));
    AFQMC_TRY(make_map(&m[2], B.hi, B.K, B.rows, B.batch, B.row_stride, B.batch_stride, BN, three_d, exact));
    AFQMC_TRY(make_map(&m[3], B.lo, B.K, B.rows, B.batch, B.row_stride, B.batch_stride, BN, three_d, exact));
    TileShape sh;
    sh.rows = rows;
    sh.cols = cols;
    sh.K = K;
    sh.nbatch = nbatch;
    sh.rt = (int)((rows + kBM - 1) / kBM);
    sh.ct = (int)((cols + BN - 1) / BN);
    sh.nk = (int)((K + kBK - 1) / kBK);
    sh.tiles = (int64_t)sh.rt * sh.ct * nbatch;
    sh.am = three_d ? amap : BatchMap{1, 1 << 30};
    sh.bm = three_d ? bmap : BatchMap{1, 1 << 30};
    sh.a_scale = A.scale;
    sh.b_scale = B.scale;
    sh.a_rows = A.rows;
    sh.b_rows = B.rows;
    if (exact) return launch_gemm<128, true>(m, sh, epi, flags, st);
    if (BN == 256) return launch_gemm<256, false>(m, sh, epi, flags, st);
    return launch_gemm<128, false>(m, sh, epi, flags, st);
}

namespace {

// Validation, tensor maps and shape of one energy contraction (brows: Theta rows per TMA box,
// 256 for one CTA per tile, 128 for CTA pairs).
int energy_setup(const SplitMat& Lt, const SplitMat& ThetaT, int Np, int Nchol, int nws, int M, cplx* t_out,
                 cplx* X_out, int terms, const uint8_t* lolo_group, const bf16* Lt_round, int BK, int brows,
                 CUtensorMap* m, EnergyShape& es, const uint8_t* single_group, const bf16* ThetaT_round) {
    if (terms != kEnergyThree && terms != kEnergyFour && terms != kEnergyRounded)
        return fail(AFQMC_ERR_BADARG, "tc_energy: terms must be 3, 4 or the rounded three");
    if (terms == kEnergyRounded && !Lt_round)
        return fail(AFQMC_ERR_BADARG, "tc_energy: rounded products need the rounded Ltilde plane");
    if (single_group && (terms != kEnergyRounded || !ThetaT_round))
        return fail(AFQMC_ERR_BADARG, "tc_energy: single-product tiles need the rounded products and Theta plane");
    if (Np < 8 || Np > 128 || Np % 8) return fail(AFQMC_ERR_UNSUPPORTED, "tc_energy: Np must be a multiple of 8 up to 128");
    if (M % kBK || M > 1024) return fail(AFQMC_ERR_UNSUPPORTED, "tc_energy: M must be a multiple of 64, <= 1024");
    if (!Lt.scale || !ThetaT.scale) return fail(AFQMC_ERR_BADARG, "tc_energy: row-scaled operands required");
    const bool rounded = terms == kEnergyRounded;
    const int swz = 2 * BK;   // bytes per swizzled row of the K chunk
    AFQMC_TRY(make_map(&m[0], Lt.hi, M, (int64_t)Nchol * Np, 1, Lt.row_stride, 0, 128, false, true, swz));
    AFQMC_TRY(make_map(&m[1], Lt.lo, M, (int64_t)Nchol * Np, 1, Lt.row_stride, 0, 128, false, true, swz));
    AFQMC_TRY(make_map(&m[2], rounded ? Lt_round : Lt.hi, M, (int64_t)Nchol * Np, 1, Lt.row_stride, 0, 128, false,
                       true, swz));
    AFQMC_TRY(make_map(&m[3], ThetaT.hi, M, (int64_t)nws * 2 * Np, 1, ThetaT.row_stride, 0, brows, false, true, swz));
    AFQMC_TRY(make_map(&m[4], ThetaT.lo, M, (int64_t)nws * 2 * Np, 1, ThetaT.row_stride, 0, brows, false, true, swz));
    AFQMC_TRY(make_map(&m[5], single_group ? ThetaT_round : ThetaT.hi, M, (int64_t)nws * 2 * Np, 1, ThetaT.row_stride,
                       0, brows, false, true, swz));
    es = EnergyShape{};
    es.Np = Np;
    es.Q = Np / 32;
    es.G = 128 / Np;
    es.np_inv = (65536u + (uint32_t)Np - 1) / (uint32_t)Np;
    es.g_inv = (65536u + (uint32_t)es.G - 1) / (uint32_t)es.G;
    es.Nchol = Nchol;
    es.nws = nws;
    es.n_groups = (Nchol + es.G - 1) / es.G;
    es.ws_groups = (nws + es.G - 1) / es.G;
    es.ws_super = std::min(es.ws_groups, launch_policy().energy_ws_super > 0 ? launch_policy().energy_ws_super
                                                                                : kEWsSuperDefault);
    es.tiles = (int64_t)es.n_groups * es.ws_groups;
    es.n_pairs = (es.n_groups + 1) / 2;
    es.tiles2 = (int64_t)es.n_pairs * es.ws_groups;
    es.nk = M / BK;
    es.lolo = terms == kEnergyFour ? 1 : 0;
    es.lolo_group = rounded ? nullptr : lolo_group;
    es.single_group = single_group;
    es.a_scale = Lt.scale;
    es.b_scale = ThetaT.scale;
    es.t_out = t_out;
    es.X_out = X_out;
    return AFQMC_OK;
}

template <int BK, int AP>
int launch_energy_multi(const EnergySys* sys, const EnergyWork* work, int64_t nwork, unsigned* flags,
                        cudaStream_t st) {
    auto kern = tc_energy_multi_kernel<BK, AP>;
    const size_t sm = energy_smem<BK, AP, 128>();
    raise_dyn_smem(kern, sm);
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kEThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)(2 * (tc_num_sms() / 2)));
    int pairs = 0;
    if (cudaOccupancyMaxActiveClusters(&pairs, kern, &cfg) != cudaSuccess || pairs < 1) {
        cudaGetLastError();
        pairs = tc_num_sms() / 2;
    }
    if (launch_policy().grid_cap > 0) pairs = std::max(1, std::min(pairs, launch_policy().grid_cap / 2));
    cfg.gridDim = dim3((unsigned)(2 * std::min<int64_t>(nwork, pairs)));
    count_launch();
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, sys, work, nwork, flags);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AFQMC_ERR_CUDA, std::string("tc_energy_multi launch: ") + cudaGetErrorString(e));
    return AFQMC_OK;
}

}  // namespace

int tc_energy(const SplitMat& Lt, const SplitMat& ThetaT, int Np, int Nchol, int nws, int M, cplx* t_out,
              cplx* X_out, int terms, const uint8_t* lolo_group, const bf16* Lt_round, unsigned* flags,
              cudaStream_t st, const uint8_t* single_group, const bf16* ThetaT_round) {
    const int BK = launch_policy().energy_bk != 0 ? launch_policy().energy_bk : kEBKDefault;
    const bool pair = launch_policy().energy_pair != 0;
    const bool rounded = terms == kEnergyRounded;
    CUtensorMap m[6];
    EnergyShape es;
    // the one-CTA form has no single-product tiles: it forms the rounded three products throughout
    AFQMC_TRY(energy_setup(Lt, ThetaT, Np, Nchol, nws, M, t_out, X_out, terms, lolo_group, Lt_round, BK,
                           pair ? 128 : 256, m, es, pair ? single_group : nullptr, ThetaT_round));
#define AFQMC_ENERGY_LAUNCH(NP, BKV, APV) \
    (pair ? launch_energy_pair<NP, BKV, APV>(m, es, flags, st) : launch_energy<NP, BKV, APV>(m, es, flags, st))
#define AFQMC_ENERGY_NP(BKV, APV)                                        \
    switch (Np) {                                                       \
        case 32: return AFQMC_ENERGY_LAUNCH(32, BKV, APV);              \
        case 64: return AFQMC_ENERGY_LAUNCH(64, BKV, APV);              \
        case 128: return AFQMC_ENERGY_LAUNCH(128, BKV, APV);            \
        default: return AFQMC_ENERGY_LAUNCH(0, BKV, APV);               \
    }
    if (BK == 32) {
        if (rounded) AFQMC_ENERGY_NP(32, 3)
        AFQMC_ENERGY_NP(32, 2)
    }
    if (rounded) AFQMC_ENERGY_NP(16, 3)
    AFQMC_ENERGY_NP(16, 2)
#undef AFQMC_ENERGY_NP
#undef AFQMC_ENERGY_LAUNCH
}

int tc_energy_describe(const SplitMat& Lt, const SplitMat& ThetaT, int Np, int Nchol, int nws, int M, cplx* t_out,
                       cplx* X_out, int terms, const uint8_t* lolo_group, const bf16* Lt_round, int BK,
                       EnergySys* out, const uint8_t* single_group, const bf16* ThetaT_round) {
    if (BK != 16 && BK != 32) return fail(AFQMC_ERR_BADARG, "tc_energy_describe: BK must be 16 or 32");
    return energy_setup(Lt, ThetaT, Np, Nchol, nws, M, t_out, X_out, terms, lolo_group, Lt_round, BK, 128, out->map,
                        out->es, single_group, ThetaT_round);
}

void energy_work_list(const EnergySys* sys, int nsys, std::vector<EnergyWork>& out) {
    out.clear();
    for (int s = 0; s < nsys; ++s) {
        const EnergyShape& es = sys[s].es;
        for (int64_t t = 0; t < es.tiles2; ++t) {   // the single-system tile order (L2 windows)
            const int64_t per_super = (int64_t)es.ws_super * es.n_pairs;
            const int64_t sup = t / per_super, rem = t % per_super;
            const int64_t first = sup * es.ws_super;
            const int width = (int)std::min<int64_t>(es.ws_groups - first, es.ws_super);
            out.push_back(EnergyWork{s, (int)(rem / width), (int)(first + rem % width), 0});
        }
    }
}

int tc_energy_multi(const EnergySys* sys, const EnergyWork* work, int64_t nwork, int BK, int terms, unsigned* flags,
                    cudaStream_t st) {
    if (nwork <= 0) return AFQMC_OK;
    const bool rounded = terms == kEnergyRounded;
    if (BK == 32) return rounded ? launch_energy_multi<32, 3>(sys, work, nwork, flags, st)
                                 : launch_energy_multi<32, 2>(sys, work, nwork, flags, st);
    return rounded ? launch_energy_multi<16, 3>(sys, work, nwork, flags, st)
                   : launch_energy_multi<16, 2>(sys, work, nwork, flags, st);
}

void select_single_groups(const double* nrm2, int nch, int G, double eta, uint8_t* flags) {
    // the complement of the four-product choice on the squared norms: a group is single when
    // every one of its vectors lies in the tail
    select_lolo_groups(nrm2, nch, G, eta, flags);
    for (int g = 0; g < (nch + G - 1) / G; ++g) flags[g] = flags[g] ? 0 : 1;
}

void select_lolo_groups(const double* nrm, int nch, int G, double eta, uint8_t* flags) {
    std::vector<int> order((size_t)nch);
    for (int n = 0; n < nch; ++n) order[(size_t)n] = n;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nrm[a] < nrm[b]; });
    double total = 0.0;
    for (int n = 0; n < nch; ++n) total += nrm[n];
    std::vector<uint8_t> three((size_t)nch, 0);
    double acc = 0.0;
    for (int n : order) {
        if (acc + nrm[n] > eta * total) break;
        acc += nrm[n];
        three[(size_t)n] = 1;
    }
    const int ng = (nch + G - 1) / G;
    for (int g = 0; g < ng; ++g) {
        uint8_t four = 0;
        for (int n = g * G; n < std::min(nch, (g + 1) * G); ++n) four |= three[(size_t)n] ? 0 : 1;
        flags[g] = four;
    }
}

void split3_rows(const double* src, int64_t rows, int64_t K, bf16* h, bf16* m, bf16* l, float* scale,
                 cudaStream_t st) {
    if (rows <= 0) return;
    count_launch();
    split3_rows_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(src, rows, K, reinterpret_cast<__half*>(h),
                                                                   reinterpret_cast<__half*>(m),
                                                                   reinterpret_cast<__half*>(l), scale);
}

int tc_gemm3(const Split3& A, BatchMap amap, const Split3& B, BatchMap bmap, int64_t rows, int64_t cols, int64_t K,
             int nbatch, const EpiParams& epi, unsigned* flags, cudaStream_t st) {
    if (rows <= 0 || cols <= 0 || K <= 0 || nbatch <= 0) return AFQMC_OK;
    if (!A.scale || !B.scale) return fail(AFQMC_ERR_BADARG, "tc_gemm3: row scales required");
    const bool three_d = nbatch > 1 || amap.mod != (1 << 30);
    CUtensorMap m[6];
    for (int q = 0; q < 3; ++q) {
        AFQMC_TRY(make_map(&m[q], A.p[q], A.K, A.rows, A.batch, A.K, A.batch_stride, kBM, three_d, true));
        AFQMC_TRY(make_map(&m[3 + q], B.p[q], B.K, B.rows, B.batch, B.K, B.batch_stride, 128, three_d, true));
    }
    TileShape sh;
    sh.rows = rows;
    sh.cols = cols;
    sh.K = K;
    sh.nbatch = nbatch;
    sh.rt = (int)((rows + kBM - 1) / kBM);
    sh.ct = (int)((cols + 127) / 128);
    sh.nk = (int)((K + kBK - 1) / kBK);
    sh.tiles = (int64_t)sh.rt * sh.ct * nbatch;
    // unbatched: 2-D maps and batch coordinate 0 (the kernel tests the same condition)
    sh.am = three_d ? amap : BatchMap{1, 1 << 30};
    sh.bm = three_d ? bmap : BatchMap{1, 1 << 30};
    sh.a_scale = A.scale;
    sh.b_scale = B.scale;
    sh.a_rows = A.rows;
    sh.b_rows = B.rows;
    const size_t smem = 1024 + (size_t)kG3Stages * kG3StageBytes + sizeof(SharedCtl);
    raise_dyn_smem(tc_gemm3_kernel, smem);
    const int cap = launch_policy().grid_cap > 0 ? std::min(launch_policy().grid_cap, tc_num_sms()) : tc_num_sms();
    const int grid = (int)std::min<int64_t>(sh.tiles, cap);
    count_launch();
    tc_gemm3_kernel<<<grid, kGemmThreads, smem, st>>>(m[0], m[1], m[2], m[3], m[4], m[5], sh, epi, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AFQMC_ERR_CUDA, std::string("tc_gemm3 launch: ") + cudaGetErrorString(e));
    return AFQMC_OK;
}

int tc_overlap3(const bf16* const* a, const float* a_scale, int nws, int rows, const bf16* const* b,
                const float* b_scale, int N, int M, double* out, unsigned* flags, cudaStream_t st) {
    if (N > 128 || M % 8 || rows <= 0 || nws <= 0)
        return fail(AFQMC_ERR_UNSUPPORTED, "tc_overlap3: needs N <= 128, M % 8 == 0");
    Split3 A, B;
    for (int q = 0; q < 3; ++q) {
        A.p[q] = a[q];
        B.p[q] = b[q];
    }
    A.scale = a_scale;
    A.K = M;
    A.rows = rows;
    A.batch = nws;
    A.batch_stride = (int64_t)rows * M;
    B.scale = b_scale;
    B.K = M;
    B.rows = N;
    B.batch = 1;
    EpiParams e;
    e.kind = EPI3_F64;
    e.rows_valid = rows;
    e.cols_valid = N;
    e.ld = N;
    e.ob = (int64_t)rows * N;
    e.out_f64 = out;
    return tc_gemm3(A, BatchMap{1, nws}, B, BatchMap{1, 1}, rows, N, M, nws, e, flags, st);
}

void split3_rows_ff(const float* hi, const float* lo, int64_t rows, int64_t K, bf16* h, bf16* m, bf16* l,
                    float* scale, cudaStream_t st) {
    if (rows <= 0) return;
    count_launch();
    split3_rows_ff_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(
        hi, lo, rows, K, reinterpret_cast<__half*>(h), reinterpret_cast<__half*>(m), reinterpret_cast<__half*>(l),
        scale);
}

// The same Taylor step for M = 128 NG: lane t handles the four consecutive orbitals
// k = 4 t + 128 i (i < NG) of both rows, kept in registers from the norm pass to the split, with
// 16-byte loads and 8-byte stores of four fp16 slices.
__device__ __forceinline__ void st4h(__half* p, __half a, __half b, __half c, __half d) {
    uint2 u;
    u.x = (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
    u.y = (uint32_t)__half_as_ushort(c) | ((uint32_t)__half_as_ushort(d) << 16);
    *reinterpret_cast<uint2*>(p) = u;
}
template <int NG>
__global__ void __launch_bounds__(256) taylor_step_ff_v4_kernel(const float* Ch, const float* Cl, float s_hi,
                                                                float s_lo, float* Ph, float* Pl, int64_t WS, int N,
                                                                int split, __half* h, __half* m, __half* l,
                                                                float* scale) {
    constexpr int M = 128 * NG;
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);   // (ws, j)
    const int lane = threadIdx.x & 31;
    if (r >= WS * N) return;
    const int64_t ws = r / N;
    const int j = (int)(r % N);
    const int64_t row0 = ws * 2 * N + j, row1 = row0 + N;   // re, im rows
    float rh[NG][4], rl[NG][4], ih[NG][4], il[NG][4];       // this step's term P (re, im)
    float ss = 0.f;
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        const int k = 4 * lane + 128 * i;
        if (Ch) {
            const float4 c0h = *reinterpret_cast<const float4*>(Ch + row0 * M + k);
            const float4 c0l = *reinterpret_cast<const float4*>(Cl + row0 * M + k);
            const float4 c1h = *reinterpret_cast<const float4*>(Ch + row1 * M + k);
            const float4 c1l = *reinterpret_cast<const float4*>(Cl + row1 * M + k);
            const float a0h[4] = {c0h.x, c0h.y, c0h.z, c0h.w}, a0l[4] = {c0l.x, c0l.y, c0l.z, c0l.w};
            const float a1h[4] = {c1h.x, c1h.y, c1h.z, c1h.w}, a1l[4] = {c1l.x, c1l.y, c1l.z, c1l.w};
            float4 p0h = *reinterpret_cast<const float4*>(Ph + row0 * M + k);
            float4 p0l = *reinterpret_cast<const float4*>(Pl + row0 * M + k);
            float4 p1h = *reinterpret_cast<const float4*>(Ph + row1 * M + k);
            float4 p1l = *reinterpret_cast<const float4*>(Pl + row1 * M + k);
            float s0h[4] = {p0h.x, p0h.y, p0h.z, p0h.w}, s0l[4] = {p0l.x, p0l.y, p0l.z, p0l.w};
            float s1h[4] = {p1h.x, p1h.y, p1h.z, p1h.w}, s1l[4] = {p1l.x, p1l.y, p1l.z, p1l.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                ff_mul(-a1h[u], -a1l[u], s_hi, s_lo, rh[i][u], rl[i][u]);   // Re P = -s Im C
                ff_mul(a0h[u], a0l[u], s_hi, s_lo, ih[i][u], il[i][u]);     // Im P =  s Re C
                ff_add(s0h[u], s0l[u], rh[i][u], rl[i][u], s0h[u], s0l[u]);
                ff_add(s1h[u], s1l[u], ih[i][u], il[i][u], s1h[u], s1l[u]);
                ss = fmaf(rh[i][u], rh[i][u], fmaf(ih[i][u], ih[i][u], ss));
            }
            *reinterpret_cast<float4*>(Ph + row0 * M + k) = make_float4(s0h[0], s0h[1], s0h[2], s0h[3]);
            *reinterpret_cast<float4*>(Pl + row0 * M + k) = make_float4(s0l[0], s0l[1], s0l[2], s0l[3]);
            *reinterpret_cast<float4*>(Ph + row1 * M + k) = make_float4(s1h[0], s1h[1], s1h[2], s1h[3]);
            *reinterpret_cast<float4*>(Pl + row1 * M + k) = make_float4(s1l[0], s1l[1], s1l[2], s1l[3]);
        } else {
            const float4 p0h = *reinterpret_cast<const float4*>(Ph + row0 * M + k);
            const float4 p0l = *reinterpret_cast<const float4*>(Pl + row0 * M + k);
            const float4 p1h = *reinterpret_cast<const float4*>(Ph + row1 * M + k);
            const float4 p1l = *reinterpret_cast<const float4*>(Pl + row1 * M + k);
            rh[i][0] = p0h.x; rh[i][1] = p0h.y; rh[i][2] = p0h.z; rh[i][3] = p0h.w;
            rl[i][0] = p0l.x; rl[i][1] = p0l.y; rl[i][2] = p0l.z; rl[i][3] = p0l.w;
            ih[i][0] = p1h.x; ih[i][1] = p1h.y; ih[i][2] = p1h.z; ih[i][3] = p1h.w;
            il[i][0] = p1l.x; il[i][1] = p1l.y; il[i][2] = p1l.z; il[i][3] = p1l.w;
#pragma unroll
            for (int u = 0; u < 4; ++u) ss = fmaf(rh[i][u], rh[i][u], fmaf(ih[i][u], ih[i][u], ss));
        }
    }
    if (!split) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    float inv, sc;
    row_scale(ss, inv, sc);
    if (lane == 0) { scale[row0] = sc; scale[row1] = sc; }
    constexpr int K2 = 2 * M;
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        const int k = 4 * lane + 128 * i;
        __half Hr[4], Mr[4], Lr[4], Hi[4], Mi[4], Li[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            slice3(rh[i][u] * inv, rl[i][u] * inv, Hr[u], Mr[u], Lr[u]);
            slice3(ih[i][u] * inv, il[i][u] * inv, Hi[u], Mi[u], Li[u]);
        }
        // doubled rows: row0 = [Re | -Im], row1 = [Im | Re]
        st4h(h + row0 * K2 + k, Hr[0], Hr[1], Hr[2], Hr[3]);
        st4h(m + row0 * K2 + k, Mr[0], Mr[1], Mr[2], Mr[3]);
        st4h(l + row0 * K2 + k, Lr[0], Lr[1], Lr[2], Lr[3]);
        st4h(h + row0 * K2 + M + k, __hneg(Hi[0]), __hneg(Hi[1]), __hneg(Hi[2]), __hneg(Hi[3]));
        st4h(m + row0 * K2 + M + k, __hneg(Mi[0]), __hneg(Mi[1]), __hneg(Mi[2]), __hneg(Mi[3]));
        st4h(l + row0 * K2 + M + k, __hneg(Li[0]), __hneg(Li[1]), __hneg(Li[2]), __hneg(Li[3]));
        st4h(h + row1 * K2 + k, Hi[0], Hi[1], Hi[2], Hi[3]);
        st4h(m + row1 * K2 + k, Mi[0], Mi[1], Mi[2], Mi[3]);
        st4h(l + row1 * K2 + k, Li[0], Li[1], Li[2], Li[3]);
        st4h(h + row1 * K2 + M + k, Hr[0], Hr[1], Hr[2], Hr[3]);
        st4h(m + row1 * K2 + M + k, Mr[0], Mr[1], Mr[2], Mr[3]);
        st4h(l + row1 * K2 + M + k, Lr[0], Lr[1], Lr[2], Lr[3]);
    }
}

void taylor_step_ff(const float* Ch, const float* Cl, float s_hi, float s_lo, float* Ph, float* Pl, int64_t WS,
                    int N, int M, bool split, bf16* h, bf16* m, bf16* l, float* scale, cudaStream_t st) {
    if (WS * N <= 0) return;
    count_launch();
    const unsigned grid = (unsigned)((WS * N + 7) / 8);
    auto v4 = [&](auto kern) {
        kern<<<grid, 256, 0, st>>>(Ch, Cl, s_hi, s_lo, Ph, Pl, WS, N, split ? 1 : 0, reinterpret_cast<__half*>(h),
                                   reinterpret_cast<__half*>(m), reinterpret_cast<__half*>(l), scale);
    };
    switch (M) {   // the register form for M = 128, 256, 384, 512
        case 128: v4(taylor_step_ff_v4_kernel<1>); return;
        case 256: v4(taylor_step_ff_v4_kernel<2>); return;
        case 384: v4(taylor_step_ff_v4_kernel<3>); return;
        case 512: v4(taylor_step_ff_v4_kernel<4>); return;
        default: break;
    }
    taylor_step_ff_kernel<<<(unsigned)((WS * N + 7) / 8), 256, 0, st>>>(
        Ch, Cl, s_hi, s_lo, Ph, Pl, WS, N, M, split ? 1 : 0, reinterpret_cast<__half*>(h),
        reinterpret_cast<__half*>(m), reinterpret_cast<__half*>(l), scale);
}

void split_rows(const double* src, int64_t src_stride, int64_t rows, int64_t K, bf16* hi, bf16* lo, float* scale,
                cudaStream_t st, bf16* rounded) {
    if (rows <= 0) return;
    count_launch();
    split_rows_kernel<double><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(
        src, src_stride, rows, K, reinterpret_cast<__half*>(hi), reinterpret_cast<__half*>(lo), scale,
        reinterpret_cast<__half*>(rounded));
}

void split_rows(const float* src, int64_t src_stride, int64_t rows, int64_t K, bf16* hi, bf16* lo, float* scale,
                cudaStream_t st, bf16* rounded) {
    if (rows <= 0) return;
    count_launch();
    split_rows_f32_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(
        src, src_stride, rows, K, reinterpret_cast<__half*>(hi), reinterpret_cast<__half*>(lo), scale,
        reinterpret_cast<__half*>(rounded));
}

}  // namespace afqmc
