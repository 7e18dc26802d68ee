// Tensor-core (tcgen05 + TMA) split-precision GEMMs of the mixed-precision walker step.
// Internal to the library.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <vector>

#include "common.cuh"

namespace afqmc {

using bf16 = __nv_bfloat16;

// A K-major 16-bit matrix stored as two planes (hi, lo) of identical layout
// [batch][rows][K] with the given element strides, plus optional per-row scales
// ([batch][rows], contiguous).  Element value = (hi + lo) * scale[row].
//
// Two encodings are used:
//  * plain (bf16):      hi = bf16(x), lo = bf16(x - hi), no scale (scale == nullptr);
//  * row-scaled (fp16): scale = 2^(e - 11) with ||x_row||_2 < 2^e, hi = rint(x / scale) an
//                       integer in [-2048, 2048] (exact in fp16), lo = fp16(x / scale - hi).
// With row-scaled operands on both sides the hi*hi products are integers and, by
// Cauchy-Schwarz, every partial sum stays below 2^23, so their fp32 tensor-memory sums are
// exact whatever rounding the tensor cores apply (they round toward zero); the remainder
// terms hi*lo + lo*hi + lo*lo go to a second accumulator ("exact" GEMMs).  Plain GEMMs put
// hi*hi + hi*lo + lo*hi in one accumulator.  The pointers are typed bf16 for both
// encodings; row-scaled planes hold IEEE fp16 bit patterns.
struct SplitMat {
    const bf16* hi = nullptr;
    const bf16* lo = nullptr;
    const float* scale = nullptr;
    int64_t K = 0, rows = 0, batch = 1;
    int64_t row_stride = 0;    // elements between rows (>= K, multiple of 8)
    int64_t batch_stride = 0;  // elements between batches
};

// Which batch coordinate each operand uses: z = (batch / div) % mod.
struct BatchMap {
    int div = 1;
    int mod = 1 << 30;
};

// Float pair of x * 2^k read from the bits of the double x: hi = its sign, exponent and leading
// 24 significant bits, lo = its remaining 29 bits rounded to float, so hi + lo = x 2^k to
// 2^-47 relative, using integer and fp32 instructions only (GB300's FP64 pipe is ~1/64 of its
// fp32 pipe).  k must keep |x 2^k| below 2^127; results below 2^-100 are flushed to zero and
// inf / NaN give NaN.
__device__ __forceinline__ void dbl_scaled_ff(double x, int k, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
    const int E = (int)((bh >> 20) & 0x7ffu);
    const int ey = E - 1023 + k;
    if (E == 0x7ff) { hi = __int_as_float(0x7fc00000); lo = 0.f; return; }
    if (E == 0 || ey < -100) { hi = 0.f; lo = 0.f; return; }
    const uint32_t sign = bh & 0x80000000u;
    hi = __uint_as_float(sign | ((uint32_t)(ey + 127) << 23) | ((bh & 0xfffffu) << 3) | (bl >> 29));
    const int el = ey - 52;   // weight of the lowest fraction bit
    lo = el < -126 ? 0.f : __uint2float_rn(bl & 0x1fffffffu) * __uint_as_float((uint32_t)(el + 127) << 23);
    if (sign) lo = -lo;
}

// Three slices of a float-float value (yh + yl already divided by the row scale, |y| < 2^11):
// h = rint(yh), r = (yh - h) + yl (|r| <= 0.5 + 2^-13), m = rint(128 r), l = fp16(128 r - m).
__device__ __forceinline__ void slice3(float yh, float yl, __half& h, __half& m, __half& l) {
    const float hv = rintf(yh);
    const float rr = ((yh - hv) + yl) * 128.0f;
    const float mv = rintf(rr);
    h = __float2half_rn(hv);
    m = __float2half_rn(mv);
    l = __float2half_rn(rr - mv);
}

// Output tile epilogues (kind selects the write pattern): EPI_F32 for the two-slice GEMM.
enum EpiKind : int {
    EPI_F32 = 0,       // out_f32[b*ob + r*ld + c]
    // three-slice GEMM (tc_gemm3) epilogues.  Values leave the accumulators as float-float
    // pairs (hi + lo, each exact in its scaling); "FF" outputs keep them as two fp32 planes
    // (out_f32 = hi, out_lo32 = lo), EPI3_F64 adds them in FP64.
    EPI3_F64 = 8,      // out_f64[b*ob + r*ld + c]
    EPI3_FF = 9,       // out_f32 / out_lo32 [b*ob + r*ld + c]
    EPI3_HSPOT_FF = 10,// A potential: row (w, c), col (i, k) -> [w][i][c*M + k] (both planes)
};

struct EpiParams {
    int kind = EPI_F32;
    int64_t rows_valid = 0, cols_valid = 0;  // per batch
    int64_t ld = 0, ob = 0;                  // row / batch strides of the output (elements)
    float* out_f32 = nullptr;
    double* out_f64 = nullptr;
    float* out_lo32 = nullptr;               // low plane of float-float outputs (EPI3_FF*)
    int M = 0;                               // orbitals (EPI3_HSPOT_FF column split)
};

// Three fp16 slices of a matrix [batch][rows][K] (planes h, m, l; see split3_rows) with
// per-row scales [batch][rows]: value = scale (h + 2^-7 (m + l)).
struct Split3 {
    const bf16* p[3] = {nullptr, nullptr, nullptr};
    const float* scale = nullptr;
    int64_t K = 0, rows = 0, batch = 1;
    int64_t batch_stride = 0;   // elements between batches (row stride = K)
};

// C[b] = A[b] . B[b]^T from three-slice operands, ~1e-9 relative, FP64 epilogue (EPI3_*),
// 128 x 128 tiles.  K <= 1024 keeps the integer accumulators exact; larger K only loses
// exactness of the h*m sums (still ~1e-8).
int tc_gemm3(const Split3& A, BatchMap amap, const Split3& B, BatchMap bmap, int64_t rows, int64_t cols, int64_t K,
             int nbatch, const EpiParams& epi, unsigned* flags, cudaStream_t st);
// Three-slice split of float-float rows (hi, lo planes [rows][K]).
void split3_rows_ff(const float* hi, const float* lo, int64_t rows, int64_t K, bf16* h, bf16* m, bf16* l,
                    float* scale, cudaStream_t st);
// One Taylor step on float-float planar data [WS][2][N][M] (hi, lo planes):
// P = i s C with s = s_hi + s_lo; Pacc += P (hi, lo planes); when `split`, P's doubled operand
// row (ws, 0, j) = [Re P_j | -Im P_j], row (ws, 1, j) = [Im P_j | Re P_j] (length 2M) as three
// slices.  With C == nullptr, P is taken from Pacc itself (the first term, s = 1, no update).
void taylor_step_ff(const float* Ch, const float* Cl, float s_hi, float s_lo, float* Ph, float* Pl, int64_t WS,
                    int N, int M, bool split, bf16* h, bf16* m, bf16* l, float* scale, cudaStream_t st);

// C[b] = A[b] . B[b]^T (split bf16, fp32 accumulation in TMEM), 128 x BN tiles.
// exact = true needs row-scaled A and B and BN = 128.
int tc_gemm(const SplitMat& A, BatchMap amap, const SplitMat& B, BatchMap bmap, int64_t rows, int64_t cols,
            int64_t K, int nbatch, const EpiParams& epi, int BN, bool exact, unsigned* flags, cudaStream_t st);

// Shape, operands and outputs of one fused energy contraction (kernels_tc.cu).
struct EnergyShape {
    int Np, Q, G;
    uint32_t np_inv, g_inv;   // ceil(2^16 / Np), ceil(2^16 / G): x / Np = (x np_inv) >> 16 for x < 256
    int Nchol, nws;
    int n_groups, ws_groups;
    int ws_super;     // ws groups per L2 super-block
    int64_t tiles;
    int n_pairs;      // CTA-pair kernel: pairs of n-groups (ceil(n_groups / 2))
    int64_t tiles2;   // CTA-pair kernel: pair tiles (n_pairs x ws_groups)
    int nk;
    int lolo;               // 1: also form lo*lo (four products), 0: three
    const uint8_t* lolo_group;   // if set: per n-group choice (1: four products, 0: three)
    const uint8_t* single_group; // if set (rounded products, CTA-pair kernels): per n-group, 1 = the
                                 // group's tiles form the one product r*r' (r' = fp16 of the scaled
                                 // Theta); a pair tile does so when both of its n-groups are flagged
    const float* a_scale;   // [Nchol*Np]
    const float* b_scale;   // [nws*2*Np]
    cplx* t_out;
    cplx* X_out;
};

// One system of a multi-system energy contraction (device array, 64-byte aligned): tensor maps
// of Ltilde hi, lo, rounded (hi again without rounded products) and Theta^T hi, lo, rounded (hi
// again without single-product tiles) (boxes of 128 Theta rows: the CTA-pair form), and its shape.
struct EnergySys {
    CUtensorMap map[6];
    EnergyShape es;
};
// One pair tile of a multi-system energy contraction: system, n-group pair, walker-spin group.
struct EnergyWork {
    int sys, ngp, wg, pad;
};

// Split products of the fused energy contraction (row-scaled operands: y = x / scale,
// hi = rint(y), lo = fp16(y - hi)):
constexpr int kEnergyThree = 3;     // hi*hi (exact) + hi*lo + lo*hi
constexpr int kEnergyFour = 4;      // hi*hi (exact) + hi*lo + lo*hi + lo*lo
constexpr int kEnergyRounded = 5;   // hi*hi (exact) + r*lo + lo*hi, r = fp16(y) of Ltilde: three
                                    // products, r carrying the leading part of lo*lo

// Fused energy contraction: T_{n,ws} = Lt_n Theta_ws^T (Np x Np complex, Np | 128) for
// all n and walker-spin pairs ws; emits t = Tr T and X = Tr(T T) per (ws, n) into
// t_out/X_out [nws][Nchol] (complex FP64).  Lt: [Nchol*Np][M], ThetaT: [nws*2*Np][M]
// (rows (ws, re/im, b)), both row-scaled; exact accumulation of the leading product.
// terms: kEnergyThree, kEnergyFour or kEnergyRounded (which needs Lt_round, the rounded plane
// r of Lt, same layout).  lolo_group (device, one byte per group of 128/Np Cholesky vectors, or
// null) overrides three/four products per group: 1 four products, 0 three.  single_group
// (device, same indexing, or null; rounded products only, with ThetaT_round the rounded plane
// r' = fp16(y) of ThetaT): the pair tiles whose n-groups are all flagged form the one product
// r*r' instead of three (the one-CTA form ignores it).
int tc_energy(const SplitMat& Lt, const SplitMat& ThetaT, int Np, int Nchol, int nws, int M, cplx* t_out,
              cplx* X_out, int terms, const uint8_t* lolo_group, const bf16* Lt_round, unsigned* flags,
              cudaStream_t st, const uint8_t* single_group = nullptr, const bf16* ThetaT_round = nullptr);

// Fills `out` for one system of a multi-system energy contraction (arguments as tc_energy; BK
// the K chunk every system of the launch uses).
int tc_energy_describe(const SplitMat& Lt, const SplitMat& ThetaT, int Np, int Nchol, int nws, int M, cplx* t_out,
                       cplx* X_out, int terms, const uint8_t* lolo_group, const bf16* Lt_round, int BK,
                       EnergySys* out, const uint8_t* single_group = nullptr, const bf16* ThetaT_round = nullptr);
// The work list of a multi-system energy contraction: every pair tile of every system, each
// system's tiles in its own L2 windows (walker-spin groups x every n-group pair).
void energy_work_list(const EnergySys* sys, int nsys, std::vector<EnergyWork>& out);
// One persistent launch (CTA pairs) over the work list: sys and work in device memory; every
// system described with the same BK and the same product set (terms).  The arithmetic of every
// tile is the single-system contraction's.
int tc_energy_multi(const EnergySys* sys, const EnergyWork* work, int64_t nwork, int BK, int terms, unsigned* flags,
                    cudaStream_t st);

// Cholesky-vector groups whose energy tiles form the lo*lo product (flags[g] = 1): every group
// except those made only of the smallest vectors, by Frobenius norm nrm[n] of Ltilde_n, whose
// norms add up to at most eta of the total.  G vectors per group, ceil(nch / G) flags.
void select_lolo_groups(const double* nrm, int nch, int G, double eta, uint8_t* flags);
// Cholesky-vector groups whose energy tiles form the single product r*r' (flags[g] = 1): the
// groups made only of the smallest vectors, by squared Frobenius norm nrm2[n] of Ltilde_n, whose
// squared norms add up to at most eta of the total.  ceil(nch / G) flags.
void select_single_groups(const double* nrm2, int nch, int G, double eta, uint8_t* flags);

// Three-slice row split (see kernels_tc.cu): h, m, l fp16 planes [rows][K] and row scales.
void split3_rows(const double* src, int64_t rows, int64_t K, bf16* h, bf16* m, bf16* l, float* scale,
                 cudaStream_t st);
// out[ws][r][c] = sum_k A[ws][r][k] B[c][k] (FP64 out, ~1e-9 relative) from three-slice operands:
// a[3] planes [nws][rows][M] with scales [nws][rows], b[3] planes [N][M] with scales [N].
int tc_overlap3(const bf16* const* a, const float* a_scale, int nws, int rows, const bf16* const* b,
                const float* b_scale, int N, int M, double* out, unsigned* flags, cudaStream_t st);

// Row-scaled (fp16) split of `rows` rows of length K (row r at src + r*src_stride) into
// hi/lo [rows][K] (row stride K) and scale[rows].  FP64 or FP32 source.
void split_rows(const double* src, int64_t src_stride, int64_t rows, int64_t K, bf16* hi, bf16* lo, float* scale,
                cudaStream_t st, bf16* rounded = nullptr);   // rounded (optional): r = fp16(x / scale)
void split_rows(const float* src, int64_t src_stride, int64_t rows, int64_t K, bf16* hi, bf16* lo, float* scale,
                cudaStream_t st, bf16* rounded = nullptr);   // rounded (optional): r = fp16(x / scale)

int tc_num_sms();

}  // namespace afqmc
