// Tensor-core (tcgen05 + TMA) split-precision GEMMs of the mixed-precision walker step.
// Internal to the library.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

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

// Output tile epilogues of the generic GEMM (kind selects the write pattern).
enum EpiKind : int {
    EPI_F32 = 0,       // out_f32[b*ob + r*ld + c]
    EPI_SPLIT = 1,     // out_hi/out_lo[b*ob + r*ld + c]  (plain bf16 pair)
    EPI_HSPOT = 2,     // A potential: row (w, c), col (i, k) -> hi/lo[w][i][c*M + k]
    EPI_BFIRST = 3,    // B Phi: doubled operand for the Taylor series + accumulator init
    EPI_TAYLOR = 4,    // (i s) P A^T: doubled operand of the next term + accumulator update
    EPI_F64 = 5,       // out_f64[b*ob + r*ld + c]
    EPI_HSPOT_F32 = 6, // A potential in fp32: row (w, c), col (i, k) -> out_f32[w][i][c*M + k]
    EPI_TAYLOR_F32 = 7,// next Taylor term i*scale*C in fp32 (planar rows) + accumulator update
    // three-slice GEMM (tc_gemm3) epilogues, FP64 values:
    EPI3_F64 = 8,      // out_f64[b*ob + r*ld + c]
    EPI3_HSPOT = 9,    // A potential: row (w, c), col (i, k) -> out_f64[w][i][c*M + k]
    EPI3_TAYLOR = 10,  // next Taylor term i*scale*C -> out_f64 (planar rows), acc64 += term
};

struct EpiParams {
    int kind = EPI_F32;
    int64_t rows_valid = 0, cols_valid = 0;  // per batch
    int64_t ld = 0, ob = 0;                  // row / batch strides of the output (elements)
    float* out_f32 = nullptr;
    bf16* out_hi = nullptr;
    bf16* out_lo = nullptr;
    double* out_f64 = nullptr;
    float* acc = nullptr;                    // Taylor accumulator (fp32)
    double* acc64 = nullptr;                 // Taylor accumulator (FP64, three-slice GEMM)
    int M = 0, N = 0;                        // orbitals, electrons per spin
    float scale = 1.0f;                      // Taylor factor sqrt(tau)/k
    double scale64 = 1.0;                    // the same in FP64 (three-slice GEMM)
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
// Doubled complex operand of a planar FP64 term P [WS][2][N][M] as three slices:
// row (ws, 0, j) = [Re P_j | -Im P_j], row (ws, 1, j) = [Im P_j | Re P_j] (length 2M).
void split3_doubled(const double* P, int64_t WS, int N, int M, bf16* h, bf16* m, bf16* l, float* scale,
                    cudaStream_t st);

// C[b] = A[b] . B[b]^T (split bf16, fp32 accumulation in TMEM), 128 x BN tiles.
// exact = true needs row-scaled A and B and BN = 128.
int tc_gemm(const SplitMat& A, BatchMap amap, const SplitMat& B, BatchMap bmap, int64_t rows, int64_t cols,
            int64_t K, int nbatch, const EpiParams& epi, int BN, bool exact, unsigned* flags, cudaStream_t st);

// Fused energy contraction: T_{n,ws} = Lt_n Theta_ws^T (Np x Np complex, Np | 128) for
// all n and walker-spin pairs ws; emits t = Tr T and X = Tr(T T) per (ws, n) into
// t_out/X_out [nws][Nchol] (complex FP64).  Lt: [Nchol*Np][M], ThetaT: [nws*2*Np][M]
// (rows (ws, re/im, b)), both row-scaled; exact accumulation of the leading product.
// terms = 3 (hi*hi exact, hi*lo + lo*hi) or 4 (+ lo*lo) split products.
int tc_energy(const SplitMat& Lt, const SplitMat& ThetaT, int Np, int Nchol, int nws, int M, cplx* t_out,
              cplx* X_out, int terms, unsigned* flags, cudaStream_t st);

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
                cudaStream_t st);
void split_rows(const float* src, int64_t src_stride, int64_t rows, int64_t K, bf16* hi, bf16* lo, float* scale,
                cudaStream_t st);

int tc_num_sms();

}  // namespace afqmc
