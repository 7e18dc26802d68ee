// Mixed-precision (BF16X3) walker-step driver.  The dense contractions of the phaseless
// step (Sec. V; Zhang & Krakauer 2003, Motta & Zhang 2018) run on tcgen05 tensor cores with
// row-scaled fp16 split operands (two slices for the Green's function and the energy, three
// for the overlap, the propagation and the QR's Gram matrix and R^-1 product); the overlap
// inverse runs in float pairs with FP64 pivots and log-determinant, the Cholesky factor and
// the energy and weight reductions in FP64 (kernels_fp64.cu).
//
// Device layouts (W walkers, both spins, N electrons per spin, complex stored planar):
//   PhiT   [W][2][2][N][M] FP64 master walkers, transposed (row (s, c, j) = column j of
//          Phi_s, re/im plane c); a second buffer holds the proposals, copied over the current
//          walkers on acceptance (the current walkers never change buffer, so captured step
//          graphs replay); PhiT3 is the three-slice split of whichever is being multiplied
//   Phi    [W][2][M][2N]   row-scaled fp16 pair, untransposed with re | im columns
//          (Green's-function GEMM operand)
//   Si     [W][2][N][N]    S^-1 of the current walkers (kept from the step that made them)
//   ThT    [W][2][2][N][M] Theta^T = (Phi S^-1)^T: fp32, and its row-scaled fp16 pair
//          (energy GEMM operand)
//   Lt     [Nchol][N][M]   Ltilde_n = Psi^T L_n (trial real, same for both spins): row-scaled
//          pair for the energy; Ltp the same rows over all N*M entries (force bias only)
//   LT3    [M*M][Nchol]    L transposed, three slices (HS potential GEMM operand)
//   A      [W][M][2M]      HS potential sum_n c_n L_n, re | im columns, float-float (+ three
//                          slices)
//   C      [W][2][2][N][M] product P_{k-1} A^T of a Taylor step, float-float; PD3
//                          [W][2][2N][2M] the doubled form [[Re, -Im], [Im, Re]] of the term
//                          P_k = (i sqrt(tau)/k) C as three slices
//   Pacc   [W][2][2][N][M] Taylor sum, float-float (three slices for the final B product)
// Contractions use row-scaled fp16 operands with exact accumulation of the leading products
// (kernels_tc.cu): the Green's-function and energy contractions with two slices (hi*hi summed
// exactly, remainders in a second accumulator), the overlap and the whole propagation with
// three slices and float-float (hi + lo fp32) intermediates (~1e-9), because the walkers'
// overlaps set the weights; the float-float arithmetic keeps that work off the narrow FP64 pipe.
#include <algorithm>
#include <utility>
#include <vector>

#include "ffc.cuh"
#include "kernels_tc.cuh"
#include "state.cuh"
#include "tc_ptx.cuh"

namespace afqmc {

struct TcState {
    int N = 0, M = 0, Nchol = 0, W = 0;
    // static operands
    bf16 *Lt_h = nullptr, *Lt_l = nullptr;
    bf16* Lt_r = nullptr;   // rounded plane r = fp16(Ltilde row / scale) of the rounded energy products
    float* Lt_s = nullptr;
    bf16 *Ltp_h = nullptr, *Ltp_l = nullptr;      // Ltilde rows n over all N*M entries, row-scaled
    float* Ltp_s = nullptr;
    bf16* LT3[3] = {nullptr, nullptr, nullptr};    // L^T [M*M][Nchol], three slices
    float* LT3_s = nullptr;
    bf16* Bh3[3] = {nullptr, nullptr, nullptr};    // B = exp(-tau h'/2) [M][M], three slices
    float* Bh3_s = nullptr;
    bf16 *PsiT_h = nullptr, *PsiT_l = nullptr;
    float* PsiT_s = nullptr;
    double* PsiT_f = nullptr;
    // walkers
    double* PhiT[2] = {nullptr, nullptr};
    bf16 *PhiT3[3] = {nullptr, nullptr, nullptr};   // three-slice split of the walkers being multiplied
    float* PhiT3_s = nullptr;
    bf16 *PsiT3[3] = {nullptr, nullptr, nullptr};   // three-slice split of the trial (static)
    float* PsiT3_s = nullptr;
    double* ST64 = nullptr;                         // [WS][2N][N] overlap (transposed, planar), FP64
    bf16 *Phi_h = nullptr, *Phi_l = nullptr;
    float* Phi_s = nullptr;
    // Green's function and energy
    cplx* S = nullptr;      // scratch: proposals' overlap inverse, Gram matrices of the QR
    cplx* ld = nullptr;     // scratch: proposals' per-spin log-determinants
    cplx* Si = nullptr;     // [W][2][N][N] S^-1 of the current walkers
    cplx* ldc = nullptr;    // [W][2] their per-spin log-determinants
    bf16 *SD_h = nullptr, *SD_l = nullptr;
    float* SD_s = nullptr;
    float* ThT_f = nullptr;
    bf16 *ThT_h = nullptr, *ThT_l = nullptr;
    bf16* ThT_r = nullptr;   // rounded plane r' = fp16(Theta row / scale) of the single-product tiles
    float* ThT_s = nullptr;
    cplx *tE = nullptr, *XE = nullptr;
    float* tFB = nullptr;
    cplx* E1 = nullptr;
    // propagation (three-slice operands, float-float intermediates)
    double* cfp = nullptr;                 // [W][2][Nchol] HS coefficients, planar
    bf16* cf3[3] = {nullptr, nullptr, nullptr};
    float* cf3_s = nullptr;
    float *A_hi = nullptr, *A_lo = nullptr;   // [W][M][2M] HS potential (re | im columns), float-float
    bf16* A3[3] = {nullptr, nullptr, nullptr};
    float* A3_s = nullptr;
    float *C_hi = nullptr, *C_lo = nullptr;   // [W][2][2][N][M] product P_{k-1} A^T of a Taylor step
    bf16* PD3[3] = {nullptr, nullptr, nullptr};   // doubled form of the term [W][2][2N][2M]
    float* PD3_s = nullptr;
    uint8_t* lolo = nullptr;   // [ceil(Nchol / (128 / N))] energy tiles that form lo*lo
    double lolo_frac = 1.0;    // fraction of those groups
    uint8_t* single = nullptr; // [ceil(Nchol / (128 / N))] energy tiles that form the one product r*r'
    double single_frac = 0.0;  // fraction of the CTA-pair tiles that do so
    int n_single = 0;          // number of such groups
    float *Pacc_hi = nullptr, *Pacc_lo = nullptr;   // Taylor sum, float-float
    bf16* Pacc3[3] = {nullptr, nullptr, nullptr};
    float* Pacc3_s = nullptr;
    bf16 *Pacc_h = nullptr, *Pacc_l = nullptr;   // scratch pair of the force-bias-only contraction
    float* Pacc_s = nullptr;
    int cur = 0;
    std::vector<void*> owned;
};

namespace {

constexpr int kT = 256;
// Split products of the energy contraction when the options leave it open: hi*hi (exact),
// r*lo and lo*hi with the rounded Ltilde plane r = fp16(y).  The two-body energy is a difference
// of large Coulomb and exchange sums, so at energies of ~1e3 Ha the lo*lo term matters; r carries
// its leading part at the cost of three products.
// Adaptive energy products (energy_terms = 1): the lo*lo product is skipped for the smallest
// Cholesky vectors whose
// Frobenius norms ||Ltilde_n|| add up to at most this fraction of the total.  The dropped term is
// ~2^-22 of |Ltilde_n| |Theta| per element, so the added error in every energy and force-bias
// term is at most this fraction of the three-product error (which is 1.35 mHa in E_mix over 10
// m512 steps, against 0.33 mHa with four products everywhere).
constexpr double kLoloTail = 0.01;
// Single-product energy tiles (energy_terms = 0, the default): the tiles of the smallest Cholesky
// vectors, whose squared norms ||Ltilde_n||_F^2 add up to at most this fraction of the total, form
// the one product r*r' of the two operands rounded to fp16 after row scaling (relative error
// ~2^-11 per product) instead of the rounded three.  Those vectors carry about this fraction of
// the two-body energy and of the force bias, so the added error is about 2^-11 of it, ~1.5e-8 of
// the two-body energy.
constexpr double kSingleTail = 0x1p-15;
inline unsigned nb(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

template <typename T>
int talloc(TcState* s, T** p, size_t count) {
    if (cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(AFQMC_ERR_OOM, "BF16X3 workspace allocation failed");
    }
    s->owned.push_back(*p);
    return AFQMC_OK;
}

// ----------------------------------------------------------------------------- pack kernels
// accepted walkers take their proposal's overlap inverse and log-determinants (both spins)
__global__ void commit_inverse_kernel(const int* accept, int W, int N, const cplx* Snew, const cplx* ldnew, cplx* Si,
                                      cplx* ldc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = 2LL * N * N;
    if (i >= (int64_t)W * per) return;
    const int64_t w = i / per;
    if (!accept[w]) return;
    Si[i] = Snew[i];
    if (i % ((int64_t)N * N) == 0) ldc[i / ((int64_t)N * N)] = ldnew[i / ((int64_t)N * N)];
}
// Psi [M][N] complex (real part) -> PsiT [N][M] FP64
__global__ void psiT_kernel(const cplx* Psi, int M, int N, double* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * N) return;
    const int a = (int)(i / M), k = (int)(i % M);
    out[i] = Psi[(int64_t)k * N + a].re;
}
// L [Nchol][MM] -> LT [MM][Nchol] FP64, 32 x 32 tiles through shared memory
__global__ void LT_kernel(const double* L, int64_t MM, int nch, double* LT) {
    __shared__ double tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32;  // along MM
    const int n0 = blockIdx.y * 32;               // along Nchol
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int n = n0 + r;
        const int64_t c = c0 + threadIdx.x;
        tile[r][threadIdx.x] = (n < nch && c < MM) ? L[(int64_t)n * MM + c] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t c = c0 + r;
        const int n = n0 + threadIdx.x;
        if (c < MM && n < nch) LT[c * nch + n] = tile[threadIdx.x][r];
    }
}
// canonical Phi_s [W][M][N] complex  <->  PhiT [W][2][2][N][M]
__global__ void canon_to_phiT_kernel(const cplx* Phi, int s, int W, int M, int N, double* PhiT) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)W * M * N) return;
    const int w = (int)(i / ((int64_t)M * N));
    const int64_t e = i % ((int64_t)M * N);
    const int k = (int)(e / N), j = (int)(e % N);
    const cplx v = Phi[i];
    const int64_t base = (((int64_t)w * 2 + s) * 2) * N * M;
    PhiT[base + (int64_t)j * M + k] = v.re;
    PhiT[base + (int64_t)N * M + (int64_t)j * M + k] = v.im;
}
template <typename Real>
__global__ void phiT_to_canon_kernel(const Real* PhiT, int s, int W, int M, int N, cplx* Phi) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)W * M * N) return;
    const int w = (int)(i / ((int64_t)M * N));
    const int64_t e = i % ((int64_t)M * N);
    const int k = (int)(e / N), j = (int)(e % N);
    const int64_t base = (((int64_t)w * 2 + s) * 2) * N * M;
    Phi[i] = cplx{(double)PhiT[base + (int64_t)j * M + k], (double)PhiT[base + (int64_t)N * M + (int64_t)j * M + k]};
}
// PhiT FP64 [WS][2N][M] -> Phi [WS][M][2N] row-scaled fp16 pair, or three slices (SLICES = 3,
// as split3_rows; planes hi, lo, lo2), row = orbital k over the 2N values re | im.  Block = (32 orbitals, one walker-spin); the 2N x 32 tile sits in
// shared memory, each orbital's scale comes from the 2-norm of its column of the tile.  The
// norm (largest exponent per column, then fp32 squares relative to it) and the split (the
// scaled value as a float pair from the double's bits) use no FP64 instructions.
template <int SLICES>
__global__ void __launch_bounds__(kT) phi_untranspose_split_kernel(const double* PhiT, int M, int N2, __half* hi,
                                                                     __half* lo, __half* lo2, float* scale) {
    extern __shared__ double tile[];  // [N2][33]
    __shared__ int cexp[8][32];
    __shared__ float css[8][32];
    __shared__ int kexp[32];
    __shared__ int cbad[32];
    const int64_t ws = blockIdx.y;
    const int k0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const double* src = PhiT + ws * (int64_t)N2 * M;
    int emax = 0, bad = 0;
    for (int r = ty; r < N2; r += 8) {
        const int k = k0 + tx;
        const double v = k < M ? src[(int64_t)r * M + k] : 0.0;
        tile[r * 33 + tx] = v;
        const int E = (int)(((uint32_t)((unsigned long long)__double_as_longlong(v) >> 32) >> 20) & 0x7ffu);
        if (E == 0x7ff) bad = 1;
        else emax = max(emax, E);
    }
    cexp[ty][tx] = emax;
    cbad[tx] = 0;
    __syncthreads();
    if (bad) cbad[tx] = 1;
    int cm = cexp[0][tx];
#pragma unroll
    for (int q = 1; q < 8; ++q) cm = max(cm, cexp[q][tx]);
    float ss = 0.f;
    if (cm > 0) {
        for (int r = ty; r < N2; r += 8) {
            const uint32_t bh = (uint32_t)((unsigned long long)__double_as_longlong(tile[r * 33 + tx]) >> 32);
            const int E = (int)((bh >> 20) & 0x7ffu);
            const int d = E - cm;
            if (E == 0 || E == 0x7ff || d < -60) continue;
            const float v = __uint_as_float(0x3f800000u | ((bh & 0xfffffu) << 3)) *
                            __uint_as_float((uint32_t)(d + 127) << 23);
            ss = fmaf(v, v, ss);
        }
    }
    css[ty][tx] = ss;
    __syncthreads();
    if (ty == 0) {
        float t = css[0][tx];
        for (int q = 1; q < 8; ++q) t += css[q][tx];
        const int k = k0 + tx;
        float sc = 1.0f;
        int kx = 0;
        if (cm > 0 && t > 0.f) {
            int en = 0;
            frexpf(sqrtf(t) * (1.0f + 0x1p-10f), &en);   // margin: truncated mantissas, fp32 sum
            const int e = en + cm - 1023;                 // ||column|| < 2^e
            kx = 11 - e;
            sc = ldexpf(1.0f, e - 11);
        } else {
            kx = 0x40000;                                 // zero column: every value flushes to 0
        }
        if (cbad[tx]) sc = __int_as_float(0x7fc00000);
        kexp[tx] = kx;
        if (k < M) scale[ws * M + k] = sc;
    }
    __syncthreads();
    // write: row k (= k0 + kk) has N2 contiguous outputs; threads along the row
    for (int kk = ty; kk < 32; kk += 8) {
        const int k = k0 + kk;
        if (k >= M) continue;
        const int64_t o = (ws * M + k) * (int64_t)N2;
        const int kx = kexp[kk];
        for (int r = tx; r < N2; r += 32) {
            float yh = 0.f, yl = 0.f;
            if (kx != 0x40000) dbl_scaled_ff(tile[r * 33 + kk], kx, yh, yl);
            if (SLICES == 3) {
                slice3(yh, yl, hi[o + r], lo[o + r], lo2[o + r]);
            } else {
                const float s1 = rintf(yh);
                hi[o + r] = __float2half_rn(s1);
                lo[o + r] = __float2half_rn((yh - s1) + yl);
            }
        }
    }
}
// ST64 [WS][2N][N] (rows (c, b), cols a) -> S [WS][N][N] complex, S[a][b]
__global__ void st64_to_S_kernel(const double* ST, int WS, int N, cplx* S) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)WS * N * N) return;
    const int64_t ws = i / ((int64_t)N * N);
    const int64_t e = i % ((int64_t)N * N);
    const int a = (int)(e / N), b = (int)(e % N);
    const double* base = ST + ws * 2 * N * N;
    S[i] = cplx{base[(int64_t)b * N + a], base[(int64_t)N * N + (int64_t)b * N + a]};
}
// S^-1 [WS][N][N] -> SD [WS][2N][2N] row-scaled fp16 pair: row (0,b) = [Re Si[j][b] | -Im Si[j][b]],
// row (1,b) = [Im | Re]; both rows of b share the scale (2-norm of column b of S^-1).
__global__ void __launch_bounds__(kT) sinv_doubled_kernel(const cplx* Si, int WS, int N, __half* hi, __half* lo,
                                                            float* scale) {
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);   // (ws, b)
    const int lane = threadIdx.x & 31;
    if (r >= (int64_t)WS * N) return;
    const int64_t ws = r / N;
    const int b = (int)(r % N);
    const cplx* col = Si + ws * N * N + b;
    double ss = 0.0;
    for (int j = lane; j < N; j += 32) {
        const cplx v = col[(int64_t)j * N];
        ss += v.re * v.re + v.im * v.im;
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const double nrm = sqrt(ss);          // 2-norm of either doubled row
    int e = 0;
    if (nrm > 0.0) frexp(nrm, &e);
    const double inv = nrm > 0.0 ? ldexp(1.0, 11 - e) : 0.0;
    const float sc = nrm > 0.0 ? (float)ldexp(1.0, e - 11) : 1.0f;
    const int64_t row0 = ws * 2 * N + b, row1 = row0 + N;  // rows (ws, 0, b), (ws, 1, b)
    if (lane == 0) { scale[row0] = sc; scale[row1] = sc; }
    const int64_t K2 = 2 * N;
    for (int j = lane; j < N; j += 32) {
        const cplx v = col[(int64_t)j * N];
        const double yr = v.re * inv, yi = v.im * inv;
        const double hr = rint(yr), hiI = rint(yi);
        const __half Hr = __double2half(hr), Lr = __double2half(yr - hr);
        const __half Hi = __double2half(hiI), Li = __double2half(yi - hiI);
        const __half nHi = __double2half(-hiI), nLi = __double2half(-(yi - hiI));
        hi[row0 * K2 + j] = Hr;      lo[row0 * K2 + j] = Lr;        // Re
        hi[row0 * K2 + N + j] = nHi; lo[row0 * K2 + N + j] = nLi;   // -Im
        hi[row1 * K2 + j] = Hi;      lo[row1 * K2 + j] = Li;        // Im
        hi[row1 * K2 + N + j] = Hr;  lo[row1 * K2 + N + j] = Lr;    // Re
    }
}
// Frobenius norm of each Ltilde_n [Nchol][N][M] (FP64, once per walker set)
__global__ void __launch_bounds__(kT) ltilde_norm_kernel(const double* Lt, int64_t NM, double* nrm) {
    __shared__ double red[kT];
    const double* x = Lt + (int64_t)blockIdx.x * NM;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < NM; i += kT) s = fma(x[i], x[i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) nrm[blockIdx.x] = sqrt(red[0]);
}
// HS coefficients c [W][Nchol] complex -> planar rows [W][2][Nchol]
// planar [w][re/im][n] copy of c (im_sign = -1: of conj(c))
__global__ void coef_planar_kernel(const cplx* c, int64_t W, int nch, double* out, double im_sign) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * nch) return;
    const int64_t w = i / nch, n = i % nch;
    out[(w * 2) * nch + n] = c[i].re;
    out[(w * 2 + 1) * nch + n] = im_sign * c[i].im;
}
__global__ void fb_combine_kernel(const float* tFB, int64_t WS, int nch, cplx* t) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= WS * nch) return;
    const int64_t ws = i / nch, n = i % nch;
    t[i] = cplx{(double)tFB[(ws * 2) * nch + n], (double)tFB[(ws * 2 + 1) * nch + n]};
}
__global__ void logS_pair_kernel(const cplx* ld, int W, cplx* out) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const cplx s = ld[2 * w] + ld[2 * w + 1];
    out[w] = cplx{s.re, atan2(sin(s.im), cos(s.im))};
}
// E1[w] = sum_s sum_{b,k} ht_s[b][k] (ThT_re + i ThT_im)[w, s][b][k]  (fp32 Theta, FP64 sum)
__global__ void __launch_bounds__(kT) e1_kernel(const cplx* ht0, const cplx* ht1, const float* th, int M, int N,
                                                cplx* E1) {
    __shared__ cplx sh[kT];
    const int w = blockIdx.x;
    cplx acc{0.0, 0.0};
    const int64_t NM = (int64_t)N * M;
    for (int s = 0; s < 2; ++s) {
        const cplx* ht = s == 0 ? ht0 : ht1;
        const int64_t base = ((int64_t)w * 2 + s) * 2 * NM;
        for (int64_t e = threadIdx.x; e < NM; e += kT)
            cfma(acc, ht[e], cplx{(double)th[base + e], (double)th[base + NM + e]});
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) E1[w] = sh[0];
}
// E_L and capped force bias from traces in walker-spin layout [W][2][Nchol]
__global__ void __launch_bounds__(kT) le_mixed_kernel(const cplx* E1, const cplx* tE, const cplx* XE, int nch,
                                                      double E0, double tau, double cap, int energy, cplx* E_L,
                                                      cplx* xbar, unsigned* flags) {
    __shared__ cplx sh[kT];
    const int w = blockIdx.x;
    const double sq = sqrt(tau);
    cplx e2{0.0, 0.0};
    for (int n = threadIdx.x; n < nch; n += kT) {
        const int64_t i0 = ((int64_t)w * 2) * nch + n, i1 = i0 + nch;
        const cplx ts = tE[i0] + tE[i1];
        if (energy) {
            cfma(e2, ts, ts);
            e2 = e2 - XE[i0] - XE[i1];
        }
        cplx xb{sq * ts.im, -sq * ts.re};
        if (cap > 0.0) {
            const double m = hypot(xb.re, xb.im);
            if (m > cap) xb = (cap / m) * xb;
        }
        xbar[(int64_t)w * nch + n] = xb;
    }
    if (!energy) return;
    sh[threadIdx.x] = e2;
    __syncthreads();
    for (int o = kT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const cplx E = cplx{E0 + E1[w].re + 0.5 * sh[0].re, E1[w].im + 0.5 * sh[0].im};
        E_L[w] = E;
        if (!(isfinite(E.re) && isfinite(E.im))) atomicOr(flags, FLAG_NONFINITE);
    }
}
// accepted walkers take their proposal: copy nxt -> cur where accept != 0 (the current
// walkers stay in one buffer, so a captured step graph can be replayed)
__global__ void commit_accepted_kernel(const int* accept, int W, int64_t per, const double* new64, double* cur64) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)W * per) return;
    if (accept[i / per]) cur64[i] = new64[i];
}
// ------------------------------------------------------------- Cholesky QR (FP64)
// Phi = Q R with diag R > 0 in three FP64 kernels, as Q = Phi R^-1 with R^H R = Phi^H Phi:
// the Gram matrix (a batched GEMM over the M orbitals), its Cholesky factor and the factor's
// inverse (on chip), and the triangular product.  Walkers are re-orthonormalised every few
// steps, so Phi stays well conditioned and one Cholesky pass leaves ||Q^H Q - I|| ~ cond(Phi)^2
// times the FP64 rounding -- the same Q as Gram-Schmidt or Householder, with about half the
// flops of Gram-Schmidt twice, all in GEMM-shaped loops.
constexpr int kQT = 64;    // output tile (rows and columns)
constexpr int kQK = 16;    // reduction chunk

// G[ws] = Phi^H Phi: G[i][j] = sum_k conj(Phi[k][i]) Phi[k][j]; Phi's column j is the planar
// row pair j of PhiT[ws].  Tiles with ti <= tj are computed and mirrored (G is Hermitian).
__global__ void __launch_bounds__(kT) gram_planar_kernel(const double* PhiT, int M, int N, const cplx* weight,
                                                         cplx* G) {
    const int ti = blockIdx.x, tj = blockIdx.y, ws = blockIdx.z;
    if (ti > tj) return;
    if (weight[ws / 2].re == 0.0 && weight[ws / 2].im == 0.0) return;
    __shared__ double xr[kQK][kQT + 1], xi[kQK][kQT + 1], yr[kQK][kQT + 1], yi[kQK][kQT + 1];
    const double* Pr = PhiT + (int64_t)ws * 2 * N * M;
    const double* Pi = Pr + (int64_t)N * M;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double ar[4][4] = {}, ai[4][4] = {};
    for (int k0 = 0; k0 < M; k0 += kQK) {
        for (int e = threadIdx.x; e < kQK * kQT; e += kT) {
            const int r = e / kQK, k = e % kQK;   // consecutive threads along k: coalesced rows
            const int i = ti * kQT + r, j = tj * kQT + r, kk = k0 + k;
            const bool ok = kk < M;
            xr[k][r] = (ok && i < N) ? Pr[(int64_t)i * M + kk] : 0.0;
            xi[k][r] = (ok && i < N) ? Pi[(int64_t)i * M + kk] : 0.0;
            yr[k][r] = (ok && j < N) ? Pr[(int64_t)j * M + kk] : 0.0;
            yi[k][r] = (ok && j < N) ? Pi[(int64_t)j * M + kk] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kQK; ++k) {
            double a_r[4], a_i[4], b_r[4], b_i[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a_r[q] = xr[k][ty + 16 * q];
                a_i[q] = xi[k][ty + 16 * q];
                b_r[q] = yr[k][tx + 16 * q];
                b_i[q] = yi[k][tx + 16 * q];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {   // conj(x) y
                    ar[a][b] = fma(a_r[a], b_r[b], fma(a_i[a], b_i[b], ar[a][b]));
                    ai[a][b] = fma(a_r[a], b_i[b], fma(-a_i[a], b_r[b], ai[a][b]));
                }
        }
        __syncthreads();
    }
    cplx* Gw = G + (int64_t)ws * N * N;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = ti * kQT + ty + 16 * a, j = tj * kQT + tx + 16 * b;
            if (i < N && j < N) {
                Gw[(int64_t)i * N + j] = cplx{ar[a][b], ai[a][b]};
                if (ti != tj) Gw[(int64_t)j * N + i] = cplx{ar[a][b], -ai[a][b]};
            }
        }
}

// In place on G[ws]: upper Cholesky factor R (G = R^H R, real positive diagonal), then its
// inverse, left in the upper triangle (the strict lower triangle is zeroed).  The upper
// triangle is staged in shared memory, packed row by row, as float pairs (ffc.cuh: ~2^-44
// relative on the fp32 pipe; the Gram matrix it factors is formed to ~1e-9), with the square
// roots and reciprocals of the diagonal in FP64.  A non-positive or non-finite pivot sets
// FLAG_NONFINITE and leaves the identity (the walker keeps its orbitals).
__device__ __forceinline__ int upk(int i, int j, int N) { return i * N - (i * (i - 1)) / 2 + (j - i); }
__device__ __forceinline__ ffc ff_from(cplx v) {
    const float rh = (float)v.re, ih = (float)v.im;
    return ffc{rh, (float)(v.re - (double)rh), ih, (float)(v.im - (double)ih)};
}
__device__ __forceinline__ cplx ff_to(const ffc& v) {
    return cplx{(double)v.rh + (double)v.rl, (double)v.ih + (double)v.il};
}
__device__ __forceinline__ ffc ff_scaled(const ffc& a, float sh, float sl) {   // a s, s real
    ffc r{0.f, 0.f, 0.f, 0.f};
    ff_fma(r.rh, r.rl, a.rh, a.rl, sh, sl);
    ff_fma(r.ih, r.il, a.ih, a.il, sh, sl);
    return r;
}
__device__ __forceinline__ void ff_sub_conj_mul(ffc& a, const ffc& x, const ffc& y) {   // a -= conj(x) y
    ff_fma(a.rh, a.rl, -x.rh, -x.rl, y.rh, y.rl);
    ff_fma(a.rh, a.rl, -x.ih, -x.il, y.ih, y.il);
    ff_fma(a.ih, a.il, -x.rh, -x.rl, y.ih, y.il);
    ff_fma(a.ih, a.il, x.ih, x.il, y.rh, y.rl);
}
__device__ __forceinline__ void ff_add_mul(ffc& a, const ffc& x, const ffc& y) {   // a += x y
    ff_fma(a.rh, a.rl, x.rh, x.rl, y.rh, y.rl);
    ff_fma(a.rh, a.rl, -x.ih, -x.il, y.ih, y.il);
    ff_fma(a.ih, a.il, x.rh, x.rl, y.ih, y.il);
    ff_fma(a.ih, a.il, x.ih, x.il, y.rh, y.rl);
}

__global__ void __launch_bounds__(kT) chol_inv_kernel(cplx* G, int N, const cplx* weight, unsigned* flags) {
    extern __shared__ __align__(16) unsigned char qsm[];
    ffc* U = reinterpret_cast<ffc*>(qsm);          // packed upper triangle, N (N+1) / 2
    __shared__ int s_bad;
    const int ws = blockIdx.x, t = threadIdx.x;
    cplx* Gw = G + (int64_t)ws * N * N;
    const bool dead = weight[ws / 2].re == 0.0 && weight[ws / 2].im == 0.0;
    const int NP = N * (N + 1) / 2;
    if (t == 0) s_bad = 0;
    for (int i = 0; i < N; ++i)
        for (int j = i + t; j < N; j += kT)
            U[upk(i, j, N)] = ff_from(dead ? cplx{i == j ? 1.0 : 0.0, 0.0} : Gw[(int64_t)i * N + j]);
    __syncthreads();
    if (!dead) {
        // right-looking Cholesky: row k of R, then the trailing upper triangle
        for (int k = 0; k < N; ++k) {
            const double d2 = (double)U[upk(k, k, N)].rh + (double)U[upk(k, k, N)].rl;
            if (!(d2 > 0.0) || !isfinite(d2)) {
                if (t == 0) s_bad = 1;
                break;
            }
            const double d = sqrt(d2), id = 1.0 / d;
            const float idh = (float)id, idl = (float)(id - (double)idh);
            __syncthreads();
            for (int j = k + t; j < N; j += kT) {
                const int e = upk(k, j, N);
                U[e] = j == k ? ff_from(cplx{d, 0.0}) : ff_scaled(U[e], idh, idl);
            }
            __syncthreads();
            const int nr = N - k - 1;
            for (int e = t; e < nr * nr; e += kT) {   // trailing upper triangle k < i <= j
                const int ii = k + 1 + e / nr, jj = k + 1 + e % nr;
                if (jj < ii) continue;
                ff_sub_conj_mul(U[upk(ii, jj, N)], U[upk(k, ii, N)], U[upk(k, jj, N)]);
            }
            __syncthreads();
        }
        __syncthreads();
        if (!s_bad) {
            // inverse of the upper triangular R, in place, column by column:
            // X[j][j] = 1 / R[j][j]; X[i][j] = -(sum_{p=i..j-1} X[i][p] R[p][j]) / R[j][j]
            // (N <= kT: thread i owns row i of column j)
            for (int j = 0; j < N; ++j) {
                const double ir = 1.0 / ((double)U[upk(j, j, N)].rh + (double)U[upk(j, j, N)].rl);
                const float irh = (float)ir, irl = (float)(ir - (double)irh);
                // row i < j reads X[i][p] (p < j, final) and R[p][j] (column j, still R): the new
                // column is written only after every row has read it
                ffc val{0.f, 0.f, 0.f, 0.f};
                if (t < j) {
                    ffc acc{0.f, 0.f, 0.f, 0.f};
                    for (int p = t; p < j; ++p) ff_add_mul(acc, U[upk(t, p, N)], U[upk(p, j, N)]);
                    val = ff_scaled(acc, -irh, -irl);
                }
                __syncthreads();
                if (t < j) U[upk(t, j, N)] = val;
                if (t == 0) U[upk(j, j, N)] = ff_from(cplx{ir, 0.0});
                __syncthreads();
            }
        }
    }
    __syncthreads();
    if (s_bad) {
        if (t == 0) atomicOr(flags, FLAG_NONFINITE);
        for (int e = t; e < NP; e += kT) U[e] = ffc{0.f, 0.f, 0.f, 0.f};
        __syncthreads();
        for (int i = t; i < N; i += kT) U[upk(i, i, N)] = ffc{1.f, 0.f, 0.f, 0.f};
        __syncthreads();
    }
    for (int e = t; e < N * N; e += kT) {
        const int i = e / N, j = e % N;
        Gw[e] = i <= j ? ff_to(U[upk(i, j, N)]) : cplx{0.0, 0.0};
    }
}

// Tensor-core Cholesky QR (M >= 2N): the Gram matrix and the product Phi R^-1 as three-slice
// GEMMs on the planar real forms, FP64 results, ~1e-9 relative.
//   Gram: C = PhiT PhiT^T per walker-spin ([2N][M] rows re | im), C [2N][2N]:
//         G[i][j] = C[i][j] + C[N+i][N+j] + i (C[i][N+j] - C[N+i][j]).
//   Apply: PhiT' = D PhiT with D [2N][2N] = [[Xr^T, -Xi^T], [Xi^T, Xr^T]], X = R^-1, formed as
//         D . (PhiT^T)^T with the untransposed walker [M][2N] as the second operand.
__global__ void gram_combine_kernel(const double* C, int WS, int N, cplx* G) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)WS * N * N) return;
    const int64_t ws = t / ((int64_t)N * N);
    const int i = (int)((t / N) % N), j = (int)(t % N);
    const int64_t N2 = 2LL * N;
    const double* c = C + ws * N2 * N2;
    G[t] = cplx{c[i * N2 + j] + c[(N + i) * N2 + N + j], c[i * N2 + N + j] - c[(N + i) * N2 + j]};
}
// D [WS][2N][2N] from X = R^-1 [WS][N][N] (complex); 32 x 32 tiles of X pass through shared
// memory so that both the reads of X rows and the writes of D rows are coalesced.
__global__ void __launch_bounds__(kT) rinv_doubled_kernel(const cplx* X, int N, double* D) {
    __shared__ cplx tile[32][33];
    const int64_t ws = blockIdx.z;
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const cplx* Xw = X + ws * (int64_t)N * N;
    for (int r = ty; r < 32; r += 8) {   // tile[i][j] = X[i0 + i][j0 + j]
        const int i = i0 + r, j = j0 + tx;
        tile[r][tx] = (i < N && j < N) ? Xw[(int64_t)i * N + j] : cplx{0.0, 0.0};
    }
    __syncthreads();
    const int64_t N2 = 2LL * N;
    double* Dw = D + ws * N2 * N2;
    for (int r = ty; r < 32; r += 8) {   // D row j = j0 + r, columns i = i0 + tx
        const int j = j0 + r, i = i0 + tx;
        if (j >= N || i >= N) continue;
        const cplx v = tile[tx][r];      // X[i][j]
        Dw[j * N2 + i] = v.re;
        Dw[j * N2 + N + i] = -v.im;
        Dw[(N + j) * N2 + i] = v.im;
        Dw[(N + j) * N2 + N + i] = v.re;
    }
}

// Q^T rows: out[ws][j] = sum_{i <= j} X[i][j] * PhiT[ws] row i (complex, planar), X = R^-1
// upper triangular.  Tile: 64 rows j x 64 orbitals k.
__global__ void __launch_bounds__(kT) apply_rinv_kernel(const double* PhiT, const cplx* X, int M, int N,
                                                        double* out) {
    const int tk = blockIdx.x, tj = blockIdx.y, ws = blockIdx.z;
    __shared__ double xr_[kQK][kQT + 1], xi_[kQK][kQT + 1], pr_[kQK][kQT + 1], pi_[kQK][kQT + 1];
    const double* Pr = PhiT + (int64_t)ws * 2 * N * M;
    const double* Pi = Pr + (int64_t)N * M;
    const cplx* Xw = X + (int64_t)ws * N * N;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double ar[4][4] = {}, ai[4][4] = {};
    const int imax = min(N, (tj + 1) * kQT);   // rows i <= j only
    for (int i0 = 0; i0 < imax; i0 += kQK) {
        for (int e = threadIdx.x; e < kQK * kQT; e += kT) {
            const int r = e % kQT, q = e / kQT;    // consecutive threads along the fast index
            const int i = i0 + q;
            const int j = tj * kQT + r, k = tk * kQT + r;
            const bool iok = i < N;
            const cplx xv = (iok && j < N) ? Xw[(int64_t)i * N + j] : cplx{0.0, 0.0};
            xr_[q][r] = xv.re;
            xi_[q][r] = xv.im;
            pr_[q][r] = (iok && k < M) ? Pr[(int64_t)i * M + k] : 0.0;
            pi_[q][r] = (iok && k < M) ? Pi[(int64_t)i * M + k] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int q = 0; q < kQK; ++q) {
            double a_r[4], a_i[4], b_r[4], b_i[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a_r[u] = xr_[q][ty + 16 * u];
                a_i[u] = xi_[q][ty + 16 * u];
                b_r[u] = pr_[q][tx + 16 * u];
                b_i[u] = pi_[q][tx + 16 * u];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    ar[a][b] = fma(a_r[a], b_r[b], fma(-a_i[a], b_i[b], ar[a][b]));
                    ai[a][b] = fma(a_r[a], b_i[b], fma(a_i[a], b_r[b], ai[a][b]));
                }
        }
        __syncthreads();
    }
    double* Or = out + (int64_t)ws * 2 * N * M;
    double* Oi = Or + (int64_t)N * M;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = tj * kQT + ty + 16 * a, k = tk * kQT + tx + 16 * b;
            if (j < N && k < M) {
                Or[(int64_t)j * M + k] = ar[a][b];
                Oi[(int64_t)j * M + k] = ai[a][b];
            }
        }
}

SplitMat smat(const bf16* h, const bf16* l, int64_t K, int64_t rows, int64_t batch = 1, const float* scale = nullptr,
              int64_t row_stride = -1, int64_t batch_stride = -1) {
    SplitMat m;
    m.hi = h;
    m.lo = l;
    m.scale = scale;
    m.K = K;
    m.rows = rows;
    m.batch = batch;
    m.row_stride = row_stride < 0 ? K : row_stride;
    m.batch_stride = batch_stride < 0 ? rows * m.row_stride : batch_stride;
    return m;
}

// untransposed operand of the current walkers (Green's-function GEMM)
void untranspose_walkers(TcState* s, cudaStream_t st) {
    dim3 g((s->M + 31) / 32, 2 * s->W);
    const size_t sm = (size_t)2 * s->N * 33 * sizeof(double);
    raise_dyn_smem(phi_untranspose_split_kernel<2>, sm);
    count_launch();
    phi_untranspose_split_kernel<2><<<g, kT, sm, st>>>(s->PhiT[s->cur], s->M, 2 * s->N,
                                                       reinterpret_cast<__half*>(s->Phi_h),
                                                       reinterpret_cast<__half*>(s->Phi_l), nullptr, s->Phi_s);
}

void refresh_operands(TcState* s, cudaStream_t st) { untranspose_walkers(s, st); }

// S = Psi^T Phi for the walkers in buffer b -> Sout (inverted in place when `inverse`), per-spin
// log-determinants -> ldout
// Three-slice operand [batch][rows][K] of tc_gemm3
Split3 sp3(bf16* const* p, const float* sc, int64_t K, int64_t rows, int64_t batch = 1) {
    Split3 x;
    for (int q = 0; q < 3; ++q) x.p[q] = p[q];
    x.scale = sc;
    x.K = K;
    x.rows = rows;
    x.batch = batch;
    x.batch_stride = rows * K;
    return x;
}

int overlap_logdet(afqmc_walkers* wk, int b, bool inverse, cplx* Sout, cplx* ldout, cudaStream_t st) {
    TcState* s = wk->tc;
    const int N = s->N, M = s->M, WS = 2 * s->W;
    // three-slice operands: the log-determinant sets the weights, so S is formed to ~1e-9
    split3_rows(s->PhiT[b], (int64_t)WS * 2 * N, M, s->PhiT3[0], s->PhiT3[1], s->PhiT3[2], s->PhiT3_s, st);
    const bf16* a3[3] = {s->PhiT3[0], s->PhiT3[1], s->PhiT3[2]};
    const bf16* b3[3] = {s->PsiT3[0], s->PsiT3[1], s->PsiT3[2]};
    AFQMC_TRY(tc_overlap3(a3, s->PhiT3_s, WS, 2 * N, b3, s->PsiT3_s, N, M, s->ST64, wk->flags, st));
    count_launch();
    st64_to_S_kernel<<<nb((int64_t)WS * N * N), kT, 0, st>>>(s->ST64, WS, N, Sout);
    // S is formed to ~1e-9 here, so the float-float elimination loses nothing
    batched_inverse_logdet(Sout, (int64_t)N * N, N, WS, ldout, inverse, wk->flags, st, true);
    return AFQMC_OK;
}

// S^-1 and log det of the current walkers, recomputed (after initialisation, QR, set_walkers)
int refresh_inverse(afqmc_walkers* wk, cudaStream_t st) {
    TcState* s = wk->tc;
    return overlap_logdet(wk, s->cur, true, s->Si, s->ldc, st);
}

}  // namespace

int tc_alloc(afqmc_walkers* wk, cudaStream_t st) {
    TcState* s = new TcState();
    wk->tc = s;
    const int N = wk->N[0], M = wk->M, nch = wk->Nchol, W = wk->W;
    s->N = N;
    s->M = M;
    s->Nchol = nch;
    s->W = W;
    const int64_t NM = (int64_t)N * M, MM = (int64_t)M * M;
    AFQMC_TRY(talloc(s, &s->Lt_h, nch * NM));
    AFQMC_TRY(talloc(s, &s->Lt_l, nch * NM));
    AFQMC_TRY(talloc(s, &s->Lt_r, nch * NM));
    AFQMC_TRY(talloc(s, &s->Lt_s, (int64_t)nch * N));
    AFQMC_TRY(talloc(s, &s->Ltp_h, nch * NM));
    AFQMC_TRY(talloc(s, &s->Ltp_l, nch * NM));
    AFQMC_TRY(talloc(s, &s->Ltp_s, nch));
    for (int q = 0; q < 3; ++q) {
        AFQMC_TRY(talloc(s, &s->LT3[q], MM * nch));
        AFQMC_TRY(talloc(s, &s->Bh3[q], MM));
    }
    AFQMC_TRY(talloc(s, &s->LT3_s, MM));
    AFQMC_TRY(talloc(s, &s->Bh3_s, M));
    AFQMC_TRY(talloc(s, &s->PsiT_h, NM));
    AFQMC_TRY(talloc(s, &s->PsiT_l, NM));
    AFQMC_TRY(talloc(s, &s->PsiT_s, N));
    AFQMC_TRY(talloc(s, &s->PsiT_f, NM));
    const int64_t wall = (int64_t)W * 4 * NM;  // PhiT elements
    for (int b = 0; b < 2; ++b) AFQMC_TRY(talloc(s, &s->PhiT[b], wall));
    for (int q = 0; q < 3; ++q) {
        AFQMC_TRY(talloc(s, &s->PhiT3[q], wall));
        AFQMC_TRY(talloc(s, &s->PsiT3[q], NM));
    }
    AFQMC_TRY(talloc(s, &s->PhiT3_s, (int64_t)W * 4 * N));
    AFQMC_TRY(talloc(s, &s->PsiT3_s, N));
    AFQMC_TRY(talloc(s, &s->ST64, (int64_t)W * 2 * 2 * N * N));
    for (int q = 0; q < 3; ++q) {
        AFQMC_TRY(talloc(s, &s->PD3[q], (int64_t)W * 2 * 2 * N * 2 * M));
        AFQMC_TRY(talloc(s, &s->Pacc3[q], wall));
        AFQMC_TRY(talloc(s, &s->A3[q], (int64_t)W * M * 2 * M));
        AFQMC_TRY(talloc(s, &s->cf3[q], (int64_t)W * 2 * nch));
    }
    AFQMC_TRY(talloc(s, &s->PD3_s, (int64_t)W * 4 * N));
    AFQMC_TRY(talloc(s, &s->Pacc3_s, (int64_t)W * 4 * N));
    AFQMC_TRY(talloc(s, &s->A3_s, (int64_t)W * M));
    AFQMC_TRY(talloc(s, &s->cf3_s, (int64_t)W * 2));
    AFQMC_TRY(talloc(s, &s->C_hi, wall));
    AFQMC_TRY(talloc(s, &s->C_lo, wall));
    AFQMC_TRY(talloc(s, &s->Pacc_hi, wall));
    AFQMC_TRY(talloc(s, &s->Pacc_lo, wall));
    AFQMC_TRY(talloc(s, &s->A_hi, (int64_t)W * M * 2 * M));
    AFQMC_TRY(talloc(s, &s->A_lo, (int64_t)W * M * 2 * M));
    AFQMC_TRY(talloc(s, &s->Phi_h, wall));
    AFQMC_TRY(talloc(s, &s->Phi_l, wall));
    AFQMC_TRY(talloc(s, &s->Phi_s, (int64_t)W * 2 * M));
    AFQMC_TRY(talloc(s, &s->S, (int64_t)W * 2 * N * N));
    AFQMC_TRY(talloc(s, &s->ld, (int64_t)W * 2));
    AFQMC_TRY(talloc(s, &s->Si, (int64_t)W * 2 * N * N));
    AFQMC_TRY(talloc(s, &s->ldc, (int64_t)W * 2));
    AFQMC_TRY(talloc(s, &s->SD_h, (int64_t)W * 2 * 4 * N * N));
    AFQMC_TRY(talloc(s, &s->SD_l, (int64_t)W * 2 * 4 * N * N));
    AFQMC_TRY(talloc(s, &s->SD_s, (int64_t)W * 2 * 2 * N));
    AFQMC_TRY(talloc(s, &s->ThT_f, wall));
    AFQMC_TRY(talloc(s, &s->ThT_h, wall));
    AFQMC_TRY(talloc(s, &s->ThT_l, wall));
    AFQMC_TRY(talloc(s, &s->ThT_r, wall));
    AFQMC_TRY(talloc(s, &s->ThT_s, (int64_t)W * 4 * N));
    AFQMC_TRY(talloc(s, &s->tE, (int64_t)W * 2 * nch));
    AFQMC_TRY(talloc(s, &s->XE, (int64_t)W * 2 * nch));
    AFQMC_TRY(talloc(s, &s->tFB, (int64_t)W * 4 * nch));
    AFQMC_TRY(talloc(s, &s->cfp, (int64_t)W * 2 * nch));

    AFQMC_TRY(talloc(s, &s->Pacc_h, wall));
    AFQMC_TRY(talloc(s, &s->Pacc_l, wall));
    AFQMC_TRY(talloc(s, &s->Pacc_s, (int64_t)W * 4 * N));
    AFQMC_TRY(talloc(s, &s->E1, W));
    // static operands
    const double* Ltr = static_cast<const double*>(wk->f.Lt[0]);  // real [Nchol][N][M]
    split_rows(Ltr, M, (int64_t)nch * N, M, s->Lt_h, s->Lt_l, s->Lt_s, st, s->Lt_r);
    {   // energy tiles that form lo*lo (adaptive energy products)
        const int G = 128 / N, ng = (nch + G - 1) / G;
        AFQMC_TRY(talloc(s, &s->lolo, ng));
        double* dn = nullptr;
        if (cudaMalloc(&dn, sizeof(double) * (size_t)nch) != cudaSuccess) {
            cudaGetLastError();
            return fail(AFQMC_ERR_OOM, "BF16X3 workspace allocation failed");
        }
        count_launch();
        ltilde_norm_kernel<<<nch, kT, 0, st>>>(Ltr, NM, dn);
        std::vector<double> hn((size_t)nch);
        std::vector<uint8_t> hf((size_t)ng);
        cudaError_t e = cudaMemcpyAsync(hn.data(), dn, sizeof(double) * (size_t)nch, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(dn);
        AFQMC_CUDA_TRY(e);
        select_lolo_groups(hn.data(), nch, G, kLoloTail, hf.data());
        int four = 0;
        for (int g = 0; g < ng; ++g) four += hf[(size_t)g];
        s->lolo_frac = (double)four / ng;
        AFQMC_CUDA_TRY(cudaMemcpyAsync(s->lolo, hf.data(), (size_t)ng, cudaMemcpyHostToDevice, st));
        // single-product groups, from the squared norms
        AFQMC_TRY(talloc(s, &s->single, ng));
        std::vector<double> hn2((size_t)nch);
        for (int n = 0; n < nch; ++n) hn2[(size_t)n] = hn[(size_t)n] * hn[(size_t)n];
        std::vector<uint8_t> hs((size_t)ng);
        select_single_groups(hn2.data(), nch, G, kSingleTail, hs.data());
        int npairs = (ng + 1) / 2, nsp = 0;
        for (int g = 0; g < ng; ++g) s->n_single += hs[(size_t)g];
        for (int p = 0; p < npairs; ++p) nsp += (hs[(size_t)(2 * p)] && (2 * p + 1 >= ng || hs[(size_t)(2 * p + 1)])) ? 1 : 0;
        s->single_frac = (double)nsp / npairs;
        AFQMC_CUDA_TRY(cudaMemcpyAsync(s->single, hs.data(), (size_t)ng, cudaMemcpyHostToDevice, st));
        AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
    }
    split_rows(Ltr, NM, nch, NM, s->Ltp_h, s->Ltp_l, s->Ltp_s, st);   // force-bias-only operand
    {   // L^T [M*M][Nchol] in FP64 (temporary), then its row-scaled pair
        double* LTd = nullptr;
        if (cudaMalloc(&LTd, sizeof(double) * (size_t)MM * nch) != cudaSuccess) {
            cudaGetLastError();
            return fail(AFQMC_ERR_OOM, "BF16X3 workspace allocation failed");
        }
        dim3 gl((unsigned)((MM + 31) / 32), (unsigned)((nch + 31) / 32));
        count_launch();
        LT_kernel<<<gl, dim3(32, 8), 0, st>>>(wk->ham->L, MM, nch, LTd);
        split3_rows(LTd, MM, nch, s->LT3[0], s->LT3[1], s->LT3[2], s->LT3_s, st);
        cudaStreamSynchronize(st);
        cudaFree(LTd);
    }
    split3_rows(wk->f.Bh, M, M, s->Bh3[0], s->Bh3[1], s->Bh3[2], s->Bh3_s, st);   // B symmetric: rows = columns
    count_launch();
    psiT_kernel<<<nb(NM), kT, 0, st>>>(wk->f.Psi[0], M, N, s->PsiT_f);
    split_rows(s->PsiT_f, M, N, M, s->PsiT_h, s->PsiT_l, s->PsiT_s, st);
    split3_rows(s->PsiT_f, N, M, s->PsiT3[0], s->PsiT3[1], s->PsiT3[2], s->PsiT3_s, st);
    return tc_sync_walkers_from_fp64(wk, st);
}

void tc_free(afqmc_walkers* wk) {
    if (!wk->tc) return;
    for (void* p : wk->tc->owned) cudaFree(p);
    delete wk->tc;
    wk->tc = nullptr;
}

int tc_sync_walkers_from_fp64(afqmc_walkers* wk, cudaStream_t st) {
    TcState* s = wk->tc;
    if (!s) return AFQMC_OK;
    const int64_t n = (int64_t)s->W * s->M * s->N;
    for (int sp = 0; sp < 2; ++sp) {
        count_launch();
        canon_to_phiT_kernel<<<nb(n), kT, 0, st>>>(wk->f.Phi[sp], sp, s->W, s->M, s->N, s->PhiT[s->cur]);
    }
    refresh_operands(s, st);
    return refresh_inverse(wk, st);
}

void tc_canon_to_T(afqmc_walkers* wk, cplx* const* Phi, double* out_T, cudaStream_t st) {
    TcState* s = wk->tc;
    const int64_t n = (int64_t)s->W * s->M * s->N;
    for (int sp = 0; sp < 2; ++sp) {
        count_launch();
        canon_to_phiT_kernel<<<nb(n), kT, 0, st>>>(Phi[sp], sp, s->W, s->M, s->N, out_T);
    }
}

void tc_T_to_canon(afqmc_walkers* wk, const double* in_T, cplx* const* Phi, cudaStream_t st) {
    TcState* s = wk->tc;
    const int64_t n = (int64_t)s->W * s->M * s->N;
    for (int sp = 0; sp < 2; ++sp) {
        count_launch();
        phiT_to_canon_kernel<double><<<nb(n), kT, 0, st>>>(in_T, sp, s->W, s->M, s->N, Phi[sp]);
    }
}

namespace {
// stream-ordered scratch of one call, freed when it goes out of scope
struct CallScratch {
    std::vector<void*> p;
    cudaStream_t st;
    explicit CallScratch(cudaStream_t s) : st(s) {}
    template <typename T>
    T* get(int64_t count) {
        void* q = nullptr;
        if (cudaMallocAsync(&q, sizeof(T) * (size_t)std::max<int64_t>(count, 1), st) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        p.push_back(q);
        return static_cast<T*>(q);
    }
    ~CallScratch() {
        for (void* q : p) cudaFreeAsync(q, st);
    }
};
}  // namespace

int tc_bp_green(afqmc_walkers* wk, const double* QT, cplx* const* Phi0, cplx* const* Theta, cudaStream_t st) {
    TcState* s = wk->tc;
    const int N = s->N, M = s->M, W = s->W, WS = 2 * W;
    const int64_t rows = (int64_t)WS * 2 * N, nT = rows * M, NN = (int64_t)N * N;
    CallScratch sc(st);
    double* P0T = sc.get<double>(nT);
    bf16* q3[3] = {sc.get<bf16>(nT), sc.get<bf16>(nT), sc.get<bf16>(nT)};
    bf16* p3[3] = {sc.get<bf16>(nT), sc.get<bf16>(nT), sc.get<bf16>(nT)};
    float* qs = sc.get<float>(rows);
    float* ps = sc.get<float>(rows);
    double* C64 = sc.get<double>((int64_t)WS * 4 * NN);
    cplx* S = sc.get<cplx>((int64_t)WS * NN);
    cplx* ld = sc.get<cplx>(WS);
    unsigned* sing = sc.get<unsigned>(1);
    bf16* SDh = sc.get<bf16>((int64_t)WS * 4 * NN);
    bf16* SDl = sc.get<bf16>((int64_t)WS * 4 * NN);
    float* SDs = sc.get<float>(rows);
    bf16* Ph = sc.get<bf16>(nT);
    bf16* Pl = sc.get<bf16>(nT);
    float* Ps = sc.get<float>((int64_t)WS * M);
    float* ThT = sc.get<float>(nT);
    if (!P0T || !q3[0] || !q3[1] || !q3[2] || !p3[0] || !p3[1] || !p3[2] || !qs || !ps || !C64 || !S || !ld ||
        !sing || !SDh || !SDl || !SDs || !Ph || !Pl || !Ps || !ThT)
        return fail(AFQMC_ERR_OOM, "bp_rdm1: tensor-core estimate workspace");
    // S = Psi_bp^+ Phi(0) per walker-spin: [Q rows re | im] . [Phi(0) rows re | im]^T (three
    // slices, FP64 out), combined as for the QR's Gram matrix
    tc_canon_to_T(wk, Phi0, P0T, st);
    split3_rows(QT, rows, M, q3[0], q3[1], q3[2], qs, st);
    split3_rows(P0T, rows, M, p3[0], p3[1], p3[2], ps, st);
    {
        EpiParams e;
        e.kind = EPI3_F64;
        e.rows_valid = 2 * N;
        e.cols_valid = 2 * N;
        e.ld = 2 * N;
        e.ob = 4 * NN;
        e.out_f64 = C64;
        AFQMC_TRY(tc_gemm3(sp3(q3, qs, M, 2 * N, WS), BatchMap{1, WS}, sp3(p3, ps, M, 2 * N, WS), BatchMap{1, WS},
                           2 * N, 2 * N, M, WS, e, wk->flags, st));
    }
    count_launch();
    gram_combine_kernel<<<nb((int64_t)WS * NN), kT, 0, st>>>(C64, WS, N, S);
    // S^-1 in float pairs (S is formed to ~1e-9); a singular S belongs to a dead walker, whose
    // weight removes it from the sum
    AFQMC_CUDA_TRY(cudaMemsetAsync(sing, 0, sizeof(unsigned), st));
    batched_inverse_logdet(S, NN, N, WS, ld, true, sing, st, true);
    // Theta^T = (Phi(0) S^-1)^T: the doubled S^-1 pair times Phi(0)'s untransposed pair (exact mode)
    count_launch();
    sinv_doubled_kernel<<<(unsigned)(((int64_t)WS * N + 7) / 8), kT, 0, st>>>(
        S, WS, N, reinterpret_cast<__half*>(SDh), reinterpret_cast<__half*>(SDl), SDs);
    {
        dim3 g((M + 31) / 32, WS);
        const size_t sm = (size_t)2 * N * 33 * sizeof(double);
        raise_dyn_smem(phi_untranspose_split_kernel<2>, sm);
        count_launch();
        phi_untranspose_split_kernel<2><<<g, kT, sm, st>>>(P0T, M, 2 * N, reinterpret_cast<__half*>(Ph),
                                                           reinterpret_cast<__half*>(Pl), nullptr, Ps);
    }
    {
        EpiParams e;
        e.kind = EPI_F32;
        e.rows_valid = 2 * N;
        e.cols_valid = M;
        e.ld = M;
        e.ob = 2LL * N * M;
        e.out_f32 = ThT;
        AFQMC_TRY(tc_gemm(smat(SDh, SDl, 2 * N, 2 * N, WS, SDs), BatchMap{1, WS}, smat(Ph, Pl, 2 * N, M, WS, Ps),
                          BatchMap{1, WS}, 2 * N, M, 2 * N, WS, e, 128, true, wk->flags, st));
    }
    const int64_t n = (int64_t)W * M * N;
    for (int sp = 0; sp < 2; ++sp) {
        count_launch();
        phiT_to_canon_kernel<float><<<nb(n), kT, 0, st>>>(ThT, sp, W, M, N, Theta[sp]);
    }
    return AFQMC_OK;
}

int tc_sync_walkers_to_fp64(afqmc_walkers* wk, cudaStream_t st) {
    TcState* s = wk->tc;
    if (!s) return AFQMC_OK;
    const int64_t n = (int64_t)s->W * s->M * s->N;
    for (int sp = 0; sp < 2; ++sp) {
        count_launch();
        phiT_to_canon_kernel<double><<<nb(n), kT, 0, st>>>(s->PhiT[s->cur], sp, s->W, s->M, s->N, wk->f.Phi[sp]);
    }
    return AFQMC_OK;
}

// Measurement of the mixed step in three phases, so that a batch of systems can run the energy
// contractions of all its systems in one launch between the first and the last:
//   tc_measure_pre:  S^-1 of the current walkers -> Theta^T (exact-mode GEMM) and its split;
//   the contraction: tc_energy (measuring) or the force-bias-only GEMM;
//   tc_measure_post: one-body energy, local energy and force bias.
// whether the walker set's energy contractions form single-product tiles
bool single_tiles(const afqmc_walkers* wk) { return wk->opts.energy_terms == 0 && wk->tc && wk->tc->n_single > 0; }

int tc_measure_pre(afqmc_walkers* wk, cudaStream_t st) {
    TcState* s = wk->tc;
    const int N = s->N, M = s->M, W = s->W, WS = 2 * W;
    // S^-1 of the current walkers is kept from the step that produced them (the proposals'
    // inverse, committed with them) or recomputed after QR / initialisation
    count_launch();
    logS_pair_kernel<<<nb(W), kT, 0, st>>>(s->ldc, W, wk->logS_old);
    count_launch();
    sinv_doubled_kernel<<<(unsigned)(((int64_t)WS * N + 7) / 8), kT, 0, st>>>(
        s->Si, WS, N, reinterpret_cast<__half*>(s->SD_h), reinterpret_cast<__half*>(s->SD_l), s->SD_s);
    {   // Theta^T = (Phi S^-1)^T  [WS][2N][M] fp32, then its row-scaled pair
        EpiParams e;
        e.kind = EPI_F32;
        e.rows_valid = 2 * N;
        e.cols_valid = M;
        e.ld = M;
        e.ob = 2LL * N * M;
        e.out_f32 = s->ThT_f;
        AFQMC_TRY(tc_gemm(smat(s->SD_h, s->SD_l, 2 * N, 2 * N, WS, s->SD_s), BatchMap{1, WS},
                          smat(s->Phi_h, s->Phi_l, 2 * N, M, WS, s->Phi_s), BatchMap{1, WS}, 2 * N, M, 2 * N, WS, e,
                          128, true, wk->flags, st));
        split_rows(s->ThT_f, M, (int64_t)WS * 2 * N, M, s->ThT_h, s->ThT_l, s->ThT_s, st,
                   single_tiles(wk) ? s->ThT_r : nullptr);
    }
    return AFQMC_OK;
}

namespace {
// energy_terms: 0 = rounded three products with single-product tail tiles (default), 2 = rounded
// three products throughout, 1 = adaptive four/three, 3, 4
int energy_terms_of(const afqmc_walkers* wk) {
    const int et = wk->opts.energy_terms;
    return (et == 0 || et == 2) ? kEnergyRounded : (et == 1 ? kEnergyFour : et);
}
}  // namespace

int tc_energy_system(afqmc_walkers* wk, int BK, EnergySys* out) {
    TcState* s = wk->tc;
    if (!s) return fail(AFQMC_ERR_BADARG, "energy_system: not a BF16X3 walker set");
    const int N = s->N, M = s->M, WS = 2 * s->W, nch = s->Nchol;
    return tc_energy_describe(smat(s->Lt_h, s->Lt_l, M, (int64_t)nch * N, 1, s->Lt_s),
                              smat(s->ThT_h, s->ThT_l, M, (int64_t)WS * 2 * N, 1, s->ThT_s), N, nch, WS, M, s->tE,
                              s->XE, energy_terms_of(wk), wk->opts.energy_terms == 1 ? s->lolo : nullptr, s->Lt_r, BK,
                              out, single_tiles(wk) ? s->single : nullptr, s->ThT_r);
}

int tc_measure_post(afqmc_walkers* wk, bool measure, cudaStream_t st) {
    TcState* s = wk->tc;
    const int N = s->N, M = s->M, W = s->W, nch = s->Nchol;
    if (measure) {
        count_launch();
        e1_kernel<<<W, kT, 0, st>>>(wk->f.ht[0], wk->f.ht[1], s->ThT_f, M, N, s->E1);
    }
    const double cap = wk->opts.weight_mode == AFQMC_WEIGHT_FREE ? 0.0 : wk->opts.fb_cap;
    count_launch();
    le_mixed_kernel<<<W, kT, 0, st>>>(s->E1, s->tE, s->XE, nch, wk->ham->E0, wk->tau, cap, measure ? 1 : 0, wk->E_L,
                                      wk->xbar, wk->flags);
    return AFQMC_OK;
}

int tc_measure(afqmc_walkers* wk, bool measure, cudaStream_t st) {
    TcState* s = wk->tc;
    const int N = s->N, M = s->M, W = s->W, WS = 2 * W, nch = s->Nchol;
    AFQMC_TRY(tc_measure_pre(wk, st));
    const bool timed = !stream_capturing(st);
    if (wk->ev0 && timed) cudaEventRecord(wk->ev0, st);
    if (measure) {
        AFQMC_TRY(tc_energy(smat(s->Lt_h, s->Lt_l, M, (int64_t)nch * N, 1, s->Lt_s),
                            smat(s->ThT_h, s->ThT_l, M, (int64_t)WS * 2 * N, 1, s->ThT_s), N, nch, WS, M, s->tE,
                            s->XE, energy_terms_of(wk), wk->opts.energy_terms == 1 ? s->lolo : nullptr, s->Lt_r,
                            wk->flags, st, single_tiles(wk) ? s->single : nullptr, s->ThT_r));
    } else {
        // force bias only: t[ws][n] = sum_{a,k} ThetaT[ws][a][k] Ltilde[n][a][k], one exact-mode GEMM
        // with K = N*M over rows (ws, re/im) of Theta^T (row-scaled pair in the Pacc scratch)
        const int64_t K = (int64_t)N * M;
        split_rows(s->ThT_f, K, 2LL * WS, K, s->Pacc_h, s->Pacc_l, s->Pacc_s, st);
        EpiParams e;
        e.kind = EPI_F32;
        e.rows_valid = 2LL * WS;
        e.cols_valid = nch;
        e.ld = nch;
        e.out_f32 = s->tFB;
        AFQMC_TRY(tc_gemm(smat(s->Pacc_h, s->Pacc_l, K, 2LL * WS, 1, s->Pacc_s), BatchMap{},
                          smat(s->Ltp_h, s->Ltp_l, K, nch, 1, s->Ltp_s), BatchMap{}, 2LL * WS, nch, K, 1, e, 128,
                          true, wk->flags, st));
        count_launch();
        fb_combine_kernel<<<nb((int64_t)WS * nch), kT, 0, st>>>(s->tFB, WS, nch, s->tE);
    }
    if (wk->ev1 && timed) {
        cudaEventRecord(wk->ev1, st);
        wk->ev_valid = true;
    }
    return tc_measure_post(wk, measure, st);
}

// Phi_out = B T_K(sign i sqrt(tau) A) B Phi_in for every walker and spin, with the HS potential
// A = sum_n c_n L_n (conj_c: of conj(c)), B = exp(-tau h'/2): three-slice tensor-core GEMMs with
// float-float intermediates, FP64 result.  Phi_in and Phi_out are in the transposed planar
// layout of PhiT ([W][2][2][N][M]); they may not alias.  The forward step uses c = x - xbar and
// sign = +1; back-propagation carries the trial through the adjoint B(k)^+ = B T_K(-i sqrt(tau)
// A^+) B with A^+ = sum_n conj(c_n) L_n (real symmetric L_n).
int tc_apply_propagator(afqmc_walkers* wk, const cplx* c, bool conj_c, double sign, const double* Phi_in,
                        double* Phi_out, cudaStream_t st) {
    TcState* s = wk->tc;
    const int N = s->N, M = s->M, W = s->W, nch = s->Nchol;
    const int64_t MM = (int64_t)M * M;
    count_launch();
    coef_planar_kernel<<<nb((int64_t)W * nch), kT, 0, st>>>(c, W, nch, s->cfp, conj_c ? -1.0 : 1.0);
    split3_rows(s->cfp, 2LL * W, nch, s->cf3[0], s->cf3[1], s->cf3[2], s->cf3_s, st);
    {   // A_w = sum_n c_wn L_n  -> float-float [W][M][2M], then its three slices
        EpiParams e;
        e.kind = EPI3_HSPOT_FF;
        e.rows_valid = 2LL * W;
        e.cols_valid = MM;
        e.M = M;
        e.out_f32 = s->A_hi;
        e.out_lo32 = s->A_lo;
        AFQMC_TRY(tc_gemm3(sp3(s->cf3, s->cf3_s, nch, 2LL * W), BatchMap{}, sp3(s->LT3, s->LT3_s, nch, MM),
                           BatchMap{}, 2LL * W, MM, nch, 1, e, wk->flags, st));
        split3_rows_ff(s->A_hi, s->A_lo, (int64_t)W * M, 2LL * M, s->A3[0], s->A3[1], s->A3[2], s->A3_s, st);
    }
    const int64_t rowsAll = (int64_t)W * 4 * N;
    const int64_t WS = 2LL * W;
    {   // P0 = B Phi -> Taylor sum (float-float), then the doubled operand of the first term
        split3_rows(Phi_in, rowsAll, M, s->PhiT3[0], s->PhiT3[1], s->PhiT3[2], s->PhiT3_s, st);
        EpiParams e;
        e.kind = EPI3_FF;
        e.rows_valid = rowsAll;
        e.cols_valid = M;
        e.ld = M;
        e.out_f32 = s->Pacc_hi;
        e.out_lo32 = s->Pacc_lo;
        AFQMC_TRY(tc_gemm3(sp3(s->PhiT3, s->PhiT3_s, M, rowsAll), BatchMap{}, sp3(s->Bh3, s->Bh3_s, M, M), BatchMap{},
                           rowsAll, M, M, 1, e, wk->flags, st));
        taylor_step_ff(nullptr, nullptr, 1.0f, 0.0f, s->Pacc_hi, s->Pacc_lo, WS, N, M, true, s->PD3[0], s->PD3[1],
                       s->PD3[2], s->PD3_s, st);
    }
    const double sq = sqrt(wk->tau);
    for (int k = 1; k <= wk->opts.k_taylor; ++k) {
        EpiParams e;   // C = P_{k-1} A^T (planar re / im rows)
        e.kind = EPI3_FF;
        e.rows_valid = 4LL * N;
        e.cols_valid = M;
        e.ld = M;
        e.ob = 4LL * N * M;
        e.out_f32 = s->C_hi;
        e.out_lo32 = s->C_lo;
        AFQMC_TRY(tc_gemm3(sp3(s->PD3, s->PD3_s, 2LL * M, 4LL * N, W), BatchMap{1, W},
                           sp3(s->A3, s->A3_s, 2LL * M, M, W), BatchMap{1, W}, 4LL * N, M, 2LL * M, W, e, wk->flags,
                           st));
        // P_k = (sign i sqrt(tau) / k) C, Pacc += P_k, doubled operand of P_k for the next term
        const double sk = sign * sq / (double)k;
        const float sh = (float)sk, sl = (float)(sk - (double)sh);
        taylor_step_ff(s->C_hi, s->C_lo, sh, sl, s->Pacc_hi, s->Pacc_lo, WS, N, M, k < wk->opts.k_taylor, s->PD3[0],
                       s->PD3[1], s->PD3[2], s->PD3_s, st);
    }
    {   // Phi_out = B Pacc  (FP64)
        split3_rows_ff(s->Pacc_hi, s->Pacc_lo, rowsAll, M, s->Pacc3[0], s->Pacc3[1], s->Pacc3[2], s->Pacc3_s, st);
        EpiParams e;
        e.kind = EPI3_F64;
        e.rows_valid = rowsAll;
        e.cols_valid = M;
        e.ld = M;
        e.out_f64 = Phi_out;
        AFQMC_TRY(tc_gemm3(sp3(s->Pacc3, s->Pacc3_s, M, rowsAll), BatchMap{}, sp3(s->Bh3, s->Bh3_s, M, M), BatchMap{},
                           rowsAll, M, M, 1, e, wk->flags, st));
    }
    return AFQMC_OK;
}

int tc_propagate_and_weight(afqmc_walkers* wk, const double* x, cudaStream_t st) {
    TcState* s = wk->tc;
    const int N = s->N, M = s->M, W = s->W, nch = s->Nchol;
    hs_coefficients(x, wk->xbar, wk->weight, W, nch, wk->coef, wk->flags, st);
    const int nxt = s->cur ^ 1;
    AFQMC_TRY(tc_apply_propagator(wk, wk->coef, false, 1.0, s->PhiT[s->cur], s->PhiT[nxt], st));
    // the proposals' inverse is the next step's S^-1 for every accepted walker
    AFQMC_TRY(overlap_logdet(wk, nxt, true, s->S, s->ld, st));
    count_launch();
    logS_pair_kernel<<<nb(W), kT, 0, st>>>(s->ld, W, wk->logS_new);
    WeightArgs a;
    a.W = W;
    a.Nchol = nch;
    a.mode = wk->opts.weight_mode;
    a.x = x;
    a.xbar = wk->xbar;
    a.logS_old = wk->logS_old;
    a.logS_new = wk->logS_new;
    a.E_L = wk->E_L;
    a.ebound = 2.0 / sqrt(wk->tau);
    a.tau = wk->tau;
    a.E_T = wk->E_T;
    a.E0 = wk->ham->E0;
    a.weight = wk->weight;
    a.accept = wk->accept;
    weight_update(a, st);
    const int64_t per = 4LL * N * M;
    count_launch();
    commit_accepted_kernel<<<nb((int64_t)W * per), kT, 0, st>>>(wk->accept, W, per, s->PhiT[nxt], s->PhiT[s->cur]);
    count_launch();
    commit_inverse_kernel<<<nb((int64_t)W * 2 * N * N), kT, 0, st>>>(wk->accept, W, N, s->S, s->ld, s->Si, s->ldc);
    refresh_operands(s, st);
    return AFQMC_OK;
}

// mean number of split products per energy tile under the walker set's energy_terms setting
int tc_energy_products(afqmc_walkers* wk, double* mean) {
    TcState* s = wk->tc;
    if (!s) return fail(AFQMC_ERR_BADARG, "energy_products: not a BF16X3 walker set");
    const int t = wk->opts.energy_terms;
    // single-product tiles exist only in the CTA-pair form (the default)
    const double one = launch_policy().energy_pair != 0 && single_tiles(wk) ? s->single_frac : 0.0;
    *mean = t == 1 ? 3.0 + s->lolo_frac : (t == 0 ? 3.0 - 2.0 * one : (t == 2 ? 3.0 : (double)t));
    return AFQMC_OK;
}

int tc_debug_terms(afqmc_walkers* wk, double* ST, double* Sinv, double* ThetaT, double* t, double* X, double* E1) {
    TcState* s = wk->tc;
    if (!s) return fail(AFQMC_ERR_BADARG, "debug_mixed_terms: not a BF16X3 walker set");
    AFQMC_TRY(refresh_inverse(wk, 0));   // overlap of the current walkers into ST64 and Si
    AFQMC_TRY(tc_measure(wk, true, 0));
    AFQMC_CUDA_TRY(cudaDeviceSynchronize());
    const int64_t nst = (int64_t)s->W * 4 * s->N * s->N;
    if (ST) AFQMC_CUDA_TRY(cudaMemcpy(ST, s->ST64, nst * 8, cudaMemcpyDeviceToHost));
    if (Sinv) AFQMC_CUDA_TRY(cudaMemcpy(Sinv, s->Si, (nst / 2) * 16, cudaMemcpyDeviceToHost));
    const int64_t nth = (int64_t)s->W * 4 * s->N * s->M;
    if (ThetaT) {
        std::vector<float> h(nth);
        AFQMC_CUDA_TRY(cudaMemcpy(h.data(), s->ThT_f, nth * 4, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < nth; ++i) ThetaT[i] = h[i];
    }
    const int64_t nt = (int64_t)s->W * 2 * s->Nchol;
    if (t) AFQMC_CUDA_TRY(cudaMemcpy(t, s->tE, nt * 16, cudaMemcpyDeviceToHost));
    if (X) AFQMC_CUDA_TRY(cudaMemcpy(X, s->XE, nt * 16, cudaMemcpyDeviceToHost));
    if (E1) AFQMC_CUDA_TRY(cudaMemcpy(E1, s->E1, (int64_t)s->W * 16, cudaMemcpyDeviceToHost));
    return AFQMC_OK;
}

int tc_qr(afqmc_walkers* wk, cudaStream_t st) {
    TcState* s = wk->tc;
    const int N = s->N, M = s->M, WS = 2 * s->W;
    if (N > kT) return fail(AFQMC_ERR_UNSUPPORTED, "tc_qr: N above the Cholesky kernel's row limit");
    const int nt = (N + kQT - 1) / kQT;
    const int nxt = s->cur ^ 1;
    const int64_t N2 = 2LL * N;
    // tensor-core path: the [2N][2N] FP64 scratch of every walker-spin fits in the proposal buffer
    const bool tc = M >= 2 * N;
    if (tc) {
        // Gram matrices: C = PhiT PhiT^T from the three slices of the current walkers
        split3_rows(s->PhiT[s->cur], (int64_t)WS * N2, M, s->PhiT3[0], s->PhiT3[1], s->PhiT3[2], s->PhiT3_s, st);
        EpiParams e;
        e.kind = EPI3_F64;
        e.rows_valid = N2;
        e.cols_valid = N2;
        e.ld = N2;
        e.ob = N2 * N2;
        e.out_f64 = s->PhiT[nxt];
        AFQMC_TRY(tc_gemm3(sp3(s->PhiT3, s->PhiT3_s, M, N2, WS), BatchMap{1, WS}, sp3(s->PhiT3, s->PhiT3_s, M, N2, WS),
                           BatchMap{1, WS}, N2, N2, M, WS, e, wk->flags, st));
        count_launch();
        gram_combine_kernel<<<nb((int64_t)WS * N * N), kT, 0, st>>>(s->PhiT[nxt], WS, N, s->S);
    } else {
        count_launch();
        gram_planar_kernel<<<dim3(nt, nt, WS), kT, 0, st>>>(s->PhiT[s->cur], M, N, wk->weight, s->S);
    }
    // Cholesky factor and its inverse X = R^-1 in place of the Gram matrices (dead walkers: X = I)
    const size_t sm = (size_t)N * (N + 1) / 2 * sizeof(cplx);
    raise_dyn_smem(chol_inv_kernel, sm);
    count_launch();
    chol_inv_kernel<<<WS, kT, sm, st>>>(s->S, N, wk->weight, wk->flags);
    // Q^T = (Phi X)^T into the proposal buffer, then back over the current walkers
    if (tc) {
        count_launch();
        rinv_doubled_kernel<<<dim3((N + 31) / 32, (N + 31) / 32, WS), kT, 0, st>>>(s->S, N, s->PhiT[nxt]);
        // D's three slices: planes of the HS-potential operand (W M 2M >= WS (2N)^2 halves for
        // M >= 2N), scales in the Taylor operand's scale buffer (W 4N = WS 2N rows); both idle here
        split3_rows(s->PhiT[nxt], (int64_t)WS * N2, N2, s->A3[0], s->A3[1], s->A3[2], s->PD3_s, st);
        // the untransposed walkers [WS][M][2N] as three slices: planes of the Taylor operand
        // (8 W N M halves each), scales in the two-slice operand's scale buffer (rebuilt below)
        dim3 g((M + 31) / 32, WS);
        const size_t tsm = (size_t)N2 * 33 * sizeof(double);
        raise_dyn_smem(phi_untranspose_split_kernel<3>, tsm);
        count_launch();
        phi_untranspose_split_kernel<3><<<g, kT, tsm, st>>>(s->PhiT[s->cur], M, (int)N2,
                                                            reinterpret_cast<__half*>(s->PD3[0]),
                                                            reinterpret_cast<__half*>(s->PD3[1]),
                                                            reinterpret_cast<__half*>(s->PD3[2]), s->Phi_s);
        EpiParams e;
        e.kind = EPI3_F64;
        e.rows_valid = N2;
        e.cols_valid = M;
        e.ld = M;
        e.ob = N2 * M;
        e.out_f64 = s->PhiT[nxt];
        AFQMC_TRY(tc_gemm3(sp3(s->A3, s->PD3_s, N2, N2, WS), BatchMap{1, WS}, sp3(s->PD3, s->Phi_s, N2, M, WS),
                           BatchMap{1, WS}, N2, M, N2, WS, e, wk->flags, st));
    } else {
        count_launch();
        apply_rinv_kernel<<<dim3((M + kQT - 1) / kQT, nt, WS), kT, 0, st>>>(s->PhiT[s->cur], s->S, M, N,
                                                                          s->PhiT[nxt]);
    }
    AFQMC_CUDA_TRY(cudaMemcpyAsync(s->PhiT[s->cur], s->PhiT[nxt], sizeof(double) * (size_t)WS * 2 * N * M,
                                   cudaMemcpyDeviceToDevice, st));
    refresh_operands(s, st);
    return refresh_inverse(wk, st);
}

}  // namespace afqmc
