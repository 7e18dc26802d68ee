// Mixed-precision (BF16X3) walker-step driver.  The dense contractions of the phaseless
// step (Sec. V; Zhang & Krakauer 2003, Motta & Zhang 2018) run on tcgen05 tensor cores
// through the split-bf16 GEMM engine; the overlap LU / log-det / inverse, the QR
// re-orthonormalisation, the energy and weight reductions stay in FP64 (kernels_fp64.cu).
//
// Device layouts (W walkers, both spins, N electrons per spin, complex stored planar):
//   PhiT   [W][2][2][N][M] FP64 master walkers, transposed (row (s, c, j) = column j of
//          Phi_s, re/im plane c), plus its bf16 (hi, lo) pair
//   Phi    [W][2][M][2N]   bf16 pair, untransposed with re | im columns (Theta GEMM operand)
//   ThT    [W][2][2][N][M] Theta^T = (Phi S^-1)^T, bf16 pair (energy GEMM operand)
//   Lt     [Nchol][N][M]   Ltilde_n = Psi^T L_n, bf16 pair (trial is real, same both spins)
//   LT     [M*M][Nchol]    L transposed, bf16 pair (HS potential GEMM operand)
//   A      [W][M][2M]      HS potential sum_n c_n L_n, re | im columns, bf16 pair
//   PD     [W][2][2N][2M]  Taylor term in doubled form [[Re, -Im], [Im, Re]] (ping-pong)
//   Pacc   [W][2][2][N][M] fp32 Taylor accumulator
#include <algorithm>
#include <utility>

#include "kernels_tc.cuh"
#include "state.cuh"
#include "tc_ptx.cuh"

namespace afqmc {

struct TcState {
    int N = 0, M = 0, Nchol = 0, W = 0;
    bf16 *Lt_h = nullptr, *Lt_l = nullptr;
    bf16 *LT_h = nullptr, *LT_l = nullptr;
    bf16 *Bh_h = nullptr, *Bh_l = nullptr;
    bf16 *PsiT_h = nullptr, *PsiT_l = nullptr;
    double* PhiT[2] = {nullptr, nullptr};
    bf16 *PhiT_h[2] = {nullptr, nullptr}, *PhiT_l[2] = {nullptr, nullptr};
    bf16 *Phi_h = nullptr, *Phi_l = nullptr;
    float* ST = nullptr;
    cplx* S = nullptr;
    cplx* ld = nullptr;
    bf16 *SD_h = nullptr, *SD_l = nullptr;
    bf16 *ThT_h = nullptr, *ThT_l = nullptr;
    cplx *tE = nullptr, *XE = nullptr;
    float* tFB = nullptr;
    bf16 *cf_h = nullptr, *cf_l = nullptr;
    bf16 *A_h = nullptr, *A_l = nullptr;
    bf16 *PD_h[2] = {nullptr, nullptr}, *PD_l[2] = {nullptr, nullptr};
    float* Pacc = nullptr;
    bf16 *Pacc_h = nullptr, *Pacc_l = nullptr;
    cplx* E1 = nullptr;
    int cur = 0;
    std::vector<void*> owned;
};

namespace {

constexpr int kT = 256;
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
__global__ void split_f64_kernel(const double* src, bf16* hi, bf16* lo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) tc::split_bf16(src[i], hi[i], lo[i]);
}
__global__ void split_f32_kernel(const float* src, bf16* hi, bf16* lo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) tc::split_bf16(src[i], hi[i], lo[i]);
}
// Psi [M][N] complex (real part) -> PsiT [N][M]
__global__ void psiT_kernel(const cplx* Psi, int M, int N, bf16* hi, bf16* lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * N) return;
    const int a = (int)(i / M), k = (int)(i % M);
    tc::split_bf16(Psi[(int64_t)k * N + a].re, hi[i], lo[i]);
}
// L [Nchol][MM] -> LT [MM][Nchol], 32 x 32 tiles through shared memory
__global__ void LT_kernel(const double* L, int64_t MM, int nch, bf16* hi, bf16* lo) {
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
        if (c < MM && n < nch) tc::split_bf16(tile[threadIdx.x][r], hi[c * nch + n], lo[c * nch + n]);
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
__global__ void phiT_to_canon_kernel(const double* PhiT, int s, int W, int M, int N, cplx* Phi) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)W * M * N) return;
    const int w = (int)(i / ((int64_t)M * N));
    const int64_t e = i % ((int64_t)M * N);
    const int k = (int)(e / N), j = (int)(e % N);
    const int64_t base = (((int64_t)w * 2 + s) * 2) * N * M;
    Phi[i] = cplx{PhiT[base + (int64_t)j * M + k], PhiT[base + (int64_t)N * M + (int64_t)j * M + k]};
}
// PhiT pair [WS][2N][M] -> Phi pair [WS][M][2N] (32 x 32 tiles)
__global__ void phiT_to_phi_kernel(const bf16* th, const bf16* tl, int M, int N2, bf16* ph, bf16* pl) {
    __shared__ bf16 sh[32][34], sl[32][34];
    const int64_t ws = blockIdx.z;
    const int r0 = blockIdx.y * 32;  // rows of PhiT (c, j)
    const int k0 = blockIdx.x * 32;  // columns k
    const bf16* TH = th + ws * (int64_t)N2 * M;
    const bf16* TL = tl + ws * (int64_t)N2 * M;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int row = r0 + r, k = k0 + threadIdx.x;
        if (row < N2 && k < M) {
            sh[r][threadIdx.x] = TH[(int64_t)row * M + k];
            sl[r][threadIdx.x] = TL[(int64_t)row * M + k];
        }
    }
    __syncthreads();
    bf16* PH = ph + ws * (int64_t)N2 * M;
    bf16* PL = pl + ws * (int64_t)N2 * M;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r, row = r0 + threadIdx.x;
        if (row < N2 && k < M) {
            PH[(int64_t)k * N2 + row] = sh[threadIdx.x][r];
            PL[(int64_t)k * N2 + row] = sl[threadIdx.x][r];
        }
    }
}
// ST [WS][2N][N] (rows (c, b), cols a) -> S [WS][N][N] complex, S[a][b]
__global__ void st_to_S_kernel(const float* ST, int WS, int N, cplx* S) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)WS * N * N) return;
    const int64_t ws = i / ((int64_t)N * N);
    const int64_t e = i % ((int64_t)N * N);
    const int a = (int)(e / N), b = (int)(e % N);
    const float* base = ST + ws * 2 * N * N;
    S[i] = cplx{(double)base[(int64_t)b * N + a], (double)base[(int64_t)N * N + (int64_t)b * N + a]};
}
// S^-1 [WS][N][N] -> SD [WS][2N][2N]: row (0,b) = [Re Si[j][b] | -Im Si[j][b]], row (1,b) = [Im | Re]
__global__ void sinv_doubled_kernel(const cplx* Si, int WS, int N, bf16* hi, bf16* lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)4 * N * N;
    if (i >= (int64_t)WS * per) return;
    const int64_t ws = i / per;
    const int64_t e = i % per;
    const int row = (int)(e / (2 * N)), col = (int)(e % (2 * N));
    const int c = row / N, b = row % N, cp = col / N, j = col % N;
    const cplx v = Si[ws * N * N + (int64_t)j * N + b];
    double x;
    if (c == 0) x = (cp == 0) ? v.re : -v.im;
    else x = (cp == 0) ? v.im : v.re;
    tc::split_bf16(x, hi[i], lo[i]);
}
__global__ void coef_split_kernel(const cplx* c, int64_t W, int nch, bf16* hi, bf16* lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * nch) return;
    const int64_t w = i / nch, n = i % nch;
    tc::split_bf16(c[i].re, hi[(w * 2) * nch + n], lo[(w * 2) * nch + n]);
    tc::split_bf16(c[i].im, hi[(w * 2 + 1) * nch + n], lo[(w * 2 + 1) * nch + n]);
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
// E1[w] = sum_s sum_{b,k} ht_s[b][k] (ThT_re + i ThT_im)[w, s][b][k]
__global__ void __launch_bounds__(kT) e1_kernel(const cplx* ht0, const cplx* ht1, const bf16* th, const bf16* tl,
                                                int M, int N, cplx* E1) {
    __shared__ cplx sh[kT];
    const int w = blockIdx.x;
    cplx acc{0.0, 0.0};
    const int64_t NM = (int64_t)N * M;
    for (int s = 0; s < 2; ++s) {
        const cplx* ht = s == 0 ? ht0 : ht1;
        const int64_t base = ((int64_t)w * 2 + s) * 2 * NM;
        for (int64_t e = threadIdx.x; e < NM; e += kT) {
            const double re = (double)__bfloat162float(th[base + e]) + (double)__bfloat162float(tl[base + e]);
            const double im = (double)__bfloat162float(th[base + NM + e]) + (double)__bfloat162float(tl[base + NM + e]);
            cfma(acc, ht[e], cplx{re, im});
        }
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
// rejected walkers keep their old state: copy cur -> nxt where accept == 0
__global__ void keep_rejected_kernel(const int* accept, int W, int64_t per, const double* old64, double* new64,
                                     const bf16* oh, const bf16* ol, bf16* nh, bf16* nl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)W * per) return;
    if (accept[i / per]) return;
    new64[i] = old64[i];
    nh[i] = oh[i];
    nl[i] = ol[i];
}
// Classical Gram-Schmidt (twice) on the N columns of one walker-spin, stored as planar
// rows of PhiT: column j = (re row j, im row j), length M.  diag R > 0.
__global__ void __launch_bounds__(kT) qr_planar_kernel(double* PhiT, int M, int N, const cplx* weight) {
    extern __shared__ double qs[];
    double* vr = qs;       // M
    double* vi = qs + M;   // M
    double* rr = vi + M;   // N
    double* ri = rr + N;   // N
    __shared__ double red[kT];
    const int ws = blockIdx.x, w = ws / 2;
    if (weight[w].re == 0.0 && weight[w].im == 0.0) return;
    double* Qr = PhiT + (int64_t)ws * 2 * N * M;
    double* Qi = Qr + (int64_t)N * M;
    const int t = threadIdx.x;
    for (int j = 0; j < N; ++j) {
        for (int k = t; k < M; k += kT) { vr[k] = Qr[(int64_t)j * M + k]; vi[k] = Qi[(int64_t)j * M + k]; }
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {
            // r_i = <q_i, v> for i < j: one warp per i, lanes over k
            const int warp = t >> 5, lane = t & 31;
            for (int i = warp; i < j; i += kT / 32) {
                double ar = 0.0, ai = 0.0;
                for (int k = lane; k < M; k += 32) {
                    const double qr = Qr[(int64_t)i * M + k], qi = Qi[(int64_t)i * M + k];
                    ar += qr * vr[k] + qi * vi[k];   // conj(q) v
                    ai += qr * vi[k] - qi * vr[k];
                }
                for (int o = 16; o > 0; o >>= 1) {
                    ar += __shfl_xor_sync(0xffffffffu, ar, o);
                    ai += __shfl_xor_sync(0xffffffffu, ai, o);
                }
                if (lane == 0) { rr[i] = ar; ri[i] = ai; }
            }
            __syncthreads();
            for (int k = t; k < M; k += kT) {
                double ar = vr[k], ai = vi[k];
                for (int i = 0; i < j; ++i) {
                    const double qr = Qr[(int64_t)i * M + k], qi = Qi[(int64_t)i * M + k];
                    ar -= qr * rr[i] - qi * ri[i];
                    ai -= qr * ri[i] + qi * rr[i];
                }
                vr[k] = ar;
                vi[k] = ai;
            }
            __syncthreads();
        }
        double p = 0.0;
        for (int k = t; k < M; k += kT) p += vr[k] * vr[k] + vi[k] * vi[k];
        red[t] = p;
        __syncthreads();
        for (int o = kT / 2; o > 0; o >>= 1) {
            if (t < o) red[t] += red[t + o];
            __syncthreads();
        }
        const double inv = 1.0 / sqrt(red[0]);
        for (int k = t; k < M; k += kT) {
            Qr[(int64_t)j * M + k] = vr[k] * inv;
            Qi[(int64_t)j * M + k] = vi[k] * inv;
        }
        __syncthreads();
    }
}

SplitMat smat(const bf16* h, const bf16* l, int64_t K, int64_t rows, int64_t batch = 1, int64_t row_stride = -1,
              int64_t batch_stride = -1) {
    SplitMat m;
    m.hi = h;
    m.lo = l;
    m.K = K;
    m.rows = rows;
    m.batch = batch;
    m.row_stride = row_stride < 0 ? K : row_stride;
    m.batch_stride = batch_stride < 0 ? rows * m.row_stride : batch_stride;
    return m;
}

// refresh the bf16 pair and the untransposed operand of the current walkers
void refresh_operands(TcState* s, cudaStream_t st) {
    const int64_t n = (int64_t)s->W * 4 * s->N * s->M;
    count_launch();
    split_f64_kernel<<<nb(n), kT, 0, st>>>(s->PhiT[s->cur], s->PhiT_h[s->cur], s->PhiT_l[s->cur], n);
    dim3 g((s->M + 31) / 32, (2 * s->N + 31) / 32, 2 * s->W);
    count_launch();
    phiT_to_phi_kernel<<<g, dim3(32, 8), 0, st>>>(s->PhiT_h[s->cur], s->PhiT_l[s->cur], s->M, 2 * s->N, s->Phi_h,
                                                  s->Phi_l);
}

// S = Psi^T Phi for the walkers held in (h, l) -> s->S; logdet into s->ld; optional inverse
int overlap_logdet(afqmc_walkers* wk, const bf16* h, const bf16* l, bool inverse, cudaStream_t st) {
    TcState* s = wk->tc;
    const int N = s->N, M = s->M, WS = 2 * s->W;
    EpiParams e;
    e.kind = EPI_F32;
    e.rows_valid = 2 * N;
    e.cols_valid = N;
    e.ld = N;
    e.ob = 2LL * N * N;
    e.out_f32 = s->ST;
    AFQMC_TRY(tc_gemm(smat(h, l, M, 2 * N, WS), BatchMap{1, WS}, smat(s->PsiT_h, s->PsiT_l, M, N, 1), BatchMap{1, 1},
                      2 * N, N, M, WS, e, 128, wk->flags, st));
    count_launch();
    st_to_S_kernel<<<nb((int64_t)WS * N * N), kT, 0, st>>>(s->ST, WS, N, s->S);
    batched_inverse_logdet(s->S, (int64_t)N * N, N, WS, s->ld, inverse, wk->flags, st);
    return AFQMC_OK;
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
    AFQMC_TRY(talloc(s, &s->LT_h, MM * nch));
    AFQMC_TRY(talloc(s, &s->LT_l, MM * nch));
    AFQMC_TRY(talloc(s, &s->Bh_h, MM));
    AFQMC_TRY(talloc(s, &s->Bh_l, MM));
    AFQMC_TRY(talloc(s, &s->PsiT_h, NM));
    AFQMC_TRY(talloc(s, &s->PsiT_l, NM));
    const int64_t wall = (int64_t)W * 4 * NM;  // PhiT elements
    for (int b = 0; b < 2; ++b) {
        AFQMC_TRY(talloc(s, &s->PhiT[b], wall));
        AFQMC_TRY(talloc(s, &s->PhiT_h[b], wall));
        AFQMC_TRY(talloc(s, &s->PhiT_l[b], wall));
        AFQMC_TRY(talloc(s, &s->PD_h[b], (int64_t)W * 2 * 2 * N * 2 * M));
        AFQMC_TRY(talloc(s, &s->PD_l[b], (int64_t)W * 2 * 2 * N * 2 * M));
    }
    AFQMC_TRY(talloc(s, &s->Phi_h, wall));
    AFQMC_TRY(talloc(s, &s->Phi_l, wall));
    AFQMC_TRY(talloc(s, &s->ST, (int64_t)W * 2 * 2 * N * N));
    AFQMC_TRY(talloc(s, &s->S, (int64_t)W * 2 * N * N));
    AFQMC_TRY(talloc(s, &s->ld, (int64_t)W * 2));
    AFQMC_TRY(talloc(s, &s->SD_h, (int64_t)W * 2 * 4 * N * N));
    AFQMC_TRY(talloc(s, &s->SD_l, (int64_t)W * 2 * 4 * N * N));
    AFQMC_TRY(talloc(s, &s->ThT_h, wall));
    AFQMC_TRY(talloc(s, &s->ThT_l, wall));
    AFQMC_TRY(talloc(s, &s->tE, (int64_t)W * 2 * nch));
    AFQMC_TRY(talloc(s, &s->XE, (int64_t)W * 2 * nch));
    AFQMC_TRY(talloc(s, &s->tFB, (int64_t)W * 4 * nch));
    AFQMC_TRY(talloc(s, &s->cf_h, (int64_t)W * 2 * nch));
    AFQMC_TRY(talloc(s, &s->cf_l, (int64_t)W * 2 * nch));
    AFQMC_TRY(talloc(s, &s->A_h, (int64_t)W * M * 2 * M));
    AFQMC_TRY(talloc(s, &s->A_l, (int64_t)W * M * 2 * M));
    AFQMC_TRY(talloc(s, &s->Pacc, wall));
    AFQMC_TRY(talloc(s, &s->Pacc_h, wall));
    AFQMC_TRY(talloc(s, &s->Pacc_l, wall));
    AFQMC_TRY(talloc(s, &s->E1, W));
    // static operands
    const double* Ltr = static_cast<const double*>(wk->f.Lt[0]);  // real [Nchol][N][M]
    count_launch();
    split_f64_kernel<<<nb(nch * NM), kT, 0, st>>>(Ltr, s->Lt_h, s->Lt_l, nch * NM);
    dim3 gl((unsigned)((MM + 31) / 32), (unsigned)((nch + 31) / 32));
    count_launch();
    LT_kernel<<<gl, dim3(32, 8), 0, st>>>(wk->ham->L, MM, nch, s->LT_h, s->LT_l);
    count_launch();
    split_f64_kernel<<<nb(MM), kT, 0, st>>>(wk->f.Bh, s->Bh_h, s->Bh_l, MM);
    count_launch();
    psiT_kernel<<<nb(NM), kT, 0, st>>>(wk->f.Psi[0], M, N, s->PsiT_h, s->PsiT_l);
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
    return AFQMC_OK;
}

int tc_sync_walkers_to_fp64(afqmc_walkers* wk, cudaStream_t st) {
    TcState* s = wk->tc;
    if (!s) return AFQMC_OK;
    const int64_t n = (int64_t)s->W * s->M * s->N;
    for (int sp = 0; sp < 2; ++sp) {
        count_launch();
        phiT_to_canon_kernel<<<nb(n), kT, 0, st>>>(s->PhiT[s->cur], sp, s->W, s->M, s->N, wk->f.Phi[sp]);
    }
    return AFQMC_OK;
}

int tc_measure(afqmc_walkers* wk, bool measure, cudaStream_t st) {
    TcState* s = wk->tc;
    const int N = s->N, M = s->M, W = s->W, WS = 2 * W, nch = s->Nchol;
    AFQMC_TRY(overlap_logdet(wk, s->PhiT_h[s->cur], s->PhiT_l[s->cur], true, st));
    count_launch();
    logS_pair_kernel<<<nb(W), kT, 0, st>>>(s->ld, W, wk->logS_old);
    count_launch();
    sinv_doubled_kernel<<<nb((int64_t)WS * 4 * N * N), kT, 0, st>>>(s->S, WS, N, s->SD_h, s->SD_l);
    {   // Theta^T = (Phi S^-1)^T  [WS][2N][M]
        EpiParams e;
        e.kind = EPI_SPLIT;
        e.rows_valid = 2 * N;
        e.cols_valid = M;
        e.ld = M;
        e.ob = 2LL * N * M;
        e.out_hi = s->ThT_h;
        e.out_lo = s->ThT_l;
        AFQMC_TRY(tc_gemm(smat(s->SD_h, s->SD_l, 2 * N, 2 * N, WS), BatchMap{1, WS},
                          smat(s->Phi_h, s->Phi_l, 2 * N, M, WS), BatchMap{1, WS}, 2 * N, M, 2 * N, WS, e,
                          M % 256 == 0 ? 256 : 128, wk->flags, st));
    }
    if (wk->ev0) cudaEventRecord(wk->ev0, st);
    if (measure) {
        AFQMC_TRY(tc_energy(smat(s->Lt_h, s->Lt_l, M, (int64_t)nch * N), smat(s->ThT_h, s->ThT_l, M, (int64_t)WS * 2 * N),
                            N, nch, WS, M, s->tE, s->XE, wk->flags, st));
    } else {
        EpiParams e;
        e.kind = EPI_F32;
        e.rows_valid = 2LL * WS;
        e.cols_valid = nch;
        e.ld = nch;
        e.out_f32 = s->tFB;
        const int64_t K = (int64_t)N * M;
        AFQMC_TRY(tc_gemm(smat(s->ThT_h, s->ThT_l, K, 2LL * WS), BatchMap{}, smat(s->Lt_h, s->Lt_l, K, nch),
                          BatchMap{}, 2LL * WS, nch, K, 1, e, 256, wk->flags, st));
        count_launch();
        fb_combine_kernel<<<nb((int64_t)WS * nch), kT, 0, st>>>(s->tFB, WS, nch, s->tE);
    }
    if (wk->ev1) {
        cudaEventRecord(wk->ev1, st);
        wk->ev_valid = true;
    }
    if (measure) e1_kernel<<<W, kT, 0, st>>>(wk->f.ht[0], wk->f.ht[1], s->ThT_h, s->ThT_l, M, N, s->E1);
    const double cap = wk->opts.weight_mode == AFQMC_WEIGHT_FREE ? 0.0 : wk->opts.fb_cap;
    count_launch();
    le_mixed_kernel<<<W, kT, 0, st>>>(s->E1, s->tE, s->XE, nch, wk->ham->E0, wk->tau, cap, measure ? 1 : 0, wk->E_L,
                                      wk->xbar, wk->flags);
    return AFQMC_OK;
}

int tc_propagate_and_weight(afqmc_walkers* wk, const double* x, cudaStream_t st) {
    TcState* s = wk->tc;
    const int N = s->N, M = s->M, W = s->W, nch = s->Nchol;
    const int64_t MM = (int64_t)M * M;
    const int BNm = M % 256 == 0 ? 256 : 128;
    hs_coefficients(x, wk->xbar, wk->weight, W, nch, wk->coef, wk->flags, st);
    count_launch();
    coef_split_kernel<<<nb((int64_t)W * nch), kT, 0, st>>>(wk->coef, W, nch, s->cf_h, s->cf_l);
    {   // A_w = sum_n c_wn L_n  -> [W][M][2M]
        EpiParams e;
        e.kind = EPI_HSPOT;
        e.rows_valid = 2LL * W;
        e.cols_valid = MM;
        e.M = M;
        e.out_hi = s->A_h;
        e.out_lo = s->A_l;
        AFQMC_TRY(tc_gemm(smat(s->cf_h, s->cf_l, nch, 2LL * W), BatchMap{}, smat(s->LT_h, s->LT_l, nch, MM), BatchMap{},
                          2LL * W, MM, nch, 1, e, 256, wk->flags, st));
    }
    const int64_t rowsAll = (int64_t)W * 4 * N;
    {   // P0 = B Phi -> doubled operand + accumulator
        EpiParams e;
        e.kind = EPI_BFIRST;
        e.rows_valid = rowsAll;
        e.cols_valid = M;
        e.M = M;
        e.N = N;
        e.out_hi = s->PD_h[0];
        e.out_lo = s->PD_l[0];
        e.acc = s->Pacc;
        AFQMC_TRY(tc_gemm(smat(s->PhiT_h[s->cur], s->PhiT_l[s->cur], M, rowsAll), BatchMap{},
                          smat(s->Bh_h, s->Bh_l, M, M), BatchMap{}, rowsAll, M, M, 1, e, BNm, wk->flags, st));
    }
    const float sq = (float)sqrt(wk->tau);
    for (int k = 1; k <= wk->opts.k_taylor; ++k) {
        const int src = (k - 1) & 1, dst = k & 1;
        EpiParams e;
        e.kind = EPI_TAYLOR;
        e.rows_valid = 4LL * N;
        e.cols_valid = M;
        e.M = M;
        e.N = N;
        e.out_hi = s->PD_h[dst];
        e.out_lo = s->PD_l[dst];
        e.acc = s->Pacc;
        e.scale = sq / (float)k;
        AFQMC_TRY(tc_gemm(smat(s->PD_h[src], s->PD_l[src], 2LL * M, 4LL * N, W), BatchMap{1, W},
                          smat(s->A_h, s->A_l, 2LL * M, M, W), BatchMap{1, W}, 4LL * N, M, 2LL * M, W, e, BNm,
                          wk->flags, st));
    }
    const int nxt = s->cur ^ 1;
    {
        const int64_t n = rowsAll * M;
        count_launch();
        split_f32_kernel<<<nb(n), kT, 0, st>>>(s->Pacc, s->Pacc_h, s->Pacc_l, n);
        EpiParams e;
        e.kind = EPI_BFINAL;
        e.rows_valid = rowsAll;
        e.cols_valid = M;
        e.ld = M;
        e.out_f64 = s->PhiT[nxt];
        e.out_hi = s->PhiT_h[nxt];
        e.out_lo = s->PhiT_l[nxt];
        AFQMC_TRY(tc_gemm(smat(s->Pacc_h, s->Pacc_l, M, rowsAll), BatchMap{}, smat(s->Bh_h, s->Bh_l, M, M), BatchMap{},
                          rowsAll, M, M, 1, e, BNm, wk->flags, st));
    }
    AFQMC_TRY(overlap_logdet(wk, s->PhiT_h[nxt], s->PhiT_l[nxt], false, st));
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
    a.tau = wk->tau;
    a.E_T = wk->E_T;
    a.E0 = wk->ham->E0;
    a.weight = wk->weight;
    a.accept = wk->accept;
    weight_update(a, st);
    const int64_t per = 4LL * N * M;
    count_launch();
    keep_rejected_kernel<<<nb((int64_t)W * per), kT, 0, st>>>(wk->accept, W, per, s->PhiT[s->cur], s->PhiT[nxt],
                                                              s->PhiT_h[s->cur], s->PhiT_l[s->cur], s->PhiT_h[nxt],
                                                              s->PhiT_l[nxt]);
    s->cur = nxt;
    dim3 g((M + 31) / 32, (2 * N + 31) / 32, 2 * W);
    count_launch();
    phiT_to_phi_kernel<<<g, dim3(32, 8), 0, st>>>(s->PhiT_h[s->cur], s->PhiT_l[s->cur], M, 2 * N, s->Phi_h, s->Phi_l);
    return AFQMC_OK;
}

int tc_qr(afqmc_walkers* wk, cudaStream_t st) {
    TcState* s = wk->tc;
    const size_t sm = (size_t)(2 * s->M + 2 * s->N) * sizeof(double);
    count_launch();
    qr_planar_kernel<<<2 * s->W, kT, sm, st>>>(s->PhiT[s->cur], s->M, s->N, wk->weight);
    refresh_operands(s, st);
    return AFQMC_OK;
}

}  // namespace afqmc
