// Back-propagated one-body density matrix: the back-propagation estimator Sec. V lists for
// observables that do not commute with H (Zhang, Carlson & Gubernatis 1997; Purwanto &
// Zhang 2004; Motta & Zhang 2017).
//
// A window opened at the walkers Phi(0) records the shifted fields c = x - xbar that drove
// each of the next n steps.  The estimate carries the trial back through the adjoints of
// those steps' propagators,
//     Psi_bp,w = B_w(1)^+ ... B_w(n)^+ Psi_T,
//     B_w(k)^+ = B T_K(-i sqrt(tau) A_w(k)^+) B,   A_w(k)^+ = sum_n conj(c_wn(k)) L_n
// (B = exp(-tau h'/2) and every L_n are Hermitian), and averages
//     G[i][j] = <c+_i c_j> = [Phi_w(0) (Psi_bp,w^+ Phi_w(0))^-1 Psi_bp,w^+]_ji
// over the walkers with their end-of-window weights (weight-0 walkers contribute nothing).
// The walker sum is one GEMM over K = W N: G^T = sum_w (w_w / sum w) Theta_w Psi_bp,w^+ with
// both factors laid out row-major over (walker, orbital).  The back-propagated trial is
// re-orthonormalised every k_qr steps, which leaves the estimate unchanged.
//
// FP64 on the DFMA pipe (zgemm and the batched inverse) whatever the walker set's precision.
#include <algorithm>

#include "state.cuh"

namespace afqmc {

namespace {

constexpr int kT = 256;

inline unsigned nb(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

__global__ void conj_kernel(const cplx* a, cplx* b, int64_t n) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) b[id] = conjg(a[id]);
}

// *tot = sum_w w[w], one block of kT threads, fixed order
__global__ void weight_total_kernel(const cplx* w, int W, cplx* tot) {
    __shared__ double re[kT], im[kT];
    double r = 0.0, i = 0.0;
    for (int k = threadIdx.x; k < W; k += kT) {
        r += w[k].re;
        i += w[k].im;
    }
    re[threadIdx.x] = r;
    im[threadIdx.x] = i;
    __syncthreads();
    for (int h = kT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            re[threadIdx.x] += re[threadIdx.x + h];
            im[threadIdx.x] += im[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *tot = cplx{re[0], im[0]};
}

// dst[i][w][a] = f_w src[w][i][a] for W walkers of M x N, with f_w = w_w / tot (exactly 0
// where w_w == 0) when weights are given, else 1.
__global__ void to_orbital_major_kernel(const cplx* src, int W, int M, int N, const cplx* weight,
                                        const cplx* tot, cplx* dst) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t mn = (int64_t)M * N;
    if (id >= (int64_t)W * mn) return;
    const int w = (int)(id / mn);
    const int64_t r = id % mn;
    const int i = (int)(r / N), a = (int)(r % N);
    cplx v = src[id];
    if (weight) {
        const cplx ww = weight[w];
        v = (ww.re == 0.0 && ww.im == 0.0) ? cplx{0.0, 0.0} : cdiv(ww, *tot) * v;
    }
    dst[((int64_t)i * W + w) * N + a] = v;
}

// Walker sum of the estimate on the tensor cores (BF16X3 walker sets).  With v_w = (w_w / sum w)
// Theta_w and K' = (walker, orbital, re|im) = 2 W N, H = sum_w v_w Q_w^+ is the real GEMM
// [A_re; A_im] . B^T: A_re[i][(w,a,0|1)] = (Re, Im) v_w[i][a], A_im[i][(w,a,0|1)] = (Im, -Re)
// v_w[i][a], B[j][(w,a,0|1)] = (Re, Im) Q_w[j][a]; then Hr = A_re B^T and Hi = A_im B^T.  K' is
// cut into nb chunks of kc (the three-slice GEMM's batches; the tail of the last is zero), so
// A is [nb][2M][kc] and B [nb][M][kc], FP64 before the row split.
__global__ void bp_pack_kernel(const cplx* Th, const cplx* Q, const cplx* weight, const cplx* tot, int W, int M,
                               int N, int64_t kc, int nb, double* A, double* B) {
    const int64_t total = (int64_t)nb * M * kc;
    const int64_t K2 = 2LL * W * N;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
        const int64_t kk = id % kc;
        const int64_t r = id / kc;
        const int i = (int)(r % M);
        const int64_t b = r / M;
        const int64_t kp = b * kc + kk;
        double are = 0.0, aim = 0.0, bv = 0.0;
        if (kp < K2) {
            const int64_t K = kp >> 1;
            const int c = (int)(kp & 1);
            const int w = (int)(K / N), a = (int)(K % N);
            const int64_t e = ((int64_t)w * M + i) * N + a;
            const cplx ww = weight[w];
            const cplx v = (ww.re == 0.0 && ww.im == 0.0) ? cplx{0.0, 0.0} : cdiv(ww, *tot) * Th[e];
            are = c == 0 ? v.re : v.im;
            aim = c == 0 ? v.im : -v.re;
            bv = c == 0 ? Q[e].re : Q[e].im;
        }
        A[(b * 2 * M + i) * kc + kk] = are;
        A[(b * 2 * M + M + i) * kc + kk] = aim;
        B[(b * M + i) * kc + kk] = bv;
    }
}

// G[j][i] = sum_b (P_b[i][j] + i P_b[M + i][j]) over the chunk products P_b [2M][M], in chunk order
__global__ void bp_combine_kernel(const double* P, int nb, int M, cplx* G) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t MM = (int64_t)M * M;
    if (id >= MM) return;
    const int i = (int)(id / M), j = (int)(id % M);
    double re = 0.0, im = 0.0;
    for (int b = 0; b < nb; ++b) {
        re += P[(int64_t)b * 2 * MM + (int64_t)i * M + j];
        im += P[(int64_t)b * 2 * MM + (int64_t)(M + i) * M + j];
    }
    G[(int64_t)j * M + i] = cplx{re, im};
}

// b = (sum_c a_c)^T over nc partial M x M products a_c = a + c M^2, summed in chunk order
__global__ void sum_transpose_kernel(const cplx* a, int nc, int M, cplx* b) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t MM = (int64_t)M * M;
    if (id >= MM) return;
    const int i = (int)(id / M), j = (int)(id % M);
    cplx acc = a[id];
    for (int c = 1; c < nc; ++c) acc = acc + a[c * MM + id];
    b[(int64_t)j * M + i] = acc;
}

// Walker chunks for the walker-sum GEMM: its M x M output alone has few 64 x 64 tiles, so the
// K = W N sum is split into chunks of whole walkers, about four CTAs per SM in all.  The
// largest divisor of W not above that target.
int walker_chunks(int W, int M) {
    const int64_t tiles = (int64_t)((M + 63) / 64) * ((M + 63) / 64);
    const int64_t target = std::max<int64_t>(1, (4 * (int64_t)tc_num_sms() + tiles - 1) / tiles);
    int best = 1;
    for (int d = 1; d <= W && d <= target; ++d)
        if (W % d == 0) best = d;
    return best;
}

struct Scratch {
    std::vector<void*> p;
    cudaStream_t st;
    explicit Scratch(cudaStream_t s) : st(s) {}
    template <typename T>
    T* get(size_t count) {
        void* q = nullptr;
        if (cudaMallocAsync(&q, sizeof(T) * std::max<size_t>(count, 1), st) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        p.push_back(q);
        return static_cast<T*>(q);
    }
    ~Scratch() {
        for (void* q : p) cudaFreeAsync(q, st);
    }
};

}  // namespace

void bp_close(afqmc_walkers* wk) {
    for (int s = 0; s < 2; ++s) {
        if (wk->bp_Phi[s]) cudaFree(wk->bp_Phi[s]);
        wk->bp_Phi[s] = nullptr;
    }
    if (wk->bp_coef) cudaFree(wk->bp_coef);
    wk->bp_coef = nullptr;
    wk->bp_n = -1;
    wk->bp_k = 0;
    wk->bp_overrun = false;
}

int bp_open(afqmc_walkers* wk, int nbp, cudaStream_t st) {
    bp_close(wk);
    const int M = wk->M, W = wk->W;
    bool ok = true;
    for (int s = 0; s < 2; ++s)
        ok = ok && cudaMalloc(&wk->bp_Phi[s], sizeof(cplx) * (size_t)W * M * wk->N[s]) == cudaSuccess;
    ok = ok && cudaMalloc(&wk->bp_coef, sizeof(cplx) * (size_t)std::max(nbp, 1) * W * wk->Nchol) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        bp_close(wk);
        return fail(AFQMC_ERR_OOM, "bp_begin: window buffers");
    }
    if (wk->opts.precision == AFQMC_PREC_BF16X3) AFQMC_TRY(tc_sync_walkers_to_fp64(wk, st));
    for (int s = 0; s < 2; ++s)
        AFQMC_CUDA_TRY(cudaMemcpyAsync(wk->bp_Phi[s], wk->f.Phi[s], sizeof(cplx) * (size_t)W * M * wk->N[s],
                                       cudaMemcpyDeviceToDevice, st));
    wk->bp_n = nbp;
    return AFQMC_OK;
}

void bp_record(afqmc_walkers* wk, cudaStream_t st) {
    if (wk->bp_n < 0) return;
    if (wk->bp_k < wk->bp_n) {
        const size_t per = (size_t)wk->W * wk->Nchol;
        cudaMemcpyAsync(wk->bp_coef + (size_t)wk->bp_k * per, wk->coef, sizeof(cplx) * per,
                        cudaMemcpyDeviceToDevice, st);
        ++wk->bp_k;
    } else {
        wk->bp_overrun = true;
    }
}

int bp_follow_comb(afqmc_walkers* wk, const int* idx, cplx* tmp, cudaStream_t st) {
    if (wk->bp_n < 0) return AFQMC_OK;
    const int W = wk->W;
    for (int s = 0; s < 2; ++s) {
        const int64_t per = (int64_t)wk->M * wk->N[s];
        gather_rows(wk->bp_Phi[s], per, idx, W, tmp, st);
        AFQMC_CUDA_TRY(cudaMemcpyAsync(wk->bp_Phi[s], tmp, sizeof(cplx) * per * W, cudaMemcpyDeviceToDevice, st));
    }
    const int64_t per = wk->Nchol;
    for (int k = 0; k < wk->bp_k; ++k) {
        cplx* slot = wk->bp_coef + (int64_t)k * W * per;
        gather_rows(slot, per, idx, W, tmp, st);
        AFQMC_CUDA_TRY(cudaMemcpyAsync(slot, tmp, sizeof(cplx) * per * W, cudaMemcpyDeviceToDevice, st));
    }
    return AFQMC_OK;
}

namespace {

// Walker sum of the estimate on the tensor cores (~1e-8 relative): G = H^T with
// H = sum_w (w_w / sum w) Theta_w Q_w^+, one three-slice GEMM over K' = 2 W N in chunks.
int bp_walker_sum_tc(afqmc_walkers* wk, const cplx* Th, const cplx* Q, int N, const cplx* tot, cplx* Gs,
                     unsigned* flag, cudaStream_t st) {
    const int M = wk->M, W = wk->W;
    const int64_t MM = (int64_t)M * M;
    const int64_t K2 = 2LL * W * N;
    const int64_t kc = std::min<int64_t>(8192, (K2 + 7) / 8 * 8);
    const int nbk = (int)((K2 + kc - 1) / kc);
    const int64_t na = (int64_t)nbk * 2 * M * kc, nbb = (int64_t)nbk * M * kc;
    Scratch ts(st);
    double* A64 = ts.get<double>(na);
    double* B64 = ts.get<double>(nbb);
    bf16* a3[3] = {ts.get<bf16>(na), ts.get<bf16>(na), ts.get<bf16>(na)};
    bf16* b3[3] = {ts.get<bf16>(nbb), ts.get<bf16>(nbb), ts.get<bf16>(nbb)};
    float* as = ts.get<float>((int64_t)nbk * 2 * M);
    float* bs = ts.get<float>((int64_t)nbk * M);
    double* Pp = ts.get<double>((int64_t)nbk * 2 * MM);
    if (!A64 || !B64 || !a3[0] || !a3[1] || !a3[2] || !b3[0] || !b3[1] || !b3[2] || !as || !bs || !Pp)
        return fail(AFQMC_ERR_OOM, "bp_rdm1: tensor-core walker sum workspace");
    count_launch();
    bp_pack_kernel<<<(unsigned)std::min<int64_t>(nb((int64_t)nbk * M * kc), 1 << 20), kT, 0, st>>>(
        Th, Q, wk->weight, tot, W, M, N, kc, nbk, A64, B64);
    split3_rows(A64, (int64_t)nbk * 2 * M, kc, a3[0], a3[1], a3[2], as, st);
    split3_rows(B64, (int64_t)nbk * M, kc, b3[0], b3[1], b3[2], bs, st);
    Split3 sa, sb;
    for (int q = 0; q < 3; ++q) {
        sa.p[q] = a3[q];
        sb.p[q] = b3[q];
    }
    sa.scale = as; sa.K = kc; sa.rows = 2LL * M; sa.batch = nbk; sa.batch_stride = 2LL * M * kc;
    sb.scale = bs; sb.K = kc; sb.rows = M; sb.batch = nbk; sb.batch_stride = (int64_t)M * kc;
    EpiParams e;
    e.kind = EPI3_F64;
    e.rows_valid = 2LL * M;
    e.cols_valid = M;
    e.ld = M;
    e.ob = 2 * MM;
    e.out_f64 = Pp;
    AFQMC_TRY(tc_gemm3(sa, BatchMap{1, nbk}, sb, BatchMap{1, nbk}, 2LL * M, M, kc, nbk, e, wk->flags, st));
    count_launch();
    bp_combine_kernel<<<nb(MM), kT, 0, st>>>(Pp, nbk, M, Gs);
    check_finite(reinterpret_cast<const double*>(Gs), 2 * MM, flag, st);
    return AFQMC_OK;
}

// G[s] (device, M x M each) from a complete window.  flag: device word, FLAG_NONFINITE when
// G is not finite.
int bp_rdm1(afqmc_walkers* wk, cplx* G[2], unsigned* flag, cudaStream_t st) {
    Fp64Buffers& f = wk->f;
    const int M = wk->M, W = wk->W, nch = wk->Nchol, K = wk->opts.k_taylor;
    const int Nmax = std::max(wk->N[0], wk->N[1]);
    const int64_t MM = (int64_t)M * M, big = (int64_t)W * M * Nmax;
    const bool rB = !wk->ham->cplx_L;   // B and L are real unless the Hamiltonian is complex
    const double sq = sqrt(wk->tau);
    Scratch sc(st);
    cplx* Qs[2] = {sc.get<cplx>(big), sc.get<cplx>(big)};
    cplx* P0 = sc.get<cplx>(big);
    cplx* P1 = sc.get<cplx>(big);
    cplx* acc = sc.get<cplx>(big);
    cplx* Th = sc.get<cplx>(big);
    cplx* cc = sc.get<cplx>((size_t)W * nch);
    cplx* S = sc.get<cplx>((size_t)W * Nmax * Nmax);
    cplx* ld = sc.get<cplx>(W);
    const int nck = walker_chunks(W, M);
    cplx* H = sc.get<cplx>(MM * nck);
    cplx* tot = sc.get<cplx>(1);
    unsigned* sing = sc.get<unsigned>(1);
    if (!Qs[0] || !Qs[1] || !P0 || !P1 || !acc || !Th || !cc || !S || !ld || !H || !tot || !sing)
        return fail(AFQMC_ERR_OOM, "bp_rdm1: workspace");
    count_launch();
    weight_total_kernel<<<1, kT, 0, st>>>(wk->weight, W, tot);
    for (int s = 0; s < 2; ++s)
        replicate(Qs[s], f.Psi[s], (int64_t)M * wk->N[s], W, (int64_t)M * wk->N[s], st);
    if (wk->tc) {
        // BF16X3 walker set: every back step on the tensor cores, through the forward step's own
        // three-slice propagation with conjugated coefficients and -i sqrt(tau) (the adjoint
        // B(k)^+ = B T_K(-i sqrt(tau) A(k)^+) B); QR in FP64 on the canonical layout
        const int64_t nT = (int64_t)W * 4 * wk->N[0] * M;
        double* QT = sc.get<double>(nT);
        double* QT2 = sc.get<double>(nT);
        if (!QT || !QT2) return fail(AFQMC_ERR_OOM, "bp_rdm1: workspace");
        tc_canon_to_T(wk, Qs, QT, st);
        for (int k = wk->bp_n - 1; k >= 0; --k) {
            AFQMC_TRY(tc_apply_propagator(wk, wk->bp_coef + (int64_t)k * W * nch, true, -1.0, QT, QT2, st));
            std::swap(QT, QT2);
            const int done = wk->bp_n - k;
            if (wk->opts.k_qr > 0 && done % wk->opts.k_qr == 0 && k > 0) {
                tc_T_to_canon(wk, QT, Qs, st);
                for (int s = 0; s < 2; ++s)
                    qr_reorthonormalise(Qs[s], (int64_t)M * wk->N[s], M, wk->N[s], W, wk->weight, st);
                tc_canon_to_T(wk, Qs, QT, st);
            }
        }
        tc_T_to_canon(wk, QT, Qs, st);
        // the estimate on the tensor cores: Green's functions of both spins, then per spin the
        // walker sum
        cplx* Ths[2] = {P0, P1};
        AFQMC_TRY(tc_bp_green(wk, QT, wk->bp_Phi, Ths, st));
        for (int s = 0; s < 2; ++s) AFQMC_TRY(bp_walker_sum_tc(wk, Ths[s], Qs[s], wk->N[s], tot, G[s], flag, st));
        return AFQMC_OK;
    }
    for (int k = wk->bp_n - 1; k >= 0; --k) {
        // A(k)^+ = sum_n conj(c_n) L_n for every walker, shared by both spins
        count_launch();
        conj_kernel<<<nb((int64_t)W * nch), kT, 0, st>>>(wk->bp_coef + (int64_t)k * W * nch, cc, (int64_t)W * nch);
        GemmArgs g;
        g.m = W; g.n = (int)MM; g.k = nch;
        g.A.ptr = cc; g.A.ld = nch;
        g.B.ptr = wk->ham->L; g.B.real = rB; g.B.ld = MM;
        g.C = f.A; g.ldc = MM;
        zgemm(g, st);
        for (int s = 0; s < 2; ++s) {
            const int N = wk->N[s];
            const int64_t mn = (int64_t)M * N;
            cplx* Q = Qs[s];
            GemmArgs b1;   // P0 = B Q
            b1.m = M; b1.n = N; b1.k = M; b1.nb1 = W;
            b1.A.ptr = f.Bh; b1.A.real = rB; b1.A.ld = M;
            b1.B.ptr = Q; b1.B.ld = N; b1.B.s1 = mn;
            b1.C = P0; b1.ldc = N; b1.sc1 = mn;
            zgemm(b1, st);
            AFQMC_CUDA_TRY(cudaMemcpyAsync(acc, P0, sizeof(cplx) * W * mn, cudaMemcpyDeviceToDevice, st));
            cplx* p0 = P0;
            cplx* p1 = P1;
            for (int t = 1; t <= K; ++t) {
                GemmArgs tg;   // p1 = (-i sqrt(tau) / t) A^+ p0 ;  acc += p1
                tg.m = M; tg.n = N; tg.k = M; tg.nb1 = W;
                tg.A.ptr = f.A; tg.A.ld = M; tg.A.s1 = MM;
                tg.B.ptr = p0; tg.B.ld = N; tg.B.s1 = mn;
                tg.alpha = cplx{0.0, -sq / t};
                tg.C = p1; tg.ldc = N; tg.sc1 = mn;
                tg.D = acc; tg.ldd = N; tg.sd1 = mn;
                zgemm(tg, st);
                std::swap(p0, p1);
            }
            GemmArgs b2;   // Q = B acc
            b2.m = M; b2.n = N; b2.k = M; b2.nb1 = W;
            b2.A.ptr = f.Bh; b2.A.real = rB; b2.A.ld = M;
            b2.B.ptr = acc; b2.B.ld = N; b2.B.s1 = mn;
            b2.C = Q; b2.ldc = N; b2.sc1 = mn;
            zgemm(b2, st);
            const int done = wk->bp_n - k;
            if (wk->opts.k_qr > 0 && done % wk->opts.k_qr == 0 && k > 0)
                qr_reorthonormalise(Q, mn, M, N, W, wk->weight, st);
        }
    }
    for (int s = 0; s < 2; ++s) {
        const int N = wk->N[s];
        const int64_t mn = (int64_t)M * N;
        const cplx* Q = Qs[s];
        {   // S = Psi_bp^+ Phi(0), inverted in place
            GemmArgs g;
            g.m = N; g.n = N; g.k = M; g.nb1 = W;
            g.A.ptr = Q; g.A.op = OP_C; g.A.ld = N; g.A.s1 = mn;
            g.B.ptr = wk->bp_Phi[s]; g.B.ld = N; g.B.s1 = mn;
            g.C = S; g.ldc = N; g.sc1 = (int64_t)N * N;
            zgemm(g, st);
        }
        AFQMC_CUDA_TRY(cudaMemsetAsync(sing, 0, sizeof(unsigned), st));
        batched_inverse_logdet(S, (int64_t)N * N, N, W, ld, true, sing, st);
        {   // Theta = Phi(0) S^-1
            GemmArgs g;
            g.m = M; g.n = N; g.k = N; g.nb1 = W;
            g.A.ptr = wk->bp_Phi[s]; g.A.ld = N; g.A.s1 = mn;
            g.B.ptr = S; g.B.ld = N; g.B.s1 = (int64_t)N * N;
            g.C = Th; g.ldc = N; g.sc1 = mn;
            zgemm(g, st);
        }
        // H = sum_w (w_w / sum w) Theta_w Psi_bp,w^+ over K = (walker, orbital); G = H^T.  The
        // K sum runs as nck batched partial products over chunks of W / nck walkers, added in
        // chunk order with the transpose
        count_launch();
        to_orbital_major_kernel<<<nb((int64_t)W * mn), kT, 0, st>>>(Th, W, M, N, wk->weight, tot, P0);
        count_launch();
        to_orbital_major_kernel<<<nb((int64_t)W * mn), kT, 0, st>>>(Q, W, M, N, nullptr, nullptr, P1);
        const int kc = (W / nck) * N;
        GemmArgs g;
        g.m = M; g.n = M; g.k = kc; g.nb1 = nck;
        g.A.ptr = P0; g.A.ld = (int64_t)W * N; g.A.s1 = kc;
        g.B.ptr = P1; g.B.op = OP_C; g.B.ld = (int64_t)W * N; g.B.s1 = kc;
        g.C = H; g.ldc = M; g.sc1 = MM;
        zgemm(g, st);
        count_launch();
        sum_transpose_kernel<<<nb(MM), kT, 0, st>>>(H, nck, M, G[s]);
        check_finite(reinterpret_cast<const double*>(G[s]), 2 * MM, flag, st);
    }
    return AFQMC_OK;
}

}  // namespace

}  // namespace afqmc

using namespace afqmc;

extern "C" {

int afqmc_bp_begin(afqmc_wk_t wk, int nbp, void* stream) {
    if (!wk) return fail(AFQMC_ERR_BADARG, "bp_begin: NULL handle");
    if (nbp < 0) return fail(AFQMC_ERR_BADARG, "bp_begin: negative window length");
    if (wk->ND > 1) return fail(AFQMC_ERR_UNSUPPORTED, "bp_begin: needs a single-determinant trial");
    if (wk->ham->Nmu > 0) return fail(AFQMC_ERR_UNSUPPORTED, "bp_begin: needs a Hamiltonian with Cholesky vectors (not THC)");
    return bp_open(wk, nbp, static_cast<cudaStream_t>(stream));
}

int afqmc_bp_rdm1(afqmc_wk_t wk, double* rdm_up, double* rdm_dn, void* stream) {
    if (!wk) return fail(AFQMC_ERR_BADARG, "bp_rdm1: NULL handle");
    if (wk->bp_n < 0) return fail(AFQMC_ERR_BADARG, "bp_rdm1: no back-propagation window is open");
    if (wk->bp_overrun) return fail(AFQMC_ERR_BADARG, "bp_rdm1: a step ran after the window was complete");
    if (wk->bp_k != wk->bp_n)
        return fail(AFQMC_ERR_BADARG, "bp_rdm1: the window has " + std::to_string(wk->bp_k) + " of its " +
                                          std::to_string(wk->bp_n) + " steps");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t MM = (int64_t)wk->M * wk->M;
    Scratch sc(st);
    cplx* G = sc.get<cplx>(2 * MM);
    unsigned* flag = sc.get<unsigned>(1);
    if (!G || !flag) return fail(AFQMC_ERR_OOM, "bp_rdm1: output buffers");
    AFQMC_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(unsigned), st));
    cplx* Gs[2] = {G, G + MM};
    AFQMC_TRY(bp_rdm1(wk, Gs, flag, st));
    bool sync = false;
    AFQMC_TRY(copy_out(rdm_up, Gs[0], sizeof(cplx) * MM, st, &sync));
    AFQMC_TRY(copy_out(rdm_dn, Gs[1], sizeof(cplx) * MM, st, &sync));
    unsigned fl = 0;
    AFQMC_TRY(read_flags(flag, st, &fl));
    if (fl & FLAG_NONFINITE)
        return fail(AFQMC_ERR_NONFINITE, "bp_rdm1: a live walker's back-propagated overlap vanished");
    AFQMC_TRY(read_flags(wk->flags, st, &fl));
    return flags_to_error(fl, "bp_rdm1");
}

}  // extern "C"
