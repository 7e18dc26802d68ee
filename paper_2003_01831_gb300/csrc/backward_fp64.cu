// Adjoint of the mixed local energy and the log-overlap (FP64).
//
// With Q_s = Psi_s^+ (E_L and logS are holomorphic in Q), S = Q Phi, Theta = Phi S^-1,
// T_n = Q L_n Theta, c_n = sum_s Tr T_ns (energy of Sec. V, Eqs. (1), (3)):
//   d logS / dQ^T   = Theta
//   d E_L  / dQ_s^T = (I - Theta Q)[h Theta + sum_n L_n U_n],   U_n = Theta (c_n I - T_n)
//   d E_L  / dL_n   = (sum_s U_ns Q_s)^T
// For the real loss  sum_w Re(conj(dE_w) E_L,w + conj(dlogS_w) logS_w):
//   dPsi_s = sum_w conj(dE_w) (dE_L/dQ_s^T)_w + conj(dlogS_w) Theta_w
//   dL_n   = Re( [ sum_s (sum_w conj(dE_w) U_nsw) Psi_s^+ ]^T )
// Theta and T are recomputed, never stored between calls.  Walkers are processed in
// chunks of Cholesky vectors so the U tensor stays bounded.
#include <algorithm>

#include "state.cuh"

namespace afqmc {

bool is_device_ptr(const void* p);

namespace {

constexpr int kT = 256;
inline unsigned nb(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

// U[w][c] += c_n Theta_w   (c_n = t0[w][n] + t1[w][n])
__global__ void add_ctheta_kernel(cplx* U, const cplx* Theta, const cplx* t0, const cplx* t1, int W, int nc, int n0,
                                  int nch, int64_t MN) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)W * nc * MN) return;
    const int64_t w = i / (nc * MN);
    const int64_t rem = i % (nc * MN);
    const int c = (int)(rem / MN);
    const int64_t e = rem % MN;
    const int64_t ti = w * nch + n0 + c;
    const cplx cn = t0[ti] + t1[ti];
    cfma(U[i], cn, Theta[w * MN + e]);
}

// V[c][e] = sum_w g_w U[w][c][e]   (fixed walker order)
__global__ void weighted_walker_sum_kernel(const cplx* U, const cplx* g, int W, int nc, int64_t MN, cplx* V) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nc * MN) return;
    cplx acc{0.0, 0.0};
    for (int w = 0; w < W; ++w) cfma(acc, g[w], U[(int64_t)w * nc * MN + i]);
    V[i] = acc;
}

// dL[n0+c][i][k] += Re(F[c][k][i])
__global__ void add_re_transpose_kernel(const cplx* F, int nc, int M, double* dL) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t MM = (int64_t)M * M;
    if (i >= (int64_t)nc * MM) return;
    const int64_t c = i / MM, e = i % MM;
    const int r = (int)(e / M), k = (int)(e % M);
    dL[i] += F[c * MM + (int64_t)k * M + r].re;
}

// out[e] = sum_w (gE_w F_w[e] + gS_w Theta_w[e])
__global__ void psi_grad_reduce_kernel(const cplx* F, const cplx* Theta, const cplx* gE, const cplx* gS, int W,
                                       int64_t MN, cplx* out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= MN) return;
    cplx acc{0.0, 0.0};
    for (int w = 0; w < W; ++w) {
        cfma(acc, gE[w], F[(int64_t)w * MN + e]);
        cfma(acc, gS[w], Theta[(int64_t)w * MN + e]);
    }
    out[e] = acc;
}

__global__ void conj_kernel(const cplx* in, cplx* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in ? conjg(in[i]) : cplx{0.0, 0.0};
}

}  // namespace

int fp64_backward(afqmc_walkers* wk, const cplx* dE, const cplx* dlogS, cplx* dPsi_up, cplx* dPsi_dn, double* dL,
                  cudaStream_t st) {
    const int M = wk->M, W = wk->W, nch = wk->Nchol;
    Fp64Buffers& f = wk->f;
    if (wk->opts.precision == AFQMC_PREC_BF16X3) AFQMC_TRY(tc_sync_walkers_to_fp64(wk, st));
    // upstream factors (conjugated), device copies
    cplx *gE = nullptr, *gS = nullptr, *dEd = nullptr, *dSd = nullptr;
    AFQMC_CUDA_TRY(cudaMallocAsync(&gE, sizeof(cplx) * W, st));
    AFQMC_CUDA_TRY(cudaMallocAsync(&gS, sizeof(cplx) * W, st));
    if (dE) {
        AFQMC_CUDA_TRY(cudaMallocAsync(&dEd, sizeof(cplx) * W, st));
        AFQMC_CUDA_TRY(cudaMemcpyAsync(dEd, dE, sizeof(cplx) * W, cudaMemcpyDefault, st));
    }
    if (dlogS) {
        AFQMC_CUDA_TRY(cudaMallocAsync(&dSd, sizeof(cplx) * W, st));
        AFQMC_CUDA_TRY(cudaMemcpyAsync(dSd, dlogS, sizeof(cplx) * W, cudaMemcpyDefault, st));
    }
    count_launch();
    conj_kernel<<<nb(W), kT, 0, st>>>(dEd, gE, W);
    count_launch();
    conj_kernel<<<nb(W), kT, 0, st>>>(dSd, gS, W);

    // Theta, t, X for both spins (FP64 path at the current walkers)
    AFQMC_TRY(fp64_measure(wk, true, st));

    const int Nmax = std::max(wk->N[0], wk->N[1]);
    const int64_t per_u = (int64_t)W * M * Nmax;                 // complex elements per Cholesky vector
    const int nu = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)f.nc, (int64_t)nch,
                                                                 ((int64_t)768 << 20) / (per_u * 16)}));
    cplx *U = nullptr, *V = nullptr, *F = nullptr, *G = nullptr, *Z = nullptr, *gP = nullptr;
    double* dLd = nullptr;
    AFQMC_CUDA_TRY(cudaMallocAsync(&U, sizeof(cplx) * nu * per_u, st));
    AFQMC_CUDA_TRY(cudaMallocAsync(&V, sizeof(cplx) * (size_t)nu * M * Nmax, st));
    AFQMC_CUDA_TRY(cudaMallocAsync(&F, sizeof(cplx) * (size_t)nu * M * M, st));
    AFQMC_CUDA_TRY(cudaMallocAsync(&G, sizeof(cplx) * per_u, st));
    AFQMC_CUDA_TRY(cudaMallocAsync(&Z, sizeof(cplx) * (size_t)W * Nmax * Nmax, st));
    AFQMC_CUDA_TRY(cudaMallocAsync(&gP, sizeof(cplx) * (size_t)M * Nmax, st));
    const bool want_L = dL != nullptr;
    if (want_L) {
        AFQMC_CUDA_TRY(cudaMallocAsync(&dLd, sizeof(double) * (size_t)nch * M * M, st));
        AFQMC_CUDA_TRY(cudaMemsetAsync(dLd, 0, sizeof(double) * (size_t)nch * M * M, st));
    }
    cplx* outs[2] = {dPsi_up, dPsi_dn};
    for (int s = 0; s < 2; ++s) {
        const int N = wk->N[s];
        const int64_t MN = (int64_t)M * N;
        fill_cplx(G, (int64_t)W * MN, cplx{0.0, 0.0}, st);
        for (int n0 = 0; n0 < nch; n0 += nu) {
            const int nc = std::min(nu, nch - n0);
            {   // T[c][w] = Lt_{n0+c} Theta_w
                GemmArgs g;
                g.m = N; g.n = N; g.k = M; g.nb1 = nc; g.nb2 = W;
                g.A.real = wk->Lt_real;
                g.A.ptr = wk->Lt_real
                              ? (const void*)(static_cast<const double*>(f.Lt[s]) + (int64_t)n0 * N * M)
                              : (const void*)(static_cast<const cplx*>(f.Lt[s]) + (int64_t)n0 * N * M);
                g.A.ld = M; g.A.s1 = (int64_t)N * M;
                g.B.ptr = f.Theta[s]; g.B.ld = N; g.B.s2 = MN;
                g.C = f.T; g.ldc = N; g.sc1 = (int64_t)W * N * N; g.sc2 = (int64_t)N * N;
                zgemm(g, st);
            }
            {   // U[w][c] = -Theta_w T[c][w]  (+ c_n Theta_w below)
                GemmArgs g;
                g.m = M; g.n = N; g.k = N; g.nb1 = W; g.nb2 = nc;
                g.A.ptr = f.Theta[s]; g.A.ld = N; g.A.s1 = MN;
                g.B.ptr = f.T; g.B.ld = N; g.B.s1 = (int64_t)N * N; g.B.s2 = (int64_t)W * N * N;
                g.alpha = cplx{-1.0, 0.0};
                g.C = U; g.ldc = N; g.sc1 = (int64_t)nc * MN; g.sc2 = MN;
                zgemm(g, st);
            }
            count_launch();
            add_ctheta_kernel<<<nb((int64_t)W * nc * MN), kT, 0, st>>>(U, f.Theta[s], f.t[0], f.t[1], W, nc, n0, nch,
                                                                       MN);
            {   // G_w += sum_{n in chunk} L_n U_nw  = X^T U_w with X[(n,k)][i] = L[n][k][i]
                GemmArgs g;
                g.m = M; g.n = N; g.k = nc * M; g.nb1 = W;
                g.A.ptr = wk->ham->L + (int64_t)n0 * M * M; g.A.real = true; g.A.op = OP_T; g.A.ld = M;
                g.B.ptr = U; g.B.ld = N; g.B.s1 = (int64_t)nc * MN;
                g.beta = cplx{1.0, 0.0};
                g.C = G; g.ldc = N; g.sc1 = MN;
                zgemm(g, st);
            }
            if (want_L) {
                count_launch();
                weighted_walker_sum_kernel<<<nb((int64_t)nc * MN), kT, 0, st>>>(U, gE, W, nc, MN, V);
                GemmArgs g;   // F[c] = V_c Psi^+   [M][M]
                g.m = M; g.n = M; g.k = N; g.nb1 = nc;
                g.A.ptr = V; g.A.ld = N; g.A.s1 = MN;
                g.B.ptr = f.Psi[s]; g.B.op = OP_C; g.B.ld = N;
                g.C = F; g.ldc = M; g.sc1 = (int64_t)M * M;
                zgemm(g, st);
                count_launch();
                add_re_transpose_kernel<<<nb((int64_t)nc * M * M), kT, 0, st>>>(F, nc, M, dLd + (int64_t)n0 * M * M);
            }
        }
        {   // Y = h Theta + G, formed in place in G
            GemmArgs g;
            g.m = M; g.n = N; g.k = M; g.nb1 = W;
            g.A.ptr = wk->ham->h; g.A.real = true; g.A.ld = M;
            g.B.ptr = f.Theta[s]; g.B.ld = N; g.B.s1 = MN;
            g.beta = cplx{1.0, 0.0};
            g.C = G; g.ldc = N; g.sc1 = MN;
            zgemm(g, st);   // G <- h Theta + G  (this is Y)
        }
        {   // Z = Psi^+ Y
            GemmArgs g;
            g.m = N; g.n = N; g.k = M; g.nb1 = W;
            g.A.ptr = f.Psi[s]; g.A.op = OP_C; g.A.ld = N;
            g.B.ptr = G; g.B.ld = N; g.B.s1 = MN;
            g.C = Z; g.ldc = N; g.sc1 = (int64_t)N * N;
            zgemm(g, st);
        }
        {   // F_w = Y - Theta Z   (in place in G)
            GemmArgs g;
            g.m = M; g.n = N; g.k = N; g.nb1 = W;
            g.A.ptr = f.Theta[s]; g.A.ld = N; g.A.s1 = MN;
            g.B.ptr = Z; g.B.ld = N; g.B.s1 = (int64_t)N * N;
            g.alpha = cplx{-1.0, 0.0};
            g.beta = cplx{1.0, 0.0};
            g.C = G; g.ldc = N; g.sc1 = MN;
            zgemm(g, st);
        }
        count_launch();
        psi_grad_reduce_kernel<<<nb(MN), kT, 0, st>>>(G, f.Theta[s], gE, gS, W, MN, gP);
        if (outs[s]) AFQMC_CUDA_TRY(cudaMemcpyAsync(outs[s], gP, sizeof(cplx) * MN, cudaMemcpyDefault, st));
    }
    if (want_L) AFQMC_CUDA_TRY(cudaMemcpyAsync(dL, dLd, sizeof(double) * (size_t)nch * M * M, cudaMemcpyDefault, st));
    void* frees[] = {U, V, F, G, Z, gP, dLd, gE, gS, dEd, dSd};
    for (void* p : frees)
        if (p) cudaFreeAsync(p, st);
    AFQMC_CUDA_TRY(cudaStreamSynchronize(st));
    unsigned fl = 0;
    AFQMC_CUDA_TRY(cudaMemcpy(&fl, wk->flags, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (fl & FLAG_NONFINITE) return fail(AFQMC_ERR_NONFINITE, "energy_backward: NaN/Inf");
    if (fl & FLAG_SINGULAR) return fail(AFQMC_ERR_SINGULAR, "energy_backward: singular overlap");
    return AFQMC_OK;
}

}  // namespace afqmc
