// FP64 walker-step driver: the phaseless AFQMC step (Sec. V; Zhang & Krakauer 2003,
// Motta & Zhang 2018) as a sequence of DFMA kernels.  This is the precision reference
// of the GPU path; the tensor-core path (step_tc.cu) replaces its contractions.
#include <algorithm>

#include "state.cuh"

namespace afqmc {

namespace {

__global__ void add_logdet_kernel(const cplx* a, const cplx* b, cplx* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const cplx s = a[i] + b[i];
    out[i] = cplx{s.re, atan2(sin(s.im), cos(s.im))};
}

template <typename T>
int dalloc(T** p, size_t count) {
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * count);
    if (e != cudaSuccess) return fail(AFQMC_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return AFQMC_OK;
}

void add_logdet(const cplx* a, const cplx* b, cplx* out, int n, cudaStream_t st) {
    count_launch();
    add_logdet_kernel<<<(n + 255) / 256, 256, 0, st>>>(a, b, out, n);
}

// Y[w] = op(X) Phi[w]-style helpers --------------------------------------------------------
// S_w = Psi^+ Phi_w   (N x N)
void overlap(const cplx* Psi, const cplx* Phi, cplx* S, int M, int N, int W, cudaStream_t st) {
    GemmArgs g;
    g.m = N; g.n = N; g.k = M; g.nb1 = W;
    g.A.ptr = Psi; g.A.op = OP_C; g.A.ld = N;
    g.B.ptr = Phi; g.B.op = OP_N; g.B.ld = N; g.B.s1 = (int64_t)M * N;
    g.C = S; g.ldc = N; g.sc1 = (int64_t)N * N;
    zgemm(g, st);
}

}  // namespace

int fp64_alloc(afqmc_walkers* wk) {
    Fp64Buffers& f = wk->f;
    const int M = wk->M, W = wk->W, nch = wk->Nchol, ND = wk->ND;
    const int Nmu = wk->ham->Nmu;   // > 0: THC Hamiltonian
    const size_t budget = (size_t)512 << 20;
    const int Nmax = std::max(wk->N[0], wk->N[1]);
    // multi-determinant trials: the measurement runs chunks of msd_nd determinants at once, their
    // Green's functions held for all walkers (both spins within the budget)
    f.msd_nd = 1;
    if (ND > 1)
        f.msd_nd = (int)std::max<size_t>(1, std::min<size_t>((size_t)ND, budget / ((size_t)2 * W * M * Nmax * sizeof(cplx))));
    const size_t nd = (size_t)f.msd_nd;
    for (int s = 0; s < 2; ++s) {
        const int N = wk->N[s];
        const size_t mn = (size_t)M * N;
        AFQMC_TRY(dalloc(&f.Psi[s], ND * mn));
        if (Nmu > 0) {
            AFQMC_TRY(dalloc(&f.Yt[s], (size_t)N * Nmu));
            AFQMC_TRY(dalloc(&f.Z[s], (size_t)W * N * Nmu));
            AFQMC_TRY(dalloc(&f.gs[s], (size_t)W * Nmu));
            AFQMC_TRY(dalloc(&f.ex[s], (size_t)W));
        } else {
            AFQMC_TRY(dalloc(reinterpret_cast<cplx**>(&f.Lt[s]), ND * (size_t)nch * mn));
            AFQMC_TRY(dalloc(reinterpret_cast<cplx**>(&f.LtT[s]), ND * (size_t)nch * mn));
        }
        AFQMC_TRY(dalloc(&f.ht[s], ND * mn));
        AFQMC_TRY(dalloc(&f.Phi[s], (size_t)W * mn));
        AFQMC_TRY(dalloc(&f.Pnew[s], (size_t)W * mn));
        AFQMC_TRY(dalloc(&f.Pa[s], (size_t)W * mn));
        AFQMC_TRY(dalloc(&f.Pb[s], (size_t)W * mn));
        AFQMC_TRY(dalloc(&f.S[s], nd * W * N * N));
        AFQMC_TRY(dalloc(&f.ld[s], nd * W));
        AFQMC_TRY(dalloc(&f.Theta[s], nd * W * mn));
        AFQMC_TRY(dalloc(&f.t[s], nd * W * nch));
        AFQMC_TRY(dalloc(&f.X[s], nd * W * nch));
    }
    AFQMC_TRY(dalloc(&f.Bh, (size_t)M * M * (wk->ham->cplx_L ? 2 : 1)));
    if (Nmu > 0) {   // walker chunks of the THC densities T and of X diag(U c)
        const size_t per_w = std::max((size_t)Nmu * Nmu, (size_t)M * Nmu) * sizeof(cplx);
        f.thc_wc = (int)std::max<size_t>(1, std::min<size_t>((size_t)W, budget / per_w));
        AFQMC_TRY(dalloc(&f.Tthc, (size_t)f.thc_wc * Nmu * Nmu));
        AFQMC_TRY(dalloc(&f.XD, (size_t)f.thc_wc * M * Nmu));
        AFQMC_TRY(dalloc(&f.dv, (size_t)W * Nmu));
    } else {
        const size_t per_n = nd * W * Nmax * Nmax * sizeof(cplx);
        f.nc = (int)std::max<size_t>(1, std::min<size_t>((size_t)nch, budget / std::max<size_t>(per_n, 1)));
        f.nc = std::min(f.nc, 65535);
        AFQMC_TRY(dalloc(&f.T, (size_t)f.nc * nd * W * Nmax * Nmax));
    }
    AFQMC_TRY(dalloc(&f.A, (size_t)W * M * M));
    if (ND > 1) {
        AFQMC_TRY(dalloc(&f.msd_cc, (size_t)ND));
        AFQMC_TRY(dalloc(&f.msd_ls, (size_t)ND * W));
        AFQMC_TRY(dalloc(&f.msd_E, (size_t)ND * W));
        AFQMC_TRY(dalloc(&f.msd_t, (size_t)ND * W * nch));
        AFQMC_TRY(dalloc(&f.msd_flag, 2));
        AFQMC_TRY(dalloc(&f.msd_Es, nd * W));
    }
    return AFQMC_OK;
}

void fp64_free(afqmc_walkers* wk) {
    Fp64Buffers& f = wk->f;
    for (int s = 0; s < 2; ++s) {
        void* ps[] = {f.Psi[s], f.Lt[s], f.LtT[s], f.ht[s], f.Phi[s], f.Pnew[s], f.Pa[s], f.Pb[s],
                      f.S[s], f.ld[s], f.Theta[s], f.t[s], f.X[s], f.Yt[s], f.Z[s], f.gs[s], f.ex[s]};
        for (void* p : ps)
            if (p) cudaFree(p);
    }
    void* more[] = {f.Bh, f.T, f.A, f.msd_cc, f.msd_ls, f.msd_E, f.msd_t, f.msd_flag, f.msd_Es, f.Tthc, f.dv, f.XD};
    for (void* p : more)
        if (p) cudaFree(p);
    f = Fp64Buffers{};
}

namespace {

// Green's function, traces, local energy and force bias at the first W walkers with the
// trial's determinant I alone: logS -> logS_out, E_L -> E_out, xbar -> wk->xbar.  Status bits
// of the inverses go to inv_flags, those of the local energy to le_flags.
void measure_det(afqmc_walkers* wk, int I, bool measure, int W, cplx* logS_out, cplx* E_out,
                 unsigned* inv_flags, unsigned* le_flags, cudaStream_t st) {
    Fp64Buffers& f = wk->f;
    const int M = wk->M, nch = wk->Nchol;
    const bool timed = !stream_capturing(st) && I == 0;
    for (int s = 0; s < 2; ++s) {
        const int N = wk->N[s];
        const int64_t mn = (int64_t)M * N, lt = (int64_t)I * nch * mn;
        const cplx* Psi = f.Psi[s] + I * mn;
        const void* Lt = wk->Lt_real ? (const void*)(static_cast<const double*>(f.Lt[s]) + lt)
                                     : (const void*)(static_cast<const cplx*>(f.Lt[s]) + lt);
        const void* LtT = wk->Lt_real ? (const void*)(static_cast<const double*>(f.LtT[s]) + lt)
                                      : (const void*)(static_cast<const cplx*>(f.LtT[s]) + lt);
        overlap(Psi, f.Phi[s], f.S[s], M, N, W, st);
        batched_inverse_logdet(f.S[s], (int64_t)N * N, N, W, f.ld[s], true, inv_flags, st);
        {   // Theta_w = Phi_w S_w^-1
            GemmArgs g;
            g.m = M; g.n = N; g.k = N; g.nb1 = W;
            g.A.ptr = f.Phi[s]; g.A.ld = N; g.A.s1 = (int64_t)M * N;
            g.B.ptr = f.S[s]; g.B.ld = N; g.B.s1 = (int64_t)N * N;
            g.C = f.Theta[s]; g.ldc = N; g.sc1 = (int64_t)M * N;
            zgemm(g, st);
        }
        if (s == 0 && wk->ev0 && timed) cudaEventRecord(wk->ev0, st);
        if (wk->ham->Nmu > 0) {
            // THC: Z = Theta^T X, densities g_mu and (measuring) T = Yt^T Z with its exchange sum,
            // then the force-bias traces t_n = sum_mu U_mu n g_mu of this spin
            const int Nmu = wk->ham->Nmu;
            GemmArgs z;
            z.m = N; z.n = Nmu; z.k = M; z.nb1 = W;
            z.A.ptr = f.Theta[s]; z.A.op = OP_T; z.A.ld = N; z.A.s1 = (int64_t)M * N;
            z.B.ptr = wk->ham->X; z.B.real = true; z.B.ld = Nmu;
            z.C = f.Z[s]; z.ldc = Nmu; z.sc1 = (int64_t)N * Nmu;
            zgemm(z, st);
            if (measure) {
                for (int w0 = 0; w0 < W; w0 += f.thc_wc) {
                    const int wc = std::min(f.thc_wc, W - w0);
                    GemmArgs g;
                    g.m = Nmu; g.n = Nmu; g.k = N; g.nb1 = wc;
                    g.A.ptr = f.Yt[s]; g.A.op = OP_T; g.A.ld = Nmu;
                    g.B.ptr = f.Z[s] + (int64_t)w0 * N * Nmu; g.B.ld = Nmu; g.B.s1 = (int64_t)N * Nmu;
                    g.C = f.Tthc; g.ldc = Nmu; g.sc1 = (int64_t)Nmu * Nmu;
                    zgemm(g, st);
                    thc_exchange(f.Tthc, wc, Nmu, wk->ham->Mk, f.gs[s] + (int64_t)w0 * Nmu, f.ex[s] + w0, st);
                }
            } else {
                thc_gdiag(f.Yt[s], f.Z[s], W, N, Nmu, f.gs[s], st);
            }
            GemmArgs t;
            t.m = W; t.n = nch; t.k = Nmu;
            t.A.ptr = f.gs[s]; t.A.ld = Nmu;
            t.B.ptr = wk->ham->U; t.B.real = true; t.B.ld = nch;
            t.C = f.t[s]; t.ldc = nch;
            zgemm(t, st);
        } else if (measure) {
            for (int n0 = 0; n0 < nch; n0 += f.nc) {
                const int nc = std::min(f.nc, nch - n0);
                GemmArgs g;   // T[c][w] = Lt_{n0+c} Theta_w
                g.m = N; g.n = N; g.k = M; g.nb1 = nc; g.nb2 = W;
                g.A.real = wk->Lt_real;
                g.A.ptr = wk->Lt_real
                              ? (const void*)(static_cast<const double*>(Lt) + (int64_t)n0 * N * M)
                              : (const void*)(static_cast<const cplx*>(Lt) + (int64_t)n0 * N * M);
                g.A.ld = M; g.A.s1 = (int64_t)N * M; g.A.s2 = 0;
                g.B.ptr = f.Theta[s]; g.B.ld = N; g.B.s1 = 0; g.B.s2 = (int64_t)M * N;
                g.C = f.T; g.ldc = N; g.sc1 = (int64_t)W * N * N; g.sc2 = (int64_t)N * N;
                zgemm(g, st);
                trace_terms(f.T, nc, W, N, n0, f.t[s], f.X[s], nch, st);
            }
        } else {
            // force bias only: t[w][n] = sum_{k,a} Theta_w[k][a] LtT_n[k][a]
            GemmArgs g;
            g.m = W; g.n = nch; g.k = M * N;
            g.A.ptr = f.Theta[s]; g.A.op = OP_N; g.A.ld = (int64_t)M * N;
            g.B.real = wk->Lt_real; g.B.ptr = LtT; g.B.op = OP_T; g.B.ld = (int64_t)M * N;
            g.C = f.t[s]; g.ldc = nch;
            zgemm(g, st);
        }
        if (s == 1 && wk->ev1 && timed) { cudaEventRecord(wk->ev1, st); wk->ev_valid = true; }
    }
    add_logdet(f.ld[0], f.ld[1], logS_out, W, st);
    LocalEnergyArgs a;
    a.W = W; a.M = M; a.Nchol = nch; a.Nup = wk->N[0]; a.Ndn = wk->N[1];
    for (int s = 0; s < 2; ++s) {
        a.ht[s] = f.ht[s] + (int64_t)I * M * wk->N[s]; a.Theta[s] = f.Theta[s]; a.t[s] = f.t[s];
        a.X[s] = measure && wk->ham->Nmu == 0 ? f.X[s] : nullptr;
        a.exch[s] = measure && wk->ham->Nmu > 0 ? f.ex[s] : nullptr;
    }
    a.E0 = wk->ham->E0; a.tau = wk->tau;
    a.fb_cap = wk->opts.weight_mode == AFQMC_WEIGHT_FREE ? 0.0 : wk->opts.fb_cap;
    a.E_L = E_out; a.xbar = wk->xbar; a.flags = le_flags;
    local_energy_forcebias(a, st);
}

// Multi-determinant trial (Sec. V, NOMSD): each determinant alone at the first W walkers, with
// the determinants as an extra GEMM batch dimension.  Per chunk of nd determinants and per spin,
// one batched GEMM over (determinant, walker) forms every overlap Psi_I^+ Phi_w, one batched
// inverse covers all nd W of them, one GEMM forms every Theta_{I,w}, and the energy GEMM runs
// over (Cholesky chunk, determinant, walker) with one trace pass; then one local-energy pass
// over all (determinant, walker) pairs (each group of W walkers reading its determinant's
// Psi^+ h).  Results: log-overlaps msd_ls, local energies msd_E and spin-summed traces msd_t,
// each [ND][wk->W].
void measure_msd(afqmc_walkers* wk, bool measure, int W, cudaStream_t st) {
    Fp64Buffers& f = wk->f;
    const int M = wk->M, nch = wk->Nchol, ND = wk->ND, Wld = wk->W;
    const bool dense = W == Wld;   // (determinant, walker) pairs contiguous in the [ND][W] outputs
    for (int I0 = 0; I0 < ND; I0 += f.msd_nd) {
        const int nd = std::min(f.msd_nd, ND - I0);
        for (int s = 0; s < 2; ++s) {
            const int N = wk->N[s];
            const int64_t mn = (int64_t)M * N, nn = (int64_t)N * N, ltI = (int64_t)nch * mn;
            GemmArgs g;   // S[I][w] = Psi_I^+ Phi_w
            g.m = N; g.n = N; g.k = M; g.nb1 = nd; g.nb2 = W;
            g.A.ptr = f.Psi[s] + I0 * mn; g.A.op = OP_C; g.A.ld = N; g.A.s1 = mn;
            g.B.ptr = f.Phi[s]; g.B.ld = N; g.B.s2 = mn;
            g.C = f.S[s]; g.ldc = N; g.sc1 = (int64_t)W * nn; g.sc2 = nn;
            zgemm(g, st);
            batched_inverse_logdet(f.S[s], nn, N, nd * W, f.ld[s], true, f.msd_flag, st);
            GemmArgs t;   // Theta[I][w] = Phi_w S[I][w]^-1
            t.m = M; t.n = N; t.k = N; t.nb1 = nd; t.nb2 = W;
            t.A.ptr = f.Phi[s]; t.A.ld = N; t.A.s2 = mn;
            t.B.ptr = f.S[s]; t.B.ld = N; t.B.s1 = (int64_t)W * nn; t.B.s2 = nn;
            t.C = f.Theta[s]; t.ldc = N; t.sc1 = (int64_t)W * mn; t.sc2 = mn;
            zgemm(t, st);
            const size_t esz = wk->Lt_real ? sizeof(double) : sizeof(cplx);
            const char* Lt = static_cast<const char*>(f.Lt[s]) + esz * (size_t)(I0 * ltI);
            const char* LtT = static_cast<const char*>(f.LtT[s]) + esz * (size_t)(I0 * ltI);
            if (measure) {
                for (int n0 = 0; n0 < nch; n0 += f.nc) {
                    const int nc = std::min(f.nc, nch - n0);
                    GemmArgs e;   // T[c][I][w] = Lt_{I, n0+c} Theta_{I,w}
                    e.m = N; e.n = N; e.k = M; e.nb0 = nc; e.nb1 = nd; e.nb2 = W;
                    e.A.real = wk->Lt_real;
                    e.A.ptr = Lt + esz * (size_t)((int64_t)n0 * N * M);
                    e.A.ld = M; e.A.s0 = (int64_t)N * M; e.A.s1 = ltI;
                    e.B.ptr = f.Theta[s]; e.B.ld = N; e.B.s1 = (int64_t)W * mn; e.B.s2 = mn;
                    e.C = f.T; e.ldc = N; e.sc0 = (int64_t)nd * W * nn; e.sc1 = (int64_t)W * nn; e.sc2 = nn;
                    zgemm(e, st);
                    trace_terms(f.T, nc, nd * W, N, n0, f.t[s], f.X[s], nch, st);
                }
            } else {
                GemmArgs b;   // force bias only: t[I][w][n] = sum_{k,a} Theta_{I,w}[k][a] LtT_{I,n}[k][a]
                b.m = W; b.n = nch; b.k = M * N; b.nb1 = nd;
                b.A.ptr = f.Theta[s]; b.A.ld = mn; b.A.s1 = (int64_t)W * mn;
                b.B.real = wk->Lt_real; b.B.ptr = LtT; b.B.op = OP_T; b.B.ld = mn; b.B.s1 = ltI;
                b.C = f.t[s]; b.ldc = nch; b.sc1 = (int64_t)W * nch;
                zgemm(b, st);
            }
        }
        LocalEnergyArgs a;
        a.W = nd * W; a.M = M; a.Nchol = nch; a.Nup = wk->N[0]; a.Ndn = wk->N[1];
        for (int s = 0; s < 2; ++s) {
            a.ht[s] = f.ht[s] + (int64_t)I0 * M * wk->N[s]; a.Theta[s] = f.Theta[s]; a.t[s] = f.t[s];
            a.X[s] = measure ? f.X[s] : nullptr;
            a.ht_stride[s] = (int64_t)M * wk->N[s];
        }
        a.wper = W;
        a.E0 = wk->ham->E0; a.tau = wk->tau; a.fb_cap = 0.0;
        a.E_L = dense ? f.msd_E + (int64_t)I0 * Wld : f.msd_Es;
        a.xbar = nullptr;   // the force bias comes from the combination
        a.flags = f.msd_flag + 1;
        local_energy_forcebias(a, st);
        if (dense) {
            add_logdet(f.ld[0], f.ld[1], f.msd_ls + (int64_t)I0 * Wld, nd * W, st);
            cplx_add(f.t[0], f.t[1], f.msd_t + (int64_t)I0 * Wld * nch, (int64_t)nd * W * nch, st);
        } else {
            for (int I = 0; I < nd; ++I) {
                add_logdet(f.ld[0] + (int64_t)I * W, f.ld[1] + (int64_t)I * W, f.msd_ls + (int64_t)(I0 + I) * Wld, W,
                           st);
                cplx_add(f.t[0] + (int64_t)I * W * nch, f.t[1] + (int64_t)I * W * nch,
                         f.msd_t + (int64_t)(I0 + I) * Wld * nch, (int64_t)W * nch, st);
            }
            if (measure)
                cudaMemcpy2DAsync(f.msd_E + (int64_t)I0 * Wld, sizeof(cplx) * Wld, f.msd_Es, sizeof(cplx) * W,
                                  sizeof(cplx) * W, nd, cudaMemcpyDeviceToDevice, st);
        }
    }
}

}  // namespace

int fp64_measure(afqmc_walkers* wk, bool measure, cudaStream_t st, int Wm) {
    const int W = Wm > 0 ? Wm : wk->W;
    if (wk->ND == 1) {
        measure_det(wk, 0, measure, W, wk->logS_old, wk->E_L, wk->flags, wk->flags, st);
        return AFQMC_OK;
    }
    // multi-determinant trial: every determinant alone (batched), then the overlap-weighted
    // combination.  A determinant with an exactly zero overlap has a non-finite term of weight
    // zero: its local-energy status goes to a discarded word, and the combination checks the
    // result.
    Fp64Buffers& f = wk->f;
    const int nch = wk->Nchol;
    cudaMemsetAsync(f.msd_flag, 0, sizeof(unsigned), st);
    measure_msd(wk, measure, W, st);
    MsdArgs a;
    a.W = W; a.ND = wk->ND; a.Nchol = nch; a.ldw = wk->W;
    a.cc = f.msd_cc; a.ls = f.msd_ls; a.E = measure ? f.msd_E : nullptr; a.t = f.msd_t;
    a.tau = wk->tau;
    a.fb_cap = wk->opts.weight_mode == AFQMC_WEIGHT_FREE ? 0.0 : wk->opts.fb_cap;
    a.logS = wk->logS_old; a.E_L = wk->E_L; a.xbar = wk->xbar;
    a.inv_flags = f.msd_flag; a.flags = wk->flags;
    msd_combine(a, st);
    return AFQMC_OK;
}

int fp64_propagate_and_weight(afqmc_walkers* wk, const double* x, cudaStream_t st) {
    Fp64Buffers& f = wk->f;
    const int M = wk->M, W = wk->W, nch = wk->Nchol;
    hs_coefficients(x, wk->xbar, wk->weight, W, nch, wk->coef, wk->flags, st);
    if (wk->ham->Nmu > 0) {   // THC: A_w = X diag(U c_w) X^T
        const int Nmu = wk->ham->Nmu;
        GemmArgs d;   // dv = c U^T   [W][Nmu]
        d.m = W; d.n = Nmu; d.k = nch;
        d.A.ptr = wk->coef; d.A.ld = nch;
        d.B.ptr = wk->ham->U; d.B.real = true; d.B.op = OP_T; d.B.ld = nch;
        d.C = f.dv; d.ldc = Nmu;
        zgemm(d, st);
        for (int w0 = 0; w0 < W; w0 += f.thc_wc) {
            const int wc = std::min(f.thc_wc, W - w0);
            thc_scale_columns(wk->ham->X, f.dv + (int64_t)w0 * Nmu, wc, M, Nmu, f.XD, st);
            GemmArgs g;
            g.m = M; g.n = M; g.k = Nmu; g.nb1 = wc;
            g.A.ptr = f.XD; g.A.ld = Nmu; g.A.s1 = (int64_t)M * Nmu;
            g.B.ptr = wk->ham->X; g.B.real = true; g.B.op = OP_T; g.B.ld = Nmu;
            g.C = f.A + (int64_t)w0 * M * M; g.ldc = M; g.sc1 = (int64_t)M * M;
            zgemm(g, st);
        }
    } else {   // A_w = sum_n c[w][n] L_n
        GemmArgs g;
        g.m = W; g.n = M * M; g.k = nch;
        g.A.ptr = wk->coef; g.A.ld = nch;
        g.B.ptr = wk->ham->L; g.B.real = !wk->ham->cplx_L; g.B.ld = (int64_t)M * M;
        g.C = f.A; g.ldc = (int64_t)M * M;
        zgemm(g, st);
    }
    const double sq = sqrt(wk->tau);
    for (int s = 0; s < 2; ++s) {
        const int N = wk->N[s];
        const int64_t mn = (int64_t)M * N;
        cplx* P0 = f.Pa[s];
        cplx* P1 = f.Pb[s];
        GemmArgs g;   // P0 = B Phi
        g.m = M; g.n = N; g.k = M; g.nb1 = W;
        g.A.ptr = f.Bh; g.A.real = !wk->ham->cplx_L; g.A.ld = M;
        g.B.ptr = f.Phi[s]; g.B.ld = N; g.B.s1 = mn;
        g.C = P0; g.ldc = N; g.sc1 = mn;
        zgemm(g, st);
        cudaMemcpyAsync(f.Pnew[s], P0, sizeof(cplx) * W * mn, cudaMemcpyDeviceToDevice, st);
        for (int k = 1; k <= wk->opts.k_taylor; ++k) {
            GemmArgs t;   // P1 = (i sqrt(tau) / k) A_w P0 ;  Pnew += P1
            t.m = M; t.n = N; t.k = M; t.nb1 = W;
            t.A.ptr = f.A; t.A.ld = M; t.A.s1 = (int64_t)M * M;
            t.B.ptr = P0; t.B.ld = N; t.B.s1 = mn;
            t.alpha = cplx{0.0, sq / k};
            t.C = P1; t.ldc = N; t.sc1 = mn;
            t.D = f.Pnew[s]; t.ldd = N; t.sd1 = mn;
            zgemm(t, st);
            std::swap(P0, P1);
        }
        GemmArgs b2;  // Phi' = B Pnew  -> Pa
        b2.m = M; b2.n = N; b2.k = M; b2.nb1 = W;
        b2.A.ptr = f.Bh; b2.A.real = !wk->ham->cplx_L; b2.A.ld = M;
        b2.B.ptr = f.Pnew[s]; b2.B.ld = N; b2.B.s1 = mn;
        b2.C = f.Pa[s]; b2.ldc = N; b2.sc1 = mn;
        zgemm(b2, st);
        if (wk->ND == 1) {
            overlap(f.Psi[s], f.Pa[s], f.S[s], M, N, W, st);
            batched_inverse_logdet(f.S[s], (int64_t)N * N, N, W, f.ld[s], false, wk->flags, st);
        }
    }
    if (wk->ND == 1) {
        add_logdet(f.ld[0], f.ld[1], wk->logS_new, W, st);
    } else {   // log <psi_T|Phi'> over the determinants
        cudaMemsetAsync(f.msd_flag, 0, sizeof(unsigned), st);
        for (int I0 = 0; I0 < wk->ND; I0 += f.msd_nd) {   // determinants batched with the walkers
            const int nd = std::min(f.msd_nd, wk->ND - I0);
            for (int s = 0; s < 2; ++s) {
                const int N = wk->N[s];
                const int64_t mn = (int64_t)M * N, nn = (int64_t)N * N;
                GemmArgs g;   // S[I][w] = Psi_I^+ Phi'_w
                g.m = N; g.n = N; g.k = M; g.nb1 = nd; g.nb2 = W;
                g.A.ptr = f.Psi[s] + I0 * mn; g.A.op = OP_C; g.A.ld = N; g.A.s1 = mn;
                g.B.ptr = f.Pa[s]; g.B.ld = N; g.B.s2 = mn;
                g.C = f.S[s]; g.ldc = N; g.sc1 = (int64_t)W * nn; g.sc2 = nn;
                zgemm(g, st);
                batched_inverse_logdet(f.S[s], nn, N, nd * W, f.ld[s], false, f.msd_flag, st);
            }
            add_logdet(f.ld[0], f.ld[1], f.msd_ls + (int64_t)I0 * W, nd * W, st);
        }
        MsdArgs a;
        a.W = W; a.ND = wk->ND; a.Nchol = nch; a.ldw = W;
        a.cc = f.msd_cc; a.ls = f.msd_ls; a.E = nullptr; a.t = nullptr;
        a.tau = wk->tau; a.fb_cap = 0.0;
        a.logS = wk->logS_new; a.E_L = nullptr; a.xbar = nullptr;
        a.inv_flags = f.msd_flag; a.flags = wk->flags;
        msd_combine(a, st);
    }
    WeightArgs a;
    a.W = W; a.Nchol = nch; a.mode = wk->opts.weight_mode;
    a.x = x; a.xbar = wk->xbar; a.logS_old = wk->logS_old; a.logS_new = wk->logS_new;
    a.E_L = wk->E_L; a.ebound = 2.0 / sqrt(wk->tau);
    a.tau = wk->tau; a.E_T = wk->E_T; a.E0 = wk->ham->E0;
    a.weight = wk->weight; a.accept = wk->accept;
    weight_update(a, st);
    for (int s = 0; s < 2; ++s)
        commit_walkers(f.Phi[s], f.Pa[s], wk->accept, W, (int64_t)M * wk->N[s], st);
    return AFQMC_OK;
}

int fp64_qr(afqmc_walkers* wk, cudaStream_t st) {
    for (int s = 0; s < 2; ++s)
        qr_reorthonormalise(wk->f.Phi[s], (int64_t)wk->M * wk->N[s], wk->M, wk->N[s], wk->W, wk->weight, st);
    return AFQMC_OK;
}

}  // namespace afqmc
