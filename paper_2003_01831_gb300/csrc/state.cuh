// Handle structures shared by the C-ABI front end and the step drivers.  Internal.
#pragma once

#include <vector>

#include "common.cuh"
#include "kernels_fp64.cuh"
#include "kernels_tc.cuh"

struct afqmc_ham {
    int device = 0;
    int M = 0, Nchol = 0;
    double E0 = 0.0;
    double* h = nullptr;    // [M][M]
    double* L = nullptr;    // [Nchol][M][M]; interleaved complex when cplx_L
    double* hp = nullptr;   // h' = h - 1/2 sum L L^+ [M][M]; interleaved complex when cplx_L
    // Built from general complex Cholesky vectors: L holds their Hermitian split (2 per input
    // vector, Nchol counts the split vectors).  Only the FP64 step supports it.
    bool cplx_L = false;
    // THC Hamiltonian (afqmc_create_hamiltonian_thc): orbital values X [M][Nmu] at the
    // interpolating points, kernel Mk [Nmu][Nmu] and its modified-Cholesky factor U [Nmu][Nchol]
    // (Nchol = its rank).  L is not formed (null); only the FP64 step runs it.
    int Nmu = 0;
    double* X = nullptr;
    double* Mk = nullptr;
    double* U = nullptr;
    unsigned* flags = nullptr;
    int live_walker_sets = 0;
};

namespace afqmc {

struct TcState;  // tensor-core buffers (kernels_tc.cu)

// Device buffers of the FP64 path.  Walkers, Green's functions and traces are kept per
// spin; complex arrays are interleaved FP64 pairs.
// Trial quantities hold one block per determinant of the trial (ND of them), the first at the
// pointer itself.
struct Fp64Buffers {
    cplx* Psi[2] = {nullptr, nullptr};     // [ND][M][N_s]
    void* Lt[2] = {nullptr, nullptr};      // Psi_s^+ L_n: [ND][Nchol][N_s][M] (double if trial real)
    void* LtT[2] = {nullptr, nullptr};     // transposed: [ND][Nchol][M][N_s] (force-bias-only path)
    cplx* ht[2] = {nullptr, nullptr};      // Psi_s^+ h: [ND][N_s][M]
    double* Bh = nullptr;                  // exp(-tau h'/2): [M][M], interleaved complex if cplx_L
    cplx* Phi[2] = {nullptr, nullptr};     // [W][M][N_s]
    cplx* Pnew[2] = {nullptr, nullptr};    // propagated walkers / Taylor accumulator
    cplx* Pa[2] = {nullptr, nullptr};      // Taylor term ping
    cplx* Pb[2] = {nullptr, nullptr};      // Taylor term pong
    cplx* S[2] = {nullptr, nullptr};       // [W][N_s][N_s] overlap, inverted in place
    cplx* ld[2] = {nullptr, nullptr};      // [W] per-spin log det
    cplx* Theta[2] = {nullptr, nullptr};   // [W][M][N_s]
    cplx* t[2] = {nullptr, nullptr};       // [W][Nchol]
    cplx* X[2] = {nullptr, nullptr};       // [W][Nchol]
    cplx* T = nullptr;                     // trace chunk [nc][W][N][N]
    int nc = 0;
    cplx* A = nullptr;                     // [W][M][M] HS potential
    // multi-determinant trial (ND > 1): per-determinant results of the current walkers
    cplx* msd_cc = nullptr;                // conj(c_I): [ND]
    cplx* msd_ls = nullptr;                // log <D_I|Phi_w>: [ND][W]
    cplx* msd_E = nullptr;                 // E_L with trial D_I: [ND][W]
    cplx* msd_t = nullptr;                 // sum_s t_n with trial D_I: [ND][W][Nchol]
    unsigned* msd_flag = nullptr;          // status of the per-determinant inverses [0], local energies [1]
    int msd_nd = 0;                        // determinants per batched chunk (S, ld, Theta, t, X hold
                                           // msd_nd x W walkers; T holds nc x msd_nd x W blocks)
    cplx* msd_Es = nullptr;                // local energies of a chunk when W < the walker count: [msd_nd][W]
    // THC Hamiltonians (Lt, LtT, T are then not allocated)
    cplx* Yt[2] = {nullptr, nullptr};      // Psi_s^+ X: [N_s][Nmu]
    cplx* Z[2] = {nullptr, nullptr};       // Theta_s^T X: [W][N_s][Nmu]
    cplx* gs[2] = {nullptr, nullptr};      // densities at the points, per spin: [W][Nmu]
    cplx* ex[2] = {nullptr, nullptr};      // exchange sums per spin: [W]
    cplx* Tthc = nullptr;                  // T = Yt^T Z for a chunk of walkers: [thc_wc][Nmu][Nmu]
    cplx* dv = nullptr;                    // U c per walker: [W][Nmu]
    cplx* XD = nullptr;                    // X diag(U c) for a chunk of walkers: [thc_wc][M][Nmu]
    int thc_wc = 0;
};

}  // namespace afqmc

struct afqmc_walkers {
    afqmc_ham* ham = nullptr;
    int device = 0;
    int M = 0, Nchol = 0, N[2] = {0, 0}, W = 0;
    int ND = 1;                       // determinants in the trial expansion
    double tau = 0.0;
    afqmc_opts opts{};
    bool trial_real = false;
    bool spin_same = false;           // Psi_up == Psi_dn exactly (checked for BF16X3 walker sets)
    bool Lt_real = false;             // Psi^+ L_n real: a real trial and real L
    double E_T = 0.0;
    int64_t step = 0;

    afqmc::Fp64Buffers f;
    afqmc::TcState* tc = nullptr;

    // shared per-walker arrays
    afqmc::cplx* weight = nullptr;    // [W]
    afqmc::cplx* logS_old = nullptr;  // [W]
    afqmc::cplx* logS_new = nullptr;  // [W]
    afqmc::cplx* E_L = nullptr;       // [W]
    afqmc::cplx* xbar = nullptr;      // [W][Nchol]
    afqmc::cplx* coef = nullptr;      // [W][Nchol]
    int* accept = nullptr;            // [W]
    double* x = nullptr;              // fields, x_cap steps of [W][Nchol]
    int x_cap = 0;
    afqmc::cplx* emix = nullptr;      // measurement trace, emix_cap entries
    afqmc::cplx* esum = nullptr;      // their partial sums (sum w E_L, sum w), 2 emix_cap entries
    int emix_cap = 0;
    int nmeas_last = 0;               // measurements made by the last step / energy call
    unsigned* flags = nullptr;

    // back-propagation window (backprop.cu): walkers at its start and the shifted fields
    // c = x - xbar of the steps recorded since
    int bp_n = -1;                    // window length in steps; -1: no window open
    int bp_k = 0;                     // steps recorded so far
    bool bp_overrun = false;          // a step ran after the window was complete
    afqmc::cplx* bp_Phi[2] = {nullptr, nullptr};   // [W][M][N_s]
    afqmc::cplx* bp_coef = nullptr;   // [bp_n][W][Nchol]

    // timing of the energy contraction (device events around it in the last step)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool ev_valid = false;
    int kernels_per_step = -1;
};

namespace afqmc {

// step drivers (step_fp64.cu / step_tc.cu)
int fp64_alloc(afqmc_walkers* wk);
void fp64_free(afqmc_walkers* wk);
// Green's function, traces, local energy and force bias at the current walkers.
// measure = compute exchange too.  Leaves logS of the current walkers in wk->logS_old.
int fp64_measure(afqmc_walkers* wk, bool measure, cudaStream_t st, int Wm = 0);
int fp64_propagate_and_weight(afqmc_walkers* wk, const double* x, cudaStream_t st);
int fp64_qr(afqmc_walkers* wk, cudaStream_t st);
int fp64_backward(afqmc_walkers* wk, const cplx* dE, const cplx* dlogS, cplx* dPsi_up, cplx* dPsi_dn,
                  double* dL, cudaStream_t st);

int tc_alloc(afqmc_walkers* wk, cudaStream_t st);
void tc_free(afqmc_walkers* wk);
int tc_measure(afqmc_walkers* wk, bool measure, cudaStream_t st);
int tc_propagate_and_weight(afqmc_walkers* wk, const double* x, cudaStream_t st);
// The measurement's phases (tc_measure = pre, the energy contraction, post) and the description
// of a walker set's energy contraction for a multi-system launch (step_tc.cu).
int tc_measure_pre(afqmc_walkers* wk, cudaStream_t st);
int tc_measure_post(afqmc_walkers* wk, bool measure, cudaStream_t st);
int tc_energy_system(afqmc_walkers* wk, int BK, afqmc::EnergySys* out);
// Phi_out = B T_K(sign i sqrt(tau) sum_n c_n L_n) B Phi_in (conj_c: with conj(c)) on the tensor
// cores, both spins, transposed planar layout [W][2][2][N][M] (step_tc.cu).
int tc_apply_propagator(afqmc_walkers* wk, const afqmc::cplx* c, bool conj_c, double sign, const double* Phi_in,
                        double* Phi_out, cudaStream_t st);
// Canonical walkers Phi[s] [W][M][N] (both spins) to / from the transposed planar layout.
void tc_canon_to_T(afqmc_walkers* wk, afqmc::cplx* const* Phi, double* out_T, cudaStream_t st);
void tc_T_to_canon(afqmc_walkers* wk, const double* in_T, afqmc::cplx* const* Phi, cudaStream_t st);
// Green's functions of a back-propagation window's estimate on the tensor cores: per walker-spin
// S = Psi_bp^+ Phi(0) (three-slice GEMM), S^-1 (float-pair Gauss-Jordan), Theta = Phi(0) S^-1
// (exact-mode GEMM), written canonical to Theta[s] [W][M][N].  QT: Psi_bp in the transposed
// planar layout; Phi0: the window's first walkers, canonical (step_tc.cu).
int tc_bp_green(afqmc_walkers* wk, const double* QT, afqmc::cplx* const* Phi0, afqmc::cplx* const* Theta,
                cudaStream_t st);
int tc_qr(afqmc_walkers* wk, cudaStream_t st);
int tc_sync_walkers_to_fp64(afqmc_walkers* wk, cudaStream_t st);
int tc_sync_walkers_from_fp64(afqmc_walkers* wk, cudaStream_t st);
int tc_debug_terms(afqmc_walkers* wk, double* ST, double* Sinv, double* ThetaT, double* t, double* X, double* E1);
int tc_energy_products(afqmc_walkers* wk, double* mean);

// back-propagation window (backprop.cu)
int bp_open(afqmc_walkers* wk, int nbp, cudaStream_t st);
void bp_close(afqmc_walkers* wk);
void bp_record(afqmc_walkers* wk, cudaStream_t st);
// after population control: every walker's window copy and history from its source idx[w];
// tmp holds at least W * max(M * max N_s, Nchol) complex elements
int bp_follow_comb(afqmc_walkers* wk, const int* idx, cplx* tmp, cudaStream_t st);

// host helpers of the C-ABI front end (afqmc_api.cu)
bool is_device_ptr(const void* p);
int copy_in(void* dst, const void* src, size_t bytes, cudaStream_t st);
// copies to a caller pointer; *needs_sync is set when the destination is host memory
int copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st, bool* needs_sync);
int read_flags(unsigned* dflags, cudaStream_t st, unsigned* out);   // synchronises st
int flags_to_error(unsigned f, const char* where);

}  // namespace afqmc
