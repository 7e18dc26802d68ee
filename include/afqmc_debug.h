/*
 * afqmc_debug.h -- diagnostic entry points of the GB300 AFQMC library.
 *
 * They expose single building blocks of the mixed-precision walker step so the test
 * suite can check each against a plain reference in isolation.  Host pointers only;
 * every call allocates its own device buffers, runs on the legacy default stream and
 * synchronises before returning.  Return AFQMC_OK or a negative AFQMC_ERR_* code
 * (messages via afqmc_last_error()).
 */
#ifndef AFQMC_GB300_DEBUG_H
#define AFQMC_GB300_DEBUG_H

#ifdef __cplusplus
extern "C" {
#endif

/* C[b] = A[b] B[b]^T for A [nbatch][rows][K], B [nbatch][cols][K] (float64, host), computed
 * by the tcgen05 split-bf16 GEMM and returned as float64 C [nbatch][rows][cols].
 * exact = 0: plain split (hi = bf16(x), lo = bf16(x - hi)), all three products in one fp32
 *            accumulator; BN = 128 or 256.
 * exact = 1: row-scaled split (hi an integer in [-128, 128] times a per-row power of two),
 *            hi*hi summed exactly in its own accumulator; BN must be 128 and K <= 1024.
 * K must be a multiple of 8.  This is the contraction primitive behind every dense product
 * of the step (Sec. V; Table II costs). */
int afqmc_debug_split_gemm(const double* A, const double* B, int nbatch, int rows, int cols, int K, int BN,
                           int exact, double* C);

/* The fused energy contraction on its own (row-scaled operands, exact leading product;
 * terms = 3: hi*hi + hi*lo + lo*hi, terms = 4: + lo*lo):
 * for Lt [Nchol][Np][M] (real) and walker-spin
 * Green's functions ThetaT [nws][2][Np][M] (re plane then im plane of Theta^T), returns
 * t [nws][Nchol] = Tr(Lt_n Theta_ws) and X [nws][Nchol] = Tr((Lt_n Theta_ws)^2) as complex
 * (interleaved float64).  Np in {32, 64, 128}, M % 64 == 0.  These traces give the force
 * bias and the Coulomb / exchange energies of the mixed estimator. */
int afqmc_debug_energy(const double* Lt, const double* ThetaT, int Np, int Nchol, int nws, int M, int terms,
                       double* t, double* X);

/* Intermediates of one measurement of a BF16X3 walker set (wk from afqmc_init_walkers with
 * AFQMC_PREC_BF16X3): runs the overlap / Green's function / energy contractions on the
 * current walkers and copies out, as float64 (host pointers, any may be NULL):
 *   ST     [W][2][2][N][N]  overlap transposed, planar: ST[w][s][c][b][a] = (re|im) S[a][b]
 *   Sinv   [W][2][N][N]     complex inverse of S
 *   ThetaT [W][2][2][N][M]  Theta^T per walker, spin, re/im plane (Theta = Phi (Psi^T Phi)^-1)
 *   t, X   [W][2][Nchol]    complex traces Tr(Ltilde_n Theta), Tr((Ltilde_n Theta)^2)
 *   E1     [W]              complex one-body energy sum_s Tr(Psi_s^T h Theta_s) */
typedef struct afqmc_walkers* afqmc_wk_debug_t;

/* Launch-shape knobs of the calling thread's later tensor-core launches (0 = default):
 * grid_cap = most CTAs per persistent launch, bn_max = 128 to narrow plain GEMM tiles,
 * energy_bk = 16 or 32, the K chunk of the fused energy kernel.  For tuning experiments;
 * results do not depend on them. */
int afqmc_debug_set_launch_policy(int grid_cap, int bn_max, int energy_bk);
int afqmc_debug_mixed_terms(afqmc_wk_debug_t wk, double* ST, double* Sinv, double* ThetaT, double* t, double* X,
                            double* E1);

#ifdef __cplusplus
}
#endif

#endif
