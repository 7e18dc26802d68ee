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
 * by the tcgen05 split-bf16 GEMM (each operand rounded to a bf16 hi + lo pair, three
 * products, fp32 accumulation) and returned as float64 C [nbatch][rows][cols].
 * BN = 128 or 256 (tile width).  K must be a multiple of 8.  This is the contraction
 * primitive behind every dense product of the step (Sec. V; Table II costs). */
int afqmc_debug_split_gemm(const double* A, const double* B, int nbatch, int rows, int cols, int K, int BN,
                           double* C);

/* The fused energy contraction on its own: for Lt [Nchol][Np][M] (real) and walker-spin
 * Green's functions ThetaT [nws][2][Np][M] (re plane then im plane of Theta^T), returns
 * t [nws][Nchol] = Tr(Lt_n Theta_ws) and X [nws][Nchol] = Tr((Lt_n Theta_ws)^2) as complex
 * (interleaved float64).  Np in {32, 64, 128}, M % 64 == 0.  These traces give the force
 * bias and the Coulomb / exchange energies of the mixed estimator. */
int afqmc_debug_energy(const double* Lt, const double* ThetaT, int Np, int Nchol, int nws, int M, double* t,
                       double* X);

#ifdef __cplusplus
}
#endif

#endif
