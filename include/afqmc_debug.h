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
 * by the tcgen05 split-operand GEMM and returned as float64 C [nbatch][rows][cols].
 * exact = 0: plain split (hi = bf16(x), lo = bf16(x - hi)), all three products in one fp32
 *            accumulator; BN = 128 or 256.
 * exact = 1: row-scaled fp16 split: per row a power of two s = 2^(e-11) with ||x||_2 < 2^e,
 *            hi = rint(x/s) (an integer, |hi| <= 2048), lo = fp16(x/s - hi); hi*hi summed
 *            exactly in its own accumulator, hi*lo + lo*hi + lo*lo in a second; BN must be 128.
 * K must be a multiple of 8.  This is the contraction primitive behind every dense product
 * of the step (Sec. V; Table II costs). */
int afqmc_debug_split_gemm(const double* A, const double* B, int nbatch, int rows, int cols, int K, int BN,
                           int exact, double* C);

/* The fused energy contraction on its own (row-scaled operands y = x / scale, hi = rint(y),
 * lo = fp16(y - hi), exact leading product; terms = 3: hi*hi + hi*lo + lo*hi, terms = 4:
 * + lo*lo, terms = 5: hi*hi + r*lo + lo*hi with r = fp16(y) of Lt; terms = 6: as 5, but the
 * tiles of n-groups 4p + 2 and 4p + 3 (groups of 128/Np Cholesky vectors) form the single
 * product r*r' with r' = fp16(y) of ThetaT (the single-product tail of the library default,
 * on alternate CTA-pair tiles); terms = 7: r*r' for every tile):
 * for Lt [Nchol][Np][M] (real) and walker-spin
 * Green's functions ThetaT [nws][2][Np][M] (re plane then im plane of Theta^T), returns
 * t [nws][Nchol] = Tr(Lt_n Theta_ws) and X [nws][Nchol] = Tr((Lt_n Theta_ws)^2) as complex
 * (interleaved float64).  Np a multiple of 8 up to 128, M % 64 == 0.  These traces give the force
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

/* Batched inverse and log-determinant of count complex N x N matrices S (host, interleaved
 * float64, row-major [count][N][N]) by FP64 Gauss-Jordan elimination with partial pivoting
 * (the LU / inverse / log-det row of the walker step, Sec. V).  logdet [count] complex
 * receives log|det S| + i arg det S; with_inverse = 1 also writes the inverses to Sout (same
 * layout).  variant: 0 = the FP64 kernel the
 * FP64 step uses, 1 = the shared-memory kernel, 2 = the register kernel, 3 = the register
 * kernel with float-pair elimination (~2^-44 relative, what the BF16X3 step uses); 2 and 3
 * apply for 32 < N <= 128 with with_inverse, other cases fall back to 1.  *ms (if not NULL) receives the kernel time.
 * Returns AFQMC_ERR_SINGULAR / AFQMC_ERR_NONFINITE (logdet = -inf + 0i for such a matrix,
 * its inverse unwritten) if a pivot column is zero / not finite. */
int afqmc_debug_inverse(const double* S, int N, int count, int variant, int with_inverse, double* Sout,
                        double* logdet, float* ms);

/* The adaptive choice of energy products (afqmc_opts.energy_terms = 1) on host data: for the
 * Frobenius norms norms[n] >= 0 of the nch rotated Cholesky vectors Ltilde_n, flags[g] = 1
 * (the lo*lo product is formed) for every group g of G consecutive vectors except the groups
 * made only of the smallest vectors whose norms add up to at most eta of the total (ties:
 * lower index first), 0 for those.  ceil(nch / G) flags.  Host only, no device work; the
 * step uses eta = 0.01 and G = 128 / N. */
int afqmc_debug_select_energy_groups(const double* norms, int nch, int G, double eta, unsigned char* flags);

/* The single-product tail of the default energy products (afqmc_opts.energy_terms = 0) on host
 * data: for the squared Frobenius norms sqnorms[n] >= 0 of the nch rotated Cholesky vectors,
 * flags[g] = 1 (the group's tiles form the one product r*r') for every group g of G
 * consecutive vectors made only of the smallest vectors whose squared norms add up to at most
 * eta of the total (ties: lower index first), 0 for the others; a CTA-pair tile forms the
 * single product when both of its groups are flagged.  ceil(nch / G) flags.  Host only; the
 * step uses eta = 2^-15 and G = 128 / N. */
int afqmc_debug_select_single_groups(const double* sqnorms, int nch, int G, double eta, unsigned char* flags);

/* Tile order of the calling thread's later energy-kernel launches: the (Cholesky vector,
 * walker-spin) tiles run in windows of ws_super walker-spin groups (0 = default), sweeping
 * every Cholesky vector inside a window, so the window's Green's functions stay in L2 while
 * Ltilde streams through once per window.  For tuning experiments; results do not depend
 * on it. */
int afqmc_debug_set_energy_window(int ws_super);

/* Form of the calling process's later fused energy contractions: pair = 1 (the default),
 * clusters of two CTAs on two SMs, each pair computing two tiles of the same walker-spin group
 * with MMAs of M = 256 issued by one CTA (cta_group::2), every SM staging half of the
 * Green's-function rows; pair = 0, one CTA per 128 x 256 tile (kind::f16 MMAs of M = 128).
 * Results are the same arithmetic in the same order.  Errors: BADARG for other values. */
int afqmc_debug_set_energy_variant(int pair);

/* Electron-count padding of batches created after the call: granule 8 (default) pads each
 * system's N to the next multiple of 8 (energy tiles of floor(128 / N') walker-spins); 32 pads
 * to 32, 64 or 128.  Errors: BADARG for any other granule. */
int afqmc_debug_set_batch_padding(int granule);

/* Energy launch of a batch's later measuring BF16X3 steps (b: an afqmc_batch_t): multi = 1 one
 * persistent launch over every system's tiles with K chunks of bk (16 or 32), multi = 0 one
 * launch per system in its graph branch.  The arithmetic of every tile is the same.  Errors:
 * BADARG. */
int afqmc_debug_set_batch_energy(void* b, int multi, int bk);
int afqmc_debug_mixed_terms(afqmc_wk_debug_t wk, double* ST, double* Sinv, double* ThetaT, double* t, double* X,
                            double* E1);

/* Mean number of split products per energy tile of a BF16X3 walker set: under the default
 * (energy_terms = 0) 3 - 2 f, f the fraction of CTA-pair tiles that form the single product
 * (0 in the one-CTA form); 3 for energy_terms = 2 or 3, 4 for 4; 3 + the fraction of tiles
 * that form lo*lo under the adaptive choice (1).  The issued tensor-core flops of the energy
 * contraction are this many times the algorithmic ones.  Host only. */
int afqmc_debug_energy_products(afqmc_wk_debug_t wk, double* mean);

/* Failure detection without a fault: one warp waits, by the library's bounded mbarrier wait
 * (try_wait polled against a clock64 budget) with a budget of limit_cycles SM clock cycles
 * (1 .. the production bound of 4e9), on a barrier phase that completes only if
 * release != 0 (one thread arrives first).  *status
 * receives the status word: FLAG_TIMEOUT (4) when the wait ran out, 0 when it completed;
 * *ms (may be NULL) the kernel's duration.  The kernel returns either way, so the context
 * stays usable.  Errors: BADARG (null status, limit out of range), OOM, CUDA. */
int afqmc_debug_wait_probe(long long limit_cycles, int release, unsigned* status, float* ms);

#ifdef __cplusplus
}
#endif

#endif
