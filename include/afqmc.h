/*
 * afqmc.h -- C ABI of the GB300 (sm_103a) phaseless-AFQMC walker step.
 *
 * The operation is the batched walker step of phaseless auxiliary-field QMC for
 * the Hamiltonian of Sec. V, Eq. (1),
 *     H = sum_ij h_ij c+_i c_j + 1/2 sum_ijkl v_ijkl c+_i c+_j c_l c_k + E0,
 * with the two-electron tensor given by the modified-Cholesky factorisation of
 * Sec. V, Eq. (3),  v_ijkl = sum_n L^n_ik L^n*_lj  (Nchol = x_c M vectors; the
 * paper notes that any 3-index tensor of this form is accepted).  The step
 * itself (overlap, half-rotated Green's function, force bias, HS propagator,
 * local energy, phaseless weights, QR) is the algorithm the paper cites for its
 * AFQMC implementation (Zhang & Krakauer 2003; Motta & Zhang 2018); Table II
 * gives its dense 3-index costs: O(N M^2) propagation and O(x_c N^2 M^2) energy
 * per walker.
 *
 * Conventions for every entry point
 *   - Return value: AFQMC_OK (0) or a negative AFQMC_ERR_* code.  No exception
 *     crosses the ABI.  afqmc_last_error() gives a message for the calling
 *     thread's last failure.
 *   - Pointers: any data pointer may be host memory (pageable or pinned) or
 *     device memory of the current device.  The library tells them apart with
 *     cudaPointerGetAttributes.  Inputs are copied (caller keeps ownership and
 *     may free them when the call returns).  Device outputs are written
 *     asynchronously on `stream`; host outputs are complete when the call
 *     returns (the call synchronises `stream`).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All device
 *     work of a call is ordered on it.
 *   - Layouts are row-major and contiguous.  "complex" means interleaved
 *     (re, im) pairs of doubles, i.e. numpy complex128 / C double _Complex.
 *   - Handles own their device memory; destroy them with the matching
 *     afqmc_destroy_* call.  A handle must not be used from two threads at once.
 */
#ifndef AFQMC_GB300_H
#define AFQMC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define AFQMC_OK               0
#define AFQMC_ERR_BADARG      -1  /* null handle/pointer, bad option value      */
#define AFQMC_ERR_SHAPE       -2  /* sizes out of the supported range           */
#define AFQMC_ERR_OOM         -3  /* device allocation failed                   */
#define AFQMC_ERR_NONFINITE   -4  /* NaN/Inf met in an input or a result        */
#define AFQMC_ERR_SINGULAR    -5  /* trial/walker overlap is exactly singular   */
#define AFQMC_ERR_TIMEOUT     -6  /* a bounded device wait gave up              */
#define AFQMC_ERR_CUDA        -7  /* a CUDA runtime call failed                 */
#define AFQMC_ERR_UNSUPPORTED -8  /* valid request the library does not handle  */

/* ---- options ----------------------------------------------------------- */
#define AFQMC_PREC_FP64    0  /* every contraction in FP64 (DFMA)                       */
#define AFQMC_PREC_BF16X3  1  /* contractions on tcgen05 tensor cores (kind::f16, FP32
                                 accumulation) on operands split into row-scaled fp16
                                 slices whose leading products sum exactly: two slices
                                 for the Green's function and the energy, three for the
                                 overlap, the propagation and the QR's Gram matrix and
                                 R^-1 product (see energy_terms for the energy's split
                                 products); the overlap inverse and the QR's Cholesky
                                 factor in float pairs with FP64 pivots, square roots and
                                 log-determinants; reductions and weights in FP64      */

#define AFQMC_WEIGHT_PHASELESS 0  /* w <- w |I| max(0, cos dtheta)  (hybrid form)        */
#define AFQMC_WEIGHT_FREE      1  /* free projection: complex weights, no cap, no cos   */
#define AFQMC_WEIGHT_LOCAL     2  /* local energy: w <- w exp(-tau (E_b - E_T)) max(0, cos dtheta),
                                     E_b = Re E_L of the pre-step walker clipped to E_T +- 2/sqrt(tau);
                                     measures E_L every step                                   */

typedef struct afqmc_opts {
    int    precision;    /* AFQMC_PREC_*                                           */
    int    k_taylor;     /* order K of the Taylor series for exp(i sqrt(tau) A), 1..32 */
    int    k_qr;         /* re-orthonormalise every k_qr steps (0 = never)         */
    int    weight_mode;  /* AFQMC_WEIGHT_*                                          */
    double fb_cap;       /* cap |xbar_n| <= fb_cap per component (<= 0: no cap)    */
    int    walker_offset;/* global index of walker 0 in the Philox counter (>= 0): a
                            population split over processes as consecutive walker
                            ranges draws exactly the fields of the whole population  */
    int    energy_terms; /* BF16X3 energy contraction's split products, with the
                            row-scaled operands y = x / scale, hi = rint(y),
                            lo = fp16(y - hi):
                            2 = hi*hi + r*lo + lo*hi, r = fp16(y) of Ltilde_n: three
                                products whose r carries the leading part of lo*lo
                                (the accuracy of four);
                            0 (default) = as 2, except for the smallest Cholesky
                                vectors, whose squared norms ||Ltilde_n||_F^2 add up
                                to at most 2^-15 of the total: their tiles form the
                                one product r*r', r' = fp16(y) of Theta (relative
                                error ~2^-11 on a share ~2^-15 of the energy; the
                                CTA-pair kernel, the default form, does this);
                            3 = hi*hi + hi*lo + lo*hi;
                            4 = + lo*lo for every Cholesky vector;
                            1 = adaptive: four products except for the smallest
                                vectors whose norms ||Ltilde_n||_F add up to at most
                                1% of the total, three for those                     */
    int    reserved[6];  /* must be zero                                           */
} afqmc_opts;

/* Fills the defaults: FP64, K = 6, k_qr = 5, phaseless, fb_cap = 1.0. */
void afqmc_default_opts(afqmc_opts* opts);

typedef struct afqmc_ham*     afqmc_ham_t;
typedef struct afqmc_walkers* afqmc_wk_t;

/* ---- Hamiltonian (Sec. V, Eqs. (1) and (3)) ----------------------------
 * h     [M][M]        real symmetric one-body matrix h_ij.
 * L     [Nchol][M][M] real Cholesky vectors L^n_ik, each symmetric
 *                     (v_ijkl = sum_n L^n_ik L^n_jl).
 * E0    constant energy (E_II of Eq. (1)).
 * Sizes: 1 <= M <= 1024, 1 <= Nchol.
 * The library keeps FP64 copies of h and L, forms h' = h - 1/2 sum_n L_n L_n^T
 * and the split-precision copies the tensor-core path needs on first use.
 * Errors: BADARG (null), SHAPE, NONFINITE (NaN/Inf in h or L), OOM, CUDA. */
int afqmc_create_hamiltonian(const double* h, const double* L, double E0, int M, int Nchol,
                             void* stream, afqmc_ham_t* out);

/* ---- Hamiltonian with general complex Cholesky vectors (Sec. V, Eq. (3)) ----
 * h     [M][M]        real symmetric one-body matrix h_ij.
 * L     [Nchol][M][M] complex128 (interleaved re, im) Cholesky vectors, any
 *                     complex matrices: v_ijkl = sum_n L^n_ik conj(L^n_lj).
 * E0    constant energy.
 * The library replaces each L_n by its Hermitian split A_n = (L_n + L_n^+)/2,
 * B_n = (L_n - L_n^+)/(2i), which gives the same two-body operator, so walker
 * sets on this Hamiltonian have 2 Nchol Cholesky vectors in the order
 * A_0, B_0, A_1, B_1, ...: caller fields x of afqmc_step are [nsteps][W][2 Nchol]
 * and Philox draws 2 Nchol fields per walker.  The one-body matrix of the
 * propagator is then the complex Hermitian h' = h - 1/2 sum_m V_m V_m^+ over the
 * split vectors V_m (= h - 1/4 sum_n (L_n L_n^+ + L_n^+ L_n)).
 * Only the FP64 path runs it: a BF16X3 walker set and afqmc_energy_backward on
 * such a walker set return UNSUPPORTED.  Device memory: 2 Nchol M^2 complex.
 * Errors: BADARG (null), SHAPE, NONFINITE (NaN/Inf in h or L), OOM, CUDA. */
int afqmc_create_hamiltonian_complex(const double* h, const double* L, double E0, int M, int Nchol,
                                     void* stream, afqmc_ham_t* out);

/* ---- Hamiltonian in tensor-hypercontraction form (Sec. V, Eqs. (4)-(6)) ----
 * h     [M][M]        real symmetric one-body matrix h_ij.
 * X     [M][Nmu]      real orbital values X_{i mu} = phi_i(r_mu) at Nmu interpolating points
 *                     (Eq. (4)).
 * Mk    [Nmu][Nmu]    real symmetric positive semidefinite Coulomb kernel M_{mu nu} between
 *                     the interpolating vectors (Eq. (6)).
 * E0    constant energy.
 * The two-electron tensor is Eq. (5): v_ijkl = sum_{mu nu} X_{i mu} X_{k mu} M_{mu nu}
 * X_{j nu} X_{l nu}.  The library factors the kernel Mk = U U^T by modified (diagonally
 * pivoted) Cholesky: each column takes the largest remaining diagonal entry (lowest index on
 * ties), and the factor stops once that entry is at most 1e-12 of the largest initial one.  Its
 * rank is the Hamiltonian's Nchol (afqmc_hamiltonian_info): afqmc_step draws, or takes from the
 * caller, Nchol fields per walker, one per column of U.  The equivalent Cholesky vectors
 * L^n = X diag(U[:, n]) X^T are never formed: the step contracts through the interpolating
 * points (per walker and spin: Z = Theta^T X, T = (Psi^+ X)^T Z, the density g_mu = T_mu mu,
 * exchange sum_{mu nu} M_{mu nu} T_{mu nu} T_{nu mu}, force bias U^T g, HS potential
 * X diag(U c) X^T), and h' = h - 1/2 X [(X^T X) o (U U^T)] X^T.  Memory: O(M Nmu + Nmu^2).
 * Only the FP64 path with a single-determinant trial runs it: BF16X3 and multi-determinant
 * walker sets, afqmc_bp_begin and afqmc_energy_backward return UNSUPPORTED.
 * Sizes: 1 <= M <= 1024, 1 <= Nmu <= 8192.  The factor runs in one CTA, O(Nmu^3) FP64.
 * Errors: BADARG (null, a kernel that is not symmetric or has no positive diagonal), SHAPE,
 * NONFINITE (NaN/Inf in h, X or Mk), OOM, CUDA. */
int afqmc_create_hamiltonian_thc(const double* h, const double* X, const double* Mk, double E0, int M, int Nmu,
                                 void* stream, afqmc_ham_t* out);

/* Sizes of a Hamiltonian: M, Nchol (fields per walker: Cholesky vectors, their Hermitian split,
 * or the rank of a THC kernel's factor) and Nmu (interpolating points of a THC Hamiltonian,
 * 0 otherwise).  Any output may be NULL.  Errors: BADARG (null handle). */
int afqmc_hamiltonian_info(afqmc_ham_t ham, int* M, int* Nchol, int* Nmu);
int afqmc_destroy_hamiltonian(afqmc_ham_t ham);

/* ---- Walker set ---------------------------------------------------------
 * Psi_up [M][Nup], Psi_dn [M][Ndn]  complex trial orbitals (single determinant
 *                                   per spin).
 * W      number of walkers (>= 1).
 * Phi0   complex [W][M*Nup + M*Ndn] initial walkers (per walker: spin-up M x Nup
 *        then spin-down M x Ndn, row-major) or NULL to start every walker at the
 *        trial.
 * tau    imaginary time step (> 0).
 * opts   NULL for defaults.
 * Sets w = 1 and E_T = E_L(trial) (the trial's own mixed energy).
 * Sizes: 1 <= Nup, Ndn <= min(M, 128).  BF16X3 additionally needs a real trial with
 * Psi_up == Psi_dn (one trial operand serves both spins), M % 64 == 0 and
 * Nchol % 8 == 0 (UNSUPPORTED otherwise); its fused
 * energy contraction further needs N % 8 == 0 and M <= 1024, so a step that measures
 * the energy of another shape returns UNSUPPORTED (steps with measure_every = 0 run;
 * afqmc_create_batch pads any shape exactly).
 * Errors: BADARG, SHAPE, UNSUPPORTED, SINGULAR (a walker with zero overlap),
 * NONFINITE, OOM, CUDA. */
int afqmc_init_walkers(afqmc_ham_t ham, const double* Psi_up, const double* Psi_dn, int Nup, int Ndn,
                       int W, const double* Phi0, double tau, const afqmc_opts* opts, void* stream,
                       afqmc_wk_t* out);

/* ---- Walker set on a multi-determinant trial (Sec. V) ----------------------
 * |psi_T> = sum_I c_I |D_I> over ND determinants, orthogonal (CI) or not (NOMSD,
 * <D_I|D_J> = S_IJ).
 * D_up [ND][M][Nup], D_dn [ND][M][Ndn]  complex orbitals of the determinants.
 * c    complex [ND] coefficients (finite, not all zero).
 * Every mixed estimate is the overlap-weighted average of the determinants' own:
 * with u_I = conj(c_I) <D_I|Phi> / <psi_T|Phi>, E_L = sum_I u_I E_L,I and the force
 * bias uses <L_n> = sum_I u_I <L_n>_I; the weights use <psi_T|Phi> (a log-sum-exp of
 * the determinants' log-overlaps).  E_T is the trial's energy shift
 * sum'_IJ conj(c_I) c_J S_IJ E_L,I(D_J) / sum'_IJ conj(c_I) c_J S_IJ over the pairs with a
 * non-singular overlap S_IJ: the variational energy of the trial when no pair of determinants
 * is orthogonal (NOMSD), a shift otherwise (orthogonal CI), since the left-out pairs' <D_I|H|D_J>
 * would need the Slater-Condon rules.  With phaseless weights E_T is a common factor, so E_mix
 * does not depend on it; with local-energy weights it also centres the clip window
 * E_T +- 2/sqrt(tau).  Without Phi0 the
 * walkers start at the determinant with the largest |c_I| (lowest index on ties).
 * Each determinant's term is formed as <D_I|Phi> times its own mixed estimate
 * (no fast updates), which needs <D_I|Phi> away from zero: orthogonal CI expansions
 * whose walkers sit exactly on the reference are ill-conditioned this way.
 * A determinant whose overlap with a walker is exactly zero contributes nothing;
 * SINGULAR is reported for a walker orthogonal to every determinant.  afqmc_energy's
 * logS is log <psi_T|Phi>; with ND = 1 the coefficient is dropped (a constant factor
 * changes no estimate) and the single-determinant path runs.
 * Other arguments, sizes and errors as afqmc_init_walkers, plus SHAPE for ND outside
 * 1..1024.  Only the FP64 path runs it: BF16X3, afqmc_energy_backward and
 * afqmc_bp_begin return UNSUPPORTED for ND > 1.  Cost per step: ND times the
 * single-determinant measurement and overlap. */
int afqmc_init_walkers_msd(afqmc_ham_t ham, int ND, const double* D_up, const double* D_dn, const double* c,
                           int Nup, int Ndn, int W, const double* Phi0, double tau, const afqmc_opts* opts,
                           void* stream, afqmc_wk_t* out);
int afqmc_destroy_walkers(afqmc_wk_t wk);

/* ---- The walker step -----------------------------------------------------
 * Runs `nsteps` phaseless steps.  Each step, for every walker with w != 0:
 *   S = Psi^+ Phi, Theta = Phi S^-1, t_n = sum_s Tr(Psi_s^+ L_n Theta_s),
 *   xbar_n = -i sqrt(tau) t_n (capped), A = sum_n (x_n - xbar_n) L_n,
 *   Phi' = B T_K(i sqrt(tau) A) B Phi with B = exp(-tau h'/2),
 *   w <- w |r e^{x.xbar - xbar.xbar/2}| e^{tau (E_T - E0)} max(0, cos arg r),
 *   r = <Psi|Phi'>/<Psi|Phi>; every k_qr-th step Phi = Q R, Phi <- Q.
 * x            fields [nsteps][W][Nchol] doubles, or NULL to draw them on the
 *              device from Philox4x32-10 keyed by `seed` (counter = (n/4,
 *              walker_offset + walker, global step index, 0), Box-Muller; see
 *              afqmc_philox_fields).
 * measure_every  if > 0, the mixed energy E_mix = sum w E_L / sum w (weights
 *              and walkers before the step's update) is measured at every step
 *              s (0-based within this call) with s % measure_every == 0 and
 *              written to E_mix_trace as complex values
 *              [ceil(nsteps / measure_every)]; 0 = no measurement.
 * Errors: BADARG, NONFINITE (NaN/Inf fields or energies), CUDA. */
int afqmc_step(afqmc_wk_t wk, int nsteps, const double* x, uint64_t seed, int measure_every,
               double* E_mix_trace, void* stream);

/* ---- Mixed-estimator local energy of the current walkers -----------------
 * E_L  complex [W] local energies <Psi|H|Phi_w>/<Psi|Phi_w>
 * w    [W] weights (real part only for free projection: see afqmc_get_walkers)
 * logS complex [W] sum_s log det(Psi_s^+ Phi_s) (imaginary part in (-pi, pi])
 * E_mix complex scalar sum_w w E_L / sum_w w
 * Any output may be NULL. */
int afqmc_energy(afqmc_wk_t wk, double* E_L, double* w, double* logS, double* E_mix, void* stream);

/* ---- Partial sums of the mixed estimator ------------------------------------
 * For a population split over processes (each holding consecutive walkers, see
 * afqmc_opts.walker_offset): E_mix of the whole population is
 * sum_r S_r / sum_r D_r over the processes r, with this walker set's partial sums
 *     S = sum_w w_w E_L,w,   D = sum_w w_w
 * (the numerator and denominator of the estimator's definition above).
 * sums [nmeas][4] doubles (host or device): (Re S, Im S, Re D, Im D) for each measurement of
 * the last afqmc_step call, in order, or for the one measurement of the last afqmc_energy
 * call.  nmeas must equal the number of measurements that call made (BADARG otherwise, and
 * after a failed call).  Formed on the device by the same FP64 reduction as E_mix; a device
 * output is written asynchronously on `stream`, so an all-reduce on that stream can follow
 * without a host round trip. */
int afqmc_mixed_sums(afqmc_wk_t wk, int nmeas, double* sums, void* stream);

/* ---- Adjoint of the local energy and log-overlap -------------------------
 * For the real loss  ell = sum_w Re(conj(dE_w) E_L,w + conj(dlogS_w) logS_w)
 * at the current walkers (Phi held fixed), writes
 *   dPsi_up [M][Nup], dPsi_dn [M][Ndn] complex: d ell/d Re Psi + i d ell/d Im Psi
 *   dL      [Nchol][M][M] real: d ell / d L^n_ik over the full (unsymmetrised)
 *           tensor.
 * dE, dlogS complex [W]; either may be NULL (treated as zero).  Theta is
 * recomputed, never stored.  Outputs may be NULL to skip them.
 * Computed in FP64 whatever the walker set's precision; UNSUPPORTED on a
 * Hamiltonian made by afqmc_create_hamiltonian_complex. */
int afqmc_energy_backward(afqmc_wk_t wk, const double* dE, const double* dlogS, double* dPsi_up,
                          double* dPsi_dn, double* dL, void* stream);

/* Comb population control (outside the step; phaseless or local-energy weights).  With
 * W_tot = sum_j w_j and the running sums c_j = w_0 + ... + w_j (FP64, left to right), new walker
 * k (k = 0..W-1) is a copy of the first walker j with c_j > (k + xi) W_tot / W (the last live
 * walker if rounding leaves none), and every new weight is W_tot / W.  A walker is copied floor
 * or ceil of W w_j / W_tot times; dead walkers are never copied.  xi in [0, 1) is the comb's one
 * random number, supplied by the caller.  idx (host or device, W ints, may be NULL) receives
 * the source walker of every new walker.  The walkers' overlaps and (BF16X3) split operands
 * are rebuilt.  Errors: BADARG (null handle, xi outside [0, 1), free-projection weights,
 * no live walker), CUDA.  The paper does not describe population control; this is the
 * standard comb, applied between steps. */
int afqmc_population_control(afqmc_wk_t wk, double xi, int* idx, void* stream);

/* The comb's selection alone, on any weight vector: w [W] real weights (host or
 * device; >= 0), xi in [0, 1) -> idx [W] (host or device) the source of every slot,
 * and *total (host or device, may be NULL) their sum, by the same kernel and rule as
 * afqmc_population_control.  A population split over processes gathers its weights,
 * runs this on every rank and moves the selected walkers between ranks.
 * Synchronises the stream.  Errors: BADARG (null pointer, xi outside [0, 1), weights
 * not summing to a positive number), SHAPE (W < 1), OOM, CUDA. */
int afqmc_comb_indices(const double* w, int W, double xi, int* idx, double* total, void* stream);

/* ---- Back-propagated one-body density matrix (Sec. V: the back-propagation
 * estimator for observables that do not commute with H) -----------------------
 * afqmc_bp_begin opens a window of nbp >= 0 steps at the current walkers: it keeps a
 * copy of them, Phi_w(0), and records for each of the next nbp steps the shifted
 * fields c_wn = x_wn - xbar_wn that drove every walker.  A window already open is
 * discarded.
 * afqmc_bp_rdm1, once exactly nbp steps have run, carries the trial back through
 * the adjoints of those steps' propagators,
 *     Psi_bp,w = B_w(1)^+ ... B_w(nbp)^+ Psi_T,
 *     B_w(k) = exp(-tau h'/2) T_K(i sqrt(tau) sum_n c_wn(k) L_n) exp(-tau h'/2),
 * and writes the one-body density matrix of each spin,
 *     G_s[i][j] = sum_w w_w <Psi_bp,w| c+_is c_js |Phi_w(0)> / <Psi_bp,w|Phi_w(0)> / sum_w w_w
 *               = sum_w w_w [Phi_w(0) (Psi_bp,w^+ Phi_w(0))^-1 Psi_bp,w^+]_ji / sum_w w_w,
 * with w the current (end-of-window) weights; walkers of weight 0 do not contribute.
 * nbp = 0 gives the mixed estimate.  The window stays open, so the call may be
 * repeated, until the next afqmc_bp_begin.
 *   rdm_up, rdm_dn  complex [M][M] (either may be NULL).
 * afqmc_population_control inside a window gives every new walker its source
 * walker's Phi_w(0) and field history; afqmc_set_walkers closes the window.
 * Precision follows the walker set: FP64 walker sets in FP64; BF16X3 walker sets on
 * the tensor cores (the forward step's three-slice propagation for the back steps,
 * three-slice GEMMs and a float-pair inverse for the estimate; ~1e-7 relative to the
 * FP64 result).  Device memory W (M (Nup + Ndn) + nbp Nchol) complex for the window
 * and ~6 W M max(Nup, Ndn) complex during afqmc_bp_rdm1 (BF16X3: about twice that).
 * Errors: BADARG (null handle, nbp < 0; for bp_rdm1: no window, fewer than nbp
 * steps recorded, or a step run after the window was complete), NONFINITE (a live
 * walker whose back-propagated overlap vanishes), OOM, CUDA. */
int afqmc_bp_begin(afqmc_wk_t wk, int nbp, void* stream);
int afqmc_bp_rdm1(afqmc_wk_t wk, double* rdm_up, double* rdm_dn, void* stream);

/* ---- Walker state (checkpoint / resume and inspection) -------------------
 * Phi  complex [W][M*Nup + M*Ndn] (layout of Phi0), w [W] (complex [W] for
 * free projection), step = global step counter (drives the Philox counter).
 * afqmc_set_walkers restores a state saved by afqmc_get_walkers; a resumed run
 * with the same seed reproduces the uninterrupted one. */
int afqmc_get_walkers(afqmc_wk_t wk, double* Phi, double* w, int64_t* step, void* stream);
int afqmc_set_walkers(afqmc_wk_t wk, const double* Phi, const double* w, int64_t step, void* stream);

/* ---- Philox fields -------------------------------------------------------
 * Writes the fields afqmc_step would draw: x [W][Nchol] for global step
 * `step` and `seed` (device or host pointer).  Counter (n/4, walker, step, 0),
 * key (seed & 0xffffffff, seed >> 32), Box-Muller on (u1, u2) =
 * ((a + 0.5) 2^-32, (b + 0.5) 2^-32): x = sqrt(-2 ln u1) (cos, sin)(2 pi u2). */
int afqmc_philox_fields(uint64_t seed, int64_t step, int W, int Nchol, double* x, void* stream);

/* ---- Batches of independent systems ----------------------------------------
 * Several independent problems -- each its own Hamiltonian (Sec. V, Eqs. (1), (3)), trial,
 * shape (M, N, Nchol) and walker count -- advanced together.  Every afqmc_batch_step step
 * replays one CUDA graph holding the whole step of every system (one chain of kernels per
 * system; the chains run as parallel graph branches, so small systems fill the GPU
 * together).  In a measuring BF16X3 step the energy contractions of all systems -- the
 * step's dominant cost -- run as one persistent tcgen05 launch over a work list of every
 * system's tiles, between the systems' Green's functions and the rest of their steps.  The
 * per-system arithmetic is exactly that of afqmc_step.
 *
 * Systems the tensor-core path cannot tile (BF16X3 with M % 64 != 0, N % 8 != 0 or
 * Nchol % 8 != 0), and every system under AFQMC_PAD_ALWAYS, are padded exactly: extra
 * orbitals on which h and every L_n vanish, one extra electron per extra orbital in the
 * trial and in every walker (S = diag(S, 1), so overlaps, Green's function block, force
 * bias and energies are unchanged), and zero Cholesky vectors up to a multiple of 8.
 * Padded shapes: N' = N rounded up to a multiple of 8 (at least 8), M' = the smallest
 * multiple of 64 >= M + N' - N, Nchol' = Nchol rounded up to a multiple of 8.  The energy
 * tiles of a system hold floor(128 / N') Cholesky vectors by floor(128 / N') walker-spins.
 * Padding needs Nup == Ndn.
 * Fields come from Philox (see afqmc_philox_fields) with key seed + s * 0x9E3779B97F4A7C15
 * (mod 2^64) for system s and the batch's global step; x[w][n] does not depend on Nchol,
 * so a padded system draws the fields of its unpadded self. */
#define AFQMC_PAD_AUTO    0   /* pad only what the precision needs                    */
#define AFQMC_PAD_ALWAYS  1   /* pad every system to the tensor-core shapes           */

typedef struct afqmc_system {
    const double* h;       /* [M][M] real symmetric                                     */
    const double* L;       /* [Nchol][M][M] real, each L_n symmetric                     */
    double E0;
    int M, Nchol;
    const double* Psi_up;  /* complex [M][Nup]                                           */
    const double* Psi_dn;  /* complex [M][Ndn]                                           */
    int Nup, Ndn;
    int W;                 /* walkers of this system (>= 1)                               */
    const double* Phi0;    /* complex [W][M*Nup + M*Ndn] or NULL (start at the trial)      */
} afqmc_system;

typedef struct afqmc_batch* afqmc_batch_t;

/* Creates every system (copies of the inputs, host or device pointers) with the common
 * tau and opts (NULL = defaults; k_qr applies to the batch's global step).
 * Errors: BADARG, SHAPE, UNSUPPORTED, SINGULAR, NONFINITE, OOM, CUDA (message names the
 * failing system). */
int afqmc_create_batch(int nsys, const afqmc_system* sys, double tau, const afqmc_opts* opts, int pad_mode,
                       void* stream, afqmc_batch_t* out);
int afqmc_destroy_batch(afqmc_batch_t b);

/* nsteps steps of every system, Philox fields (see above), E_mix measured at steps
 * s % measure_every == 0 (0 = never) into E_mix_trace, complex [nmeas][nsys]
 * (nmeas = ceil(nsteps / measure_every); NULL to skip).  Synchronises `stream` at the end
 * to read the status words.  Errors: BADARG, NONFINITE, TIMEOUT, OOM, CUDA. */
int afqmc_batch_step(afqmc_batch_t b, int nsteps, uint64_t seed, int measure_every, double* E_mix_trace,
                     void* stream);

/* afqmc_energy / afqmc_get_walkers of system `sys` (walkers in the caller's unpadded layout). */
int afqmc_batch_energy(afqmc_batch_t b, int sys, double* E_L, double* w, double* logS, double* E_mix,
                       void* stream);
int afqmc_batch_get_walkers(afqmc_batch_t b, int sys, double* Phi, double* w, int64_t* step, void* stream);

/* shape[8] = {M', N', Nchol' of system sys, graph branches, widest plain-GEMM tile,
 * persistent grid cap (0 = one CTA per SM), energy launch of a measuring BF16X3 step (1: one
 * persistent launch over every system's tiles, 0: one launch per system in its branch),
 * K chunk of that launch (16 or 32)}; kernels_per_step = kernels in the measuring step graph
 * (-1 before the first step).  Either output may be NULL. */
int afqmc_batch_info(afqmc_batch_t b, int sys, int* shape, int* kernels_per_step);

/* Autotuner: times the measuring step graph (`reps` replays after one warm-up) for a
 * coordinate search over the graph's branch count (1, 2, 4, ... up to 32), the widest
 * plain-GEMM tile (256 or 128 columns), the persistent grid size (all SMs, 1/2, 1/4) and,
 * for BF16X3, the energy launch (one multi-system launch with K chunks of 32 or 16, or one
 * launch per system),
 * keeps the fastest and restores the walkers, weights and step counters it advanced.
 * best_ms (may be NULL) = the chosen shape's time per step. */
int afqmc_batch_autotune(afqmc_batch_t b, int reps, double* best_ms, void* stream);

/* ---- Allocation-free log-overlap ---------------------------------------------
 * This entry point has no counterpart in the paper; it exists for callers that must not
 * allocate device memory when they call it -- e.g. a service that gave the whole device to
 * its own memory pool (where a cudaMalloc can fail at run time) or a latency-critical loop
 * that must stay off the allocator (which can synchronise the device).
 *
 * logS[w] = sum_s log det(Psi_s^+ Phi_s[w]) for W walkers, the same quantity afqmc_energy
 * reports, computed in FP64 (batched overlap GEMM + Gauss-Jordan log-determinant).
 *   Psi_up [M][Nup], Psi_dn [M][Ndn]  complex trial orbitals (device memory)
 *   Phi    complex [W][M*Nup + M*Ndn]  walkers in the layout of afqmc_init_walkers' Phi0
 *                                      (device memory)
 *   logS   complex [W] output (device memory), imaginary part in (-pi, pi]
 * Scratch: a fixed 16 MiB device array inside the library (every GPU that loads the library
 * holds it until the process exits); the call needs W*(Nup^2 + Ndn^2 + 2)*16 + 256 bytes of
 * it and returns AFQMC_ERR_SHAPE beyond that.  No device memory is allocated or freed.
 * The first call on a device looks up that device's scratch address (cudaGetSymbolAddress,
 * with the device current); make that first call before any stream capture.  The address is
 * kept per device together with the id of the context it belongs to; a call made after that
 * context was reset (cudaDeviceReset, or another library resetting the primary context) looks
 * the address up again, so make such a call, too, outside stream capture.
 * Every call shares the one scratch array and leaves its contents behind; calls whose device
 * work overlaps (different streams or threads on the same device) race on it, so serialise
 * them.  The call synchronises `stream` to read its status word.
 * Errors: BADARG (NULL or host pointer), SHAPE, NONFINITE, SINGULAR, CUDA. */
int afqmc_log_overlap_noalloc(const double* Psi_up, const double* Psi_dn, int Nup, int Ndn, int M, int W,
                              const double* Phi, double* logS, void* stream);

/* ---- Diagnostics -----------------------------------------------------------
 * Device time of the last afqmc_step's energy contraction (ms) and the number
 * of kernels it launched per step; -1 when unknown. */
int afqmc_last_step_stats(afqmc_wk_t wk, double* energy_kernel_ms, int* kernels_per_step);

/* Message of the calling thread's last failed call ("" if none). */
const char* afqmc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AFQMC_GB300_H */
