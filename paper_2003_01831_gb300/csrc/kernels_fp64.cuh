// Launch interfaces of the FP64 (DFMA) kernels.  Internal to the library.
#pragma once

#include "common.cuh"

namespace afqmc {

// Operand of a batched GEMM: element (row r, col c) of op(X) for batch (b0, b1, b2) is read at
//   ptr + b0*s0 + b1*s1 + b2*s2 + (op == N ? r*ld + c : c*ld + r), conjugated when op == C.
enum Op : int { OP_N = 0, OP_T = 1, OP_C = 2 };

struct GemmOperand {
    const void* ptr = nullptr;
    bool real = false;  // true: doubles, imaginary part zero
    int op = OP_N;
    int64_t ld = 0;
    int64_t s1 = 0, s2 = 0;
    int64_t s0 = 0;
};

// C[b] = alpha op(A[b]) op(B[b]) + beta C[b];  if D != null also D[b] += (that result).
// batch index b = (b0 * nb1 + b1) * nb2 + b2, nbatch = nb0 * nb1 * nb2.
struct GemmArgs {
    int m = 0, n = 0, k = 0;
    int nb1 = 1, nb2 = 1;
    GemmOperand A, B;
    cplx alpha{1.0, 0.0}, beta{0.0, 0.0};
    cplx* C = nullptr;
    int64_t ldc = 0, sc1 = 0, sc2 = 0;
    cplx* D = nullptr;
    int64_t ldd = 0, sd1 = 0, sd2 = 0;
    int nb0 = 1;
    int64_t sc0 = 0, sd0 = 0;
};

void zgemm(const GemmArgs& g, cudaStream_t st);

// In-place Gauss-Jordan inverse (with_inverse) or LU elimination (log-det only) of `count`
// complex N x N matrices at S + i*stride, partial pivoting on max |re|+|im|.  logdet[i] =
// log|det| + i arg(det) (arg wrapped to (-pi, pi]); sets FLAG_SINGULAR on an exact zero pivot.
// float_float: the register kernel's elimination in float pairs (~2^-44 relative; pivot
// reciprocals and the log-determinant stay FP64), for callers whose S is itself less exact.
void batched_inverse_logdet(cplx* S, int64_t stride, int N, int count, cplx* logdet,
                            bool with_inverse, unsigned* flags, cudaStream_t st, bool float_float = false);

// Traces of T[c][w] (N x N, chunk of Nchol entries): t = Tr T, X = Tr(T T), written to
// t_out[w*ldo + n0 + c], X_out[...].  T layout [nc][W][N][N].
void trace_terms(const cplx* T, int nc, int W, int N, int n0, cplx* t_out, cplx* X_out,
                 int64_t ldo, cudaStream_t st);

// Per walker: E_L = E0 + sum_s Tr(ht_s Theta_s) + 1/2 sum_n [(t_up + t_dn)^2 - X_up - X_dn];
// xbar_n = -i sqrt(tau) (t_up + t_dn), capped.  ht_s [N_s][M], Theta_s [W][M][N_s],
// t/X [W][Nchol] per spin.  X may be null (energy skipped, E_L untouched).
struct LocalEnergyArgs {
    int W, M, Nchol, Nup, Ndn;
    const cplx* ht[2];
    const cplx* Theta[2];
    const cplx* t[2];
    const cplx* X[2];
    // THC Hamiltonians: per-walker exchange sums sum_{mu nu} M_{mu nu} T_{mu nu} T_{nu mu} of each
    // spin, [W], in place of the per-vector X (which is then null); null otherwise
    const cplx* exch[2] = {nullptr, nullptr};
    double E0, tau, fb_cap;
    cplx* E_L;
    cplx* xbar;          // may be null: force bias not written
    unsigned* flags;
    // walkers in groups of wper sharing one trial determinant: walker w reads ht[s] +
    // (w / wper) * ht_stride[s] (wper = 0: one ht for all)
    int wper = 0;
    int64_t ht_stride[2] = {0, 0};
};
void local_energy_forcebias(const LocalEnergyArgs& a, cudaStream_t st);

// ---- tensor hypercontraction (THC, Sec. V, Eq. (5)) ----
// Diagonally pivoted (modified) Cholesky of the symmetric positive semidefinite n x n kernel
// Mk: U [n][rank] (row-major, ld = rank) with U U^T = Mk up to the stopping threshold (largest
// remaining diagonal <= rtol x largest initial one; pivot = largest remaining diagonal, lowest
// index on ties).  work: n*n + 2n doubles of device scratch.  *rank is read back (synchronises).
int thc_pivoted_cholesky(const double* Mk, int n, double rtol, double* work, double* U_out, int* rank,
                         cudaStream_t st);
// Per walker w of a chunk: g[w][mu] = T_w[mu][mu] and ex[w] = sum_{mu nu} Mk[mu][nu] T_w[mu][nu]
// T_w[nu][mu], for T [wc][Nmu][Nmu] complex (fixed summation order).
void thc_exchange(const cplx* T, int wc, int Nmu, const double* Mk, cplx* g, cplx* ex, cudaStream_t st);
// Force-bias-only densities: g[w][mu] = sum_a Yt[a][mu] Z[w][a][mu] (Yt [N][Nmu], Z [W][N][Nmu]).
void thc_gdiag(const cplx* Yt, const cplx* Z, int W, int N, int Nmu, cplx* g, cudaStream_t st);
// XD[w][i][mu] = X[i][mu] d[w][mu] for the walkers of a chunk (X real [M][Nmu]).
void thc_scale_columns(const double* X, const cplx* d, int wc, int M, int Nmu, cplx* XD, cudaStream_t st);
// out[i] = Re a[i];  out[i] = Re a[i] * b[i]
void real_part(const cplx* a, double* out, int64_t n, cudaStream_t st);
void real_part_times(const cplx* a, const double* b, double* out, int64_t n, cudaStream_t st);
// out[i] = h[i] - 0.5 * Re(R[i])
void hprime_from(const double* h, const cplx* R, double* out, int64_t n, cudaStream_t st);

// Philox4x32-10 + Box-Muller fields x[w][n] for global step `step`.
// x[w][n] for walkers w0 + w (w < W): counter (n/4, w0 + w, step, 0)
void philox_fields(uint64_t seed, int64_t step, int W, int Nchol, double* x, cudaStream_t st, int w0 = 0);
// Same fields with key params[0] + seed_add and step params[1] read from device memory
// when the kernel runs (so a captured graph draws fresh fields at every replay).
void philox_fields_dev(const int64_t* params, uint64_t seed_add, int W, int Nchol, double* x, cudaStream_t st,
                       int w0 = 0);

// c[w][n] = x[w][n] - xbar[w][n] for walkers with w != 0, else 0; flags NaN/Inf fields.
void hs_coefficients(const double* x, const cplx* xbar, const cplx* weight, int W, int Nchol,
                     cplx* c, unsigned* flags, cudaStream_t st);

// Multi-determinant trial |psi_T> = sum_I c_I |D_I> (Sec. V), ND <= kMaxDets determinants:
// per walker, <psi_T|Phi> = sum_I conj(c_I) <D_I|Phi> as a log-sum-exp of the determinants'
// log-overlaps (shifted by the largest real part), u_I = conj(c_I) <D_I|Phi> / <psi_T|Phi>,
// and, where given, E_L = sum_I u_I E_I and the force bias from t_n = sum_I u_I t_In, capped per
// component as for one determinant.  Determinants with c_I == 0 or a non-finite log-overlap
// (an exactly singular overlap) contribute nothing; a walker with no contribution at all has a
// zero overlap with the trial and sets FLAG_SINGULAR.
constexpr int kMaxDets = 1024;
struct MsdArgs {
    int W, ND, Nchol;  // walkers combined (the first W), determinants, Cholesky vectors
    int ldw;           // walker stride of the per-determinant arrays (>= W)
    const cplx* cc;    // conj(c_I) [ND]
    const cplx* ls;    // log <D_I|Phi_w> [ND][ldw]
    const cplx* E;     // E_L with trial D_I [ND][ldw], or null
    const cplx* t;     // sum over spins of t_n with trial D_I [ND][ldw][Nchol], or null
    double tau, fb_cap;
    cplx* logS;        // [W]
    cplx* E_L;         // [W] (with E)
    cplx* xbar;        // [W][Nchol] (with t)
    const unsigned* inv_flags;   // status of the per-determinant inverses: NONFINITE is passed on
    unsigned* flags;
};
void msd_combine(const MsdArgs& a, cudaStream_t st);
// out = <psi_T|H|psi_T> / <psi_T|psi_T> = sum_IJ conj(c_I) c_J S_IJ E_IJ / sum_IJ conj(c_I) c_J S_IJ
// from E_IJ (E_L of trial D_I at walker D_J) and log S_IJ = log <D_I|D_J>, both [ND][ND].
void msd_variational_energy(const cplx* cc, const cplx* E, const cplx* logS, int ND, cplx* out, cudaStream_t st);
// dst = a + b over n complex elements
void cplx_add(const cplx* a, const cplx* b, cplx* dst, int64_t n, cudaStream_t st);

// Weight update (phaseless or free) and acceptance mask.
struct WeightArgs {
    int W, Nchol, mode;
    const double* x;
    const cplx* xbar;
    const cplx* logS_old;
    const cplx* logS_new;
    double tau, E_T, E0;
    const cplx* E_L;   // local-energy mode: pre-step local energies
    double ebound;     // local-energy mode: |Re E_L - E_T| bound
    cplx* weight;      // in/out
    int* accept;       // out: 1 = take Phi'
};
void weight_update(const WeightArgs& a, cudaStream_t st);

// Comb population control: idx[k] = source walker of new walker k, *total = sum of the weights
// real parts (the new weight is total / W).  One thread, running sums left to right in FP64.
void comb_indices(const cplx* weight, int W, double xi, int* idx, double* total, cudaStream_t st);
// dst[w] = src[idx[w]] for W rows of `per` complex elements.
void gather_rows(const cplx* src, int64_t per, const int* idx, int W, cplx* dst, cudaStream_t st);
// weight[w] = total / W (real).
void equal_weights(cplx* weight, int W, const double* total, cudaStream_t st);

// Phi[w] <- Phi_new[w] where accept[w]; `per_walker` complex elements per walker.
void commit_walkers(cplx* Phi, const cplx* Phi_new, const int* accept, int W, int64_t per_walker,
                    cudaStream_t st);

// In-place Gram-Schmidt (classical, twice) of the N columns of each M x N complex matrix
// Phi[w] (row-major, stride `stride`), diag R > 0; skipped where weight == 0.
void qr_reorthonormalise(cplx* Phi, int64_t stride, int M, int N, int W, const cplx* weight,
                         cudaStream_t st);

// E_mix = sum_w w E_L / sum_w w (single block, fixed order); writes out[0].
// E_mix into out[0]; if sums is set, also (sum_w w E_L, sum_w w) into sums[0..1]
void mixed_energy(const cplx* weight, const cplx* E_L, int W, cplx* out, cudaStream_t st, cplx* sums = nullptr);

// small helpers
void fill_cplx(cplx* p, int64_t n, cplx v, cudaStream_t st);
void replicate(cplx* dst, const cplx* src, int64_t n, int copies, int64_t dst_stride, cudaStream_t st);
void real_to_cplx(const double* src, cplx* dst, int64_t n, cudaStream_t st);
void check_finite(const double* p, int64_t n, unsigned* flags, cudaStream_t st);
// h' = h - 1/2 sum_n L_n L_n^T (real, FP64)
void build_hprime(const double* h, const double* L, int M, int Nchol, double* hp, cudaStream_t st);
// h' = h - 1/2 sum_m V_m V_m^+ for Hermitian complex V [Nv][M][M] and real h (complex Hermitian h')
void build_hprime_hermitian(const double* h, const cplx* V, int M, int Nv, cplx* hp, cudaStream_t st);
// V[2n] = (L_n + L_n^+)/2, V[2n+1] = (L_n - L_n^+)/(2i) for complex L [Nchol][M][M]; V [2 Nchol][M][M]
void hermitian_split(const cplx* L, int M, int Nchol, cplx* V, cudaStream_t st);
// exp(s * X) for a real symmetric M x M matrix by scaling-and-squaring of a Taylor series (FP64).
int expm_real(const double* X, double s, int M, double* out, cudaStream_t st);
// the same for a complex M x M matrix (out must not alias X)
int expm_complex(const cplx* X, double s, int M, cplx* out, cudaStream_t st);
// max |L_n - L_n^T| > tol * max|L| sets FLAG_NONFINITE-independent flag 8
void check_symmetric(const double* L, int M, int Nchol, unsigned* flags, cudaStream_t st);

}  // namespace afqmc
