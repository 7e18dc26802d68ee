// Tensor-hypercontraction (THC) Hamiltonians on the FP64 path (Sec. V, Eqs. (4)-(6)).
//
// With orbital values X[i][mu] = phi_i(r_mu) at N_mu interpolating points and the Coulomb kernel
// M_{mu nu} between them, Eq. (5) writes v_ijkl = sum_{mu nu} X_{i mu} X_{k mu} M_{mu nu}
// X_{j nu} X_{l nu} (real orbitals).  Factoring M = U U^T (modified Cholesky of the kernel)
// turns it into Eq. (3)'s form with structured vectors L^n = X diag(U[:, n]) X^T, so the
// phaseless step runs unchanged -- but nothing of size Nchol x M^2 is ever formed:
//   * densities: with Theta = Phi S^-1 (M x N) and the half-rotated orbital values
//     Yt = Psi^+ X (N x N_mu), Z = Theta^T X (N x N_mu) and T = Yt^T Z (N_mu x N_mu) give
//     g_mu = T_{mu mu} (spin-summed: the density at r_mu) and the exchange
//     sum_{mu nu} M_{mu nu} T_{mu nu} T_{nu mu};
//   * force bias: <L_n> = sum_mu U_{mu n} g_mu;  Coulomb 1/2 sum_n <L_n>^2 = 1/2 g^T M g;
//   * HS potential: sum_n c_n L^n = X diag(U c) X^T;
//   * one-body factor: h' = h - 1/2 sum_n L^n L^nT = h - 1/2 X [(X^T X) o (U U^T)] X^T.
// Energy cost per walker and spin: 2 N M N_mu (Z) + 2 N N_mu^2 (T) complex-real products, the
// O(x_mu^2 N M^2) of Table II's THC row, against O(Nchol N^2 M) for dense Cholesky vectors.
#include <math.h>

#include <algorithm>
#include <string>

#include "kernels_fp64.cuh"

namespace afqmc {

namespace {

constexpr int kT = 256;

inline unsigned blocks(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

__device__ cplx block_sum_c(cplx v, cplx* sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) sh[t] = sh[t] + sh[t + s];
        __syncthreads();
    }
    const cplx r = sh[0];
    __syncthreads();
    return r;
}

// One CTA of 1024 threads.  Lc is column-major (column r at Lc + r n), d the remaining
// diagonal.  Step r: the pivot p is the largest remaining diagonal (lowest index on ties); if
// it is at most `stop` the factor ends; else column r = (M[:, p] - sum_{j<r} L[:, j] L[p, j]) /
// sqrt(d_p), the diagonal loses its square and d_p becomes 0.
constexpr int kCholT = 1024;
__global__ void __launch_bounds__(kCholT) pivchol_kernel(const double* Mk, int n, double rtol, double* d,
                                                         double* Lc, int* rank_out) {
    __shared__ double sv[kCholT];
    __shared__ int si[kCholT];
    __shared__ double stop_s;
    const int t = threadIdx.x;
    double m = -1.0;
    for (int i = t; i < n; i += kCholT) {
        d[i] = Mk[(int64_t)i * n + i];
        m = fmax(m, d[i]);
    }
    sv[t] = m;
    __syncthreads();
    for (int s = kCholT / 2; s > 0; s >>= 1) {
        if (t < s) sv[t] = fmax(sv[t], sv[t + s]);
        __syncthreads();
    }
    if (t == 0) stop_s = rtol * sv[0];
    __syncthreads();
    const double stop = stop_s;
    int r = 0;
    for (; r < n; ++r) {
        double bv = -INFINITY;
        int bi = n;
        for (int i = t; i < n; i += kCholT)
            if (d[i] > bv) {   // increasing i per thread: keeps the first index of a tie
                bv = d[i];
                bi = i;
            }
        sv[t] = bv;
        si[t] = bi;
        __syncthreads();
        for (int s = kCholT / 2; s > 0; s >>= 1) {
            if (t < s && (sv[t + s] > sv[t] || (sv[t + s] == sv[t] && si[t + s] < si[t]))) {
                sv[t] = sv[t + s];
                si[t] = si[t + s];
            }
            __syncthreads();
        }
        const double dp = sv[0];
        const int p = si[0];
        __syncthreads();
        if (!(dp > stop)) break;
        const double inv = 1.0 / sqrt(dp);
        double* col = Lc + (int64_t)r * n;
        for (int i = t; i < n; i += kCholT) {
            double acc = Mk[(int64_t)p * n + i];   // M[i][p] = M[p][i]
            for (int j = 0; j < r; ++j) acc -= Lc[(int64_t)j * n + i] * Lc[(int64_t)j * n + p];
            col[i] = acc * inv;
        }
        __syncthreads();
        for (int i = t; i < n; i += kCholT) d[i] -= col[i] * col[i];
        __syncthreads();
        if (t == 0) d[p] = 0.0;
        __syncthreads();
    }
    if (t == 0) *rank_out = r;
}

// U[i][j] = Lc[j n + i] for j < rank
__global__ void chol_to_rowmajor_kernel(const double* Lc, int n, int rank, double* U) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * rank) return;
    const int i = (int)(e / rank), j = (int)(e % rank);
    U[e] = Lc[(int64_t)j * n + i];
}

// One block per walker of the chunk: the exchange sum over 32 x 32 tile pairs (T[I][J] and the
// transposed T[J][I] staged in shared memory, rows read coalesced), fixed order, and the
// diagonal g.
__global__ void __launch_bounds__(kT) thc_exchange_kernel(const cplx* T, int Nmu, const double* Mk, cplx* g,
                                                          cplx* ex) {
    __shared__ cplx a[32][33];
    __shared__ cplx b[32][33];
    __shared__ cplx sh[kT];
    const int w = blockIdx.x;
    const cplx* Tw = T + (int64_t)w * Nmu * Nmu;
    const int nt = (Nmu + 31) / 32;
    cplx acc{0.0, 0.0};
    for (int I = 0; I < nt; ++I) {
        for (int J = 0; J < nt; ++J) {
            for (int e = threadIdx.x; e < 1024; e += kT) {
                const int r = e >> 5, c = e & 31;
                const int r1 = I * 32 + r, c1 = J * 32 + c;
                const int r2 = J * 32 + r, c2 = I * 32 + c;
                a[r][c] = (r1 < Nmu && c1 < Nmu) ? Tw[(int64_t)r1 * Nmu + c1] : cplx{0.0, 0.0};
                b[r][c] = (r2 < Nmu && c2 < Nmu) ? Tw[(int64_t)r2 * Nmu + c2] : cplx{0.0, 0.0};
            }
            __syncthreads();
            for (int e = threadIdx.x; e < 1024; e += kT) {
                const int r = e >> 5, c = e & 31;
                const int mu = I * 32 + r, nu = J * 32 + c;
                if (mu < Nmu && nu < Nmu) acc = acc + Mk[(int64_t)mu * Nmu + nu] * (a[r][c] * b[c][r]);
            }
            __syncthreads();
        }
    }
    acc = block_sum_c(acc, sh);
    if (threadIdx.x == 0) ex[w] = acc;
    for (int mu = threadIdx.x; mu < Nmu; mu += kT) g[(int64_t)w * Nmu + mu] = Tw[(int64_t)mu * Nmu + mu];
}

__global__ void thc_gdiag_kernel(const cplx* Yt, const cplx* Z, int N, int Nmu, cplx* g) {
    const int w = blockIdx.y;
    const int mu = blockIdx.x * blockDim.x + threadIdx.x;
    if (mu >= Nmu) return;
    const cplx* Zw = Z + (int64_t)w * N * Nmu;
    cplx acc{0.0, 0.0};
    for (int a = 0; a < N; ++a) cfma(acc, Yt[(int64_t)a * Nmu + mu], Zw[(int64_t)a * Nmu + mu]);
    g[(int64_t)w * Nmu + mu] = acc;
}

__global__ void thc_scale_columns_kernel(const double* X, const cplx* d, int wc, int M, int Nmu, cplx* XD) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)M * Nmu;
    if (e >= per * wc) return;
    const int64_t w = e / per, r = e % per;
    const int mu = (int)(r % Nmu);
    XD[e] = X[r] * d[w * Nmu + mu];
}

__global__ void real_part_kernel(const cplx* a, const double* b, double* out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = b ? a[i].re * b[i] : a[i].re;
}

__global__ void hprime_from_kernel(const double* h, const cplx* R, double* out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = h[i] - 0.5 * R[i].re;
}

}  // namespace

int thc_pivoted_cholesky(const double* Mk, int n, double rtol, double* work, double* U_out, int* rank,
                         cudaStream_t st) {
    double* d = work;
    double* Lc = work + n;
    int* dr = reinterpret_cast<int*>(work + n + (int64_t)n * n);
    count_launch();
    pivchol_kernel<<<1, kCholT, 0, st>>>(Mk, n, rtol, d, Lc, dr);
    int r = 0;
    cudaError_t e = cudaMemcpyAsync(&r, dr, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(AFQMC_ERR_CUDA, std::string("thc factor: ") + cudaGetErrorString(e));
    *rank = r;
    if (r > 0) {
        count_launch();
        chol_to_rowmajor_kernel<<<blocks((int64_t)n * r), kT, 0, st>>>(Lc, n, r, U_out);
    }
    return AFQMC_OK;
}

void thc_exchange(const cplx* T, int wc, int Nmu, const double* Mk, cplx* g, cplx* ex, cudaStream_t st) {
    if (wc <= 0) return;
    count_launch();
    thc_exchange_kernel<<<wc, kT, 0, st>>>(T, Nmu, Mk, g, ex);
}

void thc_gdiag(const cplx* Yt, const cplx* Z, int W, int N, int Nmu, cplx* g, cudaStream_t st) {
    if (W <= 0) return;
    count_launch();
    thc_gdiag_kernel<<<dim3(blocks(Nmu), W), kT, 0, st>>>(Yt, Z, N, Nmu, g);
}

void thc_scale_columns(const double* X, const cplx* d, int wc, int M, int Nmu, cplx* XD, cudaStream_t st) {
    const int64_t n = (int64_t)wc * M * Nmu;
    if (n <= 0) return;
    count_launch();
    thc_scale_columns_kernel<<<blocks(n), kT, 0, st>>>(X, d, wc, M, Nmu, XD);
}

void real_part(const cplx* a, double* out, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    real_part_kernel<<<blocks(n), kT, 0, st>>>(a, nullptr, out, n);
}

void real_part_times(const cplx* a, const double* b, double* out, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    real_part_kernel<<<blocks(n), kT, 0, st>>>(a, b, out, n);
}

void hprime_from(const double* h, const cplx* R, double* out, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    hprime_from_kernel<<<blocks(n), kT, 0, st>>>(h, R, out, n);
}

}  // namespace afqmc
