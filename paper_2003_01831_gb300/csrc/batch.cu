// Batches of independent AFQMC systems (different Hamiltonians, shapes and walker counts)
// advanced together, one CUDA-graph launch per step (afqmc_create_batch and friends,
// include/afqmc.h).
//
// Each system is an ordinary Hamiltonian + walker set.  Systems whose shapes the
// tensor-core path does not tile (M not a multiple of 64, N not a multiple of 8, Nchol not
// a multiple of 8) are padded exactly:
//   * extra orbitals are decoupled: h, every L_n and hence h' vanish on them, so
//     B = exp(-tau h'/2) is the identity there and A = sum_n c_n L_n has no entries there;
//   * extra electrons sit one per extra orbital, both in the trial and in every walker, so
//     S = Psi^+ Phi = diag(S_true, 1): log det S, Theta's true block, T_n = Psi^+ L_n Theta,
//     t_n, X_n and the local energy are unchanged, and the Taylor propagator and B leave the
//     padding orbitals exactly as they were;
//   * extra Cholesky vectors are zero: t_n = 0, xbar_n = 0 and their fields drop out of A
//     and of the importance weight (x_n xbar_n - xbar_n^2/2 = 0).
// Philox draws x[w][n] from (n/4, w, step) independently of Nchol, so the fields of the true
// Cholesky vectors are those an unpadded run draws.
//
// The step of every system is captured once into a CUDA graph whose branches (one chain of
// kernels per system, spread over `concurrency` parallel branches) the GPU overlaps; seed and
// step live in device memory, so the same graph replays every step.  An autotuner times a
// few launch shapes (branch count, plain-GEMM tile width, persistent grid size) on the real
// batch and keeps the fastest.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <string>
#include <vector>

#include "state.cuh"

using namespace afqmc;

struct afqmc_batch {
    int n = 0;
    int device = 0;
    double tau = 0.0;
    afqmc_opts opts{};
    int pad_mode = AFQMC_PAD_AUTO;
    std::vector<afqmc_ham*> ham;
    std::vector<afqmc_walkers*> wk;
    std::vector<int> M, N, Nchol, W;          // caller's shapes
    std::vector<int> Mp, Np, Ncp;             // internal (padded) shapes
    std::vector<double> cost;                 // relative cost per step (branch balancing)
    int64_t step = 0;

    int64_t* params = nullptr;       // device {seed, step}
    int* trace_idx = nullptr;        // device: next trace row
    cplx* trace = nullptr;           // device [trace_cap][n]
    int trace_cap = 0;
    const cplx** emix_ptrs = nullptr;   // device [n]: each system's E_mix slot
    unsigned** flag_ptrs = nullptr;     // device [n]: each system's status word
    unsigned* flags = nullptr;          // device: OR of the systems' status words

    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> br;
    std::vector<cudaEvent_t> ev;     // fork + one join event per branch
    cudaGraphExec_t exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [measure][qr]
    int kernels[2][2] = {{0, 0}, {0, 0}};

    // launch shape (autotuned)
    int concurrency = 0;
    int bn_max = 256;
    int grid_cap = 0;
    double tuned_ms = -1.0;
    // energy contractions of a measuring BF16X3 step: one multi-system launch (1) or one
    // launch per system in its branch (0); K chunk of the multi-system launch
    int multi_energy = 1;
    int energy_bk = 32;
    EnergySys* esys = nullptr;       // device [n]: each system's operands and shape
    EnergyWork* work = nullptr;      // device [nwork]: pair tiles of every system
    int64_t nwork = 0;
    int esys_bk = 0;                 // K chunk esys was described with (0: not built)
    std::vector<cudaEvent_t> ev2;    // second fork / join around the multi-system launch
};

namespace {

constexpr uint64_t kSeedStride = 0x9E3779B97F4A7C15ull;   // system s uses key seed + s * this

__global__ void pad_real_kernel(const double* src, int nb, int rows, int cols, double* dst, int prow, int pcol) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)prow * pcol;
    if (i >= per * nb) return;
    const int64_t b = i / per, e = i % per;
    const int r = (int)(e / pcol), c = (int)(e % pcol);
    dst[i] = (b < nb && r < rows && c < cols) ? src[(b * rows + r) * cols + c] : 0.0;
}

// Orbital blocks [M][N] (complex) -> [Mp][Np] with one extra electron per extra orbital:
// entry (M + j, N + j) = 1 for j < Np - N.  `nb` blocks, source block stride sstride
// (complex elements), destination stride Mp*Np.
__global__ void pad_orbitals_kernel(const cplx* src, int64_t sstride, int nb, int M, int N, cplx* dst, int Mp,
                                    int Np) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)Mp * Np;
    if (i >= per * nb) return;
    const int64_t b = i / per, e = i % per;
    const int r = (int)(e / Np), c = (int)(e % Np);
    cplx v{0.0, 0.0};
    if (r < M && c < N) v = src[b * sstride + (int64_t)r * N + c];
    else if (r >= M && c >= N && r - M == c - N) v = cplx{1.0, 0.0};
    dst[i] = v;
}

// Walkers [W][2][Mp][Np] -> caller layout [W][M*Nup + M*Ndn] (true block of each spin)
__global__ void unpad_walkers_kernel(const cplx* src, int W, int Mp, int Np, int M, int N0, int N1, cplx* dst) {
    const int64_t per = (int64_t)M * (N0 + N1);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= per * W) return;
    const int64_t w = i / per, e = i % per;
    const int s = e < (int64_t)M * N0 ? 0 : 1;
    const int N = s == 0 ? N0 : N1;
    const int64_t f = s == 0 ? e : e - (int64_t)M * N0;
    const int r = (int)(f / N), c = (int)(f % N);
    dst[i] = src[((w * 2 + s) * Mp + r) * (int64_t)Np + c];
}

// End of a batch step: gather each system's E_mix into the trace row, OR the status words,
// advance the device step counter.
__global__ void batch_tail_kernel(const cplx* const* emix, unsigned* const* fl, int n, int measured, cplx* trace,
                                  int* trace_idx, int trace_cap, unsigned* flags, int64_t* params) {
    __shared__ unsigned acc;
    if (threadIdx.x == 0) acc = 0u;
    __syncthreads();
    const int row = *trace_idx;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        if (measured && row < trace_cap) trace[(int64_t)row * n + s] = *emix[s];
        atomicOr(&acc, *fl[s]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (acc) atomicOr(flags, acc);
        if (measured) *trace_idx = row + 1;
        params[1] += 1;
    }
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

// Tensor-core electron count: the energy tiles pack floor(128 / N') walker-spins of any N' that
// is a multiple of 8, so N is padded to the next multiple of 8 (or, under the debug granule 32,
// to 32, 64 or 128).
int tn_pad(int N) {
    if (launch_policy().batch_n_granule == 32) return N <= 32 ? 32 : (N <= 64 ? 64 : 128);
    return std::max(8, ((N + 7) / 8) * 8);
}

// Internal shapes of system s.
void pick_shapes(afqmc_batch* b, int s, bool pad) {
    if (!pad) {
        b->Mp[s] = b->M[s];
        b->Np[s] = b->N[s];
        b->Ncp[s] = b->Nchol[s];
        return;
    }
    const int Np = tn_pad(b->N[s]);
    int Mp = ((b->M[s] + (Np - b->N[s]) + 63) / 64) * 64;
    b->Mp[s] = Mp;
    b->Np[s] = Np;
    b->Ncp[s] = ((b->Nchol[s] + 7) / 8) * 8;
}

bool tc_tiles(int M, int N, int Nup, int Ndn, int Nchol) {
    const bool n_ok = launch_policy().batch_n_granule == 32 ? (N == 32 || N == 64 || N == 128) : (N % 8 == 0 && N <= 128);
    return M % 64 == 0 && M <= 1024 && Nup == Ndn && n_ok && Nchol % 8 == 0;
}

// Device copy of a caller array (host or device); *tmp owns it when a copy was made.
int device_view(const void* src, size_t bytes, cudaStream_t st, const void** dev, void** tmp) {
    *tmp = nullptr;
    if (is_device_ptr(src)) {
        *dev = src;
        return AFQMC_OK;
    }
    if (cudaMalloc(tmp, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        return fail(AFQMC_ERR_OOM, "create_batch: staging buffer");
    }
    AFQMC_CUDA_TRY(cudaMemcpyAsync(*tmp, src, bytes, cudaMemcpyDefault, st));
    *dev = *tmp;
    return AFQMC_OK;
}

struct DevBufs {
    std::vector<void*> p;
    ~DevBufs() {
        for (void* q : p)
            if (q) cudaFree(q);
    }
    void* take(void* q) {
        p.push_back(q);
        return q;
    }
};

// Creates the Hamiltonian and walker set of system s (padded if b->Mp[s] differs).
int create_system(afqmc_batch* b, int s, const afqmc_system& y, cudaStream_t st) {
    const int M = y.M, Nc = y.Nchol, Mp = b->Mp[s], Np = b->Np[s], Ncp = b->Ncp[s];
    const bool pad = Mp != M || Np != y.Nup || Ncp != Nc;
    afqmc_opts o = b->opts;
    if (!pad) {
        AFQMC_TRY(afqmc_create_hamiltonian(y.h, y.L, y.E0, M, Nc, st, &b->ham[s]));
        return afqmc_init_walkers(b->ham[s], y.Psi_up, y.Psi_dn, y.Nup, y.Ndn, y.W, y.Phi0, b->tau, &o, st, &b->wk[s]);
    }
    DevBufs keep;
    const void *h, *L, *pu, *pd, *ph = nullptr;
    void* t;
    AFQMC_TRY(device_view(y.h, sizeof(double) * M * M, st, &h, &t));
    keep.take(t);
    AFQMC_TRY(device_view(y.L, sizeof(double) * (size_t)Nc * M * M, st, &L, &t));
    keep.take(t);
    AFQMC_TRY(device_view(y.Psi_up, sizeof(cplx) * (size_t)M * y.Nup, st, &pu, &t));
    keep.take(t);
    AFQMC_TRY(device_view(y.Psi_dn, sizeof(cplx) * (size_t)M * y.Ndn, st, &pd, &t));
    keep.take(t);
    if (y.Phi0) {
        AFQMC_TRY(device_view(y.Phi0, sizeof(cplx) * (size_t)y.W * M * (y.Nup + y.Ndn), st, &ph, &t));
        keep.take(t);
    }
    void *hp, *Lp, *Pp, *Fp = nullptr;
    const size_t mm = (size_t)Mp * Mp;
    if (cudaMalloc(&hp, sizeof(double) * mm) != cudaSuccess) return fail(AFQMC_ERR_OOM, "create_batch: padding");
    keep.take(hp);
    if (cudaMalloc(&Lp, sizeof(double) * mm * Ncp) != cudaSuccess) return fail(AFQMC_ERR_OOM, "create_batch: padding");
    keep.take(Lp);
    if (cudaMalloc(&Pp, sizeof(cplx) * 2 * (size_t)Mp * Np) != cudaSuccess)
        return fail(AFQMC_ERR_OOM, "create_batch: padding");
    keep.take(Pp);
    pad_real_kernel<<<nblk((int64_t)mm), 256, 0, st>>>(static_cast<const double*>(h), 1, M, M,
                                                        static_cast<double*>(hp), Mp, Mp);
    // L: [Nc][M][M] -> [Ncp][Mp][Mp] (zero Cholesky vectors beyond Nc): pad as Ncp blocks of
    // which the source holds Nc; the extra blocks are zero-filled first.
    AFQMC_CUDA_TRY(cudaMemsetAsync(Lp, 0, sizeof(double) * mm * Ncp, st));
    pad_real_kernel<<<nblk((int64_t)mm * Nc), 256, 0, st>>>(static_cast<const double*>(L), Nc, M, M,
                                                             static_cast<double*>(Lp), Mp, Mp);
    cplx* P = static_cast<cplx*>(Pp);
    pad_orbitals_kernel<<<nblk((int64_t)Mp * Np), 256, 0, st>>>(static_cast<const cplx*>(pu), 0, 1, M, y.Nup, P, Mp,
                                                                 Np);
    pad_orbitals_kernel<<<nblk((int64_t)Mp * Np), 256, 0, st>>>(static_cast<const cplx*>(pd), 0, 1, M, y.Ndn,
                                                                 P + (size_t)Mp * Np, Mp, Np);
    if (ph) {
        if (cudaMalloc(&Fp, sizeof(cplx) * (size_t)y.W * 2 * Mp * Np) != cudaSuccess)
            return fail(AFQMC_ERR_OOM, "create_batch: padding");
        keep.take(Fp);
        // caller walker w: [M*Nup (up) | M*Ndn (dn)] -> [w][2][Mp][Np]
        const cplx* src = static_cast<const cplx*>(ph);
        const int64_t sper = (int64_t)M * (y.Nup + y.Ndn);
        cplx* F = static_cast<cplx*>(Fp);
        for (int sp = 0; sp < 2; ++sp) {
            const int Ns = sp == 0 ? y.Nup : y.Ndn;
            // pad this spin of every walker into a staging array, then scatter it to the
            // walker stride 2*Mp*Np with one strided copy
            cplx* tmp = nullptr;
            if (cudaMalloc(&tmp, sizeof(cplx) * (size_t)y.W * Mp * Np) != cudaSuccess)
                return fail(AFQMC_ERR_OOM, "create_batch: padding");
            keep.take(tmp);
            pad_orbitals_kernel<<<nblk((int64_t)y.W * Mp * Np), 256, 0, st>>>(
                src + (sp == 0 ? 0 : (int64_t)M * y.Nup), sper, y.W, M, Ns, tmp, Mp, Np);
            AFQMC_CUDA_TRY(cudaMemcpy2DAsync(F + (size_t)sp * Mp * Np, sizeof(cplx) * 2 * Mp * Np, tmp,
                                             sizeof(cplx) * Mp * Np, sizeof(cplx) * Mp * Np, y.W,
                                             cudaMemcpyDeviceToDevice, st));
        }
    }
    AFQMC_CUDA_TRY(cudaGetLastError());
    AFQMC_TRY(afqmc_create_hamiltonian(static_cast<const double*>(hp), static_cast<const double*>(Lp), y.E0, Mp, Ncp,
                                       st, &b->ham[s]));
    const int rc = afqmc_init_walkers(b->ham[s], reinterpret_cast<const double*>(P),
                                      reinterpret_cast<const double*>(P + (size_t)Mp * Np), Np, Np, y.W,
                                      static_cast<const double*>(Fp), b->tau, &o, st, &b->wk[s]);
    cudaStreamSynchronize(st);   // staging buffers are freed on return
    return rc;
}

void destroy_graphs(afqmc_batch* b) {
    for (auto& row : b->exec)
        for (auto& g : row)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
}

// Kernels of one step of system s on stream st (the same sequence afqmc_step runs).
int system_step(afqmc_batch* b, int s, bool meas, bool qr, cudaStream_t st) {
    afqmc_walkers* wk = b->wk[s];
    const bool tc = wk->opts.precision == AFQMC_PREC_BF16X3;
    AFQMC_TRY(tc ? tc_measure(wk, meas, st) : fp64_measure(wk, meas, st));
    if (meas) mixed_energy(wk->weight, wk->E_L, wk->W, wk->emix, st);
    philox_fields_dev(b->params, (uint64_t)s * kSeedStride, wk->W, wk->Nchol, wk->x, st, wk->opts.walker_offset);
    AFQMC_TRY(tc ? tc_propagate_and_weight(wk, wk->x, st) : fp64_propagate_and_weight(wk, wk->x, st));
    if (qr) AFQMC_TRY(tc ? tc_qr(wk, st) : fp64_qr(wk, st));
    return AFQMC_OK;
}

// Operands, shapes and work list of the multi-system energy contraction (device arrays, built
// once per K chunk: the systems' buffers never move).
int ensure_energy_work(afqmc_batch* b) {
    if (b->esys && b->esys_bk == b->energy_bk) return AFQMC_OK;
    if (b->esys) cudaFree(b->esys);
    if (b->work) cudaFree(b->work);
    b->esys = nullptr;
    b->work = nullptr;
    std::vector<EnergySys> hs((size_t)b->n);
    for (int s = 0; s < b->n; ++s) AFQMC_TRY(tc_energy_system(b->wk[s], b->energy_bk, &hs[(size_t)s]));
    std::vector<EnergyWork> hw;
    energy_work_list(hs.data(), b->n, hw);
    if (cudaMalloc(&b->esys, sizeof(EnergySys) * hs.size()) != cudaSuccess ||
        cudaMalloc(&b->work, sizeof(EnergyWork) * std::max<size_t>(hw.size(), 1)) != cudaSuccess) {
        cudaGetLastError();
        return fail(AFQMC_ERR_OOM, "batch: energy work list");
    }
    AFQMC_CUDA_TRY(cudaMemcpy(b->esys, hs.data(), sizeof(EnergySys) * hs.size(), cudaMemcpyHostToDevice));
    AFQMC_CUDA_TRY(cudaMemcpy(b->work, hw.data(), sizeof(EnergyWork) * hw.size(), cudaMemcpyHostToDevice));
    b->nwork = (int64_t)hw.size();
    b->esys_bk = b->energy_bk;
    return AFQMC_OK;
}

// The rest of a measuring BF16X3 step of system s once its energy contraction has run.
int system_step_after_energy(afqmc_batch* b, int s, bool qr, cudaStream_t st) {
    afqmc_walkers* wk = b->wk[s];
    AFQMC_TRY(tc_measure_post(wk, true, st));
    mixed_energy(wk->weight, wk->E_L, wk->W, wk->emix, st);
    philox_fields_dev(b->params, (uint64_t)s * kSeedStride, wk->W, wk->Nchol, wk->x, st, wk->opts.walker_offset);
    AFQMC_TRY(tc_propagate_and_weight(wk, wk->x, st));
    if (qr) AFQMC_TRY(tc_qr(wk, st));
    return AFQMC_OK;
}

// Captures one batch step (every system) into an executable graph.
int capture(afqmc_batch* b, bool meas, bool qr, cudaGraphExec_t* out, int* nkern) {
    const int K = std::max(1, std::min(b->concurrency > 0 ? b->concurrency : b->n, (int)b->br.size()));
    // longest-processing-time assignment of systems to branches
    std::vector<int> order(b->n);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int x, int y) { return b->cost[x] > b->cost[y]; });
    std::vector<double> load(K, 0.0);
    std::vector<std::vector<int>> chain(K);
    for (int s : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        chain[k].push_back(s);
        load[k] += b->cost[s];
    }
    LaunchPolicy saved = launch_policy();
    launch_policy().grid_cap = b->grid_cap;
    launch_policy().bn_max = b->bn_max;
    const bool tc = b->opts.precision == AFQMC_PREC_BF16X3;
    const bool multi = meas && tc && b->multi_energy;
    if (multi) {
        const int r0 = ensure_energy_work(b);
        if (r0) {
            launch_policy() = saved;
            return r0;
        }
    }
    cudaGraph_t g = nullptr;
    int rc = AFQMC_OK;
    AFQMC_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    if (multi) {
        // every system's Green's function, then one energy launch over all of them, then every
        // system's local energy, propagation and weights
        cudaEventRecord(b->ev2[0], b->cap);
        for (int k = 0; k < K && rc == AFQMC_OK; ++k) {
            cudaStreamWaitEvent(b->br[k], b->ev2[0], 0);
            for (int s : chain[k]) {
                rc = tc_measure_pre(b->wk[s], b->br[k]);
                if (rc) break;
            }
            cudaEventRecord(b->ev2[1 + k], b->br[k]);
            cudaStreamWaitEvent(b->cap, b->ev2[1 + k], 0);
        }
        if (rc == AFQMC_OK)
            rc = tc_energy_multi(b->esys, b->work, b->nwork, b->energy_bk,
                                 (b->opts.energy_terms == 0 || b->opts.energy_terms == 2)
                                     ? kEnergyRounded
                                     : (b->opts.energy_terms == 1 ? kEnergyFour : b->opts.energy_terms),
                                 b->wk[0]->flags, b->cap);
    }
    cudaEventRecord(b->ev[0], b->cap);
    for (int k = 0; k < K && rc == AFQMC_OK; ++k) {
        cudaStreamWaitEvent(b->br[k], b->ev[0], 0);
        for (int s : chain[k]) {
            rc = multi ? system_step_after_energy(b, s, qr, b->br[k]) : system_step(b, s, meas, qr, b->br[k]);
            if (rc) break;
        }
        cudaEventRecord(b->ev[1 + k], b->br[k]);
        cudaStreamWaitEvent(b->cap, b->ev[1 + k], 0);
    }
    batch_tail_kernel<<<1, 256, 0, b->cap>>>(b->emix_ptrs, b->flag_ptrs, b->n, meas ? 1 : 0, b->trace, b->trace_idx,
                                             b->trace_cap, b->flags, b->params);
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    launch_policy() = saved;
    if (rc != AFQMC_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess || !g) return fail(AFQMC_ERR_CUDA, std::string("batch: graph capture: ") + cudaGetErrorString(e));
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    int nk = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(AFQMC_ERR_CUDA, std::string("batch: graph instantiate: ") + cudaGetErrorString(e));
    *nkern = nk;
    return AFQMC_OK;
}

int ensure_trace(afqmc_batch* b, int rows) {
    if (rows <= b->trace_cap) return AFQMC_OK;
    destroy_graphs(b);   // the graphs hold the trace pointer
    if (b->trace) cudaFree(b->trace);
    b->trace = nullptr;
    const int cap = std::max(rows, 64);
    if (cudaMalloc(&b->trace, sizeof(cplx) * (size_t)cap * b->n) != cudaSuccess) {
        cudaGetLastError();
        b->trace_cap = 0;
        return fail(AFQMC_ERR_OOM, "batch_step: trace buffer");
    }
    b->trace_cap = cap;
    return AFQMC_OK;
}

int graph_for(afqmc_batch* b, bool meas, bool qr, cudaGraphExec_t* out) {
    cudaGraphExec_t& g = b->exec[meas][qr];
    if (!g) AFQMC_TRY(capture(b, meas, qr, &g, &b->kernels[meas][qr]));
    *out = g;
    return AFQMC_OK;
}

// Runs nsteps on stream st (no host synchronisation); E_mix rows go to the device trace.
int run_steps(afqmc_batch* b, int nsteps, int measure_every, cudaStream_t st) {
    for (int s = 0; s < nsteps; ++s) {
        const bool meas = measure_every > 0 && s % measure_every == 0;
        const bool qr = b->opts.k_qr > 0 && (b->step + 1) % b->opts.k_qr == 0;
        cudaGraphExec_t g = nullptr;
        AFQMC_TRY(graph_for(b, meas, qr, &g));
        AFQMC_CUDA_TRY(cudaGraphLaunch(g, st));
        b->step++;
        for (auto* w : b->wk) w->step++;
    }
    return AFQMC_OK;
}

int check(afqmc_batch* b, int s) {
    if (!b) return fail(AFQMC_ERR_BADARG, "batch: NULL handle");
    if (s < 0 || s >= b->n) return fail(AFQMC_ERR_BADARG, "batch: system index out of range");
    return AFQMC_OK;
}

void free_batch(afqmc_batch* b) {
    destroy_graphs(b);
    for (int s = 0; s < b->n; ++s) {
        if (b->wk[s]) afqmc_destroy_walkers(b->wk[s]);
        if (b->ham[s]) afqmc_destroy_hamiltonian(b->ham[s]);
    }
    void* ps[] = {b->params, b->trace_idx, b->trace, b->emix_ptrs, b->flag_ptrs, b->flags, b->esys, b->work};
    for (void* p : ps)
        if (p) cudaFree(p);
    for (auto e : b->ev) cudaEventDestroy(e);
    for (auto e : b->ev2) cudaEventDestroy(e);
    for (auto q : b->br) cudaStreamDestroy(q);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

}  // namespace

extern "C" {

int afqmc_create_batch(int nsys, const afqmc_system* sys, double tau, const afqmc_opts* opts, int pad_mode,
                       void* stream, afqmc_batch_t* out) {
    if (!out) return fail(AFQMC_ERR_BADARG, "create_batch: out is NULL");
    *out = nullptr;
    if (nsys < 1 || !sys) return fail(AFQMC_ERR_BADARG, "create_batch: need nsys >= 1 systems");
    if (!(tau > 0.0) || !isfinite(tau)) return fail(AFQMC_ERR_BADARG, "create_batch: tau must be > 0");
    if (pad_mode != AFQMC_PAD_AUTO && pad_mode != AFQMC_PAD_ALWAYS)
        return fail(AFQMC_ERR_BADARG, "create_batch: pad_mode");
    afqmc_opts o;
    afqmc_default_opts(&o);
    if (opts) o = *opts;
    if (o.weight_mode == AFQMC_WEIGHT_LOCAL)   // the captured steps measure E_L only on measuring steps
        return fail(AFQMC_ERR_UNSUPPORTED, "create_batch: local-energy weights are not supported in batches");
    for (int s = 0; s < nsys; ++s) {
        const afqmc_system& y = sys[s];
        if (!y.h || !y.L || !y.Psi_up || !y.Psi_dn)
            return fail(AFQMC_ERR_BADARG, "create_batch: system " + std::to_string(s) + ": NULL h, L or trial");
        if (y.M < 1 || y.M > 1024 || y.Nchol < 1 || y.Nup < 1 || y.Ndn < 1 || y.Nup > y.M || y.Ndn > y.M ||
            y.Nup > 128 || y.Ndn > 128 || y.W < 1)
            return fail(AFQMC_ERR_SHAPE, "create_batch: system " + std::to_string(s) + ": sizes out of range");
        const bool needs_pad = o.precision == AFQMC_PREC_BF16X3 && !tc_tiles(y.M, y.Nup, y.Nup, y.Ndn, y.Nchol);
        if ((needs_pad || pad_mode == AFQMC_PAD_ALWAYS) && y.Nup != y.Ndn)
            return fail(AFQMC_ERR_UNSUPPORTED, "create_batch: system " + std::to_string(s) +
                                                   ": padding needs Nup == Ndn");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    afqmc_batch* b = new afqmc_batch();
    b->n = nsys;
    b->tau = tau;
    b->opts = o;
    b->pad_mode = pad_mode;
    b->ham.assign(nsys, nullptr);
    b->wk.assign(nsys, nullptr);
    b->M.resize(nsys); b->N.resize(nsys); b->Nchol.resize(nsys); b->W.resize(nsys);
    b->Mp.resize(nsys); b->Np.resize(nsys); b->Ncp.resize(nsys); b->cost.resize(nsys);
    auto bail = [&](int rc) {
        const std::string msg = afqmc_last_error();
        free_batch(b);
        set_error(rc, msg);
        return rc;
    };
    if (cudaGetDevice(&b->device) != cudaSuccess) return bail(fail(AFQMC_ERR_CUDA, "create_batch: no device"));
    for (int s = 0; s < nsys; ++s) {
        const afqmc_system& y = sys[s];
        b->M[s] = y.M; b->N[s] = y.Nup; b->Nchol[s] = y.Nchol; b->W[s] = y.W;
        const bool pad = pad_mode == AFQMC_PAD_ALWAYS ||
                         (o.precision == AFQMC_PREC_BF16X3 && !tc_tiles(y.M, y.Nup, y.Nup, y.Ndn, y.Nchol));
        pick_shapes(b, s, pad);
        if (!pad) b->Np[s] = std::max(y.Nup, y.Ndn);
        // energy dominates: Nchol N^2 M per walker
        b->cost[s] = (double)y.W * b->Ncp[s] * b->Np[s] * b->Np[s] * b->Mp[s];
        const int rc = create_system(b, s, y, st);
        if (rc) return bail(rc);
    }
    // device bookkeeping
    if (cudaMalloc(&b->params, 2 * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&b->trace_idx, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->emix_ptrs, nsys * sizeof(cplx*)) != cudaSuccess ||
        cudaMalloc(&b->flag_ptrs, nsys * sizeof(unsigned*)) != cudaSuccess ||
        cudaMalloc(&b->flags, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(AFQMC_ERR_OOM, "create_batch: bookkeeping"));
    }
    for (int s = 0; s < nsys; ++s) {
        // per-system field and trace buffers the graphs write
        afqmc_walkers* w = b->wk[s];
        if (w->x_cap < 1) {
            if (cudaMalloc(&w->x, sizeof(double) * (size_t)w->W * w->Nchol) != cudaSuccess)
                return bail(fail(AFQMC_ERR_OOM, "create_batch: field buffer"));
            w->x_cap = 1;
        }
        if (w->emix_cap < 1) {
            if (cudaMalloc(&w->emix, sizeof(cplx)) != cudaSuccess)
                return bail(fail(AFQMC_ERR_OOM, "create_batch: trace buffer"));
            w->emix_cap = 1;
        }
    }
    {
        std::vector<const cplx*> ep(nsys);
        std::vector<unsigned*> fp(nsys);
        for (int s = 0; s < nsys; ++s) {
            ep[s] = b->wk[s]->emix;
            fp[s] = b->wk[s]->flags;
        }
        int rc = AFQMC_OK;
        if (cudaMemcpy(b->emix_ptrs, ep.data(), nsys * sizeof(cplx*), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(b->flag_ptrs, fp.data(), nsys * sizeof(unsigned*), cudaMemcpyHostToDevice) != cudaSuccess)
            rc = fail(AFQMC_ERR_CUDA, "create_batch: bookkeeping copy");
        if (rc) return bail(rc);
    }
    cudaMemsetAsync(b->params, 0, 2 * sizeof(int64_t), st);
    cudaMemsetAsync(b->flags, 0, sizeof(unsigned), st);
    cudaMemsetAsync(b->trace_idx, 0, sizeof(int), st);
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(AFQMC_ERR_CUDA, "create_batch: stream"));
    const int nb = std::min(nsys, 32);
    b->br.resize(nb, nullptr);
    b->ev.resize(nb + 1, nullptr);
    b->ev2.resize(nb + 1, nullptr);
    for (auto& q : b->br)
        if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(AFQMC_ERR_CUDA, "create_batch: stream"));
    for (auto* evs : {&b->ev, &b->ev2})
        for (auto& e : *evs)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                return bail(fail(AFQMC_ERR_CUDA, "create_batch: event"));
    b->concurrency = nb;
    {
        const int rc = ensure_trace(b, 64);
        if (rc) return bail(rc);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(fail(AFQMC_ERR_CUDA, std::string("create_batch: ") + cudaGetErrorString(e)));
    *out = b;
    return AFQMC_OK;
}

int afqmc_destroy_batch(afqmc_batch_t b) {
    if (!b) return fail(AFQMC_ERR_BADARG, "destroy_batch: NULL handle");
    cudaDeviceSynchronize();
    free_batch(b);
    return AFQMC_OK;
}

int afqmc_batch_step(afqmc_batch_t b, int nsteps, uint64_t seed, int measure_every, double* E_mix_trace,
                     void* stream) {
    if (!b) return fail(AFQMC_ERR_BADARG, "batch_step: NULL handle");
    if (nsteps < 0 || measure_every < 0) return fail(AFQMC_ERR_BADARG, "batch_step: negative nsteps or measure_every");
    if (nsteps == 0) return AFQMC_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nmeas = measure_every > 0 ? (nsteps + measure_every - 1) / measure_every : 0;
    AFQMC_TRY(ensure_trace(b, std::max(nmeas, 1)));
    const int64_t p[2] = {(int64_t)seed, b->step};
    AFQMC_CUDA_TRY(cudaMemcpyAsync(b->params, p, sizeof(p), cudaMemcpyHostToDevice, st));
    AFQMC_CUDA_TRY(cudaMemsetAsync(b->trace_idx, 0, sizeof(int), st));
    AFQMC_TRY(run_steps(b, nsteps, measure_every, st));
    if (E_mix_trace && nmeas > 0)
        AFQMC_CUDA_TRY(cudaMemcpyAsync(E_mix_trace, b->trace, sizeof(cplx) * (size_t)nmeas * b->n, cudaMemcpyDefault,
                                       st));
    unsigned fl = 0;
    AFQMC_TRY(read_flags(b->flags, st, &fl));   // synchronises st (host p stays valid until here)
    return flags_to_error(fl, "batch_step");
}

int afqmc_batch_energy(afqmc_batch_t b, int sys, double* E_L, double* w, double* logS, double* E_mix, void* stream) {
    AFQMC_TRY(check(b, sys));
    return afqmc_energy(b->wk[sys], E_L, w, logS, E_mix, stream);
}

int afqmc_batch_get_walkers(afqmc_batch_t b, int sys, double* Phi, double* w, int64_t* step, void* stream) {
    AFQMC_TRY(check(b, sys));
    afqmc_walkers* wk = b->wk[sys];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool padded = b->Mp[sys] != b->M[sys] || b->Np[sys] != b->N[sys];
    if (!Phi || !padded) return afqmc_get_walkers(wk, Phi, w, step, stream);
    AFQMC_TRY(afqmc_get_walkers(wk, nullptr, w, step, stream));
    const int W = wk->W, Mp = b->Mp[sys], Np = b->Np[sys], M = b->M[sys], N = b->N[sys];
    cplx *full = nullptr, *out = nullptr;
    const size_t nfull = (size_t)W * 2 * Mp * Np, nout = (size_t)W * M * 2 * N;
    if (cudaMalloc(&full, sizeof(cplx) * nfull) != cudaSuccess || cudaMalloc(&out, sizeof(cplx) * nout) != cudaSuccess) {
        cudaGetLastError();
        if (full) cudaFree(full);
        return fail(AFQMC_ERR_OOM, "batch_get_walkers: staging");
    }
    int rc = afqmc_get_walkers(wk, reinterpret_cast<double*>(full), nullptr, nullptr, stream);
    if (rc == AFQMC_OK) {
        unpad_walkers_kernel<<<nblk((int64_t)nout), 256, 0, st>>>(full, W, Mp, Np, M, N, N, out);
        if (cudaMemcpyAsync(Phi, out, sizeof(cplx) * nout, cudaMemcpyDefault, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = fail(AFQMC_ERR_CUDA, "batch_get_walkers: copy");
    }
    cudaFree(full);
    cudaFree(out);
    return rc;
}

int afqmc_batch_info(afqmc_batch_t b, int sys, int* shape, int* kernels_per_step) {
    AFQMC_TRY(check(b, sys));
    if (shape) {
        shape[0] = b->Mp[sys];
        shape[1] = b->Np[sys];
        shape[2] = b->Ncp[sys];
        shape[3] = b->concurrency;
        shape[4] = b->bn_max;
        shape[5] = b->grid_cap;
        shape[6] = b->opts.precision == AFQMC_PREC_BF16X3 ? b->multi_energy : 0;
        shape[7] = b->energy_bk;
    }
    if (kernels_per_step) *kernels_per_step = b->kernels[1][0] > 0 ? b->kernels[1][0] : -1;
    return AFQMC_OK;
}

int afqmc_debug_set_batch_energy(afqmc_batch_t b, int multi, int bk) {
    if (!b) return fail(AFQMC_ERR_BADARG, "debug_set_batch_energy: NULL handle");
    if ((multi != 0 && multi != 1) || (bk != 16 && bk != 32))
        return fail(AFQMC_ERR_BADARG, "debug_set_batch_energy: multi must be 0 or 1, bk 16 or 32");
    b->multi_energy = multi;
    b->energy_bk = bk;
    destroy_graphs(b);
    return AFQMC_OK;
}

int afqmc_batch_autotune(afqmc_batch_t b, int reps, double* best_ms, void* stream) {
    if (!b) return fail(AFQMC_ERR_BADARG, "batch_autotune: NULL handle");
    if (reps < 1) reps = 2;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // save the walkers (internal layout), restore after tuning
    std::vector<void*> savedPhi(b->n, nullptr), savedW(b->n, nullptr);
    std::vector<int64_t> savedStep(b->n, 0);
    auto release = [&]() {
        for (void* p : savedPhi)
            if (p) cudaFree(p);
        for (void* p : savedW)
            if (p) cudaFree(p);
    };
    for (int s = 0; s < b->n; ++s) {
        afqmc_walkers* wk = b->wk[s];
        const size_t nphi = (size_t)wk->W * wk->M * (wk->N[0] + wk->N[1]);
        if (cudaMalloc(&savedPhi[s], sizeof(cplx) * nphi) != cudaSuccess ||
            cudaMalloc(&savedW[s], sizeof(cplx) * wk->W) != cudaSuccess) {
            cudaGetLastError();
            release();
            return fail(AFQMC_ERR_OOM, "batch_autotune: save buffers");
        }
        const int rc = afqmc_get_walkers(wk, static_cast<double*>(savedPhi[s]), static_cast<double*>(savedW[s]),
                                         &savedStep[s], stream);
        if (rc) {
            release();
            return rc;
        }
    }
    const int64_t step0 = b->step;
    const int c0 = b->concurrency, bn0 = b->bn_max, g0 = b->grid_cap, m0 = b->multi_energy, k0 = b->energy_bk;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timeit = [&](double* ms) -> int {
        destroy_graphs(b);
        cudaGraphExec_t g = nullptr;
        AFQMC_TRY(graph_for(b, true, false, &g));
        AFQMC_CUDA_TRY(cudaGraphLaunch(g, st));   // warm-up (lazy module loading, caches)
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) AFQMC_CUDA_TRY(cudaGraphLaunch(g, st));
        cudaEventRecord(e1, st);
        AFQMC_CUDA_TRY(cudaEventSynchronize(e1));
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        *ms = f / reps;
        return AFQMC_OK;
    };
    int rc = AFQMC_OK;
    double best = 1e30;
    int bc = c0, bb = bn0, bg = g0;
    AFQMC_CUDA_TRY(cudaMemsetAsync(b->trace_idx, 0, sizeof(int), st));
    // coordinate search: branch count, then GEMM tile width, then persistent grid size
    std::vector<int> conc;
    for (int k = 1; k < (int)b->br.size(); k *= 2) conc.push_back(k);
    conc.push_back((int)b->br.size());
    for (int k : conc) {
        b->concurrency = k;
        double ms = 0;
        if ((rc = timeit(&ms))) break;
        if (ms < best) { best = ms; bc = k; }
    }
    b->concurrency = bc;
    for (int bn : {256, 128}) {
        if (rc) break;
        b->bn_max = bn;
        double ms = 0;
        if ((rc = timeit(&ms))) break;
        if (ms < best) { best = ms; bb = bn; }
    }
    b->bn_max = bb;
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
    for (int gcap : {0, nsm / 2, nsm / 4}) {
        if (rc) break;
        b->grid_cap = gcap;
        double ms = 0;
        if ((rc = timeit(&ms))) break;
        if (ms < best) { best = ms; bg = gcap; }
    }
    b->grid_cap = bg;
    if (b->opts.precision == AFQMC_PREC_BF16X3) {
        // energy contractions: one multi-system launch with K chunks of 32 or 16, or one launch
        // per system in its branch
        int bm = b->multi_energy, bk = b->energy_bk;
        for (auto mk : {std::make_pair(1, 32), std::make_pair(1, 16), std::make_pair(0, 32)}) {
            if (rc) break;
            if (mk.first == bm && mk.second == bk) continue;   // timed already as the current shape
            b->multi_energy = mk.first;
            b->energy_bk = mk.second;
            double ms = 0;
            if ((rc = timeit(&ms))) break;
            if (ms < best) { best = ms; bm = mk.first; bk = mk.second; }
        }
        b->multi_energy = bm;
        b->energy_bk = bk;
    }
    destroy_graphs(b);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // restore the walkers, the step counters and the status
    for (int s = 0; s < b->n && rc == AFQMC_OK; ++s)
        rc = afqmc_set_walkers(b->wk[s], static_cast<double*>(savedPhi[s]), static_cast<double*>(savedW[s]),
                               savedStep[s], stream);
    release();
    b->step = step0;
    if (rc) {
        b->concurrency = c0;
        b->bn_max = bn0;
        b->grid_cap = g0;
        b->multi_energy = m0;
        b->energy_bk = k0;
        return rc;
    }
    unsigned fl = 0;
    AFQMC_TRY(read_flags(b->flags, st, &fl));
    AFQMC_TRY(flags_to_error(fl, "batch_autotune"));
    b->tuned_ms = best;
    if (best_ms) *best_ms = best;
    return AFQMC_OK;
}

}  // extern "C"
