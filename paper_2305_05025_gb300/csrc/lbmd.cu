// C ABI of the coupled LB-MD step (declared in include/lbmd.h): handle
// lifetime, parameter validation, device memory, the per-step CUDA graph and
// the state/diagnostic calls.
//
// One coupled step is one graph launch with two branches:
//   lattice branch (low priority):  dense stream-collide of every node (g only)
//   solute branch (high priority):  sort + interpolate + claim -> n_md+1
//                                   substep kernels -> spread
// joined by the sparse fix-up of the claimed nodes (g + G), whose last block
// advances the device step counter. The dense lattice pass does not depend on
// the solute, so the two branches overlap.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbmd_internal.cuh"

using namespace lbmd;

namespace {

thread_local std::string g_create_error;

constexpr int kFixBlocks = 152 * 8;  // grid of the fix-up kernel (grid-stride over the touched nodes)
constexpr int kFold = 128;  // bucket grid per axis (cells folded modulo this)
// Atoms per bucket: a collapsed Lennard-Jones globule (sigma 0.4) packs ~30
// atoms into a cell of side 1.3, and folding (cells 128 apart share a bucket
// once a lattice axis holds more than 128 cells) can stack two globules.
constexpr int kCap = 128;
// Atoms per MD bucket on the half-size grid (a cell of side >= 0.65 holds
// ~5 atoms of a collapsed globule; one fold can stack two regions).
constexpr int kCapFine = 48;

}  // namespace

void lbmd::set_thread_error(const std::string &msg) { g_create_error = msg; }

struct lbmd_s {
    lbmd_params p{};
    double kT = 0.0;          // thermal noise (lbmd_set_thermal)
    uint64_t seed = 0;
    float *charge = nullptr;  // device charges (lbmd_set_charges)
    float4 *unode = nullptr;  // node velocities of the step (lbmd_set_reinterpolation)
    Lat *lat_dev = nullptr;   // device copy of L for the substeps (re-interpolation), set with each graph
    cudaStream_t stream = nullptr;            // caller's stream
    cudaStream_t s_main = nullptr, s_lat = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    cudaEvent_t ev_m0 = nullptr, ev_m1 = nullptr;  // bracket the n_md + 1 substep kernels
    int na = 0, nb = 0;
    Lat L{};
    AtomArgs A{};
    CouplingArgs C{};
    void *pop[2] = {nullptr, nullptr};
    DevState *ds = nullptr;
    double *red = nullptr;  // partials
    double *red_out = nullptr;
    int red_blocks = 0;
    int fix_grid = 1;
    std::vector<void *> allocs;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node_t0 = nullptr, node_t1 = nullptr, node_m0 = nullptr, node_m1 = nullptr;
    bool state_set = false;
    long long steps = 0;
    std::string err;
    int alloc_count = 0;
    void *stage = nullptr;  // device staging for host-pointer set/get (lazily sized)
    size_t stage_bytes = 0;
    int *ident = nullptr;   // identity atom order
    // lbmd_backward buffers (allocated on first use, sized for its arguments)
    std::vector<void *> adj_allocs;
    int adj_ckpts = 0, adj_seg = 0;
    void *ck_lat = nullptr, *seg_lat = nullptr;
    double *ck_X = nullptr, *seg_X = nullptr;
    float *ck_V = nullptr, *seg_V = nullptr, *ck_F = nullptr, *seg_F = nullptr;
    float4 *recP = nullptr, *recL = nullptr;
    float *recV = nullptr, *recF = nullptr;
    float *hat[2] = {nullptr, nullptr};
    AdjArgs D{};
    int *adj_count = nullptr, *adj_slot = nullptr;
    double *obs_acc = nullptr;  // [0] sum, [1..7] scratch
    int adj_blocks = 0;
    // trajectory analysis (lbmd_analysis_*), allocated by lbmd_analysis_begin
    std::vector<void *> ana_allocs;
    AnaArgs ana{};
    double ana_ybar[3] = {0, 0, 0}, ana_ey = 0.0;
    int ana_frames = 0, ana_max = 0;
    float *ana_cov = nullptr;  // device covariance for host outputs (lazily)
};

namespace {

lbmd_status fail(lbmd_t h, lbmd_status s, const std::string &msg) {
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return s;
}

lbmd_status cuda_fail(lbmd_t h, cudaError_t e, const char *what) {
    return fail(h, e == cudaErrorMemoryAllocation ? LBMD_ERR_ALLOC : LBMD_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                                                                                 \
    do {                                                                                                            \
        cudaError_t e_ = (call);                                                                                    \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);                                                    \
    } while (0)

// Device allocation with a test hook: LBMD_TEST_FAIL_ALLOC=k makes the k-th
// allocation of a handle report failure (host-side fault injection).
// NVTX range over one call of the ABI (header-only NVTX: free unless a
// profiler is attached), so a timeline shows the calls around the graph
// launches and kernels.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

lbmd_status dalloc(lbmd_t h, void **ptr, size_t bytes) {
    *ptr = nullptr;
    ++h->alloc_count;
    if (const char *env = std::getenv("LBMD_TEST_FAIL_ALLOC")) {
        if (std::atoi(env) == h->alloc_count)
            return fail(h, LBMD_ERR_ALLOC, "simulated allocation failure (LBMD_TEST_FAIL_ALLOC)");
    }
    cudaError_t e = cudaMalloc(ptr, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return cuda_fail(h, e, "cudaMalloc");
    }
    h->allocs.push_back(*ptr);
    return LBMD_OK;
}

template <class T> lbmd_status dalloc_t(lbmd_t h, T **ptr, size_t count) {
    void *p = nullptr;
    lbmd_status s = dalloc(h, &p, count * sizeof(T));
    *ptr = (T *)p;
    return s;
}

#define TRY(expr)                                                                                                   \
    do {                                                                                                            \
        lbmd_status s_ = (expr);                                                                                    \
        if (s_ != LBMD_OK) return s_;                                                                               \
    } while (0)

std::string validate(const lbmd_params *p, int n_atoms, const double *mass, int n_bonds, const int32_t *bonds,
                     const double *bond_k, const double *bond_r0) {
    if (!p) return "params is NULL";
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return "lattice sizes must be >= 1";
    const double N = (double)p->nx * p->ny * p->nz;
    if (N >= 2147483647.0) return "nx*ny*nz must be < 2^31";
    if (!(p->tau > 0.5)) return "tau must be > 1/2 (positive viscosity)";
    if (!(p->rho0 > 0)) return "rho0 must be > 0";
    if (!(p->dt == 1.0)) return "dt must be 1 (lattice units: one LB time unit per coupled step)";
    if (!(p->gamma >= 0)) return "gamma must be >= 0";
    if (p->store < 0 || p->store > 2) return "store must be LBMD_F32, LBMD_F16_SHIFTED or LBMD_BF16_SHIFTED";
    if (p->forcing < 0 || p->forcing > 3) return "unknown forcing";
    if (p->force_dir < 0 || p->force_dir > 2 || p->force_wave_axis < 0 || p->force_wave_axis > 2)
        return "force_dir and force_wave_axis must be 0, 1 or 2";
    if (!std::isfinite(p->force_amp)) return "force_amp must be finite";
    if (p->walls_z != 0 && p->walls_z != 1) return "walls_z must be 0 or 1";
    if (p->walls_z && p->nz < 2) return "walls_z needs nz >= 2";
    if (p->deterministic != 0 && p->deterministic != 1) return "deterministic must be 0 or 1";
    if (p->check_every < 0) return "check_every must be >= 0";
    if (n_atoms < 0) return "n_atoms must be >= 0";
    if (n_bonds < 0) return "n_bonds must be >= 0";
    if (n_atoms > 0) {
        if (!mass) return "mass is NULL";
        for (int a = 0; a < n_atoms; ++a)
            if (!(mass[a] > 0) || !std::isfinite(mass[a])) return "masses must be positive and finite";
        if (p->n_md < 1) return "n_md must be >= 1";
        if (!(p->lj_sigma > 0) || !(p->lj_rcut_over_sigma > 0) || !(p->lj_eps >= 0)) return "invalid LJ parameters";
        if (!(p->skin >= 0)) return "skin must be >= 0";
        const double rc = p->lj_sigma * p->lj_rcut_over_sigma;
        const double side = rc + p->skin;
        const int L[3] = {p->nx, p->ny, p->nz};
        for (int d = 0; d < 3; ++d) {
            const int nc = (int)std::floor((double)L[d] / side);
            if (nc < 3) return "each box side must hold at least 3 pair-search cells (side >= 3 (rcut + skin))";
        }
    }
    if (n_bonds > 0) {
        if (!bonds || !bond_k || !bond_r0) return "bond arrays are NULL";
        for (int b = 0; b < n_bonds; ++b) {
            const int i = bonds[2 * b], j = bonds[2 * b + 1];
            if (i < 0 || j < 0 || i >= n_atoms || j >= n_atoms || i == j) return "bond index out of range";
            if (!std::isfinite(bond_k[b]) || !std::isfinite(bond_r0[b]) || bond_r0[b] < 0) return "invalid bond";
        }
    }
    return "";
}

void fill_physics(lbmd_t h) {
    const lbmd_params &p = h->p;
    Lat &L = h->L;
    L.nx = p.nx;
    L.ny = p.ny;
    L.nz = p.nz;
    L.N = (size_t)p.nx * p.ny * p.nz;
    L.omega = (float)(1.0 / p.tau);
    L.rho0 = (float)p.rho0;
    L.walls = p.walls_z;
    L.forcing = p.forcing;
    L.famp = (float)p.force_amp;
    L.fdir = p.force_dir;
    L.faxis = p.force_wave_axis;
    // Thermal noise amplitudes a_k = sqrt(mu (1 - (1 - omega)^2) / b_k),
    // mu = rho0 kT / c_s^2, b_k = sum_i w_i e_k(c_i)^2, in FP64.
    L.thermal = h->kT > 0.0;
    L.key0 = (unsigned)(h->seed & 0xffffffffu);
    L.key1 = (unsigned)(h->seed >> 32);
    {
        const double om = 1.0 / p.tau, g = 1.0 - om, mu = 3.0 * p.rho0 * h->kT;
        for (int k = 4; k < Q; ++k) {
            double b = 0.0;
            for (int i = 0; i < Q; ++i) {
                const double wi = i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
                b += wi * (double)emode(k, i) * (double)emode(k, i);
            }
            L.namp[k - 4] = (float)std::sqrt(mu * (1.0 - g * g) / b);
        }
    }

    AtomArgs &A = h->A;
    A.na = h->na;
    A.n_md = p.n_md > 0 ? p.n_md : 1;
    A.dt = (float)(1.0 / A.n_md);
    A.hdt = (float)(0.5 / A.n_md);
    A.gamma = (float)p.gamma;
    const double rc = p.lj_sigma * p.lj_rcut_over_sigma;
    A.lj_sig2 = (float)(p.lj_sigma * p.lj_sigma);
    A.lj_24eps = (float)(24.0 * p.lj_eps);
    const double sr6 = std::pow(p.lj_sigma / rc, 6.0);
    A.lj_fc = (float)(24.0 * p.lj_eps * (2.0 * sr6 * sr6 - sr6) / rc);
    A.rc2f = (float)(rc * rc);
    A.rl2 = (float)((rc + p.skin) * (rc + p.skin));
    A.half_skin2 = (float)(0.25 * p.skin * p.skin);
    A.det = p.deterministic;
    A.rc2d = rc * rc;
    const int Ls[3] = {p.nx, p.ny, p.nz};
    for (int d = 0; d < 3; ++d) {
        A.nc[d] = h->na > 0 ? (int)std::floor((double)Ls[d] / (rc + p.skin)) : 3;
        A.fold[d] = A.nc[d] < kFold ? A.nc[d] : kFold;
        A.fmask[d] = A.nc[d] <= kFold ? -1 : kFold - 1;
        A.Ld[d] = (double)Ls[d];
        A.hd[d] = (double)Ls[d] / A.nc[d];
        A.h[d] = (float)A.hd[d];
        A.inv_h[d] = (float)(A.nc[d] / (double)Ls[d]);
        A.Lf[d] = (float)Ls[d];
        A.inv_Lf[d] = (float)(1.0 / Ls[d]);
        double B = 1.0;
        while (B < 2.0 * Ls[d]) B *= 2.0;
        A.offd[d] = B + 0.5 * (B - Ls[d]);
        A.off[d] = (float)A.offd[d];
    }
    A.cap = kCap;
    // Half-size cells while each axis folds at most twice (a bucket then
    // stacks cells 128 apart at most once); coarse cells on larger boxes.
    bool fine = true;
    for (int d = 0; d < 3; ++d) fine = fine && std::floor((double)Ls[d] / (0.5 * (rc + p.skin))) <= 2 * kFold;
    A.bwin = fine ? 5 : 3;
    for (int d = 0; d < 3; ++d) {
        A.bnc[d] = h->na == 0 ? 6 : fine ? (int)std::floor((double)Ls[d] / (0.5 * (rc + p.skin))) : A.nc[d];
        // Folded axes: cells 128 apart share a bucket, and across the
        // periodic wrap such cells are only (bnc mod 128) apart. Keep that
        // at 0 or >= 7 (a few cells fewer, each slightly larger), so no
        // search window of up to 7 consecutive cells meets a bucket twice.
        if (A.bnc[d] > kFold && A.bnc[d] % kFold < kMaxWindow) A.bnc[d] -= A.bnc[d] % kFold;
        A.bfold[d] = A.bnc[d] < kFold ? A.bnc[d] : kFold;
        A.bfmask[d] = A.bnc[d] <= kFold ? -1 : kFold - 1;
        A.bh[d] = (float)((double)Ls[d] / A.bnc[d]);
        A.binv_h[d] = (float)(A.bnc[d] / (double)Ls[d]);
    }
    A.bcap = fine ? kCapFine : kCap;
    A.nl[0] = p.nx;
    A.nl[1] = p.ny;
    A.nl[2] = p.nz;
    A.walls = p.walls_z;
    h->C.L = L;
    h->C.na = h->na;
}

void destroy_graph(lbmd_t h) {
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
    h->node_t0 = h->node_t1 = h->node_m0 = h->node_m1 = nullptr;
}

lbmd_status enqueue_step(lbmd_t h) {
    // Lattice branch.
    CK(h, cudaEventRecord(h->ev_fork, h->s_main));
    CK(h, cudaStreamWaitEvent(h->s_lat, h->ev_fork, 0));
    CK(h, cudaEventRecordWithFlags(h->ev_t0, h->s_lat, cudaEventRecordExternal));
    CK(h, launch_lb_step(h->p.store, h->L, h->pop, h->ds, h->s_lat));
    CK(h, cudaEventRecordWithFlags(h->ev_t1, h->s_lat, cudaEventRecordExternal));
    CK(h, cudaEventRecord(h->ev_join, h->s_lat));
    // Solute branch, beside the lattice branch (at 512^3 a schedule that
    // waited for the lattice kernel before the substeps measured the same).
    if (h->na > 0) {
        CK(h, launch_md_sort(h->A, h->s_main));
        CK(h, launch_interp(h->p.store, h->C, h->A, h->pop, h->s_main));
        CK(h, cudaEventRecordWithFlags(h->ev_m0, h->s_main, cudaEventRecordExternal));
        for (int k = 0; k <= h->A.n_md; ++k) CK(h, launch_md_substep(h->A, k, h->s_main));
        CK(h, cudaEventRecordWithFlags(h->ev_m1, h->s_main, cudaEventRecordExternal));
        CK(h, launch_spread(h->C, h->s_main));
    }
    CK(h, cudaStreamWaitEvent(h->s_main, h->ev_join, 0));
    CK(h, launch_lb_fix(h->p.store, h->L, h->pop, h->C, h->fix_grid, h->s_main));
    return LBMD_OK;
}

lbmd_status build_graph(lbmd_t h) {
    destroy_graph(h);
    if (h->lat_dev) {  // every setter that changes L rebuilds the graph
        CK(h, cudaMemcpyAsync(h->lat_dev, &h->L, sizeof(Lat), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    CK(h, cudaStreamBeginCapture(h->s_main, cudaStreamCaptureModeThreadLocal));
    lbmd_status s = enqueue_step(h);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->s_main, &g);
    if (s != LBMD_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    h->graph = g;
    CK(h, cudaGraphInstantiate(&h->exec, h->graph, 0));
    size_t n = 0;
    CK(h, cudaGraphGetNodes(h->graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    CK(h, cudaGraphGetNodes(h->graph, nodes.data(), &n));
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        CK(h, cudaGraphNodeGetType(nd, &t));
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        CK(h, cudaGraphEventRecordNodeGetEvent(nd, &ev));
        if (ev == h->ev_t0) h->node_t0 = nd;
        if (ev == h->ev_t1) h->node_t1 = nd;
        if (ev == h->ev_m0) h->node_m0 = nd;
        if (ev == h->ev_m1) h->node_m1 = nd;
    }
    return LBMD_OK;
}

lbmd_status read_flags(lbmd_t h) {
    int flags = 0;
    CK(h, cudaMemcpyAsync(&flags, &h->ds->flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (!flags) return LBMD_OK;
    const int zero = 0;
    CK(h, cudaMemcpyAsync(&h->ds->flags, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (flags & FLAG_NONFINITE) return fail(h, LBMD_ERR_NONFINITE, "non-finite value in the lattice or the atoms");
    if (flags & FLAG_CELL)
        return fail(h, LBMD_ERR_CELL, "a pair-search bucket overflowed: forces of a step missed pairs");
    if (flags & FLAG_WALL) return fail(h, LBMD_ERR_STATE, "an atom's interpolation stencil crossed a z wall");
    return fail(h, LBMD_ERR_STATE, "touched-node list overflowed");
}

// Copies n bytes from a caller buffer into device memory (staging helper).
lbmd_status to_device(lbmd_t h, void *dst, const void *src, size_t n, int on_device) {
    CK(h, cudaMemcpyAsync(dst, src, n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    return LBMD_OK;
}

// Device staging area for calls with host pointers, grown on demand and kept
// for the handle's lifetime (so repeated host-pointer calls allocate nothing).
cudaError_t stage(lbmd_t h, size_t bytes, void **out) {
    if (h->stage_bytes < bytes) {
        if (h->stage) {
            cudaStreamSynchronize(h->stream);
            cudaFree(h->stage);
            h->stage = nullptr;
            h->stage_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&h->stage, bytes);
        if (e != cudaSuccess) return e;
        h->stage_bytes = bytes;
    }
    *out = h->stage;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// lbmd_backward support: checkpoints of the raw state, restore, and the
// recording re-run of one step.

lbmd_status adj_alloc(lbmd_t h, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc (adjoint)");
    h->adj_allocs.push_back(*p);
    return LBMD_OK;
}

lbmd_status adj_prepare(lbmd_t h, int n_steps, int K) {
    const int nseg = (n_steps + K - 1) / K;
    if (h->adj_ckpts >= nseg + 1 && h->adj_seg >= K) return LBMD_OK;
    for (void *p : h->adj_allocs) cudaFree(p);
    h->adj_allocs.clear();
    const size_t N = h->L.N, na = (size_t)h->na, na3 = 3 * na, nm = (size_t)h->A.n_md + 1;
    const size_t lat = N * Q * store_bytes(h->p.store);
    void *p;
    const int C = nseg + 1;
    TRY(adj_alloc(h, &h->ck_lat, lat * C));
    TRY(adj_alloc(h, &p, na3 * sizeof(double) * C)); h->ck_X = (double *)p;
    TRY(adj_alloc(h, &p, na3 * sizeof(float) * C)); h->ck_V = (float *)p;
    TRY(adj_alloc(h, &p, na3 * sizeof(float) * C)); h->ck_F = (float *)p;
    TRY(adj_alloc(h, &h->seg_lat, lat * K));
    TRY(adj_alloc(h, &p, na3 * sizeof(double) * K)); h->seg_X = (double *)p;
    TRY(adj_alloc(h, &p, na3 * sizeof(float) * K)); h->seg_V = (float *)p;
    TRY(adj_alloc(h, &p, na3 * sizeof(float) * K)); h->seg_F = (float *)p;
    TRY(adj_alloc(h, &p, nm * na * sizeof(float4))); h->recP = (float4 *)p;
    TRY(adj_alloc(h, &p, nm * na * sizeof(float4))); h->recL = (float4 *)p;
    TRY(adj_alloc(h, &p, nm * na3 * sizeof(float))); h->recV = (float *)p;
    TRY(adj_alloc(h, &p, nm * na3 * sizeof(float))); h->recF = (float *)p;
    TRY(adj_alloc(h, &p, N * Q * sizeof(float))); h->hat[0] = (float *)p;
    TRY(adj_alloc(h, &p, N * Q * sizeof(float))); h->hat[1] = (float *)p;
    AdjArgs &D = h->D;
    TRY(adj_alloc(h, &p, N * sizeof(float4))); D.Ghat = (float4 *)p;
    TRY(adj_alloc(h, &p, N * sizeof(float4))); D.Uhat = (float4 *)p;
    float **arrs[6] = {&D.xhat, &D.vhat, &D.p, &D.Jhat, &D.Uat_hat, &D.xw};
    for (float **a : arrs) {
        TRY(adj_alloc(h, &p, na3 * sizeof(float)));
        *a = (float *)p;
    }
    TRY(adj_alloc(h, &p, na * sizeof(double))); D.gam_acc = (double *)p;
    TRY(adj_alloc(h, &p, 2 * sizeof(double))); D.par_acc = (double *)p;
    h->adj_blocks = adj_lb_blocks(h->L);
    TRY(adj_alloc(h, &p, 2 * (size_t)h->adj_blocks * sizeof(double))); D.partials = (double *)p;
    const size_t B = (size_t)h->A.fold[0] * h->A.fold[1] * h->A.fold[2];
    TRY(adj_alloc(h, &p, B * sizeof(int))); h->adj_count = (int *)p;
    TRY(adj_alloc(h, &p, B * h->A.cap * sizeof(int))); h->adj_slot = (int *)p;
    TRY(adj_alloc(h, &p, 8 * sizeof(double))); h->obs_acc = (double *)p;
    h->adj_ckpts = C;
    h->adj_seg = K;
    return LBMD_OK;
}

// Saves the raw state (current storage buffer, X, V, cached F) into slot i of
// the checkpoints (ck = true) or of the segment store.
lbmd_status adj_save(lbmd_t h, int i, bool ck) {
    const size_t N = h->L.N, na3 = 3 * (size_t)h->na;
    const size_t lat = N * Q * store_bytes(h->p.store);
    char *L = (char *)(ck ? h->ck_lat : h->seg_lat) + lat * i;
    cudaStream_t s = h->stream;
    CK(h, cudaMemcpyAsync(L, h->pop[h->steps & 1], lat, cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync((ck ? h->ck_X : h->seg_X) + na3 * i, h->A.X, na3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync((ck ? h->ck_V : h->seg_V) + na3 * i, h->A.V, na3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync((ck ? h->ck_F : h->seg_F) + na3 * i, h->A.F, na3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return LBMD_OK;
}

// Restores slot i as the current state, step counter 0 (buffer 0), with fresh
// buckets, touched tags and neighbour lists, and the saved cached force.
lbmd_status adj_restore(lbmd_t h, int i, bool ck) {
    const size_t N = h->L.N, na = (size_t)h->na, na3 = 3 * na;
    const size_t lat = N * Q * store_bytes(h->p.store);
    cudaStream_t s = h->stream;
    const char *L = (const char *)(ck ? h->ck_lat : h->seg_lat) + lat * i;
    CK(h, cudaMemcpyAsync(h->pop[0], L, lat, cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemsetAsync(h->ds, 0, sizeof(DevState), s));
    const int one = 1;
    CK(h, cudaMemcpyAsync(&h->ds->nl_flag[0], &one, sizeof(int), cudaMemcpyHostToDevice, s));
    CK(h, cudaMemsetAsync(h->C.tag, 0, N * sizeof(int), s));
    CK(h, cudaMemsetAsync(h->C.G, 0, N * sizeof(float4), s));
    CK(h, cudaMemcpyAsync(h->A.X, (ck ? h->ck_X : h->seg_X) + na3 * i, na3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync(h->A.V, (ck ? h->ck_V : h->seg_V) + na3 * i, na3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    const size_t B = (size_t)h->A.bfold[0] * h->A.bfold[1] * h->A.bfold[2];
    for (int g = 0; g < 3; ++g) {
        CK(h, cudaMemsetAsync(h->A.count[g], 0, B * sizeof(int), s));
        CK(h, cudaMemsetAsync(h->A.bucket[g], 0, na * sizeof(int), s));
    }
    CK(h, cudaMemsetAsync(h->A.J, 0, na3 * sizeof(float), s));
    CK(h, cudaMemsetAsync(h->A.U, 0, na3 * sizeof(float), s));
    CK(h, cudaMemsetAsync(h->A.nnb, 0, na * sizeof(int), s));
    CK(h, cudaMemsetAsync(h->A.D, 0, na3 * sizeof(float), s));
    CK(h, cudaMemcpyAsync(h->A.order, h->ident, na * sizeof(int), cudaMemcpyDeviceToDevice, s));
    CK(h, launch_md_prime(h->A, s));
    CK(h, cudaMemcpyAsync(h->A.F, (ck ? h->ck_F : h->seg_F) + na3 * i, na3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    h->steps = 0;
    return LBMD_OK;
}

// One coupled step launched directly (not from the graph), recording the
// substep positions, input velocities and forces, and keeping G and the
// touched-node list for the reverse pass.
lbmd_status enqueue_record_step(lbmd_t h) {
    cudaStream_t s = h->stream;
    AtomArgs A = h->A;
    A.recP = h->recP;
    A.recL = h->recL;
    A.recV = h->recV;
    A.recF = h->recF;
    CouplingArgs C = h->C;
    C.keep = 1;
    CK(h, launch_md_sort(A, s));
    CK(h, launch_interp(h->p.store, C, A, h->pop, s));
    for (int k = 0; k <= A.n_md; ++k) CK(h, launch_md_substep(A, k, s));
    CK(h, launch_spread(C, s));
    CK(h, launch_lb_step(h->p.store, h->L, h->pop, h->ds, s));
    CK(h, launch_lb_fix(h->p.store, h->L, h->pop, C, h->fix_grid, s));
    ++h->steps;
    return LBMD_OK;
}

// Optimal superposition (Horn's quaternion form of the least-squares rotation,
// J. Opt. Soc. Am. A 4, 629 (1987)): for centred coordinate sets x and y with
// S[a][b] = sum_i x_ia y_ib, the rotation R maximising sum_i y_i . R x_i is
// given by the unit quaternion of the largest eigenvalue lambda of the
// symmetric 4x4 matrix N(S) below, and that maximum is lambda, so the
// least-squares residual is |x|^2 + |y|^2 - 2 lambda. Eigenpairs by cyclic
// Jacobi rotations in FP64. Returns lambda; R is row-major, y ~ R x.
double horn_rotation(const double S[9], double R[9]) {
    const double Sxx = S[0], Sxy = S[1], Sxz = S[2], Syx = S[3], Syy = S[4], Syz = S[5], Szx = S[6], Szy = S[7],
                 Szz = S[8];
    double N[4][4] = {{Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx},
                      {Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz},
                      {Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy},
                      {Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz}};
    double V[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
    // Cyclic Jacobi sweeps on the symmetric 4x4 matrix.
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int p = 0; p < 4; ++p)
            for (int q = 0; q < 4; ++q) {
                tot += N[p][q] * N[p][q];
                if (p != q) off += N[p][q] * N[p][q];
            }
        if (off <= 1e-32 * tot) break;
        for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 4; ++q) {
                if (N[p][q] == 0.0) continue;
                const double theta = (N[q][q] - N[p][p]) / (2.0 * N[p][q]);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 4; ++k) {
                    const double a = N[k][p], b = N[k][q];
                    N[k][p] = c * a - s * b;
                    N[k][q] = s * a + c * b;
                }
                for (int k = 0; k < 4; ++k) {
                    const double a = N[p][k], b = N[q][k];
                    N[p][k] = c * a - s * b;
                    N[q][k] = s * a + c * b;
                }
                for (int k = 0; k < 4; ++k) {
                    const double a = V[k][p], b = V[k][q];
                    V[k][p] = c * a - s * b;
                    V[k][q] = s * a + c * b;
                }
            }
    }
    int best = 0;
    for (int k = 1; k < 4; ++k)
        if (N[k][k] > N[best][best]) best = k;
    double q0 = V[0][best], q1 = V[1][best], q2 = V[2][best], q3 = V[3][best];
    const double nq = std::sqrt(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    q0 /= nq; q1 /= nq; q2 /= nq; q3 /= nq;
    R[0] = q0 * q0 + q1 * q1 - q2 * q2 - q3 * q3;
    R[1] = 2 * (q1 * q2 - q0 * q3);
    R[2] = 2 * (q1 * q3 + q0 * q2);
    R[3] = 2 * (q1 * q2 + q0 * q3);
    R[4] = q0 * q0 - q1 * q1 + q2 * q2 - q3 * q3;
    R[5] = 2 * (q2 * q3 - q0 * q1);
    R[6] = 2 * (q1 * q3 - q0 * q2);
    R[7] = 2 * (q2 * q3 + q0 * q1);
    R[8] = q0 * q0 - q1 * q1 - q2 * q2 + q3 * q3;
    return N[best][best];
}

void ana_free(lbmd_t h) {
    for (void *p : h->ana_allocs) cudaFree(p);
    h->ana_allocs.clear();
    h->ana = AnaArgs{};
    h->ana_cov = nullptr;
    h->ana_frames = h->ana_max = 0;
}

lbmd_status ana_alloc(lbmd_t h, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc (analysis)");
    h->ana_allocs.push_back(*p);
    return LBMD_OK;
}

// Bytes of one population buffer in the handle's storage format.
size_t pop_bytes(lbmd_t h) { return h->L.N * Q * store_bytes(h->p.store); }

lbmd_status finish_state(lbmd_t h, const double *x, const float *v, int on_device);

}  // namespace

extern "C" {

int lbmd_version(void) { return 1; }

const char *lbmd_last_error(lbmd_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

lbmd_status lbmd_create(const lbmd_params *params, int n_atoms, const double *mass, int n_bonds,
                        const int32_t *bonds, const double *bond_k, const double *bond_r0, void *cuda_stream,
                        lbmd_t *out) {
    if (!out) return fail(nullptr, LBMD_ERR_ARG, "out is NULL");
    *out = nullptr;
    std::string why = validate(params, n_atoms, mass, n_bonds, bonds, bond_k, bond_r0);
    if (!why.empty()) return fail(nullptr, LBMD_ERR_ARG, why);

    lbmd_t h = new (std::nothrow) lbmd_s();
    if (!h) return fail(nullptr, LBMD_ERR_ALLOC, "host allocation failed");
    h->p = *params;
    h->stream = (cudaStream_t)cuda_stream;
    h->na = n_atoms;
    h->nb = n_bonds;
    fill_physics(h);

    auto bail = [&](lbmd_status s) {
        g_create_error = h->err;
        lbmd_destroy(h);
        return s;
    };
#define CREATE_TRY(expr)                                                                                            \
    do {                                                                                                            \
        lbmd_status s_ = (expr);                                                                                    \
        if (s_ != LBMD_OK) return bail(s_);                                                                         \
    } while (0)
#define CREATE_CK(call)                                                                                             \
    do {                                                                                                            \
        cudaError_t e_ = (call);                                                                                    \
        if (e_ != cudaSuccess) return bail(cuda_fail(h, e_, #call));                                                \
    } while (0)

    int lo = 0, hi = 0;
    CREATE_CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CREATE_CK(cudaStreamCreateWithPriority(&h->s_main, cudaStreamNonBlocking, hi));
    CREATE_CK(cudaStreamCreateWithPriority(&h->s_lat, cudaStreamNonBlocking, lo));
    CREATE_CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    CREATE_CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    CREATE_CK(cudaEventCreate(&h->ev_t0));
    CREATE_CK(cudaEventCreate(&h->ev_t1));
    CREATE_CK(cudaEventCreate(&h->ev_m0));
    CREATE_CK(cudaEventCreate(&h->ev_m1));

    const Lat &L = h->L;
    const size_t pop_bytes = L.N * Q * store_bytes(h->p.store);
    CREATE_TRY(dalloc(h, &h->pop[0], pop_bytes));
    CREATE_TRY(dalloc(h, &h->pop[1], pop_bytes));
    CREATE_TRY(dalloc_t(h, &h->ds, 1));
    CREATE_TRY(dalloc_t(h, &h->C.G, L.N));
    CREATE_TRY(dalloc_t(h, &h->C.tag, L.N));
    h->red_blocks = (int)std::min<size_t>((L.N + 255) / 256, 1024);
    CREATE_TRY(dalloc_t(h, &h->red, (size_t)h->red_blocks * 4));
    CREATE_TRY(dalloc_t(h, &h->red_out, 8));
    CREATE_CK(cudaMemsetAsync(h->C.G, 0, L.N * sizeof(float4), h->stream));
    CREATE_CK(cudaMemsetAsync(h->C.tag, 0, L.N * sizeof(int), h->stream));
    CREATE_CK(cudaMemsetAsync(h->ds, 0, sizeof(DevState), h->stream));
    {
        // Kolmogorov wave shape per lattice row, in FP64 then rounded once.
        const int nax = h->p.force_wave_axis == 0 ? h->p.nx : (h->p.force_wave_axis == 1 ? h->p.ny : h->p.nz);
        std::vector<float> shape(nax);
        for (int c = 0; c < nax; ++c) shape[c] = (float)std::sin(6.283185307179586477 * c / nax);
        float *d_shape;
        CREATE_TRY(dalloc_t(h, &d_shape, (size_t)nax));
        CREATE_CK(cudaMemcpy(d_shape, shape.data(), nax * sizeof(float), cudaMemcpyHostToDevice));
        h->L.kshape = d_shape;
        h->C.L.kshape = d_shape;  // the coupling kernels' copy of the lattice
    }

    AtomArgs &A = h->A;
    CouplingArgs &C = h->C;
    A.ds = C.ds = h->ds;
    const int na = h->na;
    const size_t na3 = (size_t)3 * (na > 0 ? na : 1);
    if (na > 0) {
        CREATE_TRY(dalloc_t(h, &A.X, na3));
        CREATE_TRY(dalloc_t(h, &A.P[0], (size_t)na));
        CREATE_TRY(dalloc_t(h, &A.P[1], (size_t)na));
        CREATE_TRY(dalloc_t(h, &A.L[0], (size_t)na));
        CREATE_TRY(dalloc_t(h, &A.L[1], (size_t)na));
        CREATE_TRY(dalloc_t(h, &A.P0, na3));
        CREATE_TRY(dalloc_t(h, &A.R0, na3));
        CREATE_TRY(dalloc_t(h, &A.V, na3));
        CREATE_TRY(dalloc_t(h, &A.F, na3));
        CREATE_TRY(dalloc_t(h, &A.U, na3));
        CREATE_TRY(dalloc_t(h, &A.J, na3));
        CREATE_TRY(dalloc_t(h, &A.mass, (size_t)na));
        CREATE_TRY(dalloc_t(h, &A.inv_m, (size_t)na));
        CREATE_TRY(dalloc_t(h, &C.base, na3));
        CREATE_TRY(dalloc_t(h, &C.frac, na3));
        C.touched_cap = 8 * na;
        CREATE_TRY(dalloc_t(h, &C.touched, (size_t)C.touched_cap));
        if (h->p.deterministic) {  // node -> touched slot, and the fixed-point sums per slot
            CREATE_TRY(dalloc_t(h, &C.tslot, L.N));
            CREATE_TRY(dalloc_t(h, &C.gfix, 3 * (size_t)C.touched_cap));
            CREATE_CK(cudaMemsetAsync(C.tslot, 0, L.N * sizeof(int), h->stream));
            CREATE_CK(cudaMemsetAsync(C.gfix, 0, 3 * (size_t)C.touched_cap * sizeof(long long), h->stream));
        }
        const size_t B = (size_t)A.bfold[0] * A.bfold[1] * A.bfold[2];
        for (int g = 0; g < 3; ++g) {
            CREATE_TRY(dalloc_t(h, &A.count[g], B));
            CREATE_TRY(dalloc_t(h, &A.slot[g], B * A.bcap));
            CREATE_TRY(dalloc_t(h, &A.bucket[g], (size_t)na));
            CREATE_TRY(dalloc_t(h, &A.sidx[g], (size_t)na));
        }
        CREATE_TRY(dalloc_t(h, &A.order, (size_t)na));
        CREATE_TRY(dalloc_t(h, &A.scode, (size_t)na));
        CREATE_TRY(dalloc_t(h, &h->ident, (size_t)na));
        CREATE_TRY(dalloc_t(h, &A.nbr, (size_t)na * NL_MAX));
        CREATE_TRY(dalloc_t(h, &A.nnb, (size_t)na));
        CREATE_TRY(dalloc_t(h, &A.D, na3));
        CREATE_TRY(dalloc_t(h, &A.scan_local, (size_t)kMortonCodes));
        CREATE_TRY(dalloc_t(h, &A.scan_block, kMortonCodes / 1024));
        // Topology: masses and a symmetric bond CSR.
        std::vector<float> m(na), im(na);
        for (int a = 0; a < na; ++a) {
            m[a] = (float)mass[a];
            im[a] = (float)(1.0 / mass[a]);
        }
        std::vector<int> start(na + 1, 0), part(2 * (size_t)n_bonds + 1), fill(na, 0);
        std::vector<float> bk(2 * (size_t)n_bonds + 1), br0(2 * (size_t)n_bonds + 1);
        for (int b = 0; b < n_bonds; ++b) {
            start[bonds[2 * b] + 1]++;
            start[bonds[2 * b + 1] + 1]++;
        }
        for (int a = 0; a < na; ++a) start[a + 1] += start[a];
        for (int b = 0; b < n_bonds; ++b) {
            const int i = bonds[2 * b], j = bonds[2 * b + 1];
            const int si = start[i] + fill[i]++, sj = start[j] + fill[j]++;
            part[si] = j;
            part[sj] = i;
            bk[si] = bk[sj] = (float)bond_k[b];
            br0[si] = br0[sj] = (float)bond_r0[b];
        }
        int *d_start, *d_part;
        float *d_bk, *d_br0;
        CREATE_TRY(dalloc_t(h, &d_start, (size_t)na + 1));
        CREATE_TRY(dalloc_t(h, &d_part, part.size()));
        CREATE_TRY(dalloc_t(h, &d_bk, bk.size()));
        CREATE_TRY(dalloc_t(h, &d_br0, br0.size()));
        CREATE_CK(cudaMemcpy(d_start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice));
        CREATE_CK(cudaMemcpy(d_part, part.data(), part.size() * sizeof(int), cudaMemcpyHostToDevice));
        CREATE_CK(cudaMemcpy(d_bk, bk.data(), bk.size() * sizeof(float), cudaMemcpyHostToDevice));
        CREATE_CK(cudaMemcpy(d_br0, br0.data(), br0.size() * sizeof(float), cudaMemcpyHostToDevice));
        CREATE_CK(cudaMemcpy(A.mass, m.data(), na * sizeof(float), cudaMemcpyHostToDevice));
        CREATE_CK(cudaMemcpy(A.inv_m, im.data(), na * sizeof(float), cudaMemcpyHostToDevice));
        A.bstart = d_start;
        A.bpart = d_part;
        A.bk = d_bk;
        A.br0 = d_br0;
        C.X = A.X;
        C.U = A.U;
        C.J = A.J;
        C.order = A.order;
    }
    h->fix_grid = na > 0 ? std::min((C.touched_cap + 255) / 256, kFixBlocks) : 1;
    CREATE_CK(cudaStreamSynchronize(h->stream));
    *out = h;
#undef CREATE_TRY
#undef CREATE_CK
    return LBMD_OK;
}

void lbmd_destroy(lbmd_t h) {
    if (!h) return;
    if (h->stream || h->s_main) cudaStreamSynchronize(h->stream);
    destroy_graph(h);
    for (void *p : h->allocs) cudaFree(p);
    for (void *p : h->adj_allocs) cudaFree(p);
    for (void *p : h->ana_allocs) cudaFree(p);
    if (h->stage) cudaFree(h->stage);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_t0) cudaEventDestroy(h->ev_t0);
    if (h->ev_t1) cudaEventDestroy(h->ev_t1);
    if (h->ev_m0) cudaEventDestroy(h->ev_m0);
    if (h->ev_m1) cudaEventDestroy(h->ev_m1);
    if (h->s_main) cudaStreamDestroy(h->s_main);
    if (h->s_lat) cudaStreamDestroy(h->s_lat);
    delete h;
}

lbmd_status lbmd_set_state(lbmd_t h, const float *f, const float *rho, const float *u, const double *x,
                           const float *v, int on_device) {
    const Range range("lbmd_set_state");
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (!f && (!rho || !u)) return fail(h, LBMD_ERR_ARG, "give f, or rho and u");
    if (h->na > 0 && (!x || !v)) return fail(h, LBMD_ERR_ARG, "x and v are required when n_atoms > 0");
    const Lat &L = h->L;
    const float *df = f, *drho = rho, *du = u;
    if (!on_device) {
        void *p;
        CK(h, stage(h, L.N * (f ? Q : 4) * sizeof(float), &p));
        if (f) {
            TRY(to_device(h, p, f, L.N * Q * sizeof(float), 0));
            df = (const float *)p;
        } else {
            TRY(to_device(h, p, rho, L.N * sizeof(float), 0));
            TRY(to_device(h, (float *)p + L.N, u, 3 * L.N * sizeof(float), 0));
            drho = (const float *)p;
            du = (const float *)p + L.N;
        }
    }
    CK(h, launch_lb_init(h->p.store, L, h->pop[0], f ? df : nullptr, f ? nullptr : drho, f ? nullptr : du, h->stream));
    return finish_state(h, x, v, on_device);
}

lbmd_status lbmd_save_state(lbmd_t h, void *pop, double *x, float *v, int on_device) {
    const Range range("lbmd_save_state");
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (!h->state_set) return fail(h, LBMD_ERR_STATE, "lbmd_set_state has not been called");
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (pop) CK(h, cudaMemcpyAsync(pop, h->pop[h->steps & 1], pop_bytes(h), k, h->stream));
    if (h->na > 0) {
        if (x) CK(h, cudaMemcpyAsync(x, h->A.X, 3 * (size_t)h->na * sizeof(double), k, h->stream));
        if (v) CK(h, cudaMemcpyAsync(v, h->A.V, 3 * (size_t)h->na * sizeof(float), k, h->stream));
    }
    if (!on_device) CK(h, cudaStreamSynchronize(h->stream));
    return LBMD_OK;
}

lbmd_status lbmd_load_state(lbmd_t h, const void *pop, const double *x, const float *v, int on_device) {
    const Range range("lbmd_load_state");
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (!pop) return fail(h, LBMD_ERR_ARG, "pop is NULL");
    if (h->na > 0 && (!x || !v)) return fail(h, LBMD_ERR_ARG, "x and v are required when n_atoms > 0");
    TRY(to_device(h, h->pop[0], pop, pop_bytes(h), on_device));
    return finish_state(h, x, v, on_device);
}

}  // extern "C"

namespace {

// The part of setting a state shared by lbmd_set_state and lbmd_load_state,
// once the populations are in buffer 0: device state, touched tags and
// coupling force cleared, atoms uploaded with their first forces and cells,
// the lattice scanned for non-finite values.
lbmd_status finish_state(lbmd_t h, const double *x, const float *v, int on_device) {
    const Lat &L = h->L;
    CK(h, cudaMemsetAsync(h->ds, 0, sizeof(DevState), h->stream));
    CK(h, cudaMemsetAsync(h->C.tag, 0, L.N * sizeof(int), h->stream));
    CK(h, cudaMemsetAsync(h->C.G, 0, L.N * sizeof(float4), h->stream));
    if (h->C.gfix)
        CK(h, cudaMemsetAsync(h->C.gfix, 0, 3 * (size_t)h->C.touched_cap * sizeof(long long), h->stream));
    if (h->na > 0) {
        const size_t na3 = (size_t)3 * h->na;
        TRY(to_device(h, h->A.X, x, na3 * sizeof(double), on_device));
        TRY(to_device(h, h->A.V, v, na3 * sizeof(float), on_device));
        const size_t B = (size_t)h->A.bfold[0] * h->A.bfold[1] * h->A.bfold[2];
        for (int g = 0; g < 3; ++g) {
            CK(h, cudaMemsetAsync(h->A.count[g], 0, B * sizeof(int), h->stream));
            CK(h, cudaMemsetAsync(h->A.bucket[g], 0, h->na * sizeof(int), h->stream));
        }
        CK(h, cudaMemsetAsync(h->A.J, 0, na3 * sizeof(float), h->stream));
        {
            std::vector<int> ident(h->na);
            for (int i = 0; i < h->na; ++i) ident[i] = i;
            CK(h, cudaMemcpy(h->A.order, ident.data(), h->na * sizeof(int), cudaMemcpyHostToDevice));
            CK(h, cudaMemcpy(h->ident, ident.data(), h->na * sizeof(int), cudaMemcpyHostToDevice));
            CK(h, cudaMemsetAsync(h->A.nnb, 0, h->na * sizeof(int), h->stream));
            CK(h, cudaMemsetAsync(h->A.D, 0, na3 * sizeof(float), h->stream));
            const int one = 1;  // first force evaluation builds the lists
            CK(h, cudaMemcpyAsync(&h->ds->nl_flag[0], &one, sizeof(int), cudaMemcpyHostToDevice, h->stream));
        }
        CK(h, cudaMemsetAsync(h->A.U, 0, na3 * sizeof(float), h->stream));
        CK(h, launch_md_prime(h->A, h->stream));
    }
    // Scan the new lattice for NaN/Inf (raises the flag read below).
    CK(h, launch_lb_reduce(h->p.store, L, h->pop[0], h->red, h->red_blocks, h->ds, h->stream));
    if (!on_device) CK(h, cudaStreamSynchronize(h->stream));  // the caller may reuse its buffers
    h->state_set = true;
    h->steps = 0;
    return read_flags(h);
}

}  // namespace

extern "C" {

lbmd_status lbmd_step(lbmd_t h, int n_steps) {
    const Range range("lbmd_step");
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (n_steps < 0) return fail(h, LBMD_ERR_ARG, "n_steps must be >= 0");
    if (!h->state_set) return fail(h, LBMD_ERR_STATE, "lbmd_set_state has not been called");
    if (!h->exec) TRY(build_graph(h));
    for (int i = 0; i < n_steps; ++i) {
        CK(h, cudaGraphLaunch(h->exec, h->stream));
        ++h->steps;
        if (h->p.check_every > 0 && h->steps % h->p.check_every == 0) TRY(read_flags(h));
    }
    return LBMD_OK;
}

lbmd_status lbmd_get_fields(lbmd_t h, float *f, float *rho, float *u, double *x, float *v, int on_device) {
    const Range range("lbmd_get_fields");
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (!h->state_set) return fail(h, LBMD_ERR_STATE, "lbmd_set_state has not been called");
    const Lat &L = h->L;
    const void *cur = h->pop[h->steps & 1];
    if (f || rho || u) {
        float *df = f, *drho = rho, *du = u;
        if (!on_device) {
            void *p;
            CK(h, stage(h, L.N * (Q + 4) * sizeof(float), &p));
            float *base = (float *)p;
            df = f ? base : nullptr;
            drho = rho ? base + L.N * Q : nullptr;
            du = u ? base + L.N * (Q + 1) : nullptr;
        }
        CK(h, launch_lb_fields(h->p.store, L, cur, df, drho, du, h->ds, h->stream));
        if (!on_device) {
            if (f) CK(h, cudaMemcpyAsync(f, df, L.N * Q * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
            if (rho) CK(h, cudaMemcpyAsync(rho, drho, L.N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
            if (u) CK(h, cudaMemcpyAsync(u, du, 3 * L.N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        }
    }
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (h->na > 0) {
        if (x) CK(h, cudaMemcpyAsync(x, h->A.X, 3 * (size_t)h->na * sizeof(double), k, h->stream));
        if (v) CK(h, cudaMemcpyAsync(v, h->A.V, 3 * (size_t)h->na * sizeof(float), k, h->stream));
    }
    if (!on_device) CK(h, cudaStreamSynchronize(h->stream));
    return LBMD_OK;
}

lbmd_status lbmd_get_stats(lbmd_t h, double *mass, double mom_fluid[3], double mom_atoms[3]) {
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (!h->state_set) return fail(h, LBMD_ERR_STATE, "lbmd_set_state has not been called");
    const Lat &L = h->L;
    const void *cur = h->pop[h->steps & 1];
    CK(h, launch_lb_reduce(h->p.store, L, cur, h->red, h->red_blocks, h->ds, h->stream));
    CK(h, launch_reduce_finish(h->red, h->red_blocks, 4, h->red_out, h->stream));
    double out[7] = {0, 0, 0, 0, 0, 0, 0};
    if (h->na > 0) {
        const int nb = std::min(h->red_blocks, (h->na + 255) / 256);
        // Atom partials reuse the tail of the partial buffer after the lattice sum.
        CK(h, launch_atom_momentum(h->A.V, h->A.mass, h->na, h->red, nb, h->ds, h->stream));
        CK(h, launch_reduce_finish(h->red, nb, 3, h->red_out + 4, h->stream));
        CK(h, cudaMemcpyAsync(out, h->red_out, 7 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    } else {
        CK(h, cudaMemcpyAsync(out, h->red_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    if (mass) *mass = (double)L.N * h->p.rho0 + out[0];
    if (mom_fluid)
        for (int d = 0; d < 3; ++d) mom_fluid[d] = out[1 + d];
    if (mom_atoms)
        for (int d = 0; d < 3; ++d) mom_atoms[d] = out[4 + d];
    return read_flags(h);
}

lbmd_status lbmd_check(lbmd_t h) {
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    return read_flags(h);
}

lbmd_status lbmd_cell_list(lbmd_t h, int32_t *cell_of, int32_t *neighbours, int32_t *nc, int on_device) {
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (!h->state_set) return fail(h, LBMD_ERR_STATE, "lbmd_set_state has not been called");
    if (nc)
        for (int d = 0; d < 3; ++d) nc[d] = h->A.nc[d];
    if (h->na == 0 || (!cell_of && !neighbours)) return LBMD_OK;
    int *dc = cell_of, *dn = neighbours;
    if (!on_device) {
        void *p;
        CK(h, stage(h, 2 * (size_t)h->na * sizeof(int), &p));
        dc = cell_of ? (int *)p : nullptr;
        dn = neighbours ? (int *)p + h->na : nullptr;
    }
    CK(h, launch_md_diag(h->A, dc, dn, h->stream));
    if (!on_device) {
        if (cell_of) CK(h, cudaMemcpyAsync(cell_of, dc, h->na * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        if (neighbours)
            CK(h, cudaMemcpyAsync(neighbours, dn, h->na * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return LBMD_OK;
}

lbmd_status lbmd_set_physics(lbmd_t h, double gamma, double tau, double force_amp) {
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (!(tau > 0.5) || !(gamma >= 0) || !std::isfinite(force_amp) || !std::isfinite(gamma))
        return fail(h, LBMD_ERR_ARG, "need tau > 1/2, gamma >= 0 and a finite force_amp");
    h->p.gamma = gamma;
    h->p.tau = tau;
    h->p.force_amp = force_amp;
    fill_physics(h);
    destroy_graph(h);
    return LBMD_OK;
}

lbmd_status lbmd_set_charges(lbmd_t h, const double *charge, double coul_c, double coul_rc) {
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    AtomArgs &A = h->A;
    if (h->state_set)
        return fail(h, LBMD_ERR_STATE, "set the charges before lbmd_set_state (it computes the forces with them)");
    if (!charge) {
        A.coul = 0;
        A.q = nullptr;
        destroy_graph(h);
        return LBMD_OK;
    }
    if (h->na == 0) return fail(h, LBMD_ERR_ARG, "charges need atoms (n_atoms > 0)");
    const double rc = h->p.lj_sigma * h->p.lj_rcut_over_sigma;
    if (!(coul_rc > 0.0) || coul_rc > rc)
        return fail(h, LBMD_ERR_ARG, "coul_rc must be > 0 and <= the Lennard-Jones cutoff (the same pair lists)");
    if (!std::isfinite(coul_c)) return fail(h, LBMD_ERR_ARG, "coul_c must be finite");
    std::vector<float> q(h->na);
    for (int a = 0; a < h->na; ++a) {
        if (!std::isfinite(charge[a])) return fail(h, LBMD_ERR_ARG, "charges must be finite");
        q[a] = (float)charge[a];
    }
    if (!h->charge) TRY(dalloc_t(h, &h->charge, (size_t)h->na));
    CK(h, cudaMemcpyAsync(h->charge, q.data(), h->na * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    A.q = h->charge;
    A.coul = 1;
    A.coul_2c = (float)(2.0 * coul_c);
    A.coul_rc2 = (float)(coul_rc * coul_rc);
    A.coul_irc3 = (float)(1.0 / (coul_rc * coul_rc * coul_rc));
    destroy_graph(h);
    return LBMD_OK;
}

lbmd_status lbmd_set_reinterpolation(lbmd_t h, int on) {
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (on != 0 && on != 1) return fail(h, LBMD_ERR_ARG, "on must be 0 or 1");
    if (on && h->na == 0) return fail(h, LBMD_ERR_ARG, "re-interpolation needs atoms (n_atoms > 0)");
    if (on && h->p.deterministic)
        return fail(h, LBMD_ERR_ARG, "the deterministic mode covers the frozen-velocity coupling only");
    AtomArgs &A = h->A;
    CouplingArgs &C = h->C;
    if (on) {
        if (!h->unode) TRY(dalloc_t(h, &h->unode, h->L.N));
        // Each atom claims its stencil and one node of margin (4 x 4 x 4),
        // plus the nodes it reaches beyond them; a node enters once per step,
        // so N entries always suffice.
        const int cap = (int)std::min<size_t>(h->L.N, 256 * (size_t)h->na);
        if (C.touched_cap < cap) {
            int *t = nullptr;
            TRY(dalloc_t(h, &t, (size_t)cap));
            C.touched = t;
            C.touched_cap = cap;
            h->fix_grid = std::min((cap + 255) / 256, kFixBlocks);
        }
    }
    A.reinterp = C.reinterp = on;
    A.unode = C.unode = h->unode;
    A.G = C.G;
    if (on && !h->lat_dev) TRY(dalloc_t(h, &h->lat_dev, 1));
    A.lat = h->lat_dev;
    A.store = h->p.store;
    A.pop[0] = h->pop[0];
    A.pop[1] = h->pop[1];
    A.tag = C.tag;
    A.touched = C.touched;
    A.touched_cap = C.touched_cap;
    destroy_graph(h);
    return LBMD_OK;
}

lbmd_status lbmd_set_thermal(lbmd_t h, double kT, uint64_t seed) {
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (!(kT >= 0.0) || !std::isfinite(kT)) return fail(h, LBMD_ERR_ARG, "kT must be finite and >= 0");
    h->kT = kT;
    h->seed = seed;
    fill_physics(h);
    destroy_graph(h);
    return LBMD_OK;
}

lbmd_status lbmd_set_timing_events(lbmd_t h, void *ev_start, void *ev_stop) {
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if ((ev_start == nullptr) != (ev_stop == nullptr)) return fail(h, LBMD_ERR_ARG, "give both events or neither");
    if (!h->state_set) return fail(h, LBMD_ERR_STATE, "lbmd_set_state has not been called");
    if (!h->exec) TRY(build_graph(h));
    if (!h->node_t0 || !h->node_t1) return fail(h, LBMD_ERR_CUDA, "timing nodes missing from the step graph");
    cudaEvent_t a = ev_start ? (cudaEvent_t)ev_start : h->ev_t0;
    cudaEvent_t b = ev_stop ? (cudaEvent_t)ev_stop : h->ev_t1;
    CK(h, cudaGraphExecEventRecordNodeSetEvent(h->exec, h->node_t0, a));
    CK(h, cudaGraphExecEventRecordNodeSetEvent(h->exec, h->node_t1, b));
    return LBMD_OK;
}

lbmd_status lbmd_set_md_timing_events(lbmd_t h, void *ev_start, void *ev_stop) {
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if ((ev_start == nullptr) != (ev_stop == nullptr)) return fail(h, LBMD_ERR_ARG, "give both events or neither");
    if (!h->state_set) return fail(h, LBMD_ERR_STATE, "lbmd_set_state has not been called");
    if (h->na == 0) return fail(h, LBMD_ERR_ARG, "no atoms: the step has no substep kernels");
    if (!h->exec) TRY(build_graph(h));
    if (!h->node_m0 || !h->node_m1) return fail(h, LBMD_ERR_CUDA, "substep timing nodes missing from the step graph");
    cudaEvent_t a = ev_start ? (cudaEvent_t)ev_start : h->ev_m0;
    cudaEvent_t b = ev_stop ? (cudaEvent_t)ev_stop : h->ev_m1;
    CK(h, cudaGraphExecEventRecordNodeSetEvent(h->exec, h->node_m0, a));
    CK(h, cudaGraphExecEventRecordNodeSetEvent(h->exec, h->node_m1, b));
    return LBMD_OK;
}

}  // extern "C"

namespace {

// The rollout and reverse sweep of lbmd_backward; with grad_* given, also the
// adjoint of the initial state in the ABI's terms.
lbmd_status backward_impl(lbmd_t h, int n_steps, int ckpt_every, int observable, double *d_gamma, double *d_tau,
                          double *d_force_amp, double *obs, float *grad_f, float *grad_x, float *grad_v,
                          int on_device) {
    const Range range("lbmd_backward");
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (!h->state_set) return fail(h, LBMD_ERR_STATE, "lbmd_set_state has not been called");
    if (n_steps < 1 || ckpt_every < 1) return fail(h, LBMD_ERR_ARG, "need n_steps >= 1 and ckpt_every >= 1");
    if (observable != LBMD_OBS_DRAG_X && observable != LBMD_OBS_RG2) return fail(h, LBMD_ERR_ARG, "unknown observable");
    if (h->na == 0) return fail(h, LBMD_ERR_ARG, "the observables need atoms (n_atoms > 0)");
    if (h->kT > 0.0)
        return fail(h, LBMD_ERR_ARG, "the adjoint differentiates the deterministic step: set kT = 0 (lbmd_set_thermal)");
    if (h->A.reinterp)
        return fail(h, LBMD_ERR_ARG, "the adjoint covers the frozen-velocity coupling: turn re-interpolation off");
    if (h->p.deterministic)
        return fail(h, LBMD_ERR_ARG, "the adjoint runs with deterministic = 0 (its reverse sums use float atomics)");
    TRY(adj_prepare(h, n_steps, ckpt_every));
    cudaStream_t s = h->stream;
    const int K = ckpt_every, nseg = (n_steps + K - 1) / K;
    const int na = h->na;
    if (!h->exec) TRY(build_graph(h));

    // Forward pass with checkpoints, accumulating the observable.
    CK(h, cudaMemsetAsync(h->obs_acc, 0, 8 * sizeof(double), s));
    for (int n = 0; n < n_steps; ++n) {
        if (n % K == 0) TRY(adj_save(h, n / K, true));
        CK(h, cudaGraphLaunch(h->exec, s));
        ++h->steps;
        CK(h, launch_obs_accumulate(h->A, h->C, observable, h->obs_acc, s));
    }
    TRY(adj_save(h, nseg, true));  // final state, restored at the end
    double acc = 0.0;
    CK(h, cudaMemcpyAsync(&acc, h->obs_acc, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    TRY(read_flags(h));
    const double O = acc / n_steps;

    // Reverse pass, segment by segment.
    AdjArgs &D = h->D;
    D.L = h->L;
    D.na = na;
    D.obs_w = (float)(1.0 / n_steps);
    D.observable = observable;
    const size_t N = h->L.N, na3 = 3 * (size_t)na;
    CK(h, cudaMemsetAsync(h->hat[0], 0, N * Q * sizeof(float), s));
    CK(h, cudaMemsetAsync(D.Ghat, 0, N * sizeof(float4), s));
    CK(h, cudaMemsetAsync(D.Uhat, 0, N * sizeof(float4), s));
    CK(h, cudaMemsetAsync(D.xhat, 0, na3 * sizeof(float), s));
    CK(h, cudaMemsetAsync(D.vhat, 0, na3 * sizeof(float), s));
    CK(h, cudaMemsetAsync(D.gam_acc, 0, na * sizeof(double), s));
    CK(h, cudaMemsetAsync(D.par_acc, 0, 2 * sizeof(double), s));
    CK(h, cudaMemsetAsync(D.partials, 0, 2 * (size_t)h->adj_blocks * sizeof(double), s));
    int cur = 0;
    AtomArgs Aadj = h->A;
    Aadj.count[0] = h->adj_count;
    Aadj.slot[0] = h->adj_slot;
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int s0 = seg * K, s1 = std::min(s0 + K, n_steps);
        TRY(adj_restore(h, seg, true));
        for (int n = s0; n < s1; ++n) {
            TRY(adj_save(h, n - s0, false));
            CK(h, cudaGraphLaunch(h->exec, s));
            ++h->steps;
        }
        for (int n = s1 - 1; n >= s0; --n) {
            TRY(adj_restore(h, n - s0, false));
            TRY(enqueue_record_step(h));  // step n again, keeping what the reverse needs
            if (observable == LBMD_OBS_RG2) CK(h, launch_rg2_grad(h->A, h->obs_acc + 1, D.obs_w, D.xhat, s));
            D.hat_in = h->hat[cur];
            D.hat_out = h->hat[cur ^ 1];
            AtomArgs Arec = h->A;
            Arec.recP = h->recP;
            Arec.recL = h->recL;
            Arec.recV = h->recV;
            Arec.recF = h->recF;
            Aadj.recP = h->recP;
            Aadj.recL = h->recL;
            Aadj.recV = h->recV;
            Aadj.recF = h->recF;
            CK(h, launch_adjoint_step(h->p.store, D, Arec, Aadj, h->C, h->pop[0], s));
            CK(h, cudaMemsetAsync(&h->ds->n_touched, 0, sizeof(int), s));
            cur ^= 1;
        }
    }
    // Adjoint of the initial state. The ABI's populations are the pull of the
    // stored ones (f_i(x) = h_i(x - c_i)), so their adjoint is the pull of the
    // storage adjoint; positions and velocities are the atoms' adjoints.
    if (grad_f || grad_x || grad_v) {
        const size_t nf = N * Q;
        float *gf = grad_f, *gx = grad_x, *gv = grad_v;
        void *p = nullptr;
        if (!on_device) {
            CK(h, stage(h, (nf + 2 * na3) * sizeof(float), &p));
            gf = grad_f ? (float *)p : nullptr;
            gx = grad_x ? (float *)p + nf : nullptr;
            gv = grad_v ? (float *)p + nf + na3 : nullptr;
        }
        if (gf) CK(h, launch_pull_f32(h->L, h->hat[cur], gf, s));
        if (gx) CK(h, cudaMemcpyAsync(gx, D.xhat, na3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
        if (gv) CK(h, cudaMemcpyAsync(gv, D.vhat, na3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
        if (!on_device) {
            if (grad_f) CK(h, cudaMemcpyAsync(grad_f, gf, nf * sizeof(float), cudaMemcpyDeviceToHost, s));
            if (grad_x) CK(h, cudaMemcpyAsync(grad_x, gx, na3 * sizeof(float), cudaMemcpyDeviceToHost, s));
            if (grad_v) CK(h, cudaMemcpyAsync(grad_v, gv, na3 * sizeof(float), cudaMemcpyDeviceToHost, s));
            CK(h, cudaStreamSynchronize(s));
        }
    }
    // Parameter gradients: d/d gamma from the atoms, d/d omega and d/d A from
    // the lattice (block partials plus touched-node corrections).
    CK(h, launch_sum_double(D.gam_acc, na, h->obs_acc + 1, s));
    CK(h, launch_sum_double(D.partials, h->adj_blocks, h->obs_acc + 2, s));
    CK(h, launch_sum_double(D.partials + h->adj_blocks, h->adj_blocks, h->obs_acc + 3, s));
    double res[3], corr[2];
    CK(h, cudaMemcpyAsync(res, h->obs_acc + 1, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(h, cudaMemcpyAsync(corr, D.par_acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    TRY(adj_restore(h, nseg, true));  // leave the state advanced by n_steps
    CK(h, cudaStreamSynchronize(s));
    TRY(read_flags(h));
    const double om = 1.0 / h->p.tau;
    const double omh = res[1] + corr[0];
    if (obs) *obs = O;
    if (d_gamma) *d_gamma = res[0];
    if (d_tau) *d_tau = -omh * om * om;
    if (d_force_amp) *d_force_amp = res[2] + corr[1];
    return LBMD_OK;
}

}  // namespace

extern "C" {

lbmd_status lbmd_backward(lbmd_t h, int n_steps, int ckpt_every, int observable, double *d_gamma, double *d_tau,
                          double *d_force_amp, double *obs) {
    return backward_impl(h, n_steps, ckpt_every, observable, d_gamma, d_tau, d_force_amp, obs, nullptr, nullptr,
                         nullptr, 0);
}

lbmd_status lbmd_backward_state(lbmd_t h, int n_steps, int ckpt_every, int observable, double *obs, float *grad_f,
                                float *grad_x, float *grad_v, int on_device) {
    return backward_impl(h, n_steps, ckpt_every, observable, nullptr, nullptr, nullptr, obs, grad_f, grad_x, grad_v,
                         on_device);
}

lbmd_status lbmd_analysis_begin(lbmd_t h, int n_sel, const int32_t *sel, const double *x_ref, int max_frames) {
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (!h->state_set) return fail(h, LBMD_ERR_STATE, "lbmd_set_state has not been called");
    if (h->na == 0) return fail(h, LBMD_ERR_ARG, "the observables need atoms (n_atoms > 0)");
    if (max_frames < 1) return fail(h, LBMD_ERR_ARG, "max_frames must be >= 1");
    const int n = sel ? n_sel : h->na;
    if (n < 1 || n > h->na) return fail(h, LBMD_ERR_ARG, "n_sel must be in 1..n_atoms");
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) {
        idx[i] = sel ? sel[i] : i;
        if (idx[i] < 0 || idx[i] >= h->na) return fail(h, LBMD_ERR_ARG, "selection index out of range");
    }
    // Reference: the caller's, or the selected atoms' current positions.
    std::vector<double> y(3 * (size_t)n);
    if (x_ref) {
        for (size_t k = 0; k < y.size(); ++k) y[k] = x_ref[k];
    } else {
        std::vector<double> X(3 * (size_t)h->na);
        CK(h, cudaMemcpyAsync(X.data(), h->A.X, X.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        for (int d = 0; d < 3; ++d)
            for (int i = 0; i < n; ++i) y[(size_t)d * n + i] = X[(size_t)d * h->na + idx[i]];
    }
    for (double v : y)
        if (!std::isfinite(v)) return fail(h, LBMD_ERR_ARG, "x_ref holds a non-finite value");
    const size_t M = 3 * (size_t)n;
    if ((double)max_frames * (double)M * 4.0 > 64.0e9)
        return fail(h, LBMD_ERR_ARG, "max_frames x 3 n_sel x 4 bytes of frame storage exceeds 64 GB");
    ana_free(h);
    std::vector<double> yc(y);
    double ey = 0.0;
    for (int d = 0; d < 3; ++d) {
        double c = 0.0;
        for (int i = 0; i < n; ++i) c += y[(size_t)d * n + i];
        c /= n;
        h->ana_ybar[d] = c;
        for (int i = 0; i < n; ++i) {
            yc[(size_t)d * n + i] -= c;
            ey += yc[(size_t)d * n + i] * yc[(size_t)d * n + i];
        }
    }
    h->ana_ey = ey;
    AnaArgs &A = h->ana;
    A.na = h->na;
    A.n = n;
    A.X = h->A.X;
    A.mass = h->A.mass;
    void *p;
    TRY(ana_alloc(h, &p, n * sizeof(int))); A.sel = (const int *)p;
    CK(h, cudaMemcpyAsync(p, idx.data(), n * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    TRY(ana_alloc(h, &p, M * sizeof(double))); A.y = (const double *)p;
    CK(h, cudaMemcpyAsync(p, y.data(), M * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    TRY(ana_alloc(h, &p, M * sizeof(double))); A.yc = (const double *)p;
    CK(h, cudaMemcpyAsync(p, yc.data(), M * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    TRY(ana_alloc(h, &p, (size_t)ana_blocks(A) * kAnaSums * sizeof(double))); A.partials = (double *)p;
    TRY(ana_alloc(h, &p, kAnaSums * sizeof(double))); A.sums = (double *)p;
    TRY(ana_alloc(h, &p, (size_t)max_frames * M * sizeof(float))); A.frames = (float *)p;
    TRY(ana_alloc(h, &p, M * sizeof(double))); A.dsum = (double *)p;
    CK(h, cudaMemsetAsync(p, 0, M * sizeof(double), h->stream));
    TRY(ana_alloc(h, &p, M * sizeof(float))); A.meanf = (float *)p;
    CK(h, cudaStreamSynchronize(h->stream));  // the host vectors go out of scope
    h->ana_max = max_frames;
    h->ana_frames = 0;
    return LBMD_OK;
}

lbmd_status lbmd_analysis_frame(lbmd_t h, double *rg2, double *rmsd) {
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (!h->ana.frames) return fail(h, LBMD_ERR_STATE, "lbmd_analysis_begin has not been called");
    if (h->ana_frames >= h->ana_max) return fail(h, LBMD_ERR_ARG, "max_frames frames already taken");
    AnaArgs &A = h->ana;
    A.X = h->A.X;
    CK(h, launch_ana_moments(A, h->stream));
    double m[kAnaSums];
    CK(h, cudaMemcpyAsync(m, A.sums, sizeof(m), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (double v : m)
        if (!std::isfinite(v)) return fail(h, LBMD_ERR_NONFINITE, "non-finite atom position");
    const double n = A.n;
    AnaFit F{};
    double ex = m[8];
    for (int d = 0; d < 3; ++d) {
        F.xbar[d] = m[5 + d] / n;
        F.ybar[d] = h->ana_ybar[d];
        ex -= n * F.xbar[d] * F.xbar[d];
    }
    // sum x_a yc_b = sum (x - xbar)_a yc_b, since yc sums to zero.
    const double lambda = horn_rotation(m + 9, F.R);
    if (rmsd) *rmsd = std::sqrt(std::max(0.0, (ex + h->ana_ey - 2.0 * lambda) / n));
    if (rg2) {
        const double M = m[0];
        const double c[3] = {m[1] / M, m[2] / M, m[3] / M};
        *rg2 = std::max(0.0, m[4] / M - (c[0] * c[0] + c[1] * c[1] + c[2] * c[2]));
    }
    CK(h, launch_ana_store(A, h->ana_frames, F, h->stream));
    ++h->ana_frames;
    return LBMD_OK;
}

lbmd_status lbmd_analysis_result(lbmd_t h, double *mean_disp, double *rmsf, float *cov, int on_device) {
    if (!h) return fail(nullptr, LBMD_ERR_ARG, "handle is NULL");
    if (!h->ana.frames) return fail(h, LBMD_ERR_STATE, "lbmd_analysis_begin has not been called");
    if (h->ana_frames < 1) return fail(h, LBMD_ERR_STATE, "no frame taken (lbmd_analysis_frame)");
    AnaArgs &A = h->ana;
    const size_t n = A.n, M = 3 * n;
    double *dmean = mean_disp, *drmsf = rmsf;
    float *dcov = cov;
    void *p = nullptr;
    if (!on_device) {
        CK(h, stage(h, (M + n) * sizeof(double), &p));
        dmean = mean_disp ? (double *)p : nullptr;
        drmsf = rmsf ? (double *)p + M : nullptr;
        if (cov && !h->ana_cov) {
            void *c;
            TRY(ana_alloc(h, &c, M * M * sizeof(float)));
            h->ana_cov = (float *)c;
        }
        dcov = cov ? h->ana_cov : nullptr;
    }
    CK(h, launch_ana_result(A, h->ana_frames, dmean, drmsf, dcov, h->stream));
    if (!on_device) {
        if (mean_disp) CK(h, cudaMemcpyAsync(mean_disp, dmean, M * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        if (rmsf) CK(h, cudaMemcpyAsync(rmsf, drmsf, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        if (cov) CK(h, cudaMemcpyAsync(cov, dcov, M * M * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return LBMD_OK;
}

}  // extern "C"
