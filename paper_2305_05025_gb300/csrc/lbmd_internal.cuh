// Internal declarations of the sm_103a coupled LB-MD step: device state,
// kernel argument blocks of the atoms, the coupling, the adjoint and the
// analyses, and the launcher prototypes. Shared by the library's own
// translation units only.
#pragma once

#include <string>

#include "lattice.cuh"

namespace lbmd {

// ---------------------------------------------------------------------------
// Atoms.
//
// Positions: X (FP64, unwrapped) is the accumulator, advanced once per coupled
// step. Inside a step each atom carries its periodic image in the step frame,
// origin + (x mod L) with origin = B + (B - L)/2 and B the smallest power of
// two >= 2L, as an unevaluated FP32 pair hi + lo advanced with error-free
// (two-sum) updates. Every hi lies in the binade [B, 2B) (margins of at least
// L/2 absorb the drift within a step), where differences of hi values and
// folds by whole box lengths are exact: a pair displacement
// (hi_a - hi_b) - k L + (lo_a - lo_b) carries one final FP32 rounding.

constexpr int kMortonBits = 7;                              // bucket coordinates < 128
constexpr int kMortonCodes = 1 << (3 * kMortonBits);       // 2^21 Morton codes
constexpr int kMaxWindow = 7;  // consecutive bucket cells along an axis that never meet a folded bucket twice (searches take 3 or 5)
constexpr int NL_MAX = 256;    // neighbour-list capacity per atom (close packing of sigma = 0.4 beads within 1.3: ~200)

struct AtomArgs {
    int na;
    int n_md;
    float dt, hdt;        // 1/n_md and half of it
    float gamma;
    float lj_sig2, lj_24eps, lj_fc, rc2f;  // LJ constants; lj_fc = F_LJ(rc)
    double rc2d;          // rc^2 in FP64 (neighbour counts)
    int nc[3];            // cell grid (side h = L/nc >= rc + skin): the reported cell
                          // list and the adjoint's buckets
    int fold[3];          // bucket grid: cell c -> bucket c mod fold
    int cap;              // slots per bucket
    float h[3], inv_h[3];
    // Grid of the MD buckets (substeps, list builds, sort). While each axis
    // folds at most twice at half the coarse side, cells of side
    // bh = L/bnc >= (rc + skin)/2 searched as a 5x5x5 block (bwin = 5:
    // about half the candidates of 27 coarse cells); on larger boxes the
    // coarse cells searched as 3x3x3 (bwin = 3), since finer buckets folded
    // many times over would stack far-apart atoms.
    int bnc[3], bfold[3], bfmask[3], bcap, bwin;
    float bh[3], binv_h[3];
    double hd[3], Ld[3];
    float Lf[3], inv_Lf[3];  // box lengths and their inverses
    float off[3];         // step-frame origin per axis (exact in FP32)
    double offd[3];
    double *X;            // 3*na FP64 accumulator
    float4 *P[2];         // (hi x, hi y, hi z, charge) by substep parity
    float4 *L[2];         // (lo x, lo y, lo z, 0) by substep parity
    float *P0, *R0;       // 3*na step-start hi and lo parts
    float *V, *F, *U, *J; // 3*na SoA each
    float *mass, *inv_m;
    const int *bstart, *bpart;  // bond CSR
    const float *bk, *br0;
    int *count[3], *slot[3], *bucket[3], *sidx[3];  // pair-search buckets by generation mod 3
    int fmask[3];         // bucket coordinate = cell & fmask (fold = nc, or 128 with mask 127)
    int *order;           // atoms in warp-sorted (Morton bucket) order
    int *scode;           // per atom: Morton code of its 4x4x4 sub-cell within its bucket cell (sort key within a bucket)
    float4 *recP, *recL;  // adjoint recording ((n_md+1)*na): positions at x_k, or NULL
    float *recV, *recF;   // adjoint recording ((n_md+1)*3na): input velocity and force of kernel k
    int *nbr;             // na * NL_MAX neighbour lists (atom-major)
    int *nnb;             // list lengths
    float *D;             // 3*na drift since the last list build
    float rl2;            // (rc + skin)^2, list radius squared
    // Screened Coulomb pairs (charge in the w component of P): pair force
    // 2 C q_a q_b (r^-4 - rcc^-3 r^-1) d within rcc <= rc; coul = 0: off.
    int coul;
    float coul_2c, coul_rc2, coul_irc3;
    const float *q;       // na charges (by atom), or NULL
    // Re-interpolated coupling: every substep kernel interpolates U at x_k
    // from the step's node velocities and spreads its own friction impulse.
    int reinterp;
    const float4 *unode;  // node velocities of the step (w: the step's stamp), from the interpolation
    float4 *G;            // per node coupling force (the spread's target)
    int nl[3];            // lattice nodes per axis
    int walls;
    // Nodes outside the region the interpolation froze (an atom that moved
    // more than one node within the step): their velocities come from the
    // step's populations, and they join the touched-node list.
    const Lat *lat;          // device copy of the lattice description
    int store;               // LBMD_F32 / LBMD_F16_SHIFTED / LBMD_BF16_SHIFTED
    const void *pop[2];      // population buffers; the step reads pop[step & 1]
    int *tag, *touched;      // touched-node stamps and list (as the interpolation's)
    int touched_cap;
    float half_skin2;     // (skin/2)^2, drift that triggers a rebuild
    int det;              // deterministic mode: lists sorted by atom index, set-up forces in fixed point
    int *scan_local;      // Morton-code exclusive scan within blocks of 1024
    int *scan_block;      // kMortonCodes / 1024 block offsets
    DevState *ds;
};

// Step frame of an atom from its FP64 position: the periodic image in
// [0, L) shifted by the frame origin into the binade [B, 2B), split into
// hi + lo. Also the step-start copies used to advance X at the step's end.
__device__ __forceinline__ bool set_frame(const AtomArgs &A, int a, float4 &p, float4 &l) {
    bool finite = true;
    float hi[3], lo[3];
    for (int d = 0; d < 3; ++d) {
        const double x = A.X[d * A.na + a];
        finite = finite && isfinite(x);
        double w = x - floor(x / A.Ld[d]) * A.Ld[d];
        if (!(w >= 0.0 && w < A.Ld[d])) w = 0.0;  // non-finite or rounding at the top edge
        const double y = A.offd[d] + w;
        hi[d] = (float)y;
        lo[d] = (float)(y - (double)hi[d]);
        A.P0[d * A.na + a] = hi[d];
        A.R0[d * A.na + a] = lo[d];
    }
    p = make_float4(hi[0], hi[1], hi[2], A.q ? A.q[a] : 0.f);  // w: the atom's charge
    l = make_float4(lo[0], lo[1], lo[2], 0.f);
    return finite;
}

struct CouplingArgs {
    Lat L;
    int na;
    const double *X;
    float *U, *J;
    int *base;      // 3*na wrapped base node per atom (step start)
    float *frac;    // 3*na fractional offsets (step start)
    int *tag;       // per node: step stamp of the last claim
    int *touched;   // unique touched nodes of this step
    int touched_cap;
    float4 *G;      // per node coupling force (x, y, z, unused)
    const int *order;  // atoms in warp-sorted (Morton bucket) order, as AtomArgs::order
    int reinterp;      // 1: the substeps interpolate and spread (see AtomArgs)
    float4 *unode;     // node velocities of the step's region (re-interpolation only)
    DevState *ds;
    int keep;       // 1: the fix-up leaves G and the touched list for the adjoint
    // Deterministic mode: the spread adds fixed-point integers (exact, so
    // independent of the order of the atomics) per touched slot instead of
    // float4 atomics per node; tslot maps a node to its touched slot.
    int *tslot;
    long long *gfix;  // 3 per touched slot, in units of 1/kFixScale
};
constexpr double kFixScale = 1099511627776.0;  // 2^40: fixed-point unit of the deterministic spread

// Adjoint state and accumulators of lbmd_backward.
struct AdjArgs {
    Lat L;
    int na;
    float *hat_in, *hat_out;  // adjoint of the post-collision storage (19*N FP32): step n+1 in, n out
    float4 *Ghat, *Uhat;      // per node hat F and hat u_b (touched nodes only, zero elsewhere)
    float *xhat, *vhat;       // 3*na adjoint of positions and velocities
    float *p, *Jhat, *Uat_hat, *xw;  // 3*na work arrays
    double *gam_acc;          // na: d/d gamma contributions
    double *par_acc;          // 2: touched-node corrections of d/d omega and d/d A
    double *partials;         // 2*nblocks: block sums of d/d omega and d/d A
    float obs_w;              // 1/T
    int observable;
};

// Trajectory analysis (observables of the solute). Frame moments, FP64:
// [0] sum m, [1..3] sum m x, [4] sum m |x|^2 over all atoms; over the
// selection [5..7] sum x, [8] sum |x|^2, [9 + 3a + b] sum x_a yc_b (yc: the
// reference minus its centroid).
constexpr int kAnaSums = 18;
struct AnaArgs {
    int na, n;            // atoms, selected atoms
    const double *X;      // 3*na FP64 positions
    const float *mass;    // na
    const int *sel;       // n atom indices
    const double *y;      // 3n reference positions (SoA)
    const double *yc;     // 3n reference minus its centroid
    double *partials;     // ana_blocks * kAnaSums
    double *sums;         // kAnaSums
    float *frames;        // max_frames rows of 3n superposed displacements (component-major)
    double *dsum;         // 3n running sum of the displacements
    float *meanf;         // 3n mean displacement (FP32, set at the result)
};
struct AnaFit {
    double R[9];          // rotation, row-major
    double xbar[3], ybar[3];
};

// Message returned by lbmd_last_error(NULL) on the calling thread.
void set_thread_error(const std::string &msg);

// Launchers (stream-ordered, no synchronisation).
cudaError_t launch_lb_step(int store, const Lat &L, void *const buf[2], DevState *ds, cudaStream_t s);
cudaError_t launch_lb_fix(int store, const Lat &L, void *const buf[2], const CouplingArgs &c, int grid,
                          cudaStream_t s);
cudaError_t launch_lb_fields(int store, const Lat &L, const void *cur, float *f, float *rho, float *u,
                             DevState *ds, cudaStream_t s);
cudaError_t launch_lb_init(int store, const Lat &L, void *dst, const float *f, const float *rho, const float *u,
                           cudaStream_t s);
cudaError_t launch_pull_f32(const Lat &L, const float *src, float *dst, cudaStream_t s);
cudaError_t launch_lb_reduce(int store, const Lat &L, const void *cur, double *partials, int nblocks, DevState *ds,
                             cudaStream_t s);
cudaError_t launch_reduce_finish(const double *partials, int nblocks, int width, double *out, cudaStream_t s);
cudaError_t launch_atom_momentum(const float *V, const float *mass, int na, double *partials, int nblocks,
                                 DevState *ds, cudaStream_t s);

cudaError_t launch_md_prime(const AtomArgs &a, cudaStream_t s);
cudaError_t launch_md_substep(const AtomArgs &a, int k, cudaStream_t s);
cudaError_t launch_md_diag(const AtomArgs &a, int *cell_of, int *neigh, cudaStream_t s);
cudaError_t launch_md_sort(const AtomArgs &a, cudaStream_t s);

int adj_lb_blocks(const Lat &L);
cudaError_t launch_adjoint_step(int store, const AdjArgs &D, const AtomArgs &A, AtomArgs &Aadj, const CouplingArgs &C,
                                const void *h, cudaStream_t s);
cudaError_t launch_obs_accumulate(const AtomArgs &A, const CouplingArgs &C, int observable, double *out,
                                  cudaStream_t s);
cudaError_t launch_rg2_grad(const AtomArgs &A, double *scratch, float w, float *xhat, cudaStream_t s);
cudaError_t launch_sum_double(const double *v, int n, double *out, cudaStream_t s);

cudaError_t launch_interp(int store, const CouplingArgs &c, const AtomArgs &a, void *const buf[2], cudaStream_t s);

int ana_blocks(const AnaArgs &A);
cudaError_t launch_ana_moments(const AnaArgs &A, cudaStream_t s);
cudaError_t launch_ana_store(const AnaArgs &A, int frame, const AnaFit &F, cudaStream_t s);
cudaError_t launch_ana_result(const AnaArgs &A, int T, double *mean, double *rmsf, float *cov, cudaStream_t s);
cudaError_t launch_spread(const CouplingArgs &c, cudaStream_t s);

}  // namespace lbmd
