/*
 * lbmd.h -- C ABI of the GB300 (sm_103a) coupled lattice-Boltzmann /
 * molecular-dynamics step.
 *
 * Method: Lauricella et al., "Multiscale Hybrid Modeling of Proteins in
 * Solvent" (arXiv 2305.05025), Sec. 2.2. One coupled step:
 *   1. the fluid velocity u = (sum_i f_i c_i + g/2)/rho (Eq. 2, Guo half-shift
 *      of the body force g) is interpolated trilinearly at every atom from the
 *      eight nearest nodes;
 *   2. the atoms advance by n_md velocity-Verlet substeps of 1/n_md under
 *      shifted-force Lennard-Jones + harmonic bonds and the Stokes friction
 *      gamma (U - v), U held fixed over the step;
 *   3. the opposite of each atom's friction impulse is spread back onto the
 *      same eight nodes with the same weights;
 *   4. every node is collided with the BGK operator -omega (f - f_eq) and the
 *      Guo source of the total force g + G (Eq. 1), omega = 1/tau,
 *      nu = (tau - 1/2)/3, and streamed.
 * Lattice units throughout: Delta x = Delta t = 1, c_s^2 = 1/3.
 *
 * Conventions
 *  - Node (x, y, z), 0 <= x < nx ..., has linear index (z*ny + y)*nx + x.
 *  - D3Q19 speeds in this order: 0 rest; 1..6 = +x -x +y -y +z -z;
 *    7..18 = (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1)
 *    (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1). Speed 2k-1 and 2k are
 *    opposite.
 *  - Populations cross the ABI as structure-of-arrays, population i of node
 *    n at [i*N + n], N = nx*ny*nz, in FP32: the post-streaming distribution
 *    f_i(r, t) of Eq. (1), whatever the internal storage format.
 *  - Atom arrays are SoA: component d of atom a at [d*n_atoms + a].
 *    Positions are FP64 and unwrapped (periodic images are taken by the
 *    library); velocities FP32.
 *  - The caller owns every buffer it passes. The library copies on entry and
 *    exit and never keeps a caller pointer.
 *  - on_device = 1: the pointers are CUDA device pointers; 0: host pointers.
 *  - All device work is enqueued on the stream given to lbmd_create, so calls
 *    are ordered with the caller's other work on that stream. Calls that
 *    return data to the host synchronise that stream.
 *  - Every call returns a status and never aborts; lbmd_last_error gives the
 *    message. No kernel of the library traps or waits on a flag.
 *  - A handle is not thread safe: one thread at a time.
 */
#ifndef LBMD_H
#define LBMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbmd_s *lbmd_t;

typedef enum {
    LBMD_OK = 0,
    LBMD_ERR_ARG = 1,       /* invalid argument or parameter combination */
    LBMD_ERR_ALLOC = 2,     /* device or host allocation failed */
    LBMD_ERR_CUDA = 3,      /* a CUDA runtime call failed (message has the CUDA error) */
    LBMD_ERR_NONFINITE = 4, /* a NaN or Inf appeared in the lattice or the atoms */
    LBMD_ERR_CELL = 5,      /* a pair-search cell held more atoms than its capacity:
                               that step's forces miss pairs */
    LBMD_ERR_STATE = 6      /* call out of order (no state set), or an atom's
                               interpolation stencil crossed a z wall */
} lbmd_status;

/* Storage format of the populations. All arithmetic is FP32; the shifted
 * formats store delta f_i = f_i - w_i rho0 (halving the bytes per node). */
enum { LBMD_F32 = 0, LBMD_F16_SHIFTED = 1, LBMD_BF16_SHIFTED = 2 };

/* Body force g(x) (not in the paper; the workloads' driving). */
enum {
    LBMD_FORCE_NONE = 0,
    LBMD_FORCE_UNIFORM = 1,    /* g = A e_dir */
    LBMD_FORCE_KOLMOGOROV = 2, /* g = A sin(2 pi x_axis / n_axis) e_dir */
    LBMD_FORCE_POISEUILLE = 3  /* g = A e_dir, meant with walls_z = 1 */
};

/* Observables of lbmd_backward. */
enum {
    LBMD_OBS_DRAG_X = 0, /* (1/T) sum_steps sum_atoms J_x: mean friction force the
                            fluid exerts on the solute along x */
    LBMD_OBS_RG2 = 1     /* (1/T) sum_steps R_g^2 after each step (mass weighted) */
};

typedef struct {
    int nx, ny, nz;           /* lattice nodes per axis (>= 1; >= 2 along z with walls) */
    double tau;               /* BGK relaxation time, > 1/2 (omega = 1/tau) */
    double rho0;              /* reference density (shift of the stored populations) */
    double gamma;             /* Stokes friction coefficient, force = gamma (U - v) */
    double dt;                /* coupled time step in lattice units: must be 1 */
    int n_md;                 /* velocity-Verlet substeps per coupled step, >= 1 */
    double lj_eps, lj_sigma;  /* Lennard-Jones well depth and diameter */
    double lj_rcut_over_sigma;/* cutoff radius in units of sigma */
    double skin;              /* extra cell side beyond the cutoff (>= 0) */
    int forcing;              /* LBMD_FORCE_* */
    double force_amp;         /* A */
    int force_dir;            /* component of g (0, 1, 2) */
    int force_wave_axis;      /* axis of the Kolmogorov wave (0, 1, 2) */
    int walls_z;              /* 1: half-way bounce-back walls at z = -1/2, nz - 1/2 */
    int store;                /* LBMD_F32, LBMD_F16_SHIFTED, LBMD_BF16_SHIFTED */
    int deterministic;        /* 1: bitwise-reproducible lbmd_step (Verlet lists sorted by
                                 atom index, the spread summed in exact fixed point,
                                 set-up forces in fixed point); 0: the default, faster
                                 order-of-atomics sums. Mode 1 refuses the
                                 re-interpolated coupling and lbmd_backward. */
    int check_every;          /* lbmd_step polls the device error flags every this
                                 many steps (0: only lbmd_check / lbmd_get_stats do) */
} lbmd_params;

/* Creates a handle. Passage: Sec. 2.2 -- the lattice of Eq. (1) (nx, ny, nz
 * nodes, D3Q19), its relaxation omega = 1/tau with nu = (tau - 1/2)/3, the
 * friction coefficient gamma of the atom-fluid coupling, and the solute
 * (masses, bonded topology, the Lennard-Jones short-range force field that
 * stands in for the paper's force field). Validates the parameters
 * (LBMD_ERR_ARG before any device work), allocates the lattice (two population buffers of N*19 elements of
 * the storage format), the atom arrays and the pair-search cells, and uploads
 * the topology. mass: n_atoms masses (> 0). bonds: 2*n_bonds atom indices;
 * bond_k, bond_r0: n_bonds stiffnesses and rest lengths (U = k (r - r0)^2/2).
 * Bonded pairs are excluded from the Lennard-Jones sum. n_atoms may be 0 (a
 * lattice-only run). cuda_stream: a cudaStream_t (NULL: the legacy default
 * stream). Host pointers. On failure *out is NULL. */
lbmd_status lbmd_create(const lbmd_params *params, int n_atoms, const double *mass, int n_bonds,
                        const int32_t *bonds, const double *bond_k, const double *bond_r0,
                        void *cuda_stream, lbmd_t *out);

/* Sets the state (Sec. 2.2: the populations f_i(r, t) of Eq. (1) and the
 * atom positions and velocities). f: FP32 post-streaming populations (19*N SoA); or, when f
 * is NULL, rho (N) and u (3*N SoA) give f = f_eq(rho, u) (the second-order
 * equilibrium of Sec. 2.2). x (FP64) and v (FP32): 3*n_atoms SoA, required
 * when n_atoms > 0. Also computes the conservative forces at x and fills
 * the pair-search cells. Resets the step counter to 0. */
lbmd_status lbmd_set_state(lbmd_t h, const float *f, const float *rho, const float *u,
                           const double *x, const float *v, int on_device);

/* Advances n_steps coupled steps (Sec. 2.2, Eq. 1: one lattice-Boltzmann
 * update per step in lock step with the MD, which takes n_md velocity-Verlet
 * substeps; the friction gamma (u - v) couples them through trilinear
 * interpolation over the eight nearest nodes and the equal and opposite
 * source term). Asynchronous; each step is one CUDA graph launch. Returns LBMD_ERR_STATE if no state was set. Polls the device flags
 * only when check_every > 0 and a multiple of it is crossed. */
lbmd_status lbmd_step(lbmd_t h, int n_steps);

/* Snapshot of the state in the storage format (no counterpart in the paper:
 * checkpoint and restore, and the cheapest exchange with the host). pop
 * receives the lattice buffer the next step reads: 19*N elements of the
 * storage format (4 bytes for LBMD_F32, 2 for the 16-bit formats, which hold
 * delta f = f - w_i rho0, FP16 scaled by 2^10) in the library's
 * post-collision layout; treat it as opaque and give it back to
 * lbmd_load_state on a handle created with the same lattice size and
 * storage format. x (3*n_atoms FP64) and v (3*n_atoms FP32) as
 * lbmd_get_fields. Any pointer may be NULL; on_device: 1 if they are device
 * memory. Synchronises the stream when on_device = 0. */
lbmd_status lbmd_save_state(lbmd_t h, void *pop, double *x, float *v, int on_device);

/* Restores a snapshot of lbmd_save_state: the lattice bit for bit; the atoms
 * as lbmd_set_state sets them (forces and pair-search cells recomputed). The
 * step counter restarts at 0 (the thermal noise draws restart with it). pop
 * is required, x and v when n_atoms > 0 (LBMD_ERR_ARG otherwise). */
lbmd_status lbmd_load_state(lbmd_t h, const void *pop, const double *x, const float *v, int on_device);

/* Copies out the current state (Sec. 2.2; rho and u are the moments of
 * Eq. 2); any pointer may be NULL. f: FP32 post-streaming populations (19*N); rho (N); u (3*N), the velocity
 * (sum f c + g/2)/rho; x (3*n_atoms FP64); v (3*n_atoms FP32). Synchronises
 * the stream when on_device = 0. */
lbmd_status lbmd_get_fields(lbmd_t h, float *f, float *rho, float *u, double *x, float *v,
                            int on_device);

/* Conservation diagnostics (Sec. 2.2: the source term of Eq. (1) keeps mass
 * and momentum, and the fluid receives exactly the impulse the atoms lose, so
 * mass is constant and total momentum grows by sum_x g per step). FP64 global
 * sums: fluid mass sum_x sum_i f_i, fluid momentum
 * sum_x sum_i f_i c_i, solute momentum sum_a m_a v_a (host outputs, any may be
 * NULL). Synchronises; returns LBMD_ERR_NONFINITE if a NaN/Inf was found. */
lbmd_status lbmd_get_stats(lbmd_t h, double *mass, double mom_fluid[3], double mom_atoms[3]);

/* Error poll (no counterpart in the paper: a service of this library).
 * Synchronises and returns the first raised device flag as a status
 * (NONFINITE, CELL, STATE), clearing the flags. */
lbmd_status lbmd_check(lbmd_t h);

/* Pair-search diagnostics (the cell list of the short-range forces; the
 * paper's MD engine keeps one internally, Sec. 2.2, and states no layout):
 * cell_of[a] = linear
 * index (cz*ncy + cy)*ncx + cx of atom a's cell, cx = floor(x*ncx/nx) mod ncx
 * in FP64, ncx = floor(nx/(rcut + skin)); neighbours[a] = number of other
 * atoms with r^2 < rcut^2 (FP64, minimum image). nc (3 ints, host) receives
 * the cell grid. Any output may be NULL. */
lbmd_status lbmd_cell_list(lbmd_t h, int32_t *cell_of, int32_t *neighbours, int32_t *nc,
                           int on_device);

/* Changes gamma, tau and the body-force amplitude of an existing handle
 * (Sec. 2.2: the coupling and relaxation parameters the adjoint
 * differentiates); the step graph is rebuilt on the next lbmd_step. */
lbmd_status lbmd_set_physics(lbmd_t h, double gamma, double tau, double force_amp);

/* Screened electrostatics of the solute (Sec. 2.2: the force field's Coulomb
 * interactions with a distance-dependent dielectric and a cutoff). charge:
 * n_atoms host doubles (NULL: no electrostatics, the default). Non-bonded
 * pairs within coul_rc interact with the energy coul_c q_a q_b / r^2
 * (k / (eps_r r) with eps_r r the dielectric: coul_c = k / eps_r), shifted so
 * that force and energy vanish at coul_rc; coul_rc must be > 0 and no larger
 * than the Lennard-Jones cutoff (the same pair lists serve both). Must be
 * called before lbmd_set_state (LBMD_ERR_STATE after it), which computes the
 * first forces with the charges. The adjoint includes the Coulomb pairs. */
lbmd_status lbmd_set_charges(lbmd_t h, const double *charge, double coul_c, double coul_rc);

/* Coupling variant (Sec. 2.2: the friction uses the fluid velocity "at the
 * particle position"). on = 0 (the default): the velocity interpolated at the
 * start of the step is held over its n_md substeps and the total friction
 * impulse is spread with the step-start weights. on = 1: the node velocities
 * stay those of the step's start, but every half-kick interpolates at the
 * atom's position of that moment and each substep's impulse is spread with
 * the weights of that position (the fluid still receives exactly what the
 * atoms lose). The interpolation stores the node velocities of each atom's
 * stencil and one node of margin; a substep that finds its atom beyond them
 * computes the missing ones from the step's populations, so any displacement
 * within a step is handled exactly. Costs one node-velocity array (16 bytes
 * per node) and a touched-node list of min(N, 256 per atom) entries
 * (LBMD_ERR_STATE if the atoms claim more nodes in one step). The step graph
 * is rebuilt on the next lbmd_step; lbmd_backward refuses on = 1. */
lbmd_status lbmd_set_reinterpolation(lbmd_t h, int on);

/* Thermal fluctuations of the fluid (Sec. 2.2: the noise xi_i of the
 * fluctuating lattice Boltzmann source term S_i = p_i + xi_i of Eq. 1, the
 * fluid acting as the heat bath). kT > 0 adds after every collision, at every
 * node, Gaussian noise on the 15 non-conserved modes of the D3Q19 moment
 * basis with variance mu b_k (1 - (1 - omega)^2), mu = rho0 kT / c_s^2, so
 * that at rest each node's density fluctuates with variance rho0 kT / c_s^2
 * and each momentum component with rho0 kT; mass and momentum are exact.
 * kT = 0 (the default) turns it off. The random numbers are Philox4x32-10
 * with counter (node, block, step) and key `seed`: a run is reproducible for
 * a given seed and state, and the step counter restarts at lbmd_set_state.
 * The step graph is rebuilt on the next lbmd_step. lbmd_backward refuses
 * kT > 0 (LBMD_ERR_ARG). */
lbmd_status lbmd_set_thermal(lbmd_t h, double kT, uint64_t seed);

/* Timing hook (no counterpart in the paper). Routes the start/stop of the
 * lattice kernel of the NEXT step launch to two
 * caller events (cudaEvent_t, created with timing enabled), so the caller can
 * time that kernel with cudaEventElapsedTime on the stream it runs on.
 * NULL, NULL restores the library's own events. The events stay referenced
 * by the step graph until the next call replaces them: the caller keeps them
 * alive until then (destroying them first makes the next call fail with
 * LBMD_ERR_CUDA). */
lbmd_status lbmd_set_timing_events(lbmd_t h, void *ev_start, void *ev_stop);

/* Timing hook (no counterpart in the paper). Like lbmd_set_timing_events,
 * for the chain of the n_md + 1 velocity-Verlet
 * substep kernels of each step (on the library's solute stream): ev_start is
 * recorded before the first substep kernel, ev_stop after the last. Returns
 * LBMD_ERR_ARG for a lattice-only handle (n_atoms = 0). */
lbmd_status lbmd_set_md_timing_events(lbmd_t h, void *ev_start, void *ev_stop);

/* Differentiable rollout (not in the paper: the discrete adjoint of the
 * coupled step of Sec. 2.2, Eq. 1, for calibrating its gamma, tau and
 * forcing).
 * Runs n_steps steps from the current state, keeping a checkpoint every
 * ckpt_every steps, evaluates the observable (LBMD_OBS_*) and, by the
 * discrete adjoint (reverse collide-stream, reverse interpolate/spread,
 * reverse velocity Verlet), its derivatives with respect to gamma, tau and
 * force_amp. Outputs are host doubles (any may be NULL). The state ends
 * advanced by n_steps, as after lbmd_step(n_steps). */
lbmd_status lbmd_backward(lbmd_t h, int n_steps, int ckpt_every, int observable, double *d_gamma,
                          double *d_tau, double *d_force_amp, double *obs);

/* Like lbmd_backward, returning instead of the parameter gradients the
 * gradient of the observable with respect to the initial state, in the
 * ABI's terms: grad_f (19*N FP32, the post-streaming populations f_i of
 * lbmd_set_state), grad_x and grad_v (3*n_atoms FP32 SoA, positions and
 * velocities). Any output may be NULL; on_device as elsewhere. The same
 * restrictions and state advance as lbmd_backward. */
lbmd_status lbmd_backward_state(lbmd_t h, int n_steps, int ckpt_every, int observable, double *obs, float *grad_f,
                                float *grad_x, float *grad_v, int on_device);

/* Trajectory analysis of the solute (the analyses of Sec. 3 of the paper:
 * root-mean-square deviation from the starting structure, radius of
 * gyration, per-atom root-mean-square fluctuation and the principal
 * components of the atomic fluctuations), computed on the device.
 *
 * lbmd_analysis_begin selects n_sel atoms (sel: host array of atom indices;
 * NULL: all atoms, n_sel ignored) and a reference structure x_ref (host,
 * 3*n_sel FP64 SoA; NULL: the selected atoms' current positions), and
 * reserves device storage for max_frames frames (3*n_sel FP32 each); it
 * replaces any earlier analysis of the handle. LBMD_ERR_ARG for an empty or
 * out-of-range selection, a non-finite reference or more than 64 GB of
 * frames. Synchronises the stream. */
lbmd_status lbmd_analysis_begin(lbmd_t h, int n_sel, const int32_t *sel, const double *x_ref, int max_frames);

/* Takes one frame at the current positions. rg2 (host, may be NULL): the
 * mass-weighted squared radius of gyration of all atoms. rmsd (host, may be
 * NULL): the root-mean-square deviation of the selection from the reference
 * after the optimal rigid superposition (unweighted least squares, proper
 * rotation plus translation). The superposed displacements from the reference
 * are stored as frame number k (k = frames taken so far). FP64 sums on the
 * device, the 4x4 eigenproblem of the optimal rotation on the host.
 * Synchronises the stream. LBMD_ERR_ARG once max_frames frames are taken,
 * LBMD_ERR_STATE before lbmd_analysis_begin. */
lbmd_status lbmd_analysis_frame(lbmd_t h, double *rg2, double *rmsd);

/* Over the T frames taken: mean_disp (3*n_sel FP64 SoA), the mean superposed
 * displacement from the reference; rmsf (n_sel FP64), sqrt of the mean over
 * frames of |d_t - mean|^2 per atom; cov ((3 n_sel)^2 FP32, row-major,
 * coordinate index d*n_sel + i), the covariance (1/T) sum_t (d_t - mean)
 * (d_t - mean)^T whose eigenvectors are the principal components. Any output
 * may be NULL; on_device as elsewhere. The frames stay: more may be taken and
 * the result asked again. LBMD_ERR_STATE before the first frame. */
lbmd_status lbmd_analysis_result(lbmd_t h, double *mean_disp, double *rmsf, float *cov, int on_device);

/* (No counterpart in the paper.) Message of the last failed call on this handle (or of the last failed
 * lbmd_create on this thread when h is NULL). Never NULL. */
const char *lbmd_last_error(lbmd_t h);

/* (No counterpart in the paper.) Frees every resource of the handle
 * (synchronises its stream). NULL is a no-op. */
void lbmd_destroy(lbmd_t h);

/* (No counterpart in the paper.) ABI version, currently 1. */
int lbmd_version(void);

/* Largest lattice lbmd_fluid_sums_noalloc accepts: 65536 blocks of 256 nodes
 * (256^3 nodes), the capacity of its fixed 2 MiB device scratch. */
#define LBMD_NOALLOC_MAX_NODES 16777216

/* Allocation-free FP64 fluid sums (the paper has no counterpart: a service of
 * this library). For callers that cannot call cudaMalloc -- an engine or
 * plugin host that reserves the device memory up front in its own pool and
 * forbids allocations from outside it, or a time-critical loop that cannot
 * afford the device synchronisation an allocation implies. No handle is
 * needed and nothing is allocated: the per-block partial sums go to a
 * file-scope device array of LBMD_NOALLOC_MAX_NODES/256 * 4 doubles that every
 * GPU which loads the library keeps until the process exits.
 *
 * f: device pointer to FP32 populations in the ABI layout (19 * N SoA,
 * N = nx*ny*nz <= LBMD_NOALLOC_MAX_NODES, larger sizes return LBMD_ERR_ARG).
 * out: device pointer to 4 doubles, receives sum_n sum_i f_i and
 * sum_n sum_i f_i c_i (x, y, z). Both stay owned by the caller. Enqueued on
 * cuda_stream (NULL: the legacy default stream); asynchronous.
 *
 * The first call on a device (with that device current) looks up the
 * device address of the scratch array; make that first call before any
 * stream capture. All calls share the array and it keeps the last call's
 * partials: calls that may overlap on the GPU (unordered streams) race and
 * must be serialised by the caller. Errors: LBMD_ERR_ARG, LBMD_ERR_CUDA, with
 * the message from lbmd_last_error(NULL). */
lbmd_status lbmd_fluid_sums_noalloc(const float *f, int nx, int ny, int nz, double *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LBMD_H */
