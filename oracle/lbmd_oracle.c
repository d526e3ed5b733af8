/*
 * lbmd_oracle.c -- plain FP64 CPU oracle of one coupled lattice-Boltzmann /
 * molecular-dynamics time step, after Lauricella et al., "Multiscale Hybrid
 * Modeling of Proteins in Solvent: SARS-CoV2 Spike Protein as test case for
 * Lattice Boltzmann - All Atom Molecular Dynamics Coupling" (arXiv 2305.05025),
 * Sec. 2.2 ("Coupled Lattice-Boltzmann and Molecular Dynamics").
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. It shares no code, header, table or
 * helper with the CUDA path; the two meet only on the same seeded inputs.
 *
 * Everything is double precision and single threaded. Each function is one
 * whole pass over the lattice or the atoms, in the order the paper states the
 * method; nothing is fused, blocked or reordered.
 *
 * Readings taken where the paper is silent, ambiguous or garbled:
 *  R1  Eq. (1) prints "+omega[f - f_eq]"; with that sign the scheme amplifies
 *      deviations from equilibrium, so the collision is the standard BGK
 *      relaxation  -omega (f - f_eq).
 *  R2  omega = 2/(6 nu + 1) (Sec. 2.2) is tau = 1/omega, nu = (tau - 1/2)/3.
 *  R3  "i = 0, b" runs over the 19 D3Q19 speeds; their order is fixed below.
 *  R4  The source p_i of the external and coupling forces (Sec. 2.2) is the
 *      Guo forcing term; the velocity in f_eq is shifted by F/(2 rho).
 *  R5  Friction: the fluid receives gamma (v - u) (Sec. 2.2), the atom the
 *      equal and opposite gamma (u - v). The fluid's share is spread over the
 *      same eight nodes with the same trilinear weights used to interpolate u.
 *  R6  The fluid velocity interpolated at an atom includes the half-shift of
 *      the body force g only: u = (sum_i f_i c_i + g/2) / rho.
 *  R7  LB and MD advance in lock step with one LB time unit per coupled step;
 *      the MD part is n_md velocity-Verlet substeps of 1/n_md each, with the
 *      interpolated fluid velocity held fixed over the coupled step.
 *  R8  Synthetic solute: harmonic bonds U = k (r - r0)^2 / 2 and shifted-force
 *      12-6 Lennard-Jones (force zero at the cutoff), 1-2 bonded pairs excluded.
 *  R9  Nodes sit at integer coordinates 0..n-1; atoms use the same length unit
 *      and are stored unwrapped; lattice indices wrap periodically and pair
 *      distances use the minimum image.
 *  R10 Optional z walls: half-way bounce-back at z = -1/2 and z = nz - 1/2.
 *      Atoms must keep their interpolation stencil inside 0..nz-1.
 *  R11 The thermal noise xi_i of the fluctuating LB (Sec. 2.2, the source term
 *      S_i = p_i + xi_i of Eq. 1) is added after the collision when kT > 0:
 *      Gaussian noise on the 15 non-conserved modes of the weighted-orthogonal
 *      D3Q19 moment basis below, each with variance mu b_k (1 - (1 - omega)^2),
 *      mu = rho0 kT / c_s^2 (the fluctuation-dissipation amplitude of a BGK
 *      relaxation 1 - omega; rho0 rather than the local density), so that at
 *      rest every mode holds mu b_k and the fluid velocity kT/rho0 per
 *      component. Mass and momentum get no noise. Random numbers: Philox4x32-10
 *      (Salmon et al., SC'11) with counter (node, call, step low, step high)
 *      and key (seed low, seed high); uniforms ((w >> 9) + 1/2) 2^-23 (exact
 *      in FP32 as in FP64, so a single-precision implementation draws the
 *      same uniforms); normals by the Box-Muller transform.
 *  R16 Electrostatics (Sec. 2.2: Coulomb interactions with a distance-dependent
 *      dielectric and a cutoff, in the paper's implicit-solvent force field):
 *      with charges q, the pair energy k q_a q_b / (eps(r) r) with
 *      eps(r) = eps_r r is C q_a q_b / r^2, C = k / eps_r, shifted-force at
 *      the cutoff r_cc (force and energy vanish there), for non-bonded pairs
 *      within r_cc <= the Lennard-Jones cutoff; off when no charges are given.
 *  R17 Re-interpolation (an option, reinterp = 1; R7 stays the default): the
 *      node velocities u_j stay those at the start of the step, but every
 *      half-kick takes the fluid velocity interpolated at the atom's position
 *      of that moment (x^s for the first half-kick of substep s, x^(s+1) for
 *      the second), and its friction impulse is spread with the weights of
 *      that same position, so the fluid still receives exactly the impulse
 *      the atoms lose.
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

/* D3Q19 speeds (R3): rest, the six faces, the twelve edges. */
static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

/* D3Q19 weights: 1/3 rest, 1/18 faces, 1/36 edges. */
static double weight(int i) {
    if (i == 0) return 1.0 / 3.0;
    if (i <= 6) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* Index of the speed -c_i, found by search. */
static int opposite(int i) {
    for (int j = 0; j < Q; ++j)
        if (CX[j] == -CX[i] && CY[j] == -CY[i] && CZ[j] == -CZ[i]) return j;
    return -1;
}

typedef struct {
    int nx, ny, nz;
    double tau, rho0, gamma;
    int n_md;
    double lj_eps, lj_sigma, lj_rcut; /* absolute cutoff radius */
    double cell_min;                  /* minimum side of a linked-list cell */
    int forcing;                      /* 0 none, 1 uniform, 2 Kolmogorov, 3 Poiseuille */
    double force_amp;
    int force_dir, force_wave_axis;
    int walls_z;
    int brute_force;                  /* 1: all-pairs search instead of cells */
    double kT;                        /* thermal energy of the fluctuating LB (0: no noise) */
    uint64_t seed;                    /* key of the noise's random numbers */
    int64_t step0;                    /* step index of the first step of a run */
    double coul_c;                    /* C = k / eps_r of the screened Coulomb pairs (R16) */
    double coul_rc;                   /* their cutoff (<= lj_rcut) */
    int reinterp;                     /* 1: fluid velocity re-interpolated at every half-kick (R17) */
} orc_params;

typedef struct {
    int n_atoms;
    const double *mass;
    int n_bonds;
    const int32_t *bonds;  /* 2 * n_bonds atom indices */
    const double *bond_k;
    const double *bond_r0;
    const double *charge;  /* n_atoms charges, or NULL: no electrostatics */
} orc_topology;

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_ALLOC = -2, ORC_ERR_WALL = -3 };

static size_t n_nodes(const orc_params *p) { return (size_t)p->nx * p->ny * p->nz; }

static size_t node_at(const orc_params *p, int x, int y, int z) {
    return ((size_t)z * p->ny + y) * p->nx + x;
}

static int wrap(long a, int n) {
    long r = a % n;
    return (int)(r < 0 ? r + n : r);
}

/* ---------------------------------------------------------------------- */
/* Lattice tables, exported so the tests can check them against the
 * isotropy conditions a D3Q19 set must satisfy. */
void orc_lattice(int32_t *c /* 3*Q, c[3i+d] */, double *w /* Q */, int32_t *opp /* Q */) {
    for (int i = 0; i < Q; ++i) {
        c[3 * i + 0] = CX[i];
        c[3 * i + 1] = CY[i];
        c[3 * i + 2] = CZ[i];
        w[i] = weight(i);
        opp[i] = opposite(i);
    }
}

/* Second-order (Mach) truncated equilibrium, Sec. 2.2:
 * f_eq_i = w_i rho [1 + 3 c_i.u + 9/2 (c_i.u)^2 - 3/2 u.u]  (c_s^2 = 1/3). */
static double equilibrium(int i, double rho, const double u[3]) {
    double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return weight(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

void orc_equilibrium(int64_t n, const double *rho, const double *u /* 3n SoA */,
                     double *feq /* Q n SoA */) {
    for (int64_t k = 0; k < n; ++k) {
        double uk[3] = {u[k], u[n + k], u[2 * n + k]};
        for (int i = 0; i < Q; ++i) feq[(size_t)i * n + k] = equilibrium(i, rho[k], uk);
    }
}

/* Moments, Eq. (2): rho = sum_i f_i, rho u = sum_i f_i c_i. */
void orc_moments(int64_t n, const double *f, double *rho, double *j /* 3n SoA */) {
    for (int64_t k = 0; k < n; ++k) {
        double r = 0, jx = 0, jy = 0, jz = 0;
        for (int i = 0; i < Q; ++i) {
            double fi = f[(size_t)i * n + k];
            r += fi;
            jx += fi * CX[i];
            jy += fi * CY[i];
            jz += fi * CZ[i];
        }
        rho[k] = r;
        j[k] = jx;
        j[n + k] = jy;
        j[2 * n + k] = jz;
    }
}

/* Guo forcing term (R4): S_i = (1 - omega/2) w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F */
static double guo_source(int i, double omega, const double u[3], const double F[3]) {
    double c[3] = {CX[i], CY[i], CZ[i]};
    double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
    double s = 0;
    for (int d = 0; d < 3; ++d) s += (3.0 * (c[d] - u[d]) + 9.0 * cu * c[d]) * F[d];
    return (1.0 - 0.5 * omega) * weight(i) * s;
}

void orc_guo_source(double tau, const double u[3], const double F[3], double *S /* Q */) {
    for (int i = 0; i < Q; ++i) S[i] = guo_source(i, 1.0 / tau, u, F);
}

/* Collision of one node, Eq. (1) right-hand side with R1 and R4:
 * f*_i = f_i - omega (f_i - f_eq_i(rho, u)) + S_i,  u = (sum f c + F/2)/rho. */
void orc_collide_node(double tau, const double *f /* Q */, const double F[3], double *out /* Q */) {
    double omega = 1.0 / tau;
    double rho = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
        j[0] += f[i] * CX[i];
        j[1] += f[i] * CY[i];
        j[2] += f[i] * CZ[i];
    }
    double u[3];
    for (int d = 0; d < 3; ++d) u[d] = (j[d] + 0.5 * F[d]) / rho;
    for (int i = 0; i < Q; ++i)
        out[i] = f[i] - omega * (f[i] - equilibrium(i, rho, u)) + guo_source(i, omega, u, F);
}

/* ---------------------------------------------------------------------- */
/* Thermal noise (R11). Philox4x32-10 as published: ten rounds of
 * (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
 * lo(M0 c0)) with the key advanced by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * c[0], p1 = (uint64_t)M1 * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* Mode k of the D3Q19 moment basis at speed i: polynomials in c, orthogonal
 * under the weights w_i. 0: 1; 1-3: c_x, c_y, c_z; 4: c^2 - 1; 5: 3c_x^2 - c^2;
 * 6: c_y^2 - c_z^2; 7-9: c_x c_y, c_y c_z, c_x c_z; 10-12: (3c^2 - 5) c_x,y,z;
 * 13: (c_y^2 - c_z^2) c_x; 14: (c_z^2 - c_x^2) c_y; 15: (c_x^2 - c_y^2) c_z;
 * 16: 3c^4 - 6c^2 + 1; 17: (2c^2 - 3)(3c_x^2 - c^2); 18: (2c^2 - 3)(c_y^2 - c_z^2). */
static double mode_value(int k, int i) {
    const double x = CX[i], y = CY[i], z = CZ[i];
    const double c2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return c2 - 1.0;
    case 5: return 3.0 * x * x - c2;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return y * z;
    case 9: return x * z;
    case 10: return (3.0 * c2 - 5.0) * x;
    case 11: return (3.0 * c2 - 5.0) * y;
    case 12: return (3.0 * c2 - 5.0) * z;
    case 13: return (y * y - z * z) * x;
    case 14: return (z * z - x * x) * y;
    case 15: return (x * x - y * y) * z;
    case 16: return 3.0 * c2 * c2 - 6.0 * c2 + 1.0;
    case 17: return (2.0 * c2 - 3.0) * (3.0 * x * x - c2);
    default: return (2.0 * c2 - 3.0) * (y * y - z * z);
    }
}

/* E[k*Q + i] = mode k at speed i; b[k] = sum_i w_i E_ki^2. */
void orc_mode_basis(double *E, double *b) {
    for (int k = 0; k < Q; ++k) {
        b[k] = 0.0;
        for (int i = 0; i < Q; ++i) {
            E[k * Q + i] = mode_value(k, i);
            b[k] += weight(i) * E[k * Q + i] * E[k * Q + i];
        }
    }
}

/* The 16 standard normals of a node and step: four Philox blocks, each
 * giving two Box-Muller pairs from its words (w0, w1) and (w2, w3). */
static void node_normals(uint64_t seed, int64_t node, int64_t step, double n[16]) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int call = 0; call < 4; ++call) {
        const uint32_t ctr[4] = {(uint32_t)node, (uint32_t)call, (uint32_t)step, (uint32_t)((uint64_t)step >> 32)};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        for (int p = 0; p < 2; ++p) {
            const double u1 = ((double)(w[2 * p] >> 9) + 0.5) * (1.0 / 8388608.0);
            const double u2 = ((double)(w[2 * p + 1] >> 9) + 0.5) * (1.0 / 8388608.0);
            const double r = sqrt(-2.0 * log(u1));
            n[4 * call + 2 * p] = r * cos(2.0 * 3.14159265358979323846 * u2);
            n[4 * call + 2 * p + 1] = r * sin(2.0 * 3.14159265358979323846 * u2);
        }
    }
}

/* xi_i = w_i sum_{k=4..18} E_ki sqrt(mu (1 - (1 - omega)^2) / b_k) n_{k-4}. */
void orc_node_noise(const orc_params *p, int64_t node, int64_t step, double *xi /* Q */) {
    double E[Q * Q], b[Q], n[16];
    orc_mode_basis(E, b);
    node_normals(p->seed, node, step, n);
    const double omega = 1.0 / p->tau;
    const double mu = 3.0 * p->rho0 * p->kT;
    const double g = 1.0 - omega;
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int k = 4; k < Q; ++k) s += E[k * Q + i] * sqrt(mu * (1.0 - g * g) / b[k]) * n[k - 4];
        xi[i] = weight(i) * s;
    }
}

/* Body force g(x) (not in the paper; the workload's forcing): uniform or
 * Poiseuille g = A e_dir; Kolmogorov g = A sin(2 pi x_axis / n_axis) e_dir. */
static void body_force(const orc_params *p, int x, int y, int z, double g[3]) {
    g[0] = g[1] = g[2] = 0.0;
    if (p->forcing == 0) return;
    double a = p->force_amp;
    if (p->forcing == 2) {
        int coord = p->force_wave_axis == 0 ? x : (p->force_wave_axis == 1 ? y : z);
        int n = p->force_wave_axis == 0 ? p->nx : (p->force_wave_axis == 1 ? p->ny : p->nz);
        a *= sin(2.0 * 3.14159265358979323846 * (double)coord / (double)n);
    }
    g[p->force_dir] = a;
}

void orc_body_force(const orc_params *p, double *g /* 3N SoA */) {
    size_t N = n_nodes(p);
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double gg[3];
                body_force(p, x, y, z, gg);
                size_t k = node_at(p, x, y, z);
                g[k] = gg[0];
                g[N + k] = gg[1];
                g[2 * N + k] = gg[2];
            }
}

/* Trilinear stencil, Sec. 2.2 ("linear interpolation over the nearest eight
 * lattice points"), with R9/R10. Corner k has offsets (k&1, k>>1&1, k>>2&1). */
static int stencil(const orc_params *p, const double xa[3], size_t node[8], double W[8]) {
    double t[3];
    long b[3];
    for (int d = 0; d < 3; ++d) {
        double fl = floor(xa[d]);
        t[d] = xa[d] - fl;
        b[d] = (long)fl;
    }
    if (p->walls_z && (b[2] < 0 || b[2] + 1 > p->nz - 1)) return ORC_ERR_WALL;
    for (int k = 0; k < 8; ++k) {
        int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
        double wk = 1.0;
        for (int d = 0; d < 3; ++d) wk *= o[d] ? t[d] : 1.0 - t[d];
        W[k] = wk;
        node[k] = node_at(p, wrap(b[0] + o[0], p->nx), wrap(b[1] + o[1], p->ny),
                          p->walls_z ? (int)(b[2] + o[2]) : wrap(b[2] + o[2], p->nz));
    }
    return ORC_OK;
}

/* U_a = sum_j W_aj u_j  (u is a 3N SoA node field). */
int orc_interp(const orc_params *p, const double *ufield, int n_atoms, const double *x,
               double *U /* 3 n_atoms SoA */) {
    size_t N = n_nodes(p);
    for (int a = 0; a < n_atoms; ++a) {
        double xa[3] = {x[a], x[n_atoms + a], x[2 * n_atoms + a]};
        size_t node[8];
        double W[8];
        if (stencil(p, xa, node, W)) return ORC_ERR_WALL;
        for (int d = 0; d < 3; ++d) {
            double s = 0;
            for (int k = 0; k < 8; ++k) s += W[k] * ufield[d * N + node[k]];
            U[d * n_atoms + a] = s;
        }
    }
    return ORC_OK;
}

/* G_j += sum_a W_aj J_a  (adds into a 3N SoA node field; the caller supplies
 * the sign). */
int orc_spread(const orc_params *p, int n_atoms, const double *x, const double *J, double *G) {
    size_t N = n_nodes(p);
    for (int a = 0; a < n_atoms; ++a) {
        double xa[3] = {x[a], x[n_atoms + a], x[2 * n_atoms + a]};
        size_t node[8];
        double W[8];
        if (stencil(p, xa, node, W)) return ORC_ERR_WALL;
        for (int k = 0; k < 8; ++k)
            for (int d = 0; d < 3; ++d) G[d * N + node[k]] += W[k] * J[d * n_atoms + a];
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Solute forces (R8, R9). */

static void min_image(const orc_params *p, const double *x, int na, int a, int b, double d[3]) {
    const int L[3] = {p->nx, p->ny, p->nz};
    for (int k = 0; k < 3; ++k) {
        double dd = x[k * na + a] - x[k * na + b];
        dd -= (double)L[k] * nearbyint(dd / (double)L[k]);
        d[k] = dd;
    }
}

static double sq3(const double d[3]) {
    double s = d[0] * d[0];
    s += d[1] * d[1];
    s += d[2] * d[2];
    return s;
}

/* 12-6 Lennard-Jones magnitude -dU/dr and energy at distance r. */
static void lj_plain(const orc_params *p, double r, double *fmag, double *u) {
    double sr6 = pow(p->lj_sigma / r, 6.0);
    double sr12 = sr6 * sr6;
    *u = 4.0 * p->lj_eps * (sr12 - sr6);
    *fmag = 24.0 * p->lj_eps * (2.0 * sr12 - sr6) / r;
}

/* Shifted-force LJ: F(r) = F_LJ(r) - F_LJ(rc), U(r) = U_LJ(r) - U_LJ(rc) + (r - rc) F_LJ(rc). */
static void lj_shifted_force(const orc_params *p, double r, double *fmag, double *u) {
    double fr, ur, fc, uc;
    lj_plain(p, r, &fr, &ur);
    lj_plain(p, p->lj_rcut, &fc, &uc);
    *fmag = fr - fc;
    *u = ur - uc + (r - p->lj_rcut) * fc;
}

/* Screened Coulomb pair (R16): energy C q_a q_b / r^2, radial force
 * 2 C q_a q_b / r^3 (positive = repulsive), shifted so that force and energy
 * vanish at coul_rc. qq = q_a q_b. */
static void coulomb_shifted_force(const orc_params *p, double qq, double r, double *fmag, double *u) {
    const double rc = p->coul_rc, A = p->coul_c * qq;
    const double fr = 2.0 * A / (r * r * r), fc = 2.0 * A / (rc * rc * rc);
    *fmag = fr - fc;
    *u = A / (r * r) - A / (rc * rc) + (r - rc) * fc;
}

typedef struct {
    int n;
    int *start; /* n+1 */
    int *nbr;
    double *k, *r0;
} adjacency;

static int build_adjacency(const orc_topology *t, adjacency *adj) {
    int n = t->n_atoms;
    adj->n = n;
    adj->start = (int *)calloc((size_t)n + 1, sizeof(int));
    adj->nbr = (int *)malloc(sizeof(int) * (size_t)(2 * t->n_bonds + 1));
    adj->k = (double *)malloc(sizeof(double) * (size_t)(2 * t->n_bonds + 1));
    adj->r0 = (double *)malloc(sizeof(double) * (size_t)(2 * t->n_bonds + 1));
    int *fill = (int *)calloc((size_t)n + 1, sizeof(int));
    if (!adj->start || !adj->nbr || !adj->k || !adj->r0 || !fill) {
        free(fill);
        return ORC_ERR_ALLOC;
    }
    for (int b = 0; b < t->n_bonds; ++b) {
        int i = t->bonds[2 * b], j = t->bonds[2 * b + 1];
        if (i < 0 || j < 0 || i >= n || j >= n || i == j) {
            free(fill);
            return ORC_ERR_ARG;
        }
        adj->start[i + 1]++;
        adj->start[j + 1]++;
    }
    for (int a = 0; a < n; ++a) adj->start[a + 1] += adj->start[a];
    for (int b = 0; b < t->n_bonds; ++b) {
        int i = t->bonds[2 * b], j = t->bonds[2 * b + 1];
        int si = adj->start[i] + fill[i]++;
        int sj = adj->start[j] + fill[j]++;
        adj->nbr[si] = j;
        adj->k[si] = t->bond_k[b];
        adj->r0[si] = t->bond_r0[b];
        adj->nbr[sj] = i;
        adj->k[sj] = t->bond_k[b];
        adj->r0[sj] = t->bond_r0[b];
    }
    free(fill);
    return ORC_OK;
}

static void free_adjacency(adjacency *adj) {
    free(adj->start);
    free(adj->nbr);
    free(adj->k);
    free(adj->r0);
}

static int bonded(const adjacency *adj, int a, int b) {
    for (int s = adj->start[a]; s < adj->start[a + 1]; ++s)
        if (adj->nbr[s] == b) return 1;
    return 0;
}

/* Linked-cell list: cells of side >= cell_min, cell index floor(x n_c / L)
 * computed in FP64 as (x * n_c) / L, then wrapped. */
static void cell_grid(const orc_params *p, int nc[3]) {
    const int L[3] = {p->nx, p->ny, p->nz};
    for (int d = 0; d < 3; ++d) nc[d] = (int)floor((double)L[d] / p->cell_min);
}

static int cell_coord(double x, int nc, int L) {
    double s = (x * (double)nc) / (double)L;
    return wrap((long)floor(s), nc);
}

void orc_cells(const orc_params *p, int n_atoms, const double *x, int32_t *cell_of, int32_t *nc_out) {
    int nc[3];
    const int L[3] = {p->nx, p->ny, p->nz};
    cell_grid(p, nc);
    for (int d = 0; d < 3; ++d) nc_out[d] = nc[d];
    for (int a = 0; a < n_atoms; ++a) {
        int c[3];
        for (int d = 0; d < 3; ++d) c[d] = cell_coord(x[d * n_atoms + a], nc[d], L[d]);
        cell_of[a] = (c[2] * nc[1] + c[1]) * nc[0] + c[0];
    }
}

typedef struct {
    int nc[3];
    int ncell;
    int *head, *next;
} cell_list;

static int build_cells(const orc_params *p, int na, const double *x, cell_list *cl) {
    cell_grid(p, cl->nc);
    cl->ncell = cl->nc[0] * cl->nc[1] * cl->nc[2];
    cl->head = (int *)malloc(sizeof(int) * (size_t)cl->ncell);
    cl->next = (int *)malloc(sizeof(int) * (size_t)(na + 1));
    if (!cl->head || !cl->next) return ORC_ERR_ALLOC;
    for (int c = 0; c < cl->ncell; ++c) cl->head[c] = -1;
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(na + 1));
    int32_t ncd[3];
    if (!cell_of) return ORC_ERR_ALLOC;
    orc_cells(p, na, x, cell_of, ncd);
    for (int a = 0; a < na; ++a) {
        cl->next[a] = cl->head[cell_of[a]];
        cl->head[cell_of[a]] = a;
    }
    free(cell_of);
    return ORC_OK;
}

static void free_cells(cell_list *cl) {
    free(cl->head);
    free(cl->next);
}

static int use_cells(const orc_params *p) {
    int nc[3];
    if (p->brute_force) return 0;
    cell_grid(p, nc);
    return nc[0] >= 3 && nc[1] >= 3 && nc[2] >= 3;
}

/* Calls visit(a, b) for every ordered pair a != b whose atoms lie in the same
 * or adjacent cells (or for every ordered pair, when cells are not used). */
typedef void (*pair_visit)(void *ctx, int a, int b);

static int for_candidate_pairs(const orc_params *p, int na, const double *x, pair_visit visit,
                               void *ctx) {
    if (!use_cells(p)) {
        for (int a = 0; a < na; ++a)
            for (int b = 0; b < na; ++b)
                if (b != a) visit(ctx, a, b);
        return ORC_OK;
    }
    cell_list cl;
    int err = build_cells(p, na, x, &cl);
    if (err) {
        free_cells(&cl);
        return err;
    }
    const int L[3] = {p->nx, p->ny, p->nz};
    for (int a = 0; a < na; ++a) {
        int c[3];
        for (int d = 0; d < 3; ++d) c[d] = cell_coord(x[d * na + a], cl.nc[d], L[d]);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int cc = (wrap(c[2] + dz, cl.nc[2]) * cl.nc[1] + wrap(c[1] + dy, cl.nc[1])) * cl.nc[0] +
                             wrap(c[0] + dx, cl.nc[0]);
                    for (int b = cl.head[cc]; b >= 0; b = cl.next[b])
                        if (b != a) visit(ctx, a, b);
                }
    }
    free_cells(&cl);
    return ORC_OK;
}

typedef struct {
    const orc_params *p;
    int na;
    const double *x;
    const adjacency *adj;
    double *F;
    double energy2; /* every pair is visited twice */
    int32_t *counts;
    const double *charge; /* or NULL */
} pair_ctx;

static void visit_force(void *vctx, int a, int b) {
    pair_ctx *c = (pair_ctx *)vctx;
    double d[3];
    min_image(c->p, c->x, c->na, a, b, d);
    double r2 = sq3(d);
    if (!(r2 < c->p->lj_rcut * c->p->lj_rcut)) return;
    if (bonded(c->adj, a, b)) return;
    double r = sqrt(r2), fmag, u;
    lj_shifted_force(c->p, r, &fmag, &u);
    if (c->charge && r2 < c->p->coul_rc * c->p->coul_rc) {
        double fq, uq;
        coulomb_shifted_force(c->p, c->charge[a] * c->charge[b], r, &fq, &uq);
        fmag += fq;
        u += uq;
    }
    for (int k = 0; k < 3; ++k) c->F[k * c->na + a] += fmag * d[k] / r;
    c->energy2 += u;
}

static void visit_count(void *vctx, int a, int b) {
    pair_ctx *c = (pair_ctx *)vctx;
    double d[3];
    min_image(c->p, c->x, c->na, a, b, d);
    if (sq3(d) < c->p->lj_rcut * c->p->lj_rcut) c->counts[a]++;
}

static int forces_with(const orc_params *p, const orc_topology *t, const adjacency *adj,
                       const double *x, double *F, double *energy) {
    int na = t->n_atoms;
    for (int k = 0; k < 3 * na; ++k) F[k] = 0.0;
    pair_ctx ctx = {p, na, x, adj, F, 0.0, NULL, t->charge};
    int err = for_candidate_pairs(p, na, x, visit_force, &ctx);
    if (err) return err;
    double e = 0.5 * ctx.energy2;
    for (int a = 0; a < na; ++a)
        for (int s = adj->start[a]; s < adj->start[a + 1]; ++s) {
            int b = adj->nbr[s];
            double d[3];
            min_image(p, x, na, a, b, d);
            double r = sqrt(sq3(d));
            double fmag = -adj->k[s] * (r - adj->r0[s]);
            for (int k = 0; k < 3; ++k) F[k * na + a] += fmag * d[k] / r;
            e += 0.25 * adj->k[s] * (r - adj->r0[s]) * (r - adj->r0[s]); /* each bond seen twice */
        }
    if (energy) *energy = e;
    return ORC_OK;
}

/* Conservative force on every atom (3 n_atoms SoA) and the potential energy. */
int orc_forces(const orc_params *p, const orc_topology *t, const double *x, double *F, double *energy) {
    adjacency adj;
    int err = build_adjacency(t, &adj);
    if (!err) err = forces_with(p, t, &adj, x, F, energy);
    free_adjacency(&adj);
    return err;
}

/* Number of other atoms within the LJ cutoff (strict r^2 < rc^2, FP64). */
int orc_neighbour_counts(const orc_params *p, int n_atoms, const double *x, int32_t *counts) {
    for (int a = 0; a < n_atoms; ++a) counts[a] = 0;
    pair_ctx ctx = {p, n_atoms, x, NULL, NULL, 0.0, counts, NULL};
    return for_candidate_pairs(p, n_atoms, x, visit_count, &ctx);
}

/* ---------------------------------------------------------------------- */
/* One coupled step (Sec. 2.2). f holds the post-streaming populations f_i(r,t)
 * (Q*N SoA), x the unwrapped positions and v the velocities (3*n_atoms SoA).
 * obs (optional, 4 doubles): sum_a J_a (the drag impulse the atoms received,
 * per component) and the mass-weighted squared radius of gyration after the
 * step. */
static double radius_gyration2(const orc_topology *t, const double *x) {
    int na = t->n_atoms;
    double M = 0, cm[3] = {0, 0, 0};
    for (int a = 0; a < na; ++a) {
        M += t->mass[a];
        for (int d = 0; d < 3; ++d) cm[d] += t->mass[a] * x[d * na + a];
    }
    if (M <= 0) return 0;
    for (int d = 0; d < 3; ++d) cm[d] /= M;
    double s = 0;
    for (int a = 0; a < na; ++a)
        for (int d = 0; d < 3; ++d) {
            double e = x[d * na + a] - cm[d];
            s += t->mass[a] * e * e;
        }
    return s / M;
}

typedef struct {
    double *fs, *g, *rho, *j, *ub, *G;
    double *U, *J, *F;
} work;

static void free_work(work *w) {
    free(w->fs);
    free(w->g);
    free(w->rho);
    free(w->j);
    free(w->ub);
    free(w->G);
    free(w->U);
    free(w->J);
    free(w->F);
}

static int alloc_work(const orc_params *p, int na, work *w) {
    size_t N = n_nodes(p);
    size_t A = (size_t)(na > 0 ? na : 1);
    memset(w, 0, sizeof(*w));
    w->fs = (double *)malloc(sizeof(double) * Q * N);
    w->g = (double *)malloc(sizeof(double) * 3 * N);
    w->rho = (double *)malloc(sizeof(double) * N);
    w->j = (double *)malloc(sizeof(double) * 3 * N);
    w->ub = (double *)malloc(sizeof(double) * 3 * N);
    w->G = (double *)malloc(sizeof(double) * 3 * N);
    w->U = (double *)malloc(sizeof(double) * 3 * A);
    w->J = (double *)malloc(sizeof(double) * 3 * A);
    w->F = (double *)malloc(sizeof(double) * 3 * A);
    if (!w->fs || !w->g || !w->rho || !w->j || !w->ub || !w->G || !w->U || !w->J || !w->F)
        return ORC_ERR_ALLOC;
    return ORC_OK;
}

static int check_params(const orc_params *p, const orc_topology *t) {
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return ORC_ERR_ARG;
    if (!(p->tau > 0.5)) return ORC_ERR_ARG;
    if (t->n_atoms > 0 && (p->n_md < 1 || !(p->lj_rcut > 0) || !(p->cell_min >= p->lj_rcut)))
        return ORC_ERR_ARG;
    if (p->forcing < 0 || p->forcing > 3 || p->force_dir < 0 || p->force_dir > 2 ||
        p->force_wave_axis < 0 || p->force_wave_axis > 2)
        return ORC_ERR_ARG;
    if (p->walls_z && p->nz < 2) return ORC_ERR_ARG;
    if (!(p->kT >= 0.0)) return ORC_ERR_ARG;
    if (t->charge && !(p->coul_rc > 0.0 && p->coul_rc <= p->lj_rcut)) return ORC_ERR_ARG;
    return ORC_OK;
}

static int step_once(const orc_params *p, const orc_topology *t, const adjacency *adj, work *w,
                     double *f, double *x, double *v, double *obs, int64_t step) {
    const size_t N = n_nodes(p);
    const int na = t->n_atoms;
    int err;

    /* Body force and moments of the current populations, Eq. (2). */
    orc_body_force(p, w->g);
    orc_moments((int64_t)N, f, w->rho, w->j);
    for (size_t k = 0; k < N; ++k)
        for (int d = 0; d < 3; ++d) w->ub[d * N + k] = (w->j[d * N + k] + 0.5 * w->g[d * N + k]) / w->rho[k];

    /* Fluid velocity at the atoms (R6). */
    for (size_t k = 0; k < 3 * N; ++k) w->G[k] = 0.0;
    if (na > 0) {
        err = orc_interp(p, w->ub, na, x, w->U);
        if (err) return err;

        /* Velocity Verlet with Stokes drag gamma (U - v) on the atom (R5, R7).
         * J accumulates the drag impulse each half-kick applies. */
        double *xs = (double *)malloc(sizeof(double) * 3 * (size_t)na);
        if (!xs) return ORC_ERR_ALLOC;
        memcpy(xs, x, sizeof(double) * 3 * (size_t)na); /* positions at the start of the step */
        const double dt = 1.0 / (double)p->n_md;
        err = forces_with(p, t, adj, x, w->F, NULL);
        if (err) {
            free(xs);
            return err;
        }
        for (int k = 0; k < 3 * na; ++k) w->J[k] = 0.0;
        if (p->reinterp) {
            /* R17: U at the position of each half-kick, each impulse spread with
             * the weights of that position. dJ holds minus the half-kick's impulse. */
            double *dJ = (double *)malloc(sizeof(double) * 3 * (size_t)na);
            if (!dJ) {
                free(xs);
                return ORC_ERR_ALLOC;
            }
            for (int s = 0; s < p->n_md && !err; ++s) {
                for (int half = 0; half < 2 && !err; ++half) {
                    if (half == 1) {
                        for (int k = 0; k < 3 * na; ++k) x[k] += dt * v[k];
                        err = forces_with(p, t, adj, x, w->F, NULL);
                        if (!err) err = orc_interp(p, w->ub, na, x, w->U);
                        if (err) break;
                    }
                    for (int a = 0; a < na; ++a)
                        for (int d = 0; d < 3; ++d) {
                            size_t q = (size_t)d * na + a;
                            double drag = p->gamma * (w->U[q] - v[q]);
                            w->J[q] += 0.5 * dt * drag;
                            dJ[q] = -0.5 * dt * drag;
                            v[q] += 0.5 * dt * (w->F[q] + drag) / t->mass[a];
                        }
                    if (!err) err = orc_spread(p, na, x, dJ, w->G);
                }
            }
            free(dJ);
            free(xs);
            if (err) return err;
        } else {
        for (int s = 0; s < p->n_md; ++s) {
            for (int a = 0; a < na; ++a)
                for (int d = 0; d < 3; ++d) {
                    size_t q = (size_t)d * na + a;
                    double drag = p->gamma * (w->U[q] - v[q]);
                    w->J[q] += 0.5 * dt * drag;
                    v[q] += 0.5 * dt * (w->F[q] + drag) / t->mass[a];
                }
            for (int k = 0; k < 3 * na; ++k) x[k] += dt * v[k];
            err = forces_with(p, t, adj, x, w->F, NULL);
            if (err) {
                free(xs);
                return err;
            }
            for (int a = 0; a < na; ++a)
                for (int d = 0; d < 3; ++d) {
                    size_t q = (size_t)d * na + a;
                    double drag = p->gamma * (w->U[q] - v[q]);
                    w->J[q] += 0.5 * dt * drag;
                    v[q] += 0.5 * dt * (w->F[q] + drag) / t->mass[a];
                }
        }
        /* Equal and opposite force on the fluid: G = -sum_a W_aj J_a / Delta t,
         * Delta t = 1, weights at the start-of-step positions (R5). */
        for (int k = 0; k < 3 * na; ++k) w->J[k] = -w->J[k];
        err = orc_spread(p, na, xs, w->J, w->G);
        for (int k = 0; k < 3 * na; ++k) w->J[k] = -w->J[k];
        free(xs);
        if (err) return err;
        }
    }

    /* Collision with the total force F = g + G (Eq. (1), R1, R4). */
    for (size_t k = 0; k < N; ++k) {
        double fl[Q], out[Q], F[3];
        for (int i = 0; i < Q; ++i) fl[i] = f[(size_t)i * N + k];
        for (int d = 0; d < 3; ++d) F[d] = w->g[d * N + k] + w->G[d * N + k];
        orc_collide_node(p->tau, fl, F, out);
        if (p->kT > 0.0) {
            double xi[Q];
            orc_node_noise(p, (int64_t)k, step, xi);
            for (int i = 0; i < Q; ++i) out[i] += xi[i];
        }
        for (int i = 0; i < Q; ++i) w->fs[(size_t)i * N + k] = out[i];
    }

    /* Streaming, Eq. (1) left-hand side: f_i(r + c_i) <- f*_i(r); half-way
     * bounce-back at the z walls (R10). */
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x0 = 0; x0 < p->nx; ++x0) {
                size_t k = node_at(p, x0, y, z);
                for (int i = 0; i < Q; ++i) {
                    int tz = z + CZ[i];
                    if (p->walls_z && (tz < 0 || tz > p->nz - 1)) {
                        f[(size_t)opposite(i) * N + k] = w->fs[(size_t)i * N + k];
                    } else {
                        size_t tk = node_at(p, wrap(x0 + CX[i], p->nx), wrap(y + CY[i], p->ny),
                                            wrap(tz, p->nz));
                        f[(size_t)i * N + tk] = w->fs[(size_t)i * N + k];
                    }
                }
            }

    if (obs) {
        for (int d = 0; d < 3; ++d) {
            double s = 0;
            for (int a = 0; a < na; ++a) s += w->J[d * na + a];
            obs[d] = s;
        }
        obs[3] = na > 0 ? radius_gyration2(t, x) : 0.0;
    }
    return ORC_OK;
}

/* Advance n_steps coupled steps in place. obs (optional) receives 4 doubles per
 * step as described above. Returns 0 or a negative error code. */
int orc_run(const orc_params *p, const orc_topology *t, double *f, double *x, double *v, int n_steps,
            double *obs) {
    int err = check_params(p, t);
    if (err) return err;
    adjacency adj;
    err = build_adjacency(t, &adj);
    if (err) {
        free_adjacency(&adj);
        return err;
    }
    work w;
    err = alloc_work(p, t->n_atoms, &w);
    for (int s = 0; s < n_steps && !err; ++s)
        err = step_once(p, t, &adj, &w, f, x, v, obs ? obs + 4 * s : NULL, p->step0 + s);
    free_work(&w);
    free_adjacency(&adj);
    return err;
}
