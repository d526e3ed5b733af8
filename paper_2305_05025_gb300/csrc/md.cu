// Solute kernels: pair-search buckets, shifted-force Lennard-Jones + harmonic
// bonds, and the velocity-Verlet substeps with Stokes friction (Sec. 2.2: the
// atom receives gamma (u - v), u interpolated at the start of the coupled step).
//
// One kernel launch per substep, one thread per atom. Kernel k of a step
// (k = 0..n_md) finishes substep k-1 (force at x_k, second half-kick) and
// starts substep k (first half-kick, drift to x_{k+1}, insertion of the atom
// into the buckets of generation k+1). Buckets rotate over three buffers by
// generation g = step*n_md + k: kernel k reads g, fills g+1 and empties g-1.
#include "lbmd_internal.cuh"

namespace lbmd {

namespace {

__device__ __forceinline__ int wrapi(int c, int n) {
    int r = c % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ void unpack_cref(float w, int c[3]) {
    const unsigned u = __float_as_uint(w);
    c[0] = (int)(u & 1023u);
    c[1] = (int)((u >> CREF_BITS) & 1023u);
    c[2] = (int)((u >> (2 * CREF_BITS)) & 1023u);
}

__device__ __forceinline__ float pack_cref(const int c[3]) {
    return __uint_as_float((unsigned)c[0] | ((unsigned)c[1] << CREF_BITS) | ((unsigned)c[2] << (2 * CREF_BITS)));
}

// Nearest periodic image of a cell-index difference.
__device__ __forceinline__ int wrapdiff(int d, int n) {
    if (2 * d > n) return d - n;
    if (2 * d < -n) return d + n;
    return d;
}

// x_a - x_b from the per-step reference cells and FP32 offsets.
__device__ __forceinline__ void disp(const AtomArgs &A, float4 pa, const int ca[3], float4 pb, float d[3]) {
    int cb[3];
    unpack_cref(pb.w, cb);
    d[0] = (float)wrapdiff(ca[0] - cb[0], A.nc[0]) * A.h[0] + (pa.x - pb.x);
    d[1] = (float)wrapdiff(ca[1] - cb[1], A.nc[1]) * A.h[1] + (pa.y - pb.y);
    d[2] = (float)wrapdiff(ca[2] - cb[2], A.nc[2]) * A.h[2] + (pa.z - pb.z);
}

__device__ __forceinline__ int bucket_of(const AtomArgs &A, const int c[3]) {
    return ((c[2] % A.fold[2]) * A.fold[1] + (c[1] % A.fold[1])) * A.fold[0] + (c[0] % A.fold[0]);
}

// Current cell of an atom from its reference cell and FP32 offset.
__device__ __forceinline__ void current_cell(const AtomArgs &A, float4 p, const int cr[3], int c[3]) {
    c[0] = wrapi(cr[0] + (int)floorf(p.x * A.inv_h[0]), A.nc[0]);
    c[1] = wrapi(cr[1] + (int)floorf(p.y * A.inv_h[1]), A.nc[1]);
    c[2] = wrapi(cr[2] + (int)floorf(p.z * A.inv_h[2]), A.nc[2]);
}

__device__ __forceinline__ bool bonded(const AtomArgs &A, int a, int b) {
    for (int s = A.bstart[a]; s < A.bstart[a + 1]; ++s)
        if (A.bpart[s] == b) return true;
    return false;
}

// Conservative force on atom a at the positions P (buckets of generation g3).
__device__ void md_force(const AtomArgs &A, const float4 *__restrict__ P, int g3, int a, float4 pa, float F[3]) {
    int ca[3], cc[3];
    unpack_cref(pa.w, ca);
    current_cell(A, pa, ca, cc);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const int *__restrict__ cnt = A.count[g3];
    const int *__restrict__ slots = A.slot[g3];
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                const int c[3] = {wrapi(cc[0] + ox, A.nc[0]), wrapi(cc[1] + oy, A.nc[1]), wrapi(cc[2] + oz, A.nc[2])};
                const int b = bucket_of(A, c);
                const int n = min(cnt[b], A.cap);
                const int *s = slots + (size_t)b * A.cap;
                for (int j = 0; j < n; ++j) {
                    const int q = s[j];
                    if (q == a) continue;
                    float d[3];
                    disp(A, pa, ca, P[q], d);
                    const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (!(r2 < A.rc2f)) continue;
                    if (bonded(A, a, q)) continue;
                    const float inv_r2 = 1.0f / r2;
                    const float sr2 = A.lj_sig2 * inv_r2;
                    const float sr6 = sr2 * sr2 * sr2;
                    const float fr = A.lj_24eps * inv_r2 * sr6 * (2.f * sr6 - 1.f) - A.lj_fc * rsqrtf(r2);
                    fx += fr * d[0];
                    fy += fr * d[1];
                    fz += fr * d[2];
                }
            }
    for (int s = A.bstart[a]; s < A.bstart[a + 1]; ++s) {
        float d[3];
        disp(A, pa, ca, P[A.bpart[s]], d);
        const float r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const float fr = -A.bk[s] * (r - A.br0[s]) / r;
        fx += fr * d[0];
        fy += fr * d[1];
        fz += fr * d[2];
    }
    F[0] = fx;
    F[1] = fy;
    F[2] = fz;
}

__device__ __forceinline__ void insert(const AtomArgs &A, int g3, int a, const int c[3]) {
    const int b = bucket_of(A, c);
    const int s = atomicAdd(&A.count[g3][b], 1);
    if (s < A.cap)
        A.slot[g3][(size_t)b * A.cap + s] = a;
    else
        atomicOr(&A.ds->flags, FLAG_CELL);
    A.bucket[g3][a] = b;
}

// Exact FP64 cell coordinate floor((x * nc) / L) mod nc.
__device__ __forceinline__ int exact_cell(double x, int nc, double L) {
    const double s = __ddiv_rn(__dmul_rn(x, (double)nc), L);
    const double fl = floor(s);
    if (!(fabs(fl) < 4.0e15)) return 0;
    long long c = (long long)fl % nc;
    return (int)(c < 0 ? c + nc : c);
}

// set_state: reference frame at generation 0, exact binning, empty records.
__global__ void k_prime_insert(AtomArgs A) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.na) return;
    int cr[3];
    float p0[3];
    bool finite = true;
    for (int d = 0; d < 3; ++d) {
        const double x = A.X[d * A.na + a];
        finite = finite && isfinite(x);
        const double s = x * ((double)A.nc[d] / A.Ld[d]);
        double fl = floor(s);
        if (!(fabs(fl) < 4.0e15)) fl = 0.0;
        long long c = (long long)fl % A.nc[d];
        cr[d] = (int)(c < 0 ? c + A.nc[d] : c);
        p0[d] = (float)((s - fl) * A.hd[d]);
        A.P0[d * A.na + a] = p0[d];
        A.Plo[d * A.na + a] = 0.f;
    }
    if (!finite) atomicOr(&A.ds->flags, FLAG_NONFINITE);
    A.P[0][a] = make_float4(p0[0], p0[1], p0[2], pack_cref(cr));
    int c[3];
    for (int d = 0; d < 3; ++d) c[d] = exact_cell(A.X[d * A.na + a], A.nc[d], A.Ld[d]);
    insert(A, 0, a, c);
    A.bucket[2][a] = 0;
    A.bucket[1][a] = 0;
}

__global__ void k_prime_force(AtomArgs A) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.na) return;
    float F[3];
    md_force(A, A.P[0], 0, a, A.P[0][a], F);
    for (int d = 0; d < 3; ++d) A.F[d * A.na + a] = F[d];
}

__global__ void __launch_bounds__(128) k_md_substep(AtomArgs A, int k) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.na) return;
    const long long gen = (long long)A.ds->step * A.n_md + k;
    const int par = (int)(gen & 1);
    const int g3 = (int)(gen % 3), gn3 = (int)((gen + 1) % 3), gp3 = (int)((gen + 2) % 3);
    const float4 pa = A.P[par][a];
    const int na = A.na;

    float F[3];
    if (k == 0) {
        for (int d = 0; d < 3; ++d) F[d] = A.F[d * na + a];
    } else {
        md_force(A, A.P[par], g3, a, pa, F);
    }
    float v[3], U[3], J[3];
    const float im = A.inv_m[a];
    for (int d = 0; d < 3; ++d) {
        v[d] = A.V[d * na + a];
        U[d] = A.U[d * na + a];
        J[d] = k == 0 ? 0.f : A.J[d * na + a];
    }
    if (k > 0) {  // second half-kick of substep k-1, drag at v_{k-1/2}
        for (int d = 0; d < 3; ++d) {
            const float drag = A.gamma * (U[d] - v[d]);
            J[d] += A.hdt * drag;
            v[d] += A.hdt * (F[d] + drag) * im;
        }
    }
    if (k < A.n_md) {  // first half-kick of substep k, drag at v_k, then drift
        for (int d = 0; d < 3; ++d) {
            const float drag = A.gamma * (U[d] - v[d]);
            J[d] += A.hdt * drag;
            v[d] += A.hdt * (F[d] + drag) * im;
        }
        float p[3] = {pa.x, pa.y, pa.z};
        for (int d = 0; d < 3; ++d) {
            // Compensated sum p + v dt (two-sum plus the exact product error).
            const float inc = v[d] * A.dt;
            const float e_mul = fmaf(v[d], A.dt, -inc);
            const float s = p[d] + inc;
            const float bp = s - p[d];
            const float e_add = (p[d] - (s - bp)) + (inc - bp);
            p[d] = s;
            A.Plo[d * na + a] += e_add + e_mul;
        }
        const float4 pn = make_float4(p[0], p[1], p[2], pa.w);
        A.P[par ^ 1][a] = pn;
        A.count[gp3][A.bucket[gp3][a]] = 0;
        int cr[3], c[3];
        unpack_cref(pa.w, cr);
        current_cell(A, pn, cr, c);
        insert(A, gn3, a, c);
        if (!(isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]))) atomicOr(&A.ds->flags, FLAG_NONFINITE);
    } else {
        // End of the coupled step: cache the force and advance the FP64
        // accumulator by the compensated displacement.
        const float pc[3] = {pa.x, pa.y, pa.z};
        for (int d = 0; d < 3; ++d) {
            A.F[d * na + a] = F[d];
            const double disp64 = ((double)pc[d] - (double)A.P0[d * na + a]) + (double)A.Plo[d * na + a];
            A.X[d * na + a] += disp64;
        }
    }
    for (int d = 0; d < 3; ++d) {
        A.V[d * na + a] = v[d];
        A.J[d * na + a] = J[d];
    }
}

// Diagnostics: exact FP64 cells and neighbour counts (strict r^2 < rc^2,
// minimum image), searched through the buckets of the current generation.
// An atom missing from its bucket is reported as cell -1.
__global__ void k_md_diag(AtomArgs A, int *cell_of, int *neigh) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.na) return;
    const long long gen = (long long)A.ds->step * A.n_md;
    const int g3 = (int)(gen % 3);
    const int na = A.na;
    int c[3];
    for (int d = 0; d < 3; ++d) c[d] = exact_cell(A.X[d * na + a], A.nc[d], A.Ld[d]);
    const int lin = (c[2] * A.nc[1] + c[1]) * A.nc[0] + c[0];
    bool found = false;
    {
        const int b = bucket_of(A, c);
        const int n = min(A.count[g3][b], A.cap);
        for (int j = 0; j < n; ++j) found = found || A.slot[g3][(size_t)b * A.cap + j] == a;
    }
    if (cell_of) cell_of[a] = found ? lin : -1;
    if (!neigh) return;
    int count = 0;
    const double xa[3] = {A.X[a], A.X[na + a], A.X[2 * na + a]};
    // A 5x5x5 block of cells covers any bucket an atom within rc can sit in
    // after FP32 binning (at most one cell from its exact cell). The block's
    // buckets are distinct (fold >= 5, or small grids visit each residue
    // once), so every atom is seen at most once; atoms of folded far cells
    // fail the distance test.
    for (int oz = -2; oz <= 2; ++oz)
        for (int oy = -2; oy <= 2; ++oy)
            for (int ox = -2; ox <= 2; ++ox) {
                const int o[3] = {ox, oy, oz};
                int cc[3];
                bool dup = false;
                for (int d = 0; d < 3; ++d) {
                    cc[d] = wrapi(c[d] + o[d], A.nc[d]);
                    // skip offsets that alias a nearer one on small grids
                    if (A.nc[d] < 5 && (o[d] > A.nc[d] / 2 || o[d] < -((A.nc[d] - 1) / 2))) dup = true;
                }
                if (dup) continue;
                const int b = bucket_of(A, cc);
                const int n = min(A.count[g3][b], A.cap);
                for (int j = 0; j < n; ++j) {
                    const int q = A.slot[g3][(size_t)b * A.cap + j];
                    if (q == a) continue;
                    double r2 = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        double dd = __dsub_rn(xa[d], A.X[d * na + q]);
                        dd = __dsub_rn(dd, __dmul_rn(A.Ld[d], nearbyint(__ddiv_rn(dd, A.Ld[d]))));
                        r2 = __dadd_rn(r2, __dmul_rn(dd, dd));
                    }
                    if (r2 < A.rc2d) ++count;
                }
            }
    neigh[a] = count;
}

}  // namespace

cudaError_t launch_md_prime(const AtomArgs &a, cudaStream_t s) {
    if (a.na == 0) return cudaSuccess;
    const int grid = (a.na + 127) / 128;
    k_prime_insert<<<grid, 128, 0, s>>>(a);
    k_prime_force<<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_md_substep(const AtomArgs &a, int k, cudaStream_t s) {
    if (a.na == 0) return cudaSuccess;
    k_md_substep<<<(a.na + 127) / 128, 128, 0, s>>>(a, k);
    return cudaGetLastError();
}

cudaError_t launch_md_diag(const AtomArgs &a, int *cell_of, int *neigh, cudaStream_t s) {
    if (a.na == 0) return cudaSuccess;
    k_md_diag<<<(a.na + 127) / 128, 128, 0, s>>>(a, cell_of, neigh);
    return cudaGetLastError();
}

}  // namespace lbmd
