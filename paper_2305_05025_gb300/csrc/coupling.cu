// Fluid-solute coupling (Sec. 2.2): the fluid velocity is interpolated at each
// atom from the eight nearest nodes, and the opposite of the friction impulse
// each atom received is spread back onto the same nodes with the same weights.
#include "lbmd_internal.cuh"

namespace lbmd {

namespace {

__device__ __forceinline__ int wrapl(long long c, int n) {
    long long r = c % n;
    return (int)(r < 0 ? r + n : r);
}

// Start of a coupled step, one thread per atom: set the atom's FP32 step frame
// for the substeps, build its trilinear stencil from the FP64 position,
// interpolate u = (sum f c + g/2)/rho over the eight corners (pulled from the
// current post-collision buffer), and claim the corners in the touched-node
// list (each node enters once per step).
template <int S>
__global__ void __launch_bounds__(128) k_interp(CouplingArgs C, AtomArgs A, const typename Store<S>::T *b0,
                                                const typename Store<S>::T *b1) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= C.na) return;
    const int na = C.na;
    const int step = C.ds->step;
    const typename Store<S>::T *src = (step & 1) ? b1 : b0;
    const int par = (int)(((long long)step * A.n_md) & 1);
    const Lat &L = C.L;

    float4 fp, fl4;
    const bool finite = set_frame(A, a, fp, fl4);
    A.P[par][a] = fp;
    A.L[par][a] = fl4;
    if (!finite) atomicOr(&C.ds->flags, FLAG_NONFINITE);
    const double x[3] = {C.X[a], C.X[na + a], C.X[2 * na + a]};

    int b[3];
    float t[3];
    const int n[3] = {L.nx, L.ny, L.nz};
    for (int d = 0; d < 3; ++d) {
        double fl = floor(x[d]);
        if (!(fabs(fl) < 4.0e15)) fl = 0.0;
        t[d] = (float)(x[d] - fl);
        long long bl = (long long)fl;
        if (d == 2 && L.walls) {
            if (bl < 0 || bl + 1 > L.nz - 1) {
                atomicOr(&C.ds->flags, FLAG_WALL);
                bl = bl < 0 ? 0 : L.nz - 2;
            }
            b[d] = (int)bl;
        } else {
            b[d] = wrapl(bl, n[d]);
        }
        C.base[d * na + a] = b[d];
        C.frac[d * na + a] = t[d];
    }
    const int stamp = step + 1;
    float U[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
        const int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
        const int nxk = o[0] ? (b[0] + 1 == L.nx ? 0 : b[0] + 1) : b[0];
        const int nyk = o[1] ? (b[1] + 1 == L.ny ? 0 : b[1] + 1) : b[1];
        const int nzk = o[2] ? (b[2] + 1 == L.nz ? 0 : b[2] + 1) : b[2];
        const float W = (o[0] ? t[0] : 1.f - t[0]) * (o[1] ? t[1] : 1.f - t[1]) * (o[2] ? t[2] : 1.f - t[2]);
        float f[Q], g[3], u[3];
        pull<S>(src, L, nxk, nyk, nzk, f);
        body_force(L, nxk, nyk, nzk, g);
        node_velocity(L, f, g, u);
        U[0] += W * u[0];
        U[1] += W * u[1];
        U[2] += W * u[2];
        const int node = (int)(((size_t)nzk * L.ny + nyk) * L.nx + nxk);
        if (C.tag[node] != stamp && atomicExch(&C.tag[node], stamp) != stamp) {
            const int i = atomicAdd(&C.ds->n_touched, 1);
            if (i < C.touched_cap)
                C.touched[i] = node;
            else
                atomicOr(&C.ds->flags, FLAG_TOUCHED);
        }
    }
    for (int d = 0; d < 3; ++d) C.U[d * na + a] = U[d];
}

// End of the atoms' part of the step: G_j -= W_aj J_a / Delta t (Delta t = 1)
// on the eight corners of the step-start stencil.
__global__ void __launch_bounds__(128) k_spread(CouplingArgs C) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= C.na) return;
    const int na = C.na;
    const Lat &L = C.L;
    int b[3];
    float t[3], J[3];
    for (int d = 0; d < 3; ++d) {
        b[d] = C.base[d * na + a];
        t[d] = C.frac[d * na + a];
        J[d] = C.J[d * na + a];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
        const int nxk = o[0] ? (b[0] + 1 == L.nx ? 0 : b[0] + 1) : b[0];
        const int nyk = o[1] ? (b[1] + 1 == L.ny ? 0 : b[1] + 1) : b[1];
        const int nzk = o[2] ? (b[2] + 1 == L.nz ? 0 : b[2] + 1) : b[2];
        const float W = (o[0] ? t[0] : 1.f - t[0]) * (o[1] ? t[1] : 1.f - t[1]) * (o[2] ? t[2] : 1.f - t[2]);
        const size_t node = ((size_t)nzk * L.ny + nyk) * L.nx + nxk;
        atomicAdd(&C.G[node], make_float4(-W * J[0], -W * J[1], -W * J[2], 0.f));
    }
}

}  // namespace

cudaError_t launch_interp(int store, const CouplingArgs &c, const AtomArgs &a, void *const buf[2], cudaStream_t s) {
    if (c.na == 0) return cudaSuccess;
    const int grid = (c.na + 127) / 128;
    switch (store) {
    case LBMD_F32:
        k_interp<LBMD_F32><<<grid, 128, 0, s>>>(c, a, (const float *)buf[0], (const float *)buf[1]);
        break;
    case LBMD_F16_SHIFTED:
        k_interp<LBMD_F16_SHIFTED><<<grid, 128, 0, s>>>(c, a, (const __half *)buf[0], (const __half *)buf[1]);
        break;
    default:
        k_interp<LBMD_BF16_SHIFTED>
            <<<grid, 128, 0, s>>>(c, a, (const __nv_bfloat16 *)buf[0], (const __nv_bfloat16 *)buf[1]);
    }
    return cudaGetLastError();
}

cudaError_t launch_spread(const CouplingArgs &c, cudaStream_t s) {
    if (c.na == 0) return cudaSuccess;
    k_spread<<<(c.na + 127) / 128, 128, 0, s>>>(c);
    return cudaGetLastError();
}

}  // namespace lbmd
