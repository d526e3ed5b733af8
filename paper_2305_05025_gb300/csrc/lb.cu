// Lattice kernels other than the dense update (in lb_step.cu): the sparse
// re-collision of the nodes that carry a coupling force (Eq. 1 with the force
// g + G, Sec. 2.2), state set-up and read-back, the pull applied to adjoint
// fields, and the FP64 global sums. Same layout as the dense update: 19
// planes of N values, population i of node n at i*N + n.
#include "lbmd_internal.cuh"

namespace lbmd {

namespace {

// Nodes touched by atoms: redo the collision with F = g + G from the same
// pre-collision buffer, overwrite the dense kernel's result, clear G. The
// last block to finish advances the step counter and empties the list.
template <int S>
__global__ void __launch_bounds__(256) k_lb_fix(Lat L, typename Store<S>::T *b0, typename Store<S>::T *b1,
                                                const int *touched, int cap, float4 *G, long long *gfix, DevState *ds,
                                                int keep) {
    const int cnt = min(ds->n_touched, cap);
    const int step = ds->step;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const typename Store<S>::T *src = (step & 1) ? b1 : b0;
        typename Store<S>::T *dst = (step & 1) ? b0 : b1;
        const int node = touched[i];
        const int x = node % L.nx;
        const int y = (node / L.nx) % L.ny;
        const int z = node / (L.nx * L.ny);
        float f[Q], F[3];
        pull<S>(src, L, x, y, z, f);
        body_force(L, x, y, z, F);
        float4 Gn;
        if (gfix) {  // deterministic mode: the exact fixed-point sums of this touched slot
            long long *g = gfix + 3 * (size_t)i;
            Gn = make_float4((float)((double)g[0] / kFixScale), (float)((double)g[1] / kFixScale),
                             (float)((double)g[2] / kFixScale), 0.f);
            g[0] = g[1] = g[2] = 0;
        } else {
            Gn = G[node];
        }
        F[0] += Gn.x;
        F[1] += Gn.y;
        F[2] += Gn.z;
        const float rho = collide(L, f, F);
        if (!isfinite(rho)) atomicOr(&ds->flags, FLAG_NONFINITE);
        if (L.thermal) {  // the same noise the dense kernel added at this node and step
            float xi[Q];
            node_noise(L, (unsigned)node, (unsigned)step, 1.f, xi);
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] += xi[q];
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) Store<S>::st_plain(dst + (size_t)q * L.N + node, f[q]);
        if (!keep) G[node] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&ds->ticket, 1u);
        if (t == gridDim.x - 1) {
            ds->step = step + 1;
            if (!keep) ds->n_touched = 0;
            ds->ticket = 0;
            __threadfence();
        }
    }
}

// dst_i(x) = src_i(x - c_i) (or src_opp(i)(x) behind a z wall) on FP32 arrays:
// the pull of the streaming step, applied to adjoint fields.
__global__ void k_pull_f32(Lat L, const float *src, float *dst) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= L.nx || y >= L.ny) return;
    float f[Q];
    pull<LBMD_F32>(src, L, x, y, z, f);
    const size_t node = ((size_t)z * L.ny + y) * L.nx + x;
#pragma unroll
    for (int i = 0; i < Q; ++i) dst[(size_t)i * L.N + node] = f[i];
}

template <int S>
__global__ void k_lb_fields(Lat L, const typename Store<S>::T *cur, float *fout, float *rho_out, float *u_out,
                            DevState *ds) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= L.nx || y >= L.ny) return;
    float f[Q], g[3], u[3];
    pull<S>(cur, L, x, y, z, f);
    body_force(L, x, y, z, g);
    const float rho = node_velocity(L, f, g, u);
    if (!isfinite(rho)) atomicOr(&ds->flags, FLAG_NONFINITE);
    const size_t node = ((size_t)z * L.ny + y) * L.nx + x;
    if (fout)
#pragma unroll
        for (int i = 0; i < Q; ++i) fout[(size_t)i * L.N + node] = f[i] + wgt(i) * L.rho0;
    if (rho_out) rho_out[node] = rho;
    if (u_out) {
        u_out[node] = u[0];
        u_out[L.N + node] = u[1];
        u_out[2 * L.N + node] = u[2];
    }
}

// Inverse of the pull: h_j(y) = f_j(y + c_j), or f_opp(j)(y) when y + c_j is
// behind a z wall. From f itself, or from f = f_eq(rho, u) evaluated at the
// source node.
template <int S>
__global__ void k_lb_init(Lat L, typename Store<S>::T *dst, const float *f, const float *rho, const float *u) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= L.nx || y >= L.ny) return;
    const size_t node = ((size_t)z * L.ny + y) * L.nx + x;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int tz = z + cz(j);
        const bool wall = L.walls && (tz < 0 || tz > L.nz - 1);
        int q = j;
        size_t sn = node;
        if (wall) {
            q = opp(j);
        } else {
            const int tx = (x + cx(j) + L.nx) % L.nx, ty = (y + cy(j) + L.ny) % L.ny, tzz = (tz + L.nz) % L.nz;
            sn = ((size_t)tzz * L.ny + ty) * L.nx + tx;
        }
        float v;
        if (f) {
            v = f[(size_t)q * L.N + sn] - wgt(q) * L.rho0;
        } else {
            const float r = rho[sn];
            const float ux = u[sn], uy = u[L.N + sn], uz = u[2 * L.N + sn];
            const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
            const float usq = ux * ux + uy * uy + uz * uz;
            v = wgt(q) * ((r - L.rho0) + r * (3.f * cu + 4.5f * cu * cu - 1.5f * usq));
        }
        Store<S>::st_plain(dst + (size_t)j * L.N + node, v);
    }
}

// FP64 block partial sums of (sum delta f, sum delta f c) over post-streaming
// populations; the fluid mass is N rho0 + sum delta f.
template <int S>
__global__ void __launch_bounds__(256) k_lb_reduce(Lat L, const typename Store<S>::T *cur, double *partials,
                                                   DevState *ds) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < L.N; n += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(n % L.nx);
        const int y = (int)((n / L.nx) % L.ny);
        const int z = (int)(n / ((size_t)L.nx * L.ny));
        float f[Q];
        pull<S>(cur, L, x, y, z, f);
        float r = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            r += f[i];
            jx += cx(i) * f[i];
            jy += cy(i) * f[i];
            jz += cz(i) * f[i];
        }
        bad = bad || !isfinite(r) || !isfinite(jx) || !isfinite(jy) || !isfinite(jz);
        acc[0] += r;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += jz;
    }
    if (bad) atomicOr(&ds->flags, FLAG_NONFINITE);
    __shared__ double sh[4][256 / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 4; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += sh[threadIdx.x][w];
        partials[(size_t)blockIdx.x * 4 + threadIdx.x] = s;
    }
}

__global__ void __launch_bounds__(256) k_atom_momentum(const float *V, const float *mass, int na, double *partials,
                                                       DevState *ds) {
    double acc[3] = {0.0, 0.0, 0.0};
    bool bad = false;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < na; a += gridDim.x * blockDim.x) {
        for (int d = 0; d < 3; ++d) {
            const float v = V[d * na + a];
            bad = bad || !isfinite(v);
            acc[d] += (double)mass[a] * (double)v;
        }
    }
    if (bad) atomicOr(&ds->flags, FLAG_NONFINITE);
    __shared__ double sh[3][256 / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 3; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += sh[threadIdx.x][w];
        partials[(size_t)blockIdx.x * 3 + threadIdx.x] = s;
    }
}

// Deterministic final sum of block partials (fixed order, one block).
__global__ void k_reduce_finish(const double *partials, int nblocks, int width, double *out) {
    __shared__ double sh[256];
    for (int k = 0; k < width; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[(size_t)b * width + k];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sh[0];
        __syncthreads();
    }
}



}  // namespace

cudaError_t launch_lb_fix(int store, const Lat &L, void *const buf[2], const CouplingArgs &c, int grid,
                          cudaStream_t s) {
    LBMD_DISPATCH(store, (k_lb_fix<SV><<<grid, 256, 0, s>>>(L, (T *)buf[0], (T *)buf[1], c.touched, c.touched_cap,
                                                             c.G, c.gfix, c.ds, c.keep)));
    return cudaGetLastError();
}

cudaError_t launch_lb_fields(int store, const Lat &L, const void *cur, float *f, float *rho, float *u,
                             DevState *ds, cudaStream_t s) {
    const dim3 b = node_block(L), g = node_grid(L, b);
    LBMD_DISPATCH(store, (k_lb_fields<SV><<<g, b, 0, s>>>(L, (const T *)cur, f, rho, u, ds)));
    return cudaGetLastError();
}

cudaError_t launch_pull_f32(const Lat &L, const float *src, float *dst, cudaStream_t s) {
    const dim3 b = node_block(L), g = node_grid(L, b);
    k_pull_f32<<<g, b, 0, s>>>(L, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_lb_init(int store, const Lat &L, void *dst, const float *f, const float *rho, const float *u,
                           cudaStream_t s) {
    const dim3 b = node_block(L), g = node_grid(L, b);
    LBMD_DISPATCH(store, (k_lb_init<SV><<<g, b, 0, s>>>(L, (T *)dst, f, rho, u)));
    return cudaGetLastError();
}

cudaError_t launch_lb_reduce(int store, const Lat &L, const void *cur, double *partials, int nblocks, DevState *ds,
                             cudaStream_t s) {
    LBMD_DISPATCH(store, (k_lb_reduce<SV><<<nblocks, 256, 0, s>>>(L, (const T *)cur, partials, ds)));
    return cudaGetLastError();
}

cudaError_t launch_reduce_finish(const double *partials, int nblocks, int width, double *out, cudaStream_t s) {
    k_reduce_finish<<<1, 256, 0, s>>>(partials, nblocks, width, out);
    return cudaGetLastError();
}

cudaError_t launch_atom_momentum(const float *V, const float *mass, int na, double *partials, int nblocks,
                                 DevState *ds, cudaStream_t s) {
    k_atom_momentum<<<nblocks, 256, 0, s>>>(V, mass, na, partials, ds);
    return cudaGetLastError();
}

}  // namespace lbmd
