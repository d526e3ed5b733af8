// Lattice kernels: the fused pull-stream + BGK collide + Guo-force update of
// every node (Eq. 1 with the standard minus sign, Sec. 2.2), the sparse
// re-collision of the nodes that carry a coupling force, state set-up and
// read-back, and the FP64 global sums.
//
// Layout: 19 planes of N = nx*ny*nz values (SoA), population i of node n at
// i*N + n, stored as delta f = f - w_i rho0 in FP32, FP16 or BF16. Two
// buffers hold post-collision values; step s reads buffer s&1 and writes the
// other. One thread per node, threads along x within a warp, so each of the 19
// loads and stores of a warp is one contiguous run (shifted by one element for
// speeds with c_x != 0).
#include "lbmd_internal.cuh"

namespace lbmd {

namespace {

// The 19 pulled values of one node from its entry sp in plane 0; W: this z
// plane borders a wall (half-way bounce-back from the node's own opposite
// population).
template <int S, bool W>
__device__ __forceinline__ void pull_node(const typename Store<S>::T *sp, ptrdiff_t plane, int oxm, int oxp, int oym,
                                          int oyp, int ozm, int ozp, bool wlo, bool whi, float f[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int off = (cx(i) == 1 ? oxm : (cx(i) == -1 ? oxp : 0)) + (cy(i) == 1 ? oym : (cy(i) == -1 ? oyp : 0)) +
                        (cz(i) == 1 ? ozm : (cz(i) == -1 ? ozp : 0));
        const bool wall = W && ((cz(i) == 1 && wlo) || (cz(i) == -1 && whi));
        f[i] = Store<S>::ld_raw(wall ? sp + (opp(i) - i) * plane : sp + off);
        sp += plane;
    }
}

// Dense update of every node with F = g. Kept to few instructions per node
// (the kernel issues about as fast as HBM delivers): the pull's neighbour
// offsets are 32-bit per-thread constants (periodic wrap folded in), plane
// i starts at i * plane_bytes, and the collision pairs each speed with its
// opposite and is specialised on the direction FD of the body force
// (collide_g), in stored units.
template <int S, int FD, bool TH>
__global__ void __launch_bounds__(256) k_lb_step(Lat L, typename Store<S>::T *b0, typename Store<S>::T *b1,
                                                 DevState *ds) {
    using T = typename Store<S>::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= L.nx || y >= L.ny) return;
    const int step = ds->step;
    const T *src = (step & 1) ? b1 : b0;
    T *dst = (step & 1) ? b0 : b1;
    const int nx = L.nx, nxy = L.nx * L.ny;
    // Offset of the source node x - c for each sign of each component.
    const int oxm = x == 0 ? nx - 1 : -1, oxp = x == nx - 1 ? 1 - nx : 1;
    const int oym = y == 0 ? nxy - nx : -nx, oyp = y == L.ny - 1 ? nx - nxy : nx;
    const int ozm = z == 0 ? (L.nz - 1) * nxy : -nxy, ozp = z == L.nz - 1 ? (1 - L.nz) * nxy : nxy;
    const bool wlo = L.walls && z == 0, whi = L.walls && z == L.nz - 1;
    const int node = z * nxy + y * nx + x;
    const ptrdiff_t plane = (ptrdiff_t)L.N;
    float f[Q];
    // Only the first and last planes of a walled lattice test for walls (the
    // branch is uniform: a block holds one z plane).
    if (wlo || whi)
        pull_node<S, true>(src + node, plane, oxm, oxp, oym, oyp, ozm, ozp, wlo, whi, f);
    else
        pull_node<S, false>(src + node, plane, oxm, oxp, oym, oyp, ozm, ozp, false, false, f);
    const float rho = collide_g<FD, Store<S>::kScaled>(L, f, body_amp(L, x, y, z));
    if (!isfinite(rho)) atomicOr(&ds->flags, FLAG_NONFINITE);
    if (TH) {  // thermal noise, in stored units
        float xi[Q];
        node_noise(L, (unsigned)node, (unsigned)step, Store<S>::kScaled ? kF16Scale : 1.f, xi);
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] += xi[i];
    }
    T *dp = dst + node;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        Store<S>::st_raw(dp, f[i]);
        dp += plane;
    }
}

// 16-bit helpers: a pair of neighbouring nodes' values as one 32-bit word
// (node x0 in the low half, x0 + 1 in the high half).
template <int S> struct Half16;
template <> struct Half16<LBMD_F16_SHIFTED> {
    // (low, high) halves of a word as floats, in stored units.
    static __device__ __forceinline__ float2 unpack(unsigned w) {
        __half2 h;
        memcpy(&h, &w, 4);
        return __half22float2(h);
    }
    static __device__ __forceinline__ unsigned pack(float lo, float hi) {
        const __half2 h = __floats2half2_rn(lo, hi);
        unsigned w;
        memcpy(&w, &h, 4);
        return w;
    }
};
template <> struct Half16<LBMD_BF16_SHIFTED> {
    static __device__ __forceinline__ float2 unpack(unsigned w) {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    static __device__ __forceinline__ unsigned pack(float lo, float hi) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        unsigned w;
        memcpy(&w, &h, 4);
        return w;
    }
};

// The 19 pulled words (two nodes each) of a node pair from its entry sp in
// plane 0. The +-1 shift along x comes from the neighbouring lane's word
// (byte permutes), or from one 16-bit load at a row or warp edge; W: this z
// plane borders a wall.
template <int S, bool W>
__device__ __forceinline__ void pull_pair(const typename Store<S>::T *sp, ptrdiff_t plane, int oym, int oyp, int ozm,
                                          int ozp, bool wlo, bool whi, bool left_ok, bool right_ok, int xl, int xr,
                                          unsigned w[Q]) {
    using T = typename Store<S>::T;
#pragma unroll
    for (int i = 0; i < Q; ++i, sp += plane) {
        const int oyz = (cy(i) == 1 ? oym : (cy(i) == -1 ? oyp : 0)) + (cz(i) == 1 ? ozm : (cz(i) == -1 ? ozp : 0));
        const bool wall = W && ((cz(i) == 1 && wlo) || (cz(i) == -1 && whi));
        const T *row = wall ? sp + (opp(i) - i) * plane : sp + oyz;
        const unsigned v = __ldg(reinterpret_cast<const unsigned *>(row));
        if (cx(i) == 0) {
            w[i] = v;
        } else if (cx(i) == 1) {  // x0 pulls x0 - 1 (high half of the left word), x0 + 1 pulls x0
            unsigned prev = __shfl_up_sync(0xffffffffu, v, 1);
            if (!left_ok) prev = (unsigned)__ldg(reinterpret_cast<const unsigned short *>(row + xl)) << 16;
            w[i] = wall ? v : __byte_perm(prev, v, 0x5432);
        } else {  // x0 pulls x0 + 1, x0 + 1 pulls x0 + 2 (low half of the right word)
            unsigned next = __shfl_down_sync(0xffffffffu, v, 1);
            if (!right_ok) next = (unsigned)__ldg(reinterpret_cast<const unsigned short *>(row + xr));
            w[i] = wall ? v : __byte_perm(v, next, 0x5432);
        }
    }
}

// 16-bit storage, nx even: each thread updates the node pair x0 = 2t, x0 + 1.
// Every population of both nodes arrives as one aligned 32-bit load (kept
// packed until used), the +-1 shift of the pull along x is assembled from the
// neighbouring lane's word (or one 16-bit load at a row or warp edge), and
// both results leave as one 32-bit store.
template <int S, int FD, bool TH>
__global__ void __launch_bounds__(128, 7) k_lb_step_pair16(Lat L, typename Store<S>::T *b0, typename Store<S>::T *b1,
                                                        DevState *ds) {
    using T = typename Store<S>::T;
    using H = Half16<S>;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
    const int x0 = 2 * t;
    const bool active = x0 < L.nx && y < L.ny;
    const int xx = active ? x0 : 0, yy = active ? y : 0;
    const int step = ds->step;
    const T *src = (step & 1) ? b1 : b0;
    T *dst = (step & 1) ? b0 : b1;
    const int nx = L.nx, nxy = L.nx * L.ny;
    const int oym = yy == 0 ? nxy - nx : -nx, oyp = yy == L.ny - 1 ? nx - nxy : nx;
    const int ozm = z == 0 ? (L.nz - 1) * nxy : -nxy, ozp = z == L.nz - 1 ? (1 - L.nz) * nxy : nxy;
    const bool wlo = L.walls && z == 0, whi = L.walls && z == L.nz - 1;
    const int node = z * nxy + yy * nx + xx;
    // A warp covers consecutive pairs of one row; lanes at its edges (or next
    // to an inactive lane) load the shifted value themselves.
    const int left_active = __shfl_up_sync(0xffffffffu, (int)active, 1);
    const int right_active = __shfl_down_sync(0xffffffffu, (int)active, 1);
    const bool left_ok = lane > 0 && xx > 0 && left_active;
    const bool right_ok = lane < 31 && xx + 2 < nx && right_active;
    const int xl = xx == 0 ? nx - 1 : -1;      // offset of x0 - 1
    const int xr = xx + 2 == nx ? 2 - nx : 2;  // offset of x0 + 2
    unsigned w[Q];
    const ptrdiff_t plane = (ptrdiff_t)L.N;
    // Uniform branch: a block holds one z plane.
    if (wlo || whi)
        pull_pair<S, true>(src + node, plane, oym, oyp, ozm, ozp, wlo, whi, left_ok, right_ok, xl, xr, w);
    else
        pull_pair<S, false>(src + node, plane, oym, oyp, ozm, ozp, false, false, left_ok, right_ok, xl, xr, w);
    if (!active) return;
    // Both nodes share g (the pair kernel runs only when g is uniform along x);
    // their collisions run side by side in packed FP32x2 lanes.
    const float ga = body_amp(L, xx, yy, z);
    float2 fab[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fab[i] = H::unpack(w[i]);
    const float2 r = collide_g2<FD, Store<S>::kScaled>(L, fab, ga);
    if (!isfinite(r.x) || !isfinite(r.y)) atomicOr(&ds->flags, FLAG_NONFINITE);
    if (TH) {  // thermal noise of both nodes, in stored units
        const float sc = Store<S>::kScaled ? kF16Scale : 1.f;
        float xi[Q];
        node_noise(L, (unsigned)node, (unsigned)step, sc, xi);
#pragma unroll
        for (int i = 0; i < Q; ++i) fab[i].x += xi[i];
        node_noise(L, (unsigned)node + 1u, (unsigned)step, sc, xi);
#pragma unroll
        for (int i = 0; i < Q; ++i) fab[i].y += xi[i];
    }
    T *dp = dst + node;
#pragma unroll
    for (int i = 0; i < Q; ++i, dp += plane) __stcs(reinterpret_cast<unsigned *>(dp), H::pack(fab[i].x, fab[i].y));
}

// Nodes touched by atoms: redo the collision with F = g + G from the same
// pre-collision buffer, overwrite the dense kernel's result, clear G. The
// last block to finish advances the step counter and empties the list.
template <int S>
__global__ void __launch_bounds__(256) k_lb_fix(Lat L, typename Store<S>::T *b0, typename Store<S>::T *b1,
                                                const int *touched, int cap, float4 *G, DevState *ds, int keep) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int cnt = min(ds->n_touched, cap);
    const int step = ds->step;
    if (i < cnt) {
        const typename Store<S>::T *src = (step & 1) ? b1 : b0;
        typename Store<S>::T *dst = (step & 1) ? b0 : b1;
        const int node = touched[i];
        const int x = node % L.nx;
        const int y = (node / L.nx) % L.ny;
        const int z = node / (L.nx * L.ny);
        float f[Q], F[3];
        pull<S>(src, L, x, y, z, f);
        body_force(L, x, y, z, F);
        const float4 Gn = G[node];
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

dim3 node_block(const Lat &L) {
    int bx = ((L.nx + 31) / 32) * 32;
    if (bx > 256) bx = 256;
    int by = 256 / bx;
    if (by > L.ny) by = L.ny;
    return dim3(bx, by, 1);
}

dim3 node_grid(const Lat &L, dim3 b) { return dim3((L.nx + b.x - 1) / b.x, (L.ny + b.y - 1) / b.y, L.nz); }

}  // namespace

#define LBMD_DISPATCH(store, KERNEL_CALL)                                                                           \
    switch (store) {                                                                                                \
    case LBMD_F32: {                                                                                                \
        using T = float;                                                                                            \
        constexpr int SV = LBMD_F32;                                                                                \
        KERNEL_CALL;                                                                                                \
    } break;                                                                                                        \
    case LBMD_F16_SHIFTED: {                                                                                        \
        using T = __half;                                                                                           \
        constexpr int SV = LBMD_F16_SHIFTED;                                                                        \
        KERNEL_CALL;                                                                                                \
    } break;                                                                                                        \
    default: {                                                                                                      \
        using T = __nv_bfloat16;                                                                                    \
        constexpr int SV = LBMD_BF16_SHIFTED;                                                                       \
        KERNEL_CALL;                                                                                                \
    }                                                                                                               \
    }

// Runs BODY with FDV bound at compile time to the body-force direction
// (-1 without forcing) and THV to the thermal-noise switch.
#define LBMD_FD_DISPATCH1(L, BODY)                                         \
    switch ((L).forcing == LBMD_FORCE_NONE ? -1 : (L).fdir) {             \
        case -1: { constexpr int FDV = -1; BODY; } break;                  \
        case 0: { constexpr int FDV = 0; BODY; } break;                    \
        case 1: { constexpr int FDV = 1; BODY; } break;                    \
        default: { constexpr int FDV = 2; BODY; } break;                   \
    }
#define LBMD_FD_DISPATCH(L, BODY)                                          \
    if ((L).thermal) {                                                     \
        constexpr bool THV = true;                                         \
        LBMD_FD_DISPATCH1(L, BODY)                                         \
    } else {                                                               \
        constexpr bool THV = false;                                        \
        LBMD_FD_DISPATCH1(L, BODY)                                         \
    }

cudaError_t launch_lb_step(int store, const Lat &L, void *const buf[2], DevState *ds, cudaStream_t s) {
    const bool pairs = store != LBMD_F32 && L.nx % 2 == 0 &&
                       !(L.forcing == LBMD_FORCE_KOLMOGOROV && L.faxis == 0);
    if (pairs) {
        const int half = L.nx / 2;
        int bx = ((half + 31) / 32) * 32;
        if (bx > 128) bx = 128;
        int by = 128 / bx;
        if (by > L.ny) by = L.ny;
        const dim3 b(bx, by, 1), g((half + bx - 1) / bx, (L.ny + by - 1) / by, L.nz);
        if (store == LBMD_F16_SHIFTED) {
            LBMD_FD_DISPATCH(L, (k_lb_step_pair16<LBMD_F16_SHIFTED, FDV, THV>
                                 <<<g, b, 0, s>>>(L, (__half *)buf[0], (__half *)buf[1], ds)));
        } else {
            LBMD_FD_DISPATCH(L, (k_lb_step_pair16<LBMD_BF16_SHIFTED, FDV, THV>
                                 <<<g, b, 0, s>>>(L, (__nv_bfloat16 *)buf[0], (__nv_bfloat16 *)buf[1], ds)));
        }
        return cudaGetLastError();
    }
    const dim3 b = node_block(L), g = node_grid(L, b);
    LBMD_FD_DISPATCH(L, LBMD_DISPATCH(store, (k_lb_step<SV, FDV, THV><<<g, b, 0, s>>>(L, (T *)buf[0], (T *)buf[1], ds))));
    return cudaGetLastError();
}

cudaError_t launch_lb_fix(int store, const Lat &L, void *const buf[2], const CouplingArgs &c, int grid,
                          cudaStream_t s) {
    LBMD_DISPATCH(store, (k_lb_fix<SV><<<grid, 256, 0, s>>>(L, (T *)buf[0], (T *)buf[1], c.touched, c.touched_cap,
                                                             c.G, c.ds, c.keep)));
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
