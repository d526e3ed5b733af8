// The dense lattice update of every node: the fused pull-stream + BGK
// collide + Guo-force step (Eq. 1 with the standard minus sign, Sec. 2.2)
// with the body force g only; the nodes that also carry a coupling force are
// collided again by the fix-up kernel.
//
// Layout: 19 planes of N = nx*ny*nz values (SoA), population i of node n at
// i*N + n, stored as delta f = f - w_i rho0 in FP32, FP16 or BF16. Two
// buffers hold post-collision values; step s reads buffer s&1 and writes the
// other. FP32: one thread per node, threads along x within a warp, so each
// of the 19 loads and stores of a warp is one contiguous run (shifted by one
// element for speeds with c_x != 0). 16-bit formats: one thread per pair of
// nodes, one 32-bit word per population.
#include "lattice.cuh"

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
    // All 19 word loads first (and the edge lanes' 16-bit loads), so every
    // load of the thread is in flight before the first shuffle waits on one.
    const T *row[Q];
    unsigned v[Q], edge[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i, sp += plane) {
        const int oyz = (cy(i) == 1 ? oym : (cy(i) == -1 ? oyp : 0)) + (cz(i) == 1 ? ozm : (cz(i) == -1 ? ozp : 0));
        const bool wall = W && ((cz(i) == 1 && wlo) || (cz(i) == -1 && whi));
        row[i] = wall ? sp + (opp(i) - i) * plane : sp + oyz;
        v[i] = __ldg(reinterpret_cast<const unsigned *>(row[i]));
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        edge[i] = 0u;
        if (cx(i) == 1 && !left_ok) edge[i] = (unsigned)__ldg(reinterpret_cast<const unsigned short *>(row[i] + xl)) << 16;
        if (cx(i) == -1 && !right_ok) edge[i] = (unsigned)__ldg(reinterpret_cast<const unsigned short *>(row[i] + xr));
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const bool wall = W && ((cz(i) == 1 && wlo) || (cz(i) == -1 && whi));
        if (cx(i) == 0) {
            w[i] = v[i];
        } else if (cx(i) == 1) {  // x0 pulls x0 - 1 (high half of the left word), x0 + 1 pulls x0
            unsigned prev = __shfl_up_sync(0xffffffffu, v[i], 1);
            if (!left_ok) prev = edge[i];
            w[i] = wall ? v[i] : __byte_perm(prev, v[i], 0x5432);
        } else {  // x0 pulls x0 + 1, x0 + 1 pulls x0 + 2 (low half of the right word)
            unsigned next = __shfl_down_sync(0xffffffffu, v[i], 1);
            if (!right_ok) next = edge[i];
            w[i] = wall ? v[i] : __byte_perm(v[i], next, 0x5432);
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

}  // namespace

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

}  // namespace lbmd
