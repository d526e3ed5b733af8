// Discrete adjoint of the coupled step (not in the paper: it differentiates
// the method of Sec. 2.2 as implemented here). One coupled step maps
// (h^n, x^n, v^n) -> (h^{n+1}, x^{n+1}, v^{n+1}) through
//   f = pull(h^n);  u_b = (sum f c + g/2)/rho;  U_a = sum_j W_aj(x^n) u_b(j)
//   n_md velocity-Verlet substeps (forces F(x), drag gamma (U - v)) -> J_a
//   G_j = -sum_a W_aj J_a;  h^{n+1} = collide(f, g + G; omega)
// and the reverse kernels below apply the transpose of its Jacobian, in
// reverse order, to the adjoint state (hat h, hat x, hat v), accumulating
// d/d gamma, d/d omega and d/d A (the body-force amplitude).
//
// Reverse order per step: collision adjoint at the touched nodes (hat F),
// spread adjoint (hat J), reverse substeps n_md..0 (local kick/drift part,
// then the Hessian-vector product of the conservative forces), interpolation
// adjoint (hat u_b on the touched nodes), dense collide-stream adjoint at
// every node with F = g (push = transpose of pull), and the touched-node
// fix-up with F = g + G plus the interpolation's share.
#include "lbmd_internal.cuh"

namespace lbmd {

namespace {

// Body-force shape g/A at a node.
__device__ __forceinline__ void force_shape(const Lat &L, int x, int y, int z, float s[3]) {
    Lat Ls = L;
    Ls.famp = 1.f;
    body_force(Ls, x, y, z, s);
}

// Transpose of the collision Jacobian at one node. f: pulled deviations;
// F: total force; oh: adjoint of the 19 outputs. Gives the adjoint of the
// pulled inputs (fhat), of the force (Fhat) and of omega (returned).
__device__ float collide_adjoint(const Lat &L, const float f[Q], const float F[3], const float oh[Q],
                                 float fhat[Q], float Fhat[3]) {
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += f[i];
        jx += cx(i) * f[i];
        jy += cy(i) * f[i];
        jz += cz(i) * f[i];
    }
    const float rho = L.rho0 + drho;
    const float inv = 1.f / rho;
    const float u[3] = {(jx + 0.5f * F[0]) * inv, (jy + 0.5f * F[1]) * inv, (jz + 0.5f * F[2]) * inv};
    const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    const float om = L.omega, src = 1.f - 0.5f * om;
    float a = 0.f, b[3] = {0.f, 0.f, 0.f}, e[3] = {0.f, 0.f, 0.f}, omh = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float c[3] = {(float)cx(i), (float)cy(i), (float)cz(i)};
        const float cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        const float cF = c[0] * F[0] + c[1] * F[1] + c[2] * F[2];
        const float w = wgt(i);
        const float poly = 3.f * cu + 4.5f * cu * cu - 1.5f * usq;
        const float dfeq = w * (drho + rho * poly);  // f_eq - w rho0
        const float S = w * (3.f * (cF - uF) + 9.f * cu * cF);
        a += oh[i] * om * w * (1.f + poly);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            b[d] += oh[i] * (om * w * rho * (3.f * c[d] + 9.f * cu * c[d] - 3.f * u[d]) +
                             src * w * (-3.f * F[d] + 9.f * cF * c[d]));
            e[d] += oh[i] * src * w * (3.f * (c[d] - u[d]) + 9.f * cu * c[d]);
        }
        omh += oh[i] * (-(f[i] - dfeq) - 0.5f * S);
    }
#pragma unroll
    for (int k = 0; k < Q; ++k)
        fhat[k] = (1.f - om) * oh[k] + a + (b[0] * (cx(k) - u[0]) + b[1] * (cy(k) - u[1]) + b[2] * (cz(k) - u[2])) * inv;
    for (int d = 0; d < 3; ++d) Fhat[d] = e[d] + 0.5f * b[d] * inv;
    return omh;
}

__device__ __forceinline__ void load_hat(const AdjArgs &D, size_t node, float oh[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) oh[i] = D.hat_in[(size_t)i * D.L.N + node];
}

__device__ __forceinline__ void node_xyz(const Lat &L, int node, int &x, int &y, int &z) {
    x = node % L.nx;
    y = (node / L.nx) % L.ny;
    z = node / (L.nx * L.ny);
}

// K1: hat F at the touched nodes (collision with F = g + G).
template <int S>
__global__ void k_adj_force_hat(AdjArgs D, CouplingArgs C, const typename Store<S>::T *h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min(C.ds->n_touched, C.touched_cap)) return;
    const int node = C.touched[i];
    int x, y, z;
    node_xyz(D.L, node, x, y, z);
    float f[Q], F[3], oh[Q], fh[Q], Fh[3];
    pull<S>(h, D.L, x, y, z, f);
    body_force(D.L, x, y, z, F);
    const float4 G = C.G[node];
    F[0] += G.x;
    F[1] += G.y;
    F[2] += G.z;
    load_hat(D, node, oh);
    collide_adjoint(D.L, f, F, oh, fh, Fh);
    D.Ghat[node] = make_float4(Fh[0], Fh[1], Fh[2], 0.f);
}

__device__ __forceinline__ void corner(const Lat &L, const int b[3], const float t[3], int k, size_t &node, float &W,
                                       float dW[3]) {
    const int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
    const int nx = o[0] ? (b[0] + 1 == L.nx ? 0 : b[0] + 1) : b[0];
    const int ny = o[1] ? (b[1] + 1 == L.ny ? 0 : b[1] + 1) : b[1];
    const int nz = o[2] ? (b[2] + 1 == L.nz ? 0 : b[2] + 1) : b[2];
    const float w0 = o[0] ? t[0] : 1.f - t[0], w1 = o[1] ? t[1] : 1.f - t[1], w2 = o[2] ? t[2] : 1.f - t[2];
    W = w0 * w1 * w2;
    dW[0] = (o[0] ? 1.f : -1.f) * w1 * w2;
    dW[1] = (o[1] ? 1.f : -1.f) * w0 * w2;
    dW[2] = (o[2] ? 1.f : -1.f) * w0 * w1;
    node = ((size_t)nz * L.ny + ny) * L.nx + nx;
}

// K2: spread adjoint. G_j = -sum_a W_aj J_a gives hat J_a = -sum_j W_aj hat G_j
// (plus the observable's d/dJ) and a weight-gradient term for hat x_a.
__global__ void k_adj_spread(AdjArgs D, CouplingArgs C) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= D.na) return;
    const int na = D.na;
    int b[3];
    float t[3], J[3], Jh[3] = {0.f, 0.f, 0.f}, xw[3] = {0.f, 0.f, 0.f};
    for (int d = 0; d < 3; ++d) {
        b[d] = C.base[d * na + a];
        t[d] = C.frac[d * na + a];
        J[d] = C.J[d * na + a];
    }
    for (int k = 0; k < 8; ++k) {
        size_t node;
        float W, dW[3];
        corner(D.L, b, t, k, node, W, dW);
        const float4 g = D.Ghat[node];
        Jh[0] -= W * g.x;
        Jh[1] -= W * g.y;
        Jh[2] -= W * g.z;
        const float jg = J[0] * g.x + J[1] * g.y + J[2] * g.z;
        for (int d = 0; d < 3; ++d) xw[d] -= dW[d] * jg;
    }
    if (D.observable == LBMD_OBS_DRAG_X) Jh[0] += D.obs_w;
    for (int d = 0; d < 3; ++d) {
        D.Jhat[d * na + a] = Jh[d];
        D.xw[d * na + a] = xw[d];
        D.Uat_hat[d * na + a] = 0.f;
    }
}

// K3: reverse of the kick/drift part of substep kernel k for one atom.
// vhat enters as hat v_{k+1/2} (hat v_{n_md} for k = n_md) and leaves as
// hat v_{k-1/2} (hat v_0 for k = 0); xhat holds hat x_{k+1} on entry (drift
// reverse); p receives the adjoint force weight (h/m)(sum of the kick
// adjoints at x_k) for the Hessian-vector product of K4.
__global__ void k_adj_md_local(AdjArgs D, AtomArgs A, CouplingArgs C, int k) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= D.na) return;
    const int na = D.na;
    const float h = A.hdt, g = A.gamma, im = A.inv_m[a];
    const size_t rk = (size_t)k * 3 * na;
    double gam = 0.0;
    for (int d = 0; d < 3; ++d) {
        const size_t q = (size_t)d * na + a;
        const float U = C.U[q], Jh = D.Jhat[q];
        const float vin = A.recV[rk + q], Fk = A.recF[rk + q];
        const float vk = k == 0 ? vin : vin + h * im * (Fk + g * (U - vin));
        float vh = D.vhat[q], p = 0.f, Uh = D.Uat_hat[q];
        if (k < A.n_md) {
            vh += A.dt * D.xhat[q];  // x_{k+1} = x_k + dt v_{k+1/2}
            p += h * im * vh;
            Uh += h * g * im * vh + h * g * Jh;
            gam += (double)(h * im * (U - vk) * vh + h * (U - vk) * Jh);
            vh = vh * (1.f - h * g * im) - h * g * Jh;  // now hat v_k
        }
        if (k > 0) {
            p += h * im * vh;
            Uh += h * g * im * vh + h * g * Jh;
            gam += (double)(h * im * (U - vin) * vh + h * (U - vin) * Jh);
            vh = vh * (1.f - h * g * im) - h * g * Jh;  // now hat v_{k-1/2}
        }
        D.vhat[q] = vh;
        D.p[q] = p;
        D.Uat_hat[q] = Uh;
    }
    D.gam_acc[a] += gam;
}

// Adjoint buckets for positions x_k (from the records).
__global__ void k_adj_bins(AtomArgs A, int k) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.na) return;
    const float4 pa = A.recP[(size_t)k * A.na + a], la = A.recL[(size_t)k * A.na + a];
    const float v[3] = {(pa.x - A.off[0]) + la.x, (pa.y - A.off[1]) + la.y, (pa.z - A.off[2]) + la.z};
    int c[3];
    for (int d = 0; d < 3; ++d) {
        int cc = (int)floorf(v[d] * A.inv_h[d]) % A.nc[d];
        c[d] = cc < 0 ? cc + A.nc[d] : cc;
    }
    const int b = ((c[2] & A.fmask[2]) * A.fold[1] + (c[1] & A.fmask[1])) * A.fold[0] + (c[0] & A.fmask[0]);
    const int s = atomicAdd(&A.count[0][b], 1);
    if (s < A.cap)
        A.slot[0][(size_t)b * A.cap + s] = a;
    else
        atomicOr(&A.ds->flags, FLAG_CELL);
}

// x_a - x_b at the recorded positions: in the step frame the hi difference
// and the fold by whole box lengths are exact, the lo parts add below FP32
// resolution.
__device__ __forceinline__ void rec_disp(const AtomArgs &A, float4 pa, float4 la, float4 pb, float4 lb, float d[3]) {
    const float ha[3] = {pa.x, pa.y, pa.z}, hb[3] = {pb.x, pb.y, pb.z};
    const float la3[3] = {la.x, la.y, la.z}, lb3[3] = {lb.x, lb.y, lb.z};
    for (int k = 0; k < 3; ++k) {
        const float s = ha[k] - hb[k];
        d[k] = fmaf(-A.Lf[k], rintf(s * A.inv_Lf[k]), s) + (la3[k] - lb3[k]);
    }
}

__device__ __forceinline__ bool is_bonded(const AtomArgs &A, int a, int b) {
    for (int s = A.bstart[a]; s < A.bstart[a + 1]; ++s)
        if (A.bpart[s] == b) return true;
    return false;
}

// K(p_a - p_b) for a pair force f = phi(r) d: phi (p_a - p_b) + (phi'/r) d (d.(p_a - p_b)).
__device__ __forceinline__ void hvp_add(float phi, float dphi_r, const float d[3], const float dp[3], float out[3]) {
    const float dd = d[0] * dp[0] + d[1] * dp[1] + d[2] * dp[2];
    for (int k = 0; k < 3; ++k) out[k] += phi * dp[k] + dphi_r * d[k] * dd;
}

// K4: hat x_a += sum_b K_ab(x_k) (p_a - p_b), LJ pairs within rc (27 cells of
// the adjoint buckets) and bonds. One warp per atom: the candidates of the
// neighbour cells within reach of rc are numbered by a warp prefix sum over
// the cell counts and dealt to the lanes; bonded partners (the first 32) sit
// one per lane and are matched with shuffles; the lanes' terms are summed
// across the warp.
__global__ void __launch_bounds__(128) k_adj_hvp(AdjArgs D, AtomArgs A, int k) {
    const int lane = threadIdx.x & 31;
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (a >= D.na) return;  // whole warp
    const int na = D.na;
    const float4 *P = A.recP + (size_t)k * na, *Lr = A.recL + (size_t)k * na;
    const float4 pa = P[a], la = Lr[a];
    const float pA[3] = {D.p[a], D.p[na + a], D.p[2 * na + a]};
    const int b0 = A.bstart[a], b1 = A.bstart[a + 1];
    const int nbond = b1 - b0;
    const int partner = lane < nbond ? A.bpart[b0 + lane] : -1;
    const float pp[3] = {(pa.x - A.off[0]) + la.x, (pa.y - A.off[1]) + la.y, (pa.z - A.off[2]) + la.z};
    int cc[3];
    float t[3];  // position within the current cell
    for (int d = 0; d < 3; ++d) {
        const float fl = floorf(pp[d] * A.inv_h[d]);
        t[d] = pp[d] - fl * A.h[d];
        int c = (int)fl % A.nc[d];
        cc[d] = c < 0 ? c + A.nc[d] : c;
    }
    int bucket = 0, n = 0;
    if (lane < 27) {
        const int o[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
        float gap2 = 0.f;  // squared distance to the neighbour cell (conservative margin below)
        for (int d = 0; d < 3; ++d) {
            const float g = o[d] < 0 ? t[d] : (o[d] > 0 ? A.h[d] - t[d] : 0.f);
            gap2 += g * g;
        }
        if (gap2 < A.rc2f * 1.001f) {
            int c[3];
            for (int d = 0; d < 3; ++d) {
                const int v = (cc[d] + o[d]) % A.nc[d];
                c[d] = v < 0 ? v + A.nc[d] : v;
            }
            bucket = ((c[2] & A.fmask[2]) * A.fold[1] + (c[1] & A.fmask[1])) * A.fold[0] + (c[0] & A.fmask[0]);
            n = min(A.count[0][bucket], A.cap);
        }
    }
    int incl = n;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    float out[3] = {0.f, 0.f, 0.f};
    const float s6 = A.lj_sig2 * A.lj_sig2 * A.lj_sig2;
    for (int t0 = lane; t0 - lane < total; t0 += 32) {
        int pos = 0;  // cell holding candidate t0: first lane whose inclusive sum exceeds it
        for (int step = 16; step > 0; step >>= 1) {
            const int probe = __shfl_sync(0xffffffffu, incl, pos + step - 1);
            if (probe <= t0) pos += step;
        }
        const int cb = __shfl_sync(0xffffffffu, bucket, pos & 31);
        const int before = __shfl_sync(0xffffffffu, incl - n, pos & 31);
        const int q = t0 < total ? A.slot[0][(size_t)cb * A.cap + (t0 - before)] : a;
        bool use = false;
        float d[3] = {0.f, 0.f, 0.f};
        float r2 = 1.f;
        if (q != a) {
            rec_disp(A, pa, la, P[q], Lr[q], d);
            r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            use = r2 < A.rc2f;
        }
        bool bonded_q = false;
        for (int l = 0; l < min(nbond, 32); ++l) bonded_q |= __shfl_sync(0xffffffffu, partner, l) == q;
        if (use && nbond > 32 && !bonded_q) bonded_q = is_bonded(A, a, q);
        if (use && !bonded_q) {
            const float r = sqrtf(r2);
            const float ir2 = 1.f / r2;
            const float ir6 = ir2 * ir2 * ir2, ir8 = ir6 * ir2;
            // phi = 24 eps s6 (2 s6 r^-14 - r^-8) - fc / r
            const float phi = A.lj_24eps * s6 * ir8 * (2.f * s6 * ir6 - 1.f) - A.lj_fc / r;
            // phi'/r = 24 eps s6 (-28 s6 r^-16 + 8 r^-10) + fc r^-3
            const float dphi_r = A.lj_24eps * s6 * ir8 * ir2 * (-28.f * s6 * ir6 + 8.f) + A.lj_fc * ir2 / r;
            float ph = phi, dph = dphi_r;
            if (A.coul && r2 < A.coul_rc2) {
                // phi_q = 2 C q_a q_b (r^-4 - rcc^-3 r^-1), phi_q'/r = 2 C q_a q_b (-4 r^-6 + rcc^-3 r^-3)
                const float c2 = A.coul_2c * pa.w * P[q].w;
                ph += c2 * (ir2 * ir2 - A.coul_irc3 / r);
                dph += c2 * (-4.f * ir6 + A.coul_irc3 * ir2 / r);
            }
            const float dp[3] = {pA[0] - D.p[q], pA[1] - D.p[na + q], pA[2] - D.p[2 * na + q]};
            hvp_add(ph, dph, d, dp, out);
        }
    }
    for (int s = b0 + lane; s < b1; s += 32) {
        const int q = A.bpart[s];
        float d[3];
        rec_disp(A, pa, la, P[q], Lr[q], d);
        const float r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        // f = -k (1 - r0/r) d: phi = -k (1 - r0/r), phi'/r = -k r0 / r^3
        const float phi = -A.bk[s] * (1.f - A.br0[s] / r);
        const float dphi_r = -A.bk[s] * A.br0[s] / (r * r * r);
        const float dp[3] = {pA[0] - D.p[q], pA[1] - D.p[na + q], pA[2] - D.p[2 * na + q]};
        hvp_add(phi, dphi_r, d, dp, out);
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int d = 0; d < 3; ++d) out[d] += __shfl_xor_sync(0xffffffffu, out[d], o);
    if (lane == 0)
        for (int d = 0; d < 3; ++d) D.xhat[d * na + a] += out[d];
}

// K5: interpolation adjoint. U_a = sum_j W_aj u_b(j): hat u_b(j) += W_aj hat U_a
// (accumulated per node), hat x_a += sum_j grad W_aj (u_b(j) . hat U_a).
template <int S>
__global__ void k_adj_interp(AdjArgs D, CouplingArgs C, const typename Store<S>::T *h) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= D.na) return;
    const int na = D.na;
    int b[3];
    float t[3], Uh[3], xw[3];
    for (int d = 0; d < 3; ++d) {
        b[d] = C.base[d * na + a];
        t[d] = C.frac[d * na + a];
        Uh[d] = D.Uat_hat[d * na + a];
        xw[d] = D.xw[d * na + a];
    }
    for (int k = 0; k < 8; ++k) {
        size_t node;
        float W, dW[3];
        corner(D.L, b, t, k, node, W, dW);
        int x, y, z;
        node_xyz(D.L, (int)node, x, y, z);
        float f[Q], g[3], u[3];
        pull<S>(h, D.L, x, y, z, f);
        body_force(D.L, x, y, z, g);
        node_velocity(D.L, f, g, u);
        const float uU = u[0] * Uh[0] + u[1] * Uh[1] + u[2] * Uh[2];
        for (int d = 0; d < 3; ++d) xw[d] += dW[d] * uU;
        atomicAdd(&D.Uhat[node], make_float4(W * Uh[0], W * Uh[1], W * Uh[2], 0.f));
    }
    for (int d = 0; d < 3; ++d) D.xhat[d * na + a] += xw[d];
}

// Block reduction of two FP64 values into partials[2 * block + {0, 1}].
__device__ void block_sum2(double v0, double v1, double *partials) {
    __shared__ double sh[2][32];
    // Linear thread index: the lattice kernels use two-dimensional blocks.
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, o);
        v1 += __shfl_down_sync(0xffffffffu, v1, o);
    }
    if (lane == 0) {
        sh[0][warp] = v0;
        sh[1][warp] = v1;
    }
    __syncthreads();
    if (t < 2) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x * blockDim.y / 32); ++w) s += sh[t][w];
        const int nb = gridDim.x * gridDim.y * gridDim.z;
        const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[(size_t)t * nb + bid] += s;
    }
}

// K6: dense collide-stream adjoint with F = g at every node: the pulled
// inputs' adjoint goes back to the storage entries they were pulled from
// (push = transpose of pull, bounce-back included). Accumulates hat omega and
// hat A (F = g = A shape) into per-block FP64 partials.
template <int S>
__global__ void __launch_bounds__(256) k_adj_lb(AdjArgs D, const typename Store<S>::T *h) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    double om_acc = 0.0, a_acc = 0.0;
    if (x < D.L.nx && y < D.L.ny) {
        const Lat &L = D.L;
        const size_t node = ((size_t)z * L.ny + y) * L.nx + x;
        float f[Q], F[3], sh3[3], oh[Q], fh[Q], Fh[3];
        pull<S>(h, L, x, y, z, f);
        body_force(L, x, y, z, F);
        force_shape(L, x, y, z, sh3);
        load_hat(D, node, oh);
        om_acc = collide_adjoint(L, f, F, oh, fh, Fh);
        a_acc = Fh[0] * sh3[0] + Fh[1] * sh3[1] + Fh[2] * sh3[2];
        const int xm = x == 0 ? L.nx - 1 : x - 1, xp = x == L.nx - 1 ? 0 : x + 1;
        const int ym = y == 0 ? L.ny - 1 : y - 1, yp = y == L.ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? L.nz - 1 : z - 1, zp = z == L.nz - 1 ? 0 : z + 1;
#pragma unroll
        for (int i = 0; i < Q; ++i) D.hat_out[pull_index(L, i, x, y, z, xm, xp, ym, yp, zm, zp, node)] = fh[i];
    }
    block_sum2(om_acc, a_acc, D.partials);
}

// K7: touched nodes. Redo the adjoint with F = g + G, add the interpolation's
// share (u_b = (sum f c + g/2)/rho), overwrite the dense kernel's pushed
// values, correct the hat omega / hat A sums, and clear the node buffers.
template <int S>
__global__ void k_adj_fix(AdjArgs D, CouplingArgs C, const typename Store<S>::T *h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min(C.ds->n_touched, C.touched_cap)) return;
    const Lat &L = D.L;
    const int node = C.touched[i];
    int x, y, z;
    node_xyz(L, node, x, y, z);
    float f[Q], g[3], F[3], sh3[3], oh[Q], fh_d[Q], Fh_d[3], fh[Q], Fh[3];
    pull<S>(h, L, x, y, z, f);
    body_force(L, x, y, z, g);
    force_shape(L, x, y, z, sh3);
    load_hat(D, node, oh);
    const float om_d = collide_adjoint(L, f, g, oh, fh_d, Fh_d);
    const float4 G = C.G[node];
    F[0] = g[0] + G.x;
    F[1] = g[1] + G.y;
    F[2] = g[2] + G.z;
    const float om_c = collide_adjoint(L, f, F, oh, fh, Fh);
    // Interpolation share: u_b = (j + g/2)/rho.
    const float4 uh = D.Uhat[node];
    float u[3];
    const float rho = node_velocity(L, f, g, u);
    const float irho = 1.f / rho;
    const float ubu = u[0] * uh.x + u[1] * uh.y + u[2] * uh.z;
    for (int k = 0; k < Q; ++k) fh[k] += (cx(k) * uh.x + cy(k) * uh.y + cz(k) * uh.z - ubu) * irho;
    const float dA = (Fh[0] - Fh_d[0]) * sh3[0] + (Fh[1] - Fh_d[1]) * sh3[1] + (Fh[2] - Fh_d[2]) * sh3[2] +
                     0.5f * irho * (sh3[0] * uh.x + sh3[1] * uh.y + sh3[2] * uh.z);
    atomicAdd(&D.par_acc[0], (double)(om_c - om_d));
    atomicAdd(&D.par_acc[1], (double)dA);
    const int xm = x == 0 ? L.nx - 1 : x - 1, xp = x == L.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? L.ny - 1 : y - 1, yp = y == L.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? L.nz - 1 : z - 1, zp = z == L.nz - 1 ? 0 : z + 1;
    for (int q = 0; q < Q; ++q) D.hat_out[pull_index(L, q, x, y, z, xm, xp, ym, yp, zm, zp, (size_t)node)] = fh[q];
    D.Ghat[node] = make_float4(0.f, 0.f, 0.f, 0.f);
    D.Uhat[node] = make_float4(0.f, 0.f, 0.f, 0.f);
    C.G[node] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Observable pieces. DRAG_X: sum_a J_a,x of the step just taken. RG2: mass
// weighted R_g^2 of the positions X, and (for the reverse) its gradient
// w (2 m_a (x_a - x_cm) / M) added to hat x.
__global__ void k_obs_sum(const float *J, const double *X, const float *mass, int na, int observable, double *out) {
    __shared__ double sh[4][32];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int a = threadIdx.x; a < na; a += blockDim.x) {
        if (observable == LBMD_OBS_DRAG_X) {
            s[0] += (double)J[a];
        } else {
            const double m = mass[a];
            s[0] += m;
            for (int d = 0; d < 3; ++d) s[1 + d] += m * X[d * na + a];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 4; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < (int)(blockDim.x / 32); ++w)
            for (int k = 0; k < 4; ++k) t[k] += sh[k][w];
        if (observable == LBMD_OBS_DRAG_X) {
            out[0] += t[0];
        } else {
            out[1] = t[0];
            out[2] = t[1] / t[0];
            out[3] = t[2] / t[0];
            out[4] = t[3] / t[0];
        }
    }
}

__global__ void k_rg2_sum(const double *X, const float *mass, int na, double *out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int a = threadIdx.x; a < na; a += blockDim.x)
        for (int d = 0; d < 3; ++d) {
            const double e = X[d * na + a] - out[2 + d];
            s += mass[a] * e * e;
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += sh[w];
        out[0] += t / out[1];
    }
}

__global__ void k_rg2_grad(const double *X, const float *mass, int na, const double *cm, float w, float *xhat) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= na) return;
    for (int d = 0; d < 3; ++d)
        xhat[d * na + a] += (float)(w * 2.0 * mass[a] * (X[d * na + a] - cm[2 + d]) / cm[1]);
}

__global__ void k_sum_double(const double *v, int n, double *out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += sh[w];
        *out = t;
    }
}

dim3 adj_block(const Lat &L) {
    int bx = ((L.nx + 31) / 32) * 32;
    if (bx > 256) bx = 256;
    int by = 256 / bx;
    if (by > L.ny) by = L.ny;
    return dim3(bx, by, 1);
}

}  // namespace

#define ADJ_DISPATCH(store, CALL)                                                                                   \
    switch (store) {                                                                                                \
    case LBMD_F32: {                                                                                                \
        using T = float;                                                                                            \
        constexpr int SV = LBMD_F32;                                                                                \
        CALL;                                                                                                       \
    } break;                                                                                                        \
    case LBMD_F16_SHIFTED: {                                                                                        \
        using T = __half;                                                                                           \
        constexpr int SV = LBMD_F16_SHIFTED;                                                                        \
        CALL;                                                                                                       \
    } break;                                                                                                        \
    default: {                                                                                                      \
        using T = __nv_bfloat16;                                                                                    \
        constexpr int SV = LBMD_BF16_SHIFTED;                                                                       \
        CALL;                                                                                                       \
    }                                                                                                               \
    }

int adj_lb_blocks(const Lat &L) {
    const dim3 b = adj_block(L);
    return (int)(((L.nx + b.x - 1) / b.x) * ((L.ny + b.y - 1) / b.y) * L.nz);
}

cudaError_t launch_adjoint_step(int store, const AdjArgs &D, const AtomArgs &A, AtomArgs &Aadj,
                                const CouplingArgs &C, const void *h, cudaStream_t s) {
    const int na = D.na;
    const int ga = (na + 127) / 128, gt = (C.touched_cap + 255) / 256;
    if (na > 0) {
        ADJ_DISPATCH(store, (k_adj_force_hat<SV><<<gt, 256, 0, s>>>(D, C, (const T *)h)));
        k_adj_spread<<<ga, 128, 0, s>>>(D, C);
        const size_t B = (size_t)A.fold[0] * A.fold[1] * A.fold[2];
        for (int k = A.n_md; k >= 0; --k) {
            k_adj_md_local<<<ga, 128, 0, s>>>(D, A, C, k);
            cudaError_t e = cudaMemsetAsync(Aadj.count[0], 0, B * sizeof(int), s);
            if (e != cudaSuccess) return e;
            k_adj_bins<<<ga, 128, 0, s>>>(Aadj, k);
            k_adj_hvp<<<(na + 3) / 4, 128, 0, s>>>(D, Aadj, k);  // a warp per atom
        }
        ADJ_DISPATCH(store, (k_adj_interp<SV><<<ga, 128, 0, s>>>(D, C, (const T *)h)));
    }
    const dim3 b = adj_block(D.L);
    const dim3 g((D.L.nx + b.x - 1) / b.x, (D.L.ny + b.y - 1) / b.y, D.L.nz);
    ADJ_DISPATCH(store, (k_adj_lb<SV><<<g, b, 0, s>>>(D, (const T *)h)));
    if (na > 0) ADJ_DISPATCH(store, (k_adj_fix<SV><<<gt, 256, 0, s>>>(D, C, (const T *)h)));
    return cudaGetLastError();
}

cudaError_t launch_obs_accumulate(const AtomArgs &A, const CouplingArgs &C, int observable, double *out,
                                  cudaStream_t s) {
    if (A.na == 0) return cudaSuccess;
    k_obs_sum<<<1, 256, 0, s>>>(C.J, A.X, A.mass, A.na, observable, out);
    if (observable == LBMD_OBS_RG2) k_rg2_sum<<<1, 256, 0, s>>>(A.X, A.mass, A.na, out);
    return cudaGetLastError();
}

cudaError_t launch_rg2_grad(const AtomArgs &A, double *scratch, float w, float *xhat, cudaStream_t s) {
    if (A.na == 0) return cudaSuccess;
    k_obs_sum<<<1, 256, 0, s>>>(nullptr, A.X, A.mass, A.na, LBMD_OBS_RG2, scratch);
    k_rg2_grad<<<(A.na + 127) / 128, 128, 0, s>>>(A.X, A.mass, A.na, scratch, w, xhat);
    return cudaGetLastError();
}

cudaError_t launch_sum_double(const double *v, int n, double *out, cudaStream_t s) {
    k_sum_double<<<1, 256, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

}  // namespace lbmd
