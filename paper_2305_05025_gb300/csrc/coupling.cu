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

// Nodes of a block's lattice tile (the box spanned by the eight-node stencils
// of its 128 warp-sorted atoms) staged in shared memory; blocks whose atoms
// span a larger box (atoms far apart in the sort, or across a periodic seam)
// take every corner straight from global memory.
constexpr int kTileMax = 1024;

// Start of a coupled step, one thread per atom, atoms in warp-sorted order:
// set the atom's FP32 step frame for the substeps, build its trilinear stencil
// from the FP64 position, interpolate u = (sum f c + g/2)/rho over the eight
// corners (pulled from the current post-collision buffer), and claim the
// corners in the touched-node list (each node enters once per step).
//
// The block first bounds its atoms' stencils. When the box holds at most
// kTileMax nodes, u is computed once per box node into shared memory (19
// pulled loads per node instead of per corner of every atom: neighbouring
// atoms share corners), the atoms interpolate from there, and the corners
// used are claimed once per block. The sums are the same operations in the
// same order as the direct path, so both give identical U.
template <int S>
__global__ void __launch_bounds__(128) k_interp(CouplingArgs C, AtomArgs A, const typename Store<S>::T *b0,
                                                const typename Store<S>::T *b1) {
    __shared__ float4 s_u[kTileMax];
    __shared__ unsigned char s_used[kTileMax];
    __shared__ int s_box[4][6];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < C.na;
    const int a = valid ? C.order[i] : 0;
    const int na = C.na;
    const int step = C.ds->step;
    const typename Store<S>::T *src = (step & 1) ? b1 : b0;
    const int par = (int)(((long long)step * A.n_md) & 1);
    const Lat &L = C.L;
    const int n[3] = {L.nx, L.ny, L.nz};

    int b[3] = {0, 0, 0};
    float t[3] = {0.f, 0.f, 0.f};
    if (valid) {
        float4 fp, fl4;
        const bool finite = set_frame(A, a, fp, fl4);
        A.P[par][a] = fp;
        A.L[par][a] = fl4;
        if (!finite) atomicOr(&C.ds->flags, FLAG_NONFINITE);
        const double x[3] = {C.X[a], C.X[na + a], C.X[2 * na + a]};
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
    }
    // Box of the block's stencils: lowest base and highest base + 1 per axis
    // (unwrapped: base + 1 may equal n, the node at 0).
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = __reduce_min_sync(0xffffffffu, valid ? b[d] : 0x7fffffff);
        hi[d] = __reduce_max_sync(0xffffffffu, valid ? b[d] + 1 : -1);
    }
    if (lane == 0)
        for (int d = 0; d < 3; ++d) {
            s_box[warp][d] = lo[d];
            s_box[warp][3 + d] = hi[d];
        }
    __syncthreads();
    int ext[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = min(min(s_box[0][d], s_box[1][d]), min(s_box[2][d], s_box[3][d]));
        hi[d] = max(max(s_box[0][3 + d], s_box[1][3 + d]), max(s_box[2][3 + d], s_box[3][3 + d]));
        if (C.reinterp) {  // one node of margin: where the atoms' stencils move in a typical step
            lo[d] -= 1;
            hi[d] += 1;
            if (d == 2 && L.walls) {
                lo[d] = max(lo[d], 0);
                hi[d] = min(hi[d], L.nz - 1);
            }
        }
        ext[d] = hi[d] - lo[d] + 1;
    }
    const int tile = ext[0] * ext[1] * ext[2];  // > 0: every block holds at least one valid atom
    const int stamp = step + 1;
    float U[3] = {0.f, 0.f, 0.f};
    if (tile <= kTileMax) {
        for (int k = threadIdx.x; k < tile; k += blockDim.x) {
            const int ox = k % ext[0], oy = (k / ext[0]) % ext[1], oz = k / (ext[0] * ext[1]);
            int xx = lo[0] + ox, yy = lo[1] + oy, zz = lo[2] + oz;
            xx += xx < 0 ? L.nx : (xx >= L.nx ? -L.nx : 0);
            yy += yy < 0 ? L.ny : (yy >= L.ny ? -L.ny : 0);
            zz += zz < 0 ? L.nz : (zz >= L.nz ? -L.nz : 0);
            float f[Q], g[3], u[3];
            pull<S>(src, L, xx, yy, zz, f);
            body_force(L, xx, yy, zz, g);
            node_velocity(L, f, g, u);
            s_u[k] = make_float4(u[0], u[1], u[2], 0.f);
            s_used[k] = C.reinterp ? 1 : 0;  // re-interpolation claims the whole region
            if (C.reinterp)
                C.unode[((size_t)zz * L.ny + yy) * L.nx + xx] = make_float4(u[0], u[1], u[2], __int_as_float(stamp));
        }
        __syncthreads();
        if (valid) {
#pragma unroll 1
            for (int k = 0; k < 8; ++k) {
                const int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
                const float W = (o[0] ? t[0] : 1.f - t[0]) * (o[1] ? t[1] : 1.f - t[1]) * (o[2] ? t[2] : 1.f - t[2]);
                const int idx = ((b[2] + o[2] - lo[2]) * ext[1] + (b[1] + o[1] - lo[1])) * ext[0] + (b[0] + o[0] - lo[0]);
                const float4 u = s_u[idx];
                U[0] += W * u.x;
                U[1] += W * u.y;
                U[2] += W * u.z;
                s_used[idx] = 1;
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < tile; k += blockDim.x) {
            if (!s_used[k]) continue;
            const int ox = k % ext[0], oy = (k / ext[0]) % ext[1], oz = k / (ext[0] * ext[1]);
            int xx = lo[0] + ox, yy = lo[1] + oy, zz = lo[2] + oz;
            xx += xx < 0 ? L.nx : (xx >= L.nx ? -L.nx : 0);
            yy += yy < 0 ? L.ny : (yy >= L.ny ? -L.ny : 0);
            zz += zz < 0 ? L.nz : (zz >= L.nz ? -L.nz : 0);
            const int node = (int)(((size_t)zz * L.ny + yy) * L.nx + xx);
            if (C.tag[node] != stamp && atomicExch(&C.tag[node], stamp) != stamp) {
                const int j = atomicAdd(&C.ds->n_touched, 1);
                if (j < C.touched_cap) {
                    C.touched[j] = node;
                    if (C.tslot) C.tslot[node] = j;
                } else {
                    atomicOr(&C.ds->flags, FLAG_TOUCHED);
                }
            }
        }
    } else if (valid && C.reinterp) {
        // The atom's own region: its stencil and one node of margin.
#pragma unroll 1
        for (int k = 0; k < 64; ++k) {
            const int o[3] = {(k & 3) - 1, ((k >> 2) & 3) - 1, (k >> 4) - 1};
            if (L.walls && (b[2] + o[2] < 0 || b[2] + o[2] > L.nz - 1)) continue;
            const int xx = wrapl((long long)b[0] + o[0], L.nx), yy = wrapl((long long)b[1] + o[1], L.ny),
                      zz = wrapl((long long)b[2] + o[2], L.nz);
            float f[Q], g[3], u[3];
            pull<S>(src, L, xx, yy, zz, f);
            body_force(L, xx, yy, zz, g);
            node_velocity(L, f, g, u);
            const int node = (int)(((size_t)zz * L.ny + yy) * L.nx + xx);
            C.unode[node] = make_float4(u[0], u[1], u[2], __int_as_float(stamp));
            if (o[0] >= 0 && o[0] <= 1 && o[1] >= 0 && o[1] <= 1 && o[2] >= 0 && o[2] <= 1) {
                const float W = (o[0] ? t[0] : 1.f - t[0]) * (o[1] ? t[1] : 1.f - t[1]) * (o[2] ? t[2] : 1.f - t[2]);
                U[0] += W * u[0];
                U[1] += W * u[1];
                U[2] += W * u[2];
            }
            if (C.tag[node] != stamp && atomicExch(&C.tag[node], stamp) != stamp) {
                const int j = atomicAdd(&C.ds->n_touched, 1);
                if (j < C.touched_cap) {
                    C.touched[j] = node;
                    if (C.tslot) C.tslot[node] = j;
                } else {
                    atomicOr(&C.ds->flags, FLAG_TOUCHED);
                }
            }
        }
    } else if (valid) {
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
                const int j = atomicAdd(&C.ds->n_touched, 1);
                if (j < C.touched_cap) {
                    C.touched[j] = node;
                    if (C.tslot) C.tslot[node] = j;
                } else {
                    atomicOr(&C.ds->flags, FLAG_TOUCHED);
                }
            }
        }
    }
    if (valid)
        for (int d = 0; d < 3; ++d) C.U[d * na + a] = U[d];
}

// End of the atoms' part of the step: G_j -= W_aj J_a / Delta t (Delta t = 1)
// on the eight corners of the step-start stencil, one float4 atomic per
// corner. Aggregating the contributions of atoms that share a node before the
// atomics measured slower at 512^3 / 200,000 atoms (11.5 us per launch here;
// 18.3 us merging equal nodes within a warp with __match_any_sync, 24.0 us
// merging within the block's stencil tile in shared memory): with ~2 atoms
// per cell, merging removes about half of the atomics and costs more than
// they do.
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
        if (C.gfix) {  // deterministic: exact integer sums in the node's touched slot
            long long *g = C.gfix + 3 * (size_t)C.tslot[node];
#pragma unroll
            for (int d = 0; d < 3; ++d)
                atomicAdd(reinterpret_cast<unsigned long long *>(g + d),
                          (unsigned long long)llrint((double)(-W * J[d]) * kFixScale));
        } else {
            atomicAdd(&C.G[node], make_float4(-W * J[0], -W * J[1], -W * J[2], 0.f));
        }
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
    if (c.na == 0 || c.reinterp) return cudaSuccess;  // re-interpolation: the substeps spread
    k_spread<<<(c.na + 127) / 128, 128, 0, s>>>(c);
    return cudaGetLastError();
}

}  // namespace lbmd
