// Solute kernels: pair-search buckets, shifted-force Lennard-Jones + harmonic
// bonds, and the velocity-Verlet substeps with Stokes friction (Sec. 2.2: the
// atom receives gamma (u - v), u interpolated at the start of the coupled step).
//
// One kernel launch per substep. Kernel k of a step (k = 0..n_md) finishes
// substep k-1 (force at x_k, second half-kick) and starts substep k (first
// half-kick, drift to x_{k+1}, insertion of the atom into the buckets of
// generation k+1). Buckets rotate over three buffers by generation
// g = step*n_md + k: kernel k reads g, fills g+1 and empties g-1.
//
// Warp-sorted cell list: at the start of every coupled step the atoms are
// counting-sorted by bucket along a Morton curve of the bucket grid; the
// substep kernels visit atoms in that order, so neighbouring warps read
// neighbouring atoms. Forces come from per-atom Verlet lists (see below).
#include "lbmd_internal.cuh"

namespace lbmd {

namespace {

// c mod n for the usual case of c within one period of [0, n).
__device__ __forceinline__ int wrapi(int c, int n) {
    if ((unsigned)c < (unsigned)n) return c;
    if (c < 0 && c >= -n) return c + n;
    if (c >= n && c < 2 * n) return c - n;
    const int r = c % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// x_a - x_b, minimum image, as hi part dh (exact) and lo part dl. In the
// step frame every coordinate hi sits inside one binade [B, 2B) with B >= 2L,
// so hi_a - hi_b and the fold by a whole box length are exact; the lo parts
// (below one ulp of hi) differ with an error far below FP32 resolution.
__device__ __forceinline__ void pair_disp(const AtomArgs &A, float4 pa, float4 la, float4 pb, float4 lb, float dh[3],
                                          float dl[3]) {
    const float ha[3] = {pa.x, pa.y, pa.z}, hb[3] = {pb.x, pb.y, pb.z};
    const float l1[3] = {la.x, la.y, la.z}, l2[3] = {lb.x, lb.y, lb.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float s = ha[d] - hb[d];
        dh[d] = fmaf(-A.Lf[d], rintf(s * A.inv_Lf[d]), s);
        dl[d] = l1[d] - l2[d];
    }
}

// Cell of an atom from its step-frame position (hi + lo): floor of the
// offset from the frame origin over the cell side, wrapped into the grid.
__device__ __forceinline__ void cell_of(const AtomArgs &A, float4 p, float4 l, int c[3]) {
    c[0] = wrapi((int)floorf(((p.x - A.off[0]) + l.x) * A.binv_h[0]), A.bnc[0]);
    c[1] = wrapi((int)floorf(((p.y - A.off[1]) + l.y) * A.binv_h[1]), A.bnc[1]);
    c[2] = wrapi((int)floorf(((p.z - A.off[2]) + l.z) * A.binv_h[2]), A.bnc[2]);
}

// Position of an atom within its cell (0 <= t < h up to rounding), for the
// reach test of the neighbour cells.
__device__ __forceinline__ void in_cell(const AtomArgs &A, float4 p, float4 l, float t[3]) {
    const float v[3] = {(p.x - A.off[0]) + l.x, (p.y - A.off[1]) + l.y, (p.z - A.off[2]) + l.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) t[d] = v[d] - floorf(v[d] * A.binv_h[d]) * A.bh[d];
}

// Harmonic bond force factor -k (r - r0) / r with r - r0 evaluated as
// (r^2 - r0^2) / (r + r0) from a compensated r^2, so the stretch keeps its
// relative precision when r is close to r0.
__device__ __forceinline__ float bond_factor(const float dh_in[3], const float dl_in[3], float k, float r0) {
    // Renormalise hi + lo (two-sum: a component of hi may be smaller than its
    // lo) so lo is below half an ulp of hi and r = sqrt(hi part of r^2) stays
    // exact to FP32 rounding.
    float dh[3], dl[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) two_sum(dh_in[d], dl_in[d], dh[d], dl[d]);
    float p[3], pe[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        p[d] = dh[d] * dh[d];
        pe[d] = fmaf(dh[d], dh[d], -p[d]) + 2.f * dh[d] * dl[d];
    }
    float s01, e01, s, e;
    two_sum(p[0], p[1], s01, e01);
    two_sum(s01, p[2], s, e);
    const float r2_lo = (e01 + e) + (pe[0] + pe[1] + pe[2]);
    const float r0sq = r0 * r0;
    const float r0sq_lo = fmaf(r0, r0, -r0sq);
    const float diff = (s - r0sq) + (r2_lo - r0sq_lo);
    const float r = sqrtf(s);
    return -k * (diff / (r + r0)) / r;
}

// Bucket of a cell: cells fold onto a grid of at most 128 per axis (fold = nc
// when nc <= 128, otherwise 128 and fmask = 127).
__device__ __forceinline__ int bucket_of(const AtomArgs &A, const int c[3]) {
    return ((c[2] & A.bfmask[2]) * A.bfold[1] + (c[1] & A.bfmask[1])) * A.bfold[0] + (c[0] & A.bfmask[0]);
}

__device__ __forceinline__ bool bonded(const AtomArgs &A, int a, int b) {
    for (int s = A.bstart[a]; s < A.bstart[a + 1]; ++s)
        if (A.bpart[s] == b) return true;
    return false;
}

// Exact FP64 cell coordinate floor((x * nc) / L) mod nc.
__device__ __forceinline__ int exact_cell(double x, int nc, double L) {
    const double s = __ddiv_rn(__dmul_rn(x, (double)nc), L);
    const double fl = floor(s);
    if (!(fabs(fl) < 4.0e15)) return 0;
    long long c = (long long)fl % nc;
    return (int)(c < 0 ? c + nc : c);
}

// Candidate table of the W x W x W MD cells around cell cc (W = A.bwin, 3
// or 5), for one warp. A cell wholly beyond `reach` of the atom (t: its
// offset within cc; the gap along an axis is the distance to the near face
// of that cell) counts zero. tab[k], k < 128: candidates in cells 0..k
// (inclusive prefix, cells k >= W^3 empty); tab[128 + k]: bucket of cell k.
// Returns the total.
template <int W>
__device__ __forceinline__ int cell_table(const AtomArgs &A, int g3, const int cc[3], const float t[3], float reach2,
                                          int *tab) {
    const int lane = threadIdx.x & 31;
    constexpr int half = W / 2, ncell = W * W * W, rounds = (ncell + 31) / 32;
    int run = 0;
#pragma unroll
    for (int m = 0; m < rounds; ++m) {
        const int k = lane + 32 * m;
        int n = 0, b = 0;
        if (k < ncell) {
            const int o[3] = {k % W - half, (k / W) % W - half, k / (W * W) - half};
            float gap2 = 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float g = o[d] < 0   ? t[d] + (float)(-o[d] - 1) * A.bh[d]
                                : o[d] > 0 ? (A.bh[d] - t[d]) + (float)(o[d] - 1) * A.bh[d]
                                           : 0.f;
                gap2 += g * g;
            }
            if (gap2 < reach2 * 1.001f) {
                const int c[3] = {wrapi(cc[0] + o[0], A.bnc[0]), wrapi(cc[1] + o[1], A.bnc[1]),
                                  wrapi(cc[2] + o[2], A.bnc[2])};
                b = bucket_of(A, c);
                n = min(A.count[g3][b], A.bcap);
            }
        }
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        tab[k] = run + incl;
        tab[128 + k] = b;
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
#pragma unroll
    for (int k = 32 * rounds + lane; k < 128; k += 32) tab[k] = run;  // empty cells past the block
    __syncwarp();
    return run;
}

// Table cell holding candidate t (the first cell whose inclusive count
// exceeds t); `before` receives the candidates of the cells ahead of it.
__device__ __forceinline__ int cand_cell(const int *tab, int t, int &before) {
    int pos = 0;
#pragma unroll
    for (int step = 64; step > 0; step >>= 1)
        if (tab[pos + step - 1] <= t) pos += step;
    before = pos ? tab[pos - 1] : 0;
    return pos;
}

// Conservative force on atom a at the positions P, from the buckets of
// generation g3 that set_state fills with exact FP64 cells: a whole warp
// walks the candidates of the MD cells within rc around the atom's own exact
// cell (cell_table), bonds are dealt to the lanes, and the three components
// are summed across the warp. Every lane returns the full force.
__device__ void md_force_warp(const AtomArgs &A, const float4 *__restrict__ P, const float4 *__restrict__ Lq, int g3,
                              int a, float4 pa, float4 la, float F[3]) {
    __shared__ int s_tab[4][256];
    int *tab = s_tab[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    int cc[3];
    float t[3];
    for (int d = 0; d < 3; ++d) {
        const double x = A.X[d * A.na + a];
        cc[d] = exact_cell(x, A.bnc[d], A.Ld[d]);
        const double sx = x * ((double)A.bnc[d] / A.Ld[d]);
        t[d] = (float)((sx - floor(sx)) * ((double)A.Ld[d] / A.bnc[d]));
    }
    const int total = A.bwin == 5 ? cell_table<5>(A, g3, cc, t, A.rc2f, tab) : cell_table<3>(A, g3, cc, t, A.rc2f, tab);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    // Deterministic mode: each pair force also enters an exact fixed-point
    // sum (2^-32 units), independent of the candidates' order in the buckets.
    long long qx = 0, qy = 0, qz = 0;
    const double qs = 4294967296.0;
    for (int t0 = lane; t0 < total; t0 += 32) {
        int before;
        const int pos = cand_cell(tab, t0, before);
        const int q = A.slot[g3][(size_t)tab[128 + pos] * A.bcap + (t0 - before)];
        if (q == a) continue;
        float dh[3], dl[3];
        pair_disp(A, pa, la, P[q], Lq[q], dh, dl);
        const float d[3] = {dh[0] + dl[0], dh[1] + dl[1], dh[2] + dl[2]};
        const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!(r2 < A.rc2f)) continue;
        if (bonded(A, a, q)) continue;
        const float inv_r2 = 1.0f / r2;
        const float sr2 = A.lj_sig2 * inv_r2;
        const float sr6 = sr2 * sr2 * sr2;
        float fr = A.lj_24eps * inv_r2 * sr6 * (2.f * sr6 - 1.f) - A.lj_fc * rsqrtf(r2);
        if (A.coul && r2 < A.coul_rc2)
            fr += A.coul_2c * pa.w * P[q].w * (inv_r2 * inv_r2 - A.coul_irc3 * rsqrtf(r2));
        if (A.det) {
            qx += llrint((double)(fr * d[0]) * qs);
            qy += llrint((double)(fr * d[1]) * qs);
            qz += llrint((double)(fr * d[2]) * qs);
        } else {
            fx += fr * d[0];
            fy += fr * d[1];
            fz += fr * d[2];
        }
    }
    if (A.det) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            qx += __shfl_xor_sync(0xffffffffu, qx, o);
            qy += __shfl_xor_sync(0xffffffffu, qy, o);
            qz += __shfl_xor_sync(0xffffffffu, qz, o);
        }
        // every lane holds the exact sum: lane 0 carries it, the others none
        fx = lane == 0 ? (float)((double)qx / qs) : 0.f;
        fy = lane == 0 ? (float)((double)qy / qs) : 0.f;
        fz = lane == 0 ? (float)((double)qz / qs) : 0.f;
    }
    for (int sb = A.bstart[a] + lane; sb < A.bstart[a + 1]; sb += 32) {
        const int q = A.bpart[sb];
        float dh[3], dl[3];
        pair_disp(A, pa, la, P[q], Lq[q], dh, dl);
        const float fr = bond_factor(dh, dl, A.bk[sb], A.br0[sb]);
        fx += fr * (dh[0] + dl[0]);
        fy += fr * (dh[1] + dl[1]);
        fz += fr * (dh[2] + dl[2]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    __syncwarp();
    F[0] = fx;
    F[1] = fy;
    F[2] = fz;
}

__device__ __forceinline__ void insert(const AtomArgs &A, int g3, int a, const int c[3]) {
    const int b = bucket_of(A, c);
    const int s = atomicAdd(&A.count[g3][b], 1);
    if (s < A.bcap)
        A.slot[g3][(size_t)b * A.bcap + s] = a;
    else
        atomicOr(&A.ds->flags, FLAG_CELL);
    A.bucket[g3][a] = b;
    A.sidx[g3][a] = s;
}

// ---------------------------------------------------------------------------
// Warp-sorted order: counting sort of the atoms by bucket, buckets taken in
// Morton order over a 128^3 grid (codes outside the bucket grid count zero).

__device__ __forceinline__ unsigned spread3(unsigned v) {
    unsigned r = 0;
#pragma unroll
    for (int i = 0; i < kMortonBits; ++i) r |= ((v >> i) & 1u) << (3 * i);
    return r;
}

__device__ __forceinline__ unsigned morton3(int x, int y, int z) {
    return spread3((unsigned)x) | (spread3((unsigned)y) << 1) | (spread3((unsigned)z) << 2);
}

__device__ __forceinline__ int compact3(unsigned m) {
    int r = 0;
#pragma unroll
    for (int i = 0; i < kMortonBits; ++i) r |= (int)((m >> (3 * i)) & 1u) << i;
    return r;
}

// Block-local exclusive scan of the bucket counts (1024 Morton codes per block).
__global__ void __launch_bounds__(1024) k_sort_local(AtomArgs A) {
    const int step = A.ds->step;
    const int g3 = ((step % 3) * (A.n_md % 3)) % 3;
    const unsigned m = blockIdx.x * 1024u + threadIdx.x;
    const int x = compact3(m), y = compact3(m >> 1), z = compact3(m >> 2);
    int cnt = 0;
    if (x < A.bfold[0] && y < A.bfold[1] && z < A.bfold[2]) cnt = A.count[g3][(z * A.bfold[1] + y) * A.bfold[0] + x];
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    const int before = warp ? wsum[warp - 1] : 0;
    A.scan_local[m] = before + incl - cnt;
    if (threadIdx.x == 1023) A.scan_block[blockIdx.x] = before + incl;
}

// Exclusive scan of the kMortonCodes/1024 block totals (one block, two
// totals per thread).
__global__ void __launch_bounds__(1024) k_sort_top(AtomArgs A) {
    constexpr int NB = kMortonCodes / 1024;
    __shared__ int sh[1024];
    const int t = threadIdx.x;
    const int a0 = A.scan_block[2 * t], a1 = A.scan_block[2 * t + 1];
    sh[t] = a0 + a1;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = t >= o ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += v;
        __syncthreads();
    }
    const int before = t ? sh[t - 1] : 0;
    static_assert(NB == 2048, "two block totals per thread");
    A.scan_block[2 * t] = before;
    A.scan_block[2 * t + 1] = before + a0;
}

// Sub-cell of every atom within its bucket cell: 4 x 4 x 4 sub-cells in
// Morton order (from the FP64 position), the sort key within a bucket.
__global__ void __launch_bounds__(128) k_sort_code(AtomArgs A) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.na) return;
    unsigned code = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double s = A.X[d * A.na + a] * ((double)A.bnc[d] / A.Ld[d]);
        const double f = s - floor(s);
        const unsigned c = f >= 0.0 && f < 1.0 ? min(3u, (unsigned)(f * 4.0)) : 0u;
        code |= ((c & 1u) | ((c & 2u) << 2)) << d;
    }
    A.scode[a] = (int)code;
}

// Position of every atom in the sorted order: its bucket's offset plus its
// rank within the bucket by (sub-cell code, slot), so the atoms a warp takes
// from one bucket sit close together.
__global__ void __launch_bounds__(128) k_sort_scatter(AtomArgs A) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.na) return;
    const int step = A.ds->step;
    const int g3 = ((step % 3) * (A.n_md % 3)) % 3;
    const int b = A.bucket[g3][a];
    const int x = b % A.bfold[0], y = (b / A.bfold[0]) % A.bfold[1], z = b / (A.bfold[0] * A.bfold[1]);
    const unsigned m = morton3(x, y, z);
    const int s = A.sidx[g3][a];
    int rank = s;  // an atom past the bucket's capacity (an error already flagged) keeps its slot
    if (s < A.bcap) {
        const int n = min(A.count[g3][b], A.bcap);
        const int mine = A.scode[a];
        rank = 0;
        for (int t = 0; t < n; ++t) {
            const int c = A.scode[A.slot[g3][(size_t)b * A.bcap + t]];
            rank += c < mine || (c == mine && t < s);
        }
    }
    const int pos = A.scan_block[m >> 10] + A.scan_local[m] + rank;
    if (pos >= 0 && pos < A.na) A.order[pos] = a;
}


// set_state: step frame at generation 0, exact binning, empty records.
__global__ void k_prime_insert(AtomArgs A) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.na) return;
    float4 p, l;
    if (!set_frame(A, a, p, l)) atomicOr(&A.ds->flags, FLAG_NONFINITE);
    A.P[0][a] = p;
    A.L[0][a] = l;
    int c[3];
    for (int d = 0; d < 3; ++d) c[d] = exact_cell(A.X[d * A.na + a], A.bnc[d], A.Ld[d]);
    insert(A, 0, a, c);
    A.bucket[2][a] = 0;
    A.bucket[1][a] = 0;
}

__global__ void k_prime_force(AtomArgs A) {
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (a >= A.na) return;
    float F[3];
    md_force_warp(A, A.P[0], A.L[0], 0, a, A.P[0][a], A.L[0][a], F);
    if ((threadIdx.x & 31) == 0)
        for (int d = 0; d < 3; ++d) A.F[d * A.na + a] = F[d];
}

// ---------------------------------------------------------------------------
// Verlet neighbour lists. Each atom keeps the non-bonded atoms within
// rc + skin of it (at most NL_MAX). A list stays valid while no atom has
// drifted more than skin/2 since it was built; the drift check raises a
// device flag that makes the next force evaluation rebuild every list, from
// the buckets of that generation, inside the same kernel. Flags rotate over
// three slots like the buckets: kernel k reads slot g, raises g+1, clears g-1.

// Deterministic mode: a list in ascending atom index (the bucket slots fill
// in the order of atomics), so the force sums in the same order every run.
// A bitonic sort of 256 entries by the warp in its 256-int scratch row; out
// of line, so the rare path keeps its registers to itself.
__device__ __noinline__ void sort_list(int *out, int n, int *tab) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    for (int i = lane; i < 256; i += 32) tab[i] = i < n ? out[i] : 0x7fffffff;
    __syncwarp();
    for (int size = 2; size <= 256; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < 128; i += 32) {
                const int lo = 2 * stride * (i / stride) + (i % stride), hi = lo + stride;
                const int x = tab[lo], y = tab[hi];
                if ((x > y) == ((lo & size) == 0)) {
                    tab[lo] = y;
                    tab[hi] = x;
                }
            }
            __syncwarp();
        }
    for (int i = lane; i < n; i += 32) out[i] = tab[i];
    __syncwarp();
}

// Builds atom a's list with the warp: candidates of the MD cells within the
// list radius (cell_table), NBB per lane per round (all
// their slot loads issued together, then all their position loads, so a
// round costs two dependent memory latencies), ballot compaction. Bonded
// partners (the first 32) sit one per lane and are matched with shuffles,
// without touching memory per candidate.
template <int NBB, int W, bool DET>
__device__ __noinline__ void build_list(const AtomArgs &A, const float4 *__restrict__ P,
                                        const float4 *__restrict__ Lq, int g3, int a, float4 pa, float4 la, int b0,
                                        int b1) {
    __shared__ int s_tab[4][256];
    int *tab = s_tab[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    int cc[3];
    cell_of(A, pa, la, cc);
    float t[3];
    in_cell(A, pa, la, t);
    const int nbond = b1 - b0;
    const int partner = lane < nbond ? A.bpart[b0 + lane] : -1;
    // 27 coarse cells: lane k < 27 holds cell k's count, bucket and inclusive
    // prefix in registers, found by a shuffle search; 125 half-size cells:
    // the prefix table in shared memory, found by a binary search there.
    int bucket = 0, n = 0, incl = 0, total;
    if constexpr (W == 3) {
        if (lane < 27) {
            const int o[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
            float gap2 = 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float g = o[d] < 0 ? t[d] : (o[d] > 0 ? A.bh[d] - t[d] : 0.f);
                gap2 += g * g;
            }
            if (gap2 < A.rl2 * 1.001f) {
                const int c[3] = {wrapi(cc[0] + o[0], A.bnc[0]), wrapi(cc[1] + o[1], A.bnc[1]),
                                  wrapi(cc[2] + o[2], A.bnc[2])};
                bucket = bucket_of(A, c);
                n = min(A.count[g3][bucket], A.bcap);
            }
        }
        incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        total = __shfl_sync(0xffffffffu, incl, 31);
    } else {
        total = cell_table<W>(A, g3, cc, t, A.rl2, tab);
    }
    int kept = 0;
    int *__restrict__ out = A.nbr + (size_t)a * NL_MAX;
    for (int t0 = 0; t0 < total; t0 += 32 * NBB) {
        int q[NBB];
#pragma unroll
        for (int u = 0; u < NBB; ++u) {
            const int tc = t0 + 32 * u + lane;
            int cb, before;
            if constexpr (W == 3) {
                int pos = 0;  // first lane whose inclusive count exceeds tc
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int probe = __shfl_sync(0xffffffffu, incl, pos + step - 1);
                    if (probe <= tc) pos += step;
                }
                cb = __shfl_sync(0xffffffffu, bucket, pos & 31);
                before = __shfl_sync(0xffffffffu, incl - n, pos & 31);
            } else {
                const int pos = cand_cell(tab, tc < total ? tc : total - 1, before);
                cb = tab[128 + pos];
            }
            q[u] = tc < total ? A.slot[g3][(size_t)cb * A.bcap + (tc - before)] : -1;
        }
        float4 pq[NBB], lq[NBB];
#pragma unroll
        for (int u = 0; u < NBB; ++u)
            if (q[u] >= 0) {
                pq[u] = P[q[u]];
                lq[u] = Lq[q[u]];
            }
#pragma unroll
        for (int u = 0; u < NBB; ++u) {
            bool keep = false;
            if (q[u] >= 0 && q[u] != a) {
                float dh[3], dl[3];
                pair_disp(A, pa, la, pq[u], lq[u], dh, dl);
                const float d[3] = {dh[0] + dl[0], dh[1] + dl[1], dh[2] + dl[2]};
                keep = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < A.rl2;
            }
            bool is_bonded = false;
            for (int l = 0; l < min(nbond, 32); ++l) is_bonded |= __shfl_sync(0xffffffffu, partner, l) == q[u];
            if (keep && nbond > 32 && !is_bonded) is_bonded = bonded(A, a, q[u]);
            keep = keep && !is_bonded;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const int at = kept + __popc(m & ((1u << lane) - 1u));
            if (keep && at < NL_MAX) out[at] = q[u];
            kept += __popc(m);
        }
    }
    if constexpr (DET) sort_list(out, min(kept, NL_MAX), tab);
    if (lane == 0) {
        A.nnb[a] = min(kept, NL_MAX);
        if (kept > NL_MAX) atomicOr(&A.ds->flags, FLAG_CELL);
    }
    __syncwarp();
}

// The substep kernel runs TPA lanes per atom and takes NB list entries per
// lane per round (a round issues NB index loads, then NB position pairs).
// Few atoms: 8 lanes shorten each atom's chain of dependent work; many atoms
// (the GPU full several times over): 4 lanes spend fewer instructions on the
// per-atom reductions.
constexpr int NBB = 2;  // candidates per lane per round of a list build


// Conservative force on atom a from its list (nn entries) and its bonds
// (slots b0..b1), over the TPA lanes of its group; every lane of the group
// returns the full force.
template <int TPA, int NB>
__device__ __forceinline__ void list_force(const AtomArgs &A, const float4 *__restrict__ P,
                                           const float4 *__restrict__ Lq, int a, float4 pa, float4 la, int sub,
                                           int nn, int b0, int b1, float F[3]) {
    // The first bond of each lane: its loads go out with the first round.
    const int sb = b0 + sub;
    int qb = -1;
    float kb = 0.f, r0b = 0.f;
    if (sb < b1) {
        qb = A.bpart[sb];
        kb = A.bk[sb];
        r0b = A.br0[sb];
    }
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const int *__restrict__ lst = A.nbr + (size_t)a * NL_MAX;
    for (int j0 = sub; j0 < nn; j0 += TPA * NB) {
        int q[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int j = j0 + u * TPA;
            q[u] = j < nn ? lst[j] : a;
        }
        float4 ph[NB], pl[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            ph[u] = P[q[u]];
            pl[u] = Lq[q[u]];
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            if (j0 + u * TPA >= nn) continue;
            float dh[3], dl[3];
            pair_disp(A, pa, la, ph[u], pl[u], dh, dl);
            const float d[3] = {dh[0] + dl[0], dh[1] + dl[1], dh[2] + dl[2]};
            const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < A.rc2f) {
                const float inv_r2 = 1.0f / r2;
                const float sr2 = A.lj_sig2 * inv_r2;
                const float sr6 = sr2 * sr2 * sr2;
                const float ir = rsqrtf(r2);
                float fr = A.lj_24eps * inv_r2 * sr6 * (2.f * sr6 - 1.f) - A.lj_fc * ir;
                if (A.coul && r2 < A.coul_rc2)
                    fr += A.coul_2c * pa.w * ph[u].w * (inv_r2 * inv_r2 - A.coul_irc3 * ir);
                fx += fr * d[0];
                fy += fr * d[1];
                fz += fr * d[2];
            }
        }
    }
    for (int s = sb; s < b1; s += TPA) {
        int q = qb;
        float k = kb, r0 = r0b;
        if (s != sb) {
            q = A.bpart[s];
            k = A.bk[s];
            r0 = A.br0[s];
        }
        float dh[3], dl[3];
        pair_disp(A, pa, la, P[q], Lq[q], dh, dl);
        const float fr = bond_factor(dh, dl, k, r0);
        fx += fr * (dh[0] + dl[0]);
        fy += fr * (dh[1] + dl[1]);
        fz += fr * (dh[2] + dl[2]);
    }
#pragma unroll
    for (int o = TPA / 2; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    F[0] = fx;
    F[1] = fy;
    F[2] = fz;
}

__device__ __forceinline__ float4 shfl4(float4 v, int src) {
    return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                       __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}

// Component d of the velocity (sum f c + g/2)/rho of node (x, y, z) from the
// populations pulled into it: the value the interpolation computes for its
// nodes, with two running sums instead of the 19 pulled values.
template <int S>
__device__ __forceinline__ float pulled_velocity(const typename Store<S>::T *__restrict__ src, const Lat &L, int x,
                                                 int y, int z, int d) {
    const int xm = x == 0 ? L.nx - 1 : x - 1, xp = x == L.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? L.ny - 1 : y - 1, yp = y == L.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? L.nz - 1 : z - 1, zp = z == L.nz - 1 ? 0 : z + 1;
    const size_t node = ((size_t)z * L.ny + y) * L.nx + x;
    float drho = 0.f, j = 0.f;
#pragma unroll 1
    for (int i = 0; i < Q; ++i) {  // one population at a time: a rare path, kept small
        const float f = Store<S>::ld(src + pull_index(L, i, x, y, z, xm, xp, ym, yp, zm, zp, node));
        drho += f;
        if (d == 0 && cx(i)) j += cx(i) * f;
        if (d == 1 && cy(i)) j += cy(i) * f;
        if (d == 2 && cz(i)) j += cz(i) * f;
    }
    float g[3];
    body_force(L, x, y, z, g);
    const float inv = 1.f / (L.rho0 + drho);
    return (j + 0.5f * g[d]) * inv;
}

// The same for any storage format.
__device__ __forceinline__ float far_velocity(const void *src, int store, const Lat *Lp, int x, int y, int z, int d) {
    const Lat &L = *Lp;
    if (store == LBMD_F32) return pulled_velocity<LBMD_F32>((const float *)src, L, x, y, z, d);
    if (store == LBMD_F16_SHIFTED) return pulled_velocity<LBMD_F16_SHIFTED>((const __half *)src, L, x, y, z, d);
    return pulled_velocity<LBMD_BF16_SHIFTED>((const __nv_bfloat16 *)src, L, x, y, z, d);
}

// TPA lanes per atom, atoms in warp-sorted order (neighbouring warps touch
// neighbouring atoms). Every load that depends only on the atom index is
// issued at once, before any store, so a substep costs few dependent memory
// latencies: the device step and flags, the atom index, the atom's state,
// two per round of its list, and the bucket insertion. When the flag of this
// generation is up the warp first rebuilds the lists of its atoms one after
// the other (all 32 lanes on each); then each group evaluates its atom's
// force over the list, lanes 0-2 of the group integrate one component each,
// and lane 0 re-bins the atom.
// Launch bounds: 8 lanes per atom at 9 blocks per SM (56 registers: the
// 20k-atom grid fits one wave); 4 lanes at 10 blocks (48 registers): 8%
// faster than 8 blocks at 64 registers on 200k atoms, where the grid takes
// several waves and more resident warps hide more latency.
template <int TPA, int NB, int W, bool RI, bool DET>
__global__ void __launch_bounds__(128, TPA == 8 ? 9 : 10) k_md_substep(AtomArgs A, int k) {
    const int lane = threadIdx.x & 31;
    const int sub = lane & (TPA - 1);
    const int slot = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / TPA) + lane / TPA;
    const int na = A.na;
    // Launched with programmatic dependent launch: what the previous kernel
    // (substep k-1, or the interpolation for k = 0) does not write is read
    // before waiting on it: the step counter (advanced at the end of the
    // previous coupled step), the atom order (sorted before the
    // interpolation), masses and bond ranges. (An early trigger of the next
    // substep's launch measured slower: its waiting blocks hold SM slots.)
    const int step = A.ds->step;
    const int warp_first = slot - lane / TPA;
    const int a = warp_first < na ? A.order[slot < na ? slot : warp_first] : 0;
    const float im = A.inv_m[a];
    const int b0 = A.bstart[a], b1 = A.bstart[a + 1];
    cudaGridDependencySynchronize();
    const int fl0 = A.ds->nl_flag[0], fl1 = A.ds->nl_flag[1], fl2 = A.ds->nl_flag[2];
    const int g3 = ((step % 3) * (A.n_md % 3) + k) % 3;
    const int gn3 = (g3 + 1) % 3, gp3 = (g3 + 2) % 3;
    const int par = ((step & 1) * (A.n_md & 1) + k) & 1;
    const int rebuild = g3 == 0 ? fl0 : (g3 == 1 ? fl1 : fl2);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.ds->nl_flag[gp3] = 0;
        // Kernel 0 evaluates no force: hand a pending rebuild on to kernel 1.
        if (k == 0 && rebuild) atomicOr(&A.ds->nl_flag[gn3], 1);
    }
    if (warp_first >= na) return;  // whole warp past the end
    const bool valid = slot < na;
    // Everything that depends only on a, in one go: lane d < 3 of the group
    // owns component d.
    const int dcomp = sub < 3 ? sub : 0;
    const float vd = A.V[dcomp * na + a], Ud = A.U[dcomp * na + a];
    const float Jd = k == 0 ? 0.f : A.J[dcomp * na + a];
    const float Dold = A.D[dcomp * na + a];
    const float4 pa = A.P[par][a];
    const float4 la = A.L[par][a];
    const int nn = A.nnb[a];
    const int old_bucket = sub == 0 && k < A.n_md ? A.bucket[gp3][a] : 0;
    float F[3] = {0.f, 0.f, 0.f};
    if (k == 0) {
        F[0] = A.F[a];
        F[1] = A.F[na + a];
        F[2] = A.F[2 * na + a];
    }
    if (A.recP && valid) {
        if (sub == 0) {
            A.recP[(size_t)k * na + a] = pa;
            A.recL[(size_t)k * na + a] = la;
        }
        if (sub < 3) A.recV[(size_t)k * 3 * na + sub * na + a] = vd;
    }
    const bool reset = k > 0 && rebuild;
    if (k > 0) {
        int nlist = nn;
        if (reset) {
            for (int g = 0; g < 32 / TPA; ++g) {
                const int ag = __shfl_sync(0xffffffffu, a, g * TPA);
                const int vg = __shfl_sync(0xffffffffu, (int)valid, g * TPA);
                const int bg0 = __shfl_sync(0xffffffffu, b0, g * TPA), bg1 = __shfl_sync(0xffffffffu, b1, g * TPA);
                const float4 pg = shfl4(pa, g * TPA);
                const float4 lg = shfl4(la, g * TPA);
                if (vg) build_list<NBB, W, DET>(A, A.P[par], A.L[par], g3, ag, pg, lg, bg0, bg1);
            }
            __syncwarp();
            nlist = A.nnb[a];
        }
        list_force<TPA, NB>(A, A.P[par], A.L[par], a, pa, la, sub, nlist, b0, b1, F);
    }
    if (!valid) return;
    // Re-interpolated coupling: U at x_k from the step's node velocities
    // (lanes 0-2, one component each), the trilinear stencil of x_k kept for
    // the spread of this kernel's impulse below.
    float Uk = Ud, wt[3] = {0.f, 0.f, 0.f};
    int bcell[3] = {0, 0, 0};
    if (RI && sub < 3) {
        const float hi4[3] = {pa.x, pa.y, pa.z}, lo4[3] = {la.x, la.y, la.z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float s0 = hi4[d] - A.off[d];  // exact: both in the step frame's binade
            float fl = floorf(s0);
            float t = (s0 - fl) + lo4[d];
            if (t < 0.f) {
                t += 1.f;
                fl -= 1.f;
            } else if (t >= 1.f) {
                t -= 1.f;
                fl += 1.f;
            }
            wt[d] = t;
            int c = (int)fl;
            if (d == 2 && A.walls) {
                if (c < 0 || c + 1 > A.nl[2] - 1) {
                    atomicOr(&A.ds->flags, FLAG_WALL);
                    c = c < 0 ? 0 : A.nl[2] - 2;
                }
            } else {
                c = wrapi(c, A.nl[d]);
            }
            bcell[d] = c;
        }
        const int stamp = step + 1;
        float u = 0.f;
        unsigned far = 0;  // corners outside the frozen region
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int o[3] = {j & 1, (j >> 1) & 1, (j >> 2) & 1};
            const int xx = o[0] ? (bcell[0] + 1 == A.nl[0] ? 0 : bcell[0] + 1) : bcell[0];
            const int yy = o[1] ? (bcell[1] + 1 == A.nl[1] ? 0 : bcell[1] + 1) : bcell[1];
            const int zz = o[2] ? (bcell[2] + 1 == A.nl[2] ? 0 : bcell[2] + 1) : bcell[2];
            const float Wt = (o[0] ? wt[0] : 1.f - wt[0]) * (o[1] ? wt[1] : 1.f - wt[1]) * (o[2] ? wt[2] : 1.f - wt[2]);
            const float4 un = A.unode[((size_t)zz * A.nl[1] + yy) * A.nl[0] + xx];
            if (__float_as_int(un.w) == stamp)
                u += Wt * (sub == 0 ? un.x : (sub == 1 ? un.y : un.z));
            else
                far |= 1u << j;
        }
        // An atom that moved more than one node from its step-start stencil
        // within the step: the velocity of a corner the interpolation did not
        // freeze comes from the step's populations (which no kernel writes
        // during the substeps), the same value the interpolation would have
        // stored, and the node joins the step's touched list so that the
        // impulse spread onto it reaches the collision.
#pragma unroll 1
        for (int j = 0; far; ++j) {
            if (!(far >> j & 1u)) continue;
            far &= ~(1u << j);
            const int o[3] = {j & 1, (j >> 1) & 1, (j >> 2) & 1};
            const int xx = o[0] ? (bcell[0] + 1 == A.nl[0] ? 0 : bcell[0] + 1) : bcell[0];
            const int yy = o[1] ? (bcell[1] + 1 == A.nl[1] ? 0 : bcell[1] + 1) : bcell[1];
            const int zz = o[2] ? (bcell[2] + 1 == A.nl[2] ? 0 : bcell[2] + 1) : bcell[2];
            const float Wt = (o[0] ? wt[0] : 1.f - wt[0]) * (o[1] ? wt[1] : 1.f - wt[1]) * (o[2] ? wt[2] : 1.f - wt[2]);
            u += Wt * far_velocity(A.pop[step & 1], A.store, A.lat, xx, yy, zz, sub);
            const int node = (int)(((size_t)zz * A.nl[1] + yy) * A.nl[0] + xx);
            if (sub == 0 && A.tag[node] != stamp && atomicExch(&A.tag[node], stamp) != stamp) {
                const int t = atomicAdd(&A.ds->n_touched, 1);
                if (t < A.touched_cap)
                    A.touched[t] = node;
                else
                    atomicOr(&A.ds->flags, FLAG_TOUCHED);
            }
        }
        Uk = u;
    }
    // Lanes 0-2: one velocity-Verlet component each.
    float v = vd, J = Jd, p = 0.f, lo = 0.f, Dd = 0.f;
    const float Fd = sub == 0 ? F[0] : (sub == 1 ? F[1] : F[2]);
    if (A.recF && sub < 3) A.recF[(size_t)k * 3 * na + sub * na + a] = Fd;
    if (sub < 3) {
        if (k > 0) {  // second half-kick of substep k-1, drag at v_{k-1/2}
            const float drag = A.gamma * (Uk - v);
            J += A.hdt * drag;
            v += A.hdt * (Fd + drag) * im;
        }
        if (k < A.n_md) {  // first half-kick of substep k, drag at v_k, then drift
            const float drag = A.gamma * (Uk - v);
            J += A.hdt * drag;
            v += A.hdt * (Fd + drag) * im;
            p = sub == 0 ? pa.x : (sub == 1 ? pa.y : pa.z);
            lo = sub == 0 ? la.x : (sub == 1 ? la.y : la.z);
            // Error-free update of hi + lo by v dt (two-sum plus the exact
            // product error).
            const float inc = v * A.dt;
            const float e_mul = fmaf(v, A.dt, -inc);
            float s, e_add;
            two_sum(p, inc, s, e_add);
            p = s;
            lo += e_add + e_mul;
            // Drift since the last list build (which this kernel just did
            // when reset is set).
            Dd = (reset ? 0.f : Dold) + inc;
            A.D[sub * na + a] = Dd;
        } else {
            // End of the coupled step: cache the force and advance the FP64
            // accumulator by the compensated displacement.
            const float pc = sub == 0 ? pa.x : (sub == 1 ? pa.y : pa.z);
            const float lc = sub == 0 ? la.x : (sub == 1 ? la.y : la.z);
            A.F[sub * na + a] = Fd;
            A.X[sub * na + a] += ((double)pc - (double)A.P0[sub * na + a]) + ((double)lc - (double)A.R0[sub * na + a]);
            if (reset) A.D[sub * na + a] = 0.f;
        }
        A.V[sub * na + a] = v;
        A.J[sub * na + a] = J;
    }
    const int base = lane & ~(TPA - 1);
    const unsigned gm = (TPA == 32 ? 0xffffffffu : ((1u << TPA) - 1u)) << base;  // valid groups are whole
    if (RI) {
        // The fluid receives the opposite of this kernel's friction impulse,
        // with the weights U was interpolated with.
        const float dJ = sub < 3 ? J - Jd : 0.f;
        const float jx = __shfl_sync(gm, dJ, base), jy = __shfl_sync(gm, dJ, base + 1),
                    jz = __shfl_sync(gm, dJ, base + 2);
        if (sub == 0) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int o[3] = {j & 1, (j >> 1) & 1, (j >> 2) & 1};
                const int xx = o[0] ? (bcell[0] + 1 == A.nl[0] ? 0 : bcell[0] + 1) : bcell[0];
                const int yy = o[1] ? (bcell[1] + 1 == A.nl[1] ? 0 : bcell[1] + 1) : bcell[1];
                const int zz = o[2] ? (bcell[2] + 1 == A.nl[2] ? 0 : bcell[2] + 1) : bcell[2];
                const float Wt =
                    (o[0] ? wt[0] : 1.f - wt[0]) * (o[1] ? wt[1] : 1.f - wt[1]) * (o[2] ? wt[2] : 1.f - wt[2]);
                atomicAdd(&A.G[((size_t)zz * A.nl[1] + yy) * A.nl[0] + xx], make_float4(-Wt * jx, -Wt * jy, -Wt * jz, 0.f));
            }
        }
    }
    if (k == A.n_md) return;
    const float px = __shfl_sync(gm, p, base), py = __shfl_sync(gm, p, base + 1), pz = __shfl_sync(gm, p, base + 2);
    const float lx = __shfl_sync(gm, lo, base), ly = __shfl_sync(gm, lo, base + 1), lz = __shfl_sync(gm, lo, base + 2);
    const float D2 = __shfl_sync(gm, Dd * Dd, base) + __shfl_sync(gm, Dd * Dd, base + 1) +
                     __shfl_sync(gm, Dd * Dd, base + 2);
    if (sub != 0) return;
    const float4 pn = make_float4(px, py, pz, pa.w), ln = make_float4(lx, ly, lz, 0.f);  // w: charge
    A.P[par ^ 1][a] = pn;
    A.L[par ^ 1][a] = ln;
    A.count[gp3][old_bucket] = 0;
    int c[3];
    cell_of(A, pn, ln, c);
    insert(A, gn3, a, c);
    if (!(isfinite(px) && isfinite(py) && isfinite(pz))) atomicOr(&A.ds->flags, FLAG_NONFINITE);
    // Drift since the last list build: past half the skin a pair may have
    // entered the cutoff unseen, so the next force rebuilds.
    if (!(D2 <= A.half_skin2)) atomicOr(&A.ds->nl_flag[gn3], 1);
}

// Diagnostics: exact FP64 cells (of the reported grid, side >= rc + skin)
// and neighbour counts (strict r^2 < rc^2, minimum image), searched through
// the MD buckets of the current generation. An atom sits in the bucket of
// its exact MD cell or, after FP32 binning in the substeps, of a neighbour
// of it; one found in none of these is reported as cell -1.
__global__ void k_md_diag(AtomArgs A, int *cell_of, int *neigh) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.na) return;
    const long long gen = (long long)A.ds->step * A.n_md;
    const int g3 = (int)(gen % 3);
    const int na = A.na;
    int c[3], cb[3];
    for (int d = 0; d < 3; ++d) {
        c[d] = exact_cell(A.X[d * na + a], A.nc[d], A.Ld[d]);
        cb[d] = exact_cell(A.X[d * na + a], A.bnc[d], A.Ld[d]);
    }
    const int lin = (c[2] * A.nc[1] + c[1]) * A.nc[0] + c[0];
    // Offsets -r..r of a window, without those that alias a nearer one on
    // a grid of fewer than 2r + 1 cells.
    auto alias = [&](int o, int d) { return o > A.bnc[d] / 2 || o < -((A.bnc[d] - 1) / 2); };
    bool found = false;
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                const int o[3] = {ox, oy, oz};
                int cc[3];
                for (int d = 0; d < 3; ++d) cc[d] = wrapi(cb[d] + o[d], A.bnc[d]);
                const int b = bucket_of(A, cc);
                const int n = min(A.count[g3][b], A.bcap);
                for (int j = 0; j < n; ++j) found = found || A.slot[g3][(size_t)b * A.bcap + j] == a;
            }
    if (cell_of) cell_of[a] = found ? lin : -1;
    if (!neigh) return;
    int count = 0;
    const double xa[3] = {A.X[a], A.X[na + a], A.X[2 * na + a]};
    // A block of MD cells of radius R covers every cell an atom within rc
    // can be binned in: its exact cell is at most R - 1 away (R = 3 for cells
    // of side >= rc/2, 2 for side >= rc), plus one for FP32 binning. Its
    // buckets are distinct once aliased offsets are skipped, so every atom is
    // seen at most once; atoms of folded far cells fail the distance test.
    const int R = A.bwin == 5 ? 3 : 2;
    for (int oz = -R; oz <= R; ++oz)
        for (int oy = -R; oy <= R; ++oy)
            for (int ox = -R; ox <= R; ++ox) {
                const int o[3] = {ox, oy, oz};
                if (alias(ox, 0) || alias(oy, 1) || alias(oz, 2)) continue;
                int cc[3];
                for (int d = 0; d < 3; ++d) cc[d] = wrapi(cb[d] + o[d], A.bnc[d]);
                const int b = bucket_of(A, cc);
                const int n = min(A.count[g3][b], A.bcap);
                for (int j = 0; j < n; ++j) {
                    const int q = A.slot[g3][(size_t)b * A.bcap + j];
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
    k_prime_insert<<<(a.na + 127) / 128, 128, 0, s>>>(a);
    k_prime_force<<<(a.na + 3) / 4, 128, 0, s>>>(a);
    return cudaGetLastError();
}

template <int TPA, int W, bool RI, bool DET>
cudaError_t launch_substep(const AtomArgs &a, int k, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((a.na + 4 * (32 / TPA) - 1) / (4 * (32 / TPA)));  // 128 threads, TPA lanes per atom
    cfg.blockDim = dim3(128);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_md_substep<TPA, 2, W, RI, DET>, a, k);
}

cudaError_t launch_md_substep(const AtomArgs &a, int k, cudaStream_t s) {
    if (a.na == 0) return cudaSuccess;
    // Above ~64k atoms the 8-lane grid no longer fits the GPU in one wave.
    if (a.reinterp) {
        if (a.bwin == 5)
            return a.na > 65536 ? launch_substep<4, 5, true, false>(a, k, s) : launch_substep<8, 5, true, false>(a, k, s);
        return a.na > 65536 ? launch_substep<4, 3, true, false>(a, k, s) : launch_substep<8, 3, true, false>(a, k, s);
    }
    // Deterministic mode (sorted lists) in its own instantiations: the
    // default ones carry none of its code. It excludes re-interpolation.
    if (a.det) {
        if (a.bwin == 5)
            return a.na > 65536 ? launch_substep<4, 5, false, true>(a, k, s) : launch_substep<8, 5, false, true>(a, k, s);
        return a.na > 65536 ? launch_substep<4, 3, false, true>(a, k, s) : launch_substep<8, 3, false, true>(a, k, s);
    }
    if (a.bwin == 5)
        return a.na > 65536 ? launch_substep<4, 5, false, false>(a, k, s) : launch_substep<8, 5, false, false>(a, k, s);
    return a.na > 65536 ? launch_substep<4, 3, false, false>(a, k, s) : launch_substep<8, 3, false, false>(a, k, s);
}

cudaError_t launch_md_sort(const AtomArgs &a, cudaStream_t s) {
    if (a.na == 0) return cudaSuccess;
    k_sort_local<<<kMortonCodes / 1024, 1024, 0, s>>>(a);
    k_sort_top<<<1, 1024, 0, s>>>(a);
    k_sort_code<<<(a.na + 127) / 128, 128, 0, s>>>(a);
    k_sort_scatter<<<(a.na + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_md_diag(const AtomArgs &a, int *cell_of, int *neigh, cudaStream_t s) {
    if (a.na == 0) return cudaSuccess;
    k_md_diag<<<(a.na + 127) / 128, 128, 0, s>>>(a, cell_of, neigh);
    return cudaGetLastError();
}

}  // namespace lbmd
