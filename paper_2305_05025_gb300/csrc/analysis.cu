// Solute observables on the device: the trajectory analyses of Sec. 3 of the
// paper (radius of gyration, root-mean-square deviation from a reference
// structure after optimal superposition, per-atom root-mean-square
// fluctuation, and the covariance matrix whose eigenvectors are the principal
// components), for a selection of atoms of the synthetic chains.
//
// Per frame: one pass over the atoms accumulates in FP64 the mass moments of
// all atoms (R_g^2) and, over the selection, the centroid, the sum of squares
// and the 3x3 correlation with the centred reference; the host solves the
// 4x4 eigenproblem of the optimal rotation (Horn's quaternion form); a second
// pass applies the superposition to the selected atoms and stores their
// displacement from the reference as one FP32 frame row. At the end the
// covariance of the stored rows is one dense contraction over the frames,
// C = (1/T) sum_t (d_t - m)(d_t - m)^T, tiled through shared memory.
#include "lbmd_internal.cuh"

namespace lbmd {

namespace {

constexpr int kAnaThreads = 256;

// FP64 block sums of the frame moments (layout in AnaArgs).
__global__ void __launch_bounds__(kAnaThreads) k_ana_moments(AnaArgs A) {
    double acc[kAnaSums];
#pragma unroll
    for (int k = 0; k < kAnaSums; ++k) acc[k] = 0.0;
    const int stride = gridDim.x * blockDim.x;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < A.na; a += stride) {
        const double m = A.mass[a];
        const double x = A.X[a], y = A.X[A.na + a], z = A.X[2 * A.na + a];
        acc[0] += m;
        acc[1] += m * x;
        acc[2] += m * y;
        acc[3] += m * z;
        acc[4] += m * (x * x + y * y + z * z);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += stride) {
        const int a = A.sel[i];
        const double x[3] = {A.X[a], A.X[A.na + a], A.X[2 * A.na + a]};
        const double yc[3] = {A.yc[i], A.yc[A.n + i], A.yc[2 * A.n + i]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            acc[5 + d] += x[d];
            acc[8] += x[d] * x[d];
#pragma unroll
            for (int e = 0; e < 3; ++e) acc[9 + 3 * d + e] += x[d] * yc[e];
        }
    }
    __shared__ double sh[kAnaThreads / 32][kAnaSums];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kAnaSums; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kAnaSums) {
        double s = 0.0;
        for (int w = 0; w < kAnaThreads / 32; ++w) s += sh[w][threadIdx.x];
        A.partials[(size_t)blockIdx.x * kAnaSums + threadIdx.x] = s;
    }
}

// Sum of the block partials in a fixed order (one thread per moment).
__global__ void k_ana_finish(AnaArgs A, int nblocks) {
    const int k = threadIdx.x;
    if (k >= kAnaSums) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += A.partials[(size_t)b * kAnaSums + k];
    A.sums[k] = s;
}

// Superposed displacement d = R (x - xbar) + ybar - y of every selected atom,
// stored as FP32 row `frame`; its FP64 running sum feeds the mean.
__global__ void __launch_bounds__(kAnaThreads) k_ana_store(AnaArgs A, int frame, AnaFit F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const int a = A.sel[i];
    const double x[3] = {A.X[a] - F.xbar[0], A.X[A.na + a] - F.xbar[1], A.X[2 * A.na + a] - F.xbar[2]};
    float *row = A.frames + (size_t)frame * 3 * A.n;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double xf = F.R[3 * d] * x[0] + F.R[3 * d + 1] * x[1] + F.R[3 * d + 2] * x[2] + F.ybar[d];
        const double disp = xf - A.y[d * A.n + i];
        row[d * A.n + i] = (float)disp;
        A.dsum[d * A.n + i] += disp;
    }
}

// Mean displacement over the T frames (FP64 and its FP32 copy for the
// centring of the contraction) and the RMSF of each selected atom.
__global__ void __launch_bounds__(kAnaThreads) k_ana_mean_rmsf(AnaArgs A, int T, double *mean, double *rmsf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    double s2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        const int k = d * A.n + i;
        const double m = A.dsum[k] / T;
        const float mf = (float)m;
        A.meanf[k] = mf;
        if (mean) mean[k] = m;
        for (int t = 0; t < T; ++t) {
            const double e = (double)(A.frames[(size_t)t * 3 * A.n + k] - mf);
            s2 += e * e;
        }
    }
    if (rmsf) rmsf[i] = sqrt(s2 / T);
}

// C[k][l] = (1/T) sum_t (F[t][k] - m_k)(F[t][l] - m_l) over the 3n x 3n output,
// one 64 x 64 tile per block of 256 threads (4 x 4 results each), frames taken
// 16 at a time through shared memory, loads coalesced along the frame rows.
constexpr int kTile = 64, kKc = 16;
__global__ void __launch_bounds__(256) k_ana_cov(AnaArgs A, int T, float *cov) {
    __shared__ float sa[kKc][kTile], sb[kKc][kTile];
    const int M = 3 * A.n;
    const int k0 = blockIdx.y * kTile, l0 = blockIdx.x * kTile;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
    for (int t0 = 0; t0 < T; t0 += kKc) {
        for (int e = threadIdx.x; e < kKc * kTile; e += 256) {
            const int tt = e / kTile, c = e % kTile;
            const int t = t0 + tt;
            const int ka = k0 + c, lb = l0 + c;
            sa[tt][c] = (t < T && ka < M) ? A.frames[(size_t)t * M + ka] - A.meanf[ka] : 0.f;
            sb[tt][c] = (t < T && lb < M) ? A.frames[(size_t)t * M + lb] - A.meanf[lb] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int tt = 0; tt < kKc; ++tt) {
            float av[4], bv[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                av[p] = sa[tt][ty + 16 * p];
                bv[p] = sb[tt][tx + 16 * p];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
        }
        __syncthreads();
    }
    const float inv = 1.f / (float)T;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + ty + 16 * p, l = l0 + tx + 16 * q;
            if (k < M && l < M) cov[(size_t)k * M + l] = acc[p][q] * inv;
        }
}

}  // namespace

int ana_blocks(const AnaArgs &A) {
    const int n = A.na > A.n ? A.na : A.n;
    int b = (n + kAnaThreads - 1) / kAnaThreads;
    return b < 1 ? 1 : (b > 1024 ? 1024 : b);
}

cudaError_t launch_ana_moments(const AnaArgs &A, cudaStream_t s) {
    const int nb = ana_blocks(A);
    k_ana_moments<<<nb, kAnaThreads, 0, s>>>(A);
    k_ana_finish<<<1, 32, 0, s>>>(A, nb);
    return cudaGetLastError();
}

cudaError_t launch_ana_store(const AnaArgs &A, int frame, const AnaFit &F, cudaStream_t s) {
    k_ana_store<<<(A.n + kAnaThreads - 1) / kAnaThreads, kAnaThreads, 0, s>>>(A, frame, F);
    return cudaGetLastError();
}

cudaError_t launch_ana_result(const AnaArgs &A, int T, double *mean, double *rmsf, float *cov, cudaStream_t s) {
    k_ana_mean_rmsf<<<(A.n + kAnaThreads - 1) / kAnaThreads, kAnaThreads, 0, s>>>(A, T, mean, rmsf);
    if (cov) {
        const int M = 3 * A.n, g = (M + kTile - 1) / kTile;
        k_ana_cov<<<dim3(g, g), 256, 0, s>>>(A, T, cov);
    }
    return cudaGetLastError();
}

}  // namespace lbmd
