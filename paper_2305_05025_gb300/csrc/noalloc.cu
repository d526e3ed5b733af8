// Allocation-free FP64 fluid sums: a variant of the library's population
// reduction whose block partials live in a file-scope device array instead of
// memory from cudaMalloc. It serves callers that must not allocate device
// memory themselves or through the library: an MD engine or plugin host that
// reserves the GPU's memory up front in its own pool and forbids allocations
// from outside it, or a time-critical loop where a cudaMalloc would stall on
// an implicit device synchronisation.
//
// The scratch array holds one partial per 256-node block, so one call handles
// at most LBMD_NOALLOC_MAX_NODES nodes. Every call on a device uses the same
// array: two calls whose kernels overlap on the GPU (different streams, no
// ordering between them) race on it. Pass 1 overwrites every partial it later
// reads, so nothing has to be cleared between calls.
#include <mutex>
#include <string>

#include "lbmd_internal.cuh"

namespace lbmd {
namespace {

constexpr int kBlock = 256;
constexpr int kMaxPartials = LBMD_NOALLOC_MAX_NODES / kBlock;
constexpr int kMaxDevices = 64;

// 4 FP64 partial sums per block: sum f, sum f c_x, sum f c_y, sum f c_z.
static __device__ __align__(256) double g_partials[kMaxPartials * 4];

// Device address of g_partials, looked up once per device.
double *g_addr[kMaxDevices] = {};
std::mutex g_mutex;

__global__ void __launch_bounds__(kBlock) k_sums_pass1(const float *__restrict__ f, size_t N, double *partials) {
    const size_t n = (size_t)blockIdx.x * kBlock + threadIdx.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (n < N) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double v = (double)f[(size_t)i * N + n];
            acc[0] += v;
            acc[1] += cx(i) * v;
            acc[2] += cy(i) * v;
            acc[3] += cz(i) * v;
        }
    }
    __shared__ double sh[4][kBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 4; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) s += sh[threadIdx.x][w];
        partials[(size_t)blockIdx.x * 4 + threadIdx.x] = s;
    }
}

// One block sums the partials in a fixed order (deterministic result).
__global__ void __launch_bounds__(kBlock) k_sums_pass2(const double *partials, int nblocks, double *out) {
    __shared__ double sh[kBlock];
    for (int k = 0; k < 4; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += kBlock) s += partials[(size_t)b * 4 + k];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = kBlock / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sh[0];
        __syncthreads();
    }
}

lbmd_status noalloc_fail(lbmd_status s, const std::string &msg) {
    set_thread_error(msg);  // read back with lbmd_last_error(NULL)
    return s;
}

}  // namespace
}  // namespace lbmd

extern "C" lbmd_status lbmd_fluid_sums_noalloc(const float *f, int nx, int ny, int nz, double *out,
                                               void *cuda_stream) {
    using namespace lbmd;
    if (!f || !out) return noalloc_fail(LBMD_ERR_ARG, "f and out must be device pointers");
    if (nx < 1 || ny < 1 || nz < 1) return noalloc_fail(LBMD_ERR_ARG, "lattice sizes must be >= 1");
    const double nodes = (double)nx * ny * nz;
    if (nodes > (double)LBMD_NOALLOC_MAX_NODES)
        return noalloc_fail(LBMD_ERR_ARG, "lattice too large for lbmd_fluid_sums_noalloc: at most " +
                                              std::to_string(LBMD_NOALLOC_MAX_NODES) + " nodes (its fixed scratch)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(LBMD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(LBMD_ERR_ARG, "device index out of range");
    double *partials = nullptr;
    {
        // First call on this device (with it current): look up the device
        // address of the scratch array.
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_partials);
            if (e != cudaSuccess)
                return noalloc_fail(LBMD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_addr[dev] = (double *)p;
        }
        partials = g_addr[dev];
    }
    const size_t N = (size_t)nx * ny * nz;
    const int nblocks = (int)((N + kBlock - 1) / kBlock);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    k_sums_pass1<<<nblocks, kBlock, 0, s>>>(f, N, partials);
    k_sums_pass2<<<1, kBlock, 0, s>>>(partials, nblocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(LBMD_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return LBMD_OK;
}
