// noalloc.cu -- description length of a dense blockmodel without any
// device-memory allocation.
//
// For callers that must not allocate device memory once they are running:
// for example a serving process whose memory pool owns the whole device, or
// code with a latency budget that cannot afford cudaMalloc's implicit
// device synchronisation or its failure at an unpredictable moment.  The
// caller passes every input and the output; the only scratch (one partial
// sum per tile of M) lives in a fixed array of device memory that the
// library declares at file scope, so it exists on every GPU that loads the
// library until the process exits.
//
// It is a variant of the library's DL reduction: the same tiles and the
// same fixed summation order, with x ln x taken from FP64 log instead of the
// library's x ln x table (building that table would allocate).
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace sbp {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaTile = kNaThreads * 4;                  // entries of M per partial sum
constexpr int kNaMaxPartials = 16384;                    // scratch size (128 KB of doubles)
constexpr int64_t kNaMaxEntries = (int64_t)kNaTile * kNaMaxPartials;  // B*B <= 2^24, i.e. B <= 4096

// The shared scratch: one partial sum per tile.  Every call overwrites the
// partials it later reads, so nothing has to start at zero.
static __device__ __align__(256) double g_dl_partials[kNaMaxPartials];

constexpr int kNaMaxDevices = 64;
double *g_partials_addr[kNaMaxDevices] = {nullptr};
std::mutex g_na_mu;

__device__ __forceinline__ double xlogx64(int64_t x) { return x > 1 ? (double)x * log((double)x) : 0.0; }

__device__ double na_block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    return sh[0];
}

// one tile of M per block; the first B threads of the grid add the degree
// terms of their block
__global__ void __launch_bounds__(kNaThreads) k_dl_partial_noalloc(const int32_t *__restrict__ M, int64_t BB,
                                                                   const int32_t *__restrict__ dout,
                                                                   const int32_t *__restrict__ din, int B,
                                                                   double *__restrict__ partials) {
    __shared__ double sh[kNaThreads];
    double acc = 0.0;
    const int64_t base = (int64_t)blockIdx.x * kNaTile;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t e = base + i * kNaThreads + threadIdx.x;
        if (e < BB) acc += xlogx64(M[e]);
    }
    const int64_t g = (int64_t)blockIdx.x * kNaThreads + threadIdx.x;
    if (g < B) acc -= xlogx64(dout[g]) + xlogx64(din[g]);
    const double s = na_block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Eq. 2 from the partials, summed in a fixed order by one block
__global__ void __launch_bounds__(kNaThreads) k_dl_final_noalloc(const double *__restrict__ partials, int np, int64_t E,
                                                                 int64_t N, int B, double *__restrict__ dl) {
    __shared__ double sh[kNaThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partials[i];
    const double L = na_block_sum(acc, sh);
    if (threadIdx.x == 0) {
        double model = 0.0;
        if (E > 0) {
            const double x = (double)B * (double)B / (double)E;
            model = (double)E * ((1.0 + x) * log1p(x) - x * log(x));
        }
        dl[0] = model + (double)N * log((double)B) - L;
    }
}

// device address of the scratch array on the current device, looked up once
int partials_address(double **out) {
    int dev = 0;
    SBP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) return fail(SBP_EINVAL, "sbp_dense_dl_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_partials_addr[dev]) {
        double *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_dl_partials);
        if (e != cudaSuccess) return cuda_fail(e, "sbp_dense_dl_noalloc: cudaGetSymbolAddress");
        g_partials_addr[dev] = p;
    }
    *out = g_partials_addr[dev];
    return SBP_OK;
}

}  // namespace
}  // namespace sbp

extern "C" int sbp_dense_dl_noalloc(const int32_t *M, int32_t B, const int32_t *dout, const int32_t *din, int64_t E,
                                    int64_t N, double *dl_out, void *stream) {
    using namespace sbp;
    if (!M || !dout || !din || !dl_out) return fail(SBP_EINVAL, "sbp_dense_dl_noalloc: NULL pointer");
    if (B < 1 || (int64_t)B * B > kNaMaxEntries)
        return fail(SBP_EINVAL, "sbp_dense_dl_noalloc: B must be in [1, 4096] (the fixed scratch holds " +
                                    std::to_string(kNaMaxPartials) + " partial sums of " + std::to_string(kNaTile) +
                                    " entries)");
    if (E < 0 || N < 1) return fail(SBP_EINVAL, "sbp_dense_dl_noalloc: need E >= 0 and N >= 1");
    double *partials = nullptr;
    SBP_TRY(partials_address(&partials));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t BB = (int64_t)B * B;
    int64_t np = (BB + kNaTile - 1) / kNaTile;
    const int64_t deg_blocks = ((int64_t)B + kNaThreads - 1) / kNaThreads;
    if (np < deg_blocks) np = deg_blocks;
    k_dl_partial_noalloc<<<(unsigned)np, kNaThreads, 0, st>>>(M, BB, dout, din, B, partials);
    SBP_LAUNCHED();
    k_dl_final_noalloc<<<1, kNaThreads, 0, st>>>(partials, (int)np, E, N, B, dl_out);
    SBP_LAUNCHED();
    return SBP_OK;
}
