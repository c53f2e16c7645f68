// xlogx_table.cu -- tabulated f(x) = x ln x in 128-bit fixed point.
//
// Every term of the log-likelihood (Eq. 1) and of its changes is f at a
// non-negative integer count: an entry of M or a block degree.  The table
// holds round(x ln x * 2^64) for x < X as signed 128-bit integers, so a
// change f(x+k) - f(x) is one exact integer subtraction and sums of them
// carry no rounding at all.  Entries are computed on the host in long
// double (64-bit or wider significand) with logl, so each is within about
// 2^-63 * x ln x of the true value; counts at or beyond X fall back to FP64
// arithmetic in the kernels.
//
// One table per device, grown on demand (X is a power of two, at most
// kMaxTable), kept until the process exits.
#include <cmath>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace sbp {
namespace {

constexpr int kMaxDevices = 64;
struct TableSlot {
    __int128 *dev = nullptr;
    int64_t size = 0;
};
TableSlot g_tables[kMaxDevices];
std::mutex g_mu;

void fill(std::vector<__int128> &t, int64_t lo, int64_t hi) {
    const long double two64 = 18446744073709551616.0L;  // 2^64
    for (int64_t x = lo; x < hi; ++x) {
        if (x < 2) {
            t[(size_t)x] = 0;
            continue;
        }
        const long double v = (long double)x * logl((long double)x);  // > 0
        const long double ip = floorl(v);
        long double frac = (v - ip) * two64;
        long double fr = floorl(frac + 0.5L);
        unsigned __int128 whole = (unsigned __int128)(uint64_t)ip << 64;
        if (fr >= two64) {
            whole += (unsigned __int128)1 << 64;
            fr = 0.0L;
        }
        whole += (unsigned __int128)(uint64_t)fr;
        t[(size_t)x] = (__int128)whole;
    }
}

}  // namespace

int xlogx_table(int64_t need, const __int128 **table, int64_t *size) {
    int dev = 0;
    SBP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(SBP_EINVAL, "device index out of range");
    int64_t want = 1 << 12;
    if (need > kMaxTable) need = kMaxTable;
    while (want < need) want <<= 1;
    std::lock_guard<std::mutex> lock(g_mu);
    TableSlot &slot = g_tables[dev];
    if (slot.size < want) {
        std::vector<__int128> host((size_t)want);
        unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> th;
        for (unsigned i = 0; i < nt; ++i)
            th.emplace_back(fill, std::ref(host), want * i / nt, want * (i + 1) / nt);
        for (auto &x : th) x.join();
        __int128 *d = nullptr;
        if (cudaMalloc(&d, (size_t)want * sizeof(__int128)) != cudaSuccess) {
            cudaGetLastError();
            return fail(SBP_ENOMEM, "cudaMalloc failed for the x ln x table");
        }
        SBP_CUDA(cudaMemcpy(d, host.data(), (size_t)want * sizeof(__int128), cudaMemcpyHostToDevice));
        // a smaller table may still be in use by work queued on another
        // stream, so it is left allocated (at most a doubling series)
        slot.dev = d;
        slot.size = want;
    }
    *table = slot.dev;
    *size = slot.size;
    return SBP_OK;
}

}  // namespace sbp
