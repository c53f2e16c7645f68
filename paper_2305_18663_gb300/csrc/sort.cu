// sort.cu -- device-wide exclusive scan and LSD radix sort (8-bit digits).
//
// Used by the sparse blockmodel rebuild: the (b[src], b[dst]) keys of all
// edges are sorted, then run-length encoded into the nonzeros of M.
// Stable by construction: each pass keeps the order of equal digits, so the
// passes compose into a sort on the whole key.
//
// Pass structure (tile = 256 threads x 8 keys, striped: key j*256 + tid):
//   k_digit_hist: per tile, a 256-bin histogram, stored digit-major;
//   exclusive scan over the digit-major histogram gives every (digit, tile)
//   its first output position;
//   k_digit_scatter: per tile, 8 rounds of 256 keys; a key's rank among the
//   earlier keys of its digit comes from warp match/popc, per-warp digit
//   counts and a running count per digit.
#include "common.cuh"

namespace sbp {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;  // elements per thread in a scan block
constexpr int kScanBlock = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t warp_excl_scan_u32(uint32_t v, uint32_t &total) {
    const int lane = threadIdx.x & 31;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// block-wide exclusive scan of one value per thread (1024 threads)
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t *sh, uint32_t &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t wt;
    const uint32_t x = warp_excl_scan_u32(v, wt);
    if (lane == 31) sh[wid] = wt;
    __syncthreads();
    if (wid == 0) {
        const uint32_t s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
        uint32_t t2;
        const uint32_t e = warp_excl_scan_u32(s, t2);
        sh[lane] = e;
        if (lane == 0) sh[32] = t2;
    }
    __syncthreads();
    const uint32_t r = x + sh[wid];
    total = sh[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in, int64_t n,
                                                              uint32_t *__restrict__ sums) {
    __shared__ uint32_t sh[33];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    uint32_t total;
    block_excl_scan(s, sh, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// one block: exclusive scan of the block sums, in place; grand total to *total
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint32_t *__restrict__ sums, int64_t nb,
                                                            uint32_t *__restrict__ total_out) {
    __shared__ uint32_t sh[33];
    uint32_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t i0 = base + (int64_t)threadIdx.x * kScanItems;
        uint32_t v[kScanItems], s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = i0 + i < nb ? sums[i0 + i] : 0u;
            s += v[i];
        }
        uint32_t total;
        uint32_t e = block_excl_scan(s, sh, total) + carry;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            if (i0 + i < nb) sums[i0 + i] = e;
            e += v[i];
        }
        carry += total;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t *__restrict__ in, int64_t n,
                                                            const uint32_t *__restrict__ sums, uint32_t *__restrict__ out) {
    __shared__ uint32_t sh[33];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems], s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0u;
        s += v[i];
    }
    uint32_t total;
    uint32_t e = block_excl_scan(s, sh, total) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = e;
        e += v[i];
    }
}

// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

template <class K>
__device__ __forceinline__ int digit_of(K k, int shift) {
    return (int)((k >> shift) & 0xff);
}

template <class K>
__global__ void __launch_bounds__(kSortThreads) k_digit_hist(const K *__restrict__ keys, int64_t n, int shift,
                                                             int64_t ntiles, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t i = base + j * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[digit_of(keys[i], shift)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

template <class K, class V>
__global__ void __launch_bounds__(kSortThreads) k_digit_scatter(const K *__restrict__ keys, const V *__restrict__ vals,
                                                                int64_t n, int shift, int64_t ntiles,
                                                                const uint32_t *__restrict__ offs, K *__restrict__ kout,
                                                                V *__restrict__ vout) {
    __shared__ uint32_t gofs[256];
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[kSortThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    gofs[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
    run[tid] = 0;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int j = 0; j < kSortItems; ++j) {
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const int64_t i = base + j * kSortThreads + tid;
        const bool valid = i < n;
        K k = 0;
        V v = V();
        if (valid) {
            k = keys[i];
            if (vals) v = vals[i];
        }
        const int d = valid ? digit_of(k, shift) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank_w = __popc(peers & ((1u << lane) - 1u));
        if (valid && lane == __ffs(peers) - 1) wcnt[wid][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t s = run[tid];
#pragma unroll
            for (int w = 0; w < kSortThreads / 32; ++w) {
                const uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = s;
                s += c;
            }
            run[tid] = s;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = gofs[d] + wcnt[wid][d] + (uint32_t)rank_w;
            kout[pos] = k;
            if (vals) vout[pos] = v;
        }
        __syncthreads();
    }
}

}  // namespace

// Exclusive scan of n uint32 values (in may equal out).  scratch needs
// scan_scratch_words(n) words; *total_dev (device, may be NULL) gets the sum.
int64_t scan_scratch_words(int64_t n) { return (n + kScanBlock - 1) / kScanBlock + 1; }

int exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total_dev, uint32_t *scratch,
                       cudaStream_t st) {
    if (n <= 0) {
        if (total_dev) SBP_CUDA(cudaMemsetAsync(total_dev, 0, 4, st));
        return SBP_OK;
    }
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, scratch);
    SBP_LAUNCHED();
    k_scan_sums<<<1, kScanThreads, 0, st>>>(scratch, nb, total_dev);
    SBP_LAUNCHED();
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, scratch, out);
    SBP_LAUNCHED();
    return SBP_OK;
}

int64_t sort_scratch_words(int64_t n) {
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    return 256 * ntiles + scan_scratch_words(256 * ntiles);
}

// LSD radix sort on the low `bits` bits of the keys, 8 bits per pass.  The
// result lands in k0/v0 (the inputs) or k1/v1 according to the parity of
// the pass count; *in_first tells which.  vals may be NULL.
template <class K, class V>
int radix_sort(K *k0, K *k1, V *v0, V *v1, int64_t n, int bits, uint32_t *scratch, cudaStream_t st, bool *in_first) {
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    uint32_t *hist = scratch;
    uint32_t *sscr = scratch + 256 * ntiles;
    K *ks = k0, *kd = k1;
    V *vs = v0, *vd = v1;
    const int passes = (bits + 7) / 8;
    if (n > 0) {
        for (int p = 0; p < passes; ++p) {
            const int shift = 8 * p;
            k_digit_hist<K><<<(unsigned)ntiles, kSortThreads, 0, st>>>(ks, n, shift, ntiles, hist);
            SBP_LAUNCHED();
            SBP_TRY(exclusive_scan_u32(hist, hist, 256 * ntiles, nullptr, sscr, st));
            k_digit_scatter<K, V><<<(unsigned)ntiles, kSortThreads, 0, st>>>(ks, vs, n, shift, ntiles, hist, kd, vd);
            SBP_LAUNCHED();
            std::swap(ks, kd);
            std::swap(vs, vd);
        }
    }
    *in_first = (n <= 0) || (passes % 2 == 0);
    return SBP_OK;
}

template int radix_sort<uint64_t, uint64_t>(uint64_t *, uint64_t *, uint64_t *, uint64_t *, int64_t, int, uint32_t *,
                                            cudaStream_t, bool *);
template int radix_sort<uint64_t, uint32_t>(uint64_t *, uint64_t *, uint32_t *, uint32_t *, int64_t, int, uint32_t *,
                                            cudaStream_t, bool *);
template int radix_sort<uint32_t, uint64_t>(uint32_t *, uint32_t *, uint64_t *, uint64_t *, int64_t, int, uint32_t *,
                                            cudaStream_t, bool *);

}  // namespace sbp
