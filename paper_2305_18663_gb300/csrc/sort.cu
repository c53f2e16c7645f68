// sort.cu -- device-wide exclusive scan and LSD radix sort.
//
// Used by the sparse blockmodel rebuild: the (b[src], b[dst]) keys of all
// edges are sorted, then run-length encoded into the nonzeros of M.
// Stable by construction: each pass keeps the order of equal digits, so the
// passes compose into a sort on the whole key.
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

// one block for short arrays: exclusive scan of in into out (may alias)
__global__ void __launch_bounds__(kScanThreads) k_scan_small(const uint32_t *in, int64_t n, uint32_t *out,
                                                             uint32_t *__restrict__ total_out) {
    __shared__ uint32_t sh[33];
    uint32_t carry = 0;
    for (int64_t base = 0; base < n; base += kScanBlock) {
        const int64_t i0 = base + (int64_t)threadIdx.x * kScanItems;
        uint32_t v[kScanItems], s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = i0 + i < n ? in[i0 + i] : 0u;
            s += v[i];
        }
        uint32_t total;
        uint32_t e = block_excl_scan(s, sh, total) + carry;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            if (i0 + i < n) out[i0 + i] = e;
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
// Radix sort.  The keys are cut into G contiguous chunks, one CTA per chunk
// in both kernels of a pass:
//   k_rs_count: per chunk, a histogram of the pass's digit, stored
//     digit-major (hist[d * G + chunk]); an exclusive scan of it gives every
//     (digit, chunk) its first output position.  For the first pass of the
//     edge sort it also makes the keys (b[src] * B + b[dst]) and writes them;
//   k_rs_scatter: the chunk is walked in rounds of 4096 keys.  A key's rank
//     among the earlier keys of its digit in the round comes from warp
//     match/popc (per item) and per-warp digit counts; the round is
//     first placed in shared memory in digit order, then written out with
//     consecutive threads on consecutive positions of each digit's run, so
//     the global writes coalesce.
// Digits are up to 9 bits wide (512 bins), chosen so that the pass count is
// the smallest possible: ceil(bits / 9).
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 16;                       // keys per lane per round
constexpr int kRsRound = kRsThreads * kRsItems;    // keys per round
constexpr int kRsMaxBins = 512;
constexpr int64_t kRsMaxChunks = 2048;

template <class K, bool EDGES>
__device__ __forceinline__ K rs_key(const K *__restrict__ keys, const EdgeKeys &ek, int64_t i) {
    if constexpr (EDGES)
        return (K)((uint64_t)ek.b[ek.esrc[i]] * ek.B + (uint64_t)ek.b[ek.oc[i]]);
    else
        return keys[i];
}

template <class K, bool EDGES>
__global__ void __launch_bounds__(kRsThreads) k_rs_count(const K *__restrict__ keys, EdgeKeys ek, int64_t n,
                                                         int64_t chunk, int shift, int nbins, int G,
                                                         uint32_t *__restrict__ hist, K *__restrict__ kout) {
    __shared__ uint32_t h[kRsMaxBins];
    for (int d = threadIdx.x; d < nbins; d += kRsThreads) h[d] = 0;
    __syncthreads();
    const int64_t begin = (int64_t)blockIdx.x * chunk;
    const int64_t end = begin + chunk < n ? begin + chunk : n;
    const uint64_t mask = (uint64_t)nbins - 1;
    for (int64_t base = begin; base < end; base += 4 * kRsThreads) {
        K k[4];
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t i = base + j * kRsThreads + threadIdx.x;
            ok[j] = i < end;
            k[j] = ok[j] ? rs_key<K, EDGES>(keys, ek, i) : (K)0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (ok[j]) {
                if (EDGES) kout[base + j * kRsThreads + threadIdx.x] = k[j];
                atomicAdd(&h[(int)(((uint64_t)k[j] >> shift) & mask)], 1u);
            }
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nbins; d += kRsThreads) hist[(int64_t)d * G + blockIdx.x] = h[d];
}

template <class K, class V>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const K *__restrict__ keys, const V *__restrict__ vals,
                                                           int64_t n, int64_t chunk, int shift, int nbins, int G,
                                                           const uint32_t *__restrict__ offs, K *__restrict__ kout,
                                                           V *__restrict__ vout) {
    extern __shared__ __align__(16) unsigned char rs_stage[];
    K *sk = reinterpret_cast<K *>(rs_stage);                              // [kRsRound]
    V *sv = reinterpret_cast<V *>(rs_stage + (size_t)kRsRound * sizeof(K));  // [kRsRound], with vals
    __shared__ uint32_t run[kRsMaxBins];     // next output position of each digit
    __shared__ uint32_t lstart[kRsMaxBins];  // first staged slot of each digit in this round
    __shared__ uint32_t wc[kRsWarps][kRsMaxBins];
    __shared__ uint32_t wsum[kRsWarps];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const uint64_t mask = (uint64_t)nbins - 1;
    for (int d = tid; d < nbins; d += kRsThreads) run[d] = offs[(int64_t)d * G + blockIdx.x];
    const int64_t begin = (int64_t)blockIdx.x * chunk;
    const int64_t end = begin + chunk < n ? begin + chunk : n;
    const int d0 = 2 * tid;  // this thread's pair of digits in the digit scan
    for (int64_t base = begin; base < end; base += kRsRound) {
        for (int d = tid; d < nbins; d += kRsThreads) {
#pragma unroll
            for (int x = 0; x < kRsWarps; ++x) wc[x][d] = 0;
        }
        __syncthreads();
        // warp w holds keys [base + 512 w, base + 512 w + 512), item j at lane
        // offset 32 j: index order is (warp, item, lane)
        K k[kRsItems];
        V v[kRsItems];
        int dg[kRsItems];
        uint32_t rk[kRsItems];
#pragma unroll
        for (int j = 0; j < kRsItems; ++j) {
            const int64_t i = base + (int64_t)w * (32 * kRsItems) + j * 32 + lane;
            const bool ok = i < end;
            k[j] = ok ? keys[i] : (K)0;
            v[j] = (vals && ok) ? vals[i] : V();
            dg[j] = ok ? (int)(((uint64_t)k[j] >> shift) & mask) : -1;
        }
#pragma unroll
        for (int j = 0; j < kRsItems; ++j) {
            const unsigned peers = __match_any_sync(0xffffffffu, dg[j]);
            const uint32_t before = dg[j] >= 0 ? wc[w][dg[j]] : 0u;
            rk[j] = before + (uint32_t)__popc(peers & lt);
            __syncwarp();
            if (dg[j] >= 0 && lane == __ffs(peers) - 1) wc[w][dg[j]] = before + (uint32_t)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive prefix over the warps, and the round's total
        uint32_t t0 = 0, t1 = 0;
        if (d0 < nbins) {
#pragma unroll
            for (int x = 0; x < kRsWarps; ++x) {
                const uint32_t c0 = wc[x][d0], c1 = wc[x][d0 + 1];
                wc[x][d0] = t0;
                wc[x][d0 + 1] = t1;
                t0 += c0;
                t1 += c1;
            }
        }
        // block exclusive scan of the digit totals, in digit order
        uint32_t incl = t0 + t1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        uint32_t ex = incl - (t0 + t1);
        for (int x = 0; x < w; ++x) ex += wsum[x];
        if (d0 < nbins) {
            lstart[d0] = ex;
            lstart[d0 + 1] = ex + t0;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kRsItems; ++j) {
            if (dg[j] >= 0) {
                const uint32_t lp = lstart[dg[j]] + wc[w][dg[j]] + rk[j];
                sk[lp] = k[j];
                if (vals) sv[lp] = v[j];
            }
        }
        __syncthreads();
        const int cnt = (int)(end - base < kRsRound ? end - base : kRsRound);
        for (int x = tid; x < cnt; x += kRsThreads) {
            const K key = sk[x];
            const int d = (int)(((uint64_t)key >> shift) & mask);
            const uint32_t pos = run[d] + (uint32_t)x - lstart[d];
            kout[pos] = key;
            if (vals) vout[pos] = sv[x];
        }
        __syncthreads();
        if (d0 < nbins) {
            run[d0] += t0;
            run[d0 + 1] += t1;
        }
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
    if (n <= 8 * kScanBlock) {
        k_scan_small<<<1, kScanThreads, 0, st>>>(in, n, out, total_dev);
        SBP_LAUNCHED();
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

namespace {

// chunk length (a whole number of rounds) and chunk count for n keys
void rs_chunks(int64_t n, int64_t *chunk, int *G) {
    int64_t rounds = (n + kRsRound - 1) / kRsRound;
    if (rounds < 1) rounds = 1;
    const int64_t per = (rounds + kRsMaxChunks - 1) / kRsMaxChunks;
    *chunk = per * kRsRound;
    *G = (int)((n + *chunk - 1) / *chunk);
    if (*G < 1) *G = 1;
}

template <class K, class V>
size_t rs_stage_bytes(bool with_vals) {
    return (size_t)kRsRound * (sizeof(K) + (with_vals ? sizeof(V) : 0));
}

// one pass: keys from ks (or, with ek.b set, made from the edge list and
// written to kmade first), digits [shift, shift + nbits)
template <class K, class V>
int rs_pass(const K *ks, const V *vs, const EdgeKeys &ek, K *kmade, int64_t n, int shift, int nbits, K *kd, V *vd,
            uint32_t *scratch, cudaStream_t st) {
    int64_t chunk;
    int G;
    rs_chunks(n, &chunk, &G);
    const int nbins = 1 << nbits;
    uint32_t *hist = scratch;
    uint32_t *sscr = scratch + (int64_t)kRsMaxBins * kRsMaxChunks;
    if (ek.b) {
        k_rs_count<K, true><<<G, kRsThreads, 0, st>>>(nullptr, ek, n, chunk, shift, nbins, G, hist, kmade);
        ks = kmade;
    } else {
        k_rs_count<K, false><<<G, kRsThreads, 0, st>>>(ks, ek, n, chunk, shift, nbins, G, hist, nullptr);
    }
    SBP_LAUNCHED();
    SBP_TRY(exclusive_scan_u32(hist, hist, (int64_t)nbins * G, nullptr, sscr, st));
    const size_t smem = rs_stage_bytes<K, V>(vs != nullptr);
    // the staging area plus the static tables pass the default 48 KB limit
    SBP_TRY(ensure_dyn_smem((const void *)k_rs_scatter<K, V>, smem));
    k_rs_scatter<K, V><<<G, kRsThreads, smem, st>>>(ks, vs, n, chunk, shift, nbins, G, hist, kd, vd);
    SBP_LAUNCHED();
    return SBP_OK;
}

}  // namespace

int64_t sort_scratch_words(int64_t) {
    return (int64_t)kRsMaxBins * kRsMaxChunks + scan_scratch_words((int64_t)kRsMaxBins * kRsMaxChunks);
}

int sort_chunk_count(int64_t n) {
    int64_t chunk;
    int G;
    rs_chunks(n, &chunk, &G);
    return G;
}

int64_t sort_chunk_length(int64_t n) {
    int64_t chunk;
    int G;
    rs_chunks(n, &chunk, &G);
    return chunk;
}

// Stable LSD radix sort on the low `bits` bits of the keys, ceil(bits / 9)
// passes.  The result lands in k0/v0 or k1/v1 according to the parity of the
// pass count; *in_first tells which.  vals may be NULL.  With `edges`, the
// first pass makes the keys from the edge list and writes them to k0 (whose
// contents on entry are ignored).
template <class K, class V>
int radix_sort(K *k0, K *k1, V *v0, V *v1, int64_t n, int bits, uint32_t *scratch, cudaStream_t st, bool *in_first,
               const EdgeKeys *edges) {
    const int passes = (bits + 8) / 9;
    const int width = (bits + passes - 1) / passes;
    K *ks = k0, *kd = k1;
    V *vs = v0, *vd = v1;
    const EdgeKeys none{};
    if (n > 0) {
        for (int p = 0; p < passes; ++p) {
            const int shift = p * width;
            const int nbits = bits - shift < width ? bits - shift : width;
            // the first pass of the edge sort makes the keys into k0 (= ks)
            SBP_TRY((rs_pass<K, V>(ks, vs, (p == 0 && edges) ? *edges : none, ks, n, shift, nbits, kd, vd, scratch, st)));
            std::swap(ks, kd);
            std::swap(vs, vd);
        }
    }
    *in_first = (n <= 0) || (passes % 2 == 0);
    return SBP_OK;
}

#define SBP_RS_INST(K, V) \
    template int radix_sort<K, V>(K *, K *, V *, V *, int64_t, int, uint32_t *, cudaStream_t, bool *, const EdgeKeys *);
SBP_RS_INST(uint64_t, uint64_t)
SBP_RS_INST(uint64_t, uint32_t)
SBP_RS_INST(uint32_t, uint64_t)
SBP_RS_INST(uint32_t, uint32_t)
#undef SBP_RS_INST

}  // namespace sbp
