// sparse.cu -- the blockmodel as sparse rows and columns (B > dense_max_B).
//
// Section III-A (a)-(b): M held as per-row hashed sparse rows plus a stored
// transpose.  Rebuilt from the assignment by sort plus segmented count:
//   1. key of every edge = b[src] * B + b[dst], sorted.  The sort is a
//      counting sort over the B x B key space when that space is small
//      (the edge keys need no values, so its histogram already holds the
//      run lengths); otherwise an LSD radix sort of the keys;
//   2. run-length encoding gives the nonzeros (r, c, M[r][c]) in row order;
//   3. CSR: row offsets by a row histogram and scan, the inclusive prefix of
//      the counts inside each row (the proposal CDF over row u);
//   4. CSC: a stable radix sort of the nonzeros by column keeps ascending
//      rows inside each column; offsets and prefixes as for the rows;
//   5. per-row open-addressing tables (capacity the power of two at least
//      twice the row's length; each slot holds the key and the count, so a
//      probe is one 8-byte load) for M[r][c] lookups;
//   6. block degrees from the last prefix of each row / column; DL as an
//      exact fixed-point sum over the nonzeros.
#include <algorithm>

#include "apply.cuh"

namespace sbp {

namespace {

constexpr int kT = 256;

int grid_of(int64_t work, int cap) {
    int64_t g = (work + kT - 1) / kT;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// Run-length encoding of the sorted keys, chunk by chunk: count the run
// heads per chunk, scan, then write each run's start, column and row.  A
// thread takes 16 consecutive keys per round (a round is 4096 keys; chunks
// are whole rounds).
constexpr int kRleItems = 16;
constexpr int kRleRound = kT * kRleItems;

// keys [i0, i0 + 16) with i0 a multiple of 16, as 16-byte loads
template <class K>
__device__ __forceinline__ void load16(const K *__restrict__ keys, int64_t i0, K (&k)[kRleItems]) {
    const uint4 *p = reinterpret_cast<const uint4 *>(keys + i0);
    constexpr int nv = kRleItems * (int)sizeof(K) / 16;
    uint4 tmp[nv];
#pragma unroll
    for (int x = 0; x < nv; ++x) tmp[x] = p[x];
    const K *t = reinterpret_cast<const K *>(tmp);
#pragma unroll
    for (int j = 0; j < kRleItems; ++j) k[j] = t[j];
}

// head flags of the thread's keys in the round starting at base: bit j set
// when key i0 + j starts a run
template <class K>
__device__ __forceinline__ uint32_t rle_heads(const K *__restrict__ keys, int64_t i0, int64_t end, K (&k)[kRleItems]) {
    uint32_t hm = 0;
    if (i0 >= end) return 0;
    if (i0 + kRleItems <= end) {
        load16<K>(keys, i0, k);
    } else {
#pragma unroll
        for (int j = 0; j < kRleItems; ++j) k[j] = i0 + j < end ? keys[i0 + j] : (K)0;
    }
    K prev = i0 > 0 ? keys[i0 - 1] : (K)0;
#pragma unroll
    for (int j = 0; j < kRleItems; ++j) {
        if (i0 + j < end && (i0 + j == 0 || k[j] != prev)) hm |= 1u << j;
        prev = k[j];
    }
    return hm;
}

template <class K>
__global__ void __launch_bounds__(kT) k_rle_count(const K *__restrict__ keys, int64_t n, int64_t chunk,
                                                  uint32_t *__restrict__ cnt) {
    __shared__ uint32_t sh[kT / 32];
    const int64_t begin = (int64_t)blockIdx.x * chunk;
    const int64_t end = begin + chunk < n ? begin + chunk : n;
    uint32_t c = 0;
    for (int64_t base = begin; base < end; base += kRleRound) {
        K k[kRleItems];
        c += (uint32_t)__popc(rle_heads<K>(keys, base + (int64_t)threadIdx.x * kRleItems, end, k));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kT / 32; ++w) t += sh[w];
        cnt[blockIdx.x] = t;
    }
}

template <class K>
__global__ void __launch_bounds__(kT) k_rle_emit(const K *__restrict__ keys, int64_t n, int64_t chunk,
                                                 const uint32_t *__restrict__ cstart, uint64_t B,
                                                 uint32_t *__restrict__ start, int32_t *__restrict__ col,
                                                 int32_t *__restrict__ rowof, uint32_t *__restrict__ rowcnt) {
    __shared__ uint32_t wsum[kT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t begin = (int64_t)blockIdx.x * chunk;
    const int64_t end = begin + chunk < n ? begin + chunk : n;
    uint32_t running = cstart[blockIdx.x];
    for (int64_t base = begin; base < end; base += kRleRound) {
        const int64_t i0 = base + (int64_t)threadIdx.x * kRleItems;
        K k[kRleItems];
        uint32_t hm = rle_heads<K>(keys, i0, end, k);
        const uint32_t c = (uint32_t)__popc(hm);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        uint32_t before = incl - c, total = 0;
#pragma unroll
        for (int x = 0; x < kT / 32; ++x) {
            const uint32_t t = wsum[x];
            before += x < w ? t : 0u;
            total += t;
        }
        uint32_t p = running + before;
#pragma unroll
        for (int j = 0; j < kRleItems; ++j) {
            if ((hm >> j) & 1u) {
                const uint64_t key = (uint64_t)k[j];
                const uint64_t r = key / B;
                start[p] = (uint32_t)(i0 + j);
                col[p] = (int32_t)(key - r * B);
                rowof[p] = (int32_t)r;
                atomicAdd(&rowcnt[r], 1u);
                ++p;
            }
        }
        running += total;
        __syncthreads();
    }
}

// Counting-sort form (small B x B key space): the cell counts are the run
// lengths.  One warp per row: number of nonzero cells, then (after the scan
// of those numbers) the row's nonzeros in ascending column with their
// in-row inclusive prefix; the row total is dout.
__global__ void k_cell_rowcount(const int32_t *__restrict__ cells, int B, uint32_t *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < B; r += nw) {
        uint32_t c = 0;
        for (int c0 = 0; c0 < B; c0 += 32) {
            const int col = c0 + lane;
            c += (uint32_t)__popc(__ballot_sync(0xffffffffu, col < B && cells[r * B + col] != 0));
        }
        if (lane == 0) cnt[r] = c;
    }
}

__global__ void k_cell_compact(const int32_t *__restrict__ cells, int B, const uint32_t *__restrict__ rp,
                               int32_t *__restrict__ rc, int32_t *__restrict__ rv, int32_t *__restrict__ rowof,
                               uint32_t *__restrict__ rpre, int32_t *__restrict__ dout) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < B; r += nw) {
        uint32_t p = rp[r], carry = 0;
        for (int c0 = 0; c0 < B; c0 += 32) {
            const int col = c0 + lane;
            const uint32_t v = col < B ? (uint32_t)cells[r * B + col] : 0u;
            const unsigned nz = __ballot_sync(0xffffffffu, v != 0);
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (v != 0) {
                const uint32_t q = p + (uint32_t)__popc(nz & ((1u << lane) - 1u));
                rc[q] = col;
                rv[q] = (int32_t)v;
                rowof[q] = (int32_t)r;
                rpre[q] = carry + incl;
            }
            p += (uint32_t)__popc(nz);
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) dout[r] = (int32_t)carry;
    }
}

// Small B (at most kSmallRowsB blocks): the rebuild from the cell counts in
// four kernels with no host round trip -- CSR (offsets, columns, counts,
// in-row prefixes, dout), CSC the same by column (rows ascending), the
// per-row hash tables, the per-block scalars and DL (Eq. 2, exact fixed-point
// sums, the same integer L as the general path).  The nonzero count stays on
// the device.
constexpr int kSmallRowsB = 1024;
constexpr int kSmallThreads = 1024;

__device__ uint32_t cta_excl_scan_1024(uint32_t v, uint32_t *sh, uint32_t *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        const uint32_t t = sh[lane];
        uint32_t z = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        sh[lane] = z - t;
        if (lane == 31) sh[32] = z;
    }
    __syncthreads();
    const uint32_t r = sh[w] + x - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

// (1) row and column lengths: a warp per row (warps [0, B)) or per column
// (warps [B, 2B))
__global__ void k_small_lengths(const int32_t *__restrict__ cells, int B, uint32_t *__restrict__ rlen,
                                uint32_t *__restrict__ clen) {
    const int lane = threadIdx.x & 31;
    const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (w >= 2 * B) return;
    const bool col = w >= B;
    const int i = col ? w - B : w;
    uint32_t c = 0;
    for (int j0 = 0; j0 < B; j0 += 32 * 8) {
        int32_t x[8];  // eight chunks of the row (or column) in flight
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = j0 + 32 * q + lane;
            x[q] = j < B ? (col ? cells[j * B + i] : cells[i * B + j]) : 0;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) c += (uint32_t)__popc(__ballot_sync(0xffffffffu, x[q] != 0));
    }
    if (lane == 0) (col ? clen : rlen)[i] = c;
}

// (2) one CTA: offsets of the rows, the columns and the row tables
__global__ void __launch_bounds__(kSmallThreads) k_small_offsets(const uint32_t *__restrict__ rlen,
                                                                 const uint32_t *__restrict__ clen, int B,
                                                                 uint32_t *__restrict__ rp, uint32_t *__restrict__ cp,
                                                                 uint32_t *__restrict__ hoff,
                                                                 int64_t *__restrict__ nnz_out) {
    __shared__ uint32_t sh[33];
    const int tid = threadIdx.x;
    uint32_t total;
    const uint32_t lr = tid < B ? rlen[tid] : 0u;
    uint32_t ex = cta_excl_scan_1024(lr, sh, &total);
    if (tid < B) rp[tid] = ex;
    if (tid == 0) {
        rp[B] = total;
        *nnz_out = total;
    }
    ex = cta_excl_scan_1024(tid < B ? clen[tid] : 0u, sh, &total);
    if (tid < B) cp[tid] = ex;
    if (tid == 0) cp[B] = total;
    uint32_t cap = 0;
    if (tid < B) {
        cap = 2;
        while (cap < 2 * lr) cap <<= 1;
    }
    ex = cta_excl_scan_1024(cap, sh, &total);
    if (tid < B) hoff[tid] = ex;
    if (tid == 0) hoff[B] = total;
}

// (3) a warp per row (warps [0, B)): CSR entries, in-row prefixes, dout,
// the row's hash table (cleared, then filled by the same warp); a warp per
// column (warps [B, 2B)): CSC entries, prefixes, din.  Per warp, its share
// of L (Eq. 1): + x ln x of the row's counts, - dout ln dout or
// - din ln din, in fixed point.
__global__ void k_small_fill(const int32_t *__restrict__ cells, int B, const uint32_t *__restrict__ rp,
                             const uint32_t *__restrict__ cp, const uint32_t *__restrict__ hoff,
                             int32_t *__restrict__ rc, int32_t *__restrict__ rv, int32_t *__restrict__ rowof,
                             uint32_t *__restrict__ rpre, int32_t *__restrict__ cr, int32_t *__restrict__ cv,
                             uint32_t *__restrict__ cpre, int2 *__restrict__ hkv,
                             int32_t *__restrict__ dout, int32_t *__restrict__ din, const __int128 *__restrict__ T,
                             int64_t XT, __int128 *__restrict__ lpart, double *__restrict__ lfb,
                             int32_t *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (w >= 2 * B) return;
    const bool col = w >= B;
    const int i = col ? w - B : w;
    __int128 f = 0;
    double fb = 0.0;  // counts beyond the table, in FP64
    uint32_t p = col ? cp[i] : rp[i], carry = 0;
    const uint32_t off = col ? 0u : hoff[i], cap = col ? 0u : hoff[i + 1] - off;
    if (!col)
        for (uint32_t q = lane; q < cap; q += 32) hkv[off + q] = make_int2(-1, 0);
    __syncwarp();
    for (int j8 = 0; j8 < B; j8 += 32 * 8) {
        uint32_t x8[8];  // eight chunks of the row (or column) in flight
#pragma unroll
        for (int cq = 0; cq < 8; ++cq) {
            const int j = j8 + 32 * cq + lane;
            x8[cq] = j < B ? (uint32_t)(col ? cells[j * B + i] : cells[i * B + j]) : 0u;
        }
#pragma unroll
        for (int cq = 0; cq < 8; ++cq) {
            const int j0 = j8 + 32 * cq;
            if (j0 >= B) break;
            const int j = j0 + lane;
            const uint32_t v = x8[cq];
            const unsigned nz = __ballot_sync(0xffffffffu, v != 0);
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (v != 0) {
                const uint32_t q = p + (uint32_t)__popc(nz & ((1u << lane) - 1u));
                if (col) {
                    cr[q] = j;
                    cv[q] = (int32_t)v;
                    cpre[q] = carry + incl;
                } else {
                    rc[q] = j;
                    rv[q] = (int32_t)v;
                    rowof[q] = i;
                    rpre[q] = carry + incl;
                    if ((int64_t)v < XT) f += T[v];
                    else fb += (double)v * log((double)v);
                    uint32_t h = sparse_hash(j) & (cap - 1);
                    bool done = false;
                    for (uint32_t t = 0; t < cap; ++t) {
                        if (atomicCAS(&hkv[off + h].x, -1, j) == -1) {
                            hkv[off + h].y = (int32_t)v;
                            done = true;
                            break;
                        }
                        h = (h + 1) & (cap - 1);
                    }
                    if (!done) record_status(status, SBP_EHASHFULL);
                }
            }
            p += (uint32_t)__popc(nz);
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    f = warp_sum_128(f);
    fb = warp_sum(fb);
    if (lane == 0) {
        (col ? din : dout)[i] = (int32_t)carry;
        if ((int64_t)carry < XT) f -= T[carry];
        else fb -= (double)carry * log((double)carry);
        lpart[w] = f;
        lfb[w] = fb;
    }
}

// (4) one CTA: per-block scalars and DL from the warps' shares of L (fixed
// order, exact)
__global__ void __launch_bounds__(kSmallThreads) k_small_finish(const int32_t *__restrict__ dout,
                                                                const int32_t *__restrict__ din, int B,
                                                                const __int128 *__restrict__ lpart,
                                                                const double *__restrict__ lfb,
                                                                int32_t *__restrict__ dsum, double *__restrict__ rcp,
                                                                float *__restrict__ rcp32, int64_t E, int64_t N,
                                                                double *__restrict__ dl) {
    __shared__ __int128 red[kSmallThreads / 32];
    __shared__ double redd[kSmallThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    __int128 f = 0;
    double fb = 0.0;
    for (int u = tid; u < B; u += kSmallThreads) {
        const int64_t d = (int64_t)dout[u] + din[u];
        dsum[u] = (int32_t)d;
        rcp[u] = 1.0 / ((double)d + (double)B);
        rcp32[u] = 1.0f / ((float)d + (float)B);
    }
    for (int q = tid; q < 2 * B; q += kSmallThreads) {
        f += lpart[q];
        fb += lfb[q];
    }
    f = warp_sum_128(f);
    fb = warp_sum(fb);
    if (lane == 0) {
        red[w] = f;
        redd[w] = fb;
    }
    __syncthreads();
    if (tid == 0) {
        __int128 L = 0;
        double Lb = 0.0;
        for (int q = 0; q < kSmallThreads / 32; ++q) {
            L += red[q];
            Lb += redd[q];
        }
        dl[0] = dl_eq2(E, N, B, fix_to_double(L) + Lb);
    }
}

__global__ void k_run_counts(const uint32_t *__restrict__ start, int64_t nnz, int64_t n, int32_t *__restrict__ val) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = p + 1 < nnz ? start[p + 1] : (uint32_t)n;
        val[p] = (int32_t)(e - start[p]);
    }
}

// one warp per row: inclusive prefix of the row's counts; the last one is
// the row's degree
__global__ void k_row_prefix(const uint32_t *__restrict__ ptr, const int32_t *__restrict__ val, int64_t R,
                             uint32_t *__restrict__ pre, int32_t *__restrict__ deg) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < R; r += nw) {
        const uint32_t a = ptr[r], z = ptr[r + 1];
        uint32_t carry = 0;
        for (uint32_t b0 = a; b0 < z; b0 += 32) {
            const uint32_t i = b0 + lane;
            uint32_t x = i < z ? (uint32_t)val[i] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            x += carry;
            if (i < z) pre[i] = x;
            carry = __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) deg[r] = (int32_t)carry;
    }
}

// CSC source: key = column, value = (row << 32) | count, in CSR order
__global__ void k_csc_src(const int32_t *__restrict__ col, const int32_t *__restrict__ rowof,
                          const int32_t *__restrict__ val, int64_t nnz, uint32_t *__restrict__ ckey,
                          uint64_t *__restrict__ cval, uint32_t *__restrict__ colcnt) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        ckey[p] = (uint32_t)col[p];
        cval[p] = ((uint64_t)(uint32_t)rowof[p] << 32) | (uint32_t)val[p];
        atomicAdd(&colcnt[col[p]], 1u);
    }
}

__global__ void k_csc_unpack(const uint64_t *__restrict__ cval, int64_t nnz, int32_t *__restrict__ crow,
                             int32_t *__restrict__ cv) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        crow[p] = (int32_t)(cval[p] >> 32);
        cv[p] = (int32_t)(cval[p] & 0xffffffffu);
    }
}

__global__ void k_hash_caps(const uint32_t *__restrict__ ptr, int64_t R, uint32_t *__restrict__ caps) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t len = ptr[r + 1] - ptr[r];
        uint32_t c = 2;
        while (c < 2 * len) c <<= 1;
        caps[r] = c;
    }
}

__global__ void k_hash_fill(const uint32_t *__restrict__ ptr, const int32_t *__restrict__ col,
                            const int32_t *__restrict__ val, const int32_t *__restrict__ rowof, int64_t nnz,
                            const uint32_t *__restrict__ hoff, int2 *__restrict__ hkv,
                            int32_t *__restrict__ status) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int r = rowof[p], c = col[p];
        const uint32_t off = hoff[r], cap = hoff[r + 1] - off;
        uint32_t h = sparse_hash(c) & (cap - 1);
        bool done = false;
        for (uint32_t q = 0; q < cap; ++q) {
            if (atomicCAS(&hkv[off + h].x, -1, c) == -1) {
                hkv[off + h].y = val[p];
                done = true;
                break;
            }
            h = (h + 1) & (cap - 1);
        }
        if (!done) record_status(status, SBP_EHASHFULL);
    }
}

__global__ void k_block_scalars(const int32_t *__restrict__ dout, const int32_t *__restrict__ din, int B,
                                int32_t *__restrict__ dsum, double *__restrict__ rcp, float *__restrict__ rcp32) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < B; u += gridDim.x * blockDim.x) {
        const int64_t d = (int64_t)dout[u] + din[u];
        dsum[u] = (int32_t)d;
        rcp[u] = 1.0 / ((double)d + (double)B);
        rcp32[u] = 1.0f / ((float)d + (float)B);
    }
}

int bits_for(uint64_t maxval) {
    int b = 1;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b;
}

template <class T>
int alloc(sbp_model *m, T **p, int64_t count) {
    model_free(*p, m->stream);
    *p = nullptr;
    if (model_alloc((void **)p, (size_t)(count > 0 ? count : 1) * sizeof(T), m->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(SBP_ENOMEM, "cudaMalloc failed for the sparse blockmodel");
    }
    return SBP_OK;
}

// the 32 pivots of every row (threads [0, 32 B)) and column (threads
// [32 B, 64 B)) of the sparse M: pivot i is the row's inclusive prefix at the
// end of its i-th segment of ceil(len / 32) entries, all ones past the row
__global__ void k_sparse_pivots(const uint32_t *__restrict__ rp, const uint32_t *__restrict__ rpre,
                                const uint32_t *__restrict__ cp, const uint32_t *__restrict__ cpre, int B,
                                uint32_t *__restrict__ rpc, uint32_t *__restrict__ cpc) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= 64 * (int64_t)B) return;
    const bool col = x >= 32 * (int64_t)B;
    const int64_t y = col ? x - 32 * (int64_t)B : x;
    const int u = (int)(y >> 5), i = (int)(y & 31);
    const uint32_t *p = col ? cp : rp;
    const uint32_t *pre = col ? cpre : rpre;
    const uint32_t lo = p[u], len = p[u + 1] - lo;
    const uint32_t step = (len + 31) / 32;
    uint32_t v = 0xffffffffu;
    if ((uint32_t)i * step < len) {
        const uint32_t end = ((uint32_t)i + 1) * step < len ? ((uint32_t)i + 1) * step : len;
        v = pre[lo + end - 1];
    }
    (col ? cpc : rpc)[y] = v;
}

}  // namespace

// The rebuild counts cells instead of sorting keys when the B x B key space
// is small: at most 2^26 cells (B <= 8192) and at most 8 E + 2^20, so that
// zeroing and scanning the cells stays cheaper than sorting E keys.
bool sparse_by_count(int64_t B, int64_t E) {
    const int64_t cells = B * B;
    return cells <= (int64_t(1) << 26) && cells <= 8 * E + (int64_t(1) << 20);
}

int ensure_sparse_capacity(sbp_model *m, int32_t B) {
    sbp_model::Sparse &S = m->sp;
    const int64_t E = m->g->m > 0 ? m->g->m : 1;
    if (S.cap_e < E) {
        SBP_TRY(alloc(m, &S.key0, E));
        SBP_TRY(alloc(m, &S.key1, E));
        SBP_TRY(alloc(m, &S.start, E));
        SBP_TRY(alloc(m, &S.rc, E));
        SBP_TRY(alloc(m, &S.rv, E));
        SBP_TRY(alloc(m, &S.rowof, E));
        SBP_TRY(alloc(m, &S.rpre, E));
        SBP_TRY(alloc(m, &S.cr, E));
        SBP_TRY(alloc(m, &S.cv, E));
        SBP_TRY(alloc(m, &S.cpre, E));
        SBP_TRY(alloc(m, &S.ckey0, E));
        SBP_TRY(alloc(m, &S.ckey1, E));
        SBP_TRY(alloc(m, &S.cval0, E));
        SBP_TRY(alloc(m, &S.cval1, E));
        SBP_TRY(alloc(m, &S.hkv, 4 * E + 2 * (int64_t)m->g->n));
        const int64_t w = std::max(std::max(sort_scratch_words(E), scan_scratch_words(E) + 4),
                                   scan_scratch_words((int64_t)m->g->n + 1) + 4);
        SBP_TRY(alloc(m, &S.scratch, w + 1024));
        SBP_TRY(alloc(m, &S.nnz_dev, 1));
        S.cap_e = E;
    }
    if (sparse_by_count(B, m->g->m) && S.cap_cells < (int64_t)B * B) {
        SBP_TRY(alloc(m, &S.cells, (int64_t)B * B));
        S.cap_cells = (int64_t)B * B;
    }
    if (S.cap_b < B) {
        SBP_TRY(alloc(m, &S.rp, (int64_t)B + 1));
        SBP_TRY(alloc(m, &S.cp, (int64_t)B + 1));
        SBP_TRY(alloc(m, &S.hoff, (int64_t)B + 1));
        SBP_TRY(alloc(m, &S.cnt, (int64_t)B + 1));
        SBP_TRY(alloc(m, &S.rpc, (int64_t)B * 32));
        SBP_TRY(alloc(m, &S.cpc, (int64_t)B * 32));
        S.cap_b = B;
    }
    return SBP_OK;
}

namespace {

// steps 1-2 for keys of type K: sort the edge keys (the first pass makes
// them from the edge list), run-length encode; returns the nonzero count
template <class K>
int sort_and_encode(sbp_model *m, int bits, int64_t *nnz_out) {
    const sbp_graph *g = m->g;
    sbp_model::Sparse &S = m->sp;
    const int64_t E = g->m;
    cudaStream_t st = m->stream;
    K *k0 = reinterpret_cast<K *>(S.key0), *k1 = reinterpret_cast<K *>(S.key1);
    EdgeKeys ek;
    ek.esrc = g->esrc;
    ek.oc = g->oc;
    ek.b = m->b;
    ek.B = (uint64_t)m->B;
    bool in_first = true;
    SBP_TRY((radix_sort<K, uint32_t>(k0, k1, nullptr, nullptr, E, bits, S.scratch, st, &in_first, &ek)));
    const K *keys = in_first ? k0 : k1;
    const int G = sort_chunk_count(E);
    const int64_t chunk = sort_chunk_length(E);
    uint32_t *tot = S.scratch, *cnt = S.scratch + 4, *cstart = S.scratch + 4 + 2 * (int64_t)G + 4;
    uint32_t *sscr = cstart + 2 * (int64_t)G + 4;
    k_rle_count<K><<<G, kT, 0, st>>>(keys, E, chunk, cnt);
    SBP_LAUNCHED();
    SBP_TRY(exclusive_scan_u32(cnt, cstart, G, tot, sscr, st));
    uint32_t h = 0;
    SBP_CUDA(cudaMemcpyAsync(&h, tot, 4, cudaMemcpyDeviceToHost, st));
    k_rle_emit<K><<<G, kT, 0, st>>>(keys, E, chunk, cstart, (uint64_t)m->B, S.start, S.rc, S.rowof, S.cnt);
    SBP_LAUNCHED();
    SBP_CUDA(cudaStreamSynchronize(st));
    *nnz_out = h;
    return SBP_OK;
}

}  // namespace

// Rebuild of the sparse blockmodel from m->b; fills the model's degree and
// per-block arrays.  One host read-back (the nonzero count) per rebuild.
// after_pass: m->bnew holds the previous assignment, and cell counts kept
// from the previous rebuild may be updated from the moves.
int rebuild_sparse(sbp_model *m, bool after_pass, bool *dl_done) {
    const sbp_graph *g = m->g;
    sbp_model::Sparse &S = m->sp;
    const int B = m->B;
    const int64_t E = g->m;
    cudaStream_t st = m->stream;
    const int cap = 152 * 8;
    uint32_t *sscr = S.scratch + 4;
    *dl_done = false;
    if (sparse_by_count(B, E) && B <= kSmallRowsB) {
        // counting sort over the B x B keys, then everything in one CTA
        if (after_pass && S.cells_B == B)
            SBP_TRY(update_cells(m, S.cells));
        else
            SBP_TRY(count_cells(m, S.cells));
        S.cells_B = B;
        uint32_t *rlen = S.scratch + 8, *clen = rlen + kSmallRowsB;
        __int128 *lpart = reinterpret_cast<__int128 *>(S.scratch + 8 + 2 * kSmallRowsB + 8);
        double *lfb = reinterpret_cast<double *>(lpart + 2 * kSmallRowsB);
        const int wgrid = (int)((2 * (int64_t)B * 32 + kT - 1) / kT);
        k_small_lengths<<<wgrid, kT, 0, st>>>(S.cells, B, rlen, clen);
        SBP_LAUNCHED();
        k_small_offsets<<<1, kSmallThreads, 0, st>>>(rlen, clen, B, S.rp, S.cp, S.hoff, S.nnz_dev);
        SBP_LAUNCHED();
        k_small_fill<<<wgrid, kT, 0, st>>>(S.cells, B, S.rp, S.cp, S.hoff, S.rc, S.rv, S.rowof, S.rpre, S.cr, S.cv,
                                           S.cpre, S.hkv, m->dout, m->din, m->T, m->XT, lpart, lfb, m->status);
        SBP_LAUNCHED();
        k_small_finish<<<1, kSmallThreads, 0, st>>>(m->dout, m->din, B, lpart, lfb, m->dsum, m->rcp, m->rcp32, E,
                                                    g->n, m->dl);
        SBP_LAUNCHED();
        k_sparse_pivots<<<(int)((64 * (int64_t)B + kT - 1) / kT), kT, 0, st>>>(S.rp, S.rpre, S.cp, S.cpre, B, S.rpc,
                                                                              S.cpc);
        SBP_LAUNCHED();
        S.nnz = -1;  // on the device until someone asks
        *dl_done = true;
        return SBP_OK;
    }
    // 1-3. the nonzeros of M in row order: CSR offsets, columns, counts,
    // in-row prefixes, dout
    int64_t nnz = 0;
    SBP_CUDA(cudaMemsetAsync(S.cnt, 0, ((size_t)B + 1) * 4, st));
    if (sparse_by_count(B, E)) {
        // counting sort over the B x B keys: the counts are the run lengths
        if (after_pass && S.cells_B == B)
            SBP_TRY(update_cells(m, S.cells));
        else
            SBP_TRY(count_cells(m, S.cells));
        S.cells_B = B;
        k_cell_rowcount<<<grid_of((int64_t)B * 32, cap), kT, 0, st>>>(S.cells, B, S.cnt);
        SBP_LAUNCHED();
        SBP_TRY(exclusive_scan_u32(S.cnt, S.rp, (int64_t)B + 1, S.scratch, sscr, st));
        uint32_t h = 0;
        SBP_CUDA(cudaMemcpyAsync(&h, S.scratch, 4, cudaMemcpyDeviceToHost, st));
        k_cell_compact<<<grid_of((int64_t)B * 32, cap), kT, 0, st>>>(S.cells, B, S.rp, S.rc, S.rv, S.rowof, S.rpre,
                                                                        m->dout);
        SBP_LAUNCHED();
        SBP_CUDA(cudaStreamSynchronize(st));
        nnz = h;
    } else {
        S.cells_B = 0;
        // radix sort of the (row, column) keys of the edges, run-length encoding
        const int bits = bits_for((uint64_t)B * (uint64_t)B - 1);
        if (E > 0) {
            if (bits <= 32)
                SBP_TRY(sort_and_encode<uint32_t>(m, bits, &nnz));
            else
                SBP_TRY(sort_and_encode<uint64_t>(m, bits, &nnz));
            k_run_counts<<<grid_of(nnz, cap), kT, 0, st>>>(S.start, nnz, E, S.rv);
            SBP_LAUNCHED();
        }
        SBP_TRY(exclusive_scan_u32(S.cnt, S.rp, (int64_t)B + 1, nullptr, sscr, st));
        k_row_prefix<<<grid_of((int64_t)B * 32, cap), kT, 0, st>>>(S.rp, S.rv, B, S.rpre, m->dout);
        SBP_LAUNCHED();
    }
    S.nnz = nnz;
    // 4. CSC by a stable sort on the column
    SBP_CUDA(cudaMemsetAsync(S.cnt, 0, ((size_t)B + 1) * 4, st));
    if (nnz > 0) {
        k_csc_src<<<grid_of(nnz, cap), kT, 0, st>>>(S.rc, S.rowof, S.rv, nnz, S.ckey0, S.cval0, S.cnt);
        SBP_LAUNCHED();
    }
    bool cfirst = true;
    SBP_TRY((radix_sort<uint32_t, uint64_t>(S.ckey0, S.ckey1, S.cval0, S.cval1, nnz, bits_for((uint64_t)B - 1), S.scratch,
                                            st, &cfirst)));
    if (nnz > 0) {
        k_csc_unpack<<<grid_of(nnz, cap), kT, 0, st>>>(cfirst ? S.cval0 : S.cval1, nnz, S.cr, S.cv);
        SBP_LAUNCHED();
    }
    SBP_TRY(exclusive_scan_u32(S.cnt, S.cp, (int64_t)B + 1, nullptr, sscr, st));
    k_row_prefix<<<grid_of((int64_t)B * 32, cap), kT, 0, st>>>(S.cp, S.cv, B, S.cpre, m->din);
    SBP_LAUNCHED();
    k_sparse_pivots<<<(int)((64 * (int64_t)B + kT - 1) / kT), kT, 0, st>>>(S.rp, S.rpre, S.cp, S.cpre, B, S.rpc, S.cpc);
    SBP_LAUNCHED();
    // 5. per-row hash tables
    k_hash_caps<<<grid_of(B, cap), kT, 0, st>>>(S.rp, B, S.cnt);
    SBP_LAUNCHED();
    SBP_TRY(exclusive_scan_u32(S.cnt, S.hoff, (int64_t)B + 1, nullptr, sscr, st));
    // capacities are powers of two below 4 len + 2 per row
    SBP_CUDA(cudaMemsetAsync(S.hkv, 0xff, (size_t)(4 * nnz + 2 * (int64_t)B) * sizeof(int2), st));
    if (nnz > 0) {
        k_hash_fill<<<grid_of(nnz, cap), kT, 0, st>>>(S.rp, S.rc, S.rv, S.rowof, nnz, S.hoff, S.hkv, m->status);
        SBP_LAUNCHED();
    }
    // 6. per-block scalars
    k_block_scalars<<<grid_of(B, cap), kT, 0, st>>>(m->dout, m->din, B, m->dsum, m->rcp, m->rcp32);
    SBP_LAUNCHED();
    return SBP_OK;
}

int64_t sparse_nnz(sbp_model *m) {
    if (m->sp.nnz >= 0) return m->sp.nnz;
    int64_t h = 0;
    if (cudaMemcpyAsync(&h, m->sp.nnz_dev, 8, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    m->sp.nnz = h;
    return h;
}

void free_sparse(sbp_model *m) {
    sbp_model::Sparse &S = m->sp;
    void *ps[] = {S.key0, S.key1, S.start, S.rc, S.rv, S.rowof, S.rpre, S.cr, S.cv, S.cpre, S.ckey0,
                  S.ckey1, S.cval0, S.cval1, S.hkv, S.scratch, S.rp, S.cp, S.hoff, S.cnt, S.cells, S.nnz_dev,
                  S.rpc,  S.cpc};
    for (void *p : ps) model_free(p, m->stream);
    S = sbp_model::Sparse();
}

}  // namespace sbp
