// sparse.cu -- the blockmodel as sparse rows and columns (B > dense_max_B).
//
// Section III-A (a)-(b): M held as per-row hashed sparse rows plus a stored
// transpose.  Rebuilt from the assignment by sort plus segmented count:
//   1. key of every edge = b[src] * B + b[dst]; radix sort;
//   2. run-length encoding gives the nonzeros (r, c, M[r][c]) in row order;
//   3. CSR: row offsets by a row histogram and scan, the inclusive prefix of
//      the counts inside each row (the proposal CDF over row u);
//   4. CSC: a stable radix sort of the nonzeros by column keeps ascending
//      rows inside each column; offsets and prefixes as for the rows;
//   5. per-row open-addressing tables (capacity the power of two at least
//      twice the row's length) for M[r][c] lookups;
//   6. block degrees from the last prefix of each row / column; DL as an
//      exact fixed-point sum over the nonzeros.
#include <algorithm>

#include "common.cuh"

namespace sbp {

int exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total_dev, uint32_t *scratch,
                       cudaStream_t st);
int64_t scan_scratch_words(int64_t n);
int64_t sort_scratch_words(int64_t n);
template <class K, class V>
int radix_sort(K *k0, K *k1, V *v0, V *v1, int64_t n, int bits, uint32_t *scratch, cudaStream_t st, bool *in_first);

namespace {

constexpr int kT = 256;

int grid_of(int64_t work, int cap) {
    int64_t g = (work + kT - 1) / kT;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

__global__ void k_edge_keys(GraphDev g, const int32_t *__restrict__ b, int64_t B, uint64_t *__restrict__ keys) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < g.m; e += (int64_t)gridDim.x * blockDim.x)
        keys[e] = (uint64_t)b[g.esrc[e]] * (uint64_t)B + (uint64_t)b[g.oc[e]];
}

__global__ void k_run_heads(const uint64_t *__restrict__ keys, int64_t n, uint32_t *__restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

// heads: unique key, start position; row counts
__global__ void k_run_scatter(const uint64_t *__restrict__ keys, int64_t n, const uint32_t *__restrict__ flag,
                              const uint32_t *__restrict__ pos, int64_t B, uint32_t *__restrict__ start,
                              int32_t *__restrict__ col, uint32_t *__restrict__ rowcnt, int32_t *__restrict__ rowof) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (flag[i]) {
            const uint32_t p = pos[i];
            const uint64_t k = keys[i];
            const int r = (int)(k / (uint64_t)B), c = (int)(k % (uint64_t)B);
            start[p] = (uint32_t)i;
            col[p] = c;
            rowof[p] = r;
            atomicAdd(&rowcnt[r], 1u);
        }
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
                            const uint32_t *__restrict__ hoff, int32_t *__restrict__ hk, int32_t *__restrict__ hv,
                            int32_t *__restrict__ status) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int r = rowof[p], c = col[p];
        const uint32_t off = hoff[r], cap = hoff[r + 1] - off;
        uint32_t h = sparse_hash(c) & (cap - 1);
        bool done = false;
        for (uint32_t q = 0; q < cap; ++q) {
            if (atomicCAS(&hk[off + h], -1, c) == -1) {
                hv[off + h] = val[p];
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
int alloc(T **p, int64_t count) {
    cudaFree(*p);
    *p = nullptr;
    if (cudaMalloc((void **)p, (size_t)(count > 0 ? count : 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SBP_ENOMEM, "cudaMalloc failed for the sparse blockmodel");
    }
    return SBP_OK;
}

}  // namespace

int ensure_sparse_capacity(sbp_model *m, int32_t B) {
    sbp_model::Sparse &S = m->sp;
    const int64_t E = m->g->m > 0 ? m->g->m : 1;
    if (S.cap_e < E) {
        SBP_TRY(alloc(&S.key0, E));
        SBP_TRY(alloc(&S.key1, E));
        SBP_TRY(alloc(&S.flag, E));
        SBP_TRY(alloc(&S.pos, E));
        SBP_TRY(alloc(&S.start, E));
        SBP_TRY(alloc(&S.rc, E));
        SBP_TRY(alloc(&S.rv, E));
        SBP_TRY(alloc(&S.rowof, E));
        SBP_TRY(alloc(&S.rpre, E));
        SBP_TRY(alloc(&S.cr, E));
        SBP_TRY(alloc(&S.cv, E));
        SBP_TRY(alloc(&S.cpre, E));
        SBP_TRY(alloc(&S.ckey0, E));
        SBP_TRY(alloc(&S.ckey1, E));
        SBP_TRY(alloc(&S.cval0, E));
        SBP_TRY(alloc(&S.cval1, E));
        SBP_TRY(alloc(&S.hk, 4 * E + 2 * (int64_t)m->g->n));
        SBP_TRY(alloc(&S.hv, 4 * E + 2 * (int64_t)m->g->n));
        const int64_t w = std::max(std::max(sort_scratch_words(E), scan_scratch_words(E) + 4),
                                   scan_scratch_words((int64_t)m->g->n + 1) + 4);
        SBP_TRY(alloc(&S.scratch, w + 1024));
        S.cap_e = E;
    }
    if (S.cap_b < B) {
        SBP_TRY(alloc(&S.rp, (int64_t)B + 1));
        SBP_TRY(alloc(&S.cp, (int64_t)B + 1));
        SBP_TRY(alloc(&S.hoff, (int64_t)B + 1));
        SBP_TRY(alloc(&S.cnt, (int64_t)B + 1));
        S.cap_b = B;
    }
    return SBP_OK;
}

// Rebuild of the sparse blockmodel from m->b; fills the model's degree and
// per-block arrays.  One host read-back (the nonzero count) per rebuild.
int rebuild_sparse(sbp_model *m) {
    const sbp_graph *g = m->g;
    sbp_model::Sparse &S = m->sp;
    const int B = m->B;
    const int64_t E = g->m;
    cudaStream_t st = m->stream;
    const int cap = 152 * 8;
    // 1. keys, sort
    const int bits = bits_for((uint64_t)B * (uint64_t)B - 1);
    if (E > 0) {
        k_edge_keys<<<grid_of(E, cap), kT, 0, st>>>(g->dev(), m->b, B, S.key0);
        SBP_LAUNCHED();
    }
    bool in_first = true;
    SBP_TRY((radix_sort<uint64_t, uint64_t>(S.key0, S.key1, nullptr, nullptr, E, bits, S.scratch, st, &in_first)));
    const uint64_t *keys = in_first ? S.key0 : S.key1;
    // 2. run-length
    uint32_t *tot = S.scratch;  // word 0: nonzero count (scratch tail used by the scans below)
    uint32_t *sscr = S.scratch + 4;
    int64_t nnz = 0;
    SBP_CUDA(cudaMemsetAsync(S.cnt, 0, ((size_t)B + 1) * 4, st));
    if (E > 0) {
        k_run_heads<<<grid_of(E, cap), kT, 0, st>>>(keys, E, S.flag);
        SBP_LAUNCHED();
        SBP_TRY(exclusive_scan_u32(S.flag, S.pos, E, tot, sscr, st));
        uint32_t h = 0;
        SBP_CUDA(cudaMemcpyAsync(&h, tot, 4, cudaMemcpyDeviceToHost, st));
        SBP_CUDA(cudaStreamSynchronize(st));
        nnz = h;
        k_run_scatter<<<grid_of(E, cap), kT, 0, st>>>(keys, E, S.flag, S.pos, B, S.start, S.rc, S.cnt, S.rowof);
        SBP_LAUNCHED();
        k_run_counts<<<grid_of(nnz, cap), kT, 0, st>>>(S.start, nnz, E, S.rv);
        SBP_LAUNCHED();
    }
    S.nnz = nnz;
    // 3. CSR offsets and row prefixes, dout
    SBP_TRY(exclusive_scan_u32(S.cnt, S.rp, (int64_t)B + 1, nullptr, sscr, st));
    k_row_prefix<<<grid_of((int64_t)B * 32, cap), kT, 0, st>>>(S.rp, S.rv, B, S.rpre, m->dout);
    SBP_LAUNCHED();
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
    // 5. per-row hash tables
    k_hash_caps<<<grid_of(B, cap), kT, 0, st>>>(S.rp, B, S.cnt);
    SBP_LAUNCHED();
    SBP_TRY(exclusive_scan_u32(S.cnt, S.hoff, (int64_t)B + 1, nullptr, sscr, st));
    SBP_CUDA(cudaMemsetAsync(S.hk, 0xff, (size_t)(4 * S.cap_e + 2 * g->n) * 4, st));
    if (nnz > 0) {
        k_hash_fill<<<grid_of(nnz, cap), kT, 0, st>>>(S.rp, S.rc, S.rv, S.rowof, nnz, S.hoff, S.hk, S.hv, m->status);
        SBP_LAUNCHED();
    }
    // 6. per-block scalars
    k_block_scalars<<<grid_of(B, cap), kT, 0, st>>>(m->dout, m->din, B, m->dsum, m->rcp, m->rcp32);
    SBP_LAUNCHED();
    return SBP_OK;
}

void free_sparse(sbp_model *m) {
    sbp_model::Sparse &S = m->sp;
    void *ps[] = {S.key0, S.key1, S.flag, S.pos, S.start, S.rc, S.rv, S.rowof, S.rpre, S.cr, S.cv, S.cpre, S.ckey0,
                  S.ckey1, S.cval0, S.cval1, S.hk, S.hv, S.scratch, S.rp, S.cp, S.hoff, S.cnt};
    for (void *p : ps) cudaFree(p);
    S = sbp_model::Sparse();
}

}  // namespace sbp
