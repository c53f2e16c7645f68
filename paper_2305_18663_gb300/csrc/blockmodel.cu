// blockmodel.cu -- the blockmodel from the assignment, and its update after
// a pass.
//
// Section II-A: M[r][s] counts the edges from block r to block s; the block
// degrees are its row and column sums.  Alg. 5: after every pass the moves
// are applied and the blockmodel is made consistent again: each edge with a
// moved end leaves its old (block, block) cell and enters the new one when
// the moved rows hold at most a quarter of the edges (a plan taken on the
// device), else M is recounted from the new assignment.  Both give the same
// integers.  The same kernels keep the block-labelled rows in step.
//
// Dense form (B <= dense_max_B): M is B x B int32, counted by an atomic
// histogram over the out-edges with the diagonal privatised per CTA.  P
// holds, per block u, the inclusive prefix of row u followed by dout_u plus
// the inclusive prefix of column u; the nodal and merge proposals search it.
// DL (Eq. 2) is reduced in a fixed order so it is reproducible bit for bit.
#include <cmath>

#include "apply.cuh"

namespace sbp {
namespace {

constexpr int kThreads = 256;

// Atomic histogram of (b[src], b[dst]) over the out-edges, four
// consecutive edges per thread (16-byte loads, eight independent gathers in
// flight).  Diagonal counts (intra-block edges, the large majority) go to a
// per-CTA shared-memory copy of the diagonal first.
__device__ __forceinline__ void hist_add(int32_t *__restrict__ M, int *diag, int B, bool valid, int r, int t) {
    if (!valid) return;
    if (r == t) atomicAdd(&diag[r], 1);
    else atomicAdd(&M[(size_t)r * B + t], 1);
}

__global__ void __launch_bounds__(kThreads) k_hist_dense(GraphDev g, const int32_t *__restrict__ b,
                                                         int32_t *__restrict__ M, int B, const int32_t *__restrict__ skip) {
    if (skip && *skip == 1) return;
    extern __shared__ int diag[];
    for (int i = threadIdx.x; i < B; i += blockDim.x) diag[i] = 0;
    __syncthreads();
    const int64_t m4 = g.m >> 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int4 *es4 = reinterpret_cast<const int4 *>(g.esrc);
    const int4 *oc4 = reinterpret_cast<const int4 *>(g.oc);
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m4; base += stride) {
        const int64_t q = base + threadIdx.x;
        const bool valid = q < m4;
        int4 s4 = make_int4(0, 0, 0, 0), d4 = make_int4(0, 0, 0, 0);
        if (valid) {
            s4 = es4[q];
            d4 = oc4[q];
        }
        int r0 = 0, r1 = 0, r2 = 0, r3 = 0, t0 = 0, t1 = 0, t2 = 0, t3 = 0;
        if (valid) {
            r0 = b[s4.x]; r1 = b[s4.y]; r2 = b[s4.z]; r3 = b[s4.w];
            t0 = b[d4.x]; t1 = b[d4.y]; t2 = b[d4.z]; t3 = b[d4.w];
        }
        hist_add(M, diag, B, valid, r0, t0);
        hist_add(M, diag, B, valid, r1, t1);
        hist_add(M, diag, B, valid, r2, t2);
        hist_add(M, diag, B, valid, r3, t3);
    }
    // the last m % 4 edges
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const int64_t e = (m4 << 2) + threadIdx.x;
        const bool valid = e < g.m;
        const int r = valid ? b[g.esrc[e]] : 0, t = valid ? b[g.oc[e]] : 0;
        hist_add(M, diag, B, valid, r, t);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < B; i += blockDim.x)
        if (diag[i]) atomicAdd(&M[(size_t)i * B + i], diag[i]);
}

// one warp per block u
__global__ void __launch_bounds__(kThreads) k_prefix_dense(const int32_t *__restrict__ M, int B,
                                                           uint32_t *__restrict__ P, int32_t *__restrict__ dout,
                                                           int32_t *__restrict__ din, double *__restrict__ rcp,
                                                           float *__restrict__ rcp32, int32_t *__restrict__ dsum,
                                                           uint32_t *__restrict__ Pc, int pstep) {
    const int u = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (u >= B) return;
    prefix_block(M, B, u, P, dout, din, rcp, rcp32, dsum, Pc, pstep);
}

// Eq. 1 split form: sum over M of x ln x minus the degree terms, one
// partial per block, exact in fixed point inside the table
__global__ void __launch_bounds__(kThreads) k_dl_partial(const int32_t *__restrict__ M, int64_t BB,
                                                         const int32_t *__restrict__ dout,
                                                         const int32_t *__restrict__ din, int B,
                                                         const __int128 *__restrict__ T, int64_t XT,
                                                         DlPartial *__restrict__ partials) {
    __shared__ __int128 sfix[kThreads / 32];
    __shared__ double sfb[kThreads / 32];
    __int128 fix = 0;
    double fb = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < BB; i += stride) add_xlogx(T, XT, M[i], 1, fix, fb);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += stride) {
        add_xlogx(T, XT, dout[i], -1, fix, fb);
        add_xlogx(T, XT, din[i], -1, fix, fb);
    }
    fix = warp_sum_128(fix);
    fb = warp_sum(fb);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sfix[wid] = fix;
        sfb[wid] = fb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __int128 f = 0;
        double d = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) {
            f += sfix[q];
            d += sfb[q];
        }
        partials[blockIdx.x].fix = f;
        partials[blockIdx.x].fb = d;
    }
}

// Eq. 2: DL = E h(B^2/E) + N ln B - L, h(x) = (1+x) ln(1+x) - x ln x.  The
// partials are summed in a fixed order (strided per thread, then a fixed
// tree), so the result is reproducible bit for bit.
__global__ void __launch_bounds__(kThreads) k_dl_final(const DlPartial *__restrict__ partials, int np, int64_t E,
                                                       int64_t N, int B, double *__restrict__ dl) {
    __shared__ __int128 sfix[kThreads];
    __shared__ double sfb[kThreads];
    __int128 f = 0;
    double d = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        f += partials[i].fix;
        d += partials[i].fb;
    }
    sfix[threadIdx.x] = f;
    sfb[threadIdx.x] = d;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sfix[threadIdx.x] += sfix[threadIdx.x + o];
            sfb[threadIdx.x] += sfb[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        dl[0] = dl_eq2(E, N, B, fix_to_double(sfix[0]) + sfb[0]);
    }
}

// commit plan (1 = update the counts from the moved vertices' rows, when
// they hold at most a quarter of the edges; 0 = recount) and, for a recount,
// the zeroed cells: every CTA derives the plan from the counters, CTA 0
// stores it for the kernels that follow
__global__ void k_commit_plan(const DevCounters *__restrict__ c, int64_t E, int32_t *__restrict__ flag,
                              int32_t *__restrict__ M, int64_t n) {
    const int plan = (c->acc_edges * 4ull <= (unsigned long long)E) ? 1 : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) flag[0] = plan;
    if (plan != 0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) M[i] = 0;
}

// Apply step of Alg. 5 on a dense M: every edge with a moved end leaves its
// old (block, block) cell and enters the new one.  An edge is visited once:
// through the out-row of its moved source, or through the in-row of its
// moved target when the source stayed.  Lanes take the edges of one row,
// four loads in flight per lane.
// Warps [0, n_big) take one vertex each of the largest-degree group (in
// descending degree, so the longest rows start first); the remaining warps
// take 32 consecutive vertex ids each and skip the ones of that group.
__global__ void __launch_bounds__(kThreads) k_delta_dense(GraphDev g, const int32_t *__restrict__ order, int big_begin,
                                                          int n_big, const int32_t *__restrict__ bnew,
                                                          const int32_t *__restrict__ bold, int32_t *__restrict__ M,
                                                          int B, const int32_t *__restrict__ flag) {
    if (*flag != 1) return;
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w < n_big) {
        const int v = order[big_begin + w];
        const int r = bold[v], s = bnew[v];
        if (r == s) return;
        delta_out_row(g.oc, g.op[v], g.op[v + 1], r, s, bnew, bold, M, B);
        delta_in_row(g.ic, g.ip[v], g.ip[v + 1], r, s, bnew, bold, M, B);
        return;
    }
    const int64_t base = (w - n_big) * 32;
    if (base >= g.n) return;
    const int64_t vv = base + lane;
    const bool moved = vv < g.n && bnew[vv] != bold[vv];
    unsigned mm = __ballot_sync(0xffffffffu, moved);
    while (mm) {
        const int q = __ffs(mm) - 1;
        mm &= mm - 1;
        const int v = (int)(base + q);
        const int o0 = g.op[v], o1 = g.op[v + 1], i0 = g.ip[v], i1 = g.ip[v + 1];
        if ((o1 - o0) + (i1 - i0) > kWarpDeg) continue;  // a warp of its own took it
        const int r = bold[v], s = bnew[v];
        delta_out_row(g.oc, o0, o1, r, s, bnew, bold, M, B);
        delta_in_row(g.ic, i0, i1, r, s, bnew, bold, M, B);
    }
}

// Adds d to cells[key] for every lane with key >= 0.  The lanes whose key
// equals that of the first lane holding one add together with one atomic
// (most edges of a moved vertex land on the same (block, block) cell); the
// other lanes add their own.  All lanes of the warp call it.
__device__ __forceinline__ void warp_cell_add(int32_t *cells, int key, int d) {
    const unsigned act = __ballot_sync(0xffffffffu, key >= 0);
    if (!act) return;
    const int lead = __ffs(act) - 1;
    const int k0 = __shfl_sync(0xffffffffu, key, lead);
    const unsigned same = __ballot_sync(0xffffffffu, key == k0);
    if ((int)(threadIdx.x & 31) == lead)
        atomicAdd(&cells[k0], d * __popc(same));
    else if (key >= 0 && key != k0)
        atomicAdd(&cells[key], d);
}

// The same apply step driven by the accepted-move list: an item is one
// kMoveChunk-edge slice of the concatenated (out, in) row of a moved vertex,
// so hubs are spread over many warps and no warp scans unmoved vertices.
// Lane j of the warp takes edges j, j + 32, ... of the slice, all loads in
// flight together.  With nbo (not NULL) it also brings the block-labelled
// rows up to date (the twin of each edge takes v's new label), whatever the
// plan; the count update runs only when the plan chose it.
__global__ void __launch_bounds__(kThreads) k_delta_items(GraphDev g, const int2 *__restrict__ items,
                                                          const DevCounters *__restrict__ c, int64_t cap,
                                                          const int32_t *__restrict__ bnew,
                                                          const int32_t *__restrict__ bold, int32_t *__restrict__ M,
                                                          int B, const int32_t *__restrict__ flag,
                                                          int32_t *__restrict__ nbo, int32_t *__restrict__ nbi) {
    const bool counts = *flag == 1;
    if (!counts && !nbo) return;
    const int lane = threadIdx.x & 31;
    const int64_t total = (int64_t)(c->items < (unsigned long long)cap ? c->items : (unsigned long long)cap);
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int kPer = kMoveChunk / 32;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
        const int2 it = items[w];
        const int v = it.x;
        const int r = bold[v], s = bnew[v];
        if (r == s) continue;
        const int o0 = g.op[v], kout = g.op[v + 1] - o0;
        const int i0 = g.ip[v], k = kout + (g.ip[v + 1] - i0);
        const int lo = it.y * kMoveChunk;
        int nb[kPer], t[kPer], u[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int idx = lo + j * 32 + lane;
            nb[j] = idx < k ? (idx < kout ? g.oc[o0 + idx] : g.ic[i0 + idx - kout]) : -1;
        }
        if (nbo) {
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int idx = lo + j * 32 + lane;
                if (nb[j] < 0) continue;
                const int32_t x = s | (nb[j] == v ? kNbSelf : 0);
                if (idx < kout) nbi[g.tw_oi[o0 + idx]] = x;  // v -> w: in w's in-row
                else nbo[g.tw_io[i0 + idx - kout]] = x;     // w -> v: in w's out-row
            }
        }
        if (!counts) continue;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            t[j] = nb[j] >= 0 ? bold[nb[j]] : 0;
            u[j] = nb[j] >= 0 ? bnew[nb[j]] : 0;
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int idx = lo + j * 32 + lane;
            int leave = -1, enter = -1;  // cells (B * B <= 2^26) the edge leaves and enters
            if (nb[j] >= 0) {
                if (idx < kout) {
                    // out-edge v -> w: leaves (r, t), enters (s, u)
                    leave = r * B + t[j];
                    enter = s * B + u[j];
                } else if (u[j] == t[j]) {
                    // in-edge w -> v from a vertex that stayed (a moved
                    // source applies it through its own out-row)
                    leave = t[j] * B + r;
                    enter = t[j] * B + s;
                }
            }
            warp_cell_add(M, leave, -1);
            warp_cell_add(M, enter, 1);
        }
    }
}

// block-labelled rows from scratch, both CSRs in their own order (coalesced
// writes): out-entry e (u -> w) gets b[w], in-entry j (w -> u) gets b[w];
// bit 31 marks a self-loop (out-rows: from the edge's source; in-rows: set
// afterwards at the graph's self-loop positions by k_nb_self)
__global__ void k_nb_full(GraphDev g, const int32_t *__restrict__ b, int32_t *__restrict__ nbo,
                          int32_t *__restrict__ nbi) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < g.m; e += stride) {
        const int u = g.esrc[e], w = g.oc[e], x = g.ic[e];
        nbo[e] = b[w] | (u == w ? kNbSelf : 0);
        nbi[e] = b[x];
    }
}

__global__ void k_nb_self(const int32_t *__restrict__ self_in, int64_t n_self, int32_t *__restrict__ nbi) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_self; i += (int64_t)gridDim.x * blockDim.x)
        nbi[self_in[i]] |= kNbSelf;
}

// the entries that name a moved vertex, after a pass: for every item of
// the accepted-move list (a 256-edge slice of moved vertex v's rows), the
// twin of each of v's edges takes v's new label
__global__ void __launch_bounds__(kThreads) k_nb_items(GraphDev g, const int2 *__restrict__ items,
                                                       const DevCounters *__restrict__ c, int64_t cap,
                                                       const int32_t *__restrict__ b, int32_t *__restrict__ nbo,
                                                       int32_t *__restrict__ nbi) {
    const int lane = threadIdx.x & 31;
    const int64_t total = (int64_t)(c->items < (unsigned long long)cap ? c->items : (unsigned long long)cap);
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int kPer = kMoveChunk / 32;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
        const int2 it = items[w];
        const int v = it.x;
        const int s = b[v];
        const int o0 = g.op[v], kout = g.op[v + 1] - o0;
        const int i0 = g.ip[v], k = kout + (g.ip[v + 1] - i0);
        const int lo = it.y * kMoveChunk;
        int nb[kPer], tw[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int idx = lo + j * 32 + lane;
            const bool ok = idx < k, out = idx < kout;
            nb[j] = ok ? (out ? g.oc[o0 + idx] : g.ic[i0 + idx - kout]) : -1;
            tw[j] = ok ? (out ? g.tw_oi[o0 + idx] : g.tw_io[i0 + idx - kout]) : 0;
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int idx = lo + j * 32 + lane;
            if (nb[j] < 0) continue;
            const int32_t x = s | (nb[j] == v ? kNbSelf : 0);
            if (idx < kout) nbi[tw[j]] = x;  // v -> w: in w's in-row
            else nbo[tw[j]] = x;             // w -> v: in w's out-row
        }
    }
}

__global__ void k_relabel(int32_t *__restrict__ b, int32_t *__restrict__ bnew, int n, const int32_t *__restrict__ map) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int x = map[b[v]];
        b[v] = x;
        bnew[v] = x;
    }
}

__global__ void k_vertex_count(const int32_t *__restrict__ b, int n, int32_t *__restrict__ cnt) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) atomicAdd(&cnt[b[v]], 1);
}

int grid_for(int64_t work, int per_block, int cap) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

}  // namespace

int ensure_capacity(sbp_model *m, int32_t B) {
    m->dense = B <= m->p.dense_max_B;
    if (!m->dense) SBP_TRY(ensure_sparse_capacity(m, B));
    const bool need_dense = m->dense && B > m->Bdense;
    if (B <= m->Bcap && !need_dense) return SBP_OK;
    cudaStream_t st = m->stream;
    auto alloc = [&](auto **p, size_t bytes) { return model_alloc((void **)p, bytes, st) == cudaSuccess; };
    if (need_dense) {
        model_free(m->M, st);
        model_free(m->P, st);
        model_free(m->Pc, st);
        m->M = nullptr; m->P = nullptr; m->Pc = nullptr;
        m->Bdense = 0;
        const size_t BB = (size_t)B * B;
        if (!alloc(&m->M, BB * 4) || !alloc(&m->P, BB * 8) || !alloc(&m->Pc, (size_t)B * 32 * 4)) {
            cudaGetLastError();
            return fail(SBP_ENOMEM, "device allocation failed for a dense blockmodel of B = " + std::to_string(B));
        }
        m->Bdense = B;
    }
    if (B > m->Bcap) {
        void *old[] = {m->dout, m->din, m->rcp, m->rcp32, m->dsum, m->best_s, m->best_d, m->map, m->vcount};
        for (void *p : old) model_free(p, st);
        m->dout = m->din = nullptr; m->rcp = nullptr; m->rcp32 = nullptr; m->dsum = nullptr;
        m->best_s = m->map = m->vcount = nullptr; m->best_d = nullptr;
        m->Bcap = 0;
        const size_t b = (size_t)B;
        if (!alloc(&m->dout, b * 4) || !alloc(&m->din, b * 4) || !alloc(&m->rcp, b * 8) || !alloc(&m->rcp32, b * 4) ||
            !alloc(&m->dsum, b * 4) || !alloc(&m->best_s, b * 4) || !alloc(&m->best_d, b * 8) ||
            !alloc(&m->map, b * 4) || !alloc(&m->vcount, b * 4)) {
            cudaGetLastError();
            return fail(SBP_ENOMEM, "device allocation failed for the block arrays of B = " + std::to_string(B));
        }
        m->Bcap = B;
    }
    return SBP_OK;
}

// cells[r * B + t] = number of edges from block r to block t (all B * B
// cells are written); B <= 16384
int count_cells(sbp_model *m, int32_t *cells) {
    const sbp_graph *g = m->g;
    const int B = m->B;
    SBP_CUDA(cudaMemsetAsync(cells, 0, (size_t)B * B * 4, m->stream));
    if (g->m > 0) {
        const size_t smem = (size_t)B * 4;
        if (smem > 48 * 1024)
            SBP_TRY(ensure_dyn_smem((const void *)k_hist_dense, smem));
        k_hist_dense<<<grid_for((g->m + 3) / 4, kThreads, num_sms() * 8), kThreads, smem, m->stream>>>(g->dev(), m->b,
                                                                                                        cells, B, nullptr);
        SBP_LAUNCHED();
    }
    return SBP_OK;
}

// cells (the counts of the previous assignment m->bnew) brought to the
// counts of m->b: the plan kernel picks, on the device, either the update
// from the moved vertices' rows (few moved edges) or a recount; both give
// the same counts
int update_cells(sbp_model *m, int32_t *cells) {
    const sbp_graph *g = m->g;
    const int B = m->B;
    const int sms = num_sms();
    const int64_t BB = (int64_t)B * B;
    int32_t *flag = m->status + 1;
    k_commit_plan<<<grid_for(BB, kThreads, sms * 8), kThreads, 0, m->stream>>>(m->counters, g->m, flag, cells, BB);
    SBP_LAUNCHED();
    if (g->m > 0) {
        const size_t smem = (size_t)B * 4;
        if (smem > 48 * 1024)
            SBP_TRY(ensure_dyn_smem((const void *)k_hist_dense, smem));
        k_hist_dense<<<grid_for((g->m + 3) / 4, kThreads, sms * 8), kThreads, smem, m->stream>>>(g->dev(), m->b, cells, B,
                                                                                                  flag);
        SBP_LAUNCHED();
        if (m->list_ok && m->items) {
            // the block-labelled rows follow in the same pass
            const bool nb = m->nb_ok && m->nbo;
            k_delta_items<<<sms * 4, kThreads, 0, m->stream>>>(g->dev(), m->items, m->counters, m->cap_items, m->b,
                                                               m->bnew, cells, B, flag, nb ? m->nbo : nullptr,
                                                               nb ? m->nbi : nullptr);
            SBP_LAUNCHED();
            m->nb_in_commit = nb;
        } else {
            const int64_t n_big = g->n - g->bin[3];
            const int64_t warps = n_big + (g->n + 31) / 32;
            k_delta_dense<<<grid_for(warps * 32, kThreads, 1 << 30), kThreads, 0, m->stream>>>(
                g->dev(), g->order, (int)g->bin[3], (int)n_big, m->b, m->bnew, cells, B, flag);
            SBP_LAUNCHED();
        }
    }
    return SBP_OK;
}

namespace {

// M (dense, or sparse rows), P, degrees, rcp and DL from m->b.  after_pass:
// m->bnew holds the assignment the current M was built from, and the counts
// may be updated from the moves instead of recounted.
int build_blockmodel(sbp_model *m, bool after_pass) {
    const sbp_graph *g = m->g;
    const int B = m->B;
    SBP_TRY(xlogx_table(g->m + 1, &m->T, &m->XT));
    const int32_t *vals;
    int64_t nvals;
    if (m->dense) {
        const int64_t BB = (int64_t)B * B;
        if (after_pass)
            SBP_TRY(update_cells(m, m->M));
        else
            SBP_TRY(count_cells(m, m->M));
        k_prefix_dense<<<grid_for((int64_t)B * 32, kThreads, 1 << 30), kThreads, 0, m->stream>>>(
            m->M, B, m->P, m->dout, m->din, m->rcp, m->rcp32, m->dsum, m->Pc, (2 * B + 31) / 32);
        SBP_LAUNCHED();
        vals = m->M;
        nvals = BB;
    } else {
        bool dl_done = false;
        SBP_TRY(rebuild_sparse(m, after_pass, &dl_done));
        if (dl_done) {
            SBP_CUDA(cudaMemcpyAsync(m->bnew, m->b, (size_t)g->n * 4, cudaMemcpyDeviceToDevice, m->stream));
            return SBP_OK;
        }
        vals = m->sp.rv;
        nvals = m->sp.nnz;
    }
    const int np = grid_for(nvals > B ? nvals : B, kThreads * 4, m->npartials);
    DlPartial *parts = reinterpret_cast<DlPartial *>(m->partials);
    k_dl_partial<<<np, kThreads, 0, m->stream>>>(vals, nvals, m->dout, m->din, B, m->T, m->XT, parts);
    SBP_LAUNCHED();
    k_dl_final<<<1, kThreads, 0, m->stream>>>(parts, np, g->m, g->n, B, m->dl);
    SBP_LAUNCHED();
    SBP_CUDA(cudaMemcpyAsync(m->bnew, m->b, (size_t)g->n * 4, cudaMemcpyDeviceToDevice, m->stream));
    return SBP_OK;
}

}  // namespace

// a rebuild from m->b drops the pending decisions, and with them the
// accepted-move list
int rebuild_blockmodel(sbp_model *m) {
    m->nb_ok = false;
    m->list_ok = true;
    m->decided.clear();
    SBP_CUDA(cudaMemsetAsync(&m->counters->items, 0, sizeof(unsigned long long), m->stream));
    return build_blockmodel(m, false);
}

// P, Pc, degrees and reciprocals of a dense model from its M
int launch_prefix(sbp_model *m) {
    const int B = m->B;
    k_prefix_dense<<<grid_for((int64_t)B * 32, kThreads, 1 << 30), kThreads, 0, m->stream>>>(
        m->M, B, m->P, m->dout, m->din, m->rcp, m->rcp32, m->dsum, m->Pc, (2 * B + 31) / 32);
    SBP_LAUNCHED();
    return SBP_OK;
}

// After a nodal pass (m->b: new labels, m->bnew: the previous ones).  The
// counts (dense M, or the cell counts of a sparse model rebuilt by
// counting) take the incremental update when the plan kernel finds few
// moved edges (decided on the device, no host round trip); the result is
// the same M as a recount.
int commit_blockmodel(sbp_model *m) { return build_blockmodel(m, !m->p.full_rebuild); }

// block-labelled rows from m->b (allocated on first use).  Without the
// memory for them nb_ok stays false and the pass gathers labels instead.
int nb_rows_rebuild(sbp_model *m) {
    const sbp_graph *g = m->g;
    if (!m->nbo) {
        const size_t bytes = (size_t)(g->m > 0 ? g->m : 1) * 4;
        if (model_alloc((void **)&m->nbo, bytes, m->stream) != cudaSuccess ||
            model_alloc((void **)&m->nbi, bytes, m->stream) != cudaSuccess) {
            cudaGetLastError();
            model_free(m->nbo, m->stream);
            model_free(m->nbi, m->stream);
            m->nbo = m->nbi = nullptr;
            return SBP_OK;
        }
    }
    if (g->m > 0) {
        k_nb_full<<<grid_for(g->m, kThreads, num_sms() * 8), kThreads, 0, m->stream>>>(g->dev(), m->b, m->nbo, m->nbi);
        SBP_LAUNCHED();
    }
    if (g->n_self > 0) {
        k_nb_self<<<grid_for(g->n_self, kThreads, num_sms() * 8), kThreads, 0, m->stream>>>(g->self_in, g->n_self,
                                                                                           m->nbi);
        SBP_LAUNCHED();
    }
    m->nb_ok = true;
    return SBP_OK;
}

// after a commit: the block-labelled rows follow the accepted moves, or are
// marked stale when the list does not hold every change
int nb_rows_after_commit(sbp_model *m) {
    if (m->nb_in_commit) {  // updated by the apply step's kernel
        m->nb_in_commit = false;
        return SBP_OK;
    }
    if (!m->nb_ok || !m->nbo) return SBP_OK;
    if (!m->list_ok || !m->items) {
        m->nb_ok = false;
        return SBP_OK;
    }
    k_nb_items<<<num_sms() * 4, kThreads, 0, m->stream>>>(m->g->dev(), m->items, m->counters, m->cap_items, m->b,
                                                          m->nbo, m->nbi);
    SBP_LAUNCHED();
    return SBP_OK;
}

int launch_relabel(sbp_model *m, const int32_t *map_dev) {
    const int n = (int)m->g->n;
    k_relabel<<<grid_for(n, kThreads, num_sms() * 8), kThreads, 0, m->stream>>>(m->b, m->bnew, n, map_dev);
    SBP_LAUNCHED();
    return SBP_OK;
}

int launch_vertex_count(sbp_model *m) {
    const int n = (int)m->g->n;
    SBP_CUDA(cudaMemsetAsync(m->vcount, 0, (size_t)m->B * 4, m->stream));
    k_vertex_count<<<grid_for(n, kThreads, num_sms() * 8), kThreads, 0, m->stream>>>(m->b, n, m->vcount);
    SBP_LAUNCHED();
    return SBP_OK;
}

}  // namespace sbp
