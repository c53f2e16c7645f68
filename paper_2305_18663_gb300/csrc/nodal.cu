// nodal.cu -- the asynchronous-Gibbs nodal decision pass.
//
// For every vertex v (block r) against the frozen (b, M):
//   1. proposal (Alg. 2 "propose new community"): a uniformly chosen
//      incident edge (out-list then in-list) gives the neighbour block u;
//      s is drawn with probability (1 + M[u][s] + M[s][u]) / (d_u + B) by an
//      integer inverse CDF over the prefix array P[u];
//   2. neighbour-block counts kout[t], kin[t] (Section III-A (c): the sparse
//      vector of changes) aggregated with warp match/ballot and, for longer
//      rows, a shared-memory hash table;
//   3. Delta DL over the changed entries of rows r,s and columns r,s only
//      (Section II-C), block degrees included; Eq. 1-2;
//   4. Hastings-corrected Metropolis test (Alg. 2): logA = -beta dDL +
//      ln(p_bwd / p_fwd), accept iff logA >= 0 or ln(u) < logA.
// The decision goes to the pending assignment; M is untouched until commit.
//
// Work units: one lane per neighbour for k <= 32; one warp per vertex with
// a per-warp table for k <= 128; one CTA per vertex above that.
#include <cmath>

#include "common.cuh"

namespace sbp {
namespace {

struct DecideArgs {
    GraphDev g;
    ModelDev md;
    const int32_t *order;
    int64_t lo, hi;
    int64_t v_begin, v_end;
    uint64_t seed, sweep_id;
    double beta;
    sbp_vertex_trace tr;
};

struct Counts {
    unsigned long long proposed = 0, moves = 0, accepted = 0, margin = 0;
};

__device__ __forceinline__ void write_trace(const DecideArgs &a, int v, int s, int flags, double dH, double logA) {
    if (a.tr.s) a.tr.s[v] = s;
    if (a.tr.flags) a.tr.flags[v] = flags;
    if (a.tr.dH) a.tr.dH[v] = dH;
    if (a.tr.logA) a.tr.logA[v] = logA;
}

__device__ __forceinline__ int Mat(const ModelDev &md, int r, int c) { return md.M[(size_t)r * md.B + c]; }

// contribution of one neighbour block t not in {r, s}
__device__ __forceinline__ void eval_entry(const ModelDev &md, int t, int ko, int ki, int r, int s, double &dL,
                                           double &fwd, double &bwd) {
    const int B = md.B;
    const int64_t Mrt = Mat(md, r, t), Mst = Mat(md, s, t), Mtr = Mat(md, t, r), Mts = Mat(md, t, s);
    if (ko) dL += dxlogx(Mrt, -ko) + dxlogx(Mst, ko);
    if (ki) dL += dxlogx(Mtr, -ki) + dxlogx(Mts, ki);
    const double den = (double)((int64_t)md.dout[t] + md.din[t] + B);
    const double c = (double)(ko + ki);
    fwd += c * (double)(Mts + Mst + 1) / den;
    bwd += c * (double)((Mtr - ki) + (Mrt - ko) + 1) / den;
}

// cross entries, degree terms, Hastings terms of r and s, and the test
__device__ void finalize(const DecideArgs &a, int v, int r, int s, int64_t Kout, int64_t Kin, int64_t self,
                         int64_t ko_r, int64_t ki_r, int64_t ko_s, int64_t ki_s, double dL, double fwd, double bwd,
                         uint64_t w2, Counts &c) {
    const ModelDev &md = a.md;
    const int B = md.B;
    const int64_t Mrr = Mat(md, r, r), Mss = Mat(md, s, s), Mrs = Mat(md, r, s), Msr = Mat(md, s, r);
    const int64_t dor = md.dout[r], dos = md.dout[s], dir = md.din[r], dis = md.din[s];
    dL += dxlogx(Mrr, -(ko_r + ki_r + self));
    dL += dxlogx(Mss, ko_s + ki_s + self);
    dL += dxlogx(Mrs, ki_r - ko_s);
    dL += dxlogx(Msr, ko_r - ki_s);
    dL -= dxlogx(dor, -Kout) + dxlogx(dos, Kout) + dxlogx(dir, -Kin) + dxlogx(dis, Kin);
    const double dH = -dL;
    const int64_t dr = dor + dir, ds = dos + dis, K = Kout + Kin;
    fwd += (double)(ko_r + ki_r + 2 * self) * (double)(Mrs + Msr + 1) / (double)(dr + B);
    fwd += (double)(ko_s + ki_s) * (double)(2 * Mss + 1) / (double)(ds + B);
    const int64_t Mrr2 = Mrr - (ko_r + ki_r + self), Mrs2 = Mrs + ki_r - ko_s, Msr2 = Msr + ko_r - ki_s;
    bwd += (double)(ko_r + ki_r) * (double)(2 * Mrr2 + 1) / (double)(dr - K + B);
    bwd += (double)(ko_s + ki_s + 2 * self) * (double)(Msr2 + Mrs2 + 1) / (double)(ds + K + B);
    const double logA = -a.beta * dH + log(bwd) - log(fwd);
    const double uacc = (double)(w2 >> 11) * 0x1.0p-53;
    const double lnu = log(uacc);
    const bool accept = logA >= 0.0 || lnu < logA;
    const bool margin = fabs(lnu - logA) <= 1e-9 * fmax(fabs(logA), 1.0);
    if (accept) md.bnew[v] = s;
    c.proposed++;
    c.moves++;
    c.accepted += accept;
    c.margin += margin;
    write_trace(a, v, s, 1 | (accept ? 2 : 0) | (margin ? 4 : 0), dH, logA);
}

// s from u: y < B picks s = y, else the inverse CDF over row u then column u
__device__ __forceinline__ int propose_block(const ModelDev &md, int u, uint64_t w1) {
    const int B = md.B;
    const int64_t du = (int64_t)md.dout[u] + md.din[u];
    const int64_t y = draw_below(w1, (uint64_t)(du + B));
    if (y < B) return (int)y;
    const int idx = warp_upper_bound(md.P + (size_t)u * 2 * B, 2 * B, (uint32_t)(y - B));
    return idx < B ? idx : idx - B;
}

__device__ __forceinline__ unsigned hash_slot(int key, int cap_log2) {
    return ((unsigned)key * 0x9E3779B1u) >> (32 - cap_log2);
}

// insert (key, inc) into an open-addressing table; false when full
__device__ __forceinline__ bool table_add(int *keys, unsigned long long *cnt, int *list, int *nlist, int cap,
                                          int cap_log2, int key, unsigned long long inc) {
    unsigned h = hash_slot(key, cap_log2);
    for (int p = 0; p < cap; ++p) {
        const int prev = atomicCAS(&keys[h], -1, key);
        if (prev == -1) {
            list[atomicAdd(nlist, 1)] = (int)h;
            atomicAdd(&cnt[h], inc);
            return true;
        }
        if (prev == key) {
            atomicAdd(&cnt[h], inc);
            return true;
        }
        h = (h + 1) & (unsigned)(cap - 1);
    }
    return false;
}

// ---------------------------------------------------------------------------
// warp per vertex (k <= kWarpDeg)

__global__ void __launch_bounds__(kWarpsPerCta * 32) k_decide_warp(DecideArgs a) {
    __shared__ int s_keys[kWarpsPerCta][kWarpCap];
    __shared__ unsigned long long s_cnt[kWarpsPerCta][kWarpCap];
    __shared__ int s_list[kWarpsPerCta][kWarpCap];
    __shared__ int s_nlist[kWarpsPerCta];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *keys = s_keys[wid];
    unsigned long long *cnt = s_cnt[wid];
    int *list = s_list[wid];
    int *nlist = &s_nlist[wid];
    for (int i = lane; i < kWarpCap; i += 32) {
        keys[i] = -1;
        cnt[i] = 0;
    }
    if (lane == 0) *nlist = 0;
    __syncwarp();
    constexpr int cap_log2 = 8;
    static_assert((1 << cap_log2) == kWarpCap, "table size");

    const GraphDev &g = a.g;
    const ModelDev &md = a.md;
    Counts c;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerCta;
    for (int64_t i = a.lo + (int64_t)blockIdx.x * kWarpsPerCta + wid; i < a.hi; i += nw) {
        const int v = a.order[i];
        if (v < a.v_begin || v >= a.v_end) continue;
        const int r = md.b[v];
        const int o0 = g.op[v], kout = g.op[v + 1] - o0;
        const int i0 = g.ip[v], kin = g.ip[v + 1] - i0;
        const int k = kout + kin;
        if (k == 0) {
            if (lane == 0) write_trace(a, v, r, 0, 0.0, 0.0);
            continue;
        }
        const U64x4 w = philox4x64_10(a.sweep_id, (uint64_t)v, 0, 0, a.seed, 0);
        const int j = (int)draw_below(w.x, (uint64_t)k);

        int self = 0, u = r, D = 0;
        int my_t = -1, my_ko = 0, my_ki = 0;
        if (k <= kSmallDeg) {
            const bool valid = lane < k, is_out = lane < kout;
            const int nb = valid ? (is_out ? g.oc[o0 + lane] : g.ic[i0 + lane - kout]) : -1;
            const int tb = valid ? md.b[nb] : -1;
            u = __shfl_sync(0xffffffffu, tb, j);
            const bool is_self = valid && nb == v;
            self = __popc(__ballot_sync(0xffffffffu, is_self && is_out));
            const int key = (valid && !is_self) ? tb : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            const unsigned outm = __ballot_sync(0xffffffffu, valid && !is_self && is_out);
            if (key >= 0 && lane == __ffs(peers) - 1) {
                my_t = key;
                my_ko = __popc(peers & outm);
                my_ki = __popc(peers) - my_ko;
            }
        } else {
            bool ok = true;
            for (int base = 0; base < k; base += 32) {
                const int idx = base + lane;
                const bool valid = idx < k, is_out = idx < kout;
                const int nb = valid ? (is_out ? g.oc[o0 + idx] : g.ic[i0 + idx - kout]) : -1;
                const int tb = valid ? md.b[nb] : -1;
                if (j >= base && j < base + 32) u = __shfl_sync(0xffffffffu, tb, j - base);
                const bool is_self = valid && nb == v;
                self += __popc(__ballot_sync(0xffffffffu, is_self && is_out));
                const int key = (valid && !is_self) ? tb : -1;
                const unsigned peers = __match_any_sync(0xffffffffu, key);
                const unsigned outm = __ballot_sync(0xffffffffu, valid && !is_self && is_out);
                if (key >= 0 && lane == __ffs(peers) - 1) {
                    const unsigned ko = __popc(peers & outm), ki = __popc(peers) - ko;
                    ok &= table_add(keys, cnt, list, nlist, kWarpCap, cap_log2, key,
                                    (unsigned long long)ko | ((unsigned long long)ki << 32));
                }
                __syncwarp();
            }
            if (!ok) record_status(md.status, SBP_EHASHFULL);
            D = *nlist;
        }

        const int s = propose_block(md, u, w.y);
        if (s == r) {
            if (lane == 0) {
                c.proposed++;
                write_trace(a, v, r, 1, 0.0, 0.0);
            }
        } else {
            double dL = 0.0, fwd = 0.0, bwd = 0.0;
            int ko_r = 0, ki_r = 0, ko_s = 0, ki_s = 0;
            if (k <= kSmallDeg) {
                if (my_t >= 0) {
                    if (my_t == r) { ko_r = my_ko; ki_r = my_ki; }
                    else if (my_t == s) { ko_s = my_ko; ki_s = my_ki; }
                    else eval_entry(md, my_t, my_ko, my_ki, r, s, dL, fwd, bwd);
                }
            } else {
                for (int e = lane; e < D; e += 32) {
                    const int slot = list[e];
                    const int t = keys[slot];
                    const unsigned long long cc = cnt[slot];
                    const int ko = (int)(cc & 0xffffffffu), ki = (int)(cc >> 32);
                    if (t == r) { ko_r = ko; ki_r = ki; }
                    else if (t == s) { ko_s = ko; ki_s = ki; }
                    else eval_entry(md, t, ko, ki, r, s, dL, fwd, bwd);
                }
            }
            dL = warp_sum(dL);
            fwd = warp_sum(fwd);
            bwd = warp_sum(bwd);
            ko_r = warp_sum_i(ko_r);
            ki_r = warp_sum_i(ki_r);
            ko_s = warp_sum_i(ko_s);
            ki_s = warp_sum_i(ki_s);
            if (lane == 0) finalize(a, v, r, s, kout, kin, self, ko_r, ki_r, ko_s, ki_s, dL, fwd, bwd, w.z, c);
        }
        if (k > kSmallDeg) {
            __syncwarp();
            for (int e = lane; e < D; e += 32) {
                const int slot = list[e];
                keys[slot] = -1;
                cnt[slot] = 0;
            }
            __syncwarp();
            if (lane == 0) *nlist = 0;
            __syncwarp();
        }
    }
    if (lane == 0 && (c.proposed | c.moves)) {
        atomicAdd(&md.counters->proposed, c.proposed);
        atomicAdd(&md.counters->moves, c.moves);
        atomicAdd(&md.counters->accepted, c.accepted);
        atomicAdd(&md.counters->margin, c.margin);
    }
}

// ---------------------------------------------------------------------------
// CTA per vertex (k > kWarpDeg); the table lives in dynamic shared memory

__device__ double block_sum_d(double v, double *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    __syncthreads();
    return r;  // valid in thread 0
}

__device__ int block_sum_i(int v, int *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum_i(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int r = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    __syncthreads();
    return r;  // valid in thread 0
}

__global__ void __launch_bounds__(kBigThreads) k_decide_cta(DecideArgs a, int cap, int cap_log2) {
    extern __shared__ unsigned long long smem_u64[];
    unsigned long long *cnt = smem_u64;
    int *keys = reinterpret_cast<int *>(cnt + cap);
    int *list = keys + cap;
    __shared__ int s_nlist, s_self, s_u, s_s;
    __shared__ int s_ok;
    __shared__ double sh_d[kBigThreads / 32];
    __shared__ int sh_i[kBigThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < cap; i += blockDim.x) {
        keys[i] = -1;
        cnt[i] = 0;
    }
    if (tid == 0) { s_nlist = 0; s_self = 0; s_ok = 1; }
    __syncthreads();

    const GraphDev &g = a.g;
    const ModelDev &md = a.md;
    Counts c;
    for (int64_t i = a.lo + blockIdx.x; i < a.hi; i += gridDim.x) {
        const int v = a.order[i];
        if (v < a.v_begin || v >= a.v_end) continue;
        const int r = md.b[v];
        const int o0 = g.op[v], kout = g.op[v + 1] - o0;
        const int i0 = g.ip[v], kin = g.ip[v + 1] - i0;
        const int k = kout + kin;
        const U64x4 w = philox4x64_10(a.sweep_id, (uint64_t)v, 0, 0, a.seed, 0);
        const int j = (int)draw_below(w.x, (uint64_t)k);
        for (int base = 0; base < k; base += blockDim.x) {
            const int idx = base + tid;
            const bool valid = idx < k, is_out = idx < kout;
            const int nb = valid ? (is_out ? g.oc[o0 + idx] : g.ic[i0 + idx - kout]) : -1;
            const int tb = valid ? md.b[nb] : -1;
            if (idx == j) s_u = tb;
            const bool is_self = valid && nb == v;
            const int nself = __popc(__ballot_sync(0xffffffffu, is_self && is_out));
            if (lane == 0 && nself) atomicAdd(&s_self, nself);
            const int key = (valid && !is_self) ? tb : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            const unsigned outm = __ballot_sync(0xffffffffu, valid && !is_self && is_out);
            if (key >= 0 && lane == __ffs(peers) - 1) {
                const unsigned ko = __popc(peers & outm), ki = __popc(peers) - ko;
                if (!table_add(keys, cnt, list, &s_nlist, cap, cap_log2, key,
                               (unsigned long long)ko | ((unsigned long long)ki << 32)))
                    s_ok = 0;
            }
        }
        __syncthreads();
        if (tid < 32) {
            const int s = propose_block(md, s_u, w.y);
            if (tid == 0) s_s = s;
        }
        __syncthreads();
        const int s = s_s, D = s_nlist, self = s_self, u_unused = s_u;
        (void)u_unused;
        if (tid == 0 && !s_ok) record_status(md.status, SBP_EHASHFULL);
        if (s == r) {
            if (tid == 0) {
                c.proposed++;
                write_trace(a, v, r, 1, 0.0, 0.0);
            }
        } else {
            double dL = 0.0, fwd = 0.0, bwd = 0.0;
            int ko_r = 0, ki_r = 0, ko_s = 0, ki_s = 0;
            for (int e = tid; e < D; e += blockDim.x) {
                const int slot = list[e];
                const int t = keys[slot];
                const unsigned long long cc = cnt[slot];
                const int ko = (int)(cc & 0xffffffffu), ki = (int)(cc >> 32);
                if (t == r) { ko_r = ko; ki_r = ki; }
                else if (t == s) { ko_s = ko; ki_s = ki; }
                else eval_entry(md, t, ko, ki, r, s, dL, fwd, bwd);
            }
            dL = block_sum_d(dL, sh_d);
            fwd = block_sum_d(fwd, sh_d);
            bwd = block_sum_d(bwd, sh_d);
            ko_r = block_sum_i(ko_r, sh_i);
            ki_r = block_sum_i(ki_r, sh_i);
            ko_s = block_sum_i(ko_s, sh_i);
            ki_s = block_sum_i(ki_s, sh_i);
            if (tid == 0) finalize(a, v, r, s, kout, kin, self, ko_r, ki_r, ko_s, ki_s, dL, fwd, bwd, w.z, c);
        }
        __syncthreads();
        for (int e = tid; e < D; e += blockDim.x) {
            const int slot = list[e];
            keys[slot] = -1;
            cnt[slot] = 0;
        }
        if (tid == 0) { s_nlist = 0; s_self = 0; }
        __syncthreads();
    }
    if (tid == 0 && (c.proposed | c.moves)) {
        atomicAdd(&md.counters->proposed, c.proposed);
        atomicAdd(&md.counters->moves, c.moves);
        atomicAdd(&md.counters->accepted, c.accepted);
        atomicAdd(&md.counters->margin, c.margin);
    }
}

int sm_count() {
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

ModelDev model_dev(sbp_model *m) {
    ModelDev d;
    d.B = m->B;
    d.n = (int32_t)m->g->n;
    d.m = m->g->m;
    d.b = m->b;
    d.bnew = m->bnew;
    d.M = m->M;
    d.P = m->P;
    d.dout = m->dout;
    d.din = m->din;
    d.rcp = m->rcp;
    d.status = m->status;
    d.counters = m->counters;
    return d;
}

int launch_decide(sbp_model *m, uint64_t sweep_id, int64_t v_begin, int64_t v_end, const sbp_vertex_trace *trace) {
    const sbp_graph *g = m->g;
    DecideArgs a;
    a.g = g->dev();
    a.md = model_dev(m);
    a.order = g->order;
    a.v_begin = v_begin;
    a.v_end = v_end;
    a.seed = m->p.seed;
    a.sweep_id = sweep_id;
    a.beta = m->p.beta;
    a.tr = trace ? *trace : sbp_vertex_trace{nullptr, nullptr, nullptr, nullptr};
    const bool want_trace = a.tr.s || a.tr.flags || a.tr.dH || a.tr.logA;
    const int sms = sm_count();

    // k <= kWarpDeg (and k = 0 when a trace is requested)
    a.lo = want_trace ? g->bin[0] : g->bin[1];
    a.hi = g->bin[3];
    if (a.hi > a.lo) {
        const int64_t warps = a.hi - a.lo;
        int64_t blocks = (warps + kWarpsPerCta - 1) / kWarpsPerCta;
        if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
        k_decide_warp<<<(int)blocks, kWarpsPerCta * 32, 0, m->stream>>>(a);
        SBP_CUDA(cudaGetLastError());
    }
    // k > kWarpDeg
    a.lo = g->bin[3];
    a.hi = g->bin[4];
    if (a.hi > a.lo) {
        int64_t need = 2 * (int64_t)(g->max_deg < m->B ? g->max_deg : m->B) + 2;
        int cap_log2 = 6;
        while ((int64_t(1) << cap_log2) < need) ++cap_log2;
        const int cap = 1 << cap_log2;
        const size_t smem = (size_t)cap * (8 + 4 + 4);
        if (smem > 200 * 1024) return fail(SBP_ESTATE, "nodal pass: neighbour table does not fit shared memory");
        SBP_CUDA(cudaFuncSetAttribute(k_decide_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int64_t blocks = a.hi - a.lo;
        if (blocks > (int64_t)sms * 4) blocks = (int64_t)sms * 4;
        k_decide_cta<<<(int)blocks, kBigThreads, smem, m->stream>>>(a, cap, cap_log2);
        SBP_CUDA(cudaGetLastError());
    }
    return SBP_OK;
}

}  // namespace sbp
