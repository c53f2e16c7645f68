// nodal.cu -- the asynchronous-Gibbs nodal decision pass of one graph.
//
// Vertices are split by total degree into three groups (k <= 32, 33..128,
// above 128), each with its own evaluation kernel: k_eval_batch (32 movers
// per warp; for 33..128 with direct-mapped counts while B is small),
// k_eval_warp_direct (one warp per mover, direct-mapped counts) or, at
// larger B, k_eval_warp (one warp per mover with a shared-memory table) and
// k_eval_cta (one CTA per mover, very large tables).  In a pass over all
// vertices without a trace the first two kinds draw the proposals of their
// group's vertices themselves; otherwise k_propose (one lane per vertex)
// draws every proposal first and hands the moving ones (s != r) over in
// lists by group.  Only movers' rows are aggregated.  Moves the FP32 test
// cannot settle are decided after the pass by the exact evaluation
// (k_eval_cta in recheck mode).  The decision goes to the pending
// assignment; M is untouched until commit.  The steps and their numerics
// are described in nodal_dev.cuh.
#include <algorithm>
#include <cmath>

#include "nodal_dev.cuh"

// CTAs per SM the evaluation kernels are compiled for (register budget:
// 80 registers at 3, 64 at 4; the direct-mapped kernel for the largest rows
// fits 4 without spilling once the exact evaluation is a kernel of its own)
#ifndef SBP_DECIDE_MIN_BLOCKS
#define SBP_DECIDE_MIN_BLOCKS 3
#endif
#ifndef SBP_DIRECT_MIN_BLOCKS
#define SBP_DIRECT_MIN_BLOCKS 4
#endif
// 1: full-range passes draw the proposals inside the evaluation kernels;
// 0: always k_propose first (for comparison builds)
#ifndef SBP_FUSED_PROPOSALS
#define SBP_FUSED_PROPOSALS 1
#endif

namespace sbp {
namespace {

// Proposal of every vertex in [v_begin, v_end).  Proposals with s = r end
// here; the others are appended to the list of their degree group.
__global__ void __launch_bounds__(256) k_propose(DecideArgs a) {
    const ModelDev &md = a.md;
    const GraphDev &g = a.g;
    const int lane = threadIdx.x & 31;
    Counts c;
    unsigned long long medges = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = a.v_begin + (int64_t)blockIdx.x * blockDim.x; base < a.v_end; base += stride) {
        const int64_t vv = base + threadIdx.x;
        int bin = -1, s = 0, v = (int)vv;
        uint64_t w2 = 0;
        if (vv < a.v_end && !(a.skip && a.skip[v])) {
            const Proposal p = propose_vertex(g, md, a.seed, a.sweep_id, v);
            s = p.s;
            if (p.k == 0) {
                write_trace(a, v, p.r, 0, 0.0, 0.0);
            } else if (p.s == p.r) {
                c.proposed++;
                write_trace(a, v, p.r, 1, 0.0, 0.0);
            } else {
                bin = p.k <= kSmallDeg ? 0 : p.k <= kWarpDeg ? 1 : 2;
                w2 = p.w2;
                medges += (unsigned long long)p.k;
            }
        }
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
            const unsigned msk = __ballot_sync(0xffffffffu, bin == bb);
            if (msk == 0) continue;
            const int leader = __ffs(msk) - 1;
            unsigned pos0 = 0;
            if (lane == leader) pos0 = atomicAdd(&a.mcount[bb], (unsigned)__popc(msk));
            pos0 = __shfl_sync(0xffffffffu, pos0, leader);
            if (bin == bb) {
                Mover mv;
                mv.v = v;
                mv.s = s;
                mv.w2 = w2;
                a.movers[a.mbase[bb] + pos0 + __popc(msk & ((1u << lane) - 1u))] = mv;
            }
        }
    }
    flush_counts_warp(md, c, medges);
}

// One warp per mover of list `bin` (k >= 33).  Dynamic shared memory per
// warp: cap int keys, cap 32-bit counts (ko | ki << 16, degrees below
// 65536), cap 16-bit list entries, one list length.  Warps take chunks of
// `chunk` movers and prefetch their records with one lane per mover.
template <bool DL32>
__global__ void __launch_bounds__(kWarpsPerCta * 32, SBP_DECIDE_MIN_BLOCKS) k_eval_warp(DecideArgs a, int bin, int cap,
                                                                                    int cap_log2, int chunk) {
    extern __shared__ int dsm[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const ModelDev &md = a.md;
    const GraphDev &g = a.g;
    int *keys = dsm + (size_t)wid * cap;
    unsigned *cnt = reinterpret_cast<unsigned *>(dsm + (size_t)nwarps * cap) + (size_t)wid * cap;
    int *nlist = dsm + (size_t)2 * nwarps * cap + wid;
    unsigned short *list = reinterpret_cast<unsigned short *>(dsm + (size_t)2 * nwarps * cap + nwarps) + (size_t)wid * cap;
    for (int i = lane; i < cap; i += 32) {
        keys[i] = -1;
        cnt[i] = 0;
    }
    if (lane == 0) *nlist = 0;
    __syncwarp();

    const Mover *mlist = a.movers + a.mbase[bin];
    const int64_t count = *(volatile unsigned *)&a.mcount[bin];
    Counts c;
    const int64_t nw = (int64_t)gridDim.x * nwarps;
    const int64_t nchunk = (count + chunk - 1) / chunk;
    for (int64_t ch = (int64_t)blockIdx.x * nwarps + wid; ch < nchunk; ch += nw) {
        const int64_t first = ch * chunk;
        const int cnt_v = (int)(count - first < chunk ? count - first : chunk);
        int pv = 0, ps = 0, pr = 0, po = 0, pko = 0, pi = 0, pki = 0;
        uint64_t pw2 = 0;
        if (lane < cnt_v) {
            const Mover mv = mlist[first + lane];
            pv = mv.v;
            ps = mv.s;
            pw2 = mv.w2;
            pr = md.b[pv];
            po = g.op[pv];
            pko = g.op[pv + 1] - po;
            pi = g.ip[pv];
            pki = g.ip[pv + 1] - pi;
        }
        for (int q = 0; q < cnt_v; ++q) {
            const int v = __shfl_sync(0xffffffffu, pv, q);
            const int s = __shfl_sync(0xffffffffu, ps, q);
            const int r = __shfl_sync(0xffffffffu, pr, q);
            const int o0 = __shfl_sync(0xffffffffu, po, q), kout = __shfl_sync(0xffffffffu, pko, q);
            const int i0 = __shfl_sync(0xffffffffu, pi, q), kin = __shfl_sync(0xffffffffu, pki, q);
            const uint64_t w2 = __shfl_sync(0xffffffffu, pw2, q);
            const int k = kout + kin;
            // aggregate the row: four 32-neighbour chunks per round
            int self = 0;
            bool ok = true;
            for (int base = 0; base < k; base += 128) {
                int nb[4], tb[4];
                bool sf[4];
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const int idx = base + c4 * 32 + lane;
                    nb[c4] = idx < k ? nb_raw(g, md, o0, i0, kout, idx) : 0;
                }
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const int idx = base + c4 * 32 + lane;
                    sf[c4] = false;
                    tb[c4] = idx < k ? nb_block(md, nb[c4], v, sf[c4]) : -1;
                }
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const int cb = base + c4 * 32;
                    if (cb >= k) break;
                    const int idx = cb + lane;
                    const bool valid = idx < k, is_out = idx < kout;
                    const bool is_self = valid && sf[c4];
                    self += __popc(__ballot_sync(0xffffffffu, is_self && is_out));
                    const int key = (valid && !is_self) ? tb[c4] : -1;
                    const unsigned peers = __match_any_sync(0xffffffffu, key);
                    const unsigned outm = __ballot_sync(0xffffffffu, valid && !is_self && is_out);
                    if (key >= 0 && lane == __ffs(peers) - 1) {
                        const unsigned ko = __popc(peers & outm), ki = __popc(peers) - ko;
                        ok &= table_add32(keys, cnt, list, nlist, cap, cap_log2, key, ko | (ki << 16));
                    }
                    __syncwarp();
                }
            }
            if (!ok) record_status(md.status, SBP_EHASHFULL);
            const int D = *nlist;
            if (lane == 0) c.entries += (unsigned)D;
            VertexCtx x;
            x.v = v; x.r = r; x.s = s;
            x.Kout = kout; x.Kin = kin; x.self = self; x.k = k;
            evaluate_warp<DL32>(a, md, x, w2, [&](auto &&f) {
                for (int e = lane; e < D; e += 32) {
                    const int slot = list[e];
                    const unsigned cc = cnt[slot];
                    f(keys[slot], (int)(cc & 0xffffu), (int)(cc >> 16));
                }
            }, c);
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
    if (lane == 0) flush_counts(md, c);
}

// ---------------------------------------------------------------------------
// One warp per mover with direct-mapped counts (B <= kDirectMaxB): the row's
// neighbour blocks go straight into a per-warp array of B counts (ko | ki <<
// 16) with shared-memory atomics, the first touch of a block (an atomic that
// returns 0) appends it to the warp's list.  No table probing and no warp
// match; eight 32-edge chunks in flight per round.  Degrees below 65536.
constexpr int kDirectChunks = 8;

// one mover (v, s, w2) on the whole warp, counts in cnt[B] (all zero on entry
// and on return), first touches in list
template <bool DL32>
__device__ __forceinline__ void direct_mover(const DecideArgs &a, unsigned *cnt, int *list, int v, int s, uint64_t w2,
                                             Counts &c) {
    const int lane = threadIdx.x & 31;
    const ModelDev &md = a.md;
    const GraphDev &g = a.g;
    const int r = md.b[v];
    const int o0 = g.op[v], kout = g.op[v + 1] - o0;
    const int i0 = g.ip[v], kin = g.ip[v + 1] - i0;
    const int k = kout + kin;
    int nl = 0, self = 0;
    for (int base = 0; base < k; base += 32 * kDirectChunks) {
        int nb[kDirectChunks], tb[kDirectChunks];
#pragma unroll
        for (int c8 = 0; c8 < kDirectChunks; ++c8) {
            const int idx = base + c8 * 32 + lane;
            nb[c8] = idx < k ? nb_raw(g, md, o0, i0, kout, idx) : 0;
        }
        bool sf[kDirectChunks];
#pragma unroll
        for (int c8 = 0; c8 < kDirectChunks; ++c8) {
            const int idx = base + c8 * 32 + lane;
            sf[c8] = false;
            tb[c8] = idx < k ? nb_block(md, nb[c8], v, sf[c8]) : -1;
        }
#pragma unroll
        for (int c8 = 0; c8 < kDirectChunks; ++c8) {
            const int idx = base + c8 * 32 + lane;
            const bool is_out = idx < kout, is_self = idx < k && sf[c8];
            self += __popc(__ballot_sync(0xffffffffu, is_self && is_out));
            bool fresh = false;
            if (tb[c8] >= 0 && !is_self) fresh = atomicAdd(&cnt[tb[c8]], is_out ? 1u : 0x10000u) == 0u;
            const unsigned fm = __ballot_sync(0xffffffffu, fresh);
            if (fresh) list[nl + __popc(fm & ((1u << lane) - 1u))] = tb[c8];
            nl += __popc(fm);
        }
    }
    __syncwarp();
    VertexCtx x;
    x.v = v; x.r = r; x.s = s;
    x.Kout = kout; x.Kin = kin; x.self = self; x.k = k;
    const int D = nl;
    if (lane == 0) c.entries += (unsigned)D;
    evaluate_warp<DL32>(a, md, x, w2, [&](auto &&f) {
        for (int e = lane; e < D; e += 32) {
            const int t = list[e];
            const unsigned cc = cnt[t];
            f(t, (int)(cc & 0xffffu), (int)(cc >> 16));
        }
    }, c);
    __syncwarp();
    for (int e = lane; e < D; e += 32) cnt[list[e]] = 0u;
    __syncwarp();
}

// One warp per mover with direct-mapped counts.  FUSED = false: the movers
// of list `bin`.  FUSED = true: the warps draw the proposals of the group's
// vertices themselves, warp w taking the vertices w, w + W, w + 2W, ... of
// the group (W warps in the grid; the group is sorted by descending degree,
// so every warp gets a share of the largest rows), one per lane, then
// evaluates its movers one after another.
template <bool DL32, bool FUSED>
__global__ void __launch_bounds__(kWarpsPerCta * 32, SBP_DIRECT_MIN_BLOCKS) k_eval_warp_direct(DecideArgs a, int bin,
                                                                                           int warp_words) {
    extern __shared__ unsigned dmw[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const ModelDev &md = a.md;
    const int B = md.B;
    unsigned *cnt = dmw + (size_t)wid * warp_words;
    int *list = reinterpret_cast<int *>(cnt + B);
    for (int i = lane; i < B; i += 32) cnt[i] = 0u;
    __syncwarp();
    Counts c;
    const int64_t gw = (int64_t)blockIdx.x * nwarps + wid, nw = (int64_t)gridDim.x * nwarps;
    if constexpr (!FUSED) {
        const Mover *mlist = a.movers + a.mbase[bin];
        const int64_t count = *(volatile unsigned *)&a.mcount[bin];
        for (int64_t q = gw; q < count; q += nw) {
            const Mover mv = mlist[q];
            direct_mover<DL32>(a, cnt, list, mv.v, mv.s, mv.w2, c);
        }
        if (lane == 0) flush_counts(md, c);
    } else {
        const int32_t *vl = a.vlist[bin];
        const int64_t vcount = a.vcount[bin];
        unsigned long long medges = 0;
        for (int64_t j0 = 0; gw + j0 * nw < vcount; j0 += 32) {
            const int64_t i = gw + (j0 + lane) * nw;
            bool mover = false;
            int pv = 0, ps = 0;
            uint64_t pw = 0;
            if (i < vcount) {
                pv = vl[i];
                const Proposal p = propose_vertex(a.g, md, a.seed, a.sweep_id, pv);
                if (p.s == p.r) {
                    c.proposed++;
                } else {
                    mover = true;
                    ps = p.s;
                    pw = p.w2;
                    medges += (unsigned long long)p.k;
                }
            }
            unsigned mask = __ballot_sync(0xffffffffu, mover);
            while (mask) {
                const int q = __ffs(mask) - 1;
                mask &= mask - 1u;
                const int v = __shfl_sync(0xffffffffu, pv, q), s = __shfl_sync(0xffffffffu, ps, q);
                const uint64_t w2 = __shfl_sync(0xffffffffu, pw, q);
                direct_mover<DL32>(a, cnt, list, v, s, w2, c);
            }
        }
        flush_counts_warp(md, c, medges);
    }
}

// ---------------------------------------------------------------------------
// CTA per mover: tables beyond 4096 slots or degree >= 65536

struct CtaScratch {
    __int128 dl[kBigThreads / 32];
    double fb[kBigThreads / 32], pf64[kBigThreads / 32], pb64[kBigThreads / 32];
    float pf[kBigThreads / 32], pb[kBigThreads / 32], dlf[kBigThreads / 32], am[kBigThreads / 32];
    __int128 dl_tot;
    double fb_tot;
    int rs[4];
    int nlist, self, ok, dec;
};

// gtab: NULL, or a global scratch of 2 cap words per CTA for tables that do
// not fit shared memory
template <bool DL32>
__global__ void __launch_bounds__(kBigThreads) k_eval_cta(DecideArgs a, int bin, int cap, int cap_log2,
                                                          unsigned long long *gtab) {
    extern __shared__ unsigned long long smem_u64[];
    // CTAs beyond the list's length have nothing to do (the recheck launch
    // is usually nearly empty)
    if ((int64_t)blockIdx.x >= (int64_t)(*(volatile unsigned *)&a.mcount[bin])) return;
    unsigned long long *cnt = gtab ? gtab + (size_t)blockIdx.x * 2 * (size_t)cap : smem_u64;
    int *keys = reinterpret_cast<int *>(cnt + cap);
    int *list = keys + cap;
    __shared__ CtaScratch sh;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = kBigThreads / 32;
    for (int i = tid; i < cap; i += blockDim.x) {
        keys[i] = -1;
        cnt[i] = 0;
    }
    if (tid == 0) {
        sh.nlist = 0;
        sh.self = 0;
        sh.ok = 1;
    }
    __syncthreads();

    const GraphDev &g = a.g;
    const ModelDev &md = a.md;
    const Mover *mlist = a.movers + a.mbase[bin];
    const int64_t count = *(volatile unsigned *)&a.mcount[bin];
    Counts c;
    for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
        const Mover mv = mlist[i];
        const int v = mv.v, s = mv.s;
        const int r = md.b[v];
        const int o0 = g.op[v], kout = g.op[v + 1] - o0;
        const int i0 = g.ip[v], kin = g.ip[v + 1] - i0;
        const int k = kout + kin;
        if (tid < 4) sh.rs[tid] = 0;
        for (int base = 0; base < k; base += blockDim.x) {
            const int idx = base + tid;
            const bool valid = idx < k, is_out = idx < kout;
            bool sfl = false;
            const int tb = valid ? nb_block(md, nb_raw(g, md, o0, i0, kout, idx), v, sfl) : -1;
            const bool is_self = valid && sfl;
            const int nself = __popc(__ballot_sync(0xffffffffu, is_self && is_out));
            if (lane == 0 && nself) atomicAdd(&sh.self, nself);
            const int key = (valid && !is_self) ? tb : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            const unsigned outm = __ballot_sync(0xffffffffu, valid && !is_self && is_out);
            if (key >= 0 && lane == __ffs(peers) - 1) {
                const unsigned ko = __popc(peers & outm), ki = __popc(peers) - ko;
                if (!table_add(keys, cnt, list, &sh.nlist, cap, cap_log2, key,
                               (unsigned long long)ko | ((unsigned long long)ki << 32)))
                    sh.ok = 0;
            }
        }
        __syncthreads();
        const int D = sh.nlist;
        if (tid == 0 && !sh.ok) record_status(md.status, SBP_EHASHFULL);
        if (tid == 0 && !a.force_exact) c.entries += (unsigned)D;
        VertexCtx x;
        x.v = v; x.r = r; x.s = s;
        x.Kout = kout; x.Kin = kin; x.self = sh.self; x.k = k;
        for (int e = tid; e < D; e += blockDim.x) {
            const int slot = list[e];
            const int t = keys[slot];
            const unsigned long long cc = cnt[slot];
            if (t == r) { sh.rs[0] = (int)(cc & 0xffffffffu); sh.rs[1] = (int)(cc >> 32); }
            if (t == s) { sh.rs[2] = (int)(cc & 0xffffffffu); sh.rs[3] = (int)(cc >> 32); }
        }
        __syncthreads();
        x.ko_r = sh.rs[0]; x.ki_r = sh.rs[1]; x.ko_s = sh.rs[2]; x.ki_s = sh.rs[3];
        __int128 dl = 0;
        double fb = 0.0;
        float pf = 0.0f, pb = 0.0f, dlf = 0.0f, am = 0.0f;
        // the FP32 pass only feeds the FP32 test; when the exact evaluation
        // decides anyway (the recheck launch, a trace) it is skipped (the
        // exact form's pass also yields the exact Delta L, so it stays)
        const bool fast_pass = !DL32 || (!a.trace_on && !a.force_exact);
        for (int e = tid; fast_pass && e < D; e += blockDim.x) {
            const int slot = list[e];
            const int t = keys[slot];
            const unsigned long long cc = cnt[slot];
            if (t != r && t != s) {
                if (DL32)
                    entry_fast32(md, x, t, (int)(cc & 0xffffffffu), (int)(cc >> 32), dlf, am, pf, pb);
                else
                    entry_fast(md, x, t, (int)(cc & 0xffffffffu), (int)(cc >> 32), dl, fb, pf, pb);
            }
        }
        if (fast_pass && tid < 32) {
            if (DL32)
                special_terms32(md, x, tid, dlf, am);
            else
                special_terms(md, x, tid, dl, fb);
        }
        pf = warp_sum_f(pf);
        pb = warp_sum_f(pb);
        if (DL32) {
            dlf = warp_sum_f(dlf);
            am = warp_sum_f(am);
        } else {
            dl = warp_sum_128(dl);
            if (__any_sync(0xffffffffu, __double_as_longlong(fb) != 0)) fb = warp_sum(fb);
        }
        if (lane == 0) {
            sh.dl[wid] = dl;
            sh.fb[wid] = fb;
            sh.pf[wid] = pf;
            sh.pb[wid] = pb;
            sh.dlf[wid] = dlf;
            sh.am[wid] = am;
        }
        __syncthreads();
        CornerVals cv;
        Mat4corner(md, r, s, cv.Mrr, cv.Mss, cv.Mrs, cv.Msr);
        cv.dr = md.dsum[r];
        cv.ds = md.dsum[s];
        if (tid == 0) {
            __int128 dlt = 0;
            double fbt = 0.0;
            float pft = 0.0f, pbt = 0.0f, dlft = 0.0f, amt = 0.0f;
            for (int q = 0; q < nwarps; ++q) {
                dlt += sh.dl[q];
                fbt += sh.fb[q];
                pft += sh.pf[q];
                pbt += sh.pb[q];
                dlft += sh.dlf[q];
                amt += sh.am[q];
            }
            sh.dl_tot = dlt;
            sh.fb_tot = fbt;
            corner_hastings_fast(x, cv, md.B, pft, pbt);
            int dec = -1;
            if (!a.trace_on && !a.force_exact) {
                if (DL32)
                    dec = fast_decision_f(a.beta32, dlft, 0.0f, pft, pbt, mv.w2, k, dl32_error(amt, k));
                else
                    dec = fast_decision(a.beta32, dlt, __double_as_longlong(fbt) != 0, fbt, pft, pbt, mv.w2, k);
            }
            sh.dec = dec;
            if (dec >= 0) {
                if (dec) accept_move(md, v, s, x.k);
                count_result(c, dec != 0, false, x.k);
            }
        }
        __syncthreads();
        if (sh.dec < 0) {
            double pf64 = 0.0, pb64 = 0.0;
            __int128 dle = 0;
            double fbe = 0.0;
            for (int e = tid; e < D; e += blockDim.x) {
                const int slot = list[e];
                const int t = keys[slot];
                const unsigned long long cc = cnt[slot];
                if (t != r && t != s) {
                    if (DL32)
                        entry_exact_all(md, x, t, (int)(cc & 0xffffffffu), (int)(cc >> 32), dle, fbe, pf64, pb64);
                    else
                        entry_exact(md, x, t, (int)(cc & 0xffffffffu), (int)(cc >> 32), pf64, pb64);
                }
            }
            if (DL32) {
                if (tid < 32) special_terms(md, x, tid, dle, fbe);
                dle = warp_sum_128(dle);
                if (__any_sync(0xffffffffu, __double_as_longlong(fbe) != 0)) fbe = warp_sum(fbe);
                if (lane == 0) {
                    sh.dl[wid] = dle;
                    sh.fb[wid] = fbe;
                }
            }
            pf64 = warp_sum(pf64);
            pb64 = warp_sum(pb64);
            if (lane == 0) {
                sh.pf64[wid] = pf64;
                sh.pb64[wid] = pb64;
            }
            __syncthreads();
            if (tid == 0) {
                double pft = 0.0, pbt = 0.0;
                __int128 dlt = sh.dl_tot;
                double fbt = sh.fb_tot;
                if (DL32) {
                    dlt = 0;
                    fbt = 0.0;
                    for (int q = 0; q < nwarps; ++q) {
                        dlt += sh.dl[q];
                        fbt += sh.fb[q];
                    }
                }
                for (int q = 0; q < nwarps; ++q) {
                    pft += sh.pf64[q];
                    pbt += sh.pb64[q];
                }
                corner_hastings_exact(x, cv, md.B, pft, pbt);
                const Exact e = exact_decision(a.beta, dlt, fbt, pft, pbt, mv.w2);
                if (e.accept) accept_move(md, v, s, k);
                count_exact(c, e.accept, e.margin, k);
                write_trace(a, v, s, 1 | (e.accept ? 2 : 0) | (e.margin ? 4 : 0), e.dH, e.logA);
            }
        }
        __syncthreads();
        for (int e = tid; e < D; e += blockDim.x) {
            const int slot = list[e];
            keys[slot] = -1;
            cnt[slot] = 0;
        }
        if (tid == 0) {
            sh.nlist = 0;
            sh.self = 0;
        }
        __syncthreads();
    }
    if (tid == 0) flush_counts(md, c);
}

// ---------------------------------------------------------------------------
// moves of vertices with 1 <= k <= 32: batches of 32 movers per warp
//
//   P1 lane per mover: record, offsets, label; exclusive prefix of k;
//   P2 edge parallel over the batch's concatenated rows (four 32-wide
//      chunks in flight): neighbour blocks into shared memory, tagged with
//      the mover's slot;
//   P3 windows of whole rows (at most 32 edge ends): match/ballot
//      aggregation into (q, t, kout, kin) entries, compacted in place, in
//      row order;
//   P5 entry parallel: Delta L (table sums, per entry in 64-bit fixed point
//      at 2^-48) and FP32 Hastings terms, summed per mover by a segmented
//      warp scan (entries of a mover are contiguous);
//   P6 lane per mover: corner and degree terms, FP32 test with its band;
//      a move the band does not settle goes to the recheck list.

// rows of at most 32 edges: sub-batches of 512 edge ends keep a CTA's
// shared memory at 38 KB, so that 4 CTAs (64 registers each) fit an SM
#ifndef SBP_BATCH0_EDGES
#define SBP_BATCH0_EDGES 512
#endif
#ifndef SBP_BATCH0_MIN_BLOCKS
#define SBP_BATCH0_MIN_BLOCKS 4
#endif
constexpr int kBatchEdges = 32 * kSmallDeg;     // edge ends per sub-batch (33..128)
constexpr int kBatchEdges0 = SBP_BATCH0_EDGES;  // ... for rows of at most 32
constexpr int kDirectMaxB = 2048;  // direct-mapped per-warp counts up to this B

template <int EDGES>
struct BatchWarpT {
    int key[EDGES];  // edge ends (q << 26 | self << 25 | t << 1 | in), then entries (q << 26 | t)
    unsigned short ec[EDGES];  // entry counts ko | ki << 8
    int r[32], s[32], rsr[32], rss[32], hasfb[32];
    long long dl[32];  // Delta L, fixed point 2^-48
    float pf[32], pb[32];
    float dlf[32], am[32];  // FP32 Delta L and its magnitude sum (precision form)
    double fb[32];
};

template <int MODE>
using BatchWarp = BatchWarpT<MODE == 0 ? kBatchEdges0 : kBatchEdges>;


__device__ __forceinline__ float fix48_to_float(long long v) {
    return fmaf((float)(int)(v >> 32), 0x1p-16f, (float)(unsigned)(v & 0xffffffffu) * 0x1p-48f);
}
__device__ __forceinline__ double fix48_to_double(long long v) {
    return (double)(int)(v >> 32) * 0x1p-16 + (double)(unsigned)(v & 0xffffffffu) * 0x1p-48;
}

// The evaluation of up to 32 movers of one warp: lane q < nv holds mover q
// (v, s, w2).  MODE 0: rows of at most 32 edges (aggregated in windows of
// whole rows); MODE 1: rows of 33..128 edges (aggregated per mover in a
// direct-mapped count array of B entries, dcnt, with its touch list dlist,
// which follow the warp's BatchWarp in shared memory).  Movers are taken in
// sub-batches of at most kBatchEdges edge ends.
template <int MODE, bool DL32>
__device__ __forceinline__ void batch_movers(const DecideArgs &a, BatchWarp<MODE> &W, unsigned *dcnt, int *dlist,
                                             const int nv, int v, int s, uint64_t w2, Counts &c) {
    constexpr int kEdges = MODE == 0 ? kBatchEdges0 : kBatchEdges;
    const int lane = threadIdx.x & 31;
    const GraphDev &g = a.g;
    const ModelDev &md = a.md;
    const int B = md.B;
    // ---- P1 (the mover records are in registers)
    int r = 0, o0 = 0, kout = 0, i0 = 0, kin = 0, k = 0;
    if (lane < nv) {
        r = md.b[v];
        o0 = g.op[v];
        kout = g.op[v + 1] - o0;
        i0 = g.ip[v];
        kin = g.ip[v + 1] - i0;
        k = kout + kin;
    } else {
        v = 0;
        s = -1;
        w2 = 0;
    }
    int incl = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int first = incl - k;
    // sub-batches of whole rows with at most kBatchEdges edge ends
    for (int sa = 0; sa < nv;) {
    const int fs = __shfl_sync(0xffffffffu, first, sa);
    const unsigned fit = __ballot_sync(0xffffffffu, lane >= sa && lane < nv && incl - fs <= kEdges);
    const int sb = 31 - __clz(fit);
    const int total = __shfl_sync(0xffffffffu, incl, sb) - fs;
    const bool act = lane >= sa && lane <= sb;
    // ---- P2 (eight 32-edge chunks in flight for the longer rows of MODE 1)
    constexpr int kP2 = MODE == 1 ? 8 : 4;
    for (int base = 0; base < total; base += 32 * kP2) {
        int nb[kP2], vq[kP2], tag[kP2];
#pragma unroll
        for (int c4 = 0; c4 < kP2; ++c4) {
            const int pp = base + c4 * 32 + lane;
            const int p = fs + pp;
            int q = 0;
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1) {
                const int f = __shfl_sync(0xffffffffu, first, q + st);
                if (f <= p) q += st;
            }
            const int fq = __shfl_sync(0xffffffffu, first, q);
            const int kq = __shfl_sync(0xffffffffu, kout, q);
            const int oq = __shfl_sync(0xffffffffu, o0, q);
            const int iq = __shfl_sync(0xffffffffu, i0, q);
            vq[c4] = __shfl_sync(0xffffffffu, v, q);
            const int e = p - fq;
            tag[c4] = (q << 26) | (e < kq ? 0 : 1);
            nb[c4] = pp < total ? nb_raw(g, md, oq, iq, kq, e) : 0;
        }
#pragma unroll
        for (int c4 = 0; c4 < kP2; ++c4) {
            const int pp = base + c4 * 32 + lane;
            if (pp < total) {
                bool sfl;
                const int t = nb_block(md, nb[c4], vq[c4], sfl);
                W.key[pp] = sfl ? (tag[c4] | (1 << 25)) : (tag[c4] | (t << 1));
            }
        }
    }
    __syncwarp();
    int nent = 0, my_self = 0, my_est = 0, my_ecnt = 0;
    if (MODE == 0) {
    // ---- P3: windows of whole rows
    for (int qa = sa; qa <= sb;) {
        const int fa = __shfl_sync(0xffffffffu, first, qa);
        const unsigned inw = __ballot_sync(0xffffffffu, lane >= qa && lane <= sb && incl - fa <= 32);
        const int qb = 31 - __clz(inw);
        const int wend = __shfl_sync(0xffffffffu, incl, qb);
        const int p = fa + lane;
        const bool valid = p < wend;
        const int x = valid ? W.key[p - fs] : 0;
        const bool selfl = valid && ((x >> 25) & 1);
        const bool in = (x & 1) != 0;
        const bool isent = valid && !selfl;
        const int mkey = isent ? (x >> 1) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, mkey);
        const unsigned outm = __ballot_sync(0xffffffffu, isent && !in);
        const unsigned sfl = __ballot_sync(0xffffffffu, selfl && !in);
        const bool leader = isent && lane == __ffs(peers) - 1;
        const unsigned lm = __ballot_sync(0xffffffffu, leader);
        if (leader) {
            const int ko = __popc(peers & outm), ki = __popc(peers) - ko;
            const int pos = nent + __popc(lm & ((1u << lane) - 1u));
            W.key[pos] = (x & (31 << 26)) | ((x >> 1) & 0xffffff);
            W.ec[pos] = (unsigned short)(ko | (ki << 8));
        }
        if (lane >= qa && lane <= qb) {
            const int lo_l = first - fa, hi_l = incl - fa;
            const unsigned below = (1u << lo_l) - 1u;
            const unsigned mq = (hi_l >= 32 ? 0xffffffffu : ((1u << hi_l) - 1u)) & ~below;
            my_self = __popc(sfl & mq);
            my_est = nent + __popc(lm & below);
            my_ecnt = __popc(lm & mq);
        }
        nent += __popc(lm);
        qa = qb + 1;
    }
    } else {
    // ---- P3: per mover, direct-mapped counts; first touches kept in
    // order of appearance (ballot compaction), so entries are deterministic
    for (int q = sa; q <= sb; ++q) {
        const int kq = __shfl_sync(0xffffffffu, k, q);
        const int fq = __shfl_sync(0xffffffffu, first, q) - fs;
        int nl = 0, selfq = 0;
        for (int c0 = 0; c0 < kq; c0 += 32) {
            const bool valid = c0 + lane < kq;
            const int x = valid ? W.key[fq + c0 + lane] : 0;
            const bool selfl = valid && ((x >> 25) & 1);
            const bool in = (x & 1) != 0;
            const bool isent = valid && !selfl;
            const int t = isent ? ((x >> 1) & 0xffffff) : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, t);
            const unsigned outm = __ballot_sync(0xffffffffu, isent && !in);
            selfq += __popc(__ballot_sync(0xffffffffu, selfl && !in));
            const bool leader = isent && lane == __ffs(peers) - 1;
            bool fresh = false;
            if (leader) {
                const unsigned ko = __popc(peers & outm), ki = __popc(peers) - ko;
                fresh = atomicAdd(&dcnt[t], ko | (ki << 16)) == 0u;
            }
            const unsigned fm = __ballot_sync(0xffffffffu, fresh);
            if (fresh) dlist[nl + __popc(fm & ((1u << lane) - 1u))] = t;
            nl += __popc(fm);
            __syncwarp();
        }
        for (int e = lane; e < nl; e += 32) {
            const int t = dlist[e];
            const unsigned cc = dcnt[t];
            dcnt[t] = 0u;
            W.key[nent + e] = (q << 26) | t;
            W.ec[nent + e] = (unsigned short)((cc & 0xffu) | ((cc >> 16) << 8));
        }
        if (lane == q) {
            my_self = selfq;
            my_est = nent;
            my_ecnt = nl;
        }
        nent += nl;
        __syncwarp();
    }
    }
    W.r[lane] = r;
    W.s[lane] = act ? s : -1;
    W.rsr[lane] = 0;
    W.rss[lane] = 0;
    W.hasfb[lane] = 0;
    W.dl[lane] = 0;
    W.pf[lane] = 0.0f;
    W.pb[lane] = 0.0f;
    W.dlf[lane] = 0.0f;
    W.am[lane] = 0.0f;
    W.fb[lane] = 0.0;
    __syncwarp();
    // ---- P5: entry parallel, segmented sums per mover
    for (int base = 0; base < nent; base += 32) {
        const int e = base + lane;
        const bool valid = e < nent;
        const unsigned ent = valid ? (unsigned)W.key[e] : 0u;
        const int q = valid ? (int)(ent >> 26) : 32;
        long long d48 = 0;
        float pfe = 0.0f, pbe = 0.0f, dlf = 0.0f, am = 0.0f;
        double f = 0.0;
        if (valid) {
            const int t = (int)(ent & 0x3ffffffu);
            const unsigned ec = W.ec[e];
            const int ko = (int)(ec & 0xffu), ki = (int)(ec >> 8);
            const int rq = W.r[q], sq = W.s[q];
            if (t == rq) {
                W.rsr[q] = ko | (ki << 8);
            } else if (t == sq) {
                W.rss[q] = ko | (ki << 8);
            } else {
                VertexCtx x;
                x.r = rq;
                x.s = sq;
                if (DL32) {
                    entry_fast32(md, x, t, ko, ki, dlf, am, pfe, pbe);
                } else {
                    __int128 d = 0;
                    entry_fast(md, x, t, ko, ki, d, f, pfe, pbe);
                    d48 = (long long)(d >> 16);
                }
            }
        }
        const bool anyfb = !DL32 && __any_sync(0xffffffffu, __double_as_longlong(f) != 0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int qo = __shfl_up_sync(0xffffffffu, q, o);
            const float p2 = __shfl_up_sync(0xffffffffu, pfe, o);
            const float b2 = __shfl_up_sync(0xffffffffu, pbe, o);
            if (DL32) {
                const float l2 = __shfl_up_sync(0xffffffffu, dlf, o);
                const float a2 = __shfl_up_sync(0xffffffffu, am, o);
                if (lane >= o && qo == q) {
                    dlf += l2;
                    am += a2;
                }
            } else {
                const long long d2 = __shfl_up_sync(0xffffffffu, d48, o);
                if (lane >= o && qo == q) d48 += d2;
            }
            if (lane >= o && qo == q) {
                pfe += p2;
                pbe += b2;
            }
        }
        if (anyfb) {
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int qo = __shfl_up_sync(0xffffffffu, q, o);
                const double f2 = __shfl_up_sync(0xffffffffu, f, o);
                if (lane >= o && qo == q) f += f2;
            }
        }
        const int qn = __shfl_down_sync(0xffffffffu, q, 1);
        if (valid && (lane == 31 || qn != q)) {
            if (DL32) {
                W.dlf[q] += dlf;
                W.am[q] += am;
            } else {
                W.dl[q] += d48;
            }
            W.pf[q] += pfe;
            W.pb[q] += pbe;
            if (anyfb && __double_as_longlong(f) != 0) {
                W.fb[q] += f;
                W.hasfb[q] = 1;
            }
        }
        __syncwarp();
    }
    __syncwarp();
    // ---- P6: lane per mover
    if (act) {
        c.entries += (unsigned)my_ecnt;
        VertexCtx x;
        x.v = v; x.r = r; x.s = s;
        x.Kout = kout; x.Kin = kin; x.self = my_self; x.k = k;
        const int rsr = W.rsr[lane], rss = W.rss[lane];
        x.ko_r = rsr & 0xff; x.ki_r = rsr >> 8;
        x.ko_s = rss & 0xff; x.ki_s = rss >> 8;
        __int128 d = 0;
        bool has_fb = W.hasfb[lane] != 0;
        double fb = has_fb ? W.fb[lane] : 0.0;
        float dlf = W.dlf[lane], am = W.am[lane];
        CornerVals cv;
        if (DL32) {
            cv = special_terms32_lane(md, x, dlf, am);
        } else {
            cv.Mrr = special_terms(md, x, 0, d, fb);
            cv.Mss = special_terms(md, x, 1, d, fb);
            cv.Mrs = special_terms(md, x, 2, d, fb);
            cv.Msr = special_terms(md, x, 3, d, fb);
#pragma unroll
            for (int jj = 4; jj < 8; ++jj) special_terms(md, x, jj, d, fb);
            has_fb = has_fb || __double_as_longlong(fb) != 0;
        }
        cv.dr = md.dsum[r];
        cv.ds = md.dsum[s];
        long long dl48 = W.dl[lane] + (long long)(d >> 16);
        float pf = W.pf[lane], pb = W.pb[lane];
        corner_hastings_fast(x, cv, B, pf, pb);
        int dec = -1;
        if (!a.trace_on) {
            if (DL32)
                dec = fast_decision_f(a.beta32, dlf, 0.0f, pf, pb, w2, k, dl32_error(am, k));
            else
                dec = fast_decision_f(a.beta32, fix48_to_float(dl48), has_fb ? (float)fb : 0.0f, pf, pb, w2, k);
        }
        if (dec >= 0) {
            if (dec) accept_move(md, v, s, k);
            count_result(c, dec != 0, false, k);
        } else {
            push_recheck(a, v, s, w2);  // the exact evaluation follows the pass
        }
    }
    __syncwarp();
        sa = sb + 1;
    }
}

// k_eval_batch: 32 movers per warp.  FUSED = false: the movers come from the
// list of degree group `bin` that k_propose filled.  FUSED = true: the warps
// draw the proposals of that group's vertices themselves (32 per round, lane
// per vertex), keep the movers in a queue of two slots per lane (position p
// in lane p % 32, slot p / 32) and evaluate them 32 at a time, so that the
// proposals' load chains overlap other warps' evaluation.
template <int MODE, bool DL32, bool FUSED>
__global__ void __launch_bounds__(kWarpsPerCta * 32, MODE == 0 ? SBP_BATCH0_MIN_BLOCKS : SBP_DECIDE_MIN_BLOCKS)
    k_eval_batch(DecideArgs a, int bin, int warp_bytes) {
    extern __shared__ __align__(16) unsigned char bsm[];
    using BW = BatchWarp<MODE>;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    BW &W = *reinterpret_cast<BW *>(bsm + (size_t)wid * warp_bytes);
    unsigned *dcnt = reinterpret_cast<unsigned *>(bsm + (size_t)wid * warp_bytes + sizeof(BW));
    const ModelDev &md = a.md;
    const int B = md.B;
    int *dlist = reinterpret_cast<int *>(dcnt + B);
    if (MODE == 1) {
        for (int i = lane; i < B; i += 32) dcnt[i] = 0u;
        __syncwarp();
    }
    Counts c;
    const int64_t gw = (int64_t)blockIdx.x * nwarps + wid, nw = (int64_t)gridDim.x * nwarps;
    if constexpr (!FUSED) {
        const Mover *mlist = a.movers + a.mbase[bin];
        const int64_t count = *(volatile unsigned *)&a.mcount[bin];
        const int64_t nbatch = (count + 31) >> 5;
        for (int64_t bt = gw; bt < nbatch; bt += nw) {
            const int64_t first_i = bt << 5;
            const int nv = (int)(count - first_i < 32 ? count - first_i : 32);
            Mover mv{0, -1, 0ull};
            if (lane < nv) mv = mlist[first_i + lane];
            batch_movers<MODE, DL32>(a, W, dcnt, dlist, nv, mv.v, mv.s, mv.w2, c);
        }
        flush_counts_warp(md, c, 0ull);
    } else {
        const int32_t *vl = a.vlist[bin];
        const int64_t vcount = a.vcount[bin];
        const int64_t nvb = (vcount + 31) >> 5;
        unsigned long long medges = 0;
        int q0v = 0, q0s = -1, q1v = 0, q1s = -1, nq = 0;
        uint64_t q0w = 0, q1w = 0;
        for (int64_t vb = gw;; vb += nw) {
            const bool more = vb < nvb;
            if (more) {
                const int64_t i = (vb << 5) + lane;
                bool mover = false;
                int pv = 0, ps = 0;
                uint64_t pw = 0;
                if (i < vcount) {
                    pv = vl[i];
                    const Proposal p = propose_vertex(a.g, md, a.seed, a.sweep_id, pv);
                    if (p.s == p.r) {
                        c.proposed++;
                    } else {
                        mover = true;
                        ps = p.s;
                        pw = p.w2;
                        medges += (unsigned long long)p.k;
                    }
                }
                const unsigned mask = __ballot_sync(0xffffffffu, mover);
                const int cnt = __popc(mask);
                // queue positions nq .. nq + cnt - 1 take the new movers in lane order
                const int r0 = lane - nq, r1 = 32 + lane - nq;
                const bool t0 = r0 >= 0 && r0 < cnt, t1 = r1 >= 0 && r1 < cnt;
                const int src0 = t0 ? nth_set_bit(mask, r0) : lane, src1 = t1 ? nth_set_bit(mask, r1) : lane;
                const int v0 = __shfl_sync(0xffffffffu, pv, src0), s0 = __shfl_sync(0xffffffffu, ps, src0);
                const uint64_t w0 = __shfl_sync(0xffffffffu, pw, src0);
                const int v1 = __shfl_sync(0xffffffffu, pv, src1), s1 = __shfl_sync(0xffffffffu, ps, src1);
                const uint64_t w1 = __shfl_sync(0xffffffffu, pw, src1);
                if (t0) { q0v = v0; q0s = s0; q0w = w0; }
                if (t1) { q1v = v1; q1s = s1; q1w = w1; }
                nq += cnt;
            }
            while (nq >= 32 || (!more && nq > 0)) {
                const int nv = nq < 32 ? nq : 32;
                const int v = q0v, s = q0s;
                const uint64_t w2 = q0w;
                q0v = q1v; q0s = q1s; q0w = q1w;
                nq -= nv;
                batch_movers<MODE, DL32>(a, W, dcnt, dlist, nv, v, s, w2, c);
            }
            if (!more) break;
        }
        flush_counts_warp(md, c, medges);
    }
}

// ---------------------------------------------------------------------------
// Sequential part of the hybrid pass (one CTA).  The h highest-degree
// vertices, in order, each decided against the current (b, M) with the exact
// evaluation (fixed-point Delta L, FP64 Hastings and test) and, when accepted,
// applied at once: the cells of its edges, the degrees of r and s, the
// labels.  The prefix rows P are rebuilt after this kernel; here the inverse
// CDF of the proposal scans row u (then column u) of M directly.
constexpr int kHybThreads = 256;

__device__ __forceinline__ int cta_first_above(const int32_t *M, int B, int u, bool column, uint32_t t, int *s_out,
                                               uint32_t *s_carry) {
    // smallest c with sum_{c' <= c} (row u or column u of M)[c'] > t
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    __shared__ uint32_t wsum[kHybThreads / 32];
    if (tid == 0) {
        *s_out = B - 1;
        *s_carry = 0;
    }
    __syncthreads();
    for (int c0 = 0; c0 < B; c0 += kHybThreads) {
        const int c = c0 + tid;
        const uint32_t x = c < B ? (uint32_t)(column ? M[(size_t)c * B + u] : M[(size_t)u * B + c]) : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        uint32_t before = *s_carry, total = 0;
        for (int q = 0; q < kHybThreads / 32; ++q) {
            before += q < w ? wsum[q] : 0u;
            total += wsum[q];
        }
        const uint32_t p = before + incl;
        const bool found = c < B && p > t && p - x <= t;
        __syncthreads();
        if (found) *s_out = c;
        if (tid == 0) *s_carry += total;
        const int any = __syncthreads_or(found ? 1 : 0);
        if (any) break;
    }
    __syncthreads();
    return *s_out;
}

__global__ void __launch_bounds__(kHybThreads) k_hybrid_seq(DecideArgs a, const int32_t *__restrict__ order, int h,
                                                            int32_t *M, int32_t *dout, int32_t *din, int32_t *dsum,
                                                            double *rcp, float *rcp32, int32_t *b, int32_t *bnew) {
    extern __shared__ unsigned hsm[];
    const ModelDev &md = a.md;
    const GraphDev &g = a.g;
    const int B = md.B, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    unsigned *cnt = hsm;
    int *list = reinterpret_cast<int *>(hsm + B);
    __shared__ int s_nl, s_self, s_u, s_mode, s_s, s_dec, s_pick;
    __shared__ uint32_t s_t, s_carry;
    __shared__ unsigned long long s_w2;
    __shared__ __int128 r_dl[kHybThreads / 32];
    __shared__ double r_fb[kHybThreads / 32], r_pf[kHybThreads / 32], r_pb[kHybThreads / 32];
    for (int i = tid; i < B; i += kHybThreads) cnt[i] = 0u;
    if (tid == 0) {
        s_nl = 0;
        s_self = 0;
    }
    Counts c;
    __syncthreads();
    for (int i = 0; i < h; ++i) {
        const int v = order[i];
        const int r = b[v];
        const int o0 = g.op[v], kout = g.op[v + 1] - o0, i0 = g.ip[v], kin = g.ip[v + 1] - i0, k = kout + kin;
        if (k == 0) {
            if (tid == 0) write_trace(a, v, r, 0, 0.0, 0.0);
            continue;
        }
        // the proposal, as in propose_vertex, against the current state
        if (tid == 0) {
            const U64x4 wd = philox4x64_10(a.sweep_id, (uint64_t)v, 0, 0, a.seed, 0);
            const int j = (int)draw_below(wd.x, (uint64_t)k);
            const int nb = j < kout ? g.oc[o0 + j] : g.ic[i0 + j - kout];
            const int u = b[nb];
            const int64_t y = draw_below(wd.y, (uint64_t)((int64_t)dsum[u] + B));
            s_w2 = wd.z;
            s_u = u;
            if (y < B) {
                s_mode = 0;
                s_s = (int)y;
            } else if (y - B < dout[u]) {
                s_mode = 1;
                s_t = (uint32_t)(y - B);
            } else {
                s_mode = 2;
                s_t = (uint32_t)(y - B - dout[u]);
            }
        }
        __syncthreads();
        int s = s_s;
        if (s_mode != 0) s = cta_first_above(M, B, s_u, s_mode == 2, s_t, &s_pick, &s_carry);
        if (s == r) {
            if (tid == 0) {
                write_trace(a, v, r, 1, 0.0, 0.0);
                c.proposed++;
            }
            __syncthreads();
            continue;
        }
        // v's neighbour blocks: direct-mapped counts ko | ki << 16
        for (int e = tid; e < k; e += kHybThreads) {
            const bool is_out = e < kout;
            const int nb = is_out ? g.oc[o0 + e] : g.ic[i0 + e - kout];
            if (nb == v) {
                if (is_out) atomicAdd(&s_self, 1);
                continue;
            }
            const int t = b[nb];
            if (atomicAdd(&cnt[t], is_out ? 1u : 0x10000u) == 0u) list[atomicAdd(&s_nl, 1)] = t;
        }
        __syncthreads();
        VertexCtx x;
        x.v = v;
        x.r = r;
        x.s = s;
        x.Kout = kout;
        x.Kin = kin;
        x.self = s_self;
        x.k = k;
        x.ko_r = (int)(cnt[r] & 0xffffu);
        x.ki_r = (int)(cnt[r] >> 16);
        x.ko_s = (int)(cnt[s] & 0xffffu);
        x.ki_s = (int)(cnt[s] >> 16);
        const int nl = s_nl;
        __int128 dl = 0;
        double fb = 0.0, pf = 0.0, pb = 0.0;
        for (int e = tid; e < nl; e += kHybThreads) {
            const int t = list[e];
            if (t == r || t == s) continue;
            const unsigned cc = cnt[t];
            entry_exact_all(md, x, t, (int)(cc & 0xffffu), (int)(cc >> 16), dl, fb, pf, pb);
        }
        if (tid < 8) special_terms(md, x, tid, dl, fb);
        dl = warp_sum_128(dl);
        fb = warp_sum(fb);
        pf = warp_sum(pf);
        pb = warp_sum(pb);
        if (lane == 0) {
            r_dl[w] = dl;
            r_fb[w] = fb;
            r_pf[w] = pf;
            r_pb[w] = pb;
        }
        __syncthreads();
        if (tid == 0) {
            __int128 dlt = 0;
            double fbt = 0.0, pft = 0.0, pbt = 0.0;
            for (int q = 0; q < kHybThreads / 32; ++q) {
                dlt += r_dl[q];
                fbt += r_fb[q];
                pft += r_pf[q];
                pbt += r_pb[q];
            }
            CornerVals cv;
            cv.Mrr = Mat(md, r, r);
            cv.Mss = Mat(md, s, s);
            cv.Mrs = Mat(md, r, s);
            cv.Msr = Mat(md, s, r);
            cv.dr = dsum[r];
            cv.ds = dsum[s];
            corner_hastings_exact(x, cv, B, pft, pbt);
            const Exact e = exact_decision(a.beta, dlt, fbt, pft, pbt, s_w2);
            count_exact(c, e.accept, e.margin, 0);
            write_trace(a, v, s, 1 | (e.accept ? 2 : 0) | (e.margin ? 4 : 0), e.dH, e.logA);
            s_dec = e.accept ? 1 : 0;
        }
        __syncthreads();
        if (s_dec) {
            // apply the move: the cells of v's edges, then degrees and labels
            for (int e = tid; e < kout; e += kHybThreads) {
                const int wv = g.oc[o0 + e];
                const int tw = wv == v ? r : b[wv], tn = wv == v ? s : b[wv];
                atomicAdd(&M[(size_t)r * B + tw], -1);
                atomicAdd(&M[(size_t)s * B + tn], 1);
            }
            for (int e = tid; e < kin; e += kHybThreads) {
                const int wv = g.ic[i0 + e];
                if (wv == v) continue;
                const int tw = b[wv];
                atomicAdd(&M[(size_t)tw * B + r], -1);
                atomicAdd(&M[(size_t)tw * B + s], 1);
            }
            __syncthreads();
            if (tid == 0) {
                dout[r] -= kout;
                dout[s] += kout;
                din[r] -= kin;
                din[s] += kin;
                const int qs[2] = {r, s};
                for (int q = 0; q < 2; ++q) {
                    const int bq = qs[q];
                    dsum[bq] = dout[bq] + din[bq];
                    rcp[bq] = 1.0 / ((double)dout[bq] + (double)din[bq] + (double)B);
                    rcp32[bq] = 1.0f / ((float)dout[bq] + (float)din[bq] + (float)B);
                }
                b[v] = s;
                bnew[v] = s;
            }
        }
        __syncthreads();
        for (int e = tid; e < nl; e += kHybThreads) cnt[list[e]] = 0u;
        if (tid == 0) {
            s_nl = 0;
            s_self = 0;
        }
        __syncthreads();
    }
    if (tid == 0) flush_counts(md, c);
}

__global__ void k_dxlogx32(const int32_t *__restrict__ x, const int32_t *__restrict__ k, int n, float *__restrict__ val,
                           float *__restrict__ am) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a = 0.0f;
    val[i] = dxlogx32(x[i], k[i], a);
    am[i] = a;
}

__global__ void k_mark_skip(const int32_t *__restrict__ order, int h, int n, uint8_t *__restrict__ skip) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) skip[i] = 0;
}

__global__ void k_mark_skip2(const int32_t *__restrict__ order, int h, uint8_t *__restrict__ skip) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < h; i += gridDim.x * blockDim.x) skip[order[i]] = 1;
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
    d.Pc = m->Pc;
    d.pstep = (2 * m->B + 31) / 32;
    d.dout = m->dout;
    d.din = m->din;
    d.rcp = m->rcp;
    d.rcp32 = m->rcp32;
    d.dsum = m->dsum;
    d.T = m->T;
    d.XT = m->XT;
    d.sparse = m->dense ? 0 : 1;
    d.rp = m->sp.rp;
    d.cp = m->sp.cp;
    d.hoff = m->sp.hoff;
    d.rc = m->sp.rc;
    d.cr = m->sp.cr;
    d.rv = m->sp.rv;
    d.cv = m->sp.cv;
    d.rpre = m->sp.rpre;
    d.cpre = m->sp.cpre;
    d.rpc = m->sp.rpc;
    d.cpc = m->sp.cpc;
    d.hkv = m->sp.hkv;
    d.status = m->status;
    d.counters = m->counters;
    d.items = nullptr;  // set by the nodal pass only
    d.cap_items = 0;
    d.nbo = nullptr;
    d.nbi = nullptr;
    return d;
}

namespace {

// The CTA kernel's neighbour table (cap slots of 16 bytes): in shared memory
// while it fits, else a slice per CTA of a global scratch the model keeps
// (at most 1 GB, fewer CTAs for very large tables).
int cta_table(sbp_model *m, int cap, int sms, int *grid, size_t *smem, unsigned long long **gtab) {
    const size_t bytes = (size_t)cap * 16;
    *grid = sms * 4;
    *gtab = nullptr;
    *smem = bytes;
    if (bytes <= 160 * 1024) return SBP_OK;
    *smem = 0;
    const size_t per_grid = std::max<size_t>(1, (size_t(1) << 30) / bytes);
    if ((size_t)*grid > per_grid) *grid = (int)per_grid;
    const size_t need = bytes * (size_t)*grid;
    if (m->cta_tab_bytes < need) {
        model_free(m->cta_tab, m->stream);
        m->cta_tab = nullptr;
        m->cta_tab_bytes = 0;
        if (model_alloc((void **)&m->cta_tab, need, m->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(SBP_ENOMEM, "nodal pass: no device memory for the neighbour tables");
        }
        m->cta_tab_bytes = need;
    }
    *gtab = m->cta_tab;
    return SBP_OK;
}

// graphs with at least this many edges run the three degree groups'
// kernels on three streams
constexpr int64_t kSideStreamEdges = int64_t(1) << 22;

// streams of the three groups: the model's own one for the movers above 128
// edges (launched first: the longest tail), side streams for the others
// (forked after k_propose, joined back by join_evals)
int fork_evals(sbp_model *m, cudaStream_t st[3]) {
    st[0] = st[1] = st[2] = m->stream;
    if (m->g->m < kSideStreamEdges) return SBP_OK;
    if (!m->fork_ev) {
        for (int i = 0; i < 2; ++i) {
            SBP_CUDA(cudaStreamCreateWithFlags(&m->side[i], cudaStreamNonBlocking));
            SBP_CUDA(cudaEventCreateWithFlags(&m->join_ev[i], cudaEventDisableTiming));
        }
        SBP_CUDA(cudaEventCreateWithFlags(&m->fork_ev, cudaEventDisableTiming));
    }
    SBP_CUDA(cudaEventRecord(m->fork_ev, m->stream));
    for (int i = 0; i < 2; ++i) SBP_CUDA(cudaStreamWaitEvent(m->side[i], m->fork_ev, 0));
    st[0] = m->side[1];
    st[1] = m->side[0];
    return SBP_OK;
}

int join_evals(sbp_model *m) {
    if (m->g->m < kSideStreamEdges || !m->fork_ev) return SBP_OK;
    for (int i = 0; i < 2; ++i) {
        SBP_CUDA(cudaEventRecord(m->join_ev[i], m->side[i]));
        SBP_CUDA(cudaStreamWaitEvent(m->stream, m->join_ev[i], 0));
    }
    return SBP_OK;
}

// the evaluation kernels of the three degree groups: after k_propose, or
// (FUSED) drawing the proposals themselves
template <bool DL32, bool FUSED>
int launch_groups(sbp_model *m, const DecideArgs &a, int sms, const cudaStream_t st[3]) {
    const sbp_graph *g = m->g;
    const int B = m->B;
    auto warp_smem = [](int cap, int nwarps) { return (size_t)nwarps * cap * 10 + (size_t)nwarps * 4 + 16; };
    // movers with k > 128: per-warp direct-mapped counts while B is small,
    // else per-warp tables sized for min(max degree, B) distinct blocks while
    // they fit, one CTA per mover beyond that
    if (g->bin[4] > g->bin[3] && B <= kDirectMaxB && g->max_deg < 65536) {
        const int warp_words = 2 * B + 4;
        const int nwarps = warp_words * 4 * kWarpsPerCta <= 64 * 1024 ? kWarpsPerCta : kWarpsPerCta / 2;
        const size_t smem = (size_t)warp_words * 4 * nwarps;
        SBP_TRY(ensure_dyn_smem((const void *)k_eval_warp_direct<DL32, FUSED>, smem));
        k_eval_warp_direct<DL32, FUSED><<<sms * 4, nwarps * 32, smem, st[2]>>>(a, 2, warp_words);
        SBP_LAUNCHED();
    } else if (g->bin[4] > g->bin[3]) {
        const int64_t dmax = g->max_deg < B ? g->max_deg : B;
        const int64_t need = dmax + dmax / 4 + 2;
        int cap_log2 = 6;
        while ((int64_t(1) << cap_log2) < need) ++cap_log2;
        const int cap = 1 << cap_log2;
        if (cap <= 4096 && g->max_deg < 65536) {
            const int nwarps = cap <= 2048 ? 8 : 4;
            const size_t smem = warp_smem(cap, nwarps);
            SBP_TRY(ensure_dyn_smem((const void *)k_eval_warp<DL32>, smem));
            k_eval_warp<DL32><<<sms * 4, nwarps * 32, smem, st[2]>>>(a, 2, cap, cap_log2, 1);
            SBP_LAUNCHED();
        } else {
            int grid;
            size_t smem;
            unsigned long long *gtab;
            SBP_TRY(cta_table(m, cap, sms, &grid, &smem, &gtab));
            SBP_TRY(ensure_dyn_smem((const void *)k_eval_cta<DL32>, smem));
            k_eval_cta<DL32><<<grid, kBigThreads, smem, st[2]>>>(a, 2, cap, cap_log2, gtab);
            SBP_LAUNCHED();
        }
    }
    // movers with k <= 32: batches of 32 per warp
    if (g->bin[2] > g->bin[1]) {
        const int wb = (int)((sizeof(BatchWarp<0>) + 15) / 16 * 16);
        const size_t smem = (size_t)wb * kWarpsPerCta;
        SBP_TRY(ensure_dyn_smem((const void *)k_eval_batch<0, DL32, FUSED>, smem));
        k_eval_batch<0, DL32, FUSED><<<sms * SBP_BATCH0_MIN_BLOCKS, kWarpsPerCta * 32, smem, st[0]>>>(a, 0, wb);
        SBP_LAUNCHED();
    }
    // movers with 33 <= k <= 128: batches with direct-mapped counts while B is
    // small, otherwise one warp each with a 256-slot table
    if (g->bin[3] > g->bin[2]) {
        if (B <= kDirectMaxB) {
            const int wb = (int)((sizeof(BatchWarp<1>) + 4 * (size_t)B + 4 * kWarpDeg + 15) / 16 * 16);
            const int nwarps = wb <= 10 * 1024 ? kWarpsPerCta : kWarpsPerCta / 2;
            const size_t smem = (size_t)wb * nwarps;
            SBP_TRY(ensure_dyn_smem((const void *)k_eval_batch<1, DL32, FUSED>, smem));
            k_eval_batch<1, DL32, FUSED><<<sms * SBP_DECIDE_MIN_BLOCKS, nwarps * 32, smem, st[1]>>>(a, 1, wb);
            SBP_LAUNCHED();
        } else {
            const size_t smem = warp_smem(kWarpCap, kWarpsPerCta);
            SBP_TRY(ensure_dyn_smem((const void *)k_eval_warp<DL32>, smem));
            k_eval_warp<DL32><<<sms * SBP_DECIDE_MIN_BLOCKS, kWarpsPerCta * 32, smem, st[1]>>>(a, 1, kWarpCap, 8, 32);
            SBP_LAUNCHED();
        }
    }
    return SBP_OK;
}

// the movers the FP32 test left undecided (all of them when a trace is
// asked for): a CTA each, aggregated again and decided by the exact
// evaluation, after the three groups' kernels
template <bool DL32>
int launch_recheck(sbp_model *m, const DecideArgs &a0, int sms) {
    const sbp_graph *g = m->g;
    DecideArgs a = a0;
    a.force_exact = 1;
    const int64_t dmax = g->max_deg < m->B ? g->max_deg : m->B;
    const int64_t need = dmax + dmax / 4 + 2;
    int cap_log2 = 6;
    while ((int64_t(1) << cap_log2) < need) ++cap_log2;
    const int cap = 1 << cap_log2;
    int grid;
    size_t smem;
    unsigned long long *gtab;
    SBP_TRY(cta_table(m, cap, sms, &grid, &smem, &gtab));
    SBP_TRY(ensure_dyn_smem((const void *)k_eval_cta<DL32>, smem));
    k_eval_cta<DL32><<<grid, kBigThreads, smem, m->stream>>>(a, 3, cap, cap_log2, gtab);
    SBP_LAUNCHED();
    return SBP_OK;
}

template <bool DL32>
int launch_evals(sbp_model *m, const DecideArgs &a, int sms, bool fused) {
    cudaStream_t st[3];
    SBP_TRY(fork_evals(m, st));
    const int rc = fused ? launch_groups<DL32, true>(m, a, sms, st) : launch_groups<DL32, false>(m, a, sms, st);
    const int rj = join_evals(m);  // joined on every path
    if (rc != SBP_OK) return rc;
    if (rj != SBP_OK) return rj;
    return launch_recheck<DL32>(m, a, sms);
}

}  // namespace

int launch_decide(sbp_model *m, uint64_t sweep_id, int64_t v_begin, int64_t v_end, const sbp_vertex_trace *trace) {
    const sbp_graph *g = m->g;
    if (!m->movers) {
        // the degree groups' lists (n entries) and the recheck list (n more)
        if (model_alloc(&m->movers, (size_t)(g->n > 0 ? 2 * g->n : 1) * sizeof(Mover), m->stream) != cudaSuccess ||
            model_alloc((void **)&m->mcount, 4 * sizeof(unsigned), m->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(SBP_ENOMEM, "cudaMalloc failed for the mover lists");
        }
    }
    if (!m->items) {
        // at most one item per vertex plus one per kMoveChunk edge ends
        const int64_t cap = g->n + (2 * g->m) / kMoveChunk + 1;
        if (model_alloc((void **)&m->items, (size_t)cap * sizeof(int2), m->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(SBP_ENOMEM, "cudaMalloc failed for the accepted-move list");
        }
        m->cap_items = cap;
    }
    // the list holds every accepted move only while the ranges decided since
    // the last commit are disjoint
    for (const auto &rg : m->decided)
        if (v_begin < rg.second && rg.first < v_end) m->list_ok = false;
    m->decided.emplace_back(v_begin, v_end);
    DecideArgs a;
    a.g = g->dev();
    a.md = model_dev(m);
    a.md.items = m->items;
    a.md.cap_items = m->cap_items;
    const int64_t h_seq = std::min<int64_t>(m->p.hybrid_h, g->n);
    if (h_seq > 0 && m->dense && v_begin == 0 && v_end == g->n) {
        m->nb_ok = false;  // the sequential part moves vertices in place
    } else {
        if (!m->nb_ok) SBP_TRY(nb_rows_rebuild(m));
        if (m->nb_ok) {
            a.md.nbo = m->nbo;
            a.md.nbi = m->nbi;
        }
    }
    a.v_begin = v_begin;
    a.v_end = v_end;
    a.movers = static_cast<Mover *>(m->movers);
    a.mcount = m->mcount;
    // list capacities: the sizes of the degree groups
    a.mbase[0] = 0;
    a.mbase[1] = g->bin[2] - g->bin[1];
    a.mbase[2] = a.mbase[1] + (g->bin[3] - g->bin[2]);
    a.mbase[3] = g->n;  // the recheck list
    a.force_exact = 0;
    a.seed = m->p.seed;
    a.sweep_id = sweep_id;
    a.beta = m->p.beta;
    a.beta32 = (float)m->p.beta;
    a.tr = trace ? *trace : sbp_vertex_trace{nullptr, nullptr, nullptr, nullptr};
    a.skip = nullptr;
    a.trace_on = (a.tr.s || a.tr.flags || a.tr.dH || a.tr.logA) ? 1 : 0;
    const int sms = sm_count();
    const int B = m->B;
    if (B >= (1 << 24)) return fail(SBP_ESTATE, "nodal pass: B must be below 2^24");
    SBP_CUDA(cudaMemsetAsync(m->mcount, 0, 4 * sizeof(unsigned), m->stream));

    // hybrid pass: the sequential part first (full-range passes of a dense model)
    const int64_t h = std::min<int64_t>(m->p.hybrid_h, g->n);
    if (h > 0 && m->dense && v_begin == 0 && v_end == g->n) {
        if (g->max_deg >= 65536) return fail(SBP_ESTATE, "hybrid pass: degrees of 65536 or more are not supported");
        if (!m->skip) {
            if (model_alloc((void **)&m->skip, (size_t)g->n, m->stream) != cudaSuccess) {
                cudaGetLastError();
                return fail(SBP_ENOMEM, "device allocation failed for the hybrid pass");
            }
            m->skip_h = -1;
        }
        if (m->skip_h != (int32_t)h) {
            k_mark_skip<<<(int)std::min<int64_t>((g->n + 255) / 256, 1024), 256, 0, m->stream>>>(g->by_degree, (int)h,
                                                                                                 (int)g->n, m->skip);
            SBP_LAUNCHED();
            k_mark_skip2<<<(int)std::min<int64_t>((h + 255) / 256, 1024), 256, 0, m->stream>>>(g->by_degree, (int)h,
                                                                                               m->skip);
            SBP_LAUNCHED();
            m->skip_h = (int32_t)h;
        }
        const size_t smem = (size_t)B * 8;
        SBP_TRY(ensure_dyn_smem((const void *)k_hybrid_seq, smem));
        k_hybrid_seq<<<1, kHybThreads, smem, m->stream>>>(a, g->by_degree, (int)h, m->M, m->dout, m->din, m->dsum,
                                                          m->rcp, m->rcp32, m->b, m->bnew);
        SBP_LAUNCHED();
        SBP_TRY(launch_prefix(m));
        a.skip = m->skip;
    }

    // A full-range pass with no trace and no sequential part, whose degree
    // groups all take the direct-mapped kernels, draws the proposals inside
    // the evaluation kernels; any other pass proposes every vertex of its
    // range first (k_propose) and hands the movers over in lists.
    for (int i = 0; i < 3; ++i) {
        a.vlist[i] = g->order + g->bin[i + 1];
        a.vcount[i] = g->bin[i + 2] - g->bin[i + 1];
    }
    const bool fused = SBP_FUSED_PROPOSALS && v_begin == 0 && v_end == g->n && !a.skip && !a.trace_on &&
                       B <= kDirectMaxB && g->max_deg < 65536;
    if (!fused) {
        int64_t blocks = (v_end - v_begin + 255) / 256;
        if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
        if (blocks < 1) blocks = 1;
        k_propose<<<(int)blocks, 256, 0, m->stream>>>(a);
        SBP_LAUNCHED();
    }
    return m->p.dl_fp32 ? launch_evals<true>(m, a, sms, fused) : launch_evals<false>(m, a, sms, fused);
}

}  // namespace sbp

// Known-answer hook for the FP32 term of the precision form: val[i] =
// f(x[i] + k[i]) - f(x[i]) in FP32 and am[i] the magnitude its error bound
// is proportional to (host arrays).
extern "C" int sbp_dxlogx32_check(const int32_t *x, const int32_t *k, int32_t count, float *val, float *am) {
    using namespace sbp;
    if (count < 0 || count > (1 << 24) || (count > 0 && (!x || !k || !val || !am)))
        return fail(SBP_EINVAL, "sbp_dxlogx32_check: bad count or NULL array");
    for (int32_t i = 0; i < count; ++i)
        if (x[i] < 0 || (int64_t)x[i] + k[i] < 0 || (int64_t)x[i] + k[i] > INT32_MAX)
            return fail(SBP_EINVAL, "sbp_dxlogx32_check: need x >= 0 and 0 <= x + k < 2^31");
    if (count == 0) return SBP_OK;
    void *d = nullptr;
    SBP_CUDA(cudaMalloc(&d, (size_t)count * 16));
    int32_t *dx = static_cast<int32_t *>(d), *dk = dx + count;
    float *dv = reinterpret_cast<float *>(dk + count), *da = dv + count;
    cudaError_t e = cudaMemcpy(dx, x, (size_t)count * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, k, (size_t)count * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_dxlogx32<<<(count + 255) / 256, 256>>>(dx, dk, count, dv, da);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(val, dv, (size_t)count * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(am, da, (size_t)count * 4, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "sbp_dxlogx32_check");
    return SBP_OK;
}
