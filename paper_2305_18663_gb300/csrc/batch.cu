// batch.cu -- many graphs' phases in one persistent launch.
//
// The batching form of the golden-ratio search: thousands of small, uneven
// graphs each need tens of phases (Alg. 1 merges, then an Alg. 2 MCMC
// phase of a few tens of sweeps) at a few hundred blocks.  Run one graph
// at a time, every merge round and every sweep is a chain of small kernels
// with a host round trip.  Here one persistent launch takes a table of jobs
// (one phase of one graph each, every graph in its own dense model); a CTA
// pulls a job from a device queue, runs the whole phase for it and pulls
// the next, largest jobs first.  A job:
//   0. (optional) loads the phase's start state, a bracket state the model
//      no longer holds, and rebuilds the counts from it;
//   1. (optional) the merge phase: per round, every block's best merge
//      (one warp per block, the same scoring code as the per-graph kernel),
//      the scores sorted in shared memory, the merges applied in order with
//      a union-find until n_merges are done, the labels relabelled and the
//      counts rebuilt; rounds repeat as the per-graph merge does;
//   2. the MCMC phase, per sweep:
//      a. proposals, one thread per vertex (the same proposal as the
//         per-graph pass), movers (s != r) appended to the graph's list;
//      b. evaluation, G lanes per mover: the row is aggregated into
//         direct-mapped counts in shared memory (B entries), then the same
//         Delta DL, Hastings and test code as the per-graph pass;
//      c. the apply step from the moved vertices' rows.  Each cell update is
//         an atomic whose returned old count gives T[new] - T[old] (x ln x
//         in 128-bit fixed point), so sum M ln M is carried exactly from
//         sweep to sweep without a pass over the B x B cells;
//      d. prefix rows, degrees and DL (Eq. 2, the same integer L as a
//         recount, hence the same bits), and the convergence test of Alg. 2;
//   3. the compaction: empty blocks dropped, labels renumbered in order.
// The decisions are the exact ones (the precision form's band guarantees it),
// the counts are integers and L is an exact integer, so a graph's phase ends
// with the same assignment, M, DL and sweep count as the per-graph path.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "apply.cuh"
#include "sbp_check.h"
#include "batch.h"
#include "driver.h"
#include "merge_dev.cuh"
#include "nodal_dev.cuh"

namespace sbp {
namespace {

constexpr int kBatchThreads = 256;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr size_t kBatchSmemCap = 96 * 1024;  // dynamic shared memory of a CTA (two per SM)

// the blockmodel arrays the apply step writes (the decision pass sees them
// read-only through DecideArgs)
struct ModelOut {
    int32_t *b, *M, *dout, *din, *dsum;
    uint32_t *P, *Pc;
    double *rcp;
    float *rcp32;
};

struct BatchJob {
    DecideArgs a;        // graph, model, seed, beta (trace off)
    ModelOut w;
    int max_sweeps;
    int merge_x;         // proposals per block and merge round
    double reduction, t_pre, t_post;  // the search's parameters
    int lim_from;        // largest B a phase may start from here
    int max_B;           // largest B a phase may merge to
    double *hist;        // [max_sweeps + 1], the current phase's DL per sweep
    double *dl;          // the model's dl[0] (current) and dl[1] (before the last sweep)
    int32_t *best_s;     // [lim_from] the merge rounds' best proposal per block
    double *best_d;
    SearchRec *rec;      // the search, in and out
    int32_t *slots;      // its four label slots (4 n)
};

// Bracket::insert on the kernel's copy of the bracket (positions move with
// their label slots)
__host__ __device__ void search_insert(SearchRec &r, const SearchState &x) {
    if (r.s[1].B == 0) {
        r.s[1] = x;
        return;
    }
    if (x.dl < r.s[1].dl) {
        if (r.s[1].B > x.B) r.s[0] = r.s[1];
        else r.s[2] = r.s[1];
        r.s[1] = x;
    } else {
        if (x.B > r.s[1].B) r.s[0] = x;
        else r.s[2] = x;
    }
}

// Bracket::next on the kernel's copy: the next phase's start position and
// target, false when the search has ended
__host__ __device__ bool search_next(const SearchRec &r, double reduction, int &start, int &target) {
    const SearchState *s = r.s;
    if (s[2].B == 0) {
        int64_t nm = (int64_t)floor((double)s[1].B * reduction);
        if (nm > s[1].B - 1) nm = s[1].B - 1;
        if (nm < 1) return false;
        start = 1;
        target = (int)(s[1].B - nm);
        return true;
    }
    if (s[0].B - s[2].B <= 2) return false;
    const int up = s[0].B - s[1].B, low = s[1].B - s[2].B;
    int upper, lower;
    if (up >= low) {
        start = 0;
        upper = s[0].B;
        lower = s[1].B;
    } else {
        start = 1;
        upper = s[1].B;
        lower = s[2].B;
    }
    int t = upper - (int)llround(0.618 * (double)(upper - lower));
    if (t >= upper) t = upper - 1;
    if (t <= lower) t = lower + 1;
    target = t;
    return true;
}

// the label slot no bracket position uses (three positions, four slots: one
// is always free)
__host__ __device__ int search_free_slot(const SearchRec &r) {
    for (int f = 0; f < 4; ++f) {
        bool used = false;
        for (int p = 0; p < 3; ++p) used |= r.s[p].B != 0 && r.s[p].slot == f;
        if (!used) return f;
    }
    return -1;
}

// one cell update of the incremental apply with the exact change of sum x ln x
__device__ __forceinline__ void cell_add(int32_t *__restrict__ M, const __int128 *__restrict__ T, bool valid, int key,
                                         int d, __int128 &acc) {
    if (!valid) return;
    const int old = atomicAdd(&M[key], d);
    acc += T[old + d] - T[old];
}

// (labels and M through plain loads and atomics: this kernel writes all of
// them between sweeps, so no read-only-cache path may be used)
__device__ void apply_rows(const GraphDev &g, const int32_t *bold, const int32_t *bnew, int32_t *M, int B,
                           const __int128 *__restrict__ T, int v, __int128 &acc) {
    const int lane = threadIdx.x & 31;
    const int r = bold[v], s = bnew[v];
    const int o0 = g.op[v], o1 = g.op[v + 1], i0 = g.ip[v], i1 = g.ip[v + 1];
    for (int e0 = o0; e0 < o1; e0 += 32) {
        const int e = e0 + lane;
        const bool ok = e < o1;
        const int w = ok ? g.oc[e] : 0;
        const int tw = ok ? bold[w] : 0, uw = ok ? bnew[w] : 0;
        cell_add(M, T, ok, r * B + tw, -1, acc);
        cell_add(M, T, ok, s * B + uw, 1, acc);
    }
    for (int e0 = i0; e0 < i1; e0 += 32) {
        const int e = e0 + lane;
        bool ok = e < i1;
        const int w = ok ? g.ic[e] : 0;
        const int t = ok ? bold[w] : 0;
        ok = ok && bnew[w] == t;
        cell_add(M, T, ok, t * B + r, -1, acc);
        cell_add(M, T, ok, t * B + s, 1, acc);
    }
}

// the CTA's sum of one int128 per thread (every thread gets it)
__device__ __int128 cta_sum_128(__int128 v, __int128 *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum_128(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    __int128 s = 0;
    for (int q = 0; q < kBatchWarps; ++q) s += sh[q];
    __syncthreads();
    return s;
}

// The dense model of B blocks from labels b, CTA-wide (the per-graph
// rebuild's counts, prefix rows, degrees and reciprocals): M counted from the
// edge list, then the sums C = sum T[M] and D = sum T[dout] + T[din]
// (L = C - D exactly).  Every thread gets C and D.
__device__ void cta_rebuild(const GraphDev &g, const int32_t *b, const ModelOut &w, int B, int pstep,
                            const __int128 *__restrict__ T, __int128 *red, __int128 &C, __int128 &D) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int BB = B * B;
    for (int i = tid; i < BB; i += kBatchThreads) w.M[i] = 0;
    __syncthreads();
    for (int64_t e = tid; e < g.m; e += kBatchThreads) atomicAdd(&w.M[b[g.esrc[e]] * B + b[g.oc[e]]], 1);
    __syncthreads();
    __int128 dd = 0, c = 0;
    for (int u = wid; u < B; u += kBatchWarps) {
        prefix_block(w.M, B, u, w.P, w.dout, w.din, w.rcp, w.rcp32, w.dsum, w.Pc, pstep);
        if (lane == 0) {
            dd += T[w.dout[u]];
            dd += T[w.din[u]];
        }
    }
    for (int i = tid; i < BB; i += kBatchThreads) c += T[w.M[i]];
    D = cta_sum_128(dd, red);
    C = cta_sum_128(c, red);
}

// ascending sort of (key, idx) pairs, CTA-wide bitonic network (n a power
// of two; the indices are distinct, so the order is total)
__device__ void cta_sort_pairs(long long *key, int *idx, int n) {
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += kBatchThreads) {
                const int p = i ^ j;
                if (p > i) {
                    const bool up = (i & k) == 0;
                    const bool gt = key[i] > key[p] || (key[i] == key[p] && idx[i] > idx[p]);
                    if (gt == up) {
                        const long long tk = key[i];
                        key[i] = key[p];
                        key[p] = tk;
                        const int ti = idx[i];
                        idx[i] = idx[p];
                        idx[p] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ int uf_find(int *par, int x) {
    while (par[x] != x) {
        par[x] = par[par[x]];
        x = par[x];
    }
    return x;
}

// b[v] = bnew[v] = map[b[v]] for every vertex
__device__ void cta_relabel(int32_t *b, int32_t *bnew, int n, const int *map) {
    for (int v = threadIdx.x; v < n; v += kBatchThreads) {
        const int x = map[b[v]];
        b[v] = x;
        bnew[v] = x;
    }
    __syncthreads();
}

// G: lanes per mover in the evaluation (32 / G movers per warp at a time);
// group_words: shared-memory words of one group (counts, then the list);
// blk_cap: a power of two >= every job's lim_from (the merge rounds' and the
// compaction's shared arrays)
template <bool DL32, int G>
__global__ void __launch_bounds__(kBatchThreads, 2) k_batch_search(const BatchJob *__restrict__ jobs, int njobs,
                                                                  unsigned *__restrict__ queue, int group_words,
                                                                  int blk_cap) {
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ DecideArgs sa;
    __shared__ ModelOut sw;
    __shared__ SearchRec sr;
    __shared__ __int128 red[kBatchWarps];
    __shared__ unsigned s_job, s_nmov;
    __shared__ int s_stop, s_left, s_rounds, s_done, s_Bn, s_go, s_start, s_target, s_reload, s_slot;
    constexpr int V = 32 / G;  // movers per warp
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int gid = lane / G, gl = lane & (G - 1);
    const unsigned gm = group_mask<G>();
    unsigned *cnt = reinterpret_cast<unsigned *>(bsm) + ((size_t)wid * V + gid) * group_words;
    // merge rounds and compaction (the same shared memory, used between
    // sweeps only): sort keys and indices, union-find parents, labels
    long long *skey = reinterpret_cast<long long *>(bsm);
    int *sidx = reinterpret_cast<int *>(skey + blk_cap);
    int *par = sidx + blk_cap;
    int *smap = par + blk_cap;
    for (;;) {
        if (tid == 0) s_job = atomicAdd(queue, 1u);
        __syncthreads();
        const unsigned j = s_job;
        if (j >= (unsigned)njobs) return;
        if (tid == 0) {
            sa = jobs[j].a;
            sw = jobs[j].w;
            sr = *jobs[j].rec;
            sr.done = 0;
            sr.phases = sr.merged = sr.starts = 0;
        }
        __syncthreads();
        const BatchJob &J = jobs[j];
        const GraphDev &g = sa.g;
        const ModelDev &md = sa.md;
        const int n = g.n;
        int B = md.B;
        bool started = sr.started != 0;
        for (;;) {
            __int128 C = 0, D = 0;
            bool have_sums = false;
            if (!started) {
                // the next phase of the search, if it is one for this kernel
                if (tid == 0) {
                    int st = 0, tg = 0;
                    if (!search_next(sr, J.reduction, st, tg)) {
                        s_go = 0;
                        sr.done = 1;
                    } else {
                        const SearchState &from = sr.s[st];
                        s_go = from.B <= J.lim_from && tg >= 1 && tg < from.B && tg <= J.max_B ? 1 : 2;
                        s_start = st;
                        s_target = tg;
                        // decided here, once: thread 0 changes sr.holds below
                        s_reload = from.id != sr.holds ? 1 : 0;
                    }
                }
                __syncthreads();
                if (s_go != 1) break;
                // 0. the start state, when the model no longer holds it
                const SearchState from = sr.s[s_start];
                if (s_reload) {
                    const int32_t *src = J.slots + (size_t)from.slot * n;
                    for (int v = tid; v < n; v += kBatchThreads) {
                        const int x = src[v];
                        sw.b[v] = x;
                        md.bnew[v] = x;
                    }
                    B = from.B;
                    if (tid == 0) {
                        sa.md.B = B;
                        sa.md.pstep = (2 * B + 31) / 32;
                        ++sr.starts;
                    }
                    __syncthreads();
                    cta_rebuild(g, sw.b, sw, B, (2 * B + 31) / 32, md.T, red, C, D);
                    have_sums = true;
                }
                // 1. merge rounds until from.B - target blocks are gone (or a
                // round merges nothing), each from the previous round's counts
                if (tid == 0) {
                    s_left = from.B - s_target;
                    s_rounds = 0;
                    sr.holds = 0;
                    ++sr.merged;
                }
                __syncthreads();
                while (s_left > 0 && B >= 2) {
                    const uint64_t rid = sr.round_id + (uint64_t)s_rounds;
                    for (int r = wid; r < B; r += kBatchWarps) {
                        int bs;
                        double bd;
                        merge_best(md, sa.seed, rid, J.merge_x, r, bs, bd);
                        if (lane == 0) {
                            J.best_s[r] = bs;
                            J.best_d[r] = bd;
                        }
                    }
                    __syncthreads();
                    int p2 = 1;
                    while (p2 < B) p2 <<= 1;
                    for (int i = tid; i < p2; i += kBatchThreads) {
                        skey[i] = i < B ? score_key(J.best_d[i]) : LLONG_MAX;
                        sidx[i] = i < B ? i : INT_MAX;
                    }
                    __syncthreads();
                    cta_sort_pairs(skey, sidx, p2);
                    if (tid == 0) {
                        // ascending (score, block), pointer-based union, stop at
                        // the merges still owed; groups numbered by their
                        // smallest block
                        for (int c = 0; c < B; ++c) par[c] = c;
                        int done = 0;
                        for (int q = 0; q < B && done < s_left; ++q) {
                            const int r = sidx[q], s = J.best_s[r];
                            if (s < 0) continue;
                            const int a = uf_find(par, r), c = uf_find(par, s);
                            if (a == c) continue;
                            par[a] = c;
                            ++done;
                        }
                        int *lab = reinterpret_cast<int *>(skey);
                        for (int c = 0; c < B; ++c) lab[c] = -1;
                        int next = 0;
                        for (int c = 0; c < B; ++c) {
                            const int root = uf_find(par, c);
                            if (lab[root] < 0) lab[root] = next++;
                            smap[c] = lab[root];
                        }
                        s_done = done;
                        s_Bn = next;
                        s_left -= done;
                        ++s_rounds;
                        sa.md.B = next;
                        sa.md.pstep = (2 * next + 31) / 32;
                    }
                    __syncthreads();
                    cta_relabel(sw.b, md.bnew, n, smap);
                    B = s_Bn;
                    cta_rebuild(g, sw.b, sw, B, md.pstep, md.T, red, C, D);
                    have_sums = true;
                    if (s_done == 0) break;
                }
                if (tid == 0) sr.round_id += (uint64_t)s_rounds;
            }
            started = false;
            // 2. the MCMC phase (its B must fit the launch's count rows: the
            // merges end at the planned B, so this only guards the bound)
            if (2 * B + 4 > group_words) break;
            if (!have_sums) {
                // sum over the cells of T[M] and the degree terms at the phase start (exact)
                __int128 c = 0, dd = 0;
                for (int i = tid; i < B * B; i += kBatchThreads) c += md.T[md.M[i]];
                for (int u = tid; u < B; u += kBatchThreads) dd += md.T[md.dout[u]] + md.T[md.din[u]];
                C = cta_sum_128(c, red);
                D = cta_sum_128(dd, red);
            }
            int *list = reinterpret_cast<int *>(cnt + B);
            for (int i = gl; i < B; i += G) cnt[i] = 0u;
            const double dl0 = dl_eq2(g.m, g.n, B, fix_to_double(C - D));
            const double tconv = sr.s[2].B == 0 ? J.t_pre : J.t_post;
            const uint64_t sweep0 = sr.sweep_id;
            if (tid == 0) J.hist[0] = dl0;
            double prev = dl0;
            int k = 0;
            __syncthreads();
            for (;;) {
                ++k;
                const uint64_t sweep_id = sweep0 + (uint64_t)(k - 1);
                if (tid == 0) s_nmov = 0;
                __syncthreads();
                // 1. proposals
                for (int base = 0; base < n; base += kBatchThreads) {
                    const int v = base + tid;
                    bool mv = false;
                    Proposal p;
                    if (v < n) {
                        p = propose_vertex(g, md, sa.seed, sweep_id, v);
                        mv = p.k > 0 && p.s != p.r;
                    }
                    const unsigned msk = __ballot_sync(0xffffffffu, mv);
                    unsigned pos0 = 0;
                    if (msk) {
                        if (lane == __ffs(msk) - 1) pos0 = atomicAdd(&s_nmov, (unsigned)__popc(msk));
                        pos0 = __shfl_sync(0xffffffffu, pos0, __ffs(msk) - 1);
                    }
                    if (mv) {
                        Mover m;
                        m.v = v;
                        m.s = p.s;
                        m.w2 = p.w2;
                        sa.movers[pos0 + __popc(msk & ((1u << lane) - 1u))] = m;
                    }
                }
                __syncthreads();
                // 2. evaluation, G lanes per mover
                const int nmov = (int)s_nmov;
                Counts cts;
                __syncwarp();
                for (int q = wid * V + gid; q < nmov; q += kBatchWarps * V) {
                    const Mover mv = sa.movers[q];
                    const int v = mv.v;
                    const int o0 = g.op[v], kout = g.op[v + 1] - o0;
                    const int i0 = g.ip[v], kin = g.ip[v + 1] - i0;
                    const int kk = kout + kin;
                    int nl = 0, self = 0;
                    for (int base = 0; base < kk; base += G) {
                        const int idx = base + gl;
                        const bool valid = idx < kk, is_out = idx < kout;
                        const int nb = valid ? (is_out ? g.oc[o0 + idx] : g.ic[i0 + idx - kout]) : -1;
                        const bool is_self = valid && nb == v;
                        self += __popc(__ballot_sync(gm, is_self && is_out));
                        bool fresh = false;
                        int t = 0;
                        if (valid && !is_self) {
                            t = md.b[nb];
                            fresh = atomicAdd(&cnt[t], is_out ? 1u : 0x10000u) == 0u;
                        }
                        const unsigned fm = __ballot_sync(gm, fresh);  // bits of this group only
                        if (fresh) list[nl + __popc(fm & ((1u << lane) - 1u))] = t;
                        nl += __popc(fm);
                    }
                    __syncwarp(gm);
                    VertexCtx x;
                    x.v = v;
                    x.r = md.b[v];
                    x.s = mv.s;
                    x.Kout = kout;
                    x.Kin = kin;
                    x.self = self;
                    x.k = kk;
                    evaluate_group<DL32, G, true>(sa, md, x, mv.w2, [&](auto &&f) {
                        for (int e = gl; e < nl; e += G) {
                            const int t = list[e];
                            const unsigned cc = cnt[t];
                            f(t, (int)(cc & 0xffffu), (int)(cc >> 16));
                        }
                    }, cts);
                    __syncwarp(gm);
                    for (int e = gl; e < nl; e += G) cnt[list[e]] = 0u;
                    __syncwarp(gm);
                }
                __syncthreads();
                // 3. apply: warp per 32 vertex ids, rows of the moved ones
                __int128 dc = 0;
                for (int base = wid * 32; base < n; base += kBatchThreads) {
                    const int vv = base + lane;
                    const bool moved = vv < n && md.bnew[vv] != md.b[vv];
                    unsigned mm = __ballot_sync(0xffffffffu, moved);
                    while (mm) {
                        const int qq = __ffs(mm) - 1;
                        mm &= mm - 1;
                        apply_rows(g, md.b, md.bnew, sw.M, B, md.T, base + qq, dc);
                    }
                }
                C += cta_sum_128(dc, red);  // includes the barrier before the label copy
                for (int v = tid; v < n; v += kBatchThreads) sw.b[v] = md.bnew[v];
                __syncthreads();
                // 4. prefix rows, degrees, DL, the stopping rule
                __int128 dd = 0;
                for (int u = wid; u < B; u += kBatchWarps) {
                    prefix_block(sw.M, B, u, sw.P, sw.dout, sw.din, sw.rcp, sw.rcp32, sw.dsum, sw.Pc, md.pstep);
                    if (lane == 0) {
                        dd += md.T[sw.dout[u]];
                        dd += md.T[sw.din[u]];
                    }
                }
                const __int128 Dk = cta_sum_128(dd, red);
                if (tid == 0) {
                    const double dlk = dl_eq2(g.m, g.n, B, fix_to_double(C - Dk));
                    J.hist[k] = dlk;
                    const bool stop = k >= J.max_sweeps ||
                                      (k >= 3 && fabs(J.hist[k - 3] - dlk) < tconv * dlk);
                    s_stop = stop ? 1 : 0;
                    J.dl[1] = prev;
                    J.dl[0] = dlk;
                    prev = dlk;
                }
                __syncthreads();
                if (s_stop) break;
            }
            // 3. compaction: blocks left empty by the sweeps are dropped and
            // the others renumbered in order (the counts rebuilt when any was
            // empty)
            for (int i = tid; i < B; i += kBatchThreads) par[i] = 0;
            __syncthreads();
            for (int v = tid; v < n; v += kBatchThreads) atomicAdd(&par[sw.b[v]], 1);
            __syncthreads();
            if (tid == 0) {
                int next = 0;
                for (int c = 0; c < B; ++c) smap[c] = par[c] > 0 ? next++ : -1;
                s_Bn = next;
                sa.md.B = next;
                sa.md.pstep = (2 * next + 31) / 32;
                s_slot = search_free_slot(sr);
            }
            __syncthreads();
            double dlc = prev;
            if (s_Bn != B) {
                cta_relabel(sw.b, md.bnew, n, smap);
                B = s_Bn;
                cta_rebuild(g, sw.b, sw, B, md.pstep, md.T, red, C, D);
                dlc = dl_eq2(g.m, g.n, B, fix_to_double(C - D));
            }
            // 4. the phase's state joins the bracket; its labels go to the free slot
            int32_t *dst = J.slots + (size_t)s_slot * n;
            for (int v = tid; v < n; v += kBatchThreads) dst[v] = sw.b[v];
            if (tid == 0) {
                J.dl[0] = dlc;
                sr.sweep_id += (uint64_t)k;
                sr.total += k;
                SearchState x;
                x.B = B;
                x.slot = s_slot;
                x.dl = dlc;
                x.id = ++sr.last_id;
                sr.holds = x.id;
                search_insert(sr, x);
                ++sr.phases;
            }
            __syncthreads();
        }
        // the search goes back (ended, or its next phase is not one for this
        // kernel): the labels, then the record, then its ok word, each
        // visible to the host before the next
        __threadfence_system();
        __syncthreads();
        if (tid == 0) {
            sr.B_model = B;
            sr.started = 0;
            const int ok = 2 * B + 4 > group_words ? -1 : 1;
            sr.ok = 0;
            *J.rec = sr;
            __threadfence_system();
            *(volatile int32_t *)&J.rec->ok = ok;
        }
        __syncthreads();
    }
}

int sm_count_b() {
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

bool batch_graph_ok(const sbp_model *m, int64_t max_n) {
    return m->p.hybrid_h == 0 && m->g->n <= max_n && m->g->m < (int64_t(1) << 22) && m->g->max_deg < 65536 &&
           m->g->n < (int64_t(1) << 30);
}

bool batch_eligible(const sbp_model *m, int max_B, int64_t max_n) {
    return m->dense && m->B <= max_B && m->B <= kBatchMaxB && batch_graph_ok(m, max_n);
}

int32_t batch_lim_from(const sbp_model *m) {
    if (!m->dense) return 0;
    return std::min(std::min(kBatchMaxB, m->p.dense_max_B), std::min(m->Bdense, m->Bcap));
}

bool batch_phase_eligible(const sbp_model *m, int32_t B_from, int32_t target, int max_B, int64_t max_n) {
    return B_from <= batch_lim_from(m) && target >= 1 && target < B_from && target <= max_B &&
           target <= kBatchMaxB && batch_graph_ok(m, max_n);
}

int batch_enqueue(const std::vector<BatchSpec> &specs, const sbp_params &p, const BatchTuning &tune,
                  cudaStream_t st) {
    const int nj = (int)specs.size();
    if (nj == 0) return SBP_OK;
    const int max_B = std::min(tune.max_B, kBatchMaxB);
    int blk = 1;
    for (const BatchSpec &sp : specs) {
        const sbp_model *m = sp.m;
        if (!sp.rec || !sp.slots) return fail(SBP_EINVAL, "batch: search without its record or label slots");
        if (!m->dense || !batch_graph_ok(m, INT32_MAX) || sp.lim_from > batch_lim_from(m) ||
            (sp.started && m->B > max_B))
            return fail(SBP_EINVAL, "batch: model not eligible");
        blk = std::max(blk, std::max(sp.lim_from, (int)m->B));
    }
    int blk_cap = 1;
    while (blk_cap < blk) blk_cap <<= 1;
    // device scratch: jobs, hist rows, queue
    const size_t hist_stride = (size_t)p.max_sweeps + 1;
    const size_t bytes = (size_t)nj * sizeof(BatchJob) + (size_t)nj * hist_stride * 8 + 16;
    unsigned char *buf = nullptr;
    SBP_CUDA(cudaMallocAsync(&buf, bytes, st));
    BatchJob *d_jobs = reinterpret_cast<BatchJob *>(buf);
    double *d_hist = reinterpret_cast<double *>(buf + (size_t)nj * sizeof(BatchJob));
    unsigned *d_queue = reinterpret_cast<unsigned *>(d_hist + (size_t)nj * hist_stride);
    // largest graphs first
    std::vector<int> order((size_t)nj);
    for (int i = 0; i < nj; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const sbp_graph *gx = specs[(size_t)x].m->g, *gy = specs[(size_t)y].m->g;
        return gx->m + gx->n > gy->m + gy->n;
    });
    std::vector<BatchJob> jobs((size_t)nj);
    for (int q = 0; q < nj; ++q) {
        const BatchSpec &sp = specs[(size_t)order[(size_t)q]];
        sbp_model *m = sp.m;
        m->nb_ok = false;  // the persistent kernel moves labels without the block-labelled rows
        if (!m->movers) {
            // on this stream, which runs the kernel that first uses them
            // the degree groups' lists and the recheck list of the per-graph pass
            if (model_alloc(&m->movers, (size_t)(m->g->n > 0 ? 2 * m->g->n : 1) * sizeof(Mover), st) != cudaSuccess ||
                model_alloc((void **)&m->mcount, 4 * sizeof(unsigned), st) != cudaSuccess) {
                cudaGetLastError();
                cudaFreeAsync(buf, st);
                return fail(SBP_ENOMEM, "device allocation failed for the mover lists");
            }
        }
        BatchJob &J = jobs[(size_t)q];
        J.a = DecideArgs();
        J.a.g = m->g->dev();
        J.a.md = model_dev(m);
        J.a.v_begin = 0;
        J.a.v_end = m->g->n;
        J.a.movers = static_cast<Mover *>(m->movers);
        J.a.mcount = m->mcount;
        J.a.seed = m->p.seed;
        J.a.sweep_id = 0;
        J.a.beta = m->p.beta;
        J.a.beta32 = (float)m->p.beta;
        J.a.trace_on = 0;
        J.a.tr = sbp_vertex_trace{nullptr, nullptr, nullptr, nullptr};
        J.w.b = m->b;
        J.w.M = m->M;
        J.w.dout = m->dout;
        J.w.din = m->din;
        J.w.dsum = m->dsum;
        J.w.P = m->P;
        J.w.Pc = m->Pc;
        J.w.rcp = m->rcp;
        J.w.rcp32 = m->rcp32;
        J.max_sweeps = m->p.max_sweeps;
        J.merge_x = m->p.merge_proposals;
        J.reduction = m->p.reduction;
        J.t_pre = m->p.t_pre;
        J.t_post = m->p.t_post;
        J.lim_from = sp.lim_from;
        J.max_B = max_B;
        J.hist = d_hist + (size_t)q * hist_stride;
        J.dl = m->dl;
        J.best_s = m->best_s;
        J.best_d = m->best_d;
        J.rec = sp.rec;
        J.slots = sp.slots;
    }
    // the host copy is pageable: it completes before returning
    SBP_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), (size_t)nj * sizeof(BatchJob), cudaMemcpyHostToDevice, st));
    SBP_CUDA(cudaMemsetAsync(d_queue, 0, 4, st));
    // per mover group: B counts and a list of up to B blocks; as many movers
    // per warp as asked for while the CTA's share of shared memory holds them
    const int group_words = 2 * max_B + 4;
    int V = tune.movers_per_warp == 4 ? 4 : tune.movers_per_warp == 2 ? 2 : 1;
    while (V > 1 && (size_t)kBatchWarps * V * group_words * 4 > kBatchSmemCap) V /= 2;
    // the merge rounds' and the compaction's arrays share that memory
    const size_t smem = std::max((size_t)kBatchWarps * V * group_words * 4, (size_t)blk_cap * 20);
    const int per_sm = tune.ctas_per_sm > 0 ? tune.ctas_per_sm : 2;
    const int grid = std::min(nj, sm_count_b() * per_sm);
    auto launch = [&](auto kern) -> int {
        SBP_TRY(ensure_dyn_smem((const void *)kern, smem));
        kern<<<grid, kBatchThreads, smem, st>>>(d_jobs, nj, d_queue, group_words, blk_cap);
        SBP_LAUNCHED();
        return SBP_OK;
    };
    if (p.dl_fp32) {
        SBP_TRY(V == 4 ? launch(k_batch_search<true, 8>) : V == 2 ? launch(k_batch_search<true, 16>)
                                                          : launch(k_batch_search<true, 32>));
    } else {
        SBP_TRY(V == 4 ? launch(k_batch_search<false, 8>) : V == 2 ? launch(k_batch_search<false, 16>)
                                                           : launch(k_batch_search<false, 32>));
    }
    SBP_CUDA(cudaFreeAsync(buf, st));
    return SBP_OK;
}

}  // namespace sbp

// The kernel's bracket code (run here on the host) against Bracket: states
// (B[i], dl[i]) inserted in order into both; after each insert, out[12 i ..]
// holds Bracket's position B values, next()'s result, start and target, then
// the same six from the kernel's code.  *n_bad counts the steps where they
// differ, or where the positions' ids or label slots disagree.
extern "C" int sbp_bracket_check(const int32_t *B, const double *dl, int32_t count, double reduction, int32_t *out,
                                 int32_t *n_bad) {
    if (count < 0 || !n_bad || (count > 0 && (!B || !dl || !out)))
        return sbp::fail(SBP_EINVAL, "sbp_bracket_check: bad count or NULL array");
    if (!(reduction > 0 && reduction < 1)) return sbp::fail(SBP_EINVAL, "sbp_bracket_check: reduction must be in (0, 1)");
    sbp::Bracket hb;
    sbp::SearchRec dr;
    int32_t bad = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (B[i] < 1) return sbp::fail(SBP_EINVAL, "sbp_bracket_check: B must be >= 1");
        sbp::State x;
        x.B = B[i];
        x.dl = dl[i];
        x.id = (uint64_t)i + 1;
        hb.insert(std::move(x));
        sbp::SearchState y;
        y.B = B[i];
        y.dl = dl[i];
        y.id = (uint64_t)i + 1;
        y.slot = sbp::search_free_slot(dr);
        sbp::search_insert(dr, y);
        int hs = 0, ds = 0;
        int32_t ht = 0;
        int dt = 0;
        const bool hok = hb.next(reduction, hs, ht);
        const bool dok = sbp::search_next(dr, reduction, ds, dt);
        int32_t *o = out + (size_t)i * 12;
        bool same = hok == dok && (!hok || (hs == ds && ht == dt)) && y.slot >= 0;
        bool used[4] = {false, false, false, false};
        for (int p = 0; p < 3; ++p) {
            o[p] = hb.s[p].B;
            o[6 + p] = dr.s[p].B;
            same = same && hb.s[p].B == dr.s[p].B && (hb.s[p].B == 0 || hb.s[p].id == dr.s[p].id);
            if (dr.s[p].B != 0) {
                same = same && dr.s[p].slot >= 0 && dr.s[p].slot < 4 && !used[dr.s[p].slot];
                if (dr.s[p].slot >= 0 && dr.s[p].slot < 4) used[dr.s[p].slot] = true;
            }
        }
        o[3] = hok ? 1 : 0;
        o[4] = hok ? hs : 0;
        o[5] = hok ? ht : 0;
        o[9] = dok ? 1 : 0;
        o[10] = dok ? ds : 0;
        o[11] = dok ? dt : 0;
        if (!same) ++bad;
    }
    *n_bad = bad;
    return SBP_OK;
}

extern "C" int sbp_default_batch_options(sbp_batch_options *o) {
    if (!o) return sbp::fail(SBP_EINVAL, "sbp_default_batch_options: NULL");
    o->workers = 32;
    o->max_B = 512;
    o->dense_max_B = 1024;
    o->ctas_per_sm = 2;
    o->max_n = 65536;
    o->movers_per_warp = 2;
    o->mem_fraction = 0.5;
    return SBP_OK;
}
