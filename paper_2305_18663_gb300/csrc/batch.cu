// batch.cu -- many graphs' MCMC phases in one persistent launch.
//
// The batching form of the nodal sweep: thousands of small, uneven graphs
// each need a few tens of sweeps per MCMC phase (Alg. 2) at a few hundred
// blocks.  Launched one graph at a time, each sweep is a dozen small kernels
// plus a host round trip for the convergence test.  Here one persistent
// launch takes a table of jobs (one MCMC phase of one graph each, every graph
// in its own dense model); a CTA pulls a job from a device queue, runs the
// whole phase for it and pulls the next, largest jobs first.  Per sweep,
// inside the CTA:
//   1. proposals, one thread per vertex (the same proposal as the per-graph
//      pass), movers (s != r) appended to the graph's mover list;
//   2. evaluation, one warp per mover: the row is aggregated into
//      direct-mapped per-warp counts in shared memory (B entries), then the
//      same Delta DL, Hastings and test code as the per-graph pass;
//   3. the apply step from the moved vertices' rows.  Each cell update is an
//      atomic whose returned old count gives T[new] - T[old] (x ln x in
//      128-bit fixed point), so sum M ln M is carried exactly from sweep to
//      sweep without a pass over the B x B cells;
//   4. prefix rows, degrees and DL (Eq. 2, the same integer L as a recount,
//      hence the same bits), and the convergence test of Alg. 2 on the device.
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
#include "batch.h"
#include "driver.h"
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
    uint64_t sweep0;     // sweep id of the phase's first sweep
    double t;            // convergence threshold of the phase
    int max_sweeps;
    int dl32;
    double *hist;        // [max_sweeps + 1]; hist[0] = DL after the merge (set by the host)
    int *k_res;          // sweeps done (host-mapped)
    double *dl_res;      // DL after the last sweep (host-mapped)
    double *dl;          // the model's dl[0] (after) and dl[1] (before the last sweep)
};

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

// G: lanes per mover in the evaluation (32 / G movers per warp at a time);
// group_words: shared-memory words of one group (counts, then the list)
template <bool DL32, int G>
__global__ void __launch_bounds__(kBatchThreads, 2) k_batch_mcmc(const BatchJob *__restrict__ jobs, int njobs,
                                                                  unsigned *__restrict__ queue, int group_words) {
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ DecideArgs sa;
    __shared__ ModelOut sw;
    __shared__ __int128 red[kBatchWarps];
    __shared__ unsigned s_job, s_nmov;
    __shared__ int s_stop;
    constexpr int V = 32 / G;  // movers per warp
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int gid = lane / G, gl = lane & (G - 1);
    const unsigned gm = group_mask<G>();
    unsigned *cnt = reinterpret_cast<unsigned *>(bsm) + ((size_t)wid * V + gid) * group_words;
    for (;;) {
        if (tid == 0) s_job = atomicAdd(queue, 1u);
        __syncthreads();
        const unsigned j = s_job;
        if (j >= (unsigned)njobs) return;
        if (tid == 0) {
            sa = jobs[j].a;
            sw = jobs[j].w;
        }
        __syncthreads();
        const BatchJob &J = jobs[j];
        const GraphDev &g = sa.g;
        const ModelDev &md = sa.md;
        const int B = md.B, n = g.n;
        int *list = reinterpret_cast<int *>(cnt + B);
        for (int i = gl; i < B; i += G) cnt[i] = 0u;
        // sum over the cells of T[M] at the phase start (exact)
        __int128 c = 0;
        for (int64_t i = tid; i < (int64_t)B * B; i += kBatchThreads) c += md.T[md.M[i]];
        __int128 C = cta_sum_128(c, red);
        double prev = J.hist[0];
        int k = 0;
        for (;;) {
            ++k;
            const uint64_t sweep_id = J.sweep0 + (uint64_t)(k - 1);
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
            const __int128 D = cta_sum_128(dd, red);
            if (tid == 0) {
                const double dlk = dl_eq2(g.m, g.n, B, fix_to_double(C - D));
                J.hist[k] = dlk;
                const bool stop = k >= J.max_sweeps ||
                                  (k >= 3 && fabs(J.hist[k - 3] - dlk) < J.t * dlk);
                s_stop = stop ? 1 : 0;
                J.dl[1] = prev;
                J.dl[0] = dlk;
                prev = dlk;
                if (stop) {
                    *J.k_res = k;
                    *J.dl_res = dlk;
                }
            }
            __syncthreads();
            if (s_stop) break;
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

bool batch_eligible(const sbp_model *m, int max_B, int64_t max_n) {
    return m->dense && m->p.hybrid_h == 0 && m->B <= max_B && m->B <= kBatchMaxB && m->g->n <= max_n &&
           m->g->m < (int64_t(1) << 22) &&
           m->g->max_deg < 65536 && m->g->n < (int64_t(1) << 30);
}

// Enqueues one MCMC phase for each model on stream st (all eligible and
// idle; hist0[i] = DL after the merge), starting at sweep id sweep0[i] with
// threshold t[i].  When the stream reaches the end of the launch, k_res[i]
// holds the sweeps done and dl_res[i] the last DL (device-visible pointers,
// typically into host-mapped memory), and each model is in the state the
// per-graph sweeps would leave.  The launch's scratch is freed in stream
// order.
int batch_enqueue(const std::vector<sbp_model *> &models, const std::vector<uint64_t> &sweep0,
                  const std::vector<double> &t, const std::vector<double> &hist0, const std::vector<int *> &k_res,
                  const std::vector<double *> &dl_res, const BatchTuning &tune, cudaStream_t st) {
    const int nj = (int)models.size();
    if (nj == 0) return SBP_OK;
    int maxB = 1, max_sweeps = 1, dl32 = models[0]->p.dl_fp32;
    for (const sbp_model *m : models) {
        maxB = std::max(maxB, (int)m->B);
        max_sweeps = std::max(max_sweeps, m->p.max_sweeps);
        if (m->p.dl_fp32 != dl32) return fail(SBP_EINVAL, "batch: all models must share dl_fp32");
        if (!batch_eligible(m, kBatchMaxB, INT32_MAX)) return fail(SBP_EINVAL, "batch: model not eligible");
    }
    // device scratch: jobs, hist rows, queue
    const size_t hist_stride = (size_t)max_sweeps + 1;
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
        return models[(size_t)x]->g->m + models[(size_t)x]->g->n > models[(size_t)y]->g->m + models[(size_t)y]->g->n;
    });
    std::vector<BatchJob> jobs((size_t)nj);
    std::vector<double> h0((size_t)nj * hist_stride, 0.0);
    for (int q = 0; q < nj; ++q) {
        const int i = order[(size_t)q];
        sbp_model *m = models[(size_t)i];
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
        J.a.sweep_id = sweep0[(size_t)i];
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
        J.sweep0 = sweep0[(size_t)i];
        J.t = t[(size_t)i];
        J.max_sweeps = m->p.max_sweeps;
        J.dl32 = dl32;
        J.hist = d_hist + (size_t)q * hist_stride;
        J.k_res = k_res[(size_t)i];
        J.dl_res = dl_res[(size_t)i];
        J.dl = m->dl;
        h0[(size_t)q * hist_stride] = hist0[(size_t)i];
    }
    // the host copies are pageable: these copies complete before returning
    SBP_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), (size_t)nj * sizeof(BatchJob), cudaMemcpyHostToDevice, st));
    SBP_CUDA(cudaMemcpyAsync(d_hist, h0.data(), h0.size() * 8, cudaMemcpyHostToDevice, st));
    SBP_CUDA(cudaMemsetAsync(d_queue, 0, 4, st));
    // per mover group: B counts and a list of up to B blocks; as many movers
    // per warp as asked for while the CTA's share of shared memory holds them
    const int group_words = 2 * maxB + 4;
    int V = tune.movers_per_warp == 4 ? 4 : tune.movers_per_warp == 2 ? 2 : 1;
    while (V > 1 && (size_t)kBatchWarps * V * group_words * 4 > kBatchSmemCap) V /= 2;
    const size_t smem = (size_t)kBatchWarps * V * group_words * 4;
    const int per_sm = tune.ctas_per_sm > 0 ? tune.ctas_per_sm : 2;
    const int grid = std::min(nj, sm_count_b() * per_sm);
    auto launch = [&](auto kern) -> int {
        SBP_TRY(ensure_dyn_smem((const void *)kern, smem));
        kern<<<grid, kBatchThreads, smem, st>>>(d_jobs, nj, d_queue, group_words);
        SBP_LAUNCHED();
        return SBP_OK;
    };
    if (dl32) {
        SBP_TRY(V == 4 ? launch(k_batch_mcmc<true, 8>) : V == 2 ? launch(k_batch_mcmc<true, 16>)
                                                          : launch(k_batch_mcmc<true, 32>));
    } else {
        SBP_TRY(V == 4 ? launch(k_batch_mcmc<false, 8>) : V == 2 ? launch(k_batch_mcmc<false, 16>)
                                                           : launch(k_batch_mcmc<false, 32>));
    }
    SBP_CUDA(cudaFreeAsync(buf, st));
    return SBP_OK;
}

}  // namespace sbp

extern "C" int sbp_default_batch_options(sbp_batch_options *o) {
    if (!o) return sbp::fail(SBP_EINVAL, "sbp_default_batch_options: NULL");
    o->workers = 16;
    o->max_B = 512;
    o->dense_max_B = 4096;
    o->ctas_per_sm = 2;
    o->max_n = 4096;
    o->movers_per_warp = 2;
    o->mem_fraction = 0.5;
    return SBP_OK;
}
