// api.cu -- the C ABI of libsbp: handles, passes, merge phase and driver.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "driver.h"

namespace sbp {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

cudaError_t model_alloc(void **p, size_t bytes, cudaStream_t st) {
    return cudaMallocAsync(p, bytes > 0 ? bytes : 1, st);
}

void model_free(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

namespace {
std::mutex g_pinned_mu;
std::vector<void *> g_pinned_free;
}  // namespace

// 4 KB pinned buffers, never returned to the driver (cudaFreeHost would
// synchronise the device)
void *pinned_get() {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    if (!g_pinned_free.empty()) {
        void *p = g_pinned_free.back();
        g_pinned_free.pop_back();
        return p;
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, 4096) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pinned_put(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    g_pinned_free.push_back(p);
}

int ensure_dyn_smem(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> set;
    int dev = 0;
    SBP_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = set[std::make_pair(dev, func)];
    if (bytes > cur) {
        SBP_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        cur = bytes;
    }
    return SBP_OK;
}

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SBP_ENOMEM : SBP_ECUDA;
}

int check_status(const sbp_model *m) {
    int32_t st = 0;
    SBP_CUDA(cudaMemcpyAsync(&st, m->status, 4, cudaMemcpyDeviceToHost, m->stream));
    SBP_CUDA(cudaStreamSynchronize(m->stream));
    if (st != 0) {
        SBP_CUDA(cudaMemsetAsync(m->status, 0, 4, m->stream));
        return fail(st, "a kernel recorded status " + std::to_string(st) +
                             (st == SBP_EHASHFULL ? " (neighbour table full)" : ""));
    }
    return SBP_OK;
}

namespace {

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaMemcpyKind kind_from_dev(const void *dst) {
    return is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

int validate_params(const sbp_params &p) {
    if (!std::isfinite(p.beta) || p.beta < 0) return fail(SBP_EINVAL, "params: beta must be finite and >= 0");
    if (p.merge_proposals < 1) return fail(SBP_EINVAL, "params: merge_proposals must be >= 1");
    if (p.max_sweeps < 1) return fail(SBP_EINVAL, "params: max_sweeps must be >= 1");
    if (!(p.reduction > 0 && p.reduction < 1)) return fail(SBP_EINVAL, "params: reduction must be in (0, 1)");
    if (!(p.t_pre > 0) || !(p.t_post > 0)) return fail(SBP_EINVAL, "params: thresholds must be > 0");
    if (p.dense_max_B < 1 || p.dense_max_B > 16384) return fail(SBP_EINVAL, "params: dense_max_B must be in [1, 16384]");
    if (p.full_rebuild != 0 && p.full_rebuild != 1) return fail(SBP_EINVAL, "params: full_rebuild must be 0 or 1");
    if (p.dl_fp32 != 0 && p.dl_fp32 != 1) return fail(SBP_EINVAL, "params: dl_fp32 must be 0 or 1");
    if (p.hybrid_h < 0) return fail(SBP_EINVAL, "params: hybrid_h must be >= 0");
    return SBP_OK;
}

struct Stats {
    DevCounters c;
    double dl[2];
    int32_t status;
};

int read_stats(sbp_model *m, sbp_sweep_stats *out) {
    Stats *h = static_cast<Stats *>(m->pinned);
    SBP_CUDA(cudaMemcpyAsync(&h->c, m->counters, sizeof(DevCounters), cudaMemcpyDeviceToHost, m->stream));
    SBP_CUDA(cudaMemcpyAsync(h->dl, m->dl, 16, cudaMemcpyDeviceToHost, m->stream));
    SBP_CUDA(cudaMemcpyAsync(&h->status, m->status, 4, cudaMemcpyDeviceToHost, m->stream));
    SBP_CUDA(cudaStreamSynchronize(m->stream));
    if (h->status != 0) {
        const int st = h->status;
        SBP_CUDA(cudaMemsetAsync(m->status, 0, 4, m->stream));
        return fail(st, "a kernel recorded status " + std::to_string(st));
    }
    out->n_proposed = (int64_t)h->c.proposed;
    out->n_moves = (int64_t)h->c.moves;
    out->n_accepted = (int64_t)h->c.accepted;
    out->n_margin = (int64_t)h->c.margin;
    out->n_move_edges = (int64_t)h->c.move_edges;
    out->n_recheck = (int64_t)h->c.recheck;
    out->n_entries = (int64_t)h->c.entries;
    out->dl_after = h->dl[0];
    out->dl_before = h->dl[1];
    return SBP_OK;
}

// labels outside [0, B): the slot keeps INT32_MAX - (smallest such vertex)
__global__ void k_check_labels(const int32_t *__restrict__ b, int64_t n, int32_t B, int32_t *__restrict__ slot) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (b[v] < 0 || b[v] >= B) atomicMax(slot, (int32_t)(INT32_MAX - v));
}

// Labels set from outside against the current ones, with the same block
// count: the range check of k_check_labels, and every changed vertex listed
// the way the decision kernels list an accepted move (its kMoveChunk-edge
// items, its degree in acc_edges), so that the commit of a pass can apply
// the change.  Counters and item slots are taken once per warp.
__global__ void k_diff_labels(const int32_t *__restrict__ bnew, const int32_t *__restrict__ b, int64_t n, int32_t B,
                              const int32_t *__restrict__ op, const int32_t *__restrict__ ip, int2 *__restrict__ items,
                              int64_t cap, DevCounters *__restrict__ c, int32_t *__restrict__ slot) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;
        int k = 0, nch = 0;
        if (v < n) {
            const int32_t lab = bnew[v];
            if (lab < 0 || lab >= B) {
                atomicMax(slot, (int32_t)(INT32_MAX - v));
            } else if (lab != b[v]) {
                k = (op[v + 1] - op[v]) + (ip[v + 1] - ip[v]);
                nch = (k + kMoveChunk - 1) / kMoveChunk;
            }
        }
        int incl = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int wtotal = __shfl_sync(0xffffffffu, incl, 31);
        const unsigned wk = __reduce_add_sync(0xffffffffu, (unsigned)k);
        unsigned long long first = 0;
        if (lane == 0 && wtotal > 0) {
            first = atomicAdd(&c->items, (unsigned long long)wtotal);
            atomicAdd(&c->acc_edges, (unsigned long long)wk);
        }
        first = __shfl_sync(0xffffffffu, first, 0);
        for (int q = 0; q < nch; ++q) {
            const unsigned long long at = first + (unsigned long long)(incl - nch + q);
            if (at < (unsigned long long)cap) items[at] = make_int2((int)v, q);
        }
    }
}

// Labels with the block count the model already has, once it has its
// accepted-move list: the change against the current labels is applied like
// the moves of a pass (the commit's plan, on the device, updates the counts
// from the changed vertices' rows when they hold at most a quarter of the
// edges, else recounts; the block-labelled rows follow the changed vertices).
// Same counts and DL as a rebuild from scratch.
int upload_incremental(sbp_model *m, const int32_t *b) {
    const int64_t n = m->g->n;
    int32_t *slot = m->status + 2;
    SBP_CUDA(cudaMemcpyAsync(m->bnew, b, (size_t)n * 4, cudaMemcpyDefault, m->stream));
    SBP_CUDA(cudaMemsetAsync(m->counters, 0, sizeof(DevCounters), m->stream));
    SBP_CUDA(cudaMemsetAsync(slot, 0, 4, m->stream));
    k_diff_labels<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, m->stream>>>(
        m->bnew, m->b, n, m->B, m->g->op, m->g->ip, m->items, m->cap_items, m->counters, slot);
    SBP_LAUNCHED();
    int32_t *h = static_cast<int32_t *>(m->pinned);
    SBP_CUDA(cudaMemcpyAsync(h, slot, 4, cudaMemcpyDeviceToHost, m->stream));
    SBP_CUDA(cudaStreamSynchronize(m->stream));
    if (*h > 0) {
        SBP_CUDA(cudaMemcpyAsync(m->bnew, m->b, (size_t)n * 4, cudaMemcpyDeviceToDevice, m->stream));
        SBP_CUDA(cudaMemsetAsync(m->counters, 0, sizeof(DevCounters), m->stream));
        return fail(SBP_EINVAL, "label out of [0, B) at vertex " + std::to_string((int64_t)INT32_MAX - *h));
    }
    std::swap(m->b, m->bnew);
    SBP_CUDA(cudaMemcpyAsync(m->dl + 1, m->dl, 8, cudaMemcpyDeviceToDevice, m->stream));
    m->list_ok = true;  // the items list every change, once
    m->decided.clear();
    m->nb_in_commit = false;
    int rc = commit_blockmodel(m);
    if (rc == SBP_OK) rc = nb_rows_after_commit(m);
    if (rc != SBP_OK) m->nb_ok = false;
    SBP_CUDA(cudaMemsetAsync(m->counters, 0, sizeof(DevCounters), m->stream));
    return rc;
}

// The labels go to the pending buffer, are checked on the device (one read
// back), and only then become the assignment: a bad label leaves the model
// as it was.
int upload_assignment(sbp_model *m, int32_t B, const int32_t *b) {
    const int64_t n = m->g->n;
    if (B < 1 || B > n) return fail(SBP_EINVAL, "B must be in [1, n]");
    if (!b) return fail(SBP_EINVAL, "assignment pointer is NULL");
    if (B == m->B && m->items && !m->p.full_rebuild) return upload_incremental(m, b);
    int32_t *slot = m->status + 2;
    SBP_CUDA(cudaMemcpyAsync(m->bnew, b, (size_t)n * 4, cudaMemcpyDefault, m->stream));
    SBP_CUDA(cudaMemsetAsync(slot, 0, 4, m->stream));
    k_check_labels<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, m->stream>>>(m->bnew, n, B, slot);
    SBP_LAUNCHED();
    int32_t *h = static_cast<int32_t *>(m->pinned);
    SBP_CUDA(cudaMemcpyAsync(h, slot, 4, cudaMemcpyDeviceToHost, m->stream));
    SBP_CUDA(cudaStreamSynchronize(m->stream));
    if (*h > 0) {
        SBP_CUDA(cudaMemcpyAsync(m->bnew, m->b, (size_t)n * 4, cudaMemcpyDeviceToDevice, m->stream));
        return fail(SBP_EINVAL, "label out of [0, B) at vertex " + std::to_string((int64_t)INT32_MAX - *h));
    }
    SBP_TRY(ensure_capacity(m, B));
    m->B = B;
    std::swap(m->b, m->bnew);
    return rebuild_blockmodel(m);
}

int64_t merge_key(double d) { return (int64_t)std::floor(d * 1048576.0 + 0.5); }

// Alg. 1 "sort best_merges", "pop, merge c into c'": links in ascending
// (key, r), pointer-based union (Section III-A (d)), stops at n_merges.
// map[c] = new dense label, groups numbered by their smallest member.
int64_t apply_merges(int32_t B, const std::vector<int32_t> &bs, const std::vector<double> &bd, int64_t n_merges,
                     std::vector<int32_t> &map, int32_t &B_new) {
    std::vector<std::pair<int64_t, int32_t>> it((size_t)B);
    for (int32_t r = 0; r < B; ++r) it[(size_t)r] = {merge_key(bd[(size_t)r]), r};
    std::sort(it.begin(), it.end());
    std::vector<int32_t> parent((size_t)B);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int32_t x) {
        while (parent[(size_t)x] != x) {
            parent[(size_t)x] = parent[(size_t)parent[(size_t)x]];
            x = parent[(size_t)x];
        }
        return x;
    };
    int64_t done = 0;
    for (size_t k = 0; k < it.size() && done < n_merges; ++k) {
        const int32_t r = it[k].second, s = bs[(size_t)r];
        if (s < 0) continue;
        const int32_t a = find(r), c = find(s);
        if (a == c) continue;
        parent[(size_t)a] = c;
        ++done;
    }
    std::vector<int32_t> label((size_t)B, -1);
    map.assign((size_t)B, 0);
    int32_t next = 0;
    for (int32_t c = 0; c < B; ++c) {
        const int32_t root = find(c);
        if (label[(size_t)root] < 0) label[(size_t)root] = next++;
        map[(size_t)c] = label[(size_t)root];
    }
    B_new = next;
    return done;
}

int relabel_and_rebuild(sbp_model *m, const std::vector<int32_t> &map, int32_t B_new) {
    SBP_CUDA(cudaMemcpyAsync(m->map, map.data(), map.size() * 4, cudaMemcpyHostToDevice, m->stream));
    SBP_TRY(launch_relabel(m, m->map));
    SBP_CUDA(cudaStreamSynchronize(m->stream));
    SBP_TRY(ensure_capacity(m, B_new));  // dense or sparse for the new B
    m->B = B_new;
    return rebuild_blockmodel(m);
}

}  // namespace

int params_valid(const sbp_params &p) { return validate_params(p); }

}  // namespace sbp

using namespace sbp;

extern "C" size_t sbp_last_error(char *buf, size_t len) {
    const std::string &e = g_last_error;
    if (buf && len) {
        const size_t k = std::min(len - 1, e.size());
        std::memcpy(buf, e.data(), k);
        buf[k] = '\0';
    }
    return e.size();
}

extern "C" int sbp_default_params(sbp_params *p) {
    if (!p) return fail(SBP_EINVAL, "sbp_default_params: NULL");
    std::memset(p, 0, sizeof(*p));
    p->seed = 0;
    p->beta = 3.0;
    p->merge_proposals = 10;
    p->max_sweeps = 100;
    p->reduction = 0.5;
    p->t_pre = 5e-4;
    p->t_post = 1e-4;
    p->dense_max_B = 4096;
    p->full_rebuild = 0;
    p->dl_fp32 = 1;
    p->hybrid_h = 0;
    return SBP_OK;
}

extern "C" void sbp_free_model(sbp_model_t *m) {
    if (!m) return;
    cudaStream_t st = m->stream;
    if (st) cudaStreamSynchronize(st);
    void *ps[] = {m->b,        m->bnew,   m->M,        m->P,       m->Pc,     m->dout,  m->din,
                  m->rcp,      m->rcp32,  m->dsum,     m->dl,      m->partials, m->counters, m->status,
                  m->best_s,   m->best_d, m->map,      m->vcount,  m->movers, m->mcount, m->skip,
                  m->items,    m->nbo,    m->nbi,      m->cta_tab};
    for (void *p : ps) model_free(p, st);
    for (int i = 0; i < 2; ++i) {
        if (m->side[i]) cudaStreamDestroy(m->side[i]);
        if (m->join_ev[i]) cudaEventDestroy(m->join_ev[i]);
    }
    if (m->fork_ev) cudaEventDestroy(m->fork_ev);
    free_sparse(m);
    pinned_put(m->pinned);
    if (st) cudaStreamSynchronize(st);
    delete m;
}

extern "C" int sbp_build_blockmodel(const sbp_graph_t *g, int32_t B, const int32_t *b, const sbp_params *p,
                                    void *stream, sbp_model_t **out) {
    if (!out) return fail(SBP_EINVAL, "sbp_build_blockmodel: out is NULL");
    *out = nullptr;
    if (!g) return fail(SBP_EINVAL, "sbp_build_blockmodel: graph is NULL");
    sbp_params prm;
    if (p) prm = *p;
    else sbp_default_params(&prm);
    SBP_TRY(validate_params(prm));
    if (B < 1 || B > g->n) return fail(SBP_EINVAL, "sbp_build_blockmodel: B must be in [1, n]");
    auto *m = new sbp_model();
    m->g = g;
    m->p = prm;
    m->stream = static_cast<cudaStream_t>(stream);
    m->npartials = 1024;
    const size_t n = (size_t)g->n;
    cudaStream_t st = m->stream;
    m->pinned = pinned_get();
    if (model_alloc((void **)&m->b, n * 4, st) != cudaSuccess || model_alloc((void **)&m->bnew, n * 4, st) != cudaSuccess ||
        model_alloc((void **)&m->dl, 16, st) != cudaSuccess ||
        model_alloc((void **)&m->partials, (size_t)m->npartials * 32, st) != cudaSuccess ||
        model_alloc((void **)&m->counters, sizeof(DevCounters), st) != cudaSuccess ||
        model_alloc((void **)&m->status, 16, st) != cudaSuccess || !m->pinned) {
        cudaGetLastError();
        sbp_free_model(m);
        return fail(SBP_ENOMEM, "sbp_build_blockmodel: allocation failed");
    }
    cudaMemsetAsync(m->counters, 0, sizeof(DevCounters), m->stream);
    cudaMemsetAsync(m->status, 0, 4, m->stream);
    cudaMemsetAsync(m->dl, 0, 16, m->stream);
    const int rc = upload_assignment(m, B, b);
    if (rc != SBP_OK) {
        sbp_free_model(m);
        return rc;
    }
    *out = m;
    return SBP_OK;
}

extern "C" int sbp_set_assignment(sbp_model_t *m, int32_t B, const int32_t *b) {
    if (!m) return fail(SBP_EINVAL, "sbp_set_assignment: NULL model");
    return upload_assignment(m, B, b);
}

extern "C" int sbp_nodal_decide(sbp_model_t *m, uint64_t sweep_id, int64_t v_begin, int64_t v_end,
                                const sbp_vertex_trace *trace) {
    if (!m) return fail(SBP_EINVAL, "sbp_nodal_decide: NULL model");
    if (v_begin < 0 || v_end > m->g->n || v_begin > v_end) return fail(SBP_EINVAL, "sbp_nodal_decide: bad vertex range");
    if (trace) {
        const void *ps[4] = {trace->s, trace->flags, trace->dH, trace->logA};
        for (const void *q : ps)
            if (q && !is_device_ptr(q)) return fail(SBP_EINVAL, "sbp_nodal_decide: trace buffers must be device memory");
    }
    if (v_begin == v_end) return SBP_OK;
    return launch_decide(m, sweep_id, v_begin, v_end, trace);
}

namespace sbp {
namespace {

// pending labels from device memory: out-of-range labels keep the vertex in
// its block and record SBP_EINVAL
__global__ void k_set_pending(const int32_t *__restrict__ in, int64_t v_begin, int64_t count, int32_t B,
                              const int32_t *__restrict__ b, int32_t *__restrict__ bnew, int32_t *status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t lab = in[i];
        const bool ok = lab >= 0 && lab < B;
        bnew[v_begin + i] = ok ? lab : b[v_begin + i];
        if (!ok) record_status(status, SBP_EINVAL);
    }
}

}  // namespace
}  // namespace sbp

extern "C" int sbp_get_pending(const sbp_model_t *m, int64_t v_begin, int64_t v_end, int32_t *out) {
    if (!m || !out) return fail(SBP_EINVAL, "sbp_get_pending: NULL argument");
    if (v_begin < 0 || v_end > m->g->n || v_begin > v_end) return fail(SBP_EINVAL, "sbp_get_pending: bad vertex range");
    if (v_begin < v_end)
        SBP_CUDA(cudaMemcpyAsync(out, m->bnew + v_begin, (size_t)(v_end - v_begin) * 4, kind_from_dev(out), m->stream));
    return check_status(m);
}

extern "C" int sbp_set_pending(sbp_model_t *m, int64_t v_begin, int64_t v_end, const int32_t *in) {
    if (!m || !in) return fail(SBP_EINVAL, "sbp_set_pending: NULL argument");
    if (v_begin < 0 || v_end > m->g->n || v_begin > v_end) return fail(SBP_EINVAL, "sbp_set_pending: bad vertex range");
    const int64_t count = v_end - v_begin;
    if (count == 0) return SBP_OK;
    m->list_ok = false;  // the accepted-move list no longer holds every change
    if (is_device_ptr(in)) {
        const int grid = (int)std::min<int64_t>((count + 255) / 256, 4096);
        k_set_pending<<<grid, 256, 0, m->stream>>>(in, v_begin, count, m->B, m->b, m->bnew, m->status);
        SBP_LAUNCHED();
        return SBP_OK;
    }
    for (int64_t i = 0; i < count; ++i)
        if (in[i] < 0 || in[i] >= m->B)
            return fail(SBP_EINVAL, "sbp_set_pending: label out of [0, B) at vertex " + std::to_string(v_begin + i));
    SBP_CUDA(cudaMemcpyAsync(m->bnew + v_begin, in, (size_t)count * 4, cudaMemcpyHostToDevice, m->stream));
    SBP_CUDA(cudaStreamSynchronize(m->stream));
    return SBP_OK;
}

extern "C" int sbp_commit(sbp_model_t *m, sbp_sweep_stats *stats) {
    if (!m) return fail(SBP_EINVAL, "sbp_commit: NULL model");
    std::swap(m->b, m->bnew);
    SBP_CUDA(cudaMemcpyAsync(m->dl + 1, m->dl, 8, cudaMemcpyDeviceToDevice, m->stream));
    m->nb_in_commit = false;
    int rc = commit_blockmodel(m);
    if (rc == SBP_OK) rc = nb_rows_after_commit(m);
    if (rc != SBP_OK) m->nb_ok = false;
    m->list_ok = true;
    m->decided.clear();
    SBP_TRY(rc);
    if (stats) SBP_TRY(read_stats(m, stats));
    SBP_CUDA(cudaMemsetAsync(m->counters, 0, sizeof(DevCounters), m->stream));
    return SBP_OK;
}

extern "C" int sbp_nodal_sweep(sbp_model_t *m, uint64_t sweep_id, int64_t v_begin, int64_t v_end,
                               sbp_sweep_stats *stats) {
    SBP_TRY(sbp_nodal_decide(m, sweep_id, v_begin, v_end, nullptr));
    return sbp_commit(m, stats);
}

extern "C" int sbp_merge_proposals(sbp_model_t *m, uint64_t round_id, int32_t *best_s, double *best_dDL) {
    if (!m) return fail(SBP_EINVAL, "sbp_merge_proposals: NULL model");
    if (m->B < 2) return fail(SBP_ESTATE, "sbp_merge_proposals: needs B >= 2");
    SBP_TRY(launch_merge_proposals(m, round_id));
    if (best_s) SBP_CUDA(cudaMemcpyAsync(best_s, m->best_s, (size_t)m->B * 4, kind_from_dev(best_s), m->stream));
    if (best_dDL) SBP_CUDA(cudaMemcpyAsync(best_dDL, m->best_d, (size_t)m->B * 8, kind_from_dev(best_dDL), m->stream));
    SBP_CUDA(cudaStreamSynchronize(m->stream));
    return check_status(m);
}

extern "C" int sbp_merge_blocks(sbp_model_t *m, uint64_t round_id, int32_t n_merges, int32_t *B_out,
                                int32_t *rounds_used) {
    if (!m) return fail(SBP_EINVAL, "sbp_merge_blocks: NULL model");
    if (n_merges < 1 || n_merges >= m->B) return fail(SBP_EINVAL, "sbp_merge_blocks: need 1 <= n_merges < B");
    int32_t rounds = 0;
    int64_t left = n_merges;
    std::vector<int32_t> bs, map;
    std::vector<double> bd;
    while (left > 0 && m->B >= 2) {
        const int32_t B = m->B;
        SBP_TRY(launch_merge_proposals(m, round_id + (uint64_t)rounds));
        ++rounds;
        bs.resize((size_t)B);
        bd.resize((size_t)B);
        SBP_CUDA(cudaMemcpyAsync(bs.data(), m->best_s, (size_t)B * 4, cudaMemcpyDeviceToHost, m->stream));
        SBP_CUDA(cudaMemcpyAsync(bd.data(), m->best_d, (size_t)B * 8, cudaMemcpyDeviceToHost, m->stream));
        SBP_CUDA(cudaStreamSynchronize(m->stream));
        int32_t Bn = B;
        const int64_t done = apply_merges(B, bs, bd, left, map, Bn);
        SBP_TRY(relabel_and_rebuild(m, map, Bn));
        left -= done;
        if (done == 0) break;
    }
    if (B_out) *B_out = m->B;
    if (rounds_used) *rounds_used = rounds;
    return check_status(m);
}

extern "C" int sbp_compact(sbp_model_t *m, int32_t *B_out) {
    if (!m) return fail(SBP_EINVAL, "sbp_compact: NULL model");
    const int32_t B = m->B;
    SBP_TRY(launch_vertex_count(m));
    std::vector<int32_t> cnt((size_t)B), map((size_t)B, -1);
    SBP_CUDA(cudaMemcpyAsync(cnt.data(), m->vcount, (size_t)B * 4, cudaMemcpyDeviceToHost, m->stream));
    SBP_CUDA(cudaStreamSynchronize(m->stream));
    int32_t next = 0;
    for (int32_t c = 0; c < B; ++c)
        if (cnt[(size_t)c] > 0) map[(size_t)c] = next++;
    if (next != B) SBP_TRY(relabel_and_rebuild(m, map, next));
    if (B_out) *B_out = m->B;
    return SBP_OK;
}

// ---------------------------------------------------------------------------
// golden-ratio search over the number of blocks (Section II-B)
namespace sbp {
namespace {

int read_assignment(sbp_model *m, std::vector<int32_t> &b) {
    b.resize((size_t)m->g->n);
    SBP_CUDA(cudaMemcpyAsync(b.data(), m->b, b.size() * 4, cudaMemcpyDeviceToHost, m->stream));
    SBP_CUDA(cudaStreamSynchronize(m->stream));
    return SBP_OK;
}

int read_dl(sbp_model *m, double &dl) {
    SBP_CUDA(cudaMemcpyAsync(m->pinned, m->dl, 8, cudaMemcpyDeviceToHost, m->stream));
    SBP_CUDA(cudaStreamSynchronize(m->stream));
    dl = *static_cast<double *>(m->pinned);
    return SBP_OK;
}

}  // namespace

int PartitionRun::begin(sbp_model *model) {
    m = model;
    hist.assign((size_t)m->p.max_sweeps + 1, 0.0);
    State init;
    init.B = m->B;
    init.id = ++last_id;
    SBP_TRY(read_dl(m, init.dl));
    SBP_TRY(read_assignment(m, init.b));
    model_holds = init.id;
    br.insert(std::move(init));
    plan();
    return SBP_OK;
}

void PartitionRun::plan() {
    if (!br.next(m->p.reduction, start, target)) {
        done = true;
        return;
    }
    t = br.s[2].B == 0 ? m->p.t_pre : m->p.t_post;
    k = 0;
}

int PartitionRun::start_phase() {
    const State &from = br.s[start];
    // the model already holds that state (labels, counts, DL) when it is the
    // one the last phase ended in; uploading it again would rebuild the same
    if (from.id != model_holds) SBP_TRY(upload_assignment(m, from.B, from.b.data()));
    model_holds = 0;
    int32_t Bm = m->B, rounds = 0;
    SBP_TRY(sbp_merge_blocks(m, round_id, from.B - target, &Bm, &rounds));
    round_id += (uint64_t)rounds;
    SBP_TRY(read_dl(m, hist[0]));
    k = 0;
    return SBP_OK;
}

bool PartitionRun::phase_over() const {
    if (k >= m->p.max_sweeps) return true;
    return k >= 3 && std::fabs(hist[(size_t)k - 3] - hist[(size_t)k]) < t * hist[(size_t)k];
}

int PartitionRun::sweep() {
    sbp_sweep_stats st;
    SBP_TRY(sbp_nodal_sweep(m, sweep_id++, 0, m->g->n, &st));
    ++k;
    hist[(size_t)k] = st.dl_after;
    return SBP_OK;
}

int PartitionRun::end_phase() {
    total += k;
    int32_t Bc = m->B;
    SBP_TRY(sbp_compact(m, &Bc));
    State x;
    x.B = m->B;
    x.id = ++last_id;
    SBP_TRY(read_dl(m, x.dl));
    SBP_TRY(read_assignment(m, x.b));
    model_holds = x.id;
    br.insert(std::move(x));
    plan();
    return SBP_OK;
}

void PartitionRun::export_search(SearchRec &rec, int32_t *slots, bool started) const {
    const size_t n = (size_t)m->g->n;
    for (int p = 0; p < 3; ++p) {
        const State &x = br.s[p];
        rec.s[p].B = x.B;
        rec.s[p].slot = p;
        rec.s[p].dl = x.dl;
        rec.s[p].id = x.id;
        if (x.B != 0) std::memcpy(slots + (size_t)p * n, x.b.data(), n * 4);
    }
    rec.sweep_id = sweep_id;
    rec.round_id = round_id;
    rec.last_id = last_id;
    rec.holds = model_holds;
    rec.total = total;
    rec.started = started ? 1 : 0;
    rec.B_model = m->B;
    rec.done = rec.phases = rec.merged = rec.starts = rec.ok = 0;
}

void PartitionRun::import_search(const SearchRec &rec, const int32_t *slots) {
    const size_t n = (size_t)m->g->n;
    for (int p = 0; p < 3; ++p) {
        State &x = br.s[p];
        x.B = rec.s[p].B;
        x.dl = rec.s[p].dl;
        x.id = rec.s[p].id;
        if (x.B != 0) x.b.assign(slots + (size_t)rec.s[p].slot * n, slots + (size_t)rec.s[p].slot * n + n);
        else x.b.clear();
    }
    sweep_id = rec.sweep_id;
    round_id = rec.round_id;
    last_id = rec.last_id;
    model_holds = rec.holds;
    total = rec.total;
    // the model's host-side view of what the kernel left: B, and the
    // derived state a rebuild resets
    m->B = rec.B_model;
    m->nb_ok = false;
    m->list_ok = true;
    m->decided.clear();
    if (rec.done) done = true;
    else plan();
}

int PartitionRun::finish(int32_t *b_out, int32_t *B_out, double *dl_out, int64_t *n_sweeps) const {
    const State &best = br.s[1];
    if (b_out)
        SBP_CUDA(cudaMemcpy(b_out, best.b.data(), (size_t)m->g->n * 4,
                            is_device_ptr(b_out) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
    if (B_out) *B_out = best.B;
    if (dl_out) *dl_out = best.dl;
    if (n_sweeps) *n_sweeps = total;
    return SBP_OK;
}

namespace {

int run_partition(sbp_model *m, int32_t *b_out, int32_t *B_out, double *dl_out, int64_t *n_sweeps) {
    PartitionRun r;
    SBP_TRY(r.begin(m));
    while (!r.done) {
        SBP_TRY(r.start_phase());
        while (!r.phase_over()) SBP_TRY(r.sweep());
        SBP_TRY(r.end_phase());
    }
    return r.finish(b_out, B_out, dl_out, n_sweeps);
}

}  // namespace
}  // namespace sbp

extern "C" int sbp_partition(const sbp_graph_t *g, const sbp_params *p, void *stream, int32_t *b_out, int32_t *B_out,
                             double *dl_out, int64_t *n_sweeps) {
    if (!g || !b_out) return fail(SBP_EINVAL, "sbp_partition: NULL argument");
    sbp_params prm;
    if (p) prm = *p;
    else sbp_default_params(&prm);
    SBP_TRY(validate_params(prm));
    std::vector<int32_t> ident((size_t)g->n);
    std::iota(ident.begin(), ident.end(), 0);
    sbp_model_t *m = nullptr;
    SBP_TRY(sbp_build_blockmodel(g, (int32_t)g->n, ident.data(), &prm, stream, &m));
    const int rc = run_partition(m, b_out, B_out, dl_out, n_sweeps);
    sbp_free_model(m);
    return rc;
}

// ---------------------------------------------------------------------------
// read-back

extern "C" int sbp_sync(const sbp_model_t *m) {
    if (!m) return fail(SBP_EINVAL, "sbp_sync: NULL model");
    return check_status(m);
}

extern "C" int sbp_get_assignment(const sbp_model_t *m, int32_t *b_out) {
    if (!m || !b_out) return fail(SBP_EINVAL, "sbp_get_assignment: NULL argument");
    SBP_CUDA(cudaMemcpyAsync(b_out, m->b, (size_t)m->g->n * 4, kind_from_dev(b_out), m->stream));
    return check_status(m);
}

extern "C" int sbp_get_B(const sbp_model_t *m, int32_t *B_out) {
    if (!m || !B_out) return fail(SBP_EINVAL, "sbp_get_B: NULL argument");
    *B_out = m->B;
    return SBP_OK;
}

extern "C" int sbp_get_dl(const sbp_model_t *m, double *dl_out) {
    if (!m || !dl_out) return fail(SBP_EINVAL, "sbp_get_dl: NULL argument");
    SBP_CUDA(cudaMemcpyAsync(dl_out, m->dl, 8, kind_from_dev(dl_out), m->stream));
    return check_status(m);
}

extern "C" int sbp_get_blockmodel_dense(const sbp_model_t *m, int32_t *M_out) {
    if (!m || !M_out) return fail(SBP_EINVAL, "sbp_get_blockmodel_dense: NULL argument");
    if (!m->dense) return fail(SBP_ESTATE, "sbp_get_blockmodel_dense: model is not dense");
    SBP_CUDA(cudaMemcpyAsync(M_out, m->M, (size_t)m->B * m->B * 4, kind_from_dev(M_out), m->stream));
    return check_status(m);
}

extern "C" int sbp_get_blockmodel_coo(const sbp_model_t *m, int64_t capacity, int64_t *keys, int32_t *counts,
                                      int64_t *nnz) {
    if (!m || !nnz) return fail(SBP_EINVAL, "sbp_get_blockmodel_coo: NULL argument");
    SBP_TRY(check_status(m));
    const int64_t B = m->B;
    std::vector<int64_t> k;
    std::vector<int32_t> c;
    if (m->dense) {
        std::vector<int32_t> M((size_t)(B * B));
        SBP_CUDA(cudaMemcpy(M.data(), m->M, M.size() * 4, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < B * B; ++i)
            if (M[(size_t)i]) {
                k.push_back(i);
                c.push_back(M[(size_t)i]);
            }
    } else {
        const int64_t z = sparse_nnz(const_cast<sbp_model *>(m));
        std::vector<uint32_t> rp((size_t)B + 1);
        std::vector<int32_t> rc((size_t)z), rv((size_t)z);
        SBP_CUDA(cudaMemcpy(rp.data(), m->sp.rp, rp.size() * 4, cudaMemcpyDeviceToHost));
        if (z > 0) {
            SBP_CUDA(cudaMemcpy(rc.data(), m->sp.rc, (size_t)z * 4, cudaMemcpyDeviceToHost));
            SBP_CUDA(cudaMemcpy(rv.data(), m->sp.rv, (size_t)z * 4, cudaMemcpyDeviceToHost));
        }
        for (int64_t r = 0; r < B; ++r)
            for (uint32_t i = rp[(size_t)r]; i < rp[(size_t)r + 1]; ++i) {
                k.push_back(r * B + rc[i]);
                c.push_back(rv[i]);
            }
    }
    *nnz = (int64_t)k.size();
    if ((int64_t)k.size() > capacity) return fail(SBP_EINVAL, "sbp_get_blockmodel_coo: capacity too small");
    if (keys && !k.empty()) std::memcpy(keys, k.data(), k.size() * 8);
    if (counts && !c.empty()) std::memcpy(counts, c.data(), c.size() * 4);
    return SBP_OK;
}

extern "C" int sbp_get_degrees(const sbp_model_t *m, int32_t *dout, int32_t *din) {
    if (!m) return fail(SBP_EINVAL, "sbp_get_degrees: NULL model");
    if (dout) SBP_CUDA(cudaMemcpyAsync(dout, m->dout, (size_t)m->B * 4, kind_from_dev(dout), m->stream));
    if (din) SBP_CUDA(cudaMemcpyAsync(din, m->din, (size_t)m->B * 4, kind_from_dev(din), m->stream));
    return check_status(m);
}

// ---------------------------------------------------------------------------
// Philox known-answer check
namespace sbp {
namespace {
__global__ void k_philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0, uint64_t k1, int count,
                         uint64_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const U64x4 w = philox4x64_10(c0 + (uint64_t)i, c1, c2, c3, k0, k1);
    out[4 * i + 0] = w.x;
    out[4 * i + 1] = w.y;
    out[4 * i + 2] = w.z;
    out[4 * i + 3] = w.w;
}
}  // namespace
}  // namespace sbp

extern "C" int sbp_philox_check(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0, uint64_t k1,
                                int32_t count, uint64_t *out) {
    if (count < 1 || count > (1 << 20) || !out) return fail(SBP_EINVAL, "sbp_philox_check: bad count or NULL out");
    uint64_t *d = nullptr;
    SBP_CUDA(cudaMalloc(&d, (size_t)count * 32));
    k_philox<<<(count + 255) / 256, 256>>>(c0, c1, c2, c3, k0, k1, count, d);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(out, d, (size_t)count * 32, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "sbp_philox_check");
    return SBP_OK;
}

extern "C" int sbp_kernel_launches(uint64_t *out) {
    if (!out) return sbp::fail(SBP_EINVAL, "sbp_kernel_launches: NULL out");
    *out = sbp::g_launches.load(std::memory_order_relaxed);
    return SBP_OK;
}
