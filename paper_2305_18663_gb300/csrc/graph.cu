// graph.cu -- graph upload: directed COO -> CSR of out-edges and of in-edges.
//
// The graph is the fixed input "Graph G" of Alg. 1-2.  Rows are sorted by
// neighbour id (the order the nodal proposal indexes into), duplicates and
// self-loops are kept.  Vertices are also grouped by total degree so the
// nodal pass can give small, medium and large rows different work units;
// the grouping changes no result (every decision reads frozen state only).
#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void build_rows(int64_t n, int64_t m, const int32_t *from, const int32_t *to, std::vector<int32_t> &ptr,
                std::vector<int32_t> &col) {
    ptr.assign((size_t)n + 1, 0);
    for (int64_t e = 0; e < m; ++e) ptr[(size_t)from[e] + 1]++;
    for (int64_t v = 0; v < n; ++v) ptr[(size_t)v + 1] += ptr[(size_t)v];
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    col.resize((size_t)std::max<int64_t>(m, 1));
    for (int64_t e = 0; e < m; ++e) col[(size_t)fill[(size_t)from[e]]++] = to[e];
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) {
        th.emplace_back([&, t]() {
            for (int64_t v = t; v < n; v += nt) std::sort(col.begin() + ptr[(size_t)v], col.begin() + ptr[(size_t)v + 1]);
        });
    }
    for (auto &x : th) x.join();
}

template <class T>
int upload(T **dst, const T *src, size_t count) {
    if (count == 0) count = 1;
    if (cudaMalloc((void **)dst, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return sbp::fail(SBP_ENOMEM, "cudaMalloc failed while loading the graph");
    }
    SBP_CUDA(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
    return SBP_OK;
}

}  // namespace

extern "C" int sbp_load_graph(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, sbp_graph_t **out) {
    if (!out) return sbp::fail(SBP_EINVAL, "sbp_load_graph: out is NULL");
    *out = nullptr;
    if (n < 1 || n > INT32_MAX - 1) return sbp::fail(SBP_EINVAL, "sbp_load_graph: n must be in [1, 2^31-2]");
    if (m < 0 || m >= (int64_t(1) << 30)) return sbp::fail(SBP_EINVAL, "sbp_load_graph: m must be in [0, 2^30)");
    if (m > 0 && (!src || !dst)) return sbp::fail(SBP_EINVAL, "sbp_load_graph: src/dst is NULL");

    std::vector<int32_t> hs, hd;
    const int32_t *s = src, *d = dst;
    if (m > 0 && is_device_ptr(src)) {
        hs.resize((size_t)m);
        SBP_CUDA(cudaMemcpy(hs.data(), src, (size_t)m * 4, cudaMemcpyDeviceToHost));
        s = hs.data();
    }
    if (m > 0 && is_device_ptr(dst)) {
        hd.resize((size_t)m);
        SBP_CUDA(cudaMemcpy(hd.data(), dst, (size_t)m * 4, cudaMemcpyDeviceToHost));
        d = hd.data();
    }
    for (int64_t e = 0; e < m; ++e)
        if (s[e] < 0 || s[e] >= n || d[e] < 0 || d[e] >= n)
            return sbp::fail(SBP_EINVAL, "sbp_load_graph: vertex id out of range at edge " + std::to_string(e));

    std::vector<int32_t> op, oc, ip, ic;
    build_rows(n, m, s, d, op, oc);
    build_rows(n, m, d, s, ip, ic);
    std::vector<int32_t> esrc((size_t)std::max<int64_t>(m, 1));
    for (int64_t v = 0; v < n; ++v)
        for (int32_t e = op[(size_t)v]; e < op[(size_t)v + 1]; ++e) esrc[(size_t)e] = (int32_t)v;
    // twins: out-rows visited by ascending source meet every in-row's
    // entries (ascending source, duplicates adjacent) in their order, so a
    // cursor per in-row pairs the k-th copy of an edge with its k-th copy
    std::vector<int32_t> tw_oi((size_t)std::max<int64_t>(m, 1)), tw_io((size_t)std::max<int64_t>(m, 1));
    std::vector<int32_t> self_in;
    {
        std::vector<int32_t> cur(ip.begin(), ip.end() - 1);
        for (int64_t e = 0; e < m; ++e) {
            const int32_t j = cur[(size_t)oc[(size_t)e]]++;
            tw_oi[(size_t)e] = j;
            tw_io[(size_t)j] = (int32_t)e;
            if (oc[(size_t)e] == esrc[(size_t)e]) self_in.push_back(j);
        }
    }

    // degree groups: k = 0 | 1..32 | 33..128 | > 128, each in id order
    std::vector<int32_t> order((size_t)n);
    int64_t cnt[4] = {0, 0, 0, 0};
    int32_t maxk = 0;
    auto group = [&](int64_t v) {
        int32_t k = (op[(size_t)v + 1] - op[(size_t)v]) + (ip[(size_t)v + 1] - ip[(size_t)v]);
        maxk = std::max(maxk, k);
        return k == 0 ? 0 : k <= sbp::kSmallDeg ? 1 : k <= sbp::kWarpDeg ? 2 : 3;
    };
    for (int64_t v = 0; v < n; ++v) cnt[group(v)]++;
    auto *g = new sbp_graph();
    g->bin[0] = 0;
    for (int i = 0; i < 4; ++i) g->bin[i + 1] = g->bin[i] + cnt[i];
    int64_t pos[4] = {g->bin[0], g->bin[1], g->bin[2], g->bin[3]};
    for (int64_t v = 0; v < n; ++v) order[(size_t)pos[group(v)]++] = (int32_t)v;
    // the largest rows first inside the top group, for load balance
    auto deg = [&](int32_t v) { return (op[(size_t)v + 1] - op[(size_t)v]) + (ip[(size_t)v + 1] - ip[(size_t)v]); };
    std::stable_sort(order.begin() + g->bin[3], order.end(), [&](int32_t x, int32_t y) { return deg(x) > deg(y); });

    // every vertex by degree, descending, ties by id (the hybrid pass's order)
    std::vector<int32_t> by_degree((size_t)n);
    for (int64_t v = 0; v < n; ++v) by_degree[(size_t)v] = (int32_t)v;
    std::stable_sort(by_degree.begin(), by_degree.end(), [&](int32_t x, int32_t y) { return deg(x) > deg(y); });

    g->n = n;
    g->m = m;
    g->max_deg = maxk;
    cudaGetDevice(&g->device);
    int rc = SBP_OK;
    if (rc == SBP_OK) rc = upload(&g->op, op.data(), op.size());
    if (rc == SBP_OK) rc = upload(&g->ip, ip.data(), ip.size());
    if (rc == SBP_OK) rc = upload(&g->oc, oc.data(), (size_t)m);
    if (rc == SBP_OK) rc = upload(&g->ic, ic.data(), (size_t)m);
    if (rc == SBP_OK) rc = upload(&g->esrc, esrc.data(), (size_t)m);
    if (rc == SBP_OK) rc = upload(&g->tw_oi, tw_oi.data(), (size_t)m);
    if (rc == SBP_OK) rc = upload(&g->tw_io, tw_io.data(), (size_t)m);
    g->n_self = (int64_t)self_in.size();
    if (self_in.empty()) self_in.push_back(-1);  // the upload keeps one element at least
    if (rc == SBP_OK) rc = upload(&g->self_in, self_in.data(), self_in.size());
    if (rc == SBP_OK) rc = upload(&g->order, order.data(), (size_t)n);
    if (rc == SBP_OK) rc = upload(&g->by_degree, by_degree.data(), (size_t)n);
    if (rc != SBP_OK) {
        sbp_free_graph(g);
        return rc;
    }
    *out = g;
    return SBP_OK;
}

extern "C" int sbp_graph_info(const sbp_graph_t *g, int64_t *n, int64_t *m) {
    if (!g) return sbp::fail(SBP_EINVAL, "sbp_graph_info: NULL graph");
    if (n) *n = g->n;
    if (m) *m = g->m;
    return SBP_OK;
}

extern "C" void sbp_free_graph(sbp_graph_t *g) {
    if (!g) return;
    cudaFree(g->op);
    cudaFree(g->ip);
    cudaFree(g->oc);
    cudaFree(g->ic);
    cudaFree(g->esrc);
    cudaFree(g->tw_oi);
    cudaFree(g->tw_io);
    cudaFree(g->self_in);
    cudaFree(g->order);
    cudaFree(g->by_degree);
    delete g;
}
