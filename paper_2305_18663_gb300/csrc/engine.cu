// engine.cu -- the batch engine behind the batching and serving forms.
//
// Every graph runs its own golden-ratio search (PartitionRun, Section II-B;
// Alg. 1 merge phases, Alg. 2 MCMC phases), with the same result as
// sbp_partition.  Graphs can be submitted at any time.  Two kinds of work
// overlap on the device:
//   - per-graph work, driven by host worker threads: model set-up, and the
//     phases the persistent kernel does not take (merges from B above its
//     limit, big graphs, sparse rows), each with its merges, sweeps and
//     compaction on the per-graph kernels.  Workers take graphs from a
//     shared queue: first the short steps (a finished search's result, the
//     set-up of a graph whose search the persistent kernel will take), then
//     the largest (the server: the oldest); a graph's work goes to its
//     model's stream;
//   - persistent launches (batch.cu), driven by the launcher: a graph whose
//     next phase the kernel can run whole (start state, merges, sweeps,
//     compaction) hands it its search from that phase on, as does a graph
//     whose merges ran per graph and whose sweeps it can run.  The kernel
//     runs the search's phases and bracket updates until the search ends or
//     a phase is out of its bounds.  A launch starts when a GPU's worth of
//     searches is ready, when the workers have nothing else to do, or 2 ms
//     after the oldest ready search joined; up to 16 are in flight on their
//     own streams, with the searches in host-mapped memory.  A search that
//     ends is taken back as soon as its record says so (a launch can hold
//     searches of very different lengths); one whose next phase is out of
//     the kernel's bounds once its launch is over (its model's device state
//     is then complete for the per-graph kernels).  Either goes back to the
//     workers.
// Admission: graphs are admitted in submission order while their estimated
// device memory fits the budget (one is always admitted when none is
// running); a finished graph's model is freed at once, so the next request
// takes its place: continuous batching.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "batch.h"
#include "driver.h"

namespace sbp {
namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// device bytes of a graph's model at its largest: sparse rows at B = N, or
// the dense counts and prefix rows at the first dense B, min(N, dense_max_B)
size_t model_bytes(const sbp_graph *g, int dense_max_B) {
    const size_t n = (size_t)g->n, m = (size_t)std::max<int64_t>(g->m, 1);
    const size_t bd = std::min(n, (size_t)dense_max_B);
    return 152 * m + 128 * n + 12 * bd * bd + (1u << 20);
}

}  // namespace

struct Item {
    const sbp_graph *g = nullptr;
    int32_t *b_out = nullptr;
    sbp_model *m = nullptr;
    PartitionRun run;
    bool admitted = false, started = false, finished = false;
    // the persistent kernel it waits for: 1 to run the started phase's
    // sweeps and the search after it, 2 the search from the planned phase on
    int job = 0;
    bool bounced = false;  // the kernel gave the search back without a phase
    double t_ready = 0;    // when it last joined the persistent kernel's queue
    // host-mapped search record and its four label slots (4 n), and their
    // device view
    unsigned char *xfer = nullptr, *xfer_dev = nullptr;
    size_t xfer_bytes = 0;
    SearchRec *rec() const { return reinterpret_cast<SearchRec *>(xfer); }
    int32_t *slots() const { return reinterpret_cast<int32_t *>(xfer + kRecBytes); }
    static constexpr size_t kRecBytes = (sizeof(SearchRec) + 255) / 256 * 256;
    int rc = SBP_OK;
    std::string msg;
    size_t bytes = 0;
    sbp_batch_result res{};
};

struct Engine {
    sbp_params prm{};
    BatchOptions opt;
    int W = 1;
    size_t budget = 0, full_batch = 1;
    double t0 = 0;
    std::vector<cudaStream_t> streams;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::unique_ptr<Item>> items;
    size_t next_admit = 0;          // first graph not yet admitted
    std::vector<int64_t> cpu_q;     // graphs needing per-graph work
    std::vector<int64_t> ready;     // graphs whose search waits for a persistent launch
    int busy = 0;
    int64_t running = 0;            // admitted, not finished
    size_t used = 0;
    bool closing = false, aborting = false;
    int fatal = SBP_OK;             // an engine-level failure (streams, launches)
    std::string fatal_msg;
    sbp_batch_stats st{};
    std::atomic<int64_t> per_graph_phases{0};
    std::vector<std::thread> workers;
    std::thread launcher;
    // which queued graph a free worker takes: the largest (a batch call:
    // the longest runs start first, which shortens the whole call) or the
    // oldest request (the server: requests finish closer to arrival order,
    // which keeps the median latency down when the device is saturated)
    bool oldest_first = false;
    // host-mapped search records with their label slots, reused by size once
    // their graph is done
    std::mutex xfer_mu;
    std::multimap<size_t, unsigned char *> xfer_free;
    std::vector<unsigned char *> xfer_all;

    int init(const sbp_params &p, const BatchOptions &o, bool background);
    int64_t submit(const sbp_graph *g, int32_t *b_out);
    void close_and_join();
    int loop();  // the launcher

  private:
    void admit();  // under mu
    int work(Item &it, cudaStream_t s);
    void worker();
    bool whole_phase_ok(const Item &it) const;
    int ensure_xfer(Item &it);
    void release_xfer(Item &it);
};

// the planned phase can run whole in the persistent kernel
bool Engine::whole_phase_ok(const Item &it) const {
    if (it.run.done) return false;
    return batch_phase_eligible(it.m, it.run.start_state().B, it.run.target, opt.tune.max_B, opt.tune.max_n);
}

int Engine::ensure_xfer(Item &it) {
    const size_t need = Item::kRecBytes + (size_t)std::max<int64_t>(it.g->n, 1) * 16;
    if (it.xfer_bytes >= need) return SBP_OK;
    release_xfer(it);
    size_t cls = 4096;
    while (cls < need) cls <<= 1;
    unsigned char *h = nullptr;
    {
        std::lock_guard<std::mutex> lk(xfer_mu);
        auto f = xfer_free.find(cls);
        if (f != xfer_free.end()) {
            h = f->second;
            xfer_free.erase(f);
        }
    }
    if (!h) {
        if (cudaHostAlloc((void **)&h, cls, cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            return fail(SBP_ENOMEM, "batch engine: mapped host memory for a search");
        }
        std::lock_guard<std::mutex> lk(xfer_mu);
        xfer_all.push_back(h);
    }
    unsigned char *d = nullptr;
    SBP_CUDA(cudaHostGetDevicePointer((void **)&d, h, 0));
    it.xfer = h;
    it.xfer_dev = d;
    it.xfer_bytes = cls;
    return SBP_OK;
}

void Engine::release_xfer(Item &it) {
    if (!it.xfer) return;
    std::lock_guard<std::mutex> lk(xfer_mu);
    xfer_free.emplace(it.xfer_bytes, it.xfer);
    it.xfer = it.xfer_dev = nullptr;
    it.xfer_bytes = 0;
}

void Engine::admit() {
    while (next_admit < items.size()) {
        Item &it = *items[next_admit];
        it.bytes = model_bytes(it.g, prm.dense_max_B);
        if (running > 0 && used + it.bytes > budget) break;
        used += it.bytes;
        it.admitted = true;
        it.res.t_admit = now_s() - t0;
        ++running;
        cpu_q.push_back((int64_t)next_admit);
        ++next_admit;
    }
}

int Engine::init(const sbp_params &p, const BatchOptions &o, bool background) {
    prm = p;
    opt = o;
    oldest_first = background;  // the server
    prm.dense_max_B = opt.tune.dense_max_B;
    W = std::max(1, opt.workers);
    t0 = now_s();
    streams.assign((size_t)W, nullptr);
    for (auto &s : streams) SBP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    size_t free_b = 0, total_b = 0;
    SBP_CUDA(cudaMemGetInfo(&free_b, &total_b));
    budget = (size_t)((double)free_b * opt.mem_fraction);
    int dev = 0, sms = 1;
    SBP_CUDA(cudaGetDevice(&dev));
    SBP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    full_batch = (size_t)sms * (size_t)std::max(1, opt.tune.ctas_per_sm);
    for (int w = 0; w < W; ++w)
        workers.emplace_back([this, dev]() {
            cudaSetDevice(dev);
            worker();
        });
    if (background)
        launcher = std::thread([this, dev]() {
            cudaSetDevice(dev);
            loop();
        });
    return SBP_OK;
}

int64_t Engine::submit(const sbp_graph *g, int32_t *b_out) {
    auto it = std::make_unique<Item>();
    it->g = g;
    it->b_out = b_out;
    std::lock_guard<std::mutex> lk(mu);
    it->res.t_submit = now_s() - t0;
    items.push_back(std::move(it));
    admit();
    cv.notify_all();
    return (int64_t)items.size() - 1;
}

// one graph's per-graph work, until it waits for a batched phase or ends
int Engine::work(Item &it, cudaStream_t s) {
    int r = SBP_OK;
    double tm = now_s();
    if (!it.started) {
        std::vector<int32_t> ident((size_t)it.g->n);
        std::iota(ident.begin(), ident.end(), 0);
        r = sbp_build_blockmodel(it.g, (int32_t)it.g->n, ident.data(), &prm, s, &it.m);
        if (r == SBP_OK) r = it.run.begin(it.m);
        it.started = true;
    }
    double t_merge = now_s() - tm, t_sweeps = 0.0;
    while (r == SBP_OK && !it.run.done) {
        if (!it.bounced && whole_phase_ok(it)) {
            it.job = 2;
            break;
        }
        it.bounced = false;
        tm = now_s();
        r = it.run.start_phase();
        t_merge += now_s() - tm;
        if (r != SBP_OK) break;
        if (batch_eligible(it.m, opt.tune.max_B, opt.tune.max_n)) {
            it.job = 1;
            break;
        }
        tm = now_s();
        while (r == SBP_OK && !it.run.phase_over()) r = it.run.sweep();
        const double t1 = now_s();
        t_sweeps += t1 - tm;
        if (r == SBP_OK) r = it.run.end_phase();
        t_merge += now_s() - t1;
        per_graph_phases.fetch_add(1, std::memory_order_relaxed);
    }
    if (r == SBP_OK && it.job) r = ensure_xfer(it);
    if (r == SBP_OK && it.run.done) r = it.run.finish(it.b_out, &it.res.B, &it.res.dl, &it.res.n_sweeps);
    if (r != SBP_OK || it.run.done) {
        if (it.m) sbp_free_model(it.m);
        it.m = nullptr;
        release_xfer(it);
        it.job = 0;
        it.finished = true;
        it.res.t_done = now_s() - t0;
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        st.s_merge += t_merge;
        st.s_sweeps += t_sweeps;
    }
    return r;
}

void Engine::worker() {
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        cv.wait(lk, [&]() { return aborting || (closing && running == 0) || !cpu_q.empty(); });
        if (aborting || (cpu_q.empty() && closing && running == 0)) return;
        // first the short steps: graphs whose search has ended (their result
        // is out and their memory freed at once) and graphs not yet set up
        // whose searches the persistent kernel will take (the set-up hands
        // the device work that overlaps the rest); then by the engine's order
        auto rank = [&](int64_t i) {
            const Item &c = *items[(size_t)i];
            return (c.started && c.run.done) || (!c.started && c.g->n <= opt.tune.max_n) ? 0 : 1;
        };
        size_t pick = 0;
        for (size_t q = 1; q < cpu_q.size(); ++q) {
            const int64_t a = cpu_q[q], b = cpu_q[pick];
            const int ra = rank(a), rb = rank(b);
            if (ra != rb) {
                if (ra < rb) pick = q;
                continue;
            }
            if (oldest_first ? a < b : items[(size_t)a]->g->m > items[(size_t)b]->g->m) pick = q;
        }
        const int64_t idx = cpu_q[pick];
        cpu_q.erase(cpu_q.begin() + (long)pick);
        Item &it = *items[(size_t)idx];
        ++busy;
        lk.unlock();
        const double ts = now_s();
        const int r = work(it, streams[(size_t)idx % streams.size()]);
        std::string msg;
        if (r != SBP_OK) {
            char buf[1024];
            sbp_last_error(buf, sizeof buf);
            msg = buf;
        }
        lk.lock();
        st.s_per_graph += now_s() - ts;
        --busy;
        if (it.finished) {
            it.rc = r;
            it.msg = msg;
            --running;
            used -= it.bytes;
            admit();
        } else {
            it.t_ready = now_s();
            ready.push_back(idx);
        }
        cv.notify_all();
    }
}

int Engine::loop() {
    struct Launch {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        std::vector<int64_t> take;  // its graphs not yet taken back
        double t0 = 0;
    };
    // launches in flight at once: a launch runs its graphs' searches to the
    // end (or to a phase it cannot take), so it stays in flight as long as
    // its longest search
    const int kMaxInflight = 16;
    const double kMaxWait = 0.002;
    std::vector<Launch> pool((size_t)kMaxInflight);
    std::vector<int> free_slots, inflight;
    int rc = SBP_OK;
    auto engine_fail = [&](int code, const std::string &msg) {
        std::lock_guard<std::mutex> lk(mu);
        if (fatal == SBP_OK) {
            fatal = code;
            fatal_msg = msg;
        }
        aborting = true;
        cv.notify_all();
    };
    for (int q = 0; q < kMaxInflight; ++q) {
        free_slots.push_back(q);
        if (cudaStreamCreateWithFlags(&pool[(size_t)q].st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&pool[(size_t)q].ev, cudaEventDisableTiming) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "batch engine: stream or event");
            engine_fail(rc, "batch engine: stream or event creation failed");
        }
    }
    std::vector<Item *> ended;
    {
        std::unique_lock<std::mutex> lk(mu);
        while (rc == SBP_OK) {
            // a launch is due when a GPU's worth of searches is ready, when
            // the workers have nothing else to do, or when the oldest ready
            // search has waited kMaxWait: searches start soon after they
            // become batchable without a launch per search
            auto due = [&]() {
                if (ready.empty() || free_slots.empty()) return false;
                if (ready.size() >= full_batch || (cpu_q.empty() && busy < W)) return true;
                return now_s() - items[(size_t)ready.front()]->t_ready >= kMaxWait;
            };
            cv.wait_for(lk, std::chrono::microseconds(500),
                        [&]() { return aborting || (closing && running == 0) || due(); });
            for (size_t q = 0; q < inflight.size();) {
                Launch &L = pool[(size_t)inflight[q]];
                const cudaError_t e = cudaEventQuery(L.ev);
                if (e != cudaSuccess && e != cudaErrorNotReady) {
                    rc = cuda_fail(e, "persistent launch");
                    lk.unlock();
                    engine_fail(rc, std::string("batched search: ") + cudaGetErrorString(e));
                    lk.lock();
                    break;
                }
                const bool over = e == cudaSuccess;
                // searches taken back: while the launch runs, the ended ones
                // (their outcome is all in host-mapped memory, and their
                // model is only freed after), once it is over, the rest
                std::vector<int64_t> back, keep;
                for (int64_t idx : L.take) {
                    Item &it = *items[(size_t)idx];
                    const int32_t ok = __atomic_load_n(&it.rec()->ok, __ATOMIC_ACQUIRE);
                    if (over || (ok == 1 && it.rec()->done)) back.push_back(idx);
                    else keep.push_back(idx);
                }
                L.take.swap(keep);
                if (over) {
                    st.s_batched += now_s() - L.t0;
                    free_slots.push_back(inflight[q]);
                    inflight.erase(inflight.begin() + (long)q);
                } else {
                    ++q;
                }
                if (back.empty()) continue;
                // each search is taken back (the bracket's labels copied out of
                // the mapped slots) and plans its next phase, outside the
                // lock: these graphs are the launcher's until queued again
                ended.clear();
                for (int64_t idx : back) ended.push_back(items[(size_t)idx].get());
                lk.unlock();
                bool bad = false;
                int64_t ph = 0, mg = 0, sts = 0;
                for (Item *ip : ended) {
                    Item &it = *ip;
                    const SearchRec rec = *it.rec();
                    if (rec.ok != 1) {
                        bad = true;
                        break;
                    }
                    it.run.import_search(rec, it.slots());
                    it.bounced = rec.phases == 0;
                    it.job = 0;
                    ph += rec.phases;
                    mg += rec.merged;
                    sts += rec.starts;
                }
                if (bad) {
                    rc = SBP_ESTATE;
                    engine_fail(rc, "batched search: a phase did not fit the launch's bounds");
                    lk.lock();
                    break;
                }
                lk.lock();
                st.phases_batched += ph;
                st.merges_batched += mg;
                st.starts_batched += sts;
                for (int64_t idx : back) cpu_q.push_back(idx);
                cv.notify_all();
            }
            if (aborting || rc != SBP_OK) break;
            if (closing && running == 0 && inflight.empty()) break;
            if (!due()) continue;
            const int slot = free_slots.back();
            free_slots.pop_back();
            Launch &L = pool[(size_t)slot];
            L.take.swap(ready);
            ready.clear();
            inflight.push_back(slot);
            ended.clear();
            for (int64_t idx : L.take) ended.push_back(items[(size_t)idx].get());
            lk.unlock();
            // each graph's search goes to its mapped record and label slots
            std::vector<BatchSpec> specs(L.take.size());
            for (size_t u = 0; u < L.take.size(); ++u) {
                Item &it = *ended[u];
                it.run.export_search(*it.rec(), it.slots(), it.job == 1);
                BatchSpec &sp = specs[u];
                sp.m = it.m;
                sp.rec = reinterpret_cast<SearchRec *>(it.xfer_dev);
                sp.slots = reinterpret_cast<int32_t *>(it.xfer_dev + Item::kRecBytes);
                sp.lim_from = batch_lim_from(it.m);
                sp.started = it.job == 1 ? 1 : 0;
            }
            L.t0 = now_s();
            int r = batch_enqueue(specs, prm, opt.tune, L.st);
            if (r == SBP_OK && cudaEventRecord(L.ev, L.st) != cudaSuccess) r = cuda_fail(cudaGetLastError(), "cudaEventRecord");
            std::string msg;
            if (r != SBP_OK) {
                char buf[1024];
                sbp_last_error(buf, sizeof buf);
                msg = std::string("batched phase: ") + buf;
            }
            lk.lock();
            ++st.rounds;
            if (r != SBP_OK) {
                rc = r;
                lk.unlock();
                engine_fail(r, msg);
                lk.lock();
                break;
            }
        }
    }
    for (int q : inflight) cudaEventSynchronize(pool[(size_t)q].ev);
    for (Launch &L : pool) {
        if (L.ev) cudaEventDestroy(L.ev);
        if (L.st) cudaStreamDestroy(L.st);
    }
    return rc;
}

void Engine::close_and_join() {
    {
        std::lock_guard<std::mutex> lk(mu);
        closing = true;
        cv.notify_all();
    }
    if (launcher.joinable()) launcher.join();
    {
        std::lock_guard<std::mutex> lk(mu);
        if (fatal != SBP_OK) aborting = true;
        cv.notify_all();
    }
    for (auto &t : workers)
        if (t.joinable()) t.join();
    workers.clear();
    for (auto &p : items) {
        if (p->m) {
            sbp_free_model(p->m);
            p->m = nullptr;
        }
        release_xfer(*p);
    }
    for (unsigned char *h : xfer_all) cudaFreeHost(h);
    xfer_all.clear();
    xfer_free.clear();
    for (auto &s : streams)
        if (s) cudaStreamDestroy(s);
    streams.clear();
    st.phases_per_graph = per_graph_phases.load();
}

// the C ABI's option checks and conversion
int batch_options(const sbp_batch_options *o, BatchOptions &opt) {
    sbp_batch_options bo;
    if (o) bo = *o;
    else sbp_default_batch_options(&bo);
    if (bo.workers < 1 || bo.workers > 256) return fail(SBP_EINVAL, "batch options: workers must be in [1, 256]");
    if (bo.max_B < 1 || bo.max_B > kBatchMaxB)
        return fail(SBP_EINVAL, "batch options: max_B must be in [1, " + std::to_string(kBatchMaxB) + "]");
    if (bo.dense_max_B < bo.max_B || bo.dense_max_B > 16384)
        return fail(SBP_EINVAL, "batch options: dense_max_B must be in [max_B, 16384]");
    if (bo.ctas_per_sm < 1 || bo.ctas_per_sm > 8) return fail(SBP_EINVAL, "batch options: ctas_per_sm must be in [1, 8]");
    if (bo.max_n < 0) return fail(SBP_EINVAL, "batch options: max_n must be >= 0");
    if (bo.movers_per_warp != 1 && bo.movers_per_warp != 2 && bo.movers_per_warp != 4)
        return fail(SBP_EINVAL, "batch options: movers_per_warp must be 1, 2 or 4");
    if (!(bo.mem_fraction > 0.0 && bo.mem_fraction <= 0.95))
        return fail(SBP_EINVAL, "batch options: mem_fraction must be in (0, 0.95]");
    opt.workers = bo.workers;
    opt.mem_fraction = bo.mem_fraction;
    opt.tune.max_B = bo.max_B;
    opt.tune.dense_max_B = bo.dense_max_B;
    opt.tune.ctas_per_sm = bo.ctas_per_sm;
    opt.tune.max_n = bo.max_n;
    opt.tune.movers_per_warp = bo.movers_per_warp;
    return SBP_OK;
}

}  // namespace sbp

using sbp::Engine;
using sbp::fail;

extern "C" int sbp_partition_batch(const sbp_graph_t *const *graphs, int32_t count, const sbp_params *p,
                                   const sbp_batch_options *o, int32_t *const *b_out, sbp_batch_result *res,
                                   sbp_batch_stats *stats) {
    if (count < 0 || (count > 0 && (!graphs || !res))) return fail(SBP_EINVAL, "sbp_partition_batch: NULL argument");
    for (int i = 0; i < count; ++i)
        if (!graphs[i]) return fail(SBP_EINVAL, "sbp_partition_batch: NULL graph " + std::to_string(i));
    sbp_params prm;
    if (p) prm = *p;
    else sbp_default_params(&prm);
    SBP_TRY(sbp::params_valid(prm));
    sbp::BatchOptions opt;
    SBP_TRY(sbp::batch_options(o, opt));
    Engine e;
    SBP_TRY(e.init(prm, opt, false));
    for (int i = 0; i < count; ++i) e.submit(graphs[i], b_out ? b_out[i] : nullptr);
    {
        std::lock_guard<std::mutex> lk(e.mu);
        e.closing = true;
    }
    const int rc = e.loop();
    e.close_and_join();
    if (e.fatal != SBP_OK) return fail(e.fatal, e.fatal_msg);
    if (rc != SBP_OK) return rc;
    for (int i = 0; i < count; ++i) {
        const sbp::Item &it = *e.items[(size_t)i];
        if (it.rc != SBP_OK) return fail(it.rc, "graph " + std::to_string(i) + ": " + it.msg);
        res[i] = it.res;
    }
    if (stats) *stats = e.st;
    return SBP_OK;
}

// ---------------------------------------------------------------------------
// autotuner of the batching form: coordinate search over the options, each
// candidate timed on the same sample of graphs, every result checked equal

extern "C" int sbp_autotune_batch(const sbp_graph_t *const *graphs, int32_t count, const sbp_params *p,
                                  int32_t sample, int32_t start, sbp_batch_options *best, double *graphs_per_s,
                                  int32_t *trials) {
    if (!graphs || !best || count < 1) return fail(SBP_EINVAL, "sbp_autotune_batch: needs graphs and best");
    for (int i = 0; i < count; ++i)
        if (!graphs[i]) return fail(SBP_EINVAL, "sbp_autotune_batch: NULL graph " + std::to_string(i));
    // the sample: evenly spaced in size order, so that it spans the sizes
    std::vector<int> idx((size_t)count);
    for (int i = 0; i < count; ++i) idx[(size_t)i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        return graphs[x]->n + graphs[x]->m < graphs[y]->n + graphs[y]->m;
    });
    const int ns = (sample <= 0 || sample >= count) ? count : sample;
    std::vector<const sbp_graph_t *> pick((size_t)ns);
    for (int i = 0; i < ns; ++i) pick[(size_t)i] = graphs[idx[(size_t)((int64_t)i * count / ns)]];

    sbp_batch_options cur;
    if (start) cur = *best;
    else sbp_default_batch_options(&cur);
    sbp::BatchOptions chk;
    SBP_TRY(sbp::batch_options(&cur, chk));
    std::vector<sbp_batch_result> res((size_t)ns), ref((size_t)ns);
    bool have_ref = false;
    int ntr = 0;
    auto run = [&](const sbp_batch_options &o, double *rate) -> int {
        const auto t0 = std::chrono::steady_clock::now();
        SBP_TRY(sbp_partition_batch(pick.data(), ns, p, &o, nullptr, res.data(), nullptr));
        const double s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        ++ntr;
        if (!have_ref) {
            ref = res;
            have_ref = true;
        } else {
            for (int i = 0; i < ns; ++i)
                if (res[(size_t)i].B != ref[(size_t)i].B || res[(size_t)i].dl != ref[(size_t)i].dl ||
                    res[(size_t)i].n_sweeps != ref[(size_t)i].n_sweeps)
                    return fail(SBP_ESTATE, "sbp_autotune_batch: results differ between options");
        }
        *rate = ns / std::max(s, 1e-9);
        return SBP_OK;
    };
    double best_rate = 0.0;
    SBP_TRY(run(cur, &best_rate));  // warm-up: one-time set-up costs
    SBP_TRY(run(cur, &best_rate));
    struct Knob {
        int32_t sbp_batch_options::*field;
        std::vector<int32_t> values;
    };
    const Knob knobs[] = {
        {&sbp_batch_options::movers_per_warp, {1, 2, 4}},
        {&sbp_batch_options::ctas_per_sm, {1, 2, 3, 4}},
        {&sbp_batch_options::max_B, {128, 256, 512, 1024}},
        {&sbp_batch_options::max_n, {1024, 4096, 16384, 65536}},
        {&sbp_batch_options::dense_max_B, {1024, 4096}},
    };
    for (const Knob &kb : knobs) {
        for (int32_t v : kb.values) {
            if (cur.*kb.field == v) continue;
            sbp_batch_options trial = cur;
            trial.*kb.field = v;
            if (trial.dense_max_B < trial.max_B) continue;
            double rate = 0.0;
            SBP_TRY(run(trial, &rate));
            if (rate > best_rate * 1.02) {  // a clear gain only: runs are noisy
                cur = trial;
                best_rate = rate;
            }
        }
    }
    *best = cur;
    if (graphs_per_s) *graphs_per_s = best_rate;
    if (trials) *trials = ntr;
    return SBP_OK;
}

// ---------------------------------------------------------------------------
// serving: the same engine, fed while it runs

struct sbp_server {
    Engine e;
};

extern "C" int sbp_server_create(const sbp_params *p, const sbp_batch_options *o, sbp_server_t **out) {
    if (!out) return fail(SBP_EINVAL, "sbp_server_create: out is NULL");
    *out = nullptr;
    sbp_params prm;
    if (p) prm = *p;
    else sbp_default_params(&prm);
    SBP_TRY(sbp::params_valid(prm));
    sbp::BatchOptions opt;
    SBP_TRY(sbp::batch_options(o, opt));
    auto *s = new sbp_server();
    const int rc = s->e.init(prm, opt, true);
    if (rc != SBP_OK) {
        s->e.close_and_join();
        delete s;
        return rc;
    }
    *out = s;
    return SBP_OK;
}

extern "C" int sbp_server_submit(sbp_server_t *s, const sbp_graph_t *g, int32_t *b_out, int64_t *request) {
    if (!s || !g || !request) return fail(SBP_EINVAL, "sbp_server_submit: NULL argument");
    {
        std::lock_guard<std::mutex> lk(s->e.mu);
        if (s->e.fatal != SBP_OK) return fail(s->e.fatal, s->e.fatal_msg);
        if (s->e.closing) return fail(SBP_ESTATE, "sbp_server_submit: server is shutting down");
    }
    *request = s->e.submit(g, b_out);
    return SBP_OK;
}

extern "C" int sbp_server_poll(sbp_server_t *s, int64_t request, int32_t *done) {
    if (!s || !done) return fail(SBP_EINVAL, "sbp_server_poll: NULL argument");
    std::lock_guard<std::mutex> lk(s->e.mu);
    if (request < 0 || request >= (int64_t)s->e.items.size()) return fail(SBP_EINVAL, "sbp_server_poll: unknown request");
    *done = s->e.items[(size_t)request]->finished ? 1 : 0;
    return SBP_OK;
}

extern "C" int sbp_server_wait(sbp_server_t *s, int64_t request, sbp_batch_result *res) {
    if (!s) return fail(SBP_EINVAL, "sbp_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(s->e.mu);
    if (request < 0 || request >= (int64_t)s->e.items.size()) return fail(SBP_EINVAL, "sbp_server_wait: unknown request");
    sbp::Item &it = *s->e.items[(size_t)request];
    s->e.cv.wait(lk, [&]() { return it.finished || s->e.aborting; });
    if (!it.finished) return fail(s->e.fatal != SBP_OK ? s->e.fatal : SBP_ESTATE, "sbp_server_wait: " + s->e.fatal_msg);
    if (it.rc != SBP_OK) return fail(it.rc, "request " + std::to_string(request) + ": " + it.msg);
    if (res) *res = it.res;
    return SBP_OK;
}

extern "C" int sbp_server_stats(sbp_server_t *s, sbp_batch_stats *stats) {
    if (!s || !stats) return fail(SBP_EINVAL, "sbp_server_stats: NULL argument");
    std::lock_guard<std::mutex> lk(s->e.mu);
    *stats = s->e.st;
    stats->phases_per_graph = s->e.per_graph_phases.load();
    return SBP_OK;
}

extern "C" void sbp_server_destroy(sbp_server_t *s) {
    if (!s) return;
    s->e.close_and_join();
    delete s;
}
