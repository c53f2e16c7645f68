// batch.h -- the batching form: many graphs partitioned together (host side).
#pragma once

#include <vector>

#include "common.cuh"
#include "driver.h"

namespace sbp {

// largest B the persistent kernel takes (per-warp counts of B entries in
// shared memory; a per-sweep pass over the B x B prefix rows; the merge
// rounds sort B scores in shared memory)
constexpr int kBatchMaxB = 1024;

struct BatchTuning {
    int ctas_per_sm = 2;     // persistent CTAs per SM
    int max_B = 512;         // phases merging to B above this run on the per-graph kernels
    int64_t max_n = 65536;   // and so do graphs with more vertices
    int dense_max_B = 1024;  // dense / sparse switch of the models in the batch
    int movers_per_warp = 1; // evaluation: 1 (32 lanes each), 2 (16) or 4 (8)
};

struct BatchOptions {
    int workers = 32;
    double mem_fraction = 0.5;
    BatchTuning tune;
};

// One graph for the persistent kernel: its search (rec) and label slots
// (4 n entries), both device-visible; phases may start from at most
// lim_from blocks (the model's dense arrays, the kernel's shared arrays)
// and merge to at most max_B (the kernel's count rows).  The kernel runs
// phases (start state, merges, sweeps, compaction, bracket update) until
// the search ends or its next phase is out of those bounds.
struct BatchSpec {
    sbp_model *m = nullptr;
    SearchRec *rec = nullptr;
    int32_t *slots = nullptr;
    int32_t lim_from = 0;
    int32_t started = 0;  // the record's started flag (the host's copy)
};

// the graph and model conditions of the persistent kernel (dense counts,
// no hybrid pass, int32 edge ids, rows below 65536 edges)
bool batch_graph_ok(const sbp_model *m, int64_t max_n);

// an MCMC phase at the model's current B
bool batch_eligible(const sbp_model *m, int max_B, int64_t max_n);

// the largest B a phase of this model may start from in the kernel (the
// model is dense there, as the per-graph path would hold it, and its
// arrays hold that many blocks)
int32_t batch_lim_from(const sbp_model *m);

// a whole planned phase from B_from blocks merged to target
bool batch_phase_eligible(const sbp_model *m, int32_t B_from, int32_t target, int max_B, int64_t max_n);

// Enqueues the searches of specs on stream st (models eligible and idle;
// every SearchRec filled by the host, the label slots of its bracket
// positions written).  When the stream reaches the end of the launch each
// model is in the state the per-graph kernels would leave and each record
// and its slots hold the search as the kernel left it.  The launch's
// scratch is freed in stream order.
int batch_enqueue(const std::vector<BatchSpec> &specs, const sbp_params &p, const BatchTuning &tune,
                  cudaStream_t st);

}  // namespace sbp
