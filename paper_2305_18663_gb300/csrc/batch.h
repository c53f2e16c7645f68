// batch.h -- the batching form: many graphs partitioned together (host side).
#pragma once

#include <vector>

#include "common.cuh"

namespace sbp {

// largest B the persistent MCMC kernel takes (per-warp counts of B entries
// in shared memory; a per-sweep pass over the B x B prefix rows)
constexpr int kBatchMaxB = 1024;

struct BatchTuning {
    int ctas_per_sm = 2;     // persistent CTAs per SM
    int max_B = 512;         // phases at B above this run on the per-graph kernels
    int64_t max_n = 4096;    // and so do graphs with more vertices
    int dense_max_B = 4096;  // dense / sparse switch of the models in the batch
    int movers_per_warp = 1; // evaluation: 1 (32 lanes each), 2 (16) or 4 (8)
};

struct BatchOptions {
    int workers = 16;
    double mem_fraction = 0.5;
    BatchTuning tune;
};

bool batch_eligible(const sbp_model *m, int max_B, int64_t max_n);

int batch_enqueue(const std::vector<sbp_model *> &models, const std::vector<uint64_t> &sweep0,
                  const std::vector<double> &t, const std::vector<double> &hist0, const std::vector<int *> &k_res,
                  const std::vector<double *> &dl_res, const BatchTuning &tune, cudaStream_t st);

}  // namespace sbp
