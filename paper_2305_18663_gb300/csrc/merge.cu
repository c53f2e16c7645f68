// merge.cu -- block-merge proposals and merge Delta DL (Alg. 1, Alg. 4):
// one warp per block; the proposal, the Delta DL terms and the choice of the
// best proposal are in merge_dev.cuh.
#include "merge_dev.cuh"

namespace sbp {
namespace {

// One warp per block r (merge_best).
__global__ void __launch_bounds__(256) k_merge_proposals(ModelDev md, uint64_t seed, uint64_t round_id, int x,
                                                         int32_t *__restrict__ best_s, double *__restrict__ best_d) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < md.B; r += nw) {
        int bs;
        double bd;
        merge_best(md, seed, round_id, x, r, bs, bd);
        if (lane == 0) {
            best_s[r] = bs;
            best_d[r] = bd;
        }
    }
}

}  // namespace

int launch_merge_proposals(sbp_model *m, uint64_t round_id) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = ((int64_t)m->B * 32 + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    if (blocks < 1) blocks = 1;
    k_merge_proposals<<<(int)blocks, 256, 0, m->stream>>>(model_dev(m), m->p.seed, round_id, m->p.merge_proposals,
                                                          m->best_s, m->best_d);
    SBP_LAUNCHED();
    return SBP_OK;
}

}  // namespace sbp
