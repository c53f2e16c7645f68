// driver.h -- the golden-ratio search of one graph (Section II-B; Alg. 1
// merge phases, Alg. 2 MCMC phases) as a resumable state machine, so that a
// batch can advance many graphs together (host code).
#pragma once

#include <cmath>
#include <vector>

#include "common.cuh"

namespace sbp {

struct State {
    int32_t B = 0;
    double dl = 0;
    std::vector<int32_t> b;
    uint64_t id = 0;  // which state of the run this is (0: none)
};

struct Bracket {
    State s[3];  // 0 hi, 1 mid, 2 lo (B == 0: empty)
    void insert(State &&x) {
        if (s[1].B == 0) {
            s[1] = std::move(x);
            return;
        }
        if (x.dl < s[1].dl) {
            if (s[1].B > x.B) s[0] = std::move(s[1]);
            else s[2] = std::move(s[1]);
            s[1] = std::move(x);
        } else {
            if (x.B > s[1].B) s[0] = std::move(x);
            else s[2] = std::move(x);
        }
    }
    bool next(double reduction, int &start, int32_t &target) const {
        if (s[2].B == 0) {
            int64_t nm = (int64_t)std::floor((double)s[1].B * reduction);
            if (nm > s[1].B - 1) nm = s[1].B - 1;
            if (nm < 1) return false;
            start = 1;
            target = (int32_t)(s[1].B - nm);
            return true;
        }
        if (s[0].B - s[2].B <= 2) return false;
        const int32_t up = s[0].B - s[1].B, low = s[1].B - s[2].B;
        int32_t upper, lower;
        if (up >= low) { start = 0; upper = s[0].B; lower = s[1].B; }
        else { start = 1; upper = s[1].B; lower = s[2].B; }
        int32_t t = upper - (int32_t)std::llround(0.618 * (double)(upper - lower));
        if (t >= upper) t = upper - 1;
        if (t <= lower) t = lower + 1;
        target = t;
        return true;
    }
};

// One partition run (reading of Section II-B and Alg. 2 in the design
// notes): merge phases towards the golden-ratio target, MCMC phases until
// |DL_{k-3} - DL_k| < t DL_k or max_sweeps, compaction, bracket update.
struct PartitionRun {
    sbp_model *m = nullptr;
    uint64_t sweep_id = 0, round_id = 0;  // monotone counters of the run
    int64_t total = 0;                    // sweeps over all MCMC phases
    Bracket br;
    bool done = false;
    // the current MCMC phase
    double t = 0.0;          // convergence threshold of the phase
    int k = 0;               // sweeps done in the phase
    std::vector<double> hist;  // hist[0]: DL after the merge; hist[k]: after sweep k
    uint64_t last_id = 0;      // ids given to states
    uint64_t model_holds = 0;  // the state the model currently holds (0: none)

    int begin(sbp_model *model);  // bracket seeded with the model's state; first phase set up
    int sweep();                  // one nodal sweep of the phase (per-graph kernels)
    bool phase_over() const;      // the phase's stopping rule after k sweeps
    int after_sweeps(int k_done, double dl_last);  // a phase run elsewhere ended after k_done sweeps
    int end_phase();              // compaction, bracket update, next phase (or done)
    int finish(int32_t *b_out, int32_t *B_out, double *dl_out, int64_t *n_sweeps) const;

  private:
    int next_phase();  // merge towards the next target, or done
};

}  // namespace sbp
