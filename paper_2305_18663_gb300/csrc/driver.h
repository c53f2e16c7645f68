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

// A search state as the persistent kernel sees it: one bracket position
// and the label slot that holds its assignment (B = 0: empty position)
struct SearchState {
    int32_t B = 0;
    int32_t slot = 0;
    double dl = 0.0;
    uint64_t id = 0;
};

// One graph's golden-ratio search handed to the persistent kernel and back
// (device-visible, typically host-mapped): the bracket (positions 0 hi,
// 1 mid, 2 lo, as in Bracket), the run's counters, and what the kernel did.
// Four label slots of n entries each go with it.
struct SearchRec {
    SearchState s[3];
    uint64_t sweep_id = 0, round_id = 0, last_id = 0, holds = 0;
    int64_t total = 0;
    int32_t started = 0;  // in: the planned phase's merges ran already (its sweeps come next)
    int32_t B_model = 0;  // out: B of the state the model holds
    int32_t done = 0;     // out: the search ended
    int32_t phases = 0;   // out: phases run in the launch
    int32_t merged = 0;   // out: of them, with their merge phase
    int32_t starts = 0;   // out: of them, from a state the model no longer held
    int32_t ok = 0;       // out: 1 handed back; -1 a phase it took did not fit its bounds
    int32_t pad = 0;
};

// One partition run (reading of Section II-B and Alg. 2 in the design
// notes): merge phases towards the golden-ratio target, MCMC phases until
// |DL_{k-3} - DL_k| < t DL_k or max_sweeps, compaction, bracket update.
// Each phase is first planned (its start state and target from the
// bracket), then run here, on the per-graph kernels (start_phase, sweep,
// end_phase), or the search from that phase on is handed to the persistent
// kernel (export_search), which runs the same steps and the same bracket
// updates and hands it back (import_search).
struct PartitionRun {
    sbp_model *m = nullptr;
    uint64_t sweep_id = 0, round_id = 0;  // monotone counters of the run
    int64_t total = 0;                    // sweeps over all MCMC phases
    Bracket br;
    bool done = false;
    // the planned phase: from bracket state s[start], merged to B = target
    int start = 0;
    int32_t target = 0;
    // the current MCMC phase
    double t = 0.0;          // convergence threshold of the phase
    int k = 0;               // sweeps done in the phase
    std::vector<double> hist;  // hist[0]: DL after the merge; hist[k]: after sweep k
    uint64_t last_id = 0;      // ids given to states
    uint64_t model_holds = 0;  // the state the model currently holds (0: none)

    int begin(sbp_model *model);  // bracket seeded with the model's state; first phase planned
    int start_phase();            // the planned start: state uploaded unless held, merges, DL read
    int sweep();                  // one nodal sweep of the phase (per-graph kernels)
    bool phase_over() const;      // the phase's stopping rule after k sweeps
    int end_phase();              // compaction, bracket update, next phase planned (or done)
    // the search handed to the persistent kernel: the bracket into rec,
    // position p's labels into slot p of `slots` (4 n entries), the run's
    // counters; started: the planned phase's merges ran already
    void export_search(SearchRec &rec, int32_t *slots, bool started) const;
    // and back: the bracket and counters as the kernel left them (the model
    // holds the state rec names, at B_model), the next phase planned
    void import_search(const SearchRec &rec, const int32_t *slots);
    const State &start_state() const { return br.s[start]; }
    bool holds_start() const { return br.s[start].id == model_holds; }
    int finish(int32_t *b_out, int32_t *B_out, double *dl_out, int64_t *n_sweeps) const;

  private:
    void plan();  // the next phase from the bracket, or done
};

}  // namespace sbp
