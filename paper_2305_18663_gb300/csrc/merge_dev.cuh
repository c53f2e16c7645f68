// merge_dev.cuh -- device pieces of the block-merge proposals and their
// Delta DL (Alg. 1, Alg. 4), shared by the per-graph kernel (merge.cu) and
// the batched phase kernel (batch.cu), so that both score every proposal
// with the same arithmetic in the same order.
//
// One warp per block r; its lanes draw up to 32 proposals of r at once.  Proposal i
// (Philox counter (round_id, r, i), key (seed, 1)): u is the block at the
// far end of a uniformly chosen edge of block r (row r then column r of M);
// s != r is drawn with probability proportional to 1 + M[u][s] + M[s][u]
// (a uniform part over the other B-1 blocks, then row u and column u with
// block r left out).  A block with no edges draws s uniformly.
//
// Delta DL of merging r into s over rows and columns r, s only: row r moves
// into row s, column r into column s, the 2x2 corner collapses into M[s][s],
// and the block degrees of s absorb those of r.  Terms are written as
// f(a+b) - f(a) - f(b) = a log1p(b/a) + b log1p(a/b), f(x) = x ln x.  The
// model term of Eq. 2 is the same for every candidate and is left out.
// The best proposal is the smallest score on a 2^-20-nat grid, earliest i
// on a tie.
#pragma once

#include <cmath>

#include "common.cuh"

namespace sbp {
namespace {

// Proposal of block r on one lane (every search a single-lane one, so the
// lanes of a warp can draw different proposals of r at once).
__device__ __forceinline__ int merge_propose(const ModelDev &md, int r, uint64_t w0, uint64_t w1) {
    const int B = md.B;
    const int64_t dr = (int64_t)md.dout[r] + md.din[r];
    if (dr == 0) {
        const int64_t y = draw_below(w1, (uint64_t)(B - 1));
        return (int)(y + (y >= r));
    }
    const int64_t t0 = draw_below(w0, (uint64_t)dr);
    int u;
    if (md.sparse) {
        u = sparse_cdf_block(md, r, (uint32_t)t0, (uint32_t)md.dout[r]);
    } else {
        u = (int)pivot_upper(md.P + (size_t)r * 2 * B, md.Pc + (size_t)r * 32, 0, 2 * B, (uint32_t)t0);
        if (u >= B) u -= B;
    }
    const int64_t Mur = Mat(md, u, r), Mru = Mat(md, r, u);
    const int64_t du_out = md.dout[u], du = du_out + md.din[u];
    const int64_t W = (B - 1) + du - Mur - Mru;
    const int64_t y = draw_below(w1, (uint64_t)W);
    if (y < B - 1) return (int)(y + (y >= r));
    const int64_t t = y - (B - 1);
    const int64_t row_w = du_out - Mur;
    if (md.sparse) {
        // the same walks over the nonzeros of row u / column u, entry r left out
        if (t < row_w) {
            const uint32_t a = md.rp[u], z = md.rp[u + 1];
            const uint32_t pos = lane_lower_i32(md.rc, a, z, r);
            const int64_t pre = pos > a ? (int64_t)md.rpre[pos - 1] : 0;
            const int64_t tt = t >= pre ? t + Mur : t;
            return md.rc[lane_upper(md.rpre, a, z, (uint32_t)tt)];
        }
        const int64_t tc = t - row_w;
        const uint32_t a = md.cp[u], z = md.cp[u + 1];
        const uint32_t pos = lane_lower_i32(md.cr, a, z, r);
        const int64_t pre = pos > a ? (int64_t)md.cpre[pos - 1] : 0;
        const int64_t tt = tc >= pre ? tc + Mru : tc;
        return md.cr[lane_upper(md.cpre, a, z, (uint32_t)tt)];
    }
    const uint32_t *Pu = md.P + (size_t)u * 2 * B;
    if (t < row_w) {
        // row u with column r left out
        const int64_t pre = r > 0 ? (int64_t)Pu[r - 1] : 0;
        const int64_t tt = t >= pre ? t + Mur : t;
        return (int)lane_upper(Pu, 0, (uint32_t)B, (uint32_t)tt);
    }
    // column u with row r left out; Pu[B + c] = dout_u + column prefix
    const int64_t pre = r > 0 ? (int64_t)Pu[B + r - 1] : du_out;
    int64_t target = du_out + (t - row_w);
    if (target >= pre) target += Mru;
    return (int)lane_upper(Pu + B, 0, (uint32_t)B, (uint32_t)target);
}

// The terms of merging r into s that do not come from row or column r's
// other entries, on one lane: the 2x2 corner collapsing into M[s][s]
// (added) and the block degrees of s absorbing those of r (subtracted).
struct MergeCorner {
    double add, sub;
};

__device__ __forceinline__ MergeCorner merge_corner(const ModelDev &md, int r, int s) {
    const int64_t a = Mat(md, r, r), b = Mat(md, r, s), c = Mat(md, s, r), d = Mat(md, s, s);
    MergeCorner m;
    m.add = gmerge(a, b) + gmerge(a + b, c) + gmerge(a + b + c, d);
    m.sub = gmerge(md.dout[s], md.dout[r]) + gmerge(md.din[s], md.din[r]);
    return m;
}

// the entries of row r and column r other than r and s, merged into row and
// column s: the whole warp, one sum per lane then the warp total
__device__ __forceinline__ double merge_entries(const ModelDev &md, int r, int s) {
    const int B = md.B, lane = threadIdx.x & 31;
    double acc = 0.0;
    if (md.sparse) {
        for (uint32_t i = md.rp[r] + lane; i < md.rp[r + 1]; i += 32) {
            const int t = md.rc[i];
            if (t == r || t == s) continue;
            acc += gmerge(Mat(md, s, t), md.rv[i]);
        }
        for (uint32_t i = md.cp[r] + lane; i < md.cp[r + 1]; i += 32) {
            const int t = md.cr[i];
            if (t == r || t == s) continue;
            acc += gmerge(Mat(md, t, s), md.cv[i]);
        }
    } else {
        for (int t = lane; t < B; t += 32) {
            if (t == r || t == s) continue;
            const int Mrt = Mat(md, r, t);
            if (Mrt) acc += gmerge(Mat(md, s, t), Mrt);
            const int Mtr = Mat(md, t, r);
            if (Mtr) acc += gmerge(Mat(md, t, s), Mtr);
        }
    }
    return warp_sum(acc);
}

__device__ __forceinline__ long long score_key(double d) { return (long long)floor(d * 1048576.0 + 0.5); }

// One warp, block r: up to 32 proposals at a time, one per lane: each lane
// draws its proposal s_i and computes its corner and degree terms, so the
// proposals' dependent lookups and FP64 terms overlap; then the warp sums
// the row and column entries of each proposal in turn.  Delta DL of
// proposal i: -((entries + corner) - degrees); the best is the smallest
// score on the grid, the earliest i on a tie (bs = -1 when x = 0).
__device__ __forceinline__ void merge_best(const ModelDev &md, uint64_t seed, uint64_t round_id, int x, int r,
                                           int &bs_out, double &bd_out) {
    const int lane = threadIdx.x & 31;
    int bs = -1;
    double bd = 0.0;
    long long bk = 0;
    for (int i0 = 0; i0 < x; i0 += 32) {
        const int nq = x - i0 < 32 ? x - i0 : 32;
        int si = 0;
        MergeCorner ci{0.0, 0.0};
        if (lane < nq) {
            const U64x4 w = philox4x64_10(round_id, (uint64_t)r, (uint64_t)(i0 + lane), 0, seed, 1);
            si = merge_propose(md, r, w.x, w.y);
            ci = merge_corner(md, r, si);
        }
        for (int q = 0; q < nq; ++q) {
            const int s = __shfl_sync(0xffffffffu, si, q);
            double acc = merge_entries(md, r, s);
            acc += __shfl_sync(0xffffffffu, ci.add, q);
            acc -= __shfl_sync(0xffffffffu, ci.sub, q);
            const double d = -acc;
            const long long key = score_key(d);
            if (bs < 0 || key < bk) {
                bs = s;
                bd = d;
                bk = key;
            }
        }
    }
    bs_out = bs;
    bd_out = bd;
}

}  // namespace
}  // namespace sbp
