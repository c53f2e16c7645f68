// nodal_dev.cuh -- device helpers of the nodal decision pass, shared by the
// per-graph kernels (nodal.cu) and the batched MCMC kernel (batch.cu).
//
// For every vertex v (block r) against the frozen (b, M):
//   1. proposal (Alg. 2 "propose new community"): a uniformly chosen
//      incident edge (out-list then in-list) gives the neighbour block u;
//      s is drawn with probability (1 + M[u][s] + M[s][u]) / (d_u + B) by an
//      integer inverse CDF over the prefix array P[u];
//   2. neighbour-block counts kout[t], kin[t] (Section III-A (c): the sparse
//      vector of changes) aggregated with warp match/ballot and, for longer
//      rows, shared-memory tables;
//   3. Delta DL over the changed entries of rows r,s and columns r,s only
//      (Section II-C), block degrees included (Eq. 1-2).  Every term is
//      f(x+k) - f(x) with f(x) = x ln x at integer counts: in FP32 with a
//      rigorous error bound (the precision form), or summed exactly in
//      128-bit fixed point from a table (FP64 for counts beyond the table);
//   4. Hastings-corrected Metropolis test (Alg. 2): logA = -beta dDL +
//      ln(p_bwd / p_fwd), accept iff ln(u) < logA.  The Hastings sums and
//      the logarithms are first evaluated in FP32 with a rigorous error
//      bound; when ln(u) falls inside that band (or a trace is requested)
//      the sums and the test are redone exactly, so every decision equals
//      the FP64 one.
// GB300 executes one FP64 warp instruction per ~20 SM cycles, so the FP64
// work is kept off the common path and spread across lanes when it runs.
#pragma once

#include <cmath>

#include "common.cuh"

namespace sbp {
namespace {


// A proposal with s != b[v] that still needs its Delta DL and test.
struct Mover {
    int v, s;
    unsigned long long w2;  // the Philox word of the acceptance draw
};

struct DecideArgs {
    GraphDev g;
    ModelDev md;
    int64_t v_begin, v_end;
    Mover *movers;           // four lists: k <= 32, 33..128, > 128, and the movers
                             // the FP32 test left to the exact evaluation
    unsigned *mcount;        // their lengths (device counters)
    int64_t mbase[4];        // their offsets in movers
    int force_exact;         // 1: decide every mover by the exact evaluation
    uint64_t seed, sweep_id;
    double beta;
    float beta32;
    int trace_on;
    sbp_vertex_trace tr;
    const uint8_t *skip;     // NULL, or vertices this pass leaves alone (the hybrid pass's sequential part)
    // the vertices of the three degree groups (k <= 32, 33..128, > 128), for
    // the kernels that draw the proposals themselves
    const int32_t *vlist[3];
    int64_t vcount[3];
};

// position of the k-th (0-based) set bit of m, for k < popc(m)
__device__ __forceinline__ int nth_set_bit(unsigned m, int k) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const unsigned lo = m & ((1u << w) - 1u);
        const int c = __popc(lo);
        if (k >= c) {
            k -= c;
            m >>= w;
            pos += w;
        } else {
            m = lo;
        }
    }
    return pos;
}

// per-thread counts (32-bit: every sum over a pass is at most 2E < 2^32,
// since the CSR offsets are 32-bit); widened when flushed
struct Counts {
    unsigned proposed = 0, moves = 0, accepted = 0, margin = 0, acc_edges = 0, recheck = 0, entries = 0;
};

// a mover the FP32 test could not settle (or any mover when a trace is
// asked for), for the exact evaluation that follows the pass
__device__ __forceinline__ void push_recheck(const DecideArgs &a, int v, int s, uint64_t w2) {
    const unsigned i = atomicAdd(&a.mcount[3], 1u);
    Mover m;
    m.v = v;
    m.s = s;
    m.w2 = w2;
    a.movers[a.mbase[3] + i] = m;
}


__device__ __forceinline__ void write_trace(const DecideArgs &a, int v, int s, int flags, double dH, double logA) {
    if (a.tr.s) a.tr.s[v] = s;
    if (a.tr.flags) a.tr.flags[v] = flags;
    if (a.tr.dH) a.tr.dH[v] = dH;
    if (a.tr.logA) a.tr.logA[v] = logA;
}


// Per-vertex scalars shared by the evaluation steps.
struct VertexCtx {
    int v, r, s;
    int Kout, Kin, self;  // out / in degree of v (self-loops included), self-loops
    int ko_r, ki_r, ko_s, ki_s;
    int k;  // total degree, an upper bound on the number of entries
};

// one neighbour block t not in {r, s}: exact Delta L terms, FP32 Hastings terms
__device__ __forceinline__ void entry_fast(const ModelDev &md, const VertexCtx &x, int t, int ko, int ki, __int128 &dl,
                                           double &fb, float &pf, float &pb) {
    int Mrt, Mst, Mtr, Mts;
    Mat4(md, x.r, x.s, t, Mrt, Mst, Mtr, Mts);
    // a zero count gives T[x] - T[x] = 0, so no branch is needed
    dl += dT(md.T, md.XT, Mrt, -ko, fb) + dT(md.T, md.XT, Mst, ko, fb);
    dl += dT(md.T, md.XT, Mtr, -ki, fb) + dT(md.T, md.XT, Mts, ki, fb);
    const float rc = md.rcp32[t];
    const float c = (float)(ko + ki);
    pf += c * (float)(Mts + Mst + 1) * rc;
    pb += c * (float)((Mtr - ki) + (Mrt - ko) + 1) * rc;
}

// the same Hastings terms in FP64 (the expression the FP64 test uses)
__device__ __forceinline__ void entry_exact(const ModelDev &md, const VertexCtx &x, int t, int ko, int ki, double &pf,
                                            double &pb) {
    int Mrt, Mst, Mtr, Mts;
    Mat4(md, x.r, x.s, t, Mrt, Mst, Mtr, Mts);
    const double den = (double)((int64_t)md.dsum[t] + md.B);
    const double c = (double)(ko + ki);
    pf += c * (double)((int64_t)Mts + Mst + 1) / den;
    pb += c * (double)(((int64_t)Mtr - ki) + ((int64_t)Mrt - ko) + 1) / den;
}

// ---------------------------------------------------------------------------
// FP32 Delta L (the precision form).  f(x+k) - f(x), f(x) = x ln x, for
// integer counts x >= 0 and x + k >= 0, written
//   k ln(x+k) + x ln(1 + k/x)          when x + k >= x/2 (k/x >= -1/2),
//   (x+k) ln(x+k) - x ln x             otherwise (no cancellation left).
// Logarithms come from the hardware approximation __logf, whose documented
// error is at most 2^-21.41 absolute on [1/2, 2] and 3 ulp elsewhere; the
// divisions from __fdividef (2 ulp).  ln(1 + z) for |z| <= 1/2 is the series
// 2 atanh(w) = 2 (w + w^3/3 + ... + w^15/15), w = z / (2 + z), |w| <= 1/3,
// whose truncation is below 2e-9 relative; beyond that it is __logf(1 + z)
// with 1 + z >= 3/2.  With the conversions of counts above 2^24, the products
// and the final sum, each result is within kTermErr * 2^-24 of the sum of the
// magnitudes of its two parts, which is added to am; ln 1 is taken as 0
// exactly.  Summed over the terms of a move in FP32 with at most d additions
// between any term and the total, the error of Delta L stays below
// 2^-24 (kTermErr + d) sum(am), and kDl32Depth + k/32 bounds d in every
// kernel (entries per lane or per chunk, the warp tree, the eight corner and
// degree terms, the final additions).  A known-answer hook
// (sbp_dxlogx32_check) lets the tests check the bound against FP64.
constexpr float kTermErr = 28.0f;
constexpr float kDl32Depth = 26.0f;

__device__ __forceinline__ float log1p_atanh(float z) {
    const float w = __fdividef(z, 2.0f + z);
    const float w2 = w * w;
    float p = 1.0f / 15.0f;
    p = fmaf(p, w2, 1.0f / 13.0f);
    p = fmaf(p, w2, 1.0f / 11.0f);
    p = fmaf(p, w2, 1.0f / 9.0f);
    p = fmaf(p, w2, 1.0f / 7.0f);
    p = fmaf(p, w2, 1.0f / 5.0f);
    p = fmaf(p, w2, 1.0f / 3.0f);
    p = fmaf(p, w2, 1.0f);
    return 2.0f * w * p;
}

// ln y for an integer count y >= 1 (exactly 0 at 1)
__device__ __forceinline__ float ln_count(int y) { return y > 1 ? __logf((float)y) : 0.0f; }

// Both forms, and both evaluations of ln(1 + z), are computed and the one
// that applies is selected: no branches, so that the independent terms of a
// move interleave and lanes with different counts do not diverge.
__device__ __forceinline__ float dxlogx32(int x, int k, float &am) {
    const int y = x + k;
    const float xf = (float)x, yf = (float)y, kf = (float)k;
    const float ly = ln_count(y > 0 ? y : 1), lx = ln_count(x > 0 ? x : 1);
    const float fy = yf * ly, fx = xf * lx;  // (x+k) ln(x+k) - x ln x
    const float z = __fdividef(kf, x > 0 ? xf : 1.0f);
    const bool series = fabsf(z) <= 0.5f;
    const float la = log1p_atanh(series ? z : 0.0f), lb = __logf(1.0f + fmaxf(z, -0.5f));
    const float t1 = kf * ly, t2 = xf * (series ? la : lb);  // k ln(x+k) + x ln(1 + k/x)
    const bool direct = x == 0 || 2 * y < x;
    const float val = direct ? fy - fx : t1 + t2;
    const float mag = direct ? fabsf(fy) + fabsf(fx) : fabsf(t1) + fabsf(t2);
    am += k != 0 ? mag : 0.0f;
    return k != 0 ? val : 0.0f;
}

// bound on |Delta L (FP32) - Delta L| for a move of a degree-k vertex
__device__ __forceinline__ float dl32_error(float am, int k) {
    return 0x1p-24f * (kTermErr + kDl32Depth + (float)k * (1.0f / 32.0f)) * am * 1.01f + 1e-30f;
}

// entry_fast with the FP32 Delta L terms
__device__ __forceinline__ void entry_fast32(const ModelDev &md, const VertexCtx &x, int t, int ko, int ki, float &dl,
                                             float &am, float &pf, float &pb) {
    int Mrt, Mst, Mtr, Mts;
    Mat4(md, x.r, x.s, t, Mrt, Mst, Mtr, Mts);
    dl += dxlogx32(Mrt, -ko, am) + dxlogx32(Mst, ko, am);
    dl += dxlogx32(Mtr, -ki, am) + dxlogx32(Mts, ki, am);
    const float rc = md.rcp32[t];
    const float c = (float)(ko + ki);
    pf += c * (float)(Mts + Mst + 1) * rc;
    pb += c * (float)((Mtr - ki) + (Mrt - ko) + 1) * rc;
}

// the exact Delta L terms and the FP64 Hastings terms of one entry (the
// recheck of the precision form)
__device__ __forceinline__ void entry_exact_all(const ModelDev &md, const VertexCtx &x, int t, int ko, int ki,
                                                __int128 &dl, double &fb, double &pf, double &pb) {
    int Mrt, Mst, Mtr, Mts;
    Mat4(md, x.r, x.s, t, Mrt, Mst, Mtr, Mts);
    dl += dT(md.T, md.XT, Mrt, -ko, fb) + dT(md.T, md.XT, Mst, ko, fb);
    dl += dT(md.T, md.XT, Mtr, -ki, fb) + dT(md.T, md.XT, Mts, ki, fb);
    const double den = (double)((int64_t)md.dsum[t] + md.B);
    const double c = (double)(ko + ki);
    pf += c * (double)((int64_t)Mts + Mst + 1) / den;
    pb += c * (double)(((int64_t)Mtr - ki) + ((int64_t)Mrt - ko) + 1) / den;
}

// Delta L terms of the 2x2 corner (j = 0..3: (r,r) (s,s) (r,s) (s,r)) and of
// the block degrees (j = 4..7: dout_r dout_s din_r din_s, subtracted), one
// per lane, selected without divergence.  Returns the count it read (lanes
// 0..3 read the four corner entries of M).
__device__ __forceinline__ int special_terms(const ModelDev &md, const VertexCtx &x, int j, __int128 &dl, double &fb) {
    if (j >= 8) return 0;
    const int r = x.r, s = x.s, B = md.B;
    const int cr = x.ko_r + x.ki_r, cs = x.ko_s + x.ki_s;
    const int rowi = (j == 0 || j == 2) ? r : s;
    const int coli = (j == 0 || j == 3) ? r : s;
    const int blk = (j == 4 || j == 6) ? r : s;
    (void)B;
    const int kk = j == 0   ? -(cr + x.self)
                   : j == 1 ? cs + x.self
                   : j == 2 ? x.ki_r - x.ko_s
                   : j == 3 ? x.ko_r - x.ki_s
                   : j == 4 ? -x.Kout
                   : j == 5 ? x.Kout
                   : j == 6 ? -x.Kin
                            : x.Kin;
    // the corner entries through the blockmodel accessor (dense or sparse)
    const int val = j < 4 ? Mat(md, rowi, coli) : (j < 6 ? md.dout[blk] : md.din[blk]);
    double f2 = 0.0;
    const __int128 d = dT(md.T, md.XT, val, kk, f2);
    dl += j < 4 ? d : -d;
    fb += j < 4 ? f2 : -f2;
    return val;
}

// special_terms with the FP32 Delta L terms
__device__ __forceinline__ int special_terms32(const ModelDev &md, const VertexCtx &x, int j, float &dl, float &am) {
    if (j >= 8) return 0;
    const int r = x.r, s = x.s;
    const int cr = x.ko_r + x.ki_r, cs = x.ko_s + x.ki_s;
    const int rowi = (j == 0 || j == 2) ? r : s;
    const int coli = (j == 0 || j == 3) ? r : s;
    const int blk = (j == 4 || j == 6) ? r : s;
    const int kk = j == 0   ? -(cr + x.self)
                   : j == 1 ? cs + x.self
                   : j == 2 ? x.ki_r - x.ko_s
                   : j == 3 ? x.ko_r - x.ki_s
                   : j == 4 ? -x.Kout
                   : j == 5 ? x.Kout
                   : j == 6 ? -x.Kin
                            : x.Kin;
    const int val = j < 4 ? Mat(md, rowi, coli) : (j < 6 ? md.dout[blk] : md.din[blk]);
    const float d = dxlogx32(val, kk, am);
    dl += j < 4 ? d : -d;
    return val;
}


// Hastings terms of v's neighbours in r and in s (forward and backward),
// from the corner entries and the block degrees; FP32 and FP64 versions.
struct CornerVals {
    int Mrr, Mss, Mrs, Msr, dr, ds;
};

// the four corner entries M[r][r], M[s][s], M[r][s], M[s][r]; on sparse rows
// the two row offsets and then the four first probe slots are loaded
// together (collisions continue one slot at a time)
__device__ __forceinline__ void Mat4corner(const ModelDev &md, int r, int s, int &Mrr, int &Mss, int &Mrs, int &Msr) {
    if (!md.sparse) {
        const size_t B = (size_t)md.B;
        Mrr = md.M[(size_t)r * B + r];
        Mss = md.M[(size_t)s * B + s];
        Mrs = md.M[(size_t)r * B + s];
        Msr = md.M[(size_t)s * B + r];
        return;
    }
    const uint32_t o_r = md.hoff[r], c_r = md.hoff[r + 1] - o_r;
    const uint32_t o_s = md.hoff[s], c_s = md.hoff[s + 1] - o_s;
    const uint32_t hr = sparse_hash(r), hs = sparse_hash(s);
    const uint32_t h1 = hr & (c_r - 1), h2 = hs & (c_s - 1), h3 = hs & (c_r - 1), h4 = hr & (c_s - 1);
    const int2 k1 = md.hkv[o_r + h1], k2 = md.hkv[o_s + h2], k3 = md.hkv[o_r + h3], k4 = md.hkv[o_s + h4];
    Mrr = sparse_probe_from(md, o_r, c_r, h1, r, k1);
    Mss = sparse_probe_from(md, o_s, c_s, h2, s, k2);
    Mrs = sparse_probe_from(md, o_r, c_r, h3, s, k3);
    Msr = sparse_probe_from(md, o_s, c_s, h4, r, k4);
}

// the eight corner and degree terms of one move on one lane (the lane per
// mover of the batch kernels), all loads issued together and the terms
// summed as a tree: returns the corner entries, adds to dl and am
__device__ __forceinline__ CornerVals special_terms32_lane(const ModelDev &md, const VertexCtx &x, float &dl, float &am) {
    const int r = x.r, s = x.s;
    const int cr = x.ko_r + x.ki_r, cs = x.ko_s + x.ki_s;
    CornerVals cv;
    Mat4corner(md, r, s, cv.Mrr, cv.Mss, cv.Mrs, cv.Msr);
    const int dor = md.dout[r], dos = md.dout[s], dir = md.din[r], dis = md.din[s];
    cv.dr = md.dsum[r];
    cv.ds = md.dsum[s];
    const float c0 = dxlogx32(cv.Mrr, -(cr + x.self), am), c1 = dxlogx32(cv.Mss, cs + x.self, am);
    const float c2 = dxlogx32(cv.Mrs, x.ki_r - x.ko_s, am), c3 = dxlogx32(cv.Msr, x.ko_r - x.ki_s, am);
    const float d0 = dxlogx32(dor, -x.Kout, am), d1 = dxlogx32(dos, x.Kout, am);
    const float d2 = dxlogx32(dir, -x.Kin, am), d3 = dxlogx32(dis, x.Kin, am);
    dl += ((c0 + c1) + (c2 + c3)) - ((d0 + d1) + (d2 + d3));
    return cv;
}

__device__ __forceinline__ void corner_hastings_fast(const VertexCtx &x, const CornerVals &c, int B, float &pf,
                                                     float &pb) {
    const int cr = x.ko_r + x.ki_r, cs = x.ko_s + x.ki_s, K = x.Kout + x.Kin;
    pf += (float)(cr + 2 * x.self) * (float)(c.Mrs + c.Msr + 1) / (float)(c.dr + B);
    pf += (float)cs * (float)(2 * c.Mss + 1) / (float)(c.ds + B);
    pb += (float)cr * (float)(2 * (c.Mrr - cr - x.self) + 1) / (float)(c.dr - K + B);
    pb += (float)(cs + 2 * x.self) * (float)((c.Msr + x.ko_r - x.ki_s) + (c.Mrs + x.ki_r - x.ko_s) + 1) /
          (float)(c.ds + K + B);
}

__device__ __forceinline__ void corner_hastings_exact(const VertexCtx &x, const CornerVals &c, int B, double &pf,
                                                      double &pb) {
    const int64_t cr = x.ko_r + x.ki_r, cs = x.ko_s + x.ki_s, K = x.Kout + x.Kin, self = x.self;
    pf += (double)(cr + 2 * self) * (double)((int64_t)c.Mrs + c.Msr + 1) / (double)((int64_t)c.dr + B);
    pf += (double)cs * (double)(2 * (int64_t)c.Mss + 1) / (double)((int64_t)c.ds + B);
    pb += (double)cr * (double)(2 * ((int64_t)c.Mrr - cr - self) + 1) / (double)((int64_t)c.dr - K + B);
    pb += (double)(cs + 2 * self) *
          (double)(((int64_t)c.Msr + x.ko_r - x.ki_s) + ((int64_t)c.Mrs + x.ki_r - x.ko_s) + 1) /
          (double)((int64_t)c.ds + K + B);
}

// FP32 decision with its error band.  Returns 1 accept, 0 reject, -1 when
// the band does not settle it (FP64 needed).
__device__ __forceinline__ int fast_decision_f(float b32, float dl32, float fb32, float pf, float pb, uint64_t w2,
                                               int k, float eps_dl = 0.0f) {
    const uint64_t um = w2 >> 11;
    if (um == 0) return 1;  // u = 0: ln u = -inf
    const float lnpf = logf(pf), lnpb = logf(pb);
    const float logA = b32 * (dl32 + fb32) + (lnpb - lnpf);
    const float u32 = fmaf((float)(unsigned)(um >> 21), 0x1p-32f, (float)(unsigned)(um & 0x1fffffu) * 0x1p-53f);
    const float lnu = logf(u32);
    const float diff = logA - lnu;
    const float e = b32 * (eps_dl + 3.0f * 0x1p-24f * (fabsf(dl32) + fabsf(fb32) + 1.0f)) + 2.0f * (float)(k + 9) * 0x1p-24f +
                    0x1p-23f * (fabsf(lnpf) + fabsf(lnpb) + 2.0f * fabsf(lnu) + fabsf(logA) + 1.0f);
    const float band = 4.0f * e + 1e-6f;
    if (!(fabsf(diff) > band)) return -1;  // also catches NaN / inf
    return diff > 0.0f ? 1 : 0;
}

__device__ __forceinline__ int fast_decision(float b32, __int128 dl, bool has_fb, double fb, float pf, float pb,
                                             uint64_t w2, int k) {
    return fast_decision_f(b32, fix_to_float(dl), has_fb ? (float)fb : 0.0f, pf, pb, w2, k);
}

struct Exact {
    double dH, logA;
    bool accept, margin;
};

// the FP64 test: logA = -beta dDL + ln p_bwd - ln p_fwd, accept iff ln u < logA
__device__ __noinline__ Exact exact_decision_d(double beta, double dL, double pf, double pb, uint64_t w2) {
    Exact e;
    e.dH = -dL;
    e.logA = -beta * e.dH + log(pb) - log(pf);
    const double lnu = log((double)(w2 >> 11) * 0x1p-53);
    e.accept = lnu < e.logA;
    e.margin = fabs(lnu - e.logA) <= 1e-9 * fmax(fabs(e.logA), 1.0);
    return e;
}

__device__ __forceinline__ Exact exact_decision(double beta, __int128 dl, double fb, double pf, double pb, uint64_t w2) {
    return exact_decision_d(beta, fix_to_double(dl) + fb, pf, pb, w2);
}

__device__ __forceinline__ unsigned hash_slot(int key, int cap_log2) {
    return ((unsigned)key * 0x9E3779B1u) >> (32 - cap_log2);
}

// insert (key, inc) into an open-addressing table; false when full
__device__ __forceinline__ bool table_add(int *keys, unsigned long long *cnt, int *list, int *nlist, int cap,
                                          int cap_log2, int key, unsigned long long inc) {
    unsigned h = hash_slot(key, cap_log2);
    for (int p = 0; p < cap; ++p) {
        const int prev = atomicCAS(&keys[h], -1, key);
        if (prev == -1) {
            list[atomicAdd(nlist, 1)] = (int)h;
            atomicAdd(&cnt[h], inc);
            return true;
        }
        if (prev == key) {
            atomicAdd(&cnt[h], inc);
            return true;
        }
        h = (h + 1) & (unsigned)(cap - 1);
    }
    return false;
}

// the same with 32-bit counts (ko | ki << 16) and 16-bit list entries
__device__ __forceinline__ bool table_add32(int *keys, unsigned *cnt, unsigned short *list, int *nlist, int cap,
                                            int cap_log2, int key, unsigned inc) {
    unsigned h = hash_slot(key, cap_log2);
    for (int p = 0; p < cap; ++p) {
        const int prev = atomicCAS(&keys[h], -1, key);
        if (prev == -1) {
            list[atomicAdd(nlist, 1)] = (unsigned short)h;
            atomicAdd(&cnt[h], inc);
            return true;
        }
        if (prev == key) {
            atomicAdd(&cnt[h], inc);
            return true;
        }
        h = (h + 1) & (unsigned)(cap - 1);
    }
    return false;
}

// an accepted move v -> s of a vertex with k edges: the pending label and
// its items in the accepted-move list
__device__ __forceinline__ void accept_move(const ModelDev &md, int v, int s, int k) {
    md.bnew[v] = s;
    if (md.items) {
        const int nch = (k + kMoveChunk - 1) / kMoveChunk;
        const unsigned long long base = atomicAdd(&md.counters->items, (unsigned long long)nch);
        for (int c = 0; c < nch; ++c)
            if (base + c < (unsigned long long)md.cap_items) md.items[base + c] = make_int2(v, c);
    }
}

__device__ __forceinline__ void count_result(Counts &c, bool accept, bool margin, int k) {
    c.proposed++;
    c.moves++;
    c.accepted += accept;
    c.margin += margin;
    c.acc_edges += accept ? (unsigned)k : 0u;
}

// a move decided by the exact evaluation
__device__ __forceinline__ void count_exact(Counts &c, bool accept, bool margin, int k) {
    count_result(c, accept, margin, k);
    c.recheck++;
}

// ---------------------------------------------------------------------------
// proposals: one lane per vertex, all vertices of the range

__device__ __forceinline__ void flush_counts(const ModelDev &md, const Counts &c) {
    typedef unsigned long long u64;
    if (c.proposed | c.moves) {
        atomicAdd(&md.counters->proposed, (u64)c.proposed);
        atomicAdd(&md.counters->moves, (u64)c.moves);
        atomicAdd(&md.counters->accepted, (u64)c.accepted);
        atomicAdd(&md.counters->margin, (u64)c.margin);
        if (c.acc_edges) atomicAdd(&md.counters->acc_edges, (u64)c.acc_edges);
        if (c.recheck) atomicAdd(&md.counters->recheck, (u64)c.recheck);
        if (c.entries) atomicAdd(&md.counters->entries, (u64)c.entries);
    }
}

__device__ __forceinline__ void flush_counts_warp(const ModelDev &md, Counts c, unsigned long long extra_edges) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c.proposed += __shfl_xor_sync(0xffffffffu, c.proposed, o);
        c.moves += __shfl_xor_sync(0xffffffffu, c.moves, o);
        c.accepted += __shfl_xor_sync(0xffffffffu, c.accepted, o);
        c.margin += __shfl_xor_sync(0xffffffffu, c.margin, o);
        c.acc_edges += __shfl_xor_sync(0xffffffffu, c.acc_edges, o);
        c.recheck += __shfl_xor_sync(0xffffffffu, c.recheck, o);
        c.entries += __shfl_xor_sync(0xffffffffu, c.entries, o);
        extra_edges += __shfl_xor_sync(0xffffffffu, extra_edges, o);
    }
    if ((threadIdx.x & 31) == 0) {
        flush_counts(md, c);
        if (extra_edges) atomicAdd(&md.counters->move_edges, extra_edges);
    }
}

// first index i in Pu[0, len) with Pu[i] > t, searched by one lane: the 32
// pivots with vector loads, then the segment eight entries at a time
// (plain loads: the batched MCMC kernel rewrites P between its sweeps)
__device__ __forceinline__ int lane_cdf_search(const uint32_t *Pu, const uint32_t *Pcu, int len,
                                               int step, uint32_t t) {
    int lo = 0, seg = len;
    if (len > 32) {
        uint4 pv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) pv[i] = reinterpret_cast<const uint4 *>(Pcu)[i];
        int fp = 31;
#pragma unroll
        for (int i = 7; i >= 0; --i) {
            if (pv[i].w > t) fp = 4 * i + 3;
            if (pv[i].z > t) fp = 4 * i + 2;
            if (pv[i].y > t) fp = 4 * i + 1;
            if (pv[i].x > t) fp = 4 * i;
        }
        lo = fp * step;
        seg = step < len - lo ? step : len - lo;
    }
    if (seg <= 32) {
        for (int g0 = 0; g0 < seg; g0 += 8) {
            uint32_t x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = g0 + i < seg ? Pu[lo + g0 + i] : 0xffffffffu;
            int idx = -1;
#pragma unroll
            for (int i = 7; i >= 0; --i)
                if (x[i] > t) idx = i;
            if (idx >= 0) return lo + g0 + idx;
        }
        return lo + seg - 1;
    }
    int n = seg;
    while (n > 0) {
        const int half = n >> 1;
        if (Pu[lo + half] <= t) {
            lo += half + 1;
            n -= half + 1;
        } else {
            n = half;
        }
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Proposal of vertex v (Alg. 2 "propose new community"): the j-th incident
// edge (out-list then in-list) gives the neighbour block u; s is drawn with
// probability (1 + M[u][s] + M[s][u]) / (d_u + B) by the integer inverse CDF
// over row u, then column u.  k = 0: no proposal (s = r).  w2 is the Philox
// word of the acceptance draw.
struct Proposal {
    int r, s, k;
    uint64_t w2;
};

__device__ __forceinline__ Proposal propose_vertex(const GraphDev &g, const ModelDev &md, uint64_t seed,
                                                   uint64_t sweep_id, int v) {
    Proposal p;
    const int B = md.B;
    p.r = md.b[v];
    p.s = p.r;
    p.w2 = 0;
    const int o0 = g.op[v], kout = g.op[v + 1] - o0;
    const int i0 = g.ip[v], kin = g.ip[v + 1] - i0;
    p.k = kout + kin;
    if (p.k == 0) return p;
    const U64x4 w = philox4x64_10(sweep_id, (uint64_t)v, 0, 0, seed, 0);
    const int j = (int)draw_below(w.x, (uint64_t)p.k);
    bool self_nb;
    const int u = nb_block(md, nb_raw(g, md, o0, i0, kout, j), v, self_nb);
    const int64_t du = md.dsum[u];
    const int64_t y = draw_below(w.y, (uint64_t)(du + B));
    if (y < B) {
        p.s = (int)y;
    } else if (md.sparse) {
        p.s = sparse_cdf_block(md, u, (uint32_t)(y - B), (uint32_t)md.dout[u]);
    } else {
        const int idx = lane_cdf_search(md.P + (size_t)u * 2 * B, md.Pc + (size_t)u * 32, 2 * B, md.pstep,
                                        (uint32_t)(y - B));
        p.s = idx < B ? idx : idx - B;
    }
    p.w2 = w.z;
    return p;
}

// ---------------------------------------------------------------------------
// moves of vertices with 33 <= k (one warp per vertex)

// Evaluates the move v: r -> s once the entries are aggregated, on an
// aligned group of G lanes (G = 32: the whole warp; 8 or 16: several movers
// per warp).  each_entry(f) calls f(t, ko, ki) for each entry the calling
// lane holds.  All G lanes call this; the result is written by the group's
// first lane.  A move the FP32 test cannot settle is decided here by the
// exact evaluation (INLINE_EXACT) or handed to the recheck list.
template <bool DL32, int G, bool INLINE_EXACT, class EachEntry>
__device__ __forceinline__ void evaluate_group(const DecideArgs &a, const ModelDev &md, VertexCtx &x, uint64_t w2,
                                               EachEntry each_entry, Counts &c) {
    static_assert(G == 8 || G == 16 || G == 32, "group of 8, 16 or 32 lanes");
    const unsigned gm = group_mask<G>();
    const int gl = (threadIdx.x & 31) & (G - 1);
    const int gbase = (threadIdx.x & 31) & ~(G - 1);
    // neighbours in r and in s (one lane holds each); 16-bit fields when
    // the degree allows it
    if (x.k < 65536) {
        int pr = 0, ps = 0;
        each_entry([&](int t, int ko, int ki) {
            if (t == x.r) pr += ko | (ki << 16);
            else if (t == x.s) ps += ko | (ki << 16);
        });
        pr = group_sum<G>(pr, gm);
        ps = group_sum<G>(ps, gm);
        x.ko_r = pr & 0xffff;
        x.ki_r = pr >> 16;
        x.ko_s = ps & 0xffff;
        x.ki_s = ps >> 16;
    } else {
        int a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        each_entry([&](int t, int ko, int ki) {
            if (t == x.r) { a0 += ko; a1 += ki; }
            else if (t == x.s) { a2 += ko; a3 += ki; }
        });
        x.ko_r = group_sum<G>(a0, gm);
        x.ki_r = group_sum<G>(a1, gm);
        x.ko_s = group_sum<G>(a2, gm);
        x.ki_s = group_sum<G>(a3, gm);
    }

    __int128 dl = 0;
    double fb = 0.0;
    float pf = 0.0f, pb = 0.0f;
    float dlf = 0.0f, am = 0.0f;
    int val;
    if (DL32) {
        each_entry([&](int t, int ko, int ki) {
            if (t != x.r && t != x.s) entry_fast32(md, x, t, ko, ki, dlf, am, pf, pb);
        });
        val = special_terms32(md, x, gl, dlf, am);
    } else {
        each_entry([&](int t, int ko, int ki) {
            if (t != x.r && t != x.s) entry_fast(md, x, t, ko, ki, dl, fb, pf, pb);
        });
        val = special_terms(md, x, gl, dl, fb);
    }
    CornerVals cv;
    cv.Mrr = __shfl_sync(gm, val, gbase + 0);
    cv.Mss = __shfl_sync(gm, val, gbase + 1);
    cv.Mrs = __shfl_sync(gm, val, gbase + 2);
    cv.Msr = __shfl_sync(gm, val, gbase + 3);
    cv.dr = md.dsum[x.r];
    cv.ds = md.dsum[x.s];
    pf = group_sum<G>(pf, gm);
    pb = group_sum<G>(pb, gm);
    corner_hastings_fast(x, cv, md.B, pf, pb);
    int dec = -1;
    bool has_fb = false;
    if (DL32) {
        dlf = group_sum<G>(dlf, gm);
        am = group_sum<G>(am, gm);
        // at most k / G entries per lane before the group tree
        if (!a.trace_on && !a.force_exact)
            dec = fast_decision_f(a.beta32, dlf, 0.0f, pf, pb, w2, x.k, dl32_error(am, x.k * (32 / G)));
    } else {
        dl = group_sum_128<G>(dl, gm);
        has_fb = __any_sync(gm, __double_as_longlong(fb) != 0);
        if (has_fb) fb = group_sum<G>(fb, gm);
        if (!a.trace_on && !a.force_exact) dec = fast_decision(a.beta32, dl, has_fb, fb, pf, pb, w2, x.k);
    }
    if (dec >= 0) {
        if (gl == 0) {
            if (dec) accept_move(md, x.v, x.s, x.k);
            count_result(c, dec != 0, false, x.k);
        }
        return;
    }
    if constexpr (!INLINE_EXACT) {
        if (gl == 0) push_recheck(a, x.v, x.s, w2);
        return;
    }
    double pf64 = 0.0, pb64 = 0.0;
    if (DL32) {
        // the exact Delta L as well
        dl = 0;
        fb = 0.0;
        each_entry([&](int t, int ko, int ki) {
            if (t != x.r && t != x.s) entry_exact_all(md, x, t, ko, ki, dl, fb, pf64, pb64);
        });
        special_terms(md, x, gl, dl, fb);
        dl = group_sum_128<G>(dl, gm);
        if (__any_sync(gm, __double_as_longlong(fb) != 0)) fb = group_sum<G>(fb, gm);
    } else {
        each_entry([&](int t, int ko, int ki) {
            if (t != x.r && t != x.s) entry_exact(md, x, t, ko, ki, pf64, pb64);
        });
    }
    pf64 = group_sum<G>(pf64, gm);
    pb64 = group_sum<G>(pb64, gm);
    corner_hastings_exact(x, cv, md.B, pf64, pb64);
    if (gl == 0) {
        const Exact e = exact_decision(a.beta, dl, fb, pf64, pb64, w2);
        if (e.accept) accept_move(md, x.v, x.s, x.k);
        count_exact(c, e.accept, e.margin, x.k);
        write_trace(a, x.v, x.s, 1 | (e.accept ? 2 : 0) | (e.margin ? 4 : 0), e.dH, e.logA);
    }
}

// the whole warp on one mover; unsettled moves go to the recheck list
template <bool DL32, class EachEntry>
__device__ __forceinline__ void evaluate_warp(const DecideArgs &a, const ModelDev &md, VertexCtx &x, uint64_t w2,
                                              EachEntry each_entry, Counts &c) {
    evaluate_group<DL32, 32, false>(a, md, x, w2, each_entry, c);
}

}  // namespace
}  // namespace sbp
