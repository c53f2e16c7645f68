// common.cuh -- internal types and device helpers of libsbp (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "sbp.h"

namespace sbp {

// ---------------------------------------------------------------------------
// error plumbing (host)
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define SBP_CUDA(call)                                  \
    do {                                                \
        cudaError_t _e = (call);                        \
        if (_e != cudaSuccess) return sbp::cuda_fail(_e, #call); \
    } while (0)

// every kernel launch of the library goes through SBP_LAUNCHED(), which
// counts it (sbp_kernel_launches) and checks the launch error
void count_launch();
#define SBP_LAUNCHED()                           \
    do {                                         \
        sbp::count_launch();                     \
        SBP_CUDA(cudaGetLastError());            \
    } while (0)

// Device memory of a model: stream-ordered allocation on the model's stream
// (no device-wide synchronisation, so threads driving other models are not
// stalled), and a pool of small pinned host buffers for read-backs.
cudaError_t model_alloc(void **p, size_t bytes, cudaStream_t st);
void model_free(void *p, cudaStream_t st);
void *pinned_get();
void pinned_put(void *p);

// Raises the dynamic shared memory limit of kernel `func` on the current
// device to at least `bytes`; never lowers it, so threads launching the same
// kernel with different sizes cannot undercut one another's launch.
int ensure_dyn_smem(const void *func, size_t bytes);

// SBP_EINVAL with a message when a parameter is out of range
int params_valid(const sbp_params &p);

#define SBP_TRY(call)                \
    do {                             \
        int _rc = (call);            \
        if (_rc != SBP_OK) return _rc; \
    } while (0)

// device status word: first error code recorded by a kernel wins
__device__ __forceinline__ void record_status(int32_t *status, int32_t code) {
    atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// tuning constants
constexpr int kWarp = 32;
constexpr int kSmallDeg = 32;     // k <= 32: one neighbour per lane, no table
constexpr int kWarpDeg = 128;     // k <= 128: one warp per vertex, per-warp table
constexpr int kWarpCap = 256;     // per-warp table slots (>= 2 * kWarpDeg)
constexpr int kWarpsPerCta = 8;
constexpr int kBigThreads = 256;  // threads of the CTA-per-vertex kernel
constexpr int64_t kMaxTable = int64_t(1) << 22;  // largest x ln x table (entries)

// ---------------------------------------------------------------------------
// graph and model state
// keys computed on the fly from the out-edge list: key of out-edge e is
// b[esrc[e]] * B + b[oc[e]] (row block, column block)
struct EdgeKeys {
    const int32_t *esrc = nullptr, *oc = nullptr, *b = nullptr;
    uint64_t B = 0;
};

struct GraphDev {
    int32_t n;
    int64_t m;
    const int32_t *op, *ip;  // [n+1] out / in row offsets
    const int32_t *oc, *ic;  // [m] neighbours, ascending per row
    const int32_t *esrc;     // [m] source vertex of each out-edge (CSR order)
    const int32_t *tw_oi;    // [m] in-row position of each out-row entry (the same edge)
    const int32_t *tw_io;    // [m] out-row position of each in-row entry
};

}  // namespace sbp

struct sbp_graph {
    int64_t n = 0, m = 0;
    int device = 0;
    int32_t *op = nullptr, *ip = nullptr, *oc = nullptr, *ic = nullptr, *esrc = nullptr;
    int32_t *tw_oi = nullptr, *tw_io = nullptr;  // twin positions of each edge in the other CSR
    int32_t *self_in = nullptr;  // in-row positions of the self-loops
    int64_t n_self = 0;
    int32_t *order = nullptr;  // vertices grouped: k=0 | 1..32 | 33..128 | >128
    int32_t *by_degree = nullptr;  // all vertices by degree, descending (ties: lower id first)
    int64_t bin[5] = {0, 0, 0, 0, 0};
    int32_t max_deg = 0;
    sbp::GraphDev dev() const {
        sbp::GraphDev d;
        d.n = (int32_t)n; d.m = m; d.op = op; d.ip = ip; d.oc = oc; d.ic = ic; d.esrc = esrc;
        d.tw_oi = tw_oi; d.tw_io = tw_io;
        return d;
    }
};

namespace sbp {

// device-side counters of a decision pass: proposed, moves, accepted, margin
struct DevCounters {
    unsigned long long proposed, moves, accepted, margin, move_edges, acc_edges, recheck;
    unsigned long long items;  // entries appended to the accepted-move list
    unsigned long long entries;  // distinct neighbour blocks of the evaluated movers (sum of D_v)
};

// the accepted-move list: one (vertex, chunk) item per kMoveChunk edges of
// every accepted mover, so the apply step's work units are all small
constexpr int kMoveChunk = 256;

struct ModelDev {
    int32_t B;
    int32_t n;
    int64_t m;
    const int32_t *b;       // frozen assignment
    int32_t *bnew;          // pending assignment
    const int32_t *M;       // dense [B*B]
    const uint32_t *P;      // [B*2B]: row prefix of M[u][.], then dout_u + column prefix of M[.][u]
    const uint32_t *Pc;     // [B*32]: every pstep-th entry of P[u] (coarse CDF)
    int32_t pstep;          // ceil(2B / 32)
    const int32_t *dout, *din;
    const double *rcp;      // 1 / (dout_t + din_t + B)
    const float *rcp32;     // the same in FP32
    const int32_t *dsum;    // dout_t + din_t
    const __int128 *T;      // round(x ln x * 2^64), x < XT
    int64_t XT;
    // sparse form (B > dense_max_B): CSR and CSC of M with per-row / per-column
    // inclusive count prefixes, and per-row open-addressing tables
    int sparse;
    const uint32_t *rp, *cp, *hoff;   // [B+1]
    const int32_t *rc, *cr;           // column of each row entry, row of each column entry
    const int32_t *rv, *cv;           // their counts
    const uint32_t *rpre, *cpre;      // inclusive count prefixes inside each row / column
    const uint32_t *rpc, *cpc;        // [B * 32]: pivot i of a row is its prefix at the end of
                                      // the i-th of 32 equal segments (all ones past the row)
    const int2 *hkv;                  // table slots: (key, count), key -1 when empty
    int32_t *status;
    DevCounters *counters;
    int2 *items;        // accepted-move list (NULL: not kept)
    int64_t cap_items;
    // block-labelled rows: nbo[e] = b[oc[e]], nbi[j] = b[ic[j]], bit 31 set
    // when the neighbour is the row's own vertex (NULL: gather b instead)
    const int32_t *nbo, *nbi;
};

constexpr int32_t kNbSelf = INT32_MIN;  // self-loop bit of a block-labelled entry

}  // namespace sbp

struct sbp_model {
    struct Sparse {
        int64_t cap_e = 0, nnz = 0;
        int32_t cap_b = 0;
        uint64_t *key0 = nullptr, *key1 = nullptr;
        uint32_t *start = nullptr, *scratch = nullptr;
        int32_t *rc = nullptr, *rv = nullptr, *rowof = nullptr, *cr = nullptr, *cv = nullptr;
        uint32_t *rpre = nullptr, *cpre = nullptr;
        uint32_t *ckey0 = nullptr, *ckey1 = nullptr;
        uint64_t *cval0 = nullptr, *cval1 = nullptr;
        int2 *hkv = nullptr;  // per-row open-addressing slots (key, count)
        uint32_t *rp = nullptr, *cp = nullptr, *hoff = nullptr, *cnt = nullptr;
        uint32_t *rpc = nullptr, *cpc = nullptr;  // [B * 32] coarse pivots of rpre / cpre per row / column
        int32_t *cells = nullptr;  // B x B counts of the counting-sort rebuild
        int64_t cap_cells = 0;
        int32_t cells_B = 0;       // B the cells hold the counts of m->bnew for, else 0
        int64_t *nnz_dev = nullptr;  // the nonzero count when only the device has it (nnz < 0)
    };
    Sparse sp;
    const sbp_graph *g = nullptr;
    sbp_params p{};
    cudaStream_t stream = nullptr;
    int32_t B = 0, Bcap = 0, Bdense = 0;
    int32_t *b = nullptr, *bnew = nullptr;
    int32_t *M = nullptr;
    uint32_t *P = nullptr;
    uint32_t *Pc = nullptr;
    int32_t *dout = nullptr, *din = nullptr;
    double *rcp = nullptr;
    float *rcp32 = nullptr;
    int32_t *dsum = nullptr;
    const __int128 *T = nullptr;
    int64_t XT = 0;
    double *dl = nullptr;        // [2]: current DL, DL before the last commit
    double *partials = nullptr;  // reduction scratch
    int32_t npartials = 0;
    sbp::DevCounters *counters = nullptr;
    int32_t *status = nullptr;
    // merge scratch
    int32_t *best_s = nullptr;
    double *best_d = nullptr;
    int32_t *map = nullptr;
    int32_t *vcount = nullptr;
    // nodal pass: proposals with s != r, in three lists by degree
    void *movers = nullptr;
    unsigned *mcount = nullptr;
    // accepted moves since the last commit, as (vertex, edge chunk) items;
    // list_ok is false when the pending assignment has changes the list does
    // not hold (labels set from outside, overlapping decide ranges)
    int2 *items = nullptr;
    int64_t cap_items = 0;
    // block-labelled copy of the adjacency (nbo: out-rows, nbi: in-rows);
    // nb_ok: it matches m->b
    int32_t *nbo = nullptr, *nbi = nullptr;
    bool nb_ok = false;
    bool nb_in_commit = false;  // the apply step's kernel updated them in this commit
    bool list_ok = true;
    std::vector<std::pair<int64_t, int64_t>> decided;  // decide ranges since the last commit
    // side streams of the decision pass: the three degree groups' kernels
    // run concurrently so that each one's tail is filled by the others
    cudaStream_t side[2] = {nullptr, nullptr};
    cudaEvent_t fork_ev = nullptr, join_ev[2] = {nullptr, nullptr};
    uint8_t *skip = nullptr;  // the hybrid pass's sequential vertices (n flags)
    unsigned long long *cta_tab = nullptr;  // global neighbour tables of the CTA kernel
    size_t cta_tab_bytes = 0;
    int32_t skip_h = -1;      // the h skip was built for
    // pinned host mirror for small read-backs
    void *pinned = nullptr;
    bool dense = true;
};

namespace sbp {

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11): two 64x64->128 products per round
// with the published multipliers; key bumped by the published Weyl
// constants between rounds.
struct U64x4 {
    uint64_t x, y, z, w;
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                                uint64_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        const uint64_t a = 0xD2E7470EE14C6C93ULL * c0, ah = __umul64hi(0xD2E7470EE14C6C93ULL, c0);
        const uint64_t b = 0xCA5A826395121157ULL * c2, bh = __umul64hi(0xCA5A826395121157ULL, c2);
        const uint64_t n0 = bh ^ c1 ^ k0, n2 = ah ^ c3 ^ k1;
        c0 = n0; c1 = b; c2 = n2; c3 = a;
    }
    return U64x4{c0, c1, c2, c3};
}

// integer in [0, n): high word of w * n
__device__ __forceinline__ int64_t draw_below(uint64_t w, uint64_t n) { return (int64_t)__umul64hi(w, n); }

// f(x+k) - f(x) for f(x) = x ln x, as k ln(x+k) + x log1p(k/x)
__device__ __forceinline__ double dxlogx(int64_t x, int64_t k) {
    if (k == 0) return 0.0;
    if (x == 0) return (double)k * log((double)k);
    if (x + k == 0) return -(double)x * log((double)x);
    return (double)k * log((double)(x + k)) + (double)x * log1p((double)k / (double)x);
}

static __device__ __noinline__ double dxlogx_slow(int64_t x, int64_t k) { return dxlogx(x, k); }

// f(x+k) - f(x) from the fixed-point table when both counts are inside it;
// otherwise the FP64 formula above is added to fb and 0 returned
__device__ __forceinline__ __int128 dT(const __int128 *__restrict__ T, int64_t XT, int64_t x, int64_t k, double &fb) {
    if (k == 0) return 0;
    const int64_t y = x + k;
    if (x < XT && y < XT) return T[y] - T[x];
    fb += dxlogx_slow(x, k);
    return 0;
}

__device__ __forceinline__ __int128 shfl_xor_128(__int128 v, int o) {
    const unsigned long long lo = (unsigned long long)v;
    const long long hi = (long long)(v >> 64);
    const unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, lo, o);
    const long long hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
    return (__int128)(((unsigned __int128)(unsigned long long)hi2 << 64) | lo2);
}

__device__ __forceinline__ __int128 warp_sum_128(__int128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor_128(v, o);
    return v;
}

// reductions over an aligned group of G lanes (G = 8, 16, 32) that share
// a mover; every lane of the group gets the sum
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if (G == 32) return 0xffffffffu;
    return ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
}

template <int G, class T>
__device__ __forceinline__ T group_sum(T v, unsigned gm) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gm, v, o);
    return v;
}

template <int G>
__device__ __forceinline__ __int128 group_sum_128(__int128 v, unsigned gm) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        const unsigned long long lo = __shfl_xor_sync(gm, (unsigned long long)v, o);
        const long long hi = __shfl_xor_sync(gm, (long long)(v >> 64), o);
        v += (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | lo);
    }
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// fixed point (scale 2^64) to float / double
// (two 32-bit conversions: 64-bit integer conversions would use the FP64 pipe)
__device__ __forceinline__ float fix_to_float(__int128 v) {
    const int hi = (int)(v >> 72);                           // units of 2^8
    const unsigned lo = (unsigned)((v >> 40) & 0xffffffffu);  // units of 2^-24
    return fmaf((float)hi, 256.0f, (float)lo * 0x1p-24f);
}
__device__ __forceinline__ double fix_to_double(__int128 v) {
    const long long hi = (long long)(v >> 64);
    const unsigned long long lo = (unsigned long long)v;
    return (double)hi + (double)lo * 0x1p-64;
}

// f(a+b) - f(a) - f(b) = a log1p(b/a) + b log1p(a/b)
__device__ __forceinline__ double gmerge(int64_t a, int64_t b) {
    if (a == 0 || b == 0) return 0.0;
    return (double)a * log1p((double)b / (double)a) + (double)b * log1p((double)a / (double)b);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// first index i in a[0, len) with a[i] > t (a non-decreasing, a[len-1] > t),
// warp-cooperative 32-ary search; every lane returns the answer
__device__ __forceinline__ int warp_upper_bound(const uint32_t *__restrict__ a, int len, uint32_t t) {
    const int lane = threadIdx.x & 31;
    int lo = 0;
    while (len > 32) {
        const int step = (len + 31) >> 5;
        int idx = lo + (lane + 1) * step - 1;
        const int last = lo + len - 1;
        if (idx > last) idx = last;
        const uint32_t val = a[idx];
        const unsigned mask = __ballot_sync(0xffffffffu, val > t);
        const int first = __ffs(mask) - 1;  // a[last] > t, so mask != 0
        const int nlo = lo + first * step;
        const int nhi = (lo + (first + 1) * step - 1 < last) ? lo + (first + 1) * step - 1 : last;
        lo = nlo;
        len = nhi - nlo + 1;
    }
    const uint32_t val = lane < len ? a[lo + lane] : 0xffffffffu;
    const unsigned mask = __ballot_sync(0xffffffffu, val > t);
    return lo + __ffs(mask) - 1;
}

// first index i in Pu[0, len) with Pu[i] > t, given the 32 pivots
// Pcu[q] = Pu[min((q+1) step - 1, len - 1)]: the pivots pick a segment of at
// most `step` entries, searched with one more read while step <= 32
__device__ __forceinline__ int warp_cdf_search(const uint32_t *__restrict__ Pu, const uint32_t *Pcu, int len, int step,
                                               uint32_t t) {
    const int lane = threadIdx.x & 31;
    if (len <= 32) {
        const uint32_t val = lane < len ? Pu[lane] : 0xffffffffu;
        return __ffs(__ballot_sync(0xffffffffu, val > t)) - 1;
    }
    const uint32_t pv = Pcu[lane];
    const int first = __ffs(__ballot_sync(0xffffffffu, pv > t)) - 1;
    const int lo = first * step;
    const int seg = step < len - lo ? step : len - lo;
    if (seg <= 32) {
        const uint32_t val = lane < seg ? Pu[lo + lane] : 0xffffffffu;
        return lo + __ffs(__ballot_sync(0xffffffffu, val > t)) - 1;
    }
    return lo + warp_upper_bound(Pu + lo, seg, t);
}

// ---------------------------------------------------------------------------
// blockmodel access (dense or sparse, a kernel-wide flag)

__device__ __forceinline__ unsigned sparse_hash(int key) { return (unsigned)key * 0x9E3779B1u; }

// M[r][c] from row r's table (bounded probe; absent = 0)
__device__ __forceinline__ int sparse_at(const ModelDev &md, int r, int c) {
    const uint32_t off = md.hoff[r], cap = md.hoff[r + 1] - off;
    uint32_t h = sparse_hash(c) & (cap - 1);
    for (uint32_t q = 0; q < cap; ++q) {
        const int2 kv = md.hkv[off + h];  // key and count in one load
        if (kv.x == c) return kv.y;
        if (kv.x < 0) return 0;
        h = (h + 1) & (cap - 1);
    }
    return 0;
}

__device__ __forceinline__ int Mat(const ModelDev &md, int r, int c) {
    return md.sparse ? sparse_at(md, r, c) : md.M[(size_t)r * md.B + c];
}

// v's idx-th neighbour entry (out-row first): its block-labelled entry when
// the pass keeps them, else the neighbour's id
__device__ __forceinline__ int nb_raw(const GraphDev &g, const ModelDev &md, int o0, int i0, int kout, int idx) {
    if (md.nbo) return idx < kout ? md.nbo[o0 + idx] : md.nbi[i0 + idx - kout];
    return idx < kout ? g.oc[o0 + idx] : g.ic[i0 + idx - kout];
}

// the block of an entry from nb_raw, and whether the neighbour is v itself
__device__ __forceinline__ int nb_block(const ModelDev &md, int raw, int v, bool &self) {
    if (md.nbo) {
        self = raw < 0;
        return raw & 0x7fffffff;
    }
    self = raw == v;
    return md.b[raw];
}

// continues a probe of row table [off, off + cap) for key c whose first
// slot h has been loaded into kv (same bound and result as sparse_at)
__device__ __forceinline__ int sparse_probe_from(const ModelDev &md, uint32_t off, uint32_t cap, uint32_t h, int c,
                                                 int2 kv) {
    for (uint32_t q = 1;; ++q) {
        if (kv.x == c) return kv.y;
        if (kv.x < 0 || q >= cap) return 0;
        h = (h + 1) & (cap - 1);
        kv = md.hkv[off + h];
    }
}

// the four counts a neighbour block t contributes to a move r -> s:
// M[r][t], M[s][t], M[t][r], M[t][s].  On sparse rows the three row offsets
// and then the four first probe slots are loaded together (two dependent
// rounds instead of eight); collisions continue one slot at a time.
__device__ __forceinline__ void Mat4(const ModelDev &md, int r, int s, int t, int &Mrt, int &Mst, int &Mtr,
                                     int &Mts) {
    if (!md.sparse) {
        const size_t B = (size_t)md.B;
        Mrt = md.M[(size_t)r * B + t];
        Mst = md.M[(size_t)s * B + t];
        Mtr = md.M[(size_t)t * B + r];
        Mts = md.M[(size_t)t * B + s];
        return;
    }
    const uint32_t o_r = md.hoff[r], c_r = md.hoff[r + 1] - o_r;
    const uint32_t o_s = md.hoff[s], c_s = md.hoff[s + 1] - o_s;
    const uint32_t o_t = md.hoff[t], c_t = md.hoff[t + 1] - o_t;
    const uint32_t ht = sparse_hash(t);
    const uint32_t h1 = ht & (c_r - 1), h2 = ht & (c_s - 1);
    const uint32_t h3 = sparse_hash(r) & (c_t - 1), h4 = sparse_hash(s) & (c_t - 1);
    const int2 k1 = md.hkv[o_r + h1], k2 = md.hkv[o_s + h2], k3 = md.hkv[o_t + h3], k4 = md.hkv[o_t + h4];
    Mrt = sparse_probe_from(md, o_r, c_r, h1, t, k1);
    Mst = sparse_probe_from(md, o_s, c_s, h2, t, k2);
    Mtr = sparse_probe_from(md, o_t, c_t, h3, r, k3);
    Mts = sparse_probe_from(md, o_t, c_t, h4, s, k4);
}

// first i in a[lo, hi) with a[i] > t (one lane, binary search)
__device__ __forceinline__ uint32_t lane_upper(const uint32_t *__restrict__ a, uint32_t lo, uint32_t hi, uint32_t t) {
    uint32_t n = hi - lo;
    while (n > 0) {
        const uint32_t half = n >> 1;
        if (a[lo + half] <= t) {
            lo += half + 1;
            n -= half + 1;
        } else {
            n = half;
        }
    }
    return lo;
}

// first i in a[lo, hi) with a[i] >= t (one lane)
__device__ __forceinline__ uint32_t lane_lower_i32(const int32_t *__restrict__ a, uint32_t lo, uint32_t hi, int32_t t) {
    uint32_t n = hi - lo;
    while (n > 0) {
        const uint32_t half = n >> 1;
        if (a[lo + half] < t) {
            lo += half + 1;
            n -= half + 1;
        } else {
            n = half;
        }
    }
    return lo;
}

// first i in pre[lo, hi) with pre[i] > t (pre non-decreasing, pre[hi-1] > t),
// with the row's 32 pivots: the eight 16-byte pivot loads and then up to
// eight entries of the segment are in flight together
__device__ __forceinline__ uint32_t pivot_upper(const uint32_t *pre, const uint32_t *piv, uint32_t lo, uint32_t hi,
                                                uint32_t t) {
    const uint32_t len = hi - lo;
    uint32_t seg = len;
    if (len > 32) {
        uint4 pv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) pv[i] = reinterpret_cast<const uint4 *>(piv)[i];
        uint32_t fp = 31;
#pragma unroll
        for (int i = 7; i >= 0; --i) {
            if (pv[i].w > t) fp = 4 * i + 3;
            if (pv[i].z > t) fp = 4 * i + 2;
            if (pv[i].y > t) fp = 4 * i + 1;
            if (pv[i].x > t) fp = 4 * i;
        }
        const uint32_t step = (len + 31) / 32;
        lo += fp * step;
        seg = step < hi - lo ? step : hi - lo;
    }
    if (seg > 32) return lane_upper(pre, lo, lo + seg, t);
    for (uint32_t g0 = 0; g0 < seg; g0 += 8) {
        uint32_t x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = g0 + i < seg ? pre[lo + g0 + i] : 0xffffffffu;
        int idx = -1;
#pragma unroll
        for (int i = 7; i >= 0; --i)
            if (x[i] > t) idx = i;
        if (idx >= 0) return lo + g0 + (uint32_t)idx;
    }
    return lo + seg - 1;
}

// Sparse inverse CDF over row u then column u of M (weights M[u][c], then
// M[c][u]), t < dout_u + din_u: the block at that position.  One lane.
__device__ __forceinline__ int sparse_cdf_block(const ModelDev &md, int u, uint32_t t, uint32_t dout_u) {
    if (t < dout_u) {
        const uint32_t i = pivot_upper(md.rpre, md.rpc + (size_t)u * 32, md.rp[u], md.rp[u + 1], t);
        return md.rc[i];
    }
    const uint32_t i = pivot_upper(md.cpre, md.cpc + (size_t)u * 32, md.cp[u], md.cp[u + 1], t - dout_u);
    return md.cr[i];
}

// ---------------------------------------------------------------------------
// host-side launch helpers implemented in the .cu files
int rebuild_blockmodel(sbp_model *m);  // M, P, degrees, rcp, DL from m->b
int count_cells(sbp_model *m, int32_t *cells);  // cells[r * B + t] = edges r -> t
int update_cells(sbp_model *m, int32_t *cells);  // counts of m->bnew -> counts of m->b
int launch_prefix(sbp_model *m);                 // P, Pc, degrees, reciprocals from a dense M
int commit_blockmodel(sbp_model *m);   // the same after a pass: m->b new labels, m->bnew the previous ones
int launch_decide(sbp_model *m, uint64_t sweep_id, int64_t v_begin, int64_t v_end, const sbp_vertex_trace *trace);
int nb_rows_rebuild(sbp_model *m);       // block-labelled rows from m->b (nb_ok when there is memory)
int nb_rows_after_commit(sbp_model *m);  // ... brought up to date after a commit
int launch_merge_proposals(sbp_model *m, uint64_t round_id);
int launch_relabel(sbp_model *m, const int32_t *map_dev);
int launch_vertex_count(sbp_model *m);
int ensure_capacity(sbp_model *m, int32_t B);
int check_status(const sbp_model *m);
int xlogx_table(int64_t need, const __int128 **table, int64_t *size);
int ensure_sparse_capacity(sbp_model *m, int32_t B);
int rebuild_sparse(sbp_model *m, bool after_pass, bool *dl_done);
int64_t sparse_nnz(sbp_model *m);  // the nonzero count (read back once when only the device has it)
void free_sparse(sbp_model *m);

// sort.cu: exclusive scan of n uint32 (in may equal out; *total_dev, device,
// may be NULL) and the stable LSD radix sort with its scratch sizes
int exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total_dev, uint32_t *scratch,
                       cudaStream_t st);
int64_t scan_scratch_words(int64_t n);
int64_t sort_scratch_words(int64_t n);
int sort_chunk_count(int64_t n);
int64_t sort_chunk_length(int64_t n);
template <class K, class V>
int radix_sort(K *k0, K *k1, V *v0, V *v1, int64_t n, int bits, uint32_t *scratch, cudaStream_t st, bool *in_first,
               const EdgeKeys *edges = nullptr);
ModelDev model_dev(sbp_model *m);

}  // namespace sbp
