/*
 * sbp_oracle.c -- plain, slow CPU oracle of the stochastic block partitioning
 * (SBP) hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library) never calls it and shares no code with it.
 *
 * Arithmetic: FP64 throughout; block counts as int64.  Every function cites
 * the passage of the paper it follows.  Where the paper only names a step
 * ("propose new community", "compute Metropolis-Hastings ratio", the golden
 * ratio search), the reading taken is spelled out in the comment; both the
 * oracle and the CUDA path follow the same readings.
 *
 * Parity status: P1 (blockmodel, Eq. 1-2), P2 (Philox), P3-P5 (proposal,
 * move Delta-DL, Hastings, and the acceptance draw re-derived from numpy's
 * Philox words), P7 (merge Delta-DL) and P8 (merge application, including
 * its further proposal rounds) are pinned by the tests against brute force,
 * closed forms and numpy.  P9: the MCMC stop rule is pinned against DL
 * histories recomputed by numpy, and the phase sequence of a full run
 * against the bracket rule alone (itself pinned on unimodal curves); the
 * driver's constants are readings, not values from the paper.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): 10 rounds of two 64x64->128 multiplies with the
 * published multipliers, key schedule bumped by the published Weyl constants
 * between rounds. */
typedef unsigned __int128 u128;

void og_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        u128 p0 = (u128)0xD2E7470EE14C6C93ULL * c0;
        u128 p1 = (u128)0xCA5A826395121157ULL * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* An integer in [0, n): the high word of w * n. */
static int64_t draw(uint64_t w, int64_t n) { return (int64_t)(((u128)w * (uint64_t)n) >> 64); }

/* ------------------------------------------------------------------------ */
/* Graph: directed, duplicates kept, self-loops kept (they appear in both the
 * out- and in-list of their vertex).  Neighbour lists ascend by id. */
typedef struct {
    int64_t n, m;
    int64_t *op, *ip; /* [n+1] */
    int32_t *oc, *ic; /* [m]   */
} og_graph;

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}
static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static void build_csr(int64_t n, int64_t m, const int32_t *from, const int32_t *to, int64_t *ptr, int32_t *col) {
    memset(ptr, 0, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t e = 0; e < m; ++e) ptr[from[e] + 1]++;
    for (int64_t v = 0; v < n; ++v) ptr[v + 1] += ptr[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) fill[v] = ptr[v];
    for (int64_t e = 0; e < m; ++e) col[fill[from[e]]++] = to[e];
    free(fill);
    for (int64_t v = 0; v < n; ++v) qsort(col + ptr[v], (size_t)(ptr[v + 1] - ptr[v]), sizeof(int32_t), cmp_i32);
}

og_graph *og_graph_new(int64_t n, int64_t m, const int32_t *src, const int32_t *dst) {
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return NULL;
    og_graph *g = (og_graph *)calloc(1, sizeof(og_graph));
    g->n = n; g->m = m;
    g->op = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    g->ip = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    g->oc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    g->ic = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    build_csr(n, m, src, dst, g->op, g->oc);
    build_csr(n, m, dst, src, g->ip, g->ic);
    return g;
}

void og_graph_free(og_graph *g) {
    if (!g) return;
    free(g->op); free(g->ip); free(g->oc); free(g->ic); free(g);
}

void og_graph_csr(const og_graph *g, int64_t *op, int32_t *oc, int64_t *ip, int32_t *ic) {
    memcpy(op, g->op, sizeof(int64_t) * (size_t)(g->n + 1));
    memcpy(ip, g->ip, sizeof(int64_t) * (size_t)(g->n + 1));
    memcpy(oc, g->oc, sizeof(int32_t) * (size_t)g->m);
    memcpy(ic, g->ic, sizeof(int32_t) * (size_t)g->m);
}

/* ------------------------------------------------------------------------ */
/* P1. Blockmodel (Section II-A): M[r][s] = number of edges from a vertex of
 * block r to a vertex of block s; dout_r = sum_s M[r][s], din_s = sum_r
 * M[r][s].  Held sparse, as sorted (key, count) lists in row order (key =
 * r*B+s) and column order (key = s*B+r), i.e. the blockmodel and its stored
 * transpose (Section III-A (a)-(b)). */
typedef struct {
    const og_graph *g;
    int64_t B;
    int32_t *b;
    int64_t nnz;
    int64_t *rk, *rc, *rptr; /* row order */
    int64_t *ck, *cc, *cptr; /* column order */
    int64_t *dout, *din;
} og_model;

static void count_runs(int64_t *keys, int64_t m, int64_t B, int64_t **ko, int64_t **co, int64_t **ptr, int64_t *nnz) {
    qsort(keys, (size_t)m, sizeof(int64_t), cmp_i64);
    int64_t runs = 0;
    for (int64_t e = 0; e < m; ++e)
        if (e == 0 || keys[e] != keys[e - 1]) runs++;
    *ko = (int64_t *)malloc(sizeof(int64_t) * (size_t)(runs > 0 ? runs : 1));
    *co = (int64_t *)malloc(sizeof(int64_t) * (size_t)(runs > 0 ? runs : 1));
    *ptr = (int64_t *)calloc((size_t)(B + 1), sizeof(int64_t));
    int64_t k = -1;
    for (int64_t e = 0; e < m; ++e) {
        if (e == 0 || keys[e] != keys[e - 1]) {
            ++k;
            (*ko)[k] = keys[e];
            (*co)[k] = 0;
            (*ptr)[keys[e] / B + 1]++;
        }
        (*co)[k]++;
    }
    for (int64_t r = 0; r < B; ++r) (*ptr)[r + 1] += (*ptr)[r];
    *nnz = runs;
}

static void model_release(og_model *md) {
    free(md->rk); free(md->rc); free(md->rptr);
    free(md->ck); free(md->cc); free(md->cptr);
    free(md->dout); free(md->din);
    md->rk = md->rc = md->rptr = md->ck = md->cc = md->cptr = md->dout = md->din = NULL;
}

static void model_rebuild(og_model *md) {
    const og_graph *g = md->g;
    int64_t B = md->B, m = g->m;
    model_release(md);
    int64_t *keys = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t nnz_c = 0;
    for (int64_t v = 0; v < g->n; ++v)
        for (int64_t e = g->op[v]; e < g->op[v + 1]; ++e) keys[e] = (int64_t)md->b[v] * B + md->b[g->oc[e]];
    count_runs(keys, m, B, &md->rk, &md->rc, &md->rptr, &md->nnz);
    for (int64_t v = 0; v < g->n; ++v)
        for (int64_t e = g->op[v]; e < g->op[v + 1]; ++e) keys[e] = (int64_t)md->b[g->oc[e]] * B + md->b[v];
    count_runs(keys, m, B, &md->ck, &md->cc, &md->cptr, &nnz_c);
    free(keys);
    md->dout = (int64_t *)calloc((size_t)B, sizeof(int64_t));
    md->din = (int64_t *)calloc((size_t)B, sizeof(int64_t));
    for (int64_t k = 0; k < md->nnz; ++k) {
        md->dout[md->rk[k] / B] += md->rc[k];
        md->din[md->rk[k] % B] += md->rc[k];
    }
}

/* Returns NULL when a label is outside [0, B). */
og_model *og_model_new(const og_graph *g, int64_t B, const int32_t *b) {
    if (B < 1) return NULL;
    for (int64_t v = 0; v < g->n; ++v)
        if (b[v] < 0 || b[v] >= B) return NULL;
    og_model *md = (og_model *)calloc(1, sizeof(og_model));
    md->g = g;
    md->B = B;
    md->b = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n > 0 ? g->n : 1));
    memcpy(md->b, b, sizeof(int32_t) * (size_t)g->n);
    model_rebuild(md);
    return md;
}

void og_model_free(og_model *md) {
    if (!md) return;
    model_release(md);
    free(md->b);
    free(md);
}

/* Apply new assignments and rebuild M (Alg. 5: after the exchange every
 * rank's blockmodel is recomputed to agree with the assignments). */
int og_model_set_b(og_model *md, int64_t B, const int32_t *b) {
    for (int64_t v = 0; v < md->g->n; ++v)
        if (b[v] < 0 || b[v] >= B) return -1;
    md->B = B;
    memcpy(md->b, b, sizeof(int32_t) * (size_t)md->g->n);
    model_rebuild(md);
    return 0;
}

int64_t og_model_nnz(const og_model *md) { return md->nnz; }
int64_t og_model_B(const og_model *md) { return md->B; }

void og_model_get(const og_model *md, int64_t *keys, int64_t *cnt, int64_t *dout, int64_t *din, int32_t *b) {
    if (keys) memcpy(keys, md->rk, sizeof(int64_t) * (size_t)md->nnz);
    if (cnt) memcpy(cnt, md->rc, sizeof(int64_t) * (size_t)md->nnz);
    if (dout) memcpy(dout, md->dout, sizeof(int64_t) * (size_t)md->B);
    if (din) memcpy(din, md->din, sizeof(int64_t) * (size_t)md->B);
    if (b) memcpy(b, md->b, sizeof(int32_t) * (size_t)md->g->n);
}

/* M[r][s] by binary search in row r. */
static int64_t M_at(const og_model *md, int64_t r, int64_t s) {
    int64_t lo = md->rptr[r], hi = md->rptr[r + 1], key = r * md->B + s;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (md->rk[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < md->rptr[r + 1] && md->rk[lo] == key) ? md->rc[lo] : 0;
}

/* x ln x with 0 ln 0 = 0. */
static double xlogx(double x) { return x > 0.0 ? x * log(x) : 0.0; }

/* f(x+k) - f(x) for f(x) = x ln x, written k ln(x+k) + x log1p(k/x) so the
 * difference of two large terms is not formed. */
static double dxlogx(int64_t x, int64_t k) {
    if (k == 0) return 0.0;
    if (x == 0) return xlogx((double)k);
    if (x + k == 0) return -xlogx((double)x);
    return (double)k * log((double)(x + k)) + (double)x * log1p((double)k / (double)x);
}

/* f(a+b) - f(a) - f(b) = a log1p(b/a) + b log1p(a/b). */
static double gmerge(int64_t a, int64_t b) {
    if (a == 0 || b == 0) return 0.0;
    return (double)a * log1p((double)b / (double)a) + (double)b * log1p((double)a / (double)b);
}

/* Eq. 1 in the split form sum M ln M - sum dout ln dout - sum din ln din. */
double og_model_L(const og_model *md) {
    double L = 0.0;
    for (int64_t k = 0; k < md->nnz; ++k) L += xlogx((double)md->rc[k]);
    for (int64_t r = 0; r < md->B; ++r) L -= xlogx((double)md->dout[r]);
    for (int64_t r = 0; r < md->B; ++r) L -= xlogx((double)md->din[r]);
    return L;
}

/* Eq. 2: DL = E h(C^2/E) + V ln C - L, h(x) = (1+x) ln(1+x) - x ln x. */
double og_dl(int64_t E, int64_t V, int64_t C, double L) {
    /* with no edges the model term E h(C^2/E) is taken at its limit 0 */
    double model = 0.0;
    if (E > 0) {
        double x = (double)C * (double)C / (double)E;
        model = (double)E * ((1.0 + x) * log1p(x) - x * log(x));
    }
    return model + (double)V * log((double)C) - L;
}

double og_model_dl(const og_model *md) { return og_dl(md->g->m, md->g->n, md->B, og_model_L(md)); }

/* ------------------------------------------------------------------------ */
/* P3. Nodal proposal (Alg. 2 "propose new community"; the distribution is
 * the one of the SBP literature the paper cites in Section II-B):
 * j uniform over the incident edges of v (out-list, then in-list), u = b[j];
 * s drawn with probability (1 + M[u][s] + M[s][u]) / (d_u + B) by an integer
 * inverse CDF: y < B picks s = y; otherwise walk row u, then column u. */
static int64_t row_pick(const og_model *md, int64_t u, int64_t t, int64_t skip) {
    int64_t acc = 0;
    for (int64_t k = md->rptr[u]; k < md->rptr[u + 1]; ++k) {
        int64_t c = md->rk[k] % md->B;
        if (c == skip) continue;
        acc += md->rc[k];
        if (acc > t) return c;
    }
    return -1;
}
static int64_t col_pick(const og_model *md, int64_t u, int64_t t, int64_t skip) {
    int64_t acc = 0;
    for (int64_t k = md->cptr[u]; k < md->cptr[u + 1]; ++k) {
        int64_t c = md->ck[k] % md->B;
        if (c == skip) continue;
        acc += md->cc[k];
        if (acc > t) return c;
    }
    return -1;
}

typedef struct {
    int32_t t;
    int32_t dir; /* 0 out, 1 in */
} nb_entry;

static int cmp_nb(const void *a, const void *b) {
    const nb_entry *x = (const nb_entry *)a, *y = (const nb_entry *)b;
    if (x->t != y->t) return (x->t > y->t) - (x->t < y->t);
    return (x->dir > y->dir) - (x->dir < y->dir);
}

/* P4 + P5 for v moving r -> s against the frozen blockmodel.
 * Section III-A (c): only the entries of rows r,s and columns r,s that the
 * move changes enter the sum (Section II-C: "two rows and two columns").
 * Outputs dH = Delta DL = -Delta L (C fixed during the sweep), and the
 * forward / backward proposal weights pf, pb (both times k_v).
 * scratch holds at least k_v entries. */
static void move_delta(const og_model *md, int64_t v, int64_t s, nb_entry *scratch, double *dH, double *pf, double *pb) {
    const og_graph *g = md->g;
    const int64_t B = md->B;
    const int64_t r = md->b[v];
    int64_t self = 0, cnt = 0;
    for (int64_t e = g->op[v]; e < g->op[v + 1]; ++e) {
        if (g->oc[e] == v) { self++; continue; }
        scratch[cnt].t = md->b[g->oc[e]]; scratch[cnt].dir = 0; cnt++;
    }
    for (int64_t e = g->ip[v]; e < g->ip[v + 1]; ++e) {
        if (g->ic[e] == v) continue;
        scratch[cnt].t = md->b[g->ic[e]]; scratch[cnt].dir = 1; cnt++;
    }
    qsort(scratch, (size_t)cnt, sizeof(nb_entry), cmp_nb);

    /* neighbour-block counts kout[t], kin[t] in ascending t */
    int64_t kout_r = 0, kin_r = 0, kout_s = 0, kin_s = 0, Kout = self, Kin = self;
    for (int64_t i = 0; i < cnt; ++i) {
        if (scratch[i].dir == 0) Kout++; else Kin++;
        if (scratch[i].t == r) { if (scratch[i].dir == 0) kout_r++; else kin_r++; }
        if (scratch[i].t == s) { if (scratch[i].dir == 0) kout_s++; else kin_s++; }
    }

    double dL = 0.0;
    for (int64_t i = 0; i < cnt;) {
        int64_t t = scratch[i].t, ko = 0, ki = 0;
        while (i < cnt && scratch[i].t == t) { if (scratch[i].dir == 0) ko++; else ki++; ++i; }
        if (t == r || t == s) continue;
        if (ko > 0) dL += dxlogx(M_at(md, r, t), -ko) + dxlogx(M_at(md, s, t), ko);
        if (ki > 0) dL += dxlogx(M_at(md, t, r), -ki) + dxlogx(M_at(md, t, s), ki);
    }
    const int64_t Mrr = M_at(md, r, r), Mss = M_at(md, s, s), Mrs = M_at(md, r, s), Msr = M_at(md, s, r);
    dL += dxlogx(Mrr, -(kout_r + kin_r + self));
    dL += dxlogx(Mss, kout_s + kin_s + self);
    dL += dxlogx(Mrs, kin_r - kout_s);
    dL += dxlogx(Msr, kout_r - kin_s);
    dL -= dxlogx(md->dout[r], -Kout) + dxlogx(md->dout[s], Kout) + dxlogx(md->din[r], -Kin) + dxlogx(md->din[s], Kin);
    *dH = -dL;

    /* P5: Hastings weights over the blocks t of v's neighbours (and r / s
     * for self-loops, whose far end is v itself), ascending t. */
    const int64_t Mrr2 = Mrr - (kout_r + kin_r + self);
    const int64_t Mrs2 = Mrs + kin_r - kout_s, Msr2 = Msr + kout_r - kin_s;
    double f = 0.0, bsum = 0.0;
    int64_t i = 0;
    int64_t lo = r < s ? r : s, hi = r < s ? s : r;
    int done_lo = 0, done_hi = 0;
    for (;;) {
        /* next distinct t in ascending order over neighbour blocks and {r, s} */
        int64_t t;
        int64_t cand = i < cnt ? scratch[i].t : INT64_MAX;
        if (!done_lo && lo <= cand) { t = lo; done_lo = 1; }
        else if (!done_hi && hi <= cand) { t = hi; done_hi = 1; }
        else if (i < cnt) t = cand;
        else break;
        int64_t ko = 0, ki = 0;
        while (i < cnt && scratch[i].t == t) { if (scratch[i].dir == 0) ko++; else ki++; ++i; }
        if (t == lo) done_lo = 1;
        if (t == hi) done_hi = 1;
        int64_t cf = ko + ki + (t == r ? 2 * self : 0);
        int64_t cb = ko + ki + (t == s ? 2 * self : 0);
        int64_t dt = md->dout[t] + md->din[t];
        if (t == r) {
            f += (double)cf * (double)(Mrs + Msr + 1) / (double)(dt + B);
            bsum += (double)cb * (double)(2 * Mrr2 + 1) / (double)(dt - Kout - Kin + B);
        } else if (t == s) {
            f += (double)cf * (double)(2 * Mss + 1) / (double)(dt + B);
            bsum += (double)cb * (double)(Msr2 + Mrs2 + 1) / (double)(dt + Kout + Kin + B);
        } else {
            int64_t Mts = M_at(md, t, s), Mst = M_at(md, s, t), Mtr = M_at(md, t, r), Mrt = M_at(md, r, t);
            f += (double)cf * (double)(Mts + Mst + 1) / (double)(dt + B);
            bsum += (double)cb * (double)((Mtr - ki) + (Mrt - ko) + 1) / (double)(dt + B);
        }
    }
    *pf = f;
    *pb = bsum;
}

/* Delta DL, pf and pb for moving v to s (s != b[v]); for the brute-force and
 * enumeration tests. */
int og_move_delta(const og_model *md, int64_t v, int64_t s, double *dH, double *pf, double *pb) {
    const og_graph *g = md->g;
    if (v < 0 || v >= g->n || s < 0 || s >= md->B || s == md->b[v]) return -1;
    int64_t k = (g->op[v + 1] - g->op[v]) + (g->ip[v + 1] - g->ip[v]);
    nb_entry *sc = (nb_entry *)malloc(sizeof(nb_entry) * (size_t)(k > 0 ? k : 1));
    move_delta(md, v, s, sc, dH, pf, pb);
    free(sc);
    return 0;
}

/* Per-vertex outcome of one nodal decision. */
typedef struct {
    int32_t s;       /* proposed block (= r when no proposal) */
    int32_t flags;   /* 1 proposed, 2 accepted */
    double dH, logA, lnu;
} og_decision;

/* P3-P5 for vertex v: proposal, Delta DL, Hastings-corrected Metropolis test
 * (Alg. 2 lines "propose" .. "if move is accepted"). */
static void nodal_decide(const og_model *md, uint64_t seed, uint64_t sweep_id, double beta, int64_t v, nb_entry *scratch, og_decision *out) {
    const og_graph *g = md->g;
    const int64_t B = md->B, r = md->b[v];
    const int64_t kout = g->op[v + 1] - g->op[v], kin = g->ip[v + 1] - g->ip[v], k = kout + kin;
    out->s = (int32_t)r; out->flags = 0; out->dH = 0.0; out->logA = 0.0; out->lnu = 0.0;
    if (k == 0) return; /* isolated vertex: no proposal */
    uint64_t ctr[4] = {sweep_id, (uint64_t)v, 0, 0}, key[2] = {seed, 0}, w[4];
    og_philox4x64(ctr, key, w);
    int64_t j = draw(w[0], k);
    int64_t nb = j < kout ? g->oc[g->op[v] + j] : g->ic[g->ip[v] + (j - kout)];
    int64_t u = md->b[nb];
    int64_t du = md->dout[u] + md->din[u];
    int64_t y = draw(w[1], du + B), s;
    if (y < B) s = y;
    else {
        int64_t t = y - B;
        if (t < md->dout[u]) s = row_pick(md, u, t, -1);
        else s = col_pick(md, u, t - md->dout[u], -1);
    }
    out->s = (int32_t)s;
    out->flags = 1;
    if (s == r) return; /* counted proposal, no move */
    double dH, pf, pb;
    move_delta(md, v, s, scratch, &dH, &pf, &pb);
    double logA = -beta * dH + log(pb) - log(pf);
    double uacc = (double)(w[2] >> 11) * 0x1.0p-53;
    double lnu = log(uacc);
    out->dH = dH;
    out->logA = logA;
    out->lnu = lnu;
    if (logA >= 0.0 || lnu < logA) out->flags |= 2;
}

/* One asynchronous-Gibbs pass (Section II-B, Alg. 5 with one rank per
 * vertex): every v in [v_begin, v_end) decides against the frozen model.
 * Writes b_new for that range only; the model is unchanged.  Optional
 * per-vertex outputs (full length n) may be NULL.  Returns accepted count. */
int64_t og_nodal_decide(const og_model *md, uint64_t seed, uint64_t sweep_id, double beta, int64_t v_begin, int64_t v_end,
                        int32_t *b_new, int32_t *s_out, int32_t *flags_out, double *dH_out, double *logA_out, double *lnu_out,
                        int nthreads) {
    const og_graph *g = md->g;
    int64_t maxk = 0;
    for (int64_t v = v_begin; v < v_end; ++v) {
        int64_t k = (g->op[v + 1] - g->op[v]) + (g->ip[v + 1] - g->ip[v]);
        if (k > maxk) maxk = k;
    }
    int64_t accepted = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads) reduction(+ : accepted)
    {
        nb_entry *sc = (nb_entry *)malloc(sizeof(nb_entry) * (size_t)(maxk > 0 ? maxk : 1));
#pragma omp for schedule(dynamic, 512)
        for (int64_t v = v_begin; v < v_end; ++v) {
            og_decision d;
            nodal_decide(md, seed, sweep_id, beta, v, sc, &d);
            b_new[v] = (d.flags & 2) ? d.s : md->b[v];
            if (d.flags & 2) accepted++;
            if (s_out) s_out[v] = d.s;
            if (flags_out) flags_out[v] = d.flags;
            if (dH_out) dH_out[v] = d.dH;
            if (logA_out) logA_out[v] = d.logA;
            if (lnu_out) lnu_out[v] = d.lnu;
        }
        free(sc);
    }
    return accepted;
}

/* Hybrid pass: the hybrid SBP the paper adopts for the work within a node
 * (Section II-B; Section III-B, "Hybrid SBP"): informative high-degree
 * vertices are processed sequentially, the rest by asynchronous Gibbs.  The
 * h vertices of largest degree k_v (ties: lower id first) are visited in that
 * order; each draws its proposal and is decided (Metropolis-Hastings, Alg. 2)
 * against the current model, and an accepted move is applied at once (labels
 * and M; here by recounting M, the plainest correct update).  Then every
 * other vertex decides against the model the sequential part left
 * (asynchronous Gibbs).  b_new receives every vertex's label (the sequential
 * vertices' current ones); the model holds the state after the sequential
 * part.  Optional outputs as og_nodal_decide, for all vertices.  Returns the
 * number of accepted moves. */
typedef struct { int64_t k, v; } deg_key;
static int cmp_deg(const void *a, const void *b) {
    const deg_key *x = (const deg_key *)a, *y = (const deg_key *)b;
    if (x->k != y->k) return x->k > y->k ? -1 : 1;
    return (x->v > y->v) - (x->v < y->v);
}

int64_t og_hybrid_decide(og_model *md, uint64_t seed, uint64_t sweep_id, double beta, int64_t h, int32_t *b_new,
                         int32_t *s_out, int32_t *flags_out, double *dH_out, double *logA_out, double *lnu_out,
                         int nthreads) {
    const og_graph *g = md->g;
    const int64_t n = g->n;
    if (h > n) h = n;
    if (h < 0) h = 0;
    deg_key *kv = (deg_key *)malloc(sizeof(deg_key) * (size_t)(n > 0 ? n : 1));
    int64_t maxk = 0;
    for (int64_t v = 0; v < n; ++v) {
        kv[v].k = (g->op[v + 1] - g->op[v]) + (g->ip[v + 1] - g->ip[v]);
        kv[v].v = v;
        if (kv[v].k > maxk) maxk = kv[v].k;
    }
    qsort(kv, (size_t)n, sizeof(deg_key), cmp_deg);
    unsigned char *seq = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
    nb_entry *sc = (nb_entry *)malloc(sizeof(nb_entry) * (size_t)(maxk > 0 ? maxk : 1));
    int32_t *bt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t accepted = 0;
    for (int64_t i = 0; i < h; ++i) {
        const int64_t v = kv[i].v;
        seq[v] = 1;
        og_decision d;
        nodal_decide(md, seed, sweep_id, beta, v, sc, &d);
        if (s_out) s_out[v] = d.s;
        if (flags_out) flags_out[v] = d.flags;
        if (dH_out) dH_out[v] = d.dH;
        if (logA_out) logA_out[v] = d.logA;
        if (lnu_out) lnu_out[v] = d.lnu;
        if (d.flags & 2) {
            accepted++;
            memcpy(bt, md->b, sizeof(int32_t) * (size_t)n);
            bt[v] = d.s;
            og_model_set_b(md, md->B, bt);
        }
    }
    free(sc);
    free(bt);
    memcpy(b_new, md->b, sizeof(int32_t) * (size_t)n);
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads) reduction(+ : accepted)
    {
        nb_entry *sc2 = (nb_entry *)malloc(sizeof(nb_entry) * (size_t)(maxk > 0 ? maxk : 1));
#pragma omp for schedule(dynamic, 512)
        for (int64_t v = 0; v < n; ++v) {
            if (seq[v]) continue;
            og_decision d;
            nodal_decide(md, seed, sweep_id, beta, v, sc2, &d);
            b_new[v] = (d.flags & 2) ? d.s : md->b[v];
            if (d.flags & 2) accepted++;
            if (s_out) s_out[v] = d.s;
            if (flags_out) flags_out[v] = d.flags;
            if (dH_out) dH_out[v] = d.dH;
            if (logA_out) logA_out[v] = d.logA;
            if (lnu_out) lnu_out[v] = d.lnu;
        }
        free(sc2);
    }
    free(seq);
    free(kv);
    return accepted;
}

/* ------------------------------------------------------------------------ */
/* P7. Block-merge proposal and merge Delta DL (Alg. 1 lines "propose" and
 * "calculate Delta DL"; Alg. 4).  u is the block at the far end of a random
 * edge of block r; s != r is drawn with probability proportional to
 * 1 + M[u][s] + M[s][u].  Blocks with no edges draw s uniformly. */
static int64_t merge_propose(const og_model *md, uint64_t seed, uint64_t round_id, int64_t r, int64_t i) {
    const int64_t B = md->B;
    uint64_t ctr[4] = {round_id, (uint64_t)r, (uint64_t)i, 0}, key[2] = {seed, 1}, w[4];
    og_philox4x64(ctr, key, w);
    int64_t dr = md->dout[r] + md->din[r];
    if (dr == 0) {
        int64_t y = draw(w[1], B - 1);
        return y + (y >= r);
    }
    int64_t t = draw(w[0], dr), u;
    if (t < md->dout[r]) u = row_pick(md, r, t, -1);
    else u = col_pick(md, r, t - md->dout[r], -1);
    int64_t Mur = M_at(md, u, r), Mru = M_at(md, r, u);
    int64_t W = (B - 1) + md->dout[u] + md->din[u] - Mur - Mru;
    int64_t y = draw(w[1], W);
    if (y < B - 1) return y + (y >= r);
    t = y - (B - 1);
    int64_t row_w = md->dout[u] - Mur;
    if (t < row_w) return row_pick(md, u, t, r);
    return col_pick(md, u, t - row_w, r);
}

/* Delta DL of merging block r into block s (the model term of Eq. 2 is the
 * same for every candidate and is left out).  Row and column r vanish; row
 * and column s absorb them. */
static double merge_delta(const og_model *md, int64_t r, int64_t s) {
    double dL = 0.0;
    /* row r: t not in {r, s}, ascending t */
    for (int64_t k = md->rptr[r]; k < md->rptr[r + 1]; ++k) {
        int64_t t = md->rk[k] % md->B;
        if (t == r || t == s) continue;
        dL += gmerge(M_at(md, s, t), md->rc[k]);
    }
    /* column r: t not in {r, s}, ascending t */
    for (int64_t k = md->cptr[r]; k < md->cptr[r + 1]; ++k) {
        int64_t t = md->ck[k] % md->B;
        if (t == r || t == s) continue;
        dL += gmerge(M_at(md, t, s), md->cc[k]);
    }
    int64_t a = M_at(md, r, r), b = M_at(md, r, s), c = M_at(md, s, r), d = M_at(md, s, s);
    dL += gmerge(a, b) + gmerge(a + b, c) + gmerge(a + b + c, d);
    dL -= gmerge(md->dout[s], md->dout[r]) + gmerge(md->din[s], md->din[r]);
    return -dL;
}

double og_merge_delta(const og_model *md, int64_t r, int64_t s) { return merge_delta(md, r, s); }

int64_t og_merge_propose(const og_model *md, uint64_t seed, uint64_t round_id, int64_t r, int64_t i) {
    if (md->B < 2 || r < 0 || r >= md->B) return -1;
    return merge_propose(md, seed, round_id, r, i);
}

/* Scores compare on a 2^-20-nat grid; equal grid values count as ties. */
int64_t og_merge_key(double dDL) { return (int64_t)floor(dDL * 1048576.0 + 0.5); }

/* For every block r: x proposals, keep the best (smallest Delta DL, the
 * earliest proposal on a tie).  Alg. 1 / Alg. 4, "store c' and Delta DL". */
void og_merge_proposals(const og_model *md, uint64_t seed, uint64_t round_id, int64_t x, int32_t *best_s, double *best_dDL, int nthreads) {
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 64)
    for (int64_t r = 0; r < md->B; ++r) {
        int64_t bs = -1;
        double bd = 0.0;
        for (int64_t i = 0; i < x; ++i) {
            int64_t s = merge_propose(md, seed, round_id, r, i);
            double d = merge_delta(md, r, s);
            if (bs < 0 || og_merge_key(d) < og_merge_key(bd)) { bs = s; bd = d; }
        }
        best_s[r] = (int32_t)bs;
        best_dDL[r] = bd;
    }
}

/* ------------------------------------------------------------------------ */
/* P8. Merge application (Alg. 1 "sort best_merges", "repeat ... pop, merge
 * c into c' until the number of communities is halved"; Section III-A (d)
 * pointer-based tracking of merges).  Merges are taken in ascending
 * (score key, r); each one links the group holding r under the group holding
 * s unless both are already one group.  Stops after n_merges links.  Writes
 * the dense relabelling map[B] (groups numbered by their smallest member) and
 * returns the number of links made. */
static int64_t uf_find(int64_t *parent, int64_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

typedef struct { int64_t key, r; } merge_item;
static int cmp_merge(const void *a, const void *b) {
    const merge_item *x = (const merge_item *)a, *y = (const merge_item *)b;
    if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
    return (x->r > y->r) - (x->r < y->r);
}

int64_t og_merge_apply(int64_t B, const int32_t *best_s, const double *best_dDL, int64_t n_merges, int32_t *map, int64_t *B_new) {
    merge_item *it = (merge_item *)malloc(sizeof(merge_item) * (size_t)B);
    for (int64_t r = 0; r < B; ++r) { it[r].key = og_merge_key(best_dDL[r]); it[r].r = r; }
    qsort(it, (size_t)B, sizeof(merge_item), cmp_merge);
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)B);
    for (int64_t c = 0; c < B; ++c) parent[c] = c;
    int64_t done = 0;
    for (int64_t k = 0; k < B && done < n_merges; ++k) {
        int64_t r = it[k].r, s = best_s[r];
        if (s < 0) continue;
        int64_t a = uf_find(parent, r), c = uf_find(parent, s);
        if (a == c) continue;
        parent[a] = c;
        done++;
    }
    /* groups numbered in ascending order of their smallest member */
    int64_t *label_of_root = (int64_t *)malloc(sizeof(int64_t) * (size_t)B);
    for (int64_t c = 0; c < B; ++c) label_of_root[c] = -1;
    int64_t next = 0;
    for (int64_t c = 0; c < B; ++c) {
        int64_t root = uf_find(parent, c);
        if (label_of_root[root] < 0) label_of_root[root] = next++;
        map[c] = (int32_t)label_of_root[root];
    }
    *B_new = next;
    free(label_of_root); free(parent); free(it);
    return done;
}

/* Drop labels with no vertex and renumber the rest densely, ascending. */
int64_t og_compact(int64_t n, int64_t B, int32_t *b) {
    int32_t *map = (int32_t *)malloc(sizeof(int32_t) * (size_t)B);
    for (int64_t c = 0; c < B; ++c) map[c] = -1;
    for (int64_t v = 0; v < n; ++v) map[b[v]] = 0;
    int64_t next = 0;
    for (int64_t c = 0; c < B; ++c)
        if (map[c] == 0) map[c] = (int32_t)next++;
    for (int64_t v = 0; v < n; ++v) b[v] = map[b[v]];
    free(map);
    return next;
}

/* ------------------------------------------------------------------------ */
/* P9. Golden-ratio search over the number of communities (Section II-B):
 * keep up to three (C, DL, assignment) states hi > mid > lo by C. */
typedef struct {
    int64_t B[3];   /* 0 hi, 1 mid, 2 lo; 0 = empty */
    double dl[3];
    int32_t *b[3];
} og_bracket;

static void bracket_put(og_bracket *k, int idx, int64_t B, double dl, const int32_t *b, int64_t n) {
    k->B[idx] = B;
    k->dl[idx] = dl;
    if (!k->b[idx]) k->b[idx] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (b) memcpy(k->b[idx], b, sizeof(int32_t) * (size_t)n);
}
static void bracket_move(og_bracket *k, int to, int from) {
    int32_t *tmp = k->b[to];
    k->B[to] = k->B[from]; k->dl[to] = k->dl[from]; k->b[to] = k->b[from];
    k->b[from] = tmp;
}

/* Insert a new state: a new best becomes mid and the old mid moves to hi or
 * lo by C; otherwise the new state replaces hi or lo by C. */
static void bracket_insert(og_bracket *k, int64_t B, double dl, const int32_t *b, int64_t n) {
    if (k->B[1] == 0) { bracket_put(k, 1, B, dl, b, n); return; }
    if (dl < k->dl[1]) {
        if (k->B[1] > B) bracket_move(k, 0, 1); else bracket_move(k, 2, 1);
        bracket_put(k, 1, B, dl, b, n);
    } else {
        if (B > k->B[1]) bracket_put(k, 0, B, dl, b, n); else bracket_put(k, 2, B, dl, b, n);
    }
}

/* Next step: (start index, target C).  Returns 0 when done. */
static int bracket_next(const og_bracket *k, double reduction, int *start, int64_t *target) {
    if (k->B[2] == 0) {
        int64_t nm = (int64_t)floor((double)k->B[1] * reduction);
        if (nm > k->B[1] - 1) nm = k->B[1] - 1;
        if (nm < 1) return 0;
        *start = 1;
        *target = k->B[1] - nm;
        return 1;
    }
    if (k->B[0] - k->B[2] <= 2) return 0;
    int64_t up_gap = k->B[0] - k->B[1], low_gap = k->B[1] - k->B[2];
    int64_t upper, lower;
    if (up_gap >= low_gap) { *start = 0; upper = k->B[0]; lower = k->B[1]; }
    else { *start = 1; upper = k->B[1]; lower = k->B[2]; }
    int64_t t = upper - (int64_t)llround(0.618 * (double)(upper - lower));
    if (t >= upper) t = upper - 1;
    if (t <= lower) t = lower + 1;
    *target = t;
    return 1;
}

/* Standalone access to the bracket rule for tests: feed (B, DL) pairs,
 * read back the bracket and the next step. */
typedef struct { og_bracket k; } og_bracket_handle;
og_bracket_handle *og_bracket_new(void) { return (og_bracket_handle *)calloc(1, sizeof(og_bracket_handle)); }
void og_bracket_free(og_bracket_handle *h) {
    if (!h) return;
    for (int i = 0; i < 3; ++i) free(h->k.b[i]);
    free(h);
}
void og_bracket_insert(og_bracket_handle *h, int64_t B, double dl) { bracket_insert(&h->k, B, dl, NULL, 0); }
int og_bracket_next(og_bracket_handle *h, double reduction, int64_t *Bs, double *dls, int *start, int64_t *target) {
    for (int i = 0; i < 3; ++i) { Bs[i] = h->k.B[i]; dls[i] = h->k.dl[i]; }
    return bracket_next(&h->k, reduction, start, target);
}

typedef struct {
    uint64_t seed;
    double beta;
    int64_t merge_proposals;
    double reduction;
    double t_pre, t_post;
    int64_t max_sweeps;
    int64_t hybrid_h;     /* > 0: hybrid passes while B <= dense_max_B */
    int64_t dense_max_B;
} og_params;

/* Merge phase: from state b with B blocks, reach B - n_merges blocks.  When
 * a round of proposals runs out before n_merges links, the merged model is
 * rebuilt and a new round (new round_id) proposes again.  *rounds (may be
 * NULL) receives the number of proposal rounds taken. */
static int64_t merge_phase(og_model *md, const og_params *p, uint64_t *round_id, int64_t n_merges, int nthreads,
                           int64_t *rounds) {
    const og_graph *g = md->g;
    int64_t nr = 0;
    while (n_merges > 0) {
        int64_t B = md->B;
        int32_t *bs = (int32_t *)malloc(sizeof(int32_t) * (size_t)B);
        double *bd = (double *)malloc(sizeof(double) * (size_t)B);
        int32_t *map = (int32_t *)malloc(sizeof(int32_t) * (size_t)B);
        og_merge_proposals(md, p->seed, (*round_id)++, p->merge_proposals, bs, bd, nthreads);
        nr++;
        int64_t Bn;
        int64_t done = og_merge_apply(B, bs, bd, n_merges, map, &Bn);
        int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * (size_t)g->n);
        for (int64_t v = 0; v < g->n; ++v) nb[v] = map[md->b[v]];
        og_model_set_b(md, Bn, nb);
        free(nb); free(map); free(bd); free(bs);
        n_merges -= done;
        if (done == 0) break;
    }
    if (rounds) *rounds = nr;
    return md->B;
}

/* MCMC phase (Alg. 2 with the asynchronous-Gibbs pass, or the hybrid pass
 * while B <= dense_max_B when hybrid_h > 0): sweeps until
 * |DL_{k-3} - DL_k| < t DL_k (k >= 3) or max_sweeps.  hist (may be NULL,
 * else max_sweeps + 1 entries) receives DL_0 (the start) .. DL_k. */
static int64_t mcmc_phase(og_model *md, const og_params *p, uint64_t *sweep_id, double t, int nthreads, double *hist_out) {
    const og_graph *g = md->g;
    double *hist = (double *)malloc(sizeof(double) * (size_t)(p->max_sweeps + 1));
    int32_t *bn = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n > 0 ? g->n : 1));
    hist[0] = og_model_dl(md);
    int64_t k;
    for (k = 1; k <= p->max_sweeps; ++k) {
        memcpy(bn, md->b, sizeof(int32_t) * (size_t)g->n);
        if (p->hybrid_h > 0 && md->B <= p->dense_max_B)
            og_hybrid_decide(md, p->seed, (*sweep_id)++, p->beta, p->hybrid_h, bn, NULL, NULL, NULL, NULL, NULL, nthreads);
        else
            og_nodal_decide(md, p->seed, (*sweep_id)++, p->beta, 0, g->n, bn, NULL, NULL, NULL, NULL, NULL, nthreads);
        og_model_set_b(md, md->B, bn);
        hist[k] = og_model_dl(md);
        if (k >= 3 && fabs(hist[k - 3] - hist[k]) < t * hist[k]) break;
    }
    int64_t done = k > p->max_sweeps ? p->max_sweeps : k;
    if (hist_out) memcpy(hist_out, hist, sizeof(double) * (size_t)(done + 1));
    free(bn);
    free(hist);
    return done;
}

/* The two phases on their own, for the tests of their stopping rules. */
int64_t og_mcmc_phase(og_model *md, const og_params *p, uint64_t sweep_id, double t, int nthreads, double *hist) {
    return mcmc_phase(md, p, &sweep_id, t, nthreads, hist);
}

int64_t og_merge_phase(og_model *md, const og_params *p, uint64_t round_id, int64_t n_merges, int nthreads,
                       int64_t *rounds) {
    return merge_phase(md, p, &round_id, n_merges, nthreads, rounds);
}

/* Full run (Fig. 1, Section II-B): start from one block per vertex,
 * alternate merge and MCMC phases under the golden-ratio search.  log (may
 * be NULL, else log_cap rows of 7 doubles) receives one row per phase:
 * start B, target B, B after the merges, MCMC threshold t, sweeps, and the
 * compacted B and its DL inserted into the bracket; *n_log the number of
 * phases. */
int og_partition(const og_graph *g, const og_params *p, int32_t *b_out, int64_t *B_out, double *dl_out, int64_t *n_sweeps_out,
                 int nthreads, double *log, int64_t log_cap, int64_t *n_log) {
    const int64_t n = g->n;
    int32_t *b = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t v = 0; v < n; ++v) b[v] = (int32_t)v;
    og_model *md = og_model_new(g, n, b);
    if (!md) { free(b); return -1; }
    og_bracket k;
    memset(&k, 0, sizeof(k));
    bracket_insert(&k, n, og_model_dl(md), b, n);
    uint64_t sweep_id = 0, round_id = 0;
    int64_t total_sweeps = 0, phases = 0;
    int start;
    int64_t target;
    while (bracket_next(&k, p->reduction, &start, &target)) {
        int64_t B0 = k.B[start];
        double t = k.B[2] == 0 ? p->t_pre : p->t_post;
        og_model_set_b(md, B0, k.b[start]);
        merge_phase(md, p, &round_id, B0 - target, nthreads, NULL);
        int64_t Bm = md->B;
        int64_t ns = mcmc_phase(md, p, &sweep_id, t, nthreads, NULL);
        total_sweeps += ns;
        memcpy(b, md->b, sizeof(int32_t) * (size_t)n);
        int64_t Bc = og_compact(n, md->B, b);
        og_model_set_b(md, Bc, b);
        double dlc = og_model_dl(md);
        bracket_insert(&k, Bc, dlc, b, n);
        if (log && phases < log_cap) {
            double *row = log + 7 * phases;
            row[0] = (double)B0; row[1] = (double)target; row[2] = (double)Bm;
            row[3] = t; row[4] = (double)ns; row[5] = (double)Bc; row[6] = dlc;
        }
        phases++;
    }
    if (n_log) *n_log = phases;
    memcpy(b_out, k.b[1], sizeof(int32_t) * (size_t)n);
    *B_out = k.B[1];
    *dl_out = k.dl[1];
    if (n_sweeps_out) *n_sweeps_out = total_sweeps;
    og_model_free(md);
    for (int i = 0; i < 3; ++i) free(k.b[i]);
    free(b);
    return 0;
}

int og_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
