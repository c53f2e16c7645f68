// apply.cuh -- device pieces of the apply step (Alg. 5: apply the moves,
// make the blockmodel consistent) and of the DL (Eq. 1-2), shared by the
// per-graph kernels (blockmodel.cu) and the batched MCMC kernel (batch.cu).
#pragma once

#include <cmath>

#include "common.cuh"

namespace sbp {
namespace {

// Incremental apply on a dense M: every edge with a moved end leaves its old
// (block, block) cell and enters the new one.  An edge is visited once:
// through the out-row of its moved source, or through the in-row of its
// moved target when the source stayed.  Lanes take the edges of one row,
// four loads in flight per lane.
// (a dense M has B <= 16384, so a cell index fits 32 bits)
__device__ __forceinline__ void delta_add(int32_t *__restrict__ M, bool valid, int key, int d) {
    if (valid) atomicAdd(&M[key], d);
}

// out-row [a, z) of a vertex moved r -> s
__device__ __forceinline__ void delta_out_row(const int32_t *__restrict__ oc, int a, int z, int r, int s,
                                              const int32_t *__restrict__ bnew, const int32_t *__restrict__ bold,
                                              int32_t *__restrict__ M, int B) {
    const int lane = threadIdx.x & 31;
    for (int e0 = a; e0 < z; e0 += 128) {
        int w[4], t[4], u[4];
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = e0 + 32 * j + lane;
            ok[j] = e < z;
            w[j] = ok[j] ? oc[e] : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            t[j] = ok[j] ? bold[w[j]] : 0;
            u[j] = ok[j] ? bnew[w[j]] : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            delta_add(M, ok[j], r * B + t[j], -1);
            delta_add(M, ok[j], s * B + u[j], 1);
        }
    }
}

// in-row [a, z) of a vertex moved r -> s; only sources that stayed
__device__ __forceinline__ void delta_in_row(const int32_t *__restrict__ ic, int a, int z, int r, int s,
                                             const int32_t *__restrict__ bnew, const int32_t *__restrict__ bold,
                                             int32_t *__restrict__ M, int B) {
    const int lane = threadIdx.x & 31;
    for (int e0 = a; e0 < z; e0 += 128) {
        int w[4], t[4];
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = e0 + 32 * j + lane;
            ok[j] = e < z;
            w[j] = ok[j] ? ic[e] : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            t[j] = ok[j] ? bold[w[j]] : 0;
            ok[j] = ok[j] && bnew[w[j]] == t[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            delta_add(M, ok[j], t[j] * B + r, -1);
            delta_add(M, ok[j], t[j] * B + s, 1);
        }
    }
}

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += x;
    }
    return v;
}

// One warp, block u of a dense M: P[u] = inclusive prefix of row u, then
// dout_u plus the inclusive prefix of column u (the proposal CDFs); the 32
// pivots Pc[u]; degrees and the reciprocals of d_u + B.
// (M through plain loads: the batched MCMC kernel has just updated it)
__device__ __forceinline__ void prefix_block(const int32_t *M, int B, int u, uint32_t *__restrict__ P,
                                             int32_t *__restrict__ dout, int32_t *__restrict__ din,
                                             double *__restrict__ rcp, float *__restrict__ rcp32,
                                             int32_t *__restrict__ dsum, uint32_t *__restrict__ Pc, int pstep) {
    const int lane = threadIdx.x & 31;
    uint32_t *row = P + (size_t)u * 2 * B;
    uint32_t carry = 0;
    for (int c0 = 0; c0 < B; c0 += 32) {
        const int c = c0 + lane;
        uint32_t v = c < B ? (uint32_t)M[(size_t)u * B + c] : 0u;
        v = warp_incl_scan_u32(v) + carry;
        if (c < B) row[c] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
    const uint32_t du_out = carry;
    for (int c0 = 0; c0 < B; c0 += 32) {
        const int c = c0 + lane;
        uint32_t v = c < B ? (uint32_t)M[(size_t)c * B + u] : 0u;
        v = warp_incl_scan_u32(v) + carry;
        if (c < B) row[B + c] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
    __syncwarp();
    const int pi = (lane + 1) * pstep - 1 < 2 * B - 1 ? (lane + 1) * pstep - 1 : 2 * B - 1;
    Pc[(size_t)u * 32 + lane] = row[pi];
    if (lane == 0) {
        const uint32_t du_in = carry - du_out;
        dout[u] = (int32_t)du_out;
        din[u] = (int32_t)du_in;
        rcp[u] = 1.0 / ((double)du_out + (double)du_in + (double)B);
        rcp32[u] = 1.0f / ((float)du_out + (float)du_in + (float)B);
        dsum[u] = (int32_t)(du_out + du_in);
    }
}

struct DlPartial {
    __int128 fix;  // sum of x ln x * 2^64 over counts inside the table
    double fb;     // FP64 sum over counts beyond it
    double pad;
};

__device__ __forceinline__ void add_xlogx(const __int128 *__restrict__ T, int64_t XT, int64_t x, int sign, __int128 &fix,
                                          double &fb) {
    if (x < 2) return;
    if (x < XT) fix += sign > 0 ? T[x] : -T[x];
    else fb += sign * ((double)x * log((double)x));
}

// Eq. 2 from L (Eq. 1): DL = E h(B^2/E) + N ln B - L with
// h(x) = (1+x) ln(1+x) - x ln x, the E = 0 limit taken as 0
__device__ __forceinline__ double dl_eq2(int64_t E, int64_t N, int B, double L) {
    double model = 0.0;
    if (E > 0) {
        const double x = (double)B * (double)B / (double)E;
        model = (double)E * ((1.0 + x) * log1p(x) - x * log(x));
    }
    return model + (double)N * log((double)B) - L;
}

}  // namespace
}  // namespace sbp
