// fused.cu -- the hot path: one persistent kernel runs Algorithm 1 (Sec. 3.3) for
// whole days, rebuilding each day's DAR (Eq. (dar)) from its tick table on chip
// in every pass instead of reading a materialised matrix.
//
// Work decomposition.  A CTA takes a day from a device work queue and runs all
// of that day's epochs before taking the next one (days are independent
// problems, Sec. 2.7).  One epoch is a forward sweep and an adjoint sweep:
//
//  * A task is (OD pair, tile of 31 departure intervals).  Its warp walks every
//    route of the OD; lane l follows the leading vehicle that departs at
//    boundary b0 + l (Example "DAR matrix computation").  At each link the lane's
//    entry time T_j(b) and its right neighbour's T_j(b+1) (one shuffle) bound
//    the window of Eq. (dar); the entry interval selects the link time from the
//    tick table (Sec. 2.4, Eq. (cost)).  The route's links are held in registers
//    as precomputed shared-memory offsets and broadcast by shuffles, so a link
//    step touches memory only for the tick lookup and the window's one or two
//    link-interval cells.  The OD / route tables sit in shared memory.
//  * Both sweeps run in phases of F tiles in time order.  A phase stages the
//    tick rows its trajectories can reach (departure rows plus the day's
//    largest trip offset, padded past the end of the day with the last row)
//    from global memory into shared memory.
//  * Forward sweep (xhat = B q, Eq. (reverse) with (flow)): windows deposit
//    p q rho into link-interval accumulators held as 64-bit fixed point
//    (2^-20 vehicles): the low word in shared memory with native integer
//    atomics, the rare carries in a per-CTA high word in global memory.  Sums
//    are exact and independent of the deposit order, so results are bitwise
//    reproducible.  After a phase every interval before the next phase's first
//    departure is final (no vehicle arrives before it departs): those rows
//    become masked residuals r = m (xhat - x), are summed into the loss
//    (Eq. (nnls)) and are written to the CTA's residual slot (global,
//    L2-resident); the rows that spill into the next phase move to the front.
//  * Adjoint sweep (g = B^T r, Algorithm 1's gradient): a phase stages the
//    residual rows its windows can reach back into shared memory, the same walk
//    gathers r over each window, route sums are combined with the route choice
//    of Eq. (logit), and the Adagrad step and projection max(q, 0) are applied in
//    place -- every (OD, interval) belongs to exactly one lane.
//
// Days whose trajectories needed FIFO repairs read the exact repaired
// trajectories from a per-day table built once by the prepare kernel; all other
// days walk the tick table directly (which is then exact).  When the shared
// windows do not fit (very many links, long trips or ticks above 16 bits) the
// same code reads ticks and residuals from global memory and accumulates link
// flows with global float atomics.  No CTA ever waits on another CTA: the work
// queue is a single atomicAdd.
#include <climits>

#include "dode_internal.cuh"

namespace dode {

constexpr int kInactive = INT_MIN;
constexpr float kFxScale = 1048576.f;          // 2^20: fixed-point unit of the accumulators
constexpr double kFxInv = 1.0 / 1048576.0;

template <int PREC>
struct Operand;

template <>
struct Operand<0> {
    __device__ static __forceinline__ float q(const FusedParams &p, size_t i) { return p.q[i]; }
    __device__ static __forceinline__ float r(const void *rb, size_t i) {
        return static_cast<const float *>(rb)[i];
    }
    __device__ static __forceinline__ void store_r(void *rb, size_t i, float v) {
        static_cast<float *>(rb)[i] = v;
    }
};

template <>
struct Operand<1> {
    __device__ static __forceinline__ float q(const FusedParams &p, size_t i) {
        return __bfloat162float(p.qb[i]);
    }
    __device__ static __forceinline__ float r(const void *rb, size_t i) {
        return __bfloat162float(static_cast<const __nv_bfloat16 *>(rb)[i]);
    }
    __device__ static __forceinline__ void store_r(void *rb, size_t i, float v) {
        static_cast<__nv_bfloat16 *>(rb)[i] = __float2bfloat16_rn(v);
    }
};

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

struct Shared {
    uint32_t *lo;         // [O][R]: accumulator low words (forward) / residual window as float bits (adjoint)
    int *hi;              // [O][R] in global memory: accumulator high words (forward)
    uint16_t *tw;         // [A][RW]: tick window (row = h - pb)
    const uint32_t *colact;
    const int4 *rinfo;    // [P] OD-major: (route, first link, links, 0)
    const int2 *odr;      // [K] route range of each OD in rinfo
    const int *task_od;   // [K] processing order
    int *carry;           // set once any deposit of this CTA carried into a high word
    int R, RW, pb;
};

// Route links in registers: lane j holds, for link j (and j + 32) of the route,
// the offset of its tick row and of its accumulator row (kInactive when the
// link is unobserved or has no observation this day), both relative to pb.
struct RouteRegs {
    int t0, o0, t1, o1;
};

template <bool SMEM_RING, bool SMEM_TICKS>
__device__ __forceinline__ RouteRegs load_route(const FusedParams &p, const Shared &s, int l0, int beta) {
    const int lane = threadIdx.x & 31;
    RouteRegs r{0, kInactive, 0, kInactive};
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int j = lane + 32 * half;
        if (j < beta && (half == 0 || beta > 32)) {
            const int2 ao = __ldg(&p.rpack[l0 + j]);
            const int a = ao.x, o = ao.y;
            const int tb = SMEM_TICKS ? a * s.RW - s.pb : a * p.Np;
            int ob = kInactive;
            if (o >= 0 && ((s.colact[o >> 5] >> (o & 31)) & 1u)) ob = SMEM_RING ? o * s.R - s.pb : o * p.Np;
            if (half == 0) {
                r.t0 = tb;
                r.o0 = ob;
            } else {
                r.t1 = tb;
                r.o1 = ob;
            }
        }
    }
    return r;
}

// Route choice of Eq. (logit) at the lane's departure interval from the route
// times (differentiable form): shift m and reciprocal normaliser.
__device__ __forceinline__ void logit_norm(const FusedParams &p, const Shared &s, const float *Cday, int r0, int r1,
                                           int bi, float &m, float &rden) {
    m = -INFINITY;
    for (int i = r0; i < r1; ++i) m = fmaxf(m, -p.theta * Cday[(size_t)s.rinfo[i].x * p.Np + bi]);
    float den = 0.f;
    for (int i = r0; i < r1; ++i) den += expf(-p.theta * Cday[(size_t)s.rinfo[i].x * p.Np + bi] - m);
    rden = 1.f / den;
}

// Shares of a window [T, hi) of width w over the arrival intervals (Eq. (dar)).
// d0, the share of the interval h0 that contains T, is min(1, (e0 - T) / w) with
// e0 the end of h0 (a zero-length window gives 1).  When the window ends in the
// next interval its share is 1 - d0; longer windows (the travel time jumped by
// more than an interval between consecutive departures) take the loop in
// window_tail.  BF16 form: shares are rounded to BF16 and the last share of a
// window is the remainder, so each departure's mass is conserved.
template <int PREC>
__device__ __forceinline__ float first_share(int T, int e0, float inv) {
    const float d = fminf(1.f, (float)(e0 - T) * inv);
    if (PREC == 0) return d;
    return d < 1.f ? bf16_round(d) : 1.f;
}

// Add v to accumulator cell idx: 64-bit fixed point (shared low word, carries
// into the global high word) or a global float when the ring is not in shared
// memory.
// FAST: the caller guarantees 0 <= v < 3000 (then v 2^20 fits 32 unsigned bits).
template <bool SMEM_RING, bool FAST = false>
__device__ __forceinline__ void deposit(const Shared &s, float *gacc, int idx, float v) {
    if (!SMEM_RING) {
        atomicAdd(gacc + idx, v);
        return;
    }
    const float sv = v * kFxScale;
    if (FAST || (sv >= 0.f && sv < 4.0e9f)) {
        const uint32_t u = __float2uint_rn(sv);
        const uint32_t old = atomicAdd(&s.lo[idx], u);
        if (old + u < old) {
            atomicAdd(&s.hi[idx], 1);
            *s.carry = 1;
        }
        return;
    }
    const long long fx = __float2ll_rn(sv);
    const uint32_t u = (uint32_t)fx;
    const uint32_t old = atomicAdd(&s.lo[idx], u);
    const int dh = (int)(fx >> 32) + ((old + u < old) ? 1 : 0);
    if (dh) {
        atomicAdd(&s.hi[idx], dh);
        *s.carry = 1;
    }
}

// Cells h0 + 1 .. of a window spanning three or more intervals.  Forward:
// deposits f * share; adjoint: returns sum share * r.
template <int PREC, bool SMEM_RING, bool DEPOSIT>
__device__ __noinline__ float window_tail(const Shared &s, float *gacc, const void *rb, int idx, int hi, int e,
                                          int h, int N, int ipt, float inv, float used, float f) {
    float acc = 0.f;
    while (hi > e && h < N) {
        const int end = min(hi, e + ipt);
        float share;
        if (PREC == 0) {
            share = (float)(end - e) * inv;
        } else {
            share = end >= hi ? 1.f - used : bf16_round((float)(end - e) * inv);
            used += share;
        }
        if (DEPOSIT)
            deposit<SMEM_RING>(s, gacc, idx, f * share);
        else
            acc += share * (SMEM_RING ? __uint_as_float(s.lo[idx]) : Operand<PREC>::r(rb, (size_t)idx));
        ++idx;
        e += ipt;
        ++h;
    }
    return acc;
}

template <bool SMEM_TICKS, bool TAB>
__device__ __forceinline__ int next_entry(const FusedParams &p, const Shared &s, const int32_t *tick_day,
                                          const int32_t *trow, int j, int T, int tb, int h0) {
    if (TAB) return __ldg(&trow[(size_t)(j + 1) * (p.N + 1)]);
    if (SMEM_TICKS) return T + s.tw[tb + h0];
    return T + __ldg(&tick_day[tb + min(h0, p.N - 1)]);
}

// One route's forward walk: deposit f rho of every window on observed links.
// FAST: every f of the warp lies in [0, 3000), so each deposit f * share does too.
template <int PREC, bool SMEM_RING, bool SMEM_TICKS, bool TAB, bool FAST>
__device__ __forceinline__ void forward_walk(const FusedParams &p, const Shared &s, const int32_t *tick_day,
                                             const int32_t *trow, const RouteRegs &rr, float *gacc, int beta, int bb,
                                             bool vw, float f) {
    const int ipt = p.div.ipt, N = p.N;
    int T = ipt * bb;
    for (int j = 0; j < beta; ++j) {
        const int tb = __shfl_sync(0xffffffffu, j < 32 ? rr.t0 : rr.t1, j & 31);
        const int ob = __shfl_sync(0xffffffffu, j < 32 ? rr.o0 : rr.o1, j & 31);
        const int hi = __shfl_down_sync(0xffffffffu, T, 1);
        const int h0 = interval_of(T, p.div);
        if (ob != kInactive) {
            if (vw && h0 < N) {
                const int idx = ob + h0;
                const int e0 = h0 * ipt + ipt;
                const float inv = __fdividef(1.f, (float)(hi - T));
                const float d0 = first_share<PREC>(T, e0, inv);
                const float c0 = f * d0;
                deposit<SMEM_RING, FAST>(s, gacc, idx, c0);
                if (hi > e0 && h0 + 1 < N) {
                    if (hi <= e0 + ipt)
                        deposit<SMEM_RING, FAST>(s, gacc, idx + 1, f - c0);
                    else
                        window_tail<PREC, SMEM_RING, true>(s, gacc, nullptr, idx + 1, hi, e0, h0 + 1, N, ipt, inv, d0,
                                                           f);
                }
            }
        }
        T = next_entry<SMEM_TICKS, TAB>(p, s, tick_day, trow, j, T, tb, h0);
    }
}

template <int PREC, bool SMEM_RING, bool SMEM_TICKS, bool TAB>
__device__ void forward_task(const FusedParams &p, const Shared &s, int day, int od, int b0,
                             const int32_t *tab) {
    const int lane = threadIdx.x & 31;
    const int b = b0 + lane;
    const int bb = min(b, p.N);
    const bool vw = (lane < kTileW) && (b < p.N);
    const int bi = min(b, p.N - 1);
    const int32_t *tick_day = p.ticks + (size_t)day * p.A * p.Np;
    const int2 rr0 = s.odr[od];
    const float qv = vw ? Operand<PREC>::q(p, ((size_t)day * p.K + od) * p.Np + b) : 0.f;
    if (!__any_sync(0xffffffffu, qv != 0.f)) return;     // nothing departs: no deposits
    float *gacc = SMEM_RING ? nullptr : p.gring + (size_t)blockIdx.x * p.O * p.Np;
    for (int i = rr0.x; i < rr0.y; ++i) {
        const int4 ri = s.rinfo[i];
        const int k = ri.x, l0 = ri.y, beta = ri.z;
        const float f = __ldg(&p.pt[((size_t)day * p.P + k) * p.Np + bi]) * qv;
        const RouteRegs rr = load_route<SMEM_RING, SMEM_TICKS>(p, s, l0, beta);
        const int32_t *trow = TAB ? tab + (size_t)(l0 + k) * (p.N + 1) + bb : nullptr;
        if (__all_sync(0xffffffffu, f >= 0.f && f < 3000.f))
            forward_walk<PREC, SMEM_RING, SMEM_TICKS, TAB, true>(p, s, tick_day, trow, rr, gacc, beta, bb, vw, f);
        else
            forward_walk<PREC, SMEM_RING, SMEM_TICKS, TAB, false>(p, s, tick_day, trow, rr, gacc, beta, bb, vw, f);
    }
}

template <int PREC, bool SMEM_RING, bool SMEM_TICKS, bool TAB>
__device__ void adjoint_task(const FusedParams &p, const Shared &s, int day, int od, int b0, const void *rb,
                             const int32_t *tab, double *s_dth) {
    const int lane = threadIdx.x & 31;
    const int b = b0 + lane;
    const int bb = min(b, p.N);
    const bool vw = (lane < kTileW) && (b < p.N);
    const int bi = min(b, p.N - 1);
    const int32_t *tick_day = p.ticks + (size_t)day * p.A * p.Np;
    const int2 rr0 = s.odr[od];
    const int ipt = p.div.ipt, N = p.N;
    const size_t qi = ((size_t)day * p.K + od) * p.Np + b;
    const bool grad = p.mode == MODE_LOSS_GRAD;
    const float *Cday = p.C + (size_t)day * p.P * p.Np;
    float m = 0.f, rden = 1.f;
    if (grad) logit_norm(p, s, Cday, rr0.x, rr0.y, bi, m, rden);
    const float *racc = SMEM_RING ? reinterpret_cast<const float *>(s.lo) : nullptr;
    float g = 0.f;
    double dth = 0.0;
    for (int i = rr0.x; i < rr0.y; ++i) {
        const int4 ri = s.rinfo[i];
        const int k = ri.x, l0 = ri.y, beta = ri.z;
        float pk, ck = 0.f;
        if (grad) {
            ck = Cday[(size_t)k * p.Np + bi];
            pk = expf(-p.theta * ck - m) * rden;
        } else {
            pk = __ldg(&p.pt[((size_t)day * p.P + k) * p.Np + bi]);
        }
        const RouteRegs rr = load_route<SMEM_RING, SMEM_TICKS>(p, s, l0, beta);
        const int32_t *trow = TAB ? tab + (size_t)(l0 + k) * (N + 1) + bb : nullptr;
        float gp = 0.f;
        int T = ipt * bb;
        for (int j = 0; j < beta; ++j) {
            const int tb = __shfl_sync(0xffffffffu, j < 32 ? rr.t0 : rr.t1, j & 31);
            const int ob = __shfl_sync(0xffffffffu, j < 32 ? rr.o0 : rr.o1, j & 31);
            const int hi = __shfl_down_sync(0xffffffffu, T, 1);
            const int h0 = interval_of(T, p.div);
            if (ob != kInactive) {
                if (vw && h0 < N) {
                    const int idx = ob + h0;
                    const int e0 = h0 * ipt + ipt;
                    const float inv = __fdividef(1.f, (float)(hi - T));
                    const float d0 = first_share<PREC>(T, e0, inv);
                    float a = d0 * (SMEM_RING ? racc[idx] : Operand<PREC>::r(rb, (size_t)idx));
                    if (hi > e0 && h0 + 1 < N) {
                        if (hi <= e0 + ipt)
                            a += (1.f - d0) * (SMEM_RING ? racc[idx + 1] : Operand<PREC>::r(rb, (size_t)idx + 1));
                        else
                            a += window_tail<PREC, SMEM_RING, false>(s, nullptr, rb, idx + 1, hi, e0, h0 + 1, N, ipt,
                                                                     inv, d0, 0.f);
                    }
                    gp += a;
                }
            }
            T = next_entry<SMEM_TICKS, TAB>(p, s, tick_day, trow, j, T, tb, h0);
        }
        g += pk * gp;
        if (grad && vw) {
            // dp_k/dtheta = p_k (cbar - C_k) with cbar - C_k = sum_k' p_k' (C_k' - C_k):
            // differences of route times first, which avoids the cancellation
            float dc = 0.f;
            for (int i2 = rr0.x; i2 < rr0.y; ++i2) {
                const float c2 = Cday[(size_t)s.rinfo[i2].x * p.Np + bi];
                dc += expf(-p.theta * c2 - m) * rden * (c2 - ck);
            }
            dth += 2.0 * (double)p.q[qi] * (double)gp * (double)pk * (double)dc;
        }
    }
    if (!vw) return;
    if (p.mode == MODE_SOLVE) {
        const float Gv = p.G[qi] + g * g;
        float qv = p.q[qi] - p.eta * g / (sqrtf(Gv) + p.eps);
        qv = fmaxf(qv, 0.f);
        p.G[qi] = Gv;
        p.q[qi] = qv;
        if (PREC == 1) p.qb[qi] = __float2bfloat16_rn(qv);
    } else if (grad) {
        p.gout[qi] = 2.f * g;
        atomicAdd(s_dth, dth);
    }
}

__device__ __forceinline__ double block_sum(double v, double *s_red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? s_red[lane] : 0.0;
        for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    }
    return t;  // valid in thread 0
}

// Tick rows [pb, pb + RW) of every link; rows past the end of the day repeat the
// last interval (the link entry rule clamps to it).  Each warp loads four
// links' rows before storing, to keep many loads in flight.
__device__ __forceinline__ void stage_ticks(const FusedParams &p, Shared &s, const int32_t *tick_day) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int a0 = warp; a0 < p.A; a0 += 4 * nw) {
        for (int r0 = 0; r0 < s.RW; r0 += 32) {
            const int r = r0 + lane;
            int v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int a = a0 + u * nw;
                v[u] = (a < p.A && r < s.RW) ? __ldg(&tick_day[(size_t)a * p.Np + min(s.pb + r, p.N - 1)]) : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int a = a0 + u * nw;
                if (a < p.A && r < s.RW) s.tw[a * s.RW + r] = (uint16_t)v[u];
            }
        }
    }
}

// Residual rows [pb, pb + R) (clipped to the day) of every observed link, as
// float bits in the accumulator array.
template <int PREC>
__device__ __forceinline__ void stage_residual(const FusedParams &p, Shared &s, const void *rb) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int rows = min(s.R, p.N - s.pb);
    for (int o0 = warp; o0 < p.O; o0 += 4 * nw) {
        for (int r0 = 0; r0 < rows; r0 += 32) {
            const int r = r0 + lane;
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int o = o0 + u * nw;
                v[u] = (o < p.O && r < rows) ? Operand<PREC>::r(rb, (size_t)o * p.Np + s.pb + r) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int o = o0 + u * nw;
                if (o < p.O && r < rows) s.lo[o * s.R + r] = __float_as_uint(v[u]);
            }
        }
    }
}

// Flush of a phase: rows [pb0, pb0 + rows) of every observed link hold final
// link flows.  They become masked residuals r = m (xhat - x) (Eq. (nnls)),
// summed into the loss and written to the CTA's residual slot (or, FORWARD,
// the flows to xout).  EXACT (forward, loss and gradient calls) converts the
// 64-bit fixed point to FP64 and sums the loss in FP64.  The solve path
// (!EXACT) rounds the flow to FP32 once (relative error 6e-8, far below the
// residual's own scale) and sums r^2 with a compensated FP32 sum per thread,
// keeping the FP64 pipe out of the loop.  A row chunk (sel >= 0) keeps only
// the residuals of its rows for the update; the loss still covers all rows.
// High words are read only once the CTA has seen a carry.
template <int PREC, bool SMEM_RING, bool EXACT>
__device__ __forceinline__ void flush_phase(const FusedParams &p, const Shared &s, float *gacc, void *rb,
                                            const float *cnt, const uint32_t *mk, const int32_t *lab, int sel,
                                            int day, int pb0, int rows, bool carry, double &lsum, float &ks,
                                            float &kc) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int o0 = warp; o0 < p.O; o0 += 2 * nw) {
        for (int r0 = 0; r0 < rows; r0 += 32) {
            const int r = r0 + lane;
            const int h = pb0 + r;
            uint32_t lo[2];
            int hi[2];
            float xf[2], c[2];
            bool on[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int o = o0 + u * nw;
                lo[u] = 0u;
                hi[u] = 0;
                xf[u] = 0.f;
                c[u] = 0.f;
                on[u] = false;
                if (o < p.O && r < rows) {
                    if (SMEM_RING) {
                        const int idx = o * s.R + r;
                        lo[u] = s.lo[idx];
                        if (carry) hi[u] = s.hi[idx];
                    } else {
                        float *cell = gacc + (size_t)o * p.Np + h;
                        xf[u] = *cell;
                        *cell = 0.f;
                    }
                    if (p.mode != MODE_FORWARD) {
                        on[u] = (mk[(size_t)o * p.Nw + (h >> 5)] >> (h & 31)) & 1u;
                        c[u] = cnt[(size_t)o * p.Np + h];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int o = o0 + u * nw;
                if (o < p.O && r < rows) {
                    const size_t ri = (size_t)o * p.Np + h;
                    if (EXACT) {
                        const double x =
                            SMEM_RING ? (double)(((long long)hi[u] << 32) | (long long)lo[u]) * kFxInv : (double)xf[u];
                        if (p.mode == MODE_FORWARD) {
                            p.xout[(size_t)day * p.O * p.Np + ri] = (float)x;
                        } else {
                            const double rr = on[u] ? x - (double)c[u] : 0.0;
                            lsum += rr * rr;
                            Operand<PREC>::store_r(rb, ri, (float)rr);
                        }
                    } else {
                        const float x =
                            SMEM_RING ? fmaf((float)hi[u], 4096.f, __uint2float_rn(lo[u]) * 9.5367431640625e-7f)
                                      : xf[u];
                        const float rr = on[u] ? x - c[u] : 0.f;
                        const float y = rr * rr - kc;     // compensated (Kahan) sum
                        const float t = ks + y;
                        kc = (t - ks) - y;
                        ks = t;
                        const bool use = sel < 0 || (on[u] && lab[ri] == sel);
                        Operand<PREC>::store_r(rb, ri, use ? rr : 0.f);
                    }
                }
            }
        }
    }
}

// SplitMix64 (Steele, Lea and Flood, 2014) output number i of the stream that
// starts at state s: each step adds the golden-ratio constant to the state and
// mixes it, so output i is the mix of s + (i + 1) gamma.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long s, unsigned long long i) {
    unsigned long long z = s + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Row chunks of Algorithm 1 for one (day, epoch): the epoch visits the day's
// observed rows in ascending (key, row) order, row r = h O + o drawing key =
// output r of SplitMix64 seeded with seed ^ (day << 32 | epoch), and updates on
// runs of b rows.  Each observed cell gets lab = rank / b.  Ranks come from a
// histogram on the keys' top 12 bits: a bin whose rank range lies in one chunk
// labels its rows directly; the rows of a bin that straddles a chunk boundary
// are listed and ranked exactly inside the bin.  Returns the number of chunks.
__device__ int row_labels(const FusedParams &p, const uint32_t *mk, int gday, int epoch, int *s_n) {
    uint32_t *cnt = p.rc_bins + (size_t)blockIdx.x * 3 * kRankBins;
    uint32_t *first = cnt + kRankBins, *cur = first + kRankBins;
    const size_t cells = (size_t)p.O * p.N;
    unsigned long long *lkey = p.rc_key + (size_t)blockIdx.x * cells;
    int32_t *lrow = p.rc_row + (size_t)blockIdx.x * cells;
    int32_t *lab = p.lab + (size_t)blockIdx.x * p.O * p.Np;
    const unsigned long long s0 =
        p.seed ^ (((unsigned long long)(uint32_t)gday << 32) | (unsigned long long)(uint32_t)epoch);
    const uint32_t b = (uint32_t)p.row_chunk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < kRankBins; i += blockDim.x) {
        cnt[i] = 0u;
        cur[i] = 0u;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < (int)cells; c += blockDim.x) {    // O N < 2^31 (checked at create)
        const int o = c / p.N, h = c - o * p.N;
        if ((mk[(size_t)o * p.Nw + (h >> 5)] >> (h & 31)) & 1u) {
            const unsigned long long key = splitmix64_at(s0, (unsigned long long)h * p.O + o);
            atomicAdd(&cnt[key >> 52], 1u);
        }
    }
    __syncthreads();
    if (warp == 0) {       // exclusive scan of the bin counts: lane l owns 128 consecutive bins
        constexpr int per = kRankBins / 32;
        uint32_t sum = 0;
        for (int i = 0; i < per; ++i) sum += cnt[lane * per + i];
        uint32_t incl = sum;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        uint32_t run = incl - sum;
        for (int i = 0; i < per; ++i) {
            first[lane * per + i] = run;
            run += cnt[lane * per + i];
        }
        if (lane == 31) *s_n = (int)incl;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < (int)cells; c += blockDim.x) {    // O N < 2^31 (checked at create)
        const int o = c / p.N, h = c - o * p.N;
        if ((mk[(size_t)o * p.Nw + (h >> 5)] >> (h & 31)) & 1u) {
            const unsigned long long key = splitmix64_at(s0, (unsigned long long)h * p.O + o);
            const int bin = (int)(key >> 52);
            const uint32_t f = first[bin], n = cnt[bin];
            if (f / b == (f + n - 1) / b) {
                lab[(size_t)o * p.Np + h] = (int32_t)(f / b);
            } else {
                const uint32_t pos = f + atomicAdd(&cur[bin], 1u);
                lkey[pos] = key;
                lrow[pos] = h * p.O + o;
            }
        }
    }
    __syncthreads();
    for (int bin = warp; bin < kRankBins; bin += nw) {
        const uint32_t f = first[bin], n = cnt[bin];
        if (n == 0 || f / b == (f + n - 1) / b) continue;
        for (uint32_t i = lane; i < n; i += 32) {
            const unsigned long long ki = lkey[f + i];
            const int32_t ri = lrow[f + i];
            uint32_t rank = 0;
            for (uint32_t j = 0; j < n; ++j) {
                const unsigned long long kj = lkey[f + j];
                rank += (kj < ki || (kj == ki && lrow[f + j] < ri)) ? 1u : 0u;
            }
            lab[(size_t)(ri % p.O) * p.Np + ri / p.O] = (int32_t)((f + rank) / b);
        }
    }
    __syncthreads();
    return (int)((*s_n + b - 1) / b);
}

// Dynamic shared memory layout (16-byte aligned blocks):
//   rinfo int4[P] | odr int2[K] | task_od int[K] | colact u32[Ow] | lo u32[O][R] | tw u16[A][RW]
template <int PREC, bool SMEM_RING, bool SMEM_TICKS>
__global__ void __launch_bounds__(1024, 1) k_fused(const FusedParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shared s;
    s.R = SMEM_RING ? p.ring_rows : 0;
    s.RW = SMEM_TICKS ? p.tick_rows : 0;
    s.pb = 0;
    auto align16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    size_t off = 0;
    int4 *rinfo = reinterpret_cast<int4 *>(smem_raw + off);
    off = align16(off + (size_t)p.P * sizeof(int4));
    int2 *odr = reinterpret_cast<int2 *>(smem_raw + off);
    off = align16(off + (size_t)p.K * sizeof(int2));
    int *task_od = reinterpret_cast<int *>(smem_raw + off);
    off = align16(off + (size_t)p.K * sizeof(int));
    uint32_t *colact = reinterpret_cast<uint32_t *>(smem_raw + off);
    off = align16(off + (size_t)p.Ow * sizeof(uint32_t));
    s.lo = reinterpret_cast<uint32_t *>(smem_raw + off);
    if (SMEM_RING) off = align16(off + (size_t)p.O * s.R * sizeof(uint32_t));
    s.tw = reinterpret_cast<uint16_t *>(smem_raw + off);
    s.colact = colact;
    s.rinfo = rinfo;
    s.odr = odr;
    s.task_od = task_od;
    s.hi = SMEM_RING ? reinterpret_cast<int *>(p.gring) + (size_t)blockIdx.x * p.O * s.R : nullptr;
    __shared__ int s_day;
    __shared__ int s_task;
    __shared__ double s_red[32];
    __shared__ double s_dth;
    __shared__ int s_nrows;
    __shared__ int s_carry;
    s.carry = &s_carry;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nthr = blockDim.x;
    const int ntiles = (p.N + kTileW - 1) / kTileW;
    void *rb = static_cast<unsigned char *>(p.rbuf) +
               (size_t)blockIdx.x * p.O * p.Np * (PREC == 1 ? sizeof(__nv_bfloat16) : sizeof(float));
    float *gacc = SMEM_RING ? nullptr : p.gring + (size_t)blockIdx.x * p.O * p.Np;

    // network tables
    for (int i = threadIdx.x; i < p.P; i += nthr) {
        const int k = __ldg(&p.od_routes[i]);
        const int l0 = __ldg(&p.rptr[k]);
        rinfo[i] = make_int4(k, l0, __ldg(&p.rptr[k + 1]) - l0, 0);
    }
    for (int i = threadIdx.x; i < p.K; i += nthr) {
        odr[i] = make_int2(__ldg(&p.od_ptr[i]), __ldg(&p.od_ptr[i + 1]));
        task_od[i] = __ldg(&p.task_od[i]);
    }
    if (SMEM_RING) {
        for (int i = threadIdx.x; i < p.O * s.R; i += nthr) {
            s.lo[i] = 0u;
            s.hi[i] = 0;
        }
    } else {
        for (size_t i = threadIdx.x; i < (size_t)p.O * p.Np; i += nthr) gacc[i] = 0.f;
    }
    if (threadIdx.x == 0) {
        s_task = 0;
        s_carry = 0;
    }
    const bool exact = p.mode != MODE_SOLVE;

    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_day = atomicAdd(p.queue, 1);
        __syncthreads();
        const int day = s_day;
        if (day >= p.n_days) break;
        for (int i = threadIdx.x; i < p.Ow; i += nthr) colact[i] = p.colact[(size_t)day * p.Ow + i];
        const int64_t toff = p.tab_off[day];
        const int32_t *tab = toff >= 0 ? p.traj_tab + toff : nullptr;
        const int32_t *tick_day = p.ticks + (size_t)day * p.A * p.Np;
        const float *cnt = p.counts + (size_t)day * p.O * p.Np;
        const uint32_t *mk = p.mask + (size_t)day * p.O * p.Nw;
        const int maxoff = p.maxoff[day];
        // tiles per phase: the accumulators must hold a phase's arrival rows
        // (31 F + maxoff + 2) and the tick window its trajectories' entry rows
        // (31 F + maxoff + 1)
        int F = ntiles;
        if (SMEM_RING) F = min(F, (s.R - maxoff - 2) / kTileW);
        if (SMEM_TICKS) F = min(F, (s.RW - maxoff - 1) / kTileW);
        F = min(F, max(1, p.tiles_per_phase));
        if (F < 1) {
            if (threadIdx.x == 0) set_error(p.err, kErrUnsupported, day);
            continue;
        }
        const int spill = maxoff + 2;     // rows past a phase that its windows can reach
        if (threadIdx.x == 0) s_dth = 0.0;
        __syncthreads();

        // One pass = forward sweep (+ adjoint sweep and step).  Full-row updates
        // make one pass per epoch; row chunks make one per chunk, the first of
        // an epoch also giving the epoch's full masked loss.
        const bool chunked = p.mode == MODE_SOLVE && p.row_chunk > 0;
        const int32_t *lab = chunked ? p.lab + (size_t)blockIdx.x * p.O * p.Np : nullptr;
        int nch = 1;
        for (int it = 0, chunk = 0;;) {
            if (chunked && it < p.iters && chunk == 0) nch = row_labels(p, mk, p.day_base + day, it, &s_nrows);
            const int sel = (chunked && it < p.iters) ? chunk : -1;     // chunk of rows in this update
            // ------------------------------ forward sweep ------------------------------
            double lsum = 0.0;     // EXACT calls: FP64 (finite differences of the loss resolve tiny changes)
            float ks = 0.f, kc = 0.f;  // solve: compensated FP32 sum
            for (int pb0 = 0; pb0 < p.N; pb0 += F * kTileW) {
                const int nt = min(F, (p.N - pb0 + kTileW - 1) / kTileW);
                const int ntask = nt * p.K;
                s.pb = pb0;
                if (SMEM_TICKS && !tab) {
                    stage_ticks(p, s, tick_day);
                    __syncthreads();
                }
                while (true) {
                    int t = 0;
                    if (lane == 0) t = atomicAdd(&s_task, 1);
                    t = __shfl_sync(0xffffffffu, t, 0);
                    if (t >= ntask) break;
                    const int od = task_od[t / nt];
                    const int b0 = pb0 + (t % nt) * kTileW;
                    if (tab)
                        forward_task<PREC, SMEM_RING, SMEM_TICKS, true>(p, s, day, od, b0, tab);
                    else
                        forward_task<PREC, SMEM_RING, SMEM_TICKS, false>(p, s, day, od, b0, tab);
                }
                __syncthreads();
                // rows [pb0, pb0 + 31 nt) are final: residual, loss, residual slot;
                // the spill rows move to the front for the next phase
                const int span = nt * kTileW;
                const int rows = min(span, p.N - pb0);
                const bool carry = s_carry != 0;
                if (exact)
                    flush_phase<PREC, SMEM_RING, true>(p, s, gacc, rb, cnt, mk, lab, sel, day, pb0, rows, carry, lsum,
                                                       ks, kc);
                else
                    flush_phase<PREC, SMEM_RING, false>(p, s, gacc, rb, cnt, mk, lab, sel, day, pb0, rows, carry,
                                                        lsum, ks, kc);
                if (SMEM_RING) {
                    // move the spill rows [span, span + spill) to the front, zero the rest
                    __syncthreads();
                    for (int o = warp; o < p.O; o += nwarps) {
                        uint32_t *lrow = s.lo + o * s.R;
                        int *hrow = s.hi + o * s.R;
                        for (int q0 = 0; q0 < spill; q0 += 32) {
                            const int r = q0 + lane;
                            uint32_t vl = 0;
                            int vh = 0;
                            if (r < spill) {
                                vl = lrow[span + r];
                                if (carry) vh = hrow[span + r];
                            }
                            __syncwarp();
                            if (r < spill) {
                                lrow[r] = vl;
                                if (carry) hrow[r] = vh;
                            }
                            __syncwarp();
                        }
                        for (int r = spill + lane; r < span + spill; r += 32) {
                            lrow[r] = 0u;
                            if (carry) hrow[r] = 0;
                        }
                    }
                }
                if (threadIdx.x == 0) s_task = 0;
                __syncthreads();
            }
            const double loss_day = block_sum(exact ? lsum : (double)ks - (double)kc, s_red);
            if (threadIdx.x == 0 && chunk == 0) {
                if (p.mode == MODE_SOLVE && it < p.iters && p.trace) p.trace[(size_t)it * p.n_days + day] = (float)loss_day;
                if (p.mode != MODE_SOLVE || it == p.iters) p.loss[day] = loss_day;
            }
            if (p.mode == MODE_FORWARD || p.mode == MODE_LOSS || (p.mode == MODE_SOLVE && it >= p.iters)) break;
            if (chunked && nch == 0) {      // no observed row: the epoch makes no update
                ++it;
                continue;
            }

            // ------------------------------ adjoint sweep ------------------------------
            for (int pb0 = 0; pb0 < p.N; pb0 += F * kTileW) {
                const int nt = min(F, (p.N - pb0 + kTileW - 1) / kTileW);
                const int ntask = nt * p.K;
                s.pb = pb0;
                __syncthreads();                           // previous phase done with the windows
                if (SMEM_TICKS && !tab) stage_ticks(p, s, tick_day);
                if (SMEM_RING) stage_residual<PREC>(p, s, rb);
                __syncthreads();
                while (true) {
                    int t = 0;
                    if (lane == 0) t = atomicAdd(&s_task, 1);
                    t = __shfl_sync(0xffffffffu, t, 0);
                    if (t >= ntask) break;
                    const int od = task_od[t / nt];
                    const int b0 = pb0 + (t % nt) * kTileW;
                    if (tab)
                        adjoint_task<PREC, SMEM_RING, SMEM_TICKS, true>(p, s, day, od, b0, rb, tab, &s_dth);
                    else
                        adjoint_task<PREC, SMEM_RING, SMEM_TICKS, false>(p, s, day, od, b0, rb, tab, &s_dth);
                }
                __syncthreads();
                if (threadIdx.x == 0) s_task = 0;
            }
            __syncthreads();
            if (SMEM_RING) {
                for (int i = threadIdx.x; i < p.O * s.R; i += nthr) s.lo[i] = 0u;
            }
            __syncthreads();
            if (p.mode == MODE_LOSS_GRAD) {
                if (threadIdx.x == 0) p.dtheta[day] = s_dth;
                break;
            }
            if (chunked && ++chunk < nch) continue;
            chunk = 0;
            ++it;
        }
    }
}

// Raise a variant's dynamic shared-memory limit once to the largest size asked
// for (so that launches made during a stream capture need no attribute call).
template <int PREC, bool SMEM_RING, bool SMEM_TICKS>
static cudaError_t set_attr_one(size_t smem) {
    static size_t limit = 48 * 1024;
    if (smem <= limit) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_fused<PREC, SMEM_RING, SMEM_TICKS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) limit = smem;
    return e;
}

template <int PREC, bool SMEM_RING, bool SMEM_TICKS>
static cudaError_t launch_one(const FusedParams &p, int grid, int block, size_t smem, cudaStream_t s) {
    cudaError_t e = set_attr_one<PREC, SMEM_RING, SMEM_TICKS>(smem);
    if (e != cudaSuccess) return e;
    k_fused<PREC, SMEM_RING, SMEM_TICKS><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t fused_set_attr(bool smem_ring, bool smem_ticks, int precision, size_t smem) {
    if (precision == 1) {
        if (smem_ring && smem_ticks) return set_attr_one<1, true, true>(smem);
        if (smem_ring) return set_attr_one<1, true, false>(smem);
        return set_attr_one<1, false, false>(smem);
    }
    if (smem_ring && smem_ticks) return set_attr_one<0, true, true>(smem);
    if (smem_ring) return set_attr_one<0, true, false>(smem);
    return set_attr_one<0, false, false>(smem);
}

template <int PREC>
static cudaError_t launch_prec(const FusedParams &p, int grid, int block, size_t smem, cudaStream_t s) {
    const bool ring = p.ring_rows > 0, ticks = p.tick_rows > 0;
    if (ring && ticks) return launch_one<PREC, true, true>(p, grid, block, smem, s);
    if (ring) return launch_one<PREC, true, false>(p, grid, block, smem, s);
    return launch_one<PREC, false, false>(p, grid, block, smem, s);
}

cudaError_t launch_fused(const FusedParams &p, int precision, int grid, int block, size_t smem,
                         cudaStream_t s) {
    return precision == 1 ? launch_prec<1>(p, grid, block, smem, s) : launch_prec<0>(p, grid, block, smem, s);
}

cudaError_t fused_occupancy(int precision, int block, size_t smem, int *blocks_per_sm) {
    cudaError_t e;
    if (precision == 1) {
        e = cudaFuncSetAttribute(k_fused<1, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_fused<1, true, true>, block, smem);
    }
    e = cudaFuncSetAttribute(k_fused<0, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_fused<0, true, true>, block, smem);
}

}  // namespace dode
