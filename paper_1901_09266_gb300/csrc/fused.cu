// fused.cu -- the hot path: one persistent kernel runs Algorithm 1 (Sec. 3.3) for
// whole days, rebuilding each day's DAR (Eq. (dar)) from its tick table on chip
// in every pass instead of reading a materialised matrix.
//
// Work decomposition.  A CTA takes a day from a device work queue and runs all
// of that day's epochs before taking the next one (days are independent
// problems, Sec. 2.7).  One epoch is a forward sweep and an adjoint sweep:
//
//  * Routes leaving one origin share their trajectories over their common
//    link prefix, so each origin's routes are walked as a prefix tree (walk
//    groups, built once per network): every shared window is computed once.
//  * A task is (walk group, the phase's tiles of 31 departure intervals):
//    lane l follows the leading vehicles that depart at boundaries b0 + l and
//    b0 + 31 + l (Example "DAR matrix computation") -- two independent chains
//    per lane that share the route records, for instruction-level
//    parallelism.  At each link a chain's entry time T_j(b) and its right
//    neighbour's T_j(b+1) (one shuffle) bound the window of Eq. (dar); the
//    entry interval selects the link time from the tick table (Sec. 2.4,
//    Eq. (cost)).  The route's links are held in registers as precomputed
//    shared-memory offsets and broadcast by shuffles, so a link step touches
//    memory only for the tick lookup and the window's one or two link-interval
//    cells.  The walk-group and route tables sit in shared memory.
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

// Lanes that share one row of a staging or flush loop: the smallest power of
// two (at most 32) that covers the row's n chunks, as its log2.  A warp then
// takes 32 >> lg rows at a time and no index needs a division.
__device__ __forceinline__ int lane_group_log2(int n) { return n <= 1 ? 0 : min(5, 32 - __clz(n - 1)); }

// i / n for 0 <= i < 2^31 by the multiply-high of IntervalDiv (d = make_interval_div(max(n, 2))).
__device__ __forceinline__ int div_by(int i, int n, const IntervalDiv &d) { return n == 1 ? i : interval_of(i, d); }


struct Shared {
    uint32_t *lo;         // [O][R]: accumulator low words (forward) / residual window as float bits (adjoint)
    int *hi;              // [O][R] in global memory: accumulator high words (forward)
    uint16_t *tw;         // [A][RW]: tick window (row = h - pb)
    const uint32_t *colact;
    const int4 *groute;   // [P] walk order: (route, first position, links, start depth)
    const int *gptr;      // [G+1] routes of each walk group
    const int *task_grp;  // [G] processing order
    const int *god_ptr;   // [G+1] ODs owned by each walk group (shared-memory copies of the
    const int *god;       //        OD-update tables: read by every adjoint task, so they are
    const int *godr_ptr;  //        kept out of the global load path)
    const int *godr;
    const int2 *rtab;     // [L] route-position table in shared memory, or null
    const uint32_t *rtab32;  // [L] its 32-bit form in shared memory, or null
    int *carry;           // set once any deposit of this CTA carried into a high word
    int R, RW, pb;
    int *err;             // error word (index checks of the debug build)
    int ring_cells;       // accumulator / residual cells: O R (shared ring) or O Np (global)
    int tick_cells;       // tick cells: A RW (shared window) or A Np (global table)
};

// Route links in registers: lane j holds, for position j (and j + 32) of the
// route, the offset of its tick row and of its accumulator row (kInactive when
// the link is unobserved or has no observation this day), both relative to pb,
// and the position's walk-group event word (E << 1 | save).
struct RouteRegs {
    int t0, o0, e0, t1, o1, e1;
};

template <bool SMEM_RING, bool SMEM_TICKS>
__device__ __forceinline__ RouteRegs load_route(const FusedParams &p, const Shared &s, int l0, int beta) {
    const int lane = threadIdx.x & 31;
    RouteRegs r{0, kInactive, 0, 0, kInactive, 0};
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int j = lane + 32 * half;
        if (j < beta && (half == 0 || beta > 32)) {
            int a, o, ev;
            if (s.rtab32) {
                const uint32_t w = s.rtab32[l0 + j];
                a = (int)(w & 0x7ffu);
                o = (int)((w >> 11) & 0x7ffu) - 1;
                ev = (int)(w >> 22);
            } else {
                const int2 x = s.rtab ? s.rtab[l0 + j] : __ldg(&p.rtab[l0 + j]);
                a = x.x;
                o = (x.y & 0xffffff) - 1;
                ev = x.y >> 24;
            }
            const int tb = SMEM_TICKS ? a * s.RW - s.pb : a * p.Np;
            int ob = kInactive;
            if (o >= 0 && ((s.colact[o >> 5] >> (o & 31)) & 1u)) ob = SMEM_RING ? o * s.R - s.pb : o * p.Np;
            if (half == 0) {
                r.t0 = tb;
                r.o0 = ob;
                r.e0 = ev;
            } else {
                r.t1 = tb;
                r.o1 = ob;
                r.e1 = ev;
            }
        }
    }
    return r;
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
    return PREC == 0 ? d : bf16_round(d);      // 1 is exact in BF16
}

// Add v to accumulator cell idx: 64-bit fixed point (shared low word, carries
// into the global high word) or a global float when the ring is not in shared
// memory.
// FAST: the caller guarantees 0 <= v < 3000 (then v 2^20 fits 32 unsigned bits).
template <bool SMEM_RING, bool FAST = false>
__device__ __forceinline__ void deposit(const Shared &s, float *gacc, int idx, float v) {
    if (!DODE_IN_BOUNDS(idx, s.ring_cells, s.err, kSiteRingDeposit)) return;
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
        else if (DODE_IN_BOUNDS(idx, s.ring_cells, s.err, kSiteRingGather))
            acc += share * (SMEM_RING ? __uint_as_float(s.lo[idx]) : Operand<PREC>::r(rb, (size_t)idx));
        ++idx;
        e += ipt;
        ++h;
    }
    return acc;
}

// Add u units of 2^-20 vehicles (u < 2^32) to cell idx.
template <bool SMEM_RING>
__device__ __forceinline__ void deposit_u(const Shared &s, float *gacc, int idx, uint32_t u) {
    if (!DODE_IN_BOUNDS(idx, s.ring_cells, s.err, kSiteRingDeposit)) return;
    if (!SMEM_RING) {
        atomicAdd(gacc + idx, (float)((double)u * kFxInv));
        return;
    }
    const uint32_t old = atomicAdd(&s.lo[idx], u);
    if (old + u < old) {
        atomicAdd(&s.hi[idx], 1);
        *s.carry = 1;
    }
}

// Integer form of window_tail: cells h0 + 1 .. of a window spanning three or
// more intervals get rn(W share) each, the window's last cell the remainder
// of W; cells past the end of the day are dropped.
template <int PREC, bool SMEM_RING>
__device__ __noinline__ void window_tail_u(const Shared &s, float *gacc, int idx, int hi, int e, int h, int N,
                                           int ipt, float inv, float Wf, uint32_t rem) {
    while (hi > e && h < N) {
        const int end = min(hi, e + ipt);
        uint32_t u = rem;
        if (end < hi) {
            float share = (float)(end - e) * inv;
            if (PREC == 1) share = bf16_round(share);
            u = min(__float2uint_rn(Wf * share), rem);
        }
        if (u) deposit_u<SMEM_RING>(s, gacc, idx, u);
        rem -= u;
        ++idx;
        e += ipt;
        ++h;
    }
}

// Residual cell idx read by an adjoint walk: the shared window, or the CTA's
// residual slot when the ring is global.
template <int PREC, bool SMEM_RING>
__device__ __forceinline__ float rcell(const Shared &s, const float *racc, const void *rb, int idx) {
    if (!DODE_IN_BOUNDS(idx, s.ring_cells, s.err, kSiteRingGather)) return 0.f;
    return SMEM_RING ? racc[idx] : Operand<PREC>::r(rb, (size_t)idx);
}

template <bool SMEM_TICKS, bool TAB>
__device__ __forceinline__ int next_entry(const FusedParams &p, const Shared &s, const int32_t *tick_day,
                                          const int32_t *trow, int j, int T, int tb, int h0) {
    if (TAB) return __ldg(&trow[(size_t)(j + 1) * (p.N + 1)]);
    const int ti = SMEM_TICKS ? tb + h0 : tb + min(h0, p.N - 1);
    if (!DODE_IN_BOUNDS(ti, s.tick_cells, s.err, kSiteTickWindow)) return T;
    if (SMEM_TICKS) return T + s.tw[ti];
    return T + __ldg(&tick_day[ti]);
}

// Forward walk of route t of a group from depth j0: every window on an
// observed link deposits W rho, W the summed flow of the group's routes t..E
// that share the window (exclusive prefix sums S over the group, 2^-20
// vehicle units).  Integer form (every flow of the warp's group in
// [0, 2^31)): the head cell gets rn(W d0) and a two-cell window's tail
// W - rn(W d0); when the tail cell is where the next lane's window starts,
// the next lane adds the tail to its own head deposit (one atomic per window
// instead of two).  On the shared ring no lane needs a range check: lanes
// outside the tile carry W = 0, and cells past the end of the day fall in
// ring rows that are never flushed and are cleared after the sweep.  LONG:
// the route has more than 32 links (positions 32.. sit in the second register
// set).
template <int PREC, bool SMEM_RING, bool SMEM_TICKS, bool TAB, bool LONG>
__device__ __forceinline__ void forward_walk_u(const FusedParams &p, const Shared &s, const int32_t *tick_day,
                                               const int32_t *trow, const RouteRegs &rr, float *gacc, int j0, int beta,
                                               int T, bool vw, const long long *S, int t, int E, int *stk) {
    const int lane = threadIdx.x & 31;
    const int ipt = p.div.ipt, N = p.Nh;      // horizon: the day, and the first rows of a coupled next day
    if (!DODE_IN_BOUNDS(E + 1, kGroupRoutes + 1, s.err, kSiteGroupSums)) E = t;
    uint32_t Wu = (uint32_t)(S[E + 1] - S[t]);
    float Wf = __uint2float_rn(Wu);
    for (int j = j0; j < beta; ++j) {
        const bool first32 = !LONG || j < 32;
        const int tb = __shfl_sync(0xffffffffu, first32 ? rr.t0 : rr.t1, j & 31);
        const int ob = __shfl_sync(0xffffffffu, first32 ? rr.o0 : rr.o1, j & 31);
        const int ev = __shfl_sync(0xffffffffu, first32 ? rr.e0 : rr.e1, j & 31);
        if ((ev >> 1) != E) {          // routes branch off: fewer of them share this window
            E = ev >> 1;
            if (!DODE_IN_BOUNDS(E + 1, kGroupRoutes + 1, s.err, kSiteGroupSums)) E = t;
            Wu = (uint32_t)(S[E + 1] - S[t]);
            Wf = __uint2float_rn(Wu);
        }
        const int hi = __shfl_down_sync(0xffffffffu, T, 1);
        const int h0 = interval_of(T, p.div);
        if (ob != kInactive) {
            uint32_t u0 = 0, give = 0;
            int kind = 0;              // 1: the tail fills the next cell to its end; 2: three or more cells
            int e0 = 0;
            float inv = 0.f;
            if (SMEM_RING || (vw && h0 < N)) {
                e0 = h0 * ipt + ipt;
                inv = __fdividef(1.f, (float)(hi - T));
                const float d0 = first_share<PREC>(T, e0, inv);
                u0 = min(__float2uint_rn(Wf * d0), Wu);
                if (hi > e0 && (SMEM_RING || h0 + 1 < N)) {
                    if (hi < e0 + ipt)
                        give = Wu - u0;
                    else
                        kind = hi == e0 + ipt ? 1 : 2;
                }
            }
            uint32_t recv = __shfl_up_sync(0xffffffffu, give, 1);
            if (lane == 0) recv = 0;
            const uint32_t dep = u0 + recv;
            if (dep) deposit_u<SMEM_RING>(s, gacc, ob + h0, dep);
            if (kind == 1)
                deposit_u<SMEM_RING>(s, gacc, ob + h0 + 1, Wu - u0);
            else if (kind == 2)
                window_tail_u<PREC, SMEM_RING>(s, gacc, ob + h0 + 1, hi, e0, h0 + 1, N, ipt, inv, Wf, Wu - u0);
        }
        T = next_entry<SMEM_TICKS, TAB>(p, s, tick_day, trow, j, T, tb, h0);
        if ((ev & 1) && DODE_IN_BOUNDS(j + 1, kMaxRouteLinks + 1, s.err, kSiteWalkStack)) stk[j + 1] = T;
    }
}

// General form (a flow outside [0, 2^31) units): W as FP32 vehicles, one
// 64-bit fixed-point deposit per cell.
template <int PREC, bool SMEM_RING, bool SMEM_TICKS, bool TAB, bool LONG>
__device__ __forceinline__ void forward_walk_f(const FusedParams &p, const Shared &s, const int32_t *tick_day,
                                               const int32_t *trow, const RouteRegs &rr, float *gacc, int j0, int beta,
                                               int T, bool vw, const long long *S, int t, int E, int *stk) {
    const int ipt = p.div.ipt, N = p.Nh;      // horizon: the day, and the first rows of a coupled next day
    if (!DODE_IN_BOUNDS(E + 1, kGroupRoutes + 1, s.err, kSiteGroupSums)) E = t;
    float f = (float)((double)(S[E + 1] - S[t]) * kFxInv);
    for (int j = j0; j < beta; ++j) {
        const bool first32 = !LONG || j < 32;
        const int tb = __shfl_sync(0xffffffffu, first32 ? rr.t0 : rr.t1, j & 31);
        const int ob = __shfl_sync(0xffffffffu, first32 ? rr.o0 : rr.o1, j & 31);
        const int ev = __shfl_sync(0xffffffffu, first32 ? rr.e0 : rr.e1, j & 31);
        if ((ev >> 1) != E) {
            E = ev >> 1;
            if (!DODE_IN_BOUNDS(E + 1, kGroupRoutes + 1, s.err, kSiteGroupSums)) E = t;
            f = (float)((double)(S[E + 1] - S[t]) * kFxInv);
        }
        const int hi = __shfl_down_sync(0xffffffffu, T, 1);
        const int h0 = interval_of(T, p.div);
        if (ob != kInactive && vw && h0 < N) {
            const int idx = ob + h0;
            const int e0 = h0 * ipt + ipt;
            const float inv = __fdividef(1.f, (float)(hi - T));
            const float d0 = first_share<PREC>(T, e0, inv);
            const float c0 = f * d0;
            deposit<SMEM_RING>(s, gacc, idx, c0);
            if (hi > e0 && h0 + 1 < N) {
                if (hi <= e0 + ipt)
                    deposit<SMEM_RING>(s, gacc, idx + 1, f - c0);
                else
                    window_tail<PREC, SMEM_RING, true>(s, gacc, nullptr, idx + 1, hi, e0, h0 + 1, N, ipt, inv, d0, f);
            }
        }
        T = next_entry<SMEM_TICKS, TAB>(p, s, tick_day, trow, j, T, tb, h0);
        if ((ev & 1) && DODE_IN_BOUNDS(j + 1, kMaxRouteLinks + 1, s.err, kSiteWalkStack)) stk[j + 1] = T;
    }
}

// Entry time of a route's walk at its start depth s0: the departure boundary at
// the root, else the time stored by the walk that passed depth s0 - 1 (or the
// repaired trajectory table).
template <bool TAB>
__device__ __forceinline__ int walk_start(const FusedParams &p, const int32_t *trow, const int *stk, int s0, int bb) {
    if (s0 == 0) return p.div.ipt * bb;
    if (TAB) return __ldg(&trow[(size_t)s0 * (p.N + 1)]);
    return stk[s0];
}

// Route flows of one tile: exclusive prefix sums S over the group's walk order.
template <int PREC>
__device__ __forceinline__ void group_flows(const FusedParams &p, const Shared &s, int day, int i0, int m, int b,
                                            bool vw, long long *S, bool &any, bool &fast) {
    const int bi = min(b, p.N - 1);
    long long acc = 0;
    bool nonneg = true;
    any = false;
    S[0] = 0;
    for (int t0 = 0; t0 < m; t0 += 4) {
        float pv[4], qv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            pv[u] = 0.f;
            qv[u] = 0.f;
            if (vw && t0 + u < m) {
                const int4 gr = s.groute[i0 + t0 + u];
                pv[u] = __ldg(&p.pt[((size_t)day * p.P + gr.x) * p.Np + bi]);
                qv[u] = Operand<PREC>::q(p, ((size_t)day * p.K + (gr.w >> 9)) * p.Np + b);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (t0 + u < m) {
                // 32-bit conversion whenever the flow fits (the 64-bit one runs on the slow FP64 pipe)
                const float x = pv[u] * qv[u] * kFxScale;
                long long fu;
                if (x >= 0.f && x < 2147483520.f)
                    fu = __float2int_rn(x);
                else
                    fu = __float2ll_rn(x);
                nonneg = nonneg && fu >= 0;
                any = any || fu != 0;
                acc += fu;
                S[t0 + u + 1] = acc;
            }
        }
    }
    fast = nonneg && acc < (1ll << 31);
}

// Forward task: walk group g for departure boundaries b0 .. b0 + 31.
template <int PREC, bool SMEM_RING, bool SMEM_TICKS, bool TAB>
__device__ void forward_task(const FusedParams &p, const Shared &s, int day, int g, int b0, const int32_t *tab) {
    const int lane = threadIdx.x & 31;
    const int b = b0 + lane;
    const int bb = min(b, p.N);
    const bool vw = (lane < kTileW) && (b < p.N);
    const int32_t *tick_day = p.ticks + (size_t)day * p.A * p.Np;
    const int i0 = s.gptr[g], m = s.gptr[g + 1] - i0;
    if (!DODE_IN_BOUNDS(m, kGroupRoutes + 1, s.err, kSiteGroupSums)) return;
    // route flows f = p q (Eq. (flow)) in 2^-20 vehicle units and their
    // exclusive prefix sums over the group's walk order
    long long S[kGroupRoutes + 1];
    bool any, fast_lane;
    group_flows<PREC>(p, s, day, i0, m, b, vw, S, any, fast_lane);
    if (!__any_sync(0xffffffffu, any)) return;            // nothing departs: no deposits
    const bool fast = __all_sync(0xffffffffu, fast_lane);
    float *gacc = SMEM_RING ? nullptr : p.gring + (size_t)blockIdx.x * p.O * p.Np;
    int stk[kMaxRouteLinks + 1];
    for (int t = 0; t < m; ++t) {
        const int4 gr = s.groute[i0 + t];
        const int k = gr.x, l0 = gr.y, beta = gr.z, s0 = gr.w & 0xff;
        if (!DODE_IN_BOUNDS(beta - 1, kMaxRouteLinks, s.err, kSiteWalkStack) ||
            !DODE_IN_BOUNDS(s0, kMaxRouteLinks + 1, s.err, kSiteWalkStack))
            continue;
        if (s0 >= beta) continue;                         // every link walked by earlier routes
        const RouteRegs rr = load_route<SMEM_RING, SMEM_TICKS>(p, s, l0, beta);
        const int32_t *trow = TAB ? tab + (size_t)(l0 + k) * (p.N + 1) + bb : nullptr;
        const int T = walk_start<TAB>(p, trow, stk, s0, bb);
        const int E = __shfl_sync(0xffffffffu, s0 < 32 ? rr.e0 : rr.e1, s0 & 31) >> 1;
        if (fast && beta <= 32)
            forward_walk_u<PREC, SMEM_RING, SMEM_TICKS, TAB, false>(p, s, tick_day, trow, rr, gacc, s0, beta, T, vw, S,
                                                                    t, E, stk);
        else if (fast)
            forward_walk_u<PREC, SMEM_RING, SMEM_TICKS, TAB, true>(p, s, tick_day, trow, rr, gacc, s0, beta, T, vw, S, t,
                                                                   E, stk);
        else
            forward_walk_f<PREC, SMEM_RING, SMEM_TICKS, TAB, true>(p, s, tick_day, trow, rr, gacc, s0, beta, T, vw, S, t,
                                                                   E, stk);
    }
}


// Two tiles of the same walk group in one warp (A: boundaries b0 .., B: b0 + 31 ..):
// the route record shuffles and loop control are shared, the two lane chains
// are independent.  Integer form, routes of at most 32 links.  The prefix sums
// and the walk stack hold both chains' values side by side (one 8-byte local
// access for the pair).
template <int PREC, bool SMEM_RING, bool SMEM_TICKS, bool TAB>
__device__ __forceinline__ void forward_walk_u2(const FusedParams &p, const Shared &s, const int32_t *tick_day,
                                                const int32_t *trowA, const int32_t *trowB, const RouteRegs &rr,
                                                float *gacc, int j0, int beta, int TA, int TB, bool vwA, bool vwB,
                                                const uint2 *S2, int t, int E, int2 *stk2) {
    const int lane = threadIdx.x & 31;
    const int ipt = p.div.ipt, N = p.Nh;      // horizon: the day, and the first rows of a coupled next day
    if (!DODE_IN_BOUNDS(E + 1, kGroupRoutes + 1, s.err, kSiteGroupSums)) E = t;
    uint2 shi = S2[E + 1];
    const uint2 slo = S2[t];
    uint32_t WuA = shi.x - slo.x, WuB = shi.y - slo.y;
    float WfA = __uint2float_rn(WuA), WfB = __uint2float_rn(WuB);
    for (int j = j0; j < beta; ++j) {
        const int tb = __shfl_sync(0xffffffffu, rr.t0, j & 31);
        const int ob = __shfl_sync(0xffffffffu, rr.o0, j & 31);
        const int ev = __shfl_sync(0xffffffffu, rr.e0, j & 31);
        if ((ev >> 1) != E) {
            E = ev >> 1;
            if (!DODE_IN_BOUNDS(E + 1, kGroupRoutes + 1, s.err, kSiteGroupSums)) E = t;
            shi = S2[E + 1];
            WuA = shi.x - slo.x;
            WuB = shi.y - slo.y;
            WfA = __uint2float_rn(WuA);
            WfB = __uint2float_rn(WuB);
        }
        const int hiA = __shfl_down_sync(0xffffffffu, TA, 1);
        const int hiB = __shfl_down_sync(0xffffffffu, TB, 1);
        const int h0A = interval_of(TA, p.div);
        const int h0B = interval_of(TB, p.div);
        if (ob != kInactive) {
            uint32_t u0A = 0, giveA = 0, u0B = 0, giveB = 0;
            int kindA = 0, kindB = 0, e0A = 0, e0B = 0;
            float invA = 0.f, invB = 0.f;
            if (SMEM_RING || (vwA && h0A < N)) {
                e0A = h0A * ipt + ipt;
                invA = __fdividef(1.f, (float)(hiA - TA));
                u0A = min(__float2uint_rn(WfA * first_share<PREC>(TA, e0A, invA)), WuA);
                if (hiA > e0A && (SMEM_RING || h0A + 1 < N)) {
                    if (hiA < e0A + ipt)
                        giveA = WuA - u0A;
                    else
                        kindA = hiA == e0A + ipt ? 1 : 2;
                }
            }
            if (SMEM_RING || (vwB && h0B < N)) {
                e0B = h0B * ipt + ipt;
                invB = __fdividef(1.f, (float)(hiB - TB));
                u0B = min(__float2uint_rn(WfB * first_share<PREC>(TB, e0B, invB)), WuB);
                if (hiB > e0B && (SMEM_RING || h0B + 1 < N)) {
                    if (hiB < e0B + ipt)
                        giveB = WuB - u0B;
                    else
                        kindB = hiB == e0B + ipt ? 1 : 2;
                }
            }
            uint32_t recvA = __shfl_up_sync(0xffffffffu, giveA, 1);
            uint32_t recvB = __shfl_up_sync(0xffffffffu, giveB, 1);
            if (lane == 0) {
                recvA = 0;
                recvB = 0;
            }
            const uint32_t depA = u0A + recvA, depB = u0B + recvB;
            if (depA) deposit_u<SMEM_RING>(s, gacc, ob + h0A, depA);
            if (depB) deposit_u<SMEM_RING>(s, gacc, ob + h0B, depB);
            if (kindA == 1)
                deposit_u<SMEM_RING>(s, gacc, ob + h0A + 1, WuA - u0A);
            else if (kindA == 2)
                window_tail_u<PREC, SMEM_RING>(s, gacc, ob + h0A + 1, hiA, e0A, h0A + 1, N, ipt, invA, WfA, WuA - u0A);
            if (kindB == 1)
                deposit_u<SMEM_RING>(s, gacc, ob + h0B + 1, WuB - u0B);
            else if (kindB == 2)
                window_tail_u<PREC, SMEM_RING>(s, gacc, ob + h0B + 1, hiB, e0B, h0B + 1, N, ipt, invB, WfB, WuB - u0B);
        }
        TA = next_entry<SMEM_TICKS, TAB>(p, s, tick_day, trowA, j, TA, tb, h0A);
        TB = next_entry<SMEM_TICKS, TAB>(p, s, tick_day, trowB, j, TB, tb, h0B);
        if ((ev & 1) && DODE_IN_BOUNDS(j + 1, kMaxRouteLinks + 1, s.err, kSiteWalkStack)) stk2[j + 1] = make_int2(TA, TB);
    }
}

// Route flows of both tiles of a pair task: exclusive prefix sums interleaved
// per route (x: tile A, y: tile B), so that one 8-byte local access serves both
// chains; 32 bits suffice for the integer form the pair walk takes (fast).  A
// flow outside [0, 2^31) units (or not a number) makes the task not fast; it is
// then walked as two single tiles, which convert in 64 bits.
template <int PREC>
__device__ __forceinline__ void group_flows2(const FusedParams &p, const Shared &s, int day, int i0, int m, int bA,
                                             int bB, bool vwA, bool vwB, uint2 *S, bool &any, bool &fast) {
    const int biA = min(bA, p.N - 1), biB = min(bB, p.N - 1);
    long long accA = 0, accB = 0;
    bool nonneg = true;
    any = false;
    S[0] = make_uint2(0u, 0u);
    for (int t0 = 0; t0 < m; t0 += 4) {
        float pa[4], qa[4], pb[4], qb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            pa[u] = qa[u] = pb[u] = qb[u] = 0.f;
            if (t0 + u < m) {
                const int4 gr = s.groute[i0 + t0 + u];
                const size_t prow = ((size_t)day * p.P + gr.x) * p.Np, qrow = ((size_t)day * p.K + (gr.w >> 9)) * p.Np;
                if (vwA) {
                    pa[u] = __ldg(&p.pt[prow + biA]);
                    qa[u] = Operand<PREC>::q(p, qrow + bA);
                }
                if (vwB) {
                    pb[u] = __ldg(&p.pt[prow + biB]);
                    qb[u] = Operand<PREC>::q(p, qrow + bB);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (t0 + u < m) {
                // the pair walk needs every flow in [0, 2^31) units: a 32-bit
                // conversion then gives the same integer as a 64-bit one, and keeps
                // the slow FP64 pipe (which takes 64-bit conversions) free
                const float xa = pa[u] * qa[u] * kFxScale, xb = pb[u] * qb[u] * kFxScale;
                const bool in = xa >= 0.f && xa < 2147483520.f && xb >= 0.f && xb < 2147483520.f;
                const int fa = in ? __float2int_rn(xa) : 0, fb = in ? __float2int_rn(xb) : 0;
                nonneg = nonneg && in;
                any = any || fa != 0 || fb != 0 || !in;     // out of range: the single-tile walks decide
                accA += fa;
                accB += fb;
                S[t0 + u + 1] = make_uint2((uint32_t)accA, (uint32_t)accB);
            }
        }
    }
    fast = nonneg && accA < (1ll << 31) && accB < (1ll << 31);
}

// Forward task over both tiles of a phase for walk group g (b0 .. b0 + 61).
// Groups with a route past 32 links, or with a flow outside the integer form,
// take two single-tile tasks.
template <int PREC, bool SMEM_RING, bool SMEM_TICKS, bool TAB>
__device__ void forward_task2(const FusedParams &p, const Shared &s, int day, int g, int b0, const int32_t *tab) {
    const int lane = threadIdx.x & 31;
    const int bA = b0 + lane, bB = b0 + kTileW + lane;
    const int bbA = min(bA, p.N), bbB = min(bB, p.N);
    const bool vwA = (lane < kTileW) && (bA < p.N), vwB = (lane < kTileW) && (bB < p.N);
    const int32_t *tick_day = p.ticks + (size_t)day * p.A * p.Np;
    const int i0 = s.gptr[g], m = s.gptr[g + 1] - i0;
    if (!DODE_IN_BOUNDS(m, kGroupRoutes + 1, s.err, kSiteGroupSums)) return;
    uint2 S2[kGroupRoutes + 1];   // the pair walk is integer-form only
    bool any, fast;
    group_flows2<PREC>(p, s, day, i0, m, bA, bB, vwA, vwB, S2, any, fast);
    if (!__any_sync(0xffffffffu, any)) return;
    bool longr = false;                                   // a route past 32 links: single-tile walks
    for (int t = 0; t < m; ++t) longr = longr || s.groute[i0 + t].z > 32;
    if (longr || !__all_sync(0xffffffffu, fast)) {
        forward_task<PREC, SMEM_RING, SMEM_TICKS, TAB>(p, s, day, g, b0, tab);
        forward_task<PREC, SMEM_RING, SMEM_TICKS, TAB>(p, s, day, g, b0 + kTileW, tab);
        return;
    }
    float *gacc = SMEM_RING ? nullptr : p.gring + (size_t)blockIdx.x * p.O * p.Np;
    int2 stk2[kMaxRouteLinks + 1];
    for (int t = 0; t < m; ++t) {
        const int4 gr = s.groute[i0 + t];
        const int k = gr.x, l0 = gr.y, beta = gr.z, s0 = gr.w & 0xff;
        if (!DODE_IN_BOUNDS(beta - 1, kMaxRouteLinks, s.err, kSiteWalkStack) ||
            !DODE_IN_BOUNDS(s0, kMaxRouteLinks + 1, s.err, kSiteWalkStack))
            continue;
        if (s0 >= beta) continue;
        const RouteRegs rr = load_route<SMEM_RING, SMEM_TICKS>(p, s, l0, beta);
        const int32_t *trowA = TAB ? tab + (size_t)(l0 + k) * (p.N + 1) + bbA : nullptr;
        const int32_t *trowB = TAB ? tab + (size_t)(l0 + k) * (p.N + 1) + bbB : nullptr;
        int TA, TB;
        if (s0 == 0) {
            TA = p.div.ipt * bbA;
            TB = p.div.ipt * bbB;
        } else if (TAB) {
            TA = __ldg(&trowA[(size_t)s0 * (p.N + 1)]);
            TB = __ldg(&trowB[(size_t)s0 * (p.N + 1)]);
        } else {
            const int2 st = stk2[s0];
            TA = st.x;
            TB = st.y;
        }
        const int E = __shfl_sync(0xffffffffu, rr.e0, s0 & 31) >> 1;
        forward_walk_u2<PREC, SMEM_RING, SMEM_TICKS, TAB>(p, s, tick_day, trowA, trowB, rr, gacc, s0, beta, TA, TB, vwA,
                                                         vwB, S2, t, E, stk2);
    }
}

// Algorithm 1's update of one (OD, departure b) from its routes' adjoint sums
// gp_k: g = sum_k p_k gp_k (Eq. (flow) transposed).  SOLVE: Adagrad step and
// projection max(q, 0).  LOSS_GRAD: 2 g, and the dL/dtheta terms
// 2 q gp_k dp_k/dtheta with dp_k/dtheta = p_k sum_k' p_k' (C_k' - C_k)
// (Eq. (logit)), route-time differences taken first to avoid cancellation.
template <int PREC, class RouteK, class RouteGp>
__device__ __forceinline__ void od_update(const FusedParams &p, int day, int od, int b, int nr, RouteK route_k,
                                          RouteGp route_gp, double &dth) {
    if (!DODE_IN_BOUNDS(od, p.K, p.err, kSiteDemand) || !DODE_IN_BOUNDS(b, p.N, p.err, kSiteDemand)) return;
    const float *pt = p.pt + (size_t)day * p.P * p.Np;
    float g = 0.f;
    for (int i = 0; i < nr; ++i) g += __ldg(&pt[(size_t)route_k(i) * p.Np + b]) * route_gp(i);
    const size_t qi = ((size_t)day * p.K + od) * p.Np + b;
    if (p.mode == MODE_SOLVE) {
        const float Gv = p.G[qi] + g * g;
        float qv = p.q[qi] - p.eta * g / (sqrtf(Gv) + p.eps);
        qv = fmaxf(qv, 0.f);
        p.G[qi] = Gv;
        p.q[qi] = qv;
        if (PREC == 1) p.qb[qi] = __float2bfloat16_rn(qv);
    } else if (p.mode == MODE_LOSS_GRAD) {
        p.gout[qi] = 2.f * g;
        const float *Cd = p.C + (size_t)day * p.P * p.Np;
        for (int i = 0; i < nr; ++i) {
            const int k = route_k(i);
            const float ck = Cd[(size_t)k * p.Np + b];
            float dc = 0.f;
            for (int i2 = 0; i2 < nr; ++i2) {
                const int k2 = route_k(i2);
                dc += __ldg(&pt[(size_t)k2 * p.Np + b]) * (Cd[(size_t)k2 * p.Np + b] - ck);
            }
            dth += 2.0 * (double)p.q[qi] * (double)route_gp(i) * (double)__ldg(&pt[(size_t)k * p.Np + b]) *
                   (double)dc;
        }
    }
}

// The solve's update of one OD for both tiles of a pair task (departures bA,
// bB): the same arithmetic as od_update in SOLVE mode, with every global load of
// both tiles (accumulator, flow, route choice) issued before the first use, so
// that the pair pays one memory latency instead of a chain of them.
template <int PREC, class RouteK, class RouteGp2>
__device__ __forceinline__ void od_step2(const FusedParams &p, int day, int od, int bA, int bB, bool vwA, bool vwB,
                                         int nr, RouteK route_k, RouteGp2 route_gp2) {
    if (!DODE_IN_BOUNDS(od, p.K, p.err, kSiteDemand)) return;
    const float *pt = p.pt + (size_t)day * p.P * p.Np;
    const size_t row = ((size_t)day * p.K + od) * p.Np;
    const size_t qA = row + (vwA ? bA : 0), qB = row + (vwB ? bB : 0);
    const float GA = p.G[qA], GB = p.G[qB], xA = p.q[qA], xB = p.q[qB];
    float gA = 0.f, gB = 0.f;
    for (int i = 0; i < nr; ++i) {
        const float *pk = pt + (size_t)route_k(i) * p.Np;
        const float pa = __ldg(&pk[vwA ? bA : 0]), pb = __ldg(&pk[vwB ? bB : 0]);
        const float2 gp = route_gp2(i);
        gA += pa * gp.x;
        gB += pb * gp.y;
    }
    if (vwA) {
        const float Gv = GA + gA * gA;
        const float qv = fmaxf(xA - p.eta * gA / (sqrtf(Gv) + p.eps), 0.f);
        p.G[qA] = Gv;
        p.q[qA] = qv;
        if (PREC == 1) p.qb[qA] = __float2bfloat16_rn(qv);
    }
    if (vwB) {
        const float Gv = GB + gB * gB;
        const float qv = fmaxf(xB - p.eta * gB / (sqrtf(Gv) + p.eps), 0.f);
        p.G[qB] = Gv;
        p.q[qB] = qv;
        if (PREC == 1) p.qb[qB] = __float2bfloat16_rn(qv);
    }
}

__device__ __forceinline__ void add_dtheta(double dth, double *s_dth) {
    for (int off = 16; off > 0; off >>= 1) dth += __shfl_down_sync(0xffffffffu, dth, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(s_dth, dth);
}

// Adjoint walk of one route from depth j0: gathers r over every window on an
// observed link into the running route sum G.  On the shared ring no lane
// needs a range check: residual rows past the end of the day are staged as
// zeros, and lanes outside the tile never store their sums.
template <int PREC, bool SMEM_RING, bool SMEM_TICKS, bool TAB, bool LONG>
__device__ __forceinline__ float adjoint_walk(const FusedParams &p, const Shared &s, const int32_t *tick_day,
                                              const int32_t *trow, const RouteRegs &rr, const void *rb, int j0,
                                              int beta, int T, float G, bool vw, int *stk, float *gstk) {
    const int ipt = p.div.ipt, N = p.Nh;      // horizon: the day, and the first rows of a coupled next day
    const float *racc = SMEM_RING ? reinterpret_cast<const float *>(s.lo) : nullptr;
    for (int j = j0; j < beta; ++j) {
        const bool first32 = !LONG || j < 32;
        const int tb = __shfl_sync(0xffffffffu, first32 ? rr.t0 : rr.t1, j & 31);
        const int ob = __shfl_sync(0xffffffffu, first32 ? rr.o0 : rr.o1, j & 31);
        const int ev = __shfl_sync(0xffffffffu, first32 ? rr.e0 : rr.e1, j & 31);
        const int hi = __shfl_down_sync(0xffffffffu, T, 1);
        const int h0 = interval_of(T, p.div);
        if (ob != kInactive) {
            if (SMEM_RING || (vw && h0 < N)) {
                const int idx = ob + h0;
                const int e0 = h0 * ipt + ipt;
                const float inv = __fdividef(1.f, (float)(hi - T));
                const float d0 = first_share<PREC>(T, e0, inv);
                float a = d0 * rcell<PREC, SMEM_RING>(s, racc, rb, idx);
                if (hi > e0 && (SMEM_RING || h0 + 1 < N)) {
                    if (hi <= e0 + ipt)
                        a += (1.f - d0) * rcell<PREC, SMEM_RING>(s, racc, rb, idx + 1);
                    else
                        a += window_tail<PREC, SMEM_RING, false>(s, nullptr, rb, idx + 1, hi, e0, h0 + 1, N, ipt, inv,
                                                                 d0, 0.f);
                }
                G += a;
            }
        }
        T = next_entry<SMEM_TICKS, TAB>(p, s, tick_day, trow, j, T, tb, h0);
        if ((ev & 1) && DODE_IN_BOUNDS(j + 1, kMaxRouteLinks + 1, s.err, kSiteWalkStack)) {
            stk[j + 1] = T;
            gstk[j + 1] = G;
        }
    }
    return G;
}

// Adjoint task: the same walk gathers r over every window (B^T r at route
// level, Algorithm 1's gradient).  A route's sum is the partial sum stored at
// its start depth plus its own windows.  The ODs the group owns are updated
// here; routes of other ODs leave their sums in the CTA's route slot for the
// step pass.
template <int PREC, bool SMEM_RING, bool SMEM_TICKS, bool TAB>
__device__ void adjoint_task(const FusedParams &p, const Shared &s, int day, int g, int b0, const void *rb,
                             const int32_t *tab, double *s_dth) {
    const int lane = threadIdx.x & 31;
    const int b = b0 + lane;
    const int bb = min(b, p.N);
    const bool vw = (lane < kTileW) && (b < p.N);
    const int32_t *tick_day = p.ticks + (size_t)day * p.A * p.Np;
    const int N = p.N;
    const int i0 = s.gptr[g], m = s.gptr[g + 1] - i0;
    if (!DODE_IN_BOUNDS(m, kGroupRoutes + 1, s.err, kSiteGroupSums)) return;
    float *gp = p.gp + (size_t)blockIdx.x * p.P * p.Np;
    int stk[kMaxRouteLinks + 1];
    float gstk[kMaxRouteLinks + 1];
    float gpl[kGroupRoutes];
    for (int t = 0; t < m; ++t) {
        const int4 gr = s.groute[i0 + t];
        const int k = gr.x, l0 = gr.y, beta = gr.z, s0 = gr.w & 0xff;
        if (!DODE_IN_BOUNDS(beta - 1, kMaxRouteLinks, s.err, kSiteWalkStack) ||
            !DODE_IN_BOUNDS(s0, kMaxRouteLinks + 1, s.err, kSiteWalkStack))
            continue;
        const RouteRegs rr = load_route<SMEM_RING, SMEM_TICKS>(p, s, l0, beta);
        const int32_t *trow = TAB ? tab + (size_t)(l0 + k) * (N + 1) + bb : nullptr;
        const int T = walk_start<TAB>(p, trow, stk, s0, bb);
        const float G0 = s0 == 0 ? 0.f : gstk[s0];
        const float G = beta <= 32
                            ? adjoint_walk<PREC, SMEM_RING, SMEM_TICKS, TAB, false>(p, s, tick_day, trow, rr, rb, s0,
                                                                                   beta, T, G0, vw, stk, gstk)
                            : adjoint_walk<PREC, SMEM_RING, SMEM_TICKS, TAB, true>(p, s, tick_day, trow, rr, rb, s0,
                                                                                  beta, T, G0, vw, stk, gstk);
        gpl[t] = G;
        if (!((gr.w >> 8) & 1) && vw) gp[(size_t)k * p.Np + b] = G;
    }
    const int e0 = s.god_ptr[g], e1 = s.god_ptr[g + 1];
    if (e0 == e1) return;
    double dth = 0.0;
    if (vw) {
        for (int e = e0; e < e1; ++e) {
            const int r0 = s.godr_ptr[e];
            const int *gr = s.godr + r0;
            od_update<PREC>(p, day, s.god[e], b, s.godr_ptr[e + 1] - r0,
                            [&](int i) { return s.groute[i0 + gr[i]].x; }, [&](int i) { return gpl[gr[i]]; },
                            dth);
        }
    }
    if (p.mode == MODE_LOSS_GRAD) add_dtheta(dth, s_dth);
}


// Adjoint walk of one route for two tiles of the same group (see forward_walk_u2).
template <int PREC, bool SMEM_RING, bool SMEM_TICKS, bool TAB>
__device__ __forceinline__ void adjoint_walk2(const FusedParams &p, const Shared &s, const int32_t *tick_day,
                                              const int32_t *trowA, const int32_t *trowB, const RouteRegs &rr,
                                              const void *rb, int j0, int beta, int TA, int TB, float &GA, float &GB,
                                              bool vwA, bool vwB, int2 *stk2, float2 *gstk2) {
    const int ipt = p.div.ipt, N = p.Nh;      // horizon: the day, and the first rows of a coupled next day
    const float *racc = SMEM_RING ? reinterpret_cast<const float *>(s.lo) : nullptr;
    for (int j = j0; j < beta; ++j) {
        const int tb = __shfl_sync(0xffffffffu, rr.t0, j & 31);
        const int ob = __shfl_sync(0xffffffffu, rr.o0, j & 31);
        const int ev = __shfl_sync(0xffffffffu, rr.e0, j & 31);
        const int hiA = __shfl_down_sync(0xffffffffu, TA, 1);
        const int hiB = __shfl_down_sync(0xffffffffu, TB, 1);
        const int h0A = interval_of(TA, p.div);
        const int h0B = interval_of(TB, p.div);
        if (ob != kInactive) {
            if (SMEM_RING || (vwA && h0A < N)) {
                const int idx = ob + h0A;
                const int e0 = h0A * ipt + ipt;
                const float inv = __fdividef(1.f, (float)(hiA - TA));
                const float d0 = first_share<PREC>(TA, e0, inv);
                float a = d0 * rcell<PREC, SMEM_RING>(s, racc, rb, idx);
                if (hiA > e0 && (SMEM_RING || h0A + 1 < N)) {
                    if (hiA <= e0 + ipt)
                        a += (1.f - d0) * rcell<PREC, SMEM_RING>(s, racc, rb, idx + 1);
                    else
                        a += window_tail<PREC, SMEM_RING, false>(s, nullptr, rb, idx + 1, hiA, e0, h0A + 1, N, ipt, inv,
                                                                 d0, 0.f);
                }
                GA += a;
            }
            if (SMEM_RING || (vwB && h0B < N)) {
                const int idx = ob + h0B;
                const int e0 = h0B * ipt + ipt;
                const float inv = __fdividef(1.f, (float)(hiB - TB));
                const float d0 = first_share<PREC>(TB, e0, inv);
                float a = d0 * rcell<PREC, SMEM_RING>(s, racc, rb, idx);
                if (hiB > e0 && (SMEM_RING || h0B + 1 < N)) {
                    if (hiB <= e0 + ipt)
                        a += (1.f - d0) * rcell<PREC, SMEM_RING>(s, racc, rb, idx + 1);
                    else
                        a += window_tail<PREC, SMEM_RING, false>(s, nullptr, rb, idx + 1, hiB, e0, h0B + 1, N, ipt, inv,
                                                                 d0, 0.f);
                }
                GB += a;
            }
        }
        TA = next_entry<SMEM_TICKS, TAB>(p, s, tick_day, trowA, j, TA, tb, h0A);
        TB = next_entry<SMEM_TICKS, TAB>(p, s, tick_day, trowB, j, TB, tb, h0B);
        if ((ev & 1) && DODE_IN_BOUNDS(j + 1, kMaxRouteLinks + 1, s.err, kSiteWalkStack)) {
            stk2[j + 1] = make_int2(TA, TB);
            gstk2[j + 1] = make_float2(GA, GB);
        }
    }
}

// Adjoint task over both tiles of a phase for walk group g (b0 .. b0 + 61);
// stacks and route sums hold both tiles' values side by side.  Groups with a
// route past 32 links take two single-tile tasks.
template <int PREC, bool SMEM_RING, bool SMEM_TICKS, bool TAB>
__device__ void adjoint_task2(const FusedParams &p, const Shared &s, int day, int g, int b0, const void *rb,
                              const int32_t *tab, double *s_dth) {
    const int lane = threadIdx.x & 31;
    const int bA = b0 + lane, bB = b0 + kTileW + lane;
    const int bbA = min(bA, p.N), bbB = min(bB, p.N);
    const bool vwA = (lane < kTileW) && (bA < p.N), vwB = (lane < kTileW) && (bB < p.N);
    const int32_t *tick_day = p.ticks + (size_t)day * p.A * p.Np;
    const int N = p.N;
    const int i0 = s.gptr[g], m = s.gptr[g + 1] - i0;
    if (!DODE_IN_BOUNDS(m, kGroupRoutes + 1, s.err, kSiteGroupSums)) return;
    bool longr = false;                                   // a route past 32 links: single-tile walks
    for (int t = 0; t < m; ++t) longr = longr || s.groute[i0 + t].z > 32;
    if (longr) {
        adjoint_task<PREC, SMEM_RING, SMEM_TICKS, TAB>(p, s, day, g, b0, rb, tab, s_dth);
        adjoint_task<PREC, SMEM_RING, SMEM_TICKS, TAB>(p, s, day, g, b0 + kTileW, rb, tab, s_dth);
        return;
    }
    float *gp = p.gp + (size_t)blockIdx.x * p.P * p.Np;
    int2 stk2[kMaxRouteLinks + 1];
    float2 gstk2[kMaxRouteLinks + 1];
    float2 gpl2[kGroupRoutes];
    for (int t = 0; t < m; ++t) {
        const int4 gr = s.groute[i0 + t];
        const int k = gr.x, l0 = gr.y, beta = gr.z, s0 = gr.w & 0xff;
        if (!DODE_IN_BOUNDS(beta - 1, kMaxRouteLinks, s.err, kSiteWalkStack) ||
            !DODE_IN_BOUNDS(s0, kMaxRouteLinks + 1, s.err, kSiteWalkStack))
            continue;
        const RouteRegs rr = load_route<SMEM_RING, SMEM_TICKS>(p, s, l0, beta);
        const int32_t *trowA = TAB ? tab + (size_t)(l0 + k) * (N + 1) + bbA : nullptr;
        const int32_t *trowB = TAB ? tab + (size_t)(l0 + k) * (N + 1) + bbB : nullptr;
        int TA, TB;
        float GA = 0.f, GB = 0.f;
        if (s0 == 0) {
            TA = p.div.ipt * bbA;
            TB = p.div.ipt * bbB;
        } else {
            if (TAB) {
                TA = __ldg(&trowA[(size_t)s0 * (N + 1)]);
                TB = __ldg(&trowB[(size_t)s0 * (N + 1)]);
            } else {
                const int2 st = stk2[s0];
                TA = st.x;
                TB = st.y;
            }
            const float2 gs = gstk2[s0];
            GA = gs.x;
            GB = gs.y;
        }
        adjoint_walk2<PREC, SMEM_RING, SMEM_TICKS, TAB>(p, s, tick_day, trowA, trowB, rr, rb, s0, beta, TA, TB, GA, GB,
                                                       vwA, vwB, stk2, gstk2);
        gpl2[t] = make_float2(GA, GB);
        if (!((gr.w >> 8) & 1)) {
            if (vwA) gp[(size_t)k * p.Np + bA] = GA;
            if (vwB) gp[(size_t)k * p.Np + bB] = GB;
        }
    }
    const int e0 = s.god_ptr[g], e1 = s.god_ptr[g + 1];
    if (e0 == e1) return;
    if (p.mode == MODE_SOLVE) {
        for (int e = e0; e < e1; ++e) {
            const int r0 = s.godr_ptr[e];
            const int *gr = s.godr + r0;
            od_step2<PREC>(p, day, s.god[e], bA, bB, vwA, vwB, s.godr_ptr[e + 1] - r0,
                           [&](int i) { return s.groute[i0 + gr[i]].x; }, [&](int i) { return gpl2[gr[i]]; });
        }
        return;
    }
    double dth = 0.0;
    for (int e = e0; e < e1; ++e) {
        const int r0 = s.godr_ptr[e];
        const int *gr = s.godr + r0;
        const int od = s.god[e], nr = s.godr_ptr[e + 1] - r0;
        if (vwA)
            od_update<PREC>(p, day, od, bA, nr, [&](int i) { return s.groute[i0 + gr[i]].x; },
                            [&](int i) { return gpl2[gr[i]].x; }, dth);
        if (vwB)
            od_update<PREC>(p, day, od, bB, nr, [&](int i) { return s.groute[i0 + gr[i]].x; },
                            [&](int i) { return gpl2[gr[i]].y; }, dth);
    }
    if (p.mode == MODE_LOSS_GRAD) add_dtheta(dth, s_dth);
}

// After a phase's adjoint tasks: the ODs whose routes span several groups
// (only when an origin has more than kGroupRoutes routes).
template <int PREC>
__device__ void step_phase(const FusedParams &p, int day, int pb0, int span, double *s_dth) {
    const float *gp = p.gp + (size_t)blockIdx.x * p.P * p.Np;
    double dth = 0.0;
    const int n = p.n_step_ods * span;
    for (int x0 = 0; x0 < n; x0 += blockDim.x) {     // uniform trip count: add_dtheta shuffles the full warp
        const int x = x0 + threadIdx.x;
        if (x < n) {
            const int od = __ldg(&p.step_ods[x / span]);
            const int b = pb0 + (x - (x / span) * span);
            if (b < p.N) {
                const int r0 = __ldg(&p.od_ptr[od]);
                const int *rk = p.od_routes + r0;
                od_update<PREC>(p, day, od, b, __ldg(&p.od_ptr[od + 1]) - r0, [&](int i) { return __ldg(&rk[i]); },
                                [&](int i) { return gp[(size_t)__ldg(&rk[i]) * p.Np + b]; }, dth);
            }
        }
    }
    if (p.mode == MODE_LOSS_GRAD) add_dtheta(dth, s_dth);
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

// Tick rows [pb, pb + RW) of every link from the 16-bit table, whose entries
// past the end of the day repeat the last interval (the link entry rule clamps
// to it), or, for coupled days (t16n = the next day's table), continue with
// the next day's rows.  16-byte loads of 8 ticks at 8-aligned row positions,
// four per thread in flight before the shared stores; chunks past the table
// row take the last interval's value, chunks that reach past midnight of a
// coupled day are gathered tick by tick.
__device__ __forceinline__ void stage_ticks(const FusedParams &p, Shared &s, const uint16_t *t16,
                                            const uint16_t *t16n) {
    const int c0 = s.pb & ~7;
    const int nch = (s.pb + s.RW - c0 + 7) >> 3;       // 8-tick chunks per link
    const IntervalDiv dn = make_interval_div(max(nch, 2));
    const int total = p.A * nch;
    for (int i0 = threadIdx.x; i0 < total; i0 += 4 * blockDim.x) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            v[u] = make_uint4(0u, 0u, 0u, 0u);
            if (i < total) {
                const int a = div_by(i, nch, dn), c = c0 + 8 * (i - a * nch);
                const uint16_t *row = t16 + (size_t)a * p.Np;
                if (c + 8 <= (t16n ? p.N : p.Np)) {
                    v[u] = __ldg(reinterpret_cast<const uint4 *>(row + c));
                } else if (t16n) {
                    const uint16_t *nrow = t16n + (size_t)a * p.Np;
                    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int x = c + k;
                        const uint32_t t = x < p.N ? __ldg(row + x) : __ldg(nrow + min(x - p.N, p.N - 1));
                        w[k >> 1] |= t << ((k & 1) * 16);
                    }
                    v[u] = make_uint4(w[0], w[1], w[2], w[3]);
                } else {
                    uint32_t x = __ldg(row + p.Np - 1);
                    x |= x << 16;
                    v[u] = make_uint4(x, x, x, x);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < total) {
                const int a = div_by(i, nch, dn), c = c0 + 8 * (i - a * nch);
                if (!DODE_IN_BOUNDS(a, p.A, s.err, kSiteStageTicks)) continue;
                const uint32_t w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
                uint16_t *row = s.tw + a * s.RW;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int r = c + k - s.pb;
                    if (r >= 0 && r < s.RW) row[r] = (uint16_t)(w[k >> 1] >> ((k & 1) * 16));
                }
            }
        }
    }
}

// Residual of row r of the next day, seen from a coupled day: the next day's
// own deposits into its first rows (early) plus this day's spill into them
// (halo), turned into r = m (xhat - x) exactly as the next day's own flush
// does it (EXACT: FP64, else the solve path's FP32), in the residual slot's
// precision.
template <int PREC>
__device__ __forceinline__ uint32_t next_day_residual(const FusedParams &p, int day, int o, int r, bool exact) {
    const size_t S = (size_t)p.halo_rows, nc = (size_t)(day + 1) * p.O + o;
    const long long v = p.early[nc * S + r] + p.halo[((size_t)day * p.O + o) * S + r];
    const bool on = (__ldg(&p.mask[nc * p.Nw + (r >> 5)]) >> (r & 31)) & 1u;
    const float c = __ldg(&p.counts[nc * p.Np + r]);
    float rr;
    if (exact) {
        rr = on ? (float)((double)v * kFxInv - (double)c) : 0.f;
    } else {
        const float x = fmaf((float)(int)(v >> 32), 4096.f, __uint2float_rn((uint32_t)v) * 9.5367431640625e-7f);
        rr = on ? x - c : 0.f;
    }
    return __float_as_uint(PREC == 1 ? bf16_round(rr) : rr);
}

// Residual rows [pb, pb + R) of every observed link, as float bits in the
// accumulator array (rows past the end of the day are zero, or the next day's
// residuals for a coupled day): 16-byte loads (8 BF16 or 4 FP32 residuals) at
// aligned row positions, four per thread in flight.  The slot was written by
// this kernel, so the loads take the L2-coherent path, not the read-only one.
template <int PREC>
__device__ __forceinline__ void stage_residual(const FusedParams &p, Shared &s, const void *rb, int day,
                                               bool exact) {
    constexpr int E = PREC == 1 ? 8 : 4;              // residuals per 16 bytes
    const int rows = min(s.R, p.N - s.pb);
    const int c0 = s.pb & ~(E - 1);
    const int nch = (s.pb + rows - c0 + E - 1) / E;
    const IntervalDiv dn = make_interval_div(max(nch, 2));
    const int total = p.O * nch;
    for (int i0 = threadIdx.x; i0 < total; i0 += 4 * blockDim.x) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            v[u] = make_uint4(0u, 0u, 0u, 0u);
            if (i < total) {
                const int o = div_by(i, nch, dn), c = c0 + E * (i - o * nch);
                if (!DODE_IN_BOUNDS(o, p.O, s.err, kSiteStageResid)) continue;
                v[u] = __ldcg(reinterpret_cast<const uint4 *>(static_cast<const unsigned char *>(rb) +
                                                            ((size_t)o * p.Np + c) * (PREC == 1 ? 2 : 4)));
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < total) {
                const int o = div_by(i, nch, dn), c = c0 + E * (i - o * nch);
                if (!DODE_IN_BOUNDS(o, p.O, s.err, kSiteStageResid)) continue;
                const uint32_t w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
                uint32_t *row = s.lo + o * s.R;
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const int r = c + k - s.pb;
                    const uint32_t bits = PREC == 1 ? (k & 1 ? (w[k >> 1] & 0xffff0000u) : (w[k >> 1] << 16)) : w[k];
                    if (r >= 0 && r < rows) row[r] = bits;
                }
            }
        }
    }
    // rows past the end of the day gather nothing, except the first rows of a
    // coupled next day
    const int tail = s.R - rows;
    const bool next = p.coupled && day + 1 < p.n_days;
    for (int i = threadIdx.x; i < p.O * tail; i += blockDim.x) {
        const int o = i / tail, x = rows + (i - o * tail);
        const int r = s.pb + x - p.N;          // row of the next day (rows past its end: dropped)
        uint32_t bits = 0u;
        if (next && r >= 0 && r < min(p.halo_rows, p.N)) bits = next_day_residual<PREC>(p, day, o, r, exact);
        s.lo[o * s.R + x] = bits;
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
                        if (DODE_IN_BOUNDS(idx, s.ring_cells, s.err, kSiteFlushCell)) {
                            lo[u] = s.lo[idx];
                            if (carry) hi[u] = s.hi[idx];
                        }
                    } else if (DODE_IN_BOUNDS((size_t)o * p.Np + h, s.ring_cells, s.err, kSiteFlushCell)) {
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

// Solve-path flush of a phase (the !EXACT case of flush_phase), four rows per
// chunk: 16-byte loads of counts (and row-chunk labels) at 4-aligned row
// positions, one mask word, 8- or 16-byte residual stores.  Each thread issues
// the loads of U chunks before using any of them (one memory latency per U
// chunks, U kept small for the registers); chunks are summed in the same order
// as one at a time.
template <int PREC, bool SMEM_RING>
__device__ __forceinline__ void flush_solve(const FusedParams &p, const Shared &s, float *gacc, void *rb,
                                            const float *cnt, const uint32_t *mk, const int32_t *lab, int sel, int pb0,
                                            int rows, bool carry, float &ks, float &kc) {
    constexpr int U = 2;                  // chunks per thread whose loads are in flight together
    const int c0 = pb0 & ~3;
    const int nch = (pb0 + rows - c0 + 3) >> 2;
    const IntervalDiv dn = make_interval_div(max(nch, 2));
    const int total = p.O * nch;
    for (int i0 = threadIdx.x; i0 < total; i0 += U * blockDim.x) {
        float4 cv[U];
        uint32_t mw[U];
        int4 lv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * blockDim.x;
            cv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            mw[u] = 0u;
            lv[u] = make_int4(0, 0, 0, 0);
            if (i < total) {
                const int o = div_by(i, nch, dn), c = c0 + 4 * (i - o * nch);
                const size_t cell = (size_t)o * p.Np + c;
                cv[u] = __ldg(reinterpret_cast<const float4 *>(cnt + cell));
                mw[u] = (__ldg(&mk[(size_t)o * p.Nw + (c >> 5)]) >> (c & 31)) & 0xfu;
                if (sel >= 0) lv[u] = __ldcg(reinterpret_cast<const int4 *>(lab + cell));
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i >= total) continue;
            const int o = div_by(i, nch, dn), c = c0 + 4 * (i - o * nch);
            const size_t cell = (size_t)o * p.Np + c;
            const float cc[4] = {cv[u].x, cv[u].y, cv[u].z, cv[u].w};
            const int ll[4] = {lv[u].x, lv[u].y, lv[u].z, lv[u].w};
            float r4[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int r = c + k - pb0;
                const bool in = r >= 0 && r < rows;
                float x = 0.f;
                if (in) {
                    if (SMEM_RING) {
                        const int idx = o * s.R + r;
                        if (DODE_IN_BOUNDS(idx, s.ring_cells, s.err, kSiteFlushCell)) {
                            const int hw = carry ? s.hi[idx] : 0;
                            x = fmaf((float)hw, 4096.f, __uint2float_rn(s.lo[idx]) * 9.5367431640625e-7f);
                        }
                    } else if (DODE_IN_BOUNDS(cell + k, s.ring_cells, s.err, kSiteFlushCell)) {
                        x = gacc[cell + k];
                        gacc[cell + k] = 0.f;
                    }
                }
                const bool on = in && ((mw[u] >> k) & 1u);
                const float rr = on ? x - cc[k] : 0.f;
                const float y = rr * rr - kc;          // compensated (Kahan) sum
                const float t = ks + y;
                kc = (t - ks) - y;
                ks = t;
                r4[k] = (sel < 0 || (on && ll[k] == sel)) ? rr : 0.f;
            }
            if (c >= pb0 && c + 4 <= pb0 + rows) {
                if (PREC == 1) {
                    __nv_bfloat162 lo2 = __floats2bfloat162_rn(r4[0], r4[1]);
                    __nv_bfloat162 hi2 = __floats2bfloat162_rn(r4[2], r4[3]);
                    uint2 pk;
                    pk.x = *reinterpret_cast<uint32_t *>(&lo2);
                    pk.y = *reinterpret_cast<uint32_t *>(&hi2);
                    *reinterpret_cast<uint2 *>(static_cast<__nv_bfloat16 *>(rb) + cell) = pk;
                } else {
                    *reinterpret_cast<float4 *>(static_cast<float *>(rb) + cell) =
                        make_float4(r4[0], r4[1], r4[2], r4[3]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int r = c + k - pb0;
                    if (r >= 0 && r < rows) Operand<PREC>::store_r(rb, cell + k, r4[k]);
                }
            }
        }
    }
}

// Solve-path flush of a phase on the shared ring, fused with the move of its
// spill rows.  Each observed link's ring row belongs to one group of lanes of
// one warp (4-cell chunks at 4-aligned row positions), so no other warp touches
// it and the move needs no CTA barrier.  Every cell of rows [0, span) is read
// and cleared; rows [0, rows) become masked residuals r = m (xhat - x) (Eq.
// (nnls)), summed into the loss with a compensated FP32 sum and written to the
// residual slot; then the spill rows [span, span + spill) move to [0, spill) and
// are cleared.  The loads of U rows are in flight together.
template <int PREC>
__device__ __forceinline__ void flush_move_solve(const FusedParams &p, const Shared &s, void *rb, const float *cnt,
                                                 const uint32_t *mk, const int32_t *lab, int sel, int pb0, int rows,
                                                 int span, int spill, bool carry, float &ks, float &kc) {
    constexpr int U = 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c0 = pb0 & ~3;
    const int nch = (pb0 + span - c0 + 3) >> 2;          // chunks covering rows [0, span)
    const int lg = lane_group_log2(nch);
    const int L = 1 << lg, per = 32 >> lg;
    const int sub = lane >> lg, kq = lane & (L - 1);
    const int step = nw * per;
    for (int o0 = warp * per; o0 < p.O; o0 += U * step) {
        for (int k0 = 0; k0 < nch; k0 += L) {
            const int k = k0 + kq, c = c0 + 4 * k;
            float4 cv[U];
            uint32_t mw[U];
            int4 lv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int o = o0 + u * step + sub;
                cv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                mw[u] = 0u;
                lv[u] = make_int4(0, 0, 0, 0);
                if (o < p.O && k < nch && c < pb0 + rows) {
                    const size_t cell = (size_t)o * p.Np + c;
                    cv[u] = __ldg(reinterpret_cast<const float4 *>(cnt + cell));
                    mw[u] = (__ldg(&mk[(size_t)o * p.Nw + (c >> 5)]) >> (c & 31)) & 0xfu;
                    if (sel >= 0) lv[u] = __ldcg(reinterpret_cast<const int4 *>(lab + cell));
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int o = o0 + u * step + sub;
                if (o >= p.O || k >= nch) continue;
                const size_t cell = (size_t)o * p.Np + c;
                const float cc[4] = {cv[u].x, cv[u].y, cv[u].z, cv[u].w};
                const int ll[4] = {lv[u].x, lv[u].y, lv[u].z, lv[u].w};
                float r4[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = c + q - pb0;
                    float x = 0.f;
                    if (r >= 0 && r < span && DODE_IN_BOUNDS(o * s.R + r, s.ring_cells, s.err, kSiteFlushCell)) {
                        const int idx = o * s.R + r;
                        const int hw = carry ? s.hi[idx] : 0;
                        x = fmaf((float)hw, 4096.f, __uint2float_rn(s.lo[idx]) * 9.5367431640625e-7f);
                        s.lo[idx] = 0u;
                        if (carry) s.hi[idx] = 0;
                    }
                    const bool on = r >= 0 && r < rows && ((mw[u] >> q) & 1u);
                    const float rr = on ? x - cc[q] : 0.f;
                    const float y = rr * rr - kc;          // compensated (Kahan) sum
                    const float t = ks + y;
                    kc = (t - ks) - y;
                    ks = t;
                    r4[q] = (sel < 0 || (on && ll[q] == sel)) ? rr : 0.f;
                }
                if (c >= pb0 && c + 4 <= pb0 + rows) {
                    if (PREC == 1) {
                        __nv_bfloat162 lo2 = __floats2bfloat162_rn(r4[0], r4[1]);
                        __nv_bfloat162 hi2 = __floats2bfloat162_rn(r4[2], r4[3]);
                        uint2 pk;
                        pk.x = *reinterpret_cast<uint32_t *>(&lo2);
                        pk.y = *reinterpret_cast<uint32_t *>(&hi2);
                        *reinterpret_cast<uint2 *>(static_cast<__nv_bfloat16 *>(rb) + cell) = pk;
                    } else {
                        *reinterpret_cast<float4 *>(static_cast<float *>(rb) + cell) =
                            make_float4(r4[0], r4[1], r4[2], r4[3]);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int r = c + q - pb0;
                        if (r >= 0 && r < rows) Operand<PREC>::store_r(rb, cell + q, r4[q]);
                    }
                }
            }
        }
        __syncwarp();
        // spill rows to the front of each row this warp flushed
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int o = o0 + u * step + sub;
            if (o >= p.O) continue;
            uint32_t *lrow = s.lo + o * s.R;
            int *hrow = s.hi + o * s.R;
            for (int r = kq; r < spill; r += L) {
                if (!DODE_IN_BOUNDS(o * s.R + span + r, s.ring_cells, s.err, kSiteFlushCell)) break;
                lrow[r] = lrow[span + r];
                lrow[span + r] = 0u;
                if (carry) {
                    hrow[r] = hrow[span + r];
                    hrow[span + r] = 0;
                }
            }
        }
        __syncwarp();
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

// Task t of a phase of nt tiles: the first nb groups of the processing order
// (the largest walks) go as pairs of tiles when nt is even, the other groups
// as single tiles, so the tail of a phase is made of small tasks.
struct TaskRef {
    int g, b0;
    bool pair;
};

__device__ __forceinline__ int phase_tasks(int nt, int nb, int G) {
    if (nt & 1) nb = 0;
    return nb * (nt / 2) + (G - nb) * nt;
}

__device__ __forceinline__ TaskRef task_ref(int t, int nt, int nb, int pb0, const int *task_grp) {
    if (nt & 1) nb = 0;
    const int hp = nt / 2, np = nb * hp;
    if (t < np) return TaskRef{task_grp[t / hp], pb0 + (t % hp) * 2 * kTileW, true};
    t -= np;
    return TaskRef{task_grp[nb + t / nt], pb0 + (t % nt) * kTileW, false};
}

// Dynamic shared memory layout (16-byte aligned blocks):
//   groute int4[P] | gptr int[G+1] | task_grp int[G] |
//   OD tables int[G+1 + n_god + n_god+1 + n_godr] | colact u32[Ow] | lo u32[O][R] | tw u16[A][RW]
// Epoch slices.  The epochs of one day are a chain (each reads the demand and
// Adagrad state the one before wrote), so with one CTA per day the last round
// of days leaves most CTAs idle.  Cutting each day's epochs into S slices and
// handing out (slice, day) units slice-major keeps every CTA busy to within one
// slice: a day's slice s follows its slice s - 1 by D units in the queue.  The
// CTA that finishes a slice publishes it with a release store after its
// writes; the CTA that takes the next slice waits (bounded) for it with an
// acquire load.  A unit waits only on a unit taken earlier by a running CTA,
// so the waits always end.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int load_acquire(const int *a) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ void store_release(int *a, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// Thread 0: wait until day's slice count reaches `need`; false after wait_ns.
__device__ bool wait_slice(const FusedParams &p, int day, int need) {
    if (load_acquire(&p.progress[day]) >= need) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        __nanosleep(256);
        if (load_acquire(&p.progress[day]) >= need) return true;
        if ((long long)(global_ns() - t0) > p.wait_ns) return false;
    }
}

template <int PREC, bool SMEM_RING, bool SMEM_TICKS>
__global__ void __launch_bounds__(1024, 1) k_fused(const FusedParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shared s;
    s.R = SMEM_RING ? p.ring_rows : 0;
    s.RW = SMEM_TICKS ? p.tick_rows : 0;
    s.pb = 0;
    auto align16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    size_t off = 0;
    int4 *groute = reinterpret_cast<int4 *>(smem_raw + off);
    off = align16(off + (size_t)p.P * sizeof(int4));
    int *gptr = reinterpret_cast<int *>(smem_raw + off);
    off = align16(off + (size_t)(p.n_groups + 1) * sizeof(int));
    int *task_grp = reinterpret_cast<int *>(smem_raw + off);
    off = align16(off + (size_t)p.n_groups * sizeof(int));
    int *odt = reinterpret_cast<int *>(smem_raw + off);
    off = align16(off + (size_t)(p.n_groups + 1 + 2 * p.n_god + 1 + p.n_godr) * sizeof(int));
    uint32_t *colact = reinterpret_cast<uint32_t *>(smem_raw + off);
    off = align16(off + (size_t)p.Ow * sizeof(uint32_t));
    s.lo = reinterpret_cast<uint32_t *>(smem_raw + off);
    if (SMEM_RING) off = align16(off + (size_t)p.O * s.R * sizeof(uint32_t));
    s.tw = reinterpret_cast<uint16_t *>(smem_raw + off);
    s.colact = colact;
    s.groute = groute;
    s.gptr = gptr;
    s.task_grp = task_grp;
    s.god_ptr = odt;
    s.god = odt + p.n_groups + 1;
    s.godr_ptr = odt + p.n_groups + 1 + p.n_god;
    s.godr = odt + p.n_groups + 1 + 2 * p.n_god + 1;
    s.rtab = (p.rtab_off >= 0 && !p.rtab_packed) ? reinterpret_cast<const int2 *>(smem_raw + p.rtab_off) : nullptr;
    s.rtab32 = (p.rtab_off >= 0 && p.rtab_packed) ? reinterpret_cast<const uint32_t *>(smem_raw + p.rtab_off) : nullptr;
    s.hi = SMEM_RING ? reinterpret_cast<int *>(p.gring) + (size_t)blockIdx.x * p.O * s.R : nullptr;
    __shared__ int s_day;
    __shared__ int s_slice;
    __shared__ int s_task;
    __shared__ double s_red[32];
    __shared__ double s_dth;
    __shared__ int s_nrows;
    __shared__ int s_carry;
    s.carry = &s_carry;
    s.err = p.err;
    s.ring_cells = SMEM_RING ? p.O * s.R : p.O * p.Np;
    s.tick_cells = SMEM_TICKS ? p.A * s.RW : p.A * p.Np;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nthr = blockDim.x;
    const int ntiles = (p.N + kTileW - 1) / kTileW;
    void *rb = static_cast<unsigned char *>(p.rbuf) +
               (size_t)blockIdx.x * p.O * p.Np * (PREC == 1 ? sizeof(__nv_bfloat16) : sizeof(float));
    float *gacc = SMEM_RING ? nullptr : p.gring + (size_t)blockIdx.x * p.O * p.Np;

    // network tables
    for (int i = threadIdx.x; i < p.P; i += nthr) groute[i] = __ldg(&p.groute[i]);
    for (int i = threadIdx.x; i <= p.n_groups; i += nthr) gptr[i] = __ldg(&p.gptr[i]);
    for (int i = threadIdx.x; i < p.n_groups; i += nthr) task_grp[i] = __ldg(&p.task_grp[i]);
    for (int i = threadIdx.x; i <= p.n_groups; i += nthr) odt[i] = __ldg(&p.god_ptr[i]);
    for (int i = threadIdx.x; i < p.n_god; i += nthr) odt[p.n_groups + 1 + i] = __ldg(&p.god[i]);
    for (int i = threadIdx.x; i <= p.n_god; i += nthr) odt[p.n_groups + 1 + p.n_god + i] = __ldg(&p.godr_ptr[i]);
    for (int i = threadIdx.x; i < p.n_godr; i += nthr)
        odt[p.n_groups + 1 + 2 * p.n_god + 1 + i] = __ldg(&p.godr[i]);
    if (p.rtab_off >= 0 && p.rtab_packed) {
        uint32_t *rt = reinterpret_cast<uint32_t *>(smem_raw + p.rtab_off);
        for (int i = threadIdx.x; i < p.rptr_total; i += nthr) rt[i] = __ldg(&p.rtab32[i]);
    } else if (p.rtab_off >= 0) {
        int2 *rt = reinterpret_cast<int2 *>(smem_raw + p.rtab_off);
        for (int i = threadIdx.x; i < p.rptr_total; i += nthr) rt[i] = __ldg(&p.rtab[i]);
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
    const int nbg = p.n_pair_groups;                  // groups walked as tile pairs

    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int u = atomicAdd(p.queue, 1);
            const int sl = u / p.n_days, d = u - sl * p.n_days;
            int code = d;
            if (sl >= p.slices)
                code = -1;                                 // no work left
            else if (sl > 0 && !wait_slice(p, d, sl)) {
                set_error(p.err, kErrDeviceTimeout, d);
                code = -1;
            }
            s_day = code;
            s_slice = sl;
        }
        __syncthreads();
        const int day = s_day;
        if (day < 0) break;
        const int slice = s_slice;
        const int it_begin = (int)((long long)slice * p.iters / p.slices);
        const int it_end = (int)((long long)(slice + 1) * p.iters / p.slices);
        const bool has_next = p.coupled && day + 1 < p.n_days;
        // a coupled day also deposits on the next day's observed links (its trips
        // that cross midnight)
        for (int i = threadIdx.x; i < p.Ow; i += nthr)
            colact[i] = p.colact[(size_t)day * p.Ow + i] | (has_next ? p.colact[(size_t)(day + 1) * p.Ow + i] : 0u);
        const int64_t toff = p.tab_off[day];
        const int32_t *tab = toff >= 0 ? p.traj_tab + toff : nullptr;
        const int32_t *tick_day = p.ticks + (size_t)day * p.A * p.Np;
        const uint16_t *tick16_day = p.ticks16 + (size_t)day * p.A * p.Np;
        const uint16_t *tick16_next = has_next ? tick16_day + (size_t)p.A * p.Np : nullptr;
        const float *cnt = p.counts + (size_t)day * p.O * p.Np;
        const uint32_t *mk = p.mask + (size_t)day * p.O * p.Nw;
        // coupled days: every day keeps the context's largest offset, so that the
        // rows carried between phases always cover the halo rows
        const int maxoff = p.coupled ? p.halo_rows - 2 : p.maxoff[day];
        int tw_pb = -1;                   // phase whose tick rows the window holds (this day)
        // tiles per phase: the accumulators must hold a phase's arrival rows
        // (31 F + maxoff + 2) and the tick window its trajectories' entry rows
        // (31 F + maxoff + 1)
        int F = ntiles;
        if (SMEM_RING) F = min(F, (s.R - maxoff - 2) / kTileW);
        if (SMEM_TICKS) F = min(F, (s.RW - maxoff - 1) / kTileW);
        F = min(F, max(1, p.tiles_per_phase));
        if (p.mode == MODE_HALO) F = min(F, 1);      // one tile per phase: the halo pass walks two tiles
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
        for (int it = it_begin, chunk = 0;;) {
            if (chunked && it < p.iters && chunk == 0) nch = row_labels(p, mk, p.day_base + day, it, &s_nrows);
            const int sel = (chunked && it < p.iters) ? chunk : -1;     // chunk of rows in this update
            // ------------------------------ forward sweep ------------------------------
            double lsum = 0.0;     // EXACT calls: FP64 (finite differences of the loss resolve tiny changes)
            float ks = 0.f, kc = 0.f;  // solve: compensated FP32 sum
            const bool halo_pass = p.mode == MODE_HALO;
            if (SMEM_RING && p.coupled && day > 0 && !halo_pass) {
                // the previous day's trips that cross midnight: its deposits into
                // this day's first rows go in first (the ring is clear here)
                const long long *hin = p.halo + (size_t)(day - 1) * p.O * p.halo_rows;
                for (int i = threadIdx.x; i < p.O * p.halo_rows; i += nthr) {
                    const int o = i / p.halo_rows, r = i - o * p.halo_rows;
                    const long long v = hin[i];
                    s.lo[o * s.R + r] = (uint32_t)v;
                    const int hw = (int)(v >> 32);
                    if (hw) {
                        s.hi[o * s.R + r] = hw;
                        s_carry = 1;
                    }
                }
                __syncthreads();
            }
            // halo pass: only the phases that reach the first rows or midnight
            auto reaches = [&](int pb) {
                const int sp = min(F, (p.N - pb + kTileW - 1) / kTileW) * kTileW;
                return pb < p.halo_rows || pb + sp + maxoff + 2 > p.N;
            };
            int adv = F * kTileW;
            for (int pb0 = 0; pb0 < p.N; pb0 += adv) {
                adv = F * kTileW;
                const int nt = min(F, (p.N - pb0 + kTileW - 1) / kTileW);
                const int ntask = phase_tasks(nt, nbg, p.n_groups);
                const int span = nt * kTileW;
                const bool walk = !halo_pass || reaches(pb0);
                s.pb = pb0;
                // the solve and evaluation passes stage each later phase's ticks during the previous flush
                if (walk && SMEM_TICKS && !tab && (halo_pass || pb0 == 0) && tw_pb != pb0) {
                    stage_ticks(p, s, tick16_day, tick16_next);
                    tw_pb = pb0;
                    __syncthreads();
                }
                while (walk) {
                    int t = 0;
                    if (lane == 0) t = atomicAdd(&s_task, 1);
                    t = __shfl_sync(0xffffffffu, t, 0);
                    if (t >= ntask) break;
                    const TaskRef tr = task_ref(t, nt, nbg, pb0, task_grp);
                    if (tr.pair) {
                        if (tab)
                            forward_task2<PREC, SMEM_RING, SMEM_TICKS, true>(p, s, day, tr.g, tr.b0, tab);
                        else
                            forward_task2<PREC, SMEM_RING, SMEM_TICKS, false>(p, s, day, tr.g, tr.b0, tab);
                    } else {
                        if (tab)
                            forward_task<PREC, SMEM_RING, SMEM_TICKS, true>(p, s, day, tr.g, tr.b0, tab);
                        else
                            forward_task<PREC, SMEM_RING, SMEM_TICKS, false>(p, s, day, tr.g, tr.b0, tab);
                    }
                }
                __syncthreads();
                // rows [pb0, pb0 + 31 nt) are final: residual, loss, residual slot;
                // the spill rows move to the front for the next phase
                const int rows = min(span, p.N - pb0);
                const bool carry = s_carry != 0;
                if (halo_pass) {
                    if (SMEM_RING) {
                        const int S = p.halo_rows;
                        long long *early = p.early + (size_t)day * p.O * S;
                        long long *halo = p.halo + (size_t)day * p.O * S;
                        const int ne = pb0 < S ? min(rows, S - pb0) : 0;       // final rows of [0, S)
                        for (int i = threadIdx.x; i < p.O * ne; i += nthr) {
                            const int o = i / ne, r = i - o * ne, idx = o * s.R + r;
                            early[o * S + pb0 + r] = ((long long)(carry ? s.hi[idx] : 0) << 32) | (long long)s.lo[idx];
                        }
                        if (pb0 + span >= p.N) {                                // the day's last phase
                            for (int i = threadIdx.x; i < p.O * S; i += nthr) {
                                const int o = i / S, r = i - o * S, idx = o * s.R + (p.N - pb0) + r;
                                halo[i] = ((long long)(carry ? s.hi[idx] : 0) << 32) | (long long)s.lo[idx];
                            }
                        }
                    }
                } else if (exact)
                    flush_phase<PREC, SMEM_RING, true>(p, s, gacc, rb, cnt, mk, lab, sel, day, pb0, rows, carry, lsum,
                                                       ks, kc);
                else if (SMEM_RING)
                    flush_move_solve<PREC>(p, s, rb, cnt, mk, lab, sel, pb0, rows, span, spill, carry, ks, kc);
                else
                    flush_solve<PREC, SMEM_RING>(p, s, gacc, rb, cnt, mk, lab, sel, pb0, rows, carry, ks, kc);
                if (SMEM_TICKS && !tab && !halo_pass && pb0 + adv < p.N) {
                    // the tasks are done with the tick window: stage the next phase's rows now
                    s.pb = pb0 + adv;
                    stage_ticks(p, s, tick16_day, tick16_next);
                    tw_pb = pb0 + adv;
                    s.pb = pb0;
                }
                if (SMEM_RING && (halo_pass || exact)) {
                    // move the spill rows [span, span + spill) to the front, zero the rest
                    // (the solve's flush has done both for the rows it flushed)
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
                if (halo_pass) {
                    // jump over the phases it does not need; what the last walked
                    // phase left for them is not needed either: clear the ring
                    int nb = pb0 + adv;
                    while (nb < p.N && !reaches(nb)) nb += adv;
                    if (SMEM_RING && nb > pb0 + adv) {
                        const bool carry = s_carry != 0;
                        for (int i = threadIdx.x; i < p.O * s.R; i += nthr) {
                            s.lo[i] = 0u;
                            if (carry) s.hi[i] = 0;
                        }
                        __syncthreads();
                    }
                    adv = nb - pb0;
                }
            }
            if (SMEM_RING) {
                // the last phase's spill rows lie past the end of the day: clear them
                const bool carry = s_carry != 0;
                for (int i = threadIdx.x; i < p.O * spill; i += nthr) {
                    const int o = i / spill, idx = o * s.R + (i - o * spill);
                    s.lo[idx] = 0u;
                    if (carry) s.hi[idx] = 0;
                }
                __syncthreads();
            }
            const double loss_day = block_sum(exact ? lsum : (double)ks - (double)kc, s_red);
            if (threadIdx.x == 0 && chunk == 0) {
                if (p.mode == MODE_SOLVE && it < p.iters && p.trace) p.trace[(size_t)it * p.n_days + day] = (float)loss_day;
                if (!halo_pass && (p.mode != MODE_SOLVE || it == p.iters)) p.loss[day] = loss_day;
            }
            if (p.mode == MODE_FORWARD || p.mode == MODE_LOSS || halo_pass || (p.mode == MODE_SOLVE && it >= p.iters))
                break;
            if (chunked && nch == 0) {      // no observed row: the epoch makes no update
                ++it;
                continue;
            }

            // ------------------------------ adjoint sweep ------------------------------
            // last phase first: it still holds the forward's last tick window, and
            // the next forward sweep starts from the window this sweep ends with
            const int nph = (p.N + F * kTileW - 1) / (F * kTileW);
            for (int ph = nph - 1; ph >= 0; --ph) {
                const int pb0 = ph * F * kTileW;
                const int nt = min(F, (p.N - pb0 + kTileW - 1) / kTileW);
                const int ntask = phase_tasks(nt, nbg, p.n_groups);
                s.pb = pb0;
                __syncthreads();                           // previous phase done with the windows
                if (SMEM_TICKS && !tab && tw_pb != pb0) {
                    stage_ticks(p, s, tick16_day, tick16_next);
                    tw_pb = pb0;
                }
                if (SMEM_RING) stage_residual<PREC>(p, s, rb, day, exact);
                __syncthreads();
                while (true) {
                    int t = 0;
                    if (lane == 0) t = atomicAdd(&s_task, 1);
                    t = __shfl_sync(0xffffffffu, t, 0);
                    if (t >= ntask) break;
                    const TaskRef tr = task_ref(t, nt, nbg, pb0, task_grp);
                    if (tr.pair) {
                        if (tab)
                            adjoint_task2<PREC, SMEM_RING, SMEM_TICKS, true>(p, s, day, tr.g, tr.b0, rb, tab, &s_dth);
                        else
                            adjoint_task2<PREC, SMEM_RING, SMEM_TICKS, false>(p, s, day, tr.g, tr.b0, rb, tab, &s_dth);
                    } else {
                        if (tab)
                            adjoint_task<PREC, SMEM_RING, SMEM_TICKS, true>(p, s, day, tr.g, tr.b0, rb, tab, &s_dth);
                        else
                            adjoint_task<PREC, SMEM_RING, SMEM_TICKS, false>(p, s, day, tr.g, tr.b0, rb, tab, &s_dth);
                    }
                }
                __syncthreads();
                if (threadIdx.x == 0) s_task = 0;
                if (p.n_step_ods) step_phase<PREC>(p, day, pb0, nt * kTileW, &s_dth);
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
            if (p.no_final && it >= p.iters) break;        // the caller takes the final loss
            if (it >= it_end && it_end < p.iters) break;   // the slice's epochs are done
        }
        if (p.slices > 1) {
            __syncthreads();                               // the slice's writes of q and G ...
            if (threadIdx.x == 0) {
                __threadfence();
                store_release(&p.progress[day], slice + 1);   // ... before its count
            }
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
