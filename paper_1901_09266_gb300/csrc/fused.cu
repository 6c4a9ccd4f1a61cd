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
//    link-interval cells.
//  * Both sweeps run in phases of F tiles in time order.  A phase stages the
//    tick rows its trajectories can reach (departure rows plus the day's
//    largest trip offset, padded past the end of the day with the last row)
//    from global memory into shared memory.
//  * Forward sweep (xhat = B q, Eq. (reverse) with (flow)): windows deposit
//    p q rho into shared-memory accumulators for the phase's arrival rows.
//    After a phase every interval before the next phase's first departure is
//    final (no vehicle arrives before it departs): those rows become masked
//    residuals r = m (xhat - x), are summed into the loss (Eq. (nnls)) and are
//    written to the CTA's residual slot (global, L2-resident); the rows that
//    spill into the next phase are moved to the front of the accumulators.
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
// flows with global atomics.  No CTA ever waits on another CTA: the work queue
// is a single atomicAdd.
#include <climits>

#include "dode_internal.cuh"

namespace dode {

constexpr int kInactive = INT_MIN;

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
    float *acc;           // [O][R]: forward accumulators / adjoint residual window (row = h - pb)
    uint16_t *tw;         // [A][RW]: tick window (row = h - pb)
    const uint32_t *colact;
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
__device__ __forceinline__ void logit_norm(const FusedParams &p, const float *Cday, int r0, int r1, int bi,
                                           float &m, float &rden) {
    m = -INFINITY;
    for (int i = r0; i < r1; ++i) m = fmaxf(m, -p.theta * Cday[(size_t)__ldg(&p.od_routes[i]) * p.Np + bi]);
    float den = 0.f;
    for (int i = r0; i < r1; ++i) den += expf(-p.theta * Cday[(size_t)__ldg(&p.od_routes[i]) * p.Np + bi] - m);
    rden = 1.f / den;
}

// Cells of a window past its second one (the travel time jumped by more than
// one interval between consecutive departures): rare, handled by a loop.
// FP32: share = seg * scale.  BF16: share rounded, last share = remainder.
template <int PREC, bool DEPOSIT>
__device__ __noinline__ float window_tail(float *cellp, const void *rb, size_t gidx, bool smem, int hi, int e,
                                          int h, int N, int ipt, float scale, float used, float f) {
    float acc = 0.f;
    while (hi > e && h < N) {
        const int end = min(hi, e + ipt);
        float share;
        if (PREC == 0) {
            share = (float)(end - e) * scale;
        } else {
            share = end >= hi ? 1.f - used : bf16_round((float)(end - e) * scale);
            used += share;
        }
        if (DEPOSIT) {
            atomicAdd(cellp, f * share);
        } else {
            acc += share * (smem ? *cellp : Operand<PREC>::r(rb, gidx));
        }
        ++cellp;
        ++gidx;
        e += ipt;
        ++h;
    }
    return acc;
}

template <int PREC, bool SMEM_RING, bool SMEM_TICKS>
__device__ void forward_task(const FusedParams &p, const Shared &s, int day, int od, int b0,
                             const int32_t *tab) {
    const int lane = threadIdx.x & 31;
    const int b = b0 + lane;
    const int bb = min(b, p.N);
    const bool vw = (lane < kTileW) && (b < p.N);
    const int bi = min(b, p.N - 1);
    const int32_t *tick_day = p.ticks + (size_t)day * p.A * p.Np;
    const int r0 = __ldg(&p.od_ptr[od]), r1 = __ldg(&p.od_ptr[od + 1]);
    const float qv = vw ? Operand<PREC>::q(p, ((size_t)day * p.K + od) * p.Np + b) : 0.f;
    if (!__any_sync(0xffffffffu, qv != 0.f)) return;     // nothing departs: no deposits
    const int ipt = p.div.ipt, N = p.N;
    float *acc = SMEM_RING ? s.acc : p.gring + (size_t)blockIdx.x * p.O * p.Np;
    for (int i = r0; i < r1; ++i) {
        const int k = __ldg(&p.od_routes[i]);
        const float f = __ldg(&p.pt[((size_t)day * p.P + k) * p.Np + bi]) * qv;
        const int l0 = __ldg(&p.rptr[k]), beta = __ldg(&p.rptr[k + 1]) - l0;
        const RouteRegs rr = load_route<SMEM_RING, SMEM_TICKS>(p, s, l0, beta);
        const int32_t *trow = tab ? tab + (size_t)(l0 + k) * (N + 1) + bb : nullptr;
        int T = ipt * bb;
        for (int j = 0; j < beta; ++j) {
            const int tb = __shfl_sync(0xffffffffu, j < 32 ? rr.t0 : rr.t1, j & 31);
            const int ob = __shfl_sync(0xffffffffu, j < 32 ? rr.o0 : rr.o1, j & 31);
            const int hi = __shfl_down_sync(0xffffffffu, T, 1);
            const int h0 = interval_of(T, p.div);
            if (ob != kInactive && vw && h0 < N) {
                float *cell = acc + (ob + h0);
                const int w = hi - T;
                if (w == 0) {
                    atomicAdd(cell, f);
                } else {
                    const float inv = __fdividef(1.f, (float)w);
                    const int e0 = h0 * ipt + ipt;
                    const int end0 = min(hi, e0);
                    float s0, used = 0.f;
                    if (PREC == 0) {
                        s0 = (float)(end0 - T) * inv;
                    } else {
                        s0 = end0 >= hi ? 1.f : bf16_round((float)(end0 - T) * inv);
                        used = s0;
                    }
                    atomicAdd(cell, f * s0);
                    if (hi > e0 && h0 + 1 < N) {
                        const int end1 = min(hi, e0 + ipt);
                        float s1;
                        if (PREC == 0) {
                            s1 = (float)(end1 - e0) * inv;
                        } else {
                            s1 = end1 >= hi ? 1.f - used : bf16_round((float)(end1 - e0) * inv);
                            used += s1;
                        }
                        atomicAdd(cell + 1, f * s1);
                        if (hi > e0 + ipt && h0 + 2 < N)
                            window_tail<PREC, true>(cell + 2, nullptr, 0, true, hi, e0 + ipt, h0 + 2, N, ipt, inv,
                                                    used, f);
                    }
                }
            }
            if (trow) {
                T = __ldg(&trow[(size_t)(j + 1) * (N + 1)]);
            } else if (SMEM_TICKS) {
                T += s.tw[tb + h0];
            } else {
                T += __ldg(&tick_day[tb + min(h0, N - 1)]);
            }
        }
    }
}

template <int PREC, bool SMEM_RING, bool SMEM_TICKS>
__device__ void adjoint_task(const FusedParams &p, const Shared &s, int day, int od, int b0, const void *rb,
                             const int32_t *tab, double *s_dth) {
    const int lane = threadIdx.x & 31;
    const int b = b0 + lane;
    const int bb = min(b, p.N);
    const bool vw = (lane < kTileW) && (b < p.N);
    const int bi = min(b, p.N - 1);
    const int32_t *tick_day = p.ticks + (size_t)day * p.A * p.Np;
    const int r0 = __ldg(&p.od_ptr[od]), r1 = __ldg(&p.od_ptr[od + 1]);
    const int ipt = p.div.ipt, N = p.N;
    const size_t qi = ((size_t)day * p.K + od) * p.Np + b;
    const bool grad = p.mode == MODE_LOSS_GRAD;
    const float *Cday = p.C + (size_t)day * p.P * p.Np;
    float m = 0.f, rden = 1.f, cbar = 0.f;
    if (grad) {
        logit_norm(p, Cday, r0, r1, bi, m, rden);
        for (int i = r0; i < r1; ++i) {
            const float c = Cday[(size_t)__ldg(&p.od_routes[i]) * p.Np + bi];
            cbar += expf(-p.theta * c - m) * rden * c;
        }
    }
    const float *racc = SMEM_RING ? s.acc : nullptr;
    float g = 0.f, dth = 0.f;
    for (int i = r0; i < r1; ++i) {
        const int k = __ldg(&p.od_routes[i]);
        float pk, ck = 0.f;
        if (grad) {
            ck = Cday[(size_t)k * p.Np + bi];
            pk = expf(-p.theta * ck - m) * rden;
        } else {
            pk = __ldg(&p.pt[((size_t)day * p.P + k) * p.Np + bi]);
        }
        const int l0 = __ldg(&p.rptr[k]), beta = __ldg(&p.rptr[k + 1]) - l0;
        const RouteRegs rr = load_route<SMEM_RING, SMEM_TICKS>(p, s, l0, beta);
        const int32_t *trow = tab ? tab + (size_t)(l0 + k) * (N + 1) + bb : nullptr;
        float gp = 0.f;
        int T = ipt * bb;
        for (int j = 0; j < beta; ++j) {
            const int tb = __shfl_sync(0xffffffffu, j < 32 ? rr.t0 : rr.t1, j & 31);
            const int ob = __shfl_sync(0xffffffffu, j < 32 ? rr.o0 : rr.o1, j & 31);
            const int hi = __shfl_down_sync(0xffffffffu, T, 1);
            const int h0 = interval_of(T, p.div);
            if (ob != kInactive && vw && h0 < N) {
                const int idx = ob + h0;
                auto rv = [&](int d) -> float {
                    return SMEM_RING ? racc[idx + d] : Operand<PREC>::r(rb, (size_t)(idx + d));
                };
                const int w = hi - T;
                if (w == 0) {
                    gp += rv(0);
                } else {
                    const float inv = __fdividef(1.f, (float)w);
                    const int e0 = h0 * ipt + ipt;
                    const int end0 = min(hi, e0);
                    float a, used = 0.f;
                    if (PREC == 0) {
                        a = (float)(end0 - T) * rv(0);
                    } else {
                        const float s0 = end0 >= hi ? 1.f : bf16_round((float)(end0 - T) * inv);
                        used = s0;
                        a = s0 * rv(0);
                    }
                    if (hi > e0 && h0 + 1 < N) {
                        const int end1 = min(hi, e0 + ipt);
                        if (PREC == 0) {
                            a += (float)(end1 - e0) * rv(1);
                        } else {
                            const float s1 = end1 >= hi ? 1.f - used : bf16_round((float)(end1 - e0) * inv);
                            used += s1;
                            a += s1 * rv(1);
                        }
                        if (hi > e0 + ipt && h0 + 2 < N) {
                            float *cp = SMEM_RING ? const_cast<float *>(racc) + idx + 2 : nullptr;
                            a += window_tail<PREC, false>(cp, rb, (size_t)(idx + 2), SMEM_RING, hi, e0 + ipt, h0 + 2,
                                                          N, ipt, PREC == 0 ? 1.f : inv, used, 0.f);
                        }
                    }
                    gp += PREC == 0 ? a * inv : a;
                }
            }
            if (trow) {
                T = __ldg(&trow[(size_t)(j + 1) * (N + 1)]);
            } else if (SMEM_TICKS) {
                T += s.tw[tb + h0];
            } else {
                T += __ldg(&tick_day[tb + min(h0, N - 1)]);
            }
        }
        g += pk * gp;
        if (grad && vw) dth += 2.f * p.q[qi] * gp * pk * (cbar - ck);
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
        atomicAdd(s_dth, (double)dth);
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
// last interval (the link entry rule clamps to it).
__device__ __forceinline__ void stage_ticks(const FusedParams &p, Shared &s, const int32_t *tick_day) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int a = warp; a < p.A; a += nw) {
        const int32_t *src = tick_day + (size_t)a * p.Np;
        uint16_t *dst = s.tw + a * s.RW;
        for (int r = lane; r < s.RW; r += 32) dst[r] = (uint16_t)__ldg(&src[min(s.pb + r, p.N - 1)]);
    }
}

// Residual rows [pb, pb + R) (clipped to the day) of every observed link.
template <int PREC>
__device__ __forceinline__ void stage_residual(const FusedParams &p, Shared &s, const void *rb) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int rows = min(s.R, p.N - s.pb);
    for (int o = warp; o < p.O; o += nw) {
        float *dst = s.acc + o * s.R;
        for (int r = lane; r < rows; r += 32) dst[r] = Operand<PREC>::r(rb, (size_t)o * p.Np + s.pb + r);
    }
}

template <int PREC, bool SMEM_RING, bool SMEM_TICKS>
__global__ void __launch_bounds__(1024, 1) k_fused(const FusedParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shared s;
    s.R = SMEM_RING ? p.ring_rows : 0;
    s.RW = SMEM_TICKS ? p.tick_rows : 0;
    s.pb = 0;
    unsigned char *cur = smem_raw;
    s.acc = reinterpret_cast<float *>(cur);
    if (SMEM_RING) cur += (size_t)p.O * s.R * sizeof(float);
    uint32_t *colact = reinterpret_cast<uint32_t *>(cur);
    cur += (size_t)p.Ow * sizeof(uint32_t);
    cur = smem_raw + (((cur - smem_raw) + 15) & ~(size_t)15);
    s.tw = reinterpret_cast<uint16_t *>(cur);
    s.colact = colact;
    __shared__ int s_day;
    __shared__ int s_task;
    __shared__ double s_red[32];
    __shared__ double s_dth;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nthr = blockDim.x;
    const int ntiles = (p.N + kTileW - 1) / kTileW;
    void *rb = static_cast<unsigned char *>(p.rbuf) +
               (size_t)blockIdx.x * p.O * p.Np * (PREC == 1 ? sizeof(__nv_bfloat16) : sizeof(float));
    float *gacc = SMEM_RING ? nullptr : p.gring + (size_t)blockIdx.x * p.O * p.Np;

    if (SMEM_RING) {
        for (int i = threadIdx.x; i < p.O * s.R; i += nthr) s.acc[i] = 0.f;
    } else {
        for (size_t i = threadIdx.x; i < (size_t)p.O * p.Np; i += nthr) gacc[i] = 0.f;
    }
    if (threadIdx.x == 0) s_task = 0;

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

        for (int it = 0;; ++it) {
            // ------------------------------ forward sweep ------------------------------
            float lsum = 0.f;
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
                    const int od = __ldg(&p.task_od[t / nt]);
                    const int b0 = pb0 + (t % nt) * kTileW;
                    forward_task<PREC, SMEM_RING, SMEM_TICKS>(p, s, day, od, b0, tab);
                }
                __syncthreads();
                // rows [pb0, pb0 + 31 nt) are final: residual, loss, residual slot;
                // the spill rows move to the front for the next phase
                const int span = nt * kTileW;
                const int rows = min(span, p.N - pb0);
                for (int o = warp; o < p.O; o += nwarps) {
                    float *row = SMEM_RING ? s.acc + o * s.R : gacc + (size_t)o * p.Np + pb0;
                    for (int r = lane; r < rows; r += 32) {
                        const int h = pb0 + r;
                        const float x = row[r];
                        if (!SMEM_RING) row[r] = 0.f;
                        if (p.mode == MODE_FORWARD) {
                            p.xout[((size_t)day * p.O + o) * p.Np + h] = x;
                        } else {
                            const bool on = (mk[(size_t)o * p.Nw + (h >> 5)] >> (h & 31)) & 1u;
                            const float rr = on ? x - cnt[(size_t)o * p.Np + h] : 0.f;
                            lsum += rr * rr;
                            Operand<PREC>::store_r(rb, (size_t)o * p.Np + h, rr);
                        }
                    }
                    if (SMEM_RING) {
                        __syncwarp();
                        for (int q0 = 0; q0 < spill; q0 += 32) {
                            const int r = q0 + lane;
                            const float v = r < spill ? row[span + r] : 0.f;
                            __syncwarp();
                            if (r < spill) row[r] = v;
                            __syncwarp();
                        }
                        for (int r = spill + lane; r < span + spill; r += 32) row[r] = 0.f;
                    }
                }
                if (threadIdx.x == 0) s_task = 0;
                __syncthreads();
            }
            const double loss_day = block_sum((double)lsum, s_red);
            if (threadIdx.x == 0) {
                if (p.mode == MODE_SOLVE && it < p.iters && p.trace) p.trace[(size_t)it * p.n_days + day] = (float)loss_day;
                if (p.mode != MODE_SOLVE || it == p.iters) p.loss[day] = loss_day;
            }
            if (p.mode == MODE_FORWARD || p.mode == MODE_LOSS || (p.mode == MODE_SOLVE && it >= p.iters)) break;

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
                    const int od = __ldg(&p.task_od[t / nt]);
                    const int b0 = pb0 + (t % nt) * kTileW;
                    adjoint_task<PREC, SMEM_RING, SMEM_TICKS>(p, s, day, od, b0, rb, tab, &s_dth);
                }
                __syncthreads();
                if (threadIdx.x == 0) s_task = 0;
            }
            __syncthreads();
            if (SMEM_RING) {
                for (int i = threadIdx.x; i < p.O * s.R; i += nthr) s.acc[i] = 0.f;
            }
            __syncthreads();
            if (p.mode == MODE_LOSS_GRAD) {
                if (threadIdx.x == 0) p.dtheta[day] = s_dth;
                break;
            }
        }
    }
}

template <int PREC, bool SMEM_RING, bool SMEM_TICKS>
static cudaError_t launch_one(const FusedParams &p, int grid, int block, size_t smem, cudaStream_t s) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<PREC, SMEM_RING, SMEM_TICKS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_fused<PREC, SMEM_RING, SMEM_TICKS><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
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
