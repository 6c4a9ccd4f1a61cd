// api.cu -- host implementation of the C ABI declared in include/dode.h.
//
// The context owns every device buffer (cudaMalloc'd once per size change) and
// issues all work on its stream.  Inputs in the ABI's time-major layouts are
// converted to the kernels' time-innermost layouts on entry (dode_internal.cuh)
// and results converted back on exit.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "dode.h"
#include "dode_internal.cuh"

using namespace dode;

struct dode_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    int n_sm = 0;
    size_t smem_optin = 0;
    dode_options opt{};
    int N = 0, Np = 0, Nw = 0, ipt = 0, tps = 0, A = 0, O = 0, Ow = 0, K = 0, P = 0, L = 0;
    IntervalDiv div{};
    std::vector<int32_t> rptr, rlinks, rod, obs, obs_col, od_ptr, od_routes, task_od;
    std::vector<float> len;
    std::vector<int32_t> pair_k, pair_j, pair_o, rpp;  // observed (route, position) pairs
    std::vector<int2> rpack;                           // (link, observed column) per route position
    int2 *d_rpack = nullptr;
    // walk groups of the fused kernel (routes from one origin, lexicographic order)
    std::vector<int4> groute;                          // [P] (route, first position, links, start depth | flags)
    std::vector<int32_t> gptr, task_grp, rev;          // [G+1], [G], [L]
    std::vector<int32_t> god_ptr, god, godr_ptr, godr;  // ODs owned by each group and their routes
    std::vector<int32_t> step_ods;                     // ODs of groups that do not own them
    int G = 0;
    int4 *d_groute = nullptr;
    std::vector<int2> rtab;                            // [L] (link, (observed column + 1) | event word << 24)
    int2 *d_rtab = nullptr;
    std::vector<uint32_t> rtab32;                      // [L] the same in 32 bits (link | column + 1 << 11 | event
                                                       // << 22), when links and columns fit 11 bits; else empty
    uint32_t *d_rtab32 = nullptr;
    int32_t *d_gptr = nullptr, *d_task_grp = nullptr, *d_rev = nullptr;
    int32_t *d_god_ptr = nullptr, *d_god = nullptr, *d_godr_ptr = nullptr, *d_godr = nullptr, *d_step_ods = nullptr;
    float *d_pt = nullptr;                             // route choice table [D][P][Np]
    int32_t *d_rptr = nullptr, *d_rlinks = nullptr, *d_rod = nullptr, *d_obs_col = nullptr, *d_od_ptr = nullptr,
            *d_od_routes = nullptr, *d_task_od = nullptr;
    int32_t *d_pair_k = nullptr, *d_pair_j = nullptr, *d_pair_o = nullptr, *d_rpp = nullptr;
    float *d_len = nullptr;
    // days
    int D = 0;
    int32_t *d_ticks = nullptr;
    uint16_t *d_ticks16 = nullptr;
    float *d_counts = nullptr;
    uint32_t *d_mask = nullptr, *d_colact = nullptr;
    float *d_C = nullptr;
    // traffic patterns (Eq. (logit) on a pattern's mean travel times)
    float *d_Ceff = nullptr;                           // [D][P][Np] travel times of the route choice
    bool patterns = false;
    int32_t *d_maxoff = nullptr;
    unsigned long long *d_repairs = nullptr;
    int64_t *d_tab_off = nullptr;
    int32_t *d_traj_tab = nullptr;
    std::vector<int32_t> h_maxoff;
    std::vector<unsigned long long> h_repairs;
    int maxoff_max = 0;
    int max_tick = 0;
    // coupled days: early / halo rows of every day (MODE_HALO output)
    long long *d_early = nullptr, *d_halo = nullptr;
    int halo_rows = 0;
    float *d_q = nullptr, *d_G = nullptr, *d_qtmp = nullptr, *d_gout = nullptr, *d_xout = nullptr;
    __nv_bfloat16 *d_qb = nullptr;
    double *d_loss = nullptr, *d_dtheta = nullptr;
    int *d_progress = nullptr;   // [D] epoch slices done per day (fused solve with slices)
    int last_slices = 0;
    double *d_totals = nullptr;  // [2] cross-day totals (dode_last_totals)
    int totals_kind = 0;         // what d_loss / d_dtheta hold: 0 nothing, 1 losses, 2 losses and dL/dtheta
    float *d_trace = nullptr;
    size_t trace_cap = 0;
    int trace_iters = -1;
    void *d_rbuf = nullptr;
    size_t rbuf_bytes = 0;
    float *d_gring = nullptr;
    size_t gring_bytes = 0;
    // row-chunk ranking scratch (row_chunk > 0): chunk labels, key-bin counts, straddling-bin lists
    int32_t *d_lab = nullptr, *d_rc_row = nullptr;
    uint32_t *d_rc_bins = nullptr;
    unsigned long long *d_rc_key = nullptr;
    size_t rc_grid = 0;
    float *d_gp = nullptr;                             // [grid][P][Np] route-level adjoint sums
    size_t gp_bytes = 0;
    int *d_queue = nullptr, *d_err = nullptr;
    void *d_stage = nullptr;
    size_t stage_bytes = 0;
    // plain form
    int4 *d_rec = nullptr;
    float *d_p = nullptr;
    double *d_ptrace = nullptr;
    size_t ptrace_cap = 0;
    bool plain_ready = false;
    // timing
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double last_ms = 0.0;
    int64_t last_launches = 0;
    int32_t last_grid = 0;       // CTAs of the last fused-kernel launch
    int64_t total_launches = 0;
    // CUDA graph of dode_solve's device work (use_graph)
    cudaGraphExec_t graph_exec = nullptr;
    int graph_slices = 1;                  // epoch slices of the captured solve
    // the next batch of days copied ahead (dode_prefetch_days): [speeds | counts | mask]
    char *d_pref = nullptr;
    size_t pref_cap = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t pref_ev = nullptr;
    bool pref_pending = false;
    int pref_D = 0;
    const void *pref_src[3] = {nullptr, nullptr, nullptr};   // speeds, counts, mask of the pending copy
    size_t pref_off[3] = {0, 0, 0};
    cudaStream_t own_stream = nullptr;     // capture stream when the context uses the legacy default stream
    struct GraphKey {
        int iters = -1, grid = 0, block = 0, ring = 0, tick = 0, F = 0, prec = -1;
        float step = 0.f, theta = 0.f;
        const void *q_out = nullptr, *loss_out = nullptr;
        size_t smem = 0;
        bool operator==(const GraphKey &o) const {
            return iters == o.iters && grid == o.grid && block == o.block && ring == o.ring && tick == o.tick &&
                   F == o.F && prec == o.prec && step == o.step && theta == o.theta && q_out == o.q_out &&
                   loss_out == o.loss_out && smem == o.smem;
        }
    } graph_key;
    std::string err;
};

namespace {

void drop_graph(dode_ctx *ctx);

// Travel times the route choice uses: each day's own, or its pattern's mean.
const float *choice_C(const dode_ctx *ctx) { return ctx->patterns ? ctx->d_Ceff : ctx->d_C; }

int fail(dode_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

#define CU(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            (void)cudaGetLastError(); /* a non-sticky error must not surface in a later call */  \
            int code_ = (e_ == cudaErrorMemoryAllocation) ? DODE_ERR_OOM : DODE_ERR_CUDA;        \
            return fail(ctx, code_, std::string(#call) + ": " + cudaGetErrorString(e_));         \
        }                                                                                        \
    } while (0)

// a kernel launch: checked and counted
#define CUL(call)                  \
    do {                           \
        CU(call);                  \
        ++ctx->total_launches;     \
    } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t n) {
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
    }
    if (n == 0) n = 1;
    return cudaMalloc((void **)p, n * sizeof(T));
}

template <class T>
void dfree(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

template <class T>
cudaError_t upload(T **d, const std::vector<T> &h, cudaStream_t s) {
    cudaError_t e = dalloc(d, h.size());
    if (e != cudaSuccess) return e;
    if (h.empty()) return cudaSuccess;
    return cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

int set_device(dode_ctx *ctx) {
    CU(cudaSetDevice(ctx->dev));
    return DODE_OK;
}

// Staging buffer on the device for host <-> device copies in ABI layout.
int stage(dode_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->stage_bytes) return DODE_OK;
    if (ctx->d_stage) cudaFree(ctx->d_stage);
    ctx->d_stage = nullptr;
    ctx->stage_bytes = 0;
    CU(cudaMalloc(&ctx->d_stage, bytes));
    ctx->stage_bytes = bytes;
    return DODE_OK;
}

int check_device_error(dode_ctx *ctx) {
    int h[3] = {0, 0, 0};
    CU(cudaMemcpyAsync(h, ctx->d_err, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (h[0] == 0) return DODE_OK;
    long long idx = (long long)(uint32_t)h[1] | ((long long)h[2] << 31);
    char buf[256];
    if (h[0] == DODE_ERR_BAD_SPEED || h[0] == DODE_ERR_TICK_OVERFLOW) {
        long long a = idx % ctx->A, dh = idx / ctx->A;
        snprintf(buf, sizeof buf, "%s at day %lld, interval %lld, link %lld",
                 h[0] == DODE_ERR_BAD_SPEED ? "speed not finite and positive" : "link travel time above 2^24 ticks",
                 dh / ctx->N, dh % ctx->N, a);
    } else if (h[0] == DODE_ERR_BOUNDS) {
        long long i = idx & ((1ll << 40) - 1);
        if (i >= (1ll << 39)) i -= 1ll << 40;
        snprintf(buf, sizeof buf, "index check failed at site %lld: index %lld", idx >> 40, i);
    } else if (h[0] == DODE_ERR_UNSUPPORTED) {
        snprintf(buf, sizeof buf, "unsupported input at item %lld (window spans more intervals than this form handles)", idx);
    } else {
        snprintf(buf, sizeof buf, "device error %d at item %lld", h[0], idx);
    }
    CU(cudaMemsetAsync(ctx->d_err, 0, 4 * sizeof(int), ctx->stream));
    return fail(ctx, h[0], buf);
}

bool bad_ptr_kind(int k) { return k != DODE_PTR_HOST && k != DODE_PTR_DEVICE; }

// Copy an ABI-layout input to the device (no-op for device pointers).
int input(dode_ctx *ctx, const void *src, size_t bytes, int ptr_kind, size_t stage_off, const void **dev) {
    if (ptr_kind == DODE_PTR_DEVICE) {
        *dev = src;
        return DODE_OK;
    }
    char *dst = static_cast<char *>(ctx->d_stage) + stage_off;
    CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *dev = dst;
    return DODE_OK;
}

// [D][K][Np] internal -> [D][N][K] caller buffer.
int output_odmajor(dode_ctx *ctx, const float *src, float *dst, int M, float scale, int ptr_kind) {
    const size_t bytes = (size_t)ctx->D * ctx->N * M * sizeof(float);
    float *tgt = dst;
    if (ptr_kind == DODE_PTR_HOST) {
        int rc = stage(ctx, bytes);
        if (rc) return rc;
        tgt = static_cast<float *>(ctx->d_stage);
    }
    CUL(launch_transpose_out(src, tgt, ctx->D, ctx->N, ctx->Np, M, scale, ctx->stream));
    if (ptr_kind == DODE_PTR_HOST) CU(cudaMemcpyAsync(dst, tgt, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    return DODE_OK;
}

// [D][N][M] caller -> [D][M][Np] internal.
int input_odmajor(dode_ctx *ctx, const float *src, float *dst, int M, int ptr_kind) {
    const size_t bytes = (size_t)ctx->D * ctx->N * M * sizeof(float);
    const void *dsrc = src;
    if (ptr_kind == DODE_PTR_HOST) {
        int rc = stage(ctx, bytes);
        if (rc) return rc;
        rc = input(ctx, src, bytes, ptr_kind, 0, &dsrc);
        if (rc) return rc;
    }
    CUL(launch_transpose_in(static_cast<const float *>(dsrc), dst, ctx->D, ctx->N, ctx->Np, M, ctx->stream));
    return DODE_OK;
}

int output_plain(dode_ctx *ctx, const void *src, void *dst, size_t bytes, int ptr_kind) {
    CU(cudaMemcpyAsync(dst, src, bytes,
                       ptr_kind == DODE_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, ctx->stream));
    return DODE_OK;
}

struct FusedShape {
    int block, grid, ring_rows, tick_rows, tiles_per_phase;
    int rtab_off;          // byte offset of the route-position table in shared memory, -1 = read from global
    int rtab_packed;       // the shared copy is the 32-bit table
    size_t smem;
};

// Launch shape of the fused kernel: CTA size, CTAs per SM and the shared-memory
// windows.  The dynamic shared memory holds the OD / route tables, the day's
// active-column bits, the accumulators (R = 31 F + maxoff + 2 rows per observed
// link, 32-bit words) and, when every tick fits 16 bits, the tick window
// (RW = 31 F + maxoff + 1 rows per link).  The largest F up to 3 that fits is
// taken; otherwise ticks are read from global memory, and if even the
// accumulators do not fit the link flows accumulate in global memory.
static size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

size_t fused_smem_bytes(const dode_ctx *ctx, int R, int RW) {
    size_t off = align16((size_t)ctx->P * 16) + align16((size_t)(ctx->G + 1) * 4) + align16((size_t)ctx->G * 4) +
                 align16((ctx->god_ptr.size() + ctx->god.size() + ctx->godr_ptr.size() + ctx->godr.size()) * 4) +
                 align16((size_t)ctx->Ow * 4);
    if (R > 0) off = align16(off + (size_t)ctx->O * R * 4);
    if (RW > 0) off += (size_t)ctx->A * RW * 2;
    return off;
}

int fused_shape(dode_ctx *ctx, int precision, FusedShape *s) {
    const int ntiles = (ctx->N + kTileW - 1) / kTileW;
    const int per_sm = ctx->opt.ctas_per_sm > 0 ? ctx->opt.ctas_per_sm : 1;
    int block = ctx->opt.block_threads > 0 ? ctx->opt.block_threads : (per_sm == 1 ? 1024 : 512);
    block = std::max(32, std::min(1024, block / 32 * 32));
    const size_t reserve = 2048;
    size_t budget = std::min<size_t>(ctx->smem_optin, (size_t)(228 * 1024) / per_sm - 1024);
    budget = budget > reserve ? budget - reserve : 0;
    const bool ticks16 = ctx->max_tick <= 65535;
    const int mo = ctx->maxoff_max;
    int R = 0, RW = 0, F = 0;
    for (int f = std::min(3, ntiles); f >= 1 && F == 0; --f) {
        const int r = kTileW * f + mo + 2, rw = kTileW * f + mo + 1;
        if (ticks16 && fused_smem_bytes(ctx, r, rw) <= budget) {
            F = f;
            R = r;
            RW = rw;
        }
    }
    for (int f = std::min(3, ntiles); f >= 1 && F == 0; --f) {
        const int r = kTileW * f + mo + 2;
        if (fused_smem_bytes(ctx, r, 0) <= budget) {
            F = f;
            R = r;
        }
    }
    if (F == 0) F = ntiles;
    size_t smem = fused_smem_bytes(ctx, R, RW);
    // the route-position table goes to shared memory in its 32-bit form when it
    // fits beside the windows.  The 8-byte form stays in global memory: the
    // shared memory it would take costs more L1 (which holds the walks' local
    // stacks) than its loads save.
    s->rtab_off = -1;
    s->rtab_packed = 0;
    if (!ctx->rtab32.empty()) {
        const size_t rtab_bytes = align16((size_t)ctx->L * sizeof(uint32_t));
        if (align16(smem) + rtab_bytes <= budget) {
            s->rtab_off = (int)align16(smem);
            s->rtab_packed = 1;
            smem = align16(smem) + rtab_bytes;
        }
    }
    if (smem > budget + reserve)
        return fail(ctx, DODE_ERR_UNSUPPORTED, "route tables of this network do not fit in shared memory");
    if (ctx->opt.couple_days && (R == 0 || RW == 0))
        return fail(ctx, DODE_ERR_UNSUPPORTED,
                    "couple_days needs the accumulator ring and the tick window in shared memory");
    int occ = 0;
    cudaError_t e = fused_occupancy(precision, block, smem, &occ);
    if (e != cudaSuccess) return fail(ctx, DODE_ERR_CUDA, std::string("occupancy: ") + cudaGetErrorString(e));
    if (occ < 1) return fail(ctx, DODE_ERR_UNSUPPORTED, "fused kernel launch shape does not fit on an SM");
    occ = std::min(occ, per_sm);
    s->block = block;
    s->grid = std::max(1, std::min(ctx->D, ctx->n_sm * occ));
    if (ctx->opt.max_ctas > 0) s->grid = std::min(s->grid, ctx->opt.max_ctas);
    s->ring_rows = R;
    s->tick_rows = RW;
    s->tiles_per_phase = F;
    s->smem = smem;
    return DODE_OK;
}

int ensure_slots(dode_ctx *ctx, const FusedShape &s, int precision) {
    const size_t elems = (size_t)s.grid * ctx->O * ctx->Np;
    const size_t rb = elems * (precision == DODE_PREC_BF16 ? 2 : 4);
    if (rb > ctx->rbuf_bytes) {
        drop_graph(ctx);
        if (ctx->d_rbuf) cudaFree(ctx->d_rbuf);
        ctx->d_rbuf = nullptr;
        ctx->rbuf_bytes = 0;
        CU(cudaMalloc(&ctx->d_rbuf, rb));
        ctx->rbuf_bytes = rb;
    }
    // global accumulators (no shared ring) or the accumulators' high words
    const size_t gelems = (size_t)s.grid * ctx->O * std::max(ctx->Np, s.ring_rows);
    if (gelems * 4 > ctx->gring_bytes) {
        drop_graph(ctx);
        dfree(ctx->d_gring);
        ctx->gring_bytes = 0;
        CU(cudaMalloc(&ctx->d_gring, gelems * 4));
        ctx->gring_bytes = gelems * 4;
    }
    const size_t gpb = (size_t)s.grid * ctx->P * ctx->Np * sizeof(float);
    if (gpb > ctx->gp_bytes) {
        drop_graph(ctx);
        dfree(ctx->d_gp);
        ctx->gp_bytes = 0;
        CU(cudaMalloc(&ctx->d_gp, gpb));
        ctx->gp_bytes = gpb;
    }
    if (ctx->opt.row_chunk > 0 && (size_t)s.grid > ctx->rc_grid) {
        drop_graph(ctx);
        const size_t g = (size_t)s.grid, cells = (size_t)ctx->O * ctx->N;
        CU(dalloc(&ctx->d_lab, g * ctx->O * ctx->Np));
        CU(dalloc(&ctx->d_rc_bins, g * 3 * kRankBins));
        CU(dalloc(&ctx->d_rc_key, g * cells));
        CU(dalloc(&ctx->d_rc_row, g * cells));
        ctx->rc_grid = g;
    }
    return DODE_OK;
}

void slot_params(const dode_ctx *ctx, const FusedShape &s, FusedParams *p) {
    p->rbuf = ctx->d_rbuf;
    p->gring = ctx->d_gring;
    p->ring_rows = s.ring_rows;
    p->tick_rows = s.tick_rows;
    p->tiles_per_phase = s.tiles_per_phase;
    p->rtab_off = s.rtab_off;
    p->rtab_packed = s.rtab_packed;
    p->gp = ctx->d_gp;
    p->lab = ctx->d_lab;
    p->rc_bins = ctx->d_rc_bins;
    p->rc_key = ctx->d_rc_key;
    p->rc_row = ctx->d_rc_row;
}

// Walk groups of the fused kernel.  Every route leaving the same origin node
// starts at the same departure boundaries, so two such routes have identical
// trajectories over their common link prefix, and each window of that prefix
// carries the summed flow of the routes through it (forward) and is gathered
// once for all of them (adjoint).  Routes from one origin are put in
// lexicographic order of their link sequences -- a depth-first order of their
// prefix tree -- and cut into groups of at most kGroupRoutes.  In a group,
// route i is walked from its start depth s_i (its common prefix with route
// i - 1) to its end; per position j it records E (the last route of the group
// that shares the prefix up to and including link j, so the window's flow is
// routes i..E) and a save bit: a later route starts at depth j + 1 from this
// walk, which stores the entry time (and adjoint partial sum) there.
void build_groups(dode_ctx *ctx, const int32_t *link_tail) {
    const int P = ctx->P;
    auto links_of = [&](int k) {
        return std::vector<int32_t>(ctx->rlinks.begin() + ctx->rptr[k], ctx->rlinks.begin() + ctx->rptr[k + 1]);
    };
    std::vector<int> order(P);
    std::iota(order.begin(), order.end(), 0);
    std::vector<std::vector<int32_t>> seq(P);
    for (int k = 0; k < P; ++k) seq[k] = links_of(k);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const int oa = link_tail[seq[a][0]], ob = link_tail[seq[b][0]];
        if (oa != ob) return oa < ob;
        return seq[a] < seq[b];
    });
    auto lcp = [&](int a, int b) {
        const size_t n = std::min(seq[a].size(), seq[b].size());
        size_t i = 0;
        while (i < n && seq[a][i] == seq[b][i]) ++i;
        return (int)i;
    };
    ctx->groute.assign(P, make_int4(0, 0, 0, 0));
    ctx->rev.assign(ctx->L, 0);
    ctx->gptr.assign(1, 0);
    std::vector<long long> work;
    int i = 0;
    while (i < P) {
        // one origin's routes, cut into groups of at most kGroupRoutes
        int j = i;
        const int origin = link_tail[seq[order[i]][0]];
        while (j < P && link_tail[seq[order[j]][0]] == origin) ++j;
        for (int g0 = i; g0 < j; g0 += kGroupRoutes) {
            const int g1 = std::min(j, g0 + kGroupRoutes), m = g1 - g0;
            std::vector<int> r(order.begin() + g0, order.begin() + g1), st(m, 0);
            long long w = 0;
            for (int t = 0; t < m; ++t) {
                const int k = r[t];
                st[t] = t == 0 ? 0 : lcp(r[t - 1], k);
                const int beta = (int)seq[k].size();
                ctx->groute[g0 + t] = make_int4(k, ctx->rptr[k], beta, st[t]);
                w += beta - st[t];
                for (int d = st[t]; d < beta; ++d) {
                    int e = t;
                    while (e + 1 < m && lcp(k, r[e + 1]) >= d + 1) ++e;
                    ctx->rev[ctx->rptr[k] + d] = e << 1;
                }
            }
            // the walk that stores the state a later route starts from: the last
            // earlier route that passed depth s_e - 1
            for (int e = 1; e < m; ++e) {
                if (st[e] == 0) continue;
                int t = e - 1;
                while (st[t] > st[e] - 1) --t;
                ctx->rev[ctx->rptr[r[t]] + st[e] - 1] |= 1;
            }
            ctx->gptr.push_back(g1);
            work.push_back(w);
        }
        i = j;
    }
    ctx->G = (int)work.size();
    // a group owns an OD when it holds all of the OD's routes (always, unless an
    // origin has more than kGroupRoutes routes): its adjoint task then forms g
    // and takes the step itself; other ODs go through the step pass
    std::vector<int> gof(P);
    for (int g = 0; g < ctx->G; ++g)
        for (int x = ctx->gptr[g]; x < ctx->gptr[g + 1]; ++x) gof[ctx->groute[x].x] = g;
    std::vector<int> owner(ctx->K, -1);
    for (int od = 0; od < ctx->K; ++od) {
        int g0 = -1;
        bool one = true;
        for (int r = ctx->od_ptr[od]; r < ctx->od_ptr[od + 1]; ++r) {
            const int g = gof[ctx->od_routes[r]];
            if (g0 < 0) g0 = g;
            else if (g != g0) one = false;
        }
        owner[od] = one ? g0 : -1;
        if (!one) ctx->step_ods.push_back(od);
    }
    for (int x = 0; x < P; ++x)        // bit 8 of the start-depth word: the group owns the route's OD
        if (owner[ctx->rod[ctx->groute[x].x]] == gof[ctx->groute[x].x]) ctx->groute[x].w |= 1 << 8;
    for (int x = 0; x < P; ++x) ctx->groute[x].w |= ctx->rod[ctx->groute[x].x] << 9;   // bits 9..: the OD
    ctx->rtab.resize(ctx->L);
    for (int l = 0; l < ctx->L; ++l)
        ctx->rtab[l] = make_int2(ctx->rlinks[l], (ctx->obs_col[ctx->rlinks[l]] + 1) | (ctx->rev[l] << 24));
    ctx->rtab32.clear();
    if (ctx->A <= 2048 && ctx->O + 1 <= 2047) {
        ctx->rtab32.resize(ctx->L);
        for (int l = 0; l < ctx->L; ++l)
            ctx->rtab32[l] = (uint32_t)ctx->rlinks[l] | ((uint32_t)(ctx->obs_col[ctx->rlinks[l]] + 1) << 11) |
                             ((uint32_t)ctx->rev[l] << 22);
    }
    ctx->god_ptr.assign(1, 0);
    ctx->godr_ptr.assign(1, 0);
    for (int g = 0; g < ctx->G; ++g) {
        std::vector<int> ods;
        for (int x = ctx->gptr[g]; x < ctx->gptr[g + 1]; ++x) {
            const int od = ctx->rod[ctx->groute[x].x];
            if (owner[od] == g && std::find(ods.begin(), ods.end(), od) == ods.end()) ods.push_back(od);
        }
        for (int od : ods) {
            ctx->god.push_back(od);
            for (int x = ctx->gptr[g]; x < ctx->gptr[g + 1]; ++x)
                if (ctx->rod[ctx->groute[x].x] == od) ctx->godr.push_back(x - ctx->gptr[g]);
            ctx->godr_ptr.push_back((int32_t)ctx->godr.size());
        }
        ctx->god_ptr.push_back((int32_t)ctx->god.size());
    }
    ctx->task_grp.resize(ctx->G);
    std::iota(ctx->task_grp.begin(), ctx->task_grp.end(), 0);
    std::stable_sort(ctx->task_grp.begin(), ctx->task_grp.end(), [&](int a, int b) { return work[a] > work[b]; });
}

FusedParams base_params(dode_ctx *ctx) {
    FusedParams p{};
    p.N = ctx->N;
    p.Np = ctx->Np;
    p.Nw = ctx->Nw;
    p.A = ctx->A;
    p.O = ctx->O;
    p.Ow = ctx->Ow;
    p.K = ctx->K;
    p.P = ctx->P;
    p.div = ctx->div;
    p.rptr = ctx->d_rptr;
    p.rlinks = ctx->d_rlinks;
    p.obs_col = ctx->d_obs_col;
    p.od_ptr = ctx->d_od_ptr;
    p.od_routes = ctx->d_od_routes;
    p.task_od = ctx->d_task_od;
    p.rpack = ctx->d_rpack;
    p.groute = ctx->d_groute;
    p.rtab = ctx->d_rtab;
    p.rtab32 = ctx->d_rtab32;
    p.rtab_off = -1;
    p.rtab_packed = 0;
    p.rptr_total = ctx->L;
    p.gptr = ctx->d_gptr;
    p.task_grp = ctx->d_task_grp;
    p.rev = ctx->d_rev;
    p.rod = ctx->d_rod;
    p.n_groups = ctx->G;
    p.n_pair_groups = ctx->G;
    p.god_ptr = ctx->d_god_ptr;
    p.god = ctx->d_god;
    p.godr_ptr = ctx->d_godr_ptr;
    p.godr = ctx->d_godr;
    p.n_god = (int)ctx->god.size();
    p.n_godr = (int)ctx->godr.size();
    p.step_ods = ctx->d_step_ods;
    p.n_step_ods = (int)ctx->step_ods.size();
    p.pt = ctx->d_pt;
    p.ticks = ctx->d_ticks;
    p.ticks16 = ctx->d_ticks16;
    p.counts = ctx->d_counts;
    p.mask = ctx->d_mask;
    p.colact = ctx->d_colact;
    p.C = choice_C(ctx);
    p.maxoff = ctx->d_maxoff;
    p.tab_off = ctx->d_tab_off;
    p.traj_tab = ctx->d_traj_tab;
    p.q = ctx->d_q;
    p.G = ctx->d_G;
    p.qb = ctx->d_qb;
    p.loss = ctx->d_loss;
    p.dtheta = ctx->d_dtheta;
    p.n_days = ctx->D;
    p.eps = ctx->opt.eps;
    p.theta = ctx->opt.theta_per_min;
    p.queue = ctx->d_queue;
    p.err = ctx->d_err;
    p.row_chunk = 0;
    p.seed = ctx->opt.seed;
    p.day_base = ctx->opt.day_base;
    p.coupled = ctx->opt.couple_days;
    p.halo_rows = ctx->halo_rows;
    p.Nh = ctx->N + (ctx->opt.couple_days ? ctx->halo_rows : 0);
    p.early = ctx->d_early;
    p.halo = ctx->d_halo;
    p.no_final = 0;
    p.slices = 1;
    p.progress = nullptr;
    p.wait_ns = 20000000000LL;
    return p;
}

// Epoch slices of a fused solve over `grid` CTAs (see dode_options.epoch_slices):
// worth it once the days outnumber the CTAs (whole days would leave a partial
// last round); a day's next slice sits D > grid units after its last in the
// queue, about one slice's time later, so it is rarely waited for long.
int choose_slices(const dode_ctx *ctx, const FusedParams &p, int grid) {
    if (p.mode != MODE_SOLVE || p.coupled || p.iters < 2 || !ctx->d_progress) return 1;
    if (ctx->opt.epoch_slices > 0) return std::min(ctx->opt.epoch_slices, p.iters);
    if (p.iters < 8 || ctx->D <= grid) return 1;
    return std::min(16, p.iters / 4);
}

int run_fused(dode_ctx *ctx, FusedParams p, int precision) {
    FusedShape s;
    int rc = fused_shape(ctx, precision, &s);
    if (rc) return rc;
    rc = ensure_slots(ctx, s, precision);
    if (rc) return rc;
    slot_params(ctx, s, &p);
    CUL(launch_route_choice(choice_C(ctx), ctx->d_rod, ctx->d_od_ptr, ctx->d_od_routes, p.theta, ctx->D, ctx->P, ctx->N,
                            ctx->Np, ctx->d_pt, ctx->stream));
    CU(cudaEventRecord(ctx->ev0, ctx->stream));
    ctx->last_launches = 1;
    ctx->last_grid = s.grid;
    if (p.coupled) {
        // coupled days: every day's early rows and spill for this q first
        FusedParams ph = p;
        ph.mode = MODE_HALO;
        CU(cudaMemsetAsync(ctx->d_queue, 0, sizeof(int), ctx->stream));
        CUL(launch_fused(ph, precision, s.grid, s.block, s.smem, ctx->stream));
        ++ctx->last_launches;
    }
    p.slices = choose_slices(ctx, p, s.grid);
    ctx->last_slices = p.mode == MODE_SOLVE ? p.slices : ctx->last_slices;
    if (p.slices > 1) {
        p.progress = ctx->d_progress;
        CU(cudaMemsetAsync(ctx->d_progress, 0, (size_t)ctx->D * sizeof(int), ctx->stream));
    }
    CU(cudaMemsetAsync(ctx->d_queue, 0, sizeof(int), ctx->stream));
    CUL(launch_fused(p, precision, s.grid, s.block, s.smem, ctx->stream));
    CU(cudaEventRecord(ctx->ev1, ctx->stream));
    return DODE_OK;
}

// Coupled days (consecutive days solved jointly): Algorithm 1 with full-row
// updates on the joint problem.  Every epoch is a halo pass (each day's own
// deposits into its first rows and its spill past midnight, for the current
// q) and a one-epoch solve pass that adds the previous day's spill to each
// day's first rows and gathers the next day's first residual rows in the
// adjoint; the final loss is one more halo pass and a forward.
int solve_coupled(dode_ctx *ctx, FusedParams p, int iters) {
    const int prec = ctx->opt.precision;
    FusedShape s;
    int rc = fused_shape(ctx, prec, &s);
    if (rc) return rc;
    rc = ensure_slots(ctx, s, prec);
    if (rc) return rc;
    slot_params(ctx, s, &p);
    CUL(launch_route_choice(choice_C(ctx), ctx->d_rod, ctx->d_od_ptr, ctx->d_od_routes, p.theta, ctx->D, ctx->P, ctx->N,
                            ctx->Np, ctx->d_pt, ctx->stream));
    CU(cudaEventRecord(ctx->ev0, ctx->stream));
    FusedParams ph = p;
    ph.mode = MODE_HALO;
    for (int it = 0; it <= iters; ++it) {
        CU(cudaMemsetAsync(ctx->d_queue, 0, sizeof(int), ctx->stream));
        CUL(launch_fused(ph, prec, s.grid, s.block, s.smem, ctx->stream));
        FusedParams ps = p;
        ps.iters = it < iters ? 1 : 0;                  // the last pass: forward and final loss only
        ps.no_final = it < iters ? 1 : 0;
        ps.trace = (it < iters && p.trace) ? p.trace + (size_t)it * ctx->D : nullptr;
        CU(cudaMemsetAsync(ctx->d_queue, 0, sizeof(int), ctx->stream));
        CUL(launch_fused(ps, prec, s.grid, s.block, s.smem, ctx->stream));
    }
    CU(cudaEventRecord(ctx->ev1, ctx->stream));
    ctx->last_launches = 2LL * (iters + 1);
    ctx->last_grid = s.grid;
    return DODE_OK;
}

int finish_timing(dode_ctx *ctx) {
    CU(cudaEventSynchronize(ctx->ev1));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    ctx->last_ms = ms;
    return DODE_OK;
}

void drop_graph(dode_ctx *ctx) {
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
    ctx->graph_key = dode_ctx::GraphKey();
}

void free_days(dode_ctx *ctx) {
    drop_graph(ctx);
    dfree(ctx->d_ticks);
    dfree(ctx->d_ticks16);
    dfree(ctx->d_counts);
    dfree(ctx->d_mask);
    dfree(ctx->d_colact);
    dfree(ctx->d_C);
    dfree(ctx->d_Ceff);
    ctx->patterns = false;
    dfree(ctx->d_pt);
    dfree(ctx->d_maxoff);
    dfree(ctx->d_repairs);
    dfree(ctx->d_tab_off);
    dfree(ctx->d_traj_tab);
    dfree(ctx->d_q);
    dfree(ctx->d_G);
    dfree(ctx->d_qb);
    dfree(ctx->d_qtmp);
    dfree(ctx->d_gout);
    dfree(ctx->d_xout);
    dfree(ctx->d_loss);
    dfree(ctx->d_dtheta);
    dfree(ctx->d_progress);
    dfree(ctx->d_early);
    dfree(ctx->d_halo);
    ctx->halo_rows = 0;
    dfree(ctx->d_trace);
    ctx->trace_cap = 0;
    dfree(ctx->d_rec);
    dfree(ctx->d_p);
    dfree(ctx->d_ptrace);
    ctx->ptrace_cap = 0;
    ctx->plain_ready = false;
    ctx->D = 0;
}

// Plain form: build DAR records (all days) and route choice for theta.
int plain_prepare(dode_ctx *ctx, float theta, PlainParams *pp) {
    PlainParams p{};
    p.N = ctx->N;
    p.Np = ctx->Np;
    p.Nw = ctx->Nw;
    p.A = ctx->A;
    p.O = ctx->O;
    p.K = ctx->K;
    p.P = ctx->P;
    p.n_pairs = (int)ctx->pair_k.size();
    p.div = ctx->div;
    p.rptr = ctx->d_rptr;
    p.rlinks = ctx->d_rlinks;
    p.rod = ctx->d_rod;
    p.od_ptr = ctx->d_od_ptr;
    p.od_routes = ctx->d_od_routes;
    p.pair_k = ctx->d_pair_k;
    p.pair_j = ctx->d_pair_j;
    p.pair_o = ctx->d_pair_o;
    p.route_pair_ptr = ctx->d_rpp;
    p.ticks = ctx->d_ticks;
    p.tab_off = ctx->d_tab_off;
    p.traj_tab = ctx->d_traj_tab;
    p.C = choice_C(ctx);
    p.theta = theta;
    p.n_days = ctx->D;
    p.err = ctx->d_err;
    if (!ctx->plain_ready) {
        CU(dalloc(&ctx->d_rec, (size_t)ctx->D * p.n_pairs * ctx->N));
        CU(dalloc(&ctx->d_p, (size_t)ctx->D * ctx->P * ctx->Np));
    }
    p.rec = ctx->d_rec;
    p.p = ctx->d_p;
    if (!ctx->plain_ready) {
        CUL(launch_plain_build(p, ctx->stream));
        int rc = check_device_error(ctx);
        if (rc) return rc;
        ctx->plain_ready = true;
    }
    CUL(launch_plain_route_choice(p, ctx->stream));
    *pp = p;
    return DODE_OK;
}

// Fused solve as a CUDA graph: route choice, queue reset, the persistent
// kernel (between the timing events) and the copies to the caller's device
// buffers are captured once and replayed while iters, step, theta, the launch
// shape and the output pointers stay the same.
int solve_graph(dode_ctx *ctx, FusedParams p, int iters, float step, float *q_out, double *loss_out) {
    const int prec = ctx->opt.precision;
    FusedShape s;
    int rc = fused_shape(ctx, prec, &s);
    if (rc) return rc;
    rc = ensure_slots(ctx, s, prec);
    if (rc) return rc;
    CU(fused_set_attr(s.ring_rows > 0, s.tick_rows > 0, prec, s.smem));
    dode_ctx::GraphKey key;
    key.iters = iters;
    key.grid = s.grid;
    key.block = s.block;
    key.ring = s.ring_rows;
    key.tick = s.tick_rows;
    key.F = s.tiles_per_phase;
    key.prec = prec;
    key.step = step;
    key.theta = ctx->opt.theta_per_min;
    key.q_out = q_out;
    key.loss_out = loss_out;
    key.smem = s.smem;
    if (!ctx->stream && !ctx->own_stream) CU(cudaStreamCreate(&ctx->own_stream));
    cudaStream_t gs = ctx->stream ? ctx->stream : ctx->own_stream;
    int64_t kernels = 3 + (prec == DODE_PREC_BF16 ? 1 : 0) + (q_out ? 1 : 0);
    if (!ctx->graph_exec || !(key == ctx->graph_key)) {
        drop_graph(ctx);
        slot_params(ctx, s, &p);
        p.slices = choose_slices(ctx, p, s.grid);
        if (p.slices > 1) p.progress = ctx->d_progress;
        ctx->graph_slices = p.slices;
        CU(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        const int D = ctx->D;
        if (prec == DODE_PREC_BF16 && e == cudaSuccess)
            e = launch_to_bf16(ctx->d_q, ctx->d_qb, (size_t)D * ctx->K * ctx->Np, gs);
        if (e == cudaSuccess)
            e = launch_route_choice(choice_C(ctx), ctx->d_rod, ctx->d_od_ptr, ctx->d_od_routes, p.theta, D, ctx->P,
                                    ctx->N, ctx->Np, ctx->d_pt, gs);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_queue, 0, sizeof(int), gs);
        if (e == cudaSuccess && p.slices > 1)
            e = cudaMemsetAsync(ctx->d_progress, 0, (size_t)D * sizeof(int), gs);
        // external event-record nodes: the events complete with each replay, so
        // the kernel timer works for graph launches too
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(ctx->ev0, gs, cudaEventRecordExternal);
        if (e == cudaSuccess) e = launch_fused(p, prec, s.grid, s.block, s.smem, gs);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(ctx->ev1, gs, cudaEventRecordExternal);
        if (e == cudaSuccess && q_out)
            e = launch_transpose_out(ctx->d_q, q_out, D, ctx->N, ctx->Np, ctx->K, 1.f, gs);
        if (e == cudaSuccess && loss_out)
            e = cudaMemcpyAsync(loss_out, ctx->d_loss, D * sizeof(double), cudaMemcpyDeviceToDevice, gs);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(gs, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            ctx->graph_exec = nullptr;
            return fail(ctx, DODE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        }
        ctx->graph_key = key;
    }
    if (gs != ctx->stream) CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaGraphLaunch(ctx->graph_exec, gs));
    if (gs != ctx->stream) CU(cudaStreamSynchronize(gs));
    ctx->last_launches = 1;
    ctx->last_grid = s.grid;
    ctx->last_slices = ctx->graph_slices;
    ctx->total_launches += kernels;
    return DODE_OK;
}

}  // namespace

extern "C" {

int dode_set_max_ctas(dode_ctx *ctx, int32_t max_ctas) {
    if (!ctx) return DODE_ERR_ARG;
    if (max_ctas < 0) return fail(ctx, DODE_ERR_ARG, "max_ctas >= 0");
    ctx->opt.max_ctas = max_ctas;
    return DODE_OK;
}

void dode_default_options(dode_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->n_intervals = 288;
    o->interval_s = 300;
    o->ticks_per_s = 16;
    o->theta_per_min = 0.1f;
    o->eps = 1e-10f;
    o->row_chunk = 0;
    o->seed = 0;
    o->form = DODE_FORM_FUSED;
    o->precision = DODE_PREC_FP32;
    o->block_threads = 0;
    o->ctas_per_sm = 0;
    o->device = -1;
    o->stream = nullptr;
    o->use_graph = 0;
    o->max_ctas = 0;
}

const char *dode_last_error(const dode_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

double dode_last_kernel_ms(const dode_ctx *ctx) { return ctx ? ctx->last_ms : 0.0; }

int64_t dode_last_launches(const dode_ctx *ctx) { return ctx ? ctx->last_launches : 0; }

int32_t dode_last_grid(const dode_ctx *ctx) { return ctx ? ctx->last_grid : 0; }

int32_t dode_last_slices(const dode_ctx *ctx) { return ctx ? ctx->last_slices : 0; }

int32_t dode_device(const dode_ctx *ctx) { return ctx ? ctx->dev : -1; }

int64_t dode_total_launches(const dode_ctx *ctx) { return ctx ? ctx->total_launches : 0; }

int dode_create(const dode_network *net, const dode_routes *routes, const dode_options *opt, dode_ctx **out) {
    if (!out) return DODE_ERR_ARG;
    *out = nullptr;
    if (!net || !routes) return DODE_ERR_ARG;
    dode_options o;
    if (opt)
        o = *opt;
    else
        dode_default_options(&o);
    dode_ctx *ctx = new dode_ctx();
    auto bail = [&](int code, const std::string &m) {
        static thread_local std::string last;
        last = m;
        delete ctx;
        fprintf(stderr, "dode_create: %s\n", m.c_str());
        return code;
    };
    if (net->n_nodes < 1 || net->n_links < 1 || net->n_obs < 1 || !net->link_tail || !net->link_head ||
        !net->link_len_mi || !net->obs_links)
        return bail(DODE_ERR_ARG, "network sizes / pointers");
    if (routes->n_od < 1 || routes->n_routes < 1 || !routes->route_od || !routes->route_ptr || !routes->route_links)
        return bail(DODE_ERR_ARG, "route sizes / pointers");
    if (o.n_intervals < 1 || o.interval_s < 1 || o.ticks_per_s < 1 || !std::isfinite(o.theta_per_min) ||
        !(o.eps >= 0.f) || o.row_chunk < 0 || (o.form != DODE_FORM_FUSED && o.form != DODE_FORM_PLAIN) ||
        (o.precision != DODE_PREC_FP32 && o.precision != DODE_PREC_BF16) || o.block_threads < 0 || o.ctas_per_sm < 0 ||
        o.max_ctas < 0 || (o.use_graph != 0 && o.use_graph != 1) || o.day_base < 0 ||
        (o.couple_days != 0 && o.couple_days != 1) || o.epoch_slices < 0)
        return bail(DODE_ERR_ARG, "options");
    if (o.couple_days && (o.form != DODE_FORM_FUSED || o.row_chunk > 0))
        return bail(DODE_ERR_ARG, "couple_days needs the fused form with full-row updates (row_chunk = 0)");
    if (o.row_chunk > 0 && (long long)o.n_intervals * net->n_obs >= (1LL << 31))
        return bail(DODE_ERR_ARG, "row_chunk > 0 needs n_intervals * n_obs < 2^31 row ids");
    const long long ipt = (long long)o.interval_s * o.ticks_per_s;
    if (ipt < 2 || ipt > (1 << 24) || ipt * o.n_intervals > (1LL << 29))
        return bail(DODE_ERR_ARG, "interval of 2 .. 2^24 ticks and a day of at most 2^29 ticks");
    const int A = net->n_links, O = net->n_obs, K = routes->n_od, P = routes->n_routes;
    for (int a = 0; a < A; ++a) {
        if (net->link_tail[a] < 0 || net->link_tail[a] >= net->n_nodes || net->link_head[a] < 0 ||
            net->link_head[a] >= net->n_nodes)
            return bail(DODE_ERR_ARG, "link endpoint out of range at link " + std::to_string(a));
        if (!(net->link_len_mi[a] > 0.f) || !std::isfinite(net->link_len_mi[a]))
            return bail(DODE_ERR_ARG, "link length not finite and positive at link " + std::to_string(a));
    }
    std::vector<int32_t> obs_col(A, -1);
    for (int i = 0; i < O; ++i) {
        int a = net->obs_links[i];
        if (a < 0 || a >= A) return bail(DODE_ERR_ARG, "observed link id out of range");
        if (obs_col[a] >= 0) return bail(DODE_ERR_ARG, "observed link listed twice: " + std::to_string(a));
        obs_col[a] = i;
    }
    if (routes->route_ptr[0] != 0) return bail(DODE_ERR_ARG, "route_ptr[0] != 0");
    std::vector<int> od_count(K, 0);
    for (int k = 0; k < P; ++k) {
        const int od = routes->route_od[k];
        if (od < 0 || od >= K) return bail(DODE_ERR_ARG, "route_od out of range at route " + std::to_string(k));
        ++od_count[od];
        const int l0 = routes->route_ptr[k], l1 = routes->route_ptr[k + 1];
        if (l1 - l0 < 1 || l1 - l0 > DODE_MAX_ROUTE_LINKS)
            return bail(DODE_ERR_ARG, "route length outside 1..64 at route " + std::to_string(k));
        for (int j = l0; j < l1; ++j) {
            const int a = routes->route_links[j];
            if (a < 0 || a >= A) return bail(DODE_ERR_ARG, "route link out of range at route " + std::to_string(k));
            if (j + 1 < l1 && net->link_head[a] != net->link_tail[routes->route_links[j + 1]])
                return bail(DODE_ERR_ROUTE_NOT_CONTIGUOUS, "route " + std::to_string(k) + " not contiguous");
            for (int i = l0; i < j; ++i)
                if (routes->route_links[i] == a)
                    return bail(DODE_ERR_ROUTE_REPEATS_LINK, "route " + std::to_string(k) + " repeats a link");
        }
    }
    for (int od = 0; od < K; ++od)
        if (od_count[od] == 0) return bail(DODE_ERR_ARG, "OD pair without a route: " + std::to_string(od));
    if (K >= (1 << 22)) return bail(DODE_ERR_ARG, "at most 2^22 - 1 OD pairs");

    ctx->opt = o;
    ctx->N = o.n_intervals;
    ctx->Np = (o.n_intervals + 1 + 31) / 32 * 32;
    ctx->Nw = (o.n_intervals + 31) / 32;
    ctx->ipt = (int)ipt;
    ctx->tps = o.ticks_per_s;
    ctx->div = make_interval_div((int)ipt);
    ctx->A = A;
    ctx->O = O;
    ctx->Ow = (O + 31) / 32;
    ctx->K = K;
    ctx->P = P;
    ctx->L = routes->route_ptr[P];
    ctx->rptr.assign(routes->route_ptr, routes->route_ptr + P + 1);
    ctx->rlinks.assign(routes->route_links, routes->route_links + ctx->L);
    ctx->rod.assign(routes->route_od, routes->route_od + P);
    ctx->obs.assign(net->obs_links, net->obs_links + O);
    ctx->obs_col = obs_col;
    ctx->len.assign(net->link_len_mi, net->link_len_mi + A);
    // OD-major route order and OD tasks, largest walk first
    ctx->od_ptr.assign(K + 1, 0);
    for (int k = 0; k < P; ++k) ++ctx->od_ptr[ctx->rod[k] + 1];
    for (int od = 0; od < K; ++od) ctx->od_ptr[od + 1] += ctx->od_ptr[od];
    ctx->od_routes.assign(P, 0);
    {
        std::vector<int> fill(ctx->od_ptr.begin(), ctx->od_ptr.end() - 1);
        for (int k = 0; k < P; ++k) ctx->od_routes[fill[ctx->rod[k]]++] = k;
    }
    std::vector<long long> work(K, 0);
    for (int k = 0; k < P; ++k) work[ctx->rod[k]] += ctx->rptr[k + 1] - ctx->rptr[k];
    ctx->task_od.resize(K);
    std::iota(ctx->task_od.begin(), ctx->task_od.end(), 0);
    std::stable_sort(ctx->task_od.begin(), ctx->task_od.end(), [&](int a, int b) { return work[a] > work[b]; });
    ctx->rpack.resize(ctx->L);
    for (int j = 0; j < ctx->L; ++j) ctx->rpack[j] = make_int2(ctx->rlinks[j], obs_col[ctx->rlinks[j]]);
    build_groups(ctx, net->link_tail);
    // observed (route, position) pairs for the plain form
    ctx->rpp.assign(P + 1, 0);
    for (int k = 0; k < P; ++k) {
        for (int j = ctx->rptr[k]; j < ctx->rptr[k + 1]; ++j) {
            const int o2 = obs_col[ctx->rlinks[j]];
            if (o2 < 0) continue;
            ctx->pair_k.push_back(k);
            ctx->pair_j.push_back(j - ctx->rptr[k]);
            ctx->pair_o.push_back(o2);
        }
        ctx->rpp[k + 1] = (int32_t)ctx->pair_k.size();
    }

    if (o.device >= 0) {
        if (cudaSetDevice(o.device) != cudaSuccess) return bail(DODE_ERR_CUDA, "cudaSetDevice");
    }
    if (cudaGetDevice(&ctx->dev) != cudaSuccess) return bail(DODE_ERR_CUDA, "no CUDA device");
    ctx->stream = static_cast<cudaStream_t>(o.stream);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, ctx->dev) != cudaSuccess) return bail(DODE_ERR_CUDA, "device properties");
    ctx->n_sm = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
#define CUB(call)                                                              \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return bail(DODE_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)
    CUB(dalloc(&ctx->d_totals, 2));
    CUB(upload(&ctx->d_rptr, ctx->rptr, ctx->stream));
    CUB(upload(&ctx->d_rlinks, ctx->rlinks, ctx->stream));
    CUB(upload(&ctx->d_rod, ctx->rod, ctx->stream));
    CUB(upload(&ctx->d_obs_col, ctx->obs_col, ctx->stream));
    CUB(upload(&ctx->d_od_ptr, ctx->od_ptr, ctx->stream));
    CUB(upload(&ctx->d_od_routes, ctx->od_routes, ctx->stream));
    CUB(upload(&ctx->d_task_od, ctx->task_od, ctx->stream));
    CUB(upload(&ctx->d_pair_k, ctx->pair_k, ctx->stream));
    CUB(upload(&ctx->d_pair_j, ctx->pair_j, ctx->stream));
    CUB(upload(&ctx->d_pair_o, ctx->pair_o, ctx->stream));
    CUB(upload(&ctx->d_rpp, ctx->rpp, ctx->stream));
    CUB(upload(&ctx->d_len, ctx->len, ctx->stream));
    CUB(upload(&ctx->d_rpack, ctx->rpack, ctx->stream));
    CUB(upload(&ctx->d_groute, ctx->groute, ctx->stream));
    CUB(upload(&ctx->d_rtab, ctx->rtab, ctx->stream));
    if (!ctx->rtab32.empty()) CUB(upload(&ctx->d_rtab32, ctx->rtab32, ctx->stream));
    CUB(upload(&ctx->d_gptr, ctx->gptr, ctx->stream));
    CUB(upload(&ctx->d_task_grp, ctx->task_grp, ctx->stream));
    CUB(upload(&ctx->d_rev, ctx->rev, ctx->stream));
    CUB(upload(&ctx->d_god_ptr, ctx->god_ptr, ctx->stream));
    CUB(upload(&ctx->d_god, ctx->god, ctx->stream));
    CUB(upload(&ctx->d_godr_ptr, ctx->godr_ptr, ctx->stream));
    CUB(upload(&ctx->d_godr, ctx->godr, ctx->stream));
    CUB(upload(&ctx->d_step_ods, ctx->step_ods, ctx->stream));
    CUB(cudaMalloc(&ctx->d_queue, sizeof(int)));
    CUB(cudaMalloc(&ctx->d_err, 4 * sizeof(int)));
    CUB(cudaMemsetAsync(ctx->d_err, 0, 4 * sizeof(int), ctx->stream));
    CUB(cudaEventCreate(&ctx->ev0));
    CUB(cudaEventCreate(&ctx->ev1));
    CUB(cudaStreamSynchronize(ctx->stream));
#undef CUB
    *out = ctx;
    return DODE_OK;
}

void dode_destroy(dode_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->dev);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    free_days(ctx);
    dfree(ctx->d_totals);
    dfree(ctx->d_rptr);
    dfree(ctx->d_rlinks);
    dfree(ctx->d_rod);
    dfree(ctx->d_obs_col);
    dfree(ctx->d_od_ptr);
    dfree(ctx->d_od_routes);
    dfree(ctx->d_task_od);
    dfree(ctx->d_pair_k);
    dfree(ctx->d_pair_j);
    dfree(ctx->d_pair_o);
    dfree(ctx->d_rpp);
    dfree(ctx->d_len);
    dfree(ctx->d_rpack);
    dfree(ctx->d_groute);
    dfree(ctx->d_rtab);
    dfree(ctx->d_rtab32);
    dfree(ctx->d_gptr);
    dfree(ctx->d_task_grp);
    dfree(ctx->d_rev);
    dfree(ctx->d_god_ptr);
    dfree(ctx->d_god);
    dfree(ctx->d_godr_ptr);
    dfree(ctx->d_godr);
    dfree(ctx->d_step_ods);
    dfree(ctx->d_queue);
    dfree(ctx->d_err);
    if (ctx->d_rbuf) cudaFree(ctx->d_rbuf);
    dfree(ctx->d_gring);
    dfree(ctx->d_gp);
    dfree(ctx->d_lab);
    dfree(ctx->d_rc_bins);
    dfree(ctx->d_rc_key);
    dfree(ctx->d_rc_row);
    if (ctx->d_stage) cudaFree(ctx->d_stage);
    if (ctx->pref_ev) {
        cudaEventSynchronize(ctx->pref_ev);
        cudaEventDestroy(ctx->pref_ev);
    }
    if (ctx->d_pref) cudaFree(ctx->d_pref);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}

int dode_set_stream(dode_ctx *ctx, void *stream) {
    if (!ctx) return DODE_ERR_ARG;
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->opt.stream = stream;
    return DODE_OK;
}

int dode_set_launch(dode_ctx *ctx, int32_t block_threads, int32_t ctas_per_sm) {
    if (!ctx) return DODE_ERR_ARG;
    if (block_threads < 0 || block_threads > 1024 || block_threads % 32 || ctas_per_sm < 0 || ctas_per_sm > 8)
        return fail(ctx, DODE_ERR_ARG, "launch shape: block_threads multiple of 32 up to 1024, ctas_per_sm 0..8");
    ctx->opt.block_threads = block_threads;
    ctx->opt.ctas_per_sm = ctas_per_sm;
    return DODE_OK;
}

int dode_prefetch_days(dode_ctx *ctx, int32_t n_days, const float *counts, const float *speeds,
                       const uint8_t *mask) {
    if (!ctx) return DODE_ERR_ARG;
    if (n_days < 1 || !counts || !speeds) return fail(ctx, DODE_ERR_ARG, "prefetch_days arguments");
    int rc = set_device(ctx);
    if (rc) return rc;
    if (ctx->pref_pending) {                      // the previous copy must land before its buffer is reused
        CU(cudaEventSynchronize(ctx->pref_ev));
        ctx->pref_pending = false;
    }
    const size_t D = (size_t)n_days, N = ctx->N;
    const size_t sp_bytes = D * N * ctx->A * sizeof(float), ct_bytes = D * N * ctx->O * sizeof(float);
    const size_t mk_bytes = mask ? D * N * ctx->O : 0;
    auto align256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t off_ct = align256(sp_bytes), off_mk = off_ct + align256(ct_bytes);
    const size_t need = off_mk + mk_bytes;
    if (need > ctx->pref_cap) {
        if (ctx->d_pref) cudaFree(ctx->d_pref);
        ctx->d_pref = nullptr;
        ctx->pref_cap = 0;
        if (cudaMalloc(&ctx->d_pref, need) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(ctx, DODE_ERR_OOM, "prefetch buffer");
        }
        ctx->pref_cap = need;
    }
    if (!ctx->copy_stream) CU(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    if (!ctx->pref_ev) CU(cudaEventCreateWithFlags(&ctx->pref_ev, cudaEventDisableTiming));
    CU(cudaMemcpyAsync(ctx->d_pref, speeds, sp_bytes, cudaMemcpyHostToDevice, ctx->copy_stream));
    CU(cudaMemcpyAsync(ctx->d_pref + off_ct, counts, ct_bytes, cudaMemcpyHostToDevice, ctx->copy_stream));
    if (mask) CU(cudaMemcpyAsync(ctx->d_pref + off_mk, mask, mk_bytes, cudaMemcpyHostToDevice, ctx->copy_stream));
    CU(cudaEventRecord(ctx->pref_ev, ctx->copy_stream));
    ctx->pref_pending = true;
    ctx->pref_D = n_days;
    ctx->pref_src[0] = speeds;
    ctx->pref_src[1] = counts;
    ctx->pref_src[2] = mask;
    ctx->pref_off[0] = 0;
    ctx->pref_off[1] = off_ct;
    ctx->pref_off[2] = off_mk;
    return DODE_OK;
}

int dode_set_days(dode_ctx *ctx, int32_t n_days, const float *counts, const float *speeds, const uint8_t *mask,
                  int32_t ptr_kind) {
    if (!ctx) return DODE_ERR_ARG;
    if (n_days < 1 || !counts || !speeds || bad_ptr_kind(ptr_kind)) return fail(ctx, DODE_ERR_ARG, "set_days arguments");
    int rc = set_device(ctx);
    if (rc) return rc;
    if (ctx->pref_pending) {
        // host buffers copied ahead by dode_prefetch_days: take the device copies
        if (ptr_kind == DODE_PTR_HOST && n_days == ctx->pref_D && speeds == ctx->pref_src[0] &&
            counts == ctx->pref_src[1] && mask == ctx->pref_src[2]) {
            CU(cudaStreamWaitEvent(ctx->stream, ctx->pref_ev, 0));
            speeds = reinterpret_cast<const float *>(ctx->d_pref + ctx->pref_off[0]);
            counts = reinterpret_cast<const float *>(ctx->d_pref + ctx->pref_off[1]);
            if (mask) mask = reinterpret_cast<const uint8_t *>(ctx->d_pref + ctx->pref_off[2]);
            ptr_kind = DODE_PTR_DEVICE;
        } else {
            CU(cudaEventSynchronize(ctx->pref_ev));   // other inputs: the copy is not used
        }
        ctx->pref_pending = false;
    }
    CU(cudaStreamSynchronize(ctx->stream));
    const int D = n_days, N = ctx->N, Np = ctx->Np, A = ctx->A, O = ctx->O;
    if (D != ctx->D) {
        free_days(ctx);
        CU(dalloc(&ctx->d_ticks, (size_t)D * A * Np));
        CU(dalloc(&ctx->d_ticks16, (size_t)D * A * Np));
        CU(dalloc(&ctx->d_counts, (size_t)D * O * Np));
        CU(dalloc(&ctx->d_mask, (size_t)D * O * ctx->Nw));
        CU(dalloc(&ctx->d_colact, (size_t)D * ctx->Ow));
        CU(dalloc(&ctx->d_C, (size_t)D * ctx->P * Np));
        CU(dalloc(&ctx->d_pt, (size_t)D * ctx->P * Np));
        CU(dalloc(&ctx->d_maxoff, (size_t)D));
        CU(dalloc(&ctx->d_repairs, (size_t)D));
        CU(dalloc(&ctx->d_tab_off, (size_t)D));
        CU(dalloc(&ctx->d_q, (size_t)D * ctx->K * Np));
        CU(dalloc(&ctx->d_G, (size_t)D * ctx->K * Np));
        CU(dalloc(&ctx->d_qb, (size_t)D * ctx->K * Np));
        CU(dalloc(&ctx->d_qtmp, (size_t)D * ctx->K * Np));
        CU(dalloc(&ctx->d_loss, (size_t)D));
        CU(dalloc(&ctx->d_dtheta, (size_t)D));
        CU(dalloc(&ctx->d_progress, (size_t)D));
        ctx->D = D;
    }
    ctx->plain_ready = false;
    ctx->totals_kind = 0;
    ctx->trace_iters = -1;
    ctx->patterns = false;
    // speeds -> ticks (staged through the device when on the host)
    const size_t sp_bytes = (size_t)D * N * A * sizeof(float);
    const size_t ct_bytes = (size_t)D * N * O * sizeof(float);
    const size_t mk_bytes = mask ? (size_t)D * N * O : 0;
    if (ptr_kind == DODE_PTR_HOST) {
        rc = stage(ctx, std::max(sp_bytes, ct_bytes + mk_bytes));
        if (rc) return rc;
    }
    const void *dsp = nullptr;
    rc = input(ctx, speeds, sp_bytes, ptr_kind, 0, &dsp);
    if (rc) return rc;
    CU(cudaMemsetAsync(ctx->d_err, 0, 4 * sizeof(int), ctx->stream));
    CUL(launch_ticks(static_cast<const float *>(dsp), ctx->d_len, D, N, Np, A, ctx->tps, ctx->d_ticks,
                     ctx->d_ticks16, ctx->d_err + 3, ctx->d_err, ctx->stream));
    CU(cudaMemcpyAsync(&ctx->max_tick, ctx->d_err + 3, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    rc = check_device_error(ctx);
    if (rc) {
        free_days(ctx);
        return rc;
    }
    // trajectories: pass 1 (route times, offsets, repair counts)
    CU(cudaMemsetAsync(ctx->d_maxoff, 0, (size_t)D * sizeof(int32_t), ctx->stream));
    CU(cudaMemsetAsync(ctx->d_repairs, 0, (size_t)D * sizeof(unsigned long long), ctx->stream));
    CU(cudaMemsetAsync(ctx->d_tab_off, 0xff, (size_t)D * sizeof(int64_t), ctx->stream));
    PrepParams pp{};
    pp.N = N;
    pp.Np = Np;
    pp.A = A;
    pp.P = ctx->P;
    pp.tps = ctx->tps;
    pp.div = ctx->div;
    pp.rptr = ctx->d_rptr;
    pp.rlinks = ctx->d_rlinks;
    pp.ticks = ctx->d_ticks;
    pp.C = ctx->d_C;
    pp.maxoff = ctx->d_maxoff;
    pp.repairs = ctx->d_repairs;
    pp.tab_off = ctx->d_tab_off;
    pp.traj_tab = nullptr;
    pp.n_days = D;
    pp.coupled = ctx->opt.couple_days;
    CUL(launch_prepare(pp, ctx->stream));
    ctx->h_maxoff.resize(D);
    ctx->h_repairs.resize(D);
    CU(cudaMemcpyAsync(ctx->h_maxoff.data(), ctx->d_maxoff, D * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(ctx->h_repairs.data(), ctx->d_repairs, D * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->maxoff_max = *std::max_element(ctx->h_maxoff.begin(), ctx->h_maxoff.end());
    if (ctx->opt.couple_days) {
        // rows of the next day that a day's trips reach: every arrival row is at
        // most maxoff + 1 past its departure row
        dfree(ctx->d_early);
        dfree(ctx->d_halo);
        ctx->halo_rows = ctx->maxoff_max + 2;
        const size_t nh = (size_t)D * ctx->O * ctx->halo_rows;
        CU(dalloc(&ctx->d_early, nh));
        CU(dalloc(&ctx->d_halo, nh));
    }
    // pass 2 for days that needed FIFO repairs: keep their exact trajectories
    std::vector<int64_t> off(D, -1);
    const size_t per_day = (size_t)(ctx->L + ctx->P) * (N + 1);
    size_t n_tab = 0;
    for (int d = 0; d < D; ++d)
        if (ctx->h_repairs[d] > 0) {
            off[d] = (int64_t)(n_tab * per_day);
            ++n_tab;
        }
    dfree(ctx->d_traj_tab);
    if (n_tab > 0) {
        CU(dalloc(&ctx->d_traj_tab, n_tab * per_day));
        CU(cudaMemcpyAsync(ctx->d_tab_off, off.data(), D * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemsetAsync(ctx->d_repairs, 0, (size_t)D * sizeof(unsigned long long), ctx->stream));
        pp.traj_tab = ctx->d_traj_tab;
        CUL(launch_prepare(pp, ctx->stream));
    }
    // counts / mask
    rc = dode_set_counts(ctx, counts, mask, ptr_kind);
    if (rc) return rc;
    // fresh solver state
    CU(cudaMemsetAsync(ctx->d_q, 0, (size_t)D * ctx->K * Np * sizeof(float), ctx->stream));
    CU(cudaMemsetAsync(ctx->d_G, 0, (size_t)D * ctx->K * Np * sizeof(float), ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return DODE_OK;
}

int dode_set_counts(dode_ctx *ctx, const float *counts, const uint8_t *mask, int32_t ptr_kind) {
    if (!ctx) return DODE_ERR_ARG;
    if (ctx->D == 0) return fail(ctx, DODE_ERR_STATE, "no days loaded");
    if (!counts || bad_ptr_kind(ptr_kind)) return fail(ctx, DODE_ERR_ARG, "set_counts arguments");
    int rc = set_device(ctx);
    if (rc) return rc;
    const int D = ctx->D, N = ctx->N, O = ctx->O;
    const size_t ct_bytes = (size_t)D * N * O * sizeof(float);
    const size_t mk_bytes = (size_t)D * N * O;
    if (ptr_kind == DODE_PTR_HOST) {
        rc = stage(ctx, ct_bytes + mk_bytes);
        if (rc) return rc;
    }
    CU(cudaStreamSynchronize(ctx->stream));
    const void *dct = nullptr;
    rc = input(ctx, counts, ct_bytes, ptr_kind, 0, &dct);
    if (rc) return rc;
    CUL(launch_transpose_in(static_cast<const float *>(dct), ctx->d_counts, D, N, ctx->Np, O, ctx->stream));
    const void *dmk = nullptr;
    if (mask) {
        rc = input(ctx, mask, mk_bytes, ptr_kind, ct_bytes, &dmk);
        if (rc) return rc;
    }
    CUL(launch_pack_mask(static_cast<const uint8_t *>(dmk), ctx->d_mask, ctx->d_colact, D, N, ctx->Nw, O, ctx->Ow,
                        ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return DODE_OK;
}

int dode_get_state(dode_ctx *ctx, float *q, float *G, int32_t ptr_kind) {
    if (!ctx) return DODE_ERR_ARG;
    if (ctx->D == 0) return fail(ctx, DODE_ERR_STATE, "no days loaded");
    if (bad_ptr_kind(ptr_kind)) return fail(ctx, DODE_ERR_ARG, "ptr_kind");
    int rc = set_device(ctx);
    if (rc) return rc;
    if (q && (rc = output_odmajor(ctx, ctx->d_q, q, ctx->K, 1.f, ptr_kind))) return rc;
    CU(cudaStreamSynchronize(ctx->stream));
    if (G && (rc = output_odmajor(ctx, ctx->d_G, G, ctx->K, 1.f, ptr_kind))) return rc;
    CU(cudaStreamSynchronize(ctx->stream));
    return DODE_OK;
}

int dode_set_state(dode_ctx *ctx, const float *q, const float *G, int32_t ptr_kind) {
    if (!ctx) return DODE_ERR_ARG;
    if (ctx->D == 0) return fail(ctx, DODE_ERR_STATE, "no days loaded");
    if (bad_ptr_kind(ptr_kind)) return fail(ctx, DODE_ERR_ARG, "ptr_kind");
    int rc = set_device(ctx);
    if (rc) return rc;
    CU(cudaStreamSynchronize(ctx->stream));
    if (q && (rc = input_odmajor(ctx, q, ctx->d_q, ctx->K, ptr_kind))) return rc;
    CU(cudaStreamSynchronize(ctx->stream));
    if (G && (rc = input_odmajor(ctx, G, ctx->d_G, ctx->K, ptr_kind))) return rc;
    CU(cudaStreamSynchronize(ctx->stream));
    return DODE_OK;
}

int dode_solve(dode_ctx *ctx, int32_t iters, float step, int32_t batch, float *q_out, double *loss_out,
               int32_t ptr_kind) {
    if (!ctx) return DODE_ERR_ARG;
    if (ctx->D == 0) return fail(ctx, DODE_ERR_STATE, "no days loaded");
    if (iters < 0 || !(step > 0.f) || !std::isfinite(step) || batch < 0 || bad_ptr_kind(ptr_kind))
        return fail(ctx, DODE_ERR_ARG, "solve arguments");
    if (ctx->opt.row_chunk > 0 && ctx->opt.form == DODE_FORM_PLAIN)
        return fail(ctx, DODE_ERR_UNSUPPORTED, "row_chunk > 0 needs the fused form");
    int rc = set_device(ctx);
    if (rc) return rc;
    const int D = ctx->D;
    if (ctx->opt.form == DODE_FORM_PLAIN) {
        PlainParams pp;
        rc = plain_prepare(ctx, ctx->opt.theta_per_min, &pp);
        if (rc) return rc;
        if (!ctx->d_xout) CU(dalloc(&ctx->d_xout, (size_t)D * ctx->O * ctx->Np));
        const size_t need = (size_t)(iters + 1) * D;
        if (need > ctx->ptrace_cap) {
            CU(dalloc(&ctx->d_ptrace, need));
            ctx->ptrace_cap = need;
        }
        CU(cudaMemsetAsync(ctx->d_ptrace, 0, need * sizeof(double), ctx->stream));
        const size_t xbytes = (size_t)D * ctx->O * ctx->Np * sizeof(float);
        CU(cudaEventRecord(ctx->ev0, ctx->stream));
        for (int it = 0; it <= iters; ++it) {
            CU(cudaMemsetAsync(ctx->d_xout, 0, xbytes, ctx->stream));
            CUL(launch_plain_forward(pp, ctx->d_q, ctx->d_xout, ctx->stream));
            CUL(launch_plain_residual(pp, ctx->d_counts, ctx->d_mask, ctx->d_xout, ctx->d_ptrace + (size_t)it * D,
                                     nullptr, ctx->stream));
            if (it < iters)
                CUL(launch_plain_adjoint_step(pp, ctx->d_xout, ctx->d_q, ctx->d_G, step, ctx->opt.eps, ctx->stream));
        }
        CU(cudaEventRecord(ctx->ev1, ctx->stream));
        ctx->last_launches = 1 + 3LL * iters + 2;
        ctx->last_grid = 0;
        CU(cudaMemcpyAsync(ctx->d_loss, ctx->d_ptrace + (size_t)iters * D, D * sizeof(double),
                           cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
        if ((size_t)iters * D > ctx->trace_cap) {
            drop_graph(ctx);
            CU(dalloc(&ctx->d_trace, (size_t)iters * D));
            ctx->trace_cap = (size_t)iters * D;
        }
        FusedParams p = base_params(ctx);
        p.mode = MODE_SOLVE;
        p.row_chunk = ctx->opt.row_chunk;
        p.iters = iters;
        p.eta = step;
        p.trace = iters > 0 ? ctx->d_trace : nullptr;
        if (ctx->opt.couple_days) {
            if (ctx->opt.precision == DODE_PREC_BF16)
                CUL(launch_to_bf16(ctx->d_q, ctx->d_qb, (size_t)D * ctx->K * ctx->Np, ctx->stream));
            rc = solve_coupled(ctx, p, iters);
            if (rc) return rc;
        } else if (ctx->opt.use_graph && ptr_kind == DODE_PTR_DEVICE) {
            rc = solve_graph(ctx, p, iters, step, q_out, loss_out);
            if (rc) return rc;
            ctx->trace_iters = iters;
            rc = finish_timing(ctx);
            if (rc) return rc;
            rc = check_device_error(ctx);
            if (rc) return rc;
            CU(cudaStreamSynchronize(ctx->stream));
            return DODE_OK;
        }
        if (!ctx->opt.couple_days) {
            if (ctx->opt.precision == DODE_PREC_BF16)
                CUL(launch_to_bf16(ctx->d_q, ctx->d_qb, (size_t)D * ctx->K * ctx->Np, ctx->stream));
            rc = run_fused(ctx, p, ctx->opt.precision);
            if (rc) return rc;
        }
    }
    ctx->trace_iters = iters;
    rc = finish_timing(ctx);
    if (rc) return rc;
    rc = check_device_error(ctx);
    if (rc) return rc;
    if (q_out && (rc = output_odmajor(ctx, ctx->d_q, q_out, ctx->K, 1.f, ptr_kind))) return rc;
    if (loss_out && (rc = output_plain(ctx, ctx->d_loss, loss_out, D * sizeof(double), ptr_kind))) return rc;
    CU(cudaStreamSynchronize(ctx->stream));
    return DODE_OK;
}

int dode_get_loss_trace(dode_ctx *ctx, float *trace, int32_t iters) {
    if (!ctx || !trace) return DODE_ERR_ARG;
    if (ctx->trace_iters < 0) return fail(ctx, DODE_ERR_STATE, "no solve since the days were loaded");
    if (iters != ctx->trace_iters) return fail(ctx, DODE_ERR_ARG, "iters differs from the last solve");
    int rc = set_device(ctx);
    if (rc) return rc;
    const size_t n = (size_t)iters * ctx->D;
    if (n == 0) return DODE_OK;
    if (ctx->opt.form == DODE_FORM_PLAIN) {
        std::vector<double> tmp(n);
        CU(cudaMemcpyAsync(tmp.data(), ctx->d_ptrace, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        for (size_t i = 0; i < n; ++i) trace[i] = (float)tmp[i];
    } else {
        CU(cudaMemcpyAsync(trace, ctx->d_trace, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    return DODE_OK;
}

static int fused_eval(dode_ctx *ctx, int mode, const float *q, float theta, int ptr_kind) {
    int rc = set_device(ctx);
    if (rc) return rc;
    CU(cudaStreamSynchronize(ctx->stream));
    rc = input_odmajor(ctx, q, ctx->d_qtmp, ctx->K, ptr_kind);
    if (rc) return rc;
    FusedParams p = base_params(ctx);
    p.mode = mode;
    p.theta = theta;
    p.q = ctx->d_qtmp;
    p.G = nullptr;
    if (ctx->opt.precision == DODE_PREC_BF16)
        CUL(launch_to_bf16(ctx->d_qtmp, ctx->d_qb, (size_t)ctx->D * ctx->K * ctx->Np, ctx->stream));
    if (mode == MODE_FORWARD) {
        if (!ctx->d_xout) CU(dalloc(&ctx->d_xout, (size_t)ctx->D * ctx->O * ctx->Np));
        p.xout = ctx->d_xout;
    }
    if (mode == MODE_LOSS_GRAD) {
        if (!ctx->d_gout) CU(dalloc(&ctx->d_gout, (size_t)ctx->D * ctx->K * ctx->Np));
        p.gout = ctx->d_gout;
    }
    rc = run_fused(ctx, p, ctx->opt.precision);
    if (rc) return rc;
    rc = finish_timing(ctx);
    if (rc) return rc;
    return check_device_error(ctx);
}

int dode_forward(dode_ctx *ctx, const float *q, float *xhat, int32_t ptr_kind) {
    if (!ctx) return DODE_ERR_ARG;
    if (ctx->D == 0) return fail(ctx, DODE_ERR_STATE, "no days loaded");
    if (!q || !xhat || bad_ptr_kind(ptr_kind)) return fail(ctx, DODE_ERR_ARG, "forward arguments");
    int rc = fused_eval(ctx, MODE_FORWARD, q, ctx->opt.theta_per_min, ptr_kind);
    if (rc) return rc;
    rc = output_odmajor(ctx, ctx->d_xout, xhat, ctx->O, 1.f, ptr_kind);
    if (rc) return rc;
    CU(cudaStreamSynchronize(ctx->stream));
    return DODE_OK;
}

int dode_loss(dode_ctx *ctx, const float *q, float theta, double *loss, int32_t ptr_kind) {
    if (!ctx) return DODE_ERR_ARG;
    if (ctx->D == 0) return fail(ctx, DODE_ERR_STATE, "no days loaded");
    if (!q || !loss || bad_ptr_kind(ptr_kind) || !std::isfinite(theta)) return fail(ctx, DODE_ERR_ARG, "loss arguments");
    int rc = fused_eval(ctx, MODE_LOSS, q, theta, ptr_kind);
    if (rc) return rc;
    ctx->totals_kind = 1;
    CU(cudaMemcpyAsync(loss, ctx->d_loss, ctx->D * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return DODE_OK;
}

// Method 3 of dode_dense_nnls: the m right-hand sides stacked into GEMMs on the
// tensor cores (dense_tc.cu), TF32 products with FP32 accumulation.
static int dense_nnls_tc(int32_t nr, int32_t nc, int32_t m, const float *B, const float *Y, int32_t iters, float step,
                         float eps, float *X, float *G, double *loss, double *kernel_ms, int32_t ptr_kind,
                         void *stream) {
    auto bail = [&](int code, const std::string &msg) {
        fprintf(stderr, "dode_dense_nnls: %s\n", msg.c_str());
        return code;
    };
    const bool host = ptr_kind == DODE_PTR_HOST;
    if (m % 16 != 0 || nr % 4 != 0 || nc % 4 != 0 || (!host && ((uintptr_t)B % 16 || (uintptr_t)Y % 16)))
        return bail(DODE_ERR_UNSUPPORTED,
                    "tensor cores need m a multiple of 16 (16..256), n_rows and n_cols multiples of 4, 16-byte "
                    "aligned B and Y");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t nB = (size_t)nr * nc, nY = (size_t)nr * m, nX = (size_t)nc * m;
    float *dB = nullptr, *dY = nullptr, *dX = nullptr, *dG = nullptr;
    double *dl = nullptr;
    const cudaMemcpyKind in = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaSuccess;
    if (host) {
        e = cudaMalloc(&dB, nB * 4);
        if (e == cudaSuccess) e = cudaMalloc(&dY, nY * 4);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dB, B, nB * 4, in, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dY, Y, nY * 4, in, st);
    }
    if (e == cudaSuccess) e = cudaMalloc(&dX, nX * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dG, nX * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dl, (size_t)m * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dX, X, nX * 4, in, st);
    if (e == cudaSuccess) e = G ? cudaMemcpyAsync(dG, G, nX * 4, in, st) : cudaMemsetAsync(dG, 0, nX * 4, st);
    int rc = 0, herr = 0;
    float ms = 0.f;
    if (e == cudaSuccess)
        rc = dense_tc_nnls(nr, nc, m, host ? dB : B, host ? dY : Y, iters, step, eps, dX, dG, dl, &ms, &herr, st);
    const cudaMemcpyKind out = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (e == cudaSuccess && rc == 0) e = cudaMemcpyAsync(X, dX, nX * 4, out, st);
    if (e == cudaSuccess && rc == 0 && G) e = cudaMemcpyAsync(G, dG, nX * 4, out, st);
    if (e == cudaSuccess && rc == 0) e = cudaMemcpyAsync(loss, dl, (size_t)m * sizeof(double), out, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dB);
    cudaFree(dY);
    cudaFree(dX);
    cudaFree(dG);
    cudaFree(dl);
    if (e != cudaSuccess || rc != 0) {
        (void)cudaGetLastError();
        return bail(rc == -1 ? DODE_ERR_CUDA : (e == cudaErrorMemoryAllocation ? DODE_ERR_OOM : DODE_ERR_CUDA),
                    e != cudaSuccess ? cudaGetErrorString(e) : "tensor-core path failed");
    }
    if (herr) return bail(DODE_ERR_DEVICE_TIMEOUT, "a bounded wait of the tensor-core kernel ran out");
    if (kernel_ms) *kernel_ms = ms;
    return DODE_OK;
}

// Polls of a bounded wait in the one-pass dense kernel before it gives up.
static long long g_dense_wait_limit = 1ll << 26;

int dode_dense_set_wait_limit(int64_t polls) {
    if (polls < 0) return DODE_ERR_ARG;
    g_dense_wait_limit = polls;
    return DODE_OK;
}

int dode_dense_nnls(int32_t n_rows, int32_t n_cols, int32_t m, const float *B, const float *Y, int32_t iters,
                    float step, float eps, int32_t method, float *X, float *G, double *loss, double *kernel_ms,
                    int32_t ptr_kind, void *stream) {
    auto bail = [&](int code, const std::string &msg) {
        fprintf(stderr, "dode_dense_nnls: %s\n", msg.c_str());
        return code;
    };
    if (n_rows < 1 || n_cols < 1 || m < 1 || m > 256 || iters < 0 || !(step > 0.f) || !std::isfinite(step) ||
        !(eps >= 0.f) || !B || !Y || !X || !loss || (ptr_kind != DODE_PTR_HOST && ptr_kind != DODE_PTR_DEVICE) ||
        method < 0 || method > 3 || (m > 8 && method != 3))
        return bail(DODE_ERR_ARG, "arguments (1 <= m <= 8, or <= 256 with method 3; iters >= 0, step > 0, method 0..3)");
    if (method == 3) return dense_nnls_tc(n_rows, n_cols, m, B, Y, iters, step, eps, X, G, loss, kernel_ms, ptr_kind,
                                          stream);
    if ((long long)n_cols * m * sizeof(float) > 200 * 1024)
        return bail(DODE_ERR_UNSUPPORTED, "n_cols * m must be at most 51200 (x is staged in shared memory)");
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(DODE_ERR_CUDA, "no CUDA device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t nB = (size_t)n_rows * n_cols, nY = (size_t)n_rows * m, nX = (size_t)n_cols * m;
    DenseParams p{};
    p.nr = n_rows;
    p.nc = n_cols;
    p.m = m;
    p.eta = step;
    p.eps = eps;
    p.grid_r = (int)std::min<long long>(((long long)n_rows + 7) / 8, 4LL * n_sm);
    // row blocks of 32 rows (8 rows per load batch); partial gradients per block
    p.rows_per_cta = 32;
    p.grid_g = (n_rows + p.rows_per_cta - 1) / p.rows_per_cta;
    // one pass over B per iteration (bulk-copy staged) when it applies
    const bool host = ptr_kind == DODE_PTR_HOST;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t xbytes = ((size_t)n_cols * 4 + 127) & ~(size_t)127;
    const size_t room = (size_t)optin > xbytes + 2048 ? (size_t)optin - xbytes - 2048 : 0;
    // ring stages of one row: 8 or 4 (a multiple of the kernel's four residual warps)
    const int S = (int)(std::min<size_t>(8, room / ((size_t)n_cols * 4)) & ~(size_t)3);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    const bool one_ok = m == 1 && n_cols % 4 == 0 && n_cols <= 8192 && S >= 4 && coop &&
                        (host || ((uintptr_t)B % 16 == 0));
    if (method == 1 && !one_ok)
        return bail(DODE_ERR_UNSUPPORTED,
                    "one pass needs m = 1, n_cols % 4 == 0, n_cols <= 8192, 16-byte aligned B, cooperative launch");
    const bool one = method == 1 || (method == 0 && one_ok);
    const int grid_f = std::min(n_sm, 192);      // the one-pass step sums at most 192 partials per column
    // one device allocation: (B, y when on the host) x, G, r, gradient partials, loss
    // partials (of either kernel), loss, error flag; every piece starts on a
    // 256-byte boundary (the kernels use 16-byte accesses)
    size_t off = 0;
    auto take = [&](size_t n) {
        const size_t o = off;
        off += (n + 63) & ~(size_t)63;
        return o;
    };
    const size_t oB = host ? take(nB) : 0, oY = host ? take(nY) : 0;
    const size_t oX = take(nX), oG = take(nX), oR = take(nY);
    const size_t oP = take((size_t)std::max(p.grid_g, grid_f) * nX);
    const size_t n_lpart = (size_t)std::max(p.grid_r, grid_f) * m;
    const size_t d_count = n_lpart + m + 2;
    char *buf = nullptr;
    const size_t f_bytes = off * sizeof(float);
    if (cudaMalloc(&buf, f_bytes + d_count * sizeof(double)) != cudaSuccess) {
        (void)cudaGetLastError();
        return bail(DODE_ERR_OOM, "device memory");
    }
    float *f = reinterpret_cast<float *>(buf);
    p.B = host ? f + oB : B;
    p.y = host ? f + oY : Y;
    p.x = f + oX;
    p.G = f + oG;
    p.r = f + oR;
    p.gpart = f + oP;
    p.vec = n_cols % 4 == 0 && ((uintptr_t)p.B % 16 == 0) ? 1 : 0;
    p.lpart = reinterpret_cast<double *>(buf + f_bytes);
    double *dloss = p.lpart + n_lpart;
    int *derr = reinterpret_cast<int *>(dloss + m);
    unsigned int *dgbar = reinterpret_cast<unsigned int *>(dloss + m + 1);
    p.wait_limit = g_dense_wait_limit;
    const size_t fsmem = xbytes + (size_t)S * n_cols * 4;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const cudaMemcpyKind in = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaSuccess;
    if (host) e = cudaMemcpyAsync(const_cast<float *>(p.B), B, nB * sizeof(float), in, st);
    if (e == cudaSuccess && host) e = cudaMemcpyAsync(const_cast<float *>(p.y), Y, nY * sizeof(float), in, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p.x, X, nX * sizeof(float), in, st);
    if (e == cudaSuccess)
        e = G ? cudaMemcpyAsync(p.G, G, nX * sizeof(float), in, st) : cudaMemsetAsync(p.G, 0, nX * sizeof(float), st);
    if (e == cudaSuccess) e = dense_set_smem((size_t)n_cols * m * sizeof(float), (size_t)p.rows_per_cta * m * sizeof(float));
    if (e == cudaSuccess && one) e = dense_persist_set_smem(fsmem);
    if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (one) {
        // every iteration and the final residual pass in one launch; loss partials per CTA
        if (e == cudaSuccess) e = dense_persist(p, iters, grid_f, S, fsmem, derr, dgbar, st);
        DenseParams pl = p;
        pl.grid_r = grid_f;
        if (e == cudaSuccess) e = dense_loss(pl, dloss, st);
    } else {
        for (int it = 0; it < iters && e == cudaSuccess; ++it) e = dense_iteration(p, true, st);
        if (e == cudaSuccess) e = dense_iteration(p, false, st);     // residual and loss of the final x
        if (e == cudaSuccess) e = dense_loss(p, dloss, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    const cudaMemcpyKind out = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (e == cudaSuccess) e = cudaMemcpyAsync(X, p.x, nX * sizeof(float), out, st);
    if (e == cudaSuccess && G) e = cudaMemcpyAsync(G, p.G, nX * sizeof(float), out, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, dloss, m * sizeof(double), host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
    float ms = 0.f;
    if (e == cudaSuccess && kernel_ms) {
        e = cudaEventElapsedTime(&ms, e0, e1);
        *kernel_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return bail(DODE_ERR_CUDA, cudaGetErrorString(e));
    }
    if (herr) return bail(DODE_ERR_DEVICE_TIMEOUT, "a bounded wait of the one-pass kernel ran out");
    return DODE_OK;
}

int dode_set_patterns(dode_ctx *ctx, const int32_t *pattern) {
    if (!ctx) return DODE_ERR_ARG;
    if (ctx->D == 0) return fail(ctx, DODE_ERR_STATE, "no days loaded");
    int rc = set_device(ctx);
    if (rc) return rc;
    drop_graph(ctx);
    if (!pattern) {
        ctx->patterns = false;
        return DODE_OK;
    }
    const int D = ctx->D;
    // groups of days sharing a pattern, in ascending day order; a day with
    // label -1 is a group of its own
    std::vector<int> order(D);
    for (int d = 0; d < D; ++d) {
        if (pattern[d] < -1) return fail(ctx, DODE_ERR_ARG, "pattern labels must be >= -1");
        order[d] = d;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const long long ka = pattern[a] < 0 ? (1LL << 40) + a : pattern[a];
        const long long kb = pattern[b] < 0 ? (1LL << 40) + b : pattern[b];
        return ka < kb;
    });
    std::vector<int32_t> gptr(1, 0), gday(order.begin(), order.end());
    for (int i = 1; i <= D; ++i)
        if (i == D || pattern[order[i]] < 0 || pattern[order[i]] != pattern[order[i - 1]]) gptr.push_back(i);
    if (!ctx->d_Ceff) CU(dalloc(&ctx->d_Ceff, (size_t)D * ctx->P * ctx->Np));
    int32_t *dbuf = nullptr;
    CU(dalloc(&dbuf, gptr.size() + gday.size()));
    cudaError_t e = cudaMemcpyAsync(dbuf, gptr.data(), gptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dbuf + gptr.size(), gday.data(), gday.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                            ctx->stream);
    if (e == cudaSuccess)
        e = launch_pattern_times(ctx->d_C, (int)gptr.size() - 1, dbuf, dbuf + gptr.size(), ctx->P, ctx->N, ctx->Np,
                                 ctx->d_Ceff, ctx->stream);
    if (e == cudaSuccess) {
        ++ctx->total_launches;
        e = cudaStreamSynchronize(ctx->stream);
    }
    cudaFree(dbuf);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ctx, DODE_ERR_CUDA, std::string("set_patterns: ") + cudaGetErrorString(e));
    }
    ctx->patterns = true;
    return DODE_OK;
}

int dode_r2(dode_ctx *ctx, const float *q, float theta, double *r2, int32_t ptr_kind) {
    if (!ctx) return DODE_ERR_ARG;
    if (ctx->D == 0) return fail(ctx, DODE_ERR_STATE, "no days loaded");
    if (!q || !r2 || bad_ptr_kind(ptr_kind) || !std::isfinite(theta)) return fail(ctx, DODE_ERR_ARG, "r2 arguments");
    int rc = fused_eval(ctx, MODE_LOSS, q, theta, ptr_kind);
    if (rc) return rc;
    double *dbuf = nullptr;
    CU(dalloc(&dbuf, (size_t)ctx->D * 2));
    cudaError_t e = launch_r2(ctx->d_counts, ctx->d_mask, ctx->D, ctx->O, ctx->N, ctx->Np, ctx->Nw, ctx->d_loss, dbuf,
                              dbuf + ctx->D, ctx->stream);
    if (e == cudaSuccess) {
        ctx->total_launches += 2;
        e = cudaMemcpyAsync(r2, dbuf + ctx->D, ctx->D * sizeof(double),
                            ptr_kind == DODE_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(dbuf);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ctx, DODE_ERR_CUDA, std::string("r2: ") + cudaGetErrorString(e));
    }
    return DODE_OK;
}

int dode_dar_distance(dode_ctx *ctx, double *dist, double *mean_sq) {
    if (!ctx) return DODE_ERR_ARG;
    if (ctx->D == 0) return fail(ctx, DODE_ERR_STATE, "no days loaded");
    if (ctx->opt.couple_days) return fail(ctx, DODE_ERR_UNSUPPORTED, "dar_distance compares per-day DARs (couple_days = 0)");
    if (!dist) return fail(ctx, DODE_ERR_ARG, "dar_distance arguments");
    int rc = set_device(ctx);
    if (rc) return rc;
    DarParams p{};
    p.N = ctx->N;
    p.Np = ctx->Np;
    p.A = ctx->A;
    p.P = ctx->P;
    p.L = ctx->L;
    p.W = ctx->maxoff_max + 2;
    p.n_days = ctx->D;
    p.div = ctx->div;
    p.rptr = ctx->d_rptr;
    p.rlinks = ctx->d_rlinks;
    p.ticks = ctx->d_ticks;
    p.tab_off = ctx->d_tab_off;
    p.traj_tab = ctx->d_traj_tab;
    const int n_part = 4 * ctx->n_sm;
    double *buf = nullptr;
    const size_t nbar = (size_t)p.L * p.N * p.W;
    CU(dalloc(&buf, nbar + n_part + 1 + ctx->D));
    p.rbar = buf;
    double *part = buf + nbar, *sq = part + n_part, *dd = sq + 1;
    cudaError_t e = launch_dar_distance(p, part, n_part, sq, dd, ctx->stream);
    if (e == cudaSuccess) {
        ctx->total_launches += 4;
        e = cudaMemcpyAsync(dist, dd, ctx->D * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess && mean_sq) e = cudaMemcpyAsync(mean_sq, sq, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(buf);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ctx, DODE_ERR_CUDA, std::string("dar_distance: ") + cudaGetErrorString(e));
    }
    return DODE_OK;
}

int dode_loss_grad(dode_ctx *ctx, const float *q, float theta, double *loss, float *dq, double *dtheta,
                   int32_t ptr_kind) {
    if (!ctx) return DODE_ERR_ARG;
    if (ctx->D == 0) return fail(ctx, DODE_ERR_STATE, "no days loaded");
    if (!q || !loss || bad_ptr_kind(ptr_kind) || !std::isfinite(theta))
        return fail(ctx, DODE_ERR_ARG, "loss_grad arguments");
    int rc = fused_eval(ctx, MODE_LOSS_GRAD, q, theta, ptr_kind);
    if (rc) return rc;
    ctx->totals_kind = 2;
    if (dq && (rc = output_odmajor(ctx, ctx->d_gout, dq, ctx->K, 1.f, ptr_kind))) return rc;
    CU(cudaMemcpyAsync(loss, ctx->d_loss, ctx->D * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (dtheta) CU(cudaMemcpyAsync(dtheta, ctx->d_dtheta, ctx->D * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return DODE_OK;
}

int dode_last_totals(dode_ctx *ctx, double *loss_total, double *dtheta_total) {
    if (!ctx) return DODE_ERR_ARG;
    if (!loss_total) return fail(ctx, DODE_ERR_ARG, "last_totals: loss_total is NULL");
    if (ctx->totals_kind == 0) return fail(ctx, DODE_ERR_STATE, "no loss or gradient call since the days were loaded");
    if (dtheta_total && ctx->totals_kind != 2)
        return fail(ctx, DODE_ERR_STATE, "dtheta_total needs a dode_loss_grad call as the last evaluation");
    int rc = set_device(ctx);
    if (rc) return rc;
    CUL(launch_day_totals(ctx->d_loss, ctx->totals_kind == 2 ? ctx->d_dtheta : nullptr, ctx->D, ctx->d_totals,
                          ctx->stream));
    double h[2];
    CU(cudaMemcpyAsync(h, ctx->d_totals, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *loss_total = h[0];
    if (dtheta_total) *dtheta_total = h[1];
    return DODE_OK;
}

int dode_get_ticks(dode_ctx *ctx, int32_t day, int32_t *out) {
    if (!ctx || !out) return DODE_ERR_ARG;
    if (day < 0 || day >= ctx->D) return fail(ctx, DODE_ERR_ARG, "day out of range");
    int rc = set_device(ctx);
    if (rc) return rc;
    std::vector<int32_t> t((size_t)ctx->A * ctx->Np);
    CU(cudaMemcpyAsync(t.data(), ctx->d_ticks + (size_t)day * ctx->A * ctx->Np, t.size() * sizeof(int32_t),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    for (int h = 0; h < ctx->N; ++h)
        for (int a = 0; a < ctx->A; ++a) out[(size_t)h * ctx->A + a] = t[(size_t)a * ctx->Np + h];
    return DODE_OK;
}

int dode_get_route_times(dode_ctx *ctx, int32_t day, float *out) {
    if (!ctx || !out) return DODE_ERR_ARG;
    if (day < 0 || day >= ctx->D) return fail(ctx, DODE_ERR_ARG, "day out of range");
    int rc = set_device(ctx);
    if (rc) return rc;
    std::vector<float> t((size_t)ctx->P * ctx->Np);
    CU(cudaMemcpyAsync(t.data(), ctx->d_C + (size_t)day * ctx->P * ctx->Np, t.size() * sizeof(float),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    for (int h = 0; h < ctx->N; ++h)
        for (int k = 0; k < ctx->P; ++k) out[(size_t)h * ctx->P + k] = t[(size_t)k * ctx->Np + h];
    return DODE_OK;
}

int dode_get_day_info(dode_ctx *ctx, int32_t day, int64_t *n_repairs, int32_t *max_offset) {
    if (!ctx) return DODE_ERR_ARG;
    if (day < 0 || day >= ctx->D) return fail(ctx, DODE_ERR_ARG, "day out of range");
    if (n_repairs) *n_repairs = (int64_t)ctx->h_repairs[day];
    if (max_offset) *max_offset = ctx->h_maxoff[day];
    return DODE_OK;
}

int dode_get_dar(dode_ctx *ctx, int32_t day, int64_t *n, int32_t *kjh, float *rho) {
    if (!ctx || !n) return DODE_ERR_ARG;
    if (day < 0 || day >= ctx->D) return fail(ctx, DODE_ERR_ARG, "day out of range");
    if (ctx->opt.couple_days) return fail(ctx, DODE_ERR_UNSUPPORTED, "get_dar lists per-day DARs (couple_days = 0)");
    int rc = set_device(ctx);
    if (rc) return rc;
    // every (route, position) pair, not only observed links
    std::vector<int32_t> pk, pj, po, rpp(ctx->P + 1, 0);
    for (int k = 0; k < ctx->P; ++k) {
        for (int j = ctx->rptr[k]; j < ctx->rptr[k + 1]; ++j) {
            pk.push_back(k);
            pj.push_back(j - ctx->rptr[k]);
            po.push_back(0);
        }
        rpp[k + 1] = (int32_t)pk.size();
    }
    int32_t *d_pk = nullptr, *d_pj = nullptr, *d_po = nullptr, *d_rpp = nullptr;
    int4 *d_rec = nullptr;
    const int npairs = (int)pk.size();
    CU(upload(&d_pk, pk, ctx->stream));
    CU(upload(&d_pj, pj, ctx->stream));
    CU(upload(&d_po, po, ctx->stream));
    CU(upload(&d_rpp, rpp, ctx->stream));
    CU(dalloc(&d_rec, (size_t)npairs * ctx->N));
    PlainParams p{};
    p.N = ctx->N;
    p.Np = ctx->Np;
    p.A = ctx->A;
    p.P = ctx->P;
    p.n_pairs = npairs;
    p.div = ctx->div;
    p.rptr = ctx->d_rptr;
    p.rlinks = ctx->d_rlinks;
    p.pair_k = d_pk;
    p.pair_j = d_pj;
    p.pair_o = d_po;
    p.route_pair_ptr = d_rpp;
    p.ticks = ctx->d_ticks + (size_t)day * ctx->A * ctx->Np;
    p.tab_off = ctx->d_tab_off + day;
    p.traj_tab = ctx->d_traj_tab;
    p.rec = d_rec;
    p.n_days = 1;
    p.err = ctx->d_err;
    CUL(launch_plain_build(p, ctx->stream));
    std::vector<int4> rec((size_t)npairs * ctx->N);
    CU(cudaMemcpyAsync(rec.data(), d_rec, rec.size() * sizeof(int4), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    cudaFree(d_pk);
    cudaFree(d_pj);
    cudaFree(d_po);
    cudaFree(d_rpp);
    cudaFree(d_rec);
    rc = check_device_error(ctx);
    if (rc) return rc;
    int64_t m = 0;
    for (int pi = 0; pi < npairs; ++pi) {
        for (int b = 0; b < ctx->N; ++b) {
            const int4 r = rec[(size_t)pi * ctx->N + b];
            const int cnt = r.x >> 16, h2 = r.x & 0xffff;
            const int vals[3] = {r.y, r.z, r.w};
            for (int c = 0; c < cnt; ++c) {
                if (kjh) {
                    kjh[4 * m + 0] = pk[pi];
                    kjh[4 * m + 1] = pj[pi];
                    kjh[4 * m + 2] = b;
                    kjh[4 * m + 3] = h2 + c;
                }
                if (rho) {
                    float f;
                    std::memcpy(&f, &vals[c], sizeof f);
                    rho[m] = f;
                }
                ++m;
            }
        }
    }
    *n = m;
    return DODE_OK;
}


}  // extern "C"

// ---------------------------------------------------------------------------
// Loss evaluation with static scratch (no device allocation).
//
// Some callers cannot call cudaMalloc once they are running: a real-time or
// certified control loop that forbids device allocation after start-up, a
// host process whose GPU memory is entirely owned by another allocator (a
// framework's caching allocator or a fixed arena), or a latency-critical path
// where cudaMalloc's implicit device synchronisation would stall other
// streams.  dode_loss_static_scratch serves them: everything the fused kernel
// needs beyond the context's loaded days and the caller's buffers lives in
// one file-scope device array of kStaticScratchBytes, which every GPU that
// loads this library holds until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // 32 MiB
static __device__ __align__(256) unsigned char dode_static_scratch[kStaticScratchBytes];

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the static scratch on the context's device.  Host code
// only holds a host-side stand-in under the array's name, so the address is
// looked up with that device current -- on every call, which is cheap and
// stays right if the process resets the device between calls.
int static_scratch(dode_ctx *ctx, unsigned char **out) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, dode_static_scratch);
    if (e != cudaSuccess || !ptr)
        return fail(ctx, DODE_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    *out = static_cast<unsigned char *>(ptr);
    return DODE_OK;
}

}  // namespace

extern "C" int dode_loss_static_scratch(dode_ctx *ctx, const float *q, float theta, double *loss) {
    if (!ctx) return DODE_ERR_ARG;
    if (ctx->D == 0) return fail(ctx, DODE_ERR_STATE, "no days loaded");
    if (!q || !loss || !std::isfinite(theta)) return fail(ctx, DODE_ERR_ARG, "loss_static_scratch arguments");
    if (ctx->opt.couple_days) return fail(ctx, DODE_ERR_UNSUPPORTED, "loss_static_scratch takes independent days");
    int rc = set_device(ctx);
    if (rc) return rc;
    unsigned char *base = nullptr;
    rc = static_scratch(ctx, &base);
    if (rc) return rc;
    const int prec = ctx->opt.precision;
    FusedShape sh;
    rc = fused_shape(ctx, prec, &sh);
    if (rc) return rc;
    // scratch layout: queue | q (internal layout) | q BF16 copy | route choice |
    // per CTA: residual slot, accumulator words
    const size_t qn = (size_t)ctx->D * ctx->K * ctx->Np;
    size_t off = 256;
    const size_t off_q = off;
    off = align256(off + qn * sizeof(float));
    const size_t off_qb = off;
    if (prec == DODE_PREC_BF16) off = align256(off + qn * sizeof(__nv_bfloat16));
    const size_t off_pt = off;
    off = align256(off + (size_t)ctx->D * ctx->P * ctx->Np * sizeof(float));
    const size_t slot_r = align256((size_t)ctx->O * ctx->Np * (prec == DODE_PREC_BF16 ? 2 : 4));
    const size_t slot_g = align256((size_t)ctx->O * std::max(ctx->Np, sh.ring_rows) * 4);
    const size_t need_one = off + slot_r + slot_g;
    if (need_one > kStaticScratchBytes) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "these %d days need %zu bytes of scratch for a single CTA; the static scratch holds %zu bytes",
                 ctx->D, need_one, kStaticScratchBytes);
        return fail(ctx, DODE_ERR_ARG, buf);
    }
    const int grid = (int)std::min<size_t>((size_t)sh.grid, (kStaticScratchBytes - off) / (slot_r + slot_g));
    const size_t off_rb = off;
    const size_t off_g = off + (size_t)grid * slot_r;
    CU(cudaStreamSynchronize(ctx->stream));
    // every call shares the scratch: the queue counter starts at zero, the
    // accumulator words are cleared by the kernel itself, the rest is written
    // before it is read
    CU(cudaMemsetAsync(base, 0, 256, ctx->stream));
    float *qi = reinterpret_cast<float *>(base + off_q);
    CUL(launch_transpose_in(q, qi, ctx->D, ctx->N, ctx->Np, ctx->K, ctx->stream));
    __nv_bfloat16 *qb = reinterpret_cast<__nv_bfloat16 *>(base + off_qb);
    if (prec == DODE_PREC_BF16) CUL(launch_to_bf16(qi, qb, qn, ctx->stream));
    float *pt = reinterpret_cast<float *>(base + off_pt);
    CUL(launch_route_choice(choice_C(ctx), ctx->d_rod, ctx->d_od_ptr, ctx->d_od_routes, theta, ctx->D, ctx->P, ctx->N,
                            ctx->Np, pt, ctx->stream));
    FusedParams p = base_params(ctx);
    p.mode = MODE_LOSS;
    p.theta = theta;
    p.q = qi;
    p.G = nullptr;
    p.qb = qb;
    p.pt = pt;
    p.loss = loss;
    p.trace = nullptr;
    p.rbuf = base + off_rb;
    p.gring = reinterpret_cast<float *>(base + off_g);
    p.ring_rows = sh.ring_rows;
    p.tick_rows = sh.tick_rows;
    p.tiles_per_phase = sh.tiles_per_phase;
    p.rtab_off = sh.rtab_off;
    p.rtab_packed = sh.rtab_packed;
    p.queue = reinterpret_cast<int *>(base);
    CUL(launch_fused(p, prec, grid, sh.block, sh.smem, ctx->stream));
    ctx->last_grid = grid;
    CU(cudaStreamSynchronize(ctx->stream));
    return check_device_error(ctx);
}

