// dode_internal.cuh -- device-side layouts, parameter blocks and helpers of libdode.
//
// Internal layouts put TIME innermost so that the 32 lanes of a warp, which
// walk 32 consecutive departure boundaries of one route, touch consecutive
// words:
//   ticks   int32 [D][A][Np]     link travel time (ticks) by entry interval
//   counts  f32   [D][O][Np]     observed link counts
//   mask    u32   [D][O][Nw]     bit h of word h/32: cell (h, o) observed
//   colact  u32   [D][Ow]        bit o: link column o has any observation that day
//   C       f32   [D][P][Np]     route time (minutes) of departure interval h
//   q, G    f32   [D][K][Np]     OD flows and Adagrad accumulator
//   r slot  f32/bf16 [O][Np]     residual of one resident day (per CTA)
// with Np = N + 1 rounded up to a multiple of 32 and Nw = ceil(N / 32).  The
// ABI's time-major layouts (Table "DODE framework variable vectorization") are
// converted on entry and exit by tiled transposes.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dode {

constexpr int kWarp = 32;
constexpr int kTileW = 31;            // windows per warp task (32 boundaries)
constexpr int kMaxRouteLinks = 64;
constexpr int kGroupRoutes = 32;      // routes per walk group of the fused kernel
constexpr int kRankBins = 4096;       // row-chunk ranking: bins on the keys' top 12 bits

// MODE_HALO (coupled days): forward sweep only, writing each day's own deposits
// into its first halo_rows rows (early) and its deposits past midnight (halo).
enum Mode : int { MODE_SOLVE = 0, MODE_FORWARD = 1, MODE_LOSS = 2, MODE_LOSS_GRAD = 3, MODE_HALO = 4 };

// floor(t / ipt) for 0 <= t < 2^31 via a 32-bit magic multiplier (division by
// an invariant integer using multiplication, Granlund and Montgomery, 1994):
// with l = ceil(log2 ipt) and M = ceil(2^(31+l) / ipt) < 2^32,
// floor(t / ipt) = umulhi(t, M) >> (l - 1) for every t < 2^31.
struct IntervalDiv {
    uint32_t magic;
    int shift;
    int ipt;
};

// Requires ipt >= 2 (validated when the context is created).
__host__ __device__ inline IntervalDiv make_interval_div(int ipt) {
    IntervalDiv d;
    int l = 0;
    while ((1u << l) < (uint32_t)ipt) ++l;
    d.ipt = ipt;
    uint64_t num = 1ull << (31 + l);
    d.magic = (uint32_t)((num + (uint64_t)ipt - 1) / (uint64_t)ipt);
    d.shift = l - 1;
    return d;
}

__device__ __forceinline__ int interval_of(int t, const IntervalDiv &d) {
    return (int)(__umulhi((uint32_t)t, d.magic) >> d.shift);
}

struct FusedParams {
    // sizes
    int N, Np, Nw, A, O, Ow, K, P;
    int rptr_total;            // L, route positions over all routes
    IntervalDiv div;
    // network / routes (device)
    const int32_t *rptr;       // [P+1]
    const int32_t *rlinks;     // [L]
    const int32_t *obs_col;    // [A]
    const int32_t *od_ptr;     // [K+1]
    const int32_t *od_routes;  // [P] routes grouped by OD
    const int32_t *task_od;    // [K] OD processing order (largest work first)
    const int2 *rpack;         // [L] (link, observed column or -1) of every route position
    const int4 *groute;        // [P] walk order: (route, first position, links, start depth | own << 8 | OD << 9)
    const int2 *rtab;          // [L] (link, (observed column + 1) | event word << 24) of every route position
    const uint32_t *rtab32;    // [L] the same as link | (column + 1) << 11 | event word << 22, or null
    int rtab_off;              // byte offset of a shared-memory copy, -1 = read rtab from global memory
    int rtab_packed;           // the shared copy is rtab32
    const int32_t *gptr;       // [G+1] routes of each walk group in groute
    const int32_t *task_grp;   // [G] group processing order (largest walk first)
    const int32_t *rev;        // [L] (E << 1) | save of every route position (see build_groups)
    const int32_t *rod;        // [P] OD pair of each route
    int n_groups;
    int n_pair_groups;         // the first ones of task_grp are walked as tile pairs
    const int32_t *god_ptr;    // [G+1] ODs owned by each group (all their routes are in it)
    const int32_t *god;        // owned ODs
    const int32_t *godr_ptr;   // routes of each owned OD in godr
    const int32_t *godr;       // their indices in the group's walk order
    int n_god, n_godr;         // sizes of god and godr
    const int32_t *step_ods;   // [n_step_ods] ODs whose routes span groups: step pass
    int n_step_ods;
    const float *pt;           // [D][P][Np] route choice for the call's theta
    // per-day inputs
    const int32_t *ticks;
    const uint16_t *ticks16;   // [D][A][Np] 16-bit copy, entries >= N repeat row N-1 (tick windows)
    const float *counts;
    const uint32_t *mask;
    const uint32_t *colact;
    const float *C;
    const int32_t *maxoff;     // [D]
    const int64_t *tab_off;    // [D] offset of the repaired trajectory table, -1 if none
    const int32_t *traj_tab;
    // state / operands
    float *q;                  // [D][K][Np] FP32 (master in SOLVE, input otherwise)
    float *G;
    __nv_bfloat16 *qb;         // [D][K][Np] BF16 operand copy (BF16 form)
    void *rbuf;                // [grid][O][Np] residual slots (f32 or bf16)
    float *gring;              // [grid][O][Np] accumulators when the ring lives in global memory
    float *gp;                 // [grid][P][Np] route-level adjoint sums of the current phase
    // outputs
    double *loss;              // [D]
    float *trace;              // [iters][D] or null
    double *dtheta;            // [D] (LOSS_GRAD)
    float *gout;               // [D][K][Np] 2 B^T r (LOSS_GRAD)
    float *xout;               // [D][O][Np] (FORWARD)
    // control
    int n_days, iters, mode;
    float eta, eps, theta;
    int ring_rows;             // R rows per observed link in the shared ring, 0 = global ring
    int tick_rows;             // RW tick rows per link staged in shared memory, 0 = read global
    int tiles_per_phase;       // F (upper bound; the kernel lowers it for days with long trips)
    int *queue;
    int *err;
    // row chunks of Algorithm 1 (SOLVE with row_chunk = b > 0)
    int row_chunk;
    int day_base;
    unsigned long long seed;
    int32_t *lab;              // [grid][O][Np] chunk of each observed cell for the current epoch
    uint32_t *rc_bins;         // [grid][3][kRankBins] key-bin counts, first ranks, fill cursors
    unsigned long long *rc_key;  // [grid][O N] keys of the rows in bins that straddle a chunk boundary
    int32_t *rc_row;           // [grid][O N] their row ids
    // consecutive days solved jointly (trips that cross midnight reach the next day)
    int coupled;
    int halo_rows;             // S: rows of the next day that a day's trips reach
    int Nh;                    // deposit / gather horizon in rows: N, or N + S when coupled
    long long *early;          // [D][O][S] own deposits into the day's rows [0, S), 2^-20 vehicles
    long long *halo;           // [D][O][S] deposits into the next day's rows [0, S)
    int no_final;              // SOLVE: stop after the last step, no final forward
    // epoch slices (SOLVE): work unit u is slice u / D of day u % D, epochs
    // [s iters / S, (s + 1) iters / S); slice s of a day waits until slice s - 1 is done
    int slices;                // S >= 1
    int *progress;             // [D] slices done per day (zero at launch), or null when S = 1
    long long wait_ns;         // bound on that wait (globaltimer ns); past it: kErrDeviceTimeout
};

struct PrepParams {
    int N, Np, A, P, tps;
    IntervalDiv div;
    const int32_t *rptr, *rlinks;
    const int32_t *ticks;      // [D][A][Np]
    float *C;                  // [D][P][Np]
    int32_t *maxoff;           // [D]
    unsigned long long *repairs;  // [D]
    const int64_t *tab_off;    // [D] or null (pass 1)
    int32_t *traj_tab;
    int n_days;
    int coupled;               // entries past midnight take the next day's link times
};

struct PlainParams {
    int N, Np, Nw, A, O, K, P, n_pairs;
    IntervalDiv div;
    const int32_t *rptr, *rlinks, *rod, *od_ptr, *od_routes;
    const int32_t *pair_k, *pair_j, *pair_o;   // [n_pairs] (route, link position, observed column)
    const int32_t *route_pair_ptr;             // [P+1] pairs of route k
    const int32_t *ticks;
    const int64_t *tab_off;
    const int32_t *traj_tab;
    const float *C;
    float theta;
    int4 *rec;                 // [D][n_pairs][N] DAR records
    float *p;                  // [D][P][Np] route choice
    int n_days;
    int *err;
};

// DAR stability check (quality.cu): mean DAR over the loaded days, held as
// rbar[(l * N + h1) * W + (h2 - h1)] for route position l, and distances.
struct DarParams {
    int N, Np, A, P, L, W, n_days;
    IntervalDiv div;
    const int32_t *rptr, *rlinks;
    const int32_t *ticks;      // [D][A][Np]
    const int64_t *tab_off;    // [D] repaired trajectory table offset, -1 if none
    const int32_t *traj_tab;
    double *rbar;              // [L][N][W]
};

// Dense NNLS by Algorithm 1 (dense.cu): B [nr][nc], y / r [nr][m], x / G [nc][m].
struct DenseParams {
    const float *B, *y;
    float *x, *G, *r, *gpart;
    double *lpart;
    int nr, nc, m, grid_r, grid_g, rows_per_cta;
    int vec;                   // rows of B start on 16-byte boundaries (n_cols % 4 == 0, aligned base)
    float eta, eps;
    long long wait_limit;      // polls of a bounded wait on a row copy before it gives up
};

// error codes mirrored from dode.h for device use
constexpr int kErrArg = -1, kErrBadSpeed = -4, kErrTickOverflow = -5, kErrDeviceTimeout = -8, kErrUnsupported = -10,
              kErrBounds = -11;

__device__ __forceinline__ void set_error(int *err, int code, long long index) {
    if (atomicCAS(err, 0, code) == 0) {
        err[1] = (int)(index & 0x7fffffff);
        err[2] = (int)(index >> 31);
    }
}

// Index checks of the debug build (compiled with -DDODE_CHECK_BOUNDS): before a
// checked access, DODE_IN_BOUNDS(i, n, err, site) tests 0 <= i < n; a failed
// test records kErrBounds with the site number (bits 40..) and the low 40 bits
// of the index in the error word and the access is skipped, so a bad index
// never reaches memory.  The normal build compiles every check to `true`.
enum BoundsSite : int {
    kSiteRingDeposit = 1,     // accumulator cell of a deposit (shared ring or global)
    kSiteTickWindow = 2,      // tick read by a walk (shared window or global table)
    kSiteRingGather = 3,      // residual cell read by an adjoint walk
    kSiteWalkStack = 4,       // depth of a walk's branch-point stack
    kSiteGroupSums = 5,       // route index of a group's prefix sums
    kSiteFlushCell = 6,       // ring cell of a flush or a spill move
    kSiteStageTicks = 7,      // tick window row staged into shared memory
    kSiteStageResid = 8,      // residual window cell staged into shared memory
    kSiteDemand = 9,          // (day, OD, departure) cell of q and G
    kSiteDenseRing = 10,      // row copy of the dense one-pass ring
    kSiteDensePart = 11,      // gradient partial of the dense one-pass step
};

__device__ __forceinline__ bool bounds_check(long long i, long long n, int *err, int site) {
    if (i >= 0 && i < n) return true;
    set_error(err, kErrBounds, ((long long)site << 40) | (i & ((1ll << 40) - 1)));
    return false;
}

#ifdef DODE_CHECK_BOUNDS
#define DODE_IN_BOUNDS(i, n, err, site) ::dode::bounds_check((long long)(i), (long long)(n), (err), (site))
#else
#define DODE_IN_BOUNDS(i, n, err, site) true
#endif

// launchers (defined in the .cu files)
cudaError_t launch_ticks(const float *speeds, const float *len, int D, int N, int Np, int A, int tps,
                         int32_t *ticks, uint16_t *ticks16, int *maxtick, int *err, cudaStream_t s);
cudaError_t launch_prepare(const PrepParams &p, cudaStream_t s);
cudaError_t launch_transpose_in(const float *src, float *dst, int D, int N, int Np, int M,
                                cudaStream_t s);  // [D][N][M] -> [D][M][Np]
cudaError_t launch_transpose_out(const float *src, float *dst, int D, int N, int Np, int M, float scale,
                                 cudaStream_t s); // [D][M][Np] -> [D][N][M]
cudaError_t launch_pack_mask(const uint8_t *mask, uint32_t *bits, uint32_t *colact, int D, int N, int Nw,
                             int O, int Ow, cudaStream_t s);
cudaError_t launch_to_bf16(const float *src, __nv_bfloat16 *dst, size_t n, cudaStream_t s);
cudaError_t launch_route_choice(const float *C, const int32_t *rod, const int32_t *od_ptr, const int32_t *od_routes,
                                float theta, int D, int P, int N, int Np, float *pt, cudaStream_t s);
cudaError_t launch_fused(const FusedParams &p, int precision, int grid, int block, size_t smem,
                         cudaStream_t s);
cudaError_t fused_occupancy(int precision, int block, size_t smem, int *blocks_per_sm);
cudaError_t fused_set_attr(bool smem_ring, bool smem_ticks, int precision, size_t smem);
cudaError_t launch_r2(const float *counts, const uint32_t *mask, int D, int O, int N, int Np, int Nw,
                      const double *loss, double *sstot, double *r2, cudaStream_t s);
cudaError_t launch_day_totals(const double *loss, const double *dth, int D, double *out, cudaStream_t s);
cudaError_t launch_pattern_times(const float *C, int n_groups, const int32_t *gptr, const int32_t *gday, int P, int N,
                                 int Np, float *Ceff, cudaStream_t s);
cudaError_t launch_dar_distance(const DarParams &p, double *part, int n_part, double *rbar_sq, double *dist,
                                cudaStream_t s);
cudaError_t dense_iteration(const DenseParams &p, bool step, cudaStream_t s);
cudaError_t dense_loss(const DenseParams &p, double *loss, cudaStream_t s);
cudaError_t dense_set_smem(size_t resid_bytes, size_t grad_bytes);
cudaError_t dense_persist(const DenseParams &p, int iters, int grid, int S, size_t smem, int *err, unsigned int *gbar,
                          cudaStream_t s);
cudaError_t dense_persist_set_smem(size_t bytes);
// Tensor-core path (dense_tc.cu): device pointers; returns 0, -1 (no device) or
// -2 (CUDA error); *herr receives a device error code (a bounded wait ran out).
int dense_tc_nnls(int nr, int nc, int m, const float *B, const float *Y, int iters, float eta, float eps, float *X,
                  float *G, double *loss, float *kernel_ms, int *herr, cudaStream_t st);
cudaError_t launch_plain_build(const PlainParams &p, cudaStream_t s);
cudaError_t launch_plain_route_choice(const PlainParams &p, cudaStream_t s);
cudaError_t launch_plain_forward(const PlainParams &p, const float *q, float *xhat, cudaStream_t s);
cudaError_t launch_plain_residual(const PlainParams &p, const float *counts, const uint32_t *mask,
                                  float *xr, double *loss, float *trace_row, cudaStream_t s);
cudaError_t launch_plain_adjoint_step(const PlainParams &p, const float *r, float *q, float *G, float eta,
                                      float eps, cudaStream_t s);

}  // namespace dode
