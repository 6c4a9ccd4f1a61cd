// dense_tc.cu -- the paper's efficiency experiment (Sec. 5, "Algorithm
// efficiency") for many right-hand sides that share B, on the fifth-generation
// tensor cores.  With m columns stacked, Algorithm 1's two products become
// GEMMs that read B once each:
//   R = B X - Y        (M = n_rows, N = m, K = n_cols)   epilogue: residual, loss
//   g = B^T R          (M = n_cols, N = m, K = n_rows)   epilogue: Adagrad step and
//                                                        projection of X
// One kernel computes C = A Bop^T for K-major A [M][K] and Bop [N][K] in FP32
// storage with TF32 products and FP32 accumulation (tcgen05.mma kind::tf32), for
// N = m <= 256 in one tile, so that A -- the large operand -- is read exactly
// once per product.  B^T is kept as a second copy (built once per call) so that
// both products see a K-major A; X, G and R are kept transposed ([m][n]) so that
// they are K-major Bop operands and the epilogues store coalesced.
//
// Work items are (128-row M tile, range of K tiles): when there are fewer M tiles
// than SMs the K dimension is split.  Each item writes its partial product; a
// second kernel (k_tc_reduce, one block per M tile and 8 columns) sums the
// partials in K-range order and applies the epilogue, so results do not depend
// on timing.  Each item walks its K tiles from a rotated start, so that the CTAs
// do not all read the same Bop tile from L2 at the same time.
//
// Per CTA (persistent over work items):
//   warp 0   TMEM allocation; one lane issues the TMA tile loads (A: 128 x 32,
//            Bop: m x 32, 128-byte swizzle) into a ring of S stages (full[s]),
//            each holding kt consecutive K tiles (kt = 2 for m <= 128: every row
//            of A is then read in 256-byte runs)
//   warp 1   one lane issues the MMAs (four K = 8 steps per 32-wide K tile) into
//            one of two TMEM accumulators and commits them to the stage's
//            empty[s] barrier, and after the tile's last K step to tfull[a]
//   warps 4-7 drain: TMEM lane i = row i of the tile; tcgen05.ld 16 columns at
//            a time into the item's partial product; releases the accumulator
//            (tempty[a]) for the item after next
// Every wait is bounded: a wait that runs out sets the error word, the roles
// stop issuing, let their own copies and MMAs in flight complete (bounded) and
// the TMEM is released before the kernel returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "dode_internal.cuh"

namespace dode {

constexpr int kTcM = 128;                 // rows per tile (TMEM lanes)
constexpr int kTcK = 32;                  // K per tile: 32 FP32 = one 128-byte swizzle row
constexpr int kTcStages = 8;              // ring stages at most (fewer when they do not fit in shared memory)
constexpr int kTcThreads = 256;
constexpr int kTcRedCols = 8;             // columns per block of the reduce-and-epilogue kernel
constexpr long long kTcWait = 1ll << 26;

enum TcEpi : int { TC_RESID = 0, TC_STEP = 1, TC_RESID_ONLY = 2 };

struct TcParams {
    int M, K, N;                          // C [M][N] = A [M][K] Bop[N][K]^T
    int m_tiles, k_tiles;
    int ksplit, kpc;                      // split-K: work item = (M tile, K range of kpc tiles)
    int stages;                           // ring stages in use (<= kTcStages)
    int kt;                               // K tiles per stage (1 or 2, the kernel's template argument): with
                                          // 2, each row of A is read in 256-byte runs, which DRAM serves
                                          // with fewer row activations
    float *part;                          // [m_tiles * ksplit][N][128] partial products
    uint32_t idesc;                       // tcgen05 instruction descriptor
    // TC_RESID: Rt[j][i] = C[i][j] - Y[i][j], lpart[tile][j] = sum over the
    // tile's rows of (C - Y)^2
    const float *Yt;                      // [N][M] (Y transposed: coalesced per column)
    float *Rt;                            // [N][M]
    double *lpart;                        // [m_tiles][N]
    // TC_STEP: g = C; Gt[j][i] += g^2; Xt[j][i] = max(Xt[j][i] - eta g / (sqrt(Gt) + eps), 0)
    float *Xt, *Gt;                       // [N][M]
    float eta, eps;
    int *err;
};

__device__ __forceinline__ uint32_t tc_smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool tc_try(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(tc_smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, const volatile int *abort) {
    for (long long it = 0; it < kTcWait; ++it) {
        if (tc_try(bar, parity)) return true;
        if (abort && *abort) return false;
    }
    return false;
}

// Shared-memory matrix descriptor of a K-major tile stored with the 128-byte
// swizzle (rows of 128 bytes, 8-row groups 1024 bytes apart): start address,
// stride-dimension offset 1024 bytes, descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3fffu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

template <int KT>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages], tfull[2], tempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_cta;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = p.stages;
    // 1024-byte aligned stages: A tile then Bop tile
    const uint32_t sbase = (tc_smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t a_bytes = kTcM * kTcK * 4, b_bytes = (uint32_t)p.N * kTcK * 4;
    // a stage holds KT consecutive K tiles: A tiles first, then Bop tiles
    constexpr int kt = KT;
    const uint32_t stage_bytes = ((uint32_t)kt * (a_bytes + b_bytes) + 1023u) & ~1023u;
    const int ncols = p.N * 2 <= 32 ? 32 : (p.N * 2 <= 64 ? 64 : (p.N * 2 <= 128 ? 128 : (p.N * 2 <= 256 ? 256 : 512)));

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&empty[s])) : "memory");
        }
        for (int a = 0; a < 2; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&tfull[a])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(tc_smem_u32(&tempty[a])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_cta = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc_smem_u32(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = tmem_base;
    int n_local = 0;
    const int n_items = p.m_tiles * p.ksplit;
    for (int t = blockIdx.x; t < n_items; t += gridDim.x) ++n_local;
    // K tiles of work item t, walked from a rotated start
    auto krange = [&](int t, int &kb, int &nk, int &rot) {
        const int mt = t / p.ksplit, ks = t - mt * p.ksplit;
        kb = ks * p.kpc;
        nk = max(0, min(p.k_tiles, kb + p.kpc) - kb);
        rot = nk > 0 ? (int)(((unsigned)mt * 7u) % (unsigned)nk) : 0;
    };

    if (warp == 0 && lane == 0) {
        // ------------------------------ TMA producer ------------------------------
        long long it = 0, issued = 0;
        for (int lt = 0; lt < n_local && !abort_cta; ++lt) {
            const int item = blockIdx.x + lt * gridDim.x, tile = item / p.ksplit;
            int kb, nk, rot;
            krange(item, kb, nk, rot);
            for (int jk = 0; jk < nk; jk += kt, ++it) {
                const int nt = KT == 1 ? 1 : min(kt, nk - jk);
                const int s = (int)(it % S);
                if (it >= S && !tc_wait(&empty[s], (uint32_t)((it / S - 1) & 1), &abort_cta)) {
                    abort_cta = 1;
                    atomicCAS(p.err, 0, kErrDeviceTimeout);
                    break;
                }
                const uint32_t sa = sbase + (uint32_t)s * stage_bytes, sb = sa + (uint32_t)kt * a_bytes;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem_u32(&full[s])),
                             "r"((uint32_t)nt * (a_bytes + b_bytes))
                             : "memory");
                if constexpr (KT == 1) {
                    const int k = kb + (jk + rot) % nk;
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                        "%3}], [%4];" ::"r"(sa),
                        "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(k * kTcK), "r"(tile * kTcM),
                        "r"(tc_smem_u32(&full[s]))
                        : "memory");
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                        "%3}], [%4];" ::"r"(sb),
                        "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(k * kTcK), "r"(0), "r"(tc_smem_u32(&full[s]))
                        : "memory");
                } else {
                    for (int t = 0; t < nt; ++t) {
                        const int k = kb + (jk + t + rot) % nk;
                        asm volatile(
                            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                            "%3}], [%4];" ::"r"(sa + (uint32_t)t * a_bytes),
                            "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(k * kTcK), "r"(tile * kTcM),
                            "r"(tc_smem_u32(&full[s]))
                            : "memory");
                        asm volatile(
                            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                            "%3}], [%4];" ::"r"(sb + (uint32_t)t * b_bytes),
                            "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(k * kTcK), "r"(0), "r"(tc_smem_u32(&full[s]))
                            : "memory");
                    }
                }
                issued = it + 1;
            }
        }
        // the loads in flight write this CTA's shared memory: let them land
        for (long long q = issued > S ? issued - S : 0; q < issued; ++q)
            tc_wait(&full[q % S], (uint32_t)((q / S) & 1), nullptr);
    } else if (warp == 1 && lane == 0) {
        // ------------------------------ MMA issuer ------------------------------
        long long it = 0;
        bool any = false;
        uint64_t *last = nullptr;
        uint32_t last_par = 0;
        for (int lt = 0; lt < n_local && !abort_cta; ++lt) {
            const int a = lt & 1;
            if (lt >= 2 && !tc_wait(&tempty[a], (uint32_t)((lt / 2 - 1) & 1), &abort_cta)) {
                abort_cta = 1;
                atomicCAS(p.err, 0, kErrDeviceTimeout);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t d = tbase + (uint32_t)(a * p.N);
            bool ok = true;
            int kb, nk, rot;
            krange(blockIdx.x + lt * gridDim.x, kb, nk, rot);
            for (int jk = 0; jk < nk; jk += kt, ++it) {
                const int nt = KT == 1 ? 1 : min(kt, nk - jk);
                const int s = (int)(it % S);
                if (!tc_wait(&full[s], (uint32_t)((it / S) & 1), &abort_cta)) {
                    abort_cta = 1;
                    atomicCAS(p.err, 0, kErrDeviceTimeout);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = sbase + (uint32_t)s * stage_bytes, sb = sa + (uint32_t)kt * a_bytes;
                if constexpr (KT == 1) {
#pragma unroll
                    for (int kk = 0; kk < kTcK / 8; ++kk) {
                        // K = 8 TF32 elements = 32 bytes per MMA: advance the start addresses
                        const uint64_t ad = tc_desc(sa + 32u * kk), bd = tc_desc(sb + 32u * kk);
                        const uint32_t acc = (jk > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                            "l"(ad), "l"(bd), "r"(p.idesc), "r"(acc)
                            : "memory");
                    }
                } else {
                    for (int t = 0; t < nt; ++t) {
#pragma unroll
                        for (int kk = 0; kk < kTcK / 8; ++kk) {
                            // K = 8 TF32 elements = 32 bytes per MMA: advance the start addresses
                            const uint64_t ad = tc_desc(sa + (uint32_t)t * a_bytes + 32u * kk),
                                           bd = tc_desc(sb + (uint32_t)t * b_bytes + 32u * kk);
                            const uint32_t acc = (jk > 0 || t > 0 || kk > 0) ? 1u : 0u;
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                                "l"(ad), "l"(bd), "r"(p.idesc), "r"(acc)
                                : "memory");
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 tc_smem_u32(&empty[s]))
                             : "memory");
                any = true;
                last = &empty[s];
                last_par = (uint32_t)((it / S) & 1);
            }
            if (!ok) break;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tc_smem_u32(&tfull[a]))
                         : "memory");
            last = &tfull[a];
            last_par = (uint32_t)((lt / 2) & 1);
        }
        // MMAs in flight read shared memory and write TMEM: let them complete
        if (any && last) tc_wait(last, last_par, nullptr);
    } else if (warp >= 4) {
        // -------------------- drain: accumulator -> partial product --------------------
        const int w4 = warp - 4, r = w4 * 32 + lane;
        for (int lt = 0; lt < n_local; ++lt) {
            const int a = lt & 1;
            const int item = blockIdx.x + lt * gridDim.x;
            const bool got = tc_wait(&tfull[a], (uint32_t)((lt / 2) & 1), &abort_cta);
            // the four drain warps take the same decision
            uint32_t all;
            asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, 2, 128, q;\n"
                         " selp.u32 %0, 1, 0, p;\n}\n"
                         : "=r"(all)
                         : "r"(got ? 1u : 0u)
                         : "memory");
            if (!all) {
                if (lane == 0) {
                    abort_cta = 1;
                    atomicCAS(p.err, 0, kErrDeviceTimeout);
                }
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int c0 = 0; c0 < p.N; c0 += 16) {
                uint32_t v[16];
                const uint32_t taddr = tbase + ((uint32_t)(w4 * 32) << 16) + (uint32_t)(a * p.N + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float *pp = p.part + ((size_t)item * p.N + c0) * kTcM + r;
#pragma unroll
                for (int q = 0; q < 16; ++q) pp[(size_t)q * kTcM] = __uint_as_float(v[q]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_smem_u32(&tempty[a])) : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(ncols) : "memory");
}

// The split-K partials of C summed in K-range order, then the epilogue: block
// (M tile, kTcRedCols columns), thread = row of the tile; narrow column blocks
// give enough blocks to hide the partials' load latency.
//   TC_RESID: Rt[j][i] = C[i][j] - Y[i][j]; lpart[tile][j] = sum over the tile's rows of r^2
//   TC_RESID_ONLY: Rt alone (the iterations before the last need no loss, and
//            its FP64 warp sums run on the slow FP64 pipe)
//   TC_STEP:  Gt[j][i] += g^2, Xt[j][i] = max(Xt[j][i] - eta g / (sqrt(Gt) + eps), 0) with g = C[i][j]
template <int EPI>
__global__ void __launch_bounds__(kTcM) k_tc_reduce(const TcParams p) {
    __shared__ double red[4][kTcRedCols];
    const int tile = blockIdx.x, j0 = blockIdx.y * kTcRedCols, r = threadIdx.x, lane = r & 31, w = r >> 5;
    const int row = tile * kTcM + r;
    const bool live = row < p.M;
    const int nj = min(kTcRedCols, p.N - j0);
    for (int jq = 0; jq < nj; jq += 8) {
        float c[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) c[q] = 0.f;
        for (int ks = 0; ks < p.ksplit; ++ks) {
            const float *pp = p.part + ((size_t)(tile * p.ksplit + ks) * p.N + j0 + jq) * kTcM + r;
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = (jq + q < nj) ? __ldcg(pp + (size_t)q * kTcM) : 0.f;
#pragma unroll
            for (int q = 0; q < 8; ++q) c[q] += v[q];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = j0 + jq + q;
            if (jq + q >= nj) break;
            if (EPI == TC_RESID) {
                double l2 = 0.0;
                if (live) {
                    const float rr = c[q] - __ldg(p.Yt + (size_t)j * p.M + row);
                    p.Rt[(size_t)j * p.M + row] = rr;
                    l2 = (double)rr * (double)rr;
                }
                for (int off = 16; off > 0; off >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, off);
                if (lane == 0) red[w][jq + q] = l2;
            } else if (EPI == TC_RESID_ONLY) {
                if (live) p.Rt[(size_t)j * p.M + row] = c[q] - __ldg(p.Yt + (size_t)j * p.M + row);
            } else if (live) {
                const size_t e = (size_t)j * p.M + row;
                const float g = c[q];
                const float Gv = p.Gt[e] + g * g;
                p.Gt[e] = Gv;
                p.Xt[e] = fmaxf(p.Xt[e] - p.eta * g / (sqrtf(Gv) + p.eps), 0.f);
            }
        }
    }
    if (EPI == TC_RESID) {
        __syncthreads();
        if (r < nj) p.lpart[(size_t)tile * p.N + j0 + r] = ((red[0][r] + red[1][r]) + red[2][r]) + red[3][r];
    }
}

// r = B x - y and g = B^T r for m columns: column-major helpers of the host code
__global__ void k_tc_transpose(const float *__restrict__ src, float *__restrict__ dst, int rows, int cols) {
    __shared__ float tile[32][33];
    const int c = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i;
        if (r < rows && c < cols) tile[i][threadIdx.x] = src[(size_t)r * cols + c];
    }
    __syncthreads();
    const int r = r0 + threadIdx.x, cb = blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int cc = cb + i;
        if (r < rows && cc < cols) dst[(size_t)cc * rows + r] = tile[threadIdx.x][i];
    }
}

// loss[j] = sum over the tiles and warps, in that order, of the partials
__global__ void k_tc_loss(const double *__restrict__ lpart, int n_part, int N, double *__restrict__ loss) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double s = 0.0;
    for (int b = 0; b < n_part; ++b) s += lpart[(size_t)b * N + j];
    loss[j] = s;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tc_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

// Tensor map of a row-major FP32 matrix [rows][cols] (cols % 4 == 0, 16-byte
// aligned base), box [box_rows][32], 128-byte swizzle, out-of-range reads 0.
static bool tc_map(CUtensorMap *m, const float *base, int rows, int cols, int box_rows) {
    auto fn = tc_encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
    cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static uint32_t tc_idesc(int N) {
    // D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and 10-12 = 2), both K-major,
    // N >> 3 at bits 17-22, M >> 4 at bits 24-28
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

static size_t tc_stage_bytes(int N, int kt) {
    return ((size_t)kt * ((size_t)kTcM * kTcK * 4 + (size_t)N * kTcK * 4) + 1023) & ~(size_t)1023;
}

// stages that fit beside the kernel's static shared memory (about 200 KB of ring)
static int tc_stages(int N, int kt) {
    return (int)std::max<size_t>(2, std::min<size_t>(kTcStages, (200u << 10) / tc_stage_bytes(N, kt)));
}

// two K tiles per stage while at least three such stages fit (m <= 128; per iteration at
// n = 6000 / 8000: m = 64 80.8 -> 72.8 / 136.7 -> 107.7 us, m = 128 85.0 -> 79.1 / 139.9 -> 116.2 us),
// else one (at m = 256 two tiles leave only two stages: 93.8 -> 103.5 us)
static int tc_kt(int N) { return (200u << 10) / tc_stage_bytes(N, 2) >= 3 ? 2 : 1; }

static size_t tc_smem(int N) { return tc_stage_bytes(N, tc_kt(N)) * tc_stages(N, tc_kt(N)) + 1024; }

// One product: the GEMM's partial products, then their fixed-order sum and the epilogue.
template <int EPI>
static cudaError_t tc_launch(const CUtensorMap &a, const CUtensorMap &b, const TcParams &p, int grid, cudaStream_t s) {
    if (p.kt == 2)
        k_tc_gemm<2><<<grid, kTcThreads, tc_smem(p.N), s>>>(a, b, p);
    else
        k_tc_gemm<1><<<grid, kTcThreads, tc_smem(p.N), s>>>(a, b, p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tc_reduce<EPI><<<dim3(p.m_tiles, (p.N + kTcRedCols - 1) / kTcRedCols), kTcM, 0, s>>>(p);
    return cudaGetLastError();
}

// Algorithm 1 on B [nr][nc] for the m columns of Y with TF32 tensor-core
// products.  Device pointers; X, G are [nc][m] in and out; loss [m].
int dense_tc_nnls(int nr, int nc, int m, const float *B, const float *Y, int iters, float eta, float eps, float *X,
                  float *G, double *loss, float *kernel_ms, int *herr, cudaStream_t st) {
    *herr = 0;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    const size_t nB = (size_t)nr * nc;
    const int mt1 = (nr + kTcM - 1) / kTcM, mt2 = (nc + kTcM - 1) / kTcM;
    float *Bt = nullptr, *Xt = nullptr, *Gt = nullptr, *Rt = nullptr, *Yt = nullptr;
    double *lpart = nullptr;
    float *part = nullptr;
    int *derr = nullptr;
    cudaError_t e = cudaMalloc(&Bt, nB * 4);
    if (e == cudaSuccess) e = cudaMalloc(&Xt, (size_t)m * nc * 4);
    if (e == cudaSuccess) e = cudaMalloc(&Gt, (size_t)m * nc * 4);
    if (e == cudaSuccess) e = cudaMalloc(&Rt, (size_t)m * nr * 4);
    if (e == cudaSuccess) e = cudaMalloc(&Yt, (size_t)m * nr * 4);
    if (e == cudaSuccess) e = cudaMalloc(&lpart, (size_t)mt1 * m * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
    // partial products: at most max(n_sm, M tiles) work items of one GEMM, 128 x m each
    if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)std::max(n_sm, std::max(mt1, mt2)) * m * kTcM * 4);
    CUtensorMap tB, tBt, tXt, tRt;
    bool maps = e == cudaSuccess && tc_map(&tB, B, nr, nc, kTcM) && tc_map(&tBt, Bt, nc, nr, kTcM) &&
                tc_map(&tXt, Xt, m, nc, m) && tc_map(&tRt, Rt, m, nr, m);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess && !maps) e = cudaErrorInvalidValue;
    const dim3 tb(32, 8);
    if (e == cudaSuccess) {
        k_tc_transpose<<<dim3((nc + 31) / 32, (nr + 31) / 32), tb, 0, st>>>(B, Bt, nr, nc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_tc_transpose<<<dim3((m + 31) / 32, (nc + 31) / 32), tb, 0, st>>>(X, Xt, nc, m);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_tc_transpose<<<dim3((m + 31) / 32, (nr + 31) / 32), tb, 0, st>>>(Y, Yt, nr, m);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        if (G) {
            k_tc_transpose<<<dim3((m + 31) / 32, (nc + 31) / 32), tb, 0, st>>>(G, Gt, nc, m);
            e = cudaGetLastError();
        } else {
            e = cudaMemsetAsync(Gt, 0, (size_t)m * nc * 4, st);
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    TcParams p1{}, p2{};
    p1.M = nr; p1.K = nc; p1.N = m; p1.m_tiles = mt1; p1.k_tiles = (nc + kTcK - 1) / kTcK; p1.idesc = tc_idesc(m);
    p1.Yt = Yt; p1.Rt = Rt; p1.lpart = lpart; p1.err = derr;
    p2.M = nc; p2.K = nr; p2.N = m; p2.m_tiles = mt2; p2.k_tiles = (nr + kTcK - 1) / kTcK; p2.idesc = tc_idesc(m);
    p2.Xt = Xt; p2.Gt = Gt; p2.eta = eta; p2.eps = eps; p2.err = derr;
    // split K when there are fewer M tiles than SMs (at least 4 K tiles per item)
    for (TcParams *pp : {&p1, &p2}) {
        pp->ksplit = std::max(1, std::min(pp->k_tiles / 4, n_sm / pp->m_tiles));
        pp->kpc = (pp->k_tiles + pp->ksplit - 1) / pp->ksplit;
        pp->ksplit = (pp->k_tiles + pp->kpc - 1) / pp->kpc;
        pp->part = part;
        pp->kt = tc_kt(m);
        pp->stages = tc_stages(m, pp->kt);
    }
    const int g1 = std::min(n_sm, mt1 * p1.ksplit), g2 = std::min(n_sm, mt2 * p2.ksplit);
    // the iterations' launches (four per iteration) are captured once into a CUDA
    // graph on a private stream and replayed on the caller's: the host then
    // issues one launch instead of 4 iters + 3
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_kt(m) == 2 ? (const void *)k_tc_gemm<2> : (const void *)k_tc_gemm<1>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(m));
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t ec = cudaSuccess;
        for (int it = 0; it < iters && ec == cudaSuccess; ++it) {
            ec = tc_launch<TC_RESID_ONLY>(tB, tXt, p1, g1, cs);
            if (ec == cudaSuccess) ec = tc_launch<TC_STEP>(tBt, tRt, p2, g2, cs);
        }
        if (ec == cudaSuccess) ec = tc_launch<TC_RESID>(tB, tXt, p1, g1, cs);    // residual and loss of the final X
        if (ec == cudaSuccess) {
            k_tc_loss<<<(m + 127) / 128, 128, 0, cs>>>(lpart, mt1, m, loss);
            ec = cudaGetLastError();
        }
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = ec;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) {
        k_tc_transpose<<<dim3((nc + 31) / 32, (m + 31) / 32), tb, 0, st>>>(Xt, X, m, nc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && G) {
        k_tc_transpose<<<dim3((nc + 31) / 32, (m + 31) / 32), tb, 0, st>>>(Gt, G, m, nc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && kernel_ms) e = cudaEventElapsedTime(kernel_ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    cudaFree(Bt);
    cudaFree(Xt);
    cudaFree(Gt);
    cudaFree(Rt);
    cudaFree(Yt);
    cudaFree(lpart);
    cudaFree(part);
    cudaFree(derr);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return -2;
    }
    return 0;
}

}  // namespace dode
