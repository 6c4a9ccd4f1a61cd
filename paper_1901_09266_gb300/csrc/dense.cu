// dense.cu -- the paper's efficiency experiment (Sec. 5, "Algorithm
// efficiency"): NNLS(B, y) for a dense random B solved by Algorithm 1 (SPGD
// with Adagrad and projection, full-row updates), for m right-hand sides that
// share B.  Each iteration reads B twice, once per product:
//   k_dense_resid  r = B x - y      one warp per row, x staged in shared memory,
//                                   16-byte loads along the row, warp-sum;
//                                   per-CTA FP64 loss partials
//   k_dense_grad   g = B^T r        a CTA per (block of rows, 1024 columns),
//                                   each thread a 4-column strip, 16-byte
//                                   loads; partial gradients per row block
//   k_dense_step   sums the partials in a fixed order, then G += g^2,
//                  x = max(x - eta g / (sqrt(G) + eps), 0)
// All sums have a fixed order: results do not depend on timing.
#include "dode_internal.cuh"

namespace dode {

constexpr int kDenseMaxRhs = 8;

// r[i][j] = sum_c B[i][c] x[c][j] - y[i][j]; lpart[cta][j] = sum over the CTA's rows of r^2.
__global__ void __launch_bounds__(256) k_dense_resid(const float *__restrict__ B, const float *__restrict__ x,
                                                     const float *__restrict__ y, int nr, int nc, int m, int vec16,
                                                     float *__restrict__ r, double *__restrict__ lpart) {
    extern __shared__ __align__(16) float xs[];      // [nc][m]
    __shared__ double red[8][kDenseMaxRhs];
    for (int i = threadIdx.x; i < nc * m; i += blockDim.x) xs[i] = x[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double l2[kDenseMaxRhs];
#pragma unroll
    for (int j = 0; j < kDenseMaxRhs; ++j) l2[j] = 0.0;
    const bool vec = vec16 != 0;                        // rows 16-byte aligned
    for (int i = blockIdx.x * nw + warp; i < nr; i += gridDim.x * nw) {
        const float *row = B + (size_t)i * nc;
        float acc[kDenseMaxRhs];
#pragma unroll
        for (int j = 0; j < kDenseMaxRhs; ++j) acc[j] = 0.f;
        if (vec) {
            for (int c0 = 4 * lane; c0 < nc; c0 += 512) {
                float4 b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c = c0 + 128 * u;
                    b[u] = c < nc ? __ldg(reinterpret_cast<const float4 *>(row + c)) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c = c0 + 128 * u;
                    if (c < nc)
#pragma unroll
                        for (int j = 0; j < kDenseMaxRhs; ++j)
                            if (j < m)
                                acc[j] += b[u].x * xs[c * m + j] + b[u].y * xs[(c + 1) * m + j] +
                                          b[u].z * xs[(c + 2) * m + j] + b[u].w * xs[(c + 3) * m + j];
                }
            }
        } else {
            for (int c = lane; c < nc; c += 32) {
                const float b = __ldg(row + c);
#pragma unroll
                for (int j = 0; j < kDenseMaxRhs; ++j)
                    if (j < m) acc[j] += b * xs[c * m + j];
            }
        }
#pragma unroll
        for (int j = 0; j < kDenseMaxRhs; ++j) {
            if (j >= m) break;
            float v = acc[j];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            const float ri = v - y[(size_t)i * m + j];
            if (lane == 0) r[(size_t)i * m + j] = ri;
            l2[j] += (double)ri * (double)ri;
        }
    }
#pragma unroll
    for (int j = 0; j < kDenseMaxRhs; ++j)
        if (lane == 0 && j < m) red[warp][j] = l2[j];
    __syncthreads();
    if (threadIdx.x < m) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w][threadIdx.x];
        lpart[(size_t)blockIdx.x * m + threadIdx.x] = s;
    }
}

// gpart[rb][c][j] = sum over the rows i of row block rb of B[i][c] r[i][j]:
// blockIdx.y is the row block, blockIdx.x a 1024-column tile, each thread one
// 4-column strip; eight rows' 16-byte loads in flight.
__global__ void __launch_bounds__(256) k_dense_grad(const float *__restrict__ B, const float *__restrict__ r, int nr,
                                                    int nc, int m, int vec16, int rows_per_cta,
                                                    float *__restrict__ gpart) {
    extern __shared__ __align__(16) float rs[];      // [rows_per_cta][m]
    const int r0 = blockIdx.y * rows_per_cta, r1 = min(nr, r0 + rows_per_cta);
    for (int i = threadIdx.x; i < (r1 - r0) * m; i += blockDim.x) rs[i] = r[(size_t)r0 * m + i];
    __syncthreads();
    const int c = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= nc) return;
    float *gp = gpart + (size_t)blockIdx.y * nc * m;
    const bool vec = vec16 != 0;
    float acc[4][kDenseMaxRhs];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j < kDenseMaxRhs; ++j) acc[u][j] = 0.f;
    for (int i0 = r0; i0 < r1; i0 += 8) {
        float b[8][4];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int i = i0 + v;
            if (i < r1 && vec) {
                const float4 x = __ldg(reinterpret_cast<const float4 *>(B + (size_t)i * nc + c));
                b[v][0] = x.x;
                b[v][1] = x.y;
                b[v][2] = x.z;
                b[v][3] = x.w;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) b[v][u] = (i < r1 && c + u < nc) ? __ldg(B + (size_t)i * nc + c + u) : 0.f;
            }
        }
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int i = i0 + v;
            if (i >= r1) break;
            const float *ri = rs + (size_t)(i - r0) * m;
#pragma unroll
            for (int j = 0; j < kDenseMaxRhs; ++j)
                if (j < m) {
                    const float rv = ri[j];
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[u][j] += b[v][u] * rv;
                }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (c + u < nc)
#pragma unroll
            for (int j = 0; j < kDenseMaxRhs; ++j)
                if (j < m) gp[(size_t)(c + u) * m + j] = acc[u][j];
}

// g = sum of the partials in a fixed order; Adagrad step and projection.  A
// CTA takes 32 entries; warp w sums the partials b = w, w + 8, ... of each
// (coalesced rows of 32), and the eight warp sums are added in warp order.
__global__ void __launch_bounds__(256) k_dense_step(const float *__restrict__ gpart, int n_part, int nc, int m,
                                                    float eta, float eps, float *__restrict__ x, float *__restrict__ G) {
    __shared__ float red[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t ne = (size_t)nc * m;
    const size_t e = (size_t)blockIdx.x * 32 + lane;
    float g = 0.f;
    if (e < ne)
        for (int b = warp; b < n_part; b += 8) g += gpart[(size_t)b * ne + e];
    red[warp][lane] = g;
    __syncthreads();
    if (warp != 0 || e >= ne) return;
    g = 0.f;
    for (int w = 0; w < 8; ++w) g += red[w][lane];
    const float Gv = G[e] + g * g;
    G[e] = Gv;
    x[e] = fmaxf(x[e] - eta * g / (sqrtf(Gv) + eps), 0.f);
}

__global__ void k_dense_loss(const double *__restrict__ lpart, int n_part, int m, double *__restrict__ loss) {
    const int j = threadIdx.x;
    if (j >= m) return;
    double s = 0.0;
    for (int b = 0; b < n_part; ++b) s += lpart[(size_t)b * m + j];
    loss[j] = s;
}

// ---------------------------------------------------------------------------
// One pass over B per iteration, every iteration in one cooperative launch
// (one right-hand side, n_cols % 4 == 0, n_cols <= 8192, 16-byte aligned B).
// CTA c (one per SM, all resident) owns rows [c rpc, (c + 1) rpc) of B and
// streams them, row by row, through a ring of S shared-memory stages with bulk
// asynchronous copies (TMA).  B does not change between iterations, so the
// copies run on into the next iteration's rows while the grid synchronises.
// Warp roles, synchronised by mbarriers only:
//   warp 8      producer: one lane issues row copies into free stages
//               (full[s] completes when the row has landed; empty[s] when the
//               consumers are done with the stage)
//   warps 0..3  residuals: warp w takes the row copies q = w mod 4 (counted
//               over the whole launch) and forms r_j = B_j . x - y_j from shared
//               memory (a warp sum), publishing it through rready[s]
//   warps 4..7  gradient: thread t owns the 4-column strips c = 4 t + 512 k and
//               adds r_j B_j to them, rows in order
// After its rows the CTA writes its partial gradient to gpart[cta]; grid
// barrier; CTA c sums the partials of its columns in a fixed order and takes
// Algorithm 1's step for them (Adagrad and projection); grid barrier; every CTA
// reloads x.  Pass `iters` forms the residuals and the loss of the final x only.
// Every wait is bounded (wait_limit polls for the stream, a fixed limit for the
// drain and the grid barriers); a wait that runs out sets the error word, the
// producer stops issuing and lets its copies in flight land (bounded), the grid
// barriers give up once the error word is set, and the kernel returns.
// ---------------------------------------------------------------------------
constexpr int kPersistStages = 8;                   // ring stages (rows): 4 or 8, a multiple of the residual warps
constexpr int kPersistStrips = 16;                  // n_cols <= 16 * 512
constexpr int kReloadVecs = kPersistStrips * 512 / 4 / 256;   // 16-byte loads per compute thread for x
constexpr int kPersistThreads = 288;                // 8 compute warps + 1 producer warp
constexpr long long kDrainLimit = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase of `bar` with this parity: at most `limit` polls, and none
// once *abort is set.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit, const volatile int *abort) {
    for (long long it = 0; it < limit; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (abort && *abort) return false;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Grid barrier number k of the launch (all CTAs resident: cooperative launch):
// one thread per CTA arrives on the counter and polls it, at most `limit`
// polls, giving up once the error word is set.
__device__ bool grid_barrier(unsigned int *count, unsigned int k, const volatile int *err, long long limit) {
    __threadfence();
    atomicAdd(count, 1u);
    const unsigned int target = gridDim.x * (k + 1);
    for (long long it = 0; it < limit; ++it) {
        unsigned int v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
        if (v >= target) return true;
        if (*err) return false;
        __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void bar_compute() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__global__ void __launch_bounds__(kPersistThreads, 1)
    k_dense_persist(const DenseParams p, int iters, int S, int *err, unsigned int *gbar) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kPersistStages], empty[kPersistStages], rready[kPersistStages];
    __shared__ float rval[kPersistStages];
    __shared__ float gred[8][32];
    __shared__ double lred[4];
    __shared__ int abort_cta;    // set by any warp whose wait ran out (the producer stops issuing)
    __shared__ int stop_cta;     // the compute warps' common decision to stop, taken by thread 0 between barriers
    const int nc = p.nc, nr = p.nr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *xs = reinterpret_cast<float *>(smem_raw);
    const size_t xbytes = ((size_t)nc * 4 + 127) & ~(size_t)127;
    float *ring = reinterpret_cast<float *>(smem_raw + xbytes);
    const int rpc = (nr + gridDim.x - 1) / gridDim.x;
    const int row0 = blockIdx.x * rpc;
    const int nrow = max(0, min(rpc, nr - row0));
    const long long nseq = (long long)(iters + 1) * nrow;

    if (tid == 0) {
        for (int st = 0; st < S; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[st])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&rready[st])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 5;" ::"r"(smem_u32(&empty[st])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_cta = 0;
        stop_cta = 0;
    }
    for (int i = tid; i < nc; i += blockDim.x) xs[i] = __ldcg(p.x + i);
    __syncthreads();

    if (warp == 8) {
        // ------------------------------ producer ------------------------------
        if (lane == 0) {
            long long issued = 0;
            for (long long q = 0; q < nseq; ++q) {
                const int st = (int)(q % S);
                if (q >= S && !mbar_wait(&empty[st], (uint32_t)((q / S - 1) & 1), p.wait_limit, &abort_cta)) {
                    abort_cta = 1;
                    atomicCAS(err, 0, kErrDeviceTimeout);
                    break;
                }
                if (abort_cta) break;
                const uint32_t bytes = (uint32_t)nc * 4u;
                float *dst = ring + (size_t)st * nc;
                if (!DODE_IN_BOUNDS(row0 + (int)(q % nrow), nr, err, kSiteDenseRing)) {
                    abort_cta = 1;
                    break;
                }
                const float *src = p.B + (size_t)(row0 + (int)(q % nrow)) * nc;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&full[st])),
                             "r"(bytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(dst)),
                    "l"(src), "r"(bytes), "r"(smem_u32(&full[st]))
                    : "memory");
                issued = q + 1;
            }
            // the copies in flight write this CTA's shared memory: let them land
            for (long long q = max(0ll, issued - S); q < issued; ++q)
                mbar_wait(&full[q % S], (uint32_t)((q / S) & 1), kDrainLimit, nullptr);
        }
    } else {
        // --------------------------- compute warps ----------------------------
        const bool resid = warp < 4;
        float acc[kPersistStrips][4];
        unsigned int nbar = 0;
        for (int it = 0; it <= iters; ++it) {
            const bool last = it == iters;
#pragma unroll
            for (int k = 0; k < kPersistStrips; ++k)
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[k][u] = 0.f;
            double l2 = 0.0;
            if (resid) {
                // warp w takes the copies q = w mod 4 of the whole launch; with S a
                // multiple of 4 the previous use of a stage (q - S) was this warp's
                // too, so every wait is on the phase right after one it has seen
                // complete (a parity wait cannot alias an older phase)
                const long long qb = (long long)it * nrow, qe = qb + nrow;
                for (long long q = qb + (((warp - qb) % 4) + 4) % 4; q < qe; q += 4) {
                    const int j = (int)(q - qb);
                    const int st = (int)(q % S);
                    const bool ok = mbar_wait(&full[st], (uint32_t)((q / S) & 1), p.wait_limit, &abort_cta);
                    float v = 0.f;
                    if (ok) {
                        const float *row = ring + (size_t)st * nc;
                        for (int c = 4 * lane; c < nc; c += 128) {
                            const float4 b = *reinterpret_cast<const float4 *>(row + c);
                            const float4 xv = *reinterpret_cast<const float4 *>(xs + c);
                            v += b.x * xv.x + b.y * xv.y + b.z * xv.z + b.w * xv.w;
                        }
                    } else if (lane == 0) {
                        abort_cta = 1;
                        atomicCAS(err, 0, kErrDeviceTimeout);
                    }
                    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                    const float ri = v - __ldg(p.y + row0 + j);
                    l2 += (double)ri * (double)ri;
                    __syncwarp();
                    if (lane == 0) {
                        rval[st] = ri;
                        mbar_arrive(&rready[st]);
                        mbar_arrive(&empty[st]);
                    }
                }
            } else {
                const int t = tid - 128;
                for (int j = 0; j < nrow; ++j) {
                    const long long q = (long long)it * nrow + j;
                    const int st = (int)(q % S);
                    const uint32_t par = (uint32_t)((q / S) & 1);
                    const bool ok = mbar_wait(&rready[st], par, p.wait_limit, &abort_cta) &&
                                    mbar_wait(&full[st], par, p.wait_limit, &abort_cta);
                    if (ok && !last) {
                        const float rv = rval[st];
                        const float *row = ring + (size_t)st * nc;
#pragma unroll
                        for (int k = 0; k < kPersistStrips; ++k) {
                            const int c = 4 * t + 512 * k;
                            if (c < nc) {
                                const float4 b = *reinterpret_cast<const float4 *>(row + c);
                                acc[k][0] += b.x * rv;
                                acc[k][1] += b.y * rv;
                                acc[k][2] += b.z * rv;
                                acc[k][3] += b.w * rv;
                            }
                        }
                    } else if (!ok && lane == 0) {
                        abort_cta = 1;
                        atomicCAS(err, 0, kErrDeviceTimeout);
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[st]);
                }
                if (!last) {
                    float *gp = p.gpart + (size_t)blockIdx.x * nc;
#pragma unroll
                    for (int k = 0; k < kPersistStrips; ++k) {
                        const int c = 4 * t + 512 * k;
                        if (c < nc)
                            *reinterpret_cast<float4 *>(gp + c) = make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
                    }
                }
            }
            if (resid && lane == 0) lred[warp] = l2;
            bar_compute();
            if (last) {
                if (tid == 0) p.lpart[blockIdx.x] = ((lred[0] + lred[1]) + lred[2]) + lred[3];
                break;
            }
            // partial gradients of every CTA are written: sum them per column
            if (tid == 0) {
                if (!abort_cta && !grid_barrier(gbar, nbar, err, kDrainLimit)) {
                    abort_cta = 1;
                    atomicCAS(err, 0, kErrDeviceTimeout);
                }
                stop_cta = abort_cta;
            }
            ++nbar;
            bar_compute();
            if (stop_cta) break;
            const int cpc = (nc + gridDim.x - 1) / gridDim.x;
            const int c0 = blockIdx.x * cpc, c1 = min(nc, c0 + cpc);
            for (int cb = c0; cb < c1; cb += 32) {
                const int c = cb + lane;
                float g = 0.f;
                if (c < c1)
                    for (int b = warp; b < (int)gridDim.x; b += 8)
                        if (DODE_IN_BOUNDS((long long)b * nc + c, (long long)gridDim.x * nc, err, kSiteDensePart))
                            g += __ldcg(p.gpart + (size_t)b * nc + c);
                gred[warp][lane] = g;
                bar_compute();
                if (warp == 0 && c < c1) {
                    float gs = 0.f;
                    for (int w = 0; w < 8; ++w) gs += gred[w][lane];
                    const float Gv = __ldcg(p.G + c) + gs * gs;
                    p.G[c] = Gv;
                    p.x[c] = fmaxf(__ldcg(p.x + c) - p.eta * gs / (sqrtf(Gv) + p.eps), 0.f);
                }
                bar_compute();
            }
            // every CTA's columns are stepped: reload x
            if (tid == 0) {
                if (!abort_cta && !grid_barrier(gbar, nbar, err, kDrainLimit)) {
                    abort_cta = 1;
                    atomicCAS(err, 0, kErrDeviceTimeout);
                }
                stop_cta = abort_cta;
            }
            ++nbar;
            bar_compute();
            if (stop_cta) break;
            {
                // all of x in one round trip: n_cols <= 8192, 16-byte loads
                const int n4 = nc >> 2;
                float4 xv[kReloadVecs];
#pragma unroll
                for (int u = 0; u < kReloadVecs; ++u) {
                    const int i = tid + 256 * u;
                    xv[u] = i < n4 ? __ldcg(reinterpret_cast<const float4 *>(p.x) + i) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < kReloadVecs; ++u) {
                    const int i = tid + 256 * u;
                    if (i < n4) reinterpret_cast<float4 *>(xs)[i] = xv[u];
                }
            }
            bar_compute();
        }
    }
    __syncthreads();
}

cudaError_t dense_persist(const DenseParams &p, int iters, int grid, int S, size_t smem, int *err, unsigned int *gbar,
                          cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(gbar, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    DenseParams pp = p;
    void *args[] = {&pp, &iters, &S, &err, &gbar};
    return cudaLaunchCooperativeKernel((const void *)k_dense_persist, dim3(grid), dim3(kPersistThreads), args, smem, s);
}

cudaError_t dense_persist_set_smem(size_t bytes) {
    return cudaFuncSetAttribute(k_dense_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t dense_iteration(const DenseParams &p, bool step, cudaStream_t s) {
    k_dense_resid<<<p.grid_r, 256, (size_t)p.nc * p.m * sizeof(float), s>>>(p.B, p.x, p.y, p.nr, p.nc, p.m, p.vec,
                                                                              p.r, p.lpart);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !step) return e;
    const dim3 gg((p.nc + 1023) / 1024, p.grid_g);
    k_dense_grad<<<gg, 256, (size_t)p.rows_per_cta * p.m * sizeof(float), s>>>(p.B, p.r, p.nr, p.nc, p.m, p.vec,
                                                                                p.rows_per_cta, p.gpart);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_dense_step<<<(p.nc * p.m + 31) / 32, 256, 0, s>>>(p.gpart, p.grid_g, p.nc, p.m, p.eta, p.eps, p.x, p.G);
    return cudaGetLastError();
}

cudaError_t dense_loss(const DenseParams &p, double *loss, cudaStream_t s) {
    k_dense_loss<<<1, 32, 0, s>>>(p.lpart, p.grid_r, p.m, loss);
    return cudaGetLastError();
}

cudaError_t dense_set_smem(size_t resid_bytes, size_t grad_bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_dense_resid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)resid_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_dense_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_bytes);
}

}  // namespace dode
