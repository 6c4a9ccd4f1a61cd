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
// One pass over B per iteration (one right-hand side, n_cols % 4 == 0 and
// n_cols <= 8192): a persistent CTA per SM streams blocks of RB rows of B into
// shared memory with bulk asynchronous copies (TMA, two stages completed on
// mbarriers), forms the block's residuals r = B x - y from shared memory, and
// adds r B to a partial gradient held in registers (each thread owns 4-column
// strips c = 4 tid + 1024 k).  Partials go to gpart[cta], reduced by
// k_dense_step.  Every mbarrier wait is bounded: on expiry the kernel records
// an error, waits (bounded) for its copies in flight and returns.
// ---------------------------------------------------------------------------
constexpr int kFusedStrips = 8;                      // n_cols <= 8 * 1024

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < (1ll << 26); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Thread 0: expect `bytes` on bar, then copy rows [r0, r0 + n) of B into dst.
__device__ __forceinline__ void issue_rows(const float *B, int nc, int r0, int n, float *dst, uint64_t *bar) {
    const uint32_t bytes = (uint32_t)n * (uint32_t)nc * 4u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    for (int i = 0; i < n; ++i)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(dst + (size_t)i * nc)),
            "l"(B + (size_t)(r0 + i) * nc), "r"((uint32_t)nc * 4u), "r"(smem_u32(bar))
            : "memory");
}

__global__ void __launch_bounds__(256, 1) k_dense_fused(const DenseParams p, int RB, int *err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float rblk[8];
    __shared__ double lred[8];
    const int nc = p.nc, nr = p.nr;
    float *xs = reinterpret_cast<float *>(smem_raw);
    const size_t xbytes = ((size_t)nc * 4 + 127) & ~(size_t)127;
    float *buf[2] = {reinterpret_cast<float *>(smem_raw + xbytes),
                     reinterpret_cast<float *>(smem_raw + xbytes + (size_t)RB * nc * 4)};
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < nc; i += blockDim.x) xs[i] = p.x[i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int nblk = (nr + RB - 1) / RB;
    float acc[kFusedStrips][4];
#pragma unroll
    for (int k = 0; k < kFusedStrips; ++k)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[k][u] = 0.f;
    double l2 = 0.0;
    int blk = blockIdx.x, it = 0;
    if (tid == 0 && blk < nblk) issue_rows(p.B, nc, blk * RB, min(RB, nr - blk * RB), buf[0], &bar[0]);
    bool ok = true;
    for (; blk < nblk; blk += gridDim.x, ++it) {
        const int st = it & 1;
        const int nxt = blk + gridDim.x;
        if (tid == 0 && nxt < nblk) issue_rows(p.B, nc, nxt * RB, min(RB, nr - nxt * RB), buf[st ^ 1], &bar[st ^ 1]);
        const bool landed = mbar_wait(&bar[st], (uint32_t)((it >> 1) & 1));
        if (!__syncthreads_and(landed)) {                 // the same decision in every thread
            ok = false;
            break;
        }
        const int r0 = blk * RB, nrow = min(RB, nr - r0);
        const float *rows = buf[st];
        // residuals of the block: warp w takes row w
        if (warp < nrow) {
            const float *row = rows + (size_t)warp * nc;
            float v = 0.f;
            for (int c = 4 * lane; c < nc; c += 128) {
                const float4 b = *reinterpret_cast<const float4 *>(row + c);
                const float4 xv = *reinterpret_cast<const float4 *>(xs + c);
                v += b.x * xv.x + b.y * xv.y + b.z * xv.z + b.w * xv.w;
            }
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            const float ri = v - p.y[r0 + warp];
            if (lane == 0) {
                rblk[warp] = ri;
                p.r[r0 + warp] = ri;
            }
            l2 += (double)ri * (double)ri;
        }
        __syncthreads();
        // g += r B over the block's rows
#pragma unroll
        for (int k = 0; k < kFusedStrips; ++k) {
            const int c = 4 * tid + 1024 * k;
            if (c < nc)
                for (int i = 0; i < nrow; ++i) {
                    const float4 b = *reinterpret_cast<const float4 *>(rows + (size_t)i * nc + c);
                    const float rv = rblk[i];
                    acc[k][0] += b.x * rv;
                    acc[k][1] += b.y * rv;
                    acc[k][2] += b.z * rv;
                    acc[k][3] += b.w * rv;
                }
        }
        __syncthreads();                                  // stage st free for the copy after next
    }
    if (!ok) {
        if (tid == 0) {
            atomicCAS(err, 0, kErrDeviceTimeout);
            // the copies in flight target this CTA's shared memory: let them land
            const int st = it & 1;
            mbar_wait(&bar[st], (uint32_t)((it >> 1) & 1));
            if (blk + (int)gridDim.x < nblk) mbar_wait(&bar[st ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
        }
        return;
    }
    float *gp = p.gpart + (size_t)blockIdx.x * nc;
#pragma unroll
    for (int k = 0; k < kFusedStrips; ++k) {
        const int c = 4 * tid + 1024 * k;
        if (c < nc) *reinterpret_cast<float4 *>(gp + c) = make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
    }
    if (lane == 0) lred[warp] = l2;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += lred[w];
        p.lpart[blockIdx.x] = t;
    }
}

cudaError_t dense_fused_iteration(const DenseParams &p, int grid, int RB, size_t smem, int *err, cudaStream_t s) {
    k_dense_fused<<<grid, 256, smem, s>>>(p, RB, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_dense_step<<<(p.nc + 31) / 32, 256, 0, s>>>(p.gpart, grid, p.nc, 1, p.eta, p.eps, p.x, p.G);
    return cudaGetLastError();
}

cudaError_t dense_fused_set_smem(size_t bytes) {
    return cudaFuncSetAttribute(k_dense_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
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
