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
//   k_dense_step   sums the partials in CTA order, then G += g^2,
//                  x = max(x - eta g / (sqrt(G) + eps), 0)
// All sums have a fixed order: results do not depend on timing.
#include "dode_internal.cuh"

namespace dode {

constexpr int kDenseMaxRhs = 8;

// r[i][j] = sum_c B[i][c] x[c][j] - y[i][j]; lpart[cta][j] = sum over the CTA's rows of r^2.
__global__ void __launch_bounds__(256) k_dense_resid(const float *__restrict__ B, const float *__restrict__ x,
                                                     const float *__restrict__ y, int nr, int nc, int m,
                                                     float *__restrict__ r, double *__restrict__ lpart) {
    extern __shared__ __align__(16) float xs[];      // [nc][m]
    __shared__ double red[8][kDenseMaxRhs];
    for (int i = threadIdx.x; i < nc * m; i += blockDim.x) xs[i] = x[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double l2[kDenseMaxRhs];
#pragma unroll
    for (int j = 0; j < kDenseMaxRhs; ++j) l2[j] = 0.0;
    const bool vec = (nc & 3) == 0;                     // rows 16-byte aligned
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
                                                    int nc, int m, int rows_per_cta, float *__restrict__ gpart) {
    extern __shared__ __align__(16) float rs[];      // [rows_per_cta][m]
    const int r0 = blockIdx.y * rows_per_cta, r1 = min(nr, r0 + rows_per_cta);
    for (int i = threadIdx.x; i < (r1 - r0) * m; i += blockDim.x) rs[i] = r[(size_t)r0 * m + i];
    __syncthreads();
    const int c = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= nc) return;
    float *gp = gpart + (size_t)blockIdx.y * nc * m;
    const bool vec = (nc & 3) == 0;
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

// g = sum of the partials in CTA order; Adagrad step and projection.
__global__ void __launch_bounds__(256) k_dense_step(const float *__restrict__ gpart, int n_part, int nc, int m,
                                                    float eta, float eps, float *__restrict__ x, float *__restrict__ G) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nc * m) return;
    float g = 0.f;
    for (int b = 0; b < n_part; ++b) g += gpart[(size_t)b * nc * m + e];
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

cudaError_t dense_iteration(const DenseParams &p, bool step, cudaStream_t s) {
    k_dense_resid<<<p.grid_r, 256, (size_t)p.nc * p.m * sizeof(float), s>>>(p.B, p.x, p.y, p.nr, p.nc, p.m, p.r,
                                                                              p.lpart);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !step) return e;
    const dim3 gg((p.nc + 1023) / 1024, p.grid_g);
    k_dense_grad<<<gg, 256, (size_t)p.rows_per_cta * p.m * sizeof(float), s>>>(p.B, p.r, p.nr, p.nc, p.m,
                                                                                p.rows_per_cta, p.gpart);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_dense_step<<<(p.nc * p.m + 255) / 256, 256, 0, s>>>(p.gpart, p.grid_g, p.nc, p.m, p.eta, p.eps, p.x, p.G);
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
