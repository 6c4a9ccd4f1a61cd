// quality.cu -- stability of the DAR across days (Sec. 5, "Empirical test on
// the DAR matrix"): the mean DAR over the loaded days and each day's l2
// distance from it.  The DAR of Eq. (dar) is indexed by route position l
// (route k, link position j), departure interval h1 and arrival interval h2;
// since h1 <= h2 <= h1 + W - 1 for every entry (W = the days' largest
// trajectory offset + 2), the mean is held densely as
// rbar[(l * N + h1) * W + (h2 - h1)].  Shares are computed in FP32 as in the
// fused kernel, sums and distances in FP64; every sum has a fixed order, so
// results are reproducible.
#include "dode_internal.cuh"

namespace dode {

// Visit the DAR entries of one route and day for the lane's departure
// interval: fn(l, h2, rho) for every window cell before the end of the day
// (a zero-length window puts its whole share in its interval).
template <class Fn>
__device__ __forceinline__ void route_dar(const DarParams &p, int day, int k, int b0, Fn fn) {
    const int lane = threadIdx.x & 31;
    const int b = b0 + lane;
    const int bb = min(b, p.N);
    const bool vw = lane < kTileW && b < p.N;
    const int ipt = p.div.ipt;
    const int l0 = __ldg(&p.rptr[k]), beta = __ldg(&p.rptr[k + 1]) - l0;
    const int32_t *tk = p.ticks + (size_t)day * p.A * p.Np;
    const int64_t toff = __ldg(&p.tab_off[day]);
    const int32_t *trow = toff >= 0 ? p.traj_tab + toff + (size_t)(l0 + k) * (p.N + 1) + bb : nullptr;
    int T = ipt * bb;
    for (int j = 0; j < beta; ++j) {
        const int hi = __shfl_down_sync(0xffffffffu, T, 1);
        const int h0 = interval_of(T, p.div);
        if (vw && h0 < p.N) {
            if (hi == T) {
                fn(l0 + j, h0, 1.f);
            } else {
                const float w = (float)(hi - T);
                for (int h2 = h0; h2 < p.N && h2 * ipt < hi; ++h2) {
                    const int lo = max(T, h2 * ipt), up = min(hi, h2 * ipt + ipt);
                    fn(l0 + j, h2, __fdiv_rn((float)(up - lo), w));
                }
            }
        }
        if (trow) {
            T = __ldg(&trow[(size_t)(j + 1) * (p.N + 1)]);
        } else {
            const int a = __ldg(&p.rlinks[l0 + j]);
            T += __ldg(&tk[(size_t)a * p.Np + min(h0, p.N - 1)]);
        }
    }
}

// Mean DAR: one warp per (route, tile of 31 departures); every lane owns its
// departure's entries and sums them over the days in day order.
__global__ void __launch_bounds__(256) k_dar_mean(const DarParams p) {
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int ntiles = (p.N + kTileW - 1) / kTileW;
    if (gw >= (long long)p.P * ntiles) return;
    const int k = (int)(gw / ntiles), b0 = (int)(gw % ntiles) * kTileW;
    const int h1 = b0 + (threadIdx.x & 31);
    for (int d = 0; d < p.n_days; ++d)
        route_dar(p, d, k, b0, [&](int l, int h2, float rho) {
            p.rbar[((size_t)l * p.N + h1) * p.W + (h2 - h1)] += (double)rho;
        });
    const double inv = 1.0 / (double)p.n_days;
    const int l0 = __ldg(&p.rptr[k]), beta = __ldg(&p.rptr[k + 1]) - l0;
    if ((threadIdx.x & 31) < kTileW && h1 < p.N)
        for (int j = 0; j < beta; ++j)
            for (int w = 0; w < p.W; ++w) p.rbar[((size_t)(l0 + j) * p.N + h1) * p.W + w] *= inv;
}

__device__ double block_sum_fixed(double v, double *red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    __syncthreads();
    return t;
}

// ||rbar||^2 in fixed-order partial sums (one per block), then one block adds them.
__global__ void __launch_bounds__(256) k_sq_partial(const double *__restrict__ x, size_t n, double *__restrict__ part) {
    __shared__ double red[8];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        s += x[i] * x[i];
    s = block_sum_fixed(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_sum_partials(const double *__restrict__ part, int n, double *__restrict__ out) {
    __shared__ double red[8];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = block_sum_fixed(s, red);
    if (threadIdx.x == 0) *out = s;
}

// dist_d^2 = ||rbar||^2 + sum over day d's entries of (rho^2 - 2 rho rbar):
// one block per day, its warps over (route, tile) pairs.
__global__ void __launch_bounds__(256) k_dar_dist(const DarParams p, const double *__restrict__ rbar_sq,
                                                  double *__restrict__ dist) {
    __shared__ double red[8];
    const int d = blockIdx.x;
    const int ntiles = (p.N + kTileW - 1) / kTileW;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double s = 0.0;
    for (int t = warp; t < p.P * ntiles; t += nw) {
        const int k = t / ntiles, b0 = (t % ntiles) * kTileW;
        const int h1 = b0 + (threadIdx.x & 31);
        route_dar(p, d, k, b0, [&](int l, int h2, float rho) {
            const double r = (double)rho;
            s += r * r - 2.0 * r * p.rbar[((size_t)l * p.N + h1) * p.W + (h2 - h1)];
        });
    }
    s = block_sum_fixed(s, red);
    if (threadIdx.x == 0) dist[d] = sqrt(fmax(*rbar_sq + s, 0.0));
}

cudaError_t launch_dar_distance(const DarParams &p, double *part, int n_part, double *rbar_sq, double *dist,
                                cudaStream_t s) {
    const int ntiles = (p.N + kTileW - 1) / kTileW;
    const long long warps = (long long)p.P * ntiles;
    cudaError_t e = cudaMemsetAsync(p.rbar, 0, (size_t)p.L * p.N * p.W * sizeof(double), s);
    if (e != cudaSuccess) return e;
    k_dar_mean<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_sq_partial<<<n_part, 256, 0, s>>>(p.rbar, (size_t)p.L * p.N * p.W, part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_sum_partials<<<1, 256, 0, s>>>(part, n_part, rbar_sq);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_dar_dist<<<p.n_days, 256, 0, s>>>(p, rbar_sq, dist);
    return cudaGetLastError();
}

// Cross-day totals of the per-day results (Sec. 2.7: the multi-year objective
// is the sum of the independent days' objectives): FP64 sums in day order, by
// one thread, so that the total does not depend on any launch shape.
__global__ void k_day_totals(const double *__restrict__ loss, const double *__restrict__ dth, int D,
                             double *__restrict__ out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double l = 0.0, t = 0.0;
    for (int d = 0; d < D; ++d) {
        l += loss[d];
        if (dth) t += dth[d];
    }
    out[0] = l;
    out[1] = t;
}

cudaError_t launch_day_totals(const double *loss, const double *dth, int D, double *out, cudaStream_t s) {
    k_day_totals<<<1, 32, 0, s>>>(loss, dth, D, out);
    return cudaGetLastError();
}

}  // namespace dode
