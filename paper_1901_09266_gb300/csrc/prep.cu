// prep.cu -- once-per-load kernels: link travel-time ticks (Sec. 2.4), exact
// leading-vehicle trajectories with FIFO repair and route times (Eq. (cost),
// Sec. 2.2), and the layout conversions between the ABI's time-major arrays and
// the internal time-innermost ones.
#include "dode_internal.cuh"

namespace dode {

// ---------------------------------------------------------------------------
// Tick table: c[d][a][h] = max(1, rint(fl32(fl32(len_a * 3600 tps) / v[d][h][a]))).
// IEEE FP32 multiply and divide with round-to-nearest-even and an IEEE
// round-half-even conversion, so every implementation gets the same integers.
// 32 x 32 tiles are transposed through shared memory: reads run along links,
// writes along intervals.
// ---------------------------------------------------------------------------
// Link travel time in ticks at speed v (Eq. (cost)): rint(fl32(fl32(len * 3600 tps) / v)), at least 1;
// 0 marks an invalid speed or an overflow.
__device__ __forceinline__ int32_t tick_of(float len, float scale, float v) {
    if (!(v > 0.f) || !isfinite(v)) return 0;
    const float t = __fdiv_rn(__fmul_rn(len, scale), v);
    if (!(t <= 16777216.f)) return 0;
    return max(__float2int_rn(t), 1);
}

__global__ void k_ticks(const float *__restrict__ speeds, const float *__restrict__ len, int N, int Np,
                        int A, float scale, int32_t *__restrict__ ticks, uint16_t *__restrict__ ticks16, int *maxtick,
                        int *err) {
    __shared__ int32_t tile[32][33];
    const int d = blockIdx.z;
    const int a0 = blockIdx.x * 32, h0 = blockIdx.y * 32;
    const float *sp = speeds + (size_t)d * N * A;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int h = h0 + i, a = a0 + threadIdx.x;
        int32_t c = 1;
        if (h < N && a < A) {
            const float v = sp[(size_t)h * A + a];
            if (!(v > 0.f) || !isfinite(v)) {
                set_error(err, kErrBadSpeed, ((long long)d * N + h) * A + a);
            } else {
                const float num = __fmul_rn(len[a], scale);
                const float t = __fdiv_rn(num, v);
                if (!(t <= 16777216.f)) {
                    set_error(err, kErrTickOverflow, ((long long)d * N + h) * A + a);
                } else {
                    c = max(__float2int_rn(t), 1);
                }
            }
        }
        tile[i][threadIdx.x] = c;
    }
    __syncthreads();
    int32_t *tk = ticks + (size_t)d * A * Np;
    uint16_t *tk16 = ticks16 + (size_t)d * A * Np;
    int mx = 0;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int a = a0 + i, h = h0 + threadIdx.x;
        if (a < A && h < Np) {
            const int32_t c = h < N ? tile[threadIdx.x][i] : 1;
            tk[(size_t)a * Np + h] = c;
            mx = max(mx, c);
            // 16-bit copy for the fused kernel's tick windows: entries past the end
            // of the day repeat the last interval (the link entry rule clamps to
            // it); values above 16 bits saturate and the kernel does not use it
            const int32_t c16 = h < N ? c : max(tick_of(len[a], scale, sp[(size_t)(N - 1) * A + a]), 1);
            tk16[(size_t)a * Np + h] = (uint16_t)min(c16, 65535);
        }
    }
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, off));
    if (threadIdx.x == 0) atomicMax(maxtick, mx);
}

cudaError_t launch_ticks(const float *speeds, const float *len, int D, int N, int Np, int A, int tps,
                         int32_t *ticks, uint16_t *ticks16, int *maxtick, int *err, cudaStream_t s) {
    dim3 block(32, 8), grid((A + 31) / 32, (Np + 31) / 32, D);
    k_ticks<<<grid, block, 0, s>>>(speeds, len, N, Np, A, (float)(tps * 3600), ticks, ticks16, maxtick, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exact trajectories, one warp per (day, route).  Lanes take boundaries
// b = 32 c + lane in chunks c; at link position j the raw entry time of link
// j+1 is T_j(b) + c_{a_j}(T_j(b)) and the FIFO rule makes T_{j+1}(b) the running
// maximum of the raw values over all boundaries <= b: a warp max-scan plus the
// carry of the previous chunk (kept per link position in shared memory).
// Outputs: route time C[k][b] in minutes, the largest interval offset of any
// trajectory point, the number of repairs, and (pass 2, repaired days only) the
// full trajectory table T[(rptr[k] + k + j)][b], b = 0..N.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_prepare(const PrepParams p) {
    __shared__ int32_t s_carry[8][kMaxRouteLinks + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (gw >= (long long)p.n_days * p.P) return;
    const int day = (int)(gw / p.P), k = (int)(gw % p.P);
    const int l0 = p.rptr[k], l1 = p.rptr[k + 1], beta = l1 - l0;
    const int32_t *tk = p.ticks + (size_t)day * p.A * p.Np;
    // coupled days: a link entered after midnight takes the next day's link time
    const int32_t *tk_next = (p.coupled && day + 1 < p.n_days) ? tk + (size_t)p.A * p.Np : nullptr;
    const int ipt = p.div.ipt;
    int32_t *tab = nullptr;
    if (p.tab_off && p.tab_off[day] >= 0) tab = p.traj_tab + p.tab_off[day] + (size_t)(l0 + k) * (p.N + 1);
    int32_t *carry = s_carry[warp];
    for (int j = lane; j <= beta; j += 32) carry[j] = INT_MIN;
    __syncwarp();
    int maxoff = 0;
    unsigned long long reps = 0;
    const float inv_min = 1.f / (float)(60 * p.tps);
    for (int b0 = 0; b0 <= p.N; b0 += 32) {
        const int b = b0 + lane;
        const bool valid = b <= p.N;
        int T = valid ? ipt * b : INT_MAX;
        if (valid && tab) tab[b] = T;
        for (int j = 0; j < beta; ++j) {
            const int a = p.rlinks[l0 + j];
            int raw = INT_MAX;
            if (valid) {
                const int h = interval_of(T, p.div);
                if (h < p.N)
                    raw = T + tk[(size_t)a * p.Np + h];
                else if (tk_next)
                    raw = T + tk_next[(size_t)a * p.Np + min(h - p.N, p.N - 1)];
                else
                    raw = T + tk[(size_t)a * p.Np + p.N - 1];
            }
            // inclusive running max over lanes, seeded with the previous chunk
            int v = raw;
            for (int off = 1; off < 32; off <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, off);
                if (lane >= off) v = max(v, u);
            }
            const int prev_excl = max(__shfl_up_sync(0xffffffffu, v, 1), carry[j + 1]);
            const int before = lane == 0 ? carry[j + 1] : prev_excl;
            v = max(v, carry[j + 1]);
            if (valid && raw < before) ++reps;
            __syncwarp();
            if (lane == 31) carry[j + 1] = v;   // lane 31 holds the chunk maximum (INT_MAX past the end)
            __syncwarp();
            T = valid ? v : INT_MAX;
            if (valid) {
                maxoff = max(maxoff, interval_of(T, p.div) - b);
                if (tab) tab[(size_t)(j + 1) * (p.N + 1) + b] = T;
            }
        }
        if (valid && b < p.N) p.C[((size_t)day * p.P + k) * p.Np + b] = (float)(T - ipt * b) * inv_min;
    }
    for (int off = 16; off > 0; off >>= 1) {
        maxoff = max(maxoff, __shfl_down_sync(0xffffffffu, maxoff, off));
        reps += __shfl_down_sync(0xffffffffu, reps, off);
    }
    if (lane == 0) {
        atomicMax(&p.maxoff[day], maxoff);
        if (reps) atomicAdd(&p.repairs[day], reps);
    }
}

cudaError_t launch_prepare(const PrepParams &p, cudaStream_t s) {
    const long long warps = (long long)p.n_days * p.P;
    const int block = 256;
    const long long grid = (warps + 7) / 8;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_prepare<<<(unsigned)grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// [D][N][M] (time-major) <-> [D][M][Np] (time innermost), 32 x 32 tiles.
// ---------------------------------------------------------------------------
__global__ void k_transpose_in(const float *__restrict__ src, float *__restrict__ dst, int N, int Np, int M) {
    __shared__ float tile[32][33];
    const int d = blockIdx.z, m0 = blockIdx.x * 32, h0 = blockIdx.y * 32;
    const float *s = src + (size_t)d * N * M;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int h = h0 + i, m = m0 + threadIdx.x;
        tile[i][threadIdx.x] = (h < N && m < M) ? s[(size_t)h * M + m] : 0.f;
    }
    __syncthreads();
    float *t = dst + (size_t)d * M * Np;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int m = m0 + i, h = h0 + threadIdx.x;
        if (m < M && h < Np) t[(size_t)m * Np + h] = tile[threadIdx.x][i];
    }
}

__global__ void k_transpose_out(const float *__restrict__ src, float *__restrict__ dst, int N, int Np, int M,
                                float scale) {
    __shared__ float tile[32][33];
    const int d = blockIdx.z, m0 = blockIdx.y * 32, h0 = blockIdx.x * 32;
    const float *s = src + (size_t)d * M * Np;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int m = m0 + i, h = h0 + threadIdx.x;
        tile[i][threadIdx.x] = (m < M && h < N) ? s[(size_t)m * Np + h] : 0.f;
    }
    __syncthreads();
    float *t = dst + (size_t)d * N * M;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int h = h0 + i, m = m0 + threadIdx.x;
        if (h < N && m < M) t[(size_t)h * M + m] = scale * tile[threadIdx.x][i];
    }
}

cudaError_t launch_transpose_in(const float *src, float *dst, int D, int N, int Np, int M, cudaStream_t s) {
    dim3 block(32, 8), grid((M + 31) / 32, (Np + 31) / 32, D);
    k_transpose_in<<<grid, block, 0, s>>>(src, dst, N, Np, M);
    return cudaGetLastError();
}

cudaError_t launch_transpose_out(const float *src, float *dst, int D, int N, int Np, int M, float scale,
                                 cudaStream_t s) {
    dim3 block(32, 8), grid((N + 31) / 32, (M + 31) / 32, D);
    k_transpose_out<<<grid, block, 0, s>>>(src, dst, N, Np, M, scale);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// u8 mask [D][N][O] -> bits [D][O][Nw] and per-day active-column bits [D][Ow].
// ---------------------------------------------------------------------------
__global__ void k_pack_mask(const uint8_t *__restrict__ mask, uint32_t *__restrict__ bits,
                            uint32_t *__restrict__ colact, int N, int Nw, int O, int Ow) {
    const int d = blockIdx.y;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    bool any = false;
    if (o < O) {
        const uint8_t *m = mask ? mask + (size_t)d * N * O : nullptr;
        for (int w = 0; w < Nw; ++w) {
            uint32_t word = 0;
            for (int i = 0; i < 32; ++i) {
                const int h = w * 32 + i;
                if (h < N && (m == nullptr || m[(size_t)h * O + o])) word |= 1u << i;
            }
            bits[((size_t)d * O + o) * Nw + w] = word;
            any |= word != 0;
        }
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, any);
    if ((threadIdx.x & 31) == 0) {
        const int wo = o >> 5;
        if (wo < Ow) colact[(size_t)d * Ow + wo] = bal;
    }
}

cudaError_t launch_pack_mask(const uint8_t *mask, uint32_t *bits, uint32_t *colact, int D, int N, int Nw,
                             int O, int Ow, cudaStream_t s) {
    dim3 block(128), grid((O + 127) / 128, D);
    k_pack_mask<<<grid, block, 0, s>>>(mask, bits, colact, N, Nw, O, Ow);
    return cudaGetLastError();
}

__global__ void k_to_bf16(const float *__restrict__ src, __nv_bfloat16 *__restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

cudaError_t launch_to_bf16(const float *src, __nv_bfloat16 *dst, size_t n, cudaStream_t s) {
    const int block = 256;
    size_t g = (n + block - 1) / block;
    if (g > 65536) g = 65536;
    if (g == 0) return cudaSuccess;
    k_to_bf16<<<(unsigned)g, block, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

// Route choice portions pt[d][k][h] = logit over the OD's routes of -theta C
// (Eq. (logit), (rt)), for every day, route and departure interval.
__global__ void k_route_choice(const float *__restrict__ C, const int32_t *__restrict__ rod,
                               const int32_t *__restrict__ od_ptr, const int32_t *__restrict__ od_routes, float theta,
                               int D, int P, int N, int Np, float *__restrict__ pt) {
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= (long long)D * P * Np) return;
    const int h = (int)(gid % Np);
    const long long dk = gid / Np;
    const int k = (int)(dk % P), d = (int)(dk / P);
    if (h >= N) {
        pt[gid] = 0.f;
        return;
    }
    const float *Cd = C + (size_t)d * P * Np;
    const int od = rod[k];
    float m = -INFINITY;
    for (int i = od_ptr[od]; i < od_ptr[od + 1]; ++i) m = fmaxf(m, -theta * Cd[(size_t)od_routes[i] * Np + h]);
    float den = 0.f;
    for (int i = od_ptr[od]; i < od_ptr[od + 1]; ++i) den += expf(-theta * Cd[(size_t)od_routes[i] * Np + h] - m);
    pt[gid] = expf(-theta * Cd[(size_t)k * Np + h] - m) / den;
}

cudaError_t launch_route_choice(const float *C, const int32_t *rod, const int32_t *od_ptr, const int32_t *od_routes,
                                float theta, int D, int P, int N, int Np, float *pt, cudaStream_t s) {
    const long long n = (long long)D * P * Np;
    k_route_choice<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(C, rod, od_ptr, od_routes, theta, D, P, N, Np, pt);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Goodness of fit (Step 6 of the framework, Sec. 4): per-day total sum of
// squares of the observed counts about their masked mean, two passes in FP64
// (block per day), and R^2 = 1 - SS_res / SS_tot from the day's masked loss.
// ---------------------------------------------------------------------------
__device__ double block_sum_d(double v, double *red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];      // same order in every thread
    return t;
}

__global__ void __launch_bounds__(256) k_sstot(const float *__restrict__ counts, const uint32_t *__restrict__ mask,
                                               int O, int N, int Np, int Nw, double *__restrict__ sstot) {
    __shared__ double red[8];
    const int d = blockIdx.x;
    const float *c = counts + (size_t)d * O * Np;
    const uint32_t *m = mask + (size_t)d * O * Nw;
    double s = 0.0, n = 0.0;
    for (int i = threadIdx.x; i < O * N; i += blockDim.x) {
        const int o = i / N, h = i - o * N;
        if ((m[(size_t)o * Nw + (h >> 5)] >> (h & 31)) & 1u) {
            s += c[(size_t)o * Np + h];
            n += 1.0;
        }
    }
    s = block_sum_d(s, red);
    n = block_sum_d(n, red);
    const double mean = n > 0.0 ? s / n : 0.0;
    double ss = 0.0;
    for (int i = threadIdx.x; i < O * N; i += blockDim.x) {
        const int o = i / N, h = i - o * N;
        if ((m[(size_t)o * Nw + (h >> 5)] >> (h & 31)) & 1u) {
            const double e = (double)c[(size_t)o * Np + h] - mean;
            ss += e * e;
        }
    }
    ss = block_sum_d(ss, red);
    if (threadIdx.x == 0) sstot[d] = ss;
}

__global__ void k_r2(const double *__restrict__ loss, const double *__restrict__ sstot, int D, double *__restrict__ r2) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d < D) r2[d] = sstot[d] > 0.0 ? 1.0 - loss[d] / sstot[d] : __longlong_as_double(0x7ff8000000000000ll);
}

cudaError_t launch_r2(const float *counts, const uint32_t *mask, int D, int O, int N, int Np, int Nw,
                      const double *loss, double *sstot, double *r2, cudaStream_t s) {
    k_sstot<<<D, 256, 0, s>>>(counts, mask, O, N, Np, Nw, sstot);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_r2<<<(D + 127) / 128, 128, 0, s>>>(loss, sstot, D, r2);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pattern-level route choice (Eq. (logit) takes the mean travel time of each
// path over the days of a traffic pattern): Ceff[d] = mean over the days of
// d's group of C[d'], FP64 sums in ascending day order.  One thread per
// (group, route, interval).
// ---------------------------------------------------------------------------
__global__ void k_pattern_times(const float *__restrict__ C, int n_groups, const int32_t *__restrict__ gptr,
                                const int32_t *__restrict__ gday, int P, int N, int Np, float *__restrict__ Ceff) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)n_groups * P * N) return;
    const int g = (int)(i / ((long long)P * N));
    const int rest = (int)(i - (long long)g * P * N);
    const int k = rest / N, h = rest - k * N;
    const int d0 = gptr[g], d1 = gptr[g + 1];
    double s = 0.0;
    for (int x = d0; x < d1; ++x) s += (double)C[((size_t)gday[x] * P + k) * Np + h];
    const float m = (float)(s / (double)(d1 - d0));
    for (int x = d0; x < d1; ++x) Ceff[((size_t)gday[x] * P + k) * Np + h] = m;
}

cudaError_t launch_pattern_times(const float *C, int n_groups, const int32_t *gptr, const int32_t *gday, int P, int N,
                                 int Np, float *Ceff, cudaStream_t s) {
    const long long n = (long long)n_groups * P * N;
    if (n == 0) return cudaSuccess;
    k_pattern_times<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(C, n_groups, gptr, gday, P, N, Np, Ceff);
    return cudaGetLastError();
}

}  // namespace dode
