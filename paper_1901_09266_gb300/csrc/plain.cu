// plain.cu -- the plain FP32 form: the straightforward GPU rendering of the
// paper's implementation (Sec. 3.1-3.3), kept as the baseline the fused kernel
// is measured against.  The DAR (Eq. (dar)) is built once and materialised in
// HBM as one 16-byte record per (observed route link, departure interval); each
// SPGD epoch is three separate kernels: forward scatter (B q, atomics), masked
// residual + loss, and adjoint gather + Adagrad step + projection.
//
// Record layout (int4): x = first arrival interval h2 | (cell count << 16),
// y, z, w = the DAR fractions of up to three consecutive arrival intervals.
// A window that spans more than three intervals is reported as
// DODE_ERR_UNSUPPORTED (the fused form has no such limit).
#include "dode_internal.cuh"

namespace dode {

// One thread per (day, route, departure interval): walks boundaries b and b+1
// together and emits the record of every listed link position of the route.
__global__ void k_plain_build(const PlainParams p) {
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= (long long)p.n_days * p.P * p.N) return;
    const int b = (int)(gid % p.N);
    const long long dk = gid / p.N;
    const int k = (int)(dk % p.P), day = (int)(dk / p.P);
    const int l0 = p.rptr[k], l1 = p.rptr[k + 1];
    const int32_t *tk = p.ticks + (size_t)day * p.A * p.Np;
    const int64_t toff = p.tab_off[day];
    const int32_t *tab = toff >= 0 ? p.traj_tab + toff + (size_t)(l0 + k) * (p.N + 1) : nullptr;
    const int ipt = p.div.ipt;
    int lo = ipt * b, hi = ipt * (b + 1);
    int pi = p.route_pair_ptr[k];
    const int pe = p.route_pair_ptr[k + 1];
    for (int j = 0; j < l1 - l0 && pi < pe; ++j) {
        if (p.pair_j[pi] == j) {
            int4 rec = make_int4(0, 0, 0, 0);
            const int h0 = interval_of(lo, p.div);
            if (h0 < p.N) {
                float f[3] = {0.f, 0.f, 0.f};
                int n = 0;
                if (hi == lo) {
                    f[0] = 1.f;
                    n = 1;
                } else {
                    const float inv = 1.f / (float)(hi - lo);
                    int s = lo, e = (h0 + 1) * ipt, h = h0;
                    while (true) {
                        const int end = min(hi, e);
                        if (n < 3) f[n] = (float)(end - s) * inv;
                        ++n;
                        if (end >= hi || h + 1 >= p.N) break;
                        s = end;
                        e += ipt;
                        ++h;
                    }
                    if (n > 3) {
                        set_error(p.err, kErrUnsupported, gid);
                        n = 3;
                    }
                }
                rec = make_int4(h0 | (n << 16), __float_as_int(f[0]), __float_as_int(f[1]), __float_as_int(f[2]));
            }
            p.rec[((size_t)day * p.n_pairs + pi) * p.N + b] = rec;
            ++pi;
        }
        const int a = p.rlinks[l0 + j];
        if (tab) {
            lo = tab[(size_t)(j + 1) * (p.N + 1) + b];
            hi = tab[(size_t)(j + 1) * (p.N + 1) + b + 1];
        } else {
            lo += tk[(size_t)a * p.Np + min(interval_of(lo, p.div), p.N - 1)];
            hi += tk[(size_t)a * p.Np + min(interval_of(hi, p.div), p.N - 1)];
        }
    }
}

cudaError_t launch_plain_build(const PlainParams &p, cudaStream_t s) {
    const long long n = (long long)p.n_days * p.P * p.N;
    const int block = 256;
    k_plain_build<<<(unsigned)((n + block - 1) / block), block, 0, s>>>(p);
    return cudaGetLastError();
}

// Route choice portions p[d][k][b] (Eq. (logit), (rt)).
__global__ void k_plain_route_choice(const PlainParams p) {
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= (long long)p.n_days * p.P * p.N) return;
    const int b = (int)(gid % p.N);
    const long long dk = gid / p.N;
    const int k = (int)(dk % p.P), day = (int)(dk / p.P);
    const int od = p.rod[k];
    const float *Cd = p.C + (size_t)day * p.P * p.Np;
    float m = -INFINITY;
    for (int i = p.od_ptr[od]; i < p.od_ptr[od + 1]; ++i)
        m = fmaxf(m, -p.theta * Cd[(size_t)p.od_routes[i] * p.Np + b]);
    float den = 0.f;
    for (int i = p.od_ptr[od]; i < p.od_ptr[od + 1]; ++i)
        den += expf(-p.theta * Cd[(size_t)p.od_routes[i] * p.Np + b] - m);
    p.p[((size_t)day * p.P + k) * p.Np + b] = expf(-p.theta * Cd[(size_t)k * p.Np + b] - m) / den;
}

cudaError_t launch_plain_route_choice(const PlainParams &p, cudaStream_t s) {
    const long long n = (long long)p.n_days * p.P * p.N;
    k_plain_route_choice<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p);
    return cudaGetLastError();
}

// xhat[d][o][h2] += rho * p * q (scatter with atomics).
__global__ void k_plain_forward(const PlainParams p, const float *__restrict__ q, float *__restrict__ xhat) {
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= (long long)p.n_days * p.n_pairs * p.N) return;
    const int b = (int)(gid % p.N);
    const long long dp = gid / p.N;
    const int pi = (int)(dp % p.n_pairs), day = (int)(dp / p.n_pairs);
    const int4 rec = p.rec[gid];
    const int n = rec.x >> 16;
    if (n == 0) return;
    const int k = p.pair_k[pi], o = p.pair_o[pi];
    const float f = p.p[((size_t)day * p.P + k) * p.Np + b] * q[((size_t)day * p.K + p.rod[k]) * p.Np + b];
    if (f == 0.f) return;
    float *x = xhat + ((size_t)day * p.O + o) * p.Np + (rec.x & 0xffff);
    atomicAdd(x, f * __int_as_float(rec.y));
    if (n > 1) atomicAdd(x + 1, f * __int_as_float(rec.z));
    if (n > 2) atomicAdd(x + 2, f * __int_as_float(rec.w));
}

cudaError_t launch_plain_forward(const PlainParams &p, const float *q, float *xhat, cudaStream_t s) {
    const long long n = (long long)p.n_days * p.n_pairs * p.N;
    k_plain_forward<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, q, xhat);
    return cudaGetLastError();
}

// r = m (xhat - x) in place; loss[d] += sum r^2.
__global__ void k_plain_residual(const PlainParams p, const float *__restrict__ counts,
                                 const uint32_t *__restrict__ mask, float *__restrict__ xr, double *loss) {
    const int day = blockIdx.y;
    const size_t cells = (size_t)p.O * p.Np;
    float acc = 0.f;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < cells; c += (size_t)gridDim.x * blockDim.x) {
        const int o = (int)(c / p.Np), h = (int)(c % p.Np);
        const size_t i = (size_t)day * cells + c;
        float r = 0.f;
        if (h < p.N && ((mask[((size_t)day * p.O + o) * p.Nw + (h >> 5)] >> (h & 31)) & 1u)) r = xr[i] - counts[i];
        xr[i] = r;
        acc += r * r;
    }
    double v = acc;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(&loss[day], v);
}

cudaError_t launch_plain_residual(const PlainParams &p, const float *counts, const uint32_t *mask, float *xr,
                                  double *loss, float *trace_row, cudaStream_t s) {
    (void)trace_row;
    dim3 grid(8, p.n_days);
    k_plain_residual<<<grid, 256, 0, s>>>(p, counts, mask, xr, loss);
    return cudaGetLastError();
}

// g = B^T r per (day, OD, interval), then Adagrad + projection.
__global__ void k_plain_adjoint_step(const PlainParams p, const float *__restrict__ r, float *__restrict__ q,
                                     float *__restrict__ G, float eta, float eps) {
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= (long long)p.n_days * p.K * p.N) return;
    const int b = (int)(gid % p.N);
    const long long dod = gid / p.N;
    const int od = (int)(dod % p.K), day = (int)(dod / p.K);
    float g = 0.f;
    for (int i = p.od_ptr[od]; i < p.od_ptr[od + 1]; ++i) {
        const int k = p.od_routes[i];
        float gp = 0.f;
        for (int pi = p.route_pair_ptr[k]; pi < p.route_pair_ptr[k + 1]; ++pi) {
            const int4 rec = p.rec[((size_t)day * p.n_pairs + pi) * p.N + b];
            const int n = rec.x >> 16;
            if (n == 0) continue;
            const float *rr = r + ((size_t)day * p.O + p.pair_o[pi]) * p.Np + (rec.x & 0xffff);
            gp += __int_as_float(rec.y) * rr[0];
            if (n > 1) gp += __int_as_float(rec.z) * rr[1];
            if (n > 2) gp += __int_as_float(rec.w) * rr[2];
        }
        g += p.p[((size_t)day * p.P + k) * p.Np + b] * gp;
    }
    const size_t qi = ((size_t)day * p.K + od) * p.Np + b;
    const float Gv = G[qi] + g * g;
    const float qv = fmaxf(q[qi] - eta * g / (sqrtf(Gv) + eps), 0.f);
    G[qi] = Gv;
    q[qi] = qv;
}

cudaError_t launch_plain_adjoint_step(const PlainParams &p, const float *r, float *q, float *G, float eta,
                                      float eps, cudaStream_t s) {
    const long long n = (long long)p.n_days * p.K * p.N;
    k_plain_adjoint_step<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, r, q, G, eta, eps);
    return cudaGetLastError();
}

}  // namespace dode
