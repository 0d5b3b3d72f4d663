// Band-wise vector kernels of the solver: residual norms and inner products
// (warp-shuffle + shared-memory tree, one block per band, fixed order so that
// repeated runs give identical bits), the preconditioned residual, row
// normalisation, start-block generation and precision conversion.
#include "fs_common.cuh"

#include <algorithm>

namespace {

constexpr int RT = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the block; every thread gets the result
__device__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0;
    const int nw = blockDim.x >> 5;
    if (wid == 0) {
        t = lane < nw ? sh[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

// dot = <x, y>, resid = || y - dot x ||
template <typename T2>
__global__ void __launch_bounds__(RT) resid_kernel(const T2* __restrict__ X, const T2* __restrict__ Y, long npw,
                                                   double* resid, double2* dot) {
    __shared__ double sh[33];
    const T2* x = X + blockIdx.x * npw;
    const T2* y = Y + blockIdx.x * npw;
    double dr = 0, di = 0;
    for (long g = threadIdx.x; g < npw; g += blockDim.x) {
        T2 a = x[g], b = y[g];
        dr += (double)a.x * b.x + (double)a.y * b.y;
        di += (double)a.x * b.y - (double)a.y * b.x;
    }
    dr = block_sum(dr, sh);
    di = block_sum(di, sh);
    double s = 0;
    for (long g = threadIdx.x; g < npw; g += blockDim.x) {
        T2 a = x[g], b = y[g];
        double rx = (double)b.x - (dr * a.x - di * a.y);
        double ry = (double)b.y - (dr * a.y + di * a.x);
        s += rx * rx + ry * ry;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        resid[blockIdx.x] = sqrt(s);
        if (dot) dot[blockIdx.x] = make_double2(dr, di);
    }
}

// resid = || y - shift_i x ||
template <typename T2>
__global__ void __launch_bounds__(RT) resid_shift_kernel(const T2* __restrict__ X, const T2* __restrict__ Y,
                                                         const double* __restrict__ shift, long npw, double* resid) {
    __shared__ double sh[33];
    const T2* x = X + blockIdx.x * npw;
    const T2* y = Y + blockIdx.x * npw;
    const double s0 = shift[blockIdx.x];
    double s = 0;
    for (long g = threadIdx.x; g < npw; g += blockDim.x) {
        T2 a = x[g], b = y[g];
        double rx = (double)b.x - s0 * a.x, ry = (double)b.y - s0 * a.y;
        s += rx * rx + ry * ry;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) resid[blockIdx.x] = sqrt(s);
}

template <typename T2>
__global__ void __launch_bounds__(RT) row_norm_kernel(const T2* __restrict__ X, const int* __restrict__ map, long npw,
                                                      double* out) {
    __shared__ double sh[33];
    long row = map ? map[blockIdx.x] : blockIdx.x;
    const T2* x = X + row * npw;
    double s = 0;
    for (long g = threadIdx.x; g < npw; g += blockDim.x) {
        T2 a = x[g];
        s += (double)a.x * a.x + (double)a.y * a.y;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(s);
}

// kinetic energy of each band: sum_g |q_g|^2/2 |x_g|^2 / sum_g |x_g|^2
template <typename T2>
__global__ void __launch_bounds__(RT) band_kin_kernel(const T2* __restrict__ X, const double* __restrict__ kin, long npw,
                                                      double* out) {
    __shared__ double sh[33];
    const T2* x = X + (long)blockIdx.x * npw;
    double s = 0, n = 0;
    for (long g = threadIdx.x; g < npw; g += blockDim.x) {
        T2 a = x[g];
        double p = (double)a.x * a.x + (double)a.y * a.y;
        s += kin[g] * p;
        n += p;
    }
    s = block_sum(s, sh);
    n = block_sum(n, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = n > 0 ? s / n : 0.0;
}

template <typename T2>
__global__ void scale_rows_kernel(T2* X, const int* __restrict__ map, long npw, const double* __restrict__ nrm) {
    using R = typename real_of<T2>::t;
    long row = map ? map[blockIdx.y] : blockIdx.y;
    double f = nrm[blockIdx.y];
    R inv = (R)(f > 0 ? 1.0 / f : 0.0);
    T2* x = X + row * npw;
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < npw; g += (long)gridDim.x * blockDim.x)
        x[g] = cscale(x[g], inv);
}

// W[a] = M_i(q) R[act[a]]
//   precond 0: paper's M(q) = 1 / ((|q|^2/2 - E)^2 + dE^2)
//   precond 1: folded Teter-Payne-Allan form K(x)^2 / T_i^2 with x = (|q|^2/2) / T_i
template <typename T2>
__global__ void make_w_kernel(const T2* __restrict__ R, const int* __restrict__ act, long npw, T2* __restrict__ W,
                              const double* __restrict__ kin, double e_ref, double dE2, int precond,
                              const double* __restrict__ band_kin) {
    using Rl = typename real_of<T2>::t;
    const int i = act[blockIdx.y];
    const T2* r = R + (long)i * npw;
    T2* w = W + (long)blockIdx.y * npw;
    double tk = band_kin ? fmax(band_kin[i], 1e-3) : 1.0;
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < npw; g += (long)gridDim.x * blockDim.x) {
        double m;
        if (precond == 1) {
            double xx = kin[g] / tk;
            double num = 27.0 + xx * (18.0 + xx * (12.0 + 8.0 * xx));
            double kk = num / (num + 16.0 * xx * xx * xx * xx);
            m = kk * kk / (tk * tk);
        } else if (precond == 2) {  // lowest states of H itself: 1 / (1 + |q|^2 / 2)
            m = 1.0 / (1.0 + kin[g]);
        } else {
            double d = kin[g] - e_ref;
            m = 1.0 / (d * d + dE2);
        }
        T2 a = r[g];
        w[g] = mk((Rl)m * a.x, (Rl)m * a.y);
    }
}

// RH[i] = y_i - d_i x_i with d_i = <x_i, y_i>  (the H residual of band i)
template <typename T2>
__global__ void rh_kernel(const T2* __restrict__ X, const T2* __restrict__ Y, const double2* __restrict__ dots,
                          long npw, T2* __restrict__ RH) {
    using Rl = typename real_of<T2>::t;
    const long i = blockIdx.y;
    const double2 d = dots[i];
    const T2* x = X + i * npw;
    const T2* y = Y + i * npw;
    T2* o = RH + i * npw;
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < npw; g += (long)gridDim.x * blockDim.x) {
        T2 a = x[g], b = y[g];
        o[g] = mk((Rl)(b.x - (d.x * a.x - d.y * a.y)), (Rl)(b.y - (d.x * a.y + d.y * a.x)));
    }
}

// A residual from the H residual r = y - d x:  (H-E)^2 x - theta x
//   = (H-E) r + d r + (d^2 - theta) x,   written over RH;  ra_i = its norm.
// Every term is computed from the small vector r, so its rounding error
// scales with ||r|| instead of with ||(H-E) y||.
template <typename T2>
__global__ void __launch_bounds__(RT) a_resid_kernel(const T2* __restrict__ ZR, T2* RH, const T2* __restrict__ X,
                                                     const double2* __restrict__ dots,
                                                     const double* __restrict__ theta, long npw, double* ra) {
    using Rl = typename real_of<T2>::t;
    __shared__ double sh[33];
    const long i = blockIdx.x;
    const double2 d = dots[i];
    const double c0x = d.x * d.x - d.y * d.y - theta[i], c0y = 2.0 * d.x * d.y;
    const T2* z = ZR + i * npw;
    const T2* x = X + i * npw;
    T2* r = RH + i * npw;
    double s = 0;
    for (long g = threadIdx.x; g < npw; g += blockDim.x) {
        T2 a = z[g], b = r[g], c = x[g];
        double ox = (double)a.x + (d.x * b.x - d.y * b.y) + (c0x * c.x - c0y * c.y);
        double oy = (double)a.y + (d.x * b.y + d.y * b.x) + (c0x * c.y + c0y * c.x);
        r[g] = mk((Rl)ox, (Rl)oy);
        s += ox * ox + oy * oy;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) ra[i] = sqrt(s);
}

// splitmix64 (Steele, Lea and Flood 2014) as a counter-based generator
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void damp_random_kernel(double2* X, long npw, int first, unsigned long long seed,
                                   const double* __restrict__ kin) {
    const long band = first + blockIdx.y;
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < npw; g += (long)gridDim.x * blockDim.x) {
        unsigned long long ctr = ((unsigned long long)band << 32) ^ (unsigned long long)g;
        unsigned long long h1 = splitmix64(seed ^ splitmix64(2 * ctr));
        unsigned long long h2 = splitmix64(seed ^ splitmix64(2 * ctr + 1));
        double u1 = ((h1 >> 11) + 1) * (1.0 / 9007199254740993.0);  // (0, 1]
        double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);        // [0, 1)
        double r = sqrt(-2.0 * log(u1));
        double s, c;
        sincospi(2.0 * u2, &s, &c);
        double d = 1.0 / (1.0 + kin[g]);
        X[band * npw + g] = make_double2(r * c * d, r * s * d);
    }
}

__global__ void damp_kernel(double2* X, long npw, const double* __restrict__ kin) {
    double2* x = X + (long)blockIdx.y * npw;
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < npw; g += (long)gridDim.x * blockDim.x) {
        double d = 1.0 / (1.0 + kin[g]);
        x[g] = make_double2(x[g].x * d, x[g].y * d);
    }
}

template <typename S2, typename T2>
__global__ void convert_kernel(const S2* __restrict__ in, T2* __restrict__ out, long count) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count; t += (long)gridDim.x * blockDim.x)
        out[t] = conv<T2>(in[t]);
}

inline int gx_for(long npw) { return (int)std::min<long>(64, (npw + 255) / 256); }

}  // namespace

template <typename T2> void vec_resid(fs_ctx* c, const T2* X, const T2* Y, int m, double* resid, double2* dot) {
    if (m <= 0) return;
    ProfScope ps(c, ks_prec<T2>(KS_VECTOR), 2.0 * m * c->npw * sizeof(T2), 16.0 * m * c->npw);
    resid_kernel<T2><<<m, RT, 0, c->stream>>>(X, Y, c->npw, resid, dot);
    FS_CUDA(cudaGetLastError());
}

template <typename T2>
void vec_resid_shift(fs_ctx* c, const T2* X, const T2* Y, const double* shift, int m, double* resid) {
    if (m <= 0) return;
    ProfScope ps(c, ks_prec<T2>(KS_VECTOR), 2.0 * m * c->npw * sizeof(T2), 8.0 * m * c->npw);
    resid_shift_kernel<T2><<<m, RT, 0, c->stream>>>(X, Y, shift, c->npw, resid);
    FS_CUDA(cudaGetLastError());
}

template <typename T2>
void vec_make_w(fs_ctx* c, const T2* R, const int* act, int na, T2* W, double e_ref, double dE, int precond,
                const double* band_kin) {
    if (na <= 0) return;
    ProfScope ps(c, ks_prec<T2>(KS_VECTOR), 2.0 * na * c->npw * sizeof(T2) + c->npw * 8.0, 6.0 * na * c->npw);
    dim3 g(gx_for(c->npw), na);
    make_w_kernel<T2><<<g, 256, 0, c->stream>>>(R, act, c->npw, W, c->kin.as<double>(), e_ref, dE * dE, precond,
                                                 band_kin);
    FS_CUDA(cudaGetLastError());
}

template <typename T2> void vec_rh(fs_ctx* c, const T2* X, const T2* Y, const double2* dots, int m, T2* RH) {
    if (m <= 0) return;
    ProfScope ps(c, ks_prec<T2>(KS_VECTOR), 3.0 * m * c->npw * sizeof(T2), 8.0 * m * c->npw);
    dim3 g(gx_for(c->npw), m);
    rh_kernel<T2><<<g, 256, 0, c->stream>>>(X, Y, dots, c->npw, RH);
    FS_CUDA(cudaGetLastError());
}

template <typename T2>
void vec_a_resid(fs_ctx* c, const T2* ZR, T2* RH, const T2* X, const double2* dots, const double* theta, int m,
                 double* ra) {
    if (m <= 0) return;
    ProfScope ps(c, ks_prec<T2>(KS_VECTOR), 4.0 * m * c->npw * sizeof(T2), 20.0 * m * c->npw);
    a_resid_kernel<T2><<<m, RT, 0, c->stream>>>(ZR, RH, X, dots, theta, c->npw, ra);
    FS_CUDA(cudaGetLastError());
}

template <typename T2> void vec_row_norms(fs_ctx* c, const T2* X, const int* map, int nrows, double* out) {
    if (nrows <= 0) return;
    ProfScope ps(c, ks_prec<T2>(KS_VECTOR), 1.0 * nrows * c->npw * sizeof(T2), 4.0 * nrows * c->npw);
    row_norm_kernel<T2><<<nrows, RT, 0, c->stream>>>(X, map, c->npw, out);
    FS_CUDA(cudaGetLastError());
}

template <typename T2> void vec_band_kin(fs_ctx* c, const T2* X, int m, double* out) {
    if (m <= 0) return;
    ProfScope ps(c, ks_prec<T2>(KS_VECTOR), 1.0 * m * c->npw * sizeof(T2) + 8.0 * c->npw, 6.0 * m * c->npw);
    band_kin_kernel<T2><<<m, RT, 0, c->stream>>>(X, c->kin.as<double>(), c->npw, out);
    FS_CUDA(cudaGetLastError());
}

template <typename T2> void vec_scale_rows(fs_ctx* c, T2* X, const int* map, int nrows, const double* nrm) {
    if (nrows <= 0) return;
    ProfScope ps(c, ks_prec<T2>(KS_VECTOR), 2.0 * nrows * c->npw * sizeof(T2), 2.0 * nrows * c->npw);
    dim3 g(gx_for(c->npw), nrows);
    scale_rows_kernel<T2><<<g, 256, 0, c->stream>>>(X, map, c->npw, nrm);
    FS_CUDA(cudaGetLastError());
}

void vec_damp_random(fs_ctx* c, double2* X, int m, int first, unsigned long long seed) {
    if (m - first <= 0) return;
    dim3 g(gx_for(c->npw), m - first);
    damp_random_kernel<<<g, 256, 0, c->stream>>>(X, c->npw, first, seed, c->kin.as<double>());
    FS_CUDA(cudaGetLastError());
}

void vec_damp(fs_ctx* c, double2* X, int m) {
    if (m <= 0) return;
    dim3 g(gx_for(c->npw), m);
    damp_kernel<<<g, 256, 0, c->stream>>>(X, c->npw, c->kin.as<double>());
    FS_CUDA(cudaGetLastError());
}

template <typename S2, typename T2> void vec_convert(fs_ctx* c, const S2* in, T2* out, size_t count) {
    if (count == 0) return;
    int b = (int)std::min<size_t>(4096, (count + 255) / 256);
    convert_kernel<S2, T2><<<b, 256, 0, c->stream>>>(in, out, (long)count);
    FS_CUDA(cudaGetLastError());
}

#define INST(T2)                                                                                           \
    template void vec_resid<T2>(fs_ctx*, const T2*, const T2*, int, double*, double2*);                     \
    template void vec_resid_shift<T2>(fs_ctx*, const T2*, const T2*, const double*, int, double*);          \
    template void vec_make_w<T2>(fs_ctx*, const T2*, const int*, int, T2*, double, double, int, const double*); \
    template void vec_rh<T2>(fs_ctx*, const T2*, const T2*, const double2*, int, T2*);                      \
    template void vec_a_resid<T2>(fs_ctx*, const T2*, T2*, const T2*, const double2*, const double*, int,   \
                                  double*);                                                                 \
    template void vec_row_norms<T2>(fs_ctx*, const T2*, const int*, int, double*);                          \
    template void vec_band_kin<T2>(fs_ctx*, const T2*, int, double*);                                       \
    template void vec_scale_rows<T2>(fs_ctx*, T2*, const int*, int, const double*);
INST(double2)
INST(float2)
template void vec_convert<double2, float2>(fs_ctx*, const double2*, float2*, size_t);
template void vec_convert<float2, double2>(fs_ctx*, const float2*, double2*, size_t);
