// Complex GEMMs of the solver on CUDA cores (FP64 or FP32 operands).
//
//   gemm_gram : C(i, j) = alpha * sum_k conj(A[i][k]) B[j][k] + beta * C(i, j)
//               the inner products of two row blocks over the long plane-wave
//               index k (projections <beta|psi>, Gram matrices of the
//               Rayleigh-Ritz step).  Split over k, partial tiles summed in a
//               fixed order (deterministic), result in FP64.
//   gemm_nn   : C[i][n] = alpha * sum_k A(i, k) B[k][n] + beta * D[i][n]
//               a small coefficient matrix applied to a row block (basis
//               rotations, projector application).
#include "fs_common.cuh"


#include <algorithm>

namespace {

constexpr int BM = 64, BN = 64, BK = 16, THREADS = 256;

template <typename T2> struct acc_of;
template <> struct acc_of<double2> { using t = double; };
template <> struct acc_of<float2> { using t = float; };

template <typename T2>
__global__ void __launch_bounds__(THREADS)
gram_kernel(int M, int N, int K, const T2* __restrict__ A, long lda, const int* __restrict__ amap,
            const T2* __restrict__ B, long ldb, const int* __restrict__ bmap, double2* __restrict__ part, int kchunk) {
    using R = typename acc_of<T2>::t;
    __shared__ T2 As[BK][BM + 1];
    __shared__ T2 Bs[BK][BN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    R ar[4][4], ai[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) ar[a][b] = ai[a][b] = (R)0;
    const int lk = threadIdx.x % BK, lr = threadIdx.x / BK;  // 16 rows per pass
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
        for (int p = 0; p < BM / 16; ++p) {
            int r = lr + 16 * p;
            int k = k0 + lk;
            int gi = i0 + r, gj = j0 + r;
            T2 va = mk((R)0, (R)0), vb = mk((R)0, (R)0);
            if (k < kend) {
                if (gi < M) va = A[(amap ? (long)amap[gi] : (long)gi) * lda + k];
                if (gj < N) vb = B[(bmap ? (long)bmap[gj] : (long)gj) * ldb + k];
            }
            As[lk][r] = va;
            Bs[lk][r] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T2 a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty + 16 * q];
                b[q] = Bs[kk][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    // conj(a) * b
                    ar[p][q] += a[p].x * b[q].x + a[p].y * b[q].y;
                    ai[p][q] += a[p].x * b[q].y - a[p].y * b[q].x;
                }
        }
        __syncthreads();
    }
    double2* out = part + (long)blockIdx.z * M * N;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        int gi = i0 + ty + 16 * p;
        if (gi >= M) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int gj = j0 + tx + 16 * q;
            if (gj < N) out[(long)gi * N + gj] = make_double2((double)ar[p][q], (double)ai[p][q]);
        }
    }
}

__global__ void gram_reduce_kernel(int M, int N, int splits, const double2* __restrict__ part, double2* C, long ci,
                                   long cj, double alpha, double beta) {
    long total = (long)M * N;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        double sx = 0, sy = 0;
        for (int s = 0; s < splits; ++s) {
            double2 v = part[(long)s * total + t];
            sx += v.x;
            sy += v.y;
        }
        long i = t / N, j = t - i * N;
        double2* dst = C + i * ci + j * cj;
        double2 o = make_double2(alpha * sx, alpha * sy);
        if (beta != 0.0) {
            o.x += beta * dst->x;
            o.y += beta * dst->y;
        }
        *dst = o;
    }
}

template <typename T2, typename A2>
__global__ void __launch_bounds__(THREADS)
nn_kernel(int M, int N, int K, const A2* __restrict__ A, long ai_, long ak_, const T2* __restrict__ B, long ldb,
          const int* __restrict__ bmap, T2* C, long ldc, const int* __restrict__ cmap, double alpha, double beta,
          const T2* D, long ldd) {
    using R = typename acc_of<T2>::t;
    __shared__ T2 As[BK][BM + 1];
    __shared__ T2 Bs[BK][BN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int i0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    R cr[4][4], ci[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cr[a][b] = ci[a][b] = (R)0;
    for (int k0 = 0; k0 < K; k0 += BK) {
        // A tile: BM rows (i) x BK (k)
        {
            int kk = threadIdx.x % BK, r = threadIdx.x / BK;
#pragma unroll
            for (int p = 0; p < BM / 16; ++p) {
                int i = i0 + r + 16 * p, k = k0 + kk;
                T2 v = mk((R)0, (R)0);
                if (i < M && k < K) v = conv<T2>(A[(long)i * ai_ + (long)k * ak_]);
                As[kk][r + 16 * p] = v;
            }
        }
        // B tile: BK rows (k) x BN (n)
        {
            int nn = threadIdx.x % BN, r = threadIdx.x / BN;  // 4 rows per pass
#pragma unroll
            for (int p = 0; p < BK / 4; ++p) {
                int k = k0 + r + 4 * p, n = n0 + nn;
                T2 v = mk((R)0, (R)0);
                if (k < K && n < N) v = B[(bmap ? (long)bmap[k] : (long)k) * ldb + n];
                Bs[r + 4 * p][nn] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T2 a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty + 16 * q];
                b[q] = Bs[kk][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    cr[p][q] += a[p].x * b[q].x - a[p].y * b[q].y;
                    ci[p][q] += a[p].x * b[q].y + a[p].y * b[q].x;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        int i = i0 + ty + 16 * p;
        if (i >= M) continue;
        long row = cmap ? (long)cmap[i] : (long)i;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int n = n0 + tx + 16 * q;
            if (n >= N) continue;
            R ox = (R)alpha * cr[p][q], oy = (R)alpha * ci[p][q];
            if (beta != 0.0) {
                T2 d = D[row * ldd + n];
                ox += (R)beta * d.x;
                oy += (R)beta * d.y;
            }
            C[row * ldc + n] = mk(ox, oy);
        }
    }
}

}  // namespace

template <typename T2>
void gemm_gram(fs_ctx* c, int M, int N, int K, const T2* A, long lda, const int* amap, const T2* B, long ldb,
               const int* bmap, double2* C, long ci, long cj, double alpha, double beta, int kid) {
    if (M <= 0 || N <= 0) return;
    if constexpr (sizeof(T2) == 8) {
        if (c->gemm_path == FS_GEMM_TENSOR) {
            tc_gemm_gram(c, M, N, K, A, lda, amap, B, ldb, bmap, C, ci, cj, alpha, beta, kid);
            return;
        }
    }
    ProfScope ps(c, ks_prec<T2>(kid), ((double)M + N) * K * sizeof(T2) + (double)M * N * sizeof(double2),
                 8.0 * M * N * K);
    if constexpr (sizeof(T2) == 16) {
        // FP64 without row maps and with C column-major is a plain GEMM, C = alpha A^H B + beta C
        // (A, B column-major K x M and K x N): the dense FP64 GEMM (split K when the output is
        // small), about three times the rate of the row-mapped kernel below
        if (!amap && !bmap && ci == 1) {
            dense_gemm(c, 1, 0, M, N, K, alpha, (const double2*)A, (int)lda, (const double2*)B, (int)ldb, beta, C,
                       (int)cj);
            return;
        }
    }
    int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
    int want = std::max(1, (2 * 152 + tm * tn - 1) / (tm * tn));
    int maxs = std::max(1, K / 512);
    int splits = std::min(want, maxs);
    int kchunk = (K + splits - 1) / splits;
    kchunk = ((kchunk + BK - 1) / BK) * BK;
    splits = std::max(1, (K + kchunk - 1) / kchunk);
    c->splitk.ensure((size_t)splits * M * N * sizeof(double2));
    dim3 g(tm, tn, splits);
    gram_kernel<T2><<<g, THREADS, 0, c->stream>>>(M, N, K, A, lda, amap, B, ldb, bmap, c->splitk.as<double2>(), kchunk);
    long total = (long)M * N;
    int rb = (int)std::min<long>(2048, (total + 255) / 256);
    gram_reduce_kernel<<<rb, 256, 0, c->stream>>>(M, N, splits, c->splitk.as<double2>(), C, ci, cj, alpha, beta);
    FS_CUDA(cudaGetLastError());
}

template <typename T2, typename A2>
void gemm_nn(fs_ctx* c, int M, int N, int K, const A2* A, long ai, long ak, const T2* B, long ldb, const int* bmap,
             T2* C, long ldc, const int* cmap, double alpha, double beta, const T2* D, long ldd, int kid) {
    if (M <= 0 || N <= 0) return;
    if constexpr (sizeof(T2) == 8) {
        if (c->gemm_path == FS_GEMM_TENSOR) {
            tc_gemm_nn<A2>(c, M, N, K, A, ai, ak, B, ldb, bmap, C, ldc, cmap, alpha, beta, D, ldd, kid);
            return;
        }
    }
    ProfScope ps(c, ks_prec<T2>(kid), ((double)K + M * (beta != 0.0 ? 2.0 : 1.0)) * N * sizeof(T2) + (double)M * K * sizeof(A2),
                 8.0 * M * N * K);
    if constexpr (sizeof(T2) == 16 && sizeof(A2) == 16) {
        // FP64 without row maps, D aliasing C (or beta = 0) and a unit stride in the coefficients
        // is a plain GEMM on the column-major views: C (N x M) = B (N x K) op(Acoef) (K x M)
        if (!bmap && !cmap && (beta == 0.0 || (D == C && ldd == ldc)) && (ak == 1 || ai == 1)) {
            dense_gemm(c, 0, ak == 1 ? 0 : 2, N, M, K, alpha, (const double2*)B, (int)ldb, (const double2*)A,
                       (int)(ak == 1 ? ai : ak), beta, (double2*)C, (int)ldc);
            return;
        }
    }
    dim3 g((N + BN - 1) / BN, (M + BM - 1) / BM);
    nn_kernel<T2, A2><<<g, THREADS, 0, c->stream>>>(M, N, K, A, ai, ak, B, ldb, bmap, C, ldc, cmap, alpha, beta, D,
                                                    ldd);
    FS_CUDA(cudaGetLastError());
}

template void gemm_gram<double2>(fs_ctx*, int, int, int, const double2*, long, const int*, const double2*, long,
                                 const int*, double2*, long, long, double, double, int);
template void gemm_gram<float2>(fs_ctx*, int, int, int, const float2*, long, const int*, const float2*, long,
                                const int*, double2*, long, long, double, double, int);
template void gemm_nn<double2, double2>(fs_ctx*, int, int, int, const double2*, long, long, const double2*, long,
                                        const int*, double2*, long, const int*, double, double, const double2*, long,
                                        int);
template void gemm_nn<float2, double2>(fs_ctx*, int, int, int, const double2*, long, long, const float2*, long,
                                       const int*, float2*, long, const int*, double, double, const float2*, long,
                                       int);

// Gram form with caller-provided split-K scratch (no allocation): the same
// kernels as gemm_gram on CUDA cores; part must hold splits * M * N double2.
// Returns false when the scratch is too small for even one split.
template <typename T2>
bool gemm_gram_scratch(cudaStream_t st, int M, int N, int K, const T2* A, long lda, const T2* B, long ldb, double2* C,
                       long ci, long cj, double2* part, size_t part_bytes) {
    if (M <= 0 || N <= 0) return true;
    const size_t per_split = (size_t)M * N * sizeof(double2);
    if (per_split > part_bytes) return false;
    int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
    int want = std::max(1, (2 * 152 + tm * tn - 1) / (tm * tn));
    int maxs = std::max(1, K / 512);
    int splits = std::min(std::min(want, maxs), (int)std::min<size_t>(part_bytes / per_split, 1 << 20));
    int kchunk = (K + splits - 1) / splits;
    kchunk = ((kchunk + BK - 1) / BK) * BK;
    splits = std::max(1, (K + kchunk - 1) / kchunk);
    dim3 g(tm, tn, splits);
    gram_kernel<T2><<<g, THREADS, 0, st>>>(M, N, K, A, lda, nullptr, B, ldb, nullptr, part, kchunk);
    long total = (long)M * N;
    int rb = (int)std::min<long>(2048, (total + 255) / 256);
    gram_reduce_kernel<<<rb, 256, 0, st>>>(M, N, splits, part, C, ci, cj, 1.0, 0.0);
    return true;
}

// Apply form on CUDA cores without the profiling scope (used by the static-scratch entry point).
void gemm_nn_plain64(cudaStream_t st, int M, int N, int K, const double2* A, long ai, long ak, const double2* B,
                     long ldb, double2* C, long ldc, double alpha, double beta, const double2* D, long ldd) {
    if (M <= 0 || N <= 0) return;
    dim3 g((N + BN - 1) / BN, (M + BM - 1) / BM);
    nn_kernel<double2, double2><<<g, THREADS, 0, st>>>(M, N, K, A, ai, ak, B, ldb, nullptr, C, ldc, nullptr, alpha,
                                                       beta, D, ldd);
}

template bool gemm_gram_scratch<double2>(cudaStream_t, int, int, int, const double2*, long, const double2*, long,
                                         double2*, long, long, double2*, size_t);
