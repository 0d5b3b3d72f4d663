// Small dense FP64 linear algebra of the Rayleigh-Ritz steps, on the GPU.
//
// Matrices are complex double, column-major, leading dimension = rows.
//   dense_gemm   C = alpha op(A) op(B) + beta C, op = N, C (conjugate transpose) or,
//                for B, T (transpose);
//                32 x 32 tiles staged in shared memory (FP64 FMA).
//   dense_potrf  Cholesky A = L L^H of the lower triangle, blocked (32): the
//                diagonal block factorised in shared memory, the panel by a
//                row-wise triangular solve, the trailing matrix by dense_gemm.
//                Reports the first non-positive pivot (LAPACK's info).
//   dense_trsm   B <- L^-1 B or L^-H B, blocked (32) the same way.
//   dense_heev   the m lowest eigenpairs of a Hermitian matrix:
//     1. Householder reduction to a real symmetric tridiagonal T = Q^H A Q
//        (Q = H_0 ... H_{n-2}, H_i = I - tau_i v_i v_i^H, the LAPACK zhetd2
//        steps), all n - 1 steps in one cooperative kernel whose blocks meet
//        at a bounded grid barrier twice per step;
//     2. eigenvalues of T by bisection on Sturm counts (a warp evaluates 31
//        points of the bracket at once, so each round narrows it 32-fold; the
//        counts come from the leading minors, rescaled, without division);
//     3. eigenvectors of T by inverse iteration (Gaussian elimination with
//        partial pivoting on T - lambda I), vectors of eigenvalues closer
//        than 1e-10 ||T|| handled as one cluster and made orthogonal to each
//        other by modified Gram-Schmidt (a warp per cluster);
//     4. back-transformation Z = Q z in blocks of 32 reflectors (compact WY
//        form), each block as three GEMMs, then one Cholesky QR pass on Z.
// Every device-side wait (the grid barrier) is bounded: on expiry the
// context's error flag is raised and the kernel returns.
#include "fs_common.cuh"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

namespace {

constexpr int TB = 32;       // GEMM tile
constexpr int TK = 16;       // GEMM k step
constexpr int NBLK = 32;     // block size of the blocked factorisations
constexpr long long BAR_LIMIT = 1ll << 22;

__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }

// ------------------------------------------------------------------ GEMM
// C[M x N] = alpha op(A) op(B) + beta C; opA/opB: 0 = N, 1 = C (conjugate transpose), opB 2 = T
// Split K (gridDim.z > 1): block z takes k in [z kc, min(K, (z + 1) kc)) and
// writes its partial product to C + z M N (ld M) with alpha = 1, beta = 0.
// lower = 1: tiles wholly above the diagonal (every row index below every column
// index) are skipped, for updates of which only the lower triangle is used.
__global__ void __launch_bounds__(256) zgemm_kernel(int M, int N, int K, int opA, int opB, double alpha,
                                                    const double2* __restrict__ A, int lda,
                                                    const double2* __restrict__ B, int ldb, double beta,
                                                    double2* __restrict__ C, int ldc, int kc, int lower) {
    __shared__ double2 As[TK][TB + 1];
    __shared__ double2 Bs[TK][TB + 1];
    const int m0 = blockIdx.x * TB, n0 = blockIdx.y * TB;
    if (lower && m0 + TB <= n0) return;
    if (gridDim.z > 1) {
        const int k0 = blockIdx.z * kc;
        K = min(K - k0, kc);
        A += opA == 0 ? (long)k0 * lda : k0;
        B += opB == 0 ? k0 : (long)k0 * ldb;  // C and T read B[n + k ldb]
        C += (size_t)blockIdx.z * M * N;
        ldc = M;
    }
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    double2 acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc[a][b] = make_double2(0.0, 0.0);
    // tile element e (0 .. 511) of op(A) and op(B) for the k step at k0; the next step's
    // elements are loaded into registers while the current step's are multiplied
    auto load = [&](int k0, double2 (&va)[2], double2 (&vb)[2]) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = t + u * 256;
            // op(A)(m, k): N -> A[m + k lda] (m fastest), C -> conj(A[k + m lda]) (k fastest)
            int mm, kk;
            if (opA == 0) { mm = e & (TB - 1); kk = e >> 5; } else { kk = e & (TK - 1); mm = e >> 4; }
            const int gm = m0 + mm, gk = k0 + kk;
            double2 v = make_double2(0.0, 0.0);
            if (gm < M && gk < K) v = opA == 0 ? A[gm + (long)gk * lda] : zconj(A[gk + (long)gm * lda]);
            va[u] = v;
            // op(B)(k, n): N -> B[k + n ldb] (k fastest), C and T -> B[n + k ldb] (n fastest)
            int nn;
            if (opB == 0) { kk = e & (TK - 1); nn = e >> 4; } else { nn = e & (TB - 1); kk = e >> 5; }
            const int gn = n0 + nn, gk2 = k0 + kk;
            v = make_double2(0.0, 0.0);
            if (gn < N && gk2 < K) {
                v = opB == 0 ? B[gk2 + (long)gn * ldb] : B[gn + (long)gk2 * ldb];
                if (opB == 1) v = zconj(v);
            }
            vb[u] = v;
        }
    };
    auto store = [&](const double2 (&va)[2], const double2 (&vb)[2]) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = t + u * 256;
            int mm, kk, nn;
            if (opA == 0) { mm = e & (TB - 1); kk = e >> 5; } else { kk = e & (TK - 1); mm = e >> 4; }
            As[kk][mm] = va[u];
            if (opB == 0) { kk = e & (TK - 1); nn = e >> 4; } else { nn = e & (TB - 1); kk = e >> 5; }
            Bs[kk][nn] = vb[u];
        }
    };
    double2 va[2], vb[2];
    if (K > 0) load(0, va, vb);
    for (int k0 = 0; k0 < K; k0 += TK) {
        store(va, vb);
        __syncthreads();
        if (k0 + TK < K) load(k0 + TK, va, vb);
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            const double2 a0 = As[kk][tx], a1 = As[kk][tx + 16];
            const double2 b0 = Bs[kk][ty], b1 = Bs[kk][ty + 16];
            acc[0][0] = cadd(acc[0][0], cmul(a0, b0));
            acc[0][1] = cadd(acc[0][1], cmul(a0, b1));
            acc[1][0] = cadd(acc[1][0], cmul(a1, b0));
            acc[1][1] = cadd(acc[1][1], cmul(a1, b1));
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int gm = m0 + tx + 16 * a, gn = n0 + ty + 16 * b;
            if (gm < M && gn < N) {
                double2* c = C + gm + (long)gn * ldc;
                double2 o = make_double2(alpha * acc[a][b].x, alpha * acc[a][b].y);
                if (beta != 0.0) {
                    o.x += beta * c->x;
                    o.y += beta * c->y;
                }
                *c = o;
            }
        }
}

// ------------------------------------------------------------------ Cholesky
// Factor the b x b diagonal block at A + j0 (1 + lda) in shared memory; squared
// pivots to piv[j0 + j]; the first non-positive pivot sets *info = j0 + j + 1
// (once) and is replaced by 1 so that the arithmetic stays finite.
__global__ void potrf_diag_kernel(double2* A, int lda, int j0, int b, double* piv, int* info) {
    __shared__ double2 S[NBLK][NBLK + 1];
    const int r = threadIdx.x & (NBLK - 1), c = threadIdx.x >> 5;  // 1024 threads
    double2* D = A + j0 + (long)j0 * lda;
    if (r < b && c < b) S[r][c] = D[r + (long)c * lda];
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        if (threadIdx.x == 0) {
            double p = S[j][j].x;
            if (piv) piv[j0 + j] = p;
            if (!(p > 0.0)) {
                atomicCAS(info, 0, j0 + j + 1);
                p = 1.0;
            }
            S[j][j] = make_double2(sqrt(p), 0.0);
        }
        __syncthreads();
        if (c == j && r > j && r < b) S[r][j] = cscale(S[r][j], 1.0 / S[j][j].x);
        __syncthreads();
        if (c > j && r >= c && r < b) S[r][c] = csub(S[r][c], cmul(S[r][j], zconj(S[c][j])));
        __syncthreads();
    }
    if (r < b && c < b && r >= c) D[r + (long)c * lda] = S[r][c];
}

// rows r >= j0 + b of the panel: A[r, j0:j0+b] <- A[r, j0:j0+b] L^-H (L the
// factored block); one warp per row, lane c holding column c.
__global__ void potrf_panel_kernel(double2* A, int lda, int n, int j0, int b) {
    __shared__ double2 Ls[NBLK][NBLK + 1];
    for (int i = threadIdx.x; i < b * b; i += blockDim.x) {
        const int rr = i % b, cc = i / b;
        Ls[rr][cc] = A[j0 + rr + (long)(j0 + cc) * lda];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int r = j0 + b + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (r >= n) return;
    double2 xv = lane < b ? A[r + (long)(j0 + lane) * lda] : make_double2(0.0, 0.0);
    // x_c = (a_c - sum_{k<c} x_k conj(L[c][k])) / L[c][c]
    for (int c = 0; c < b; ++c) {
        if (lane == c) xv = cscale(xv, 1.0 / Ls[c][c].x);
        const double2 xc = make_double2(__shfl_sync(0xffffffffu, xv.x, c), __shfl_sync(0xffffffffu, xv.y, c));
        if (lane > c && lane < b) xv = csub(xv, cmul(xc, zconj(Ls[lane][c])));
    }
    if (lane < b) A[r + (long)(j0 + lane) * lda] = xv;
}

// ------------------------------------------------------------------ triangular solves
// Diagonal block solve for every column: conj = 0: x = L_bb^-1 b (forward);
// conj = 1: x = L_bb^-H b (backward).  One warp per column, lane r holding row r.
__global__ void trsm_diag_kernel(const double2* L, int lda, int j0, int b, double2* B, int ldb, int ncols, int conj) {
    __shared__ double2 Ls[NBLK][NBLK + 1];
    for (int i = threadIdx.x; i < b * b; i += blockDim.x) {
        const int rr = i % b, cc = i / b;
        Ls[rr][cc] = L[j0 + rr + (long)(j0 + cc) * lda];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (col >= ncols) return;
    double2* x = B + j0 + (long)col * ldb;
    double2 v = lane < b ? x[lane] : make_double2(0.0, 0.0);
    if (!conj) {
        for (int r = 0; r < b; ++r) {
            if (lane == r) v = cscale(v, 1.0 / Ls[r][r].x);
            const double2 xr = make_double2(__shfl_sync(0xffffffffu, v.x, r), __shfl_sync(0xffffffffu, v.y, r));
            if (lane > r && lane < b) v = csub(v, cmul(Ls[lane][r], xr));
        }
    } else {
        for (int r = b - 1; r >= 0; --r) {
            if (lane == r) v = cscale(v, 1.0 / Ls[r][r].x);
            const double2 xr = make_double2(__shfl_sync(0xffffffffu, v.x, r), __shfl_sync(0xffffffffu, v.y, r));
            if (lane < r) v = csub(v, cmul(zconj(Ls[r][lane]), xr));
        }
    }
    if (lane < b) x[lane] = v;
}

__global__ void conj_transpose_kernel(int n, int m, const double2* A, int lda, double2* out, int ldo) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * m) return;
    const int r = (int)(t % n), c = (int)(t / n);
    out[c + (long)r * ldo] = zconj(A[r + (long)c * lda]);
}

// A <- (A + A^H) / 2 (exactly Hermitian input for the reduction)
__global__ void hermitize_kernel(double2* A, int n) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    const int r = (int)(t % n), c = (int)(t / n);
    if (r < c) return;
    const double2 a = A[r + (long)c * n], b = A[c + (long)r * n];
    const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    A[r + (long)c * n] = h;
    A[c + (long)r * n] = zconj(h);
    if (r == c) A[r + (long)c * n].y = 0.0;
}

// ------------------------------------------------------------------ grid barrier
// Blocks of a cooperative launch meet here.  Bounded: after BAR_LIMIT polls the
// waiting block raises the error flag and reports failure.
__device__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, int* err) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok_s = 1;
        volatile unsigned int* gen = bar + 1;
        const unsigned int g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long it = 0;
            while (*gen == g) {
                if (++it > BAR_LIMIT || *(volatile int*)err) {
                    atomicExch(err, 1);
                    ok_s = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok_s != 0;
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0;
    for (int i = 0; i < nw; ++i) s += red[i];
    return s;
}

// ------------------------------------------------------------------ tridiagonal reduction
// Full Hermitian A (n x n, both triangles).  Step i: reflector v_i (v[0] = 1 at
// row i + 1) with H^H x = beta e_1 for x = A[i+1:, i]; y_i = A22 v_i;
// s_i = v_i^H y_i; w_i = tau_i y_i - (|tau_i|^2 s_i / 2) v_i;
// A22 -= v_i w_i^H + w_i v_i^H.  Outputs: d, e (real), tau, V[:, i] = v_i.
//
// One grid barrier per step: after it, every block forms w_i from the segment
// sums of y_i, rebuilds the updated column i + 1 itself (old column minus the
// rank-2 term; no block writes that column) and from it the reflector v_{i+1};
// then (column, segment of SEG rows) units update A22 in place and, from the
// values they just wrote, form the segment sums of y_{i+1}.  Row i + 1 and
// column i + 1 of A are never updated in place: they are not read again.
constexpr int SEG = 256;

// reflector from x[0..L) (smem v holds x on entry, v on exit); every block
__device__ void make_reflector(double2* v, int L, double* red, double2& tau_out, double& beta_out) {
    __shared__ double2 sh_tau, sh_sc;
    __shared__ double sh_beta;
    double ss = 0;
    for (int k = 1 + threadIdx.x; k < L; k += blockDim.x) ss += v[k].x * v[k].x + v[k].y * v[k].y;
    const double xn2 = block_sum(ss, red);
    if (threadIdx.x == 0) {
        const double2 al = v[0];
        if (xn2 == 0.0 && al.y == 0.0) {  // nothing to eliminate: H = I
            sh_tau = make_double2(0.0, 0.0);
            sh_beta = al.x;
            sh_sc = make_double2(0.0, 0.0);
        } else {
            const double beta = -copysign(sqrt(al.x * al.x + al.y * al.y + xn2), al.x);
            sh_tau = make_double2((beta - al.x) / beta, -al.y / beta);
            sh_beta = beta;
            const double2 den = make_double2(al.x - beta, al.y);  // 1 / (alpha - beta)
            const double dd = den.x * den.x + den.y * den.y;
            sh_sc = make_double2(den.x / dd, -den.y / dd);
        }
    }
    __syncthreads();
    const double2 sc = sh_sc;
    for (int k = threadIdx.x; k < L; k += blockDim.x) v[k] = k == 0 ? make_double2(1.0, 0.0) : cmul(v[k], sc);
    tau_out = sh_tau;
    beta_out = sh_beta;
    __syncthreads();
}

__global__ void __launch_bounds__(256)
hetrd_kernel(int n, double2* A, double2* V, double2* tau, double* d, double* e, double2* Yp, unsigned int* bar,
             int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* v = reinterpret_cast<double2*>(smem_raw);  // v_i (length n - i - 1)
    double2* w = v + n;                                  // w_i
    double2* vn = w + n;                                 // v_{i+1}
    __shared__ double red[32];
    const unsigned int nb = gridDim.x;
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    constexpr int PER = SEG / 32;
    if (n < 2) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && n == 1) d[0] = A[0].x;
        return;
    }
    // step 0: reflector from column 0, segment sums of y_0 = A22 v_0
    double2 t;
    double beta;
    {
        const int L = n - 1;
        for (int k = threadIdx.x; k < L; k += blockDim.x) v[k] = __ldcg(A + 1 + k);
        __syncthreads();
        make_reflector(v, L, red, t, beta);
        if (blockIdx.x == 0) {
            for (int k = threadIdx.x; k < L; k += blockDim.x) V[1 + k] = v[k];
            if (threadIdx.x == 0) {
                tau[0] = t;
                e[0] = beta;
                d[0] = __ldcg(A).x;
            }
        }
        const int nseg = (L + SEG - 1) / SEG;
        for (int u = gwarp; u < L * nseg; u += nwarps) {
            const int k = u / nseg, sg = u - k * nseg;
            const double2* col = A + 1 + (long)(1 + k) * n;
            const int c0 = sg * SEG + lane;
            double2 a[PER];
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int cc = c0 + 32 * q;
                a[q] = cc < L ? __ldcg(col + cc) : make_double2(0.0, 0.0);
            }
            double2 acc = make_double2(0.0, 0.0);
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int cc = c0 + 32 * q;
                if (cc < L) acc = cadd(acc, cmulc(a[q], v[cc]));
            }
            for (int o = 16; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (lane == 0) Yp[(long)sg * n + k] = acc;
        }
        if (!grid_barrier(bar, nb, err)) return;
    }
    for (int i = 0; i < n - 1; ++i) {
        const int L = n - i - 1;  // A22 of step i: rows/columns i + 1 .. n - 1
        const int nseg = (L + SEG - 1) / SEG;
        // w_i from the segment sums of y_i
        double sp = 0;
        for (int k = threadIdx.x; k < L; k += blockDim.x) {
            double2 y = __ldcg(Yp + k);
            for (int sg = 1; sg < nseg; ++sg) y = cadd(y, __ldcg(Yp + (long)sg * n + k));
            w[k] = y;
            sp += v[k].x * y.x + v[k].y * y.y;
        }
        const double sv = block_sum(sp, red);
        const double h = 0.5 * (t.x * t.x + t.y * t.y) * sv;
        for (int k = threadIdx.x; k < L; k += blockDim.x) w[k] = csub(cmul(t, w[k]), cscale(v[k], h));
        __syncthreads();
        const double2 v0c = zconj(v[0]), w0c = zconj(w[0]);
        if (L == 1) {  // last step: the remaining 1 x 1 block
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                const double2 a = __ldcg(A + (n - 1) + (long)(n - 1) * n);
                d[n - 1] = csub(a, cadd(cmul(v[0], w0c), cmul(w[0], v0c))).x;
            }
            break;
        }
        // updated column i + 1 (rows i + 1 .. n - 1) and the reflector v_{i+1}
        const double2* colx = A + (i + 1) + (long)(i + 1) * n;
        for (int k = threadIdx.x; k < L; k += blockDim.x)
            vn[k] = csub(__ldcg(colx + k), cadd(cmul(v[k], w0c), cmul(w[k], v0c)));
        __syncthreads();
        const double dnext = vn[0].x;
        const int L1 = L - 1;  // A22 of step i + 1
        double2 tn;
        double bn;
        make_reflector(vn + 1, L1, red, tn, bn);
        if (blockIdx.x == 0) {
            for (int k = threadIdx.x; k < L1; k += blockDim.x) V[(i + 2 + k) + (long)(i + 1) * n] = vn[1 + k];
            if (threadIdx.x == 0) {
                tau[i + 1] = tn;
                e[i + 1] = bn;
                d[i + 1] = dnext;
            }
        }
        // fused units: update A22_{i+1} = rows/columns i + 2 .. n - 1 by step i's rank-2
        // term, then the segment sums of y_{i+1} = A22_{i+1} v_{i+1}
        const int nseg1 = (L1 + SEG - 1) / SEG;
        const double2* vv = vn + 1;
        for (int u = gwarp; u < L1 * nseg1; u += nwarps) {
            const int cidx = u / nseg1, sg = u - cidx * nseg1;
            double2* col = A + (i + 2) + (long)(i + 2 + cidx) * n;
            const double2 vc = zconj(v[1 + cidx]), wc = zconj(w[1 + cidx]);
            const int r0 = sg * SEG + lane;
            double2 a[PER];
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int r = r0 + 32 * q;
                if (r < L1) a[q] = __ldcg(col + r);
            }
            double2 acc = make_double2(0.0, 0.0);
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int r = r0 + 32 * q;
                if (r < L1) {
                    const double2 nv = csub(a[q], cadd(cmul(v[1 + r], wc), cmul(w[1 + r], vc)));
                    col[r] = nv;
                    acc = cadd(acc, cmulc(nv, vv[r]));
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (lane == 0) Yp[(long)sg * n + cidx] = acc;
        }
        // the next step works with v_{i+1}
        __syncthreads();
        for (int k = threadIdx.x; k < L1; k += blockDim.x) v[k] = vv[k];
        t = tn;
        if (!grid_barrier(bar, nb, err)) return;
    }
}

// ------------------------------------------------------------------ tridiagonal eigenvalues
// number of eigenvalues of T (d, e) below x: sign changes of the leading
// principal minors p_j = (d_j - x) p_{j-1} - e_{j-1}^2 p_{j-2} (p_{-1} = 1),
// carried with exact power-of-two rescaling (no division); a zero minor counts
// as a change of sign, the role of LAPACK's pivmin in the ratio form.
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int n, double x, double) {
    const double big = 0x1p+500, small = 0x1p-500;
    double pm = 1.0, p = d[0] - x;
    int cnt = !(p > 0.0);
    if (p == 0.0) p = -small;
    for (int j = 1; j < n; ++j) {
        double q = (d[j] - x) * p - e2[j - 1] * pm;
        if (q == 0.0) q = p > 0.0 ? -small : small;
        cnt += (q > 0.0) != (p > 0.0);
        pm = p;
        p = q;
        const double ap = fabs(p);
        if (ap > big) {
            p *= small;
            pm *= small;
        } else if (ap < small && fabs(pm) < small) {
            p *= big;
            pm *= big;
        }
    }
    return cnt;
}

// e2 = e^2 and the Gershgorin interval, pivmin (one block)
__global__ void tri_prep_kernel(const double* d, const double* e, double* e2, int n, double* info3) {
    __shared__ double lo_s[256], hi_s[256], em_s[256];
    double lo = 1e300, hi = -1e300, em = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double a = j > 0 ? fabs(e[j - 1]) : 0.0, b = j < n - 1 ? fabs(e[j]) : 0.0;
        lo = fmin(lo, d[j] - a - b);
        hi = fmax(hi, d[j] + a + b);
        if (j < n - 1) {
            e2[j] = e[j] * e[j];
            em = fmax(em, e2[j]);
        }
    }
    lo_s[threadIdx.x] = lo;
    hi_s[threadIdx.x] = hi;
    em_s[threadIdx.x] = em;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            lo_s[threadIdx.x] = fmin(lo_s[threadIdx.x], lo_s[threadIdx.x + o]);
            hi_s[threadIdx.x] = fmax(hi_s[threadIdx.x], hi_s[threadIdx.x + o]);
            em_s[threadIdx.x] = fmax(em_s[threadIdx.x], em_s[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double tnorm = fmax(fabs(lo_s[0]), fabs(hi_s[0]));
        const double pad = 2.0 * DBL_EPSILON * tnorm + 1e-300;
        info3[0] = lo_s[0] - pad;
        info3[1] = hi_s[0] + pad;
        info3[2] = fmax(1e-300, DBL_MIN * fmax(1.0, em_s[0]));  // pivmin
        info3[3] = tnorm;
    }
}

// eigenvalue k (ascending) of T, one warp per index: 31 interior points of the
// bracket per round, each round narrowing it 32-fold
__global__ void tri_bisect_kernel(const double* d, const double* e2, int n, int m, const double* info3, double* w) {
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= m) return;
    double a = info3[0], b = info3[1];
    const double pivmin = info3[2];
    for (int round = 0; round < 24; ++round) {
        const double tol = 2.0 * DBL_EPSILON * fmax(fabs(a), fabs(b)) + 2.0 * pivmin;
        if (b - a <= tol) break;
        const double x = a + (b - a) * (double)(lane + 1) * (1.0 / 32.0);
        const int cnt = lane < 31 ? sturm_count(d, e2, n, x, pivmin) : n + 1;
        // the first point whose count exceeds k bounds eigenvalue k from above
        const unsigned int above = __ballot_sync(0xffffffffu, cnt > k);
        const int f = __ffs(above) - 1;  // lane 31 always qualifies
        const double nb_ = a + (b - a) * (double)(f + 1) * (1.0 / 32.0);
        const double na_ = f > 0 ? a + (b - a) * (double)f * (1.0 / 32.0) : a;
        a = na_;
        b = f < 31 ? nb_ : b;
    }
    if (lane == 0) w[k] = 0.5 * (a + b);
}

// ------------------------------------------------------------------ tridiagonal eigenvectors
// Inverse iteration for the clusters of w (ascending), one warp (block) per
// index: the block of index k0 starts a cluster when w[k0] - w[k0 - 1] >
// 1e-10 ||T|| and computes the cluster's vectors in order, each made
// orthogonal to the cluster's earlier ones.  An eigenvector from inverse
// iteration is accurate to about eps ||T|| / gap, so vectors outside a cluster
// are orthogonal to 1e-6 or better; eigenvalues closer than that (the E +- d
// pairs of the folded spectrum, an orthonormal block's unit eigenvalues) share
// a cluster.  Lane 0 runs the elimination and the substitutions (sequential in
// the position) on shared-memory copies of T, of the factors and of the
// vector; all lanes run the Gram-Schmidt steps and the norms.  z: [n][m] real
// (position-major).  Dynamic shared memory: 8 n doubles.
__global__ void __launch_bounds__(32) tri_invit_kernel(const double* d, const double* e, int n, int m,
                                                       const double* w, const double* info3, double* z) {
    extern __shared__ __align__(16) double tsm[];
    double* dd = tsm;          // diagonal of T
    double* ee = dd + n;       // off-diagonal of T (ee[n - 1] = 0)
    double* ri = ee + n;       // pivot of row i of U
    double* u1 = ri + n;       // first and second super-diagonals of U
    double* u2 = u1 + n;
    double* mu = u2 + n;       // multipliers
    double* sw = mu + n;       // 1 where rows i and i + 1 were swapped
    double* zv = sw + n;       // the vector being iterated
    const int k0 = blockIdx.x;
    const int lane = threadIdx.x;
    if (k0 >= m) return;
    const double tnorm = fmax(info3[3], 1e-300);
    const double ctol = 1e-10 * tnorm;
    if (k0 > 0 && w[k0] - w[k0 - 1] <= ctol) return;  // not a cluster start (block-uniform)
    int k1 = k0 + 1;
    while (k1 < m && w[k1] - w[k1 - 1] <= ctol) ++k1;
    for (int i = lane; i < n; i += 32) {
        dd[i] = d[i];
        ee[i] = i < n - 1 ? e[i] : 0.0;
    }
    __syncwarp();
#define ZV(q, i) z[(long)(i) * m + (q)]
    const double sep = 10.0 * DBL_EPSILON * tnorm;
    double lam_prev = -1e300;
    for (int k = k0; k < k1; ++k) {
        double lam = w[k];
        if (lam - lam_prev < sep) lam = lam_prev + sep;  // separate equal eigenvalues of a cluster
        lam_prev = lam;
        if (lane == 0) {
            // elimination with partial pivoting of T - lam I: U rows (pivot, u1, u2), multipliers, swaps
            double p0 = dd[0] - lam, p1 = n > 1 ? ee[0] : 0.0, p2 = 0.0;
            for (int i = 0; i < n - 1; ++i) {
                const double sv = ee[i], a = dd[i + 1] - lam, t = ee[i + 1];
                if (fabs(p0) >= fabs(sv)) {
                    if (p0 == 0.0) p0 = sep;
                    const double f = sv / p0;
                    ri[i] = p0; u1[i] = p1; u2[i] = p2; mu[i] = f; sw[i] = 0.0;
                    p0 = a - f * p1;
                    p1 = t - f * p2;
                    p2 = 0.0;
                } else {
                    const double f = p0 / sv;
                    ri[i] = sv; u1[i] = a; u2[i] = t; mu[i] = f; sw[i] = 1.0;
                    p0 = p1 - f * a;
                    p1 = p2 - f * t;
                    p2 = 0.0;
                }
            }
            ri[n - 1] = p0 == 0.0 ? sep : p0;
            for (int i = 0; i < n - 1; ++i) {
                const double u = ri[i];
                if (fabs(u) < sep) ri[i] = u < 0 ? -sep : sep;
            }
            // start vector: a fixed pseudo-random sequence per index
            unsigned int st = 2654435761u * (unsigned int)(k + 1) + 12345u;
            for (int i = 0; i < n; ++i) {
                st = st * 1664525u + 1013904223u;
                zv[i] = 0.5 + (double)(st >> 8) * (1.0 / 16777216.0);
            }
        }
        __syncwarp();
        for (int it = 0; it < 4; ++it) {
            if (lane == 0) {
                // forward: apply the row operations
                double xi = zv[0];
                for (int i = 0; i < n - 1; ++i) {
                    const double xn = zv[i + 1];
                    if (sw[i] != 0.0) {
                        zv[i] = xn;
                        xi = xi - mu[i] * xn;
                    } else {
                        zv[i] = xi;
                        xi = xn - mu[i] * xi;
                    }
                }
                zv[n - 1] = xi;
                // back substitution with the three diagonals of U
                double x2 = 0.0, x1 = zv[n - 1] / ri[n - 1];
                zv[n - 1] = x1;
                for (int i = n - 2; i >= 0; --i) {
                    const double x0 = (zv[i] - u1[i] * x1 - u2[i] * x2) / ri[i];
                    zv[i] = x0;
                    x2 = x1;
                    x1 = x0;
                }
            }
            __syncwarp();
            // orthogonalise against the cluster's earlier vectors (warp-parallel), normalise
            for (int q = k0; q < k; ++q) {
                double dot = 0;
                for (int i = lane; i < n; i += 32) dot += ZV(q, i) * zv[i];
                for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
                for (int i = lane; i < n; i += 32) zv[i] -= dot * ZV(q, i);
                __syncwarp();
            }
            double nrm = 0;
            for (int i = lane; i < n; i += 32) nrm += zv[i] * zv[i];
            for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
            const double inv = nrm > 0 ? 1.0 / sqrt(nrm) : 1.0;
            for (int i = lane; i < n; i += 32) zv[i] *= inv;
            __syncwarp();
        }
        for (int i = lane; i < n; i += 32) ZV(k, i) = zv[i];
        __syncwarp();
    }
#undef ZV
}

// ------------------------------------------------------------------ back-transformation
// Z = Q z with Q = H_0 ... H_{n-2}, applied in blocks of NBLK reflectors from
// the last block to the first: Q_b = H_j0 ... H_j1-1 = I - V_b T_b V_b^H
// (compact WY form; T_b upper triangular, T_jj = tau_j,
// T[0:j, j] = -tau_j T[0:j, 0:j] (V_b^H v_j)[0:j]), Z <- Z - V_b (T_b (V_b^H Z)).

// z (position-major [n][m], real) -> Z (column-major, complex)
__global__ void tri_z_to_Z_kernel(int n, int m, const double* z, double2* Z, int ldz) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * m) return;
    const int i = (int)(t % n), j = (int)(t / n);
    Z[i + (long)j * ldz] = make_double2(z[(long)i * m + j], 0.0);
}

// T_b of every block of reflectors at once: block b (reflectors j0 = b NBLK ..)
// forms G = V_b^H V_b (rows j0 + 1 .. n - 1) and then T_b column by column;
// T_b goes to T + b NBLK NBLK (ld NBLK).
__global__ void __launch_bounds__(256) wy_t_kernel(int n, const double2* V, const double2* tau, double2* T) {
    __shared__ double2 Ts[NBLK][NBLK + 1];
    __shared__ double2 Gs[NBLK][NBLK + 1];
    __shared__ double2 ts[NBLK];
    const int j0 = blockIdx.x * NBLK, nbk = min(NBLK, n - 1 - j0), r0 = j0 + 1;
    const double2* Vb = V + (long)j0 * n;
    // G[p][q] = sum_rows conj(V[row][j0 + p]) V[row][j0 + q]: a warp per (p, q) entry
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int e = wp; e < nbk * nbk; e += 8) {
        const int p = e % nbk, q = e / nbk;
        double2 acc = make_double2(0.0, 0.0);
        for (int row = r0 + lane; row < n; row += 32)
            acc = cadd(acc, cmulc(Vb[row + (long)p * n], Vb[row + (long)q * n]));
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) Gs[p][q] = acc;
    }
    if (threadIdx.x < nbk) ts[threadIdx.x] = tau[j0 + threadIdx.x];
    __syncthreads();
    T += (size_t)blockIdx.x * NBLK * NBLK;
    const int r = threadIdx.x;
    for (int j = 0; j < nbk; ++j) {
        // column j: T[r][j] = -tau_j sum_{q<j} T[r][q] G[q][j] for r < j; T[j][j] = tau_j
        double2 v = make_double2(0.0, 0.0);
        if (r < j) {
            for (int q = r; q < j; ++q) v = cadd(v, cmul(Ts[r][q], Gs[q][j]));
            v = cmul(make_double2(-ts[j].x, -ts[j].y), v);
        } else if (r == j) {
            v = ts[j];
        }
        __syncthreads();
        if (r < nbk) Ts[r][j] = v;
        __syncthreads();
    }
    for (int j = 0; j < nbk; ++j)
        if (r < nbk) T[r + (long)j * nbk] = r <= j ? Ts[r][j] : make_double2(0.0, 0.0);
}


inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

// C = alpha sum_z P[z] + beta C, z in order
__global__ void gemm_sum_kernel(int M, int N, int splits, const double2* P, double alpha, double beta, double2* C,
                                int ldc, int lower) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)M * N) return;
    const int r = (int)(t % M), col = (int)(t / M);
    if (lower && (r / TB + 1) * TB <= (col / TB) * TB) return;  // a tile the GEMM skipped
    double2 s = P[t];
    for (int z = 1; z < splits; ++z) s = cadd(s, P[(size_t)z * M * N + t]);
    double2* c = C + r + (long)col * ldc;
    double2 o = make_double2(alpha * s.x, alpha * s.y);
    if (beta != 0.0) {
        o.x += beta * c->x;
        o.y += beta * c->y;
    }
    *c = o;
}

}  // namespace

// ------------------------------------------------------------------ host side
// C = alpha op(A) op(B) + beta C; when the output has few tiles and K is long,
// K is split over the grid's z dimension into partial products that a second
// kernel adds in a fixed order (deterministic).
namespace {
void dense_gemm_impl(fs_ctx* c, int opA, int opB, int M, int N, int K, double alpha, const double2* A, int lda,
                     const double2* B, int ldb, double beta, double2* C, int ldc, int lower) {
    if (M <= 0 || N <= 0) return;
    K = std::max(K, 0);
    const int tiles = cdiv(M, TB) * cdiv(N, TB);
    int splits = 1;
    if (tiles < 152 && K >= 8 * TK) splits = std::min(std::max(1, 304 / tiles), std::max(1, K / (4 * TK)));
    if (splits <= 1) {
        dim3 g(cdiv(M, TB), cdiv(N, TB));
        zgemm_kernel<<<g, 256, 0, c->stream>>>(M, N, K, opA, opB, alpha, A, lda, B, ldb, beta, C, ldc, K, lower);
        FS_CUDA(cudaGetLastError());
        return;
    }
    const int kc = cdiv(cdiv(K, splits), TK) * TK;
    splits = cdiv(K, kc);
    DenseWork& D = c->dense;
    D.gpart.ensure((size_t)splits * M * N * sizeof(double2));
    double2* P = D.gpart.as<double2>();
    dim3 g(cdiv(M, TB), cdiv(N, TB), splits);
    zgemm_kernel<<<g, 256, 0, c->stream>>>(M, N, K, opA, opB, 1.0, A, lda, B, ldb, 0.0, P, M, kc, lower);
    gemm_sum_kernel<<<cdiv((long)M * N, 256), 256, 0, c->stream>>>(M, N, splits, P, alpha, beta, C, ldc, lower);
    FS_CUDA(cudaGetLastError());
}
}  // namespace

void dense_gemm(fs_ctx* c, int opA, int opB, int M, int N, int K, double alpha, const double2* A, int lda,
                const double2* B, int ldb, double beta, double2* C, int ldc) {
    dense_gemm_impl(c, opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 0);
}

// Cholesky of the lower triangle of A (n x n, ld lda); squared pivots to piv
// (device, may be null).  Returns the LAPACK info (0, or the first failing
// column + 1).  Synchronises the context's stream.
int dense_potrf(fs_ctx* c, int n, double2* A, int lda, double* piv) {
    ProfScope ps(c, KS_SUB_POTRF, 0.0, 8.0 * n * (double)n * n / 3.0);
    DenseWork& D = c->dense;
    D.info.ensure(sizeof(int));
    int* info = D.info.as<int>();
    FS_CUDA(cudaMemsetAsync(info, 0, sizeof(int), c->stream));
    for (int j0 = 0; j0 < n; j0 += NBLK) {
        const int b = std::min(NBLK, n - j0);
        potrf_diag_kernel<<<1, NBLK * NBLK, 0, c->stream>>>(A, lda, j0, b, piv, info);
        const int rest = n - j0 - b;
        if (rest > 0) {
            potrf_panel_kernel<<<cdiv((long)rest * 32, 256), 256, 0, c->stream>>>(A, lda, n, j0, b);
            // trailing update of the lower triangle (the upper one is never read)
            dense_gemm_impl(c, 0, 1, rest, rest, b, -1.0, A + j0 + b + (long)j0 * lda, lda,
                            A + j0 + b + (long)j0 * lda, lda, 1.0, A + j0 + b + (long)(j0 + b) * lda, lda, 1);
        }
    }
    FS_CUDA(cudaGetLastError());
    int h = 0;
    FS_CUDA(cudaMemcpyAsync(&h, info, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return h;
}

// B <- L^-1 B (conj = 0) or L^-H B (conj = 1); L lower n x n (ld lda), B n x ncols (ld ldb)
void dense_trsm(fs_ctx* c, int conj, int n, int ncols, const double2* L, int lda, double2* B, int ldb) {
    if (n <= 0 || ncols <= 0) return;
    ProfScope ps(c, KS_SUB_TRSM, 0.0, 4.0 * n * (double)n * ncols);
    const int nblk = cdiv(n, NBLK);
    for (int q = 0; q < nblk; ++q) {
        const int bi = conj ? nblk - 1 - q : q;
        const int j0 = bi * NBLK, b = std::min(NBLK, n - j0);
        trsm_diag_kernel<<<cdiv((long)ncols * 32, 256), 256, 0, c->stream>>>(L, lda, j0, b, B, ldb, ncols, conj);
        if (!conj) {
            const int rest = n - j0 - b;
            if (rest > 0)
                dense_gemm(c, 0, 0, rest, ncols, b, -1.0, L + j0 + b + (long)j0 * lda, lda, B + j0, ldb, 1.0,
                           B + j0 + b, ldb);
        } else if (j0 > 0) {
            // B[0:j0] -= (L[j0:j0+b, 0:j0])^H X_b
            dense_gemm(c, 1, 0, j0, ncols, b, -1.0, L + j0, lda, B + j0, ldb, 1.0, B, ldb);
        }
    }
    FS_CUDA(cudaGetLastError());
}

void dense_conj_transpose(fs_ctx* c, int n, int m, const double2* A, int lda, double2* out, int ldo) {
    conj_transpose_kernel<<<cdiv((long)n * m, 256), 256, 0, c->stream>>>(n, m, A, lda, out, ldo);
    FS_CUDA(cudaGetLastError());
}

// The m lowest eigenpairs of the Hermitian A (n x n, ld n, destroyed): w[0..m)
// ascending (device), Z (n x m, ld ldz, device) orthonormal eigenvectors.
void dense_heev(fs_ctx* c, int n, double2* A, int m, double* w, double2* Z, int ldz) {
    if (n <= 0 || m <= 0) return;
    if (n > FS_DENSE_MAX_N) throw fs_error(FS_ERR_ARG, "dense eigensolve larger than " + std::to_string(FS_DENSE_MAX_N));
    DenseWork& D = c->dense;
    D.V.ensure((size_t)n * n * sizeof(double2));
    D.tau.ensure((size_t)n * sizeof(double2));
    D.d.ensure((size_t)n * sizeof(double));
    D.e.ensure((size_t)n * sizeof(double));
    D.e2.ensure((size_t)n * sizeof(double));
    D.Y.ensure((size_t)((n + SEG - 1) / SEG) * n * sizeof(double2));
    D.z.ensure((size_t)n * m * sizeof(double));
    D.info3.ensure(4 * sizeof(double));
    D.bar.ensure(2 * sizeof(unsigned int));
    int dev = 0, nsm = 0;
    FS_CUDA(cudaGetDevice(&dev));
    FS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = (size_t)3 * n * sizeof(double2);
    if (!D.attr_set) {
        FS_CUDA(cudaFuncSetAttribute((const void*)hetrd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     3 * FS_DENSE_MAX_N * (int)sizeof(double2)));
        FS_CUDA(cudaFuncSetAttribute((const void*)tri_invit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     8 * FS_DENSE_MAX_N * (int)sizeof(double)));
        D.attr_set = true;
    }
    int per_sm = 0;
    FS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hetrd_kernel, 256, smem));
    // enough warps for the (column, segment) units, at most one block per SM
    const int nblocks = std::max(1, std::min({nsm, nsm * std::max(per_sm, 1), (n + 3) / 4}));
    {
    ProfScope ps_h(c, KS_SUB_HETRD, 0.0, 16.0 * n * (double)n * n / 3.0);
    hermitize_kernel<<<cdiv((long)n * n, 256), 256, 0, c->stream>>>(A, n);
    FS_CUDA(cudaMemsetAsync(D.bar.p, 0, 2 * sizeof(unsigned int), c->stream));
    FS_CUDA(cudaMemsetAsync(D.V.p, 0, (size_t)n * n * sizeof(double2), c->stream));
    {
        int nn = n;
        double2* Ap = A;
        double2* Vp = D.V.as<double2>();
        double2* tp = D.tau.as<double2>();
        double* dp = D.d.as<double>();
        double* ep = D.e.as<double>();
        double2* Yp = D.Y.as<double2>();
        unsigned int* bp = D.bar.as<unsigned int>();
        int* errp = ctx_errflag(c);
        void* args[] = {&nn, &Ap, &Vp, &tp, &dp, &ep, &Yp, &bp, &errp};
        FS_CUDA(cudaLaunchCooperativeKernel((const void*)hetrd_kernel, nblocks, 256, args, smem, c->stream));
    }
    if (n == 1) {
        // no reflector: T = A
        FS_CUDA(cudaMemsetAsync(D.tau.p, 0, sizeof(double2), c->stream));
    }
    }
    {
    ProfScope ps_t(c, KS_SUB_TRIEIG, 0.0, 0.0);
    tri_prep_kernel<<<1, 256, 0, c->stream>>>(D.d.as<double>(), D.e.as<double>(), D.e2.as<double>(), n,
                                              D.info3.as<double>());
    tri_bisect_kernel<<<m, 32, 0, c->stream>>>(D.d.as<double>(), D.e2.as<double>(), n, m,
                                                                      D.info3.as<double>(), w);
    tri_invit_kernel<<<m, 32, (size_t)8 * n * sizeof(double), c->stream>>>(D.d.as<double>(), D.e.as<double>(), n, m,
                                                                           w, D.info3.as<double>(), D.z.as<double>());
    tri_z_to_Z_kernel<<<cdiv((long)n * m, 256), 256, 0, c->stream>>>(n, m, D.z.as<double>(), Z, ldz);
    FS_CUDA(cudaGetLastError());
    }
    if (n > 1) {
        ProfScope ps_b(c, KS_SUB_BACK, 0.0, 8.0 * n * (double)n * m);
        const int nref = n - 1, nblkr = cdiv(nref, NBLK);
        D.wyT.ensure((size_t)nblkr * NBLK * NBLK * sizeof(double2));
        D.wyW.ensure((size_t)NBLK * m * sizeof(double2));
        D.wyW2.ensure((size_t)NBLK * m * sizeof(double2));
        double2* W = D.wyW.as<double2>();
        double2* W2 = D.wyW2.as<double2>();
        const double2* V = D.V.as<double2>();
        wy_t_kernel<<<nblkr, 256, 0, c->stream>>>(n, V, D.tau.as<double2>(), D.wyT.as<double2>());
        for (int b = nblkr - 1; b >= 0; --b) {
            const int j0 = b * NBLK, nbk = std::min(NBLK, nref - j0);
            const int r0 = j0 + 1, rows = n - r0;  // v_j0 starts at row j0 + 1
            const double2* Vb = V + r0 + (long)j0 * n;
            const double2* Tb = D.wyT.as<double2>() + (size_t)b * NBLK * NBLK;
            dense_gemm(c, 1, 0, nbk, m, rows, 1.0, Vb, n, Z + r0, ldz, 0.0, W, nbk);
            dense_gemm(c, 0, 0, nbk, m, nbk, 1.0, Tb, nbk, W, nbk, 0.0, W2, nbk);
            dense_gemm(c, 0, 0, rows, m, nbk, -1.0, Vb, n, W2, nbk, 1.0, Z + r0, ldz);
        }
        FS_CUDA(cudaGetLastError());
    }
    // one Cholesky QR pass: the vectors of eigenvalues outside a common cluster are orthogonal
    // only to about eps ||T|| / gap; their Gram matrix is I + O(that), so Z <- Z L^-H with
    // Z^H Z = L L^H restores orthonormality to working precision (it mixes only nearly
    // degenerate vectors)
    if (m > 1) {
        D.qrG.ensure((size_t)m * m * sizeof(double2));
        D.qrT.ensure((size_t)m * n * sizeof(double2));
        double2* G = D.qrG.as<double2>();
        double2* T = D.qrT.as<double2>();
        dense_gemm(c, 1, 0, m, m, n, 1.0, Z, ldz, Z, ldz, 0.0, G, m);
        if (dense_potrf(c, m, G, m, nullptr) == 0) {
            dense_conj_transpose(c, n, m, Z, ldz, T, m);
            dense_trsm(c, 0, m, n, G, m, T, m);
            dense_conj_transpose(c, m, n, T, m, Z, ldz);
        }
    }
    ctx_check_errflag(c);
}

// Generalised Hermitian problem GA x = lambda GB x (both n x n, ld n; GB positive
// definite): the m lowest pairs; eigenvectors (GB-orthonormal) overwrite GA's
// first m columns, eigenvalues to w.  GB is overwritten by its Cholesky factor.
// Returns the Cholesky info (0 = success).
int dense_hegv(fs_ctx* c, int n, double2* GA, double2* GB, int m, double* w) {
    int info = dense_potrf(c, n, GB, n, nullptr);
    if (info != 0) return info;
    DenseWork& D = c->dense;
    D.T.ensure((size_t)n * n * sizeof(double2));
    D.U.ensure((size_t)n * m * sizeof(double2));
    double2* T = D.T.as<double2>();
    dense_trsm(c, 0, n, n, GB, n, GA, n);              // L^-1 GA
    dense_conj_transpose(c, n, n, GA, n, T, n);         // (L^-1 GA)^H = GA L^-H
    dense_trsm(c, 0, n, n, GB, n, T, n);               // L^-1 GA L^-H
    dense_heev(c, n, T, m, w, D.U.as<double2>(), n);
    dense_trsm(c, 1, n, m, GB, n, D.U.as<double2>(), n);  // x = L^-H y
    FS_CUDA(cudaMemcpyAsync(GA, D.U.p, (size_t)n * m * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    return 0;
}

// ------------------------------------------------------------------ C ABI (checking the dense solvers)
extern "C" fs_status fs_dense_eigh(fs_ctx* c, int n, const void* A, const void* B, int m, double* w, void* Z) {
    if (!c) return FS_ERR_ARG;
    if (n <= 0 || n > FS_DENSE_MAX_N || m <= 0 || m > n || !A || !w || !Z) {
        c->err = "fs_dense_eigh: bad arguments";
        return FS_ERR_ARG;
    }
    try {
        const size_t bytes = (size_t)n * n * sizeof(double2);
        dbuf dA, dB, dZ, dw;
        dA.alloc(bytes);
        dZ.alloc((size_t)n * m * sizeof(double2));
        dw.alloc((size_t)n * sizeof(double));
        FS_CUDA(cudaMemcpyAsync(dA.p, A, bytes, cudaMemcpyHostToDevice, c->stream));
        if (B) {
            dB.alloc(bytes);
            FS_CUDA(cudaMemcpyAsync(dB.p, B, bytes, cudaMemcpyHostToDevice, c->stream));
            const int info = dense_hegv(c, n, dA.as<double2>(), dB.as<double2>(), m, dw.as<double>());
            if (info != 0) throw fs_error(FS_ERR_NUMERIC, "fs_dense_eigh: B is not positive definite (column " +
                                                              std::to_string(info) + ")");
            FS_CUDA(cudaMemcpyAsync(dZ.p, dA.p, (size_t)n * m * sizeof(double2), cudaMemcpyDeviceToDevice,
                                    c->stream));
        } else {
            dense_heev(c, n, dA.as<double2>(), m, dw.as<double>(), dZ.as<double2>(), n);
        }
        FS_CUDA(cudaMemcpyAsync(w, dw.p, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaMemcpyAsync(Z, dZ.p, (size_t)n * m * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        ctx_check_errflag(c);
        c->err.clear();
        return FS_OK;
    } catch (const fs_error& e) {
        c->err = e.msg;
        return e.code;
    }
}
