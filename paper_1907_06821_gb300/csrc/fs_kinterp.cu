// Wave-function interpolation between two k-points (paper Sec. II.D).
//
// With orthonormal eigenpairs (eps_i(k1), psi_i(k1)), i < n1, and
// (eps_l(k2), psi_l(k2)), l < n2, of two nearby k-points, H(k) between them is
// taken as alpha H(k1) + (1 - alpha) H(k2); in the basis psi_i(k1) its matrix is
//     H_ij(k) = alpha eps_i(k1) delta_ij + (1 - alpha) sum_m U*_im U_jm eps_m(k2),
// with U the rows of the overlap S_il = <psi_l(k2)|psi_i(k1)> made orthonormal
// by Gram-Schmidt in index order.  Its eigenpairs give eps(k) and
//     psi_q(k) = alpha sum_j C_jq psi_j(k1) + (1 - alpha) sum_{j,l} C_jq U_jl psi_l(k2).
// The Gram-Schmidt process in row order is U = L^-1 S with S S^H = L L^H
// (L lower triangular, positive diagonal): a Cholesky QR of the rows, taken
// twice for orthogonality to working precision.  Every product is a dense FP64
// GEMM on the device; the eigensolve is the library's dense eigensolver.
#include "fs_common.cuh"

#include <algorithm>
#include <cmath>

namespace {

// rows m of Q (n2 x n1 column-major) times w[m]
__global__ void scale_rows_kernel(const double2* Q, const double* w, int n2, int n1, double2* out) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n2 * n1) return;
    const int m = (int)(t % n2);
    out[t] = make_double2(Q[t].x * w[m], Q[t].y * w[m]);
}

__global__ void add_diag_kernel(double2* H, int n, const double* e, double a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) H[i + (long)i * n].x += a * e[i];
}

inline int nblk(long t) { return (int)((t + 255) / 256); }

// One Cholesky QR pass on the columns of Q (n2 x n1, column-major): Q <- Q L^-H
// with Q^H Q = L L^H; work: G (n1 x n1), T (n1 x n2).  Returns the Cholesky info.
int chol_qr(fs_ctx* c, int n2, int n1, double2* Q, double2* G, double2* T) {
    dense_gemm(c, 1, 0, n1, n1, n2, 1.0, Q, n2, Q, n2, 0.0, G, n1);
    const int info = dense_potrf(c, n1, G, n1, nullptr);
    if (info != 0) return info;
    dense_conj_transpose(c, n2, n1, Q, n2, T, n1);   // Q^H (n1 x n2)
    dense_trsm(c, 0, n1, n2, G, n1, T, n1);          // L^-1 Q^H = (Q L^-H)^H
    dense_conj_transpose(c, n1, n2, T, n1, Q, n2);
    return 0;
}

}  // namespace

extern "C" fs_status fs_kinterp(fs_ctx* c, double alpha, int n1, const double* eps1, const void* psi1, int n2,
                                const double* eps2, const void* psi2, double* eps, void* psi) {
    if (!c) return FS_ERR_ARG;
    if (n1 <= 0 || n2 < n1 || n1 > FS_DENSE_MAX_N || !eps1 || !eps2 || !psi1 || !psi2 || !eps || !psi ||
        !std::isfinite(alpha)) {
        c->err = "fs_kinterp: bad arguments (need 0 < n1 <= n2, n1 <= 2048)";
        return FS_ERR_ARG;
    }
    try {
        const long N = c->npw;
        const double2* P1 = static_cast<const double2*>(psi1);  // column-major N x n1 (rows of [n1][npw])
        const double2* P2 = static_cast<const double2*>(psi2);
        double2* Out = static_cast<double2*>(psi);
        dbuf Q, G, T, Hk, C, M2, dw, de1, de2;
        Q.alloc((size_t)n2 * n1 * sizeof(double2));
        G.alloc((size_t)n1 * n1 * sizeof(double2));
        T.alloc((size_t)n1 * n2 * sizeof(double2));
        Hk.alloc((size_t)n1 * n1 * sizeof(double2));
        C.alloc((size_t)n1 * n1 * sizeof(double2));
        M2.alloc((size_t)n2 * n1 * sizeof(double2));
        dw.alloc((size_t)n1 * sizeof(double));
        de1.alloc((size_t)n1 * sizeof(double));
        de2.alloc((size_t)n2 * sizeof(double));
        FS_CUDA(cudaMemcpyAsync(de1.p, eps1, n1 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        FS_CUDA(cudaMemcpyAsync(de2.p, eps2, n2 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        // S^T (n2 x n1): column i = the components of psi_i(k1) on the psi_l(k2), i.e. row i of S
        dense_gemm(c, 1, 0, n2, n1, (int)N, 1.0, P2, (int)N, P1, (int)N, 0.0, Q.as<double2>(), n2);
        // Gram-Schmidt of the rows of S in index order (two Cholesky QR passes): Q = U^T
        for (int pass = 0; pass < 2; ++pass) {
            const int info = chol_qr(c, n2, n1, Q.as<double2>(), G.as<double2>(), T.as<double2>());
            if (info != 0)
                throw fs_error(FS_ERR_NUMERIC, "fs_kinterp: the overlap is rank deficient (row " +
                                                   std::to_string(info) + ")");
        }
        // H_ij(k) = (1 - alpha) (Q^H diag(eps2) Q)_ij + alpha eps1_i delta_ij
        scale_rows_kernel<<<nblk((long)n2 * n1), 256, 0, c->stream>>>(Q.as<double2>(), de2.as<double>(), n2, n1,
                                                                       M2.as<double2>());
        dense_gemm(c, 1, 0, n1, n1, n2, 1.0 - alpha, Q.as<double2>(), n2, M2.as<double2>(), n2, 0.0,
                   Hk.as<double2>(), n1);
        add_diag_kernel<<<nblk(n1), 256, 0, c->stream>>>(Hk.as<double2>(), n1, de1.as<double>(), alpha);
        FS_CUDA(cudaGetLastError());
        dense_heev(c, n1, Hk.as<double2>(), n1, dw.as<double>(), C.as<double2>(), n1);
        // psi = alpha P1 C + (1 - alpha) P2 (U^T C),  U^T = Q
        dense_gemm(c, 0, 0, n2, n1, n1, 1.0, Q.as<double2>(), n2, C.as<double2>(), n1, 0.0, M2.as<double2>(), n2);
        dense_gemm(c, 0, 0, (int)N, n1, n1, alpha, P1, (int)N, C.as<double2>(), n1, 0.0, Out, (int)N);
        dense_gemm(c, 0, 0, (int)N, n1, n2, 1.0 - alpha, P2, (int)N, M2.as<double2>(), n2, 1.0, Out, (int)N);
        FS_CUDA(cudaMemcpyAsync(eps, dw.p, n1 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        ctx_check_errflag(c);
        c->err.clear();
        return FS_OK;
    } catch (const fs_error& e) {
        c->err = e.msg;
        return e.code;
    }
}
