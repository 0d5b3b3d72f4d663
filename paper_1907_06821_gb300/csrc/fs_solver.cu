// Folded-spectrum all-band PCG (locally optimal block form) on the GPU.
//
// Operator A = (H - E)^2 (paper Sec. II.C, Eq. wl1); its lowest eigenvectors
// are the eigenvectors of H nearest E.  Per iteration, for the m bands X with
// Y = (H-E)X, Z = AX (all kept on the device):
//   r_i  = || y_i - <x_i,y_i> x_i ||              H residual (convergence test)
//   act  = bands with r_i > tol                    (soft locking)
//   W    = M (Z - X Theta) on act, W -= X (X^H W), rows normalised
//   YW   = (H-E) W, ZW = (H-E) YW                  two H applications
//   P    = previous directions on act, made orthogonal to X, normalised
//   Rayleigh-Ritz of A on S = [X W P]: G_A c = theta G_B c (FP64, cuSOLVER)
//   X <- S c (lowest m), P <- [W P] c_WP; same for Y and Z by linearity.
// Finally a Rayleigh-Ritz step on H in span X gives eps and the states.
// Mixed precision: the vectors, FFTs and GEMMs run in FP32 with FP64 small
// dense algebra until the FP32 residuals reach tol (or stall); the bands are
// then carried to FP64 and the same iteration continues in FP64 until the
// FP64 residuals reach tol.
#include "fs_common.cuh"

#include <cuComplex.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <numeric>

void ctx_ensure_fp32(fs_ctx* c);

namespace {

template <typename T2> struct Blocks {
    dbuf X, Y, Z, W, YW, ZW, P, YP, ZP, tX, tY, tZ, tP, tYP, tZP;
    bool haveP = false;
    void alloc(int m, long npw) {
        size_t b = (size_t)m * npw * sizeof(T2);
        for (dbuf* d : {&X, &Y, &Z, &W, &YW, &ZW, &P, &YP, &ZP, &tX, &tY, &tZ, &tP, &tYP, &tZP}) d->alloc(b);
        haveP = false;
    }
    void free_all() {
        for (dbuf* d : {&X, &Y, &Z, &W, &YW, &ZW, &P, &YP, &ZP, &tX, &tY, &tZ, &tP, &tYP, &tZP}) d->release();
    }
};

void swapb(dbuf& a, dbuf& b) {
    std::swap(a.p, b.p);
    std::swap(a.bytes, b.bytes);
}

struct Small {
    dbuf GA, GB, T1, T2, evals, work, info, theta, act, resid, dots, nrm, shift, dscale;
    int lwork = 0;
    int nbmax = 0;
};

__global__ void add_diag_kernel(double2* A, int n, double v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) A[(long)i * n + i].x += v;
}

__global__ void shift_kernel(const double* ev, double e, double* out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ev[i] - e;
}

// d_i = 1 / sqrt(Re GB_ii)
__global__ void diag_invsqrt_kernel(const double2* GB, int n, double* d) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        double g = GB[(long)i * n + i].x;
        d[i] = g > 0 ? rsqrt(g) : 0.0;
    }
}

// G_ij *= d_i d_j for both matrices
__global__ void sym_scale_kernel(double2* GA, double2* GB, int n, const double* d) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    int i = (int)(t % n), j = (int)(t / n);
    double f = d[i] * d[j];
    GA[t].x *= f;
    GA[t].y *= f;
    GB[t].x *= f;
    GB[t].y *= f;
}

// column j of T (n x k, ld n) *= 1 / sqrt(lam[j])
__global__ void col_invsqrt_kernel(double2* T, int n, int k, const double* lam) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * k) return;
    int j = (int)(t / n);
    double f = rsqrt(lam[j]);
    T[t].x *= f;
    T[t].y *= f;
}

// row i of C (n x m, ld n) *= d[i]
__global__ void row_scale_kernel(double2* C, int n, int m, const double* d) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * m) return;
    int i = (int)(t % n);
    C[t].x *= d[i];
    C[t].y *= d[i];
}

inline int nblk(long total) { return (int)((total + 255) / 256); }

struct Solver {
    fs_ctx* c;
    double E;
    int nstates, m;
    double tol;
    Small s;
    long long n_hpsi = 0;
    int verbose = 0;

    template <typename T2> void HE(const T2* in, T2* out, int nb, const int* map = nullptr) {
        apply_H_impl<T2>(c, in, out, nb, E, map);
        n_hpsi += nb;
    }

    void ensure_small(int nbmax) {
        if (nbmax <= s.nbmax) return;
        s.nbmax = nbmax;
        s.GA.alloc((size_t)nbmax * nbmax * sizeof(double2));
        s.GB.alloc((size_t)nbmax * nbmax * sizeof(double2));
        s.T1.alloc((size_t)nbmax * nbmax * sizeof(double2));
        s.T2.alloc((size_t)nbmax * nbmax * sizeof(double2));
        s.dscale.alloc(nbmax * sizeof(double));
        s.evals.alloc(nbmax * sizeof(double));
        s.info.alloc(sizeof(int));
        s.theta.alloc(nbmax * sizeof(double));
        s.act.alloc(nbmax * sizeof(int));
        s.resid.alloc(nbmax * sizeof(double));
        s.dots.alloc(nbmax * sizeof(double2));
        s.nrm.alloc(nbmax * sizeof(double));
        s.shift.alloc(nbmax * sizeof(double));
        int lw1 = 0, lw2 = 0;
        FS_SOLVER(cusolverDnZhegvd_bufferSize(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                              CUBLAS_FILL_MODE_LOWER, nbmax, s.GA.as<cuDoubleComplex>(), nbmax,
                                              s.GB.as<cuDoubleComplex>(), nbmax, s.evals.as<double>(), &lw1));
        FS_SOLVER(cusolverDnZheevd_bufferSize(c->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, nbmax,
                                              s.GA.as<cuDoubleComplex>(), nbmax, s.evals.as<double>(), &lw2));
        s.lwork = std::max(lw1, lw2);
        s.work.alloc((size_t)s.lwork * sizeof(cuDoubleComplex));
    }

    // generalized Hermitian eigenproblem GA c = lambda GB c, n x n column-major; returns info
    int hegvd(int n) {
        ProfScope ps(c, KS_DENSE_LA, 0.0, 0.0);
        FS_SOLVER(cusolverDnZhegvd(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                   s.GA.as<cuDoubleComplex>(), n, s.GB.as<cuDoubleComplex>(), n, s.evals.as<double>(),
                                   s.work.as<cuDoubleComplex>(), s.lwork, s.info.as<int>()));
        int info = 0;
        FS_CUDA(cudaMemcpyAsync(&info, s.info.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        return info;
    }
    int heevd(int n, double2* A = nullptr) {
        if (!A) A = s.GA.as<double2>();
        ProfScope ps(c, KS_DENSE_LA, 0.0, 0.0);
        FS_SOLVER(cusolverDnZheevd(c->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                   (cuDoubleComplex*)A, n, s.evals.as<double>(), s.work.as<cuDoubleComplex>(),
                                   s.lwork, s.info.as<int>()));
        int info = 0;
        FS_CUDA(cudaMemcpyAsync(&info, s.info.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        return info;
    }

    // Rayleigh-Ritz of A on a basis of nb vectors with Gram matrices GA = <S, AS>
    // and GB = <S, S> (column-major in s.GA, s.GB).  On return s.GA holds the
    // nb x m coefficients of the m lowest Ritz vectors (column j = vector j)
    // and s.evals[0..m) their Ritz values.  robust = true selects the basis
    // by an eigendecomposition of the diagonally scaled GB, dropping the
    // directions whose eigenvalue is below tau * max (near-dependent vectors
    // in FP32), instead of a Cholesky factorisation of GB.  Returns the
    // cuSOLVER info (0 = success).
    int rr_basis(int nb, bool robust, double tau) {
        double2* GA = s.GA.as<double2>();
        double2* GB = s.GB.as<double2>();
        if (!robust) return hegvd(nb);
        diag_invsqrt_kernel<<<nblk(nb), 256, 0, c->stream>>>(GB, nb, s.dscale.as<double>());
        sym_scale_kernel<<<nblk((long)nb * nb), 256, 0, c->stream>>>(GA, GB, nb, s.dscale.as<double>());
        int info = heevd(nb, GB);
        if (info != 0) return info;
        std::vector<double> lam(nb);
        FS_CUDA(cudaMemcpyAsync(lam.data(), s.evals.p, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        double lmax = lam[nb - 1];
        int k = 0;
        for (int i = nb - 1; i >= 0 && lam[i] > tau * lmax; --i) ++k;
        if (k < m) return -1;
        double2* T = GB + (long)(nb - k) * nb;  // kept eigenvectors, nb x k
        col_invsqrt_kernel<<<nblk((long)nb * k), 256, 0, c->stream>>>(T, nb, k, s.evals.as<double>() + (nb - k));
        const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0);
        double2* tmp = s.T1.as<double2>();
        double2* GAp = s.T2.as<double2>();
        {
        ProfScope ps(c, KS_DENSE_LA, 0.0, 8.0 * nb * (double)nb * k + 8.0 * k * (double)k * nb);
        FS_BLAS(cublasZgemm(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, nb, k, nb, &one, (cuDoubleComplex*)GA, nb,
                            (cuDoubleComplex*)T, nb, &zero, (cuDoubleComplex*)tmp, nb));
        FS_BLAS(cublasZgemm(c->blas, CUBLAS_OP_C, CUBLAS_OP_N, k, k, nb, &one, (cuDoubleComplex*)T, nb,
                            (cuDoubleComplex*)tmp, nb, &zero, (cuDoubleComplex*)GAp, k));
        }
        info = heevd(k, GAp);
        if (info != 0) return info;
        {
        ProfScope ps(c, KS_DENSE_LA, 0.0, 8.0 * nb * (double)m * k);
        FS_BLAS(cublasZgemm(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, nb, m, k, &one, (cuDoubleComplex*)T, nb,
                            (cuDoubleComplex*)GAp, k, &zero, (cuDoubleComplex*)GA, nb));
        }
        row_scale_kernel<<<nblk((long)nb * m), 256, 0, c->stream>>>(GA, nb, m, s.dscale.as<double>());
        FS_CUDA(cudaGetLastError());
        last_kept = k;
        return 0;
    }
    int last_kept = 0;

    template <typename T2> static constexpr bool is_fp32() { return sizeof(T2) == 8; }
    template <typename T2> static double tau_for() { return sizeof(T2) == 8 ? 1e-6 : 1e-11; }

    // Gram matrix of the basis blocks into G (nb x nb column-major): G(i, j) = <S_i, T_j>
    template <typename T2>
    void gram_blocks(double2* G, int nb, const T2* const* S, const T2* const* T, const int* const* maps,
                     const int* sizes, const int* offs, int nblk) {
        for (int I = 0; I < nblk; ++I)
            for (int J = 0; J < nblk; ++J)
                gemm_gram<T2>(c, sizes[I], sizes[J], c->npw, S[I], c->npw, maps[I], T[J], c->npw, maps[J],
                              G + offs[I] + (long)offs[J] * nb, 1, nb, 1.0, 0.0);
    }

    // Initial Rayleigh-Ritz on A in span X (X need not be orthonormal).
    template <typename T2> void init_block(Blocks<T2>& B) {
        T2* X = B.X.template as<T2>();
        T2* Y = B.Y.template as<T2>();
        T2* Z = B.Z.template as<T2>();
        HE(X, Y, m);
        HE(Y, Z, m);
        ensure_small(3 * m);
        double2* GA = s.GA.as<double2>();
        double2* GB = s.GB.as<double2>();
        gemm_gram<T2>(c, m, m, c->npw, Y, c->npw, nullptr, Y, c->npw, nullptr, GA, 1, m, 1.0, 0.0);
        gemm_gram<T2>(c, m, m, c->npw, X, c->npw, nullptr, X, c->npw, nullptr, GB, 1, m, 1.0, 0.0);
        int info = rr_basis(m, is_fp32<T2>(), tau_for<T2>());
        if (info != 0) info = rr_basis(m, true, tau_for<T2>());
        if (info != 0) throw fs_error(FS_ERR_NUMERIC, "start block is rank deficient (info " + std::to_string(info) + ")");
        rotate_simple(B, m);
        FS_CUDA(cudaMemcpyAsync(s.theta.p, s.evals.p, m * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        B.haveP = false;
    }

    // X, Y, Z <- (X, Y, Z) V[:, :m] with V = GA (n x n, column-major)
    template <typename T2> void rotate_simple(Blocks<T2>& B, int n) {
        const double2* V = s.GA.as<double2>();
        dbuf* src[3] = {&B.X, &B.Y, &B.Z};
        dbuf* dst[3] = {&B.tX, &B.tY, &B.tZ};
        for (int q = 0; q < 3; ++q)
            gemm_nn<T2, double2>(c, m, c->npw, n, V, n, 1, src[q]->template as<T2>(), c->npw, nullptr,
                                 dst[q]->template as<T2>(), c->npw, nullptr, 1.0, 0.0, nullptr, 0);
        swapb(B.X, B.tX);
        swapb(B.Y, B.tY);
        swapb(B.Z, B.tZ);
    }

    // Residuals of all bands; returns them on the host.
    template <typename T2> std::vector<double> residuals(Blocks<T2>& B) {
        vec_resid<T2>(c, B.X.template as<T2>(), B.Y.template as<T2>(), m, s.resid.as<double>(),
                      s.dots.as<double2>());
        std::vector<double> r(m);
        FS_CUDA(cudaMemcpyAsync(r.data(), s.resid.p, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        ctx_check_errflag(c);
        prof_flush(c);
        return r;
    }

    // One block iteration on the active set; returns false if the basis broke down.
    template <typename T2> void iterate(Blocks<T2>& B, const std::vector<int>& act_h) {
        const int na = (int)act_h.size();
        const long npw = c->npw;
        int* act = s.act.as<int>();
        FS_CUDA(cudaMemcpyAsync(act, act_h.data(), na * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        T2 *X = B.X.template as<T2>(), *Y = B.Y.template as<T2>(), *Z = B.Z.template as<T2>();
        T2 *W = B.W.template as<T2>(), *YW = B.YW.template as<T2>(), *ZW = B.ZW.template as<T2>();
        T2 *P = B.P.template as<T2>(), *YP = B.YP.template as<T2>(), *ZP = B.ZP.template as<T2>();
        double2* GA = s.GA.as<double2>();
        double2* GB = s.GB.as<double2>();
        // W = M (Z - X Theta), made orthogonal to X and normalised
        vec_make_w<T2>(c, X, Z, s.theta.as<double>(), act, na, W, E, c->opt.dE,
                       c->opt.precond == FS_PREC_TETER ? 1 : 0, nullptr);
        gemm_gram<T2>(c, m, na, npw, X, npw, nullptr, W, npw, nullptr, GB, 1, m, 1.0, 0.0);
        gemm_nn<T2, double2>(c, na, npw, m, GB, m, 1, X, npw, nullptr, W, npw, nullptr, -1.0, 1.0, W, npw);
        vec_row_norms<T2>(c, W, nullptr, na, s.nrm.as<double>());
        vec_scale_rows<T2>(c, W, nullptr, na, s.nrm.as<double>());
        HE(W, YW, na);
        HE(YW, ZW, na);
        bool useP = B.haveP;
        if (useP) {
            // P[act] -= X (X^H P[act]); same combination for YP, ZP; then normalise
            gemm_gram<T2>(c, m, na, npw, X, npw, nullptr, P, npw, act, GB, 1, m, 1.0, 0.0);
            gemm_nn<T2, double2>(c, na, npw, m, GB, m, 1, X, npw, nullptr, P, npw, act, -1.0, 1.0, P, npw);
            gemm_nn<T2, double2>(c, na, npw, m, GB, m, 1, Y, npw, nullptr, YP, npw, act, -1.0, 1.0, YP, npw);
            gemm_nn<T2, double2>(c, na, npw, m, GB, m, 1, Z, npw, nullptr, ZP, npw, act, -1.0, 1.0, ZP, npw);
            vec_row_norms<T2>(c, P, act, na, s.nrm.as<double>());
            vec_scale_rows<T2>(c, P, act, na, s.nrm.as<double>());
            vec_scale_rows<T2>(c, YP, act, na, s.nrm.as<double>());
            vec_scale_rows<T2>(c, ZP, act, na, s.nrm.as<double>());
        }
        for (int attempt = 0; attempt < 2; ++attempt) {
            int nblk = useP ? 3 : 2;
            const T2* S[3] = {X, W, P};
            const T2* SZ[3] = {Z, ZW, ZP};
            const int* maps[3] = {nullptr, nullptr, act};
            int sizes[3] = {m, na, na};
            int offs[3] = {0, m, m + na};
            int nb = m + na + (useP ? na : 0);
            gram_blocks<T2>(GA, nb, S, SZ, maps, sizes, offs, nblk);
            gram_blocks<T2>(GB, nb, S, S, maps, sizes, offs, nblk);
            int info = rr_basis(nb, is_fp32<T2>(), tau_for<T2>());
            if (info != 0 && !is_fp32<T2>()) {
                gram_blocks<T2>(GA, nb, S, SZ, maps, sizes, offs, nblk);
                gram_blocks<T2>(GB, nb, S, S, maps, sizes, offs, nblk);
                info = rr_basis(nb, true, tau_for<T2>());
            }
            if (info != 0) {
                if (useP) {
                    useP = false;
                    continue;
                }
                throw fs_error(FS_ERR_NUMERIC, "Rayleigh-Ritz basis is not positive definite (info " +
                                                   std::to_string(info) + ")");
            }
            // rotation: Pn = W Vw + P Vp ; Xn = X Vx + Pn  (and the same for Y, Z)
            const double2* V = s.GA.as<double2>();  // nb x m coefficients
            const T2* srcX[3] = {X, Y, Z};
            const T2* srcW[3] = {W, YW, ZW};
            const T2* srcP[3] = {P, YP, ZP};
            dbuf* dP[3] = {&B.tP, &B.tYP, &B.tZP};
            dbuf* dX[3] = {&B.tX, &B.tY, &B.tZ};
            for (int q = 0; q < 3; ++q) {
                T2* pn = dP[q]->template as<T2>();
                gemm_nn<T2, double2>(c, m, npw, na, V + m, nb, 1, srcW[q], npw, nullptr, pn, npw, nullptr, 1.0, 0.0,
                                     nullptr, 0);
                if (useP)
                    gemm_nn<T2, double2>(c, m, npw, na, V + m + na, nb, 1, srcP[q], npw, act, pn, npw, nullptr, 1.0,
                                         1.0, pn, npw);
                gemm_nn<T2, double2>(c, m, npw, m, V, nb, 1, srcX[q], npw, nullptr, dX[q]->template as<T2>(), npw,
                                     nullptr, 1.0, 1.0, pn, npw);
            }
            swapb(B.X, B.tX);
            swapb(B.Y, B.tY);
            swapb(B.Z, B.tZ);
            swapb(B.P, B.tP);
            swapb(B.YP, B.tYP);
            swapb(B.ZP, B.tZP);
            B.haveP = true;
            FS_CUDA(cudaMemcpyAsync(s.theta.p, s.evals.p, m * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            return;
        }
    }

    // Run block iterations until the nstates lowest bands have r <= tol, the
    // cap is reached, or (stall_check) the largest residual stops improving.
    template <typename T2>
    int run(Blocks<T2>& B, int maxit, double target, bool stall_check, int& iters_done, double& worst,
            int restart_every = 0) {
        double best = 1e300;
        int since_best = 0;
        for (int it = 0;; ++it) {
            if (restart_every > 0 && it > 0 && it % restart_every == 0) init_block<T2>(B);
            std::vector<double> r = residuals(B);
            worst = 0;
            for (int i = 0; i < nstates; ++i) worst = std::max(worst, std::isfinite(r[i]) ? r[i] : 1e300);
            if (!std::isfinite(worst) || worst >= 1e299)
                throw fs_error(FS_ERR_NUMERIC, "NaN/Inf in the residuals");
            if (verbose)
                fprintf(stderr, "[fs] it %d (%s) max resid %.3e\n", iters_done, sizeof(T2) == 16 ? "fp64" : "fp32",
                        worst);
            if (worst <= target) return 1;
            if (it >= maxit) return 0;
            if (stall_check) {
                if (worst < 0.7 * best) {
                    best = worst;
                    since_best = 0;
                } else if (++since_best >= 15 && worst < 1e-3) {
                    return 2;
                }
            }
            std::vector<int> act;
            for (int i = 0; i < m; ++i)
                if (r[i] > target) act.push_back(i);
            if (act.empty()) return 1;
            iterate<T2>(B, act);
            ++iters_done;
        }
    }

    template <typename T2> void final_rr(Blocks<T2>& B, std::vector<double>& eps, std::vector<double>& res) {
        T2* X = B.X.template as<T2>();
        T2* Y = B.Y.template as<T2>();
        double2* GA = s.GA.as<double2>();
        gemm_gram<T2>(c, m, m, c->npw, X, c->npw, nullptr, Y, c->npw, nullptr, GA, 1, m, 1.0, 0.0);
        add_diag_kernel<<<(m + 127) / 128, 128, 0, c->stream>>>(GA, m, E);
        int info = heevd(m);
        if (info != 0) throw fs_error(FS_ERR_NUMERIC, "final Rayleigh-Ritz failed (info " + std::to_string(info) + ")");
        // rotate X, Y only
        const double2* V = s.GA.as<double2>();
        gemm_nn<T2, double2>(c, m, c->npw, m, V, m, 1, X, c->npw, nullptr, B.tX.template as<T2>(), c->npw, nullptr,
                             1.0, 0.0, nullptr, 0);
        gemm_nn<T2, double2>(c, m, c->npw, m, V, m, 1, Y, c->npw, nullptr, B.tY.template as<T2>(), c->npw, nullptr,
                             1.0, 0.0, nullptr, 0);
        swapb(B.X, B.tX);
        swapb(B.Y, B.tY);
        shift_kernel<<<(m + 127) / 128, 128, 0, c->stream>>>(s.evals.as<double>(), E, s.shift.as<double>(), m);
        vec_resid_shift<T2>(c, B.X.template as<T2>(), B.Y.template as<T2>(), s.shift.as<double>(), m,
                            s.resid.as<double>());
        eps.resize(m);
        res.resize(m);
        FS_CUDA(cudaMemcpyAsync(eps.data(), s.evals.p, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaMemcpyAsync(res.data(), s.resid.p, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
    }
};

}  // namespace

fs_status solve_impl(fs_ctx* c, double e_ref, int nstates, double tol, fs_result* res) {
    auto t0 = std::chrono::steady_clock::now();
    Solver S;
    S.c = c;
    S.E = e_ref;
    S.nstates = nstates;
    S.tol = tol;
    S.verbose = c->opt.verbose;
    int guard = c->opt.guard >= 0 ? c->opt.guard : std::max(4, nstates / 16);
    S.m = nstates + guard;
    const int m = S.m;
    if (m > c->npw) throw fs_error(FS_ERR_ARG, "nstates + guard exceeds the number of plane waves");
    S.ensure_small(3 * m);
    const long npw = c->npw;
    // start block in FP64
    dbuf x0;
    x0.alloc((size_t)m * npw * sizeof(double2));
    int ncopy = std::min(c->ninit, m);
    if (ncopy > 0) {
        FS_CUDA(cudaMemcpyAsync(x0.p, c->init_states.p, (size_t)ncopy * npw * sizeof(double2),
                                cudaMemcpyDeviceToDevice, c->stream));
        if (c->init_damp) vec_damp(c, x0.as<double2>(), ncopy);
    }
    vec_damp_random(c, x0.as<double2>(), m, ncopy, c->opt.seed);

    int iters = 0, iters_mixed = 0;
    double worst = 0;
    int status = 0;
    std::vector<double> eps, resid;
    Blocks<double2> B64;
    if (c->opt.precision == FS_MIXED) {
        ctx_ensure_fp32(c);
        Blocks<float2> B32;
        B32.alloc(m, npw);
        vec_convert<double2, float2>(c, x0.as<double2>(), B32.X.as<float2>(), (size_t)m * npw);
        S.init_block<float2>(B32);
        status = S.run<float2>(B32, c->opt.maxit, tol, true, iters, worst, 10);
        iters_mixed = iters;
        // carry the bands to FP64 (through x0, so that both block sets never coexist)
        vec_convert<float2, double2>(c, B32.X.as<float2>(), x0.as<double2>(), (size_t)m * npw);
        FS_CUDA(cudaStreamSynchronize(c->stream));
        B32.free_all();
        B64.alloc(m, npw);
        FS_CUDA(cudaMemcpyAsync(B64.X.p, x0.p, (size_t)m * npw * sizeof(double2), cudaMemcpyDeviceToDevice,
                                c->stream));
    } else {
        B64.alloc(m, npw);
        FS_CUDA(cudaMemcpyAsync(B64.X.p, x0.p, (size_t)m * npw * sizeof(double2), cudaMemcpyDeviceToDevice,
                                c->stream));
    }
    x0.release();
    S.init_block<double2>(B64);
    status = S.run<double2>(B64, std::max(0, c->opt.maxit - iters), tol, false, iters, worst);
    S.final_rr<double2>(B64, eps, resid);
    // order by (|eps - E|, eps)
    std::vector<int> order(m);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        double da = std::fabs(eps[a] - e_ref), db = std::fabs(eps[b] - e_ref);
        if (da != db) return da < db;
        return eps[a] < eps[b];
    });
    c->result_states.ensure((size_t)nstates * npw * sizeof(double2));
    int nconv = 0;
    for (int i = 0; i < nstates; ++i) {
        int j = order[i];
        res->eps[i] = eps[j];
        res->resid[i] = resid[j];
        if (resid[j] <= tol) ++nconv;
        FS_CUDA(cudaMemcpyAsync(c->result_states.as<double2>() + (size_t)i * npw, B64.X.as<double2>() + (size_t)j * npw,
                                npw * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    }
    FS_CUDA(cudaStreamSynchronize(c->stream));
    c->nresult = nstates;
    res->nconv = nconv;
    res->iters = iters;
    res->iters_mixed = iters_mixed;
    res->n_hpsi = S.n_hpsi;
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    (void)status;
    return nconv == nstates ? FS_OK : FS_ERR_NOT_CONVERGED;
}
