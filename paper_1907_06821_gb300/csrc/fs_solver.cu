// Folded-spectrum all-band PCG (locally optimal block form) on the GPU.
//
// Operator A = (H - E)^2 (paper Sec. II.C, Eq. wl1); its lowest eigenvectors
// are the eigenvectors of H nearest E.  State: m bands X (A-Ritz vectors, Ritz
// values theta) and their images Y = (H-E)X.  Per iteration:
//   d_i = <x_i, y_i>, r_i = y_i - d_i x_i       H residual vectors (all bands)
//   R_i = (H-E) r_i + d_i r_i + (d_i^2 - theta_i) x_i   = A x_i - theta_i x_i
//        (one H application per band; every term scales with ||r_i||, so the
//         A residual stays accurate in FP32 down to the FP32 noise of r_i)
//   act  = bands whose ||R_i|| is above the threshold matching an H residual tol
//   W    = M R on act, W -= X (X^H W), rows normalised, YW = (H-E) W
//   P    = previous directions on act, made orthogonal to X, normalised
//   Rayleigh-Ritz of A on S = [X W P]: G_A = ((H-E)S)^H (H-E)S, G_B = S^H S,
//   robust basis selection (FP64 dense eigensolves);
//   X <- S c (lowest m), P <- [W P] c_WP; Y, YP by linearity.
// Convergence: a Rayleigh-Ritz step on H within the wanted bands; their H
// residuals must be <= tol for the nstates pairs nearest E.
// Mixed precision: vectors, FFTs and GEMMs in FP32 (tensor-core TF32 x3),
// dense algebra in FP64, Y (and YP) recomputed every 10 iterations; then an
// FP64 check of the wanted bands, and FP64 iterations only if it fails.
//
// Lowest-state mode (the all-band CG of the ground-state codes the paper
// builds on): the same block iteration on H itself, Y = H X, Rayleigh
// quotients <s_i, H s_j>, residual R = Y - theta X (one H application per
// band per iteration, half of the folded form), preconditioner
// 1 / (1 + |q|^2 / 2), results ordered by eigenvalue.
#include "fs_common.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <numeric>

void ctx_ensure_fp32(fs_ctx* c);

namespace {

// Band blocks, backed by the context's persistent workspace (12 buffers).
template <typename T2> struct Blocks {
    dbuf &X, &Y, &W, &YW, &P, &YP, &RH, &ZR, &tX, &tY, &tP, &tYP;
    bool haveP = false;
    explicit Blocks(dbuf* d)
        : X(d[0]), Y(d[1]), W(d[2]), YW(d[3]), P(d[4]), YP(d[5]), RH(d[6]), ZR(d[7]), tX(d[8]), tY(d[9]), tP(d[10]),
          tYP(d[11]) {}
    // full = false: only X, Y and the rotation targets tX, tY (what the FP64 check
    // of an FP32 result uses); the rest is allocated when FP64 iterations start
    void alloc(int m, long npw, bool full = true) {
        size_t b = (size_t)m * npw * sizeof(T2);
        for (dbuf* d : {&X, &Y, &tX, &tY}) d->ensure(b);
        if (full)
            for (dbuf* d : {&W, &YW, &P, &YP, &RH, &ZR, &tP, &tYP}) d->ensure(b);
        haveP = false;
    }
};

void swapb(dbuf& a, dbuf& b) {
    std::swap(a.p, b.p);
    std::swap(a.bytes, b.bytes);
}


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

// smallest squared diagonal entry of the Cholesky factor left in L (n x n)
__global__ void min_pivot_kernel(const double2* L, int n, double* out) {
    __shared__ double sh[256];
    double v = 1e300;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double d = L[(long)i * n + i].x;
        v = fmin(v, d * d);
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}
inline int nblk_(long total) { return nblk(total); }

// out (k x k) = G[keep, keep] for G n x n (all column-major)
__global__ void gather_sym_kernel(const double2* G, int n, const int* keep, int k, double2* out) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)k * k) return;
    int i = (int)(t % k), j = (int)(t / k);
    out[t] = G[keep[i] + (long)keep[j] * n];
}

// C (n x m, ld n): row r = U row pos[r] (U k x m, ld k), or 0 where pos[r] < 0
__global__ void scatter_rows_kernel(double2* C, int n, int m, const double2* U, int k, const int* pos) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * m) return;
    int r = (int)(t % n), j = (int)(t / n);
    int p = pos[r];
    C[t] = p >= 0 ? U[p + (long)j * k] : make_double2(0.0, 0.0);
}

// G(i, j) = conj(G(j, i)) where the block of i (boundaries b1 <= b2) is below the block of j
__global__ void herm_fill_kernel(double2* G, int n, int b1, int b2) {
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    int i = (int)(t % n), j = (int)(t / n);
    int bi = (i >= b1) + (i >= b2), bj = (j >= b1) + (j >= b2);
    if (bi < bj) {
        double2 v = G[(long)i * n + j];
        G[t] = make_double2(v.x, -v.y);
    }
}

struct Solver {
    fs_ctx* c;
    double E;
    int nstates, m;
    double tol;
    SolverSmall& s;
    explicit Solver(fs_ctx* c_) : c(c_), s(c_->smem.small) {}
    long long n_hpsi = 0;
    int verbose = 0;
    bool lowest = false;  // lowest eigenpairs of H instead of the pairs nearest E

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
        s.bkin.alloc(nbmax * sizeof(double));
        s.hres.alloc(nbmax * sizeof(double));
        s.evals.alloc(nbmax * sizeof(double));
        s.theta.alloc(nbmax * sizeof(double));
        s.act.alloc(2 * nbmax * sizeof(int));
        s.resid.alloc(nbmax * sizeof(double));
        s.dots.alloc(nbmax * sizeof(double2));
        s.nrm.alloc(nbmax * sizeof(double));
        s.shift.alloc(nbmax * sizeof(double));
        s.keep.alloc(2 * nbmax * sizeof(int));
    }

    // generalized Hermitian eigenproblem GA c = lambda GB c, n x n column-major:
    // every eigenpair, vectors into GA, values into s.evals; returns the Cholesky info
    int hegvd(int n) {
        ProfScope ps(c, KS_DENSE_LA, 0.0, 0.0);
        return dense_hegv(c, n, s.GA.as<double2>(), s.GB.as<double2>(), n, s.evals.as<double>());
    }
    // every eigenpair of the Hermitian A (n x n, default s.GA): vectors overwrite A
    int heevd(int n, double2* A = nullptr) {
        if (!A) A = s.GA.as<double2>();
        ProfScope ps(c, KS_DENSE_LA, 0.0, 0.0);
        DenseWork& D = c->dense;
        D.U.ensure((size_t)n * n * sizeof(double2));
        dense_heev(c, n, A, n, s.evals.as<double>(), D.U.as<double2>(), n);
        FS_CUDA(cudaMemcpyAsync(A, D.U.p, (size_t)n * n * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
        return 0;
    }

    // Rayleigh-Ritz of A on a basis of nb vectors with Gram matrices GA = <S, AS>
    // and GB = <S, S> (column-major in s.GA, s.GB).  On return s.GA holds the
    // nb x m coefficients of the m lowest Ritz vectors (column j = vector j)
    // and s.evals[0..m) their Ritz values.  robust = true scales both matrices
    // to a unit-diagonal GB and selects the basis by a Cholesky factorisation
    // of GB that drops every direction whose pivot (squared distance from the
    // span of the directions before it) is below piv_floor, refactorising
    // without them; should that not settle, the basis comes from an
    // eigendecomposition of GB, dropping eigenvalues below tau * max.  Returns
    // the factorisation info (0 = success, else the failing column + 1).
    int rr_basis(int nb, bool robust, double tau, double piv_floor) {
        double2* GA = s.GA.as<double2>();
        double2* GB = s.GB.as<double2>();
        if (!robust) return hegvd(nb);
        diag_invsqrt_kernel<<<nblk(nb), 256, 0, c->stream>>>(GB, nb, s.dscale.as<double>());
        sym_scale_kernel<<<nblk((long)nb * nb), 256, 0, c->stream>>>(GA, GB, nb, s.dscale.as<double>());
        FS_CUDA(cudaGetLastError());
        std::vector<int> keep(nb);
        std::iota(keep.begin(), keep.end(), 0);
        std::vector<double> piv;
        for (int attempt = 0; attempt < 6 && (int)keep.size() >= m; ++attempt) {
            const int info = chol_kept(nb, keep, piv);
            const int k = (int)keep.size();
            const int valid = info > 0 ? info - 1 : k;  // pivots known before the failing column
            std::vector<char> drop(k, 0);
            bool any = info > 0;
            if (info > 0) drop[info - 1] = 1;
            for (int i = 0; i < valid; ++i)
                if (!(piv[i] > piv_floor)) drop[i] = 1, any = true;
            if (!any) return rr_reduced(nb, keep);
            std::vector<int> kept;
            for (int i = 0; i < k; ++i)
                if (!drop[i]) kept.push_back(keep[i]);
            keep.swap(kept);
        }
        return rr_svqb(nb, tau);
    }

    // Cholesky factor of GB[keep, keep] into s.T2 (k x k) and GA[keep, keep]
    // into s.T1; squared pivots to piv; returns the potrf info.
    int chol_kept(int nb, const std::vector<int>& keep, std::vector<double>& piv) {
        ProfScope ps(c, KS_DENSE_LA, 0.0, 0.0);
        const int k = (int)keep.size();
        double2* T1 = s.T1.as<double2>();
        double2* T2 = s.T2.as<double2>();
        if (k == nb) {
            const size_t bytes = (size_t)nb * nb * sizeof(double2);
            FS_CUDA(cudaMemcpyAsync(T1, s.GA.p, bytes, cudaMemcpyDeviceToDevice, c->stream));
            FS_CUDA(cudaMemcpyAsync(T2, s.GB.p, bytes, cudaMemcpyDeviceToDevice, c->stream));
        } else {
            int* kd = s.keep.as<int>();
            FS_CUDA(cudaMemcpyAsync(kd, keep.data(), k * sizeof(int), cudaMemcpyHostToDevice, c->stream));
            gather_sym_kernel<<<nblk((long)k * k), 256, 0, c->stream>>>(s.GA.as<double2>(), nb, kd, k, T1);
            gather_sym_kernel<<<nblk((long)k * k), 256, 0, c->stream>>>(s.GB.as<double2>(), nb, kd, k, T2);
            FS_CUDA(cudaGetLastError());
        }
        const int info = dense_potrf(c, k, T2, k, s.nrm.as<double>());  // squared pivots to s.nrm
        piv.resize(k);
        FS_CUDA(cudaMemcpyAsync(piv.data(), s.nrm.p, k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        return info;
    }

    // Standard form of the kept problem, C = L^-1 GA L^-H, its m lowest
    // eigenpairs, coefficients L^-H V scattered back to the nb rows (rows of
    // dropped directions 0) and unscaled.
    int rr_reduced(int nb, const std::vector<int>& keep) {
        const int k = (int)keep.size();
        double2* L = s.T2.as<double2>();
        double2* C = s.T1.as<double2>();
        double2* T = s.GA.as<double2>();  // free here: chol_kept copied what it needs into T1
        int info = 0;
        {
            ProfScope ps(c, KS_DENSE_LA, 0.0, 8.0 * k * (double)k * k);
            dense_trsm(c, 0, k, k, L, k, C, k);               // L^-1 GA
            dense_conj_transpose(c, k, k, C, k, T, k);          // GA L^-H
            dense_trsm(c, 0, k, k, L, k, T, k);               // L^-1 GA L^-H
            dense_heev(c, k, T, m, s.evals.as<double>(), C, k);  // m lowest pairs, vectors into C
            dense_trsm(c, 1, k, m, L, k, C, k);               // L^-H V
        }
        if (info != 0) return info;
        double2* GA = s.GA.as<double2>();
        if (k == nb) {
            FS_CUDA(cudaMemcpyAsync(GA, C, (size_t)nb * m * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
        } else {
            std::vector<int> pos(nb, -1);
            for (int i = 0; i < k; ++i) pos[keep[i]] = i;
            int* pd = s.keep.as<int>() + nb;
            FS_CUDA(cudaMemcpyAsync(pd, pos.data(), nb * sizeof(int), cudaMemcpyHostToDevice, c->stream));
            scatter_rows_kernel<<<nblk((long)nb * m), 256, 0, c->stream>>>(GA, nb, m, (const double2*)C, k, pd);
        }
        row_scale_kernel<<<nblk((long)nb * m), 256, 0, c->stream>>>(GA, nb, m, s.dscale.as<double>());
        FS_CUDA(cudaGetLastError());
        last_kept = k;
        ++n_chol_drop[k < nb];
        return 0;
    }
    long long n_chol_drop[2] = {0, 0};  // Rayleigh-Ritz steps without / with dropped directions
    long long n_svqb = 0;               // steps that needed the eigendecomposition of GB

    // Basis from the eigendecomposition of the scaled GB (s.GA, s.GB scaled).
    int rr_svqb(int nb, double tau) {
        double2* GA = s.GA.as<double2>();
        double2* GB = s.GB.as<double2>();
        ++n_svqb;
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
        double2* tmp = s.T1.as<double2>();
        double2* GAp = s.T2.as<double2>();
        {
        ProfScope ps(c, KS_DENSE_LA, 0.0, 8.0 * nb * (double)nb * k + 8.0 * k * (double)k * nb);
        dense_gemm(c, 0, 0, nb, k, nb, 1.0, GA, nb, T, nb, 0.0, tmp, nb);
        dense_gemm(c, 1, 0, k, k, nb, 1.0, T, nb, tmp, nb, 0.0, GAp, k);
        }
        info = heevd(k, GAp);
        if (info != 0) return info;
        {
        ProfScope ps(c, KS_DENSE_LA, 0.0, 8.0 * nb * (double)m * k);
        dense_gemm(c, 0, 0, nb, m, k, 1.0, T, nb, GAp, k, 0.0, GA, nb);
        }
        row_scale_kernel<<<nblk((long)nb * m), 256, 0, c->stream>>>(GA, nb, m, s.dscale.as<double>());
        FS_CUDA(cudaGetLastError());
        last_kept = k;
        return 0;
    }
    int last_kept = 0;
    double last_hworst = -1;  // worst wanted H residual of the last H check of run() (-1: none)

    template <typename T2> static constexpr bool is_fp32() { return sizeof(T2) == 8; }
    template <typename T2> static double tau_for() { return sizeof(T2) == 8 ? 1e-6 : 1e-11; }
    // pivot floor of the Cholesky fast path (the scaled G_B has unit diagonal)
    template <typename T2> static double piv_for() { return sizeof(T2) == 8 ? 1e-3 : 1e-8; }

    // Hermitian Gram matrix of the basis blocks into G (nb x nb column-major):
    // G(i, j) = <S_i, T_j> computed for row block >= column block (T = S or
    // T = A S, both Hermitian forms), the upper blocks filled by conjugation.
    template <typename T2>
    void gram_blocks(double2* G, int nb, const T2* const* S, const T2* const* T, const int* const* maps,
                     const int* sizes, const int* offs, int nblk) {
        for (int I = 0; I < nblk; ++I)
            for (int J = 0; J <= I; ++J)
                gemm_gram<T2>(c, sizes[I], sizes[J], c->npw, S[I], c->npw, maps[I], T[J], c->npw, maps[J],
                              G + offs[I] + (long)offs[J] * nb, 1, nb, 1.0, 0.0);
        int b1 = nblk > 1 ? offs[1] : nb, b2 = nblk > 2 ? offs[2] : nb;
        herm_fill_kernel<<<nblk_((long)nb * nb), 256, 0, c->stream>>>(G, nb, b1, b2);
        FS_CUDA(cudaGetLastError());
    }

    // Initial Rayleigh-Ritz on A in span X (X need not be orthonormal).
    template <typename T2> void init_block(Blocks<T2>& B) {
        T2* X = B.X.template as<T2>();
        T2* Y = B.Y.template as<T2>();
        HE(X, Y, m);
        ensure_small(3 * m);
        double2* GA = s.GA.as<double2>();
        double2* GB = s.GB.as<double2>();
        // folded: <s_i, A s_j> = <(H-E) s_i, (H-E) s_j>; lowest: <s_i, H s_j>
        gemm_gram<T2>(c, m, m, c->npw, lowest ? X : Y, c->npw, nullptr, Y, c->npw, nullptr, GA, 1, m, 1.0, 0.0);
        gemm_gram<T2>(c, m, m, c->npw, X, c->npw, nullptr, X, c->npw, nullptr, GB, 1, m, 1.0, 0.0);
        {
            // a non-finite start block (or H image) is reported before a dense eigensolve sees it:
            // the diagonals of G_B and G_A are the squared norms of the bands and of their images
            std::vector<double2> dg(2 * (size_t)m);
            FS_CUDA(cudaMemcpy2DAsync(dg.data(), sizeof(double2), GB, (m + 1) * sizeof(double2), sizeof(double2), m,
                                      cudaMemcpyDeviceToHost, c->stream));
            FS_CUDA(cudaMemcpy2DAsync(dg.data() + m, sizeof(double2), GA, (m + 1) * sizeof(double2), sizeof(double2),
                                      m, cudaMemcpyDeviceToHost, c->stream));
            FS_CUDA(cudaStreamSynchronize(c->stream));
            for (const double2& v : dg)
                if (!std::isfinite(v.x)) throw fs_error(FS_ERR_NUMERIC, "non-finite values in the block or its H image");
        }
        int info = rr_basis(m, true, tau_for<T2>(), piv_for<T2>());
        if (info != 0) throw fs_error(FS_ERR_NUMERIC, "start block is rank deficient (info " + std::to_string(info) + ")");
        rotate_simple(B, m);
        FS_CUDA(cudaMemcpyAsync(s.theta.p, s.evals.p, m * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        B.haveP = false;
    }

    // FP32 stage: the images Y (and YP) are carried by linear updates and
    // drift from (H-E)X in FP32; recompute them from X and P, then redo the
    // Rayleigh-Ritz step on X.  P is kept.
    template <typename T2> void refresh(Blocks<T2>& B) {
        bool keepP = B.haveP;
        init_block<T2>(B);
        if (keepP) {
            HE(B.P.template as<T2>(), B.YP.template as<T2>(), m);
            B.haveP = true;
        }
    }

    // X, Y <- (X, Y) V[:, :m] with V = GA (n x n, column-major)
    template <typename T2> void rotate_simple(Blocks<T2>& B, int n) {
        const double2* V = s.GA.as<double2>();
        dbuf* src[2] = {&B.X, &B.Y};
        dbuf* dst[2] = {&B.tX, &B.tY};
        for (int q = 0; q < 2; ++q)
            gemm_nn<T2, double2>(c, m, c->npw, n, V, n, 1, src[q]->template as<T2>(), c->npw, nullptr,
                                 dst[q]->template as<T2>(), c->npw, nullptr, 1.0, 0.0, nullptr, 0);
        swapb(B.X, B.tX);
        swapb(B.Y, B.tY);
    }

    // A residuals R_i = A x_i - theta_i x_i of all bands (left in B.RH), their
    // norms and the Ritz values on the host.  Costs one H application per band.
    std::vector<double> hres_h;  // H residuals ||y_i - <x_i,y_i> x_i|| of the last a_residuals call

    template <typename T2> void a_residuals(Blocks<T2>& B, std::vector<double>& ra, std::vector<double>& th) {
        T2* X = B.X.template as<T2>();
        T2* Y = B.Y.template as<T2>();
        T2* RH = B.RH.template as<T2>();
        T2* ZR = B.ZR.template as<T2>();
        vec_resid<T2>(c, X, Y, m, s.hres.as<double>(), s.dots.as<double2>());
        hres_h.resize(m);
        FS_CUDA(cudaMemcpyAsync(hres_h.data(), s.hres.p, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        vec_rh<T2>(c, X, Y, s.dots.as<double2>(), m, RH);
        ra.resize(m);
        th.resize(m);
        if (lowest) {
            // the H residual y - <x, y> x is the residual of the lowest-state iteration
            FS_CUDA(cudaMemcpyAsync(ra.data(), s.hres.p, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        } else {
            HE(RH, ZR, m);
            vec_a_resid<T2>(c, ZR, RH, X, s.dots.as<double2>(), s.theta.as<double>(), m, s.resid.as<double>());
            FS_CUDA(cudaMemcpyAsync(ra.data(), s.resid.p, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        }
        FS_CUDA(cudaMemcpyAsync(th.data(), s.theta.p, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        ctx_check_errflag(c);
        prof_flush(c);
    }

    // Threshold on the A residual matching an H residual of about tol: for an
    // isolated eigenvector at distance d = sqrt(theta) from E the A residual is
    // about 2 d times the H residual (factor floored at 1e-3).
    double tol_a(double theta, double target) const {
        return lowest ? target : target * std::max(std::sqrt(std::max(theta, 0.0)), 1e-3);
    }

    // Rayleigh-Ritz on H within the wanted A-Ritz vectors (the nstates lowest
    // theta plus bands tied with the nstates-th within 1e-3): H-Ritz pairs and
    // their H residuals.  The rotated vectors are left in B.tX (rows 0..n).
    // Outputs: n, eps (E + Ritz values of H - E), res, and order (the nstates
    // pairs nearest E by (|eps - E|, eps)).
    template <typename T2>
    void h_ritz(Blocks<T2>& B, const std::vector<double>& th, int& n, std::vector<double>& eps,
                std::vector<double>& res, std::vector<int>& order) {
        n = nstates;
        const double tie = lowest ? 1e-3 * std::max(1.0, std::fabs(th[nstates - 1])) : 1e-3 * th[nstates - 1];
        while (n < m && th[n] <= th[nstates - 1] + tie) ++n;
        T2* X = B.X.template as<T2>();
        T2* Y = B.Y.template as<T2>();
        double2* GA = s.GA.as<double2>();
        double2* GB = s.GB.as<double2>();
        // generalized form with the overlap <x_i, x_j>: the Ritz vectors come out
        // orthonormal in the working precision even when X came from the FP32 stage
        gemm_gram<T2>(c, n, n, c->npw, X, c->npw, nullptr, Y, c->npw, nullptr, GA, 1, n, 1.0, 0.0);
        gemm_gram<T2>(c, n, n, c->npw, X, c->npw, nullptr, X, c->npw, nullptr, GB, 1, n, 1.0, 0.0);
        int info = hegvd(n);
        if (info != 0) throw fs_error(FS_ERR_NUMERIC, "Rayleigh-Ritz on H failed (info " + std::to_string(info) + ")");
        const double2* U = s.GA.as<double2>();
        gemm_nn<T2, double2>(c, n, c->npw, n, U, n, 1, X, c->npw, nullptr, B.tX.template as<T2>(), c->npw, nullptr,
                             1.0, 0.0, nullptr, 0);
        gemm_nn<T2, double2>(c, n, c->npw, n, U, n, 1, Y, c->npw, nullptr, B.tY.template as<T2>(), c->npw, nullptr,
                             1.0, 0.0, nullptr, 0);
        vec_resid_shift<T2>(c, B.tX.template as<T2>(), B.tY.template as<T2>(), s.evals.as<double>(), n,
                            s.resid.as<double>());
        std::vector<double> lam(n);
        res.resize(n);
        FS_CUDA(cudaMemcpyAsync(lam.data(), s.evals.p, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaMemcpyAsync(res.data(), s.resid.p, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        eps.resize(n);
        for (int i = 0; i < n; ++i) eps[i] = lam[i] + E;
        order.resize(n);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            if (lowest) return eps[a] < eps[b];
            double da = std::fabs(eps[a] - E), db = std::fabs(eps[b] - E);
            if (da != db) return da < db;
            return eps[a] < eps[b];
        });
        order.resize(nstates);
    }

    // Training rows for the learned preconditioner: for the wanted bands that are
    // still active, the A residual (in B.RH) and the correction that would take
    // the band into the span of the reference states (a converged solve).
    template <typename T2> void record_pairs(Blocks<T2>& B, const std::vector<int>& act_h) {
        Mlp& L = c->mlp;
        std::vector<int> sel;
        for (int i : act_h)
            if (i < nstates) sel.push_back(i);
        const int nr = (int)sel.size();
        const long long rows = (long long)nr * L.nshell;
        if (nr == 0 || L.nrec + rows > L.cap) return;
        const long npw = c->npw;
        const T2* Xref = sizeof(T2) == 8 ? (const T2*)L.xref32.p : (const T2*)L.xref64.p;
        int* map = s.act.as<int>() + m;  // second half of the index buffer
        FS_CUDA(cudaMemcpyAsync(map, sel.data(), nr * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        L.proj.ensure((size_t)nr * npw * sizeof(T2));
        L.err.ensure((size_t)nr * npw * sizeof(T2));
        double2* Cg = s.GB.as<double2>();
        gemm_gram<T2>(c, L.nref, nr, npw, Xref, npw, nullptr, B.X.template as<T2>(), npw, map, Cg, 1, L.nref, 1.0,
                      0.0);
        gemm_nn<T2, double2>(c, nr, npw, L.nref, Cg, L.nref, 1, Xref, npw, nullptr, L.proj.template as<T2>(), npw,
                             nullptr, 1.0, 0.0, nullptr, 0);
        mlp_err_from_proj<T2>(c, L.proj.template as<T2>(), B.X.template as<T2>(), map, nr, L.err.template as<T2>());
        mlp_features<T2>(c, B.RH.template as<T2>(), map, nr, s.dots.as<double2>(), L.err.template as<T2>(),
                         L.recF.as<float>() + L.nrec * 4, L.recz.as<float>() + L.nrec, L.recw.as<float>() + L.nrec);
        L.nrec += rows;
        L.nrec_bands += nr;
    }

    // One block iteration on the active set (B.RH holds the A residuals of all bands).
    template <typename T2> void iterate(Blocks<T2>& B, const std::vector<int>& act_h) {
        const int na = (int)act_h.size();
        const long npw = c->npw;
        int* act = s.act.as<int>();
        FS_CUDA(cudaMemcpyAsync(act, act_h.data(), na * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        T2 *X = B.X.template as<T2>(), *Y = B.Y.template as<T2>();
        T2 *W = B.W.template as<T2>(), *YW = B.YW.template as<T2>();
        T2 *P = B.P.template as<T2>(), *YP = B.YP.template as<T2>();
        double2* GA = s.GA.as<double2>();
        double2* GB = s.GB.as<double2>();
        // W = M R on the active bands, made orthogonal to X and normalised
        if (c->mlp.record && !lowest) record_pairs<T2>(B, act_h);
        const bool teter = c->opt.precond == FS_PREC_TETER;
        if (lowest) {
            vec_make_w<T2>(c, B.RH.template as<T2>(), act, na, W, 0.0, 1.0, 2, nullptr);
        } else if (c->opt.precond == FS_PREC_LEARNED) {
            mlp_make_w<T2>(c, B.RH.template as<T2>(), act, na, W, s.dots.as<double2>());
        } else {
            if (teter) vec_band_kin<T2>(c, X, m, s.bkin.as<double>());
            vec_make_w<T2>(c, B.RH.template as<T2>(), act, na, W, E, c->opt.dE, teter ? 1 : 0,
                           teter ? s.bkin.as<double>() : nullptr);
        }
        gemm_gram<T2>(c, m, na, npw, X, npw, nullptr, W, npw, nullptr, GB, 1, m, 1.0, 0.0);
        gemm_nn<T2, double2>(c, na, npw, m, GB, m, 1, X, npw, nullptr, W, npw, nullptr, -1.0, 1.0, W, npw);
        vec_row_norms<T2>(c, W, nullptr, na, s.nrm.as<double>());
        vec_scale_rows<T2>(c, W, nullptr, na, s.nrm.as<double>());
        HE(W, YW, na);
        bool useP = B.haveP;
        if (useP) {
            // P[act] -= X (X^H P[act]); the same combination for YP; then normalise
            gemm_gram<T2>(c, m, na, npw, X, npw, nullptr, P, npw, act, GB, 1, m, 1.0, 0.0);
            gemm_nn<T2, double2>(c, na, npw, m, GB, m, 1, X, npw, nullptr, P, npw, act, -1.0, 1.0, P, npw);
            gemm_nn<T2, double2>(c, na, npw, m, GB, m, 1, Y, npw, nullptr, YP, npw, act, -1.0, 1.0, YP, npw);
            vec_row_norms<T2>(c, P, act, na, s.nrm.as<double>());
            vec_scale_rows<T2>(c, P, act, na, s.nrm.as<double>());
            vec_scale_rows<T2>(c, YP, act, na, s.nrm.as<double>());
        }
        for (int attempt = 0; attempt < 2; ++attempt) {
            int nblk = useP ? 3 : 2;
            const T2* S[3] = {X, W, P};
            const T2* SY[3] = {Y, YW, YP};
            const int* maps[3] = {nullptr, nullptr, act};
            int sizes[3] = {m, na, na};
            int offs[3] = {0, m, m + na};
            int nb = m + na + (useP ? na : 0);
            // <s_i, A s_j> = <(H-E)s_i, (H-E)s_j>: the Y images keep the small
            // Rayleigh quotients of A accurate in the FP32 stage
            gram_blocks<T2>(GA, nb, lowest ? S : SY, SY, maps, sizes, offs, nblk);
            gram_blocks<T2>(GB, nb, S, S, maps, sizes, offs, nblk);
            int info = rr_basis(nb, true, tau_for<T2>(), piv_for<T2>());
            if (info != 0) {
                if (useP) {
                    useP = false;
                    continue;
                }
                throw fs_error(FS_ERR_NUMERIC, "Rayleigh-Ritz basis selection failed (info " +
                                                   std::to_string(info) + ")");
            }
            // rotation: Pn = W Vw + P Vp ; Xn = X Vx + Pn  (and the same for Y)
            const double2* V = s.GA.as<double2>();  // nb x m coefficients
            const T2* srcX[2] = {X, Y};
            const T2* srcW[2] = {W, YW};
            const T2* srcP[2] = {P, YP};
            dbuf* dP[2] = {&B.tP, &B.tYP};
            dbuf* dX[2] = {&B.tX, &B.tY};
            for (int q = 0; q < 2; ++q) {
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
            swapb(B.P, B.tP);
            swapb(B.YP, B.tYP);
            B.haveP = true;
            FS_CUDA(cudaMemcpyAsync(s.theta.p, s.evals.p, m * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            return;
        }
    }

    // Block iterations until the H residuals of the nstates pairs nearest E
    // are <= target (returns 1, results filled), the cap is reached (0), or,
    // with stall_check, the wanted A residuals stop improving (2).
    template <typename T2>
    int run(Blocks<T2>& B, int maxit, double target, bool stall_check, int& iters_done, int refresh_every,
            std::vector<double>& eps, std::vector<double>& res, std::vector<int>& order, int& nres) {
        double best = 1e300;
        int since_best = 0;
        last_hworst = -1;
        std::vector<double> ra, th;
        for (int it = 0;; ++it) {
            if (refresh_every > 0 && it > 0 && it % refresh_every == 0) refresh<T2>(B);
            a_residuals(B, ra, th);
            double worst = 0;  // largest wanted A residual relative to its threshold
            for (int i = 0; i < nstates; ++i) {
                double q = ra[i] / tol_a(th[i], target);
                if (!std::isfinite(q)) throw fs_error(FS_ERR_NUMERIC, "NaN/Inf in the residuals");
                worst = std::max(worst, q);
            }
            double hworst = -1;
            // the H check runs once every wanted A residual is below its threshold,
            // and every 5 iterations once they are within 100x of it (the FP32 A
            // residual has a noise floor that can keep the first gate shut)
            // (in FP32 the A residual of states close to E carries the noise of the
            // FP32 (H-E)x, so the H check itself also runs every 5 iterations)
            if (worst <= 1.0 || (it % 5 == 0 && (worst <= 100.0 || is_fp32<T2>()))) {
                h_ritz<T2>(B, th, nres, eps, res, order);
                hworst = 0;
                for (int i : order) hworst = std::max(hworst, res[i]);
                last_hworst = hworst;
                if (hworst <= target) return 1;
            }
            if (verbose)
                fprintf(stderr, "[fs] it %d (%s) wanted A-residual/threshold %.3e  H-check %.3e\n", iters_done,
                        is_fp32<T2>() ? "fp32" : "fp64", worst, hworst);
            if (it >= maxit) return 0;
            if (stall_check) {
                // geometric mean of the wanted bands' excess over their thresholds:
                // it keeps falling while the bulk of the block converges even when
                // the hardest band sits on a plateau
                double lg = 0;
                for (int i = 0; i < nstates; ++i) lg += std::log(std::max(ra[i] / tol_a(th[i], target), 1.0));
                double metric = std::exp(lg / nstates);
                if (hworst >= 0) metric = hworst / target;
                else if (best < 1e299 && it % 5 != 0) metric = best;  // decided by the H check when it runs
                if (metric < 0.7 * best) {
                    best = metric;
                    since_best = 0;
                } else if (++since_best >= 30) {
                    return 2;
                }
            }
            // soft locking: a band stops contributing directions once its A residual
            // is below its threshold (locking on the H residual as well was measured
            // to cost iterations on the wire workload: 135 against 125)
            std::vector<int> act;
            for (int i = 0; i < m; ++i)
                if (ra[i] > tol_a(th[i], target)) act.push_back(i);
            if (act.empty())
                for (int i = 0; i < m; ++i) act.push_back(i);
            iterate<T2>(B, act);
            ++iters_done;
        }
    }
};

}  // namespace

fs_status solve_impl(fs_ctx* c, double e_ref, int nstates, double tol, fs_result* res, bool lowest) {
    auto t0 = std::chrono::steady_clock::now();
    Solver S(c);
    S.lowest = lowest;
    S.E = lowest ? 0.0 : e_ref;
    S.nstates = nstates;
    S.tol = tol;
    S.verbose = c->opt.verbose;
    int guard = c->opt.guard >= 0 ? c->opt.guard : std::max(4, nstates / 16);
    S.m = nstates + guard;
    const int m = S.m;
    if (m > c->npw) throw fs_error(FS_ERR_ARG, "nstates + guard exceeds the number of plane waves");
    S.ensure_small(3 * m);
    const long npw = c->npw;
    if (!lowest && (c->opt.precond == FS_PREC_LEARNED || c->mlp.record)) {
        mlp_setup(c);
        if (c->mlp.e_ref != e_ref || !c->mlp.Mdev.p) {
            c->mlp.e_ref = e_ref;
            c->mlp.Mdev.release();
        }
    }
    // start block in FP64
    dbuf& x0 = c->smem.x0;
    x0.ensure((size_t)m * npw * sizeof(double2));
    int ncopy = std::min(c->ninit, m);
    if (ncopy > 0) {
        FS_CUDA(cudaMemcpyAsync(x0.p, c->init_states.p, (size_t)ncopy * npw * sizeof(double2),
                                cudaMemcpyDeviceToDevice, c->stream));
        if (c->init_damp) vec_damp(c, x0.as<double2>(), ncopy);
    }
    vec_damp_random(c, x0.as<double2>(), m, ncopy, c->opt.seed);

    int iters = 0, iters_mixed = 0;
    int status = 0;
    std::vector<double> eps, resid;
    std::vector<int> order;
    int nres = 0;
    Blocks<double2> B64(c->smem.b64);
    bool done = false;
    if (c->opt.precision == FS_MIXED) {
        ctx_ensure_fp32(c);
        Blocks<float2> B32(c->smem.b32);
        B32.alloc(m, npw);
        vec_convert<double2, float2>(c, x0.as<double2>(), B32.X.as<float2>(), (size_t)m * npw);
        S.init_block<float2>(B32);
        B64.alloc(m, npw, false);
        // FP32 stage to a margin below tol (its residuals carry FP32 noise), then
        // an FP64 check of the wanted bands: Y = (H-E)X in FP64 for those bands
        // only, Rayleigh-Ritz on H with the FP64 overlap, FP64 residuals.  A
        // failed check tightens the FP32 target.  A stalled FP32 stage is
        // checked the same way when its last H check was already within tol;
        // otherwise, or when that check fails, FP64 iterations take over.
        for (double margin : {0.5, 0.25, 0.125}) {
            status = S.run<float2>(B32, c->opt.maxit - iters, margin * tol, true, iters, 10, eps, resid, order, nres);
            if (S.verbose)
                fprintf(stderr, "[fs] FP32 stage to %.2f tol: %d iterations, %.2f s, status %d, last H check %.3e\n",
                        margin, iters, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(),
                        status, S.last_hworst);
            vec_convert<float2, double2>(c, B32.X.as<float2>(), B64.X.as<double2>(), (size_t)m * npw);
            const bool stalled_close = status == 2 && S.last_hworst >= 0 && S.last_hworst <= tol;
            if (status != 1 && !stalled_close) break;
            std::vector<double> th(m);
            FS_CUDA(cudaMemcpyAsync(th.data(), S.s.theta.p, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            FS_CUDA(cudaStreamSynchronize(c->stream));
            int nw = nstates;
            const double tie = lowest ? 1e-3 * std::max(1.0, std::fabs(th[nstates - 1])) : 1e-3 * th[nstates - 1];
            while (nw < m && th[nw] <= th[nstates - 1] + tie) ++nw;
            S.HE(B64.X.as<double2>(), B64.Y.as<double2>(), nw);
            S.h_ritz<double2>(B64, th, nres, eps, resid, order);
            done = true;
            for (int i : order) done = done && resid[i] <= tol;
            if (S.verbose)
                fprintf(stderr, "[fs] FP64 check of the FP32 result: %s\n", done ? "passed" : "failed");
            if (done || iters >= c->opt.maxit || status != 1) break;
        }
        iters_mixed = iters;
    } else {
        B64.alloc(m, npw);
        FS_CUDA(cudaMemcpyAsync(B64.X.p, x0.p, (size_t)m * npw * sizeof(double2), cudaMemcpyDeviceToDevice,
                                c->stream));
    }
    if (!done) {
        B64.alloc(m, npw);
        S.init_block<double2>(B64);
        status = S.run<double2>(B64, std::max(0, c->opt.maxit - iters), tol, false, iters, 0, eps, resid, order, nres);
    }
    if (status != 1 && !done) {
        // not converged: report the current H-Ritz pairs of the wanted block
        // (a passed FP64 check of a stalled FP32 stage has already filled them;
        // the residual blocks exist only once FP64 iterations have run)
        B64.alloc(m, npw);
        std::vector<double> ra, th;
        S.a_residuals(B64, ra, th);
        S.h_ritz<double2>(B64, th, nres, eps, resid, order);
    }
    if (S.verbose)
        fprintf(stderr, "[fs] done: %d iterations, %.2f s; Rayleigh-Ritz bases: %lld full, %lld with dropped "
                        "directions, %lld by eigendecomposition\n", iters,
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(), S.n_chol_drop[0],
                S.n_chol_drop[1], S.n_svqb);
    c->result_states.ensure((size_t)nstates * npw * sizeof(double2));
    int nconv = 0;
    for (int i = 0; i < nstates; ++i) {
        int j = order[i];
        res->eps[i] = eps[j];
        res->resid[i] = resid[j];
        if (resid[j] <= tol) ++nconv;
        FS_CUDA(cudaMemcpyAsync(c->result_states.as<double2>() + (size_t)i * npw, B64.tX.as<double2>() + (size_t)j * npw,
                                npw * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    }
    FS_CUDA(cudaStreamSynchronize(c->stream));
    c->nresult = nstates;
    c->result_eps.assign(res->eps, res->eps + nstates);
    c->result_resid.assign(res->resid, res->resid + nstates);
    res->nconv = nconv;
    res->iters = iters;
    res->iters_mixed = iters_mixed;
    res->n_hpsi = S.n_hpsi;
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    (void)status;
    return nconv == nstates ? FS_OK : FS_ERR_NOT_CONVERGED;
}
