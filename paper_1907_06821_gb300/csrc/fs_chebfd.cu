// Chebyshev filter diagonalisation (paper Sec. II.C) and spectral bounds.
//
// ChebFD: a block of vectors is filtered by p(Hs) = sum_n g_n mu_n T_n(Hs),
// Hs = (H - c)/e the spectrum mapped to [-1, 1], mu_n the Chebyshev
// coefficients of the indicator of the window [E - d, E + d] and g_n the
// Jackson damping for degree N; T_n by the three-term recurrence
// T_{n+1} = 2 Hs T_n - T_{n-1}, one batched H application per degree.  Then a
// Rayleigh-Ritz step of H on the filtered block (basis from the eigenvectors
// of its overlap, dropping eigenvalues below 1e-12 of the largest) gives the
// vectors of the next step.  FP64 throughout.  The pairs inside the window,
// ordered by (|eps - E|, eps), become the context's result (fs_get_states,
// fs_set_linear_states with phi = NULL).
//
// Spectral bounds: k Lanczos steps on one seeded vector; the extreme
// eigenvalues of the tridiagonal matrix widened by the norm of the last
// residual vector (the estimate used to place Chebyshev filters).
#include "fs_common.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <vector>

namespace {

constexpr int CT = 256;

inline int cblocks(long total) { return (int)std::min<long>(152 * 8, (total + CT - 1) / CT); }

// T_next = s HT - T_prev (written over T_prev);  Y += coef T_next
__global__ void cheb_step_kernel(const double2* __restrict__ HT, double2* __restrict__ Tp, double2* __restrict__ Y,
                                 double s, double coef, long total) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const double2 h = HT[t], p = Tp[t];
        const double2 n = make_double2(s * h.x - p.x, s * h.y - p.y);
        Tp[t] = n;
        const double2 y = Y[t];
        Y[t] = make_double2(y.x + coef * n.x, y.y + coef * n.y);
    }
}

// T1 = s HT;  Y = c0 X + c1 T1
__global__ void cheb_first_kernel(const double2* __restrict__ X, const double2* __restrict__ HT,
                                  double2* __restrict__ T1, double2* __restrict__ Y, double s, double c0, double c1,
                                  long total) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const double2 x = X[t], h = HT[t];
        const double2 t1 = make_double2(s * h.x, s * h.y);
        T1[t] = t1;
        Y[t] = make_double2(c0 * x.x + c1 * t1.x, c0 * x.y + c1 * t1.y);
    }
}

// column j of T (n x k, ld n) *= 1 / sqrt(lam[j])
__global__ void col_rsqrt_kernel(double2* T, int n, int k, const double* lam) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)n * k) return;
    const double f = rsqrt(lam[t / n]);
    T[t].x *= f;
    T[t].y *= f;
}

double jackson(int n, int N) {
    const double a = M_PI / (N + 1);
    return ((N - n + 1) * std::cos(a * n) + std::sin(a * n) / std::tan(a)) / (N + 1);
}

// mu_n g_n of the window [t1, t2] in [-1, 1], n = 0..N
std::vector<double> window_coefficients(double t1, double t2, int N) {
    const double th1 = std::acos(std::max(-1.0, std::min(1.0, t1)));
    const double th2 = std::acos(std::max(-1.0, std::min(1.0, t2)));
    std::vector<double> c(N + 1);
    c[0] = (th1 - th2) / M_PI * jackson(0, N);
    for (int n = 1; n <= N; ++n)
        c[n] = 2.0 * (std::sin(n * th1) - std::sin(n * th2)) / (n * M_PI) * jackson(n, N);
    return c;
}

// number of eigenvalues below x of the symmetric tridiagonal (a, b) (Sturm count)
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
    int cnt = 0;
    double q = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        const double off = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
        q = a[i] - x - (i > 0 ? off / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// k-th smallest eigenvalue (0-based) of the tridiagonal by bisection on the Sturm count
double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int k) {
    double lo = 1e300, hi = -1e300;
    for (size_t i = 0; i < a.size(); ++i) {
        const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < a.size() ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-14 * std::max(1.0, std::fabs(hi) + std::fabs(lo)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(a, b, mid) > k) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Re sum conj(x) y over n entries: per-block partial sums in a fixed order,
// added on the host in block order (deterministic)
constexpr int DOT_BLOCKS = 256;
__global__ void dot_re_kernel(const double2* __restrict__ x, const double2* __restrict__ y, long n, double* part) {
    __shared__ double sh[CT];
    double s = 0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        s += x[t].x * y[t].x + x[t].y * y[t].y;
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = CT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// y += a x
__global__ void axpy_kernel(long n, double a, const double2* __restrict__ x, double2* __restrict__ y) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        y[t] = make_double2(y[t].x + a * x[t].x, y[t].y + a * x[t].y);
}

// x *= a
__global__ void scal_kernel(long n, double a, double2* __restrict__ x) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        x[t] = make_double2(a * x[t].x, a * x[t].y);
}

double zdot_re(fs_ctx* c, long n, const double2* x, const double2* y) {
    dbuf& part = c->dense.gpart;
    part.ensure(DOT_BLOCKS * sizeof(double));
    dot_re_kernel<<<DOT_BLOCKS, CT, 0, c->stream>>>(x, y, n, part.as<double>());
    FS_CUDA(cudaGetLastError());
    std::vector<double> h(DOT_BLOCKS);
    FS_CUDA(cudaMemcpyAsync(h.data(), part.p, DOT_BLOCKS * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    double s = 0;
    for (double v : h) s += v;
    return s;
}

double znrm2(fs_ctx* c, long n, const double2* x) { return std::sqrt(std::max(0.0, zdot_re(c, n, x, x))); }

void zaxpy(fs_ctx* c, long n, double a, const double2* x, double2* y) {
    axpy_kernel<<<cblocks(n), CT, 0, c->stream>>>(n, a, x, y);
    FS_CUDA(cudaGetLastError());
}

void zscal(fs_ctx* c, long n, double a, double2* x) {
    scal_kernel<<<cblocks(n), CT, 0, c->stream>>>(n, a, x);
    FS_CUDA(cudaGetLastError());
}

// every eigenpair of the Hermitian n x n matrix A (column-major): vectors overwrite A, values to w (device)
void heevd(fs_ctx* c, int n, double2* A, double* w) {
    dbuf& Z = c->dense.U;
    Z.ensure((size_t)n * n * sizeof(double2));
    dense_heev(c, n, A, n, w, Z.as<double2>(), n);
    FS_CUDA(cudaMemcpyAsync(A, Z.p, (size_t)n * n * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
}

}  // namespace

void spectral_bounds_impl(fs_ctx* c, int iters, double* emin, double* emax) {
    const long npw = c->npw;
    dbuf v, vp, f;
    v.alloc(npw * sizeof(double2));
    vp.alloc(npw * sizeof(double2));
    f.alloc(npw * sizeof(double2));
    vec_damp_random(c, v.as<double2>(), 1, 0, 20191907ull);
    zscal(c, npw, 1.0 / znrm2(c, npw, v.as<double2>()), v.as<double2>());
    std::vector<double> a, b;
    double beta = 0;
    const int k = std::max(2, std::min(iters, (int)npw));
    for (int j = 0; j < k; ++j) {
        apply_H_impl<double2>(c, v.as<double2>(), f.as<double2>(), 1, 0.0, nullptr);
        if (j > 0) zaxpy(c, npw, -beta, vp.as<double2>(), f.as<double2>());
        const double alpha = zdot_re(c, npw, v.as<double2>(), f.as<double2>());
        zaxpy(c, npw, -alpha, v.as<double2>(), f.as<double2>());
        a.push_back(alpha);
        beta = znrm2(c, npw, f.as<double2>());
        if (j + 1 == k || beta < 1e-12) break;
        b.push_back(beta);
        std::swap(v.p, vp.p);
        FS_CUDA(cudaMemcpyAsync(v.p, f.p, npw * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
        zscal(c, npw, 1.0 / beta, v.as<double2>());
    }
    *emin = tridiag_eig(a, b, 0) - beta;
    *emax = tridiag_eig(a, b, (int)a.size() - 1) + beta;
    FS_CUDA(cudaStreamSynchronize(c->stream));
}

fs_status chebfd_impl(fs_ctx* c, double e_ref, double d, double emin, double emax, int degree, int nvec, int steps,
                      unsigned long long seed, int nwant, fs_chebfd_result* res) {
    auto t0 = std::chrono::steady_clock::now();
    const long npw = c->npw;
    long long n_hpsi = 0;
    const double cc = 0.5 * (emax + emin), e = 0.5 * (emax - emin);
    const std::vector<double> coef = window_coefficients((e_ref - d - cc) / e, (e_ref + d - cc) / e, degree);
    const size_t vb = (size_t)nvec * npw * sizeof(double2);
    dbuf X, Tp, Tc, HT, Y, small, small2, evals;
    for (dbuf* q : {&X, &Tp, &Tc, &HT, &Y}) q->alloc(vb);
    small.alloc((size_t)nvec * nvec * sizeof(double2));
    small2.alloc((size_t)nvec * nvec * sizeof(double2));
    dbuf small3;
    small3.alloc((size_t)nvec * nvec * sizeof(double2));
    evals.alloc(nvec * sizeof(double));
    vec_damp_random(c, X.as<double2>(), nvec, 0, seed);
    int m = nvec;  // vectors in the block
    std::vector<double> eps_h;
    for (int step = 0; step < steps; ++step) {
        const long total = (long)m * npw;
        // filter: Y = p(Hs) X
        double2* x = X.as<double2>();
        apply_H_impl<double2>(c, x, HT.as<double2>(), m, cc, nullptr);
        n_hpsi += m;
        {
            ProfScope ps(c, KS_VECTOR64, 4.0 * total * sizeof(double2), 6.0 * total);
            cheb_first_kernel<<<cblocks(total), CT, 0, c->stream>>>(x, HT.as<double2>(), Tc.as<double2>(),
                                                                    Y.as<double2>(), 1.0 / e, coef[0],
                                                                    degree >= 1 ? coef[1] : 0.0, total);
            FS_CUDA(cudaMemcpyAsync(Tp.p, x, (size_t)total * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
        }
        for (int n = 2; n <= degree; ++n) {
            apply_H_impl<double2>(c, Tc.as<double2>(), HT.as<double2>(), m, cc, nullptr);
            n_hpsi += m;
            ProfScope ps(c, KS_VECTOR64, 5.0 * total * sizeof(double2), 6.0 * total);
            cheb_step_kernel<<<cblocks(total), CT, 0, c->stream>>>(HT.as<double2>(), Tp.as<double2>(), Y.as<double2>(),
                                                                   2.0 / e, coef[n], total);
            FS_CUDA(cudaGetLastError());
            std::swap(Tp.p, Tc.p);
        }
        // Rayleigh-Ritz of H on Y: GB = Y^H Y, GA = Y^H H Y
        double2* y = Y.as<double2>();
        double2* hy = HT.as<double2>();
        apply_H_impl<double2>(c, y, hy, m, 0.0, nullptr);
        n_hpsi += m;
        double2* GB = small.as<double2>();
        double2* GA = small2.as<double2>();
        gemm_gram<double2>(c, m, m, (int)npw, y, npw, nullptr, y, npw, nullptr, GB, 1, m, 1.0, 0.0, KS_GRAM);
        gemm_gram<double2>(c, m, m, (int)npw, y, npw, nullptr, hy, npw, nullptr, GA, 1, m, 1.0, 0.0, KS_GRAM);
        std::vector<double> lam(m);
        {
            ProfScope ps(c, KS_DENSE_LA, 0.0, 0.0);
            heevd(c, m, GB, evals.as<double>());
        }
        FS_CUDA(cudaMemcpyAsync(lam.data(), evals.p, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        int k = 0;
        for (int i = m - 1; i >= 0 && lam[i] > 1e-12 * lam[m - 1]; --i) ++k;
        if (k == 0) throw fs_error(FS_ERR_NUMERIC, "ChebFD: the filtered block vanished (window outside the bounds?)");
        double2* T = GB + (long)(m - k) * m;  // kept eigenvectors, m x k
        col_rsqrt_kernel<<<(int)(((long)m * k + 255) / 256), 256, 0, c->stream>>>(T, m, k, evals.as<double>() + (m - k));
        FS_CUDA(cudaGetLastError());
        double2* tmp = small3.as<double2>();
        double2* Ar = GA;  // reuse after the product: A_r = T^H GA T into small3 then back
        {
            ProfScope ps(c, KS_DENSE_LA, 0.0, 16.0 * (double)m * m * k);
            dense_gemm(c, 0, 0, m, k, m, 1.0, GA, m, T, m, 0.0, tmp, m);
            dense_gemm(c, 1, 0, k, k, m, 1.0, T, m, tmp, m, 0.0, Ar, k);
            heevd(c, k, Ar, evals.as<double>());
            // coefficients C = T V (m x k) into tmp
            dense_gemm(c, 0, 0, m, k, k, 1.0, T, m, Ar, k, 0.0, tmp, m);
        }
        eps_h.assign(k, 0.0);
        FS_CUDA(cudaMemcpyAsync(eps_h.data(), evals.p, k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        // X = C^T Y rows (k vectors), HX = C^T HY (into Tc)
        gemm_nn<double2, double2>(c, k, (int)npw, m, tmp, m, 1, y, npw, nullptr, X.as<double2>(), npw, nullptr, 1.0,
                                  0.0, nullptr, 0, KS_ROTATE);
        gemm_nn<double2, double2>(c, k, (int)npw, m, tmp, m, 1, hy, npw, nullptr, Tc.as<double2>(), npw, nullptr, 1.0,
                                  0.0, nullptr, 0, KS_ROTATE);
        FS_CUDA(cudaStreamSynchronize(c->stream));
        m = k;
    }
    // residuals of the final Ritz pairs (X, HX in Tc, eigenvalues in evals)
    std::vector<double> resid(m);
    vec_resid_shift<double2>(c, X.as<double2>(), Tc.as<double2>(), evals.as<double>(), m, small.as<double>());
    FS_CUDA(cudaMemcpyAsync(resid.data(), small.p, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    std::vector<int> order;
    for (int i = 0; i < m; ++i)
        if (std::fabs(eps_h[i] - e_ref) <= d) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) {
        const double dp = std::fabs(eps_h[p] - e_ref), dq = std::fabs(eps_h[q] - e_ref);
        if (dp != dq) return dp < dq;
        return eps_h[p] < eps_h[q];
    });
    const int nf = std::min((int)order.size(), nwant);
    c->result_states.ensure((size_t)std::max(nf, 1) * npw * sizeof(double2));
    c->result_eps.assign(nf, 0.0);
    c->result_resid.assign(nf, 0.0);
    for (int i = 0; i < nf; ++i) {
        const int j = order[i];
        FS_CUDA(cudaMemcpyAsync(c->result_states.as<double2>() + (size_t)i * npw, X.as<double2>() + (size_t)j * npw,
                                npw * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
        c->result_eps[i] = eps_h[j];
        c->result_resid[i] = resid[j];
        if (res->eps) res->eps[i] = eps_h[j];
        if (res->resid) res->resid[i] = resid[j];
    }
    FS_CUDA(cudaStreamSynchronize(c->stream));
    ctx_check_errflag(c);
    c->nresult = nf;
    res->nfound = nf;
    res->n_hpsi = n_hpsi;
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return FS_OK;
}

extern "C" {

fs_status fs_spectral_bounds(fs_ctx* c, int iters, double* emin, double* emax) {
    if (!c) return FS_ERR_ARG;
    if (iters < 2 || !emin || !emax) {
        c->err = "fs_spectral_bounds: bad arguments";
        return FS_ERR_ARG;
    }
    try {
        spectral_bounds_impl(c, iters, emin, emax);
        c->err.clear();
        return FS_OK;
    } catch (const fs_error& e) {
        c->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        c->err = "host allocation failed";
        return FS_ERR_OOM;
    }
}

fs_status fs_chebfd(fs_ctx* c, double e_ref, double half_width, double emin, double emax, int degree, int nvec,
                    int steps, unsigned long long seed, int nwant, fs_chebfd_result* res) {
    if (!c) return FS_ERR_ARG;
    if (!res || !(half_width > 0) || !(emax > emin) || degree < 1 || nvec < 1 || nvec > c->npw || steps < 1 ||
        nwant < 0 || (nwant > 0 && (!res->eps || !res->resid)) || !std::isfinite(e_ref) || e_ref < emin ||
        e_ref > emax) {
        c->err = "fs_chebfd: bad arguments";
        return FS_ERR_ARG;
    }
    try {
        fs_status st = chebfd_impl(c, e_ref, half_width, emin, emax, degree, nvec, steps, seed, nwant, res);
        c->err.clear();
        return st;
    } catch (const fs_error& e) {
        c->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        c->err = "host allocation failed";
        return FS_ERR_OOM;
    }
}

}  // extern "C"
