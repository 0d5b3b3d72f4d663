// Folded-spectrum linear solve (paper Sec. II.C, Eq. wl1) on the GPU.
//
// For each right-hand side w_l the PCG minimises
//   F = 1/2 <psi|(H - E)^2|psi> - Re<psi|w'>,   w' = (H - E) w,
// i.e. solves (H - E)^2 psi = (H - E) w, whose solution solves the
// scattering-state equation (H - E) psi = w (Eq. wl) where H - E is
// invertible.  Preconditioner: the G-space M(G) = 1 / ((|q|^2/2 - E)^2 + dE^2),
// or, with eigenstates set, the paper's
//   M' = M (1 - sum_i |phi_i><phi_i|) + sum_i |phi_i><phi_i| / ((eps_i - E)^2 + Delta_i^2)
// applied as written.  Directions: Polak-Ribiere coefficient clamped at zero.
// Error: ||(H - E) psi - w||, with (H - E) psi carried by linearity during the
// iteration and recomputed from psi at the end.  FP64 throughout; all right-
// hand sides iterate together (one batched H application per step), a
// converged one is frozen (step length zero).
#include "fs_common.cuh"


#include <algorithm>
#include <chrono>
#include <cmath>

namespace {

constexpr int LT = 256;      // threads per block
constexpr int LCH = 64;      // blocks per row in the row reductions (partial sums, fixed order)

__device__ __forceinline__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = LT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// part[row][chunk] = (Re, Im) of sum over the chunk of conj(a) b
__global__ void __launch_bounds__(LT)
dot_part_kernel(const double2* __restrict__ A, const double2* __restrict__ B, long npw, double2* __restrict__ part) {
    __shared__ double sh[LT];
    const int row = blockIdx.y;
    const long per = (npw + LCH - 1) / LCH;
    const long g0 = blockIdx.x * per, g1 = min(npw, g0 + per);
    const double2* a = A + (long)row * npw;
    const double2* b = B + (long)row * npw;
    double re = 0, im = 0;
    for (long g = g0 + threadIdx.x; g < g1; g += LT) {
        const double2 x = a[g], y = b[g];
        re += x.x * y.x + x.y * y.y;
        im += x.x * y.y - x.y * y.x;
    }
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    if (threadIdx.x == 0) part[(long)row * LCH + blockIdx.x] = make_double2(re, im);
}

// out[row] = sum over chunks of part[row][chunk], in chunk order
__global__ void part_sum_kernel(const double2* __restrict__ part, int nrow, double2* __restrict__ out) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nrow) return;
    double re = 0, im = 0;
    for (int k = 0; k < LCH; ++k) {
        re += part[(long)row * LCH + k].x;
        im += part[(long)row * LCH + k].y;
    }
    out[row] = make_double2(re, im);
}

// psi += a p;  y += a yp;  r_old = r;  r -= a ap;  part = |y - w|^2 over the chunk
__global__ void __launch_bounds__(LT)
update_kernel(double2* __restrict__ psi, double2* __restrict__ y, double2* __restrict__ r, double2* __restrict__ r_old,
              const double2* __restrict__ p, const double2* __restrict__ yp, const double2* __restrict__ ap,
              const double2* __restrict__ w, const double* __restrict__ alpha, long npw, double2* __restrict__ part) {
    __shared__ double sh[LT];
    const int row = blockIdx.y;
    const long per = (npw + LCH - 1) / LCH;
    const long g0 = blockIdx.x * per, g1 = min(npw, g0 + per);
    const double a = alpha[row];
    const long o = (long)row * npw;
    double e2 = 0;
    for (long g = g0 + threadIdx.x; g < g1; g += LT) {
        const long i = o + g;
        const double2 pp = p[i], yy = yp[i], aa = ap[i], rr = r[i];
        double2 s = psi[i];
        psi[i] = make_double2(s.x + a * pp.x, s.y + a * pp.y);
        double2 t = y[i];
        t = make_double2(t.x + a * yy.x, t.y + a * yy.y);
        y[i] = t;
        r_old[i] = rr;
        r[i] = make_double2(rr.x - a * aa.x, rr.y - a * aa.y);
        const double2 ww = w[i];
        const double dx = t.x - ww.x, dy = t.y - ww.y;
        e2 += dx * dx + dy * dy;
    }
    e2 = block_sum(e2, sh);
    if (threadIdx.x == 0) part[(long)row * LCH + blockIdx.x] = make_double2(e2, 0.0);
}

// out = a - b (elementwise over total complex entries)
__global__ void sub_kernel(const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ out,
                           long total) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x)
        out[t] = make_double2(a[t].x - b[t].x, a[t].y - b[t].y);
}

// Z = M(G) U for every row, M(G) = 1 / ((kin - E)^2 + dE^2)
__global__ void precond_kernel(const double2* __restrict__ U, double2* __restrict__ Z, const double* __restrict__ kin,
                               long npw, long total, double e_ref, double dE2) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const double d = kin[t % npw] - e_ref;
        const double m = 1.0 / (d * d + dE2);
        Z[t] = make_double2(m * U[t].x, m * U[t].y);
    }
}

// T[i + j n] *= c[i]
__global__ void scale_coef_kernel(double2* __restrict__ T, const double* __restrict__ c, int n, int nrhs) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * nrhs) return;
    const double f = c[t % n];
    T[t] = make_double2(f * T[t].x, f * T[t].y);
}

// P = Z + beta P per row
__global__ void xpby_kernel(const double2* __restrict__ Z, double2* __restrict__ P, const double* __restrict__ beta,
                            long npw, long total) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const double b = beta[t / npw];
        P[t] = make_double2(Z[t].x + b * P[t].x, Z[t].y + b * P[t].y);
    }
}

inline int eblocks(long total) { return (int)std::min<long>(152 * 8, (total + LT - 1) / LT); }

struct Lin {
    fs_ctx* c;
    double E;
    int nrhs;
    long npw;
    long long n_hpsi = 0;
    double2 *psi, *y, *r, *r_old, *p, *yp, *ap, *z, *u;
    double2 *T, *part, *dots;  // [lin_n][nrhs], [nrhs][LCH], [nrhs]
    double *cvec, *scal;       // [lin_n], [nrhs]

    void HE(const double2* in, double2* out) {
        apply_H_impl<double2>(c, in, out, nrhs, E, nullptr);
        n_hpsi += nrhs;
    }

    // Re<a_l, b_l> for every row (host)
    std::vector<double> re_dots(const double2* a, const double2* b) {
        ProfScope ps(c, KS_VECTOR64, 2.0 * nrhs * npw * sizeof(double2), 8.0 * nrhs * npw);
        dot_part_kernel<<<dim3(LCH, nrhs), LT, 0, c->stream>>>(a, b, npw, part);
        part_sum_kernel<<<(nrhs + 127) / 128, 128, 0, c->stream>>>(part, nrhs, dots);
        FS_CUDA(cudaGetLastError());
        std::vector<double2> h(nrhs);
        FS_CUDA(cudaMemcpyAsync(h.data(), dots, nrhs * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        std::vector<double> out(nrhs);
        for (int l = 0; l < nrhs; ++l) out[l] = h[l].x;
        return out;
    }

    void upload_scal(const std::vector<double>& v) {
        FS_CUDA(cudaMemcpyAsync(scal, v.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    }

    // z = M' r (M alone without eigenstates)
    void precond(const double2* R, double2* Z) {
        const long total = (long)nrhs * npw;
        const double dE = c->opt.dE > 0 ? c->opt.dE : 0.5;
        const int n = c->lin_n;
        if (n == 0) {
            ProfScope ps(c, KS_VECTOR64, 2.0 * total * sizeof(double2), 6.0 * total);
            precond_kernel<<<eblocks(total), LT, 0, c->stream>>>(R, Z, c->kin.as<double>(), npw, total, E, dE * dE);
            FS_CUDA(cudaGetLastError());
            return;
        }
        const double2* phi = c->lin_phi.as<double2>();
        // T = <phi_i|r_l>;  u = r - Phi T;  z = M u;  z += Phi (c T)
        gemm_gram<double2>(c, n, nrhs, (int)npw, phi, npw, nullptr, R, npw, nullptr, T, 1, n, 1.0, 0.0, KS_GRAM);
        FS_CUDA(cudaMemcpyAsync(u, R, total * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
        gemm_nn<double2, double2>(c, nrhs, (int)npw, n, T, n, 1, phi, npw, nullptr, u, npw, nullptr, -1.0, 1.0, u, npw,
                                  KS_ROTATE);
        {
            ProfScope ps(c, KS_VECTOR64, 2.0 * total * sizeof(double2), 6.0 * total);
            precond_kernel<<<eblocks(total), LT, 0, c->stream>>>(u, Z, c->kin.as<double>(), npw, total, E, dE * dE);
            scale_coef_kernel<<<(n * nrhs + 255) / 256, 256, 0, c->stream>>>(T, cvec, n, nrhs);
            FS_CUDA(cudaGetLastError());
        }
        gemm_nn<double2, double2>(c, nrhs, (int)npw, n, T, n, 1, phi, npw, nullptr, Z, npw, nullptr, 1.0, 1.0, Z, npw,
                                  KS_ROTATE);
    }

    // ||a_l - b_l|| for every row (host), via u as scratch
    std::vector<double> diff_norms(const double2* a, const double2* b) {
        const long total = (long)nrhs * npw;
        sub_kernel<<<eblocks(total), LT, 0, c->stream>>>(a, b, u, total);
        FS_CUDA(cudaGetLastError());
        std::vector<double> d = re_dots(u, u);
        for (double& v : d) v = std::sqrt(std::max(v, 0.0));
        return d;
    }
};

}  // namespace

fs_status linear_solve_impl(fs_ctx* c, double e_ref, const double2* w, double2* psi_out, int nrhs, bool from_psi,
                            double tol, int maxit, fs_linres* res) {
    auto t0 = std::chrono::steady_clock::now();
    Lin L;
    L.c = c;
    L.E = e_ref;
    L.nrhs = nrhs;
    L.npw = c->npw;
    const size_t vb = (size_t)nrhs * c->npw * sizeof(double2);
    for (dbuf& d : c->lin_vec) d.ensure(vb);
    double2** vecs[9] = {&L.psi, &L.y, &L.r, &L.r_old, &L.p, &L.yp, &L.ap, &L.z, &L.u};
    for (int i = 0; i < 9; ++i) *vecs[i] = c->lin_vec[i].as<double2>();
    const int n = c->lin_n;
    const size_t sb = sizeof(double2) * ((size_t)std::max(n, 1) * nrhs + (size_t)nrhs * LCH + nrhs) +
                      sizeof(double) * ((size_t)std::max(n, 1) + nrhs);
    c->lin_small.ensure(sb);
    L.T = c->lin_small.as<double2>();
    L.part = L.T + (size_t)std::max(n, 1) * nrhs;
    L.dots = L.part + (size_t)nrhs * LCH;
    L.cvec = reinterpret_cast<double*>(L.dots + nrhs);
    L.scal = L.cvec + std::max(n, 1);
    if (n > 0) {
        std::vector<double> cv(n);
        for (int i = 0; i < n; ++i) {
            const double d = c->lin_eps[i] - e_ref;
            cv[i] = 1.0 / (d * d + c->lin_delta[i] * c->lin_delta[i]);
        }
        FS_CUDA(cudaMemcpyAsync(L.cvec, cv.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    }
    const long total = (long)nrhs * L.npw;
    // start: psi_0 (given or zero), y = (H - E) psi_0, r = (H - E)(w - y)
    if (from_psi) {
        FS_CUDA(cudaMemcpyAsync(L.psi, psi_out, vb, cudaMemcpyDeviceToDevice, c->stream));
        L.HE(L.psi, L.y);
    } else {
        FS_CUDA(cudaMemsetAsync(L.psi, 0, vb, c->stream));
        FS_CUDA(cudaMemsetAsync(L.y, 0, vb, c->stream));
    }
    sub_kernel<<<eblocks(total), LT, 0, c->stream>>>(w, L.y, L.yp, total);
    FS_CUDA(cudaGetLastError());
    std::vector<double> err(nrhs);
    {
        std::vector<double> e2 = L.re_dots(L.yp, L.yp);
        for (int l = 0; l < nrhs; ++l) err[l] = std::sqrt(std::max(e2[l], 0.0));
    }
    L.HE(L.yp, L.r);
    L.precond(L.r, L.z);
    FS_CUDA(cudaMemcpyAsync(L.p, L.z, vb, cudaMemcpyDeviceToDevice, c->stream));
    std::vector<double> zr = L.re_dots(L.z, L.r);
    std::vector<char> done(nrhs);
    bool all = true;
    for (int l = 0; l < nrhs; ++l) {
        done[l] = err[l] <= tol;
        all = all && done[l];
    }
    int it = 0;
    std::vector<double> a(nrhs), b(nrhs);
    while (!all && it < maxit) {
        L.HE(L.p, L.yp);
        L.HE(L.yp, L.ap);
        std::vector<double> pap = L.re_dots(L.p, L.ap);
        for (int l = 0; l < nrhs; ++l) a[l] = (done[l] || !(pap[l] > 0)) ? 0.0 : zr[l] / pap[l];
        L.upload_scal(a);
        {
            ProfScope ps(c, KS_VECTOR64, 9.0 * total * sizeof(double2), 12.0 * total);
            update_kernel<<<dim3(LCH, nrhs), LT, 0, c->stream>>>(L.psi, L.y, L.r, L.r_old, L.p, L.yp, L.ap, w,
                                                                 L.scal, L.npw, L.part);
            part_sum_kernel<<<(nrhs + 127) / 128, 128, 0, c->stream>>>(L.part, nrhs, L.dots);
            FS_CUDA(cudaGetLastError());
        }
        std::vector<double2> e2(nrhs);
        FS_CUDA(cudaMemcpyAsync(e2.data(), L.dots, nrhs * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        ++it;
        all = true;
        for (int l = 0; l < nrhs; ++l) {
            err[l] = std::sqrt(std::max(e2[l].x, 0.0));
            if (!std::isfinite(err[l])) throw fs_error(FS_ERR_NUMERIC, "NaN/Inf in the linear-solve residual");
            done[l] = done[l] || err[l] <= tol;
            all = all && done[l];
        }
        if (all) break;
        L.precond(L.r, L.z);
        std::vector<double> zr_new = L.re_dots(L.z, L.r);
        std::vector<double> zro = L.re_dots(L.z, L.r_old);
        for (int l = 0; l < nrhs; ++l)
            b[l] = (done[l] || zr[l] == 0.0) ? 0.0 : std::max(0.0, (zr_new[l] - zro[l]) / zr[l]);
        L.upload_scal(b);
        xpby_kernel<<<eblocks(total), LT, 0, c->stream>>>(L.z, L.p, L.scal, L.npw, total);
        FS_CUDA(cudaGetLastError());
        zr = zr_new;
    }
    // the reported error is recomputed from psi
    L.HE(L.psi, L.y);
    err = L.diff_norms(L.y, w);
    FS_CUDA(cudaMemcpyAsync(psi_out, L.psi, vb, cudaMemcpyDeviceToDevice, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    ctx_check_errflag(c);
    bool conv = true;
    for (int l = 0; l < nrhs; ++l) {
        if (res->err) res->err[l] = err[l];
        conv = conv && err[l] <= tol;
    }
    res->iters = it;
    res->n_hpsi = L.n_hpsi;
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return conv ? FS_OK : FS_ERR_NOT_CONVERGED;
}

extern "C" {

fs_status fs_set_linear_states(fs_ctx* c, const void* phi, const double* eps, const double* delta, int n,
                               int where) {
    if (!c) return FS_ERR_ARG;
    if (n < 0 || (where != FS_HOST && where != FS_DEVICE) || (phi && (!eps || !delta)) ||
        (!phi && n > c->nresult)) {
        c->err = "fs_set_linear_states: bad arguments (n beyond the last solve's states?)";
        return FS_ERR_ARG;
    }
    try {
        c->lin_n = 0;
        c->lin_eps.clear();
        c->lin_delta.clear();
        if (n == 0) return FS_OK;
        const size_t bytes = (size_t)n * c->npw * sizeof(double2);
        c->lin_phi.ensure(bytes);
        if (phi) {
            FS_CUDA(cudaMemcpyAsync(c->lin_phi.p, phi, bytes,
                                    where == FS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                    c->stream));
            c->lin_eps.assign(eps, eps + n);
            c->lin_delta.assign(delta, delta + n);
        } else {
            FS_CUDA(cudaMemcpyAsync(c->lin_phi.p, c->result_states.p, bytes, cudaMemcpyDeviceToDevice, c->stream));
            c->lin_eps.assign(c->result_eps.begin(), c->result_eps.begin() + n);
            c->lin_delta.assign(c->result_resid.begin(), c->result_resid.begin() + n);
        }
        FS_CUDA(cudaStreamSynchronize(c->stream));
        c->lin_n = n;
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

fs_status fs_linear_solve(fs_ctx* c, double e_ref, const void* w, void* psi, int nrhs, int where, int from_psi,
                          double tol, int maxit, fs_linres* res) {
    if (!c) return FS_ERR_ARG;
    if (nrhs < 0 || (nrhs > 0 && (!w || !psi)) || (where != FS_HOST && where != FS_DEVICE) || !res ||
        !(tol > 0) || maxit < 0 || !std::isfinite(e_ref)) {
        c->err = "fs_linear_solve: bad arguments";
        return FS_ERR_ARG;
    }
    res->iters = 0;
    res->n_hpsi = 0;
    res->seconds = 0;
    if (nrhs == 0) return FS_OK;
    try {
        const size_t vb = (size_t)nrhs * c->npw * sizeof(double2);
        const double2* wd = (const double2*)w;
        double2* pd = (double2*)psi;
        if (where == FS_HOST) {
            // host buffers are staged through two context buffers
            c->lin_io[0].ensure(vb);
            c->lin_io[1].ensure(vb);
            FS_CUDA(cudaMemcpyAsync(c->lin_io[0].p, w, vb, cudaMemcpyHostToDevice, c->stream));
            if (from_psi) FS_CUDA(cudaMemcpyAsync(c->lin_io[1].p, psi, vb, cudaMemcpyHostToDevice, c->stream));
            wd = c->lin_io[0].as<double2>();
            pd = c->lin_io[1].as<double2>();
        }
        fs_status st = linear_solve_impl(c, e_ref, wd, pd, nrhs, from_psi != 0, tol, maxit, res);
        if (where == FS_HOST) {
            FS_CUDA(cudaMemcpyAsync(psi, pd, vb, cudaMemcpyDeviceToHost, c->stream));
            FS_CUDA(cudaStreamSynchronize(c->stream));
        }
        c->err = st == FS_OK ? "" : "fs_linear_solve: some right-hand side did not reach tol";
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
