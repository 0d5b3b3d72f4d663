// C ABI of the learned G-shell preconditioner: training from the context's own
// solves, weight import/export, and direct evaluation of the network's output,
// loss and gradient (for checking against a reference implementation).
#include "fs_common.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

void ctx_ensure_fp32(fs_ctx* c);

namespace {
template <typename Fn> fs_status guard(fs_ctx* c, Fn fn) {
    try {
        fn();
        c->err.clear();
        return FS_OK;
    } catch (const fs_error& e) {
        c->err = e.msg;
        return e.code;
    }
}

__global__ void d2f_kernel(const double2* in, float2* out, long n) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        out[t] = make_float2((float)in[t].x, (float)in[t].y);
}

// Features (and labels) of caller-given residual rows, through the same device
// steps a recording solve takes: the correction E = Xref Xref^H x - x by the
// solver's GEMMs and kernel, the shell sums and the feature/label kernel.
template <typename T2>
void features_of(fs_ctx* c, const T2* R, const T2* X, const T2* Xref, int nref, const double* d, int nb, float* F,
                 float* zt, float* wt) {
    Mlp& L = c->mlp;
    const long npw = c->npw;
    std::vector<double2> dots(nb);
    std::vector<int> ident(nb);
    for (int i = 0; i < nb; ++i) {
        dots[i] = make_double2(d[i], 0.0);
        ident[i] = i;
    }
    dbuf dd, map;
    dd.alloc(nb * sizeof(double2));
    map.alloc(nb * sizeof(int));
    FS_CUDA(cudaMemcpyAsync(dd.p, dots.data(), nb * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    FS_CUDA(cudaMemcpyAsync(map.p, ident.data(), nb * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    const T2* Err = nullptr;
    dbuf cg;
    if (X) {
        cg.alloc((size_t)nref * nb * sizeof(double2));
        L.proj.ensure((size_t)nb * npw * sizeof(T2));
        L.err.ensure((size_t)nb * npw * sizeof(T2));
        gemm_gram<T2>(c, nref, nb, npw, Xref, npw, nullptr, X, npw, map.as<int>(), cg.as<double2>(), 1, nref, 1.0,
                      0.0);
        gemm_nn<T2, double2>(c, nb, npw, nref, cg.as<double2>(), nref, 1, Xref, npw, nullptr, L.proj.as<T2>(), npw,
                             nullptr, 1.0, 0.0, nullptr, 0);
        mlp_err_from_proj<T2>(c, L.proj.as<T2>(), X, map.as<int>(), nb, L.err.as<T2>());
        Err = L.err.as<T2>();
    }
    mlp_features<T2>(c, R, map.as<int>(), nb, dd.as<double2>(), Err, F, zt, wt);
    FS_CUDA(cudaStreamSynchronize(c->stream));
}
}  // namespace

extern "C" {

fs_status fs_precond_train(fs_ctx* c, double e_ref, int nstates, double tol, int epochs, float lr, float* loss) {
    if (!c) return FS_ERR_ARG;
    if (nstates <= 0 || !(tol > 0) || epochs < 0 || !(lr > 0) || !loss) {
        c->err = "fs_precond_train: bad arguments";
        return FS_ERR_ARG;
    }
    const int saved = c->opt.precond;
    fs_status st = guard(c, [&] {
        mlp_setup(c);
        Mlp& L = c->mlp;
        std::vector<double> eps(nstates), res(nstates);
        fs_result r{};
        r.eps = eps.data();
        r.resid = res.data();
        // 1. reference solve with the paper's M(G)
        c->opt.precond = FS_PREC_M;
        fs_status s1 = solve_impl(c, e_ref, nstates, tol, &r);
        if (s1 != FS_OK && s1 != FS_ERR_NOT_CONVERGED) throw fs_error(s1, "reference solve failed");
        const long npw = c->npw;
        L.nref = nstates;
        L.xref64.ensure((size_t)nstates * npw * sizeof(double2));
        L.xref32.ensure((size_t)nstates * npw * sizeof(float2));
        FS_CUDA(cudaMemcpyAsync(L.xref64.p, c->result_states.p, (size_t)nstates * npw * sizeof(double2),
                                cudaMemcpyDeviceToDevice, c->stream));
        d2f_kernel<<<1024, 256, 0, c->stream>>>(L.xref64.as<double2>(), L.xref32.as<float2>(), (long)nstates * npw);
        // 2. the same solve again, recording residual / correction rows
        L.cap = std::max<long long>(1, (4ll << 20));
        L.recF.ensure((size_t)L.cap * 4 * sizeof(float));
        L.recz.ensure((size_t)L.cap * sizeof(float));
        L.recw.ensure((size_t)L.cap * sizeof(float));
        L.nrec = 0;
        L.nrec_bands = 0;
        L.record = true;
        fs_status s2 = solve_impl(c, e_ref, nstates, tol, &r);
        L.record = false;
        if (s2 != FS_OK && s2 != FS_ERR_NOT_CONVERGED) throw fs_error(s2, "recording solve failed");
        // 3. full-batch Adam on the recorded rows
        double l = 0;
        const double sw = std::max<double>(1.0, (double)L.nrec_bands);
        for (int e = 0; e < epochs; ++e) {
            l = mlp_loss_grad(c, L.recF.as<float>(), L.recz.as<float>(), L.recw.as<float>(), (int)L.nrec, sw);
            mlp_adam(c, lr);
        }
        if (epochs > 0 || L.nrec > 0)
            l = L.nrec > 0 ? mlp_loss_grad(c, L.recF.as<float>(), L.recz.as<float>(), L.recw.as<float>(),
                                           (int)L.nrec, sw)
                           : 0.0;
        *loss = (float)l;
    });
    c->opt.precond = saved;
    return st;
}

fs_status fs_precond_rows(fs_ctx* c, long long* nrows) {
    if (!c || !nrows) return FS_ERR_ARG;
    *nrows = c->mlp.nrec;
    return FS_OK;
}

fs_status fs_precond_weights(fs_ctx* c, float* w, int n, int set) {
    if (!c) return FS_ERR_ARG;
    if (!w || n != mlp_nparam()) {
        c->err = "fs_precond_weights: n must be " + std::to_string(mlp_nparam());
        return FS_ERR_ARG;
    }
    return guard(c, [&] {
        mlp_setup(c);
        Mlp& L = c->mlp;
        if (set) {
            FS_CUDA(cudaMemcpyAsync(L.P.p, w, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            FS_CUDA(cudaMemsetAsync(L.m.p, 0, n * sizeof(float), c->stream));
            FS_CUDA(cudaMemsetAsync(L.v.p, 0, n * sizeof(float), c->stream));
            L.step = 0;
            mlp_prepare(c);
        } else {
            FS_CUDA(cudaMemcpyAsync(w, L.P.p, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        }
        FS_CUDA(cudaStreamSynchronize(c->stream));
    });
}

fs_status fs_precond_eval(fs_ctx* c, const float* features, int rows, float* z) {
    if (!c) return FS_ERR_ARG;
    if (rows < 0 || (rows > 0 && (!features || !z))) {
        c->err = "fs_precond_eval: bad arguments";
        return FS_ERR_ARG;
    }
    return guard(c, [&] {
        mlp_setup(c);
        mlp_forward(c, features, rows, z);
        FS_CUDA(cudaStreamSynchronize(c->stream));
        ctx_check_errflag(c);  // a bounded wait of the tensor-core forward that gave up
    });
}

fs_status fs_precond_features(fs_ctx* c, double e_ref, const void* R, const void* X, const void* Xref, int nref,
                               const double* d, int nb, int precision, float* F, float* zt, float* wt) {
    if (!c) return FS_ERR_ARG;
    if (nb < 0 || !std::isfinite(e_ref) || (precision != FS_FP64 && precision != FS_MIXED) ||
        (nb > 0 && (!R || !d || !F)) || (X && (!Xref || nref <= 0 || !zt || !wt))) {
        c->err = "fs_precond_features: bad arguments";
        return FS_ERR_ARG;
    }
    if (nb == 0) return FS_OK;
    return guard(c, [&] {
        mlp_setup(c);
        Mlp& L = c->mlp;
        if (L.e_ref != e_ref || !L.Mdev.p) {
            L.e_ref = e_ref;
            L.Mdev.release();
        }
        if (precision == FS_MIXED) {
            ctx_ensure_fp32(c);
            features_of<float2>(c, (const float2*)R, (const float2*)X, (const float2*)Xref, nref, d, nb, F, zt, wt);
        } else {
            features_of<double2>(c, (const double2*)R, (const double2*)X, (const double2*)Xref, nref, d, nb, F, zt,
                                 wt);
        }
    });
}

fs_status fs_precond_loss_grad(fs_ctx* c, const float* features, const float* target, const float* weight, int rows,
                               float* loss, float* grad) {
    if (!c) return FS_ERR_ARG;
    if (rows <= 0 || !features || !target || !weight || !loss || !grad) {
        c->err = "fs_precond_loss_grad: bad arguments";
        return FS_ERR_ARG;
    }
    return guard(c, [&] {
        mlp_setup(c);
        std::vector<float> wh(rows);
        FS_CUDA(cudaMemcpy(wh.data(), weight, rows * sizeof(float), cudaMemcpyDeviceToHost));
        double sw = 0;
        for (float v : wh) sw += v;
        if (!(sw > 0)) throw fs_error(FS_ERR_ARG, "fs_precond_loss_grad: weights sum to zero");
        *loss = (float)mlp_loss_grad(c, features, target, weight, rows, sw);
        FS_CUDA(cudaMemcpyAsync(grad, c->mlp.g.p, mlp_nparam() * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
    });
}

}  // extern "C"
