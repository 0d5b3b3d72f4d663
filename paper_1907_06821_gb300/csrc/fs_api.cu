// C ABI entry points: context set-up (plane-wave sphere, FFT column tables,
// local potential, projector table), H application and state I/O.
#include "fs_common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

namespace {

// beta[(a*nproj + c)][g] for the Gaussian s/p projectors (header fs.h gives the form)
__global__ void beta_kernel(double2* __restrict__ beta, const int* __restrict__ miller, long npw, double b0, double b1,
                            double b2, double k0, double k1, double k2, const double* __restrict__ pos, int natom,
                            const int* __restrict__ pl, const int* __restrict__ pax, const double* __restrict__ pw,
                            int nproj, double inv_sqrt_omega) {
    const long row = blockIdx.y;  // a * nproj + c
    const int a = (int)(row / nproj), c = (int)(row % nproj);
    const double w = pw[c];
    const double ns = pow(M_PI * w * w, -0.75);
    const double pref = inv_sqrt_omega * ns * pow(2.0 * M_PI * w * w, 1.5);
    const double Rx = pos[3 * a], Ry = pos[3 * a + 1], Rz = pos[3 * a + 2];
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < npw; g += (long)gridDim.x * blockDim.x) {
        double qx = k0 + miller[3 * g] * b0;
        double qy = k1 + miller[3 * g + 1] * b1;
        double qz = k2 + miller[3 * g + 2] * b2;
        double q2 = qx * qx + qy * qy + qz * qz;
        double radial = pref * exp(-0.5 * w * w * q2);
        double s, co;
        sincos(qx * Rx + qy * Ry + qz * Rz, &s, &co);  // e^{-i q.R} = (co, -s)
        double2 out;
        if (pl[c] == 0) {
            out = make_double2(radial * co, -radial * s);
        } else {
            double qa = pax[c] == 0 ? qx : (pax[c] == 1 ? qy : qz);
            double cc = radial * sqrt(2.0) * w * qa;  // beta = -i cc e^{-i q.R}
            out = make_double2(-cc * s, -cc * co);
        }
        beta[row * npw + g] = out;
    }
}

template <typename Fn> fs_status guarded(fs_ctx* c, Fn fn) {
    try {
        fn();
        if (c) c->err.clear();
        return FS_OK;
    } catch (const fs_error& e) {
        if (c) c->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (c) c->err = "host allocation failed";
        return FS_ERR_OOM;
    }
}

int posmod(long a, int n) { return (int)(((a % n) + n) % n); }

void build_sphere(fs_ctx* c) {
    const double b[3] = {2.0 * M_PI / c->L[0], 2.0 * M_PI / c->L[1], 2.0 * M_PI / c->L[2]};
    const double qmax = std::sqrt(2.0 * c->ecut);
    int h[3];
    for (int d = 0; d < 3; ++d) h[d] = (int)std::floor((qmax + std::fabs(c->k[d])) / b[d]) + 1;
    std::vector<int>& mil = c->miller;
    mil.clear();
    c->kin_h.clear();
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    for (int g0 = -h[0]; g0 <= h[0]; ++g0)
        for (int g1 = -h[1]; g1 <= h[1]; ++g1)
            for (int g2 = -h[2]; g2 <= h[2]; ++g2) {
                double q0 = c->k[0] + g0 * b[0];
                double q1 = c->k[1] + g1 * b[1];
                double q2 = c->k[2] + g2 * b[2];
                double kin = 0.5 * ((q0 * q0 + q1 * q1) + q2 * q2);
                if (kin <= c->ecut) {
                    mil.push_back(g0);
                    mil.push_back(g1);
                    mil.push_back(g2);
                    c->kin_h.push_back(kin);
                    const int gg[3] = {g0, g1, g2};
                    for (int d = 0; d < 3; ++d) {
                        lo[d] = std::min(lo[d], gg[d]);
                        hi[d] = std::max(hi[d], gg[d]);
                    }
                }
            }
    c->npw = (int)c->kin_h.size();
    if (c->npw == 0) throw fs_error(FS_ERR_ARG, "empty plane-wave sphere (ecut too small)");
    for (int d = 0; d < 3; ++d)
        if (hi[d] - lo[d] + 1 > c->n[d])
            throw fs_error(FS_ERR_GRID_TOO_SMALL, "axis " + std::to_string(d) + ": sphere spans " +
                                                      std::to_string(hi[d] - lo[d] + 1) + " > grid " +
                                                      std::to_string(c->n[d]));
    // z-columns
    std::vector<int> cstart, cxy, ecol(c->npw), ez(c->npw);
    for (int g = 0; g < c->npw; ++g) {
        int g0 = mil[3 * g], g1 = mil[3 * g + 1], g2 = mil[3 * g + 2];
        bool newcol = (g == 0) || g0 != mil[3 * (g - 1)] || g1 != mil[3 * (g - 1) + 1];
        if (newcol) {
            cstart.push_back(g);
            cxy.push_back(posmod(g0, c->n[0]) * c->n[1] + posmod(g1, c->n[1]));
        }
        ecol[g] = (int)cstart.size() - 1;
        ez[g] = posmod(g2, c->n[2]);
    }
    c->ncol = (int)cstart.size();
    cstart.push_back(c->npw);
    c->col_start.alloc(cstart.size() * sizeof(int));
    c->col_xy.alloc(cxy.size() * sizeof(int));
    c->ent_col.alloc(ecol.size() * sizeof(int));
    c->ent_z.alloc(ez.size() * sizeof(int));
    c->kin.alloc(c->kin_h.size() * sizeof(double));
    FS_CUDA(cudaMemcpy(c->col_start.p, cstart.data(), cstart.size() * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->col_xy.p, cxy.data(), cxy.size() * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->ent_col.p, ecol.data(), ecol.size() * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->ent_z.p, ez.data(), ez.size() * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->kin.p, c->kin_h.data(), c->kin_h.size() * sizeof(double), cudaMemcpyHostToDevice));
}

void upload_potential(fs_ctx* c, const double* vloc) {
    const int n0 = c->n[0], n1 = c->n[1], n2 = c->n[2];
    const size_t ng = (size_t)n0 * n1 * n2;
    std::vector<double> vz(ng);
    std::vector<float> vzf(ng);
    // plane-major [z][x][y]; on the register-FFT path each axis is stored in
    // the permuted order its inverse transform leaves ([p_z][p_x][p_y])
    std::vector<int> ix[3];
    for (int d = 0; d < 3; ++d) {
        ix[d].resize(c->n[d]);
        for (int p = 0; p < c->n[d]; ++p) ix[d][p] = c->fast ? fft_perm_index(c, d, p) : p;
    }
    for (int pz = 0; pz < n2; ++pz)
        for (int px = 0; px < n0; ++px)
            for (int py = 0; py < n1; ++py) {
                double v = vloc[((size_t)ix[0][px] * n1 + ix[1][py]) * n2 + ix[2][pz]];
                if (!std::isfinite(v)) throw fs_error(FS_ERR_ARG, "vloc holds NaN/Inf");
                size_t o = (size_t)pz * n0 * n1 + (size_t)px * n1 + py;
                vz[o] = v;
                vzf[o] = (float)v;
            }
    c->vz64.alloc(ng * sizeof(double));
    c->vz32.alloc(ng * sizeof(float));
    FS_CUDA(cudaMemcpy(c->vz64.p, vz.data(), ng * sizeof(double), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->vz32.p, vzf.data(), ng * sizeof(float), cudaMemcpyHostToDevice));
}

void build_projectors(fs_ctx* c, const fs_projectors* pr) {
    c->natom = pr ? pr->natom : 0;
    c->nproj = pr ? pr->nproj : 0;
    if (c->natom < 0 || c->nproj < 0) throw fs_error(FS_ERR_ARG, "negative projector counts");
    c->nptot = c->natom * c->nproj;
    if (c->nptot == 0) return;
    if (!pr->pos || !pr->l || !pr->axis || !pr->width || !pr->D) throw fs_error(FS_ERR_ARG, "null projector array");
    for (int i = 0; i < c->nproj; ++i) {
        if (pr->l[i] < 0 || pr->l[i] > 1) throw fs_error(FS_ERR_ARG, "projector l must be 0 or 1");
        if (pr->l[i] == 1 && (pr->axis[i] < 0 || pr->axis[i] > 2)) throw fs_error(FS_ERR_ARG, "p axis must be 0..2");
        if (!(pr->width[i] > 0)) throw fs_error(FS_ERR_ARG, "projector width must be > 0");
    }
    dbuf dmil, dpos, dl, dax, dw;
    dmil.alloc(c->miller.size() * sizeof(int));
    dpos.alloc((size_t)c->natom * 3 * sizeof(double));
    dl.alloc(c->nproj * sizeof(int));
    dax.alloc(c->nproj * sizeof(int));
    dw.alloc(c->nproj * sizeof(double));
    FS_CUDA(cudaMemcpy(dmil.p, c->miller.data(), c->miller.size() * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(dpos.p, pr->pos, (size_t)c->natom * 3 * sizeof(double), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(dl.p, pr->l, c->nproj * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(dax.p, pr->axis, c->nproj * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(dw.p, pr->width, c->nproj * sizeof(double), cudaMemcpyHostToDevice));
    const double omega = c->L[0] * c->L[1] * c->L[2];
    const double table_bytes = (double)c->nptot * c->npw * sizeof(double2);
    c->beta_gen = c->opt.projectors == FS_PROJ_GENERATED ||
                  (c->opt.projectors == FS_PROJ_AUTO && table_bytes > 16e9);
    if (c->beta_gen) {
        beta_gen_setup(c, pr, omega);
        const size_t nd = (size_t)c->natom * c->nproj * c->nproj;
        c->Dmat.alloc(nd * sizeof(double));
        FS_CUDA(cudaMemcpy(c->Dmat.p, pr->D, nd * sizeof(double), cudaMemcpyHostToDevice));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        return;
    }
    c->beta64.alloc((size_t)c->nptot * c->npw * sizeof(double2));
    dim3 g((unsigned)std::min<long>(256, (c->npw + 255) / 256), c->nptot);
    beta_kernel<<<g, 256, 0, c->stream>>>(c->beta64.as<double2>(), dmil.as<int>(), c->npw, 2.0 * M_PI / c->L[0],
                                          2.0 * M_PI / c->L[1], 2.0 * M_PI / c->L[2], c->k[0], c->k[1], c->k[2],
                                          dpos.as<double>(), c->natom, dl.as<int>(), dax.as<int>(), dw.as<double>(),
                                          c->nproj, 1.0 / std::sqrt(omega));
    FS_CUDA(cudaGetLastError());
    const size_t nd = (size_t)c->natom * c->nproj * c->nproj;
    c->Dmat.alloc(nd * sizeof(double));
    FS_CUDA(cudaMemcpy(c->Dmat.p, pr->D, nd * sizeof(double), cudaMemcpyHostToDevice));
    FS_CUDA(cudaStreamSynchronize(c->stream));
}

void ensure_fp32_tables(fs_ctx* c) {
    if (c->nptot > 0 && !c->beta_gen && !c->beta32.p) {
        size_t cnt = (size_t)c->nptot * c->npw;
        c->beta32.alloc(cnt * sizeof(float2));
        vec_convert<double2, float2>(c, c->beta64.as<double2>(), c->beta32.as<float2>(), cnt);
    }
}

}  // namespace

void ctx_ensure_fp32(fs_ctx* c) { ensure_fp32_tables(c); }

int* ctx_errflag(fs_ctx* c) { return c->errflag.as<int>(); }

// raise FS_ERR_TIMEOUT if a device-side bounded wait gave up (clears the flag)
void ctx_check_errflag(fs_ctx* c) {
    int v = 0;
    FS_CUDA(cudaMemcpyAsync(&v, c->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    if (v) {
        FS_CUDA(cudaMemsetAsync(c->errflag.p, 0, sizeof(int), c->stream));
        throw fs_error(FS_ERR_TIMEOUT, "a tensor-core pipeline wait exceeded its limit");
    }
}

extern "C" {

fs_status fs_create(const fs_grid* grid, double ecut, const double k[3], const double* vloc,
                    const fs_projectors* proj, const fs_options* opts, fs_ctx** out) {
    if (!out) return FS_ERR_ARG;
    *out = nullptr;
    if (!grid || !k || !vloc) return FS_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(grid->L[d] > 0) || grid->n[d] < 2 || grid->n[d] > 4096) return FS_ERR_ARG;
    if (!(ecut > 0) || !std::isfinite(ecut)) return FS_ERR_ARG;
    fs_ctx* c = new (std::nothrow) fs_ctx();
    if (!c) return FS_ERR_OOM;
    fs_status st = guarded(c, [&] {
        std::memcpy(c->L, grid->L, sizeof(c->L));
        std::memcpy(c->n, grid->n, sizeof(c->n));
        std::memcpy(c->k, k, sizeof(c->k));
        c->ecut = ecut;
        std::memset(&c->opt, 0, sizeof(c->opt));
        c->opt.guard = -1;
        if (opts) c->opt = *opts;
        if (!(c->opt.dE > 0)) c->opt.dE = 0.5;
        if (c->opt.maxit <= 0) c->opt.maxit = 5000;
        if (c->opt.precision != FS_FP64 && c->opt.precision != FS_MIXED) throw fs_error(FS_ERR_ARG, "bad precision");
        if (c->opt.precond < FS_PREC_M || c->opt.precond > FS_PREC_LEARNED) throw fs_error(FS_ERR_ARG, "bad precond");
        if (c->opt.projectors < FS_PROJ_AUTO || c->opt.projectors > FS_PROJ_GENERATED)
            throw fs_error(FS_ERR_ARG, "bad projectors mode");
        if (c->opt.gemm_path != FS_GEMM_TENSOR && c->opt.gemm_path != FS_GEMM_CUDA_CORES)
            throw fs_error(FS_ERR_ARG, "bad gemm_path");
        c->gemm_path = c->opt.gemm_path;
        FS_CUDA(cudaGetDevice(&c->device));
        c->errflag.alloc(sizeof(int));
        FS_CUDA(cudaMemset(c->errflag.p, 0, sizeof(int)));
        if (c->opt.cuda_stream) {
            c->stream = (cudaStream_t)c->opt.cuda_stream;
        } else {
            FS_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
            c->own_stream = true;
        }
        build_sphere(c);
        ctx_prepare_fft(c);
        upload_potential(c, vloc);
        build_projectors(c, proj);
        if (c->opt.precision == FS_MIXED) ensure_fp32_tables(c);
        FS_CUDA(cudaStreamSynchronize(c->stream));
    });
    if (st != FS_OK) {
        fs_destroy(c);
        return st;
    }
    *out = c;
    return FS_OK;
}

fs_status fs_npw(const fs_ctx* c, int* npw) {
    if (!c || !npw) return FS_ERR_ARG;
    *npw = c->npw;
    return FS_OK;
}

fs_status fs_gvectors(const fs_ctx* c, int* miller) {
    if (!c || !miller) return FS_ERR_ARG;
    std::memcpy(miller, c->miller.data(), c->miller.size() * sizeof(int));
    return FS_OK;
}

fs_status fs_apply_H(fs_ctx* c, const void* psi, void* hpsi, int nband, double shift, int precision) {
    if (!c) return FS_ERR_ARG;
    if (nband < 0 || (nband > 0 && (!psi || !hpsi || psi == hpsi)) || !std::isfinite(shift)) {
        c->err = "fs_apply_H: bad arguments";
        return FS_ERR_ARG;
    }
    if (precision != FS_FP64 && precision != FS_MIXED) {
        c->err = "fs_apply_H: bad precision";
        return FS_ERR_ARG;
    }
    return guarded(c, [&] {
        if (nband == 0) return;
        if (precision == FS_FP64) {
            apply_H_impl<double2>(c, (const double2*)psi, (double2*)hpsi, nband, shift);
        } else {
            ensure_fp32_tables(c);
            apply_H_impl<float2>(c, (const float2*)psi, (float2*)hpsi, nband, shift);
        }
        FS_CUDA(cudaStreamSynchronize(c->stream));
        ctx_check_errflag(c);
    });
}

fs_status fs_set_initial_states(fs_ctx* c, const void* psi, int n, int damp, int where) {
    if (!c) return FS_ERR_ARG;
    if (n < 0 || (n > 0 && !psi) || (where != FS_HOST && where != FS_DEVICE)) {
        c->err = "fs_set_initial_states: bad arguments";
        return FS_ERR_ARG;
    }
    return guarded(c, [&] {
        c->ninit = n;
        c->init_damp = damp ? 1 : 0;
        if (n == 0) return;
        size_t bytes = (size_t)n * c->npw * sizeof(double2);
        c->init_states.ensure(bytes);
        FS_CUDA(cudaMemcpyAsync(c->init_states.p, psi, bytes,
                                where == FS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
    });
}

fs_status fs_solve(fs_ctx* c, double e_ref, int nstates, double tol, fs_result* res) {
    if (!c) return FS_ERR_ARG;
    if (!res || !res->eps || !res->resid || nstates <= 0 || !(tol > 0) || !std::isfinite(e_ref)) {
        c->err = "fs_solve: bad arguments";
        return FS_ERR_ARG;
    }
    fs_status st = FS_OK;
    fs_status g = guarded(c, [&] { st = solve_impl(c, e_ref, nstates, tol, res); });
    return g != FS_OK ? g : st;
}

fs_status fs_solve_lowest(fs_ctx* c, int nstates, double tol, fs_result* res) {
    if (!c) return FS_ERR_ARG;
    if (!res || !res->eps || !res->resid || nstates <= 0 || !(tol > 0)) {
        c->err = "fs_solve_lowest: bad arguments";
        return FS_ERR_ARG;
    }
    fs_status st = FS_OK;
    fs_status g = guarded(c, [&] { st = solve_impl(c, 0.0, nstates, tol, res, true); });
    return g != FS_OK ? g : st;
}

fs_status fs_get_states(fs_ctx* c, void* psi, int n, int where) {
    if (!c) return FS_ERR_ARG;
    if (n < 0 || n > c->nresult || (n > 0 && !psi) || (where != FS_HOST && where != FS_DEVICE)) {
        c->err = "fs_get_states: bad arguments (n exceeds the states of the last solve?)";
        return FS_ERR_ARG;
    }
    return guarded(c, [&] {
        if (n == 0) return;
        size_t bytes = (size_t)n * c->npw * sizeof(double2);
        FS_CUDA(cudaMemcpyAsync(psi, c->result_states.p, bytes,
                                where == FS_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));
    });
}

void fs_destroy(fs_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    prof_release(c);
    cudaStream_t s = c->stream;
    bool own = c->own_stream;
    delete c;
    if (own && s) cudaStreamDestroy(s);
}

const char* fs_last_error(const fs_ctx* c) {
    if (!c) return "no context";
    return c->err.c_str();
}

}  // extern "C"
