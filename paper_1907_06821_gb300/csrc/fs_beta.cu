// Generated projectors: the tables behind beta_value (fs_beta.cuh) and the
// nonlocal term for contexts that store no projector table.
//
// The Gaussian s/p projectors of the H definition (fs.h) at q = k + G,
//     beta_s(q)   = Omega^-1/2 (pi w^2)^{-3/4} (2 pi w^2)^{3/2} e^{-w^2 q^2/2} e^{-i q.R_a},
//     beta_p,x(q) = beta_s(q) (sqrt(2)/w) (-i w^2 q_x)   (and y, z),
// split into a radial factor per type and plane wave and a phase that, in an
// orthorhombic cell, is a product of three one-axis factors per atom.  A long
// wire (7,920 projectors, 1.3 M plane waves) needs 83 MB of radial factors and
// a few MB of phases instead of a 165 GB FP64 table.
#include "fs_beta.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

// out[(p - p0) npw + g] = beta_p(q_g) for p in [p0, p0 + np), in the precision of T2
template <typename T2>
__global__ void beta_rows_kernel(BetaGen B, int p0, int np, T2* __restrict__ out) {
    const int p = p0 + blockIdx.y;
    if (blockIdx.y >= np) return;
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < B.npw; g += (long)gridDim.x * blockDim.x) {
        if constexpr (sizeof(T2) == 8)
            out[(long)blockIdx.y * B.npw + g] = beta_value32(B, p, g);
        else
            out[(long)blockIdx.y * B.npw + g] = beta_value(B, p, g);
    }
}

}  // namespace

BetaGen beta_gen_of(const fs_ctx* c) {
    BetaGen B;
    B.rad = c->bg_rad.as<double>();
    B.ph = c->bg_ph.as<double2>();
    B.rad32 = c->bg_rad32.as<float>();
    B.ph32 = c->bg_ph32.as<float2>();
    B.gidx = c->bg_gidx.as<int>();
    B.pl = c->bg_pl.as<int>();
    B.nproj = c->nproj;
    B.span = c->bg_span;
    B.npw = c->npw;
    return B;
}

void beta_gen_setup(fs_ctx* c, const fs_projectors* pr, double omega) {
    const long npw = c->npw;
    const double b[3] = {2.0 * M_PI / c->L[0], 2.0 * M_PI / c->L[1], 2.0 * M_PI / c->L[2]};
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    for (long g = 0; g < npw; ++g)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], c->miller[3 * g + d]);
            hi[d] = std::max(hi[d], c->miller[3 * g + d]);
        }
    int span = 1;
    for (int d = 0; d < 3; ++d) span = std::max(span, hi[d] - lo[d] + 1);
    if (span > 1024) throw fs_error(FS_ERR_ARG, "generated projectors: more than 1024 Miller indices on an axis");
    std::vector<double> rad((size_t)c->nproj * npw);
    std::vector<int> gidx(npw), pl(c->nproj);
    for (int p = 0; p < c->nproj; ++p) {
        const double w = pr->width[p];
        const double pref = std::pow(omega, -0.5) * std::pow(M_PI * w * w, -0.75) * std::pow(2.0 * M_PI * w * w, 1.5);
        pl[p] = pr->l[p];
        for (long g = 0; g < npw; ++g) {
            double q[3];
            for (int d = 0; d < 3; ++d) q[d] = c->k[d] + c->miller[3 * g + d] * b[d];
            const double q2 = (q[0] * q[0] + q[1] * q[1]) + q[2] * q[2];
            double r = pref * std::exp(-0.5 * w * w * q2);
            if (pr->l[p] == 1) r *= std::sqrt(2.0) * w * q[pr->axis[p]];
            rad[(size_t)p * npw + g] = r;
        }
    }
    for (long g = 0; g < npw; ++g)
        gidx[g] = (c->miller[3 * g] - lo[0]) | ((c->miller[3 * g + 1] - lo[1]) << 10) |
                  ((c->miller[3 * g + 2] - lo[2]) << 20);
    std::vector<double2> ph((size_t)c->natom * 3 * span);
    for (int a = 0; a < c->natom; ++a)
        for (int d = 0; d < 3; ++d)
            for (int j = 0; j < span; ++j) {
                const double qd = c->k[d] + (lo[d] + j) * b[d];
                const double ang = qd * pr->pos[3 * a + d];
                ph[((size_t)a * 3 + d) * span + j] = make_double2(std::cos(ang), -std::sin(ang));
            }
    c->bg_span = span;
    c->bg_rad.alloc(rad.size() * sizeof(double));
    c->bg_gidx.alloc(gidx.size() * sizeof(int));
    c->bg_pl.alloc(pl.size() * sizeof(int));
    c->bg_ph.alloc(ph.size() * sizeof(double2));
    FS_CUDA(cudaMemcpy(c->bg_rad.p, rad.data(), rad.size() * sizeof(double), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->bg_gidx.p, gidx.data(), gidx.size() * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->bg_pl.p, pl.data(), pl.size() * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->bg_ph.p, ph.data(), ph.size() * sizeof(double2), cudaMemcpyHostToDevice));
    std::vector<float> rad32(rad.begin(), rad.end());
    std::vector<float2> ph32(ph.size());
    for (size_t i = 0; i < ph.size(); ++i) ph32[i] = make_float2((float)ph[i].x, (float)ph[i].y);
    c->bg_rad32.alloc(rad32.size() * sizeof(float));
    c->bg_ph32.alloc(ph32.size() * sizeof(float2));
    FS_CUDA(cudaMemcpy(c->bg_rad32.p, rad32.data(), rad32.size() * sizeof(float), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->bg_ph32.p, ph32.data(), ph32.size() * sizeof(float2), cudaMemcpyHostToDevice));
}

// Nonlocal term with generated projectors on the CUDA-core GEMMs (FP64, or
// FP32 on the CUDA-core path): the table is formed in chunks of projector rows
// (at most 2 GiB) and each chunk contracted as the stored table would be.
// P[b * nptot + p] = <beta_p | psi_b>;  after the D step, hpsi += sum_p Q beta_p.
template <typename T2>
void beta_project_chunked(fs_ctx* c, const T2* psi, const int* rowmap, int nb, double2* P) {
    const long npw = c->npw;
    const int rows = (int)std::max<long>(1, std::min<long>(c->nptot, (2l << 30) / (npw * (long)sizeof(T2))));
    c->beta_chunk.ensure((size_t)rows * npw * sizeof(T2));
    const BetaGen B = beta_gen_of(c);
    for (int p0 = 0; p0 < c->nptot; p0 += rows) {
        const int np = std::min(rows, c->nptot - p0);
        dim3 g((unsigned)std::min<long>(64, (npw + 255) / 256), np);
        beta_rows_kernel<T2><<<g, 256, 0, c->stream>>>(B, p0, np, c->beta_chunk.as<T2>());
        FS_CUDA(cudaGetLastError());
        gemm_gram<T2>(c, np, nb, (int)npw, c->beta_chunk.as<T2>(), npw, nullptr, psi, npw, rowmap, P + p0, 1,
                      c->nptot, 1.0, 0.0, ks_prec<T2>(KS_NL_PROJ));
    }
}

template <typename T2> void beta_add_chunked(fs_ctx* c, const double2* Q, int nb, T2* hpsi) {
    const long npw = c->npw;
    const int rows = (int)std::max<long>(1, std::min<long>(c->nptot, (2l << 30) / (npw * (long)sizeof(T2))));
    c->beta_chunk.ensure((size_t)rows * npw * sizeof(T2));
    const BetaGen B = beta_gen_of(c);
    for (int p0 = 0; p0 < c->nptot; p0 += rows) {
        const int np = std::min(rows, c->nptot - p0);
        dim3 g((unsigned)std::min<long>(64, (npw + 255) / 256), np);
        beta_rows_kernel<T2><<<g, 256, 0, c->stream>>>(B, p0, np, c->beta_chunk.as<T2>());
        FS_CUDA(cudaGetLastError());
        gemm_nn<T2, double2>(c, nb, (int)npw, np, Q + p0, c->nptot, 1, c->beta_chunk.as<T2>(), npw, nullptr, hpsi,
                             npw, nullptr, 1.0, 1.0, hpsi, npw, ks_prec<T2>(KS_NL_ADD));
    }
}

template void beta_project_chunked<double2>(fs_ctx*, const double2*, const int*, int, double2*);
template void beta_project_chunked<float2>(fs_ctx*, const float2*, const int*, int, double2*);
template void beta_add_chunked<double2>(fs_ctx*, const double2*, int, double2*);
template void beta_add_chunked<float2>(fs_ctx*, const double2*, int, float2*);
