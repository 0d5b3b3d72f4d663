// Application of the plane-wave Hamiltonian: hpsi = (H - shift) psi.
//
// Local part (kinetic + V_loc), two-pass 3-D FFT decomposition:
//   1. col_inverse : unpack each sphere z-column into a zero-filled line of
//                    n2, inverse FFT along z, write to the column buffer
//                    [band][z][column] (only the ncol columns that hold
//                    plane waves exist; the rest of the grid is zero).
//   2. plane       : per (band, z) plane: scatter the columns into an n0 x n1
//                    plane in shared memory, inverse 2-D FFT, multiply by
//                    V(r), forward 2-D FFT, gather the columns back.
//   3. col_forward : forward FFT along z, scale by 1/N, pick the sphere
//                    entries and add (|q|^2/2 - shift) psi.
// Nonlocal part: P = B^H psi (Gram GEMM), Q = D P per atom, hpsi += B Q.
#include "fs_beta.cuh"
#include "fs_common.cuh"
#include "fs_fft.cuh"

#include <algorithm>
#include <cmath>

// q = a / d (integer quotient) for 0 <= a < 2^22, d >= 1, without an integer
// division: (a + 1/2) / d = q + (r + 1/2) / d lies at least 1/(2d) from the
// nearest integer, and the float product (a + 1/2) fl(1/d) differs from it by
// less than (a + 1/2) 2^-23 / d < 1/(2d), so truncation gives q exactly.
__device__ __forceinline__ int qdiv(int a, float inv_d) { return (int)(((float)a + 0.5f) * inv_d); }

// One Stockham stage over `nl` lines of length n held in shared memory.
// All reads of the stage are staged in registers before any write, so the
// stage runs in place.  KM butterflies per thread must cover nl * n / R.
template <typename T2, int R, int KM>
__device__ __forceinline__ void fft_stage(T2* buf, int n, int nl, int lstride, int estride, int Ns,
                                          const T2* __restrict__ tw, int sign) {
    const int nb = n / R;
    const int total = nb * nl;
    const float inb = 1.0f / (float)nb, ins = 1.0f / (float)Ns;
    const int wstep = n / (Ns * R);
    T2 v[KM][R];
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) {
        int t = threadIdx.x + kk * blockDim.x;
        if (t < total) {
            int line = qdiv(t, inb), j = t - line * nb;
            const T2* base = buf + (long)line * lstride;
            int tj = j - qdiv(j, ins) * Ns;
            int step = wstep * tj;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                T2 x = base[(j + r * nb) * estride];
                if (r > 0 && step > 0) {
                    T2 w = __ldg(&tw[r * step]);
                    if (sign > 0) w.y = -w.y;
                    x = cmul(x, w);
                }
                v[kk][r] = x;
            }
            Bfly<T2, R>::run(v[kk], sign);
        }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) {
        int t = threadIdx.x + kk * blockDim.x;
        if (t < total) {
            const int line = qdiv(t, inb), j = t - line * nb;
            T2* base = buf + (long)line * lstride;
            const int jq = qdiv(j, ins), tj = j - jq * Ns;
            int idxD = jq * Ns * R + tj;
#pragma unroll
            for (int r = 0; r < R; ++r) base[(idxD + r * Ns) * estride] = v[kk][r];
        }
    }
    __syncthreads();
}

// Transform nlines lines (groups of plan.group lines at a time); EPT = element budget per thread.
template <typename T2, int EPT>
__device__ void fft_lines(T2* buf, const FftPlan<T2>& p, int nlines, int lstride, int estride, int sign) {
    for (int l0 = 0; l0 < nlines; l0 += p.group) {
        int nl = min(p.group, nlines - l0);
        T2* b = buf + (long)l0 * lstride;
        int Ns = 1;
        for (int s = 0; s < p.nst; ++s) {
            int R = p.rad[s];
            if (R == 4)
                fft_stage<T2, 4, (EPT + 3) / 4>(b, p.n, nl, lstride, estride, Ns, p.tw, sign);
            else if (R == 2)
                fft_stage<T2, 2, (EPT + 1) / 2>(b, p.n, nl, lstride, estride, Ns, p.tw, sign);
            else if (R == 3)
                fft_stage<T2, 3, (EPT + 2) / 3>(b, p.n, nl, lstride, estride, Ns, p.tw, sign);
            else
                fft_stage<T2, 5, (EPT + 4) / 5>(b, p.n, nl, lstride, estride, Ns, p.tw, sign);
            Ns *= R;
        }
    }
}

constexpr int COL_THREADS = 256;
constexpr int COL_EPT = 8;
constexpr int PLANE_THREADS = 512;
constexpr int PLANE_EPT = 8;

// ------------------------------------------------------------------ kernels
template <typename T2>
__global__ void __launch_bounds__(COL_THREADS)
col_inverse_kernel(const T2* __restrict__ psi, const int* __restrict__ rowmap, long ldpsi, T2* __restrict__ colbuf,
                   const int* __restrict__ col_start, const int* __restrict__ ent_col, const int* __restrict__ ent_z,
                   int ncol, int cpb, FftPlan<T2> pz) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* lines = reinterpret_cast<T2*>(smem_raw);
    const int n2 = pz.n;
    const int band = blockIdx.y;
    const int c0 = blockIdx.x * cpb;
    const int nc = min(cpb, ncol - c0);
    const long src = rowmap ? rowmap[band] : band;
    for (int i = threadIdx.x; i < nc * n2; i += blockDim.x) lines[i] = mk((typename real_of<T2>::t)0, (typename real_of<T2>::t)0);
    __syncthreads();
    const int g0 = col_start[c0], g1 = col_start[c0 + nc];
    const T2* p = psi + src * ldpsi;
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) lines[(ent_col[g] - c0) * n2 + ent_z[g]] = p[g];
    __syncthreads();
    fft_lines<T2, COL_EPT>(lines, pz, nc, n2, 1, +1);
    T2* out = colbuf + (long)band * n2 * ncol;
    for (int i = threadIdx.x; i < nc * n2; i += blockDim.x) {
        int z = i / nc, cc = i - z * nc;
        out[(long)z * ncol + c0 + cc] = lines[cc * n2 + z];
    }
}

template <typename T2, typename R>
__global__ void __launch_bounds__(PLANE_THREADS)
plane_kernel(T2* __restrict__ colbuf, const int* __restrict__ col_xy, int ncol, const R* __restrict__ vz,
             FftPlan<T2> px, FftPlan<T2> py) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* plane = reinterpret_cast<T2*>(smem_raw);
    const int n0 = px.n, n1 = py.n, n2 = gridDim.x;
    const int z = blockIdx.x, band = blockIdx.y;
    const int np = n0 * n1;
    for (int i = threadIdx.x; i < np; i += blockDim.x) plane[i] = mk((R)0, (R)0);
    __syncthreads();
    T2* cb = colbuf + ((long)band * n2 + z) * ncol;
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) plane[col_xy[c]] = cb[c];
    __syncthreads();
    fft_lines<T2, PLANE_EPT>(plane, py, n0, n1, 1, +1);   // along y (contiguous rows)
    fft_lines<T2, PLANE_EPT>(plane, px, n1, 1, n1, +1);   // along x
    const R* v = vz + (long)z * np;
    for (int i = threadIdx.x; i < np; i += blockDim.x) plane[i] = cscale(plane[i], v[i]);
    __syncthreads();
    fft_lines<T2, PLANE_EPT>(plane, px, n1, 1, n1, -1);
    fft_lines<T2, PLANE_EPT>(plane, py, n0, n1, 1, -1);
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) cb[c] = plane[col_xy[c]];
}

template <typename T2>
__global__ void __launch_bounds__(COL_THREADS)
col_forward_kernel(const T2* __restrict__ colbuf, const T2* __restrict__ psi, const int* __restrict__ rowmap,
                   long ldpsi, T2* __restrict__ hpsi, const int* __restrict__ col_start,
                   const int* __restrict__ ent_col, const int* __restrict__ ent_z, const double* __restrict__ kin,
                   int ncol, int cpb, FftPlan<T2> pz, double inv_ng, double shift, long npw) {
    using R = typename real_of<T2>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* lines = reinterpret_cast<T2*>(smem_raw);
    const int n2 = pz.n;
    const int band = blockIdx.y;
    const int c0 = blockIdx.x * cpb;
    const int nc = min(cpb, ncol - c0);
    const T2* in = colbuf + (long)band * n2 * ncol;
    for (int i = threadIdx.x; i < nc * n2; i += blockDim.x) {
        int z = i / nc, cc = i - z * nc;
        lines[cc * n2 + z] = in[(long)z * ncol + c0 + cc];
    }
    __syncthreads();
    fft_lines<T2, COL_EPT>(lines, pz, nc, n2, 1, -1);
    const int g0 = col_start[c0], g1 = col_start[c0 + nc];
    const long src = rowmap ? rowmap[band] : band;
    const T2* p = psi + src * ldpsi;
    T2* o = hpsi + (long)band * npw;
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        T2 a = lines[(ent_col[g] - c0) * n2 + ent_z[g]];
        T2 x = p[g];
        R f = (R)(kin[g] - shift);
        o[g] = mk((R)(a.x * (R)inv_ng) + f * x.x, (R)(a.y * (R)inv_ng) + f * x.y);
    }
}

// Q[b][a*np + i] = sum_j D[a][i][j] P[b][a*np + j]
template <typename T2>
__global__ void apply_D_kernel(const T2* __restrict__ P, T2* __restrict__ Q, const double* __restrict__ D, int natom,
                               int nproj, int nb) {
    using R = typename real_of<T2>::t;
    long total = (long)nb * natom * nproj;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        int i = (int)(t % nproj);
        long ba = t / nproj;
        int a = (int)(ba % natom);
        const T2* pr = P + ba * nproj;
        const double* d = D + ((long)a * nproj + i) * nproj;
        double sx = 0, sy = 0;
        for (int j = 0; j < nproj; ++j) {
            sx += d[j] * (double)pr[j].x;
            sy += d[j] * (double)pr[j].y;
        }
        Q[t] = mk((R)sx, (R)sy);
    }
}

// ------------------------------------------------------------------ register-FFT kernels
// The same three passes with every line transformed by the two-pass register
// scheme of fs_fft.cuh.  The z axis of the column buffer, and the x and y axes
// inside a plane, are carried in the permuted layout the inverse transforms
// leave; V(r) is stored permuted the same way (context set-up), so the
// multiply needs no reordering.
constexpr int ZF_THREADS = 256;
constexpr int PF_MAX_THREADS = 768;

// unpack the sphere z-columns of a tile, inverse z-FFT, write [band][p_z][column]
template <typename T2, bool BIG>
__global__ void __launch_bounds__(ZF_THREADS)
zinv_kernel(const T2* __restrict__ psi, const int* __restrict__ rowmap, long ldpsi, T2* __restrict__ colbuf,
            const int* __restrict__ col_start, const int* __restrict__ ent_cz, int ncol, int cpb, LineGeo gz, int Pz,
            const T2* __restrict__ twz) {
    using R = typename real_of<T2>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* tw = reinterpret_cast<T2*>(smem_raw);
    T2* lines = tw + gz.L;
    const int band = blockIdx.y, c0 = blockIdx.x * cpb, nc = min(cpb, ncol - c0);
    const long src = rowmap ? rowmap[band] : band;
    for (int i = threadIdx.x; i < gz.L; i += blockDim.x) tw[i] = twz[i];
    for (int i = threadIdx.x; i < nc * Pz; i += blockDim.x) lines[i] = mk((R)0, (R)0);
    __syncthreads();
    const int g0 = col_start[c0], g1 = col_start[c0 + nc];
    const T2* p = psi + src * ldpsi;
    // four loads in flight per thread before the shared-memory stores
    for (int g = g0 + threadIdx.x; g < g1; g += 4 * blockDim.x) {
        T2 v[4];
        int e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int gg = g + u * blockDim.x;
            if (gg < g1) {
                v[u] = p[gg];
                e[u] = ent_cz[gg];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (g + u * (int)blockDim.x < g1) lines[((e[u] >> 16) - c0) * Pz + (e[u] & 0xFFFF)] = v[u];
    }
    __syncthreads();
    // lanes of a warp: the same role in consecutive lines
    for (int i = threadIdx.x; i < nc * gz.B; i += blockDim.x) {
        const int r = i / nc;
        stride_pass<+1, true, BIG>(lines + (i - r * nc) * Pz, gz, r, tw);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nc * gz.A; i += blockDim.x) {
        const int k = i / nc;
        block_pass<+1, false, BIG>(lines + (i - k * nc) * Pz, gz, k, tw);
    }
    __syncthreads();
    T2* out = colbuf + (long)band * gz.L * ncol + c0;
    for (int i = threadIdx.x; i < nc * gz.L; i += blockDim.x) {
        const int pz = i / nc, cc = i - pz * nc;
        out[(long)pz * ncol + cc] = lines[cc * Pz + line_slot(gz, pz)];
    }
}

// inverse x pass 2, x V(r), forward x pass 1 on the block k1 of one x line
template <int B, typename T2, typename R>
__device__ __forceinline__ void fused_v_block(T2* line, const LineGeo& g, int k1, const T2* tw,
                                              const R* __restrict__ v, int vstride) {
    T2 a[B];
    const int base = g.Bp * k1;
#pragma unroll
    for (int j = 0; j < B; ++j) a[j] = line[(base + j) * g.es];
    RDft<B>::template run<+1>(a, tw, g.A);
#pragma unroll
    for (int j = 0; j < B; ++j) a[j] = cscale(a[j], __ldg(v + (long)(g.B * k1 + j) * vstride));
    RDft<B>::template run<-1>(a, tw, g.A);
#pragma unroll
    for (int m = 1; m < B; ++m)
        if (k1) a[m] = cmul(a[m], twid<-1>(tw, k1 * m));
#pragma unroll
    for (int j = 0; j < B; ++j) line[(base + j) * g.es] = a[j];
}

template <typename T2, typename R>
__device__ __forceinline__ void fused_v(T2* line, const LineGeo& g, int k1, const T2* tw, const R* v, int vstride) {
    switch (g.B) {
#define FS_CASE(n) \
    case n: fused_v_block<n>(line, g, k1, tw, v, vstride); break;
        FS_FFT_SIZES_S(FS_CASE)
#undef FS_CASE
        default: break;
    }
}

// One (band, z position) plane: scatter the columns, inverse y on the rows that
// hold columns, inverse x, x V(r), forward x, forward y on those rows, gather.
template <typename T2, typename R>
__global__ void __launch_bounds__(sizeof(T2) == 16 ? PF_MAX_THREADS / 2 : PF_MAX_THREADS)
plane_fast_kernel(T2* __restrict__ colbuf, const int* __restrict__ col_slot, int ncol,
                  const int* __restrict__ xrows, int nxr, const R* __restrict__ vperm, LineGeo gx, LineGeo gy, int P,
                  const T2* __restrict__ twx_g, const T2* __restrict__ twy_g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n0 = gx.L, n1 = gy.L, nz = gridDim.x;
    T2* twx = reinterpret_cast<T2*>(smem_raw);
    T2* twy = twx + n0;
    T2* plane = twy + n1;
    const int pz = blockIdx.x, band = blockIdx.y;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) twx[i] = twx_g[i];
    for (int i = threadIdx.x; i < n1; i += blockDim.x) twy[i] = twy_g[i];
    for (int i = threadIdx.x; i < n0 * P; i += blockDim.x) plane[i] = mk((R)0, (R)0);
    __syncthreads();
    T2* cb = colbuf + ((long)band * nz + pz) * ncol;
    for (int c = threadIdx.x; c < ncol; c += 4 * blockDim.x) {
        T2 v[4];
        int e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int cc = c + u * blockDim.x;
            if (cc < ncol) {
                v[u] = cb[cc];
                e[u] = col_slot[cc];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (c + u * (int)blockDim.x < ncol) plane[e[u]] = v[u];
    }
    __syncthreads();
    // y passes: lanes of a warp take the same role in consecutive rows
    for (int i = threadIdx.x; i < nxr * gy.B; i += blockDim.x) {
        const int r = i / nxr;
        stride_pass<+1, true, false>(plane + xrows[i - r * nxr] * P, gy, r, twy);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nxr * gy.A; i += blockDim.x) {
        const int k = i / nxr;
        block_pass<+1, false, false>(plane + xrows[i - k * nxr] * P, gy, k, twy);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n1 * gx.B; i += blockDim.x) {
        const int r = i / n1, q = i - r * n1;
        stride_pass<+1, true, false>(plane + line_slot(gy, q), gx, r, twx);
    }
    __syncthreads();
    const R* vz = vperm + (long)pz * n0 * n1;
    for (int i = threadIdx.x; i < n1 * gx.A; i += blockDim.x) {
        const int k = i / n1, q = i - k * n1;
        fused_v(plane + line_slot(gy, q), gx, k, twx, vz + q, n1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n1 * gx.B; i += blockDim.x) {
        const int r = i / n1, q = i - r * n1;
        stride_pass<-1, false, false>(plane + line_slot(gy, q), gx, r, twx);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nxr * gy.A; i += blockDim.x) {
        const int k = i / nxr;
        block_pass<-1, true, false>(plane + xrows[i - k * nxr] * P, gy, k, twy);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nxr * gy.B; i += blockDim.x) {
        const int r = i / nxr;
        stride_pass<-1, false, false>(plane + xrows[i - r * nxr] * P, gy, r, twy);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) cb[c] = plane[col_slot[c]];
}

// forward z-FFT of a tile of columns, x 1/N, pick the sphere entries, + (|q|^2/2 - shift) psi
template <typename T2, bool BIG>
__global__ void __launch_bounds__(ZF_THREADS)
zfwd_kernel(const T2* __restrict__ colbuf, const T2* __restrict__ psi, const int* __restrict__ rowmap, long ldpsi,
            T2* __restrict__ hpsi, const int* __restrict__ col_start, const int* __restrict__ ent_cz,
            const double* __restrict__ kin, int ncol, int cpb, LineGeo gz, int Pz, const T2* __restrict__ twz,
            double inv_ng, double shift, long npw) {
    using R = typename real_of<T2>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* tw = reinterpret_cast<T2*>(smem_raw);
    T2* lines = tw + gz.L;
    const int band = blockIdx.y, c0 = blockIdx.x * cpb, nc = min(cpb, ncol - c0);
    for (int i = threadIdx.x; i < gz.L; i += blockDim.x) tw[i] = twz[i];
    const T2* in = colbuf + (long)band * gz.L * ncol + c0;
    const int tot = nc * gz.L;
    for (int i = threadIdx.x; i < tot; i += 4 * blockDim.x) {
        T2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int ii = i + u * blockDim.x;
            if (ii < tot) {
                const int pz = ii / nc, cc = ii - pz * nc;
                v[u] = in[(long)pz * ncol + cc];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int ii = i + u * blockDim.x;
            if (ii < tot) {
                const int pz = ii / nc, cc = ii - pz * nc;
                lines[cc * Pz + line_slot(gz, pz)] = v[u];
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nc * gz.A; i += blockDim.x) {
        const int k = i / nc;
        block_pass<-1, true, BIG>(lines + (i - k * nc) * Pz, gz, k, tw);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nc * gz.B; i += blockDim.x) {
        const int r = i / nc;
        stride_pass<-1, false, BIG>(lines + (i - r * nc) * Pz, gz, r, tw);
    }
    __syncthreads();
    const int g0 = col_start[c0], g1 = col_start[c0 + nc];
    const long src = rowmap ? rowmap[band] : band;
    const T2* p = psi + src * ldpsi;
    T2* o = hpsi + (long)band * npw;
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        const int e = ent_cz[g];
        T2 a = lines[((e >> 16) - c0) * Pz + (e & 0xFFFF)];
        T2 x = p[g];
        R f = (R)(kin[g] - shift);
        o[g] = mk((R)(a.x * (R)inv_ng) + f * x.x, (R)(a.y * (R)inv_ng) + f * x.y);
    }
}

// ------------------------------------------------------------------ host side
static int col_smem(int cpb, int n2, size_t esz) { return (int)(cpb * n2 * esz); }

template <typename T2> static const FftPlan<T2>& plan_of(fs_ctx* c, int d);
template <> const FftPlan<double2>& plan_of<double2>(fs_ctx* c, int d) { return c->plan64[d]; }
template <> const FftPlan<float2>& plan_of<float2>(fs_ctx* c, int d) { return c->plan32[d]; }

static std::vector<int> factor_radices(int n) {
    std::vector<int> r;
    while (n % 4 == 0) { r.push_back(4); n /= 4; }
    while (n % 2 == 0) { r.push_back(2); n /= 2; }
    while (n % 3 == 0) { r.push_back(3); n /= 3; }
    while (n % 5 == 0) { r.push_back(5); n /= 5; }
    if (n != 1) return {};
    return r;
}

// lines of length n that one block of `threads` threads with element budget ept can hold
static int group_lines(int n, const std::vector<int>& rads, int threads, int ept) {
    int cap = 1 << 30;
    for (int R : rads) {
        int km = (ept + R - 1) / R;
        cap = std::min(cap, threads * km * R);
    }
    return cap / n;
}

// The dynamic shared-memory ceiling is a per-kernel attribute shared by every
// context in the process; it is set once to the device maximum (227 KB) so that
// contexts with different grids can coexist (each launch asks for what it needs).
template <typename T2> static void set_attr_smem(const void* fn, int bytes) {
    (void)bytes;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

// A = B * ... : the split L = A * B (A >= B, both register DFT sizes) with the smallest A.
static bool pick_split(int L, int& A, int& B) {
    A = 0;
    for (int b = 1; b * b <= L; ++b) {
        if (L % b) continue;
        const int a = L / b;
        if (fft_size_ok(a) && fft_size_ok(b) && (A == 0 || a < A)) {
            A = a;
            B = b;
        }
    }
    return A > 0;
}

static inline int posmod_(int a, int n) { return ((a % n) + n) % n; }

// Plan of the register-FFT path (fs_fft.cuh) when every axis splits into
// register DFT sizes and the padded plane fits in shared memory in FP64.
static void prepare_fast_fft(fs_ctx* c) {
    c->fast = false;
    LineGeo g[3];
    for (int d = 0; d < 3; ++d) {
        int A = 0, B = 0;
        if (!pick_split(c->n[d], A, B)) return;
        if (d < 2 && !(fft_size_small(A) && fft_size_small(B))) return;  // plane axes: small register DFTs
        g[d] = LineGeo{c->n[d], A, B, B, 1};
    }
    const int n0 = c->n[0], n1 = c->n[1], n2 = c->n[2];
    // odd pitches: the lanes of a warp take the same position in consecutive
    // lines (rows of a plane, columns of a tile), so an odd line pitch spreads
    // them over all banks
    const int P = n1 | 1, Pz = n2 | 1;
    const size_t plane_bytes = ((size_t)n0 * P + n0 + n1) * sizeof(double2);
    if (plane_bytes > 227 * 1024) return;
    int cpb = 32;
    while (cpb > 1 && ((size_t)cpb * Pz + n2) * sizeof(double2) > 100 * 1024) cpb /= 2;
    g[0].es = P;
    // columns in sphere order (a new column starts where (g0, g1) changes)
    if (c->ncol >= (1 << 16) || Pz >= (1 << 16)) return;  // packed (column, z slot) entries
    std::vector<int> cslot, ecz(c->npw), rows;
    std::vector<char> has_row(n0, 0);
    const std::vector<int>& mil = c->miller;
    for (int i = 0; i < c->npw; ++i) {
        const int g0 = mil[3 * i], g1 = mil[3 * i + 1], g2 = mil[3 * i + 2];
        if (i == 0 || g0 != mil[3 * (i - 1)] || g1 != mil[3 * (i - 1) + 1]) {
            const int x = posmod_(g0, n0);
            cslot.push_back(x * P + geo_slot(g[1], posmod_(g1, n1)));
            has_row[x] = 1;
        }
        ecz[i] = (((int)cslot.size() - 1) << 16) | geo_slot(g[2], posmod_(g2, n2));
    }
    for (int x = 0; x < n0; ++x)
        if (has_row[x]) rows.push_back(x);
    if ((int)cslot.size() != c->ncol) return;
    c->col_slot.alloc(cslot.size() * sizeof(int));
    c->ent_cz.alloc(ecz.size() * sizeof(int));
    c->xrows.alloc(rows.size() * sizeof(int));
    FS_CUDA(cudaMemcpy(c->col_slot.p, cslot.data(), cslot.size() * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->ent_cz.p, ecz.data(), ecz.size() * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->xrows.p, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice));
    c->gx = g[0];
    c->gy = g[1];
    c->gz = g[2];
    c->P = P;
    c->Pz = Pz;
    c->nxr = (int)rows.size();
    c->pf_items = std::max(n1 * std::max(g[0].A, g[0].B), c->nxr * std::max(g[1].A, g[1].B));
    c->cpb = cpb;
    c->zbig = !(fft_size_small(g[2].A) && fft_size_small(g[2].B));
    c->fast = true;
}

// spatial index held at position p of an axis in the permuted layout
int fft_perm_index(const fs_ctx* c, int d, int p) {
    const LineGeo& g = d == 0 ? c->gx : d == 1 ? c->gy : c->gz;
    return p / g.B + g.A * (p % g.B);
}

void ctx_prepare_fft(fs_ctx* c) {
    for (int d = 0; d < 3; ++d) {
        int n = c->n[d];
        std::vector<int> rads = factor_radices(n);
        if (rads.empty() || (int)rads.size() > FS_MAX_STAGES)
            throw fs_error(FS_ERR_ARG, "grid size " + std::to_string(n) + " is not of the form 2^a 3^b 5^c");
        std::vector<double2> t64(n);
        std::vector<float2> t32(n);
        for (int p = 0; p < n; ++p) {
            // exp(-2 pi i p / n), from the exact rational angle
            double ang = -2.0 * M_PI * (double)p / (double)n;
            t64[p] = make_double2(std::cos(ang), std::sin(ang));
            t32[p] = make_float2((float)t64[p].x, (float)t64[p].y);
        }
        c->tw64[d].alloc(n * sizeof(double2));
        c->tw32[d].alloc(n * sizeof(float2));
        FS_CUDA(cudaMemcpy(c->tw64[d].p, t64.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
        FS_CUDA(cudaMemcpy(c->tw32[d].p, t32.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
        int threads = (d == 2) ? COL_THREADS : PLANE_THREADS;
        int ept = (d == 2) ? COL_EPT : PLANE_EPT;
        int grp = group_lines(n, rads, threads, ept);
        if (grp < 1) throw fs_error(FS_ERR_ARG, "FFT length " + std::to_string(n) + " too long for one block");
        FftPlan<double2> p64{};
        FftPlan<float2> p32{};
        p64.n = p32.n = n;
        p64.nst = p32.nst = (int)rads.size();
        for (size_t s = 0; s < rads.size(); ++s) p64.rad[s] = p32.rad[s] = rads[s];
        p64.group = p32.group = grp;
        p64.tw = c->tw64[d].as<double2>();
        p32.tw = c->tw32[d].as<float2>();
        c->plan64[d] = p64;
        c->plan32[d] = p32;
    }
    size_t plane64 = (size_t)c->n[0] * c->n[1] * sizeof(double2);
    if (plane64 > 227 * 1024)
        throw fs_error(FS_ERR_ARG, "n0 * n1 plane does not fit in shared memory");
    c->cpb = 16;
    while (c->cpb > 1 && (size_t)col_smem(c->cpb, c->n[2], sizeof(double2)) > 200 * 1024) c->cpb /= 2;
    set_attr_smem<double2>((const void*)col_inverse_kernel<double2>, col_smem(c->cpb, c->n[2], sizeof(double2)));
    set_attr_smem<double2>((const void*)col_forward_kernel<double2>, col_smem(c->cpb, c->n[2], sizeof(double2)));
    set_attr_smem<float2>((const void*)col_inverse_kernel<float2>, col_smem(c->cpb, c->n[2], sizeof(float2)));
    set_attr_smem<float2>((const void*)col_forward_kernel<float2>, col_smem(c->cpb, c->n[2], sizeof(float2)));
    set_attr_smem<double2>((const void*)plane_kernel<double2, double>, (int)plane64);
    set_attr_smem<float2>((const void*)plane_kernel<float2, float>, (int)(plane64 / 2));
    set_attr_smem<double2>((const void*)zinv_kernel<double2, true>, 0);
    set_attr_smem<double2>((const void*)zfwd_kernel<double2, true>, 0);
    set_attr_smem<float2>((const void*)zinv_kernel<float2, true>, 0);
    set_attr_smem<float2>((const void*)zfwd_kernel<float2, true>, 0);
    set_attr_smem<double2>((const void*)zinv_kernel<double2, false>, 0);
    set_attr_smem<double2>((const void*)zfwd_kernel<double2, false>, 0);
    set_attr_smem<float2>((const void*)zinv_kernel<float2, false>, 0);
    set_attr_smem<float2>((const void*)zfwd_kernel<float2, false>, 0);
    set_attr_smem<double2>((const void*)plane_fast_kernel<double2, double>, 0);
    set_attr_smem<float2>((const void*)plane_fast_kernel<float2, float>, 0);
    prepare_fast_fft(c);
}

template <typename T2> static const void* vz_of(fs_ctx* c);
template <> const void* vz_of<double2>(fs_ctx* c) { return c->vz64.p; }
template <> const void* vz_of<float2>(fs_ctx* c) { return c->vz32.p; }
template <typename T2> static const T2* beta_of(fs_ctx* c);
template <> const double2* beta_of<double2>(fs_ctx* c) { return c->beta64.as<double2>(); }
template <> const float2* beta_of<float2>(fs_ctx* c) { return c->beta32.as<float2>(); }

// Local part (kinetic + V) of nbc bands through the column buffer cb:
// hpsi[b] = FFT(V FFT^-1 psi[b]) / N + (|q|^2/2 - shift) psi[b].  src rows are
// src[rm[b]] when rm is given, else consecutive.  prof: time each kernel class.
template <typename T2>
static void local_part(fs_ctx* c, const T2* src, const int* rm, T2* cb, T2* dst, int nbc, double shift, bool prof) {
    using R = typename real_of<T2>::t;
    const int n0 = c->n[0], n1 = c->n[1], n2 = c->n[2];
    const long colband = (long)n2 * c->ncol;
    const int cpb = c->cpb;
    const int ncb = (c->ncol + cpb - 1) / cpb;
    const double inv_ng = 1.0 / ((double)n0 * n1 * n2);
    const double colb = (double)nbc * colband * sizeof(T2), sphb = (double)nbc * c->npw * sizeof(T2);
    const double ng = (double)n0 * n1 * n2;
    fs_ctx* pc = prof ? c : nullptr;
    dim3 gc(ncb, nbc), gp(n2, nbc);
    if (c->fast) {
        const int zsm = (int)(((size_t)cpb * c->Pz + n2) * sizeof(T2));
        const int psm = (int)(((size_t)n0 * c->P + n0 + n1) * sizeof(T2));
        {
            ProfScope ps(pc, ks_prec<T2>(KS_COL_INV), sphb + colb, 5.0 * nbc * c->ncol * n2 * std::log2((double)n2));
            auto k = c->zbig ? zinv_kernel<T2, true> : zinv_kernel<T2, false>;
            k<<<gc, ZF_THREADS, zsm, c->stream>>>(src, rm, c->npw, cb, c->col_start.as<int>(), c->ent_cz.as<int>(),
                                                  c->ncol, cpb, c->gz, c->Pz, plan_of<T2>(c, 2).tw);
        }
        {
            ProfScope ps(pc, ks_prec<T2>(KS_PLANE), 2.0 * colb + ng * sizeof(R),
                         2.0 * 5.0 * nbc * ng * std::log2((double)n0 * n1));
            const int ipt = std::max(1, c->pf_ipt);
            const int pt = std::min(sizeof(T2) == 16 ? PF_MAX_THREADS / 2 : PF_MAX_THREADS,
                                    ((c->pf_items + ipt - 1) / ipt + 31) / 32 * 32);
            plane_fast_kernel<T2, R><<<gp, pt, psm, c->stream>>>(
                cb, c->col_slot.as<int>(), c->ncol, c->xrows.as<int>(), c->nxr,
                (const R*)vz_of<T2>(c), c->gx, c->gy, c->P, plan_of<T2>(c, 0).tw, plan_of<T2>(c, 1).tw);
        }
        {
            ProfScope ps(pc, ks_prec<T2>(KS_COL_FWD), colb + 2.0 * sphb, 5.0 * nbc * c->ncol * n2 * std::log2((double)n2));
            auto k = c->zbig ? zfwd_kernel<T2, true> : zfwd_kernel<T2, false>;
            k<<<gc, ZF_THREADS, zsm, c->stream>>>(cb, src, rm, c->npw, dst, c->col_start.as<int>(),
                                                  c->ent_cz.as<int>(), c->kin.as<double>(), c->ncol, cpb, c->gz,
                                                  c->Pz, plan_of<T2>(c, 2).tw, inv_ng, shift, c->npw);
        }
        return;
    }
    const FftPlan<T2>& px = plan_of<T2>(c, 0);
    const FftPlan<T2>& py = plan_of<T2>(c, 1);
    const FftPlan<T2>& pz = plan_of<T2>(c, 2);
    const int csm = col_smem(cpb, n2, sizeof(T2));
    const int psm = n0 * n1 * (int)sizeof(T2);
    {
        ProfScope ps(pc, ks_prec<T2>(KS_COL_INV), sphb + colb, 5.0 * nbc * c->ncol * n2 * std::log2((double)n2));
        col_inverse_kernel<T2><<<gc, COL_THREADS, csm, c->stream>>>(src, rm, c->npw, cb, c->col_start.as<int>(),
                                                                     c->ent_col.as<int>(), c->ent_z.as<int>(),
                                                                     c->ncol, cpb, pz);
    }
    {
        ProfScope ps(pc, ks_prec<T2>(KS_PLANE), 2.0 * colb + ng * sizeof(R), 2.0 * 5.0 * nbc * ng * std::log2((double)n0 * n1));
        plane_kernel<T2, R><<<gp, PLANE_THREADS, psm, c->stream>>>(cb, c->col_xy.as<int>(), c->ncol,
                                                                   (const R*)vz_of<T2>(c), px, py);
    }
    {
        ProfScope ps(pc, ks_prec<T2>(KS_COL_FWD), colb + 2.0 * sphb, 5.0 * nbc * c->ncol * n2 * std::log2((double)n2));
        col_forward_kernel<T2><<<gc, COL_THREADS, csm, c->stream>>>(
            cb, src, rm, c->npw, dst, c->col_start.as<int>(), c->ent_col.as<int>(), c->ent_z.as<int>(),
            c->kin.as<double>(), c->ncol, cpb, pz, inv_ng, shift, c->npw);
    }
}

// Bands are processed in chunks: on the register-FFT path a chunk's column
// buffer is sized to stay in L2 between the three passes.
template <typename T2>
void apply_H_impl(fs_ctx* c, const T2* psi, T2* hpsi, int nb, double shift, const int* rowmap) {
    if (nb <= 0) return;
    const long colband = (long)c->n[2] * c->ncol;
    const long max_chunk_bytes = c->fast ? (long)c->hchunk_bytes : (2L << 30);
    int chunk = (int)std::max(1L, std::min((long)nb, max_chunk_bytes / (colband * (long)sizeof(T2))));
    c->colbuf.ensure((size_t)chunk * colband * sizeof(T2));
    T2* cb = c->colbuf.as<T2>();
    for (int b0 = 0; b0 < nb; b0 += chunk) {
        int nbc = std::min(chunk, nb - b0);
        const T2* src = rowmap ? psi : psi + (long)b0 * c->npw;
        const int* rm = rowmap ? rowmap + b0 : nullptr;
        local_part<T2>(c, src, rm, cb, hpsi + (long)b0 * c->npw, nbc, shift, true);
        FS_CUDA(cudaGetLastError());
    }
    if (c->nptot > 0) {
        // P[b][p] = sum_g conj(beta[p][g]) psi[b][g]   -> written as P[b * nptot + p]
        c->projbuf.ensure((size_t)nb * c->nptot * sizeof(double2));
        c->projbuf2.ensure((size_t)nb * c->nptot * sizeof(double2));
        double2* P = c->projbuf.as<double2>();
        bool tc_gen = false;
        if constexpr (sizeof(T2) == 8) tc_gen = c->beta_gen && c->gemm_path == FS_GEMM_TENSOR;
        const BetaGen gen = c->beta_gen ? beta_gen_of(c) : BetaGen{};
        if (tc_gen) {
            if constexpr (sizeof(T2) == 8)
                tc_gemm_gram(c, c->nptot, nb, c->npw, nullptr, 0, nullptr, psi, c->npw, rowmap, P, 1, c->nptot, 1.0,
                             0.0, KS_NL_PROJ, &gen);
        } else if (c->beta_gen) {
            beta_project_chunked<T2>(c, psi, rowmap, nb, P);
        } else {
            gemm_gram<T2>(c, c->nptot, nb, c->npw, beta_of<T2>(c), c->npw, nullptr, psi, c->npw, rowmap, P, 1,
                          c->nptot, 1.0, 0.0, ks_prec<T2>(KS_NL_PROJ));
        }
        double2* Q = c->projbuf2.as<double2>();
        int blocks = (int)std::min<long>(4096, ((long)nb * c->nptot + 255) / 256);
        {
            ProfScope ps(c, KS_NL_D, 2.0 * nb * c->nptot * sizeof(double2), 4.0 * nb * c->nptot * c->nproj);
            apply_D_kernel<double2><<<blocks, 256, 0, c->stream>>>(P, Q, c->Dmat.as<double>(), c->natom, c->nproj, nb);
        }
        FS_CUDA(cudaGetLastError());
        // hpsi[b][g] += sum_p Q[b][p] beta[p][g]
        if (tc_gen) {
            if constexpr (sizeof(T2) == 8)
                tc_gemm_nn<double2>(c, nb, c->npw, c->nptot, Q, c->nptot, 1, nullptr, c->npw, nullptr, hpsi, c->npw,
                                    nullptr, 1.0, 1.0, hpsi, c->npw, KS_NL_ADD, &gen);
        } else if (c->beta_gen) {
            beta_add_chunked<T2>(c, Q, nb, hpsi);
        } else {
            gemm_nn<T2, double2>(c, nb, c->npw, c->nptot, Q, c->nptot, 1, beta_of<T2>(c), c->npw, nullptr, hpsi,
                                 c->npw, nullptr, 1.0, 1.0, hpsi, c->npw, ks_prec<T2>(KS_NL_ADD));
        }
    }
}

template void apply_H_impl<double2>(fs_ctx*, const double2*, double2*, int, double, const int*);
template void apply_H_impl<float2>(fs_ctx*, const float2*, float2*, int, double, const int*);

// ------------------------------------------------------------------ static-scratch H application
// fs_apply_H_static: the FP64 H application with every intermediate in one
// file-scope device array instead of buffers the library allocates.  Callers
// that may not allocate device memory at the time of the call (for example
// code running under an allocator that forbids cudaMalloc, or a host that
// pre-plans all of its device memory) use it after fs_create.
template <typename T2>
bool gemm_gram_scratch(cudaStream_t st, int M, int N, int K, const T2* A, long lda, const T2* B, long ldb, double2* C,
                       long ci, long cj, double2* part, size_t part_bytes);
void gemm_nn_plain64(cudaStream_t st, int M, int N, int K, const double2* A, long ai, long ak, const double2* B,
                     long ldb, double2* C, long ldc, double alpha, double beta, const double2* D, long ldd);

#include <mutex>

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[FS_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the context's device, which must be
// the current device (looked up once per device).
fs_status scratch_address(int ctx_dev, void** out, std::string& err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        err = "fs_apply_H_static: no usable current device";
        return FS_ERR_CUDA;
    }
    if (dev != ctx_dev) {
        err = "fs_apply_H_static: the current device (" + std::to_string(dev) + ") is not the context's device (" +
              std::to_string(ctx_dev) + "); make the context's device current first";
        return FS_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("fs_apply_H_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
            return FS_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return FS_OK;
}

}  // namespace

extern "C" fs_status fs_apply_H_static(fs_ctx* c, const void* psi, void* hpsi, int nband, double shift) {
    if (!c) return FS_ERR_ARG;
    if (nband < 0 || (nband > 0 && (!psi || !hpsi || psi == hpsi)) || !std::isfinite(shift)) {
        c->err = "fs_apply_H_static: bad arguments";
        return FS_ERR_ARG;
    }
    if (nband == 0) return FS_OK;
    if (c->beta_gen) {
        c->err = "fs_apply_H_static: the context generates its projectors (no stored table); create it with "
                 "projectors = FS_PROJ_STORED";
        return FS_ERR_ARG;
    }
    void* base = nullptr;
    fs_status st = scratch_address(c->device, &base, c->err);
    if (st != FS_OK) return st;
    const size_t colband = (size_t)c->n[2] * c->ncol * sizeof(double2);
    const size_t projband = (size_t)c->nptot * sizeof(double2);
    // one band needs its column buffer, P and Q, and one split of the Gram partial sums
    const size_t per_band = colband + 3 * projband;
    if (per_band > (size_t)FS_STATIC_SCRATCH_BYTES) {
        c->err = "fs_apply_H_static: one band needs " + std::to_string(per_band) + " bytes of scratch, more than the " +
                 std::to_string((size_t)FS_STATIC_SCRATCH_BYTES) + " bytes of the static array";
        return FS_ERR_ARG;
    }
    int chunk = (int)std::max<size_t>(1, std::min<size_t>(nband, FS_STATIC_SCRATCH_BYTES / per_band));
    unsigned char* s = static_cast<unsigned char*>(base);
    double2* cb = reinterpret_cast<double2*>(s);
    double2* P = reinterpret_cast<double2*>(s + chunk * colband);
    double2* Q = P + (size_t)chunk * c->nptot;
    double2* part = Q + (size_t)chunk * c->nptot;
    const size_t part_bytes = (size_t)FS_STATIC_SCRATCH_BYTES - (size_t)((unsigned char*)part - s);
    const double2* in = static_cast<const double2*>(psi);
    double2* out = static_cast<double2*>(hpsi);
    for (int b0 = 0; b0 < nband; b0 += chunk) {
        const int nbc = std::min(chunk, nband - b0);
        const double2* src = in + (long)b0 * c->npw;
        double2* dst = out + (long)b0 * c->npw;
        local_part<double2>(c, src, nullptr, cb, dst, nbc, shift, false);
        if (c->nptot > 0) {
            if (!gemm_gram_scratch<double2>(c->stream, c->nptot, nbc, c->npw, c->beta64.as<double2>(), c->npw, src,
                                            c->npw, P, 1, c->nptot, part, part_bytes)) {
                c->err = "fs_apply_H_static: projections do not fit in the static scratch";
                return FS_ERR_ARG;
            }
            int blocks = (int)std::min<long>(4096, ((long)nbc * c->nptot + 255) / 256);
            apply_D_kernel<double2><<<blocks, 256, 0, c->stream>>>(P, Q, c->Dmat.as<double>(), c->natom, c->nproj,
                                                                   nbc);
            gemm_nn_plain64(c->stream, nbc, c->npw, c->nptot, Q, c->nptot, 1, c->beta64.as<double2>(), c->npw, dst,
                            c->npw, 1.0, 1.0, dst, c->npw);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            c->err = std::string("fs_apply_H_static: ") + cudaGetErrorString(e);
            return FS_ERR_CUDA;
        }
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("fs_apply_H_static: ") + cudaGetErrorString(e);
        return FS_ERR_CUDA;
    }
    c->err.clear();
    return FS_OK;
}
