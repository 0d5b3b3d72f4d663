// Shared device helpers and the context layout of the folded-spectrum library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fs.h"

// size of the file-scope scratch array used by fs_apply_H_static (64 MiB)
#define FS_STATIC_SCRATCH_BYTES (64ull << 20)

// ------------------------------------------------------------------ complex
template <typename R> struct cplx;
template <> struct cplx<double> { using t = double2; };
template <> struct cplx<float> { using t = float2; };

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

template <typename T2> __host__ __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T2> __host__ __device__ __forceinline__ T2 csub(T2 a, T2 b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T2> __host__ __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename T2> __host__ __device__ __forceinline__ T2 cmulc(T2 a, T2 b) {
    return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename T2, typename R> __host__ __device__ __forceinline__ T2 cscale(T2 a, R s) {
    return mk(a.x * s, a.y * s);
}

template <typename T2> struct real_of;
template <> struct real_of<double2> { using t = double; };
template <> struct real_of<float2> { using t = float; };

__device__ __forceinline__ double2 to_c(double2 a, double2*) { return a; }
__device__ __forceinline__ float2 to_c(double2 a, float2*) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ float2 to_c(float2 a, float2*) { return a; }
__device__ __forceinline__ double2 to_c(float2 a, double2*) { return make_double2(a.x, a.y); }
template <typename T2, typename S2> __device__ __forceinline__ T2 conv(S2 a) { return to_c(a, (T2*)nullptr); }

// ------------------------------------------------------------------ FFT plan
// A 1-D length-n transform as a list of radix-2/3/4/5 Stockham stages.
// tw points to n twiddles w^p = exp(-2 pi i p / n) in the transform's precision.
// group = how many lines the kernel's thread block transforms at once.
#define FS_MAX_STAGES 12
template <typename T2> struct FftPlan {
    int n;
    int nst;
    int rad[FS_MAX_STAGES];
    int group;
    const T2* tw;
};

// Geometry of one line family of the register FFTs (fs_fft.cuh): length
// L = A * B, element stride es (in elements), block pitch Bp = B + pad (pad 0
// or 1 slot after every block of B positions).
struct LineGeo {
    int L, A, B, Bp, es;
};
__host__ __device__ inline int geo_slot(const LineGeo& g, int p) { return p + (g.Bp - g.B) * (p / g.B); }

// ------------------------------------------------------------------ errors
#define FS_CUDA(call)                                                                    \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            throw fs_error(FS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                \
    } while (0)

struct fs_error {
    fs_status code;
    std::string msg;
    fs_error(fs_status c, std::string m) : code(c), msg(std::move(m)) {}
};

// ------------------------------------------------------------------ device buffer
struct dbuf {
    void* p = nullptr;
    size_t bytes = 0;
    void alloc(size_t nb) {
        release();
        if (nb == 0) return;
        cudaError_t e = cudaMalloc(&p, nb);
        if (e != cudaSuccess) {
            p = nullptr;
            (void)cudaGetLastError();
            throw fs_error(FS_ERR_OOM, "cudaMalloc of " + std::to_string(nb) + " bytes failed");
        }
        bytes = nb;
    }
    void ensure(size_t nb) {
        if (nb > bytes) alloc(nb);
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
    ~dbuf() { release(); }
    dbuf() = default;
    dbuf(const dbuf&) = delete;
    dbuf& operator=(const dbuf&) = delete;
};

// ------------------------------------------------------------------ kernel timing
// Optional per-kernel-class timing with CUDA events on the context's stream
// (enabled by fs_profile); each launch also adds its algorithmic bytes/flops.
enum {
    KS_COL_INV = 0,  // unpack + inverse z-FFT
    KS_PLANE,        // xy-plane FFTs with the V(r) multiply
    KS_COL_FWD,      // forward z-FFT + pack + kinetic/shift
    KS_NL_PROJ,      // <beta|psi> projections
    KS_NL_D,         // D contraction per atom
    KS_NL_ADD,       // hpsi += beta Q
    KS_GRAM,         // solver Gram matrices / inner products
    KS_ROTATE,       // solver basis rotations and projections
    KS_VECTOR,       // residuals, preconditioner, norms, scaling
    KS_DENSE_LA,     // FP64 small dense eigensolves and products
    // the same work in FP64 (FP64 stage and the FP64 check of the FP32 result)
    KS_COL_INV64,
    KS_PLANE64,
    KS_COL_FWD64,
    KS_NL_PROJ64,
    KS_NL_ADD64,
    KS_GRAM64,
    KS_ROTATE64,
    KS_VECTOR64,
    // parts of the dense FP64 algebra, timed inside the scopes above (their
    // times are contained in those of the enclosing classes, not added to them)
    KS_SUB_POTRF,    // blocked Cholesky
    KS_SUB_TRSM,     // blocked triangular solves
    KS_SUB_HETRD,    // Householder reduction to tridiagonal form
    KS_SUB_TRIEIG,   // tridiagonal eigenvalues (bisection) and vectors (inverse iteration)
    KS_SUB_BACK,     // back-transformation of the eigenvectors (compact WY)
    KS_COUNT
};
// class of a step in the arithmetic of T2 (FP64 steps are counted apart)
template <typename T2> constexpr int ks_prec(int id) {
    if (sizeof(T2) != 16) return id;
    switch (id) {
        case KS_COL_INV: return KS_COL_INV64;
        case KS_PLANE: return KS_PLANE64;
        case KS_COL_FWD: return KS_COL_FWD64;
        case KS_NL_PROJ: return KS_NL_PROJ64;
        case KS_NL_ADD: return KS_NL_ADD64;
        case KS_GRAM: return KS_GRAM64;
        case KS_ROTATE: return KS_ROTATE64;
        case KS_VECTOR: return KS_VECTOR64;
        default: return id;
    }
}
struct KStat {
    long long launches = 0;
    double ms = 0, bytes = 0, flops = 0;
};
struct Prof {
    bool on = false;
    KStat st[KS_COUNT];
    struct Pend {
        int id;
        cudaEvent_t a, b;
    };
    std::vector<Pend> pend;
    std::vector<cudaEvent_t> pool;
};

// ------------------------------------------------------------------ learned preconditioner state
struct Mlp {
    bool ready = false;
    int nshell = 32;
    dbuf shell_of, perm, off;      // shell of each plane wave; plane waves grouped by shell
    dbuf P, T, m, v, g;            // master params, prepared (BF16, transposed), Adam moments, gradient
    dbuf gpart, lpart;             // per-block partial gradients / losses
    dbuf r2, num, den;             // shell sums
    dbuf F, z;                     // features and outputs of the current iteration
    dbuf Mdev;                     // the paper's M(G) at e_ref
    double e_ref = 0;
    int step = 0;
    // recording of training rows during a solve
    bool record = false;
    int nref = 0;
    dbuf xref64, xref32;           // reference states [nref][npw]
    dbuf recF, recz, recw;         // recorded rows
    long long nrec = 0, cap = 0, nrec_bands = 0;
    dbuf proj, err;                // work: projections onto the reference span, errors
};

// ------------------------------------------------------------------ solver workspace
// Kept by the context between solves (allocated on first use, grown when
// needed, released by fs_destroy), so that repeated and concurrent solves do
// not allocate or free device memory (cudaFree synchronises the device).
// formatted operand images of the tensor-core apply form: the projector table
// is kept formatted when its image fits this size; a band block is formatted
// in chunks of plane-wave tiles of at most the second size
constexpr size_t FS_TABLE_FMT_MAX_BYTES = 32ull << 30;
constexpr size_t FS_FMT_CHUNK_BYTES = 4ull << 30;

// Workspace of the dense FP64 linear algebra (fs_dense.cu), kept by the context.
#define FS_DENSE_MAX_N 2048
struct DenseWork {
    dbuf V, tau, d, e, e2, Y, z, work, info3, bar, info, T, U, wyG, wyT, wyW, wyW2, gpart, qrG, qrT;
    bool attr_set = false;
};

struct SolverSmall {
    dbuf GA, GB, T1, T2, evals, work, info, theta, act, resid, dots, nrm, shift, dscale, bkin, hres, keep;
    int lwork = 0;
    int nbmax = 0;
};
struct SolverMem {
    dbuf b32[12], b64[12];   // band blocks of the FP32 and FP64 stages
    dbuf x0;                 // start block
    SolverSmall small;
};

// ------------------------------------------------------------------ context
struct fs_ctx {
    // geometry and basis
    double L[3];
    int n[3];
    double ecut;
    double k[3];
    int npw = 0;
    int ncol = 0;
    int natom = 0, nproj = 0, nptot = 0;
    std::vector<int> miller;      // [npw][3]
    std::vector<double> kin_h;    // [npw]
    fs_options opt;

    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;   // the device that was current at fs_create (every buffer lives there)

    // basis tables (device)
    dbuf col_start;   // int [ncol+1]
    dbuf col_xy;      // int [ncol] : (g0 mod n0) * n1 + (g1 mod n1)
    dbuf ent_col;     // int [npw]  : column of each sphere entry
    dbuf ent_z;       // int [npw]  : g2 mod n2
    dbuf kin;         // double [npw] : |k+G|^2 / 2
    dbuf vz64;        // double [n2][n0*n1]
    dbuf vz32;        // float  [n2][n0*n1]
    dbuf tw64[3];     // double2 [n_d]
    dbuf tw32[3];     // float2  [n_d]
    FftPlan<double2> plan64[3];
    FftPlan<float2> plan32[3];
    int cpb = 16;     // columns per block in the column kernels
    // register-FFT path: line geometries of x (rows of a plane), y (within a
    // row, padded) and z (columns, padded); row pitch P of a plane, line pitch
    // Pz of a column tile; rows of a plane that hold sphere columns; per-column
    // slot in the plane (x P + y slot); per sphere entry its column and z slot
    // packed as (column << 16 | z slot).  V(r) (vz64/vz32) is then stored in
    // the permuted layout [p_z][p_x][p_y].
    bool fast = false;
    bool zbig = false;  // the z split needs the large register DFT sizes (16, 27)
    LineGeo gx{}, gy{}, gz{};
    int P = 0, Pz = 0, nxr = 0, pf_items = 0;  // pf_items: line items of the busiest plane pass
    int pf_ipt = 4;                              // items per thread of the plane kernel
    dbuf xrows, col_slot, ent_cz;
    size_t hchunk_bytes = 96ull << 20;  // column-buffer bytes per band chunk (kept in L2 between passes)

    // projectors
    bool beta_gen = false;  // no table: projector values formed where they are used (fs_beta.cuh)
    dbuf bg_rad, bg_ph, bg_rad32, bg_ph32, bg_gidx, bg_pl;
    int bg_span = 0;
    dbuf beta_chunk;  // generated rows of the table for the CUDA-core GEMMs
    dbuf beta64;      // double2 [nptot][npw]
    dbuf beta32;      // float2  [nptot][npw]
    dbuf Dmat;        // double  [natom][nproj][nproj]

    // workspace for H application
    dbuf colbuf;      // [nb][n2][ncol] complex
    dbuf projbuf;     // [nb][nptot] complex (P)
    dbuf projbuf2;    // [nb][nptot] complex (Q = D P)
    dbuf splitk;      // split-K partial sums
    dbuf beta32_fmt;  // projector table as tensor-core apply-form operand images (formatted once)
    dbuf afmt;        // apply-form operand images of a band block (per call)
    dbuf bfmt;        // apply-form coefficient images (per call)
    dbuf beta32_gfmt; // projector table as Gram-form operand images (formatted once)
    dbuf gfmt_a;      // Gram-form images of the first operand (per call)
    dbuf gfmt_b;      // Gram-form images of the second operand with rotated rows (per call)

    // solver state
    dbuf init_states; // double2 [ninit][npw]
    int ninit = 0;
    int init_damp = 1;
    dbuf result_states;  // double2 [nstates][npw]
    int nresult = 0;
    std::vector<double> result_eps, result_resid;  // eigenvalues and H residuals of the last solve

    // folded linear solve: eigenstates of the M' preconditioner and the PCG vectors
    dbuf lin_phi;        // double2 [lin_n][npw]
    int lin_n = 0;
    std::vector<double> lin_eps, lin_delta;
    dbuf lin_vec[9];     // psi, y, r, r_old, p, yp, ap, z, u: [nrhs][npw] each
    dbuf lin_small;      // projections <phi_i|r_l>, coefficients, per-row scalars and partial sums
    dbuf lin_io[2];      // device copies of host right-hand sides and solutions

    Prof prof;
    Mlp mlp;
    DenseWork dense;
    SolverMem smem;
    dbuf errflag;     // int: set by a device-side wait that gave up
    int gemm_path = 0;
    std::string err;
};

void prof_flush(fs_ctx* c);
void prof_release(fs_ctx* c);
// RAII scope around one launch (or a short sequence) of kernel class id
struct ProfScope {
    fs_ctx* c;
    int id;
    cudaEvent_t a = nullptr;
    ProfScope(fs_ctx* c_, int id_, double bytes, double flops);
    ~ProfScope();
};

// ------------------------------------------------------------------ internal entry points
// H application (fs_h.cu)
template <typename T2>
void apply_H_impl(fs_ctx* c, const T2* psi, T2* hpsi, int nb, double shift, const int* rowmap_in = nullptr);

void ctx_prepare_fft(fs_ctx* c);
int fft_perm_index(const fs_ctx* c, int d, int p);  // spatial index at position p of axis d (register-FFT path)

// folded linear solve (fs_linear.cu): device w and psi [nrhs][npw] complex128
fs_status linear_solve_impl(fs_ctx* c, double e_ref, const double2* w, double2* psi, int nrhs, bool from_psi,
                            double tol, int maxit, fs_linres* res);

// GEMMs (fs_gemm.cu)
// Gram form: C(i, j) = alpha * sum_k conj(A[ia(i)][k]) * B[ib(j)][k]  (+ beta * C(i, j))
// A rows: M, stride lda; B rows: N, stride ldb; K contiguous.  Optional row maps.
// C(i, j) is written as double2 at C[i * ci + j * cj].
template <typename T2>
void gemm_gram(fs_ctx* c, int M, int N, int K, const T2* A, long lda, const int* amap, const T2* B, long ldb,
               const int* bmap, double2* C, long ci, long cj, double alpha, double beta, int kid = KS_GRAM);
// Rotation/apply form: C[ic(i)][n] = alpha * sum_k Acoef(i, k) * B[ib(k)][n] + beta * D[ic(i)][n]
// Acoef(i, k) = A[i * ai + k * ak] (A2 complex coefficients, double2 or T2);  D may equal C or be null.
template <typename T2, typename A2>
void gemm_nn(fs_ctx* c, int M, int N, int K, const A2* A, long ai, long ak, const T2* B, long ldb, const int* bmap,
             T2* C, long ldc, const int* cmap, double alpha, double beta, const T2* D, long ldd, int kid = KS_ROTATE);

// tensor-core GEMMs for the FP32 stage (fs_tc.cu); gen: the table operand (A of the
// Gram form, B of the apply form) is the generated projector table (fs_beta.cuh)
struct BetaGen;
void tc_gemm_gram(fs_ctx* c, int M, int N, int K, const float2* A, long lda, const int* amap, const float2* B,
                  long ldb, const int* bmap, double2* C, long ci, long cj, double alpha, double beta, int kid,
                  const BetaGen* gen = nullptr);
template <typename A2>
void tc_gemm_nn(fs_ctx* c, int M, int N, int K, const A2* A, long ai, long ak, const float2* B, long ldb,
                const int* bmap, float2* C, long ldc, const int* cmap, double alpha, double beta, const float2* D,
                long ldd, int kid, const BetaGen* gen = nullptr);
// generated projectors (fs_beta.cu)
void beta_gen_setup(fs_ctx* c, const fs_projectors* pr, double omega);
template <typename T2> void beta_project_chunked(fs_ctx* c, const T2* psi, const int* rowmap, int nb, double2* P);
template <typename T2> void beta_add_chunked(fs_ctx* c, const double2* Q, int nb, T2* hpsi);
int* ctx_errflag(fs_ctx* c);
void ctx_check_errflag(fs_ctx* c);

// vector kernels (fs_vec.cu)
template <typename T2> void vec_resid(fs_ctx* c, const T2* X, const T2* Y, int m, double* resid, double2* dot);
template <typename T2>
void vec_make_w(fs_ctx* c, const T2* R, const int* act, int na, T2* W, double e_ref, double dE, int precond,
                const double* band_kin);
template <typename T2> void vec_rh(fs_ctx* c, const T2* X, const T2* Y, const double2* dots, int m, T2* RH);
template <typename T2>
void vec_a_resid(fs_ctx* c, const T2* ZR, T2* RH, const T2* X, const double2* dots, const double* theta, int m,
                 double* ra);
template <typename T2> void vec_row_norms(fs_ctx* c, const T2* X, const int* map, int nrows, double* out);
template <typename T2> void vec_band_kin(fs_ctx* c, const T2* X, int m, double* out);
template <typename T2> void vec_scale_rows(fs_ctx* c, T2* X, const int* map, int nrows, const double* nrm);
template <typename T2>
void vec_resid_shift(fs_ctx* c, const T2* X, const T2* Y, const double* shift, int m, double* resid);
void vec_damp_random(fs_ctx* c, double2* X, int m, int first, unsigned long long seed);
void vec_damp(fs_ctx* c, double2* X, int m);
template <typename S2, typename T2> void vec_convert(fs_ctx* c, const S2* in, T2* out, size_t count);

// learned preconditioner (fs_mlp.cu)
int mlp_nparam();
void mlp_setup(fs_ctx* c);
void mlp_prepare(fs_ctx* c);
void mlp_forward(fs_ctx* c, const float* F, int rows, float* z);
double mlp_loss_grad(fs_ctx* c, const float* F, const float* zt, const float* wt, int rows, double sw);
void mlp_adam(fs_ctx* c, float lr);
template <typename T2>
void mlp_features(fs_ctx* c, const T2* R, const int* act, int na, const double2* dots, const T2* Err, float* F,
                  float* zt, float* wt);
template <typename T2> void mlp_make_w(fs_ctx* c, const T2* R, const int* act, int na, T2* W, const double2* dots);
template <typename T2> void mlp_err_from_proj(fs_ctx* c, const T2* proj, const T2* X, const int* act, int na, T2* E);

// dense FP64 linear algebra (fs_dense.cu); column-major complex, op 0 = N, 1 = C
void dense_gemm(fs_ctx* c, int opA, int opB, int M, int N, int K, double alpha, const double2* A, int lda,
                const double2* B, int ldb, double beta, double2* C, int ldc);
int dense_potrf(fs_ctx* c, int n, double2* A, int lda, double* piv);
void dense_trsm(fs_ctx* c, int conj, int n, int ncols, const double2* L, int lda, double2* B, int ldb);
void dense_conj_transpose(fs_ctx* c, int n, int m, const double2* A, int lda, double2* out, int ldo);
void dense_heev(fs_ctx* c, int n, double2* A, int m, double* w, double2* Z, int ldz);
int dense_hegv(fs_ctx* c, int n, double2* GA, double2* GB, int m, double* w);

// solver (fs_solver.cu)
fs_status solve_impl(fs_ctx* c, double e_ref, int nstates, double tol, fs_result* res, bool lowest = false);
