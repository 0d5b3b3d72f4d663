/*
 * fs.h - C ABI of the GB300 folded-spectrum eigensolver.
 *
 * The library finds the eigenpairs of a plane-wave Kohn-Sham Hamiltonian H
 * that lie nearest a reference energy E by minimising the folded operator
 * A = (H - E)^2 (paper, Sec. II.C, Eq. wl1 and the folded-spectrum method it
 * cites), using an all-band preconditioned conjugate-gradient method in its
 * locally optimal block form with the paper's G-space diagonal preconditioner
 * M(G) = 1/((G^2 - E)^2 + dE^2) (Sec. II.C, the definition under the M'
 * equation), taken in Hartree as M(q) = 1/((|q|^2/2 - E)^2 + dE^2).
 *
 * Units: Hartree atomic units (bohr, Ha).
 *
 * H on the sphere S = { q = k + G : |q|^2/2 <= ecut } of plane waves
 * G = 2 pi (g0/L0, g1/L1, g2/L2):
 *   kinetic   |q|^2 / 2 on the diagonal;
 *   local     Hloc[G,G'] = Vt((g - g') mod n), Vt = N^-1 sum_j V(r_j) e^{-2 pi i h.j/n},
 *             applied as  FFT^-1 -> multiply by V(r) -> FFT  on the n0 x n1 x n2 grid;
 *   nonlocal  sum_a sum_ij |beta_ai> D^a_ij <beta_aj| with Gaussian s/p projectors
 *             beta_s(q)  = Omega^-1/2 (pi w^2)^{-3/4} (2 pi w^2)^{3/2} e^{-w^2 q^2/2} e^{-i q.R_a}
 *             beta_p,x(q) = beta_s(q) (sqrt(2)/w) (-i w^2 q_x)   (and y, z).
 *
 * Sphere order: z-columns sorted by (g0, g1) ascending, each column by g2
 * ascending.  Coefficient vectors are [nband][npw], complex interleaved
 * (re, im): complex128 for FS_FP64, complex64 for FS_MIXED.
 *
 * Conventions:
 *   - Every call returns fs_status; nothing throws across this boundary.
 *   - fs_create copies every host input to the device; the caller keeps
 *     ownership of its arrays and may free them on return.
 *   - Device buffers passed in are caller-owned and must stay valid until
 *     the call returns; all work runs on the context's stream and every call
 *     returns only after that work has finished.
 *   - A context is not thread-safe: one thread (one stream) per context.
 *   - fs_last_error returns the message of the last failure on that context.
 */
#ifndef FS_H
#define FS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fs_ctx fs_ctx;

typedef enum {
    FS_OK = 0,
    FS_ERR_ARG = 1,             /* invalid argument (null pointer, size, range) */
    FS_ERR_GRID_TOO_SMALL = 2,  /* some axis needs more than n_d distinct Miller indices */
    FS_ERR_OOM = 3,             /* device allocation failed */
    FS_ERR_CUDA = 4,            /* a CUDA runtime or library call failed */
    FS_ERR_NUMERIC = 5,         /* NaN/Inf or a Gram matrix that is not positive definite */
    FS_ERR_NOT_CONVERGED = 6,   /* iteration cap reached; results are still filled */
    FS_ERR_TIMEOUT = 7,         /* a bounded device-side wait gave up */
    FS_ERR_UNIMPLEMENTED = 8
} fs_status;

enum { FS_FP64 = 0, FS_MIXED = 1 };                     /* arithmetic of the vector work */
enum { FS_PREC_M = 0, FS_PREC_TETER = 1, FS_PREC_LEARNED = 2 };
enum { FS_HOST = 0, FS_DEVICE = 1 };                     /* where a state buffer lives */
enum { FS_GEMM_TENSOR = 0, FS_GEMM_CUDA_CORES = 1 };     /* FP32-stage GEMM engine */

/* Orthorhombic cell (bohr) and FFT grid.  Grid point j sits at r_j = (j_d L_d / n_d). */
typedef struct {
    double L[3];
    int n[3];
} fs_grid;

/* Gaussian s/p projectors, the same set on every atom.
 *   pos   [natom][3]          atom positions, bohr
 *   l     [nproj]             0 = s, 1 = p
 *   axis  [nproj]             Cartesian axis of a p projector (0 = x, 1 = y, 2 = z); ignored for s
 *   width [nproj]             Gaussian width w, bohr (exp(-r^2 / (2 w^2)))
 *   D     [natom][nproj][nproj] real symmetric coupling, Ha
 * natom = 0 or nproj = 0 means no nonlocal term. */
typedef struct {
    int natom;
    int nproj;
    const double* pos;
    const int* l;
    const int* axis;
    const double* width;
    const double* D;
} fs_projectors;

typedef struct {
    int precision;             /* FS_FP64 or FS_MIXED */
    int precond;               /* FS_PREC_M (default), FS_PREC_TETER, FS_PREC_LEARNED */
    double dE;                 /* preconditioner broadening, Ha (default 0.5 when <= 0) */
    int maxit;                 /* iteration cap (default 5000 when <= 0) */
    int guard;                 /* extra bands beyond nstates (< 0: max(4, nstates/16)) */
    unsigned long long seed;   /* start block when none is supplied */
    void* cuda_stream;         /* cudaStream_t to run on (NULL: the library's own stream) */
    int verbose;               /* > 0: one line per iteration on stderr */
    int gemm_path;             /* FP32-stage GEMMs: FS_GEMM_TENSOR (default, tcgen05 TF32 x3 split)
                                  or FS_GEMM_CUDA_CORES (FP32 FMA); FP64 work always uses FP64 FMA */
    int projectors;            /* FS_PROJ_AUTO (0, default): the projector table beta[N_p][npw] is
                                  stored when its FP64 form takes at most 16 GB, else generated;
                                  FS_PROJ_STORED; FS_PROJ_GENERATED: beta is formed where it is used
                                  from per-type radial factors and per-atom one-axis phase tables
                                  (beta = f_c(|q|) exp(-i q_x X_a) exp(-i q_y Y_a) exp(-i q_z Z_a)), so
                                  no N_p x npw table exists (fs_apply_H_static then refuses) */
} fs_options;

enum { FS_PROJ_AUTO = 0, FS_PROJ_STORED = 1, FS_PROJ_GENERATED = 2 };

typedef struct {
    int nconv;                 /* states among the nstates wanted with resid <= tol */
    int iters;                 /* block iterations taken */
    long long n_hpsi;          /* band applications of H (one per band per H call) */
    double* eps;               /* caller-allocated [nstates]: eigenvalues, Ha, ordered by (|eps-E|, eps) */
    double* resid;             /* caller-allocated [nstates]: ||H psi - eps psi|| (FP64) */
    double seconds;            /* wall time of the solve */
    int iters_mixed;           /* iterations taken in the mixed-precision stage */
} fs_result;

/* Build a context: enumerate the plane-wave sphere, upload V(r) and build the
 * projector table.  vloc is host [n0][n1][n2] C-order, Ha.  k is Cartesian,
 * 1/bohr.  opts may be NULL (defaults).  On failure *out is NULL and the status
 * says why (FS_ERR_GRID_TOO_SMALL when 2 h_d + 1 > n_d on some axis). */
fs_status fs_create(const fs_grid* grid, double ecut, const double k[3],
                    const double* vloc, const fs_projectors* proj,
                    const fs_options* opts, fs_ctx** out);

/* Number of plane waves in the sphere. */
fs_status fs_npw(const fs_ctx* ctx, int* npw);

/* Miller indices of the sphere, host [npw][3] int, in sphere order. */
fs_status fs_gvectors(const fs_ctx* ctx, int* miller);

/* hpsi = (H - shift) psi for nband bands.  psi and hpsi are DEVICE pointers,
 * [nband][npw] complex128 (precision FS_FP64) or complex64 (FS_MIXED); they
 * must not overlap.  The local term runs through the fused column/plane FFT
 * kernels, the nonlocal term through the projector contractions. */
fs_status fs_apply_H(fs_ctx* ctx, const void* psi, void* hpsi, int nband,
                     double shift, int precision);

/* hpsi = (H - shift) psi in FP64, like fs_apply_H with precision FS_FP64, but
 * without allocating device memory during the call: every intermediate (column
 * buffer, projections, partial sums) lives in one 64 MiB array the library
 * declares at file scope on the device, so callers that cannot call cudaMalloc
 * at that point (a restricted allocator, a fully pre-planned memory budget) can
 * still apply H.  The paper has no counterpart of this call.
 *   - psi, hpsi: DEVICE pointers, [nband][npw] complex128, not overlapping.
 *   - Bands are processed in chunks sized to the array; if a single band
 *     needs more than 64 MiB of scratch the call returns FS_ERR_ARG and says
 *     how much it needed (fs_last_error).
 *   - The array is shared by every context and every call on a device and
 *     keeps the last call's contents; each call overwrites what it reads, so
 *     nothing needs clearing, but calls that overlap on the GPU (two streams,
 *     two threads) race on it: serialise them.
 *   - The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress; the context's device (the one current at
 *     fs_create) must be the current device, else FS_ERR_ARG.  Each GPU that
 *     loads the library holds the 64 MiB until the process exits.
 *   - The call ends by synchronising the context's stream, so it must not be
 *     made while that stream is being captured into a CUDA graph.
 *   - The context itself (fs_create) still allocates; create it beforehand. */
fs_status fs_apply_H_static(fs_ctx* ctx, const void* psi, void* hpsi, int nband, double shift);

/* Supply the start block used by the next fs_solve: n bands, [n][npw]
 * complex128, host or device (where = FS_HOST / FS_DEVICE).  damp = 1 scales
 * each coefficient by 1/(1 + |q|^2/2) before use (raw random draws); damp = 0
 * takes them as they are (warm start, e.g. from fs_get_states).  Bands beyond
 * n are drawn from the seeded generator. */
fs_status fs_set_initial_states(fs_ctx* ctx, const void* psi, int n, int damp, int where);

/* Solve for the nstates eigenpairs nearest e_ref to residual tol (Ha).
 * res->eps and res->resid must hold nstates doubles.  Returns
 * FS_ERR_NOT_CONVERGED (results filled) when the cap is reached;
 * FS_ERR_NUMERIC when the block or its H image is not finite (a non-finite
 * start block is caught before any dense eigensolve) or the basis selection
 * fails; FS_ERR_TIMEOUT when a bounded device wait gave up.  The context
 * stays usable after any of these. */
fs_status fs_solve(fs_ctx* ctx, double e_ref, int nstates, double tol, fs_result* res);

/* The nstates lowest eigenpairs of H to residual tol (Ha): the all-band
 * conjugate-gradient minimisation of the ground-state codes the paper builds
 * on (Sec. II.A-B, PEtot and LS3DF), in the same locally optimal block form as
 * fs_solve but on H itself (Rayleigh quotients <s_i, H s_j>, residual
 * H x - theta x, one H application per band per iteration, preconditioner
 * 1 / (1 + |q|^2/2)), with the same precision ladder (opts.precision) and
 * guard bands.  Results ordered by eigenvalue; fs_get_states returns the
 * states.  Return codes as fs_solve. */
fs_status fs_solve_lowest(fs_ctx* ctx, int nstates, double tol, fs_result* res);

/* Copy the n first states of the last solve (in the order of res->eps), or of
 * the last fs_chebfd (in the order of its eps), [n][npw] complex128, to host or
 * device memory. */
fs_status fs_get_states(fs_ctx* ctx, void* psi, int n, int where);

/* Per-kernel-class timing.  fs_profile(ctx, 1) resets the counters and
 * starts recording a CUDA event pair on the context's stream around every
 * launch of the library's kernels (and around its small dense FP64 solves);
 * fs_profile(ctx, 0) stops.  fs_kernel_stats copies up to max entries: the
 * class name (static string), launches, summed event time (ms), and the
 * algorithmic bytes and flops of those launches (the minimum traffic the
 * kernel's function implies: each operand read once, each result written
 * once).  FP64 work (the FP64 stage, the FP64 check of an FP32 result, the
 * linear solve, ChebFD) is counted in its own classes, named with "_fp64".
 * *count receives the number of classes. */
typedef struct {
    const char* name;
    long long launches;
    double ms;
    double bytes;
    double flops;
} fs_kernel_stat;

fs_status fs_profile(fs_ctx* ctx, int enable);
fs_status fs_kernel_stats(fs_ctx* ctx, fs_kernel_stat* out, int max, int* count);

/* Learned G-shell preconditioner (precond = FS_PREC_LEARNED).  It scales the
 * paper's G-space diagonal preconditioner M(G) (Sec. II.C) per band and per
 * kinetic-energy shell of the plane waves:  W_G = M(G) exp(z_{i,s(G)}) R_G,
 * z = f(features) with f a 4-128-128-128-1 perceptron (tanh hidden layers,
 * BF16 hidden weights in the forward pass, FP32 arithmetic).  Features of
 * (band i, shell s): shell centre / ecut, log10 of the shell's share of
 * |R_i|^2, d_i / 0.1 Ha with d_i = <x_i,(H-E)x_i>, log10 ||R_i|| / 10.  The
 * untrained network has a zero output layer, i.e. it is exactly M(G).
 * Parameters: 33,793 floats, W1[128][4] b1 W2[128][128] b2 W3[128][128] b3
 * W4[128] b4.
 *
 * fs_precond_train: solves (e_ref, nstates, tol) once with M(G), solves again
 * from the same start recording, for each wanted band still iterating, the
 * residual features and the per-shell log-gain that maps M R onto the
 * correction into the span of the first solve's states (weight: the shell's
 * share of |M R|^2); then takes `epochs` full-batch Adam steps (rate lr) on
 * the weighted squared error and returns the final loss.  Needs a start block
 * (fs_set_initial_states) or the seeded default.  At most 4 Mi rows are kept. */
fs_status fs_precond_train(fs_ctx* ctx, double e_ref, int nstates, double tol, int epochs, float lr, float* loss);
/* rows recorded by the last fs_precond_train */
fs_status fs_precond_rows(fs_ctx* ctx, long long* nrows);
/* get (set = 0) or set (set = 1) the n = 33,793 parameters, host float array */
fs_status fs_precond_weights(fs_ctx* ctx, float* w, int n, int set);
/* z = f(features) for rows of 4 features; DEVICE arrays [rows][4] and [rows] */
fs_status fs_precond_eval(fs_ctx* ctx, const float* features, int rows, float* z);
/* weighted loss sum w (f(x) - t)^2 / sum w (host *loss) and its gradient
 * (DEVICE grad[33,793]) with respect to the parameters; DEVICE inputs */
fs_status fs_precond_loss_grad(fs_ctx* ctx, const float* features, const float* target, const float* weight,
                               int rows, float* loss, float* grad);
/* Features and training labels of given residual rows, by the device steps a
 * recording solve of fs_precond_train takes (for checking them against a
 * reference implementation).  nb residual rows R, their bands X and nref
 * reference states Xref are DEVICE arrays [..][npw], complex128 (precision
 * FS_FP64) or complex64 (FS_MIXED); d is a HOST array [nb] of the distances
 * d_i = <x_i, (H - E) x_i> (Ha).  The correction of band i is
 * e_i = Xref Xref^H x_i - x_i; with it, per (band i, shell s), the label is
 * log max(Re<M R_i, e_i>_s / ||M R_i||_s^2, 1e-3) minus its weighted mean over s
 * and the weight the shell's share of ||M R_i||^2, M = M(G) at e_ref.  Shells:
 * 32 uniform bins of |q|^2/2 over [0, ecut].  Outputs are DEVICE float arrays:
 * F [nb * 32][4] (row i * 32 + s), zt and wt [nb * 32].  X = NULL computes the
 * features only (Xref, zt, wt ignored). */
fs_status fs_precond_features(fs_ctx* ctx, double e_ref, const void* R, const void* X, const void* Xref, int nref,
                              const double* d, int nb, int precision, float* F, float* zt, float* wt);

/* Batched independent boxes (the fragment setting of the paper's LS3DF step,
 * Sec. II.B: many small problems of uneven size solved independently).  A
 * batch groups nbox existing contexts, each on its own stream (contexts must
 * be distinct and must not share a stream), and fs_batch_solve runs their
 * solves concurrently from nthreads host threads (<= 0: 8) so that the
 * boxes' kernels overlap on the GPU.  Box i is solved for e_ref[i] and
 * nstates[i]; res[i].eps / res[i].resid must hold nstates[i] doubles;
 * status[i] receives each box's status.  The contexts stay owned by the
 * caller; fs_batch_destroy releases only the grouping. */
typedef struct fs_batch fs_batch;
fs_status fs_batch_create(int nbox, fs_ctx* const* ctxs, int nthreads, fs_batch** out);
fs_status fs_batch_solve(fs_batch* batch, const double* e_ref, const int* nstates, double tol, fs_result* res,
                         fs_status* status);
void fs_batch_destroy(fs_batch* batch);

/* FFT launch-shape autotuner: times H applications of 32 bands for this
 * context's grid and precision with 2, 4, 8, 16 and 32 z-columns per thread
 * block, then (register-FFT grids) 1 to 4 line items per thread of the plane
 * kernel and band chunks of 16 to 96 MiB of column buffer, keeping the fastest
 * of each in turn (cached per grid shape for the process); *cpb receives the
 * column tile (may be NULL).  With opts.verbose each timing goes to stderr. */
fs_status fs_autotune(fs_ctx* ctx, int* cpb);

/* ---- folded-spectrum linear solve (Sec. II.C, Eq. wl1 and the M' preconditioner) ----
 *
 * For each right-hand side w_l, PCG minimises F = 1/2 <psi|(H - E)^2|psi> - Re<psi|w'>
 * with w' = (H - E) w, i.e. solves (H - E)^2 psi = (H - E) w (Eq. wl1), whose solution
 * solves the scattering-state equation (H - E) psi = w (Eq. wl) where H - E is
 * invertible.  FP64 throughout; Polak-Ribiere directions (clamped at zero).
 * Preconditioner: M(G) = 1/((|q|^2/2 - E)^2 + dE^2) with dE from the options, or,
 * once eigenstates are set, the paper's
 *   M' = M (1 - sum_i |phi_i><phi_i|) + sum_i |phi_i><phi_i| / ((eps_i - E)^2 + Delta_i^2)
 * applied as written.  The error reported is ||(H - E) psi - w|| per right-hand side,
 * recomputed from psi on return. */
typedef struct {
    int iters;                 /* PCG iterations taken (all right-hand sides step together) */
    long long n_hpsi;          /* band applications of H */
    double seconds;            /* wall time of the call */
    double* err;               /* caller-allocated [nrhs], or NULL: ||(H - E) psi_l - w_l|| */
} fs_linres;

/* Eigenstates for M'.  n = 0 clears them (M alone).  phi = NULL takes the first n
 * states of the context's last fs_solve with their eigenvalues and residuals
 * (n <= nstates of that solve; eps and delta are ignored).  Otherwise phi holds n
 * states [n][npw] complex128 (host or device per `where`, copied), eps[n] their
 * eigenvalues (Ha) and delta[n] their residuals ||H phi - eps phi|| (host arrays).
 * The states are used as given (orthonormal states are what the formula assumes). */
fs_status fs_set_linear_states(fs_ctx* ctx, const void* phi, const double* eps, const double* delta, int n,
                               int where);

/* Solve for nrhs right-hand sides.  w and psi are [nrhs][npw] complex128, both on the
 * host or both on the device (`where`), caller-owned; psi receives the solution and,
 * when from_psi != 0, also holds the start guess on entry (else the start is 0).
 * tol > 0 is the target of ||(H - E) psi - w||; maxit caps the iterations.
 * FS_ERR_NOT_CONVERGED when some right-hand side missed tol (psi and res filled);
 * nrhs = 0 is a no-op. */
fs_status fs_linear_solve(fs_ctx* ctx, double e_ref, const void* w, void* psi, int nrhs, int where, int from_psi,
                          double tol, int maxit, fs_linres* res);

/* ---- Chebyshev filter diagonalisation (Sec. II.C, the ChebFD producer of the states near E) ----
 *
 * A block of nvec seeded random vectors is filtered by p(Hs) = sum_n g_n mu_n T_n(Hs),
 * Hs = (H - c)/e mapping [emin, emax] to [-1, 1], mu_n the Chebyshev coefficients of the
 * indicator of the window [E - half_width, E + half_width] and g_n the Jackson damping
 * for the given degree (T_n by the three-term recurrence, one H application per degree),
 * then a Rayleigh-Ritz step of H on the filtered block gives the block of the next step;
 * `steps` steps in all, FP64.  [emin, emax] must contain the spectrum of H
 * (fs_spectral_bounds gives an estimate).  The pairs inside the window, ordered by
 * (|eps - E|, eps), at most nwant of them, become the context's result: their states
 * are read with fs_get_states and serve fs_set_linear_states(phi = NULL).  Pairs with a
 * large residual ("ghost states") can appear; their residuals say so. */
typedef struct {
    int nfound;                /* pairs reported (inside the window, at most nwant) */
    long long n_hpsi;          /* band applications of H */
    double seconds;            /* wall time of the call */
    double* eps;               /* caller-allocated [nwant]: eigenvalues, Ha */
    double* resid;             /* caller-allocated [nwant]: ||H phi - eps phi|| */
} fs_chebfd_result;

fs_status fs_chebfd(fs_ctx* ctx, double e_ref, double half_width, double emin, double emax, int degree, int nvec,
                    int steps, unsigned long long seed, int nwant, fs_chebfd_result* res);

/* Estimated spectral bounds of H: iters (>= 2) Lanczos steps on one seeded vector; the
 * extreme eigenvalues of the tridiagonal matrix widened by the norm of the last
 * residual vector. */
fs_status fs_spectral_bounds(fs_ctx* ctx, int iters, double* emin, double* emax);

/* Wave-function interpolation between two k-points (Sec. II.D): from orthonormal
 * eigenpairs of k1 (n1 states) and k2 (n2 >= n1 states), H(k) = alpha H(k1) +
 * (1 - alpha) H(k2) in the basis psi_i(k1) is
 *     H_ij = alpha eps1_i delta_ij + (1 - alpha) sum_m U*_im U_jm eps2_m,
 * U the rows of S_il = <psi_l(k2)|psi_i(k1)> made orthonormal by Gram-Schmidt in
 * index order (U = L^-1 S, S S^H = L L^H); its eigenvalues (ascending) go to eps
 * (host [n1]) and the states psi_q = alpha sum_j C_jq psi_j(k1) + (1 - alpha)
 * sum_{j,l} C_jq U_jl psi_l(k2) to psi.  psi1 [n1][npw], psi2 [n2][npw] and psi
 * [n1][npw] are DEVICE arrays of complex128 on one common set of npw plane waves
 * (the context's sphere: periodic parts of the states of both k-points); eps1,
 * eps2 are host arrays.  FS_ERR_NUMERIC when S has dependent rows. */
fs_status fs_kinterp(fs_ctx* ctx, double alpha, int n1, const double* eps1, const void* psi1, int n2,
                     const double* eps2, const void* psi2, double* eps, void* psi);

/* The library's dense FP64 eigensolver (the one its Rayleigh-Ritz steps use): the m
 * lowest eigenpairs of the Hermitian A (B = NULL) or of the generalized problem
 * A x = lambda B x with B Hermitian positive definite (Cholesky reduction).  A and B
 * are HOST arrays, n x n complex128, column-major (1 <= n <= 2048); w receives the m
 * eigenvalues in ascending order, Z the eigenvectors (n x m, column-major;
 * orthonormal, or B-orthonormal).  FS_ERR_NUMERIC when B is not positive definite.
 * Method: Householder reduction to a real tridiagonal matrix, bisection on Sturm
 * counts, inverse iteration with Gram-Schmidt inside eigenvalue clusters,
 * back-transformation; Cholesky and triangular solves for B.  (Sec. II.C: the
 * subspace diagonalisation of the eigensolvers.) */
fs_status fs_dense_eigh(fs_ctx* ctx, int n, const void* A, const void* B, int m, double* w, void* Z);

/* Failure-path check without a GPU fault: runs the library's bounded device wait (the one
 * the tensor-core pipelines use) on a barrier that nothing completes, polling `polls`
 * times (1 .. 2^24); the wait gives up, raises the context's error flag, and the call
 * returns FS_ERR_TIMEOUT as a pipeline timeout would.  The context stays usable. */
fs_status fs_wait_selftest(fs_ctx* ctx, long long polls);

/* Release everything the context holds.  NULL is accepted. */
void fs_destroy(fs_ctx* ctx);

/* Message of the last failure on ctx ("" when none); static text when ctx is NULL. */
const char* fs_last_error(const fs_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* FS_H */
