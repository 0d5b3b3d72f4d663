"""GB300 folded-spectrum eigensolver: Python binding of the C ABI in include/fs.h.

This module only marshals arguments: every step of H application and of the
solve runs in the CUDA library ``libfs_gb300.so`` built in-tree by
``paper_1907_06821_gb300.build``.  PyTorch is used only to hold device
memory.  There is no CPU fallback: if the library is missing the import of
the binding fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfs_gb300.so")

FS_OK, FS_ERR_ARG, FS_ERR_GRID_TOO_SMALL, FS_ERR_OOM, FS_ERR_CUDA, FS_ERR_NUMERIC, \
    FS_ERR_NOT_CONVERGED, FS_ERR_TIMEOUT, FS_ERR_UNIMPLEMENTED = range(9)
FS_FP64, FS_MIXED = 0, 1
FS_PREC_M, FS_PREC_TETER, FS_PREC_LEARNED = 0, 1, 2
FS_HOST, FS_DEVICE = 0, 1
FS_GEMM_TENSOR, FS_GEMM_CUDA_CORES = 0, 1
FS_PROJ_AUTO, FS_PROJ_STORED, FS_PROJ_GENERATED = 0, 1, 2

STATUS_NAMES = {0: "FS_OK", 1: "FS_ERR_ARG", 2: "FS_ERR_GRID_TOO_SMALL", 3: "FS_ERR_OOM",
                4: "FS_ERR_CUDA", 5: "FS_ERR_NUMERIC", 6: "FS_ERR_NOT_CONVERGED",
                7: "FS_ERR_TIMEOUT", 8: "FS_ERR_UNIMPLEMENTED"}


class fs_grid(C.Structure):
    _fields_ = [("L", C.c_double * 3), ("n", C.c_int * 3)]


class fs_projectors(C.Structure):
    _fields_ = [("natom", C.c_int), ("nproj", C.c_int), ("pos", C.POINTER(C.c_double)),
                ("l", C.POINTER(C.c_int)), ("axis", C.POINTER(C.c_int)),
                ("width", C.POINTER(C.c_double)), ("D", C.POINTER(C.c_double))]


class fs_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("precond", C.c_int), ("dE", C.c_double),
                ("maxit", C.c_int), ("guard", C.c_int), ("seed", C.c_ulonglong),
                ("cuda_stream", C.c_void_p), ("verbose", C.c_int), ("gemm_path", C.c_int),
                ("projectors", C.c_int)]


class fs_result(C.Structure):
    _fields_ = [("nconv", C.c_int), ("iters", C.c_int), ("n_hpsi", C.c_longlong),
                ("eps", C.POINTER(C.c_double)), ("resid", C.POINTER(C.c_double)),
                ("seconds", C.c_double), ("iters_mixed", C.c_int)]


class fs_linres(C.Structure):
    _fields_ = [("iters", C.c_int), ("n_hpsi", C.c_longlong), ("seconds", C.c_double),
                ("err", C.POINTER(C.c_double))]


class fs_chebfd_result(C.Structure):
    _fields_ = [("nfound", C.c_int), ("n_hpsi", C.c_longlong), ("seconds", C.c_double),
                ("eps", C.POINTER(C.c_double)), ("resid", C.POINTER(C.c_double))]


class fs_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_longlong), ("ms", C.c_double),
                ("bytes", C.c_double), ("flops", C.c_double)]


class FSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1907_06821_gb300.build.build()")
    lib = C.CDLL(path)
    vp, ip, dp = C.c_void_p, C.c_int, C.c_double
    lib.fs_create.argtypes = [C.POINTER(fs_grid), dp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                              C.POINTER(fs_projectors), C.POINTER(fs_options), C.POINTER(vp)]
    lib.fs_create.restype = ip
    lib.fs_npw.argtypes = [vp, C.POINTER(C.c_int)]
    lib.fs_npw.restype = ip
    lib.fs_gvectors.argtypes = [vp, C.POINTER(C.c_int)]
    lib.fs_gvectors.restype = ip
    lib.fs_apply_H.argtypes = [vp, vp, vp, ip, dp, ip]
    lib.fs_apply_H.restype = ip
    lib.fs_set_initial_states.argtypes = [vp, vp, ip, ip, ip]
    lib.fs_set_initial_states.restype = ip
    lib.fs_solve.argtypes = [vp, dp, ip, dp, C.POINTER(fs_result)]
    lib.fs_solve.restype = ip
    lib.fs_solve_lowest.argtypes = [vp, ip, dp, C.POINTER(fs_result)]
    lib.fs_solve_lowest.restype = ip
    lib.fs_get_states.argtypes = [vp, vp, ip, ip]
    lib.fs_get_states.restype = ip
    lib.fs_apply_H_static.argtypes = [vp, vp, vp, ip, dp]
    lib.fs_apply_H_static.restype = ip
    lib.fs_precond_train.argtypes = [vp, dp, ip, dp, ip, C.c_float, C.POINTER(C.c_float)]
    lib.fs_precond_train.restype = ip
    lib.fs_precond_rows.argtypes = [vp, C.POINTER(C.c_longlong)]
    lib.fs_precond_rows.restype = ip
    lib.fs_precond_weights.argtypes = [vp, C.POINTER(C.c_float), ip, ip]
    lib.fs_precond_weights.restype = ip
    lib.fs_precond_eval.argtypes = [vp, vp, ip, vp]
    lib.fs_precond_eval.restype = ip
    lib.fs_precond_loss_grad.argtypes = [vp, vp, vp, vp, ip, C.POINTER(C.c_float), vp]
    lib.fs_precond_loss_grad.restype = ip
    lib.fs_precond_features.argtypes = [vp, dp, vp, vp, vp, ip, C.POINTER(C.c_double), ip, ip, vp, vp, vp]
    lib.fs_precond_features.restype = ip
    lib.fs_batch_create.argtypes = [ip, C.POINTER(vp), ip, C.POINTER(vp)]
    lib.fs_batch_create.restype = ip
    lib.fs_batch_solve.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int), dp, vp, C.POINTER(C.c_int)]
    lib.fs_batch_solve.restype = ip
    lib.fs_batch_destroy.argtypes = [vp]
    lib.fs_batch_destroy.restype = None
    lib.fs_set_linear_states.argtypes = [vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_double), ip, ip]
    lib.fs_set_linear_states.restype = ip
    lib.fs_linear_solve.argtypes = [vp, C.c_double, vp, vp, ip, ip, ip, C.c_double, ip, C.POINTER(fs_linres)]
    lib.fs_linear_solve.restype = ip
    lib.fs_chebfd.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double, ip, ip, ip, C.c_ulonglong, ip,
                              C.POINTER(fs_chebfd_result)]
    lib.fs_chebfd.restype = ip
    lib.fs_spectral_bounds.argtypes = [vp, ip, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.fs_spectral_bounds.restype = ip
    lib.fs_kinterp.argtypes = [vp, dp, ip, C.POINTER(C.c_double), vp, ip, C.POINTER(C.c_double), vp,
                               C.POINTER(C.c_double), vp]
    lib.fs_kinterp.restype = ip
    lib.fs_dense_eigh.argtypes = [vp, ip, vp, vp, ip, C.POINTER(C.c_double), vp]
    lib.fs_dense_eigh.restype = ip
    lib.fs_wait_selftest.argtypes = [vp, C.c_longlong]
    lib.fs_wait_selftest.restype = ip
    lib.fs_autotune.argtypes = [vp, C.POINTER(C.c_int)]
    lib.fs_autotune.restype = ip
    lib.fs_profile.argtypes = [vp, ip]
    lib.fs_profile.restype = ip
    lib.fs_kernel_stats.argtypes = [vp, C.POINTER(fs_kernel_stat), ip, C.POINTER(C.c_int)]
    lib.fs_kernel_stats.restype = ip
    lib.fs_destroy.argtypes = [vp]
    lib.fs_destroy.restype = None
    lib.fs_last_error.argtypes = [vp]
    lib.fs_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _torch_c128():
    import torch
    return torch.complex128


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


class Context:
    """One fs_ctx: a Hamiltonian on one plane-wave sphere.

    Arguments mirror fs_create: cell ``L`` (bohr), grid ``n``, cutoff ``ecut``
    (Ha), ``k`` (1/bohr), ``vloc`` [n0][n1][n2] (Ha), projector set
    (``pos`` [natom][3], ``proj`` [(l, axis, width)], ``D`` [natom][np][np]).
    """

    def __init__(self, L, n, ecut, k, vloc, pos=None, proj=(), D=None, precision=FS_FP64,
                 precond=FS_PREC_M, dE=0.5, maxit=5000, guard=-1, seed=1, stream=None, verbose=0,
                 gemm_path=FS_GEMM_TENSOR, projectors=0):
        self.lib = load_library()
        self._keep = []
        g = fs_grid((C.c_double * 3)(*[float(x) for x in L]), (C.c_int * 3)(*[int(x) for x in n]))
        kk = np.ascontiguousarray(k, dtype=np.float64)
        v = np.ascontiguousarray(vloc, dtype=np.float64)
        if v.shape != tuple(int(x) for x in n):
            raise ValueError("vloc shape does not match the grid")
        pr = fs_projectors()
        proj = list(proj)
        if pos is not None and len(proj) > 0 and len(pos) > 0:
            posa = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
            la = np.ascontiguousarray([p[0] for p in proj], dtype=np.int32)
            axa = np.ascontiguousarray([p[1] for p in proj], dtype=np.int32)
            wa = np.ascontiguousarray([p[2] for p in proj], dtype=np.float64)
            Da = np.ascontiguousarray(D, dtype=np.float64).reshape(posa.shape[0], len(proj), len(proj))
            self._keep += [posa, la, axa, wa, Da]
            pr.natom, pr.nproj = posa.shape[0], len(proj)
            pr.pos, pr.l, pr.axis, pr.width, pr.D = _dptr(posa), _iptr(la), _iptr(axa), _dptr(wa), _dptr(Da)
        opt = fs_options(precision, precond, dE, maxit, guard, seed,
                         C.c_void_p(stream) if stream else None, verbose, gemm_path, projectors)
        self.precision = precision
        h = C.c_void_p()
        st = self.lib.fs_create(C.byref(g), float(ecut), _dptr(kk), _dptr(v), C.byref(pr), C.byref(opt),
                                C.byref(h))
        if st != FS_OK:
            raise FSError(st, "fs_create failed")
        self.h = h

    @classmethod
    def from_workload(cls, w, **kw):
        """Build from an fs_inputs.Workload."""
        return cls(w.L, w.n, w.ecut, w.k, w.vloc, pos=w.pos, proj=w.proj, D=w.D, **kw)

    def _check(self, st, what):
        if st != FS_OK:
            msg = self.lib.fs_last_error(self.h)
            raise FSError(st, f"{what}: {msg.decode() if msg else ''}")

    @property
    def npw(self):
        v = C.c_int()
        self._check(self.lib.fs_npw(self.h, C.byref(v)), "fs_npw")
        return v.value

    def gvectors(self):
        out = np.empty((self.npw, 3), dtype=np.int32)
        self._check(self.lib.fs_gvectors(self.h, _iptr(out)), "fs_gvectors")
        return out

    def apply_H(self, psi, out=None, shift=0.0, precision=None):
        """(H - shift) psi for a device tensor psi [nband][npw] (complex128 or complex64)."""
        import torch
        prec = FS_FP64 if psi.dtype == torch.complex128 else FS_MIXED
        if precision is not None and precision != prec:
            raise ValueError("tensor dtype does not match the requested precision")
        if not psi.is_cuda or not psi.is_contiguous() or psi.dim() != 2 or psi.shape[1] != self.npw:
            raise ValueError("psi must be a contiguous CUDA tensor [nband][npw]")
        if out is None:
            out = torch.empty_like(psi)
        self._check(self.lib.fs_apply_H(self.h, C.c_void_p(psi.data_ptr()), C.c_void_p(out.data_ptr()),
                                        psi.shape[0], float(shift), prec), "fs_apply_H")
        return out

    def apply_H_static(self, psi, out=None, shift=0.0):
        """FP64 (H - shift) psi through fs_apply_H_static: no device allocation in
        the library during the call (intermediates live in its static scratch)."""
        import torch
        if psi.dtype != torch.complex128 or not psi.is_cuda or not psi.is_contiguous() or psi.dim() != 2:
            raise ValueError("psi must be a contiguous complex128 CUDA tensor [nband][npw]")
        if out is None:
            out = torch.empty_like(psi)
        self._check(self.lib.fs_apply_H_static(self.h, C.c_void_p(psi.data_ptr()), C.c_void_p(out.data_ptr()),
                                               psi.shape[0], float(shift)), "fs_apply_H_static")
        return out

    def set_initial_states(self, psi, damp=True):
        """Start block [n][npw] complex128: a numpy array or CPU tensor (host, e.g. pinned)
        or a CUDA tensor (device)."""
        if isinstance(psi, np.ndarray):
            a = np.ascontiguousarray(psi, dtype=np.complex128)
            self._check(self.lib.fs_set_initial_states(self.h, a.ctypes.data_as(C.c_void_p), a.shape[0],
                                                       int(damp), FS_HOST), "fs_set_initial_states")
        else:
            if psi.dtype != _torch_c128() or not psi.is_contiguous():
                raise ValueError("start block tensor must be contiguous complex128")
            where = FS_DEVICE if psi.is_cuda else FS_HOST
            self._check(self.lib.fs_set_initial_states(self.h, C.c_void_p(psi.data_ptr()), psi.shape[0],
                                                       int(damp), where), "fs_set_initial_states")

    def solve(self, e_ref, nstates, tol=1e-6, allow_unconverged=False):
        eps = np.zeros(nstates)
        res = np.zeros(nstates)
        r = fs_result()
        r.eps = _dptr(eps)
        r.resid = _dptr(res)
        st = self.lib.fs_solve(self.h, float(e_ref), int(nstates), float(tol), C.byref(r))
        if st not in (FS_OK, FS_ERR_NOT_CONVERGED) or (st == FS_ERR_NOT_CONVERGED and not allow_unconverged):
            self._check(st, "fs_solve")
        return dict(eps=eps, resid=res, nconv=r.nconv, iters=r.iters, iters_mixed=r.iters_mixed,
                    n_hpsi=r.n_hpsi, seconds=r.seconds, status=st)

    def solve_lowest(self, nstates, tol=1e-6, allow_unconverged=False):
        """The nstates lowest eigenpairs of H (fs_solve_lowest); eps ascending."""
        eps = np.zeros(nstates)
        res = np.zeros(nstates)
        r = fs_result()
        r.eps = _dptr(eps)
        r.resid = _dptr(res)
        st = self.lib.fs_solve_lowest(self.h, int(nstates), float(tol), C.byref(r))
        if st not in (FS_OK, FS_ERR_NOT_CONVERGED) or (st == FS_ERR_NOT_CONVERGED and not allow_unconverged):
            self._check(st, "fs_solve_lowest")
        return dict(eps=eps, resid=res, nconv=r.nconv, iters=r.iters, iters_mixed=r.iters_mixed,
                    n_hpsi=r.n_hpsi, seconds=r.seconds, status=st)

    def get_states(self, n, device=False, out=None):
        """The n states nearest E [n][npw] complex128: a numpy array, a CUDA tensor
        (device=True), or written into `out` (a contiguous complex128 tensor, host or
        device, e.g. pinned host memory) and returned."""
        if out is not None:
            if out.dtype != _torch_c128() or not out.is_contiguous() or tuple(out.shape) != (n, self.npw):
                raise ValueError("out must be a contiguous complex128 tensor of shape (n, npw)")
            self._check(self.lib.fs_get_states(self.h, C.c_void_p(out.data_ptr()), n,
                                               FS_DEVICE if out.is_cuda else FS_HOST), "fs_get_states")
            return out
        if device:
            import torch
            out = torch.empty((n, self.npw), dtype=torch.complex128, device="cuda")
            self._check(self.lib.fs_get_states(self.h, C.c_void_p(out.data_ptr()), n, FS_DEVICE),
                        "fs_get_states")
            return out
        out = np.empty((n, self.npw), dtype=np.complex128)
        self._check(self.lib.fs_get_states(self.h, out.ctypes.data_as(C.c_void_p), n, FS_HOST),
                    "fs_get_states")
        return out

    # ------------------------------------------------ folded linear solve
    def set_linear_states(self, n, phi=None, eps=None, delta=None):
        """Eigenstates for the M' preconditioner of linear_solve: the first n states of
        the last solve (phi None), or n given states (numpy/CPU tensor or CUDA tensor
        [n][npw] complex128) with eigenvalues eps[n] and residuals delta[n]; n = 0 clears."""
        if phi is None:
            self._check(self.lib.fs_set_linear_states(self.h, None, None, None, int(n), FS_HOST),
                        "fs_set_linear_states")
            return
        e = np.ascontiguousarray(eps, dtype=np.float64)
        d = np.ascontiguousarray(delta, dtype=np.float64)
        if isinstance(phi, np.ndarray):
            a = np.ascontiguousarray(phi, dtype=np.complex128)
            ptr, where = a.ctypes.data_as(C.c_void_p), FS_HOST
        else:
            if phi.dtype != _torch_c128() or not phi.is_contiguous():
                raise ValueError("phi must be a contiguous complex128 tensor")
            ptr, where = C.c_void_p(phi.data_ptr()), (FS_DEVICE if phi.is_cuda else FS_HOST)
        self._check(self.lib.fs_set_linear_states(self.h, ptr, _dptr(e), _dptr(d), int(n), where),
                    "fs_set_linear_states")

    def linear_solve(self, w, e_ref, tol=1e-8, maxit=100000, psi=None, allow_unconverged=False):
        """Solve (H - E)^2 psi = (H - E) w for the rows of w (numpy array: host; CUDA
        tensor: device), starting from psi when given.  Returns (psi, info)."""
        nrhs = int(w.shape[0])
        err = np.zeros(max(nrhs, 1))
        r = fs_linres()
        r.err = _dptr(err)
        if isinstance(w, np.ndarray):
            wa = np.ascontiguousarray(w, dtype=np.complex128)
            out = np.zeros_like(wa) if psi is None else np.ascontiguousarray(psi, dtype=np.complex128).copy()
            st = self.lib.fs_linear_solve(self.h, float(e_ref), wa.ctypes.data_as(C.c_void_p),
                                          out.ctypes.data_as(C.c_void_p), nrhs, FS_HOST, int(psi is not None),
                                          float(tol), int(maxit), C.byref(r))
        else:
            import torch
            out = torch.zeros_like(w) if psi is None else psi.clone()
            st = self.lib.fs_linear_solve(self.h, float(e_ref), C.c_void_p(w.data_ptr()), C.c_void_p(out.data_ptr()),
                                          nrhs, FS_DEVICE, int(psi is not None), float(tol), int(maxit),
                                          C.byref(r))
        if st not in (FS_OK, FS_ERR_NOT_CONVERGED) or (st == FS_ERR_NOT_CONVERGED and not allow_unconverged):
            self._check(st, "fs_linear_solve")
        return out, dict(iters=r.iters, n_hpsi=r.n_hpsi, seconds=r.seconds, err=err[:nrhs].copy(), status=st)

    def kinterp(self, alpha, eps1, psi1, eps2, psi2):
        """Interpolated eigenpairs at alpha (fs_kinterp); psi1 [n1][npw], psi2 [n2][npw] CUDA
        complex128 tensors, eps1/eps2 host arrays.  Returns (eps [n1], psi CUDA [n1][npw])."""
        import torch
        n1, n2 = psi1.shape[0], psi2.shape[0]
        e1 = np.ascontiguousarray(eps1, dtype=np.float64)
        e2 = np.ascontiguousarray(eps2, dtype=np.float64)
        eps = np.empty(n1)
        out = torch.empty((n1, self.npw), dtype=torch.complex128, device=psi1.device)
        self._check(self.lib.fs_kinterp(self.h, float(alpha), n1, _dptr(e1), C.c_void_p(psi1.data_ptr()), n2,
                                        _dptr(e2), C.c_void_p(psi2.data_ptr()), _dptr(eps),
                                        C.c_void_p(out.data_ptr())), "fs_kinterp")
        return eps, out

    def dense_eigh(self, A, m=None, B=None):
        """The m lowest eigenpairs of the Hermitian A (or of A x = lambda B x) by the library's
        dense FP64 eigensolver; A, B host complex arrays (n x n).  Returns (w, Z [n x m])."""
        A = np.asfortranarray(A, dtype=np.complex128)
        n = A.shape[0]
        m = n if m is None else int(m)
        Bf = None if B is None else np.asfortranarray(B, dtype=np.complex128)
        w = np.empty(m, dtype=np.float64)
        Z = np.empty((n, m), dtype=np.complex128, order="F")
        self._check(self.lib.fs_dense_eigh(self.h, n, A.ctypes.data, None if Bf is None else Bf.ctypes.data, m,
                                           _dptr(w), Z.ctypes.data), "fs_dense_eigh")
        return w, Z

    def wait_selftest(self, polls=4096):
        """Run the bounded device wait on a barrier nothing completes; raises FSError
        with FS_ERR_TIMEOUT (the failure path of the tensor-core pipelines)."""
        self._check(self.lib.fs_wait_selftest(self.h, int(polls)), "fs_wait_selftest")

    # ------------------------------------------------ ChebFD
    def spectral_bounds(self, iters=40):
        """(emin, emax) estimated by Lanczos steps widened by the last residual norm."""
        lo, hi = C.c_double(), C.c_double()
        self._check(self.lib.fs_spectral_bounds(self.h, int(iters), C.byref(lo), C.byref(hi)), "fs_spectral_bounds")
        return lo.value, hi.value

    def chebfd(self, e_ref, half_width, emin, emax, degree, nvec, steps, seed=1, nwant=None):
        """Chebyshev filter diagonalisation; returns dict(eps, resid, nfound, n_hpsi, seconds)
        for the pairs inside the window (states via get_states)."""
        nwant = nvec if nwant is None else int(nwant)
        eps = np.zeros(max(nwant, 1))
        res = np.zeros(max(nwant, 1))
        r = fs_chebfd_result()
        r.eps = _dptr(eps)
        r.resid = _dptr(res)
        self._check(self.lib.fs_chebfd(self.h, float(e_ref), float(half_width), float(emin), float(emax), int(degree),
                                       int(nvec), int(steps), int(seed), nwant, C.byref(r)), "fs_chebfd")
        n = r.nfound
        return dict(eps=eps[:n].copy(), resid=res[:n].copy(), nfound=n, n_hpsi=r.n_hpsi, seconds=r.seconds)

    # ------------------------------------------------ learned preconditioner
    N_PRECOND_PARAMS = 33793
    N_SHELL = 32

    def precond_train(self, e_ref, nstates, tol=1e-6, epochs=200, lr=1e-3):
        """Train the learned G-shell preconditioner from this context's own solves; returns the loss."""
        loss = C.c_float()
        self._check(self.lib.fs_precond_train(self.h, float(e_ref), int(nstates), float(tol), int(epochs),
                                              C.c_float(lr), C.byref(loss)), "fs_precond_train")
        n = C.c_longlong()
        self._check(self.lib.fs_precond_rows(self.h, C.byref(n)), "fs_precond_rows")
        return float(loss.value), int(n.value)

    def precond_weights(self, w=None):
        """Return the parameters (w None) or set them from a float array."""
        if w is None:
            out = np.empty(self.N_PRECOND_PARAMS, dtype=np.float32)
            self._check(self.lib.fs_precond_weights(self.h, out.ctypes.data_as(C.POINTER(C.c_float)), out.size, 0),
                        "fs_precond_weights")
            return out
        a = np.ascontiguousarray(w, dtype=np.float32)
        self._check(self.lib.fs_precond_weights(self.h, a.ctypes.data_as(C.POINTER(C.c_float)), a.size, 1),
                    "fs_precond_weights")

    def precond_eval(self, features):
        """z = f(features) for a CUDA float32 tensor [rows][4]."""
        import torch
        z = torch.empty(features.shape[0], dtype=torch.float32, device=features.device)
        self._check(self.lib.fs_precond_eval(self.h, C.c_void_p(features.data_ptr()), features.shape[0],
                                             C.c_void_p(z.data_ptr())), "fs_precond_eval")
        return z

    def precond_loss_grad(self, features, target, weight):
        import torch
        g = torch.empty(self.N_PRECOND_PARAMS, dtype=torch.float32, device=features.device)
        loss = C.c_float()
        self._check(self.lib.fs_precond_loss_grad(self.h, C.c_void_p(features.data_ptr()),
                                                  C.c_void_p(target.data_ptr()), C.c_void_p(weight.data_ptr()),
                                                  features.shape[0], C.byref(loss), C.c_void_p(g.data_ptr())),
                    "fs_precond_loss_grad")
        return float(loss.value), g

    def precond_features(self, e_ref, R, d, X=None, Xref=None):
        """Features [nb*32][4] (and labels, weights [nb*32] when X and Xref are given) of the
        residual rows R (CUDA complex128 or complex64 tensors [nb][npw]; d: host distances)."""
        import torch
        nb = R.shape[0]
        prec = FS_FP64 if R.dtype == torch.complex128 else FS_MIXED
        F = torch.empty((nb * self.N_SHELL, 4), dtype=torch.float32, device=R.device)
        zt = torch.empty(nb * self.N_SHELL, dtype=torch.float32, device=R.device)
        wt = torch.empty(nb * self.N_SHELL, dtype=torch.float32, device=R.device)
        dd = np.ascontiguousarray(d, dtype=np.float64)
        lab = X is not None
        self._check(self.lib.fs_precond_features(
            self.h, float(e_ref), C.c_void_p(R.data_ptr()), C.c_void_p(X.data_ptr() if lab else None),
            C.c_void_p(Xref.data_ptr() if lab else None), Xref.shape[0] if lab else 0, _dptr(dd), nb, prec,
            C.c_void_p(F.data_ptr()), C.c_void_p(zt.data_ptr()), C.c_void_p(wt.data_ptr())),
            "fs_precond_features")
        return (F, zt, wt) if lab else F

    def autotune(self):
        """Pick the FFT column tile for this grid by timing; returns columns per block."""
        v = C.c_int()
        self._check(self.lib.fs_autotune(self.h, C.byref(v)), "fs_autotune")
        return v.value

    def profile(self, enable=True):
        """Reset and start (or stop) per-kernel-class event timing."""
        self._check(self.lib.fs_profile(self.h, int(enable)), "fs_profile")

    def kernel_stats(self):
        """{class: dict(launches, ms, bytes, flops)} since the last profile(True)."""
        arr = (fs_kernel_stat * 32)()
        n = C.c_int()
        self._check(self.lib.fs_kernel_stats(self.h, arr, 32, C.byref(n)), "fs_kernel_stats")
        return {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].ms, bytes=arr[i].bytes,
                                           flops=arr[i].flops) for i in range(n.value)}

    def close(self):
        if getattr(self, "h", None):
            self.lib.fs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Independent boxes solved concurrently (fs_batch_*); the contexts stay owned by the caller."""

    def __init__(self, contexts, nthreads=8):
        self.lib = load_library()
        self.contexts = list(contexts)
        arr = (C.c_void_p * len(self.contexts))(*[c.h.value for c in self.contexts])
        h = C.c_void_p()
        st = self.lib.fs_batch_create(len(self.contexts), arr, int(nthreads), C.byref(h))
        if st != FS_OK:
            raise FSError(st, "fs_batch_create failed")
        self.h = h

    def solve(self, e_refs, nstates, tol=1e-6):
        n = len(self.contexts)
        eps = [np.zeros(k) for k in nstates]
        res = [np.zeros(k) for k in nstates]
        results = (fs_result * n)()
        for i in range(n):
            results[i].eps = _dptr(eps[i])
            results[i].resid = _dptr(res[i])
        e = np.ascontiguousarray(e_refs, dtype=np.float64)
        ns = np.ascontiguousarray(nstates, dtype=np.int32)
        status = (C.c_int * n)()
        self.lib.fs_batch_solve(self.h, _dptr(e), _iptr(ns), float(tol), C.cast(results, C.c_void_p), status)
        out = []
        for i in range(n):
            r = results[i]
            out.append(dict(eps=eps[i], resid=res[i], nconv=r.nconv, iters=r.iters, n_hpsi=r.n_hpsi,
                            seconds=r.seconds, status=status[i]))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.fs_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
