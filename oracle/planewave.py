"""CPU FP64 oracle: the plane-wave Kohn-Sham Hamiltonian of the folded-spectrum path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this module; only tests, the package's smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA library.

The paper (Sec. II) uses a Kohn-Sham Hamiltonian in a plane-wave basis with a
local potential and norm-conserving (separable) nonlocal projectors; its
scattering-state equation (Eq. wl) and the folded operator (Eq. wl1) are
built from that H.  The synthetic H here is, in Hartree atomic units:

  basis   S = { q = k + G : |q|^2 / 2 <= ecut },  G = 2 pi (g0/L0, g1/L1, g2/L2)
  kinetic T[G,G]  = |q|^2 / 2
  local   Hloc[G,G'] = Vt((g - g') mod n),  Vt(h) = N^-1 sum_j V(r_j) exp(-2 pi i h.j / n)
          (the grid-aliased convolution, which an FFT on this grid realises exactly)
  nonlocal H_NL = sum_a sum_ij |beta_ai> D^a_ij <beta_aj|, with the analytic
          Fourier transforms of normalised real-space Gaussians:
            s : beta(q) = Omega^-1/2 N_s (2 pi w^2)^{3/2} exp(-w^2 |q|^2 / 2) exp(-i q.R)
            p_x: beta(q) = beta_s(q) * (sqrt(2)/w) * (-i w^2 q_x)
          N_s = (pi w^2)^{-3/4}.

Sphere order (also the CUDA library's): z-columns sorted by (g0, g1)
ascending, each column g2 ascending, with g in [-h, h] on every axis.
"""
from __future__ import annotations

import numpy as np

PARITY_PINS = """
sphere      : brute-force count (pure loop) and the count 1069 for the tiny cell
kinetic     : V = 0, no projectors -> eigenvalues |q|^2/2 with multiplicities
local       : constant V shifts every eigenvalue; cosine V couples G +- G0 by V0;
              Vt vs the analytic Gaussian transform
nonlocal    : projector norm -> 1 at large cutoff (Parseval); numerical FT of the
              real-space Gaussians; one projector -> secular equation roots
full H      : Hermitian; matrix-free apply == dense apply; spectrum invariant
              under a grid translation of wells and atoms together
chunked     : the nonlocal term applied atom chunk by atom chunk equals the stored-table apply
"""


class GridTooSmall(ValueError):
    pass


def sphere(L, n, ecut, k):
    """Miller indices (N,3) int64 and q = k + G (N,3) of the plane waves with
    |q|^2/2 <= ecut, in z-column order.  Raises GridTooSmall when some axis
    needs more than n_d distinct indices (2 h_d + 1 > n_d)."""
    L = np.asarray(L, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    b = 2.0 * np.pi / L
    qmax = np.sqrt(2.0 * ecut)
    hmax = [int(np.floor((qmax + abs(k[d])) / b[d])) + 1 for d in range(3)]
    rng = [np.arange(-hmax[d], hmax[d] + 1) for d in range(3)]
    g0, g1, g2 = np.meshgrid(*rng, indexing="ij")
    g = np.stack([g0.ravel(), g1.ravel(), g2.ravel()], axis=1)
    q = k[None, :] + g * b[None, :]
    keep = 0.5 * np.sum(q * q, axis=1) <= ecut
    g = g[keep]
    # z-column order: sort by (g0, g1, g2)
    order = np.lexsort((g[:, 2], g[:, 1], g[:, 0]))
    g = g[order]
    for d in range(3):
        span = int(g[:, d].max() - g[:, d].min() + 1) if g.shape[0] else 0
        if span > int(n[d]):
            raise GridTooSmall(f"axis {d}: sphere spans {span} > grid {n[d]}")
    q = k[None, :] + g * b[None, :]
    return g.astype(np.int64), q


def kinetic(q):
    return 0.5 * np.sum(q * q, axis=1)


def vtilde(vloc):
    """Vt(h) = N^-1 sum_j V(r_j) exp(-2 pi i h.j/n), indexed by h mod n."""
    return np.fft.fftn(vloc) / vloc.size


def beta_matrix(w, g, q, atoms=None):
    """B[G, a*nproj + c] = beta_{a,c}(q_G) (complex128, (N, natom*nproj)); with
    `atoms`, only the columns of those atoms (in that order)."""
    L = w.L
    omega = float(np.prod(L))
    q2 = np.sum(q * q, axis=1)
    # the factor of each projector type without the atom's phase
    shapes = []
    for (l, ax, wid) in w.proj:
        ns = (np.pi * wid * wid) ** (-0.75)
        radial = omega ** -0.5 * ns * (2.0 * np.pi * wid * wid) ** 1.5 \
            * np.exp(-0.5 * wid * wid * q2)
        if l == 0:
            f = radial.astype(np.complex128)
        elif l == 1:
            f = radial * (np.sqrt(2.0) / wid) * (-1j * wid * wid * q[:, ax])
        else:
            raise ValueError("only s and p projectors")
        shapes.append(f)
    cols = []
    for a in (range(w.natom) if atoms is None else atoms):
        phase = np.exp(-1j * (q @ w.pos[a]))
        for f in shapes:
            cols.append(f * phase)
    if not cols:
        return np.zeros((q.shape[0], 0), dtype=np.complex128)
    return np.stack(cols, axis=1)


def _at_origin(w):
    """The workload with one atom at the origin (its projectors without a phase)."""
    import copy
    w0 = copy.copy(w)
    w0.pos = np.zeros((1, 3))
    return w0


def block_D(w):
    """Block-diagonal D over (atom, projector) as a dense matrix."""
    npj = w.nproj
    Dfull = np.zeros((w.natom * npj, w.natom * npj), dtype=np.complex128)
    for a in range(w.natom):
        Dfull[a * npj:(a + 1) * npj, a * npj:(a + 1) * npj] = w.D[a]
    return Dfull


def dense_H(w, include=("T", "V", "NL")):
    """The Hamiltonian as an explicit dense Hermitian matrix on the sphere."""
    g, q = sphere(w.L, w.n, w.ecut, w.k)
    N = g.shape[0]
    H = np.zeros((N, N), dtype=np.complex128)
    if "T" in include:
        H[np.arange(N), np.arange(N)] += kinetic(q)
    if "V" in include:
        vt = vtilde(w.vloc)
        n = np.asarray(w.n)
        dg = (g[:, None, :] - g[None, :, :]) % n[None, None, :]
        H += vt[dg[..., 0], dg[..., 1], dg[..., 2]]
    if "NL" in include and w.nproj > 0:
        B = beta_matrix(w, g, q)
        H += B @ block_D(w) @ B.conj().T
    return H


class Hamiltonian:
    """Matrix-free H (and H - s) on the sphere, FP64, via numpy.fft.

    The projector table B (N x natom*nproj) is stored when it takes at most
    table_bytes (default 16 GB); otherwise the nonlocal term is applied atom
    chunk by atom chunk from the same beta_matrix, never holding all of B."""

    def __init__(self, w, table_bytes=16e9, atom_chunk=128):
        self.w = w
        self.g, self.q = sphere(w.L, w.n, w.ecut, w.k)
        self.npw = self.g.shape[0]
        self.kin = kinetic(self.q)
        n = np.asarray(w.n)
        self.gi = tuple((self.g % n[None, :]).T)
        self.atom_chunk = atom_chunk
        store = w.nproj > 0 and self.npw * w.natom * w.nproj * 16 <= table_bytes
        self.B = beta_matrix(w, self.g, self.q) if store else None
        self.Dfull = block_D(w) if store else None
        self.chunked = w.nproj > 0 and not store
        self.F = None
        self.napply = 0

    def apply(self, X, shift=0.0):
        """(H - shift) X for X of shape [nband][npw] (complex128)."""
        X = np.atleast_2d(X)
        out = np.empty_like(X, dtype=np.complex128)
        n = self.w.n
        for b in range(X.shape[0]):
            c = np.zeros(n, dtype=np.complex128)
            c[self.gi] = X[b]
            psi_r = np.fft.ifftn(c) * c.size        # psi(r_j) = sum_G c_G e^{i G.r_j}
            vpsi = np.fft.fftn(self.w.vloc * psi_r) / c.size
            out[b] = vpsi[self.gi] + (self.kin - shift) * X[b]
        if self.B is not None:
            P = self.B.conj().T @ X.T                 # <beta|psi>, (Np, nband)
            out += (self.B @ (self.Dfull @ P)).T
        elif self.chunked:
            # beta_{a,c}(q) = f_c(q) e^{-i q.R_a}: the projections and the sum over the
            # projectors, atom chunk by atom chunk, with the phases of the chunk's atoms
            # E[G, a] = e^{-i q_G.R_a} (f_c = the type factors, beta_matrix with no phase)
            w = self.w
            if self.F is None:
                self.F = beta_matrix(_at_origin(w), self.g, self.q, [0]).T  # (nproj, N)
            nb = X.shape[0]
            U = [np.conj(self.F) * X[b][None, :] for b in range(nb)]         # (nproj, N) per band
            acc = np.zeros((nb, w.nproj, X.shape[1]), dtype=np.complex128)   # sum_a E Q per type
            for a0 in range(0, w.natom, self.atom_chunk):
                atoms = list(range(a0, min(w.natom, a0 + self.atom_chunk)))
                E = np.exp(-1j * (self.q @ w.pos[atoms].T))                  # (N, na)
                for b in range(nb):
                    P = (U[b] @ np.conj(E)).T                                # <beta_ac|psi_b>, (na, nproj)
                    Q = np.matmul(w.D[atoms], P[:, :, None])[:, :, 0]        # D_a P_a
                    acc[b] += (E @ Q).T
            out += np.sum(self.F[None, :, :] * acc, axis=1)                  # sum_c f_c sum_a E Q
        self.napply += X.shape[0]
        return out


def brute_nearest(w, e_ref, nstates):
    """The nstates eigenpairs of the dense H nearest e_ref, ordered by
    (|eps - e_ref|, eps).  Returns (eps, vecs[nstates][npw], all_eigs)."""
    H = dense_H(w)
    eps, V = np.linalg.eigh(H)
    order = np.lexsort((eps, np.abs(eps - e_ref)))
    sel = order[:nstates]
    return eps[sel], V[:, sel].T.copy(), eps
