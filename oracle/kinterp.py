"""CPU FP64 oracle: wave-function interpolation between two k-points (Sec. II.D).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this module; only tests, the package's smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA library.

Sec. II.D: with orthonormal eigenpairs (eps_i(k1), psi_i(k1)) and (eps_j(k2),
psi_j(k2)) of two nearby k-points, H(k) for k between them is taken as the
linear interpolation alpha H(k1) + (1 - alpha) H(k2), alpha = (k - k2)/(k1 - k2).
In the basis psi_i(k1) its matrix is

    H_ij(k) = alpha eps_i(k1) delta_ij + (1 - alpha) sum_m U*_im U_jm eps_m(k2),

where U is made unitary from the overlap S_ij = <psi_j(k2)|psi_i(k1)> by a
Gram-Schmidt process (exact, U = S, when every eigenstate is kept).
Diagonalising H(k) gives eps(k) and coefficients c; the interpolated state

    psi(k) = alpha sum_j c_j psi_j(k1) + (1 - alpha) sum_{j,l} c_j U_jl psi_l(k2)

is continuous in k (it is the k1-expansion at alpha = 1 and the U-mapped
k2-expansion at alpha = 0).

Readings: the states of both k-points are periodic parts u_k(r) on one common
set of plane waves G (|G| below a fixed cut), so that overlaps between k-points
are plain inner products; the Gram-Schmidt process runs over the rows of S in
index order (row i = the components of psi_i(k1) on the psi_l(k2)).
"""
from __future__ import annotations

import numpy as np

PARITY_PINS = """
complete    : with every eigenstate kept, U = S is unitary and the eigenvalues of H(k)
              equal those of alpha H(k1) + (1 - alpha) H(k2) built densely
endpoints   : alpha = 1 gives eps(k1) exactly; alpha = 0 with a complete basis gives eps(k2)
unitary     : the Gram-Schmidt U is unitary for any full-rank S; rows of U span the rows of S
              in order (U = L S with L lower triangular)
"""


def overlap(psi1, psi2):
    """S_ij = <psi_j(k2)|psi_i(k1)> for rows psi1 [n1][N], psi2 [n2][N]."""
    return psi1 @ psi2.conj().T


def gram_schmidt_rows(S):
    """Orthonormalise the rows of S in index order (modified Gram-Schmidt)."""
    U = np.array(S, dtype=np.complex128, copy=True)
    for i in range(U.shape[0]):
        for l in range(i):
            U[i] -= np.vdot(U[l], U[i]) * U[l]
        U[i] /= np.linalg.norm(U[i])
    return U


def interpolated_hamiltonian(alpha, eps1, eps2, U):
    """H_ij(k) = alpha eps_i(k1) delta_ij + (1 - alpha) sum_m U*_im U_jm eps_m(k2)."""
    return alpha * np.diag(eps1) + (1.0 - alpha) * (U.conj() * eps2[None, :]) @ U.T


def interpolate(alpha, eps1, psi1, eps2, psi2):
    """eps(k) ascending and the interpolated states [n][N] for one alpha."""
    U = gram_schmidt_rows(overlap(psi1, psi2))
    Hk = interpolated_hamiltonian(alpha, eps1, eps2, U)
    e, C = np.linalg.eigh(0.5 * (Hk + Hk.conj().T))
    # column q of C holds c_j of state q; psi_q = alpha sum_j c_jq psi1_j + (1-alpha) sum_{j,l} c_jq U_jl psi2_l
    psi = alpha * (C.T @ psi1) + (1.0 - alpha) * (C.T @ (U @ psi2))
    return e, psi


def dense_H_common(w, k, gmax):
    """Dense H(k) on the plane waves G with |G| <= gmax (common to every k):
    kinetic |k + G|^2 / 2, the local potential of the workload, and its
    projectors evaluated at q = k + G.  Returns (H, miller)."""
    from . import planewave as pw
    g, _ = pw.sphere(w.L, w.n, 0.5 * gmax * gmax, (0.0, 0.0, 0.0))
    b = 2.0 * np.pi / np.asarray(w.L)
    q = np.asarray(k)[None, :] + g * b[None, :]
    N = g.shape[0]
    H = np.zeros((N, N), dtype=np.complex128)
    H[np.arange(N), np.arange(N)] += 0.5 * np.sum(q * q, axis=1)
    vt = pw.vtilde(w.vloc)
    n = np.asarray(w.n)
    dg = (g[:, None, :] - g[None, :, :]) % n[None, None, :]
    H += vt[dg[..., 0], dg[..., 1], dg[..., 2]]
    if w.nproj > 0:
        B = pw.beta_matrix(w, g, q)
        H += B @ pw.block_D(w) @ B.conj().T
    return H, g
