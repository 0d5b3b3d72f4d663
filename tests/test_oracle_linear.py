"""Pins of the folded-spectrum linear-solve oracle (Sec. II.C, Eq. wl1 and the
M' preconditioner) against what the mathematics fixes: a library solve of
(H - E) psi = w, the eigen-decomposition of the dense H, and the action of M'
on exact eigenvectors."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import fs_inputs as fi  # noqa: E402
from oracle import linear as lin  # noqa: E402
from oracle import planewave as pw  # noqa: E402


def _box():
    return fi.make_box(L=(10.0, 10.0, 20.0), n=(16, 16, 32), ecut=5.0, natom=4, widths=(1.0,), nstates=6,
                       e_ref=0.3, seed=3)


def _rhs(w, ham):
    return fi.wavepacket_rhs(ham.g, w.L, [(5.0, 5.0, 6.0), (4.0, 6.0, 14.0)])


def test_spectral_solution_is_the_solution_of_eq_wl():
    w = _box()
    H = pw.dense_H(w)
    h = pw.Hamiltonian(w)
    W = _rhs(w, h)
    psi = lin.spectral_solution(H, w.e_ref, W)
    ref = np.linalg.solve(H - w.e_ref * np.eye(H.shape[0]), W.T).T
    assert np.abs(psi - ref).max() <= 1e-9 * np.abs(ref).max()


def test_pcg_reaches_the_spectral_expansion():
    w = _box()
    h = pw.Hamiltonian(w)
    W = _rhs(w, h)
    psi, it, err = lin.pcg_folded(h, w.e_ref, W, tol=1e-9, maxit=20000)
    ref = lin.spectral_solution(pw.dense_H(w), w.e_ref, W)
    assert np.all(err <= 1e-9)
    assert np.linalg.norm(psi - ref) <= 1e-7 * np.linalg.norm(ref)


def _eigs(w):
    H = pw.dense_H(w)
    eps, V = np.linalg.eigh(H)
    return H, eps, V


def _eigenvector_pin_error(w, h, eps, V):
    """max |M' phi_j - phi_j / (eps_j - E)^2| relative, for the 6 exact eigenvectors nearest E."""
    near = np.argsort(np.abs(eps - w.e_ref))[:6]
    phi = V[:, near].T
    z = lin.apply_mprime(h.kin, w.e_ref, 0.5, phi, phi, eps[near], np.zeros(6))
    want = phi / ((eps[near] - w.e_ref) ** 2)[:, None]
    return np.abs(z - want).max() / np.abs(want).max()


def test_mprime_is_the_folded_inverse_on_eigenvectors():
    w = _box()
    h = pw.Hamiltonian(w)
    H, eps, V = _eigs(w)
    assert _eigenvector_pin_error(w, h, eps, V) <= 1e-10
    near = np.argsort(np.abs(eps - w.e_ref))[:6]
    phi = V[:, near].T
    # a vector orthogonal to the phi_i sees M alone
    rng = np.random.default_rng(1)
    r = rng.normal(size=(1, h.npw)) + 1j * rng.normal(size=(1, h.npw))
    r = r - (phi.T @ (phi.conj() @ r.T)).T
    z = lin.apply_mprime(h.kin, w.e_ref, 0.5, r, phi, eps[near], np.zeros(6))
    m = 1.0 / ((h.kin - w.e_ref) ** 2 + 0.25)
    # (the rounding left in <phi_i|r> is amplified by c_i up to 1/(eps_i - E)^2 ~ 5e5 here)
    assert np.abs(z - m[None, :] * r).max() <= 1e-9 * np.abs(z).max()


def test_pin_catches_dropped_projector_term(monkeypatch):
    """Plant a mistake in the oracle's M' (the -M P term dropped): the
    eigenvector pin fails."""
    monkeypatch.setattr(lin, "_project_out", lambda R, phi, T: R)
    w = _box()
    h = pw.Hamiltonian(w)
    H, eps, V = _eigs(w)
    assert _eigenvector_pin_error(w, h, eps, V) > 1e-7


def test_eigenstate_preconditioner_accelerates_pcg():
    """With M' built from the exact eigenstates nearest E the PCG needs fewer
    iterations than with M alone, and both reach the same solution."""
    w = _box()
    h = pw.Hamiltonian(w)
    W = _rhs(w, h)
    H, eps, V = _eigs(w)
    near = np.argsort(np.abs(eps - w.e_ref))[:8]
    psi_m, it_m, err_m = lin.pcg_folded(h, w.e_ref, W, tol=1e-8)
    psi_p, it_p, err_p = lin.pcg_folded(h, w.e_ref, W, tol=1e-8, phi=V[:, near].T, eps=eps[near],
                                        delta=np.zeros(8))
    assert np.all(err_m <= 1e-8) and np.all(err_p <= 1e-8)
    assert it_p < it_m
    assert np.linalg.norm(psi_p - psi_m) <= 1e-6 * np.linalg.norm(psi_m)


def test_wavepacket_coefficients_are_the_fourier_transform_of_the_packet():
    """The analytic plane-wave coefficients of the wave-packet right-hand side
    equal the FFT of the periodised packet sampled on the grid (Poisson
    summation; the grid is fine enough that aliasing and the sphere cut-off
    are negligible)."""
    w = fi.make_box(L=(12.0, 12.0, 24.0), n=(48, 48, 96), ecut=60.0, natom=1, widths=(), nstates=1, e_ref=0.0,
                    seed=0)
    g, _ = pw.sphere(w.L, w.n, w.ecut, w.k)
    x0, y0, z0, k0, sxy, sz = 6.0, 5.0, 11.0, 0.8, 1.2, 1.8
    W = fi.wavepacket_rhs(g, w.L, [(x0, y0, z0)], k0=k0, s_xy=sxy, s_z=sz)[0]
    n = np.asarray(w.n)
    r = [np.arange(n[d]) * w.L[d] / n[d] for d in range(3)]
    X, Y, Z = np.meshgrid(*r, indexing="ij")
    f = np.zeros(X.shape, dtype=np.complex128)
    for a in (-1, 0, 1):                                 # the images that reach the cell
        for b in (-1, 0, 1):
            for d in (-1, 0, 1):
                Xs, Ys, Zs = X + a * w.L[0], Y + b * w.L[1], Z + d * w.L[2]
                f += np.exp(-((Xs - x0) ** 2 + (Ys - y0) ** 2) / (2 * sxy ** 2) - (Zs - z0) ** 2 / (2 * sz ** 2)
                            + 1j * k0 * Zs)
    F = np.fft.fftn(f)                                   # sum_j f(r_j) e^{-i G.r_j}
    c = F[tuple((g % n[None, :]).T)]
    c = c / np.linalg.norm(c)
    assert np.abs(c - W).max() <= 1e-10
