"""Plain FP64 CPU oracle for the gradient of the anomalous Hall sum with respect to H(R).

TEST INFRASTRUCTURE ONLY (same rules as ``kubo_oracle``: only the tests, the smoke check
and the bench's CPU arms may import it; the library never does).  It shares no code with
the CUDA path; it reuses the forward steps of ``kubo_oracle``.

Quantity.  For weights g[e, j] on the outputs S_e(E_F_j) of Eq. 2 (eta_e, E_F_j),
L = sum_{e,j} g[e, j] S_e(E_F_j).  The oracle returns, for every R of the input set,

    G(R) = dL/dRe H(R) + i dL/dIm H(R)                    (complex [N_R, W, W])

where L is extended off the Hermitian-paired inputs by taking the Hermitian part of H(k),
d_x H(k) and d_y H(k) (so G(-R) = G(R)^dagger).  For a Hermitian-paired real perturbation
of H(R)_ij and H(-R)_ji (R != 0, or i != j at R = 0) the first-order change of L is
2 Re G(R)_ij per unit step; for an imaginary one it is 2 Im G(R)_ij.

Reverse-mode steps, in the order of the forward pass (Sec. 2.2 steps (1)-(4), Eq. 2-3),
written out with the library primitives numpy offers:
  (4') Omega_bar[e, n] = sum_j g[e, j] occ_j(E_n) / N_k;
       E_bar[n]       += sum_{e,j} g[e, j] occ_j'(E_n) Omega[e, n] / N_k   (Fermi-Dirac only;
                          the step function contributes nothing almost everywhere)
       T_nm = num_nm / D_nm with num_nm = -2 Im(v^x_nm v^y_mn), D_nm = (E_n - E_m)^2 + eta^2:
       num_bar = sum_e T_bar / D,  D_bar = -T_bar num / D^2,
       E_bar[p] += sum_m 2 (E_p - E_m) (D_bar_pm + D_bar_mp)
  (3') v^x_bar_nm = -2 i num_bar_nm conj(v^y_mn), v^y_bar_mn = -2 i num_bar_nm conj(v^x_nm)
       (for f = Im(z w): df/dRe z + i df/dIm z = i conj(w)).
       v^a = U^dagger dH_a U: dH_a_bar = herm(U v^a_bar U^dagger),
       U_bar = sum_a dH_a U (v^a_bar + v^a_bar^dagger).
  (2') first-order perturbation theory of the Hermitian eigenproblem (dE_n = (U^dagger dH U)_nn,
       dU = U C with C_ij = (U^dagger dH U)_ij / (E_j - E_i), i != j):
       H_bar = U [diag(E_bar) + F o (U^dagger U_bar - U_bar^dagger U) / 2] U^dagger,
       F_ij = (E_j - E_i) / ((E_j - E_i)^2 + eps^2), F_ii = 0 (degeneracy-broadened 1/dE,
       eps = grad_eps, or 1e-12 max|E(k)| when grad_eps is 0).
  (1') H(k) = sum_R e^{ik.R} H(R), d_a H(k) = sum_R i R_a e^{ik.R} H(R):
       G(R) = sum_k e^{-ik.R} [H_bar(k) - i R_x dH_x_bar(k) - i R_y dH_y_bar(k)].
"""
from __future__ import annotations

import numpy as np

from . import kubo_oracle as O

__all__ = ["occupation_derivative", "ahc_grad"]


def occupation_derivative(E, E_F, kT):
    """d occ / dE_n for the Fermi-Dirac factor ([..., n_EF, W]); zero for the step function."""
    f = O.occupation(E, E_F, kT)
    if kT == 0.0:
        return np.zeros_like(f)
    return -f * (1.0 - f) / kT


def _herm(M):
    return 0.5 * (M + np.conj(np.swapaxes(M, -1, -2)))


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def ahc_grad(H_R, R, kmesh, E_F, g, etas=(1e-3,), kT=0.0, kidx=None, grad_eps=0.0,
             batch=128):
    """G(R) [N_R, W, W] complex128 for L = sum_{e,j} g[e, j] S_e(E_F_j) (see module doc).

    ``kidx`` restricts the k-sum to a subset of mesh points (weight stays 1/N_k), as in
    ``kubo_oracle.ahc``.
    """
    H_R = np.asarray(H_R, dtype=np.complex128)
    N_R, W, _ = H_R.shape
    Rf = np.asarray(R, dtype=np.float64)
    kmesh = tuple(int(x) for x in kmesh)
    N_k = int(np.prod(kmesh))
    if kidx is None:
        kidx = np.arange(N_k, dtype=np.int64)
    kidx = np.asarray(kidx, dtype=np.int64)
    E_F = np.atleast_1d(np.asarray(E_F, dtype=np.float64))
    etas = np.atleast_1d(np.asarray(etas, dtype=np.float64))
    g = np.asarray(g, dtype=np.float64).reshape(etas.size, E_F.size)
    G = np.zeros((N_R, W * W), dtype=np.complex128)
    off = ~np.eye(W, dtype=bool)
    for s in range(0, kidx.size, batch):
        kb = kidx[s:s + batch]
        ph = O.phases_mesh(R, kmesh, kb)                        # [n, N_R]
        Hk, dHx, dHy = O.bloch(H_R, R, kmesh, kb)
        E, U = O.eigh(Hk)
        vx, vy = O.velocity(U, dHx), O.velocity(U, dHy)
        n = E.shape[0]
        # ---- forward quantities of step (4)
        dE = E[:, :, None] - E[:, None, :]                       # E_n - E_m
        num = -2.0 * np.imag(vx * np.swapaxes(vy, -1, -2))       # [n, W, W]
        scale = np.max(np.abs(E), axis=-1)[:, None, None]
        occ = O.occupation(E, E_F, kT)                           # [n, n_EF, W]
        docc = occupation_derivative(E, E_F, kT)                 # [n, n_EF, W]
        Ebar = np.zeros_like(E)
        num_bar = np.zeros_like(num)
        for e, eta in enumerate(etas):
            if eta == 0.0:
                keep = off[None] & (np.abs(dE) > O.DEGENERATE_REL * scale)
            else:
                keep = np.broadcast_to(off[None], dE.shape)
            D = np.where(keep, dE * dE + eta * eta, 1.0)
            T = np.where(keep, num / D, 0.0)
            Om = T.sum(axis=-1)                                   # [n, W]
            Om_bar = np.einsum("j,kjw->kw", g[e], occ) / N_k
            Ebar += np.einsum("j,kjw->kw", g[e], docc) * Om / N_k
            T_bar = np.where(keep, Om_bar[:, :, None], 0.0)
            num_bar += T_bar / D
            D_bar = np.where(keep, -T_bar * num / (D * D), 0.0)
            Ebar += np.sum(2.0 * dE * (D_bar + np.swapaxes(D_bar, -1, -2)), axis=-1)
        # ---- step (3'): velocities
        vx_bar = -2j * num_bar * np.conj(np.swapaxes(vy, -1, -2))
        vy_bar = np.swapaxes(-2j * num_bar * np.conj(vx), -1, -2)
        Xbar = _herm(U @ vx_bar @ _dag(U))
        Ybar = _herm(U @ vy_bar @ _dag(U))
        U_bar = dHx @ U @ (vx_bar + _dag(vx_bar)) + dHy @ U @ (vy_bar + _dag(vy_bar))
        # ---- step (2'): eigen-adjoint
        eps = grad_eps if grad_eps > 0.0 else 1e-12 * scale
        dji = -dE                                                 # E_j - E_i at [i, j]
        F = np.where(off[None], dji / (dji * dji + eps * eps), 0.0)
        inner = F * 0.5 * (_dag(U) @ U_bar - _dag(U_bar) @ U)
        inner = inner + np.einsum("kw,wv->kwv", Ebar, np.eye(W))
        Hbar = _herm(U @ inner @ _dag(U))
        # ---- step (1'): transposed Fourier sum
        cph = np.conj(ph)                                         # e^{-ik.R}  [n, N_R]
        G += cph.T @ Hbar.reshape(n, W * W)
        G += (-1j * Rf[:, 0])[:, None] * (cph.T @ Xbar.reshape(n, W * W))
        G += (-1j * Rf[:, 1])[:, None] * (cph.T @ Ybar.reshape(n, W * W))
    return G.reshape(N_R, W, W)
