"""Plain FP64 CPU oracle for the Kubo-formula anomalous Hall conductivity (AHC).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct definition
that the CUDA path is checked against.  Only the test-suite, the smoke check and
the bench's CPU-baseline / reference arm may import it; the library never does.
It shares no code with the CUDA path (it imports only numpy, math and the seeded
input generator ``tbgen``, which holds no arithmetic of the method).

What it computes (paper: Sec. 2.1 Eqs. 2-3, Sec. 2.2 "Baseline implementation",
List 1 -- steps (1) define matrices, (2) diagonalise, (3) convert the currents to
the eigenbasis, (4) evaluate and accumulate), per k-point of a uniform mesh:

  (1) H(k)      = sum_R e^{i k.R} H(R)
      d_a H(k)  = sum_R i R_a e^{i k.R} H(R)          (a = x, y: velocity / current)
  (2) H(k) = U diag(E) U^dagger, E ascending (LAPACK ``eigh`` as a library step)
  (3) v^a = U^dagger (d_a H) U                         (columns of U are eigenvectors)
  (4) Omega_n = -2 sum_{m != n} Im(v^x_nm v^y_mn) / ((E_n - E_m)^2 + eta^2)
      S(E_F)  = (1/N_k) sum_k sum_n occ(E_n(k); E_F) Omega_n(k)

Readings of the paper (Eqs. 2-3 are silent or ambiguous on these points):
  * Normalisation/prefactor: the paper's hbar/pi prefactor omits e^2, the cell volume
    and the (2 pi)^-3 of the Brillouin-zone integral (Sec. 2.1).  The oracle returns the
    dimensionless mesh average S(E_F) above; for a 2-D layer the Chern number is
    C = 2 pi S.
  * Sign: the paper writes sigma_yx with Im[J_y]_nm[J_x]_mn.  With J = d H (Hermitian),
    Im([v^y]_nm [v^x]_mn) = -Im(v^x_nm v^y_mn), so the paper's integrand is proportional
    to sum_{n occ} Omega_n as defined here (the Berry curvature Omega_z).
  * Broadening: the paper's denominator is (E_m - E_n)^2; eta enters as
    (E_n - E_m)^2 + eta^2.  With eta = 0, pairs with |E_n - E_m| <= 1e-12 max|E| are
    skipped (they only arise between degenerate copies, where they cancel).
  * Occupation: theta(E_F - E_n) with occupied iff E_n < E_F (strict); with kT > 0 the
    Fermi-Dirac factor 1 / (1 + exp((E_n - E_F)/kT)).
  * Mesh: Gamma-centred uniform N1 x N2 x N3, k_j = 2 pi (j1/N1, j2/N2, j3/N3), weight
    1/N_k; linear index (j1 N2 + j2) N3 + j3.  Phases use exact integer argument
    reduction: k.R = 2 pi sum_a ((j_a R_a) mod N_a) / N_a.
  * Lattice (tight-binding) gauge: orbital positions are not used; velocities are the
    k-derivatives of the integer-R Fourier sum.

Batching over k (many k-points per numpy call) is the paper's own equivalence,
Eq. 4: the batched sum equals the per-k sum exactly; nothing else is reordered.
"""
from __future__ import annotations

import math
import numpy as np

__all__ = [
    "kfrac_of_index", "phases_mesh", "phases_frac", "bloch", "bloch_frac",
    "eigh", "velocity", "berry_terms", "berry_curvature", "occupation",
    "kubo_per_k", "ahc", "ahc_occ_unocc_per_k", "DEGENERATE_REL",
]

# eta = 0 degenerate-pair skip threshold (relative to max|E| at that k)
DEGENERATE_REL = 1e-12


def kfrac_of_index(kmesh, kidx) -> np.ndarray:
    """Integer mesh coordinates (j1, j2, j3) [n, 3] of linear k-indices (j3 fastest)."""
    N1, N2, N3 = (int(x) for x in kmesh)
    kidx = np.asarray(kidx, dtype=np.int64)
    j3 = kidx % N3
    j2 = (kidx // N3) % N2
    j1 = kidx // (N2 * N3)
    return np.stack([j1, j2, j3], axis=-1)


def phases_mesh(R, kmesh, kidx) -> np.ndarray:
    """e^{i k.R} for mesh points: [n_k, N_R] complex128, exact argument reduction.

    k.R = 2 pi sum_a (j_a R_a mod N_a)/N_a; the fraction is reduced mod 1 before the
    trigonometric evaluation so that |argument| < 2 pi.
    """
    j = kfrac_of_index(kmesh, kidx)                       # [n, 3]
    R = np.asarray(R, dtype=np.int64)                     # [N_R, 3]
    N = np.asarray(kmesh, dtype=np.int64)
    num = np.zeros((j.shape[0], R.shape[0]), dtype=np.float64)
    for a in range(3):
        num += np.mod(np.outer(j[:, a], R[:, a]), N[a]) / float(N[a])
    frac = np.mod(num, 1.0)
    return np.exp(2j * np.pi * frac)


def phases_frac(R, kfrac) -> np.ndarray:
    """e^{i k.R} at arbitrary k = 2 pi * kfrac (kfrac [n, 3] in units of the reciprocal basis)."""
    kfrac = np.atleast_2d(np.asarray(kfrac, dtype=np.float64))
    return np.exp(2j * np.pi * (kfrac @ np.asarray(R, dtype=np.float64).T))


def _fourier(H_R, R, ph):
    """H(k), d_x H(k), d_y H(k) from phases ph [n, N_R] (Sec. 2.2 step (1)).

    Written as the matrix product of the phase rows with the flattened H(R) blocks.
    """
    NR, W, _ = H_R.shape
    flat = H_R.reshape(NR, W * W)
    Rf = np.asarray(R, dtype=np.float64)
    Hk = (ph @ flat).reshape(-1, W, W)
    dHx = ((1j * ph * Rf[None, :, 0]) @ flat).reshape(-1, W, W)
    dHy = ((1j * ph * Rf[None, :, 1]) @ flat).reshape(-1, W, W)
    return Hk, dHx, dHy


def bloch(H_R, R, kmesh, kidx):
    """Step (1) on mesh points: (H(k), d_x H(k), d_y H(k)), each [n, W, W] complex128."""
    return _fourier(np.asarray(H_R), R, phases_mesh(R, kmesh, kidx))


def bloch_frac(H_R, R, kfrac):
    """Step (1) at arbitrary k = 2 pi kfrac (used for finite-difference and loop checks)."""
    return _fourier(np.asarray(H_R), R, phases_frac(R, kfrac))


def eigh(Hk):
    """Step (2): Hermitian eigendecomposition H = U diag(E) U^dagger, E ascending.

    Library primitive (LAPACK via numpy); columns of U are the eigenvectors.  The paper's
    List 1 writes the rotation as U J U^dagger with eigenvectors as rows; with columns the
    same rotation reads U^dagger J U.
    """
    return np.linalg.eigh(Hk)


def velocity(U, dH):
    """Step (3): v = U^dagger dH U (velocity / current operator in the eigenbasis)."""
    return np.conj(np.swapaxes(U, -1, -2)) @ dH @ U


def berry_terms(E, vx, vy, eta):
    """Pair terms T_nm = -2 Im(v^x_nm v^y_mn) / ((E_n - E_m)^2 + eta^2), T_nn = 0.

    Eq. 3 with the eta-broadened denominator.  For eta == 0 degenerate pairs
    (|E_n - E_m| <= 1e-12 max|E|) are set to zero.
    """
    E = np.asarray(E)
    dE = E[..., :, None] - E[..., None, :]
    num = -2.0 * np.imag(vx * np.swapaxes(vy, -1, -2))
    W = E.shape[-1]
    off = ~np.eye(W, dtype=bool)
    if eta == 0.0:
        scale = np.max(np.abs(E), axis=-1, keepdims=True)[..., None]
        keep = off & (np.abs(dE) > DEGENERATE_REL * scale)
        den = np.where(keep, dE * dE, 1.0)
        return np.where(keep, num / den, 0.0)
    den = dE * dE + eta * eta
    return np.where(off, num / den, 0.0)


def berry_curvature(E, vx, vy, eta):
    """Omega_n = sum_{m != n} T_nm (per band Berry curvature, z component)."""
    return np.sum(berry_terms(E, vx, vy, eta), axis=-1)


def occupation(E, E_F, kT):
    """occ(E_n; E_F): theta(E_F - E_n) (strict, kT == 0) or Fermi-Dirac (kT > 0).

    Returns [..., n_EF, W].
    """
    E = np.asarray(E)[..., None, :]
    EF = np.asarray(E_F, dtype=np.float64)[:, None]
    if kT == 0.0:
        return (E < EF).astype(np.float64)
    x = (E - EF) / kT
    # numerically stable logistic: 1/(1+e^x)
    return np.where(x > 0, np.exp(-np.abs(x)) / (1.0 + np.exp(-np.abs(x))),
                    1.0 / (1.0 + np.exp(-np.abs(x))))


def kubo_per_k(H_R, R, kmesh, kidx, etas=(1e-3,)):
    """Steps (1)-(4) for a list of mesh points.

    Returns (E [n, W], Omega [n_eta, n, W]).
    """
    Hk, dHx, dHy = bloch(H_R, R, kmesh, kidx)
    E, U = eigh(Hk)
    vx = velocity(U, dHx)
    vy = velocity(U, dHy)
    Om = np.stack([berry_curvature(E, vx, vy, float(eta)) for eta in etas])
    return E, Om


def ahc_occ_unocc_per_k(H_R, R, kmesh, kidx, E_F, eta):
    """North-star form: -2 Im sum_{n occ, m unocc} v^x_nm v^y_mn / ((E_n-E_m)^2+eta^2).

    Returns [n, n_EF] per-k sums (kT = 0).  Equal to sum_{n occ} Omega_n because
    T_nm = -T_mn (occupied-occupied pairs cancel); the tests check that identity.
    """
    Hk, dHx, dHy = bloch(H_R, R, kmesh, kidx)
    E, U = eigh(Hk)
    T = berry_terms(E, velocity(U, dHx), velocity(U, dHy), float(eta))
    out = np.zeros((E.shape[0], len(E_F)))
    for j, ef in enumerate(E_F):
        occ = E < ef
        mask = occ[:, :, None] & (~occ)[:, None, :]
        out[:, j] = np.sum(np.where(mask, T, 0.0), axis=(1, 2))
    return out


def ahc(H_R, R, kmesh, E_F, etas=(1e-3,), kT=0.0, kidx=None, batch=256,
        return_per_k=False):
    """S(E_F) = (1/N_k) sum_k sum_n occ(E_n(k)) Omega_n(k)  (Eq. 2 summed over the mesh).

    ``kidx`` restricts the sum to a subset of mesh points (weight stays 1/N_k, so the
    sum over a partition of the mesh adds up to the full result).  The k-sum is exactly
    rounded (math.fsum) per E_F and eta.  Returns [n_eta, n_EF]; with return_per_k also
    the per-k contributions [n_k, n_eta, n_EF].
    """
    H_R = np.asarray(H_R, dtype=np.complex128)
    kmesh = tuple(int(x) for x in kmesh)
    N_k = int(np.prod(kmesh))
    if kidx is None:
        kidx = np.arange(N_k, dtype=np.int64)
    kidx = np.asarray(kidx, dtype=np.int64)
    E_F = np.atleast_1d(np.asarray(E_F, dtype=np.float64))
    etas = np.atleast_1d(np.asarray(etas, dtype=np.float64))
    partials = [[[] for _ in E_F] for _ in etas]
    per_k = [] if return_per_k else None
    for s in range(0, kidx.size, batch):
        kb = kidx[s:s + batch]
        E, Om = kubo_per_k(H_R, R, kmesh, kb, etas)
        occ = occupation(E, E_F, kT)                     # [n, n_EF, W]
        f = np.einsum("kjw,ekw->kej", occ, Om)           # [n, n_eta, n_EF]
        if per_k is not None:
            per_k.append(f / N_k)
        for e in range(len(etas)):
            for j in range(len(E_F)):
                partials[e][j].extend(f[:, e, j].tolist())
    out = np.array([[math.fsum(partials[e][j]) / N_k for j in range(len(E_F))]
                    for e in range(len(etas))])
    if return_per_k:
        return out, np.concatenate(per_k, axis=0)
    return out
