"""Pins of the FP64 gradient oracle (dL/dH(R) of L = sum g[e,j] S_e(E_F_j)).

The pin is brute force: central finite differences of the forward oracle under
Hermitian-paired perturbations of single entries of H(R), which is independent of the
reverse-mode derivation (a dropped term, a wrong sign or a transposed factor in any of
its steps changes the comparison by O(1)).  Cases cover Fermi-Dirac and step occupation,
eta = 0 (degenerate-pair skip) and eta > 0, several Fermi levels and broadenings at once,
and exactly degenerate bands (two identical decoupled layers).
"""
import numpy as np
import pytest

import tbgen
from oracle import kubo_oracle as O
from oracle import kubo_grad_oracle as OG


def _paired_fd(H_R, R, neg, kmesh, E_F, g, etas, kT, r, i, j, imag, h):
    """Central difference of L under H(R_r)_ij += d, H(-R_r)_ji += conj(d) (d = h or i h)."""
    def L(sign):
        H = H_R.copy()
        d = sign * h * (1j if imag else 1.0)
        H[r, i, j] += d
        if not (neg[r] == r and i == j):
            H[neg[r], j, i] += np.conj(d)
        else:
            H[r, i, i] = H[r, i, i].real + 0j   # a diagonal entry of H(0) stays real
        S = O.ahc(H, R, kmesh, E_F, etas=etas, kT=kT)
        return float(np.sum(g * S))
    return (L(+1) - L(-1)) / (2 * h)


def _neg_index(R):
    idx = {tuple(r): q for q, r in enumerate(np.asarray(R).tolist())}
    return np.array([idx[tuple((-np.asarray(r)).tolist())] for r in np.asarray(R)])


def _expected(G, neg, r, i, j, imag):
    if neg[r] == r and i == j:
        return 0.0 if imag else G[r, i, i].real
    return 2.0 * (G[r, i, j].imag if imag else G[r, i, j].real)


def _entries(rng, N_R, W, neg, n):
    out = [(int(np.where(neg == np.arange(N_R))[0][0]), 0, 0, False)]   # H(0) diagonal
    while len(out) < n:
        r = int(rng.integers(N_R)); i = int(rng.integers(W)); j = int(rng.integers(W))
        imag = bool(rng.integers(2))
        if neg[r] == r and i == j:
            continue
        out.append((r, i, j, imag))
    return out


@pytest.mark.parametrize("kT,etas,E_F", [
    (0.05, [1e-2, 0.1], [-0.4, 0.3]),     # Fermi-Dirac, two broadenings, two Fermi levels
    (0.0, [0.05], [0.1]),                 # step occupation
    (0.02, [0.0], [0.0, 0.5]),            # eta = 0 (degenerate-pair skip path)
])
def test_gradient_matches_central_differences(kT, etas, E_F):
    m = tbgen.random_tb(4, 1, 1.0, 3)
    kmesh = (3, 4, 2)
    rng = np.random.default_rng(17)
    g = rng.standard_normal((len(etas), len(E_F)))
    G = OG.ahc_grad(m.H_R, m.R, kmesh, E_F, g, etas=etas, kT=kT)
    neg = _neg_index(m.R)
    scale = np.max(np.abs(G))
    for (r, i, j, imag) in _entries(rng, m.N_R, m.W, neg, 8):
        fd = _paired_fd(m.H_R, m.R, neg, kmesh, E_F, g, etas, kT, r, i, j, imag, 1e-5)
        assert abs(fd - _expected(G, neg, r, i, j, imag)) <= 2e-6 * scale, (r, i, j, imag, fd)


def test_gradient_is_hermitian_paired():
    m = tbgen.random_tb(3, 1, 1.0, 5)
    G = OG.ahc_grad(m.H_R, m.R, (3, 3, 2), [0.0], [[1.0]], etas=[1e-2], kT=0.05)
    neg = _neg_index(m.R)
    assert np.allclose(G[neg], np.conj(np.swapaxes(G, -1, -2)), rtol=0, atol=1e-14 * np.max(np.abs(G)))


def test_gradient_with_exactly_degenerate_bands():
    """Two identical decoupled layers: every level is doubly degenerate at every k."""
    m = tbgen.stack_layers(tbgen.qwz(-1.2, tz=0.3, c0=0.2), 2)
    kmesh = (4, 3, 3)
    E_F, etas, kT = [0.1], [0.05], 0.1
    g = np.array([[1.0]])
    G = OG.ahc_grad(m.H_R, m.R, kmesh, E_F, g, etas=etas, kT=kT)
    assert np.all(np.isfinite(G))
    neg = _neg_index(m.R)
    rng = np.random.default_rng(2)
    scale = np.max(np.abs(G))
    for (r, i, j, imag) in _entries(rng, m.N_R, m.W, neg, 8):
        fd = _paired_fd(m.H_R, m.R, neg, kmesh, E_F, g, etas, kT, r, i, j, imag, 1e-5)
        assert abs(fd - _expected(G, neg, r, i, j, imag)) <= 2e-6 * scale, (r, i, j, imag, fd)


def test_gradient_of_a_partition_adds_up():
    m = tbgen.random_tb(3, 1, 1.0, 8)
    kmesh = (3, 2, 2)
    N = 12
    full = OG.ahc_grad(m.H_R, m.R, kmesh, [0.2], [[1.0]], etas=[0.1], kT=0.05)
    a = OG.ahc_grad(m.H_R, m.R, kmesh, [0.2], [[1.0]], etas=[0.1], kT=0.05, kidx=np.arange(5))
    b = OG.ahc_grad(m.H_R, m.R, kmesh, [0.2], [[1.0]], etas=[0.1], kT=0.05, kidx=np.arange(5, N))
    assert np.allclose(a + b, full, rtol=0, atol=1e-14 * np.max(np.abs(full)))
