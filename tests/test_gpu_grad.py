"""Reverse mode (kubo_ahc_grad, FP64) against the FP64 gradient oracle and central differences.

Bars: element-wise |G - G_oracle| <= 1e-9 max|G_oracle| on the same seeded inputs; central
differences (step 1e-6) of the CUDA forward S under Hermitian-paired perturbations of 200
random entries of H(R) at the differentiable-sigma workload's model (W = 32, N_R = 729,
48^3 mesh, kT = 25 meV, eta = 5e-3, E_F = 0), within 1e-6 max|G|.
"""
import numpy as np
import pytest

import tbgen
from oracle import kubo_oracle as O
from oracle import kubo_grad_oracle as OG

pytestmark = pytest.mark.gpu

REL_G = 1e-9


@pytest.fixture(scope="module")
def kubo():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_06675_gb300 import _build
    _build.build()
    import paper_2309_06675_gb300 as k
    k.lib()
    return k


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def cuda(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def neg_index(R):
    idx = {tuple(r): q for q, r in enumerate(np.asarray(R).tolist())}
    return np.array([idx[tuple((-np.asarray(r)).tolist())] for r in np.asarray(R)])


def assert_grad_close(G, G_ref, rel=REL_G):
    scale = np.max(np.abs(G_ref))
    err = np.max(np.abs(G - G_ref))
    assert err <= rel * scale, err / scale


@pytest.fixture(scope="module")
def m32():
    return tbgen.random_tb(32, 4, 1.5, 0)


@pytest.mark.parametrize("W,hw,kmesh,E_F,etas,kT", [
    (4, 1, (3, 4, 2), [-0.4, 0.3], [1e-2, 0.1], 0.05),
    (8, 1, (4, 4, 3), [0.1], [0.05], 0.0),
    (6, 2, (3, 3, 3), [0.0, 0.5], [0.0, 1e-3], 0.02),
    (16, 2, (4, 3, 3), [-1.0, 0.0, 1.0], [5e-3], 0.025),
])
def test_grad_matches_oracle_small(kubo, torch, W, hw, kmesh, E_F, etas, kT):
    m = tbgen.random_tb(W, hw, 1.0, 40 + W)
    rng = np.random.default_rng(W)
    g = rng.standard_normal((len(etas), len(E_F)))
    G_ref = OG.ahc_grad(m.H_R, m.R, kmesh, E_F, g, etas=etas, kT=kT)
    G, S = kubo.ahc_grad(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, np.array(E_F)), cuda(torch, g),
                         etas=etas, kT=kT, chunk_k=7, with_value=True)
    assert_grad_close(G.cpu().numpy(), G_ref)
    S_ref = O.ahc(m.H_R, m.R, kmesh, E_F, etas=etas, kT=kT)
    assert np.max(np.abs(S.cpu().numpy() - S_ref)) <= 1e-10 * np.max(np.abs(S_ref))


def test_grad_exactly_degenerate_bands(kubo, torch):
    m = tbgen.stack_layers(tbgen.qwz(-1.2, tz=0.3, c0=0.2), 2)
    kmesh = (4, 3, 3)
    G_ref = OG.ahc_grad(m.H_R, m.R, kmesh, [0.1], [[1.0]], etas=[0.05], kT=0.1)
    G = kubo.ahc_grad(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, np.array([0.1])),
                      cuda(torch, np.array([[1.0]])), eta=0.05, kT=0.1).cpu().numpy()
    assert_grad_close(G, G_ref, 1e-8)


def test_grad_large_w(kubo, torch):
    m = tbgen.random_tb(72, 1, 1.0, 9)
    kmesh = (3, 3, 2)
    G_ref = OG.ahc_grad(m.H_R, m.R, kmesh, [0.0], [[1.0]], etas=[5e-3], kT=0.025)
    G = kubo.ahc_grad(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, np.array([0.0])),
                      cuda(torch, np.array([[1.0]])), eta=5e-3, kT=0.025).cpu().numpy()
    assert_grad_close(G, G_ref)


def test_grad_w32_model_on_a_mesh_plane_vs_oracle(kubo, torch, m32):
    """The differentiable-sigma model (W=32, N_R=729) on one 48x48 plane of the 48^3 mesh."""
    kmesh = (48, 48, 48)
    rng = (17 * 2304, 18 * 2304)
    G = kubo.ahc_grad(cuda(torch, m32.H_R), m32.R, kmesh, cuda(torch, np.array([0.0])),
                      cuda(torch, np.array([[1.0]])), eta=5e-3, kT=0.025, k_range=rng).cpu().numpy()
    G_ref = OG.ahc_grad(m32.H_R, m32.R, kmesh, [0.0], [[1.0]], etas=[5e-3], kT=0.025,
                        kidx=np.arange(*rng))
    assert_grad_close(G, G_ref)


def test_grad_w32_central_differences_200_entries(kubo, torch, m32):
    """Central differences (step 1e-6) of the CUDA forward on 200 random entries."""
    kmesh = (48, 48, 48)
    rng_k = (5 * 2304, 6 * 2304)
    H = cuda(torch, m32.H_R)
    EF = cuda(torch, np.array([0.0]))
    G = kubo.ahc_grad(H, m32.R, kmesh, EF, cuda(torch, np.array([[1.0]])), eta=5e-3, kT=0.025,
                      k_range=rng_k).cpu().numpy()
    neg = neg_index(m32.R)
    rs = np.random.default_rng(123)
    h = 1e-6
    scale = np.max(np.abs(G))
    worst = 0.0
    for _ in range(200):
        r = int(rs.integers(m32.N_R)); i = int(rs.integers(32)); j = int(rs.integers(32))
        imag = bool(rs.integers(2)) and not (neg[r] == r and i == j)
        d = h * (1j if imag else 1.0)
        vals = []
        for sgn in (1, -1):
            Hp = m32.H_R.copy()
            Hp[r, i, j] += sgn * d
            if not (neg[r] == r and i == j):
                Hp[neg[r], j, i] += np.conj(sgn * d)
            vals.append(float(kubo.ahc(cuda(torch, Hp), m32.R, kmesh, EF, eta=5e-3, kT=0.025,
                                       k_range=rng_k).cpu().numpy()[0, 0]))
        fd = (vals[0] - vals[1]) / (2 * h)
        if neg[r] == r and i == j:
            want = G[r, i, i].real
        else:
            want = 2.0 * (G[r, i, j].imag if imag else G[r, i, j].real)
        worst = max(worst, abs(fd - want) / scale)
    assert worst <= 1e-6, worst


def test_grad_full_mesh_equals_sum_of_halves(kubo, torch, m32):
    kmesh = (48, 48, 48)
    N = 48 ** 3
    H = cuda(torch, m32.H_R)
    EF = cuda(torch, np.array([0.0]))
    g = cuda(torch, np.array([[1.0]]))
    G, S = kubo.ahc_grad(H, m32.R, kmesh, EF, g, eta=5e-3, kT=0.025, with_value=True)
    a = kubo.ahc_grad(H, m32.R, kmesh, EF, g, eta=5e-3, kT=0.025, k_range=(0, N // 2))
    b = kubo.ahc_grad(H, m32.R, kmesh, EF, g, eta=5e-3, kT=0.025, k_range=(N // 2, N))
    G, a, b = G.cpu().numpy(), a.cpu().numpy(), b.cpu().numpy()
    assert np.max(np.abs(a + b - G)) <= 1e-12 * np.max(np.abs(G))
    assert np.allclose(G[neg_index(m32.R)], np.conj(np.swapaxes(G, -1, -2)), rtol=0,
                       atol=1e-14 * np.max(np.abs(G)))
    S_fwd = kubo.ahc(H, m32.R, kmesh, EF, eta=5e-3, kT=0.025).cpu().numpy()
    assert np.array_equal(S.cpu().numpy(), S_fwd)


def test_autograd_function_matches_parameter_finite_differences(kubo, torch):
    """H(R) built from free complex parameters; torch autograd through AHC vs central FD."""
    m = tbgen.random_tb(6, 1, 1.0, 77)
    R = np.asarray(m.R)
    neg = neg_index(R)
    canon = [q for q in range(m.N_R) if tuple(R[q]) > (0, 0, 0)]
    zero = int(np.where((R == 0).all(axis=1))[0][0])
    kmesh = (4, 3, 3)
    EF = cuda(torch, np.array([-0.2, 0.4]))
    etas = [1e-2, 0.1]
    w = cuda(torch, np.array([[0.7, -1.3], [0.4, 2.0]]))

    def build(P, P0):
        H = torch.zeros((m.N_R, 6, 6), dtype=torch.complex128, device="cuda:0")
        for c, q in enumerate(canon):
            H[q] = P[c]
            H[neg[q]] = P[c].conj().T
        H[zero] = 0.5 * (P0 + P0.conj().T)
        return H

    P = cuda(torch, m.H_R[canon]).requires_grad_(True)
    P0 = cuda(torch, m.H_R[zero]).requires_grad_(True)
    S = kubo.AHC.apply(build(P, P0), m.R, kmesh, EF, 1e-3, etas, 0.05)
    L = (S * w).sum()
    L.backward()
    gP = P.grad.cpu().numpy()

    def loss(Pn):
        with torch.no_grad():
            S = kubo.ahc(build(cuda(torch, Pn), P0.detach()), m.R, kmesh, EF, etas=etas, kT=0.05)
            return float((S * w).sum())

    rs = np.random.default_rng(5)
    base = m.H_R[canon]
    scale = np.max(np.abs(gP))
    for _ in range(10):
        c = int(rs.integers(len(canon))); i = int(rs.integers(6)); j = int(rs.integers(6))
        for d in (1e-6, 1e-6j):
            Pp, Pm = base.copy(), base.copy()
            Pp[c, i, j] += d
            Pm[c, i, j] -= d
            fd = (loss(Pp) - loss(Pm)) / (2e-6)
            want = gP[c, i, j].real if d == 1e-6 else gP[c, i, j].imag
            assert abs(fd - want) <= 1e-6 * scale, (c, i, j, d, fd, want)
