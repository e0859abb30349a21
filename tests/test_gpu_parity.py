"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (FP64 path): relative 1e-10 on S(E_F) (max over E_F of |diff| / max |S_ref|),
and 1e-9 * ||Omega(k)||_inf per k-point for the band curvatures.  Eigenvalues are compared
at 1e-12 * ||H||; eigenvectors through gauge-invariant quantities (residuals, curvatures).
"""
import json
import os

import numpy as np
import pytest

import tbgen
from oracle import kubo_oracle as O

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
REL_S = 1e-10
REL_OM = 1e-9


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


def rel_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def assert_omega_close(Om_gpu, Om_ref):
    """Per-k tolerance REL_OM * ||Omega(k)||_inf."""
    scale = np.max(np.abs(Om_ref), axis=-1, keepdims=True)
    assert np.all(np.abs(Om_gpu - Om_ref) <= REL_OM * np.maximum(scale, 1e-300)), \
        np.max(np.abs(Om_gpu - Om_ref) / np.maximum(scale, 1e-300))


@pytest.fixture(scope="module")
def m16():
    return tbgen.random_tb(16, 2, 1.0, 0)


@pytest.fixture(scope="module")
def m64():
    return tbgen.random_tb(64, 5, 1.5, 0)


# ---------------------------------------------------------------- step (1): Fourier sum
@pytest.mark.parametrize("which", ["m16", "m64"])
def test_bloch_matches_oracle(kubo, torch, request, which):
    m = request.getfixturevalue(which)
    kmesh = (24, 24, 24) if which == "m16" else (128, 128, 128)
    kidx = tbgen.k_sample(kmesh, 37, seed=5)
    Hp, Xp, Yp = kubo.bloch(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, kidx))
    ref = O.bloch(m.H_R, m.R, kmesh, kidx)
    for got, want in zip((Hp, Xp, Yp), ref):
        G = kubo.unpack_hermitian(got, m.W).cpu().numpy()
        assert rel_err(G, want) < 1e-12


# ---------------------------------------------------------------- step (2): eigensolver
def _random_hermitian(rng, n, W):
    X = rng.standard_normal((n, W, W)) + 1j * rng.standard_normal((n, W, W))
    return X + np.conj(np.swapaxes(X, -1, -2))


@pytest.mark.parametrize("W", [1, 2, 3, 5, 16, 33, 64])
def test_eigh_batched(kubo, torch, W):
    rng = np.random.default_rng(W)
    n = 67
    A = _random_hermitian(rng, n, W)
    # a few structured cases: diagonal, already tridiagonal, exactly degenerate blocks
    A[0] = np.diag(rng.standard_normal(W))
    if W >= 4:
        T = np.diag(rng.standard_normal(W)) + np.diag(rng.standard_normal(W - 1), 1)
        A[1] = T + T.T
        h = W // 2
        B = _random_hermitian(rng, 1, h)[0]
        A[2] = 0
        A[2][:h, :h] = B
        A[2][h:2 * h, h:2 * h] = B
    if W >= 6:
        # exactly triple-degenerate spectrum (three identical blocks)
        t3 = W // 3
        C = _random_hermitian(rng, 1, t3)[0]
        A[3] = 0
        for q in range(3):
            A[3][q * t3:(q + 1) * t3, q * t3:(q + 1) * t3] = C
        # clusters: eigenvalue pairs split by 1e-9 in a random unitary basis
        lam = np.sort(rng.standard_normal(W))
        lam[1::2] = lam[0::2][: W // 2] + 1e-9
        X = rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W))
        Q, _ = np.linalg.qr(X)
        A[4] = (Q * lam) @ np.conj(Q.T)
        # a diagonal matrix beside a dense one: the two k-points of one reduction CTA at
        # W <= 64 (one half reflects every column, the other none)
        A[6] = np.diag(rng.standard_normal(W))
    At = cuda(torch, A)
    E, U = kubo.eigh_batched(kubo.pack_hermitian(At), W)
    E, U = E.cpu().numpy(), U.cpu().numpy()
    nrm = np.max(np.abs(np.linalg.eigvalsh(A)), axis=-1)[:, None]
    assert np.all(np.abs(E - np.linalg.eigvalsh(A)) <= 1e-12 * np.maximum(nrm, 1))
    assert np.all(np.diff(E, axis=-1) >= 0)
    res = np.abs(A @ U - U * E[:, None, :]).max(axis=(1, 2))
    assert np.all(res <= 1e-12 * np.maximum(nrm[:, 0], 1))
    I = np.eye(W)
    orth = np.abs(np.conj(np.swapaxes(U, -1, -2)) @ U - I).max(axis=(1, 2))
    assert np.all(orth <= 1e-13 * max(W, 8))


@pytest.mark.parametrize("W", [24, 80])
@pytest.mark.parametrize("lg", [-400, 400])
def test_fp64_eigensolver_at_extreme_magnitudes(kubo, torch, W, lg):
    """A scaling by 2^lg (exact) scales the eigenvalues by 2^lg and leaves the eigenvectors:
    the inverse iterations (the fused FP64 kernel at W <= 64, the persistent one above) rescale
    their iterate between solves by powers of two on the bit patterns and compare pivots as
    integers, so FP64 results hold far outside the FP32 range too."""
    rng = np.random.default_rng(W + 7)
    A = _random_hermitian(rng, 9, W)
    f = 2.0 ** lg
    E0, _ = kubo.eigh_batched(kubo.pack_hermitian(cuda(torch, A)), W)
    E1, U1 = kubo.eigh_batched(kubo.pack_hermitian(cuda(torch, A * f)), W)
    E0, E1, U1 = E0.cpu().numpy(), E1.cpu().numpy() / f, U1.cpu().numpy()
    nrm = np.max(np.abs(E0), axis=-1)[:, None]
    assert np.all(np.isfinite(E1)) and np.all(np.isfinite(U1))
    assert np.all(np.abs(E1 - E0) <= 1e-12 * nrm)
    res = np.abs(A @ U1 - U1 * E1[:, None, :]).max(axis=(1, 2))
    assert np.all(res <= 1e-12 * nrm[:, 0])
    orth = np.abs(np.conj(np.swapaxes(U1, -1, -2)) @ U1 - np.eye(W)).max(axis=(1, 2))
    assert np.all(orth <= 1e-13 * max(W, 8))


def test_eigh_values_only(kubo, torch):
    rng = np.random.default_rng(1)
    A = _random_hermitian(rng, 9, 12)
    E, U = kubo.eigh_batched(kubo.pack_hermitian(cuda(torch, A)), 12, vectors=False)
    assert U is None
    assert np.allclose(E.cpu().numpy(), np.linalg.eigvalsh(A), rtol=0, atol=1e-12 * 20)


# ---------------------------------------------------------------- steps (3)-(4)
def test_berry_batched_matches_oracle(kubo, torch, m16):
    kmesh = (24, 24, 24)
    kidx = tbgen.k_sample(kmesh, 50, seed=9)
    Hk, dHx, dHy = O.bloch(m16.H_R, m16.R, kmesh, kidx)
    E, U = np.linalg.eigh(Hk)
    etas = [0.0, 1e-3, 5e-2]
    Om = kubo.berry_batched(cuda(torch, E), cuda(torch, U),
                            kubo.pack_hermitian(cuda(torch, dHx)),
                            kubo.pack_hermitian(cuda(torch, dHy)), etas=etas).cpu().numpy()
    vx, vy = O.velocity(U, dHx), O.velocity(U, dHy)
    for e, eta in enumerate(etas):
        assert_omega_close(Om[e], O.berry_curvature(E, vx, vy, eta))


# ---------------------------------------------------------------- per-k pipeline
@pytest.mark.parametrize("chunk", [0, 64, 100])
def test_ahc_k_per_k_matches_oracle_w16(kubo, torch, m16, chunk):
    kmesh = (24, 24, 24)
    kidx = tbgen.k_sample(kmesh, 300, seed=chunk)
    etas = [1e-3, 1e-2]
    E, Om = kubo.ahc_k(cuda(torch, m16.H_R), m16.R, kmesh, cuda(torch, kidx), etas=etas, chunk_k=chunk)
    E_ref, Om_ref = O.kubo_per_k(m16.H_R, m16.R, kmesh, kidx, etas)
    assert rel_err(E.cpu().numpy(), E_ref) < 1e-12
    for e in range(2):
        assert_omega_close(Om.cpu().numpy()[e], Om_ref[e])


def test_ahc_k_per_k_matches_oracle_w64_full_size_model(kubo, torch, m64):
    """W=64, N_R=1331, 128^3 mesh: sampled k-points in the default (bench) batch size."""
    kmesh = (128, 128, 128)
    kidx = tbgen.k_sample(kmesh, 96, seed=2)
    E, Om = kubo.ahc_k(cuda(torch, m64.H_R), m64.R, kmesh, cuda(torch, kidx), eta=1e-3)
    E_ref, Om_ref = O.kubo_per_k(m64.H_R, m64.R, kmesh, kidx, [1e-3])
    assert rel_err(E.cpu().numpy(), E_ref) < 1e-12
    assert_omega_close(Om.cpu().numpy()[0], Om_ref[0])


# ---------------------------------------------------------------- k-summed results
def test_ahc_config_w16_full_mesh_vs_golden(kubo, torch, m16):
    g = json.load(open(os.path.join(GOLDEN, "w16_r125_k24.json")))
    S = kubo.ahc(cuda(torch, m16.H_R), m16.R, (24, 24, 24), cuda(torch, np.array(g["E_F"])),
                 etas=g["etas"]).cpu().numpy()
    assert rel_err(S, np.array(g["S"])) < REL_S


def test_ahc_ragged_batches_and_partition(kubo, torch, m16):
    kmesh = (9, 7, 5)
    EF = np.array([0.7, -0.3, 0.0, 2.5, -1e3, 1e3])  # unsorted, includes empty/full cases
    H = cuda(torch, m16.H_R)
    EFt = cuda(torch, EF)
    S_ref = O.ahc(m16.H_R, m16.R, kmesh, EF, etas=[1e-3])
    S_all = kubo.ahc(H, m16.R, kmesh, EFt, eta=1e-3, chunk_k=37).cpu().numpy()
    assert rel_err(S_all, S_ref) < REL_S
    a = kubo.ahc(H, m16.R, kmesh, EFt, eta=1e-3, k_range=(0, 101)).cpu().numpy()
    b = kubo.ahc(H, m16.R, kmesh, EFt, eta=1e-3, k_range=(101, 315)).cpu().numpy()
    assert rel_err(a + b, S_ref) < REL_S
    assert S_all[0, 4] == 0.0                               # no occupied band
    assert abs(S_all[0, 5]) < 1e-12 * np.max(np.abs(S_ref))  # all bands: sum rule


def test_ahc_fermi_dirac_and_multi_eta(kubo, torch):
    m = tbgen.random_tb(8, 1, 1.0, 3)
    kmesh = (6, 6, 6)
    EF = np.array([-0.4, 0.1])
    etas = [0.0, 1e-4, 1e-3, 5e-3, 1e-2]
    for kT in [0.0, 0.025]:
        S = kubo.ahc(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, EF), etas=etas, kT=kT).cpu().numpy()
        S_ref = O.ahc(m.H_R, m.R, kmesh, EF, etas=etas, kT=kT)
        assert rel_err(S, S_ref) < REL_S


def test_two_band_closed_form_on_gpu(kubo, torch):
    """QWZ model: the GPU's per-k curvature equals the closed form d.(d_x d x d_y d)/(2|d|^3)."""
    model = tbgen.qwz(-0.7, tz=0.4, c0=0.3)
    kmesh = (7, 9, 5)
    kidx = np.arange(np.prod(kmesh))
    E, Om = kubo.ahc_k(cuda(torch, model.H_R), model.R, kmesh, cuda(torch, kidx), eta=0.0)
    j = O.kfrac_of_index(kmesh, kidx)
    k = 2 * np.pi * j / np.array(kmesh)
    d = np.stack([np.sin(k[:, 0]), np.sin(k[:, 1]),
                  -0.7 + np.cos(k[:, 0]) + np.cos(k[:, 1]) + 0.4 * np.cos(k[:, 2])], -1)
    dx = np.stack([np.cos(k[:, 0]), 0 * k[:, 0], -np.sin(k[:, 0])], -1)
    dy = np.stack([0 * k[:, 1], np.cos(k[:, 1]), -np.sin(k[:, 1])], -1)
    nd = np.linalg.norm(d, axis=-1)
    ref = np.einsum("ka,ka->k", d, np.cross(dx, dy)) / (2 * nd ** 3)
    assert np.allclose(Om.cpu().numpy()[0, :, 0], ref, rtol=1e-10, atol=1e-12)


def test_haldane_chern_number_on_gpu(kubo, torch):
    base = tbgen.haldane()
    for L in (1, 3):
        m = tbgen.stack_layers(base, L)
        S = kubo.ahc(cuda(torch, m.H_R), m.R, (96, 96, 1), cuda(torch, np.array([0.0])), eta=0.0)
        C = 2 * np.pi * S.cpu().numpy()[0, 0]
        assert abs(abs(C) - L) < 1e-6, (L, C)


def test_single_band_gives_zero(kubo, torch):
    m = tbgen.random_tb(1, 1, 1.0, 0)
    S = kubo.ahc(cuda(torch, m.H_R), m.R, (4, 4, 4), cuda(torch, np.array([0.0, 5.0])), eta=1e-3)
    assert np.all(S.cpu().numpy() == 0.0)


def test_host_buffers_match_device_buffers(kubo, torch, m16):
    kmesh = (8, 8, 8)
    EF = np.array([-0.2, 0.3])
    S_dev = kubo.ahc(cuda(torch, m16.H_R), m16.R, kmesh, cuda(torch, EF)).cpu().numpy()
    S_host = kubo.ahc_host(m16.H_R, m16.R, kmesh, EF)
    assert np.array_equal(S_dev, S_host)


# ---------------------------------------------------------------- errors
def test_non_hermitian_input_is_rejected_and_out_untouched(kubo, torch, m16):
    H = m16.H_R.copy()
    H[3, 1, 2] += 1e-6
    out = torch.full((1, 1), 7.0, dtype=torch.float64, device="cuda:0")
    with pytest.raises(kubo.KuboError) as ei:
        kubo.ahc(cuda(torch, H), m16.R, (4, 4, 4), cuda(torch, np.array([0.0])), out=out)
    assert ei.value.name == "KUBO_ERR_NOT_HERMITIAN"
    assert out.item() == 7.0
    H = m16.H_R.copy()
    H[0, 0, 0] = np.nan
    with pytest.raises(kubo.KuboError) as ei:
        kubo.ahc(cuda(torch, H), m16.R, (4, 4, 4), cuda(torch, np.array([0.0])), out=out)
    assert ei.value.name == "KUBO_ERR_NOT_HERMITIAN"
    assert out.item() == 7.0
    # the library stays usable after an error
    S = kubo.ahc(cuda(torch, m16.H_R), m16.R, (4, 4, 4), cuda(torch, np.array([0.0])))
    assert np.isfinite(S.cpu().numpy()).all()


def test_caller_workspace(kubo, torch, m16):
    kmesh = (6, 6, 6)
    n = kubo.workspace_size(16, m16.N_R, kmesh, 1)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda:0")
    S1 = kubo.ahc(cuda(torch, m16.H_R), m16.R, kmesh, cuda(torch, np.array([0.0])), workspace=ws)
    S2 = kubo.ahc(cuda(torch, m16.H_R), m16.R, kmesh, cuda(torch, np.array([0.0])))
    assert torch.equal(S1, S2)
    small = torch.empty(n // 2, dtype=torch.uint8, device="cuda:0")
    with pytest.raises(kubo.KuboError) as ei:
        kubo.ahc(cuda(torch, m16.H_R), m16.R, kmesh, cuda(torch, np.array([0.0])), workspace=small)
    assert ei.value.name == "KUBO_ERR_WORKSPACE"


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_padding_ablation_gives_identical_sums(kubo, torch, m64, precision):
    """The unpadded shared-memory layout (padding ablation) changes addresses only."""
    kmesh = (128, 128, 128)
    EF = cuda(torch, np.linspace(-1.0, 1.0, 64))
    H = cuda(torch, m64.H_R)
    rng = (9 * 16384, 9 * 16384 + 4096)
    # in the mixed mode the layouts compared are those of the SIMT rotation kernel
    a = kubo.ahc(H, m64.R, kmesh, EF, k_range=rng, precision=precision, rotation="simt").cpu().numpy()
    b = kubo.ahc(H, m64.R, kmesh, EF, k_range=rng, precision=precision, unpadded=True).cpu().numpy()
    assert np.array_equal(a, b)


def test_bounded_wait_gives_up_and_reports_timeout(kubo, torch, m16):
    """The tensor-core pipeline's bounded wait, on a barrier nothing completes, returns
    KUBO_ERR_TIMEOUT (9) instead of hanging; the context stays usable."""
    stream = torch.cuda.current_stream().cuda_stream
    assert kubo.lib().kubo_check_bounded_wait(2000, stream) == 9
    assert kubo.lib().kubo_check_bounded_wait(0, stream) == 1
    S = kubo.ahc(cuda(torch, m16.H_R), m16.R, (4, 4, 4), cuda(torch, np.array([0.0])))
    assert np.all(np.isfinite(S.cpu().numpy()))
