"""Separable Fourier sum (three one-axis sums over the bounding box of the R set) against the
dense contraction and the oracle.  Same sums up to rounding order: relative 1e-12 against the
dense FP64 path, 1e-10 against the oracle, 1e-5 with FP32 rotations."""
import json
import os

import numpy as np
import pytest

import tbgen
from oracle import kubo_oracle as O

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_separable_w16_full_mesh_vs_golden(kubo, torch):
    g = json.load(open(os.path.join(GOLDEN, "w16_r125_k24.json")))
    m = tbgen.random_tb(16, 2, 1.0, 0)
    S = kubo.ahc(cuda(torch, m.H_R), m.R, (24, 24, 24), cuda(torch, np.array(g["E_F"])),
                 etas=g["etas"], separable=True).cpu().numpy()
    assert rel(S, np.array(g["S"])) < 1e-10


def test_separable_w64_slab_vs_dense(kubo, torch):
    m = tbgen.random_tb(64, 5, 1.5, 0)
    kmesh = (128, 128, 128)
    EF = cuda(torch, np.linspace(-1.0, 1.0, 64))
    H = cuda(torch, m.H_R)
    rng = (20 * 16384, 24 * 16384)
    a = kubo.ahc(H, m.R, kmesh, EF, k_range=rng).cpu().numpy()
    b = kubo.ahc(H, m.R, kmesh, EF, k_range=rng, separable=True).cpu().numpy()
    assert rel(b, a) < 1e-12
    c = kubo.ahc(H, m.R, kmesh, EF, k_range=rng, separable=True, precision="mixed_rotation").cpu().numpy()
    assert rel(c, a) < 1e-5


def test_separable_box_with_holes_and_uneven_extent(kubo, torch):
    """R set: a 5 x 3 x 7 box with several +-R pairs removed; Fermi-Dirac, two etas."""
    full = tbgen.random_tb(6, 3, 1.2, 21)
    R = np.asarray(full.R)
    keep = (np.abs(R[:, 0]) <= 2) & (np.abs(R[:, 1]) <= 1)
    rng = np.random.default_rng(3)
    for _ in range(6):                      # drop random pairs (never R = 0)
        q = int(rng.integers(R.shape[0]))
        if not R[q].any():
            continue
        neg = np.where((R == -R[q]).all(axis=1))[0][0]
        keep[q] = keep[neg] = False
    H_R, Rk = full.H_R[keep], R[keep]
    kmesh = (5, 4, 6)
    EF = np.array([-0.3, 0.2])
    S = kubo.ahc(cuda(torch, H_R), Rk, kmesh, cuda(torch, EF), etas=[1e-3, 0.05], kT=0.03,
                 separable=True).cpu().numpy()
    ref = O.ahc(H_R, Rk, kmesh, EF, etas=[1e-3, 0.05], kT=0.03)
    assert rel(S, ref) < 1e-10


def test_separable_partial_planes_and_chunks(kubo, torch):
    m = tbgen.random_tb(12, 2, 1.0, 5)
    kmesh = (6, 5, 4)
    EF = cuda(torch, np.array([0.0, 0.4]))
    H = cuda(torch, m.H_R)
    full = kubo.ahc(H, m.R, kmesh, EF).cpu().numpy()
    parts = sum(kubo.ahc(H, m.R, kmesh, EF, k_range=(a * 20, b * 20), separable=True, chunk_k=7).cpu().numpy()
                for a, b in ((0, 2), (2, 3), (3, 6)))
    assert rel(parts, full) < 1e-12


def test_separable_host_buffers(kubo, torch):
    m = tbgen.random_tb(8, 1, 1.0, 9)
    S = kubo.ahc_host(m.H_R, m.R, (4, 4, 4), np.array([0.1]), separable=True)
    ref = O.ahc(m.H_R, m.R, (4, 4, 4), [0.1])
    assert rel(S, ref) < 1e-10


def test_separable_unsupported_cases(kubo, torch):
    m = tbgen.random_tb(8, 1, 1.0, 9)
    H, EF = cuda(torch, m.H_R), cuda(torch, np.array([0.1]))
    for kw in (dict(k_range=(3, 40)), dict(precision="mixed")):
        with pytest.raises(kubo.KuboError) as ei:
            kubo.ahc(H, m.R, (4, 4, 4), EF, separable=True, **kw)
        assert ei.value.name == "KUBO_ERR_UNSUPPORTED"
