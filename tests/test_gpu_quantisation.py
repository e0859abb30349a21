"""Quantisation check of the large sweep: a stacked Haldane model (t1 = 1, t2 = 0.1,
phi = pi/2, M = 0; L = 3 decoupled layers, W = 6) on a 512 x 512 x 1 mesh.

2 pi S(E_F in the gap) = L C with |C| = 1 for every layer.  The broadened denominator
(dE^2 + eta^2) lowers each pair term by at most a factor 1 / (1 + (eta / gap)^2), with the gap
6 sqrt(3) t2 of this model, so |2 pi S| lies within L (eta / gap)^2 of L; the uniform-mesh
sum of the smooth, periodic curvature adds nothing visible at 512^2.
"""
import numpy as np
import pytest

import tbgen

pytestmark = pytest.mark.gpu

GAP = 6.0 * np.sqrt(3.0) * 0.1


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


def test_stacked_haldane_512_fp64_all_sweep_etas(kubo, torch):
    L = 3
    m = tbgen.stack_layers(tbgen.haldane(), L)
    etas = [0.0, 1e-4, 1e-3, 5e-3, 1e-2]
    S = kubo.ahc(cuda(torch, m.H_R), m.R, (512, 512, 1), cuda(torch, np.array([0.0, -0.3, 0.3])),
                 etas=etas).cpu().numpy()
    for e, eta in enumerate(etas):
        for j in range(3):
            C = 2 * np.pi * S[e, j]
            assert abs(abs(C) - L) <= L * (eta / GAP) ** 2 + 1e-7, (eta, j, C)
            if eta > 0:
                assert abs(C) <= L + 1e-9


def test_haldane_512_mixed(kubo, torch):
    m = tbgen.haldane()
    S = kubo.ahc(cuda(torch, m.H_R), m.R, (512, 512, 1), cuda(torch, np.array([0.0])), eta=0.0,
                 precision="mixed").cpu().numpy()
    assert abs(abs(2 * np.pi * S[0, 0]) - 1) < 1e-5
