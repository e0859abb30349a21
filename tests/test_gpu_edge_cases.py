"""Edge cases of the CUDA path against the oracle: the smallest orders in every precision,
degenerate (size-1) mesh axes, many Fermi levels in both occupation kernels, the maximum
number of broadenings, unsorted / repeated per-k lists, a one-model batch."""
import numpy as np
import pytest

import tbgen
from oracle import kubo_oracle as O

pytestmark = pytest.mark.gpu


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
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("W", [1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_fourier", "mixed_rotation", "mixed_df"])
def test_smallest_orders_every_precision(kubo, torch, W, precision):
    m = tbgen.random_tb(W, 1, 1.0, 60 + W)
    kmesh = (5, 1, 3)                       # a size-1 axis
    EF = np.array([-0.5, 0.0, 0.7])
    S = kubo.ahc(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, EF), etas=[1e-3, 0.1],
                 precision=precision).cpu().numpy()
    ref = O.ahc(m.H_R, m.R, kmesh, EF, etas=[1e-3, 0.1])
    if W == 1:
        assert np.all(S == 0.0)
        return
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert np.max(np.abs(S - ref)) <= tol * max(np.max(np.abs(ref)), 1e-12)


@pytest.mark.parametrize("kT", [0.0, 0.04])
def test_many_fermi_levels(kubo, torch, kT):
    m = tbgen.random_tb(10, 1, 1.0, 70)
    kmesh = (4, 3, 5)
    EF = np.linspace(-4.0, 4.0, 2500)
    S = kubo.ahc(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, EF), kT=kT).cpu().numpy()
    ref = O.ahc(m.H_R, m.R, kmesh, EF, kT=kT)
    assert rel(S, ref) < 1e-10


def test_maximum_number_of_broadenings(kubo, torch):
    m = tbgen.random_tb(12, 1, 1.0, 71)
    kmesh = (3, 4, 4)
    etas = [0.0, 1e-5, 1e-4, 1e-3, 5e-3, 1e-2, 5e-2, 0.2]
    EF = np.array([0.0, 0.5])
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-5), ("mixed_df", 1e-5)):
        S = kubo.ahc(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, EF), etas=etas,
                     precision=prec).cpu().numpy()
        ref = O.ahc(m.H_R, m.R, kmesh, EF, etas=etas)
        for e in range(len(etas)):
            assert rel(S[e], ref[e]) < tol, (prec, e)
    with pytest.raises(kubo.KuboError):
        kubo.ahc(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, EF), etas=etas + [1.0])


def test_unsorted_and_repeated_k_list(kubo, torch):
    m = tbgen.random_tb(9, 1, 1.0, 72)
    kmesh = (6, 5, 4)
    kidx = np.array([17, 3, 3, 119, 0, 64, 17, 5], dtype=np.int64)
    E, Om = kubo.ahc_k(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, kidx), eta=1e-3)
    E_ref, Om_ref = O.kubo_per_k(m.H_R, m.R, kmesh, kidx, [1e-3])
    assert rel(E.cpu().numpy(), E_ref) < 1e-12
    scale = np.max(np.abs(Om_ref[0]), axis=-1, keepdims=True)
    assert np.all(np.abs(Om.cpu().numpy()[0] - Om_ref[0]) <= 1e-9 * scale)
    bad = cuda(torch, np.array([0, 120], dtype=np.int64))     # 120 = N_k: out of range
    with pytest.raises(kubo.KuboError):
        kubo.ahc_k(cuda(torch, m.H_R), m.R, kmesh, bad, eta=1e-3)


def test_one_model_batch(kubo, torch):
    m = tbgen.random_tb(7, 1, 1.0, 73)
    kmesh = (3, 3, 3)
    EF = np.array([0.2])
    outs, sched, status = kubo.ahc_batched([(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, EF))],
                                           tune=True)
    assert status == ["KUBO_OK"] and sched["streams"] == 1
    assert rel(outs[0].cpu().numpy(), O.ahc(m.H_R, m.R, kmesh, EF)) < 1e-10
