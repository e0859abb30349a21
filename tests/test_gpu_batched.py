"""kubo_ahc_batched: many models of uneven W, N_R and k-mesh in one call.

Checks: every model of a mixed batch against the FP64 oracle (relative 1e-10 in FP64, 1e-5
mixed); the batch against one kubo_ahc call per model; graph and direct issue give
identical results for the same schedule; the autotuner times candidates once per batch
signature and its schedule gives the same sums; a non-Hermitian model is reported in its
own status while the rest of the batch runs.
"""
import ctypes

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


def median_level_at_gamma(m):
    """The recipe's Fermi level "at the median band energy", read as the midpoint of the two
    middle levels of H(k = 0) (levels ceil(W/2) - 1 and ceil(W/2), ascending; the median for
    even W).  For odd W the median itself is a level at k = 0, a mesh point, where the step
    occupation would be decided by rounding.  Computed by the oracle."""
    Hk, _, _ = O.bloch(m.H_R, m.R, (1, 1, 1), np.array([0]))
    E = O.eigh(Hk)[0][0]
    W = E.size
    if W == 1:
        return float(E[0]) + 1.0
    h = (W + 1) // 2
    return float(0.5 * (E[h - 1] + E[h]))


SMALL = [  # (W, half_width, mesh, seed): uneven orders (incl. > 64), R boxes and meshes
    (3, 1, (4, 3, 5), 1), (8, 2, (5, 5, 4), 2), (17, 1, (6, 4, 4), 3),
    (40, 2, (3, 4, 3), 4), (64, 1, (4, 4, 2), 5), (72, 1, (3, 3, 3), 6),
]


@pytest.fixture(scope="module")
def small_batch():
    out = []
    for W, h, mesh, seed in SMALL:
        m = tbgen.random_tb(W, h, 1.5, seed)
        out.append((m, mesh, np.array([median_level_at_gamma(m), 0.3])))
    return out


def problems(torch, batch):
    return [(cuda(torch, m.H_R), m.R, mesh, cuda(torch, ef)) for m, mesh, ef in batch]


def test_batched_fp64_matches_oracle(kubo, torch, small_batch):
    etas = [1e-3, 2e-2]
    outs, sched, status = kubo.ahc_batched(problems(torch, small_batch), etas=etas, streams=3)
    assert status == ["KUBO_OK"] * len(SMALL)
    assert sched["streams"] == 3 and sched["graph"] == 1
    for (m, mesh, ef), S in zip(small_batch, outs):
        ref = O.ahc(m.H_R, m.R, mesh, ef, etas=etas)
        assert np.max(np.abs(S.cpu().numpy() - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_batched_matches_single_model_calls(kubo, torch, small_batch):
    outs, _, _ = kubo.ahc_batched(problems(torch, small_batch), kT=0.05, streams=2)
    for (m, mesh, ef), S in zip(small_batch, outs):
        one = kubo.ahc(cuda(torch, m.H_R), m.R, mesh, cuda(torch, ef), kT=0.05).cpu().numpy()
        assert np.max(np.abs(S.cpu().numpy() - one)) <= 1e-13 * np.max(np.abs(one))


def test_graph_and_direct_issue_are_identical(kubo, torch, small_batch):
    P = problems(torch, small_batch)
    a, _, _ = kubo.ahc_batched(P, streams=4, chunk_k=16, graph=True)    # several batches per model
    b, sb, _ = kubo.ahc_batched(P, streams=4, chunk_k=16, graph=False)
    assert sb["graph"] == -1
    for x, y in zip(a, b):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_autotuner_runs_once_per_signature(kubo, torch, small_batch):
    P = problems(torch, small_batch)
    ref, _, _ = kubo.ahc_batched(P, streams=1, chunk_k=65536)
    a, s1, _ = kubo.ahc_batched(P, tune=True)
    b, s2, _ = kubo.ahc_batched(P, tune=True)
    assert s1["tuned_candidates"] >= 2 and s1["probe_ms"] > 0
    assert s2["tuned_candidates"] == 0
    assert (s1["streams"], s1["chunk_k"]) == (s2["streams"], s2["chunk_k"])
    # the tuner also chose the reduction's symv partition cap (FP64: no tensor-core Fourier sum,
    # no FP32 rotation to tune), and the cached schedule carries it
    assert s1["symv_parts"] in (2, 4, 8) and s1["symv_parts"] == s2["symv_parts"]
    assert s1["fourier_group_m"] == 8 and s1["rotation"] == 0
    for x, y, r in zip(a, b, ref):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())
        rr = r.cpu().numpy()
        assert np.max(np.abs(x.cpu().numpy() - rr)) <= 1e-12 * np.max(np.abs(rr))


def test_autotuned_kernel_parameters_mixed(kubo, torch, small_batch):
    """Mixed batch: the tuner picks the Fourier rasterisation group, the symv partition cap and
    the rotation kernel as well; every choice stays within the mixed tolerance, and fixed
    parameters are respected and reported."""
    P = problems(torch, small_batch)
    outs, sc, _ = kubo.ahc_batched(P, precision="mixed", tune=True)
    assert sc["tuned_candidates"] >= 2 + 6
    assert sc["fourier_group_m"] in (4, 8, 16)
    assert sc["symv_parts"] in (2, 4, 8)
    assert sc["rotation"] in (0, 2, 3)
    for (m, mesh, ef), S in zip(small_batch, outs):
        ref = O.ahc(m.H_R, m.R, mesh, ef)
        assert np.max(np.abs(S.cpu().numpy() - ref)) <= 1e-5 * np.max(np.abs(ref))
    fixed, sf, _ = kubo.ahc_batched(P, precision="mixed", streams=2, chunk_k=8192,
                                   fourier_group_m=2, symv_parts=1, rotation="tf32")
    assert (sf["fourier_group_m"], sf["symv_parts"], sf["rotation"]) == (2, 1, 3)
    for (m, mesh, ef), S in zip(small_batch, fixed):
        ref = O.ahc(m.H_R, m.R, mesh, ef)
        assert np.max(np.abs(S.cpu().numpy() - ref)) <= 1e-5 * np.max(np.abs(ref))
    # the rasterisation order does not change any tile's sums
    g4, _, _ = kubo.ahc_batched(P, precision="mixed", streams=2, chunk_k=8192, fourier_group_m=4,
                                symv_parts=4, rotation="simt")
    g16, _, _ = kubo.ahc_batched(P, precision="mixed", streams=2, chunk_k=8192, fourier_group_m=16,
                                 symv_parts=4, rotation="simt")
    for x, y in zip(g4, g16):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_mixed_precision_batch(kubo, torch, small_batch):
    outs, _, _ = kubo.ahc_batched(problems(torch, small_batch), precision="mixed", streams=2)
    for (m, mesh, ef), S in zip(small_batch, outs):
        ref = O.ahc(m.H_R, m.R, mesh, ef)
        assert np.max(np.abs(S.cpu().numpy() - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_non_hermitian_model_is_reported_and_the_rest_runs(kubo, torch, small_batch):
    P = problems(torch, small_batch)
    bad = P[2][0].clone()
    bad[0, 0, 1] += 0.5            # breaks H(-R) = H(R)^dagger for R = (-1,-1,-1)
    P[2] = (bad,) + P[2][1:]
    with pytest.raises(kubo.KuboError) as ei:
        kubo.ahc_batched(P, streams=2)
    assert ei.value.name == "KUBO_ERR_NOT_HERMITIAN"
    # the same batch through the C ABI: per-model statuses, good models computed
    n = len(P)
    arr = (kubo.Problem * n)()
    keep, outs = [], []
    for i, (H, R, mesh, ef) in enumerate(P):
        Rh = np.ascontiguousarray(R, dtype=np.int32)
        keep.append(Rh)
        out = torch.full((1, ef.numel()), 7.0, dtype=torch.float64, device="cuda:0")
        outs.append(out)
        a = arr[i]
        a.H_R, a.R_vecs = H.data_ptr(), Rh.ctypes.data
        a.W, a.N_R = H.shape[1], H.shape[0]
        for q in range(3):
            a.kmesh[q] = mesh[q]
        a.E_F, a.n_EF, a.eta, a.out = ef.data_ptr(), ef.numel(), 1e-3, out.data_ptr()
    o = kubo.Options()
    kubo.lib().kubo_options_init(ctypes.byref(o))
    o.stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = kubo.lib().kubo_ahc_batched(arr, n, ctypes.byref(o), None)
    assert code == 2
    assert [arr[i].status for i in range(n)] == [0, 0, 2, 0, 0, 0]
    assert np.all(outs[2].cpu().numpy() == 7.0)           # untouched
    m, mesh, ef = small_batch[4]
    ref = O.ahc(m.H_R, m.R, mesh, ef)
    assert np.max(np.abs(outs[4].cpu().numpy() - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_batch_recipe_shapes_reduced_meshes(kubo, torch):
    """All 64 model shapes of the uneven batch (W 8..96, N_R 343..1331) on 4^3 meshes:
    the batch agrees with one call per model; a sample of models agrees with the oracle."""
    rec = tbgen.batch_recipe()
    models = [tbgen.random_tb(r["W"], r["half_width"], r["decay"], r["seed"]) for r in rec]
    efs = [np.array([median_level_at_gamma(m)]) for m in models]
    mesh = (4, 4, 4)
    P = [(cuda(torch, m.H_R), m.R, mesh, cuda(torch, ef)) for m, ef in zip(models, efs)]
    outs, sched, status = kubo.ahc_batched(P, streams=8)
    assert status == ["KUBO_OK"] * 64
    for i in (0, 17, 40):
        one = kubo.ahc(P[i][0], models[i].R, mesh, P[i][3]).cpu().numpy()
        assert np.max(np.abs(outs[i].cpu().numpy() - one)) <= 1e-13 * np.max(np.abs(one))
    for i in (3, 29):
        ref = O.ahc(models[i].H_R, models[i].R, mesh, efs[i])
        assert np.max(np.abs(outs[i].cpu().numpy() - ref)) <= 1e-10 * np.max(np.abs(ref))
