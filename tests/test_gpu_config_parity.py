"""S(E_F) against the oracle on the exact workload models, and the failure paths on the GPU.

* Config-level parity (Eq. 2 summed over a k-range of the real workload, weight 1/N_k):
  the W = 64, N_R = 1331 model (64 Fermi levels, eta = 1e-3), the W = 32, N_R = 729 model
  (Fermi-Dirac kT = 25 meV, eta = 5e-3) and the W = 128, N_R = 1331 model (512 Fermi levels x
  4 broadenings), each on a few thousand k-points of its own mesh, with ragged batches.
  Tolerance: 1e-10 relative in FP64, 1e-5 in every reduced-precision mode (max over Fermi
  levels of |diff| / max |S_ref|, per broadening).
* theta(0): a level exactly at E_F is empty, on the GPU as in the oracle.
* Magnitude range: H(R), E_F, eta, kT scaled by 2^+-46 and 2^+-83; S must not change.
* Failure paths made on the host: a QL sweep cap (KUBO_ERR_NO_CONVERGENCE) and a simulated
  allocation failure (KUBO_ERR_OOM), each leaving the output untouched and the next call fine.
"""
import numpy as np
import pytest

import tbgen
from oracle import kubo_oracle as O

pytestmark = pytest.mark.gpu

MIXED_MODES = ["mixed", "mixed_df", "mixed_fourier", "mixed_rotation"]


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


def rel_rows(a, b):
    """max over broadenings of max_j |a - b| / max_j |b| (reading of the 1e-5 target)."""
    a, b = np.atleast_2d(a), np.atleast_2d(b)
    return max(np.max(np.abs(a[e] - b[e])) / max(np.max(np.abs(b[e])), 1e-300) for e in range(b.shape[0]))


def _range_parity(kubo, torch, name, n_k, start, modes, chunk):
    model, kmesh, E_F, etas, kT = tbgen.config(name)
    H, EF = cuda(torch, model.H_R), cuda(torch, E_F)
    rng = (start, start + n_k)
    ref = O.ahc(model.H_R, model.R, kmesh, E_F, etas=etas, kT=kT, kidx=np.arange(*rng))
    errs = {}
    for prec in modes:
        S = kubo.ahc(H, model.R, kmesh, EF, etas=list(etas), kT=kT, precision=prec, k_range=rng,
                     chunk_k=chunk).cpu().numpy()
        errs[prec] = rel_rows(S, ref)
    print(name, {k: f"{v:.2e}" for k, v in errs.items()})
    for prec, e in errs.items():
        assert e < (1e-10 if prec == "fp64" else 1e-5), (prec, e)


def test_sigma_w64_r1331_k128_64_fermi_levels(kubo, torch):
    """4096 k-points of the 128^3 mesh (crossing a k1-plane boundary), batches of 1500."""
    _range_parity(kubo, torch, "w64_r1331_k128", 4096, 37 * 16384 - 1000,
                  ["fp64", "mixed", "mixed_df"], 1500)


def test_sigma_w32_r729_k48_fermi_dirac(kubo, torch):
    _range_parity(kubo, torch, "w32_r729_k48_fd", 4096, 20 * 48 * 48 + 333, ["fp64"], 1777)


def test_sigma_w128_r1331_k96_sweep(kubo, torch):
    """512 Fermi levels x 4 broadenings on 1024 k-points of the 96^3 mesh."""
    _range_parity(kubo, torch, "w128_r1331_k96", 1024, 48 * 96 * 96 + 4000,
                  ["fp64", "mixed", "mixed_df"], 384)


# ---------------------------------------------------------------- theta(0)
@pytest.mark.parametrize("prec", ["fp64"] + MIXED_MODES)
def test_level_exactly_at_fermi_energy_is_empty(kubo, torch, prec):
    """QWZ, m = -3/2 at Gamma: levels exactly -1/2 and +1/2, Omega_lower = 2 (closed form,
    eta = 0).  S(+1/2) = 2 / N_k (strict theta; "<=" gives 0), S(-1/2) = 0 ("<=" gives 2 / N_k),
    S(3/4) = 0 (both bands: the sum rule)."""
    m = tbgen.qwz(-1.5)
    kmesh, Nk = (8, 8, 1), 64
    H = cuda(torch, m.H_R)
    E, Om = kubo.ahc_k(H, m.R, kmesh, torch.zeros(1, dtype=torch.int64, device="cuda:0"),
                       eta=0.0, precision=prec)
    assert E.cpu().numpy().tolist() == [[-0.5, 0.5]]
    S = kubo.ahc(H, m.R, kmesh, cuda(torch, np.array([-0.5, 0.5, 0.75])), eta=0.0,
                 precision=prec, k_range=(0, 1)).cpu().numpy()[0]
    tol = 1e-13 if prec in ("fp64", "mixed_fourier") else 1e-6
    assert S[0] == 0.0
    assert abs(S[1] * Nk - 2.0) < 2.0 * tol, S[1] * Nk
    assert abs(S[2] * Nk) < 2.0 * tol, S[2] * Nk


# ---------------------------------------------------------------- magnitude range
@pytest.mark.parametrize("prec", ["mixed", "mixed_df", "mixed_rotation"])
@pytest.mark.parametrize("lg", [-83, -46, 46, 83])
def test_reduced_precision_modes_have_no_magnitude_range(kubo, torch, prec, lg):
    """H(R), E_F, eta and kT scaled by 2^lg (exact): S is unchanged in exact arithmetic, and
    the FP64 path reproduces it; the modes with FP32 steps must too (2^+-83 squares leave the
    FP32 range, so without the library's internal rescaling they would fail)."""
    m = tbgen.random_tb(16, 2, 1.0, 0)
    kmesh = (6, 5, 4)
    EF = np.array([-0.5, 0.0, 0.7])
    etas = [1e-2, 5e-2]
    f = 2.0 ** lg
    for kT in (0.0, 0.02):
        ref = kubo.ahc(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, EF), etas=etas, kT=kT,
                       chunk_k=37).cpu().numpy()
        S = kubo.ahc(cuda(torch, m.H_R * f), m.R, kmesh, cuda(torch, EF * f),
                     etas=[e * f for e in etas], kT=kT * f, precision=prec,
                     chunk_k=37).cpu().numpy()
        assert np.all(np.isfinite(S))
        assert rel_rows(S, ref) < 1e-5, (prec, lg, kT, rel_rows(S, ref))
    # per-k eigenvalues come back in the caller's units
    kidx = cuda(torch, np.array([0, 7, 55, 119], dtype=np.int64))
    E64, _ = kubo.ahc_k(cuda(torch, m.H_R), m.R, kmesh, kidx, eta=1e-2)
    E, _ = kubo.ahc_k(cuda(torch, m.H_R * f), m.R, kmesh, kidx, eta=1e-2 * f, precision=prec)
    assert np.max(np.abs(E.cpu().numpy() / f - E64.cpu().numpy())) < 1e-7 * np.max(np.abs(E64.cpu().numpy()))


def test_batched_models_of_very_different_magnitudes(kubo, torch):
    m = tbgen.random_tb(12, 1, 1.0, 3)
    kmesh = (5, 4, 3)
    EF = np.array([-0.4, 0.3])
    ref = O.ahc(m.H_R, m.R, kmesh, EF, etas=[0.02])
    probs = []
    for lg in (-83, 0, 83):
        f = 2.0 ** lg
        probs.append((cuda(torch, m.H_R * f), m.R, kmesh, cuda(torch, EF * f), 0.02 * f))
    outs, _, status = kubo.ahc_batched(probs, precision="mixed", streams=2)
    assert status == ["KUBO_OK"] * 3
    for o in outs:
        assert rel_rows(o.cpu().numpy(), ref) < 1e-5


# ---------------------------------------------------------------- failure paths
@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_df"])
def test_ql_sweep_cap_reports_no_convergence_and_leaves_out_untouched(kubo, torch, prec):
    m = tbgen.random_tb(16, 2, 1.0, 11)
    kmesh = (4, 4, 4)
    H, EF = cuda(torch, m.H_R), cuda(torch, np.array([0.0, 0.5]))
    out = torch.full((1, 2), 12345.0, dtype=torch.float64, device="cuda:0")
    with pytest.raises(kubo.KuboError) as ei:
        kubo.ahc(H, m.R, kmesh, EF, precision=prec, out=out, ql_max_sweeps=1)
    assert ei.value.name == "KUBO_ERR_NO_CONVERGENCE"
    assert torch.all(out == 12345.0)
    # the default cap converges, on the same context
    S = kubo.ahc(H, m.R, kmesh, EF, precision=prec).cpu().numpy()
    ref = O.ahc(m.H_R, m.R, kmesh, [0.0, 0.5])
    assert rel_rows(S, ref) < (1e-10 if prec == "fp64" else 1e-5)


def test_ql_sweep_cap_in_the_eigensolver_entry_point(kubo, torch):
    rng = np.random.default_rng(5)
    X = rng.standard_normal((20, 24, 24)) + 1j * rng.standard_normal((20, 24, 24))
    A = kubo.pack_hermitian(cuda(torch, X + np.conj(np.swapaxes(X, -1, -2))))
    with pytest.raises(kubo.KuboError) as ei:
        kubo.eigh_batched(A, 24, ql_max_sweeps=1)
    assert ei.value.name == "KUBO_ERR_NO_CONVERGENCE"
    E, _ = kubo.eigh_batched(A, 24)
    assert torch.isfinite(E).all()


def test_simulated_allocation_failure(kubo, torch):
    m = tbgen.random_tb(8, 1, 1.0, 12)
    kmesh = (3, 3, 3)
    H, EF = cuda(torch, m.H_R), cuda(torch, np.array([0.1]))
    out = torch.full((1, 1), -7.0, dtype=torch.float64, device="cuda:0")
    kubo.debug_fail_allocations(1)
    try:
        with pytest.raises(kubo.KuboError) as ei:
            kubo.ahc(H, m.R, kmesh, EF, out=out, precision="mixed")
        assert ei.value.name == "KUBO_ERR_OOM"
        assert torch.all(out == -7.0)
        kubo.debug_fail_allocations(1)
        with pytest.raises(kubo.KuboError) as ei:
            kubo.ahc_batched([(H, m.R, kmesh, EF)])
        assert ei.value.name == "KUBO_ERR_OOM"
    finally:
        kubo.debug_fail_allocations(0)
    S = kubo.ahc(H, m.R, kmesh, EF, out=out).cpu().numpy()
    assert rel_rows(S, O.ahc(m.H_R, m.R, kmesh, [0.1])) < 1e-10
