"""Mixed-precision path (tensor-core Fourier sum with fixed-point BF16 slices, FP32 rotations,
FP64 eigenvectors and eigenvalues, denominators and k-sum) against the FP64 oracle and the FP64 GPU path; the
double-float eigensolver variant (MIXED_DF) to the same tolerance.

Tolerance: relative 1e-5 on S(E_F) (max over E_F of |diff| / max |S_ref|).  The tensor-core
Fourier sum itself is exact up to its 31-bit fixed-point slicing: 2e-8 relative to max |H|
(split-BF16 products with FP32 accumulation reach ~3e-7 on the same workload).
"""
import json
import os

import numpy as np
import pytest

import tbgen
from oracle import kubo_oracle as O

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
REL_MIXED = 1e-5


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


@pytest.fixture(scope="module")
def m64():
    return tbgen.random_tb(64, 5, 1.5, 0)


@pytest.mark.parametrize("W,hw,n", [(16, 2, 37), (8, 1, 130), (20, 1, 129), (64, 5, 200)])
def test_tensor_core_fourier_sum(kubo, torch, W, hw, n):
    """Step (1) on tcgen05 vs the oracle: ragged k counts (not multiples of the 128-row tile),
    orders whose 3 W^2 columns are not multiples of the 128-column tile."""
    m = tbgen.random_tb(W, hw, 1.5, seed=W)
    kmesh = (17, 11, 13)
    kidx = tbgen.k_sample(kmesh, n, seed=3)
    got = kubo.bloch(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, kidx), precision="mixed")
    ref = O.bloch(m.H_R, m.R, kmesh, kidx)
    for g, r in zip(got, ref):
        G = kubo.unpack_hermitian(g, W).cpu().numpy()
        assert rel_err(G, r) < 2e-8, rel_err(G, r)


def test_mixed_w16_full_mesh_vs_golden(kubo, torch):
    g = json.load(open(os.path.join(GOLDEN, "w16_r125_k24.json")))
    m = tbgen.random_tb(16, 2, 1.0, 0)
    S = kubo.ahc(cuda(torch, m.H_R), m.R, (24, 24, 24), cuda(torch, np.array(g["E_F"])),
                 etas=g["etas"], precision="mixed").cpu().numpy()
    assert rel_err(S, np.array(g["S"])) < REL_MIXED


@pytest.mark.parametrize("prec", ["mixed", "mixed_df"])
def test_mixed_per_k_w64(kubo, torch, m64, prec):
    """Per-k parity on 200 k-points of the 128^3 mesh of the W = 64, N_R = 1331 model.

    Error budget per k (relative to ||Omega(k)||_inf): the FP64 (or pair) eigenvalues are
    within ~1e-12 of the oracle's, so the denominators are exact to FP64 grade; the FP32
    rotation rounds U and dH to 2^-24 and accumulates W = 64 products, so each v_nm carries
    ~sqrt(W) 2^-24 ||dH|| ~ 5e-7 ||dH|| of absolute error and a pair term T_nm = -2 Im(v v) /
    (dE^2 + eta^2) a relative error of ~1e-6 ||dH||^2 / |v_nm v_mn|.  The dominant pair of a
    k-point has |v_nm| ~ ||dH|| / 10, so ~1e-4 at worst; the median k-point sits near 1e-6."""
    kmesh = (128, 128, 128)
    kidx = tbgen.k_sample(kmesh, 200, seed=21)
    E, Om = kubo.ahc_k(cuda(torch, m64.H_R), m64.R, kmesh, cuda(torch, kidx), eta=1e-3,
                       precision=prec)
    E_ref, Om_ref = O.kubo_per_k(m64.H_R, m64.R, kmesh, kidx, [1e-3])
    E, Om = E.cpu().numpy(), Om.cpu().numpy()[0]
    # the eigenvalues inherit the tensor-core H(k)'s ~2^-31 entry error (||dH||_2 <= W max|dH|)
    assert np.max(np.abs(E - E_ref)) <= 1e-7 * np.max(np.abs(E_ref)), np.max(np.abs(E - E_ref))
    scale = np.max(np.abs(Om_ref[0]), axis=-1)
    err = np.max(np.abs(Om - Om_ref[0]), axis=-1) / scale
    print(f"{prec}: per-k Omega error max {np.max(err):.3e} median {np.median(err):.3e} "
          f"E error {np.max(np.abs(E - E_ref)) / np.max(np.abs(E_ref)):.3e}")
    assert np.max(err) < 1e-4, np.max(err)
    assert np.median(err) < 3e-6, np.median(err)


def test_mixed_vs_fp64_on_a_mesh_plane_w64(kubo, torch, m64):
    """One k1-plane (16,384 k-points) of the 128^3 mesh, 64 Fermi levels: the benchmark's
    batch configuration, mixed (and its double-float eigensolver variant) vs FP64 GPU."""
    kmesh = (128, 128, 128)
    EF = np.linspace(-1.0, 1.0, 64)
    H = cuda(torch, m64.H_R)
    EFt = cuda(torch, EF)
    rng = (37 * 16384, 38 * 16384)
    S64 = kubo.ahc(H, m64.R, kmesh, EFt, eta=1e-3, k_range=rng).cpu().numpy()
    Smx = kubo.ahc(H, m64.R, kmesh, EFt, eta=1e-3, k_range=rng, precision="mixed").cpu().numpy()
    assert rel_err(Smx, S64) < REL_MIXED, rel_err(Smx, S64)
    Sdf = kubo.ahc(H, m64.R, kmesh, EFt, eta=1e-3, k_range=rng, precision="mixed_df").cpu().numpy()
    assert rel_err(Sdf, S64) < REL_MIXED, rel_err(Sdf, S64)
    # the tensor-core Fourier sum alone is FP64-grade: only the FP32 rotations remain
    Sfo = kubo.ahc(H, m64.R, kmesh, EFt, eta=1e-3, k_range=rng,
                   precision="mixed_fourier").cpu().numpy()
    assert rel_err(Sfo, S64) < 1e-6, rel_err(Sfo, S64)


def test_mixed_fixup_redoes_flagged_k_points_in_fp64(kubo, torch, m64):
    """Opt-in fix-up: k-points with a level near a Fermi level, or in the top 0.5 % of
    ||Omega(k)||, are recomputed on the FP64 path and overwrite their mixed results."""
    kmesh = (128, 128, 128)
    EF = np.linspace(-1.0, 1.0, 64)
    H = cuda(torch, m64.H_R)
    EFt = cuda(torch, EF)
    rng = (90 * 16384, 90 * 16384 + 5000)
    S64 = kubo.ahc(H, m64.R, kmesh, EFt, eta=1e-3, k_range=rng).cpu().numpy()
    prof = kubo.Profile()
    Sfx = kubo.ahc(H, m64.R, kmesh, EFt, eta=1e-3, k_range=rng, precision="mixed",
                   profile=prof, fixup_rel=4e-6, chunk_k=1500).cpu().numpy()
    assert 0 < prof.fixup_k < 0.1 * 5000
    assert prof.launches[kubo.STAGES.index("fixup")] > 0
    assert rel_err(Sfx, S64) < REL_MIXED


def test_mixed_multi_eta_fermi_dirac_ragged(kubo, torch):
    m = tbgen.random_tb(12, 1, 1.0, 5)
    kmesh = (7, 6, 5)
    EF = np.array([-0.3, 0.2, 1e3])
    etas = [1e-3, 5e-3, 1e-2]
    for kT in (0.0, 0.025):
        S = kubo.ahc(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, EF), etas=etas, kT=kT,
                     precision="mixed", chunk_k=61).cpu().numpy()
        S_ref = O.ahc(m.H_R, m.R, kmesh, EF, etas=etas, kT=kT)
        assert rel_err(S, S_ref) < REL_MIXED


def test_mixed_haldane_chern(kubo, torch):
    """Quantised Chern number through the mixed path (single layer, eta = 0; exactly degenerate
    stacked copies at eta = 0 are ill-conditioned once H carries FP32-level errors)."""
    m = tbgen.haldane()
    S = kubo.ahc(cuda(torch, m.H_R), m.R, (96, 96, 1), cuda(torch, np.array([0.0])), eta=0.0,
                 precision="mixed")
    C = 2 * np.pi * S.cpu().numpy()[0, 0]
    assert abs(abs(C) - 1) < 1e-5


def test_rotation_kernels_vs_fp64(kubo, torch, m64):
    """Step (3) on the tensor cores in 3xTF32 (the default at W = 64), with exact fixed-point
    BF16-slice products, and in FP32 on the FMA pipe, against the FP64 path on a slab of the W = 64
    workload: all three within 1e-5 of FP64 (one accuracy class), through the FP64 Fourier
    sum (MIXED_ROTATION) and the tensor-core one (MIXED)."""
    kmesh = (128, 128, 128)
    EF = cuda(torch, np.linspace(-1.0, 1.0, 64))
    H = cuda(torch, m64.H_R)
    rng = (77 * 16384, 77 * 16384 + 8192)
    S64 = kubo.ahc(H, m64.R, kmesh, EF, k_range=rng).cpu().numpy()
    errs = {}
    for prec in ("mixed_rotation", "mixed"):
        for rot in ("tf32", "exact", "simt"):
            S = kubo.ahc(H, m64.R, kmesh, EF, k_range=rng, precision=prec, rotation=rot,
                         chunk_k=3000).cpu().numpy()
            errs[(prec, rot)] = rel_err(S, S64)
    print({f"{a}/{b}": f"{e:.2e}" for (a, b), e in errs.items()})
    for key, e in errs.items():
        assert e < 1e-5, (key, e)
    # with a fresh accumulator per K-quarter the 3xTF32 products are FP32-grade: no less
    # accurate than the FP32 FMA rotation (measured 2.4e-7 vs 4.3e-7 with the FP64 Fourier sum)
    assert errs[("mixed_rotation", "tf32")] <= 1.5 * errs[("mixed_rotation", "simt")]


@pytest.mark.parametrize("prec", ["mixed_rotation", "mixed"])
@pytest.mark.parametrize("rot", ["tf32", "exact"])
@pytest.mark.parametrize("W", [5, 16, 33, 64])
def test_tensor_core_rotation_small_orders_per_k(kubo, torch, W, rot, prec):
    """Per-k parity of the tensor-core rotations at orders padded to 64, odd ones included:
    from the FP64 Fourier sum (MIXED_ROTATION: FP64 velocity rows, U assembled inside the
    kernel) and from the tensor-core one (MIXED: FP32 velocity rows, 3xTF32 with U formed by
    its own kernel)."""
    m = tbgen.random_tb(W, 2 if W < 64 else 1, 1.2, 300 + W)
    kmesh = (16, 16, 16)
    kidx = tbgen.k_sample(kmesh, 150, seed=W)
    E, Om = kubo.ahc_k(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, kidx), etas=[1e-3, 0.05],
                       precision=prec, rotation=rot)
    E_ref, Om_ref = O.kubo_per_k(m.H_R, m.R, kmesh, kidx, [1e-3, 0.05])
    # FP64 Fourier sum: FP64-grade eigenvalues; tensor-core one: its 2^-31 slicing of H(k)
    etol = 1e-12 if prec == "mixed_rotation" else 1e-7
    assert np.max(np.abs(E.cpu().numpy() - E_ref)) <= etol * np.max(np.abs(E_ref))
    for e in range(2):
        scale = np.max(np.abs(Om_ref[e]), axis=-1)
        err = np.max(np.abs(Om.cpu().numpy()[e] - Om_ref[e]), axis=-1) / scale
        assert np.median(err) < 1e-5, np.median(err)
        assert np.max(err) < 1e-3, np.max(err)


def test_tf32_rotation_many_broadenings_and_ragged_persistent_grid(kubo, torch):
    """Eight broadenings (the curvature's partials then exceed the operand stage, one CTA per
    SM) and k counts that leave the persistent grid's last round ragged."""
    m = tbgen.random_tb(24, 1, 1.0, 77)
    kmesh = (9, 7, 5)
    etas = [0.0, 1e-5, 1e-4, 1e-3, 5e-3, 1e-2, 5e-2, 0.2]
    EF = np.array([-0.6, 0.0, 0.4])
    for chunk in (1, 97, 315):
        S = kubo.ahc(cuda(torch, m.H_R), m.R, kmesh, cuda(torch, EF), etas=etas,
                     precision="mixed", chunk_k=chunk, rotation="tf32").cpu().numpy()
        ref = O.ahc(m.H_R, m.R, kmesh, EF, etas=etas)
        for e in range(len(etas)):
            assert rel_err(S[e], ref[e]) < REL_MIXED, (chunk, e, rel_err(S[e], ref[e]))


@pytest.mark.parametrize("W,hw", [(2, 1), (5, 2), (33, 1), (64, 5), (100, 1)])
def test_double_float_eigenvalues(kubo, torch, W, hw):
    """The MIXED_DF mode's double-float eigenvalues (Householder reduction and QL iteration in
    FP32 pairs) against the FP64 ones: MIXED_DF and MIXED read the same tensor-core rows of H
    and differ only there.  Bound: the reduction's backward error ~W 2^-46 max|E| plus at
    most W deflations of the QL at |e| <= 2^-44 (|d_m| + |d_m+1|), each moving the eigenvalues
    by at most |e| (Weyl): 16 W 2^-46 max|E| in all."""
    m = tbgen.random_tb(W, hw, 1.5, 500 + W)
    kmesh = (16, 16, 16)
    kidx = tbgen.k_sample(kmesh, 97, seed=W)
    H, K = cuda(torch, m.H_R), cuda(torch, kidx)
    Emx, _ = kubo.ahc_k(H, m.R, kmesh, K, precision="mixed_df")
    Efx, _ = kubo.ahc_k(H, m.R, kmesh, K, precision="mixed")
    Emx, Efx = Emx.cpu().numpy(), Efx.cpu().numpy()
    scale = np.max(np.abs(Efx))
    assert np.max(np.abs(Emx - Efx)) <= 16 * W * 2.0 ** -46 * scale, \
        np.max(np.abs(Emx - Efx)) / scale


@pytest.mark.parametrize("W,hw,layers", [(2, 1, 1), (5, 2, 1), (33, 1, 1), (64, 5, 1),
                                         (100, 1, 1), (4, 1, 2)])
def test_rayleigh_quotient_eigenvalues(kubo, torch, W, hw, layers):
    """MIXED reports the FP64 Rayleigh quotients z^T T z of its FP64 inverse-iteration vectors
    (its QL iteration, in FP32 pairs, only supplies the shifts); MIXED_FOURIER reads the same
    tensor-core rows of H and takes its eigenvalues from the FP64 QL iteration.  Both are
    backward stable for the same tridiagonal T, so they agree to a few W eps ||T||; the
    quotients of a unit vector with residual r lie within ||r|| of an eigenvalue, and the
    reported levels stay ascending.  layers = 2: exactly degenerate pairs (a doubled model)."""
    if layers == 1:
        m = tbgen.random_tb(W, hw, 1.5, 700 + W)
    else:
        m = tbgen.stack_layers(tbgen.qwz(-1.2, tz=0.3, c0=0.2), 2)
        W = m.H_R.shape[-1]
    kmesh = (16, 16, 16)
    kidx = tbgen.k_sample(kmesh, 97, seed=W + 1)
    H, K = cuda(torch, m.H_R), cuda(torch, kidx)
    Erq, _ = kubo.ahc_k(H, m.R, kmesh, K, precision="mixed")
    Eql, _ = kubo.ahc_k(H, m.R, kmesh, K, precision="mixed_fourier")
    Erq, Eql = Erq.cpu().numpy(), Eql.cpu().numpy()
    scale = np.max(np.abs(Eql))
    assert np.all(np.diff(Erq, axis=-1) >= 0)
    assert np.max(np.abs(Erq - Eql)) <= 16 * W * 2.0 ** -52 * scale, \
        np.max(np.abs(Erq - Eql)) / scale


def test_mixed_with_fp64_ql_option(kubo, torch, m64):
    """kubo_options.ql_fp64 = 1 keeps the MIXED mode's QL iteration in FP64 and reports its
    eigenvalues: the eigenvalues agree with the default's Rayleigh quotients within a few
    W eps max|E| and S(E_F) to rounding (both eigensolvers FP64-accurate)."""
    kmesh = (128, 128, 128)
    H = cuda(torch, m64.H_R)
    kidx = cuda(torch, tbgen.k_sample(kmesh, 300, seed=5))
    Erq, Orq = kubo.ahc_k(H, m64.R, kmesh, kidx, precision="mixed")
    Eql, Oql = kubo.ahc_k(H, m64.R, kmesh, kidx, precision="mixed", ql_fp64=True)
    Erq, Eql = Erq.cpu().numpy(), Eql.cpu().numpy()
    assert np.max(np.abs(Erq - Eql)) <= 16 * 64 * 2.0 ** -52 * np.max(np.abs(Eql))
    EF = cuda(torch, np.linspace(-1.0, 1.0, 64))
    rng = (11 * 16384, 11 * 16384 + 4096)
    S0 = kubo.ahc(H, m64.R, kmesh, EF, k_range=rng, precision="mixed").cpu().numpy()
    S1 = kubo.ahc(H, m64.R, kmesh, EF, k_range=rng, precision="mixed", ql_fp64=True).cpu().numpy()
    assert rel_err(S1, S0) < 1e-9, rel_err(S1, S0)


def test_double_float_reduction_degenerate_bands(kubo, torch):
    """Exactly degenerate bands (two identical layers): the double-float reduction keeps the
    pairs degenerate to its precision and the curvature sums match the FP64 path."""
    m = tbgen.stack_layers(tbgen.qwz(-1.2, tz=0.3, c0=0.2), 2)
    kmesh = (24, 24, 4)
    EF = cuda(torch, np.array([-0.5, 0.1, 0.7]))
    H = cuda(torch, m.H_R)
    S64 = kubo.ahc(H, m.R, kmesh, EF, eta=0.05).cpu().numpy()
    Smx = kubo.ahc(H, m.R, kmesh, EF, eta=0.05, precision="mixed_df").cpu().numpy()
    assert rel_err(Smx, S64) < REL_MIXED, rel_err(Smx, S64)
