"""Pins of the FP64 oracle against facts fixed by the paper and the mathematics.

None of these re-types the oracle's formula: each compares it with something
independent of it -- a closed form of a two-band model, a published Chern number,
an invariant of Eq. 3, a finite difference, or a Berry phase around a small loop
(a geometric quantity the Kubo sum must reproduce).
"""
import json
import math
import os

import numpy as np
import pytest

import tbgen
from oracle import kubo_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- two-band closed forms
def _qwz_d(kf, m, tz=0.0, c0=0.0):
    k1, k2, k3 = (2 * np.pi * kf[:, a] for a in range(3))
    d0 = c0 * np.cos(k1 + k2)
    d = np.stack([np.sin(k1), np.sin(k2), m + np.cos(k1) + np.cos(k2) + tz * np.cos(k3)], -1)
    dx = np.stack([np.cos(k1), 0 * k1, -np.sin(k1)], -1)
    dy = np.stack([0 * k2, np.cos(k2), -np.sin(k2)], -1)
    return d0, d, dx, dy


def _mesh_frac(kmesh):
    """Fractional k of every mesh point in linear-index order (j3 fastest), built by loops."""
    import itertools
    N1, N2, N3 = kmesh
    return np.array([(a / N1, b / N2, c / N3)
                     for a, b, c in itertools.product(range(N1), range(N2), range(N3))])


def _closed_omega_lower(d, dx, dy, eta):
    """Berry curvature of the lower band of d0 + d.sigma with an eta-broadened denominator.

    Omega = d.(d_x d x d_y d) / (2|d|^3) * 4|d|^2 / (4|d|^2 + eta^2); derived by hand for
    d = (k_x, k_y, m) at k = 0 (|down> lower, <down|sx|up><up|sy|down> = -i).
    """
    nd = np.linalg.norm(d, axis=-1)
    trip = np.einsum("ka,ka->k", d, np.cross(dx, dy))
    return trip / (2 * nd ** 3) * (4 * nd ** 2) / (4 * nd ** 2 + eta ** 2)


@pytest.mark.parametrize("m,tz,c0", [(1.0, 0.0, 0.0), (-0.7, 0.4, 0.3), (2.6, 0.0, -0.5)])
@pytest.mark.parametrize("eta", [0.0, 1e-3, 0.3])
def test_p1_two_band_closed_form_per_k(m, tz, c0, eta):
    model = tbgen.qwz(m, tz=tz, c0=c0)
    kmesh = (7, 9, 5)
    kidx = np.arange(np.prod(kmesh))
    jf = _mesh_frac(kmesh)
    d0, d, dx, dy = _qwz_d(jf, m, tz, c0)
    E, Om = O.kubo_per_k(model.H_R, model.R, kmesh, kidx, etas=[eta])
    nd = np.linalg.norm(d, axis=-1)
    assert np.allclose(E[:, 0], d0 - nd, atol=1e-13)
    assert np.allclose(E[:, 1], d0 + nd, atol=1e-13)
    ref = _closed_omega_lower(d, dx, dy, eta)
    assert np.allclose(Om[0, :, 0], ref, rtol=1e-11, atol=1e-13)
    assert np.allclose(Om[0, :, 1], -ref, rtol=1e-11, atol=1e-13)


def test_p1_velocity_closed_form():
    """d_x H = cos k1 sx - sin k1 sz - c0 sin(k1+k2) I for the QWZ model (Fourier convention e^{+ik.R})."""
    c0 = 0.3
    model = tbgen.qwz(0.5, c0=c0)
    kmesh = (6, 5, 1)
    kidx = np.arange(30)
    jf = _mesh_frac(kmesh)
    k1, k2 = 2 * np.pi * jf[:, 0], 2 * np.pi * jf[:, 1]
    _, dHx, dHy = O.bloch(model.H_R, model.R, kmesh, kidx)
    sx = np.array([[0, 1], [1, 0]]); sy = np.array([[0, -1j], [1j, 0]]); sz = np.diag([1, -1])
    I2 = np.eye(2)
    refx = (np.cos(k1)[:, None, None] * sx - np.sin(k1)[:, None, None] * sz
            - (c0 * np.sin(k1 + k2))[:, None, None] * I2)
    refy = (np.cos(k2)[:, None, None] * sy - np.sin(k2)[:, None, None] * sz
            - (c0 * np.sin(k1 + k2))[:, None, None] * I2)
    assert np.allclose(dHx, refx, atol=1e-14)
    assert np.allclose(dHy, refy, atol=1e-14)


# ---------------------------------------------------------------- Chern numbers
def _chern(model, n=64, eta=0.0, E_F=0.0):
    S = O.ahc(model.H_R, model.R, (n, n, 1), [E_F], etas=[eta])[0, 0]
    return 2 * np.pi * S


def test_p2_qwz_chern_numbers():
    g = json.load(open(os.path.join(GOLDEN, "chern_phase_diagram.json")))["qwz"]
    got = {}
    for case in g["cases"]:
        C = _chern(tbgen.qwz(case["m"]), n=48)
        got[case["m"]] = C
        assert abs(abs(C) - case["abs_C"]) < 1e-8, (case, C)
        if "opposite_of_m" in case:
            assert abs(C + got[case["opposite_of_m"]]) < 1e-8


def test_p2_qwz_chern_sign_from_closed_form():
    """Integrating the closed-form curvature on the same mesh fixes the sign of C."""
    n = 48
    jf = np.stack(np.meshgrid(np.arange(n) / n, np.arange(n) / n, [0.0], indexing="ij"), -1).reshape(-1, 3)
    _, d, dx, dy = _qwz_d(jf, 1.0)
    C_closed = 2 * np.pi * np.mean(_closed_omega_lower(d, dx, dy, 0.0))
    assert abs(C_closed - round(C_closed)) < 1e-8
    assert abs(_chern(tbgen.qwz(1.0), n=n) - C_closed) < 1e-10


def test_p2_haldane_chern_numbers():
    g = json.load(open(os.path.join(GOLDEN, "chern_phase_diagram.json")))["haldane"]
    got = {}
    for case in g["cases"]:
        m = tbgen.haldane(case["t1"], case["t2"], case["phi"], case["M"])
        C = _chern(m, n=96)
        got[case["phi"], case["M"]] = C
        assert abs(abs(C) - case["abs_C"]) < 1e-6, (case, C)
        if "opposite_of_phi" in case:
            assert abs(C + got[case["opposite_of_phi"], case["M"]]) < 1e-8


def test_p2_haldane_stack_gives_L():
    base = tbgen.haldane()
    C1 = _chern(base, n=64)
    C3 = _chern(tbgen.stack_layers(base, 3), n=64)
    assert abs(abs(C1) - 1) < 1e-6
    assert abs(C3 - 3 * C1) < 1e-6


def test_p2_haldane_eta_broadening_small():
    """With eta > 0 the Chern sum deviates from the integer by O(eta^2 / gap^2)."""
    m = tbgen.haldane()
    gap = 6 * np.sqrt(3) * 0.1
    for eta in [1e-3, 1e-2]:
        C = _chern(m, n=64, eta=eta)
        assert abs(abs(C) - 1) <= 4 * (eta / gap) ** 2 + 1e-9


# ---------------------------------------------------------------- independent Chern: link variables
def _haldane_hk_closed(k1, k2, t1, t2, phi, M):
    """Haldane H(k) from its d-vector (independent of the oracle's Fourier sum)."""
    bs = [(1, 0), (-1, 1), (0, -1)]
    cs = sum(np.cos(k1 * b[0] + k2 * b[1]) for b in bs)
    ss = sum(np.sin(k1 * b[0] + k2 * b[1]) for b in bs)
    d0 = 2 * t2 * np.cos(phi) * cs
    dz = M - 2 * t2 * np.sin(phi) * ss
    off = t1 * (1 + np.exp(-1j * k1) + np.exp(-1j * k2))   # d_x - i d_y
    return np.array([[d0 + dz, off], [np.conj(off), d0 - dz]])


def test_p5_fukui_hatsugai_suzuki_matches_kubo_sum():
    """Lattice link-variable Chern number (Fukui, Hatsugai, Suzuki, JPSJ 74, 1674 (2005)).

    The Berry phase of a counter-clockwise plaquette is -arg(U1 U2 U1'^* U2'^*) with links
    U = <u(k)|u(k')>; summed over the plaquettes it is 2 pi C.
    """
    t1, t2, phi, M = 1.0, 0.1, np.pi / 2, 0.2
    n = 32
    u = np.zeros((n, n, 2), dtype=complex)
    for a in range(n):
        for b in range(n):
            _, V = np.linalg.eigh(_haldane_hk_closed(2 * np.pi * a / n, 2 * np.pi * b / n, t1, t2, phi, M))
            u[a, b] = V[:, 0]
    tot = 0.0
    for a in range(n):
        for b in range(n):
            a1, b1 = (a + 1) % n, (b + 1) % n
            p = (np.vdot(u[a, b], u[a1, b]) * np.vdot(u[a1, b], u[a1, b1])
                 * np.vdot(u[a1, b1], u[a, b1]) * np.vdot(u[a, b1], u[a, b]))
            tot += -np.angle(p)
    C_fhs = tot / (2 * np.pi)
    assert abs(C_fhs - round(C_fhs)) < 1e-9
    C_kubo = _chern(tbgen.haldane(t1, t2, phi, M), n=96)
    assert abs(C_kubo - round(C_fhs)) < 1e-6


def test_p4_per_k_curvature_equals_small_loop_berry_phase():
    """Omega_n(k) from Eq. 3 (eta = 0) equals the Berry phase of a small loop / its area."""
    m = tbgen.random_tb(5, 1, 1.0, seed=3)
    rng = np.random.default_rng(7)
    for _ in range(3):
        k0 = rng.uniform(0, 1, 3)
        E, U = O.eigh(O.bloch_frac(m.H_R, m.R, k0)[0])
        gaps = np.diff(E[0])
        assert gaps.min() > 1e-3
        Hk, dHx, dHy = O.bloch_frac(m.H_R, m.R, k0)
        E0, U0 = O.eigh(Hk)
        Om = O.berry_curvature(E0, O.velocity(U0, dHx), O.velocity(U0, dHy), 0.0)[0]
        h = 2e-4                                    # loop side in radians
        df = h / (2 * np.pi)
        corners = [(-0.5, -0.5), (0.5, -0.5), (0.5, 0.5), (-0.5, 0.5)]
        vecs = []
        for cx, cy in corners:
            kf = k0 + np.array([cx * df, cy * df, 0.0])
            _, V = O.eigh(O.bloch_frac(m.H_R, m.R, kf)[0])
            vecs.append(V[0])
        for n in range(m.W):
            p = 1.0 + 0j
            for c in range(4):
                p *= np.vdot(vecs[c][:, n], vecs[(c + 1) % 4][:, n])
            berry = -np.angle(p) / h ** 2
            assert abs(berry - Om[n]) <= 1e-5 * max(1.0, abs(Om[n])), (n, berry, Om[n])


# ---------------------------------------------------------------- invariants of Eq. 3
@pytest.fixture(scope="module")
def small():
    return tbgen.random_tb(6, 1, 1.0, seed=11)


def test_p3_sum_rule_all_bands(small):
    kmesh = (4, 3, 5)
    E, Om = O.kubo_per_k(small.H_R, small.R, kmesh, np.arange(60), etas=[0.0, 1e-3, 0.1])
    scale = np.max(np.abs(Om), axis=-1)
    assert np.all(np.abs(Om.sum(-1)) <= 1e-12 * np.maximum(scale, 1.0))


def test_p3_empty_and_full_bands(small):
    kmesh = (4, 4, 4)
    S = O.ahc(small.H_R, small.R, kmesh, [-1e3, 1e3], etas=[1e-3])
    assert S[0, 0] == 0.0
    assert abs(S[0, 1]) < 1e-12


def test_p3_occ_unocc_equals_occupied_sum(small):
    kmesh = (3, 3, 3)
    kidx = np.arange(27)
    EF = np.array([-1.0, 0.0, 0.7])
    a = O.ahc_occ_unocc_per_k(small.H_R, small.R, kmesh, kidx, EF, 1e-3)
    _, per_k = O.ahc(small.H_R, small.R, kmesh, EF, etas=[1e-3], return_per_k=True)
    assert np.allclose(a / 27.0, per_k[:, 0, :], rtol=1e-10, atol=1e-12)


def test_p3_unitary_orbital_rotation_invariance(small):
    rng = np.random.default_rng(5)
    X = rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6))
    V, _ = np.linalg.qr(X)
    H2 = V[None] @ small.H_R @ np.conj(V.T)[None]
    kmesh = (3, 4, 3)
    EF = [-0.5, 0.3]
    S1 = O.ahc(small.H_R, small.R, kmesh, EF, etas=[1e-2])
    S2 = O.ahc(H2, small.R, kmesh, EF, etas=[1e-2])
    assert np.allclose(S1, S2, rtol=1e-9, atol=1e-12)


def test_p3_energy_scale_invariance(small):
    lam = 2.5
    kmesh = (3, 3, 4)
    S1 = O.ahc(small.H_R, small.R, kmesh, [0.2], etas=[1e-2])
    S2 = O.ahc(lam * small.H_R, small.R, kmesh, [0.2 * lam], etas=[1e-2 * lam])
    assert np.allclose(S1, S2, rtol=1e-9, atol=1e-13)


def test_p3_time_reversal_gives_zero():
    """Real H(R) with H(-R) = H(R)^T (time-reversal symmetric) has S = 0 on a symmetric mesh."""
    m = tbgen.random_tb(5, 1, 1.0, seed=2)
    Hr = np.real(m.H_R).astype(np.complex128)
    kmesh = (4, 4, 4)
    S = O.ahc(Hr, m.R, kmesh, [-0.5, 0.0, 0.5], etas=[1e-3])
    S_ref = O.ahc(m.H_R, m.R, kmesh, [0.0], etas=[1e-3])
    assert np.max(np.abs(S)) < 1e-12 * max(1.0, abs(S_ref[0, 0])) + 1e-14
    assert abs(S_ref[0, 0]) > 1e-4


def test_p3_partition_of_mesh_adds_up(small):
    kmesh = (4, 3, 3)
    N = 36
    full = O.ahc(small.H_R, small.R, kmesh, [0.0, 0.5], etas=[1e-3])
    a = O.ahc(small.H_R, small.R, kmesh, [0.0, 0.5], etas=[1e-3], kidx=np.arange(0, 20))
    b = O.ahc(small.H_R, small.R, kmesh, [0.0, 0.5], etas=[1e-3], kidx=np.arange(20, N))
    assert np.allclose(full, a + b, rtol=1e-13, atol=1e-15)


def test_p3_fermi_dirac_limit(small):
    kmesh = (3, 3, 3)
    E, _ = O.kubo_per_k(small.H_R, small.R, kmesh, np.arange(27))
    EF = 0.5 * (np.sort(E.ravel())[80] + np.sort(E.ravel())[81])
    gap = np.min(np.abs(E - EF))
    S0 = O.ahc(small.H_R, small.R, kmesh, [EF], etas=[1e-2], kT=0.0)
    S1 = O.ahc(small.H_R, small.R, kmesh, [EF], etas=[1e-2], kT=gap / 60.0)
    assert np.allclose(S0, S1, rtol=1e-9, atol=1e-13)
    f = O.occupation(np.array([0.3]), [0.3], 0.01)
    assert f[0, 0] == 0.5


# ---------------------------------------------------------------- sub-step checks
def test_p4_hermitian_unitary_residuals_and_fd_velocity():
    m = tbgen.random_tb(8, 2, 1.0, seed=4)
    kmesh = (5, 6, 7)
    kidx = np.array([0, 17, 101, 209])
    Hk, dHx, dHy = O.bloch(m.H_R, m.R, kmesh, kidx)
    nrm = np.max(np.abs(Hk))
    assert np.max(np.abs(Hk - np.conj(np.swapaxes(Hk, -1, -2)))) <= 1e-13 * nrm
    E, U = O.eigh(Hk)
    I = np.eye(8)
    assert np.max(np.abs(np.conj(np.swapaxes(U, -1, -2)) @ U - I)) < 1e-13
    assert np.max(np.abs(Hk @ U - U * E[:, None, :])) < 1e-12 * nrm
    assert np.all(np.diff(E, axis=-1) >= 0)
    jf = O.kfrac_of_index(kmesh, kidx) / np.array(kmesh, dtype=float)
    # mesh phases with exact reduction agree with direct evaluation at the same k
    Hd, dxd, dyd = O.bloch_frac(m.H_R, m.R, jf)
    assert np.allclose(Hd, Hk, atol=1e-12) and np.allclose(dxd, dHx, atol=1e-12)
    h = 1e-5
    for a, dH in ((0, dHx), (1, dHy)):
        e = np.zeros(3); e[a] = h / (2 * np.pi)
        fd = (O.bloch_frac(m.H_R, m.R, jf + e)[0] - O.bloch_frac(m.H_R, m.R, jf - e)[0]) / (2 * h)
        assert np.max(np.abs(fd - dH)) < 1e-7 * max(1.0, np.max(np.abs(dH)))


def test_p4_eta_zero_degenerate_pairs_skipped():
    """Two uncoupled copies: degenerate pairs are skipped at eta = 0, result = 2x one copy."""
    base = tbgen.qwz(1.0)
    two = tbgen.stack_layers(base, 2)
    kmesh = (8, 8, 1)
    S1 = O.ahc(base.H_R, base.R, kmesh, [0.0], etas=[0.0])
    S2 = O.ahc(two.H_R, two.R, kmesh, [0.0], etas=[0.0])
    assert np.isfinite(S2).all()
    assert abs(S2[0, 0] - 2 * S1[0, 0]) < 1e-10


def test_theta_at_zero_a_level_exactly_at_the_fermi_energy_is_empty():
    """Reading of theta(0) (Eqs. 2-3 leave it open): a level exactly at E_F is not occupied.

    QWZ with m = -3/2 at Gamma: every hopping is a dyadic rational and every phase is 1, so
    H(Gamma) = (m + 2) sigma_z = diag(1/2, -1/2) exactly and the levels are exactly -1/2 and
    +1/2.  The lower band's curvature there is the closed form d.(d_x d x d_y d) / (2|d|^3)
    with d = (0, 0, 1/2), d_x d = (1, 0, 0), d_y d = (0, 1, 0): Omega_lower = 2 (eta = 0).
    S at E_F = +1/2 counts the lower band only (strict reading; "<=" would add the upper
    band's -2 and give 0); at E_F = -1/2 no band counts (the "<=" reading gives 2 / N_k).
    """
    m = tbgen.qwz(-1.5)
    kmesh = (8, 8, 1)
    Nk = 64
    d = np.array([[0.0, 0.0, 0.5]])
    om = _closed_omega_lower(d, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]), 0.0)[0]
    assert om == 2.0
    E, Om = O.kubo_per_k(m.H_R, m.R, kmesh, np.array([0]), etas=[0.0])
    assert E[0, 0] == -0.5 and E[0, 1] == 0.5
    S = O.ahc(m.H_R, m.R, kmesh, [-0.5, 0.5, 0.75], etas=[0.0], kidx=np.array([0]))
    assert S[0, 0] == 0.0
    assert abs(S[0, 1] - om / Nk) < 1e-14
    assert abs(S[0, 2]) < 1e-14       # both bands occupied: the sum rule gives 0
    occ = O.occupation(np.array([[-0.5, 0.5]]), [0.5], 0.0)
    assert occ.tolist() == [[[1.0, 0.0]]]
