"""Seeded synthetic tight-binding inputs shared by the oracle, the tests and the bench.

This module only *draws and lays out* inputs: lattice-vector lists R, hopping blocks
H(R), k-mesh shapes, Fermi-energy grids and k-point samples.  It contains none of
the Kubo method's arithmetic (no Fourier sum, no diagonalisation, no curvature),
so the CPU oracle and the CUDA path can both consume it without sharing any
computation.

Layouts (the library's input format):
  * ``R``   : int32 [N_R, 3], sorted lexicographically, closed under R -> -R,
              containing R = 0.
  * ``H_R`` : complex128 [N_R, W, W], row-major, with H(-R) = H(R)^dagger, so that
              H(k) = sum_R exp(i k.R) H(R) is Hermitian for every k.

The paper's benchmark models are Wannier tight-binding models of bcc Fe and its
supercells (Sec. 3); they are not available here, so random decaying-hopping
models of the same matrix dimensions (N_d = 16..128) stand in for them.  The
two-band models (Qi-Wu-Zhang, Haldane) are textbook models with closed-form
Berry curvature / Chern numbers that pin the oracle.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "TBModel", "r_box", "random_tb", "qwz", "haldane", "stack_layers",
    "k_sample", "config", "CONFIGS", "batch_recipe",
]


@dataclasses.dataclass
class TBModel:
    """A Wannier tight-binding model: H(R) blocks on integer lattice vectors R."""
    H_R: np.ndarray   # complex128 [N_R, W, W]
    R: np.ndarray     # int32 [N_R, 3]

    @property
    def W(self) -> int:
        return int(self.H_R.shape[1])

    @property
    def N_R(self) -> int:
        return int(self.R.shape[0])


def r_box(half_width: int) -> np.ndarray:
    """All integer R in {-h..h}^3, sorted lexicographically (R_1 slowest)."""
    h = int(half_width)
    ax = np.arange(-h, h + 1, dtype=np.int32)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    return np.ascontiguousarray(g, dtype=np.int32)


def _is_canonical(r) -> bool:
    """True when the first non-zero component of r is positive."""
    for c in r:
        if c != 0:
            return c > 0
    return False


def _index_of(R: np.ndarray) -> dict:
    return {tuple(int(c) for c in r): i for i, r in enumerate(R)}


def random_tb(W: int, half_width: int, decay: float, seed: int = 0) -> TBModel:
    """Random Hermitian-paired TB model with hoppings N(0,1) * exp(-|R|/decay) and random phases.

    Reading of the synthetic recipe (entries "N(0,1) exp(-|R|/decay) with random complex
    phases"): each drawn entry is a * exp(i phi), a ~ N(0,1), phi ~ U[0, 2 pi), scaled by
    exp(-|R|/decay) with |R| the Euclidean norm of the integer vector.
      * R = 0: diagonal real N(0,1); strict upper triangle drawn as above; lower = conj.
      * canonical half-set R (first non-zero component > 0): the full W x W block is drawn.
      * the partner block is H(-R) = H(R)^dagger.
    Draw order: R in sorted order; numpy PCG64 ``default_rng(seed)``.
    The random phases break time reversal, so the anomalous Hall response is non-zero.
    """
    rng = np.random.default_rng(seed)
    R = r_box(half_width)
    idx = _index_of(R)
    H = np.zeros((R.shape[0], W, W), dtype=np.complex128)
    iu = np.triu_indices(W, k=1)
    for i, r in enumerate(R):
        rt = tuple(int(c) for c in r)
        scale = float(np.exp(-np.sqrt(float(np.dot(r, r))) / decay))
        if rt == (0, 0, 0):
            d = rng.standard_normal(W)
            n_off = iu[0].size
            a = rng.standard_normal(n_off)
            ph = rng.uniform(0.0, 2.0 * np.pi, n_off)
            blk = np.zeros((W, W), dtype=np.complex128)
            blk[np.arange(W), np.arange(W)] = d
            blk[iu] = a * np.exp(1j * ph)
            blk[(iu[1], iu[0])] = np.conj(blk[iu])
            H[i] = blk * scale
        elif _is_canonical(rt):
            a = rng.standard_normal((W, W))
            ph = rng.uniform(0.0, 2.0 * np.pi, (W, W))
            H[i] = a * np.exp(1j * ph) * scale
    for rt, i in idx.items():
        if rt != (0, 0, 0) and _is_canonical(rt):
            j = idx[(-rt[0], -rt[1], -rt[2])]
            H[j] = np.conj(H[i].T)
    return TBModel(H_R=H, R=R)


def _assemble(blocks: dict, W: int) -> TBModel:
    """Build a TBModel from {R-tuple: W x W block}; missing -R partners are added as H^dagger."""
    full = dict(blocks)
    for rt, b in list(blocks.items()):
        mr = (-rt[0], -rt[1], -rt[2])
        if mr not in full:
            full[mr] = np.conj(np.asarray(b).T)
    if (0, 0, 0) not in full:
        full[(0, 0, 0)] = np.zeros((W, W), dtype=np.complex128)
    keys = sorted(full.keys())
    R = np.array(keys, dtype=np.int32).reshape(-1, 3)
    H = np.stack([np.asarray(full[k], dtype=np.complex128) for k in keys])
    return TBModel(H_R=H, R=R)


_SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def qwz(m: float, tz: float = 0.0, c0: float = 0.0) -> TBModel:
    """Qi-Wu-Zhang two-band model, optionally with a k_3 mass term and an identity term.

    H(k) = c0 cos(k1+k2) I + sin k1 sx + sin k2 sy + (m + cos k1 + cos k2 + tz cos k3) sz,
    written as hopping blocks on R in {0, +-e1, +-e2, +-e3, +-(e1+e2)} under the
    convention H(k) = sum_R exp(i k.R) H(R).
    """
    b = {}
    b[(0, 0, 0)] = m * _SZ
    b[(1, 0, 0)] = -0.5j * _SX + 0.5 * _SZ
    b[(0, 1, 0)] = -0.5j * _SY + 0.5 * _SZ
    if tz != 0.0:
        b[(0, 0, 1)] = 0.5 * tz * _SZ
    if c0 != 0.0:
        b[(1, 1, 0)] = 0.5 * c0 * _I2
    return _assemble(b, 2)


def haldane(t1: float = 1.0, t2: float = 0.1, phi: float = np.pi / 2, M: float = 0.0) -> TBModel:
    """Haldane honeycomb model on integer lattice coordinates (orbitals A=0, B=1).

    H(R)_{ij} is the amplitude <i, cell 0| H |j, cell R>.  Nearest-neighbour A->B hopping
    t1 into the cells R in {(0,0), (-1,0), (0,-1)}; next-nearest-neighbour vectors
    b in {(1,0), (-1,1), (0,-1)} carry t2 e^{+i phi} on A and t2 e^{-i phi} on B; onsite
    +M on A and -M on B.  Every hopping is added together with its Hermitian partner
    H(-R)_{ji} = conj(H(R)_{ij}).
    """
    acc = {}

    def hop(r, i, j, val):
        for rr, ii, jj, vv in ((r, i, j, val), ((-r[0], -r[1], -r[2]), j, i, np.conj(val))):
            blk = acc.setdefault(rr, np.zeros((2, 2), dtype=np.complex128))
            blk[ii, jj] += vv

    acc[(0, 0, 0)] = np.diag([M, -M]).astype(np.complex128)
    for r in [(0, 0, 0), (-1, 0, 0), (0, -1, 0)]:
        hop(r, 0, 1, t1)
    for r in [(1, 0, 0), (-1, 1, 0), (0, -1, 0)]:
        hop(r, 0, 0, t2 * np.exp(1j * phi))
        hop(r, 1, 1, t2 * np.exp(-1j * phi))
    keys = sorted(acc.keys())
    R = np.array(keys, dtype=np.int32).reshape(-1, 3)
    H = np.stack([acc[k] for k in keys])
    return TBModel(H_R=H, R=R)


def stack_layers(model: TBModel, L: int) -> TBModel:
    """L uncoupled copies of a model (block-diagonal H(R), W -> L*W)."""
    W = model.W
    H = np.zeros((model.N_R, L * W, L * W), dtype=np.complex128)
    for l in range(L):
        H[:, l * W:(l + 1) * W, l * W:(l + 1) * W] = model.H_R
    return TBModel(H_R=H, R=model.R.copy())


def k_sample(kmesh, n: int, seed: int = 0) -> np.ndarray:
    """A seeded sample of n distinct linear k-indices of the mesh (sorted, int64).

    Linear index of k = (j1, j2, j3) is (j1 * N2 + j2) * N3 + j3 (j3 fastest).
    """
    N = int(np.prod(kmesh))
    rng = np.random.default_rng(seed)
    n = min(int(n), N)
    return np.sort(rng.choice(N, size=n, replace=False)).astype(np.int64)


# The five synthetic workloads.  Each entry is a recipe; ``config(name)`` draws it.
CONFIGS = {
    "w16_r125_k24": dict(W=16, half_width=2, decay=1.0, seed=0, kmesh=(24, 24, 24),
                         E_F=[0.0], etas=[1e-3], kT=0.0),
    "w64_r1331_k128": dict(W=64, half_width=5, decay=1.5, seed=0, kmesh=(128, 128, 128),
                           E_F=list(np.linspace(-1.0, 1.0, 64)), etas=[1e-3], kT=0.0),
    "w32_r729_k48_fd": dict(W=32, half_width=4, decay=1.5, seed=0, kmesh=(48, 48, 48),
                            E_F=[0.0], etas=[5e-3], kT=0.025),
    "w128_r1331_k96": dict(W=128, half_width=5, decay=1.5, seed=0, kmesh=(96, 96, 96),
                           E_F=list(np.linspace(-2.0, 2.0, 512)),
                           etas=[1e-4, 1e-3, 5e-3, 1e-2], kT=0.0),
}


def batch_recipe(n_models: int = 64, seed: int = 7, w_range=(8, 96), hw_range=(3, 5),
                 mesh_range=(32, 64), decay: float = 1.5, model_seed0: int = 1000):
    """Shapes of the uneven-model batch: per model (W, half_width, mesh N, model seed).

    W uniform in w_range, cubic R box of half-width uniform in hw_range ((2h+1)^3 vectors),
    k-mesh N^3 with N uniform in mesh_range, hoppings as ``random_tb`` with the given decay
    and seed model_seed0 + i.  Draw with ``random_tb(W, h, decay, seed)``; the Fermi level
    of each model (its median band energy at k = 0) is for the caller to compute.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(int(n_models)):
        W = int(rng.integers(w_range[0], w_range[1] + 1))
        h = int(rng.integers(hw_range[0], hw_range[1] + 1))
        N = int(rng.integers(mesh_range[0], mesh_range[1] + 1))
        out.append(dict(W=W, half_width=h, mesh=N, decay=decay, seed=model_seed0 + i))
    return out


def config(name: str):
    """Draw a named workload: returns (TBModel, kmesh tuple, E_F float64 array, etas, kT)."""
    c = CONFIGS[name]
    m = random_tb(c["W"], c["half_width"], c["decay"], c["seed"])
    return (m, tuple(c["kmesh"]), np.asarray(c["E_F"], dtype=np.float64),
            np.asarray(c["etas"], dtype=np.float64), float(c["kT"]))
