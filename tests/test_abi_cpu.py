"""CPU-side checks of the C ABI: the library builds and loads, exports every symbol declared
in include/kubo.h, and rejects bad arguments on the host before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2309_06675_gb300 as kubo
import tbgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2309_06675_gb300 import _build
    _build.build()
    return kubo.lib()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "kubo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kubo_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = _declared_functions()
    assert "kubo_ahc" in names and "kubo_eigh_batched" in names
    for n in names:
        assert hasattr(L, n), n


def test_status_strings(L):
    for code in range(9):
        s = L.kubo_status_string(code).decode()
        assert s.startswith("KUBO_")
    assert kubo.max_orbitals("fp64") >= 64


def _call_ahc(L, H, R, W, N_R, kmesh, n_EF=1, eta=1e-3, opt=None):
    km = np.asarray(kmesh, dtype=np.int32)
    Rh = np.ascontiguousarray(R, dtype=np.int32)
    dummy = ctypes.c_void_p(16)   # never dereferenced: validation fails first
    return L.kubo_ahc(dummy if H is None else H, Rh.ctypes.data_as(ctypes.c_void_p), W, N_R,
                      km.ctypes.data_as(ctypes.c_void_p), dummy, n_EF, eta, dummy, opt)


def test_host_validation_rejects_bad_sizes(L):
    m = tbgen.random_tb(4, 1, 1.0, 0)
    assert _call_ahc(L, None, m.R, 0, m.N_R, (4, 4, 4)) == 1          # W = 0
    assert _call_ahc(L, None, m.R, 4, m.N_R, (0, 4, 4)) == 1          # empty mesh
    assert _call_ahc(L, None, m.R, 4, m.N_R, (4, 4, 4), n_EF=0) == 1  # no Fermi level
    assert _call_ahc(L, None, m.R, 4, m.N_R, (4, 4, 4), eta=-1.0) == 1
    assert _call_ahc(L, None, m.R, 4, m.N_R, (4, 4, 4), eta=float("nan")) == 1
    assert _call_ahc(L, None, m.R, 4096, m.N_R, (4, 4, 4)) == 4       # W beyond this build


def test_host_validation_rejects_open_R_sets(L):
    m = tbgen.random_tb(4, 1, 1.0, 0)
    R = m.R.copy()
    R_missing = R[R[:, 0] != -1]                                          # drops some -R
    assert _call_ahc(L, None, R_missing, 4, R_missing.shape[0], (4, 4, 4)) == 3
    R_dup = R.copy(); R_dup[1] = R_dup[0]
    assert _call_ahc(L, None, R_dup, 4, R_dup.shape[0], (4, 4, 4)) == 3
    R_no0 = np.array([[1, 0, 0], [-1, 0, 0]], dtype=np.int32)
    assert _call_ahc(L, None, R_no0, 4, 2, (4, 4, 4)) == 3


def test_options_validation(L):
    m = tbgen.random_tb(4, 1, 1.0, 0)
    o = kubo.Options()
    L.kubo_options_init(ctypes.byref(o))
    assert o.precision == 0 and o.n_eta == 0 and o.kT == 0.0
    o.kT = -1.0
    assert _call_ahc(L, None, m.R, 4, m.N_R, (4, 4, 4), opt=ctypes.byref(o)) == 1
    o.kT = 0.0
    o.k_begin, o.k_end = 10, 5
    assert _call_ahc(L, None, m.R, 4, m.N_R, (4, 4, 4), opt=ctypes.byref(o)) == 1
    o.k_begin, o.k_end = 0, 0
    e = np.zeros(9)
    o.n_eta = 9
    o.etas = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert _call_ahc(L, None, m.R, 4, m.N_R, (4, 4, 4), opt=ctypes.byref(o)) == 4


def test_workspace_size_scales_with_batch(L):
    small = kubo.workspace_size(16, 125, (24, 24, 24), 1, chunk_k=1024)
    big = kubo.workspace_size(16, 125, (24, 24, 24), 1, chunk_k=4096)
    assert 0 < small < big
    assert kubo.workspace_size(0, 125, (24, 24, 24), 1) == 0


def test_pack_unpack_roundtrip():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    X = rng.standard_normal((3, 5, 5)) + 1j * rng.standard_normal((3, 5, 5))
    A = torch.from_numpy(X + np.conj(np.swapaxes(X, -1, -2)))
    P = kubo.pack_hermitian(A)
    assert P.shape == (3, 25)
    assert torch.allclose(kubo.unpack_hermitian(P, 5), A)
