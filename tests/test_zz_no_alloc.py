"""The allocation-free eigensolver entry point against the allocating one.

kubo_eigh_batched_noalloc exists for callers that cannot let a library allocate device
memory mid-call (their own allocator holds the GPU's memory, or an allocation would
synchronise a latency-critical loop).  It keeps its intermediates in a fixed block compiled
into the library, shared by every call, so this test makes two calls in a row with
different sizes and checks each against kubo_eigh_batched at the eigensolver tolerance
used by the other tests.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_06675_gb300 import _build
    _build.build()
    import paper_2309_06675_gb300 as kubo
    L = kubo.lib()
    f = L.kubo_eigh_batched_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    return torch, kubo, f


def _noalloc(env, A, W):
    torch, kubo, f = env
    n = A.shape[0]
    E = torch.empty((n, W), dtype=torch.float64, device=A.device)
    U = torch.empty((n, W, W), dtype=torch.complex128, device=A.device)
    stream = torch.cuda.current_stream().cuda_stream
    code = f(A.data_ptr(), W, n, E.data_ptr(), U.data_ptr(), stream)
    assert code == 0, kubo.lib().kubo_status_string(code).decode()
    return E, U


def _hermitian_packed(torch, kubo, rng, n, W):
    X = rng.standard_normal((n, W, W)) + 1j * rng.standard_normal((n, W, W))
    H = X + np.conj(np.swapaxes(X, -1, -2))
    return kubo.pack_hermitian(torch.from_numpy(H).to("cuda:0"))


def test_noalloc_matches_allocating_entry_point_two_calls(env):
    torch, kubo, f = env
    rng = np.random.default_rng(2024)
    # call 1: W = 64, more matrices than one pass of the fixed block holds
    # call 2: W = 16, so the block is reused with a different layout
    for W, n in ((64, 300), (16, 2500)):
        A = _hermitian_packed(torch, kubo, rng, n, W)
        E, U = _noalloc(env, A, W)
        E_ref, U_ref = kubo.eigh_batched(A, W)
        torch.cuda.synchronize()
        nrm = E_ref.abs().max(dim=1).values[:, None]
        assert torch.all((E - E_ref).abs() <= 1e-12 * nrm.clamp(min=1.0))
        # eigenvectors are unique up to a phase: compare the gauge-invariant projector check
        overlap = (U_ref.conj().transpose(-1, -2) @ U).abs()
        eye = torch.eye(W, dtype=torch.float64, device=A.device)
        assert torch.all((overlap - eye).abs() <= 1e-9)


def test_noalloc_rejects_orders_beyond_its_limit(env):
    torch, kubo, f = env
    dummy = 256
    code = f(dummy, 65, 1, dummy, dummy, None)
    assert kubo.lib().kubo_status_string(code).decode().startswith("KUBO_ERR_UNSUPPORTED")
