"""The allocation-free eigensolver entry point against the allocating one.

kubo_eigh_batched_noalloc exists for callers that cannot let a library allocate device
memory mid-call (their own allocator holds the GPU's memory, or an allocation would
synchronise a latency-critical loop).  It keeps its intermediates in a fixed block compiled
into the library, shared by every call, so this test makes two calls in a row with
different sizes -- each spanning several passes of the block, the last one short -- and checks
each against kubo_eigh_batched and against LAPACK eigenvalues, the residual and unitarity at
the eigensolver tolerances used by the other tests.  The file is named to be collected last.
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


def _hermitian(rng, n, W):
    X = rng.standard_normal((n, W, W)) + 1j * rng.standard_normal((n, W, W))
    return X + np.conj(np.swapaxes(X, -1, -2))


# Matrices per pass of the fixed 32 MiB block: (4 W + 2 W + 2 W^2) doubles per matrix, so
# 489 at W = 64 and 6,898 at W = 16 (the block also holds the status word).
PASS_W64, PASS_W16 = 489, 6898


def test_noalloc_matches_allocating_entry_point_two_calls(env):
    torch, kubo, f = env
    rng = np.random.default_rng(2024)
    # call 1: W = 64, two full passes of the block and a short third one
    # call 2: W = 16, one full pass and a short second one, the block reused with another layout
    for W, n in ((64, 2 * PASS_W64 + 122), (16, PASS_W16 + 102)):
        A_h = _hermitian(rng, n, W)
        A = kubo.pack_hermitian(torch.from_numpy(A_h).to("cuda:0"))
        E, U = _noalloc(env, A, W)
        E_ref, U_ref = kubo.eigh_batched(A, W)
        torch.cuda.synchronize()
        nrm = E_ref.abs().max(dim=1).values[:, None]
        assert torch.all((E - E_ref).abs() <= 1e-12 * nrm.clamp(min=1.0))
        # eigenvectors are unique up to a phase: compare the gauge-invariant projector check
        overlap = (U_ref.conj().transpose(-1, -2) @ U).abs()
        eye = torch.eye(W, dtype=torch.float64, device=A.device)
        assert torch.all((overlap - eye).abs() <= 1e-9)
        # and against references that share nothing with the library: LAPACK's eigenvalues,
        # the residual A U - U E and the unitarity of U, at the eigensolver tests' tolerances
        E, U = E.cpu().numpy(), U.cpu().numpy()
        lam = np.linalg.eigvalsh(A_h)
        scale = np.maximum(np.max(np.abs(lam), axis=-1), 1.0)
        assert np.all(np.max(np.abs(E - lam), axis=-1) <= 1e-12 * scale)
        res = np.abs(A_h @ U - U * E[:, None, :]).max(axis=(1, 2))
        assert np.all(res <= 1e-12 * scale)
        orth = np.abs(np.conj(np.swapaxes(U, -1, -2)) @ U - np.eye(W)).max(axis=(1, 2))
        assert np.all(orth <= 1e-13 * max(W, 8))


def test_noalloc_rejects_orders_beyond_its_limit(env):
    torch, kubo, f = env
    dummy = 256
    code = f(dummy, 65, 1, dummy, dummy, None)
    assert kubo.lib().kubo_status_string(code).decode().startswith("KUBO_ERR_UNSUPPORTED")
