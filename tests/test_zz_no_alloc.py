"""The allocation-free SVD entry point (ipeps_kernel_svd_noalloc) against the allocating one.

For callers that cannot call cudaMalloc, the library offers a variant of ipeps_kernel_svd that keeps
its per-call scratch (operand pointer tables and error word) in a fixed device array instead of a
fresh allocation.  This file is collected last on purpose; it must pass on its own in a fresh process
and after the other tests.  Two calls in a row check that the shared array's leftover contents from
the previous call do not leak into the next result.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _run(fn, dA, m, n, batch):
    dU = torch.zeros((batch, m, n), dtype=torch.complex128, device="cuda")
    dS = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    dV = torch.zeros((batch, n, n), dtype=torch.complex128, device="cuda")
    rc = fn(m, n, batch, _p(dA), _p(dU), _p(dS), _p(dV), 4e-16 * m, 80, None, None)
    assert rc == 0
    torch.cuda.synchronize()
    return dU.cpu().numpy(), dS.cpu().numpy(), dV.cpu().numpy()


@pytest.mark.parametrize("m,n,batch", [(48, 48, 5), (162, 26, 3)])
def test_noalloc_svd_matches_allocating_entry_point(m, n, batch):
    import paper_1910_11359_gb300 as pkg
    lib = pkg.lib()
    for call in range(2):
        rng = np.random.default_rng(100 + call)
        A = rng.standard_normal((batch, m, n)) + 1j * rng.standard_normal((batch, m, n))
        dA = torch.from_numpy(A).cuda()
        U0, S0, V0 = _run(lib.ipeps_kernel_svd, dA, m, n, batch)
        U1, S1, V1 = _run(lib.ipeps_kernel_svd_noalloc, dA, m, n, batch)
        scale = np.max(S0)
        assert np.max(np.abs(S1 - S0)) < 1e-13 * scale
        for b in range(batch):
            rec = (U1[b] * S1[b]) @ V1[b].conj().T
            assert np.max(np.abs(rec - A[b])) < 1e-13 * scale
        assert np.max(np.abs(U1 - U0)) < 1e-12 and np.max(np.abs(V1 - V0)) < 1e-12


def test_noalloc_error_word_is_cleared_between_calls():
    """The error word lives in the shared array too: a call on a matrix holding a NaN must report
    IPEPS_ENAN (4), and the next call on clean input, on a non-default stream, must succeed and
    match the allocating entry point."""
    import paper_1910_11359_gb300 as pkg
    lib = pkg.lib()
    m, n, batch = 40, 24, 2
    rng = np.random.default_rng(5)
    A = rng.standard_normal((batch, m, n)) + 1j * rng.standard_normal((batch, m, n))
    bad = A.copy()
    bad[1, 3, 4] = np.nan
    dbad = torch.from_numpy(bad).cuda()
    dS = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    rc = lib.ipeps_kernel_svd_noalloc(m, n, batch, _p(dbad), None, _p(dS), None, 4e-16 * m, 80, None, None)
    assert rc == 4
    side = torch.cuda.Stream()
    dA = torch.from_numpy(A).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        dU = torch.zeros((batch, m, n), dtype=torch.complex128, device="cuda")
        dS1 = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
        dV = torch.zeros((batch, n, n), dtype=torch.complex128, device="cuda")
        rc = lib.ipeps_kernel_svd_noalloc(m, n, batch, _p(dA), _p(dU), _p(dS1), _p(dV), 4e-16 * m, 80,
                                          None, ctypes.c_void_p(side.cuda_stream))
    assert rc == 0
    side.synchronize()
    U0, S0, V0 = _run(lib.ipeps_kernel_svd, dA, m, n, batch)
    assert np.max(np.abs(dS1.cpu().numpy() - S0)) < 1e-13 * np.max(S0)
    assert np.max(np.abs(dU.cpu().numpy() - U0)) < 1e-12


def test_noalloc_rejects_oversized_batch():
    import paper_1910_11359_gb300 as pkg
    lib = pkg.lib()
    dA = torch.zeros((1, 4, 4), dtype=torch.complex128, device="cuda")
    rc = lib.ipeps_kernel_svd_noalloc(4, 4, 1025, _p(dA), None, _p(dA), None, 1e-15, 10, None, None)
    assert rc == 1
    assert b"1024" in lib.ipeps_last_error(None)
