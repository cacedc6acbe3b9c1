"""GPU checks of the FP64 building blocks through the C ABI (kernel entry points of libipeps)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    import paper_1910_11359_gb300 as pkg
    return pkg.lib()


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (17, 33, 5), (162, 162, 162), (18, 162, 81)])
@pytest.mark.parametrize("opA,opB", [(0, 0), (2, 0), (0, 1), (1, 2)])
def test_zgemm(M, N, K, opA, opB):
    batch = 3
    A = _rand((batch, M, K) if opA == 0 else (batch, K, M), 1)
    B = _rand((batch, K, N) if opB == 0 else (batch, N, K), 2)
    opa = {0: lambda x: x, 1: lambda x: np.swapaxes(x, 1, 2), 2: lambda x: np.swapaxes(x, 1, 2).conj()}
    ref = opa[opA](A) @ opa[opB](B)
    dA, dB = _dev(A), _dev(B)
    dC = torch.zeros((batch, M, N), dtype=torch.complex128, device="cuda")
    lda = A.shape[2]
    ldb = B.shape[2]
    rc = _lib().ipeps_kernel_zgemm(M, N, K, batch, opA, opB, _p(dA), lda, A.shape[1] * A.shape[2],
                                   _p(dB), ldb, B.shape[1] * B.shape[2], _p(dC), N, M * N, None)
    assert rc == 0
    torch.cuda.synchronize()
    err = np.max(np.abs(dC.cpu().numpy() - ref)) / max(1.0, np.max(np.abs(ref)))
    assert err < 1e-14 * max(K, 1) ** 0.5 * 10


def test_permute():
    x = _rand((2, 3, 4, 5, 6), 3)
    perm = [0, 3, 2, 1]
    ref = np.stack([np.transpose(x[b], perm) for b in range(2)])
    dx = _dev(x)
    dy = torch.zeros_like(dx)
    dims = (ctypes.c_int * 4)(3, 4, 5, 6)
    pm = (ctypes.c_int * 4)(*perm)
    rc = _lib().ipeps_kernel_permute(_p(dx), _p(dy), 4, dims, pm, 2, 360, 360, None)
    assert rc == 0
    torch.cuda.synchronize()
    assert np.array_equal(dy.cpu().numpy().reshape(ref.shape), ref)


@pytest.mark.parametrize("m,n", [(12, 12), (27, 12), (48, 48), (32, 32), (162, 36), (7, 3), (64, 64)])
def test_jacobi_svd(m, n):
    batch = 4
    A = _rand((batch, m, n), 5)
    A[1, :, 2] = 0.0                                    # a zero column
    A[2] = A[2] @ np.diag(np.logspace(0, -12, n))       # graded spectrum
    A[3, :, 1] = A[3, :, 0]                              # rank deficiency
    dA = _dev(A)
    dU = torch.zeros((batch, m, n), dtype=torch.complex128, device="cuda")
    dS = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    dV = torch.zeros((batch, n, n), dtype=torch.complex128, device="cuda")
    rc = _lib().ipeps_kernel_svd(m, n, batch, _p(dA), _p(dU), _p(dS), _p(dV), 4e-16 * m, 80, None, None)
    assert rc == 0
    U, S, V = dU.cpu().numpy(), dS.cpu().numpy(), dV.cpu().numpy()
    for b in range(batch):
        s_ref = np.linalg.svd(A[b], compute_uv=False)
        assert np.max(np.abs(S[b] - s_ref)) < 1e-13 * s_ref[0]
        rec = (U[b] * S[b]) @ V[b].conj().T
        assert np.max(np.abs(rec - A[b])) < 1e-13 * s_ref[0]
        nz = S[b] > 1e-10 * S[b][0]
        Ub = U[b][:, nz]
        assert np.max(np.abs(Ub.conj().T @ Ub - np.eye(nz.sum()))) < 1e-12
        assert np.max(np.abs(V[b].conj().T @ V[b] - np.eye(n))) < 1e-13


@pytest.mark.parametrize("J,V,h,delta", [(1.0, 1.0, 5.0, 0.02), (0.7, 0.0, 10.0, 0.05), (1.0, 1.0, 1.0, 0.025)])
def test_gate_matches_oracle(J, V, h, delta):
    from oracle import model
    out = np.zeros((16, 16), dtype=np.complex128)
    rc = _lib().ipeps_kernel_gate(J, V, h, delta, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert rc == 0
    assert np.max(np.abs(out - model.gate(J, V, h, delta))) < 1e-14


@pytest.mark.parametrize("m,n", [(2400, 40), (1300, 100), (1000, 100), (2600, 120)])
def test_jacobi_svd_tall_blocks(m, n):
    """Tall blocks: 16-CTA clusters (m >= 1024, where the part allows them) and, when the row
    slices exceed shared memory, columns kept in a global buffer ((1000, 100) on 8-CTA clusters,
    (2600, 120) on either)."""
    batch = 2
    A = _rand((batch, m, n), 11)
    A[1] = A[1] @ np.diag(np.logspace(0, -10, n))       # graded spectrum
    dA = _dev(A)
    dU = torch.zeros((batch, m, n), dtype=torch.complex128, device="cuda")
    dS = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    dV = torch.zeros((batch, n, n), dtype=torch.complex128, device="cuda")
    rc = _lib().ipeps_kernel_svd(m, n, batch, _p(dA), _p(dU), _p(dS), _p(dV), 4e-16 * m, 80, None, None)
    assert rc == 0
    U, S, V = dU.cpu().numpy(), dS.cpu().numpy(), dV.cpu().numpy()
    for b in range(batch):
        s_ref = np.linalg.svd(A[b], compute_uv=False)
        assert np.max(np.abs(S[b] - s_ref)) < 1e-12 * s_ref[0]
        rec = (U[b] * S[b]) @ V[b].conj().T
        assert np.max(np.abs(rec - A[b])) < 1e-12 * s_ref[0]
        assert np.max(np.abs(V[b].conj().T @ V[b] - np.eye(n))) < 1e-13


@pytest.mark.parametrize("N,k,batch", [(162, 26, 3), (512, 40, 2), (2592, 80, 1)])
def test_orth_cholesky_qr(N, k, batch):
    """Column-scaled Cholesky QR: orthonormal columns (Q^+ Q = I to rounding) spanning the input's
    (Q Q^+ X = X), on blocks shaped like the projector subspace blocks.  The columns of X are scaled
    over ten orders of magnitude, as the blocks M V are; one column is exactly zero and must stay
    zero."""
    rng = np.random.default_rng(11)
    X = rng.standard_normal((batch, N, k)) + 1j * rng.standard_normal((batch, N, k))
    X *= 10.0 ** (-10.0 * np.arange(k) / k)[None, None, :]
    X[:, :, k // 2] = 0.0
    dX = _dev(X)
    dQ = torch.zeros_like(dX)
    fail = (ctypes.c_int * batch)()
    rc = _lib().ipeps_kernel_orth(N, k, batch, _p(dX), _p(dQ), 3, fail, None)
    assert rc == 0
    assert list(fail) == [0] * batch
    Q = dQ.cpu().numpy()
    live = [j for j in range(k) if j != k // 2]
    for b in range(batch):
        q = Q[b][:, live]
        assert np.max(np.abs(q.conj().T @ q - np.eye(len(live)))) < 1e-13
        assert np.max(np.abs(Q[b][:, k // 2])) == 0.0
        proj = q @ (q.conj().T @ X[b])
        err = np.max(np.abs(proj - X[b]) / np.maximum(np.linalg.norm(X[b], axis=0), 1e-300)[None, :])
        assert err < 1e-11, err


def test_orth_flags_dependent_columns():
    """Columns that are exactly parallel cannot be orthonormalised by Cholesky QR: the problem is
    flagged (and the caller falls back) rather than returning a Q that is not orthonormal."""
    N, k = 100, 8
    rng = np.random.default_rng(3)
    X = rng.standard_normal((1, N, k)) + 1j * rng.standard_normal((1, N, k))
    X[0, :, 5] = 3.0 * X[0, :, 2]
    dX = _dev(X)
    dQ = torch.zeros_like(dX)
    fail = (ctypes.c_int * 1)()
    rc = _lib().ipeps_kernel_orth(N, k, 1, _p(dX), _p(dQ), 2, fail, None)
    assert rc == 0
    if not fail[0]:
        q = dQ.cpu().numpy()[0]
        assert np.max(np.abs(q.conj().T @ q - np.eye(k))) < 1e-10


def test_orth_ill_conditioned_block():
    """A block whose columns stay far from orthogonal after scaling (singular values spread over ten
    orders of magnitude, mixed by a random unitary: condition ~1e10) is orthonormalised by the
    three-pass shifted Cholesky QR and spans the input to its conditioning."""
    N, k = 300, 40
    rng = np.random.default_rng(5)
    base = np.linalg.qr(rng.standard_normal((N, k)) + 1j * rng.standard_normal((N, k)))[0]
    W = np.linalg.qr(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))[0]
    X = ((base * 10.0 ** (-10.0 * np.arange(k) / (k - 1))) @ W.conj().T)[None]
    dX = _dev(X)
    dQ = torch.zeros_like(dX)
    fail = (ctypes.c_int * 1)()
    assert _lib().ipeps_kernel_orth(N, k, 1, _p(dX), _p(dQ), 3, fail, None) == 0
    assert fail[0] == 0
    q = dQ.cpu().numpy()[0]
    assert np.max(np.abs(q.conj().T @ q - np.eye(k))) < 1e-12
    err = np.linalg.norm(q @ (q.conj().T @ X[0]) - X[0]) / np.linalg.norm(X[0])
    assert err < 1e-12
