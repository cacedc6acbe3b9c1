"""tcgen05 split-precision (3-term BF16) complex GEMM through the C ABI, against float64 NumPy."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("M,N,K,batch,opA,opB", [(64, 128, 32, 1, 0, 0), (128, 256, 96, 2, 0, 0),
                                                 (162, 162, 162, 3, 0, 0), (75, 131, 51, 2, 2, 0),
                                                 (100, 40, 300, 1, 0, 1),
                                                 # 128 x 256 tiles (ragged N) and transposed operands
                                                 (1024, 520, 40, 4, 0, 0), (1500, 700, 70, 3, 1, 2)])
def test_split_gemm_matches_fp64(M, N, K, batch, opA, opB):
    import paper_1910_11359_gb300 as pkg
    rng = np.random.default_rng(7)
    A = rng.standard_normal((batch,) + ((M, K) if opA == 0 else (K, M))) * (1 + 1j)
    A = A + 1j * rng.standard_normal(A.shape)
    B = rng.standard_normal((batch,) + ((K, N) if opB == 0 else (N, K))) + 1j * rng.standard_normal(
        (batch,) + ((K, N) if opB == 0 else (N, K)))
    ops = {0: lambda x: x, 1: lambda x: np.swapaxes(x, 1, 2), 2: lambda x: np.swapaxes(x, 1, 2).conj()}
    ref = ops[opA](A) @ ops[opB](B)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.zeros((batch, M, N), dtype=torch.complex128, device="cuda")
    rc = pkg.lib().ipeps_kernel_zgemm_split(M, N, K, batch, opA, opB, _p(dA), A.shape[2],
                                            A.shape[1] * A.shape[2], _p(dB), B.shape[2],
                                            B.shape[1] * B.shape[2], _p(dC), N, M * N, None)
    assert rc == 0, pkg.lib().ipeps_last_error(None)
    C = dC.cpu().numpy()
    # error against the typical size of one output: |a||b| sqrt(K)
    scale = np.sqrt(K) * np.sqrt(np.mean(np.abs(A) ** 2)) * np.sqrt(np.mean(np.abs(B) ** 2))
    err = np.max(np.abs(C - ref)) / scale
    print("split GEMM relative error %.2e" % err)
    assert err < 1e-4
    assert err > 1e-9            # it really is reduced precision, not an FP64 path


def _obs_keys():
    return ("nA", "nB", "imbalance", "energy", "purityA")


def _spectra_err(pairs):
    """Largest difference of normalised corner spectra over the values above 1e-2 of the largest
    (the part the split-precision contractions determine; the tail sits at their noise level and
    decides truncation ranks there), and over all values."""
    lead = max(np.max(np.abs(a - b)[b > 1e-2]) for a, b in pairs)
    full = max(np.max(np.abs(a - b)) for a, b in pairs)
    return lead, full


def test_split_ctmrg_matches_oracle_d3():
    """Split-precision contractions inside CTMRG (D = 3, chi = 18, 6 sweeps from the traced start,
    FP64 projectors): observables and normalised corner spectra within 1e-4 of the FP64 oracle."""
    import paper_1910_11359_gb300 as pkg
    from oracle import ctmrg, evolve, measure
    p = dict(J=1.0, V=1.0, h=5.0, D=3, order=2, dt=0.05)
    GA, GB, lam, _ = evolve.evolve_tensors(p, 6)
    chi = 18
    sim = pkg.IPEPS([1.0], [1.0], [5.0], D=3, chi=chi, order=2, dt=0.05, precision=pkg.SPLIT_BF16X3)
    sim.set_tensors(GA[None], GB[None], lam[None])
    sim.ctmrg_converge(tol=0.0, max_sweeps=6)
    obs = sim.measure()[0]
    spec = {(i, pos): sim.corner_spectrum(0, pos, i) for i in range(4) for pos in range(4)}
    sim.close()
    A, B, a = evolve.ctm_state(GA, GB, lam)
    env = ctmrg.init_env(a, 2, 2, chi, 3)
    env, n, _ = ctmrg.ctmrg(a, env, chi, tol=0.0, max_sweeps=6)
    ref = measure.observables(A, B, env, 1.0, 1.0, 5.0)
    cs = ctmrg.corner_spectra(env, chi)
    err_s, err_all = _spectra_err([(s, cs[(i, (pos % 2, pos // 2))]) for (i, pos), s in spec.items()])
    err_o = max(abs(obs[k] - ref[k]) for k in _obs_keys())
    print("split CTMRG vs FP64 oracle: observables %.1e, leading spectra %.1e (all values %.1e)"
          % (err_o, err_s, err_all))
    # imbalance and the other local observables: the 1e-4 bar of the split path; the corner spectra
    # after 6 unconverged sweeps carry the contraction noise amplified by the projector iteration
    # (observed 2e-3..2e-2), so they are only held to a sanity bound
    assert err_o < 1e-4 and err_s < 5e-2
    assert err_o > 1e-13          # the contractions really ran in reduced precision


def test_split_ctmrg_random_d4_vs_fp64():
    """Random tensors at D = 4, chi = 32 (N = 512), 4 sweeps: split path against the FP64 path."""
    import paper_1910_11359_gb300 as pkg
    from inputs import random_ctmrg_tensors
    A, B = random_ctmrg_tensors(4)
    res = []
    for prec in (pkg.FP64, pkg.SPLIT_BF16X3):
        sim = pkg.IPEPS([1.0], [1.0], [5.0], D=4, chi=32, order=2, dt=0.05, precision=prec)
        sim.set_tensors(A[None], B[None], None)
        sim.ctmrg_converge(tol=0.0, max_sweeps=4)
        res.append((sim.measure()[0], [sim.corner_spectrum(0, pos, i) for i in range(4)
                                       for pos in range(4)]))
        sim.close()
    (o64, s64), (o3, s3) = res
    err_o = max(abs(o64[k] - o3[k]) for k in _obs_keys())
    err_s, err_all = _spectra_err(list(zip(s3, s64)))
    print("split vs FP64 at D=4 chi=32: observables %.1e, leading spectra %.1e (all values %.1e)"
          % (err_o, err_s, err_all))
    assert err_o < 1e-4 and err_s < 5e-2


@pytest.mark.parametrize("M,N,K,batch,opA,opB", [(64, 128, 32, 1, 0, 0), (162, 162, 162, 3, 0, 0),
                                                 (75, 131, 51, 2, 2, 0), (1024, 520, 40, 4, 0, 0),
                                                 (1500, 700, 70, 3, 1, 2), (96, 200, 1200, 1, 0, 0)])
def test_split_gemm_tf32_matches_fp64(M, N, K, batch, opA, opB):
    """TF32x3 (kind::tf32): two TF32 terms per value, three products.  The tensor cores' truncating
    accumulation biases each MMA by ~2^-24 of the accumulator; with one accumulator over all of K
    that bias grew like 1e-7 K relative to |a| |b| sqrt(K) (1.4e-5 at K = 162).  Accumulating each
    K tile of four MMAs separately and summing the tiles in FP32 (round to nearest) leaves the
    tiles' own bias and the summation's rounding, ~2^-24 sqrt(number of tiles) of the result:
    measured 6e-7 (K = 32) to 3e-6 (K = 1200, 225 tiles) as the largest error over all outputs, a
    tenth of the BF16x3 split's."""
    import paper_1910_11359_gb300 as pkg
    rng = np.random.default_rng(9)
    A = rng.standard_normal((batch,) + ((M, K) if opA == 0 else (K, M))) \
        + 1j * rng.standard_normal((batch,) + ((M, K) if opA == 0 else (K, M)))
    B = rng.standard_normal((batch,) + ((K, N) if opB == 0 else (N, K))) \
        + 1j * rng.standard_normal((batch,) + ((K, N) if opB == 0 else (N, K)))
    ops = {0: lambda x: x, 1: lambda x: np.swapaxes(x, 1, 2), 2: lambda x: np.swapaxes(x, 1, 2).conj()}
    ref = ops[opA](A) @ ops[opB](B)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.zeros((batch, M, N), dtype=torch.complex128, device="cuda")
    rc = pkg.lib().ipeps_kernel_zgemm_split_tf32(M, N, K, batch, opA, opB, _p(dA), A.shape[2],
                                                 A.shape[1] * A.shape[2], _p(dB), B.shape[2],
                                                 B.shape[1] * B.shape[2], _p(dC), N, M * N, None)
    assert rc == 0, pkg.lib().ipeps_last_error(None)
    C = dC.cpu().numpy()
    scale = np.sqrt(K) * np.sqrt(np.mean(np.abs(A) ** 2)) * np.sqrt(np.mean(np.abs(B) ** 2))
    err = np.max(np.abs(C - ref)) / scale
    print("TF32x3 split GEMM relative error %.2e" % err)
    assert err < 5e-6
    assert err > 1e-12


def test_tf32x3_ctmrg_matches_oracle_d3():
    """TF32x3 contractions inside CTMRG (D = 3, chi = 18, 6 sweeps from the traced start): one-site
    observables within 1e-6 of the FP64 oracle (BF16x3: ~1e-5)."""
    import paper_1910_11359_gb300 as pkg
    from oracle import ctmrg, evolve, measure
    p = dict(J=1.0, V=1.0, h=5.0, D=3, order=2, dt=0.05)
    GA, GB, lam, _ = evolve.evolve_tensors(p, 6)
    sim = pkg.IPEPS([1.0], [1.0], [5.0], D=3, chi=18, order=2, dt=0.05, precision=pkg.SPLIT_TF32X3)
    sim.set_tensors(GA[None], GB[None], lam[None])
    sim.ctmrg_converge(tol=0.0, max_sweeps=6)
    obs = sim.measure()[0]
    sim.close()
    A, B, a = evolve.ctm_state(GA, GB, lam)
    env = ctmrg.init_env(a, 2, 2, 18, 3)
    env, _, _ = ctmrg.ctmrg(a, env, 18, tol=0.0, max_sweeps=6)
    ref = measure.observables(A, B, env, 1.0, 1.0, 5.0)
    err = max(abs(obs[k] - ref[k]) for k in ("nA", "nB", "imbalance", "energy"))
    print("TF32x3 CTMRG vs FP64 oracle: observables %.1e" % err)
    assert err < 1e-6 and err > 1e-14


def test_tile_width_leaves_results_unchanged(tmp_path):
    """The autotuner picks the tcgen05 output-tile width (128 or 256 columns) by timing; the width
    must not enter the arithmetic.  The same BF16x3 product computed with each width forced
    (IPEPS_TUNE=128 / 256, separate processes) is identical bit for bit."""
    import os
    import subprocess
    import sys
    code = """
import ctypes, sys
import numpy as np, torch
sys.path.insert(0, %r)
import paper_1910_11359_gb300 as pkg
rng = np.random.default_rng(5)
M, N, K, batch = 300, 700, 90, 2
A = rng.standard_normal((batch, M, K)) + 1j * rng.standard_normal((batch, M, K))
B = rng.standard_normal((batch, K, N)) + 1j * rng.standard_normal((batch, K, N))
dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
dC = torch.zeros((batch, M, N), dtype=torch.complex128, device="cuda")
p = lambda t: ctypes.c_void_p(t.data_ptr())
rc = pkg.lib().ipeps_kernel_zgemm_split(M, N, K, batch, 0, 0, p(dA), K, M * K, p(dB), N, K * N, p(dC), N,
                                        M * N, None)
assert rc == 0
np.save(sys.argv[1], dC.cpu().numpy())
""" % os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for bn in ("128", "256"):
        f = str(tmp_path / ("c%s.npy" % bn))
        env = dict(os.environ, IPEPS_TUNE=bn)
        subprocess.run([sys.executable, "-c", code, f], check=True, env=env, timeout=300)
        out[bn] = np.load(f)
    assert np.array_equal(out["128"], out["256"])
