"""Dilated site, bond Hamiltonian, Trotter gate and initial state (FP64, plain NumPy).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Paper: Sec. "Set up for iPEPS".  The disorder h_i S^z_i of Eq. (Hori) is carried by one auxiliary
spin per site prepared in |+>, coupled to the physical spin by h S^z_p S^z_a (Eq. Hanc); tracing the
auxiliaries out gives the exact disorder average (Readout, the E<O(t)> identity).  The number of
disorder levels is d_A, with the field values spaced uniformly in [-h, h] (+h, -h for d_A = 2).

Hamiltonian form used here (hard-core bosons; V/J = 2 Delta in the paper's convention):

    H = sum_<ij> [ -J (b_i^+ b_j + h.c.) + V n_i n_j ] + h sum_i tau_i n_i

where tau_i is the auxiliary "field level" operator with eigenvalues 1 - 2a/(d_A - 1),
a = 0..d_A-1 (so tau^z = +1, -1 for d_A = 2).  The on-site term is folded into the bond terms with
weight h/z, z = 4, so that each site collects h tau n once from its four bonds.

Local basis: s = n * d_A + a, n in {0, 1} (boson occupation), a the auxiliary level; d = 2 d_A.

Parity: pinned by tests/test_oracle_model.py (gate unitarity and conservation laws, the J = 0
closed form, the two-site exact short-time expansion).
"""
import numpy as np

Z_COORD = 4  # coordination number of the square lattice


def local_ops(d_A=2):
    """Return (b, n, tau, eye) as d x d complex matrices for the dilated site, d = 2 d_A."""
    d = 2 * d_A
    b = np.zeros((d, d), dtype=np.complex128)
    for a in range(d_A):
        b[a, d_A + a] = 1.0          # b |n=1, a> = |n=0, a>
    n = b.conj().T @ b
    levels = np.array([1.0 - 2.0 * a / (d_A - 1) for a in range(d_A)]) if d_A > 1 else np.zeros(1)
    tau = np.diag(np.concatenate([levels, levels])).astype(np.complex128)
    return b, n, tau, np.eye(d, dtype=np.complex128)


def bond_hamiltonian(J, V, h, d_A=2):
    """Two-site term h_b on basis index s_i * d + s_j (d^2 x d^2, Hermitian).

    h_b = -J (b_i^+ b_j + b_j^+ b_i) + V n_i n_j + (h / z) (tau_i n_i + tau_j n_j).
    """
    b, n, tau, I = local_ops(d_A)
    bd = b.conj().T
    tn = tau @ n
    return (-J * (np.kron(bd, b) + np.kron(b, bd)) + V * np.kron(n, n)
            + (h / Z_COORD) * (np.kron(tn, I) + np.kron(I, tn)))


def gate(J, V, h, delta, d_A=2):
    """Trotter gate exp(-i h_b delta) via the Hermitian eigendecomposition (LAPACK zheevd)."""
    w, W = np.linalg.eigh(bond_hamiltonian(J, V, h, d_A))
    return (W * np.exp(-1j * w * delta)) @ W.conj().T


def initial_tensors(D, d_A=2):
    """CDW (x) |+> product state as a D=1 iPEPS, zero-padded to bond dimension D.

    Sublattice A is occupied, B empty, every auxiliary spin in |+> = d_A^{-1/2} sum_a |a>
    (Sec. "Set up for iPEPS", Initialization; Fig. 1).  Returns Gamma_A, Gamma_B of shape
    (d, D, D, D, D) with leg order (s, u, l, d, r) and the four bond-weight vectors lam (4, D)
    in leg order (u, l, d, r) as seen from A, each equal to (1, 0, ..., 0).
    """
    d = 2 * d_A
    GA = np.zeros((d, D, D, D, D), dtype=np.complex128)
    GB = np.zeros((d, D, D, D, D), dtype=np.complex128)
    for a in range(d_A):
        GA[d_A + a, 0, 0, 0, 0] = 1.0 / np.sqrt(d_A)
        GB[a, 0, 0, 0, 0] = 1.0 / np.sqrt(d_A)
    lam = np.zeros((4, D))
    lam[:, 0] = 1.0
    return GA, GB, lam
