"""Simple update (Jiang, Weng & Xiang, PRL 101, 090603 (2008)) for the two-site checkerboard iPEPS.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Paper: Sec. "Set up for iPEPS" (Quench) and the Appendix choose the simple update for the real-time
evolution |Psi(t)> = exp(-iHt)|Psi_0>, with Trotter steps; the local truncation error is the sum of
the squares of the discarded weights for one site (Sec. "Results for interacting case").

State: Gamma_A, Gamma_B with legs (s, u, l, d, r) and four bond-weight vectors lam[g], g = u, l, d, r
as seen from A.  A's leg g joins B's opposite leg (g + 2) mod 4, so B's leg g carries lam[(g+2)%4].

One bond update, written plainly (no QR reduction):
  1. multiply each tensor by the weights of its three other legs;
  2. theta = A (x) lam_g (x) B contracted over the bond;
  3. apply the two-site gate to the physical pair;
  4. full SVD of theta as a (d D^3) x (d D^3) matrix;
  5. keep D values (degenerate multiplets at the cut are kept whole or dropped whole),
     eps += discarded weight sum_{k>=K} s_k^2 / sum_k s_k^2;
  6. lam_g <- s_kept / ||s_kept||; the singular vectors become the new Gammas after dividing the
     other legs' weights back out (pseudo-inverse: weights below 1e-14 of the leg's largest -> 0).

Trotter sequences (bond types named by A's leg: R = 3, U = 0, L = 1, D = 2):
  first order : R, U, L, D                      all with delta = dt
  second order: R, U, L (dt/2), D (dt), L, U, R (dt/2)

Parity: pinned by tests/test_oracle_su.py (J = 0 exactness, D = 1 brute-force product-state
propagation, dimer exactness, unitarity of the kept norm, sublattice-gauge and field-flip symmetry).
"""
import numpy as np

LEG_U, LEG_L, LEG_D, LEG_R = 0, 1, 2, 3
DEGEN_RTOL = 1e-10   # multiplet detection at a truncation cut
TINY_REL = 1e-14     # values below this fraction of the largest count as zero
PINV_REL = 1e-14     # weight pseudo-inverse threshold


def trotter_sequence(order, dt):
    """List of (leg, delta) bond updates making one Trotter step."""
    if order == 1:
        return [(LEG_R, dt), (LEG_U, dt), (LEG_L, dt), (LEG_D, dt)]
    if order == 2:
        h = dt / 2
        return [(LEG_R, h), (LEG_U, h), (LEG_L, h), (LEG_D, dt), (LEG_L, h), (LEG_U, h), (LEG_R, h)]
    raise ValueError("trotter order must be 1 or 2")


def truncation_rank(s, keep, degen_rtol=DEGEN_RTOL, tiny_rel=TINY_REL, degen_abs=0.0):
    """Number of singular values kept at a cut of nominal size ``keep``.

    If the last kept and first dropped values form one multiplet (relative gap below
    ``degen_rtol``, or absolute gap below ``degen_abs`` times the largest value) and the dropped
    one is not numerically zero, the cut moves down to the multiplet's upper edge, so that a
    multiplet is never split.
    """
    K = min(keep, len(s))
    while 1 < K < len(s) and s[K] > tiny_rel * s[0] and (
            s[K - 1] / s[K] - 1.0 < degen_rtol or s[K - 1] - s[K] < degen_abs * s[0]):
        K -= 1
    return K


def _pinv_weights(w):
    out = np.zeros_like(w)
    big = w > PINV_REL * w.max()
    out[big] = 1.0 / w[big]
    return out


def _scale_legs(G, weights, skip):
    """Multiply leg g (axis 1+g) of G by weights[g] for every g != skip."""
    out = G.copy()
    for g in range(4):
        if g == skip:
            continue
        shape = [1] * 5
        shape[1 + g] = -1
        out = out * weights[g].reshape(shape)
    return out


def b_weights(lam):
    """Weights seen by B's legs (u, l, d, r): B's leg g joins A's leg (g+2) % 4."""
    return np.stack([lam[(g + 2) % 4] for g in range(4)])


def bond_update(GA, GB, lam, leg, U):
    """Apply the gate U (d^2 x d^2, index sA*d + sB) on the bond at A's leg ``leg``.

    Returns (GA', GB', lam', eps) with eps the discarded weight of this update.
    """
    d, D = GA.shape[0], GA.shape[1]
    legB = (leg + 2) % 4
    lamB = b_weights(lam)
    A = _scale_legs(GA, lam, leg)
    B = _scale_legs(GB, lamB, legB)
    # bond leg of A last, bond leg of B right after the physical leg
    Am = np.moveaxis(A, 1 + leg, 4)          # (s, o1, o2, o3, k)
    Bm = np.moveaxis(B, 1 + legB, 1)         # (t, k, p1, p2, p3)
    theta = np.einsum('sabck,k,tkefg->sabctefg', Am, lam[leg], Bm)
    U4 = U.reshape(d, d, d, d)               # [sA', sB', sA, sB]
    theta = np.einsum('xyst,sabctefg->xabcyefg', U4, theta)
    M = theta.reshape(d * D ** 3, d * D ** 3)
    X, s, Yh = np.linalg.svd(M, full_matrices=False)
    K = truncation_rank(s, D)
    total = float(np.sum(s ** 2))
    eps = float(np.sum(s[K:] ** 2)) / total if total > 0 else 0.0
    lam_new = lam.copy()
    lam_new[leg] = 0.0
    nk = np.linalg.norm(s[:K])
    lam_new[leg, :K] = s[:K] / nk
    Xk = np.zeros((d * D ** 3, D), dtype=np.complex128)
    Xk[:, :K] = X[:, :K]
    Yk = np.zeros((D, d * D ** 3), dtype=np.complex128)
    Yk[:K] = Yh[:K]
    An = np.moveaxis(Xk.reshape(d, D, D, D, D), 4, 1 + leg)
    Bn = np.moveaxis(Yk.reshape(D, d, D, D, D), 0, 1 + legB)
    # divide the other legs' weights back out (the bond weights themselves live in lam)
    inv = np.stack([_pinv_weights(lam[g]) for g in range(4)])
    invB = b_weights(inv)
    An = _scale_legs(An, inv, leg)
    Bn = _scale_legs(Bn, invB, legB)
    return An, Bn, lam_new, eps


def trotter_step(GA, GB, lam, gates, order, dt):
    """One Trotter step; ``gates`` maps delta -> gate matrix.  Returns (GA, GB, lam, eps_sum)."""
    eps = 0.0
    for leg, delta in trotter_sequence(order, dt):
        GA, GB, lam, e = bond_update(GA, GB, lam, leg, gates[delta])
        eps += e
    return GA, GB, lam, eps


def physical_tensors(GA, GB, lam):
    """Tensors contracted by CTMRG: Gamma with sqrt(lam) absorbed on all four legs."""
    sq = np.sqrt(lam)
    A = _scale_legs(GA, sq, -1)
    B = _scale_legs(GB, b_weights(sq), -1)
    return A, B
