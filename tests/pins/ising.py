"""Closed forms of the 2D classical Ising model (J = 1, square lattice) used as CTMRG pins.

Onsager (1944): free energy and internal energy; Yang (1952): spontaneous magnetisation.
The Ising PEPS psi(s) = prod_<ij> exp(beta s_i s_j / 2) has <psi|psi> = Z_Ising(beta), so its
CTM norm per site is exp(-beta f), its one-site <sigma^z> is the magnetisation and its
nearest-neighbour <sigma^z sigma^z> is -u/2.
"""
import numpy as np
from scipy.special import ellipk

BETA_C = 0.5 * np.log(1 + np.sqrt(2))


def peps_tensor(beta):
    """A[s, u, l, d, r] = prod_legs Q[s, leg], Q Q^T = [[e^{b/2}, e^{-b/2}], [e^{-b/2}, e^{b/2}]]."""
    W = np.array([[np.exp(beta / 2), np.exp(-beta / 2)], [np.exp(-beta / 2), np.exp(beta / 2)]])
    w, V = np.linalg.eigh(W)
    Q = (V * np.sqrt(w)) @ V.T
    A = np.einsum('su,sl,sd,sr->suldr', Q, Q, Q, Q)
    return A.astype(np.complex128)


def magnetisation(beta):
    if beta <= BETA_C:
        return 0.0
    return (1 - np.sinh(2 * beta) ** -4) ** 0.125


def nn_correlation(beta):
    """<s_i s_j> for nearest neighbours = -u / 2 with Onsager's internal energy per site u."""
    k = 2 * np.sinh(2 * beta) / np.cosh(2 * beta) ** 2
    K = ellipk(k * k)
    u = -1 / np.tanh(2 * beta) * (1 + 2 / np.pi * (2 * np.tanh(2 * beta) ** 2 - 1) * K)
    return -u / 2


def z_per_site(beta, n=800):
    """exp(-beta f) from Onsager's double integral (periodic trapezoid rule, spectrally accurate)."""
    th = 2 * np.pi * np.arange(n) / n
    c1, c2 = np.meshgrid(np.cos(th), np.cos(th))
    integrand = np.log(np.cosh(2 * beta) ** 2 - np.sinh(2 * beta) * (c1 + c2))
    return np.exp(np.log(2) + 0.5 * integrand.mean())
