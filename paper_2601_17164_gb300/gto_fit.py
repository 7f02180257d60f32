"""Ground-state GTO expansions used as target inputs (paper App. B.1).

The paper fits the ground state from a time-independent Schroedinger solve to
a GTO basis with fixed exponents by linear regression (6-311G for H 1s,
cc-pV5Z for Ar 3p).  Those basis tables are not available here, so this module
fits its own even-tempered exponents:

* H 1s:  psi0 = e^{-r}/sqrt(pi) projected in L2(R^3) onto
  {e^{-alpha_j r^2}}, alpha_j = 0.05 * 3^j, j = 0..7.
* Ar 3p0: radial finite-difference solve of -u''/2 + [V(r) + 1/r^2] u = E u
  with the Tong-Lin SAE potential, second l = 1 eigenstate; the p_z orbital
  psi0 = sqrt(3/4pi) u(r)/r^2 * z is projected onto {z e^{-alpha_j r^2}},
  alpha_j = 0.04 * 2.2^j, j = 0..13.

Running ``python -m paper_2601_17164_gb300.gto_fit`` prints the coefficients
that ``workloads.py`` stores as literals.  This is input preparation, not part
of the trajectory path.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, linalg

H_ALPHA = [0.05 * 3.0 ** j for j in range(8)]
AR_ALPHA = [0.04 * 2.2 ** j for j in range(14)]
TONGLIN_AR = (1.0, 16.039, 2.007, -25.543, 4.525, 0.961, 0.443)


def _gauss_overlap(ai, aj, l):
    """int e^{-(ai+aj) r^2} d^3r (l=0) or int z^2 e^{-(ai+aj) r^2} d^3r (l=1)."""
    s = ai + aj
    if l == 0:
        return (np.pi / s) ** 1.5
    return 0.5 * np.pi ** 1.5 * s ** -2.5


def fit_h1s():
    a = np.array(H_ALPHA)
    S = np.array([[_gauss_overlap(x, y, 0) for y in a] for x in a])
    b = np.array([4.0 * np.pi / np.sqrt(np.pi) *
                  integrate.quad(lambda r, al=al: r * r * np.exp(-al * r * r - r), 0, np.inf,
                                 epsabs=1e-15, epsrel=1e-13, limit=400)[0] for al in a])
    return linalg.solve(S, b, assume_a="pos")


def tonglin_V(r, p=TONGLIN_AR):
    Zc, a1, a2, a3, a4, a5, a6 = p
    return -(Zc + a1 * np.exp(-a2 * r) + a3 * r * np.exp(-a4 * r) + a5 * np.exp(-a6 * r)) / r


def ar_3p_radial(n=12000, rmax=60.0):
    """Second l=1 eigenpair of the radial equation on a uniform grid (3-point FD)."""
    h = rmax / (n + 1)
    r = h * np.arange(1, n + 1)
    diag = 1.0 / h ** 2 + tonglin_V(r) + 1.0 / r ** 2
    off = -0.5 / h ** 2 * np.ones(n - 1)
    w, v = linalg.eigh_tridiagonal(diag, off, select="i", select_range=(0, 1))
    u = v[:, 1] / np.sqrt(h)
    if u[np.argmax(np.abs(u))] < 0 and u[-n // 4] < 0:
        u = -u
    # outer lobe positive
    i_out = np.argmax(np.abs(u) * (r > 1.0))
    if u[i_out] < 0:
        u = -u
    return r, u, w[1]


def fit_ar3p():
    r, u, E = ar_3p_radial()
    h = r[1] - r[0]
    f = np.sqrt(3.0 / (4.0 * np.pi)) * u / r ** 2       # psi0 = f(r) z
    a = np.array(AR_ALPHA)
    S = np.array([[_gauss_overlap(x, y, 1) for y in a] for x in a])
    # <z e^{-a r^2} | f z> = (4 pi / 3) int r^4 f e^{-a r^2} dr
    b = np.array([(4.0 * np.pi / 3.0) * np.sum(r ** 4 * f * np.exp(-al * r * r)) * h for al in a])
    c = linalg.solve(S, b, assume_a="pos")
    return c, E


if __name__ == "__main__":
    np.set_printoptions(precision=17)
    print("H_C =", repr(list(fit_h1s())))
    c, E = fit_ar3p()
    print("AR_C =", repr(list(c)))
    print("AR_E3p =", E)
