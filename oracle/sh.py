"""Real spherical harmonics and the (l,m,s) coupling matrices, by brute-force quadrature on the sphere.

TEST INFRASTRUCTURE ONLY.  This module belongs to the CPU oracle: a plain, slow, FP64 restatement
of the paper's method that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may import it; the
product path never does, and it shares no code with the CUDA library.

What it computes (paper: arXiv:2501.05110, "Sapphire++"):

* ``Y_lms`` from the definition of App. A (Eq. spherical-harmonics, normalisation N_lm,
  associated Legendre functions with the Condon--Shortley phase inside P_l^m, Legendre
  polynomials by Rodrigues' formula).
* The index map j(l,m,s) = l(l+1) + (-1)^(s+1) m (Sec. 2.1, Eq. ordering-expansion-coefficients).
* The direction matrices A^a_ij = <Y_i, p_a Y_j> with p = (cos t, sin t cos f, sin t sin f)
  (polar axis along x, Sec. 1), the rotation generators Omega^a_ij = <Y_i, (p x grad)_a Y_j>,
  and the collision matrix C = diag(l(l+1)/2) (Eq. real-C-matrix).  Matrix products are
  formed at L = lmax + 1 and then cut to n x n (Sec. 2.1, last paragraph).

The integrals use a Gauss--Legendre rule in cos(theta) and a uniform rule in phi, both with
more points than the polynomial degree of any integrand needs, so they are exact up to rounding.
"""
from __future__ import annotations

from functools import lru_cache
from math import factorial, pi, sqrt

import numpy as np
from numpy.polynomial import polynomial as npoly


# --------------------------------------------------------------------------------------------
# index map (Sec. 2.1)
# --------------------------------------------------------------------------------------------
def index_map(l: int, m: int, s: int) -> int:
    """j(l,m,s) = l(l+1) + (-1)^(s+1) m, starting at zero."""
    return l * (l + 1) + (-1) ** (s + 1) * m


def lms_list(lmax: int) -> list[tuple[int, int, int]]:
    """All (l,m,s) with l <= lmax, 0 <= m <= l, s in {0,1}, s=1 only for m >= 1, in index order."""
    out = [None] * ((lmax + 1) ** 2)
    for l in range(lmax + 1):
        for m in range(l + 1):
            for s in ((0,) if m == 0 else (0, 1)):
                out[index_map(l, m, s)] = (l, m, s)
    return out


# --------------------------------------------------------------------------------------------
# Legendre polynomials and associated Legendre functions (App. A)
# --------------------------------------------------------------------------------------------
@lru_cache(maxsize=None)
def _legendre_coeffs(l: int) -> np.ndarray:
    """Power-series coefficients of P_l(x) = 1/(2^l l!) d^l/dx^l (x^2 - 1)^l (Rodrigues)."""
    base = npoly.polypow(np.array([-1.0, 0.0, 1.0]), l)  # (x^2 - 1)^l
    d = npoly.polyder(base, l) if l > 0 else base
    return d / (2.0 ** l * factorial(l))


def _dm_legendre(l: int, m: int) -> np.ndarray:
    """Coefficients of d^m P_l / dx^m."""
    c = _legendre_coeffs(l)
    return npoly.polyder(c, m) if m > 0 else c


def assoc_legendre(l: int, m: int, x: np.ndarray) -> np.ndarray:
    """P_l^m(x) = (-1)^m (1 - x^2)^(m/2) d^m/dx^m P_l(x)  (Condon--Shortley phase included)."""
    q = npoly.polyval(x, _dm_legendre(l, m))
    return (-1.0) ** m * (1.0 - x * x) ** (m / 2.0) * q


def _assoc_legendre_dtheta(l: int, m: int, theta: np.ndarray) -> np.ndarray:
    """d/dtheta of P_l^m(cos theta), from the product rule on (-1)^m sin^m(t) Q(cos t)."""
    st, ct = np.sin(theta), np.cos(theta)
    q = npoly.polyval(ct, _dm_legendre(l, m))
    dq = npoly.polyval(ct, npoly.polyder(_dm_legendre(l, m))) if l - m > 0 else 0.0 * ct
    term1 = m * st ** (m - 1) * ct * q if m > 0 else 0.0 * ct
    return (-1.0) ** m * (term1 - st ** (m + 1) * dq)


def norm_lm(l: int, m: int) -> float:
    """N_lm = sqrt((2l+1)/(2 pi (1+delta_m0)) (l-m)!/(l+m)!)  (Eq. normalisation-spherical-harmonics)."""
    return sqrt((2 * l + 1) / (2 * pi * (1 + (m == 0))) * factorial(l - m) / factorial(l + m))


def real_Y(l: int, m: int, s: int, theta, phi) -> np.ndarray:
    """Y_lms(theta, phi) = N_lm P_l^m(cos theta) (delta_s0 cos m phi + delta_s1 sin m phi)."""
    theta = np.asarray(theta, dtype=float)
    phi = np.asarray(phi, dtype=float)
    ang = np.cos(m * phi) if s == 0 else np.sin(m * phi)
    return norm_lm(l, m) * assoc_legendre(l, m, np.cos(theta)) * ang


def _real_Y_derivs(l, m, s, theta, phi):
    """(Y, dY/dtheta, dY/dphi)."""
    nlm = norm_lm(l, m)
    ang = np.cos(m * phi) if s == 0 else np.sin(m * phi)
    dang = -m * np.sin(m * phi) if s == 0 else m * np.cos(m * phi)
    P = assoc_legendre(l, m, np.cos(theta))
    dP = _assoc_legendre_dtheta(l, m, theta)
    return nlm * P * ang, nlm * dP * ang, nlm * P * dang


# --------------------------------------------------------------------------------------------
# sphere quadrature
# --------------------------------------------------------------------------------------------
def sphere_rule(L: int):
    """Nodes (theta, phi) and weights of a product rule exact for polynomials of degree <= 2L+3.

    Gauss--Legendre in mu = cos(theta) with 2L+4 points; uniform phi with 4L+8 points."""
    nmu, nphi = 2 * L + 4, 4 * L + 8
    mu, wmu = np.polynomial.legendre.leggauss(nmu)
    phi = 2 * pi * np.arange(nphi) / nphi
    th = np.arccos(mu)
    TH, PH = np.meshgrid(th, phi, indexing="ij")
    W = np.outer(wmu, np.full(nphi, 2 * pi / nphi))
    return TH.ravel(), PH.ravel(), W.ravel()


def direction(theta, phi):
    """p_hat = (cos t, sin t cos f, sin t sin f): polar axis along x (Sec. 1)."""
    return np.stack([np.cos(theta), np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi)])


def _L_operator(dth, dph, theta, phi):
    """(p_hat x grad)_a g for a = x,y,z, given dg/dtheta and dg/dphi.

    On the unit sphere grad g = e_theta dg/dtheta + e_phi (1/sin t) dg/dphi, and with the
    right-handed frame (p_hat, e_theta, e_phi): p_hat x e_theta = e_phi, p_hat x e_phi = -e_theta,
    so p_hat x grad g = e_phi dg/dtheta - e_theta (1/sin t) dg/dphi."""
    st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    e_th = np.stack([-st, ct * cp, ct * sp])
    e_ph = np.stack([0.0 * st, -sp, cp])
    return e_ph * dth - e_th * (dph / st)


@lru_cache(maxsize=None)
def full_tables(L: int):
    """A^a, Omega^a (a = x,y,z) and C for the untruncated index set l <= L, by quadrature."""
    TH, PH, W = sphere_rule(L)
    idx = lms_list(L)
    nL = len(idx)
    Y = np.empty((nL, TH.size))
    LY = np.empty((3, nL, TH.size))
    for j, (l, m, s) in enumerate(idx):
        y, dth, dph = _real_Y_derivs(l, m, s, TH, PH)
        Y[j] = y
        LY[:, j] = _L_operator(dth, dph, TH, PH)
    p = direction(TH, PH)
    A = np.stack([(Y * W) @ (p[a] * Y).T for a in range(3)])
    Om = np.stack([(Y * W) @ LY[a].T for a in range(3)])
    C = np.diag([l * (l + 1) / 2.0 for (l, m, s) in idx])
    return A, Om, C


def levi_civita(a: int, b: int, c: int) -> int:
    return int((a - b) * (b - c) * (c - a) / 2)


@lru_cache(maxsize=None)
def tables(lmax: int) -> dict:
    """All n x n matrices the system of PDEs needs, n = (lmax+1)^2.

    Keys: 'A' (3,n,n), 'Om' (3,n,n), 'C' (n,n), 'AA' (3,3,n,n) = A^a A^b,
    'E' (3,n,n) = eps_abc A^b Om^c, 'F' (3,3,n,n) = A^a E^b = eps_bcd A^a A^c Om^d.
    Products are formed with the L = lmax+1 matrices and then truncated (Sec. 2.1)."""
    L = lmax + 1
    n = (lmax + 1) ** 2
    A_L, Om_L, C_L = full_tables(L)
    E_L = np.zeros_like(A_L)
    for a in range(3):
        for b in range(3):
            for c in range(3):
                e = levi_civita(a, b, c)
                if e:
                    E_L[a] += e * A_L[b] @ Om_L[c]
    AA_L = np.einsum("aij,bjk->abik", A_L, A_L)
    F_L = np.einsum("aij,bjk->abik", A_L, E_L)
    t = slice(0, n)

    def clean(M):
        # the exact matrix elements are either zero (selection rules) or O(1); quadrature leaves
        # rounding residue ~1e-16 where they vanish, which is set to zero here
        M = M.copy()
        M[np.abs(M) < 1e-12] = 0.0
        return M

    A_L, Om_L, E_L, AA_L, F_L = (clean(M) for M in (A_L, Om_L, E_L, AA_L, F_L))
    return {
        "n": n,
        "A": A_L[:, t, t].copy(),
        "Om": Om_L[:, t, t].copy(),
        "C": C_L[t, t].copy(),
        "AA": AA_L[:, :, t, t].copy(),
        "E": E_L[:, t, t].copy(),
        "F": F_L[:, :, t, t].copy(),
    }
