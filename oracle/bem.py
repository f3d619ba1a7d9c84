"""FP64 CPU oracle of the continuum (BEM) operator of Section 2.3 (Eq. 21, Eq. 22).

TEST INFRASTRUCTURE ONLY: imported by tests/ and the CPU legs of bench.py, never by
the product package.  Plain numpy in FP64, one row at a time, so that each line can
be checked against the equations by eye.

What it computes.  Eq. 21 is (Lambda(w) I + F) sigma = -dphi/dn on N surface elements
with Lambda(w) = 2 pi (eps_out + eps_in(w)) / (eps_out - eps_in(w)) and, by Eq. 22,
F_ij = n_i . grad_{r_j} 1/|r_i - r_j| = n_i . (r_i - r_j) / |r_i - r_j|^3.  The
library solves it in the same form as the omega-FQ system, (A - zI) q = R, with:

  * unknowns q_i = sigma_i a_i (charge of element i, a_i its area), so that the
    polarizability is sum_i q_i r_i / E0 exactly as for the omega-FQ charges;
  * A_ij = a_i F_ij (i != j): Eq. 22 integrated over element j by its collocation
    point gives F_ij a_j sigma_j = F_ij q_j; row i is multiplied by a_i so that the
    shift acts on q_i = a_i sigma_i;
  * A_ii = H_i sqrt(pi a_i): the principal value of Eq. 22 over element i itself,
    taken as a flat disk of the element's area on a surface of mean curvature H_i
    (zero for a flat element); the caller supplies H_i;
  * z(w) = -Lambda(w);
  * R_i = a_i dphi/dn (r_i) = -E0 a_i n_i . k for the uniform field phi = -E0 k . r.
    The printed Eq. 21 has -dphi/dn on the right; with the printed signs of Lambda and
    F that yields -sigma (for instance a negative static polarizability of a metal
    sphere), so the right-hand side is taken with the sign that gives the physical
    charge.  The signs of Lambda and F are kept as printed: together they put the
    sphere's dipole resonance at eps_in = -2 eps_out.
  * eps_in(w) = eps_inf - wp^2 / (w (w + i gamma)) (Drude); the paper leaves
    eps(w) to the material.

Pins (tests/test_oracle_bem_pins.py): the sphere's multipole eigenvalues
2 pi / (2l + 1); Gauss's law (column sums of A tend to 2 pi on any closed surface);
the quasi-static polarizabilities of a sphere and of a prolate spheroid
(depolarization factors); the resonance condition z(w_F) = 2 pi / 3; a real spectrum;
passivity (Im eps_in > 0, eps_in equal to eps_inf + 4 pi i sigma / w for the Drude
conductivity in the time convention of Eq. 5, Im alpha_kk >= 0).
"""
import math

import numpy as np

from . import oracle as _core


def eps_in(omega, bem):
    """Drude permittivity of the particle at angular frequency omega (hartree)."""
    w = complex(omega)
    return bem["eps_inf"] - bem["omega_p"] ** 2 / (w * (w + 1j * bem["gamma"]))


def z_of_omega(omega, bem):
    """Eq. 21 written as A - zI: z(w) = -Lambda(w) = -2 pi (eps_out + eps_in) / (eps_out - eps_in)."""
    eo = bem["eps_out"]
    ei = eps_in(omega, bem)
    return -2.0 * math.pi * (eo + ei) / (eo - ei)


def a_matrix(xyz, normal, area, curvature):
    """A of (A - zI) q = R for the BEM operator: A_ij = a_i n_i . (r_i - r_j) / |r_i - r_j|^3
    (Eq. 22, collocation, charge unknowns), A_ii = H_i sqrt(pi a_i)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    normal = np.asarray(normal, dtype=np.float64)
    area = np.asarray(area, dtype=np.float64)
    curvature = np.zeros(len(xyz)) if curvature is None else np.asarray(curvature, dtype=np.float64)
    n = len(xyz)
    A = np.empty((n, n))
    for i in range(n):
        d = xyz[i] - xyz                     # r_i - r_j, every j
        r2 = np.einsum("jk,jk->j", d, d)
        r2[i] = 1.0                          # the diagonal is set below
        A[i] = area[i] * (d @ normal[i]) / (r2 * np.sqrt(r2))
        A[i, i] = curvature[i] * math.sqrt(math.pi * area[i])
    return A


def rhs(normal, area, kdir, E0=1.0):
    """R_i = -E0 a_i (n_i . k): element i's area times the normal derivative of
    phi = -E0 k . r (see the module header for the sign)."""
    normal = np.asarray(normal, dtype=np.float64)
    return -E0 * np.asarray(area, dtype=np.float64) * (normal @ np.asarray(kdir, dtype=np.float64))


def solve(A, z, R):
    """(A - zI) q = R by the oracle's LU with partial pivoting."""
    return _core.lu_solve(A, z, R)


def alpha(xyz, q, E0=1.0):
    """alpha_{k'} = sum_i q_i r_{i,k'} / E0 (Eq. 28 with element charges)."""
    return _core.alpha(xyz, q, E0)
