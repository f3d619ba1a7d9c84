"""Pins of the BEM oracle (Section 2.3, Eq. 21-22) against closed forms of potential
theory, not against the oracle itself: the sphere's multipole eigenvalues
2 pi / (2l + 1), Gauss's law on a closed spheroid, the quasi-static polarizabilities
of a sphere and of a prolate spheroid (depolarization factors), the resonance
condition eps_in = -2 eps_out, a real spectrum, and passivity of the lossy particle
(Im eps_in > 0 with eps_in rebuilt from the Drude conductivity in the time convention
of the paper's Eq. 5, Im alpha_kk >= 0).  The discretisation error of
one-point collocation falls as N^-1/2; each tolerance is a fixed multiple of N^-1/2
that the correct operator meets and a transposed normal, the other element's area,
a missing self term or a flipped sign misses; a flipped damping sign fails the
passivity pin.  CPU only."""
import math

import numpy as np
import pytest

KX, KY, KZ = np.eye(3)


@pytest.fixture(scope="module")
def bem():
    from oracle import bem
    return bem


def _sphere(S, n, R=40.0):
    return S.spheroid_surface(n, R, R)


def _alpha_sphere(R, ei, eo=1.0):
    return R ** 3 * (ei - eo) / (ei + 2.0 * eo)


def _depolarization_prolate(a, b):
    """L_z and L_x of a prolate spheroid (semi-axes a > b = c), closed form."""
    e = math.sqrt(1.0 - b * b / (a * a))
    Lz = (1.0 - e * e) / (e * e) * (-1.0 + math.log((1.0 + e) / (1.0 - e)) / (2.0 * e))
    return Lz, 0.5 * (1.0 - Lz)


def test_sphere_multipole_eigenvalues(bem, S):
    # the single-layer potential of Y_lm on a sphere is 4 pi a / (2l+1) Y_lm, so Eq. 22's
    # operator has eigenvalue 2 pi / (2l + 1) on degree-l harmonics
    for n in (1000, 4000):
        s = _sphere(S, n)
        A = bem.a_matrix(s["xyz"], s["normal"], s["area"], s["curvature"])
        nx, ny, nz = s["normal"].T
        cases = [(0, np.ones(n)), (1, nz), (1, nx), (2, 1.5 * nz * nz - 0.5), (2, nx * ny)]
        for l, f in cases:
            lam = f @ (A @ f) / (f @ f)
            exact = 2.0 * math.pi / (2 * l + 1)
            assert abs(lam / exact - 1.0) < 0.7 / math.sqrt(n), (n, l, lam, exact)
            # and f is (nearly) an eigenvector, not just a good Rayleigh quotient
            assert np.linalg.norm(A @ f - exact * f) / np.linalg.norm(f) < 2.0 * exact / math.sqrt(n)


def test_gauss_law_column_sums_on_spheroid(bem, S):
    # sum_i a_i n_i . (r_i - r_j) / |r_i - r_j|^3 is the solid angle of the closed surface
    # seen from r_j on it: 2 pi.  Holds only with the normal and area of the field point i.
    for n in (1000, 3000):
        s = S.spheroid_surface(n, 60.0, 30.0)
        A = bem.a_matrix(s["xyz"], s["normal"], s["area"], s["curvature"])
        dev = np.abs(A.sum(axis=0) / (2.0 * math.pi) - 1.0)
        assert dev.max() < 0.5 / math.sqrt(n), (n, dev.max())


def test_gauss_law_fails_for_planted_mistakes(bem, S):
    # the pin above separates the operator from its plausible mistakes
    n = 1500
    s = S.spheroid_surface(n, 60.0, 30.0)
    x, nrm, a, H = s["xyz"], s["normal"], s["area"], s["curvature"]
    good = bem.a_matrix(x, nrm, a, H)
    d = x[:, None, :] - x[None, :, :]
    r2 = np.einsum("ijk,ijk->ij", d, d)
    np.fill_diagonal(r2, 1.0)
    r3 = r2 * np.sqrt(r2)
    diag = np.diag(good).copy()
    planted = {
        "normal of j": a[:, None] * np.einsum("ijk,jk->ij", d, nrm) / r3,
        "area of j": a[None, :] * np.einsum("ijk,ik->ij", d, nrm) / r3,
        "no self term": good - np.diag(diag),
    }
    for name, M in planted.items():
        if name != "no self term":
            np.fill_diagonal(M, diag)
        dev = np.abs(M.sum(axis=0) / (2.0 * math.pi) - 1.0).max()
        assert dev > 2.0 / math.sqrt(n), name


def test_sphere_polarizability_quasistatic(bem, S):
    n, R = 2000, 40.0
    s = _sphere(S, n, R)
    A = bem.a_matrix(s["xyz"], s["normal"], s["area"], s["curvature"])
    m = S.drude_metal_params()
    for w_ev in (1.0, 2.5, 4.5):
        w = S.ev(w_ev)
        z = bem.z_of_omega(w, m)
        for k in (KX, KZ):
            q = bem.solve(A, z, bem.rhs(s["normal"], s["area"], k))
            al = bem.alpha(s["xyz"], q) @ k
            ex = _alpha_sphere(R, bem.eps_in(w, m))
            assert abs(al / ex - 1.0) < 1.2 / math.sqrt(n), (w_ev, al, ex)
    # static dielectric limit: eps_in = 5 through z directly; alpha > 0
    z = -2.0 * math.pi * (1.0 + 5.0) / (1.0 - 5.0)
    q = bem.solve(A, complex(z), bem.rhs(s["normal"], s["area"], KZ))
    al = bem.alpha(s["xyz"], q)[2]
    assert al.real > 0 and abs(al / _alpha_sphere(R, 5.0) - 1.0) < 0.5 / math.sqrt(n)


def test_prolate_spheroid_depolarization(bem, S):
    n, a, b = 2500, 60.0, 30.0
    s = S.spheroid_surface(n, a, b)
    A = bem.a_matrix(s["xyz"], s["normal"], s["area"], s["curvature"])
    Lz, Lx = _depolarization_prolate(a, b)
    m = S.drude_metal_params()
    for w_ev in (1.5, 4.5):
        w = S.ev(w_ev)
        ei = bem.eps_in(w, m)
        z = bem.z_of_omega(w, m)
        for k, L in ((KZ, Lz), (KX, Lx)):
            q = bem.solve(A, z, bem.rhs(s["normal"], s["area"], k))
            al = bem.alpha(s["xyz"], q) @ k
            ex = a * b * b / 3.0 * (ei - 1.0) / (1.0 + L * (ei - 1.0))
            assert abs(al / ex - 1.0) < 1.0 / math.sqrt(n), (w_ev, L, al, ex)


def test_shift_at_the_sphere_resonance(bem, S):
    # eps_in = -2 eps_out (Froehlich) makes Lambda = -2 pi / 3: z equals the dipole eigenvalue
    for eo in (1.0, 1.77):
        m = S.drude_metal_params(gamma_ev=0.0, eps_inf=1.0, eps_out=eo)
        wF = m["omega_p"] / math.sqrt(m["eps_inf"] + 2.0 * eo)
        assert abs(bem.eps_in(wF, m) + 2.0 * eo) < 1e-12
        z = bem.z_of_omega(wF, m)
        assert abs(z - 2.0 * math.pi / 3.0) < 1e-12
    # far above the plasma frequency eps_in -> eps_inf = eps_out: z -> infinity
    m = S.drude_metal_params()
    assert abs(bem.z_of_omega(1e3, m)) > 1e4


def test_real_spectrum_and_largest_eigenvalue(bem, S):
    n = 500
    s = S.spheroid_surface(n, 60.0, 30.0)
    A = bem.a_matrix(s["xyz"], s["normal"], s["area"], s["curvature"])
    ev = np.linalg.eigvals(A)
    assert np.abs(ev.imag).max() <= 1e-9 * np.abs(ev).max()
    assert abs(ev.real.max() / (2.0 * math.pi) - 1.0) < 0.5 / math.sqrt(n)


def test_rhs_is_normal_flux_of_the_field(bem, S):
    s = _sphere(S, 600, 10.0)
    for k in (KX, KY, KZ, np.array([1.0, 2.0, 2.0]) / 3.0):
        R = bem.rhs(s["normal"], s["area"], k, E0=0.5)
        # element i: -E0 a_i cos(angle between n_i and k); on a sphere n_i = r_i / R
        assert np.allclose(R, -0.5 * s["area"] * (s["xyz"] @ k) / 10.0, rtol=0, atol=1e-14)


def test_two_spheres_couple_as_point_dipoles(bem, S):
    # Two equal spheres a distance d apart, each much smaller than d, interact through
    # their induced dipoles: along the axis alpha_pair = 2 alpha / (1 - 2 alpha / d^3),
    # across it 2 alpha / (1 + alpha / d^3) (coupled point dipoles; the next multipole
    # corrections are O((R/d)^5)).  With alpha the same mesh's single-sphere value, the
    # collocation error cancels and what is left checks the operator's far blocks: the
    # field of one body's charges at the other's elements, with its sign.
    n, R, d = 1000, 10.0, 50.0
    s = S.spheroid_surface(n, R, R)
    two = {k: np.concatenate([v, v]) for k, v in s.items()}
    two["xyz"] = np.concatenate([s["xyz"] - [0.0, 0.0, d / 2], s["xyz"] + [0.0, 0.0, d / 2]])
    A1 = bem.a_matrix(s["xyz"], s["normal"], s["area"], s["curvature"])
    A2 = bem.a_matrix(two["xyz"], two["normal"], two["area"], two["curvature"])
    z = complex(-2.0 * math.pi * (1.0 + 5.0) / (1.0 - 5.0))     # static dielectric, eps_in = 5
    for k, g in ((2, 2.0), (0, -1.0)):
        kd = np.eye(3)[k]
        a1 = bem.alpha(s["xyz"], bem.solve(A1, z, bem.rhs(s["normal"], s["area"], kd)))[k]
        a2 = bem.alpha(two["xyz"], bem.solve(A2, z, bem.rhs(two["normal"], two["area"], kd)))[k]
        pred = 2.0 * a1 / (1.0 - g * a1 / d ** 3)
        assert abs(pred / (2.0 * a1) - 1.0) > 4e-3            # the coupling is visible ...
        assert abs(a2 / pred - 1.0) < 1e-4, (k, a2, pred)     # ... and has the dipole form


def _eps_from_drude_conductivity(omega, m):
    """The particle's permittivity rebuilt from its Drude conductivity in the time
    convention fixed by the paper's Drude factor 2 n0 / (1/tau - i w) (Eq. 5, Eq. 9):
    sigma(w) = (wp^2 / 4 pi) / (gamma - i w) and eps = eps_inf + 4 pi i sigma(w) / w."""
    sigma = m["omega_p"] ** 2 / (4.0 * math.pi) / (m["gamma"] - 1j * omega)
    return m["eps_inf"] + 4j * math.pi * sigma / omega


def _passivity_failures(bem, S):
    """Where a lossy particle (gamma > 0) is not passive: Im eps_in <= 0, eps_in off the
    conductivity form above, or a negative absorption Im alpha_kk of the sphere or of the
    2:1 spheroid (three frequencies, field along and across the axis)."""
    fails = []
    m = S.drude_metal_params()
    assert m["gamma"] > 0
    for w_ev in (0.5, 1.5, 2.5, 3.5, 4.5, 8.0):
        w = S.ev(w_ev)
        ei = bem.eps_in(w, m)
        if not ei.imag > 0:
            fails.append(("Im eps", w_ev, ei))
        ref = _eps_from_drude_conductivity(w, m)
        if abs(ei - ref) > 1e-13 * abs(ref):
            fails.append(("conductivity form", w_ev, ei, ref))
    for a, b, n in ((40.0, 40.0, 800), (60.0, 30.0, 1000)):
        s = S.spheroid_surface(n, a, b)
        A = bem.a_matrix(s["xyz"], s["normal"], s["area"], s["curvature"])
        for w_ev in (1.5, 2.5, 4.5):
            z = bem.z_of_omega(S.ev(w_ev), m)
            for k in (KX, KZ):
                q = bem.solve(A, z, bem.rhs(s["normal"], s["area"], k))
                al = bem.alpha(s["xyz"], q) @ k
                if not al.imag >= 0:
                    fails.append(("Im alpha", a, b, w_ev, al))
    return fails


def test_lossy_particle_is_passive(bem, S):
    # gamma > 0 absorbs: Im eps_in > 0, and Im alpha_kk >= 0 for every shape and field
    # (the omega-FQ oracle's modal pin asks the same of Im alpha)
    assert _passivity_failures(bem, S) == []


def test_passivity_pin_catches_flipped_damping(bem, S):
    # a copy of the BEM oracle with w (w - i gamma) in place of w (w + i gamma) -- a gain
    # medium -- fails the pin above
    import os
    src = open(os.path.join(os.path.dirname(bem.__file__), "bem.py")).read()
    old = 'w * (w + 1j * bem["gamma"])'
    assert src.count(old) == 1
    ns = {"__name__": "oracle.bem_planted", "__package__": "oracle"}
    exec(compile(src.replace(old, 'w * (w - 1j * bem["gamma"])'), "bem_planted", "exec"), ns)
    planted = type(bem)("bem_planted")
    planted.__dict__.update(ns)
    fails = _passivity_failures(planted, S)
    assert any(f[0] == "Im eps" for f in fails)
    assert any(f[0] == "Im alpha" for f in fails)
