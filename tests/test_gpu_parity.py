"""GPU parity of libwfq against the FP64 CPU oracle (through the C ABI).

Tolerances:
  * integer / structural results (Kbar pair count): exact.
  * FP64 operator and FP64 solves: 1e-12 relative (operator), q and alpha to 1e-9 / 1e-10
    against LU (solution error <= cond * 1e-12 tolerance of the solve).
  * mixed operator (3 bf16 products, FP32 accumulation): per element,
        |dy_i| <= TAU_MIXED * (sum_p Kbar_ip (s_i + s_j) + |z| |x_i|),  s = |D| |x|,
    where TAU_MIXED covers the split error of D and x (each <= 2^-18 relative, three
    products -> 3 * 2^-18 = 1.1e-5) plus FP32 accumulation over N terms.
  * mixed solves (FP64 refinement): the acceptance bar -- alpha relative error <= 1e-6 and
    FP64 true residual <= 1e-8 relative, the residual re-measured by the oracle.
"""
import os
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TAU_MIXED = 4e-5


@pytest.fixture(scope="module")
def W():
    from paper_2103_00438_gb300 import wfq
    wfq.load()
    return wfq


@pytest.fixture(scope="module")
def ctx(W):
    c = W.Context(0)
    yield c
    c.close()


def _carbon(S, **kw):
    p = S.carbon_params(1.51)
    p.update(kw)
    return p


def _oracle_csr(orc, xyz, p):
    return orc.kbar_csr(xyz, p, cutoff_eps=p["cutoff_eps"])


# ----------------------------------------------------------------------------- structure

@pytest.mark.parametrize("n_rings", [3, 7, 13])
def test_kbar_pair_count_exact(W, ctx, orc, S, n_rings):
    xyz = S.honeycomb_flake(n_rings)
    p = _carbon(S)
    g = W.Geometry(ctx, xyz, p, store=W.STORE_FP64)
    rowptr, col, val = _oracle_csr(orc, xyz, p)
    assert g.info()["nnz"] == len(col)


def test_rhs_matches_oracle(W, ctx, orc, S):
    xyz = S.random_cluster(777, seed=21)
    p = _carbon(S, r0=2.7)
    g = W.Geometry(ctx, xyz, p, store=0)
    dirs = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0], [0.6, 0.8, 0.0]])
    R = g.rhs(dirs, E0=0.7)
    csr = _oracle_csr(orc, xyz, p)
    for d in range(4):
        ref = orc.rhs_csr(xyz, csr, dirs[d], E0=0.7)
        assert np.abs(R[:, d] - ref).max() <= 1e-13 * np.abs(ref).max()


# ----------------------------------------------------------------------------- operator

def _oracle_apply(orc, sysm, z, x):
    return orc.Operator.stored(sysm.D, sysm.csr).apply(z, x)


@pytest.mark.parametrize("n,store,ncplx", [(1000, "fp64", 1), (1333, "fp64", 3), (1333, "fp64", 7),
                                           (1100, "otf", 2), (1100, "otf", 5), (257, "otf", 1)])
def test_apply_fp64_matches_oracle(W, ctx, orc, S, n, store, ncplx):
    xyz = S.random_cluster(n, seed=n)
    p = _carbon(S, r0=2.7)
    g = W.Geometry(ctx, xyz, p, store=W.STORE_FP64 if store == "fp64" else 0)
    sysm = orc.System(xyz, p)
    om = S.ev(np.linspace(0.2, 1.9, ncplx))
    x = S.random_complex((n, ncplx), seed=5)
    y = np.empty_like(x)
    g.apply(om, x, y, prec=W.PREC_FP64)
    for c in range(ncplx):
        ref = _oracle_apply(orc, sysm, sysm.z(om[c]), x[:, c])
        assert np.abs(y[:, c] - ref).max() <= 1e-12 * np.abs(ref).max(), c


def _mixed_bound(sysm, z, x):
    s = np.abs(sysm.D) @ np.abs(x)
    K = sysm.K
    return K @ s + K.sum(axis=1) * s + abs(z) * np.abs(x)


@pytest.mark.parametrize("n,ncplx", [(1000, 1), (1337, 3), (2049, 8), (129, 2)])
def test_apply_mixed_within_derived_bound(W, ctx, orc, S, n, ncplx):
    xyz = S.random_cluster(n, seed=n + 1)
    p = _carbon(S, r0=2.7)
    g = W.Geometry(ctx, xyz, p, store=W.STORE_BF16X2)
    sysm = orc.System(xyz, p)
    om = S.ev(np.linspace(0.3, 1.5, ncplx))
    x = S.random_complex((n, ncplx), seed=9).astype(np.complex64)
    y = np.empty_like(x)
    g.apply(om, x, y, prec=W.PREC_MIXED)
    worst = 0.0
    for c in range(ncplx):
        z = sysm.z(om[c])
        xc = x[:, c].astype(np.complex128)
        ref = _oracle_apply(orc, sysm, z, xc)
        bound = _mixed_bound(sysm, z, xc)
        worst = max(worst, float(np.max(np.abs(y[:, c] - ref) / bound)))
    print("mixed apply: max |dy| / unit bound =", worst)
    assert worst <= TAU_MIXED


@pytest.mark.parametrize("n,ncplx,store", [(1000, 3, "fp64"), (1333, 7, "fp64"), (2049, 40, "fp64"),
                                           (1333, 7, "f32x2"), (2049, 40, "f32x2"), (1333, 7, "sym"),
                                           (2049, 40, "sym")])
def test_apply_double_float_within_derived_bound(W, ctx, orc, S, n, ncplx, store):
    """Double-float D products: operands split into float pairs (48 significant bits),
    products and sums error-free up to ~2^-48 each, so per element
        |dy_i| <= TAU_DF * (sum_p Kbar_ip (s_i + s_j) + |z| |x_i|),  s = |D| |x|,
    with TAU_DF = 8 * 2^-48 * sqrt(N): rounding errors of 2^-48 per step that add up
    like a random walk over the N-term sum, with a factor 8 of margin.  D split from the
    stored FP64 D, or read from the stored FP32 pair planes or symmetric pair tiles (the same
    48-bit pair; the tiles four real columns per pass, for any number of columns)."""
    TAU_DF = 8 * 2.0 ** -48 * np.sqrt(n)
    xyz = S.random_cluster(n, seed=n + 5)
    p = _carbon(S, r0=2.7)
    g = W.Geometry(ctx, xyz, p, store={"fp64": W.STORE_FP64, "f32x2": W.STORE_F32X2,
                                       "sym": W.STORE_F32X2_SYM}[store])
    sysm = orc.System(xyz, p)
    om = S.ev(np.linspace(0.2, 1.9, ncplx))
    x = S.random_complex((n, ncplx), seed=11)
    y = np.empty_like(x)
    g.apply(om, x, y, prec=W.PREC_DF)
    worst = 0.0
    for c in range(ncplx):
        z = sysm.z(om[c])
        ref = _oracle_apply(orc, sysm, z, x[:, c])
        worst = max(worst, float(np.max(np.abs(y[:, c] - ref) / _mixed_bound(sysm, z, x[:, c]))))
    print("double-float apply: max |dy| / unit bound =", worst)
    assert worst <= TAU_DF


@pytest.mark.parametrize("n,ncplx,store", [(1000, 1, "f32x2"), (1333, 4, "f32x2"), (1100, 2, "f32x2sym"),
                                           (1333, 3, "f32x2sym"), (200, 1, "f32x2sym")])
def test_apply_fp64_from_float_pairs_within_double_float_bound(W, ctx, orc, S, n, ncplx, store):
    """A geometry that stores only the float-pair D (full planes or symmetric tiles) applies
    WFQ_PREC_FP64 with the double-float product of those pairs (up to four columns): the
    double-float bound of the test above, TAU_DF = 8 * 2^-48 * sqrt(N)."""
    TAU_DF = 8 * 2.0 ** -48 * np.sqrt(n)
    xyz = S.random_cluster(n, seed=n + 9)
    p = _carbon(S, r0=2.7)
    g = W.Geometry(ctx, xyz, p, store=W.STORE_F32X2 if store == "f32x2" else W.STORE_F32X2_SYM)
    sysm = orc.System(xyz, p)
    om = S.ev(np.linspace(0.2, 1.9, ncplx))
    x = S.random_complex((n, ncplx), seed=12)
    y = np.empty_like(x)
    g.apply(om, x, y, prec=W.PREC_FP64)
    worst = 0.0
    for c in range(ncplx):
        z = sysm.z(om[c])
        ref = _oracle_apply(orc, sysm, z, x[:, c])
        worst = max(worst, float(np.max(np.abs(y[:, c] - ref) / _mixed_bound(sysm, z, x[:, c]))))
    print("FP64 apply from float pairs: max |dy| / unit bound =", worst)
    assert worst <= TAU_DF


@pytest.mark.parametrize("n,ncplx", [(1000, 1), (1337, 3), (2049, 8), (129, 2), (3000, 40)])
def test_apply_mixed_matrix_free_within_derived_bound(W, ctx, orc, S, n, ncplx):
    """Matrix-free tensor-core path: D tiles generated in FP32 from the coordinates and
    split into bf16 hi + lo in shared memory; same bound as the stored mixed path."""
    xyz = S.random_cluster(n, seed=n + 2)
    p = _carbon(S, r0=2.7)
    g = W.Geometry(ctx, xyz, p, store=0)
    sysm = orc.System(xyz, p)
    om = S.ev(np.linspace(0.3, 1.5, ncplx))
    x = S.random_complex((n, ncplx), seed=19).astype(np.complex64)
    y = np.empty_like(x)
    g.apply(om, x, y, prec=W.PREC_MIXED)
    worst = 0.0
    for c in range(ncplx):
        z = sysm.z(om[c])
        xc = x[:, c].astype(np.complex128)
        ref = _oracle_apply(orc, sysm, z, xc)
        worst = max(worst, float(np.max(np.abs(y[:, c] - ref) / _mixed_bound(sysm, z, xc))))
    print("matrix-free mixed apply: max |dy| / unit bound =", worst)
    assert worst <= TAU_MIXED


def test_matrix_free_equals_stored_mixed(W, ctx, S):
    """The generated tiles are the stored bf16 planes up to FP32 rounding of D: the two
    mixed applies agree far inside the mixed tolerance."""
    n = 2500
    xyz = S.random_cluster(n, seed=77)
    p = _carbon(S, r0=2.7)
    gs = W.Geometry(ctx, xyz, p, store=W.STORE_BF16X2)
    gm = W.Geometry(ctx, xyz, p, store=0)
    om = S.ev([0.4, 1.1])
    x = S.random_complex((n, 2), seed=4).astype(np.complex64)
    ys, ym = np.empty_like(x), np.empty_like(x)
    gs.apply(om, x, ys, prec=W.PREC_MIXED)
    gm.apply(om, x, ym, prec=W.PREC_MIXED)
    assert np.abs(ys - ym).max() <= 1e-4 * np.abs(ys).max()


@pytest.mark.parametrize("n,ncplx", [(1000, 2), (1333, 7), (2049, 20), (600, 40)])
def test_apply_double_float_matrix_free_within_derived_bound(W, ctx, orc, S, n, ncplx):
    """Matrix-free double-float product: far-pair 1/r from float-pair coordinates with one
    double-float Newton step on the FP32 rsqrt (entry error ~1e-13 relative), near pairs in
    FP64.  Per element |dy_i| <= TAU * (sum_p Kbar_ip (s_i + s_j) + |z| |x_i|) with
    TAU = 1e-12: entry error 1e-13 plus the double-float accumulation of the stored case."""
    xyz = S.random_cluster(n, seed=n + 9) + 37.0     # away from the origin: tests the coordinate split
    p = _carbon(S, r0=2.7)
    g = W.Geometry(ctx, xyz, p, store=0)
    sysm = orc.System(xyz, p)
    om = S.ev(np.linspace(0.2, 1.9, ncplx))
    x = S.random_complex((n, ncplx), seed=13)
    y = np.empty_like(x)
    g.apply(om, x, y, prec=W.PREC_DF)
    worst = 0.0
    for c in range(ncplx):
        z = sysm.z(om[c])
        ref = _oracle_apply(orc, sysm, z, x[:, c])
        worst = max(worst, float(np.max(np.abs(y[:, c] - ref) / _mixed_bound(sysm, z, x[:, c]))))
    print("matrix-free double-float apply: max |dy| / unit bound =", worst)
    assert worst <= 1e-12


def test_apply_device_pointers_and_stream(W, ctx, orc, S):
    torch = pytest.importorskip("torch")
    n, ncplx = 900, 4
    xyz = S.random_cluster(n, seed=31)
    p = _carbon(S, r0=2.7)
    g = W.Geometry(ctx, xyz, p, store=W.STORE_FP64 | W.STORE_BF16X2)
    om = S.ev([0.4, 0.8, 1.2, 1.6])
    x = S.random_complex((n, ncplx), seed=3)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        g.apply(om, xd, yd, prec=W.PREC_FP64, stream=st)
    st.synchronize()
    yh = np.empty_like(x)
    g.apply(om, x, yh, prec=W.PREC_FP64)
    assert np.array_equal(yd.cpu().numpy(), yh)


# ----------------------------------------------------------------------------- solves

@pytest.fixture(scope="module")
def flake(orc, S):
    wl = S.workload("flake1k")
    sysm = orc.System(wl["xyz"], wl["params"])
    om = float(wl["omega"][0])
    q_lu, _ = sysm.solve(om, np.array([1.0, 0, 0]), method="lu")
    return wl, sysm, om, q_lu


def test_gmres_fp64_flake1k_matches_lu(W, ctx, orc, flake):
    """The flake1k case: complex128 throughout, unrestarted GMRES to 1e-10, vs LU."""
    wl, sysm, om, q_lu = flake
    g = W.Geometry(ctx, wl["xyz"], wl["params"], store=W.STORE_FP64)
    q, st, status = g.solve_gmres([om], [[1.0, 0, 0]], m=0, rel_tol=1e-10, max_iter=2000, prec=W.PREC_FP64)
    assert status == "WFQ_OK" and st[0]["rel_residual"] <= 1e-10
    assert np.linalg.norm(q[:, 0] - q_lu) <= 1e-8 * np.linalg.norm(q_lu)
    a = g.polarizability(q)[0]
    a_ref = orc.alpha(wl["xyz"], q_lu)
    assert np.abs(a - a_ref).max() <= 1e-9 * np.abs(a_ref).max()
    assert abs(q[:, 0].sum()) <= 1e-10 * np.abs(q[:, 0]).sum()


@pytest.mark.parametrize("m", [0, 30])
def test_gmres_mixed_flake1k_acceptance(W, ctx, orc, flake, m):
    wl, sysm, om, q_lu = flake
    g = W.Geometry(ctx, wl["xyz"], wl["params"], store=W.STORE_FP64 | W.STORE_BF16X2)
    q, st, status = g.solve_gmres([om], [[1.0, 0, 0]], m=m, rel_tol=1e-8, max_iter=2000, prec=W.PREC_MIXED)
    assert status == "WFQ_OK", st
    a = g.polarizability(q)[0, 0]
    a_ref = orc.alpha(wl["xyz"], q_lu)[0]
    assert abs(a - a_ref) <= 1e-6 * abs(a_ref)
    z = sysm.z(om)
    R = sysm.rhs(np.array([1.0, 0, 0])).astype(complex)
    rr = sysm.operator().residual_norm(z, R, q[:, 0]) / np.linalg.norm(R)
    assert rr <= 1e-8 and abs(rr - st[0]["rel_residual"]) <= 1e-10
    print("mixed GMRES stats", st[0])


def test_gmres_mixed_matrix_free_flake1k_acceptance(W, ctx, orc, flake):
    """No D stored at all: matrix-free tensor-core inner products, FP64 recomputed
    residual; same acceptance bar."""
    wl, sysm, om, q_lu = flake
    g = W.Geometry(ctx, wl["xyz"], wl["params"], store=0)
    q, st, status = g.solve_gmres([om], [[1.0, 0, 0]], m=30, rel_tol=1e-8, max_iter=2000, prec=W.PREC_MIXED)
    assert status == "WFQ_OK", st
    a = g.polarizability(q)[0, 0]
    a_ref = orc.alpha(wl["xyz"], q_lu)[0]
    assert abs(a - a_ref) <= 1e-6 * abs(a_ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_qmr_flake1k(W, ctx, orc, flake, prec):
    wl, sysm, om, q_lu = flake
    g = W.Geometry(ctx, wl["xyz"], wl["params"], store=W.STORE_FP64 | W.STORE_BF16X2)
    P = W.PREC_FP64 if prec == "fp64" else W.PREC_MIXED
    q, st, status = g.solve_qmr([om], [[1.0, 0, 0]], rel_tol=1e-10 if prec == "fp64" else 1e-8,
                                max_iter=3000, prec=P)
    assert status == "WFQ_OK", st
    a = g.polarizability(q)[0, 0]
    a_ref = orc.alpha(wl["xyz"], q_lu)[0]
    assert abs(a - a_ref) <= (1e-9 if prec == "fp64" else 1e-6) * abs(a_ref)
    print("QMR", prec, st[0])


def test_qmr_iterates_match_oracle_qmr(W, ctx, orc, S):
    """Same method, two derivations: the GPU's direction-vector QMR recurrence and the
    oracle's smoothing of BCG iterates agree step by step (FP64, capped iterations)."""
    xyz = S.honeycomb_flake(6)
    p = _carbon(S)
    g = W.Geometry(ctx, xyz, p, store=W.STORE_FP64)
    sysm = orc.System(xyz, p)
    om = S.ev(0.9)
    R = sysm.rhs(np.array([1.0, 0, 0])).astype(complex)
    op = sysm.operator()
    for k in (1, 2, 5, 9):
        q, st, status = g.solve_qmr([om], [[1.0, 0, 0]], rel_tol=1e-14, max_iter=k, prec=W.PREC_FP64)
        qo, info = op.qmr(sysm.z(om), R, rel_tol=1e-300, max_iter=k)
        assert st[0]["iters"] == k
        assert np.linalg.norm(q[:, 0] - qo) <= 1e-10 * np.linalg.norm(qo), k


def test_gmres_iterates_match_oracle_gmres(W, ctx, orc, S):
    xyz = S.honeycomb_flake(6)
    p = _carbon(S)
    g = W.Geometry(ctx, xyz, p, store=W.STORE_FP64)
    sysm = orc.System(xyz, p)
    om = S.ev(0.7)
    R = sysm.rhs(np.array([0, 1.0, 0])).astype(complex)
    op = sysm.operator()
    for k in (1, 3, 8):
        q, st, _ = g.solve_gmres([om], [[0, 1.0, 0]], m=0, rel_tol=1e-14, max_iter=k, prec=W.PREC_FP64)
        qo, _ = op.gmres(sysm.z(om), R, restart=0, rel_tol=1e-300, max_iter=k)
        assert np.linalg.norm(q[:, 0] - qo) <= 1e-10 * np.linalg.norm(qo), k


def test_batched_columns_each_match_oracle(W, ctx, orc, S):
    """nfreq x ndir columns in one launch: each column equals its own oracle LU solve."""
    xyz = S.nanotube(5, 5, 30)          # 600 atoms, axis z
    p = S.carbon_params(1.04)
    g = W.Geometry(ctx, xyz, p, store=W.STORE_FP64 | W.STORE_BF16X2)
    sysm = orc.System(xyz, p)
    om = S.ev([0.15, 0.6, 1.1, 1.9])
    dirs = np.eye(3)
    for prec, tol, atol in ((W.PREC_FP64, 1e-11, 1e-8), (W.PREC_MIXED, 1e-8, 1e-6)):
        q, st, status = g.solve_gmres(om, dirs, m=40, rel_tol=tol, max_iter=4000, prec=prec)
        assert status == "WFQ_OK"
        al = g.polarizability(q)
        for f in range(4):
            for d in range(3):
                c = f * 3 + d
                q_lu, _ = sysm.solve(om[f], dirs[d], method="lu")
                a_ref = orc.alpha(xyz, q_lu)
                assert np.abs(al[c] - a_ref).max() <= atol * np.abs(a_ref).max(), (prec, f, d)
                assert st[c]["rel_residual"] <= tol


# ----------------------------------------------------------------------------- shifted GMRES

@pytest.mark.parametrize("store", ["f32x2", "f32x2sym"])
def test_shifted_gmres_iterates_match_oracle_gmres(W, ctx, orc, S, store):
    """After k Arnoldi steps every (omega, direction) column of the shifted solver holds
    the k-step unrestarted GMRES iterate of its own system (A - z(omega) I) q = R_dir:
    the Krylov space of A - zI from R does not depend on z.  D from the full FP32 pair
    planes or from the symmetric upper-triangle tiles (216 atoms: 4 tile rows, a ragged
    last tile)."""
    xyz = S.honeycomb_flake(6)
    p = _carbon(S)
    g = W.Geometry(ctx, xyz, p, store=W.STORE_F32X2 if store == "f32x2" else W.STORE_F32X2_SYM)
    sysm = orc.System(xyz, p)
    om = S.ev([0.3, 0.7, 1.4])
    dirs = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    op = sysm.operator()
    for k in (1, 3, 8):
        q, st, status = g.solve_gmres_shifted(om, dirs, m_max=k, rel_tol=1e-14, max_iter=k, prec=W.PREC_FP64)
        assert status == "WFQ_ENOCONV"
        for f in range(len(om)):
            for d in range(2):
                c = f * 2 + d
                assert st[c]["iters"] == k
                R = sysm.rhs(dirs[d]).astype(complex)
                qo, _ = op.gmres(sysm.z(om[f]), R, restart=0, rel_tol=1e-300, max_iter=k)
                assert np.linalg.norm(q[:, c] - qo) <= 1e-10 * np.linalg.norm(qo), (k, f, d)


@pytest.mark.parametrize("store", ["f32x2", "fp64", "f32x2sym"])
def test_shifted_gmres_columns_match_lu(W, ctx, orc, S, store):
    """All frequencies x directions from the shared real Arnoldi processes; each column's
    alpha equals its own oracle LU solve and its FP64 residual meets the tolerance without
    any block-GMRES continuation."""
    xyz = S.nanotube(5, 5, 30)          # 600 atoms, axis z
    p = S.carbon_params(1.04)
    flag = {"f32x2": W.STORE_F32X2, "fp64": W.STORE_FP64, "f32x2sym": W.STORE_F32X2_SYM}[store]
    g = W.Geometry(ctx, xyz, p, store=flag)
    sysm = orc.System(xyz, p)
    om = S.ev([0.15, 0.6, 1.1, 1.9])
    dirs = np.eye(3)
    q, st, status = g.solve_gmres_shifted(om, dirs, rel_tol=1e-10, max_iter=2000, prec=W.PREC_FP64)
    assert status == "WFQ_OK"
    al = g.polarizability(q)
    for f in range(4):
        for d in range(3):
            c = f * 3 + d
            q_lu, _ = sysm.solve(om[f], dirs[d], method="lu")
            a_ref = orc.alpha(xyz, q_lu)
            assert np.abs(al[c] - a_ref).max() <= 1e-8 * np.abs(a_ref).max(), (f, d)
            assert st[c]["rel_residual"] <= 1e-10 and st[c]["restarts"] == 0, st[c]
            assert abs(q[:, c].sum()) <= 1e-10 * np.abs(q[:, c]).sum()


def test_shifted_gmres_more_than_four_directions(W, ctx, orc, S):
    """Five field directions: the D product of the Arnoldi vectors runs in groups of at most
    four vectors (and the sparse term likewise); every column still equals its LU solve."""
    xyz = S.nanotube(5, 5, 15)
    p = S.carbon_params(1.04)
    g = W.Geometry(ctx, xyz, p, store=W.STORE_F32X2)
    sysm = orc.System(xyz, p)
    om = S.ev([0.4, 1.5])
    dirs = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0], [0.6, 0.8, 0], [0, 0.6, 0.8]])
    q, st, status = g.solve_gmres_shifted(om, dirs, rel_tol=1e-10, max_iter=2000, prec=W.PREC_FP64)
    assert status == "WFQ_OK"
    al = g.polarizability(q)
    for f in range(2):
        for d in range(5):
            c = f * 5 + d
            q_lu, _ = sysm.solve(om[f], dirs[d], method="lu")
            a_ref = orc.alpha(xyz, q_lu)
            assert np.abs(al[c] - a_ref).max() <= 1e-8 * np.abs(a_ref).max(), (f, d)


def test_shifted_gmres_capped_basis_continues_in_block_gmres(W, ctx, orc, S):
    """A basis cap far below the iterations needed: every column continues from its
    shifted iterate in mixed block GMRES(50) with FP64 refinement and meets the bar."""
    wl = S.workload("flake1k")
    xyz, p = wl["xyz"], wl["params"]
    g = W.Geometry(ctx, xyz, p, store=W.STORE_F32X2 | W.STORE_BF16X2)
    sysm = orc.System(xyz, p)
    om = S.ev([0.2, 0.52, 1.3])
    q, st, status = g.solve_gmres_shifted(om, [[1.0, 0, 0]], m_max=6, rel_tol=1e-8, max_iter=3000,
                                          prec=W.PREC_MIXED)
    assert status == "WFQ_OK"
    al = g.polarizability(q)
    for f in range(3):
        q_lu, _ = sysm.solve(om[f], np.array([1.0, 0, 0]), method="lu")
        a_ref = orc.alpha(xyz, q_lu)
        assert np.abs(al[f] - a_ref).max() <= 1e-6 * np.abs(a_ref).max(), f
        assert st[f]["rel_residual"] <= 1e-8 and st[f]["restarts"] >= 1 and st[f]["iters"] > 6


def test_shifted_gmres_bitwise_repeatable_across_contexts(W, S):
    """The shifted solver's D product is autotuned per context (the first product of a shape
    times every tiling); every tiling sums each row in the same order, so two contexts give
    bitwise-identical solutions whichever tilings they picked."""
    xyz = S.nanotube(5, 5, 60)
    p = S.carbon_params(1.04)
    om = S.ev([0.3, 1.2])
    out = []
    for _ in range(2):
        c = W.Context(0)
        g = W.Geometry(c, xyz, p, store=W.STORE_F32X2)
        q, st, status = g.solve_gmres_shifted(om, np.eye(3), rel_tol=1e-9, prec=W.PREC_FP64)
        assert status == "WFQ_OK"
        out.append(q.copy())
        g.close()
        c.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("store", ["bf16x2", "matrix_free"])
def test_mixed_apply_bitwise_repeatable_across_contexts(W, S, store):
    """The tensor-core GEMMs (stored planes and matrix-free) are autotuned per context: the
    first product of a shape times several pipeline depths and keeps the fastest.  The depth
    changes only how far loads run ahead, so two contexts agree bitwise whichever depth
    each picked, product after product."""
    xyz = S.random_cluster(2300, seed=12)
    p = dict(S.carbon_params(1.2), r0=2.7)
    om = S.ev(np.linspace(0.2, 1.6, 24))
    x = S.random_complex((len(xyz), 24), seed=13).astype(np.complex64)
    out = []
    for _ in range(2):
        c = W.Context(0)
        g = W.Geometry(c, xyz, p, store=W.STORE_BF16X2 if store == "bf16x2" else 0)
        ys = [g.apply(om, x, np.empty_like(x), prec=W.PREC_MIXED) for _ in range(2)]
        assert np.array_equal(ys[0], ys[1])
        out.append(ys[1])
        g.close()
        c.close()
    assert np.array_equal(out[0], out[1])


def test_shifted_gmres_symmetric_tiles_equal_full_planes(W, ctx, S):
    """The symmetric tiled D (each stored tile used for D_IJ x_J and D_IJ^T x_I) gives the
    same solves as the full FP32 pair planes up to double-float rounding: 3000 atoms, 47 tile
    rows (a ragged last tile), several work items per tile row."""
    xyz = S.random_cluster(3000, seed=9)
    p = _carbon(S, r0=2.7)
    om = S.ev([0.35, 1.1])
    ga = W.Geometry(ctx, xyz, p, store=W.STORE_F32X2)
    gb = W.Geometry(ctx, xyz, p, store=W.STORE_F32X2_SYM)
    qa, sa, st_a = ga.solve_gmres_shifted(om, np.eye(3), rel_tol=1e-10, prec=W.PREC_FP64)
    qb, sb, st_b = gb.solve_gmres_shifted(om, np.eye(3), rel_tol=1e-10, prec=W.PREC_FP64)
    assert st_a == "WFQ_OK" and st_b == "WFQ_OK"
    assert [s["iters"] for s in sa] == [s["iters"] for s in sb]
    assert np.linalg.norm(qa - qb) <= 1e-10 * np.linalg.norm(qa)
    assert max(s["rel_residual"] for s in sb) <= 1e-10


def test_shifted_gmres_matrix_free_matches_lu(W, ctx, orc, S):
    """No D stored: the shifted solver regenerates D from the coordinates in double-float
    for every product (near pairs in FP64); every column equals its LU solve."""
    xyz = S.nanotube(5, 5, 30)          # 600 atoms
    p = S.carbon_params(1.04)
    g = W.Geometry(ctx, xyz, p, store=0)
    sysm = orc.System(xyz, p)
    om = S.ev([0.2, 1.3])
    dirs = np.eye(3)[:2]
    q, st, status = g.solve_gmres_shifted(om, dirs, rel_tol=1e-10, max_iter=2000, prec=W.PREC_FP64)
    assert status == "WFQ_OK"
    al = g.polarizability(q)
    for f in range(2):
        for d in range(2):
            c = f * 2 + d
            q_lu, _ = sysm.solve(om[f], dirs[d], method="lu")
            a_ref = orc.alpha(xyz, q_lu)
            assert np.abs(al[c] - a_ref).max() <= 1e-8 * np.abs(a_ref).max(), (f, d)
            assert st[c]["rel_residual"] <= 1e-10 and st[c]["restarts"] == 0


@pytest.mark.parametrize("solver", ["gmres", "qmr"])
def test_fp64_solvers_matrix_free_match_lu(W, ctx, orc, S, solver):
    """No D stored: the FP64 block GMRES and QMR iterations and their true residuals take
    the double-float products that regenerate D per product (~2^-48 each, far below the
    requested residual); every column still equals its LU solve."""
    xyz = S.nanotube(5, 5, 30)          # 600 atoms
    p = S.carbon_params(1.04)
    g = W.Geometry(ctx, xyz, p, store=0)
    sysm = orc.System(xyz, p)
    om = S.ev([0.2, 1.3])
    dirs = np.eye(3)[:2]
    if solver == "gmres":
        q, st, status = g.solve_gmres(om, dirs, m=60, rel_tol=1e-10, max_iter=3000, prec=W.PREC_FP64)
    else:
        q, st, status = g.solve_qmr(om, dirs, rel_tol=1e-10, max_iter=3000, prec=W.PREC_FP64)
    assert status == "WFQ_OK", st
    al = g.polarizability(q)
    for f in range(2):
        for d in range(2):
            c = f * 2 + d
            q_lu, _ = sysm.solve(om[f], dirs[d], method="lu")
            a_ref = orc.alpha(xyz, q_lu)
            assert np.abs(al[c] - a_ref).max() <= 1e-8 * np.abs(a_ref).max(), (solver, f, d)
            assert st[c]["rel_residual"] <= 1e-10


@pytest.mark.parametrize("solver", ["gmres", "qmr"])
def test_mixed_solvers_on_symmetric_pair_tiles_match_lu(W, ctx, orc, S, solver):
    """The storage of the 150k-atom sphere's solver comparison: bf16 planes for the mixed
    iterations, symmetric FP32 pair tiles for the refinement residuals (their double-float
    product, four real columns per pass, 12 columns here); every column meets the acceptance
    bar against its LU solve."""
    xyz = S.nanotube(5, 5, 30)          # 600 atoms
    p = S.carbon_params(1.04)
    g = W.Geometry(ctx, xyz, p, store=W.STORE_F32X2_SYM | W.STORE_BF16X2)
    sysm = orc.System(xyz, p)
    om = S.ev([0.3, 0.9, 1.3, 1.8])
    dirs = np.eye(3)
    if solver == "gmres":
        q, st, status = g.solve_gmres(om, dirs, m=30, rel_tol=1e-8, max_iter=4000, prec=W.PREC_MIXED)
    else:
        q, st, status = g.solve_qmr(om, dirs, rel_tol=1e-8, max_iter=4000, prec=W.PREC_MIXED)
    assert status == "WFQ_OK", st
    al = g.polarizability(q)
    for f in range(len(om)):
        for d in range(3):
            c = f * 3 + d
            q_lu, _ = sysm.solve(om[f], dirs[d], method="lu")
            a_ref = orc.alpha(xyz, q_lu)
            assert np.abs(al[c] - a_ref).max() <= 1e-6 * np.abs(a_ref).max(), (solver, f, d)
            assert st[c]["rel_residual"] <= 1e-8


# ----------------------------------------------------------------------------- edge cases

def test_edge_single_atom_and_dimer(W, ctx, orc, S):
    p = _carbon(S)
    g1 = W.Geometry(ctx, np.zeros((1, 3)), p, store=W.STORE_FP64)
    q, st, status = g1.solve_gmres([0.02], [[1.0, 0, 0]], prec=W.PREC_FP64)
    assert status == "WFQ_OK" and np.all(q == 0)
    a = 3.1
    xyz = np.array([[0.0, 0, 0], [a, 0, 0]])
    g2 = W.Geometry(ctx, xyz, p, store=W.STORE_FP64 | W.STORE_BF16X2)
    om = 0.03
    q, st, status = g2.solve_gmres([om], [[1.0, 0, 0]], rel_tol=1e-12, prec=W.PREC_FP64)
    k12 = orc.kbar_entry(a, p)
    d12 = orc.d_matrix(xyz, p["eta"])[0, 1]
    ref = k12 * a * a / (2 * k12 * (p["eta"] - d12) + orc.z_of_omega(om, p))
    assert abs(g2.polarizability(q)[0, 0] - ref) <= 1e-11 * abs(ref)


def test_edge_field_normal_to_flake_gives_zero(W, ctx, S):
    xyz = S.honeycomb_flake(4)
    g = W.Geometry(ctx, xyz, _carbon(S), store=W.STORE_BF16X2)
    q, st, status = g.solve_gmres(S.ev([0.5]), [[0, 0, 1.0]], prec=W.PREC_MIXED)
    assert status == "WFQ_OK" and np.all(q == 0)


def test_edge_errors(W, ctx, S):
    p = _carbon(S)
    xyz = S.honeycomb_flake(3)
    g = W.Geometry(ctx, xyz, p, store=W.STORE_FP64)
    with pytest.raises(W.WfqError) as e:
        g.solve_gmres([0.0], [[1.0, 0, 0]])
    assert e.value.code == -2                       # omega = 0 (singular)
    with pytest.raises(W.WfqError) as e:
        g.solve_gmres([0.02], [[1.0, 0, 0]], prec=7)
    assert e.value.code == -1                       # unknown precision
    dup = np.vstack([xyz, xyz[:1]])
    with pytest.raises(W.WfqError) as e:
        W.Geometry(ctx, dup, p)
    assert e.value.code == -1                       # r_ij = 0
    bad = xyz.copy()
    bad[2, 1] = np.nan
    with pytest.raises(W.WfqError):
        W.Geometry(ctx, bad, p)
    with pytest.raises(W.WfqError):
        W.Geometry(ctx, xyz, dict(p, tau=-1.0))
    q, st, status = g.solve_gmres([0.02], [[1.0, 0, 0]], max_iter=2, rel_tol=1e-12)
    assert status == "WFQ_ENOCONV" and st[0]["iters"] == 2


def test_edge_dense_kbar_no_cutoff(W, ctx, orc, S):
    xyz = S.random_cluster(300, seed=44)
    p = _carbon(S, r0=2.7, cutoff_eps=0.0)
    g = W.Geometry(ctx, xyz, p, store=W.STORE_FP64)
    assert g.info()["nnz"] == 300 * 299
    sysm = orc.System(xyz, p)
    om = S.ev(0.8)
    x = S.random_complex((300, 1), seed=1)
    y = np.empty_like(x)
    g.apply([om], x, y)
    ref = _oracle_apply(orc, sysm, sysm.z(om), x[:, 0])
    assert np.abs(y[:, 0] - ref).max() <= 1e-12 * np.abs(ref).max()


# ----------------------------------------------------------------------------- full size

@pytest.mark.slow
def test_cnt20k_full_size_mixed_block_gmres(W, ctx, orc, S):
    """The cnt20k workload as the bench runs it (64 frequencies x 3 directions, mixed
    GMRES(50) with FP64 refinement): every column's FP64 residual <= 1e-8; sampled
    columns re-checked by the oracle's own operator (on-the-fly D, its own CSR)."""
    wl = S.workload("cnt20k")
    xyz, p = wl["xyz"], wl["params"]
    g = W.Geometry(ctx, xyz, p, store=W.STORE_FP64 | W.STORE_BF16X2)
    q, st, status = g.solve_gmres(wl["omega"], wl["dirs"], m=50, rel_tol=1e-8, max_iter=3000,
                                  prec=W.PREC_MIXED)
    assert status == "WFQ_OK"
    assert max(s["rel_residual"] for s in st) <= 1e-8
    csr = _oracle_csr(orc, xyz, p)
    op = orc.Operator.on_the_fly(xyz, p["eta"], csr)
    rng = np.random.default_rng(7)
    for c in rng.choice(q.shape[1], size=3, replace=False):
        f, d = divmod(int(c), 3)
        R = orc.rhs_csr(xyz, csr, wl["dirs"][d]).astype(complex)
        rr = op.residual_norm(orc.z_of_omega(wl["omega"][f], p), R, q[:, c]) / np.linalg.norm(R)
        assert rr <= 1.2e-8, (c, rr)
        assert abs(q[:, c].sum()) <= 1e-9 * np.abs(q[:, c]).sum()


@pytest.mark.slow
@pytest.mark.parametrize("solver", ["gmres", "qmr"])
def test_mixed_low_frequency_large_flake_meets_bar(W, ctx, orc, S, solver):
    """Low frequencies on a 15,000-atom flake with the field in plane: ||A|| ||q|| / ||R|| is
    large there, so the mixed refinement (double-float residuals) stalls just above the
    1e-8 bar; such columns are finished by FP64 GMRES from the mixed iterate (for mixed GMRES
    and mixed QMR alike).  Every column must meet the bar, re-measured by the oracle's
    operator, and the first column's alpha must match the oracle's own FP64 GMRES solution
    to 1e-6."""
    xyz = S.honeycomb_flake(50)
    p = S.carbon_params(1.51)
    om = S.ev(np.array([0.0555, 0.067, 0.3]))
    g = W.Geometry(ctx, xyz, p, store=W.STORE_FP64 | W.STORE_BF16X2)
    if solver == "gmres":
        q, st, status = g.solve_gmres(om, [[1.0, 0, 0]], m=50, rel_tol=1e-8, max_iter=3000, prec=W.PREC_MIXED)
    else:
        q, st, status = g.solve_qmr(om, [[1.0, 0, 0]], rel_tol=1e-8, max_iter=3000, prec=W.PREC_MIXED)
    assert status == "WFQ_OK", st
    assert max(s["rel_residual"] for s in st) <= 1e-8
    csr = _oracle_csr(orc, xyz, p)
    op = orc.Operator.stored(orc.d_matrix(xyz, p["eta"]), csr)
    R = orc.rhs_csr(xyz, csr, np.array([1.0, 0, 0])).astype(complex)
    for c in range(len(om)):
        rr = op.residual_norm(orc.z_of_omega(om[c], p), R, q[:, c]) / np.linalg.norm(R)
        assert rr <= 1.2e-8, (c, rr)
    q_ref, info = op.gmres(orc.z_of_omega(om[0], p), R, restart=50, rel_tol=1e-11, max_iter=20000)
    assert info["status"] == 0
    a = g.polarizability(q[:, :1])[0]
    a_ref = orc.alpha(xyz, q_ref)
    assert np.abs(a - a_ref).max() <= 1e-6 * np.abs(a_ref).max()


@pytest.mark.slow
@pytest.mark.parametrize("name", ["disk1m", "sphere150k"])
def test_full_size_mixed_apply_sampled_rows(W, ctx, orc, S, name):
    """The two large workloads in the launch configuration the bench times (all columns of
    the workload in one mixed apply; matrix-free for the 1M-atom disk, stored bf16 planes
    for the 150k sphere): sampled rows against the oracle, which recomputes each row from
    Eq. 3 with a brute-force neighbour scan, within the mixed per-element bound."""
    wl = S.workload(name)
    xyz, p = wl["xyz"], wl["params"]
    n = len(xyz)
    store = 0 if name == "disk1m" else W.STORE_BF16X2
    g = W.Geometry(ctx, xyz, p, store=store)
    ncplx = len(wl["omega"]) * len(wl["dirs"])
    omc = np.repeat(wl["omega"], len(wl["dirs"]))
    rng = np.random.default_rng(5)
    x = ((rng.standard_normal((n, ncplx)) + 1j * rng.standard_normal((n, ncplx))) / np.sqrt(2)).astype(np.complex64)
    y = np.empty_like(x)
    g.apply(omc, x, y, prec=W.PREC_MIXED)
    rows = rng.choice(n, size=12, replace=False)
    for c in (0, ncplx - 1):
        yo, bnd = orc.apply_rows(xyz, p, orc.z_of_omega(omc[c], p), x[:, c].astype(complex), rows)
        ratio = float(np.max(np.abs(y[rows, c] - yo) / bnd))
        print(name, "column", c, "max |dy| / unit bound =", ratio)
        assert ratio <= TAU_MIXED
    g.close()


def test_solver_trace_on_stderr(S):
    """WFQ_TRACE=1: the solvers report each restart cycle on stderr; unset, nothing."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("from paper_2103_00438_gb300 import wfq, structures as S\n"
            "ctx = wfq.Context(0)\n"
            "g = wfq.Geometry(ctx, S.honeycomb_flake(6), S.carbon_params(1.51), store=wfq.STORE_BF16X2)\n"
            "q, st, status = g.solve_gmres(S.ev([0.6]), [[1.0, 0, 0]], m=20, rel_tol=1e-8, prec=wfq.PREC_MIXED)\n"
            "assert status == 'WFQ_OK', st\n")
    for flag, expect in (("1", True), ("0", False)):
        env = dict(os.environ, WFQ_TRACE=flag)
        r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                           timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        lines = [ln for ln in r.stderr.splitlines() if ln.startswith("[wfq")]
        if expect:
            assert any("gmres(20) mixed cycle" in ln for ln in lines), r.stderr[-2000:]
        else:
            assert not lines
