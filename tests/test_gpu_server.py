"""Serving: requests submitted at once over several resident structures are merged into
block solves (continuous batching) and run on concurrent streams; every request's result
equals the same request solved alone (wfq_solve_gmres) and the FP64 oracle's LU solution,
within the acceptance tolerance (alpha relative error 1e-6; both residuals <= 1e-8).
Admission counts the device bytes of the structures in use against the budget."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_server_results_same_alone_and_in_the_mix(S, orc):
    from paper_2103_00438_gb300 import wfq
    ctx = wfq.Context(0)
    # stored D: batches run shifted GMRES; the bf16-only geometry: mixed block GMRES
    store = wfq.STORE_F32X2 | wfq.STORE_BF16X2
    inputs = [(S.honeycomb_flake(10), S.carbon_params(1.51), store),
              (S.nanotube(5, 5, 40), S.carbon_params(1.04), wfq.STORE_FP64),
              (S.random_cluster(900, seed=4), dict(S.carbon_params(1.2), r0=2.7), wfq.STORE_BF16X2)]
    geoms = [wfq.Geometry(ctx, xyz, p, store=st) for xyz, p, st in inputs]
    systems = [orc.System(xyz, p) for xyz, p, _ in inputs]
    rng = np.random.default_rng(7)
    reqs = []
    for k in range(14):
        gi = int(rng.integers(0, len(geoms)))
        nf = int(rng.integers(1, 6))
        nd = int(rng.integers(1, 4))
        om = S.ev(np.sort(rng.uniform(0.1, 1.9, size=nf)))
        dirs = np.eye(3)[:nd]
        reqs.append((gi, om, dirs))
    sv = wfq.Server(ctx, nworkers=3, budget_bytes=8 << 30, max_columns=48)
    ids = [sv.submit(geoms[gi], om, dirs, m=30, rel_tol=1e-8) for gi, om, dirs in reqs]
    res = [sv.poll(i, wait=True) for i in ids]
    sv.close()
    merged = 0
    for (gi, om, dirs), r in zip(reqs, res):
        assert r["status"] == "WFQ_OK", r["stats"]
        assert max(s["rel_residual"] for s in r["stats"]) <= 1e-8
        ncols = len(om) * len(dirs)
        merged += r["batch_columns"] > ncols
        g = geoms[gi]
        q_alone, st, status = g.solve_gmres(om, dirs, m=30, rel_tol=1e-8, max_iter=4000, prec=wfq.PREC_MIXED)
        assert status == "WFQ_OK"
        a_mix = g.polarizability(r["q"])
        a_alone = g.polarizability(q_alone)
        assert np.abs(a_mix - a_alone).max() <= 1e-6 * np.abs(a_alone).max()
        assert r["latency_s"] >= r["queue_s"] >= 0.0
        # the first and the last column of the request against the oracle's LU solve
        for c in {0, ncols - 1}:
            f, d = divmod(c, len(dirs))
            q_lu, _ = systems[gi].solve(om[f], dirs[d], method="lu")
            a_ref = orc.alpha(inputs[gi][0], q_lu)
            assert np.abs(a_mix[c] - a_ref).max() <= 1e-6 * np.abs(a_ref).max(), (gi, c)
    assert merged >= 2, "no request shared a block solve"
    for g in geoms:
        g.close()
    ctx.close()


def test_server_rejects_bad_requests(S):
    from paper_2103_00438_gb300 import wfq
    ctx = wfq.Context(0)
    g = wfq.Geometry(ctx, S.honeycomb_flake(4), S.carbon_params(1.51), store=wfq.STORE_BF16X2)
    sv = wfq.Server(ctx, nworkers=1, budget_bytes=1 << 20, max_columns=8)
    with pytest.raises(wfq.WfqError) as e:
        sv.submit(g, [0.0], [[1, 0, 0]])
    assert e.value.code == -2
    with pytest.raises(wfq.WfqError) as e:
        sv.submit(g, S.ev(np.linspace(0.2, 1.0, 5)), np.eye(3))   # 15 columns > 8
    assert e.value.code == -1
    sv.close()
    g.close()
    ctx.close()


def test_server_admission_counts_resident_structures(S):
    """A structure's device bytes count against the budget while it has requests: a
    request whose structure alone fills the budget is refused, and two structures that
    each fit with their batch but not together run one after the other."""
    from paper_2103_00438_gb300 import wfq
    ctx = wfq.Context(0)
    p = S.carbon_params(1.04)
    ga = wfq.Geometry(ctx, S.nanotube(5, 5, 300), p, store=wfq.STORE_F32X2)    # 6000 atoms
    gb = wfq.Geometry(ctx, S.nanotube(5, 5, 250), p, store=wfq.STORE_F32X2)    # 5000 atoms
    ba, bb = ga.info()["device_bytes"], gb.info()["device_bytes"]
    om, kz = S.ev(np.linspace(0.2, 1.6, 4)), np.array([[0.0, 0.0, 1.0]])
    # the structure fills the budget: refused at submit
    sv = wfq.Server(ctx, nworkers=2, budget_bytes=ba + (1 << 20), max_columns=64)
    with pytest.raises(wfq.WfqError) as e:
        sv.submit(ga, om, kz)
    assert e.value.code == -3
    sv.close()
    # each structure fits with its batch (a batch's footprint, ~70 MB for 4 columns of one
    # direction, is well below the other structure's ~200 MB), both together do not: the
    # second waits for the first
    runs = {}
    for label, budget in (("tight", ba + bb), ("ample", 8 * (ba + bb))):
        sv = wfq.Server(ctx, nworkers=2, budget_bytes=budget, max_columns=64)
        ia = sv.submit(ga, om, kz)
        ib = sv.submit(gb, om, kz)
        ra, rb = sv.poll(ia, wait=True), sv.poll(ib, wait=True)
        sv.close()
        assert ra["status"] == "WFQ_OK" and rb["status"] == "WFQ_OK"
        runs[label] = (ra, rb)
    ra, rb = runs["tight"]
    assert rb["queue_s"] >= ra["latency_s"] - 5e-3, (ra["latency_s"], rb["queue_s"])
    ra, rb = runs["ample"]
    assert rb["queue_s"] < 0.5 * ra["latency_s"], (ra["latency_s"], rb["queue_s"])
    ga.close()
    gb.close()
    ctx.close()
