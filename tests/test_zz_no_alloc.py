"""wfq_apply_mixed_noalloc -- the mixed apply for callers that cannot allocate device
memory (fixed arenas, contexts where cudaMalloc is not allowed) -- must give what the
allocating wfq_apply(..., WFQ_PREC_MIXED) gives, call after call, using only its static
scratch array.  Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_apply_matches_allocating_apply_twice(S):
    torch = pytest.importorskip("torch")
    from paper_2103_00438_gb300 import wfq
    ctx = wfq.Context(0)
    n = 1500
    xyz = S.random_cluster(n, seed=77)
    p = S.carbon_params(1.51)
    p["r0"] = 2.7
    g = wfq.Geometry(ctx, xyz, p, store=wfq.STORE_BF16X2)
    # two calls in a row with different sizes and inputs: the second must not see the
    # first one's leftovers in the shared array
    for call, (ncplx, seed) in enumerate(((5, 1), (3, 2))):
        om = S.ev(np.linspace(0.2, 1.7, ncplx))
        x = torch.from_numpy(S.random_complex((n, ncplx), seed=seed).astype(np.complex64)).cuda()
        y_ref = torch.empty_like(x)
        y = torch.full_like(x, float("nan"))
        g.apply(om, x, y_ref, prec=wfq.PREC_MIXED)
        torch.cuda.synchronize()
        before, free_before = ctx.memory_stats(), torch.cuda.mem_get_info()[0]
        g.apply_mixed_noalloc(om, x, y)
        torch.cuda.synchronize()
        after, free_after = ctx.memory_stats(), torch.cuda.mem_get_info()[0]
        if call > 0:
            # set-up (the array's address) is done by the first call; from then on the
            # library requests no device memory and the device's free memory does not move
            assert after["allocs"] == before["allocs"], (before, after)
            assert after["pool_reserved"] == before["pool_reserved"], (before, after)
            assert after["pool_used_high"] == before["pool_used_high"], (before, after)
            assert free_after == free_before, (free_before, free_after)
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        # same kernels on the same inputs; the tolerance of the mixed-apply tests bounds any
        # difference far above what is seen (identical results)
        assert np.all(np.isfinite(a)), call
        assert np.abs(a - b).max() <= 4e-5 * np.abs(b).max(), call
    # more columns than the frequency argument holds are refused with a clear error
    wide = 1500
    xb = torch.zeros((n, wide), dtype=torch.complex64, device="cuda")
    yb = torch.empty_like(xb)
    with pytest.raises(wfq.WfqError) as e:
        g.apply_mixed_noalloc(S.ev(np.full(wide, 0.5)), xb, yb)
    assert e.value.code == -1 and "1024" in str(e.value)
    # host pointers are refused (staging them would allocate)
    xh = np.zeros((n, 1), dtype=np.complex64)
    with pytest.raises(wfq.WfqError):
        g.apply_mixed_noalloc([0.02], xh, np.empty_like(xh))
    g.close()
    # sizes beyond the static array are refused with a clear error: 4000 atoms x 600
    # columns need 4*1216*4096 + 8*4000*600 + 9600 bytes > 32 MiB
    n2 = 4000
    g2 = wfq.Geometry(ctx, S.random_cluster(n2, seed=78), p, store=wfq.STORE_BF16X2)
    x2 = torch.zeros((n2, 600), dtype=torch.complex64, device="cuda")
    with pytest.raises(wfq.WfqError) as e:
        g2.apply_mixed_noalloc(S.ev(np.full(600, 0.5)), x2, torch.empty_like(x2))
    assert e.value.code == -1 and "static" in str(e.value)
    g2.close()
    ctx.close()
