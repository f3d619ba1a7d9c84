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
        g.apply_mixed_noalloc(om, x, y)
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        # same kernels on the same inputs; the tolerance of the mixed-apply tests bounds any
        # difference far above what is seen (identical results)
        assert np.all(np.isfinite(a)), call
        assert np.abs(a - b).max() <= 4e-5 * np.abs(b).max(), call
    # sizes beyond the static array are refused with a clear error, nothing allocated:
    # 1500 columns need 4*3008*1536 + 8*1500*1500 bytes > 32 MiB
    wide = 1500
    xb = torch.zeros((n, wide), dtype=torch.complex64, device="cuda")
    yb = torch.empty_like(xb)
    with pytest.raises(wfq.WfqError) as e:
        g.apply_mixed_noalloc(S.ev(np.full(wide, 0.5)), xb, yb)
    assert e.value.code == -1 and "static" in str(e.value)
    # host pointers are refused (staging them would allocate)
    xh = np.zeros((n, 1), dtype=np.complex64)
    with pytest.raises(wfq.WfqError):
        g.apply_mixed_noalloc([0.02], xh, np.empty_like(xh))
    g.close()
    ctx.close()
