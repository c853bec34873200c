"""vl_apply_A_noalloc against vl_apply(VL_OP_A), through the C ABI.

The no-allocation product serves callers that cannot allocate device memory at
call time (their memory already handed to a pool of their own, or a path that
must not enter the allocator); it keeps its intermediates in a fixed array built
into the library. It must give the same result as the workspace-based product,
call after call, and refuse problems larger than that array."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_apply_A_noalloc_matches_workspace_product():
    import torch

    import paper_2310_12000_gb300 as vl
    import workloads as wl
    P = wl.make_problem("c1_n2000", n=12000)
    ctx = vl.Context(0, ws_bytes=1 << 30)
    opts = vl.Opts.make(cg_tol=1e-10)
    fac = ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts)
    st = fac.find_mode(P.lik, P.y, P.F, opts)
    for call, t in enumerate((7, 7, 1, 40)):        # several calls in a row
        X = np.random.default_rng(call).standard_normal((P.n, t))
        ref = st.apply(vl.OP_A, X, opts)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.full_like(Xd, float("nan"))
        torch.cuda.synchronize()
        mem_before = ctx.mem()
        st.apply_A_noalloc(Xd, Yd)
        torch.cuda.synchronize()
        # the context workspace is not touched: neither its use nor its peak moves
        assert ctx.mem() == mem_before, (call, t)
        Y = Yd.cpu().numpy()
        assert np.max(np.abs(Y - ref)) <= 1e-12 * np.max(np.abs(ref)), (call, t)
    # beyond the fixed array: a clear error, nothing written
    Xd = torch.ones((P.n, 256), dtype=torch.float64, device="cuda")
    Yd = torch.zeros_like(Xd)
    with pytest.raises(vl.VLError) as e:
        st.apply_A_noalloc(Xd, Yd)
    assert "64 MiB" in str(e.value) and e.value.status == 1
    torch.cuda.synchronize()
    assert int(torch.count_nonzero(Yd)) == 0
    # host buffers are refused by the entry point (it has nowhere to stage them)
    with pytest.raises(vl.VLError) as e:
        st.apply_A_noalloc(np.zeros((P.n, 2)), Yd[:, :2].contiguous())
    assert "device pointers" in str(e.value)
