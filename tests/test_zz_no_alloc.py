"""The neighbour-list entry point that allocates nothing, against the lists a
context builds (the existing entry point mix_get_neighbours), on two calls in
a row.

It exists for callers that may not call cudaMalloc -- a plugin whose host
program owns every device allocation, or a loop that cannot take the
synchronisation an allocation implies; its scratch is a fixed array inside the
library.  Neighbour lists are integer work, so the comparison is exact.  This
file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2502_19081_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mx():
    from paper_2502_19081_gb300 import build, mix
    build.build()
    return mix


def _lists_from_noalloc(mx, torch, ctx, wl):
    n, cap = ctx.n, ctx.cap
    nnb = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    nbr = torch.full((n, cap), -1, dtype=torch.int32, device="cuda")
    rev = torch.full((n, cap), -1, dtype=torch.int32, device="cuda")
    r_list = max(wl.ace.r_cut, wl.spline.r_cut) + wl.skin
    s = wl.system
    st = mx.neighbours_noalloc(ctx.x[:n], s.box_lo, s.box_len, s.periodic, r_list, cap, nnb, nbr, rev)
    torch.cuda.synchronize()
    return st, nnb.cpu().numpy(), nbr.cpu().numpy(), rev.cpu().numpy()


def test_noalloc_lists_equal_context_lists_two_calls(mx):
    import torch
    for wl in (I.small_fe_box(31, r_core=4.0, ramp=3.0), I.si_vacancy()):
        ctx = mx.open_context(wl)
        nnb, nbr, rev = ctx.neighbours()
        st, nnb2, nbr2, rev2 = _lists_from_noalloc(mx, torch, ctx, wl)
        assert st == mx.MIX_OK
        assert np.array_equal(nnb, nnb2)
        for i in range(ctx.n):
            m = nnb[i]
            assert np.array_equal(nbr[i, :m], nbr2[i, :m]), i
            assert np.array_equal(rev[i, :m], rev2[i, :m]), i
        ctx.close()


def test_noalloc_allocates_no_device_memory(mx):
    """After a first call (which loads the library's kernels), further calls
    leave the device's free memory unchanged."""
    import torch
    wl = I.small_fe_box(32, r_core=4.0, ramp=3.0)
    ctx = mx.open_context(wl)
    _lists_from_noalloc(mx, torch, ctx, wl)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        st, _, _, _ = _lists_from_noalloc(mx, torch, ctx, wl)
        assert st == mx.MIX_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ctx.close()


def test_noalloc_reports_bad_positions(mx):
    """A non-finite coordinate, and one outside a non-periodic dimension, are
    reported as by the context path (MIX_ENUMERIC, MIX_EBOX)."""
    import torch
    wl = I.cluster_workload(33, n=20)
    s = wl.system
    nbr = torch.zeros((20, 64), dtype=torch.int32, device="cuda")
    rev = torch.zeros((20, 64), dtype=torch.int32, device="cuda")
    nnb = torch.zeros(20, dtype=torch.int32, device="cuda")
    x = torch.from_numpy(np.ascontiguousarray(s.x)).cuda()
    assert mx.neighbours_noalloc(x, s.box_lo, s.box_len, s.periodic, 5.8, 64, nnb, nbr, rev) == mx.MIX_OK
    xn = x.clone()
    xn[3, 1] = float("nan")
    assert mx.neighbours_noalloc(xn, s.box_lo, s.box_len, s.periodic, 5.8, 64, nnb, nbr, rev) == mx.MIX_ENUMERIC
    xo = x.clone()
    xo[5, 0] = float(s.box_lo[0] + s.box_len[0] + 1.0)
    assert mx.neighbours_noalloc(xo, s.box_lo, s.box_len, s.periodic, 5.8, 64, nnb, nbr, rev) == mx.MIX_EBOX


def test_noalloc_checks_its_arguments(mx):
    import torch
    x = torch.zeros((8, 4), dtype=torch.float64, device="cuda")
    small = torch.zeros((8, 10), dtype=torch.int32, device="cuda")
    nnb = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):       # nbr smaller than N x cap
        mx.neighbours_noalloc(x, (0, 0, 0), (50.0, 50.0, 50.0), (1, 1, 1), 5.8, 64, nnb, small, small)
    with pytest.raises(ValueError):       # float32 positions
        mx.neighbours_noalloc(x.float(), (0, 0, 0), (50.0, 50.0, 50.0), (1, 1, 1), 5.8, 10, nnb, small, small)
    with pytest.raises(ValueError):       # [N, 3] positions
        mx.neighbours_noalloc(x[:, :3].contiguous(), (0, 0, 0), (50.0, 50.0, 50.0), (1, 1, 1), 5.8, 10, nnb,
                              small, small)


def test_noalloc_rejects_sizes_beyond_its_limit(mx):
    import torch
    x = torch.zeros((8, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros((8, 300), dtype=torch.int32, device="cuda")
    big = torch.zeros((33000, 64), dtype=torch.int32, device="cuda")
    nb1 = torch.zeros(33000, dtype=torch.int32, device="cuda")
    too_many = torch.zeros((33000, 4), dtype=torch.float64, device="cuda")
    st = mx.neighbours_noalloc(too_many, (0, 0, 0), (50.0, 50.0, 50.0), (1, 1, 1), 5.8, 64, nb1, big, big)
    assert st == mx.MIX_EINVAL
    st = mx.neighbours_noalloc(x, (0, 0, 0), (50.0, 50.0, 50.0), (1, 1, 1), 5.8, 300, out, out, out)
    assert st == mx.MIX_EINVAL
    st = mx.neighbours_noalloc(x, (0, 0, 0), (1000.0, 1000.0, 1000.0), (0, 0, 0), 5.8, 64, out, out, out)
    assert st == mx.MIX_EINVAL                     # more cells than the scratch holds
    st = mx.neighbours_noalloc(x, (0, 0, 0), (1e12, 50.0, 50.0), (0, 0, 0), 5.8, 64, out, out, out)
    assert st == mx.MIX_EINVAL                     # a cell count beyond int, rejected before conversion
