"""The bf16 tensor-core readout (precision MIX_BF16, hi/lo split MIX_BF16_SPLIT)
against the FP64 oracle, through the C ABI.

* the MMA building block (shared-memory operand layout, tcgen05.mma with
  M = 128 and M = 64, TMEM read-back) equals a float64 product of the same
  bf16 matrices to the rounding of a float accumulation, each row of D in the
  TMEM lane the readout expects;
* forces and site energies of every parity case: the hi/lo split within
  1e-4 eV/A (float-like: about 16 significant bits per product) and 1e-4
  relative in site energy; plain bf16 (8 significant bits for Z and W)
  within 5 % of the RMS force and 2e-2 relative in site energy, and never
  closer to the oracle than the split.  Plain bf16 does not meet the 1e-3
  eV/A gate on most of these potentials (measured 2.4e-4 to 4e-2 eV/A): the
  benchmark reports that as failing and takes the split as the fallback;
* sets and weights bit-exact (they do not depend on the potential
  arithmetic), the tensor-core kernel really running (CTAs of 4 warps,
  results different from the CUDA-core float path);
* a short trajectory re-evaluated by the oracle on the GPU's own bits;
* the 256,000-atom screw cylinder on 64 sampled atoms.
"""
import numpy as np
import pytest

import oracle
from paper_2502_19081_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GATE = 1e-3


@pytest.fixture(scope="module")
def mx():
    from paper_2502_19081_gb300 import build, mix
    build.build()
    return mix


def _max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) if np.size(a) else 0.0


def _lanes(m):
    """TMEM lane of each row of an M x N accumulator: row i in lane i for
    M = 128; for M = 64, rows 16 w .. 16 w + 15 in the first 16 lanes of
    warp w's 32-lane quarter."""
    r = np.arange(m)
    return r if m == 128 else 32 * (r // 16) + r % 16


@pytest.mark.parametrize("m,n,k", [(128, 16, 16), (128, 16, 112), (128, 16, 144), (128, 32, 160), (128, 144, 16),
                                   (128, 256, 64), (128, 192, 128), (64, 16, 16), (64, 16, 144), (64, 48, 80)])
def test_mma_building_block(mx, m, n, k):
    torch = pytest.importorskip("torch")
    g = torch.Generator().manual_seed(m * 100000 + n * 1000 + k)
    a = torch.randn(m, k, generator=g).to(torch.bfloat16)
    b = torch.randn(n, k, generator=g).to(torch.bfloat16)
    ad, bd = a.cuda(), b.cuda()
    d = torch.full((128, n), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mx.tc_selftest(ad, bd, d, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    a64, b64 = a.double().numpy(), b.double().numpy()
    ref = a64 @ b64.T
    bound = (np.abs(a64) @ np.abs(b64).T) * (k * 2.0 ** -23) + 1e-30
    dl = d.cpu().double().numpy()
    got = dl[_lanes(m)]
    err = np.abs(got - ref)
    if not np.all(err <= bound):
        # where each row of the product does lie (for the assertion message)
        where = {i: [int(l) for l in range(128) if np.all(np.abs(dl[l] - ref[i]) <= bound[i])] for i in range(m)}
        pytest.fail(f"rows of D not in the expected lanes: {where}")


def test_mma_building_block_rejects_bad_shapes(mx):
    torch = pytest.importorskip("torch")
    a = torch.zeros(128, 24, dtype=torch.bfloat16, device="cuda")
    b = torch.zeros(16, 24, dtype=torch.bfloat16, device="cuda")
    d = torch.zeros(128, 16, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(mx.MixError) as e:
        mx.tc_selftest(a, b, d, st)
    assert e.value.code == mx.MIX_EINVAL


def _cases():
    return {
        "fe_box_685": lambda: I.small_fe_box(11, r_core=4.0, ramp=3.0),
        "fe_box_l4": lambda: I.small_fe_box(12, n_rad=5, l_max=4, r_core=3.0, ramp=2.5),
        "cluster_60": lambda: I.cluster_workload(13, n=60, radius=8.0, n_rad=6, l_max=3, r_core=3.5, ramp=2.0),
        "screw_3000": lambda: I.fe_screw(n_atoms=3000, nrep_z=4),
        "fe_box_n11": lambda: I.small_fe_box(15, n_rad=11, l_max=3, r_core=3.0, ramp=2.0),
        "fe_box_n12_l5": lambda: I.small_fe_box(21, n_rad=12, l_max=5, r_core=4.0, ramp=3.0),
        "fe_box_n10_l4": lambda: I.small_fe_box(22, n_rad=10, l_max=4, r_core=4.0, ramp=3.0),
        "fe_box_n14_l6": lambda: I.small_fe_box(24, n_rad=14, l_max=6, r_core=3.0, ramp=2.0),
        "fe_box_n4_l2": lambda: I.small_fe_box(25, n_rad=4, l_max=2, r_core=3.0, ramp=2.0),
    }


@pytest.mark.parametrize("name", list(_cases()))
def test_bf16_forces_against_oracle(mx, name):
    wl = _cases()[name]()
    om = oracle.Model(wl)
    res = {}
    for prec in (mx.MIX_FP32, mx.MIX_BF16, mx.MIX_BF16_SPLIT):
        ctx = mx.open_context(wl, precision=prec)
        x, _, F, _ = ctx.get_state()
        fl, _, _ = ctx.sets()
        ee, ec = ctx.site_energies()
        res[prec] = (x, F, fl, ee, ec, ctx.info())
        ctx.close()
    x = res[mx.MIX_FP32][0]
    FB, Ee, Ec = om.forces(x, oracle.MODE_METHOD)
    fl_o = om.sets(x)
    err = {}
    rms = float(np.sqrt(np.mean(FB[:, :3] ** 2)))
    # plain bf16 rounds Z and W to 8 significant bits, about 4e-3 relative per
    # product before the nu = 3 sums cancel: a loose sanity bound
    erel = {mx.MIX_FP32: 1e-5, mx.MIX_BF16: 2e-2, mx.MIX_BF16_SPLIT: 1e-4}
    for prec, (xp, F, fl, ee, ec, info) in res.items():
        assert np.array_equal(xp, x)
        assert np.array_equal(fl, fl_o)
        err[prec] = _max_abs(F[:, :3], FB[:, :3])
        ev = (fl & 4) > 0
        rel = np.abs(ee[ev] - Ee[ev]) / (np.abs(Ee[ev]) + 1.0)
        assert float(rel.max()) <= erel[prec], (prec, float(rel.max()))
        if prec != mx.MIX_FP32:
            assert info["exp_tensor_cores"] == 1 and info["exp_threads"] == 128   # the tensor-core kernel ran
    assert err[mx.MIX_FP32] <= GATE, err
    assert err[mx.MIX_BF16_SPLIT] <= 1e-4, err
    assert err[mx.MIX_BF16] <= 0.05 * rms, err
    # the tensor-core path is not the CUDA-core float path, and the split is the
    # more accurate of the two bf16 variants
    assert not np.array_equal(res[mx.MIX_BF16][1], res[mx.MIX_FP32][1])
    assert err[mx.MIX_BF16_SPLIT] < err[mx.MIX_BF16]


def test_bf16_deterministic_and_trajectory(mx):
    wl = I.small_fe_box(23, r_core=4.0, ramp=3.0, sigma=0.15)
    a = mx.open_context(wl, precision=mx.MIX_BF16)
    b = mx.open_context(wl, precision=mx.MIX_BF16)
    a.step(1.0, 10)
    b.step(1.0, 10)
    xa, va, fa, _ = a.get_state()
    xb, vb, fb, _ = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(fa, fb)
    om = oracle.Model(wl)
    fl, _, _ = a.sets()
    assert np.array_equal(fl, om.sets(xa))
    FB, _, _ = om.forces(xa, oracle.MODE_METHOD)
    assert _max_abs(fa[:, :3], FB[:, :3]) <= 0.05 * float(np.sqrt(np.mean(FB[:, :3] ** 2)))
    c = mx.open_context(wl, precision=mx.MIX_BF16_SPLIT)
    c.step(1.0, 10)
    xc, _, fc, _ = c.get_state()
    FC, _, _ = om.forces(xc, oracle.MODE_METHOD)
    assert _max_abs(fc[:, :3], FC[:, :3]) <= 1e-4


def test_bf16_in_a_batch_equals_alone(mx):
    """Batches holding tensor-core contexts step them as child graphs (the
    fused batch kernels are CUDA-core only): each member ends where it ends
    alone, bit for bit."""
    wls = [I.small_fe_box(24 + k, r_core=3.0, ramp=2.0) for k in range(3)]
    alone = []
    for wl in wls:
        c = mx.open_context(wl, precision=mx.MIX_BF16)
        c.step(1.0, 6)
        alone.append(c.get_state())
        c.close()
    ctxs = [mx.open_context(wl, precision=mx.MIX_BF16) for wl in wls]
    b = mx.Batch(ctxs)
    assert not b.info()["fused"]
    b.step(1.0, 6)
    b.sync()
    for c, (x, v, f, _) in zip(ctxs, alone):
        xc, vc, fc, _ = c.get_state()
        assert np.array_equal(xc, x) and np.array_equal(vc, v) and np.array_equal(fc, f)
    b.close()


def test_screw_cylinder_full_size_bf16_sampled(mx):
    """C3 (256,000 atoms, n = 12, lmax = 5) in bf16 and bf16 hi/lo: 64 sampled
    atoms (core, ramp, expensive buffer, cheap only) against the oracle (RMS
    force about 1 eV/A: plain bf16 within 5 %, the split within 1e-4 eV/A)."""
    wl = I.fe_screw()
    om = oracle.Model(wl)
    for prec, tol in ((mx.MIX_BF16, 0.05), (mx.MIX_BF16_SPLIT, 1e-4)):
        ctx = mx.open_context(wl, precision=prec)
        x, _, F, _ = ctx.get_state()
        fl, _, _ = ctx.sets()
        lam, _ = ctx.lam()
        rng = np.random.default_rng(1)
        pick = []
        for sel in (lam == 1.0, (lam > 0) & (lam < 1), (lam == 0) & ((fl & 4) > 0), (fl & 4) == 0):
            idx = np.nonzero(sel)[0]
            pick += list(rng.choice(idx, 16, replace=False))
        Fs = om.forces_sampled(x, np.array(pick))
        assert _max_abs(F[pick, :3], Fs[:, :3]) <= tol
        assert ctx.info()["exp_tensor_cores"] == 1
        ctx.close()
