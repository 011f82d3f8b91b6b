"""Temporal slabs (Sec. 5) on the GPU: the lattice cut into 1, 2 or 4 slab
contexts on one device, driven by the package's slab driver (the paper's
boundary protocol; the boundary links move by device copies), against the
whole lattice's context and the FP64 oracle.  The slabs run the same kernels
in the same launch configuration on the same links, so the swept field is the
whole lattice's bit for bit, in FP64 and FP32 storage, OR and SR, both gauges,
with the reunitarisation schedule (every 2 sweeps) and the SR streams following
the global sweep and site."""
import numpy as np
import pytest

import oracle as O
from paper_1305_3440_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS = (8, 6, 10, 14)  # 4 tiles of 128 sites per slice and parity, the last partial


@pytest.fixture(scope="module")
def lgt():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1305_3440_gb300 import build
    build.build()
    from paper_1305_3440_gb300 import lgt as mod
    return mod


def _slabs(lgt, p, U, n, stream, split=False):
    """n slab contexts on this device driven through a local ring; split: update the
    first slice and the interior in two launches (the order a ring across devices
    uses to overlap the return transfer)."""
    from paper_1305_3440_gb300.slab import GpuSlab, LocalRing, SlabDriver

    class SplitRing(LocalRing):
        overlap = True

    L = U.shape[0] // n
    engines = [GpuSlab(p, r * L, L, np.ascontiguousarray(U[r * L:(r + 1) * L]), stream) for r in range(n)]
    return SlabDriver(engines, SplitRing(n) if split else LocalRing(n))


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("n", [1, 2, 4])
@pytest.mark.parametrize("bulk,cfg", [("fp64", 1), ("fp32_12", 9), ("fp32_12", 15), ("fp32_12", 16), ("fp32_18", 8)])
@pytest.mark.parametrize("gauge,algo", [("landau", "or"), ("landau", "sr"), ("coulomb", "or")])
def test_gpu_slabs_reproduce_the_whole_lattice(lgt, split, n, bulk, cfg, gauge, algo):
    import torch
    g = lgt.LGT_LANDAU if gauge == "landau" else lgt.LGT_COULOMB
    a = lgt.LGT_OR if algo == "or" else lgt.LGT_SR
    U = synth.field(DIMS, 0.5, 44)
    stream = torch.cuda.Stream()
    p = lgt.lgt_params_default(dims=DIMS, bulk=getattr(lgt, "LGT_" + bulk.upper()), gauge=g, algo=a, omega=1.7,
                               p=0.8, seed=7, launch_config=cfg, reunit_every=2)
    ctx = lgt.lgt_create(p, U, stream=stream)
    try:
        lgt.lgt_sweep(ctx, 3)
        whole = lgt.lgt_get_working_links(ctx, DIMS)
        F_w, th_w, _, _ = lgt.lgt_estimate(ctx, DIMS[0])
    finally:
        lgt.lgt_destroy(ctx)
    drv = _slabs(lgt, p, U, n, stream, split)
    try:
        with torch.cuda.stream(stream):
            drv.sweep(3)
            got = np.concatenate([e.links() for e in drv.engines])
            F_s, th_s = drv.estimate()
            m = drv.measure()
    finally:
        for e in drv.engines:
            e.close()
    assert np.array_equal(got, whole)
    assert abs(F_s - F_w) < 1e-13 and abs(th_s - th_w) < 1e-13 * th_w
    r = O.measure(got, g)  # the gathered working field, measured by the oracle
    assert abs(m["F"] - r["F"]) < 1e-13 and abs(m["theta"] - r["theta"]) < 1e-12 * r["theta"]
    if bulk == "fp64":
        ref = U.copy()
        O.sweeps(ref, 3, gauge=g, algo=a, omega=1.7, p=0.8, seed=7)
        assert np.abs(got - ref).max() < 1e-12


def test_gpu_slab_driver_fixes_to_the_oracle_F(lgt):
    """The slab driver's fix (checks on the fused estimate, the exact measurement to
    certify) over 4 slabs in FP64: the oracle's converged F (1e-10) and theta < 1e-14
    on the gathered field."""
    import torch
    dims = (8, 8, 8, 8)
    U = synth.field(dims, 0.3, 1)
    stream = torch.cuda.Stream()
    p = lgt.lgt_params_default(dims=dims, omega=1.7)
    drv = _slabs(lgt, p, U, 4, stream)
    try:
        with torch.cuda.stream(stream):
            res = drv.fix(tol=1e-14, max_sweeps=2000)
            got = np.concatenate([e.links() for e in drv.engines])
    finally:
        for e in drv.engines:
            e.close()
    ref = U.copy()
    r = O.fix(ref, omega=1.7, tol=1e-14, max_sweeps=2000)
    assert res["converged"] and abs(res["F"] - r["F"]) < 1e-10
    m = O.measure(got)
    assert m["theta"] < 1e-14 and abs(m["F"] - res["F"]) < 1e-13


def test_slab_contexts_reject_the_one_lattice_calls(lgt):
    dims = (4, 4, 4, 4)
    U = synth.field(dims, 0.3, 2)
    p = lgt.lgt_params_default(dims=dims)
    ctx = lgt.lgt_slab_create(p, 8, 2, U)
    try:
        for call in (lambda: lgt.lgt_sweep(ctx, 1), lambda: lgt.lgt_measure(ctx), lambda: lgt.lgt_fix(ctx),
                     lambda: lgt.lgt_half_sweep(ctx, 0), lambda: lgt.lgt_slab_half_sweep(ctx, 0, 3, 2)):
            with pytest.raises(lgt.LgtError) as e:
                call()
            assert e.value.status == lgt.LGT_EINVAL
    finally:
        lgt.lgt_destroy(ctx)
    for nt, t0 in [(8, 1), (8, 6), (7, 0)]:
        with pytest.raises(lgt.LgtError):
            lgt.lgt_slab_create(p, nt, t0, U)
