"""The measurement entry point that allocates nothing (lgt_measure_noalloc).

Some callers of this library cannot allocate device memory -- an application
that hands out every byte of HBM through its own memory plan, or code that must
measure where no allocation may happen -- so they cannot create a context.  This
test checks that the no-allocation variant, called through the C ABI on links
in device memory, gives what the FP64 oracle's measurement gives and what the
context-based lgt_measure / lgt_measure_slices give, on two calls in a row (the
shared scratch keeps the previous call's contents).  The file is named to be
collected last.
"""
import numpy as np
import pytest

import oracle as O
from paper_1305_3440_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lgt():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1305_3440_gb300 import build
    build.build()
    from paper_1305_3440_gb300 import lgt as mod
    return mod


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (4, 6, 10, 14), (2, 2, 2, 2), (16, 8, 4, 6)])
def test_no_alloc_measure_matches_context_measure(lgt, dims):
    import torch
    U = synth.field(dims, 0.5, 21)
    dev = torch.from_numpy(U).cuda()
    nt = dims[0]
    p = lgt.lgt_params_default(dims=dims)
    ctx = lgt.lgt_create(p, dev)
    try:
        F, th, pl = lgt.lgt_measure(ctx)
        Ft, tht = lgt.lgt_measure_slices(ctx, nt)
    finally:
        lgt.lgt_destroy(ctx)
    ref = O.measure(U)
    ref_c = O.measure(U, O.COULOMB)
    stream = torch.cuda.Stream()
    out = torch.empty(8 + 2 * nt, dtype=torch.float64, device="cuda")
    for call in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        lgt.lgt_measure_noalloc(dims, dev, out, stream)
        stream.synchronize()
        o = out.cpu().numpy()
        assert abs(o[0] - F) < 1e-13 and abs(o[2] - pl) < 1e-13
        assert abs(o[1] - th) < 1e-13 * th
        assert np.allclose(o[8:8 + nt], Ft, rtol=0, atol=1e-13)
        assert np.allclose(o[8 + nt:], tht, rtol=1e-13, atol=0)
        assert abs(o[4] - tht.max()) < 1e-13 * tht.max() and abs(o[3] - Ft.mean()) < 1e-13
        assert abs(o[5] - tht.mean()) < 1e-13 * tht.mean() and o[6] == 0.0 and o[7] == 0.0
        # the oracle on the same field: Landau F, theta, plaquette; Coulomb F_t, theta_t
        assert abs(o[0] - ref["F"]) < 1e-13 and abs(o[2] - ref["plaq"]) < 1e-13
        assert abs(o[1] - ref["theta"]) < 1e-13 * ref["theta"]
        assert np.allclose(o[8:8 + nt], ref_c["F_t"], rtol=0, atol=1e-13)
        assert np.allclose(o[8 + nt:], ref_c["theta_t"], rtol=1e-13, atol=0)


def test_no_alloc_measure_rejects_sizes_beyond_its_scratch(lgt):
    import torch
    dev = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lgt.LgtError) as e:
        lgt.lgt_measure_noalloc((1026, 2, 2, 2), dev, out)
    assert e.value.status == lgt.LGT_EINVAL and "1024" in lgt.lgt_last_error()
    with pytest.raises(lgt.LgtError):
        lgt.lgt_measure_noalloc((4, 4, 4, 3), dev, out)
