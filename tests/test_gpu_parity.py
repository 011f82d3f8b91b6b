"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: one sweep from the same input agrees to 1e-12 max-abs per link
entry in FP64 and 5e-6 on FP32 link storage; converged runs agree in F to
1e-10 with theta below the requested 1e-14 (converged links are not unique:
a global gauge rotation or another Gribov copy changes them, so links are only
compared after a fixed number of sweeps).
"""
import time

import numpy as np
import pytest

import oracle as O
from paper_1305_3440_gb300 import synth
from lattice_np import check_fp32_bound, fp32_half_sweep_bound, fp32_sweep_bound, plaquettes, unitarity_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lgt():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1305_3440_gb300 import build
    build.build()
    from paper_1305_3440_gb300 import lgt as mod
    return mod


GAUGES = {"landau": O.LANDAU, "coulomb": O.COULOMB}
ALGOS = {"or": O.OR, "sr": O.SR}
# several tiles per timeslice and a ragged tail (block 128: vs_half = 420 -> 3 full + 36)
DIMS_RAGGED = (4, 6, 10, 14)


def gpu_run(lgt, U, n, working=False, **kw):
    dims = U.shape[:4]
    p = lgt.lgt_params_default(dims=dims, **kw)
    ctx = lgt.lgt_create(p, U)
    try:
        if n:
            lgt.lgt_sweep(ctx, n)
        out = lgt.lgt_get_working_links(ctx, dims) if working else lgt.lgt_get_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    return out


def test_layout_roundtrip_is_exact(lgt):
    U = synth.field(DIMS_RAGGED, 0.5, 3)
    assert np.array_equal(gpu_run(lgt, U, 0), U)
    for bulk, tol in [(lgt.LGT_FP32_18, 1.5e-7), (lgt.LGT_FP32_12, 1e-6)]:
        assert np.array_equal(gpu_run(lgt, U, 0, bulk=bulk), U)  # G = 1 on the FP64 input
        assert np.abs(gpu_run(lgt, U, 0, working=True, bulk=bulk) - U).max() < tol


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), DIMS_RAGGED, (2, 2, 2, 2), (6, 2, 4, 2)])
def test_measurement_matches_oracle(lgt, dims):
    U = synth.field(dims, 0.6, 4)
    p = lgt.lgt_params_default(dims=dims)
    ctx = lgt.lgt_create(p, U)
    try:
        F, th, pl = lgt.lgt_measure(ctx)
        Ft, tht = lgt.lgt_measure_slices(ctx, dims[0])
    finally:
        lgt.lgt_destroy(ctx)
    m = O.measure(U)
    mc = O.measure(U, O.COULOMB)
    assert abs(F - m["F"]) < 1e-13 and abs(pl - m["plaq"]) < 1e-13
    assert abs(th - m["theta"]) < 1e-13 * m["theta"]
    assert np.allclose(Ft, mc["F_t"], rtol=0, atol=1e-13)
    assert np.allclose(tht, mc["theta_t"], rtol=1e-13, atol=0)


@pytest.mark.parametrize("gauge", list(GAUGES))
@pytest.mark.parametrize("algo", list(ALGOS))
@pytest.mark.parametrize("dims,block", [(DIMS_RAGGED, 128), ((8, 8, 8, 8), 64), ((2, 4, 2, 6), 256)])
def test_one_sweep_fp64_matches_oracle(lgt, gauge, algo, dims, block):
    U = synth.field(dims, 0.5, 5)
    kw = dict(gauge=GAUGES[gauge], algo=ALGOS[algo], omega=1.7, p=0.8, seed=77, sweep_offset=3)
    got = gpu_run(lgt, U, 2, block_size=block, **kw)
    ref = U.copy()
    O.sweeps(ref, 2, gauge=kw["gauge"], algo=kw["algo"], omega=1.7, p=0.8, seed=77, sweep0=3)
    assert np.abs(got - ref).max() < 1e-12


def gpu_half(lgt, U, parity, working=True, **kw):
    dims = U.shape[:4]
    p = lgt.lgt_params_default(dims=dims, **kw)
    ctx = lgt.lgt_create(p, U)
    try:
        lgt.lgt_half_sweep(ctx, parity)
        out = lgt.lgt_get_working_links(ctx, dims) if working else lgt.lgt_get_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    return out


@pytest.mark.parametrize("bulk", ["fp32_18", "fp32_12"])
@pytest.mark.parametrize("gauge", list(GAUGES))
@pytest.mark.parametrize("algo", list(ALGOS))
@pytest.mark.parametrize("parity", [0, 1])
def test_half_sweep_fp32_matches_oracle(lgt, bulk, gauge, algo, parity):
    """The kernel's unit of work, one parity, from the same rough random-gauge field:
    within 5e-6 per link entry on FP32 link storage."""
    U = synth.field(DIMS_RAGGED, 0.5, 6)
    b = lgt.LGT_FP32_18 if bulk == "fp32_18" else lgt.LGT_FP32_12
    kw = dict(gauge=GAUGES[gauge], algo=ALGOS[algo], omega=1.7, p=0.8, seed=78)
    got = gpu_half(lgt, U, parity, bulk=b, reunit_every=0, **kw)
    ref = U.copy()
    O.half_sweep(ref, parity, gauge=kw["gauge"], algo=kw["algo"], omega=1.7, p=0.8, seed=78)
    assert np.abs(got - ref).max() < 5e-6
    full = gpu_half(lgt, U, parity, working=False, bulk=b, reunit_every=0, **kw)
    assert np.abs(full - ref).max() < 5e-6  # G U G^dagger on the FP64 input


def sweep_kappas(U, **kw):
    """The oracle's conditioning of every site update of one sweep from U: the even
    sites on U, the odd sites on the field the oracle's even half leaves."""
    half = U.copy()
    O.half_sweep(half, 0, **kw)
    ck = {k: v for k, v in kw.items() if k in ("gauge", "algo", "omega", "p", "seed")}
    return O.site_conditioning(U, 0, **ck), O.site_conditioning(half, 1, **ck)


@pytest.mark.parametrize("bulk", ["fp32_18", "fp32_12"])
@pytest.mark.parametrize("algo", list(ALGOS))
def test_one_sweep_fp32_matches_oracle(lgt, bulk, algo):
    """A full sweep (both parities) on FP32 link storage.  On a field already
    relaxed by 30 sweeps (the bulk phase's regime) every entry is within 5e-6.  On
    the raw random-gauge field the odd half reads links the even half wrote, so an
    FP32 deviation of the even half is amplified by the conditioning of the odd
    site's update: every entry is within max(5e-6, B) of the oracle, B the
    first-order bound of its link from the oracle's conditioning kappa = 1/|q|_min
    of the two site updates that wrote it (lattice_np.fp32_sweep_bound)."""
    b = lgt.LGT_FP32_18 if bulk == "fp32_18" else lgt.LGT_FP32_12
    kw = dict(algo=ALGOS[algo], omega=1.7, p=0.8, seed=79)
    raw = synth.field(DIMS_RAGGED, 0.5, 6)
    relaxed = raw.copy()
    O.sweeps(relaxed, 30, omega=1.7)
    for U, derived in [(relaxed, False), (raw, True)]:
        got = gpu_run(lgt, U, 1, working=True, bulk=b, reunit_every=0, **kw)
        ref = U.copy()
        O.sweeps(ref, 1, **kw)
        err = np.abs(got - ref)
        if not derived:
            assert err.max() < 5e-6, err.max()
            continue
        ratio, n_above, n_links = check_fp32_bound(err, fp32_sweep_bound(*sweep_kappas(U, **kw)))
        assert ratio <= 1.0, (ratio, err.max(), n_above, n_links)


@pytest.mark.parametrize("gauge", ["landau", "coulomb", "mag"])
@pytest.mark.parametrize("bulk", ["fp64", "fp32_12"])
def test_fused_estimate_matches_oracle(lgt, gauge, bulk):
    """The sweeps' own F/theta estimate (what lgt_fix's checks read) after one full
    sweep, against the oracle on the fields each half started from: F (and F_t)
    is the F of the starting field (every link once in the even sites' K), theta
    sums tr[Delta Delta^dagger] of the even sites on the starting field and of the
    odd sites after the oracle's even half.  FP64: F within 1e-13 (it is ~0 on a
    random-gauge field), theta within 1e-13 relative.  FP32 link storage: an entry
    of a site's K carries at most 64u of rounding (8 stored entries and 7 sums of
    terms up to 8), its Re tr K at most 192u, the 8-site FP32 group sum at most
    168u per site more; over the 3 N_d sites' worth of links per site F is off by
    at most 16u (a slice's F_t, N_d = 3: 32u).  By Cauchy-Schwarz the theta sum
    is off by at most 2 x 64u x 8 / rms|Delta| relative (rms over the sites, per
    slice for theta_t; the rough field's Delta is O(1))."""
    g = {"landau": O.LANDAU, "coulomb": O.COULOMB, "mag": O.MAG}[gauge]
    dims = DIMS_RAGGED
    U = synth.field(dims, 0.5, 81)
    b = lgt.LGT_FP64 if bulk == "fp64" else lgt.LGT_FP32_12
    p = lgt.lgt_params_default(dims=dims, gauge=g, bulk=b, omega=1.7, reunit_every=0)
    ctx = lgt.lgt_create(p, U)
    try:
        lgt.lgt_sweep(ctx, 1)
        F, theta, F_t, th_t = lgt.lgt_estimate(ctx, dims[0])
    finally:
        lgt.lgt_destroy(ctx)
    half = U.copy()
    O.half_sweep(half, 0, gauge=g, omega=1.7)
    viol = O.parity_violation(U, 0, g) + O.parity_violation(half, 1, g)
    vs = dims[1] * dims[2] * dims[3]
    m = O.measure(U, g)
    th_t_ref = viol / (3 * vs)
    theta_ref = th_t_ref.max() if g == O.COULOMB else viol.sum() / (3 * vs * dims[0])
    Ft_ref = O.measure(U, O.COULOMB)["F_t"] if g == O.COULOMB else None
    theta_sum_ref = viol.sum() / (3 * vs * dims[0])  # the Landau-normalised theta of the sweep
    if bulk == "fp64":
        tol_F, tol_Ft = 1e-13, 1e-13
        tol_th, tol_tht = 1e-13, np.full(dims[0], 1e-13)
    else:
        u = 2.0 ** -24
        tol_F, tol_Ft = 16 * u, 32 * u
        tol_th = 2 * 64 * u * 8 / np.sqrt(3 * theta_sum_ref)
        tol_tht = 2 * 64 * u * 8 / np.sqrt(3 * th_t_ref)
    assert abs(F - m["F"]) <= tol_F, (F, m["F"])
    assert abs(theta - theta_ref) <= tol_th * theta_ref, (theta, theta_ref)
    assert np.all(np.abs(th_t - th_t_ref) <= tol_tht * th_t_ref), (th_t, th_t_ref)
    if Ft_ref is not None:
        assert np.all(np.abs(F_t - Ft_ref) <= tol_Ft), (F_t, Ft_ref)


def test_half_sweep_counts_and_fp64_parity(lgt):
    U = synth.field(DIMS_RAGGED, 0.5, 8)
    p = lgt.lgt_params_default(dims=DIMS_RAGGED, algo=lgt.LGT_SR, p=0.8, seed=3)
    ctx = lgt.lgt_create(p, U)
    try:
        lgt.lgt_half_sweep(ctx, 0)
        assert lgt.lgt_get_progress(ctx) == (0, 0, 1)
        lgt.lgt_half_sweep(ctx, 1)
        lgt.lgt_half_sweep(ctx, 0)
        assert lgt.lgt_get_progress(ctx) == (0, 1, 1)
        got = lgt.lgt_get_links(ctx, DIMS_RAGGED)
    finally:
        lgt.lgt_destroy(ctx)
    ref = U.copy()
    O.sweeps(ref, 1, algo=O.SR, p=0.8, seed=3)
    O.half_sweep(ref, 0, algo=O.SR, p=0.8, seed=3, sweep=1)
    assert np.abs(got - ref).max() < 1e-12


def test_coulomb_temporal_option(lgt):
    U = synth.field((4, 4, 6, 4), 0.5, 7)
    got = gpu_run(lgt, U, 2, gauge=lgt.LGT_COULOMB, transform_temporal=0, omega=1.5)
    ref = U.copy()
    O.sweeps(ref, 2, gauge=O.COULOMB, omega=1.5, transform_temporal=0)
    assert np.abs(got - ref).max() < 1e-12
    assert np.array_equal(got[..., 0, :, :], U[..., 0, :, :])


@pytest.mark.parametrize("bulk", ["fp64", "fp32_18", "fp32_12"])
def test_fix_8x4_matches_oracle(lgt, bulk):
    """SU(3) Landau 8^4, eps = 0.3, seed 1, OR omega = 1.7 to theta < 1e-14."""
    b = {"fp64": lgt.LGT_FP64, "fp32_18": lgt.LGT_FP32_18, "fp32_12": lgt.LGT_FP32_12}[bulk]
    dims = (8, 8, 8, 8)
    U = synth.field(dims, 0.3, 1)
    p = lgt.lgt_params_default(dims=dims, omega=1.7, bulk=b, max_sweeps=1000)
    ctx = lgt.lgt_create(p, U)
    try:
        st, res = lgt.lgt_fix(ctx)
        V = lgt.lgt_get_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    ref = U.copy()
    r = O.fix(ref, omega=1.7, tol=1e-14, max_sweeps=1000)
    assert st == lgt.LGT_OK and res.status == lgt.LGT_OK
    assert res.theta < 1e-14 and abs(res.F - r["F"]) < 1e-10
    m = O.measure(V)  # the oracle certifies the returned field
    assert m["theta"] < 1e-14 and abs(m["F"] - res.F) < 1e-13
    assert np.abs(plaquettes(V) - plaquettes(U)).max() < 1e-12
    e, d = unitarity_error(V)
    assert e < 1e-12 and d < 1e-12
    if b == lgt.LGT_FP64:
        assert res.sweeps_bulk == 0 and res.sweeps_fp64 > 0
    else:
        assert res.sweeps_bulk > 0


@pytest.mark.parametrize("bulk", ["fp64", "fp32_12"])
def test_fix_coulomb_matches_oracle(lgt, bulk):
    b = lgt.LGT_FP64 if bulk == "fp64" else lgt.LGT_FP32_12
    dims = (6, 8, 8, 8)
    U = synth.field(dims, 0.5, 3)
    p = lgt.lgt_params_default(dims=dims, gauge=lgt.LGT_COULOMB, omega=1.7, bulk=b, max_sweeps=2000)
    ctx = lgt.lgt_create(p, U)
    try:
        st, res = lgt.lgt_fix(ctx)
        V = lgt.lgt_get_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    ref = U.copy()
    r = O.fix(ref, gauge=O.COULOMB, omega=1.7, tol=1e-14, max_sweeps=2000)
    assert st == lgt.LGT_OK and r["converged"]
    mg = O.measure(V, O.COULOMB)
    mo = O.measure(ref, O.COULOMB)
    assert np.all(mg["theta_t"] < 1e-14)
    assert np.abs(mg["F_t"] - mo["F_t"]).max() < 1e-10
    assert np.abs(plaquettes(V) - plaquettes(U)).max() < 1e-12


def test_stochastic_relaxation_fix(lgt):
    dims = (8, 8, 8, 8)
    U = synth.field(dims, 0.3, 9)
    p = lgt.lgt_params_default(dims=dims, algo=lgt.LGT_SR, p=0.8, seed=5, bulk=lgt.LGT_FP32_18,
                               max_sweeps=3000)
    ctx = lgt.lgt_create(p, U)
    try:
        st, res = lgt.lgt_fix(ctx)
    finally:
        lgt.lgt_destroy(ctx)
    ref = U.copy()
    r = O.fix(ref, algo=O.SR, p=0.8, seed=5, tol=1e-14, max_sweeps=3000)
    assert st == lgt.LGT_OK and r["converged"] and abs(res.F - r["F"]) < 1e-10


def test_results_are_deterministic_and_load_restarts(lgt):
    dims = (4, 8, 8, 8)
    U = synth.field(dims, 0.5, 10)
    p = lgt.lgt_params_default(dims=dims, bulk=lgt.LGT_FP32_12, max_sweeps=3000)
    ctx = lgt.lgt_create(p, U)
    try:
        st1, r1 = lgt.lgt_fix(ctx)
        V1 = lgt.lgt_get_links(ctx, dims)
        lgt.lgt_load(ctx, U)
        assert lgt.lgt_get_progress(ctx) == (0, 0, 0)
        st2, r2 = lgt.lgt_fix(ctx)
        V2 = lgt.lgt_get_links(ctx, dims)
        stats = lgt.lgt_get_stats(ctx)
    finally:
        lgt.lgt_destroy(ctx)
    assert st1 == st2 == lgt.LGT_OK
    assert r1.F == r2.F and r1.theta == r2.theta and r1.sweeps_bulk == r2.sweeps_bulk
    assert np.array_equal(V1, V2)
    assert stats.sweep_launches[0] == 2 * r2.sweeps_bulk and stats.sweep_ms[0] > 0
    assert stats.site_updates[0] == r2.sweeps_bulk * np.prod(dims)


def test_device_resident_links(lgt):
    import torch
    dims = (4, 4, 6, 8)
    U = synth.field(dims, 0.5, 11)
    dev = torch.from_numpy(U).cuda()
    out = torch.empty_like(dev)
    p = lgt.lgt_params_default(dims=dims, omega=1.7)
    s = torch.cuda.Stream()
    ctx = lgt.lgt_create(p, dev, stream=s)
    try:
        lgt.lgt_sweep(ctx, 3)
        lgt.lgt_get_links(ctx, out=out)
    finally:
        lgt.lgt_destroy(ctx)
    ref = U.copy()
    O.sweeps(ref, 3, omega=1.7)
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-12


def test_rejects_non_su3_and_non_finite(lgt):
    dims = (4, 4, 4, 4)
    U = synth.field(dims, 0.5, 12)
    p = lgt.lgt_params_default(dims=dims)
    bad = U.copy()
    bad[1, 2, 3, 0, 2, 1, 1] *= 1.001
    with pytest.raises(lgt.LgtError) as e:
        lgt.lgt_create(p, bad)
    assert e.value.status == lgt.LGT_EINVAL and "SU(3)" in lgt.lgt_last_error()
    bad = U.copy()
    bad[0, 0, 0, 1, 0, 0, 0] = np.nan
    with pytest.raises(lgt.LgtError):
        lgt.lgt_create(p, bad)


def test_not_converged_is_reported(lgt):
    dims = (4, 4, 4, 4)
    U = synth.field(dims, 0.5, 13)
    p = lgt.lgt_params_default(dims=dims, max_sweeps=4, check_every=2)
    ctx = lgt.lgt_create(p, U)
    try:
        st, res = lgt.lgt_fix(ctx)
        # the state is kept: continuing converges
        p2 = lgt.lgt_get_progress(ctx)
    finally:
        lgt.lgt_destroy(ctx)
    assert st == lgt.LGT_ENOTCONV and res.status == lgt.LGT_ENOTCONV and res.sweeps_fp64 == 4
    assert p2[1] == 4


# ----------------------------------------------- FP32-pair polishing sweeps
@pytest.fixture(scope="module")
def near_fixed_8():
    """8^4 fields relaxed by the oracle to theta ~ 1e-10 and ~ 1e-12 (the polish
    regime), per gauge."""
    out = {}
    for gauge in (O.LANDAU, O.COULOMB):
        for theta0 in (1e-10, 1e-12):
            U = synth.field((8, 8, 8, 8), 0.3, 1)
            r = O.fix(U, gauge=gauge, omega=1.7, tol=theta0, max_sweeps=2000, check_every=1)
            assert r["converged"]
            out[(gauge, theta0)] = U
    return out


POLISH = {"pair": (0, 2), "anchor": (2, 3)}  # polish kind -> (lgt_polish, phase after promotion)


def promoted_ctx(lgt, U, polish="pair", **kw):
    kw.setdefault("omega_polish", 0.0)  # polish at the same omega as the oracle below
    pk, phase = POLISH[polish]
    p = lgt.lgt_params_default(dims=U.shape[:4], bulk=lgt.LGT_FP32_12, polish=pk, **kw)
    ctx = lgt.lgt_create(p, U)
    lgt.lgt_promote(ctx)  # G = 1: the polish starts from the input (pairs: to ~2^-48)
    assert lgt.lgt_get_progress(ctx)[2] == phase
    return ctx


def test_pair_storage_roundtrip(lgt):
    U = synth.field(DIMS_RAGGED, 0.5, 16)
    ctx = promoted_ctx(lgt, U)
    try:
        V = lgt.lgt_get_links(ctx, DIMS_RAGGED)
        F, th, pl = lgt.lgt_measure(ctx)
    finally:
        lgt.lgt_destroy(ctx)
    assert np.abs(V - U).max() < 2e-15
    m = O.measure(U)
    assert abs(F - m["F"]) < 1e-13 and abs(th - m["theta"]) < 1e-12 * m["theta"]


@pytest.mark.parametrize("gauge", list(GAUGES))
@pytest.mark.parametrize("algo", list(ALGOS))
def test_anchor_polish_launch_configurations_agree(lgt, near_fixed_8, gauge, algo):
    """The anchored polish in each of its launch configurations (0-3: block sizes
    and register budgets; 11: 80 registers, 24 warps per SM): two polish sweeps
    are the oracle's sweeps to the polish tolerance (1e-12 at theta ~ 1e-12)."""
    U = near_fixed_8[(GAUGES[gauge], 1e-12)]
    kw = dict(gauge=GAUGES[gauge], algo=ALGOS[algo], omega=1.7, p=0.8, seed=81)
    ref = U.copy()
    O.sweeps(ref, 2, gauge=kw["gauge"], algo=kw["algo"], omega=1.7, p=0.8, seed=81)
    out = {}
    for k in (0, 1, 2, 3, 11):
        ctx = promoted_ctx(lgt, U, "anchor", launch_config=k + 1, **kw)
        try:
            assert lgt.lgt_get_stats(ctx).launch_config[1] == k
            lgt.lgt_sweep(ctx, 2)
            out[k] = lgt.lgt_get_links(ctx, U.shape[:4])
        finally:
            lgt.lgt_destroy(ctx)
        assert np.abs(out[k] - ref).max() < 1e-12, k


@pytest.mark.parametrize("polish", list(POLISH))
@pytest.mark.parametrize("gauge", list(GAUGES))
@pytest.mark.parametrize("algo", list(ALGOS))
@pytest.mark.parametrize("theta0,tol", [(1e-10, 2e-11), (1e-12, 1e-12)])
def test_pair_polish_sweep_matches_oracle(lgt, near_fixed_8, polish, gauge, algo, theta0, tol):
    """Two polish sweeps against the FP64 oracle.  The rotation angles are FP32, so a
    sweep deviates from the FP64 trajectory by ~|g - 1| 2^-24 (the applied rotations
    stay exact gauge transformations): within 2e-11 at theta ~ 1e-10 (|g - 1| ~ 1e-5,
    SR doubling the angle) and within 1e-12 per link entry at theta ~ 1e-12."""
    U = near_fixed_8[(GAUGES[gauge], theta0)]
    kw = dict(gauge=GAUGES[gauge], algo=ALGOS[algo], omega=1.7, p=0.8, seed=80)
    ctx = promoted_ctx(lgt, U, polish, **kw)
    try:
        lgt.lgt_sweep(ctx, 2)
        got = lgt.lgt_get_links(ctx, U.shape[:4])
    finally:
        lgt.lgt_destroy(ctx)
    ref = U.copy()
    O.sweeps(ref, 2, gauge=kw["gauge"], algo=kw["algo"], omega=1.7, p=0.8, seed=80)
    assert np.abs(got - ref).max() < tol


@pytest.mark.parametrize("polish", list(POLISH))
@pytest.mark.parametrize("gauge", list(GAUGES))
def test_pair_polish_is_an_exact_gauge_transformation(lgt, polish, gauge):
    """Even far from convergence (FP32-accurate angles) every pair update is a gauge
    transformation up to the ~2^-48 rounding of pair storage (~1e-14 per update, a
    random walk): after 20 sweeps plaquettes and unitarity hold to 3e-13 (FP32
    storage would give ~1e-7)."""
    U = synth.field(DIMS_RAGGED, 0.5, 14)
    ctx = promoted_ctx(lgt, U, polish, gauge=GAUGES[gauge], omega=1.7)
    try:
        lgt.lgt_half_sweep(ctx, 0)
        half = lgt.lgt_get_links(ctx, DIMS_RAGGED)
        lgt.lgt_half_sweep(ctx, 1)
        lgt.lgt_sweep(ctx, 19)
        V = lgt.lgt_get_links(ctx, DIMS_RAGGED)
    finally:
        lgt.lgt_destroy(ctx)
    ref = U.copy()
    O.half_sweep(ref, 0, gauge=GAUGES[gauge], omega=1.7)
    assert np.abs(half - ref).max() < 5e-6
    assert np.abs(plaquettes(V) - plaquettes(U)).max() < 3e-13
    e, d = unitarity_error(V)
    assert e < 3e-13 and d < 3e-13


@pytest.mark.parametrize("polish", ["pair", "fp64", "anchor"])
def test_fix_with_each_polish_kernel(lgt, polish):
    dims = (4, 8, 8, 8)
    U = synth.field(dims, 0.5, 15)
    pk = {"pair": lgt.LGT_POLISH_PAIR, "fp64": lgt.LGT_POLISH_FP64, "anchor": lgt.LGT_POLISH_ANCHOR}[polish]
    p = lgt.lgt_params_default(dims=dims, bulk=lgt.LGT_FP32_12, polish=pk, theta_switch=1e-8, max_sweeps=4000)
    ctx = lgt.lgt_create(p, U)
    try:
        st, res = lgt.lgt_fix(ctx)
        V = lgt.lgt_get_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    ref = U.copy()
    r = O.fix(ref, omega=1.7, tol=1e-14, max_sweeps=4000)
    assert st == lgt.LGT_OK and res.sweeps_fp64 > 0 and abs(res.F - r["F"]) < 1e-10
    m = O.measure(V)
    assert m["theta"] < 1e-14
    e, d = unitarity_error(V)
    assert e < 1e-12 and d < 1e-12
    assert np.abs(plaquettes(V) - plaquettes(U)).max() < 1e-12


# ------------------------------------------------------- full size: 32^4
@pytest.fixture(scope="module")
def field_32():
    """SU(3) Landau 32^4, eps = 0.5, seed 2 (the benchmark's field)."""
    return synth.field((32, 32, 32, 32), 0.5, 2)


@pytest.mark.parametrize("bulk", ["fp64", "fp32_18", "fp32_12"])
def test_full_size_one_sweep_32(lgt, field_32, bulk):
    """32^4 (the benchmark's field and launch configuration), every link: the even half
    within 1e-12 (FP64) / 5e-6 (FP32); the full sweep within 1e-12 (FP64) and, on FP32
    storage, every entry within max(5e-6, B) with B the link's first-order bound
    from the conditioning of the two site updates that wrote it (see the
    small-lattice test)."""
    b = {"fp64": lgt.LGT_FP64, "fp32_18": lgt.LGT_FP32_18, "fp32_12": lgt.LGT_FP32_12}[bulk]
    fp64 = b == lgt.LGT_FP64
    half = gpu_half(lgt, field_32, 0, bulk=b, omega=1.7, reunit_every=0)
    ref = field_32.copy()
    O.half_sweep(ref, 0, omega=1.7)
    err = np.abs(half - ref).max()
    assert err < (1e-12 if fp64 else 5e-6), err
    del half
    got = gpu_run(lgt, field_32, 1, working=True, bulk=b, omega=1.7, reunit_every=0)
    k_even = O.site_conditioning(field_32, 0, omega=1.7)
    k_odd = O.site_conditioning(ref, 1, omega=1.7)
    O.half_sweep(ref, 1, omega=1.7)
    err = np.abs(got - ref)
    del got
    if fp64:
        assert err.max() < 1e-12, err.max()
    else:
        ratio, n_above, n_links = check_fp32_bound(err, fp32_sweep_bound(k_even, k_odd))
        assert ratio <= 1.0, (ratio, err.max(), n_above, n_links)


def test_full_size_fix_32_properties(lgt, field_32):
    """The benchmark's run (FP32-12 bulk + anchored polish to 1e-14): the oracle
    certifies theta < 1e-14 on the returned field; every plaquette and unitarity are
    kept to 1e-12 (the output is G U' G^+ formed in FP64 with G orthonormalised in
    FP64: an exact gauge transform up to FP64 rounding)."""
    dims = (32, 32, 32, 32)
    p = lgt.lgt_params_default(dims=dims, omega=1.7, bulk=lgt.LGT_FP32_12, max_sweeps=20000)
    ctx = lgt.lgt_create(p, field_32)
    try:
        st, res = lgt.lgt_fix(ctx)
        V = lgt.lgt_get_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    assert st == lgt.LGT_OK and res.theta < 1e-14
    m = O.measure(V)
    assert m["theta"] < 1e-14 and abs(m["F"] - res.F) < 1e-12
    assert np.abs(plaquettes(V) - plaquettes(field_32)).max() < 1e-12
    e, d = unitarity_error(V)
    assert e < 1e-12 and d < 1e-12


def test_resume_is_bit_identical(lgt):
    """A job's state is its links and its sweep counter: stopping after 10 sweeps and
    restarting from the saved links with sweep_offset = 10 gives the same bits."""
    dims = (4, 6, 4, 8)
    U = synth.field(dims, 0.5, 31)
    kw = dict(dims=dims, algo=lgt.LGT_SR, p=0.8, seed=9)
    ctx = lgt.lgt_create(lgt.lgt_params_default(**kw), U)
    try:
        lgt.lgt_sweep(ctx, 10)
        mid = lgt.lgt_get_links(ctx, dims)
        lgt.lgt_sweep(ctx, 5)
        straight = lgt.lgt_get_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    ctx = lgt.lgt_create(lgt.lgt_params_default(sweep_offset=10, **kw), mid)
    try:
        lgt.lgt_sweep(ctx, 5)
        resumed = lgt.lgt_get_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    assert np.array_equal(straight, resumed)


# ------------------------------------------------ full size, sampled sites
def _sampled_half_sweep_check(lgt, U, gauge, n_samples, seed):
    """Even half-sweep on the GPU (FP32-12 bulk kernel, and the default polish kernel
    after promotion) against the oracle's update of randomly sampled even sites from
    the same input."""
    from lattice_np import AXIS
    dims = U.shape[:4]
    rng = np.random.default_rng(seed)
    V = int(np.prod(dims))
    sites = []
    while len(sites) < n_samples:
        s = int(rng.integers(V))
        t, x3, x2, x1 = np.unravel_index(s, dims)
        if (t + x3 + x2 + x1) % 2 == 0:
            sites.append(s)
    ref = {s: O.site_new_links(U, s, gauge=gauge, omega=1.7) for s in sites}
    for bulk, promote in [(lgt.LGT_FP32_12, False), (lgt.LGT_FP32_12, True)]:
        p = lgt.lgt_params_default(dims=dims, gauge=gauge, omega=1.7, omega_polish=0.0, bulk=bulk,
                                   reunit_every=0)
        ctx = lgt.lgt_create(p, U)
        try:
            if promote:
                lgt.lgt_promote(ctx)
            lgt.lgt_half_sweep(ctx, 0)
            got = lgt.lgt_get_working_links(ctx, dims)
        finally:
            lgt.lgt_destroy(ctx)
        worst = 0.0
        for s in sites:
            fwd, bwd = ref[s]
            c = np.unravel_index(s, dims)
            worst = max(worst, np.abs(got[c] - fwd).max())
            for mu in range(4):
                cb = list(c)
                cb[AXIS[mu]] = (cb[AXIS[mu]] - 1) % dims[AXIS[mu]]
                worst = max(worst, np.abs(got[tuple(cb)][mu] - bwd[mu]).max())
        assert worst < 5e-6, (bulk, promote, worst)
        del got


def test_full_size_64x4_sampled(lgt):
    """SU(3) Landau 64^4, eps = 0.7, seed 5: 400 sampled sites."""
    U = synth.field((64, 64, 64, 64), 0.7, 5)
    _sampled_half_sweep_check(lgt, U, O.LANDAU, 400, 1)


def test_full_size_coulomb_48x3x96_sampled(lgt):
    """SU(3) Coulomb 48^3 x 96, eps = 0.5, seed 3 (96 slices in one launch): 400 sampled sites."""
    U = synth.field((96, 48, 48, 48), 0.5, 3)
    _sampled_half_sweep_check(lgt, U, O.COULOMB, 400, 2)


def test_omega_polish_drives_the_sweeps_after_promotion(lgt, near_fixed_8):
    U = near_fixed_8[(O.LANDAU, 1e-12)]
    ctx = promoted_ctx(lgt, U, omega=1.7, omega_polish=1.9)
    try:
        lgt.lgt_sweep(ctx, 2)
        got = lgt.lgt_get_links(ctx, U.shape[:4])
    finally:
        lgt.lgt_destroy(ctx)
    ref = U.copy()
    O.sweeps(ref, 2, omega=1.9)
    assert np.abs(got - ref).max() < 1e-12
    ref17 = U.copy()
    O.sweeps(ref17, 2, omega=1.7)
    assert np.abs(got - ref17).max() > 1e-11


@pytest.mark.parametrize("polish", ["pair", "anchor"])
def test_polish_algo_switches_stochastic_relaxation_to_overrelaxation(lgt, near_fixed_8, polish):
    """polish_algo = LGT_POLISH_OR: a stochastic-relaxation job's sweeps after
    promotion are the oracle's overrelaxation sweeps at omega_polish (Sec. 3.1);
    with the default LGT_POLISH_SAME they stay the oracle's stochastic-relaxation
    sweeps (Sec. 3.2, same random stream).  8^4 field near the maximum (theta ~
    1e-12), two sweeps after promotion, to the polish tolerance."""
    U = near_fixed_8[(O.LANDAU, 1e-12)]
    kw = dict(algo=lgt.LGT_SR, p=0.8, seed=5)
    out = {}
    for pa in (lgt.LGT_POLISH_OR, lgt.LGT_POLISH_SAME):
        ctx = promoted_ctx(lgt, U, polish=polish, omega_polish=1.3, polish_algo=pa, **kw)
        try:
            lgt.lgt_sweep(ctx, 2)
            out[pa] = lgt.lgt_get_links(ctx, U.shape[:4])
        finally:
            lgt.lgt_destroy(ctx)
    tol = 1e-12  # the polish kernels' FP32 rotation angles at theta ~ 1e-12 (test above)
    ref_or = U.copy()
    O.sweeps(ref_or, 2, omega=1.3)
    assert np.abs(out[lgt.LGT_POLISH_OR] - ref_or).max() < tol
    ref_sr = U.copy()
    O.sweeps(ref_sr, 2, algo=O.SR, p=0.8, seed=5)
    assert np.abs(out[lgt.LGT_POLISH_SAME] - ref_sr).max() < tol
    assert np.abs(out[lgt.LGT_POLISH_OR] - ref_sr).max() > 10 * tol


def test_polish_algo_fix_reaches_the_stochastic_relaxation_maximum(lgt):
    """A stochastic-relaxation fix (FP32-12 bulk, p 0.8) polished by overrelaxation
    ends at the oracle's stochastic-relaxation F to 1e-10 with theta certified,
    in fewer polish sweeps than the same job polished by stochastic relaxation;
    served, it converges the same way."""
    dims = (8, 8, 8, 8)
    U = synth.field(dims, 0.3, 9)
    ref = U.copy()
    r = O.fix(ref, algo=O.SR, p=0.8, seed=5, tol=1e-14, max_sweeps=6000)
    assert r["converged"]
    res = {}
    links = {}
    for pa in (lgt.LGT_POLISH_OR, lgt.LGT_POLISH_SAME):
        p = lgt.lgt_params_default(dims=dims, algo=lgt.LGT_SR, p=0.8, seed=5, bulk=lgt.LGT_FP32_12,
                                   max_sweeps=6000, polish_algo=pa)
        ctx = lgt.lgt_create(p, U)
        try:
            st, res[pa] = lgt.lgt_fix(ctx)
            links[pa] = lgt.lgt_get_links(ctx, dims)
        finally:
            lgt.lgt_destroy(ctx)
        assert st == lgt.LGT_OK and res[pa].theta < 1e-14
        assert abs(res[pa].F - r["F"]) < 1e-10, (pa, res[pa].F, r["F"])
    m = O.measure(links[lgt.LGT_POLISH_OR])
    assert m["theta"] < 1e-14
    assert res[lgt.LGT_POLISH_OR].sweeps_fp64 < res[lgt.LGT_POLISH_SAME].sweeps_fp64
    p = lgt.lgt_params_default(dims=dims, algo=lgt.LGT_SR, p=0.8, seed=5, bulk=lgt.LGT_FP32_12,
                               max_sweeps=6000, polish_algo=lgt.LGT_POLISH_OR)
    srv = lgt.lgt_server_create(1 << 30)
    try:
        jid = lgt.lgt_submit(srv, p, U)
        out = np.empty_like(U)
        while True:
            st, sres = lgt.lgt_poll(srv, jid, out)
            if st != lgt.LGT_EAGAIN:
                break
            time.sleep(0.01)
    finally:
        lgt.lgt_server_destroy(srv)
    assert st == lgt.LGT_OK and sres.theta < 1e-14 and abs(sres.F - r["F"]) < 1e-10
    assert sres.sweeps_fp64 < res[lgt.LGT_POLISH_SAME].sweeps_fp64
    assert O.measure(out)["theta"] < 1e-14


@pytest.mark.parametrize("bulk", ["fp32_18", "fp32_12"])
@pytest.mark.parametrize("gauge", list(GAUGES))
@pytest.mark.parametrize("algo", list(ALGOS))
def test_launch_configurations_agree(lgt, bulk, gauge, algo):
    """Every launch configuration (one or four threads per site, every block size,
    pipelined through shared memory, lean, streaming) groups the fused estimate
    by the same 8 sites; they differ in FP32 rounding only (the lean ones sum
    K(x) link by link, the others pairwise, and the compiler fuses multiply-adds
    differently in each kernel), which an ill-conditioned site update amplifies.
    So the test compares what the method fixes: each configuration's half-sweep
    is within the per-site FP32 bound of the oracle's, and ladder runs converge
    to the same F.  The ragged lattice leaves a partial block in every
    configuration."""
    U = synth.field(DIMS_RAGGED, 0.5, 21)
    kw = dict(bulk=getattr(lgt, "LGT_" + bulk.upper()), gauge=GAUGES[gauge], algo=ALGOS[algo], p=0.8, seed=5,
              reunit_every=2)
    ncfg = 16
    half = U.copy()
    O.half_sweep(half, 0, gauge=GAUGES[gauge], algo=ALGOS[algo], omega=1.7, p=0.8, seed=5)
    kappa = O.site_conditioning(U, 0, gauge=GAUGES[gauge], algo=ALGOS[algo], omega=1.7, p=0.8, seed=5)
    bound = fp32_half_sweep_bound(kappa, 0, 16.0)
    for k in range(ncfg):
        p = lgt.lgt_params_default(dims=U.shape[:4], launch_config=k + 1, **kw)
        ctx = lgt.lgt_create(p, U)
        try:
            lgt.lgt_half_sweep(ctx, 0)
            out = lgt.lgt_get_working_links(ctx, U.shape[:4])
        finally:
            lgt.lgt_destroy(ctx)
        ratio, n_above, n_links = check_fp32_bound(np.abs(out - half), bound)
        assert ratio <= 1.0, f"launch configuration {k}: {ratio} of the allowed error after a half-sweep"
    ref = None
    for k in range(ncfg):
        p = lgt.lgt_params_default(dims=U.shape[:4], launch_config=k + 1, theta_tol=1e-12, max_sweeps=3000, **kw)
        ctx = lgt.lgt_create(p, U)
        try:
            st, res = lgt.lgt_fix(ctx)
            cfgs = lgt.lgt_get_stats(ctx).launch_config
        finally:
            lgt.lgt_destroy(ctx)
        supported = k not in (7, 10, 12, 13, 14, 15) or bulk == "fp32_12"  # the staged layouts hold 12-real links only
        assert st == lgt.LGT_OK and cfgs[0] == (k if supported else 0) and res.theta < 1e-12
        if ref is None:
            ref = res.F
        assert abs(res.F - ref) < 1e-10, f"launch configuration {k}: F {res.F} vs {ref}"


@pytest.mark.parametrize("gauge", list(GAUGES))
@pytest.mark.parametrize("algo", list(ALGOS))
def test_streaming_sweeps_match_the_pipelined_kernel(lgt, gauge, algo):
    """The streaming configuration runs up to 64 half-sweeps per launch and starts
    a slice of half-sweep h as soon as half-sweep h - 1 has finished it and its
    two neighbours.  Its site update is the pipelined configuration's, so any
    read of a link before its writer finished would show as a difference:
    40 sweeps (80 half-sweeps, two launches) from a rough field, with the SR
    counter and the reunitarisation schedule (every 3 sweeps) taken per item,
    give the pipelined kernel's links bit for bit, and stay within FP32
    rounding of the one-thread kernel.  12 slices of a ragged 6x10x14 volume
    (4 tiles per slice, the last partial); a single odd half-sweep first."""
    dims = (12, 6, 10, 14)
    U = synth.field(dims, 0.5, 23)
    kw = dict(dims=dims, bulk=lgt.LGT_FP32_12, gauge=GAUGES[gauge], algo=ALGOS[algo], omega=1.7, p=0.8, seed=9,
              reunit_every=3)
    out = {}
    for k in (0, 7, 10, 12):
        ctx = lgt.lgt_create(lgt.lgt_params_default(launch_config=k + 1, **kw), U)
        try:
            lgt.lgt_half_sweep(ctx, 1)
            lgt.lgt_sweep(ctx, 40)
            out[k] = lgt.lgt_get_working_links(ctx, dims)
            st = lgt.lgt_get_stats(ctx)
            sb, _, _ = lgt.lgt_get_progress(ctx)
        finally:
            lgt.lgt_destroy(ctx)
        assert st.launch_config[0] == k and sb == 41 and st.sweep_launches[0] == 81
    assert np.array_equal(out[10], out[7])
    assert np.array_equal(out[12], out[7])
    assert np.abs(out[10] - out[0]).max() < 1e-4
    assert max(unitarity_error(out[10])) < 1e-5


@pytest.mark.parametrize("band,tiles", [("2,1", "1"), ("3,3", "3"), ("6,2", "2"), ("1,5", "4"), ("12,1", "1")])
def test_rolling_band_shapes_match_the_pipelined_kernel(lgt, band, tiles, monkeypatch):
    """Configuration 12 with other band shapes (LGT_STREAM_BAND="B,G": about B
    half-sweeps at once, G slices apart; D = max(ceil(nt / B), G + 1) waves of
    stagger, S = D - G) and item sizes: 30 sweeps (60 half-sweeps, one launch)
    of stochastic relaxation from a rough field give the pipelined kernel's
    links bit for bit, and so does a launch of 3 half-sweeps.  14 slices of a
    ragged 6x10x14 volume."""
    dims = (14, 6, 10, 14)
    U = synth.field(dims, 0.5, 24)
    kw = dict(dims=dims, bulk=lgt.LGT_FP32_12, algo=lgt.LGT_SR, p=0.8, seed=11, reunit_every=4)
    monkeypatch.setenv("LGT_STREAM_BAND", band)
    monkeypatch.setenv("LGT_STREAM_BAND_TILES", tiles)
    out = {}
    for k in (7, 12):
        ctx = lgt.lgt_create(lgt.lgt_params_default(launch_config=k + 1, **kw), U)
        try:
            lgt.lgt_sweep(ctx, 30)
            lgt.lgt_half_sweep(ctx, 0)
            lgt.lgt_sweep(ctx, 1)
            lgt.lgt_half_sweep(ctx, 1)
            out[k] = lgt.lgt_get_working_links(ctx, dims)
            st = lgt.lgt_get_stats(ctx)
        finally:
            lgt.lgt_destroy(ctx)
        assert st.launch_config[0] == k and st.sweep_launches[0] == 64
    assert np.array_equal(out[12], out[7])


@pytest.mark.parametrize("bulk", ["fp64", "fp32_12"])
@pytest.mark.parametrize("gauge", list(GAUGES))
@pytest.mark.parametrize("algo", list(ALGOS))
def test_device_loop_is_bit_identical(lgt, bulk, gauge, algo):
    """lgt_fix runs whole chunks (check_every sweeps, the estimate, the decision) as
    a CUDA graph with a conditional while node; the host-driven chunks
    (LGT_FIX_GRAPHS=0) make the same decisions on the same estimates, so results,
    sweep counts and links agree bit for bit.  max_sweeps is not a multiple of
    check_every, so the host also runs a short last chunk when it is reached."""
    import os
    dims = (4, 6, 8, 10)
    U = synth.field(dims, 0.5, 41)
    kw = dict(dims=dims, bulk=getattr(lgt, "LGT_" + bulk.upper()), gauge=GAUGES[gauge], algo=ALGOS[algo],
              p=0.8, seed=3, theta_tol=1e-13, max_sweeps=2003)
    out = {}
    for mode in ("1", "0"):
        old = os.environ.get("LGT_FIX_GRAPHS")
        os.environ["LGT_FIX_GRAPHS"] = mode
        try:
            ctx = lgt.lgt_create(lgt.lgt_params_default(**kw), U)
        finally:
            if old is None:
                del os.environ["LGT_FIX_GRAPHS"]
            else:
                os.environ["LGT_FIX_GRAPHS"] = old
        try:
            st, res = lgt.lgt_fix(ctx)
            links = lgt.lgt_get_links(ctx, dims)
            stats = lgt.lgt_get_stats(ctx)
        finally:
            lgt.lgt_destroy(ctx)
        out[mode] = (st, res.as_dict(), links, stats.as_dict())
    (s1, r1, l1, t1), (s0, r0, l0, t0) = out["1"], out["0"]
    assert s1 == s0 and r1["sweeps_bulk"] == r0["sweeps_bulk"] and r1["sweeps_fp64"] == r0["sweeps_fp64"]
    assert r1["F"] == r0["F"] and r1["theta"] == r0["theta"] and np.array_equal(l1, l0)
    assert t1["site_updates"] == t0["site_updates"] and t1["sweep_launches"] == t0["sweep_launches"]
    assert t0["loop_launches"] == 0 and t1["loop_launches"] > 0 and t1["loop_chunks"] >= t1["loop_launches"]
    if s1 == lgt.LGT_OK:
        assert r1["theta"] < 1e-13


def test_coulomb_bulk_runs_to_the_fp32_floor(lgt):
    """Coulomb 32^3 x 64 (eps 0.5176, seed 1003; a job of the served stream): the
    estimate (a max over 64 slices) can stall for a few checks far above any FP32
    floor; the bulk phase must not stop there (that left the polish a large
    transformation and a floor above 1e-14)."""
    dims = (64, 32, 32, 32)
    U = synth.field(dims, 0.5175765603053992, 1003)
    p = lgt.lgt_params_default(dims=dims, gauge=lgt.LGT_COULOMB, bulk=lgt.LGT_FP32_12, theta_tol=1e-14,
                               max_sweeps=20000)
    ctx = lgt.lgt_create(p, U)
    try:
        st, res = lgt.lgt_fix(ctx)
    finally:
        lgt.lgt_destroy(ctx)
    assert st == lgt.LGT_OK and res.theta < 1e-14, res.as_dict()
    assert res.sweeps_bulk > 1000, res.as_dict()


def test_anchored_polish_from_an_early_promotion(lgt):
    """Promoted far from convergence (after 10 sweeps), the anchored polish carries
    a large transformation; renewing the anchor every 500 sweeps keeps its FP32
    correction small, so it still reaches 1e-14 (>= 500 polish sweeps here, so at
    least one renewal), the result is a gauge transform of the input, and F is the
    one the normal ladder reaches."""
    dims = (16, 16, 16, 16)
    U = synth.field(dims, 0.5, 17)
    p = lgt.lgt_params_default(dims=dims, bulk=lgt.LGT_FP32_12, theta_tol=1e-14, max_sweeps=20000)
    ctx = lgt.lgt_create(p, U)
    try:
        lgt.lgt_sweep(ctx, 10)
        lgt.lgt_promote(ctx)
        st, res = lgt.lgt_fix(ctx)
        V = lgt.lgt_get_links(ctx, dims)
        lgt.lgt_load(ctx, U)
        st2, res2 = lgt.lgt_fix(ctx)
    finally:
        lgt.lgt_destroy(ctx)
    assert st == lgt.LGT_OK and res.sweeps_fp64 >= 500, res.as_dict()
    assert st2 == lgt.LGT_OK and abs(res.F - res2.F) < 1e-10
    m = O.measure(V)
    assert m["theta"] < 1e-14
    assert np.abs(plaquettes(V) - plaquettes(U)).max() < 1e-12


@pytest.mark.parametrize("skip", [1, 3])
def test_streaming_wait_times_out_and_the_context_recovers(lgt, skip):
    """The streaming launches' bounded waits, made to expire on purpose from the
    host (lgt_inject_stream_stall): the launch's first items are never taken, so
    the next half-sweep waits for slices that never become ready.  After the 1 ms
    limit the launch ends with LGT_ETIMEOUT, every later synchronisation of the
    context reports it, and lgt_load clears it: the next sweeps give the bits of a
    fresh context.  8 slices of 8x8x16 (4 tiles each, one item per slice)."""
    import time
    dims = (8, 8, 8, 16)
    U = synth.field(dims, 0.5, 24)
    p = lgt.lgt_params_default(dims=dims, bulk=lgt.LGT_FP32_12, omega=1.7, launch_config=11)
    ctx = lgt.lgt_create(p, U)
    try:
        lgt.lgt_inject_stream_stall(ctx, 1_000_000, skip)
        t0 = time.perf_counter()
        with pytest.raises(lgt.LgtError) as e:
            lgt.lgt_sweep(ctx, 2)
        assert e.value.status == lgt.LGT_ETIMEOUT and "timed out" in lgt.lgt_last_error()
        assert time.perf_counter() - t0 < 1.5  # the 1 ms limit, not the built-in 2 s
        with pytest.raises(lgt.LgtError) as e:
            lgt.lgt_measure(ctx)
        assert e.value.status == lgt.LGT_ETIMEOUT
        lgt.lgt_load(ctx, U)
        lgt.lgt_sweep(ctx, 3)
        got = lgt.lgt_get_working_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    ctx = lgt.lgt_create(p, U)
    try:
        lgt.lgt_sweep(ctx, 3)
        fresh = lgt.lgt_get_working_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    assert np.array_equal(got, fresh)


@pytest.mark.parametrize("graphs", ["1", "0"])
def test_omega_schedule_switches_at_a_check(lgt, graphs, monkeypatch):
    """The omega schedule (Sec. 3.1 overrelaxation with a late omega): lgt_fix
    sweeps at omega until a check finds the estimate below theta_omega, then at
    omega_late.  theta_omega sits between theta of the input and theta after the
    first chunk of 10 sweeps, so the result of 20 sweeps is 10 oracle sweeps at
    omega = 1.7 and 10 at omega_late = 1.2 (FP64, 1e-11), whether the chunks run
    as the device loop or from the host (LGT_FIX_GRAPHS=0)."""
    monkeypatch.setenv("LGT_FIX_GRAPHS", graphs)
    dims = (4, 6, 4, 8)
    U = synth.field(dims, 0.5, 25)
    th0 = O.measure(U)["theta"]
    ref = U.copy()
    O.sweeps(ref, 10, omega=1.7)
    th10 = O.measure(ref)["theta"]
    switch = np.sqrt(th0 * th10)
    p = lgt.lgt_params_default(dims=dims, omega=1.7, omega_late=1.2, theta_omega=switch, max_sweeps=20)
    ctx = lgt.lgt_create(p, U)
    try:
        st, res = lgt.lgt_fix(ctx)
        got = lgt.lgt_get_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    assert st == lgt.LGT_ENOTCONV and res.sweeps_fp64 == 20
    O.sweeps(ref, 10, omega=1.2, sweep0=10)
    assert np.abs(got - ref).max() < 1e-11
    late = U.copy()
    O.sweeps(late, 20, omega=1.2)
    assert np.abs(got - late).max() > 1e-6  # the first chunk did run at omega = 1.7


@pytest.mark.parametrize("bulk", ["fp64", "fp32_12"])
def test_omega_schedule_converges_to_the_oracle_F(lgt, bulk):
    """A fix with the schedule (omega 1.5, then 1.1 below theta 1e-4) ends at the
    oracle's converged F (1e-10; the oracle relaxes at a fixed omega = 1.7) and the
    oracle certifies theta < 1e-14 on the returned field; served alike."""
    dims = (8, 8, 8, 8)
    U = synth.field(dims, 0.3, 1)
    ref = U.copy()
    r = O.fix(ref, omega=1.7, tol=1e-14, max_sweeps=1000)
    kw = dict(dims=dims, bulk=getattr(lgt, "LGT_" + bulk.upper()), omega=1.5, omega_late=1.1, theta_omega=1e-4,
              max_sweeps=1000)
    ctx = lgt.lgt_create(lgt.lgt_params_default(**kw), U)
    try:
        st, res = lgt.lgt_fix(ctx)
        V = lgt.lgt_get_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    assert st == lgt.LGT_OK and abs(res.F - r["F"]) < 1e-10
    assert O.measure(V)["theta"] < 1e-14
    srv = lgt.lgt_server_create(1 << 30, 0)
    try:
        jid = lgt.lgt_submit(srv, lgt.lgt_params_default(**kw), U)
        while True:
            st2, res2 = lgt.lgt_poll(srv, jid)
            if st2 != lgt.LGT_EAGAIN:
                break
            time.sleep(0.002)
    finally:
        lgt.lgt_server_destroy(srv)
    assert st2 == lgt.LGT_OK and abs(res2.F - r["F"]) < 1e-10


# ------------------------------------------------ simulated annealing
@pytest.mark.parametrize("gauge", list(GAUGES))
def test_annealing_sweeps_match_the_oracle(lgt, gauge):
    """The heat-bath sweeps draw from the same Philox streams as the oracle; in
    FP64 the Kennedy-Pendleton accept/reject decisions agree (they differ only if
    a comparison falls within rounding of its threshold), so three annealing
    sweeps agree with the oracle to FP64 rounding.  In FP32 storage and
    arithmetic a few decisions may flip; nearly every entry still agrees to
    FP32 accuracy and the result is a gauge transform of the input."""
    U = synth.field(DIMS_RAGGED, 0.5, 51)
    g = GAUGES[gauge]
    ref = U.copy()
    O.sa_sweeps(ref, 3, 2.0, 20.0, gauge=g, seed=13)
    for bulk, tol in [(lgt.LGT_FP64, 1e-11), (lgt.LGT_FP32_12, 1e-5)]:
        p = lgt.lgt_params_default(dims=U.shape[:4], gauge=g, bulk=bulk, seed=13, sa_sweeps=3, sa_beta0=2.0,
                                   sa_beta1=20.0, max_sweeps=3, reunit_every=0)
        ctx = lgt.lgt_create(p, U)
        try:
            st, res = lgt.lgt_fix(ctx)  # the 3 annealing sweeps use up max_sweeps
            V = lgt.lgt_get_links(ctx, U.shape[:4]) if bulk == lgt.LGT_FP64 else lgt.lgt_get_working_links(ctx, U.shape[:4])
            Vg = lgt.lgt_get_links(ctx, U.shape[:4])
        finally:
            lgt.lgt_destroy(ctx)
        assert st == lgt.LGT_ENOTCONV and res.sweeps_bulk + res.sweeps_fp64 == 3
        err = np.abs(V - ref)
        if bulk == lgt.LGT_FP64:
            assert err.max() < tol, err.max()
        # (FP32: element by element in test_fp32_annealing_sweep_matches_the_oracle_but_near_thresholds)
        assert np.abs(plaquettes(Vg) - plaquettes(U)).max() < 1e-12


@pytest.mark.parametrize("gauge", list(GAUGES))
def test_fp32_annealing_sweep_matches_the_oracle_but_near_thresholds(lgt, gauge):
    """One FP32 annealing sweep (beta = 2) against the oracle's, element by element.
    The heat bath draws from the same Philox streams; FP32 rounding moves a
    Kennedy-Pendleton comparison u^2 <= 1 - delta/2 across its threshold only where
    the oracle's margin is within it, and there the site may draw another element
    (and the odd sites next to such an even site see another K).  Those sites are
    the ones whose smallest relative margin (oracle, each half on the field it
    started from) is below 1e-4, two orders above the FP32 error of delta (~8u
    times (1 + kappa)); their links are excused, they must be few, and every other
    entry agrees within 1e-5."""
    from lattice_np import link_endpoint, parity_field, shift
    g = GAUGES[gauge]
    dims = DIMS_RAGGED
    U = synth.field(dims, 0.5, 51)
    beta = 2.0
    ref = U.copy()
    O.sa_sweeps(ref, 1, beta, beta, gauge=g, seed=13)
    p = lgt.lgt_params_default(dims=dims, gauge=g, bulk=lgt.LGT_FP32_12, seed=13, sa_sweeps=1, sa_beta0=beta,
                               sa_beta1=beta, max_sweeps=1, reunit_every=0)
    ctx = lgt.lgt_create(p, U)
    try:
        st, res = lgt.lgt_fix(ctx)
        V = lgt.lgt_get_working_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    assert st == lgt.LGT_ENOTCONV and res.sweeps_bulk == 1
    _, m_even = O.sa_site_stats(U, 0, beta, gauge=g, seed=13)
    half = U.copy()
    O.sa_half_sweep(half, 0, beta, gauge=g, seed=13)
    _, m_odd = O.sa_site_stats(half, 1, beta, gauge=g, seed=13)
    par = parity_field(dims)
    near_even = (par == 0) & (np.nan_to_num(m_even, nan=1.0) < 1e-4)
    near_odd = (par == 1) & (np.nan_to_num(m_odd, nan=1.0) < 1e-4)
    beside = np.zeros(dims, bool)
    for mu in range(4):
        beside |= shift(near_even, mu, 1) | shift(near_even, mu, -1)
    flagged = (near_even | near_odd | ((par == 1) & beside)).astype(float)
    excused = (link_endpoint(flagged, 0) + link_endpoint(flagged, 1)) > 0
    err = np.abs(V - ref).max(axis=(-1, -2))
    assert excused.mean() < 0.02, excused.mean()
    assert err[~excused].max() < 1e-5, (err[~excused].max(), int(excused.sum()))


def test_annealing_then_relaxation(lgt):
    """lgt_fix with annealing first: the FP64 path follows the oracle's annealing
    and relaxation to the same converged F; the mixed ladder converges too."""
    dims = (4, 6, 4, 8)
    U = synth.field(dims, 0.6, 52)
    kw = dict(dims=dims, seed=21, sa_sweeps=40, sa_beta0=1.0, sa_beta1=100.0, theta_tol=1e-14, max_sweeps=5000)
    ref = U.copy()
    O.sa_sweeps(ref, 40, 1.0, 100.0, seed=21)
    r = O.fix(ref, omega=1.7, tol=1e-14, max_sweeps=5000)
    out = {}
    for bulk in (lgt.LGT_FP64, lgt.LGT_FP32_12):
        ctx = lgt.lgt_create(lgt.lgt_params_default(bulk=bulk, **kw), U)
        try:
            st, res = lgt.lgt_fix(ctx)
            V = lgt.lgt_get_links(ctx, dims)
        finally:
            lgt.lgt_destroy(ctx)
        assert st == lgt.LGT_OK and O.measure(V)["theta"] < 1e-14
        assert np.abs(plaquettes(V) - plaquettes(U)).max() < 1e-12
        out[bulk] = res.F
    assert abs(out[lgt.LGT_FP64] - r["F"]) < 1e-10


@pytest.mark.parametrize("bulk", ["fp32_12", "fp32_18"])
def test_long_fp32_annealing_stays_unitary(lgt, bulk):
    """Hundreds of heat-bath sweeps at low beta rotate every site far from the
    identity.  G (and 12-real links) keep two rows in FP32 and rebuild the third,
    which under such rotations amplifies the rows' norm error by about 4/3 per
    update; without reprojection it overflows within some 50 sweeps.  After 300
    FP32 annealing sweeps the working links and the transformed FP64 field are
    finite and unitary, the plaquettes are those of the input, and the ladder
    then converges."""
    dims = (8, 8, 8, 8)
    U = synth.field(dims, 1.0, 302)
    kw = dict(dims=dims, bulk=getattr(lgt, "LGT_" + bulk.upper()), seed=3, sa_sweeps=300, sa_beta0=0.5,
              sa_beta1=50.0, reunit_every=0)
    ctx = lgt.lgt_create(lgt.lgt_params_default(max_sweeps=300, **kw), U)
    try:
        st, res = lgt.lgt_fix(ctx)  # the annealing sweeps use up max_sweeps
        W = lgt.lgt_get_working_links(ctx, dims)
        V = lgt.lgt_get_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    assert st == lgt.LGT_ENOTCONV and res.sweeps_bulk == 300
    for X in (W, V):
        assert np.isfinite(X.view(np.float64)).all()
    assert max(unitarity_error(W)) < 1e-5 and max(unitarity_error(V)) < 1e-12
    assert np.abs(plaquettes(V) - plaquettes(U)).max() < 1e-12
    ctx = lgt.lgt_create(lgt.lgt_params_default(max_sweeps=40000, theta_tol=1e-14, **kw), U)
    try:
        st, res = lgt.lgt_fix(ctx)
        V = lgt.lgt_get_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    assert st == lgt.LGT_OK and O.measure(V)["theta"] < 1e-14
    assert np.abs(plaquettes(V) - plaquettes(U)).max() < 1e-12


def test_annealing_is_not_served(lgt):
    srv = lgt.lgt_server_create(1 << 30, 0)
    try:
        p = lgt.lgt_params_default(dims=(4, 4, 4, 4), sa_sweeps=5)
        with pytest.raises(lgt.LgtError) as e:
            lgt.lgt_submit(srv, p, synth.field((4, 4, 4, 4), 0.3, 1))
        assert e.value.status == lgt.LGT_EINVAL
    finally:
        lgt.lgt_server_destroy(srv)


# ------------------------------------------------- maximally Abelian gauge
def _abelian_transformed(dims, seed, spread=0.35):
    """A diagonal (Abelian) field under a random gauge transformation near 1: its
    maximally Abelian gauge has F_MAG = 1."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(-np.pi, np.pi, size=tuple(dims) + (4, 2))
    A = np.zeros(tuple(dims) + (4, 3, 3), np.complex128)
    A[..., 0, 0] = np.exp(1j * phi[..., 0])
    A[..., 1, 1] = np.exp(1j * phi[..., 1])
    A[..., 2, 2] = np.exp(-1j * (phi[..., 0] + phi[..., 1]))
    from lattice_np import GELL_MANN, expm_herm, transform_field
    n = int(np.prod(dims))
    G = np.stack([expm_herm(spread * np.einsum("a,aij->ij", rng.normal(size=8), GELL_MANN))
                  for _ in range(n)]).reshape(tuple(dims) + (3, 3))
    return A, np.ascontiguousarray(transform_field(A, G))


@pytest.mark.parametrize("dims", [DIMS_RAGGED, (2, 2, 2, 2)])
def test_mag_measurement_matches_oracle(lgt, dims):
    """F_MAG, theta_MAG and the plaquette of the exact FP64 measurement kernel."""
    U = synth.field(dims, 0.5, 61)
    ctx = lgt.lgt_create(lgt.lgt_params_default(dims=dims, gauge=lgt.LGT_MAG), U)
    try:
        F, theta, plaq = lgt.lgt_measure(ctx)
    finally:
        lgt.lgt_destroy(ctx)
    m = O.measure(U, O.MAG)
    assert abs(F - m["F"]) < 1e-14 and abs(theta - m["theta"]) < 1e-12 * m["theta"]
    assert abs(plaq - m["plaq"]) < 1e-14


@pytest.mark.parametrize("bulk", ["fp64", "fp32_18", "fp32_12"])
@pytest.mark.parametrize("algo", list(ALGOS))
@pytest.mark.parametrize("parity", [0, 1])
def test_mag_half_sweep_matches_oracle(lgt, bulk, algo, parity):
    """One half-sweep of the maximally Abelian gauge against the oracle, every launch
    configuration that has its kernel (0-3; 13 and 14, staged, on FP32-12 links,
    the others falling back to 0): FP64 within 1e-12.  On FP32 link storage every entry is
    within max(5e-6, B), B = 32 u kappa of the site update that wrote its link
    (lattice_np.fp32_half_sweep_bound; kappa from the oracle): the subgroup element
    is the maximiser nearest the identity, whose derivative with respect to v has
    norm kappa_s / 2 (pinned), and v sums 16 terms formed in FP32 (root-sum-square
    rounding ~16u) before the factor a = 2 of overrelaxation or the
    stochastic-relaxation square: c = 2 x 16."""
    U = synth.field(DIMS_RAGGED, 0.5, 62)
    b = getattr(lgt, "LGT_" + bulk.upper())
    ref = U.copy()
    O.half_sweep(ref, parity, gauge=O.MAG, algo=ALGOS[algo], omega=1.7, p=0.8, seed=63)
    kappa = O.site_conditioning(U, parity, gauge=O.MAG, algo=ALGOS[algo], omega=1.7, p=0.8, seed=63)
    bound = fp32_half_sweep_bound(kappa, parity, 32.0)
    for k in (0, 1, 2, 3, 13, 14):
        got = gpu_half(lgt, U, parity, bulk=b, gauge=lgt.LGT_MAG, algo=ALGOS[algo], omega=1.7, p=0.8, seed=63,
                       reunit_every=0, launch_config=k + 1)
        err = np.abs(got - ref)
        if bulk == "fp64":
            assert err.max() < 1e-12, (k, err.max())
        else:
            ratio, n_above, n_links = check_fp32_bound(err, bound)
            assert ratio <= 1.0, (k, ratio, err.max(), n_above, n_links)


def test_mag_sweeps_match_the_oracle(lgt):
    """Ten FP64 sweeps (both parities, fused estimates on) follow the oracle's
    trajectory to 1e-11."""
    U = synth.field(DIMS_RAGGED, 0.5, 64)
    got = gpu_run(lgt, U, 10, gauge=lgt.LGT_MAG, omega=1.7)
    ref = U.copy()
    O.sweeps(ref, 10, gauge=O.MAG, omega=1.7)
    assert np.abs(got - ref).max() < 1e-11


@pytest.mark.parametrize("bulk", ["fp64", "fp32_12"])
def test_mag_fix_matches_oracle(lgt, bulk):
    """lgt_fix in the maximally Abelian gauge: the FP64 path ends where the oracle's
    fix ends (same F_MAG to 1e-10), the mixed ladder (FP32-12 bulk, FP64 polish)
    converges to the same maximum, and both outputs are gauge transforms of the
    input (plaquettes to 1e-12) certified by the oracle."""
    dims = (4, 6, 4, 8)
    U = synth.field(dims, 0.4, 65)
    ref = U.copy()
    r = O.fix(ref, gauge=O.MAG, omega=1.7, tol=1e-13, max_sweeps=20000, check_every=10)
    assert r["converged"]
    p = lgt.lgt_params_default(dims=dims, gauge=lgt.LGT_MAG, bulk=getattr(lgt, "LGT_" + bulk.upper()),
                               omega=1.7, theta_tol=1e-13, max_sweeps=20000)
    ctx = lgt.lgt_create(p, U)
    try:
        st, res = lgt.lgt_fix(ctx)
        V = lgt.lgt_get_links(ctx, dims)
        cfgs = lgt.lgt_get_stats(ctx).launch_config
    finally:
        lgt.lgt_destroy(ctx)
    assert st == lgt.LGT_OK and all(0 <= k <= 3 or k in (13, 14) for k in cfgs)
    m = O.measure(V, O.MAG)
    assert m["theta"] < 1e-13 and abs(m["F"] - res.F) < 1e-12
    assert abs(res.F - r["F"]) < 1e-10, (res.F, r["F"])
    assert np.abs(plaquettes(V) - plaquettes(U)).max() < 1e-12


def test_mag_recovers_a_transformed_abelian_field(lgt):
    """A gauge-transformed Abelian field: the ladder climbs back to F_MAG = 1."""
    dims = (8, 8, 8, 8)
    A, U = _abelian_transformed(dims, 66)
    p = lgt.lgt_params_default(dims=dims, gauge=lgt.LGT_MAG, bulk=lgt.LGT_FP32_12, omega=1.7, theta_tol=1e-14,
                               max_sweeps=20000)
    ctx = lgt.lgt_create(p, U)
    try:
        st, res = lgt.lgt_fix(ctx)
        V = lgt.lgt_get_links(ctx, dims)
    finally:
        lgt.lgt_destroy(ctx)
    assert st == lgt.LGT_OK and abs(res.F - 1) < 1e-12
    assert np.abs(plaquettes(V) - plaquettes(A)).max() < 1e-12


def test_mag_is_not_served_nor_annealed(lgt):
    srv = lgt.lgt_server_create(1 << 30, 0)
    try:
        with pytest.raises(lgt.LgtError) as e:
            lgt.lgt_submit(srv, lgt.lgt_params_default(dims=(4, 4, 4, 4), gauge=lgt.LGT_MAG),
                           synth.field((4, 4, 4, 4), 0.3, 1))
        assert e.value.status == lgt.LGT_EINVAL
    finally:
        lgt.lgt_server_destroy(srv)
    with pytest.raises(lgt.LgtError):
        lgt.lgt_create(lgt.lgt_params_default(dims=(4, 4, 4, 4), gauge=lgt.LGT_MAG, sa_sweeps=3),
                       synth.field((4, 4, 4, 4), 0.3, 1))
