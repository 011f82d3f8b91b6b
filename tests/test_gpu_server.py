"""The continuous-batching server: every job's result is the same alone and in a
mix (bit for bit: each job's kernels and decisions depend only on its own
parameters), matches the single-context driver, and admission respects the
device-memory budget."""
import time

import numpy as np
import pytest

import oracle as O
from paper_1305_3440_gb300 import synth
from lattice_np import plaquettes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lgt():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1305_3440_gb300 import build
    build.build()
    from paper_1305_3440_gb300 import lgt as mod
    return mod


# (dims, gauge, algo, bulk, tol, eps, seed)
JOBS = [
    ((4, 4, 4, 4), 0, 0, 2, 1e-14, 0.3, 101),
    ((6, 4, 4, 8), 1, 0, 1, 1e-12, 0.5, 102),
    ((8, 8, 8, 8), 0, 0, 0, 1e-14, 0.4, 103),
    ((4, 8, 8, 8), 1, 0, 2, 1e-14, 0.5, 104),
    ((8, 4, 4, 4), 0, 1, 2, 1e-14, 0.3, 105),
    ((8, 8, 8, 8), 0, 0, 2, 1e-12, 0.6, 106),
]


def params_of(lgt, spec):
    dims, gauge, algo, bulk, tol, eps, seed = spec
    return lgt.lgt_params_default(dims=dims, gauge=gauge, algo=algo, bulk=bulk, theta_tol=tol, p=0.8,
                                  seed=seed, max_sweeps=5000)


def wait_all(lgt, srv, ids, dims_of, timeout=300):
    out = {}
    t0 = time.time()
    while len(out) < len(ids):
        assert time.time() - t0 < timeout, "server jobs did not finish"
        for jid in ids:
            if jid in out:
                continue
            links = np.empty(tuple(dims_of[jid]) + (4, 3, 3), np.complex128)
            st, res = lgt.lgt_poll(srv, jid, links)
            if st != lgt.LGT_EAGAIN:
                out[jid] = (st, res.as_dict(), links)
        time.sleep(0.005)
    return out


def run_server(lgt, specs, budget=8 << 30, graphs=True, counters=None):
    import os
    old = os.environ.get("LGT_SERVER_GRAPHS")
    os.environ["LGT_SERVER_GRAPHS"] = "1" if graphs else "0"
    try:
        srv = lgt.lgt_server_create(budget, 0)
    finally:
        if old is None:
            del os.environ["LGT_SERVER_GRAPHS"]
        else:
            os.environ["LGT_SERVER_GRAPHS"] = old
    try:
        ids, dims_of = [], {}
        for spec in specs:
            U = synth.field(spec[0], spec[5], spec[6])
            jid = lgt.lgt_submit(srv, params_of(lgt, spec), U)
            ids.append(jid)
            dims_of[jid] = spec[0]
        res = wait_all(lgt, srv, ids, dims_of)
        done, live, used = lgt.lgt_server_stats(srv)
        assert done == len(specs) and live == 0 and used == 0
        if counters is not None:
            counters.update(lgt.lgt_server_counters(srv))
    finally:
        lgt.lgt_server_destroy(srv)
    return [res[j] for j in ids]


def test_server_results_same_alone_and_in_mix(lgt):
    mix = run_server(lgt, JOBS)
    for spec, (st, res, links) in zip(JOBS, mix):
        assert st == lgt.LGT_OK and res["theta"] < spec[4]
        if spec[3] != 0:  # an FP32 job relaxes in FP32 first: its first exact theta_t are far above theta_switch
            assert res["sweeps_bulk"] > 0, (spec, res)
        st1, res1, links1 = run_server(lgt, [spec])[0]
        assert st1 == st and (spec[3] == 0 or res1["sweeps_bulk"] > 0), (spec, res1)
        assert res1["F"] == res["F"] and res1["theta"] == res["theta"]
        assert res1["sweeps_bulk"] == res["sweeps_bulk"] and res1["sweeps_fp64"] == res["sweeps_fp64"]
        assert np.array_equal(links1, links)


def test_server_graph_replay_changes_nothing(lgt):
    """Ticks replayed from captured CUDA graphs run the same kernels on the same
    tables as directly issued ticks: every job's result and links are bit-identical
    with and without graphs, and with graphs most ticks are replays."""
    cg, cd = {}, {}
    with_g = run_server(lgt, JOBS, counters=cg)
    without = run_server(lgt, JOBS, graphs=False, counters=cd)
    for (s1, r1, l1), (s2, r2, l2) in zip(with_g, without):
        assert s1 == s2 == lgt.LGT_OK
        assert r1["F"] == r2["F"] and r1["theta"] == r2["theta"]
        assert r1["sweeps_bulk"] == r2["sweeps_bulk"] and r1["sweeps_fp64"] == r2["sweeps_fp64"]
        assert np.array_equal(l1, l2)
    # tick counts depend on when the submissions arrive, not on the graphs
    assert cd["graph_launches"] == 0 and cd["graph_captures"] == 0 and cd["ticks"] > 0
    assert 0 < cg["graph_captures"] <= 16 and cg["graph_launches"] > 0, cg
    # one job alone: its launch shape changes only at the start, at promotion and
    # at certification, so all but a few ticks are replays
    one = {}
    (st, res, _), = run_server(lgt, [JOBS[0]], counters=one)
    assert st == lgt.LGT_OK
    assert one["graph_launches"] >= one["ticks"] - 12, one


def test_server_matches_single_context_and_oracle(lgt):
    mix = run_server(lgt, JOBS[:4])
    for spec, (st, res, links) in zip(JOBS[:4], mix):
        dims, gauge, algo, bulk, tol, eps, seed = spec
        U = synth.field(dims, eps, seed)
        ctx = lgt.lgt_create(params_of(lgt, spec), U)
        try:
            st2, r2 = lgt.lgt_fix(ctx)
        finally:
            lgt.lgt_destroy(ctx)
        assert st2 == st == lgt.LGT_OK
        assert abs(r2.F - res["F"]) < 1e-12
        assert r2.sweeps_bulk == res["sweeps_bulk"] and r2.sweeps_fp64 == res["sweeps_fp64"]
        m = O.measure(links, gauge)
        assert m["theta"] < tol
        assert np.abs(plaquettes(links) - plaquettes(U)).max() < 1e-12
        ref = U.copy()
        r = O.fix(ref, gauge=gauge, algo=algo, p=0.8, seed=seed, tol=tol, max_sweeps=5000)
        assert r["converged"] and abs(r["F"] - res["F"]) < 1e-10


def test_server_admission_respects_budget(lgt):
    """A budget that fits one 8^4 FP32 job at a time: jobs run one after another."""
    spec = ((8, 8, 8, 8), 0, 0, 2, 1e-12, 0.3, 200)
    one = 8 * 8 * 8 * 8 * (576 + 192 + 36 + 576) + (1 << 20)
    srv = lgt.lgt_server_create(int(one * 1.2), 0)
    try:
        ids, dims_of = [], {}
        for k in range(4):
            s = spec[:6] + (200 + k,)
            jid = lgt.lgt_submit(srv, params_of(lgt, s), synth.field(s[0], s[5], s[6]))
            ids.append(jid)
            dims_of[jid] = s[0]
        peak_live = 0
        t0 = time.time()
        while True:
            done, live, used = lgt.lgt_server_stats(srv)
            peak_live = max(peak_live, live)
            assert used <= int(one * 1.2)
            if done == 4:
                break
            assert time.time() - t0 < 120
            time.sleep(0.002)
        res = wait_all(lgt, srv, ids, dims_of)
    finally:
        lgt.lgt_server_destroy(srv)
    assert peak_live <= 1
    assert all(st == lgt.LGT_OK for st, _, _ in res.values())


def test_server_errors_and_cancel(lgt):
    srv = lgt.lgt_server_create(256 << 20, 0)
    try:
        big = lgt.lgt_params_default(dims=(32, 32, 32, 32))
        with pytest.raises(lgt.LgtError) as e:
            lgt.lgt_submit(srv, big, np.zeros((32, 32, 32, 32, 4, 3, 3), np.complex128))
        assert e.value.status == lgt.LGT_ENOMEM
        bad = lgt.lgt_params_default(dims=(4, 4, 4, 5))
        with pytest.raises(lgt.LgtError) as e:
            lgt.lgt_submit(srv, bad, np.zeros((4, 4, 4, 5, 4, 3, 3), np.complex128))
        assert e.value.status == lgt.LGT_EINVAL
        with pytest.raises(lgt.LgtError) as e:
            lgt.lgt_poll(srv, 12345)
        assert e.value.status == lgt.LGT_ENOTFOUND
        # non-SU(3) input finishes with EINVAL; a long job is cancelled
        U = synth.field((4, 4, 4, 4), 0.3, 2)
        U[0, 0, 0, 0, 0] *= 2
        j_bad = lgt.lgt_submit(srv, lgt.lgt_params_default(dims=(4, 4, 4, 4)), U)
        # theta cannot reach 1e-300 (FP64 rounding leaves ~1e-32): the job runs until cancelled
        p_long = lgt.lgt_params_default(dims=(16, 16, 16, 16), theta_tol=1e-300, max_sweeps=2**31 - 1, bulk=0)
        j_long = lgt.lgt_submit(srv, p_long, synth.field((16, 16, 16, 16), 0.3, 3))
        time.sleep(0.5)
        lgt.lgt_cancel(srv, j_long)
        res = wait_all(lgt, srv, [j_bad, j_long], {j_bad: (4, 4, 4, 4), j_long: (16, 16, 16, 16)}, timeout=60)
        assert res[j_bad][0] == lgt.LGT_EINVAL
        assert res[j_long][0] == lgt.LGT_ECANCELLED
    finally:
        lgt.lgt_server_destroy(srv)


def test_server_from_several_threads(lgt):
    """Submit, poll and cancel from four host threads at once (the server is
    thread-safe; ctypes releases the GIL around each call): every job ends
    converged or, the one cancelled, LGT_ECANCELLED, and the server is empty."""
    import threading
    srv = lgt.lgt_server_create(8 << 30, 0)
    fields = {k: synth.field((4, 4, 4, 8), 0.4, 300 + k) for k in range(12)}
    results, errors = {}, []

    def worker(w):
        try:
            mine = []
            for k in range(3 * w, 3 * w + 3):
                p = lgt.lgt_params_default(dims=(4, 4, 4, 8), bulk=lgt.LGT_FP32_12, theta_tol=1e-13, max_sweeps=5000)
                mine.append((k, lgt.lgt_submit(srv, p, fields[k])))
            if w == 1:
                lgt.lgt_cancel(srv, mine[0][1])
            t0 = time.time()
            pending = dict(mine)
            while pending and time.time() - t0 < 120:
                for k, jid in list(pending.items()):
                    st, res = lgt.lgt_poll(srv, jid)
                    if st != lgt.LGT_EAGAIN:
                        results[k] = (st, res.theta)
                        del pending[k]
                time.sleep(0.002)
        except Exception as e:  # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(w,)) for w in range(4)]
    try:
        for th in threads:
            th.start()
        for th in threads:
            th.join(180)
        done, live, used = lgt.lgt_server_stats(srv)
    finally:
        lgt.lgt_server_destroy(srv)
    assert not errors, errors
    assert len(results) == 12 and done == 12 and live == 0 and used == 0
    for k, (st, theta) in results.items():
        if k == 3:
            assert st in (lgt.LGT_ECANCELLED, lgt.LGT_OK)
        else:
            assert st == lgt.LGT_OK and theta < 1e-13, (k, st, theta)
