"""The temporal slab decomposition (Sec. 5) driven by the package's slab driver
over the FP64 oracle, on CPU: several slabs in one process, and one slab per
gloo rank (world size 2 and 4).  Sweeping the slabs with the paper's boundary
protocol reproduces the whole lattice's oracle sweeps bit for bit (sites of one
parity are independent and the random streams follow the global site), and the
exact F and theta gathered over the slabs equal the oracle's measurement."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1305_3440_gb300 import synth
from paper_1305_3440_gb300.slab import LocalRing, SlabDriver

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS = (8, 4, 4, 6)


def _engines(U, n, **kw):
    from slab_oracle import OracleSlab
    L = U.shape[0] // n
    return [OracleSlab(U[r * L:(r + 1) * L].copy(), U.shape[0], r * L, **kw) for r in range(n)]


@pytest.mark.parametrize("n", [1, 2, 4])
@pytest.mark.parametrize("gauge,algo", [(O.LANDAU, O.OR), (O.LANDAU, O.SR), (O.COULOMB, O.OR)])
def test_slabs_in_one_process_reproduce_the_whole_lattice(n, gauge, algo):
    pytest.importorskip("torch")
    U = synth.field(DIMS, 0.5, 41)
    kw = dict(gauge=gauge, algo=algo, omega=1.7, p=0.8, seed=5)
    drv = SlabDriver(_engines(U, n, **kw), LocalRing(n))
    drv.sweep(3)
    got = np.concatenate([e.links() for e in drv.engines])
    ref = U.copy()
    O.sweeps(ref, 3, **kw)
    assert np.array_equal(got, ref)
    m, r = drv.measure(), O.measure(ref, gauge)
    assert abs(m["F"] - r["F"]) < 1e-14 and abs(m["theta"] - r["theta"]) < 1e-13 * r["theta"]


def test_boundary_links_cross_the_cut():
    """With the return transfer left out, the slabs' result differs: the protocol
    is what carries the boundary updates."""
    pytest.importorskip("torch")
    U = synth.field(DIMS, 0.5, 42)

    class OneWay(SlabDriver):
        def half_sweep(self, parity):
            q = 1 - parity
            got = self.ring.shift_start([e.boundary_out(e.L - 1, q) for e in self.engines], +1).wait()
            for e, b in zip(self.engines, got):
                e.boundary_in(-1, q, b)
            for e in self.engines:
                e.half_sweep(parity, 0, e.L)

    drv = OneWay(_engines(U, 2, omega=1.7), LocalRing(2))
    drv.sweep(1)
    got = np.concatenate([e.links() for e in drv.engines])
    ref = U.copy()
    O.sweeps(ref, 1, omega=1.7)
    assert not np.array_equal(got, ref)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, algo, out):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as Or
        from paper_1305_3440_gb300 import synth as sy
        from paper_1305_3440_gb300.slab import DistRing, SlabDriver as Drv
        from slab_oracle import OracleSlab
        U = sy.field(DIMS, 0.5, 43)
        L = DIMS[0] // world
        kw = dict(gauge=Or.LANDAU, algo=algo, omega=1.7, p=0.8, seed=6)
        eng = OracleSlab(U[rank * L:(rank + 1) * L].copy(), DIMS[0], rank * L, **kw)
        drv = Drv([eng], DistRing())
        drv.sweep(3)
        m = drv.measure()
        out.put((rank, eng.links(), m["F"], m["theta"]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("algo", [O.OR, O.SR])
def test_slabs_on_gloo_ranks_reproduce_the_whole_lattice(world, algo):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, algo, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    U = synth.field(DIMS, 0.5, 43)
    ref = U.copy()
    O.sweeps(ref, 3, gauge=O.LANDAU, algo=algo, omega=1.7, p=0.8, seed=6)
    got = np.concatenate([r[1] for r in res])
    assert np.array_equal(got, ref)
    m = O.measure(ref)
    for _, _, F, th in res:
        assert abs(F - m["F"]) < 1e-14 and abs(th - m["theta"]) < 1e-13 * m["theta"]
