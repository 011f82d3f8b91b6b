"""Temporal slab decomposition across devices (Sec. 5 of Schroeck & Vogt).

The lattice is cut along t into slabs of L slices, slab r holding the global
slices r L .. r L + L - 1 (L even).  A site of the first owned slice t_min has
its backward temporal link U_0(t_min - 1) on the slab before it, so every
half-sweep of parity p moves U_0 of the inactive parity q = 1 - p across each
cut, in the order of the paper's list:

  1-3  U_0(t_max, q) of slab r goes to slab r + 1, where it lands in the halo
       as U_0(t_min - 1, q);
  4    slab r + 1 updates its first slice, which changes U_0(t_min - 1, q);
  5-7  U_0(t_min - 1, q) goes back to slab r, into U_0(t_max, q), overlapped
       with the update of the interior slices.

Slab r's own half-sweep never touches U_0(t_max, q) (its parity-p sites there
write U_0(t_max, p)), and the links are back before its next half-sweep, whose
parity-q sites at t_max update them.  Sites of one parity touch disjoint links
and the random streams are keyed by the global site, so a decomposed sweep
reproduces the whole lattice's sweep bit for bit.

Engines hold one slab: `GpuSlab` (a liblgt slab context, lgt_slab_*).  Rings
move the boundary links: `LocalRing` for all slabs in one process (one device,
one stream; the links move by device copies), `DistRing` for one slab per
process over torch.distributed (NCCL between GPUs; gloo moves CPU tensors).
`SlabDriver` runs the protocol, the sweeps' fused estimate and the exact
measurement over every slab of the ring.
"""
from __future__ import annotations

import numpy as np

HALO = -1  # the owned-slice index of the halo slice (U_0(t_min - 1))


class GpuSlab:
    """One slab as a liblgt slab context on the current CUDA device.

    params: lgt_params of the whole lattice (dims = the global dims); the slab
    owns global slices t0 .. t0 + L - 1 of `links`, which holds those slices in
    the public layout (numpy host array or torch CUDA tensor).  `stream` is the
    torch stream every operation of the slab runs on (the ring's collectives are
    enqueued on it too)."""

    def __init__(self, params, t0: int, L: int, links, stream):
        import ctypes

        import torch
        from . import lgt
        self.lgt = lgt
        self.torch = torch
        self.stream = stream
        self.t0, self.L = int(t0), int(L)
        self.nt_global = int(params.dims[0])
        self.dims = (self.L,) + tuple(int(d) for d in params.dims[1:])
        p = lgt.lgt_params()
        ctypes.pointer(p)[0] = params
        p.dims[0] = self.L
        self.gauge = int(p.gauge)
        self.ctx = lgt.lgt_slab_create(p, self.nt_global, self.t0, links, stream=stream)
        self.nbytes = lgt.lgt_slab_boundary_bytes(self.ctx)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def boundary_out(self, slice_: int, parity: int):
        with self.torch.cuda.stream(self.stream):
            buf = self.torch.empty(self.nbytes, dtype=self.torch.uint8, device=self.device)
        self.lgt.lgt_slab_boundary(self.ctx, slice_, parity, buf, False)
        return buf

    def boundary_in(self, slice_: int, parity: int, buf) -> None:
        self.lgt.lgt_slab_boundary(self.ctx, slice_, parity, buf, True)

    def half_sweep(self, parity: int, first: int, count: int) -> None:
        self.lgt.lgt_slab_half_sweep(self.ctx, parity, first, count)

    def slice_sums(self) -> np.ndarray:
        """Exact per-slice sums of the owned slices (lgt_measure_slice_sums), (L, 5)."""
        return self.lgt.lgt_measure_slice_sums(self.ctx, self.L)

    def estimate_slices(self):
        """(F_t, theta_t) of the sweeps' fused estimate on the owned slices (the
        Landau or Coulomb normalisation per slice)."""
        _, _, F_t, th_t = self.lgt.lgt_estimate(self.ctx, self.L)
        return F_t, th_t

    def links(self) -> np.ndarray:
        return self.lgt.lgt_get_working_links(self.ctx, self.dims)

    def sync(self) -> None:
        self.lgt.lgt_slab_sync(self.ctx)

    def close(self) -> None:
        if self.ctx:
            self.lgt.lgt_destroy(self.ctx)
            self.ctx = None


class _Done:
    def __init__(self, bufs):
        self.bufs = bufs

    def wait(self):
        return self.bufs


class LocalRing:
    """Every slab in this process (ranks 0 .. n-1 of the ring); the boundary
    buffers are handed on directly (the engines share one stream, so the
    copies into and out of them are ordered).  Nothing runs concurrently on one
    stream, so the driver does not split the half-sweep for overlap."""

    overlap = False

    def __init__(self, n: int):
        self.n = int(n)

    def shift_start(self, bufs, step: int):
        """Each slab r sends bufs[r] to r + step and receives from r - step."""
        n = self.n
        return _Done([bufs[(r - step) % n] for r in range(n)])

    def allreduce(self, values: np.ndarray, op: str) -> np.ndarray:
        """values: (local slabs, ...) -> the reduction over all slabs."""
        return values.sum(axis=0) if op == "sum" else values.max(axis=0)


class _DistPending:
    def __init__(self, reqs, recv):
        self.reqs, self.recv = reqs, recv

    def wait(self):
        for r in self.reqs:
            r.wait()
        return [self.recv]


class DistRing:
    """One slab per process of a torch.distributed group (NCCL for CUDA
    tensors, gloo for CPU tensors); the ring follows the ranks."""

    overlap = True

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.n = dist.get_world_size(group)

    def shift_start(self, bufs, step: int):
        import torch
        (buf,) = bufs
        if self.n == 1:
            return _Done([buf])
        recv = torch.empty_like(buf)
        dst = (self.rank + step) % self.n
        src = (self.rank - step) % self.n
        reqs = [self.dist.isend(buf, dst, group=self.group), self.dist.irecv(recv, src, group=self.group)]
        return _DistPending(reqs, recv)

    def allreduce(self, values: np.ndarray, op: str) -> np.ndarray:
        import torch
        t = torch.from_numpy(np.ascontiguousarray(values[0], dtype=np.float64))
        if self.dist.get_backend(self.group) == "nccl":
            t = t.cuda()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM if op == "sum" else self.dist.ReduceOp.MAX,
                             group=self.group)
        return t.cpu().numpy()


class SlabDriver:
    """Sweeps, estimates and measurements of a lattice cut into temporal slabs.

    engines: the slabs this process holds (all of them for a LocalRing, one for
    a DistRing), each with owned slices t0 .. t0 + L - 1, in ring order."""

    def __init__(self, engines, ring):
        self.engines = list(engines)
        self.ring = ring
        e0 = self.engines[0]
        self.L = e0.L
        self.nt_global = e0.nt_global
        self.gauge = e0.gauge

    # ---------------------------------------------------------- Sec. 5 steps
    def half_sweep(self, parity: int) -> None:
        q = 1 - parity
        E = self.engines
        # 1-3: U_0(t_max) of the inactive parity to the next slab's halo
        got = self.ring.shift_start([e.boundary_out(e.L - 1, q) for e in E], +1).wait()
        for e, b in zip(E, got):
            e.boundary_in(HALO, q, b)
        if not self.ring.overlap:  # 4 with the interior in one launch, then 5-7
            for e in E:
                e.half_sweep(parity, 0, e.L)
            got = self.ring.shift_start([e.boundary_out(HALO, q) for e in E], -1).wait()
            for e, b in zip(E, got):
                e.boundary_in(e.L - 1, q, b)
            return
        # 4: the first slice, whose update changes U_0(t_min - 1)
        for e in E:
            e.half_sweep(parity, 0, 1)
        # 5-7: U_0(t_min - 1) back to its owner, in flight while the interior is updated
        pending = self.ring.shift_start([e.boundary_out(HALO, q) for e in E], -1)
        for e in E:
            if e.L > 1:
                e.half_sweep(parity, 1, e.L - 1)
        for e, b in zip(E, pending.wait()):
            e.boundary_in(e.L - 1, q, b)

    def sweep(self, n: int = 1) -> None:
        for _ in range(int(n)):
            self.half_sweep(0)
            self.half_sweep(1)

    def refresh_halo(self) -> None:
        """Both parities of U_0(t_min - 1) from the slab before (the exact
        measurement's violation at t_min needs them)."""
        for q in (0, 1):
            got = self.ring.shift_start([e.boundary_out(e.L - 1, q) for e in self.engines], +1).wait()
            for e, b in zip(self.engines, got):
                e.boundary_in(HALO, q, b)

    # ------------------------------------------------------- measurements
    def measure(self) -> dict:
        """Exact F and theta of the whole lattice (Sec. 2) from every slab's
        per-slice sums: Landau over all slices, Coulomb per slice (F = mean F_t,
        theta = max theta_t)."""
        self.refresh_halo()
        sums = np.stack([e.slice_sums() for e in self.engines])  # (local, L, 5)
        tot = self.ring.allreduce(sums.sum(axis=1)[:, None, :], "sum")[0]
        vs = None
        for e in self.engines:
            vs = int(np.prod(e.dims[1:]))
        V = vs * self.nt_global
        out = {"F_landau": tot[0] / (12.0 * V), "theta_landau": tot[2] / (3.0 * V)}
        Ft = sums[..., 1] / (9.0 * vs)
        tht = sums[..., 3] / (3.0 * vs)
        out["F_coulomb"] = float(self.ring.allreduce(Ft.sum(axis=1)[:, None], "sum")[0]) / self.nt_global
        out["theta_coulomb"] = float(self.ring.allreduce(tht.max(axis=1)[:, None], "max")[0])
        coulomb = self.gauge == 1
        out["F"] = out["F_coulomb"] if coulomb else out["F_landau"]
        out["theta"] = out["theta_coulomb"] if coulomb else out["theta_landau"]
        return out

    def estimate(self) -> tuple:
        """(F, theta) of the sweeps' fused estimate of the last sweep, over the
        whole lattice (a check of the Sec. 4 driver)."""
        rows = [e.estimate_slices() for e in self.engines]
        F_t = np.stack([r[0] for r in rows])
        th_t = np.stack([r[1] for r in rows])
        F = float(self.ring.allreduce(F_t.sum(axis=1)[:, None], "sum")[0]) / self.nt_global
        if self.gauge == 1:
            theta = float(self.ring.allreduce(th_t.max(axis=1)[:, None], "max")[0])
        else:
            theta = float(self.ring.allreduce(th_t.sum(axis=1)[:, None], "sum")[0]) / self.nt_global
        return F, theta

    def fix(self, tol: float = 1e-14, max_sweeps: int = 10000, check_every: int = 10) -> dict:
        """Sweeps until the exact theta is below tol (Sec. 4 driver over the
        slabs): a check every check_every sweeps on the fused estimate, the
        exact measurement to certify."""
        done = 0
        while done < max_sweeps:
            n = min(check_every, max_sweeps - done)
            self.sweep(n)
            done += n
            _, theta = self.estimate()
            if theta < tol:
                m = self.measure()
                if m["theta"] < tol:
                    return dict(m, sweeps=done, converged=True)
        m = self.measure()
        return dict(m, sweeps=done, converged=bool(m["theta"] < tol))
