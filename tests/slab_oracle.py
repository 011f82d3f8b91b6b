"""The FP64 oracle as a slab engine of paper_1305_3440_gb300.slab (test
infrastructure): one temporal slab of a lattice, held as the owned slices after
two halo slices (the layout of the library's slab contexts), swept by the
oracle's half-sweep restricted to the owned slices with the random streams
keyed by the global site.  Boundary buffers are CPU tensors (gloo moves them)."""
import numpy as np

import oracle as O


class OracleSlab:
    def __init__(self, U_owned, nt_global, t0, gauge=O.LANDAU, algo=O.OR, omega=1.0, p=0.0, seed=0):
        self.L = U_owned.shape[0]
        self.nt_global, self.t0 = int(nt_global), int(t0)
        self.dims = U_owned.shape[:4]
        self.gauge, self.algo, self.omega, self.p, self.seed = gauge, algo, omega, p, seed
        local = (self.L + 2,) + U_owned.shape[1:4]
        self.U = np.zeros(local + (4, 3, 3), np.complex128)
        self.U[...] = np.eye(3)
        self.U[2:] = U_owned
        self.vs = int(np.prod(U_owned.shape[1:4]))
        self.site_offset = (self.t0 - 2) * self.vs
        self.sweep_index = 0
        x3, x2, x1 = np.indices(U_owned.shape[1:4])
        self.spatial_parity = (x3 + x2 + x1) & 1

    def _mask(self, t_local, parity):
        return self.spatial_parity == ((parity + t_local) & 1)  # t0 even: local and global parity agree

    def boundary_out(self, slice_, parity):
        import torch
        t = slice_ + 2
        data = self.U[t, :, :, :, 0][self._mask(t, parity)]
        return torch.from_numpy(np.ascontiguousarray(data).view(np.float64).ravel().copy())

    def boundary_in(self, slice_, parity, buf):
        t = slice_ + 2
        arr = buf.numpy().view(np.complex128).reshape(-1, 3, 3)
        view = self.U[t, :, :, :, 0]
        view[self._mask(t, parity)] = arr

    def half_sweep(self, parity, first, count):
        active = np.zeros(self.L + 2, np.uint8)
        active[2 + first:2 + first + count] = 1
        O.half_sweep(self.U, parity, gauge=self.gauge, algo=self.algo, omega=self.omega, p=self.p, seed=self.seed,
                     sweep=self.sweep_index, active=active, site_offset=self.site_offset)
        if parity == 1 and first + count == self.L:
            self.sweep_index += 1

    def slice_sums(self):
        """Per owned slice: [sum_mu Re tr U, spatial part, tr Delta^2 (4-D, from the
        oracle's site violation), spatial part, 0]."""
        out = np.zeros((self.L, 5))
        retr = np.real(np.trace(self.U, axis1=-2, axis2=-1))  # (t, x3, x2, x1, mu)
        v4 = O.parity_violation(self.U, 0, O.LANDAU) + O.parity_violation(self.U, 1, O.LANDAU)
        v3 = O.parity_violation(self.U, 0, O.COULOMB) + O.parity_violation(self.U, 1, O.COULOMB)
        out[:, 0] = retr[2:].sum(axis=(1, 2, 3, 4))
        out[:, 1] = retr[2:, ..., 1:].sum(axis=(1, 2, 3, 4))
        out[:, 2] = v4[2:]
        out[:, 3] = v3[2:]
        return out

    def links(self):
        return self.U[2:].copy()

    def sync(self):
        pass
