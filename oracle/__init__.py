"""FP64 CPU oracle for relaxation gauge fixing (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package.  The CUDA library neither imports nor links it, and it shares no code
with the library: the C source ``lgt_oracle.c`` restates the paper's Sections 2
and 3 on its own (see its header for every reading of the text it takes).

Every function takes and returns links as complex128 arrays of shape
``(N_t, N_3, N_2, N_1, 4, 3, 3)`` (direction 0 = t, 1..3 = x1..x3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lgt_oracle.c")
_LIB = os.path.join(_HERE, "liblgt_oracle.so")
_lock = threading.Lock()
_lib = None

LANDAU, COULOMB, MAG = 0, 1, 2
OR, SR, SA = 0, 1, 2

_dp = ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
             _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.orc_measure.argtypes = [_i32p, _dp, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
            L.orc_half_sweep.argtypes = [_i32p, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_int, _dp, _dp]
            L.orc_half_sweep_offset.argtypes = [_i32p, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                                ctypes.c_uint64, ctypes.c_int, _dp, ctypes.c_int64]
            L.orc_sweeps.argtypes = [_i32p, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_int, ctypes.c_int, _dp]
            L.orc_site_new_links.argtypes = [_i32p, _dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                             ctypes.c_uint64, ctypes.c_int, _dp]
            L.orc_local_update.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           _dp, _dp, _dp, _dp]
            L.orc_local_update.restype = None
            L.orc_gather_K.argtypes = [_i32p, _dp, ctypes.c_int64, ctypes.c_int, _dp]
            L.orc_su2_maximum.argtypes = [_dp, _dp]
            L.orc_su2_maximum.restype = None
            L.orc_philox4x32_10.argtypes = [_dp, _dp, _dp]
            L.orc_philox4x32_10.restype = None
            L.orc_sr_draws.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, _dp]
            L.orc_sr_draws.restype = None
            L.orc_fix.argtypes = [_i32p, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                  _dp, _dp]
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_sa_sweeps.argtypes = [_i32p, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
            L.orc_kp_draws.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, _dp]
            L.orc_su2_heatbath.argtypes = [_dp, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                           ctypes.c_int, _dp]
            L.orc_su2_heatbath.restype = None
            L.orc_sa_beta.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
            L.orc_sa_beta.restype = ctypes.c_double
            L.orc_mag_subgroup.argtypes = [_dp, ctypes.c_int, _dp, _dp]
            L.orc_mag_subgroup.restype = None
            L.orc_site_conditioning.argtypes = [_i32p, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                                ctypes.c_uint64, _dp]
            L.orc_parity_violation.argtypes = [_i32p, _dp, ctypes.c_int, ctypes.c_int, _dp]
            L.orc_sa_half_sweep.argtypes = [_i32p, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
            L.orc_sa_site_stats.argtypes = [_i32p, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_uint64, ctypes.c_uint64, _dp, _dp]
            L.orc_set_threads.restype = None
            L.orc_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dims_of(links: np.ndarray):
    if links.dtype != np.complex128 or links.ndim != 7 or links.shape[4:] != (4, 3, 3):
        raise ValueError("links must be complex128 of shape (N_t, N_3, N_2, N_1, 4, 3, 3)")
    if not links.flags.c_contiguous:
        raise ValueError("links must be C-contiguous")
    return (ctypes.c_int32 * 4)(*links.shape[:4])


def _check(rc, what):
    if rc < 0:
        raise RuntimeError(f"{what} failed ({rc})")
    return rc


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def measure(links: np.ndarray, gauge: int = LANDAU):
    """Exact F, theta, plaquette (and per-timeslice F_t, theta_t)."""
    d = _dims_of(links)
    nt = links.shape[0]
    F = ctypes.c_double()
    th = ctypes.c_double()
    pl = ctypes.c_double()
    ft = np.zeros(nt)
    tt = np.zeros(nt)
    _check(_load().orc_measure(d, links.ctypes.data, gauge, ctypes.addressof(F), ctypes.addressof(th),
                               ctypes.addressof(pl), ft.ctypes.data, tt.ctypes.data), "orc_measure")
    return dict(F=F.value, theta=th.value, plaq=pl.value, F_t=ft, theta_t=tt)


def half_sweep(links, parity, gauge=LANDAU, algo=OR, omega=1.0, p=0.0, seed=0, sweep=0,
               transform_temporal=1, active=None, order=None, site_offset=0):
    """In-place half-sweep over one parity.  site_offset: the links are a slab of a
    larger lattice and the random streams are keyed by site + site_offset."""
    d = _dims_of(links)
    act = None
    if active is not None:
        act = np.ascontiguousarray(active, dtype=np.uint8)
    if site_offset:
        assert order is None
        _check(_load().orc_half_sweep_offset(d, links.ctypes.data, gauge, parity, algo, omega, p, seed, sweep,
                                             transform_temporal, None if act is None else act.ctypes.data,
                                             int(site_offset)), "orc_half_sweep_offset")
        return links
    od = None
    if order is not None:
        od = np.ascontiguousarray(order, dtype=np.int64)
        assert od.size == links[..., 0, 0, 0].size // 2
    _check(_load().orc_half_sweep(d, links.ctypes.data, gauge, parity, algo, omega, p, seed, sweep,
                                  transform_temporal, None if act is None else act.ctypes.data,
                                  None if od is None else od.ctypes.data), "orc_half_sweep")
    return links


def sweeps(links, n, gauge=LANDAU, algo=OR, omega=1.0, p=0.0, seed=0, sweep0=0,
           transform_temporal=1, active=None):
    """In-place n full sweeps (even half, then odd half)."""
    d = _dims_of(links)
    act = None
    if active is not None:
        act = np.ascontiguousarray(active, dtype=np.uint8)
    _check(_load().orc_sweeps(d, links.ctypes.data, gauge, algo, omega, p, seed, sweep0, n,
                              transform_temporal, None if act is None else act.ctypes.data),
           "orc_sweeps")
    return links


def site_new_links(links, site, gauge=LANDAU, algo=OR, omega=1.0, p=0.0, seed=0, sweep=0,
                   transform_temporal=1):
    """(fwd[4,3,3], bwd[4,3,3]) that one site update would write."""
    d = _dims_of(links)
    out = np.empty((8, 3, 3), dtype=np.complex128)
    _check(_load().orc_site_new_links(d, links.ctypes.data, int(site), gauge, algo, omega, p, seed,
                                      sweep, transform_temporal, out.ctypes.data), "orc_site_new_links")
    return out[:4], out[4:]


def local_update(K: np.ndarray, algo=OR, omega=1.0, p=0.0, draws=(0, 0, 0)):
    """g, W[3], R[3] of one Cabibbo-Marinari update of K (3x3 complex)."""
    K = np.ascontiguousarray(K, dtype=np.complex128)
    g = np.empty((3, 3), np.complex128)
    W = np.empty((3, 3, 3), np.complex128)
    R = np.empty((3, 3, 3), np.complex128)
    dr = np.ascontiguousarray(draws, dtype=np.uint32)
    _load().orc_local_update(K.ctypes.data, algo, omega, p, dr.ctypes.data, g.ctypes.data,
                             W.ctypes.data, R.ctypes.data)
    return g, W, R


def site_conditioning(links, parity, gauge=LANDAU, algo=OR, omega=1.0, p=0.0, seed=0, sweep=0):
    """Per-site conditioning of the site updates of one parity on these links
    (test infrastructure for the FP32 parity bounds; see the C source): an array
    of shape (N_t, N_3, N_2, N_1), NaN at the sites of the other parity."""
    d = _dims_of(links)
    out = np.full(links.shape[:4], np.nan)
    _check(_load().orc_site_conditioning(d, links.ctypes.data, gauge, parity, algo, omega, p, seed, sweep,
                                         out.ctypes.data), "orc_site_conditioning")
    return out


def parity_violation(links, parity, gauge=LANDAU):
    """Per timeslice, the sum of tr[Delta Delta^dagger] (Sec. 2) over the sites of
    one parity (test infrastructure for the fused estimate).  Shape (N_t,)."""
    d = _dims_of(links)
    out = np.zeros(links.shape[0])
    _check(_load().orc_parity_violation(d, links.ctypes.data, gauge, parity, out.ctypes.data),
           "orc_parity_violation")
    return out


def gather_K(links, site, gauge=LANDAU):
    d = _dims_of(links)
    K = np.empty((3, 3), np.complex128)
    _check(_load().orc_gather_K(d, links.ctypes.data, int(site), gauge, K.ctypes.data), "orc_gather_K")
    return K


def su2_maximum(M: np.ndarray):
    M = np.ascontiguousarray(M, dtype=np.complex128)
    r = np.empty(4)
    _load().orc_su2_maximum(M.ctypes.data, r.ctypes.data)
    return r


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.empty(4, np.uint32)
    _load().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, o.ctypes.data)
    return tuple(int(v) for v in o)


def sr_draws(seed, sweep, site):
    o = np.empty(3, np.uint32)
    _load().orc_sr_draws(seed, sweep, site, o.ctypes.data)
    return o


def fix(links, gauge=LANDAU, algo=OR, omega=1.7, p=0.0, seed=0, tol=1e-14, max_sweeps=1000,
        check_every=10, transform_temporal=1):
    """In-place gauge fixing to theta < tol.  Returns dict(converged, sweeps, F, theta)."""
    d = _dims_of(links)
    sw = ctypes.c_int()
    F = ctypes.c_double()
    th = ctypes.c_double()
    rc = _check(_load().orc_fix(d, links.ctypes.data, gauge, algo, omega, p, seed, tol, max_sweeps,
                                check_every, transform_temporal, ctypes.byref(sw), ctypes.addressof(F),
                                ctypes.addressof(th)), "orc_fix")
    return dict(converged=(rc == 0), sweeps=sw.value, F=F.value, theta=th.value)


def sa_sweeps(links, n, beta0, beta1, gauge=LANDAU, seed=0, sweep0=0, transform_temporal=1):
    """n simulated-annealing (SU(2) heat-bath) sweeps in place, beta rising
    geometrically from beta0 to beta1 (see the C source for the reading)."""
    L = _load()
    d = _dims_of(links)
    _check(L.orc_sa_sweeps(d, links.ctypes.data, gauge, float(beta0), float(beta1), int(n), seed, sweep0,
                           transform_temporal), "orc_sa_sweeps")
    return links


def sa_half_sweep(links, parity, beta, gauge=LANDAU, seed=0, sweep=0, transform_temporal=1):
    """One simulated-annealing half-sweep in place (the heat-bath steps of sa_sweeps)."""
    d = _dims_of(links)
    _check(_load().orc_sa_half_sweep(d, links.ctypes.data, gauge, parity, float(beta), seed, sweep,
                                     transform_temporal), "orc_sa_half_sweep")
    return links


def sa_site_stats(links, parity, beta, gauge=LANDAU, seed=0, sweep=0):
    """(kappa, margin) per site of one parity for the annealing update (test
    infrastructure; see the C source); NaN at the other parity."""
    d = _dims_of(links)
    kap = np.full(links.shape[:4], np.nan)
    mar = np.full(links.shape[:4], np.nan)
    _check(_load().orc_sa_site_stats(d, links.ctypes.data, gauge, parity, float(beta), seed, sweep,
                                     kap.ctypes.data, mar.ctypes.data), "orc_sa_site_stats")
    return kap, mar


def kp_draws(alpha, n, seed=0):
    """(draws, failures): n Kennedy-Pendleton draws of x with density
    ~ sqrt(1 - x^2) exp(alpha x) on [-1, 1] (NaN where every attempt failed)."""
    L = _load()
    out = np.empty(int(n), np.float64)
    fails = L.orc_kp_draws(float(alpha), int(n), seed, out.ctypes.data)
    return out, fails


def su2_heatbath(q, beta, seed=0, sweep=0, site=0, subgroup=0):
    """The heat-bath SU(2) element (quaternion) for a block projection q."""
    L = _load()
    qq = np.ascontiguousarray(q, np.float64)
    r = np.empty(4, np.float64)
    L.orc_su2_heatbath(qq.ctypes.data, float(beta), seed, sweep, site, subgroup, r.ctypes.data)
    return r


def sa_beta(beta0, beta1, n, i):
    """beta of annealing sweep i of n (geometric from beta0 to beta1)."""
    return _load().orc_sa_beta(float(beta0), float(beta1), int(n), int(i))


def mag_subgroup(links8: np.ndarray, s: int):
    """Maximally Abelian gauge, subgroup s of one site update on the site's 8 links
    (4 forward then 4 backward, complex 3x3): (v, r), r the maximising element."""
    L8 = np.ascontiguousarray(links8, dtype=np.complex128).reshape(8, 3, 3)
    v, r = np.zeros(3), np.zeros(4)
    _load().orc_mag_subgroup(L8.ctypes.data, int(s), v.ctypes.data, r.ctypes.data)
    return v, r
