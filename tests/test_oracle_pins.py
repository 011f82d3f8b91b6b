"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an invariant, a special case that reduces to the paper's SU(2) formula,
brute force on small inputs, or published known-answer vectors.  The test-side
arithmetic lives in ``lattice_np`` (numpy), independent of the oracle's C code.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1305_3440_gb300 import synth
from lattice_np import (GELL_MANN, coords_of, dag, expm_herm, parity_of, plaquettes,
                        random_su3, su2_grid, su2_matrices, su2_quaternion_matrix,
                        transform_field, transform_global, transform_site, unitarity_error)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def unit_field(dims):
    U = np.zeros(tuple(dims) + (4, 3, 3), np.complex128)
    U[..., :, :, :] = np.eye(3)
    return U


# ------------------------------------------------------------------ RNG
def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(w, 16) for w in line.split()]
            rows.append((v[0:4], v[4:6], tuple(v[6:10])))
    return rows


@pytest.mark.parametrize("row", _kat_rows())
def test_philox_known_answers(row):
    """Salmon et al. (SC'11) known-answer vectors, for the oracle's and the
    generator's separate Philox4x32-10 implementations."""
    ctr, key, expect = row
    assert O.philox(ctr, key) == expect
    assert synth.philox(ctr, key) == expect


def test_sr_draws_are_philox_words():
    """The stochastic-relaxation stream is word s of the Philox block counted
    by (site, sweep, tag) under the seed (the reading of Sec. 3.2)."""
    seed, sweep, site = 0x123456789ABCDEF0, 17, 4242
    blk = O.philox([site, 0, sweep, 0x53524C58], [seed & 0xFFFFFFFF, seed >> 32])
    assert tuple(O.sr_draws(seed, sweep, site)) == blk[:3]


# ------------------------------------------------- Sec. 2: F and theta
def test_unit_field_F_is_one_theta_zero():
    """Unit links: tr 1 = N_c on all N_d V links gives F = 1; Delta = 0 gives theta = 0."""
    for dims in [(2, 2, 2, 2), (4, 2, 6, 4)]:
        U = unit_field(dims)
        m = O.measure(U)
        assert m["F"] == 1.0 and m["theta"] == 0.0 and m["plaq"] == 1.0
        mc = O.measure(U, O.COULOMB)
        assert mc["F"] == 1.0 and mc["theta"] == 0.0
        assert np.all(mc["F_t"] == 1.0) and np.all(mc["theta_t"] == 0.0)


def test_constant_diagonal_field_closed_form():
    """Constant links diag(e^{ia}, e^{ib}, e^{-i(a+b)}): F = (cos a + cos b + cos(a+b))/3,
    and Delta = sum_mu (A - A) = 0 so theta = 0."""
    a, b = 0.37, -1.21
    U = unit_field((4, 4, 4, 4))
    U[...] = np.diag([np.exp(1j * a), np.exp(1j * b), np.exp(-1j * (a + b))])
    m = O.measure(U)
    assert abs(m["F"] - (np.cos(a) + np.cos(b) + np.cos(a + b)) / 3) < 1e-13
    assert m["theta"] < 1e-30


def test_single_link_theta_closed_form():
    """One non-trivial link exp(i a lambda_3/2) on a unit field: A = diag(s, -s, 0) with
    s = sin(a/2); Delta = +A at x and -A at x+mu, so theta = 2 * 2 s^2 / (3 V)."""
    dims = (4, 4, 4, 4)
    V = 256
    a = 0.8
    for mu in range(4):
        U = unit_field(dims)
        U[1, 2, 3, 0, mu] = np.diag([np.exp(0.5j * a), np.exp(-0.5j * a), 1.0])
        m = O.measure(U)
        s = np.sin(a / 2)
        assert abs(m["theta"] - 4 * s * s / (3 * V)) < 1e-16
        assert abs(m["F"] - 1 + (2 - 2 * np.cos(a / 2)) / (12 * V)) < 1e-15


def test_global_gauge_invariance_of_F_theta():
    """A constant g leaves F, theta and every plaquette unchanged."""
    U = synth.field((4, 4, 4, 4), 0.5, 11)
    g = random_su3(np.random.default_rng(3))
    m0 = O.measure(U)
    m1 = O.measure(np.ascontiguousarray(transform_global(U, g)))
    assert abs(m0["F"] - m1["F"]) < 1e-14
    assert abs(m0["theta"] - m1["theta"]) < 1e-14 * max(1.0, m0["theta"])
    assert abs(m0["plaq"] - m1["plaq"]) < 1e-14


def _theta_from_gradient(U, gauge):
    """theta rebuilt from central differences of F under g = exp(i e lambda_a/2) at
    each site: dF/de_a = -tr(T_a Delta(x))/(N_c N_d V), and tr Delta^2 = 2 sum_a c_a^2."""
    dims = U.shape[:4]
    nd = 3 if gauge == O.COULOMB else 4
    nt = dims[0]
    vs = dims[1] * dims[2] * dims[3]
    eps = 1e-4
    theta_t = np.zeros(nt)
    for site in range(U[..., 0, 0, 0].size):
        c = coords_of(site, dims)
        grad = np.zeros(8)
        for a in range(8):
            gp = expm_herm(eps * GELL_MANN[a] / 2)
            Fp = O.measure(np.ascontiguousarray(transform_site(U, c, gp)), gauge)
            Fm = O.measure(np.ascontiguousarray(transform_site(U, c, dag(gp))), gauge)
            if gauge == O.COULOMB:
                d = (Fp["F_t"][c[0]] - Fm["F_t"][c[0]]) / (2 * eps)
                grad[a] = d * (3 * nd * vs)
            else:
                d = (Fp["F"] - Fm["F"]) / (2 * eps)
                grad[a] = d * (3 * nd * vs * nt)
        theta_t[c[0]] += 2 * np.sum(grad ** 2)
    return theta_t / (3 * vs)


def test_theta_is_the_gradient_of_F_landau():
    """Sec. 2: theta = 0 iff F is stationary.  Quantitatively theta equals the squared
    gauge gradient of F (with A_mu the traceless part of (U - U^dagger)/(2i))."""
    U = synth.field((2, 4, 2, 4), 0.6, 5)
    m = O.measure(U)
    th = _theta_from_gradient(U, O.LANDAU).sum() / U.shape[0]
    assert abs(th - m["theta"]) < 1e-7 * m["theta"]


def test_theta_is_the_gradient_of_F_coulomb():
    """Per timeslice: theta_t is the squared spatial gauge gradient of F_t."""
    U = synth.field((4, 2, 4, 2), 0.6, 6)
    m = O.measure(U, O.COULOMB)
    th_t = _theta_from_gradient(U, O.COULOMB)
    assert np.allclose(th_t, m["theta_t"], rtol=1e-7, atol=0)
    assert m["theta"] == m["theta_t"].max()
    assert abs(m["F"] - m["F_t"].mean()) < 1e-15


def test_coulomb_ignores_temporal_links():
    """Coulomb functional per slice uses spatial links only: unit spatial links with
    arbitrary temporal links give F_t = 1, theta_t = 0."""
    U = synth.field((4, 4, 4, 4), 0.5, 8)
    U[..., 1:, :, :] = np.eye(3)
    m = O.measure(U, O.COULOMB)
    assert np.all(np.abs(m["F_t"] - 1) < 1e-15) and m["theta"] < 1e-30


# --------------------------------------------------------- Sec. 3: K(x)
def test_K_gives_the_local_functional():
    """For any g at site x: F(g at x) - F(1) = (Re tr[g K(x)] - Re tr K(x)) / (N_c N_d V).
    Pins which links enter K(x) and in which form (U or U^dagger)."""
    rng = np.random.default_rng(7)
    dims = (4, 4, 4, 4)
    V = 256
    U = synth.field(dims, 0.7, 9)
    F0 = O.measure(U)["F"]
    for site in [0, 1, 77, 200, 255]:
        K = O.gather_K(U, site)
        c = coords_of(site, dims)
        for _ in range(3):
            g = random_su3(rng)
            F1 = O.measure(np.ascontiguousarray(transform_site(U, c, g)))["F"]
            lhs = F1 - F0
            rhs = (np.real(np.trace(g @ K)) - np.real(np.trace(K))) / (12 * V)
            assert abs(lhs - rhs) < 1e-14


def test_K_coulomb_spatial_only():
    rng = np.random.default_rng(8)
    dims = (4, 4, 4, 4)
    U = synth.field(dims, 0.7, 10)
    site = 123
    c = coords_of(site, dims)
    F0 = O.measure(U, O.COULOMB)["F_t"][c[0]]
    K = O.gather_K(U, site, O.COULOMB)
    g = random_su3(rng)
    V2 = np.ascontiguousarray(transform_site(U, c, g))
    F1 = O.measure(V2, O.COULOMB)["F_t"][c[0]]
    assert abs((F1 - F0) - (np.real(np.trace(g @ K)) - np.real(np.trace(K))) / (9 * 64)) < 1e-14


def test_parity_sums_of_K_give_F():
    """Every link joins one even and one odd site: sum over one parity of Re tr K = N_c N_d V F."""
    dims = (4, 2, 4, 2)
    U = synth.field(dims, 0.5, 12)
    F = O.measure(U)["F"]
    for p in (0, 1):
        s = sum(np.real(np.trace(O.gather_K(U, x))) for x in range(64) if parity_of(x, dims) == p)
        assert abs(s / (12 * 64) - F) < 1e-14


# ------------------------------------------ Sec. 3: SU(2) closed form
def test_su2_formula_of_the_paper_on_su2_blocks():
    """For a block M = c S (S in SU(2), c > 0) the result is g = M^dagger / sqrt(det M^dagger)."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        M = 2.7 * su2_quaternion_matrix(q)
        r = O.su2_maximum(M)
        g = su2_quaternion_matrix(r)
        Md = dag(M)
        expect = Md / np.sqrt(np.linalg.det(Md))
        assert np.abs(g - expect).max() < 1e-14


def test_su2_closed_form_beats_brute_force():
    """For general complex 2x2 blocks: Re tr(r M) at the closed form is 2|q| and is not
    below any point of a dense SU(2) sample (random + Hopf grid)."""
    rng = np.random.default_rng(2)
    grid = su2_matrices(su2_grid(20000, rng))
    for _ in range(40):
        M = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
        r = O.su2_maximum(M)
        assert abs(np.linalg.norm(r) - 1) < 1e-15
        best = np.real(np.trace(su2_quaternion_matrix(r) @ M))
        brute = np.real(np.einsum("nij,ji->n", grid, M)).max()
        q = np.array([np.real(M[0, 0] + M[1, 1]), np.imag(M[0, 1] + M[1, 0]),
                      np.real(M[0, 1] - M[1, 0]), np.imag(M[0, 0] - M[1, 1])]) / 2
        assert abs(best - 2 * np.linalg.norm(q)) < 1e-13
        assert best >= brute - 1e-12
        assert brute > best - 0.05  # the sample is dense enough to be a real check


def test_su2_degenerate_block_keeps_identity():
    r = O.su2_maximum(np.zeros((2, 2), np.complex128))
    assert tuple(r) == (1.0, 0.0, 0.0, 0.0)


SUBGROUPS = [(0, 1), (0, 2), (1, 2)]


def _check_cm_steps(K, g, W, R, grid):
    """W[0] = K, W[s+1] = R[s] W[s], g = R[2] R[1] R[0]; R[s] is an SU(2) embedding in
    subgroup s that maximises Re tr(R W[s]) over that subgroup (brute force)."""
    assert np.abs(W[0] - K).max() < 1e-15
    for s in range(3):
        i, j = SUBGROUPS[s]
        k = 3 - i - j
        Rs = R[s]
        assert abs(Rs[k, k] - 1) < 1e-15 and np.abs(Rs[k, [i, j]]).max() == 0 and np.abs(Rs[[i, j], k]).max() == 0
        blk = Rs[np.ix_([i, j], [i, j])]
        assert np.abs(dag(blk) @ blk - np.eye(2)).max() < 1e-14 and abs(np.linalg.det(blk) - 1) < 1e-14
        if s < 2:
            assert np.abs(W[s + 1] - Rs @ W[s]).max() < 1e-13 * max(1, np.abs(W[s]).max())
        Ws = W[s]
        Mb = Ws[np.ix_([i, j], [i, j])]
        val = np.real(np.trace(blk @ Mb))
        brute = np.real(np.einsum("nij,ji->n", grid, Mb)).max()
        assert val >= brute - 1e-12 * max(1, abs(brute))
    assert np.abs(g - R[2] @ R[1] @ R[0]).max() < 1e-14


def test_cabibbo_marinari_steps_random_K():
    rng = np.random.default_rng(4)
    grid = su2_matrices(su2_grid(5000, rng))
    for _ in range(20):
        K = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        g, W, R = O.local_update(K, O.OR, 1.0)
        _check_cm_steps(K, g, W, R, grid)
        assert np.real(np.trace(g @ K)) >= np.real(np.trace(K)) - 1e-13


def test_cabibbo_marinari_on_every_site_of_2_4():
    """Every site, every subgroup of a 2^4 lattice (where x+mu = x-mu)."""
    rng = np.random.default_rng(5)
    grid = su2_matrices(su2_grid(3000, rng))
    U = synth.field((2, 2, 2, 2), 0.8, 13)
    for site in range(16):
        K = O.gather_K(U, site)
        g, W, R = O.local_update(K, O.OR, 1.0)
        _check_cm_steps(K, g, W, R, grid)


# --------------------------------------------- Sec. 3.1 overrelaxation
def test_overrelaxation_is_first_order_power():
    """Each subgroup element becomes (1 - w) 1 + w r, rescaled onto SU(2) (2x2 matrix form),
    and the local value Re tr(R W) never falls below its value at R = 1."""
    rng = np.random.default_rng(6)
    for omega in (1.0, 1.3, 1.7, 1.95):
        for _ in range(10):
            K = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
            g, W, R = O.local_update(K, O.OR, omega)
            for s in range(3):
                i, j = SUBGROUPS[s]
                Mb = W[s][np.ix_([i, j], [i, j])]
                r_plain = su2_quaternion_matrix(O.su2_maximum(np.ascontiguousarray(Mb)))
                lin = (1 - omega) * np.eye(2) + omega * r_plain
                expect = lin / np.sqrt(np.linalg.det(lin))
                got = R[s][np.ix_([i, j], [i, j])]
                assert np.abs(got - expect).max() < 1e-13
                assert np.real(np.trace(got @ Mb)) >= np.real(np.trace(Mb)) - 1e-12


# -------------------------------------- Sec. 3.2 stochastic relaxation
def test_stochastic_relaxation_square_and_threshold():
    rng = np.random.default_rng(7)
    K = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    g1, W1, R1 = O.local_update(K, O.OR, 1.0)
    # p = 0: never square -> plain update
    g0, W0, R0 = O.local_update(K, O.SR, 1.9, p=0.0, draws=(0, 0, 0))
    assert np.abs(g0 - g1).max() < 1e-15
    # p = 1: always square; each R is the square of the plain maximum of its own W
    g2, W2, R2 = O.local_update(K, O.SR, 1.9, p=1.0, draws=(0xFFFFFFFF,) * 3)
    for s in range(3):
        i, j = SUBGROUPS[s]
        Mb = W2[s][np.ix_([i, j], [i, j])]
        r = su2_quaternion_matrix(O.su2_maximum(np.ascontiguousarray(Mb)))
        assert np.abs(R2[s][np.ix_([i, j], [i, j])] - r @ r).max() < 1e-14
        # microcanonical: Re tr(r^2 M) = Re tr(M)
        assert abs(np.real(np.trace(r @ r @ Mb)) - np.real(np.trace(Mb))) < 1e-12
    # threshold: draw < floor(p 2^32) decides each subgroup separately
    p = 0.8
    thr = int(np.floor(p * 2 ** 32))
    ga, Wa, Ra = O.local_update(K, O.SR, 1.0, p=p, draws=(thr - 1, thr, 0))
    for s, squared in enumerate([True, False, True]):
        i, j = SUBGROUPS[s]
        Mb = Wa[s][np.ix_([i, j], [i, j])]
        r = su2_quaternion_matrix(O.su2_maximum(np.ascontiguousarray(Mb)))
        assert np.abs(Ra[s][np.ix_([i, j], [i, j])] - (r @ r if squared else r)).max() < 1e-14


def test_stochastic_relaxation_p1_keeps_F():
    """With p = 1 every subgroup step is microcanonical: a full sweep leaves F unchanged
    while it moves the links."""
    U = synth.field((4, 4, 4, 4), 0.5, 14)
    F0 = O.measure(U)["F"]
    V0 = U.copy()
    O.sweeps(U, 3, algo=O.SR, p=1.0, seed=99)
    assert abs(O.measure(U)["F"] - F0) < 1e-13
    assert np.abs(U - V0).max() > 1e-2


def test_stochastic_relaxation_acceptance_rate():
    """Fraction of squared updates is p (binomial, 5 sigma)."""
    n = 20000
    p = 0.8
    thr = int(np.floor(p * 2 ** 32))
    acc = 0
    for site in range(n // 3):
        acc += int(np.sum(O.sr_draws(5, 3, site) < thr))
    m = 3 * (n // 3)
    assert abs(acc / m - p) < 5 * np.sqrt(p * (1 - p) / m)


# ----------------------------------------------- half-sweeps and sweeps
def test_half_sweep_is_independent_site_updates():
    """Sites of one parity only touch their own links (Sec. 3): the half-sweep equals
    every site's own update computed from the field before it, for every parity."""
    dims = (4, 2, 4, 2)
    U = synth.field(dims, 0.6, 15)
    for parity in (0, 1):
        for gauge in (O.LANDAU, O.COULOMB):
            V = U.copy()
            O.half_sweep(V, parity, gauge=gauge, omega=1.7, sweep=3)
            expect = U.copy()
            for site in range(64):
                if parity_of(site, dims) != parity:
                    continue
                fwd, bwd = O.site_new_links(U, site, gauge=gauge, omega=1.7, sweep=3)
                t, x3, x2, x1 = coords_of(site, dims)
                expect[t, x3, x2, x1] = fwd
                for mu, (ax, n) in enumerate([(0, 4), (3, 2), (2, 4), (1, 2)]):
                    c = [t, x3, x2, x1]
                    c[ax] = (c[ax] - 1) % n
                    expect[c[0], c[1], c[2], c[3], mu] = bwd[mu]
            assert np.array_equal(V, expect)


def test_site_order_and_threads_do_not_matter():
    U = synth.field((4, 4, 4, 4), 0.5, 16)
    ref = U.copy()
    O.half_sweep(ref, 0, omega=1.7)
    rng = np.random.default_rng(0)
    sh = U.copy()
    O.half_sweep(sh, 0, omega=1.7, order=rng.permutation(128))
    assert np.array_equal(ref, sh)
    n = O.max_threads()
    try:
        O.set_threads(1)
        one = U.copy()
        O.half_sweep(one, 0, omega=1.7)
    finally:
        O.set_threads(n)
    assert np.array_equal(ref, one)


@pytest.mark.parametrize("omega", [1.0, 1.7])
def test_F_never_decreases_per_half_sweep(omega):
    """Local maximisation (omega = 1) and first-order overrelaxation (omega < 2) never
    lower any local value, so F is non-decreasing after every half-sweep."""
    U = synth.field((4, 4, 4, 4), 0.7, 17)
    F = O.measure(U)["F"]
    for s in range(20):
        for parity in (0, 1):
            O.half_sweep(U, parity, omega=omega, sweep=s)
            F1 = O.measure(U)["F"]
            assert F1 >= F - 1e-15
            F = F1


def test_plaquettes_are_invariant():
    """Every update is a gauge transformation: every plaquette is unchanged (max over
    plaquettes), for OR and SR, Landau and Coulomb (with temporal links transformed)."""
    U = synth.field((4, 4, 4, 4), 0.7, 18)
    P0 = plaquettes(U)
    for gauge, algo in [(O.LANDAU, O.OR), (O.LANDAU, O.SR), (O.COULOMB, O.OR)]:
        V = U.copy()
        O.sweeps(V, 30, gauge=gauge, algo=algo, omega=1.7, p=0.8, seed=3)
        assert np.abs(plaquettes(V) - P0).max() < 1e-12


def test_coulomb_without_temporal_transform():
    """transform_temporal = 0 leaves U_0 untouched: the spatial plaquettes are invariant
    while space-time plaquettes change."""
    U = synth.field((4, 4, 4, 4), 0.7, 19)
    P0 = plaquettes(U)
    V = U.copy()
    O.sweeps(V, 5, gauge=O.COULOMB, omega=1.5, transform_temporal=0)
    assert np.array_equal(V[..., 0, :, :], U[..., 0, :, :])
    P1 = plaquettes(V)
    assert np.abs(P1[..., 3:] - P0[..., 3:]).max() < 1e-12  # planes (1,2), (1,3), (2,3)
    assert np.abs(P1[..., :3] - P0[..., :3]).max() > 1e-3


def test_links_stay_unitary():
    U = synth.field((2, 2, 4, 4), 0.7, 20)
    O.sweeps(U, 1000, omega=1.7)
    e, d = unitarity_error(U)
    assert e < 1e-13 and d < 1e-13


# ------------------------------------------------------- convergence
def test_pure_gauge_converges_to_unit_F():
    """eps = 0 gives h(x) h(x+mu)^dagger: gauge fixing recovers F = 1 and theta < tol."""
    for dims in [(4, 4, 4, 4), (6, 4, 4, 8)]:
        U = synth.field(dims, 0.0, 21)
        r = O.fix(U, omega=1.7, tol=1e-14, max_sweeps=3000)
        assert r["converged"] and r["theta"] < 1e-14
        assert abs(r["F"] - 1) < 1e-12


def test_fix_landau_and_coulomb_converge():
    U = synth.field((8, 8, 8, 8), 0.3, 1)
    r = O.fix(U, omega=1.7, tol=1e-14, max_sweeps=1000)
    assert r["converged"] and r["theta"] < 1e-14
    m = O.measure(U)
    assert m["theta"] == r["theta"] and m["F"] == r["F"]
    U = synth.field((4, 8, 8, 8), 0.5, 3)
    r = O.fix(U, gauge=O.COULOMB, omega=1.7, tol=1e-14, max_sweeps=1000)
    assert r["converged"]
    assert np.all(O.measure(U, O.COULOMB)["theta_t"] < 1e-14)


def test_fix_reports_not_converged():
    U = synth.field((4, 4, 4, 4), 0.5, 22)
    r = O.fix(U, omega=1.7, tol=1e-14, max_sweeps=5, check_every=2)
    assert not r["converged"] and r["sweeps"] == 5


def test_odd_extent_rejected():
    U = np.zeros((4, 4, 4, 3, 4, 3, 3), np.complex128)
    with pytest.raises(RuntimeError):
        O.measure(U)


# ------------------------------------------------------------ generator
def test_generator_pure_gauge_and_unitary():
    U = synth.field((4, 4, 2, 6), 0.0, 30)
    assert np.abs(plaquettes(U) - 1).max() < 1e-14
    e, d = unitarity_error(U)
    assert e < 1e-14 and d < 1e-14
    V = synth.field((4, 4, 2, 6), 0.5, 30)
    e, d = unitarity_error(V)
    assert e < 1e-14 and d < 1e-14


def test_generator_is_deterministic_and_seeded():
    a = synth.field((2, 2, 2, 4), 0.4, 31)
    b = synth.field((2, 2, 2, 4), 0.4, 31)
    c = synth.field((2, 2, 2, 4), 0.4, 32)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_generator_roughness_scales_with_eps_squared():
    """Small eps: 1 - <plaquette> grows like eps^2."""
    d = (4, 4, 4, 4)
    p1 = 1 - plaquettes(synth.field(d, 0.05, 33)).mean()
    p2 = 1 - plaquettes(synth.field(d, 0.1, 33)).mean()
    assert 3.7 < p2 / p1 < 4.3


def test_haar_moments():
    """Haar SU(3): E tr h = 0, E |tr h|^2 = 1."""
    h = synth.haar(40, 100000)
    tr = np.trace(h, axis1=1, axis2=2)
    assert abs(tr.mean()) < 5 * np.sqrt(1 / 100000)
    assert abs(np.mean(np.abs(tr) ** 2) - 1) < 0.03
    e, d = unitarity_error(h)
    assert e < 1e-14 and d < 1e-14


# ------------------------------------------- simulated annealing (heat bath)
@pytest.mark.parametrize("alpha", [0.8, 4.0, 16.0, 64.0])
def test_kp_draws_follow_the_heat_bath_density(alpha):
    """x with density ~ sqrt(1 - x^2) exp(alpha x) on [-1, 1] has the closed-form
    moments E[x] = I2(alpha)/I1(alpha) and E[x^2] = 1 - 3 I2/(alpha I1) (modified
    Bessel functions; derivatives of the normalisation pi I1(alpha)/alpha)."""
    from scipy.special import iv
    n = 200000
    x, fails = O.kp_draws(alpha, n, seed=11)
    assert fails <= 2e-3 * n
    x = x[np.isfinite(x)]
    assert np.all(np.abs(x) <= 1.0)
    m1 = iv(2, alpha) / iv(1, alpha)
    m2 = 1.0 - 3.0 * iv(2, alpha) / (alpha * iv(1, alpha))
    var = m2 - m1 * m1
    assert abs(x.mean() - m1) < 5 * np.sqrt(var / x.size)
    # fourth central moment bound for the second-moment check
    assert abs((x * x).mean() - m2) < 5 * np.sqrt(np.var(x * x) / x.size)


@pytest.mark.parametrize("alpha", [1.0, 10.0])
def test_heat_bath_element_is_distributed_around_the_maximum(alpha):
    """The drawn SU(2) element r is unit, its overlap x = r . p with the maximum p
    follows the heat-bath moments, and its part orthogonal to p points uniformly
    (zero mean, isotropic covariance in the 3-space orthogonal to p)."""
    from scipy.special import iv
    rng = np.random.default_rng(5)
    q = rng.normal(size=4)
    beta = alpha / (2.0 * np.linalg.norm(q))
    p = np.array([q[0], -q[1], -q[2], -q[3]]) / np.linalg.norm(q)
    n = 40000
    r = np.array([O.su2_heatbath(q, beta, seed=9, sweep=3, site=k, subgroup=1) for k in range(n)])
    assert np.abs(np.linalg.norm(r, axis=1) - 1).max() < 1e-14
    x = r @ p
    m1 = iv(2, alpha) / iv(1, alpha)
    assert abs(x.mean() - m1) < 5 * x.std() / np.sqrt(n)
    basis = np.linalg.qr(np.column_stack([p, rng.normal(size=(4, 3))]))[0][:, 1:]  # orthonormal, p-orthogonal
    v = r @ basis
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    assert np.abs(v.mean(axis=0)).max() < 5 / np.sqrt(3 * n)
    cov = v.T @ v / n
    assert np.abs(cov - np.eye(3) / 3).max() < 0.02


def test_heat_bath_at_large_beta_is_the_maximum():
    rng = np.random.default_rng(6)
    for _ in range(20):
        q = rng.normal(size=4)
        p = np.array([q[0], -q[1], -q[2], -q[3]]) / np.linalg.norm(q)
        r = O.su2_heatbath(q, 1e8, seed=1, sweep=0, site=int(rng.integers(1 << 30)), subgroup=2)
        assert np.abs(r - p).max() < 1e-3


def test_annealing_schedule_is_geometric():
    b = [O.sa_beta(0.5, 50.0, 5, i) for i in range(5)]
    assert b[0] == pytest.approx(0.5) and b[-1] == pytest.approx(50.0)
    assert np.allclose(np.diff(np.log(b)), np.log(100.0) / 4)
    assert O.sa_beta(0.5, 50.0, 1, 0) == 50.0


@pytest.mark.parametrize("gauge", [O.LANDAU, O.COULOMB])
def test_annealing_sweeps_are_gauge_transformations(gauge):
    """Heat-bath updates are gauge transformations like the relaxation's: every
    plaquette is kept, links stay unitary; at high beta the functional rises."""
    dims = (4, 4, 6, 4)
    U = synth.field(dims, 0.5, 41)
    V = U.copy()
    O.sa_sweeps(V, 5, 1.0, 10.0, gauge=gauge, seed=3)
    assert np.abs(plaquettes(V) - plaquettes(U)).max() < 1e-12
    e, d = unitarity_error(V)
    assert e < 1e-13 and d < 1e-13
    W = V.copy()
    O.sa_sweeps(W, 10, 1e3, 1e4, gauge=gauge, seed=4, sweep0=5)
    assert O.measure(W, gauge)["F"] > O.measure(V, gauge)["F"]


def test_annealing_then_relaxation_converges():
    dims = (4, 4, 4, 4)
    U = synth.field(dims, 0.5, 42)
    O.sa_sweeps(U, 30, 1.0, 100.0, seed=7)
    r = O.fix(U, omega=1.7, tol=1e-14, max_sweeps=3000)
    assert r["converged"] and O.measure(U)["theta"] < 1e-14


# ------------------------------------------------- maximally Abelian gauge
def _diag_field(dims, rng):
    """Abelian field: every link diagonal, exp(i phi_a) with sum phi_a = 0."""
    phi = rng.uniform(-np.pi, np.pi, size=tuple(dims) + (4, 2))
    U = np.zeros(tuple(dims) + (4, 3, 3), np.complex128)
    U[..., 0, 0] = np.exp(1j * phi[..., 0])
    U[..., 1, 1] = np.exp(1j * phi[..., 1])
    U[..., 2, 2] = np.exp(-1j * (phi[..., 0] + phi[..., 1]))
    return U


def _mag_site_functional(R, fwd, bwd):
    """sum of |diagonal|^2 of the site's links after g = R at the site (numpy)"""
    s = 0.0
    for U in fwd:
        s += np.sum(np.abs(np.diagonal(R @ U)) ** 2)
    for W in bwd:
        s += np.sum(np.abs(np.diagonal(W @ dag(R))) ** 2)
    return s


def test_mag_functional_closed_forms():
    """F_MAG = 1/(N_c N_d V) sum |U_aa|^2: 1 and theta_MAG = 0 on an Abelian (diagonal)
    field, whatever its phases; on Haar-random links E|U_aa|^2 = 1/3 (|U_aa|^2 of a
    Haar SU(3) matrix is Beta(1, 2)), so F_MAG = 1/3 within 5 standard errors."""
    rng = np.random.default_rng(31)
    dims = (4, 4, 2, 4)
    m = O.measure(_diag_field(dims, rng), O.MAG)
    assert abs(m["F"] - 1) < 1e-15 and m["theta"] < 1e-30
    z = rng.normal(size=tuple(dims) + (4, 3, 3)) + 1j * rng.normal(size=tuple(dims) + (4, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    q = q / (np.linalg.det(q) ** (1 / 3))[..., None, None]
    m = O.measure(np.ascontiguousarray(q), O.MAG)
    n = q[..., 0, 0].size * 3
    assert abs(m["F"] - 1 / 3) < 5 * np.sqrt(1 / 18 / n)
    # the plaquette is the gauge-invariant one, unchanged by the choice of functional
    assert abs(m["plaq"] - O.measure(np.ascontiguousarray(q))["plaq"]) < 1e-15


def test_mag_theta_is_the_gradient_of_F():
    """theta_MAG = 0 iff F_MAG is stationary under gauge transformations, and
    quantitatively theta_MAG is the squared gauge gradient of F_MAG: the functional
    is quadratic in the links, so under g = exp(i e lambda_a/2) at x,
    dF/de_a = -2 tr(T_a Delta_MAG(x))/(N_c N_d V), twice the Landau-type expression
    that _theta_from_gradient inverts."""
    U = synth.field((2, 4, 2, 4), 0.6, 35)
    m = O.measure(U, O.MAG)
    th = _theta_from_gradient(U, O.MAG).sum() / U.shape[0] / 4
    assert m["theta"] > 1e-3
    assert abs(th - m["theta"]) < 1e-7 * m["theta"]


def test_mag_subgroup_step_is_the_maximum():
    """One subgroup step: the element r maximises the site's MAG functional over the
    subgroup (brute force over random and gridded SU(2) elements), is stationary
    (no generator increases it to first or second order), the maximum is
    const + |v|/2, left factors exp(i phi sigma_3) keep the value (a circle of
    maximisers), and r is the one of that circle nearest the identity (r3 = 0,
    r0 >= 0)."""
    rng = np.random.default_rng(36)
    grid = su2_grid(2000, rng)[::9]
    for trial in range(4):
        links = np.stack([random_su3(rng) for _ in range(8)])
        fwd, bwd = links[:4], links[4:]
        for s, (i, j) in enumerate([(0, 1), (0, 2), (1, 2)]):
            v, r = O.mag_subgroup(links, s)
            def emb(q):
                R = np.eye(3, dtype=np.complex128)
                R[np.ix_([i, j], [i, j])] = su2_quaternion_matrix(q)
                return R
            f_r = _mag_site_functional(emb(r), fwd, bwd)
            f_1 = _mag_site_functional(np.eye(3), fwd, bwd)
            best = max(_mag_site_functional(emb(q), fwd, bwd) for q in grid)
            assert f_r >= best - 1e-12
            assert abs(f_r - (f_1 - v[2] / 2 + np.linalg.norm(v) / 2)) < 1e-12
            for k in range(3):
                for e in (1e-3, -1e-3):
                    gen = np.zeros(4)
                    gen[0], gen[k + 1] = np.cos(e), np.sin(e)
                    R2 = emb(gen) @ emb(r)
                    assert _mag_site_functional(R2, fwd, bwd) <= f_r + 1e-12
            for phi in (0.3, 1.1, 2.5):
                D = emb(np.array([np.cos(phi), 0, 0, np.sin(phi)]))
                assert abs(_mag_site_functional(D @ emb(r), fwd, bwd) - f_r) < 1e-12
            assert abs(r[3]) < 1e-15 and r[0] >= 0 and abs(np.linalg.norm(r) - 1) < 1e-15


def _site_links(U, site):
    """the 4 forward and 4 backward links of a site (numpy copies)"""
    dims = U.shape[:4]
    t, x3, x2, x1 = coords_of(site, dims)
    fwd, bwd = [], []
    for mu in range(4):
        c = {0: t, 1: x1, 2: x2, 3: x3}
        fwd.append(U[t, x3, x2, x1, mu].copy())
        c[mu] = (c[mu] - 1) % dims[{0: 0, 1: 3, 2: 2, 3: 1}[mu]]
        bwd.append(U[c[0], c[3], c[2], c[1], mu].copy())
    return np.array(fwd), np.array(bwd)


@pytest.mark.parametrize("omega", [1.0, 1.7])
def test_mag_site_update_composes_the_subgroup_steps(omega):
    """A site update is the three subgroup steps (0,1), (0,2), (1,2) in turn, each
    taken on the links as the steps before left them (forward links R U, backward
    links U R^dagger, applied here in numpy), each element overrelaxed to first
    order: the links the oracle's site update writes are those."""
    U = synth.field((4, 4, 2, 4), 0.6, 39)
    for site in (0, 5, 37, 90, 127):
        fwd, bwd = _site_links(U, site)
        for s, (i, j) in enumerate([(0, 1), (0, 2), (1, 2)]):
            _, r = O.mag_subgroup(np.concatenate([fwd, bwd]), s)
            q = np.array([1 - omega + omega * r[0], omega * r[1], omega * r[2], omega * r[3]])
            q /= np.linalg.norm(q)
            R = np.eye(3, dtype=np.complex128)
            R[np.ix_([i, j], [i, j])] = su2_quaternion_matrix(q)
            fwd = R @ fwd
            bwd = bwd @ dag(R)
        nf, nb = O.site_new_links(U, site, gauge=O.MAG, omega=omega)
        assert np.abs(nf - fwd).max() < 1e-13 and np.abs(nb - bwd).max() < 1e-13


@pytest.mark.parametrize("omega", [1.0, 1.7])
def test_mag_sweeps_raise_F_and_keep_the_field(omega):
    """Relaxation (omega = 1) never lowers F_MAG: every subgroup step maximises the
    site functional; overrelaxed sweeps raise it overall.  Plaquettes and unitarity
    are kept (each update is a gauge transformation)."""
    U = synth.field((4, 4, 2, 4), 0.5, 37)
    P0 = plaquettes(U)
    F = [O.measure(U, O.MAG)["F"]]
    for s in range(12):
        O.half_sweep(U, 0, gauge=O.MAG, omega=omega)
        F.append(O.measure(U, O.MAG)["F"])
        O.half_sweep(U, 1, gauge=O.MAG, omega=omega)
        F.append(O.measure(U, O.MAG)["F"])
    if omega == 1.0:
        assert all(b >= a - 1e-14 for a, b in zip(F, F[1:]))
    assert F[-1] > F[0] + 0.05
    assert np.abs(plaquettes(U) - P0).max() < 1e-12
    assert max(unitarity_error(U)) < 1e-12


def test_mag_recovers_a_transformed_abelian_field():
    """A random gauge transform of an Abelian field has F_MAG < 1; MAG fixing climbs back
    to the global maximum F_MAG = 1 (theta_MAG -> 0), a case whose answer the
    functional fixes without reference to the update."""
    rng = np.random.default_rng(38)
    dims = (4, 4, 4, 4)
    A = _diag_field(dims, rng)
    small = np.stack([expm_herm(0.35 * np.einsum("a,aij->ij", rng.normal(size=8), GELL_MANN))
                      for _ in range(int(np.prod(dims)))]).reshape(tuple(dims) + (3, 3))
    U = np.ascontiguousarray(transform_field(A, small))
    assert O.measure(U, O.MAG)["F"] < 0.9
    r = O.fix(U, gauge=O.MAG, omega=1.7, tol=1e-24, max_sweeps=3000, check_every=10)
    m = O.measure(U, O.MAG)
    assert r["converged"] and m["theta"] < 1e-24 and abs(m["F"] - 1) < 1e-13
    assert np.abs(plaquettes(U) - plaquettes(A)).max() < 1e-12


def test_mag_annealing_is_rejected():
    U = synth.field((2, 2, 2, 2), 0.3, 1)
    with pytest.raises(Exception):
        O.sa_sweeps(U, 1, 1.0, 2.0, gauge=O.MAG)


# ------------------------------- conditioning of a site update (test support)
def test_site_conditioning_is_the_smallest_subgroup_maximum():
    """Landau and Coulomb: kappa = 1/min_s |q_s|.  At omega = 1 each step reaches
    its block's maximum Re tr(R_s W_s) = 2|q_s| (the closed form's value, pinned
    against brute force above), so kappa = 2 / min_s of that value: every site of
    both parities of a rough field."""
    dims = (4, 4, 2, 6)
    U = synth.field(dims, 0.6, 71)
    for gauge in (O.LANDAU, O.COULOMB):
        for p in (0, 1):
            kap = O.site_conditioning(U, p, gauge=gauge, omega=1.0)
            for site in range(int(np.prod(dims))):
                c = coords_of(site, dims)
                if parity_of(site, dims) != p:
                    assert np.isnan(kap[c])
                    continue
                g, W, R = O.local_update(O.gather_K(U, site, gauge), O.OR, 1.0)
                vals = [np.real(np.trace((R[s] @ W[s])[np.ix_([i, j], [i, j])])) for s, (i, j) in enumerate(SUBGROUPS)]
                assert abs(kap[c] - 2 / min(vals)) < 1e-12 * kap[c]


def test_landau_conditioning_bounds_the_step_sensitivity():
    """The first-order change of the closed-form element r = (q0, -q)/|q| is at
    most |dq|/|q| (finite differences of the oracle's maximum on perturbed blocks;
    the ratio reaches 1 for perturbations across q)."""
    rng = np.random.default_rng(72)
    worst = 0.0
    for _ in range(400):
        M = (rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))) * rng.uniform(0.05, 3)
        d = (rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))) * 1e-8
        q = lambda m: np.array([np.real(m[0, 0] + m[1, 1]), np.imag(m[0, 1] + m[1, 0]),
                                np.real(m[0, 1] - m[1, 0]), np.imag(m[0, 0] - m[1, 1])]) / 2
        dr = np.linalg.norm(O.su2_maximum(M + d) - O.su2_maximum(M))
        ratio = dr / (np.linalg.norm(q(M + d) - q(M)) / np.linalg.norm(q(M)))
        worst = max(worst, ratio)
    assert 0.5 < worst < 1 + 1e-5


def _mag_chain_kappa(U, site, omega):
    """kappa of a maximally Abelian site update, from the pinned subgroup steps
    composed in numpy (as test_mag_site_update_composes_the_subgroup_steps)."""
    fwd, bwd = _site_links(U, site)
    kap = 0.0
    for s, (i, j) in enumerate([(0, 1), (0, 2), (1, 2)]):
        v, r = O.mag_subgroup(np.concatenate([fwd, bwd]), s)
        nv = np.linalg.norm(v)
        kap += np.sqrt(2 / (nv * (nv + v[2])))
        q = np.array([1 - omega + omega * r[0], omega * r[1], omega * r[2], omega * r[3]])
        q /= np.linalg.norm(q)
        R = np.eye(3, dtype=np.complex128)
        R[np.ix_([i, j], [i, j])] = su2_quaternion_matrix(q)
        fwd = R @ fwd
        bwd = bwd @ dag(R)
    return kap


@pytest.mark.parametrize("omega", [1.0, 1.7])
def test_mag_conditioning_sums_the_steps(omega):
    """Maximally Abelian gauge: kappa = sum_s sqrt(2/(|v_s|(|v_s| + v_s3))), v_s of
    each step on the links as the steps before left them."""
    U = synth.field((4, 4, 2, 4), 0.6, 73)
    for p in (0, 1):
        kap = O.site_conditioning(U, p, gauge=O.MAG, omega=omega)
        for site in (0, 1, 5, 37, 90, 127):
            c = coords_of(site, U.shape[:4])
            if parity_of(site, U.shape[:4]) == p:
                assert abs(kap[c] - _mag_chain_kappa(U, site, omega)) < 1e-12 * kap[c]


def test_mag_conditioning_is_twice_the_derivative_of_the_maximum():
    """The term sqrt(2/(|v|(|v| + v_3))) is twice the spectral norm of the
    derivative of the maximiser r(v) (the oracle's, by finite differences of the
    links: |dr| <= term/2 |dv| to first order, with equality in the worst
    direction), including near v = -|v| e_3 where the rotation axis turns fast."""
    rng = np.random.default_rng(74)
    worst = 0.0
    base = synth.field((2, 2, 2, 2), 0.9, 75).reshape(-1, 3, 3)
    for k in range(300):
        L8 = base[rng.choice(len(base), 8, replace=False)].copy()
        if k % 3 == 0:  # steer v towards -e_3: swap the first two rows of the forward links
            L8[:4] = L8[:4][:, [1, 0, 2], :]
        v, r = O.mag_subgroup(L8, 0)
        nv = np.linalg.norm(v)
        term = np.sqrt(2 / (nv * (nv + v[2])))
        d = (rng.normal(size=L8.shape) + 1j * rng.normal(size=L8.shape)) * 1e-9
        v2, r2 = O.mag_subgroup(L8 + d, 0)
        worst = max(worst, np.linalg.norm(r2 - r) / (term / 2 * np.linalg.norm(v2 - v)))
    assert 0.3 < worst < 1 + 1e-4


# ------------------------------------- the sweeps' fused estimate (test support)
@pytest.mark.parametrize("gauge", [O.LANDAU, O.COULOMB])
def test_parity_violation_is_the_violation_of_K(gauge):
    """The per-parity sums of tr[Delta Delta^dagger] (Delta from the A_mu, Sec. 2)
    equal those of the traceless part of (K - K^dagger)/(2i), K(x) the site's
    local matrix (the identity the sweep kernels' estimate relies on; numpy from
    gather_K), and the two parities add up to the measured theta."""
    dims = (4, 2, 4, 6)
    U = synth.field(dims, 0.6, 76)
    vs = dims[1] * dims[2] * dims[3]
    m = O.measure(U, gauge)
    both = np.zeros(dims[0])
    for p in (0, 1):
        got = O.parity_violation(U, p, gauge)
        expect = np.zeros(dims[0])
        for site in range(int(np.prod(dims))):
            if parity_of(site, dims) != p:
                continue
            K = O.gather_K(U, site, gauge)
            D = (K - dag(K)) / 2j
            D -= np.eye(3) * np.trace(D) / 3
            expect[coords_of(site, dims)[0]] += np.sum(np.abs(D) ** 2)
        assert np.allclose(got, expect, rtol=1e-12, atol=0)
        both += got
    if gauge == O.COULOMB:
        assert np.allclose(both / (3 * vs), m["theta_t"], rtol=1e-12, atol=0)
    else:
        assert abs(both.sum() / (3 * np.prod(dims)) - m["theta"]) < 1e-12 * m["theta"]


# ------------------------------- annealing decision margins (test support)
def test_annealing_half_sweeps_and_decision_margins():
    """Two annealing half-sweeps are the oracle's annealing sweep; and the
    reported margins of the Kennedy-Pendleton comparisons mark where a decision
    can flip.  Stepping beta by a relative h moves delta (proportional to 1/beta)
    by h |delta|, so the comparison u^2 <= 1 - delta/2 can change side over a
    step only where its relative margin is below h/2 on one side of the step:
    across a fine scan every jump of a site's element (a flipped decision) sits
    at such a margin, and there are jumps to check."""
    dims = (4, 4, 6, 4)
    U = synth.field(dims, 0.6, 77)
    ref = U.copy()
    O.sa_sweeps(ref, 1, 1.5, 1.5, seed=19)
    h = U.copy()
    O.sa_half_sweep(h, 0, 1.5, seed=19)
    O.sa_half_sweep(h, 1, 1.5, seed=19)
    assert np.array_equal(h, ref)
    betas = np.linspace(1.0, 2.0, 401)
    prev = prev_m = None
    jumps = 0
    for b0, b in zip(np.r_[np.nan, betas[:-1]], betas):
        a = U.copy()
        O.sa_half_sweep(a, 0, b, seed=19)
        _, m = O.sa_site_stats(U, 0, b, seed=19)
        if prev is not None:
            moved = np.abs(a - prev).max(axis=(-3, -2, -1))  # per site: its forward links
            step = (b - b0) / b0
            jump = ~np.isnan(m) & (moved > 5e-2)
            jumps += int(jump.sum())
            assert np.all(np.minimum(m[jump], prev_m[jump]) <= 0.5 * step * 1.05)
        prev, prev_m = a, m
    assert jumps > 20


def test_generator_values_do_not_depend_on_its_thread_count():
    """The served-stream client makes inputs on fewer cores than the default team;
    every element of a field comes from its own counter, so the field is the same
    bit for bit on 1, 3 or all threads (ragged extents, Haar and link draws)."""
    dims = (4, 6, 2, 8)
    ref = synth.field(dims, 0.45, 77)
    for n in (1, 3):
        assert np.array_equal(synth.field(dims, 0.45, 77, threads=n), ref)
    assert not np.array_equal(synth.field(dims, 0.45, 78), ref)
