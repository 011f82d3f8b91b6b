"""Small numpy helpers for the tests (independent of the oracle and the library).

Links are complex128 arrays of shape (N_t, N_3, N_2, N_1, 4, 3, 3); direction
mu = 0 is t (array axis 0), mu = 1, 2, 3 are x1, x2, x3 (array axes 3, 2, 1).
"""
import numpy as np

AXIS = {0: 0, 1: 3, 2: 2, 3: 1}  # direction mu -> array axis

GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
GELL_MANN[0][0, 1] = GELL_MANN[0][1, 0] = 1
GELL_MANN[1][0, 1] = -1j
GELL_MANN[1][1, 0] = 1j
GELL_MANN[2][0, 0] = 1
GELL_MANN[2][1, 1] = -1
GELL_MANN[3][0, 2] = GELL_MANN[3][2, 0] = 1
GELL_MANN[4][0, 2] = -1j
GELL_MANN[4][2, 0] = 1j
GELL_MANN[5][1, 2] = GELL_MANN[5][2, 1] = 1
GELL_MANN[6][1, 2] = -1j
GELL_MANN[6][2, 1] = 1j
GELL_MANN[7] = np.diag([1, 1, -2]) / np.sqrt(3)


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def shift(field, mu, step):
    """field(x + step*mu) as an array indexed by x (periodic)."""
    return np.roll(field, -step, axis=AXIS[mu])


def plaquettes(U):
    """Re tr of every plaquette / 3, shape (N_t, N_3, N_2, N_1, 6)."""
    out = []
    for mu in range(4):
        for nu in range(mu + 1, 4):
            a = U[..., mu, :, :]
            b = shift(U[..., nu, :, :], mu, 1)
            c = shift(U[..., mu, :, :], nu, 1)
            d = U[..., nu, :, :]
            p = a @ b @ dag(c) @ dag(d)
            out.append(np.real(np.trace(p, axis1=-2, axis2=-1)) / 3)
    return np.stack(out, axis=-1)


def unitarity_error(U):
    m = U.reshape(-1, 3, 3)
    e = np.abs(dag(m) @ m - np.eye(3)).max()
    d = np.abs(np.linalg.det(m) - 1).max()
    return e, d


def expm_herm(h):
    """exp(i h) for a Hermitian 3x3 h via its eigendecomposition."""
    w, v = np.linalg.eigh(h)
    return (v * np.exp(1j * w)) @ dag(v)


def random_su3(rng, n=None):
    shape = (n,) if n is not None else ()
    h = np.einsum("...a,aij->...ij", rng.normal(size=shape + (8,)), GELL_MANN) * 0.9
    return expm_herm(h)


def transform_site(U, site_coords, g):
    """Copy of U with the gauge transformation g applied at one site only:
    U_mu(x) -> g U_mu(x), U_mu(x - mu) -> U_mu(x - mu) g^dagger."""
    V = U.copy()
    t, x3, x2, x1 = site_coords
    coords = {0: t, 1: x1, 2: x2, 3: x3}
    dims = U.shape[:4]
    for mu in range(4):
        V[t, x3, x2, x1, mu] = g @ V[t, x3, x2, x1, mu]
        c = dict(coords)
        c[mu] = (c[mu] - 1) % dims[AXIS[mu]]
        V[c[0], c[3], c[2], c[1], mu] = V[c[0], c[3], c[2], c[1], mu] @ dag(g)
    return V


def transform_global(U, g):
    """Constant gauge transformation g U g^dagger on every link."""
    return g @ U @ dag(g)


def transform_field(U, G):
    """U_mu(x) -> G(x) U_mu(x) G(x+mu)^dagger for a field G of shape (N_t,N_3,N_2,N_1,3,3)."""
    V = np.empty_like(U)
    for mu in range(4):
        V[..., mu, :, :] = G @ U[..., mu, :, :] @ dag(shift(G, mu, 1))
    return V


def coords_of(site, dims):
    nt, n3, n2, n1 = dims
    x1 = site % n1
    r = site // n1
    x2 = r % n2
    r //= n2
    x3 = r % n3
    t = r // n3
    return (t, x3, x2, x1)


def parity_of(site, dims):
    return sum(coords_of(site, dims)) & 1


def su2_quaternion_matrix(r):
    r0, r1, r2, r3 = r
    return np.array([[r0 + 1j * r3, r2 + 1j * r1], [-r2 + 1j * r1, r0 - 1j * r3]])


def su2_grid(n_random, rng):
    """Brute-force SU(2) sample: random unit quaternions plus a regular Hopf-type grid."""
    q = rng.normal(size=(n_random, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    # regular grid in Hopf coordinates (eta, xi1, xi2)
    m = 24
    eta = (np.arange(m) + 0.5) * (np.pi / 2) / m
    xi = np.arange(2 * m) * (2 * np.pi) / (2 * m)
    E, X1, X2 = np.meshgrid(eta, xi, xi, indexing="ij")
    g = np.stack([np.cos(E) * np.cos(X1), np.cos(E) * np.sin(X1), np.sin(E) * np.cos(X2),
                  np.sin(E) * np.sin(X2)], axis=-1).reshape(-1, 4)
    return np.concatenate([q, g])


def su2_matrices(quats):
    r0, r1, r2, r3 = quats.T
    m = np.empty((len(quats), 2, 2), np.complex128)
    m[:, 0, 0] = r0 + 1j * r3
    m[:, 0, 1] = r2 + 1j * r1
    m[:, 1, 0] = -r2 + 1j * r1
    m[:, 1, 1] = r0 - 1j * r3
    return m


# ----------------------------------------------- FP32 parity bounds
U_FP32 = 2.0 ** -24  # unit roundoff of binary32


def parity_field(dims):
    t, x3, x2, x1 = np.indices(tuple(dims))
    return (t + x3 + x2 + x1) & 1


def link_endpoint(site_values, parity):
    """Per link (z, mu): the value at the link's endpoint of the given parity --
    z if z has that parity, else z + mu.  Shape (N_t, N_3, N_2, N_1, 4)."""
    par = parity_field(site_values.shape)
    return np.stack([np.where(par == parity, site_values, shift(site_values, mu, 1)) for mu in range(4)], axis=-1)


def fp32_half_sweep_bound(kappa, parity, c):
    """Per link: c u kappa(w), w the link's endpoint of the updated parity (the
    site whose update wrote it)."""
    return c * U_FP32 * link_endpoint(kappa, parity)


def fp32_sweep_bound(kappa_even, kappa_odd, c=16.0, a=2.0):
    """Per link, the first-order FP32 error of one full sweep (even half, then odd
    half) from the conditioning kappa of every site update (the oracle's, on the
    field each half starts from).  A site update turns an error d of its K(x) into
    an error ~ a d kappa of g (a = 2 bounds the overrelaxation factor omega < 2 and
    the doubled angle of a stochastic-relaxation square); its own K carries the
    rounding eps = 8u of 8 FP32 links and 7 sums (root-sum-square), so c = a eps /
    u = 16.  The odd site y also reads the 8 links the even half wrote, each off
    by ~ c u kappa of its writer: its K is off by eps (1 + a nu(y)), nu the
    root-sum-square of the 8 neighbours' kappa.  A link is written once in each
    half, by its even endpoint x and its odd endpoint y:
        B = c u (kappa(x) + kappa(y) (1 + a nu(y))).
    Shape (N_t, N_3, N_2, N_1, 4)."""
    par = parity_field(kappa_even.shape)
    kap = np.where(par == 0, kappa_even, kappa_odd)
    nu = np.sqrt(sum(shift(kap, mu, s) ** 2 for mu in range(4) for s in (1, -1)))
    return c * U_FP32 * (link_endpoint(kap, 0) + link_endpoint(kap, 1) * (1 + a * link_endpoint(nu, 1)))


def check_fp32_bound(err, bound, floor=5e-6):
    """Every entry within max(floor, its link's bound); returns (worst err / allowed,
    entries above the floor, links whose bound exceeds the floor)."""
    allowed = np.maximum(floor, bound)[..., None, None]
    return float((err / allowed).max()), int((err > floor).sum()), int((bound > floor).sum())
