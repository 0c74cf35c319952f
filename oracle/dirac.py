"""Oracle: the finite-density Wilson kernel H(mu) = gamma5 Dw(mu) (Sec. 1, Eq. (1.1)).

Test infrastructure only (see the package docstring).

The paper names Dw(mu) but does not write it out.  The reading used here is the
standard exponential (Hasenfratz-Karsch) form of the Wilson operator at chemical
potential mu, with Wilson parameter r and mass m_w:

  (Dw psi)(x) = (4r + m_w) psi(x)
               - 1/2 sum_nu [ f+_nu (r - gamma_nu) U_nu(x) psi(x+nu)
                            + f-_nu (r + gamma_nu) U_nu(x-nu)^dag psi(x-nu) ],
  f+-_nu = 1 for nu = x, y, z and f+-_t = exp(+-mu);

a hop across the time boundary carries a factor -1 (antiperiodic in time), space is
periodic.  Gamma matrices in the chiral basis: gamma_k = [[0, -i s_k], [i s_k, 0]],
gamma_t = [[0, 1], [1, 0]], gamma5 = gamma_x gamma_y gamma_z gamma_t = diag(1,1,-1,-1).

Fields: spinors complex128 [V][4][3] (site s = x + nx(y + ny(z + nz t))), links
complex128 [4][V][3][3].  Internally the vectorised stencil reshapes to
(nt, nz, ny, nx, 4, 3) so that np.roll walks the lattice axes.

Two independent codings are given and tested against each other: a vectorised
np.roll stencil (apply_*) and an explicit per-site loop assembly of the dense matrix
(dense_*).  Both are pinned by the free-field closed form (oracle.free_field).
"""
import numpy as np

AXIS = {0: 3, 1: 2, 2: 1, 3: 0}   # direction nu -> array axis of (nt, nz, ny, nx, ...)


def gammas():
    """Chiral-basis Euclidean gamma matrices [gx, gy, gz, gt] and gamma5."""
    s = [np.array([[0, 1], [1, 0]], complex),
         np.array([[0, -1j], [1j, 0]], complex),
         np.array([[1, 0], [0, -1]], complex)]
    Z = np.zeros((2, 2), complex)
    I2 = np.eye(2, dtype=complex)
    g = [np.block([[Z, -1j * sk], [1j * sk, Z]]) for sk in s]
    g.append(np.block([[Z, I2], [I2, Z]]))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


def gell_mann():
    """The eight Gell-Mann matrices lambda_a (tr lambda_a lambda_b = 2 delta_ab)."""
    l = np.zeros((8, 3, 3), complex)
    l[0][[0, 1], [1, 0]] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][[0, 2], [2, 0]] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][[1, 2], [2, 1]] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return l


class Lattice:
    """Lattice geometry and the Wilson parameters (m_w, r)."""

    def __init__(self, dims, m_w=-2.0, r=1.0, antiperiodic_t=True):
        self.dims = tuple(int(d) for d in dims)
        self.nt, self.nx, self.ny, self.nz = self.dims
        self.V = self.nt * self.nx * self.ny * self.nz
        self.n = 12 * self.V
        self.m_w = float(m_w)
        self.r = float(r)
        self.apbc = bool(antiperiodic_t)

    # --- layout helpers -------------------------------------------------------
    def grid(self, psi):
        return np.asarray(psi).reshape(self.nt, self.nz, self.ny, self.nx, 4, 3)

    def links_grid(self, U):
        return np.asarray(U).reshape(4, self.nt, self.nz, self.ny, self.nx, 3, 3)

    def flat(self, psi_grid):
        return np.ascontiguousarray(psi_grid).reshape(self.V, 4, 3)

    def coords(self, s):
        x = s % self.nx
        y = (s // self.nx) % self.ny
        z = (s // (self.nx * self.ny)) % self.nz
        t = s // (self.nx * self.ny * self.nz)
        return x, y, z, t

    def site(self, x, y, z, t):
        return x + self.nx * (y + self.ny * (z + self.nz * t))

    def neighbour(self, s, nu, step):
        """Site s + step*nu-hat and the boundary sign (-1 across the time boundary)."""
        c = list(self.coords(s))
        ext = [self.nx, self.ny, self.nz, self.nt][nu]
        c[nu] += step
        sign = 1.0
        if c[nu] >= ext or c[nu] < 0:
            c[nu] %= ext
            if nu == 3 and self.apbc:
                sign = -1.0
        return self.site(*c), sign


def _shift(lat, field, nu, step):
    """field(x + step*nu) on the (nt, nz, ny, nx, ...) grid, with the time-boundary sign."""
    ax = AXIS[nu]
    out = np.roll(field, -step, axis=ax)
    if nu == 3 and lat.apbc:
        out = out.copy()
        if step == 1:
            out[lat.nt - 1] *= -1.0
        else:
            out[0] *= -1.0
    return out


def _wilson_grid(lat, psi, links, diag, fwd, bwd, fwd_proj_sign):
    """diag*psi - 1/2 sum_nu [fwd[nu] (r + s*gamma) L psi(x+nu) + bwd[nu] (r - s*gamma) L(x-nu)^dag psi(x-nu)]
    with s = fwd_proj_sign (s = -1 gives the Wilson projectors of Dw)."""
    g, _ = gammas()
    I4 = np.eye(4)
    out = diag * psi
    for nu in range(4):
        L = links[nu]
        if fwd[nu] != 0:
            nb = _shift(lat, psi, nu, +1)
            Lpsi = np.einsum("...ab,...sb->...sa", L, nb)
            P = lat.r * I4 + fwd_proj_sign * g[nu]
            out = out - 0.5 * fwd[nu] * np.einsum("st,...tc->...sc", P, Lpsi)
        if bwd[nu] != 0:
            nb = _shift(lat, psi, nu, -1)
            Lb = np.roll(L, 1, axis=AXIS[nu])        # L(x - nu)
            Lpsi = np.einsum("...ba,...sb->...sa", Lb.conj(), nb)
            P = lat.r * I4 - fwd_proj_sign * g[nu]
            out = out - 0.5 * bwd[nu] * np.einsum("st,...tc->...sc", P, Lpsi)
    return out


def _g5(psi_grid):
    _, g5 = gammas()
    return np.einsum("st,...tc->...sc", g5, psi_grid)


def _factors(mu):
    return [1.0, 1.0, 1.0, np.exp(mu)], [1.0, 1.0, 1.0, np.exp(-mu)]


def apply_Dw(lat, U, psi, mu):
    fwd, bwd = _factors(mu)
    out = _wilson_grid(lat, lat.grid(psi), lat.links_grid(U), 4 * lat.r + lat.m_w, fwd, bwd, -1.0)
    return lat.flat(out)


def apply_H(lat, U, psi, mu):
    """H(mu) psi = gamma5 Dw(mu) psi (Eq. (1.1))."""
    fwd, bwd = _factors(mu)
    out = _wilson_grid(lat, lat.grid(psi), lat.links_grid(U), 4 * lat.r + lat.m_w, fwd, bwd, -1.0)
    return lat.flat(_g5(out))


def apply_Hdag(lat, U, psi, mu):
    """H(mu)^dag psi = Dw(mu)^dag gamma5 psi, written as the literal adjoint of the
    stencil: the forward hop carries conj(f-) (r + gamma) U(x), the backward hop
    conj(f+) (r - gamma) U(x-nu)^dag.  (gamma5-hermiticity H(mu)^dag = H(-mu) is a
    tested property, not used here.)"""
    fwd, bwd = _factors(mu)
    out = _wilson_grid(lat, _g5(lat.grid(psi)), lat.links_grid(U), 4 * lat.r + lat.m_w,
                       [np.conj(b) for b in bwd], [np.conj(f) for f in fwd], +1.0)
    return lat.flat(out)


def apply_dH_dmu(lat, U, psi, mu):
    """d H(mu)/d mu psi: only the time hops, with d exp(+-mu)/d mu = +-exp(+-mu)."""
    fwd = [0.0, 0.0, 0.0, np.exp(mu)]
    bwd = [0.0, 0.0, 0.0, -np.exp(-mu)]
    out = _wilson_grid(lat, lat.grid(psi), lat.links_grid(U), 0.0, fwd, bwd, -1.0)
    return lat.flat(_g5(out))


def apply_dH_dmu_dag(lat, U, psi, mu):
    fwd = [0.0, 0.0, 0.0, np.conj(-np.exp(-mu))]
    bwd = [0.0, 0.0, 0.0, np.conj(np.exp(mu))]
    out = _wilson_grid(lat, _g5(lat.grid(psi)), lat.links_grid(U), 0.0, fwd, bwd, +1.0)
    return lat.flat(out)


def su3_tangent(omega):
    """Omega_nu(x) = sum_a omega^a lambda_a / 2, from float64 [4][V][8]."""
    return np.einsum("dsa,aij->dsij", np.asarray(omega), gell_mann() / 2)


def link_derivative(U, omega=None, theta=None):
    """d/dt of U_nu(x) -> exp(i t Omega_nu(x)) U_nu(x) at t = 0: Y = i Omega U.
    For a U(1) direction theta_nu(x), Omega = theta * 1 (the paper's external field, Sec. 4)."""
    U = np.asarray(U)
    if omega is not None:
        Om = su3_tangent(omega)
        return 1j * np.einsum("dsij,dsjk->dsik", Om, U)
    th = np.asarray(theta)
    return 1j * th[:, :, None, None] * U


def apply_dH_dir(lat, U, Y, psi, mu):
    """d_t H psi for a link-direction derivative with dU/dt = Y: the hopping part of
    H(mu) with U replaced by Y (forward) and U^dag by Y^dag (backward), no diagonal."""
    fwd, bwd = _factors(mu)
    out = _wilson_grid(lat, lat.grid(psi), lat.links_grid(Y), 0.0, fwd, bwd, -1.0)
    return lat.flat(_g5(out))


def apply_dH_dir_dag(lat, U, Y, psi, mu):
    fwd, bwd = _factors(mu)
    out = _wilson_grid(lat, _g5(lat.grid(psi)), lat.links_grid(Y), 0.0,
                       [np.conj(b) for b in bwd], [np.conj(f) for f in fwd], +1.0)
    return lat.flat(out)


# --- dense assembly: an independent, per-site coding of the same operators ---------

def _dense_wilson(lat, links, diag, fwd, bwd):
    """Dense n x n matrix of diag*1 - 1/2 sum hops (forward projector r - gamma)."""
    g, g5 = gammas()
    I4 = np.eye(4)
    n = lat.n
    D = np.zeros((n, n), complex)
    L = np.asarray(links)
    for s in range(lat.V):
        D[12 * s:12 * s + 12, 12 * s:12 * s + 12] += diag * np.eye(12)
        for nu in range(4):
            sp, sgn_p = lat.neighbour(s, nu, +1)
            sm, sgn_m = lat.neighbour(s, nu, -1)
            blk_f = -0.5 * fwd[nu] * sgn_p * np.kron(lat.r * I4 - g[nu], L[nu][s])
            blk_b = -0.5 * bwd[nu] * sgn_m * np.kron(lat.r * I4 + g[nu], L[nu][sm].conj().T)
            D[12 * s:12 * s + 12, 12 * sp:12 * sp + 12] += blk_f
            D[12 * s:12 * s + 12, 12 * sm:12 * sm + 12] += blk_b
    G5 = np.kron(np.eye(lat.V), np.kron(g5, np.eye(3)))
    return G5 @ D


def dense_H(lat, U, mu):
    fwd, bwd = _factors(mu)
    return _dense_wilson(lat, U, 4 * lat.r + lat.m_w, fwd, bwd)


def dense_dH_dmu(lat, U, mu):
    return _dense_wilson(lat, U, 0.0, [0, 0, 0, np.exp(mu)], [0, 0, 0, -np.exp(-mu)])


def dense_dH_dir(lat, U, Y, mu):
    fwd, bwd = _factors(mu)
    return _dense_wilson(lat, Y, 0.0, fwd, bwd)
