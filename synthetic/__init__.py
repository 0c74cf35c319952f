"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module only draws random numbers and shapes them into the input types of the
method: SU(3) gauge fields, colour-spinor sources and tangent directions.  It holds
none of the method's arithmetic (no Dirac operator, no Krylov recurrence, no matrix
function).  The paper's quenched Luescher-Weisz configurations (Sec. 4) are not
available; these fields stand in for them with the paper's lattice shapes.

Conventions (shared by every consumer):
  * lattice dims (nt, nx, ny, nz); site s = x + nx*(y + ny*(z + nz*t)).
  * gauge field: complex128 array [4][V][3][3], direction nu = 0..3 = x, y, z, t;
    U[nu][s] is the link from s to s + nu-hat.
  * colour-spinor field: complex128 array [V][4][3] (spin, colour), flattened n = 12 V.
  * su(3) tangent direction: float64 array [4][V][8] of Gell-Mann coefficients
    omega^a, Omega = sum_a omega^a lambda_a / 2.
"""
import numpy as np

__all__ = ["volume", "gauge_field", "gaussian_source", "z2_source",
           "su3_direction", "u1_direction", "RAGGED_BATCH", "RAGGED_MU"]

# The ragged batch of the batching workload: four lattices of uneven size, link spread eps
# and Krylov depth k, as (dims, eps, k, gauge seed); Z2-noise sources; mu = RAGGED_MU.
RAGGED_BATCH = [((6, 6, 6, 6), 0.3, 100, 31), ((8, 8, 8, 8), 0.5, 200, 32),
                ((8, 12, 12, 12), 0.3, 250, 33), ((10, 10, 10, 10), 0.5, 300, 34)]
RAGGED_MU = 0.2


def volume(dims):
    nt, nx, ny, nz = dims
    return nt * nx * ny * nz


def _gell_mann():
    g = np.zeros((8, 3, 3), dtype=np.complex128)
    g[0][0, 1] = g[0][1, 0] = 1
    g[1][0, 1] = -1j
    g[1][1, 0] = 1j
    g[2][0, 0] = 1
    g[2][1, 1] = -1
    g[3][0, 2] = g[3][2, 0] = 1
    g[4][0, 2] = -1j
    g[4][2, 0] = 1j
    g[5][1, 2] = g[5][2, 1] = 1
    g[6][1, 2] = -1j
    g[6][2, 1] = 1j
    g[7][0, 0] = g[7][1, 1] = 1 / np.sqrt(3)
    g[7][2, 2] = -2 / np.sqrt(3)
    return g


def _reunitarise(u):
    """Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1): an exact SU(3) matrix."""
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(r0.conj() * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def gauge_field(dims, eps, seed):
    """U = exp(i*eps*X) per link, X = sum_a c_a lambda_a/2 with c_a ~ N(0,1), then
    reunitarised to SU(3).  Returns complex128 [4][V][3][3]."""
    V = volume(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.standard_normal((4, V, 8))
    X = np.einsum("dsa,aij->dsij", c, _gell_mann() / 2)
    w, Q = np.linalg.eigh(X)
    U = np.einsum("dsij,dsj,dskj->dsik", Q, np.exp(1j * eps * w), Q.conj())
    return np.ascontiguousarray(_reunitarise(U))


def gaussian_source(dims, seed, nsrc=None):
    """Complex Gaussian colour-spinor field(s) normalised to unit 2-norm.
    Returns complex128 [V][4][3] (or [nsrc][V][4][3])."""
    V = volume(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (V, 4, 3) if nsrc is None else (nsrc, V, 4, 3)
    x = rng.standard_normal(shape + (2,))
    x = x[..., 0] + 1j * x[..., 1]
    axes = tuple(range(x.ndim - 3, x.ndim))
    x /= np.sqrt(np.sum(np.abs(x) ** 2, axis=axes, keepdims=True))
    return np.ascontiguousarray(x)


def z2_source(dims, seed, nsrc=None):
    """Z2 noise (eta_r + i eta_i)/sqrt(2), eta = +-1, per component (unnormalised:
    every component has modulus 1)."""
    V = volume(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (V, 4, 3) if nsrc is None else (nsrc, V, 4, 3)
    eta = rng.integers(0, 2, size=shape + (2,)) * 2.0 - 1.0
    return np.ascontiguousarray((eta[..., 0] + 1j * eta[..., 1]) / np.sqrt(2.0))


def su3_direction(dims, seed):
    """A global su(3) tangent field: omega^a_nu(x) ~ N(0,1) over all 4V links and 8
    generators, normalised to ||omega||_2 = 1.  Returns float64 [4][V][8]."""
    V = volume(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((4, V, 8))
    return np.ascontiguousarray(w / np.linalg.norm(w))


def u1_direction(dims, seed):
    """A U(1) tangent field theta_nu(x) ~ N(0,1), normalised to unit 2-norm.
    Returns float64 [4][V]."""
    V = volume(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    th = rng.standard_normal((4, V))
    return np.ascontiguousarray(th / np.linalg.norm(th))
