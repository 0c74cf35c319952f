"""Oracle pin: closed forms for the free field U = 1 in momentum space.

Test infrastructure only (see the package docstring).

For U = 1 a plane wave exp(i p.x) chi is an eigenfunction of every hop.  With
p_k = 2 pi n_k / N_k in space and p_t = 2 pi (n_t + 1/2) / N_t (antiperiodic time), and
the shifted temporal momentum pt~ = p_t - i mu, the Wilson operator of Sec. 1 becomes
  D(p) = M(p) + i sum_nu gamma_nu sin(p~_nu),   M(p) = m_w + r sum_nu (1 - cos p~_nu),
and H(p) = gamma5 D(p) squares to the scalar z(p) = M^2 + sum_nu sin^2(p~_nu) (the
gamma matrices anticommute).  Hence sgn(H(p)) = H(p) z(p)^{-1/2} with the principal
square root (Re sqrt > 0), valid while no eigenvalue sits on the imaginary axis, and
its mu-derivative follows by differentiating with d p~_t / d mu = -i.
"""
import numpy as np

from .dirac import gammas


def _momenta(lat):
    pt = 2 * np.pi * np.fft.fftfreq(lat.nt) + (np.pi / lat.nt if lat.apbc else 0.0)
    pz = 2 * np.pi * np.fft.fftfreq(lat.nz)
    py = 2 * np.pi * np.fft.fftfreq(lat.ny)
    px = 2 * np.pi * np.fft.fftfreq(lat.nx)
    return np.meshgrid(pt, pz, py, px, indexing="ij")


def _symbols(lat, mu):
    g, g5 = gammas()
    pt, pz, py, px = _momenta(lat)
    ps = [px, py, pz, pt - 1j * mu]
    s = [np.sin(p) for p in ps]
    c = [np.cos(p) for p in ps]
    M = lat.m_w + lat.r * sum(1 - ci for ci in c)
    D = M[..., None, None] * np.eye(4) + 1j * sum(si[..., None, None] * g[nu] for nu, si in enumerate(s))
    H = np.einsum("st,...tu->...su", g5, D)
    z = M ** 2 + sum(si ** 2 for si in s)
    # mu-derivatives (d p~_t / d mu = -i)
    dM = lat.r * s[3] * (-1j)
    dD = dM[..., None, None] * np.eye(4) + 1j * g[3] * (c[3] * (-1j))[..., None, None]
    dH = np.einsum("st,...tu->...su", g5, dD)
    dz = 2 * M * dM + 2 * s[3] * c[3] * (-1j)
    return H, z, dH, dz


def _apply_symbol(lat, sym, psi):
    """psi(x) = exp(i pi t / N_t) phi(x) with phi periodic; multiply phi~(p) by sym(p)."""
    grid = lat.grid(psi)
    t = np.arange(lat.nt)
    tw = np.exp(1j * np.pi * t / lat.nt) if lat.apbc else np.ones(lat.nt)
    phi = grid / tw[:, None, None, None, None, None]
    phik = np.fft.fftn(phi, axes=(0, 1, 2, 3))
    outk = np.einsum("...st,...tc->...sc", sym, phik)
    out = np.fft.ifftn(outk, axes=(0, 1, 2, 3)) * tw[:, None, None, None, None, None]
    return lat.flat(out)


def free_H(lat, psi, mu):
    H, _, _, _ = _symbols(lat, mu)
    return _apply_symbol(lat, H, psi)


def free_sign(lat, psi, mu):
    """sgn(H(mu)) psi for U = 1: H(p) / sqrt(z(p))."""
    H, z, _, _ = _symbols(lat, mu)
    return _apply_symbol(lat, H / np.sqrt(z)[..., None, None], psi)


def free_sign_dmu(lat, psi, mu):
    """d/dmu sgn(H(mu)) psi for U = 1: dH z^{-1/2} - H dz z^{-3/2} / 2."""
    H, z, dH, dz = _symbols(lat, mu)
    sym = dH / np.sqrt(z)[..., None, None] - 0.5 * H * (dz / z ** 1.5)[..., None, None]
    return _apply_symbol(lat, sym, psi)


def free_spectrum(lat, mu):
    """Eigenvalues of H(mu) at U = 1: +-sqrt(z(p)), each with multiplicity 2 x 3 colours."""
    _, z, _, _ = _symbols(lat, mu)
    r = np.sqrt(z).ravel()
    return np.concatenate([r, -r])
