"""Shared test helpers: oracle operator closures and error norms (no method arithmetic)."""
import numpy as np

from oracle import dirac as od


def relerr(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def oracle_ops(dims, U, mu, kind=0, field=None, m_w=-2.0):
    """(lat, A, Ah, E, Eh) closures of the oracle for a derivative direction.
    kind 0: d/dmu; 1: su(3) field [4][V][8]; 2: U(1) field [4][V]."""
    lat = od.Lattice(dims, m_w=m_w)

    def A(v):
        return od.apply_H(lat, U, v, mu).ravel()

    def Ah(v):
        return od.apply_Hdag(lat, U, v, mu).ravel()

    if kind == 0:
        def E(v):
            return od.apply_dH_dmu(lat, U, v, mu).ravel()

        def Eh(v):
            return od.apply_dH_dmu_dag(lat, U, v, mu).ravel()
    else:
        Y = od.link_derivative(U, omega=field) if kind == 1 else od.link_derivative(U, theta=field)

        def E(v):
            return od.apply_dH_dir(lat, U, Y, v, mu).ravel()

        def Eh(v):
            return od.apply_dH_dir_dag(lat, U, Y, v, mu).ravel()
    return lat, A, Ah, E, Eh
