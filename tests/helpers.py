"""Shared test helpers: oracle operator closures and error norms (no method arithmetic)."""
import numpy as np

from oracle import dirac as od


# Parity bounds in units of the oracle's own rounding sensitivity at the same Krylov depth.  The
# non-symmetric Lanczos process amplifies rounding, so two correct implementations differ by about
# the change of the oracle's result under a perturbation of rounding size: 1e-16 relative on the
# input for FP64, 6e-8 relative on every operator application for FP32.  Each factor is about
# 2.7 times the largest ratio (GPU error / that sensitivity) seen on the GB300 over every case of
# the suite: 1.87 for FP64 (a ragged-batch member), 7.3 for the FP32 stencil schedules at k = 40
# (one FP32 rounding per operation against a 6e-8 model of the whole step), 22 for the precision
# workload (8^4, k = 200, mu = 0.1: two hundred steps of that model mismatch, amplified by a process
# far from converged), 6.7 for the scalar S of the adjoint, whose sensitivity is measured on the
# force.
FP64_SENS_FACTOR = 5.0
FP32_SENS_FACTOR = 20.0
FP32_DEEP_SENS_FACTOR = 60.0
ADJ_SENS_FACTOR = 18.0
# float-float: relative noise of one operator application in the oracle's sensitivity runs, 2^-44
# (a float-float result carries a few units of 2^-47 after the sums of a Wilson hop), and the
# factor allowed over the oracle's response to it: about 2.7 times the largest ratio observed on
# the GB300 (2.19, an su(3) direction at k = 60), like the other factors
FF_STEP_NOISE = 2.0 ** -44
FF_SENS_FACTOR = 6.0


def round_bf16(a):
    """Complex FP64 array -> the values of its BF16 storage: each real part rounded to FP32
    (nearest), then to BF16 (8-bit significand, nearest even on the FP32 bit pattern), back to
    FP64 exactly.  An input transformation for the BF16-link tests (no method arithmetic)."""
    a = np.asarray(a, dtype=np.complex128)

    def r(x):
        b = np.ascontiguousarray(x, dtype=np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
        b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
        return b.astype(np.uint32).view(np.float32).astype(np.float64)
    return r(a.real) + 1j * r(a.imag)


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


def oracle_block_tsl_run(job):
    """One oracle block-TSL run (Eq. (2.6), d/dmu) for a process pool, built from seeds so that
    nothing but plain data crosses the process boundary.  job = (dims, eps, gauge_seed,
    source_seed, mu, k, perturbation, perturbation_seed); perturbation None, "input" (1e-16
    relative noise on the source: the FP64 rounding sensitivity), "step" (6e-8 relative noise
    on every operator application: the FP32 sensitivity) or "step_ff" (FF_STEP_NOISE on every
    operator application: the float-float sensitivity).  Returns (d sgn(H) x, sgn(H) x)."""
    import synthetic as syn
    from oracle import tsl as ot
    dims, eps, gseed, sseed, mu, k, pert, pseed = job
    U = syn.gauge_field(dims, eps, gseed)
    x = syn.gaussian_source(dims, sseed, nsrc=1)[0].ravel()
    lat, A, Ah, E, Eh = oracle_ops(dims, U, mu)
    rng = np.random.default_rng(pseed)
    if pert == "input":
        x = x * (1 + 1e-16 * rng.standard_normal(x.shape))
    elif pert in ("step", "step_ff"):
        size = 6e-8 if pert == "step" else FF_STEP_NOISE

        def wrap(op):
            def f(v):
                y = op(v)
                return y * (1 + size * (rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape)) / np.sqrt(2))
            return f
        A, Ah, E, Eh = wrap(A), wrap(Ah), wrap(E), wrap(Eh)
    rd, rs, _ = ot.tsl_sign_derivative(A, Ah, E, Eh, x, k)
    return rd, rs
