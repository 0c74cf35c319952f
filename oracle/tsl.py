"""Oracle: the two-sided Lanczos (TSL) approximation of sgn(A)x and of d_t sgn(A)x.

Test infrastructure only (see the package docstring).

The paper (Sec. 2) names the TSL method and applies it to sgn(A)x and, through
Eq. (2.6), to the block matrix B = [[A, dA], [0, A]] with the sparse source (0, x);
it does not print the recurrences.  The reading used here is the standard
non-symmetric Lanczos process with biorthogonal bases V, W (W^H V = 1) and the
tridiagonal projection T = W^H A V:

  v_1 = w_1 = x / |x|;  for j = 1..k:
    alpha_j = <w_j, A v_j>                                (<a, b> = sum conj(a_i) b_i)
    vh = A v_j - alpha_j v_j - beta_{j-1} v_{j-1}
    wh = A^H w_j - conj(alpha_j) w_j - conj(delta_{j-1}) w_{j-1}
    omega = <wh, vh>;  delta_j = sqrt|omega|;  beta_j = omega / delta_j
    v_{j+1} = vh / delta_j;  w_{j+1} = wh / conj(beta_j)
  T = tridiag(sub = delta, diag = alpha, super = beta);  k = dim T = number of A-applies.
  sgn(A)x ~ |x| V_k sgn(T_k) e_1.

The projected sign sgn(T_k) is evaluated by the ordered-Schur method (oracle.sign),
a different algorithm from the Newton iteration of the CUDA path.  A serious
breakdown |omega| < tol |wh| |vh| stops the process early (k_eff < k), and so does an
invariant subspace (the paper is silent on both): |vh| <= invariant_tol |A v_j| or
|wh| <= invariant_tol |A^H w_j|, where the recurrence has cancelled to rounding.  On an
invariant right subspace A V_j = V_j T_j holds exactly, so f(A)x = |x| V_j f(T_j) e_1 is
then the exact result (a free-field plane wave stops at k_eff = 2).

Re-biorthogonalisation (not in the paper; the remedy for the loss of biorthogonality in finite
precision): with period p, the three-term step that makes v_{j+1}, w_{j+1} (j = 1, 2, ...) is
followed, when j or j - 1 is divisible by p, by a projection of the new pair against all j
earlier pairs before omega is formed,
    vh <- vh - V_j (W_j^H vh),   wh <- wh - W_j (V_j^H wh),
with V_j = [v_1 .. v_j], W_j = [w_1 .. w_j] (W_j^H V_j = 1).  T keeps its three-term entries.
Two consecutive pairs are corrected because the recurrence forms each new pair from the last
two: a lone corrected pair next to an uncorrected one hands the lost biorthogonality straight
to the following vectors (the rule of periodic reorthogonalisation in the symmetric Lanczos
method, Grcar 1981; Simon, Math. Comp. 42 (1984) 115).  p = 1 corrects every pair.
"""
import numpy as np

from .sign import sign_schur


def tsl(apply_A, apply_Ah, v1, w1, k, breakdown_tol=1e-14, rebiorth=0, invariant_tol=1e-10):
    """Run k steps; returns dict(T, V [k_eff][n], W [k_eff][n], k_eff, alpha, beta, delta).
    rebiorth: 0 (off) or the period p of the re-biorthogonalisation (True is p = 1)."""
    period = int(rebiorth)
    V = [np.asarray(v1, dtype=complex)]
    W = [np.asarray(w1, dtype=complex)]
    alpha, beta, delta = [], [], []
    k_eff = k
    for j in range(k):
        Av = apply_A(V[j])
        a = np.vdot(W[j], Av)
        alpha.append(a)
        if j == k - 1:
            break
        Aw = apply_Ah(W[j])
        vh = Av - a * V[j]
        wh = Aw - np.conj(a) * W[j]
        if j > 0:
            vh = vh - beta[j - 1] * V[j - 1]
            wh = wh - np.conj(delta[j - 1]) * W[j - 1]
        if period > 0 and ((j + 1) % period == 0 or (j > 0 and j % period == 0)):
            Vm, Wm = np.array(V), np.array(W)
            vh = vh - Vm.T @ (Wm.conj() @ vh)
            wh = wh - Wm.T @ (Vm.conj() @ wh)
        if (np.linalg.norm(vh) <= invariant_tol * np.linalg.norm(Av)
                or np.linalg.norm(wh) <= invariant_tol * np.linalg.norm(Aw)):
            k_eff = j + 1          # invariant subspace
            break
        om = np.vdot(wh, vh)
        if abs(om) < breakdown_tol * np.linalg.norm(wh) * np.linalg.norm(vh):
            k_eff = j + 1
            break
        d = np.sqrt(abs(om))
        b = om / d
        delta.append(d)
        beta.append(b)
        V.append(vh / d)
        W.append(wh / np.conj(b))
    m = len(alpha)
    T = np.diag(np.array(alpha, dtype=complex))
    if m > 1:
        T += np.diag(np.array(beta[:m - 1], dtype=complex), 1)
        T += np.diag(np.array(delta[:m - 1], dtype=complex), -1)
    return dict(T=T, V=np.array(V[:m]), W=np.array(W[:m]), k_eff=k_eff,
                alpha=np.array(alpha), beta=np.array(beta[:m - 1]), delta=np.array(delta[:m - 1]))


def projected_sign_e1(T):
    """sgn(T) e_1 by the ordered-Schur oracle."""
    return sign_schur(T)[:, 0]


def tsl_sign(apply_A, apply_Ah, x, k, **kw):
    """sgn(A)x ~ |x| V_k sgn(T_k) e_1 (Sec. 2)."""
    x = np.asarray(x, dtype=complex).ravel()
    nx = np.linalg.norm(x)
    r = tsl(apply_A, apply_Ah, x / nx, x / nx, k, **kw)
    c = projected_sign_e1(r["T"])
    return nx * (r["V"].T @ c), r


def block_ops(apply_A, apply_Ah, apply_E, apply_Eh, n):
    """B = [[A, E], [0, A]] and B^H = [[A^H, 0], [E^H, A^H]] on stacked (top, bottom) vectors."""
    def B(tb):
        t, b = tb[:n], tb[n:]
        return np.concatenate([apply_A(t) + apply_E(b), apply_A(b)])

    def Bh(tb):
        t, b = tb[:n], tb[n:]
        return np.concatenate([apply_Ah(t), apply_Eh(t) + apply_Ah(b)])
    return B, Bh


def tsl_resolvent(apply_A, apply_Ah, b, sigma, k, **kw):
    """(sigma - A)^{-1} b ~ |b| V_k (sigma - T_k)^{-1} e_1: the TSL approximation of Sec. 2 for
    f(a) = 1/(sigma - a) (the projected system solved densely)."""
    b = np.asarray(b, dtype=complex).ravel()
    nb = np.linalg.norm(b)
    r = tsl(apply_A, apply_Ah, b / nb, b / nb, k, **kw)
    e1 = np.zeros(r["T"].shape[0], complex)
    e1[0] = 1.0
    c = np.linalg.solve(sigma * np.eye(len(e1)) - r["T"], e1)
    return nb * (r["V"].T @ c), r


def tsl_sign_block(apply_A, apply_Ah, apply_E, apply_Eh, t0, b0, k, **kw):
    """sgn(B)(t0, b0) by the TSL on the block operator B of Eq. (2.5) from v_1 = (t0, b0)/|(t0, b0)|
    with the left start w_1 proportional to (b0, b0), normalised to <w_1, v_1> = 1 (the reading
    that reduces to (x, x)/|x| for the sparse source (0, x) of Eq. (2.6)).  Returns (top, bottom, record)."""
    t0 = np.asarray(t0, dtype=complex).ravel()
    b0 = np.asarray(b0, dtype=complex).ravel()
    n = b0.size
    B, Bh = block_ops(apply_A, apply_Ah, apply_E, apply_Eh, n)
    psi = np.concatenate([t0, b0])
    npsi = np.linalg.norm(psi)
    v1 = psi / npsi
    w1 = np.concatenate([b0, b0])
    w1 = w1 / np.conj(np.vdot(w1, v1))
    r = tsl(B, Bh, v1, w1, k, **kw)
    c = projected_sign_e1(r["T"])
    y = npsi * (r["V"].T @ c)
    return y[:n], y[n:], r


def tsl_sign_derivative(apply_A, apply_Ah, apply_E, apply_Eh, x, k, left_start="xx", **kw):
    """Eq. (2.6): sgn(B)(0, x) = (d_t sgn(A) x, sgn(A) x), with the TSL applied to the
    2n x 2n block operator B of Eq. (2.5) from the right start v_1 = (0, x)/|x|.

    The paper does not fix the left start vector.  The reading used here is
    w_1 = (x, x)/|x| (so that <w_1, v_1> = 1).  The alternative w_1 = v_1 = (0, x)/|x|
    keeps every left vector in {0} x C^n, which reduces the process to TSL(A) and lets
    the top block grow without bound as Ritz values converge (numerically unstable);
    it is kept as left_start="zero-top" for the tests that document this.
    Returns (d_t sgn(A) x, sgn(A) x, tsl-record)."""
    x = np.asarray(x, dtype=complex).ravel()
    n = x.size
    B, Bh = block_ops(apply_A, apply_Ah, apply_E, apply_Eh, n)
    nx = np.linalg.norm(x)
    v1 = np.concatenate([np.zeros(n, complex), x]) / nx
    if left_start == "xx":
        w1 = np.concatenate([x, x]) / nx
    elif left_start == "zero-top":
        w1 = v1.copy()
    else:
        raise ValueError(left_start)
    r = tsl(B, Bh, v1, w1, k, **kw)
    c = projected_sign_e1(r["T"])
    y = nx * (r["V"].T @ c)
    return y[:n], y[n:], r


def error_estimate(apply_A, apply_Ah, psi, k, **kw):
    """eps_A = ||sgn(A)^2 psi - psi|| / (2 ||psi||), two TSL applications (Sec. 4)."""
    psi = np.asarray(psi, dtype=complex).ravel()
    y1, _ = tsl_sign(apply_A, apply_Ah, psi, k, **kw)
    y2, _ = tsl_sign(apply_A, apply_Ah, y1, k, **kw)
    return np.linalg.norm(y2 - psi) / (2 * np.linalg.norm(psi))


def error_estimate_derivative(apply_A, apply_Ah, apply_E, apply_Eh, phi, k, **kw):
    """The derivative version of eps_A (Sec. 4): B in place of A and (0, phi) in place
    of psi.  The second application acts on the non-sparse (y_d, y_s) = sgn(B)(0, phi);
    by linearity sgn(B)(y_d, y_s) = (sgn(A) y_d + d_t sgn(A) y_s, sgn(A) y_s), and each
    term is one TSL approximation (sign of y_d; derivative solve from y_s)."""
    phi = np.asarray(phi, dtype=complex).ravel()
    yd, ys, _ = tsl_sign_derivative(apply_A, apply_Ah, apply_E, apply_Eh, phi, k, **kw)
    zd, zs, _ = tsl_sign_derivative(apply_A, apply_Ah, apply_E, apply_Eh, ys, k, **kw)
    sd, _ = tsl_sign(apply_A, apply_Ah, yd, k, **kw)
    top = sd + zd
    bot = zs - phi
    return np.sqrt(np.linalg.norm(top) ** 2 + np.linalg.norm(bot) ** 2) / (2 * np.linalg.norm(phi))
