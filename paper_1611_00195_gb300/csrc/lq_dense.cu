// Small dense complex linear algebra on the host (the Rayleigh-Ritz steps of the eigensolver for
// the deflation space): the eigen-decomposition of a general complex matrix by Householder
// reduction to Hessenberg form and the shifted QR algorithm (Golub & Van Loan, "Matrix
// Computations", ch. 7: complex Schur form with Wilkinson shifts, eigenvectors by back
// substitution on the triangular factor), plus Cholesky and triangular solves.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "../../include/lq.h"
#include "lq_dense.h"

namespace lq {

using cd = std::complex<double>;

namespace {

// A (n x n, row-major) -> Hessenberg H = Q^H A Q, Q accumulated.
void hessenberg(int n, std::vector<cd>& A, std::vector<cd>& Q) {
    for (int k = 0; k + 2 < n; ++k) {
        double nx = 0.0;
        for (int i = k + 1; i < n; ++i) nx += std::norm(A[i * n + k]);
        nx = std::sqrt(nx);
        if (nx == 0.0) continue;
        const cd x0 = A[(k + 1) * n + k];
        const cd ph = (std::abs(x0) > 0.0) ? x0 / std::abs(x0) : cd(1.0, 0.0);
        std::vector<cd> v(n, 0.0);
        for (int i = k + 1; i < n; ++i) v[i] = A[i * n + k];
        v[k + 1] += ph * nx;                    // v = x + e^{i arg x0} |x| e_1
        double vv = 0.0;
        for (int i = k + 1; i < n; ++i) vv += std::norm(v[i]);
        if (vv == 0.0) continue;
        // A <- (I - 2 v v^H / vv) A
        for (int j = 0; j < n; ++j) {
            cd s = 0.0;
            for (int i = k + 1; i < n; ++i) s += std::conj(v[i]) * A[i * n + j];
            s *= 2.0 / vv;
            for (int i = k + 1; i < n; ++i) A[i * n + j] -= v[i] * s;
        }
        // A <- A (I - 2 v v^H / vv), Q <- Q (I - 2 v v^H / vv)
        for (int i = 0; i < n; ++i) {
            cd s = 0.0, t = 0.0;
            for (int j = k + 1; j < n; ++j) { s += A[i * n + j] * v[j]; t += Q[i * n + j] * v[j]; }
            s *= 2.0 / vv;
            t *= 2.0 / vv;
            for (int j = k + 1; j < n; ++j) { A[i * n + j] -= s * std::conj(v[j]); Q[i * n + j] -= t * std::conj(v[j]); }
        }
    }
}

// Givens rotation [c s; -conj(s) c] with c real that zeroes b in (a, b)^T.
void givens(cd a, cd b, double& c, cd& s) {
    const double na = std::abs(a), nb = std::abs(b);
    if (nb == 0.0) { c = 1.0; s = 0.0; return; }
    if (na == 0.0) { c = 0.0; s = std::conj(b) / nb; return; }
    const double r = std::hypot(na, nb);
    c = na / r;
    s = (a / na) * std::conj(b) / r;
}

}  // namespace

int dense_eig(int n, const cd* Ain, cd* w, cd* Vr) {
    if (n <= 0) return LQ_ERR_ARG;
    std::vector<cd> A(Ain, Ain + (size_t)n * n), Q((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
    hessenberg(n, A, Q);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j + 1 < i; ++j) A[i * n + j] = 0.0;
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, iter = 0, total = 0;
    while (hi > 0) {
        // find the start of the unreduced block ending at hi
        int l = hi;
        while (l > 0) {
            const double s = std::abs(A[(l - 1) * n + l - 1]) + std::abs(A[l * n + l]);
            if (std::abs(A[l * n + l - 1]) <= eps * (s > 0.0 ? s : 1.0)) { A[l * n + l - 1] = 0.0; break; }
            --l;
        }
        if (l == hi) { --hi; iter = 0; continue; }
        if (++total > 100 * n) return LQ_ERR_NEWTON;   // no convergence
        ++iter;
        // Wilkinson shift: eigenvalue of the trailing 2x2 closest to A[hi][hi]
        const cd a = A[(hi - 1) * n + hi - 1], b = A[(hi - 1) * n + hi], c = A[hi * n + hi - 1], d = A[hi * n + hi];
        const cd tr = a + d, det = a * d - b * c;
        const cd disc = std::sqrt(tr * tr / 4.0 - det);
        const cd e1 = tr / 2.0 + disc, e2 = tr / 2.0 - disc;
        cd mu = (std::abs(e1 - d) < std::abs(e2 - d)) ? e1 : e2;
        if (iter % 11 == 10) mu = d + cd(std::abs(A[hi * n + hi - 1]), 0.0) * 0.75;   // exceptional shift
        // explicit shifted QR step on rows/cols l..hi via Givens rotations
        std::vector<double> cs(hi - l);
        std::vector<cd> sn(hi - l);
        for (int k = l; k <= hi; ++k) A[k * n + k] -= mu;
        for (int k = l; k < hi; ++k) {
            double cc;
            cd ss;
            givens(A[k * n + k], A[(k + 1) * n + k], cc, ss);
            cs[k - l] = cc;
            sn[k - l] = ss;
            for (int j = k; j < n; ++j) {       // rows k, k+1 (left multiplication by G^H)
                const cd x = A[k * n + j], y = A[(k + 1) * n + j];
                A[k * n + j] = cc * x + ss * y;
                A[(k + 1) * n + j] = -std::conj(ss) * x + cc * y;
            }
        }
        for (int k = l; k < hi; ++k) {
            const double cc = cs[k - l];
            const cd ss = sn[k - l];
            const int rmax = std::min(k + 2, hi);
            for (int i = 0; i <= rmax; ++i) {    // columns k, k+1 (right multiplication by G)
                const cd x = A[i * n + k], y = A[i * n + k + 1];
                A[i * n + k] = cc * x + std::conj(ss) * y;
                A[i * n + k + 1] = -ss * x + cc * y;
            }
            for (int i = 0; i < n; ++i) {
                const cd x = Q[i * n + k], y = Q[i * n + k + 1];
                Q[i * n + k] = cc * x + std::conj(ss) * y;
                Q[i * n + k + 1] = -ss * x + cc * y;
            }
        }
        for (int k = l; k <= hi; ++k) A[k * n + k] += mu;
    }
    for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
    if (Vr) {
        // eigenvectors of the triangular T: T x = t_ii x, then v = Q x
        std::vector<cd> x(n);
        double tn = 0.0;
        for (int i = 0; i < n * n; ++i) tn = std::max(tn, std::abs(A[i]));
        const double small = eps * (tn > 0.0 ? tn : 1.0);
        for (int i = 0; i < n; ++i) {
            std::fill(x.begin(), x.end(), cd(0.0));
            x[i] = 1.0;
            for (int j = i - 1; j >= 0; --j) {
                cd s = 0.0;
                for (int m = j + 1; m <= i; ++m) s += A[j * n + m] * x[m];
                cd den = A[j * n + j] - A[i * n + i];
                if (std::abs(den) < small) den = small;
                x[j] = -s / den;
            }
            double nv = 0.0;
            for (int r = 0; r < n; ++r) {
                cd s = 0.0;
                for (int m = 0; m <= i; ++m) s += Q[r * n + m] * x[m];
                Vr[r * n + i] = s;
                nv += std::norm(s);
            }
            nv = std::sqrt(nv);
            for (int r = 0; r < n; ++r) Vr[r * n + i] /= nv;
        }
    }
    return LQ_OK;
}

int dense_cholesky(int n, cd* G) {   // lower factor in place (row-major), upper part zeroed
    for (int j = 0; j < n; ++j) {
        double d = G[j * n + j].real();
        for (int m = 0; m < j; ++m) d -= std::norm(G[j * n + m]);
        if (!(d > 0.0)) return LQ_ERR_BREAKDOWN;
        const double ljj = std::sqrt(d);
        G[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            cd s = G[i * n + j];
            for (int m = 0; m < j; ++m) s -= G[i * n + m] * std::conj(G[j * n + m]);
            G[i * n + j] = s / ljj;
        }
        for (int i = 0; i < j; ++i) G[i * n + j] = 0.0;
    }
    return LQ_OK;
}

int dense_inverse(int n, cd* A) {   // Gauss-Jordan with partial pivoting, in place
    std::vector<int> piv(n);
    for (int p = 0; p < n; ++p) {
        int r = p;
        for (int i = p + 1; i < n; ++i) if (std::abs(A[i * n + p]) > std::abs(A[r * n + p])) r = i;
        piv[p] = r;
        if (std::abs(A[r * n + p]) == 0.0) return LQ_ERR_BREAKDOWN;
        if (r != p) for (int j = 0; j < n; ++j) std::swap(A[p * n + j], A[r * n + j]);
        const cd inv = 1.0 / A[p * n + p];
        A[p * n + p] = 1.0;
        for (int j = 0; j < n; ++j) A[p * n + j] *= inv;
        for (int i = 0; i < n; ++i) {
            if (i == p) continue;
            const cd f = A[i * n + p];
            A[i * n + p] = 0.0;
            for (int j = 0; j < n; ++j) A[i * n + j] -= f * A[p * n + j];
        }
    }
    for (int p = n - 1; p >= 0; --p)
        if (piv[p] != p) for (int i = 0; i < n; ++i) std::swap(A[i * n + p], A[i * n + piv[p]]);
    return LQ_OK;
}

}  // namespace lq

extern "C" int lq_dense_eig(int n, const double* A, double* w, double* V) {
    if (n < 1 || !A || !w) return LQ_ERR_ARG;
    return lq::dense_eig(n, reinterpret_cast<const lq::cd*>(A), reinterpret_cast<lq::cd*>(w), reinterpret_cast<lq::cd*>(V));
}
