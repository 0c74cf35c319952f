// Batched FP64 matrix sign by the scaled Newton iteration (Higham 2008, ch. 5):
//     X_0 = T,   X_{i+1} = (m_i X_i + (m_i X_i)^{-1}) / 2,   m_i = sqrt(||X_i^{-1}||_F / ||X_i||_F),
// the projected step sgn(T_k) e_1 of the two-sided Lanczos approximation (Sec. 2).
// Norm scaling is switched off once the relative change drops below 1e-2; the iteration
// stops when the relative Frobenius change is <= tol, or when (unscaled) it no longer
// decreases quadratically below 1e-6 (rounding floor), or at max_iter (status LQ_ERR_NEWTON).
//
// The inverse is an in-place Gauss-Jordan elimination with partial (row) pivoting over the
// whole device: one launch per pivot step eliminates column p from every other row of every
// matrix in the batch; the block that finishes last for a matrix (atomic counter) chooses and
// normalises the next pivot row.  After k steps the row interchanges are undone by column
// interchanges in reverse order.
#include "lq_internal.cuh"
#include "lq_launch.h"

#include <cstring>

namespace lq {

constexpr int kNtThreads = 256;

__device__ __forceinline__ bool nt_last_block(int* counter, int nblocks) {
    __shared__ int is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int prev = atomicAdd(counter, 1);
        is_last = (prev == nblocks - 1);
        if (is_last) *counter = 0;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last != 0;
}

__device__ __forceinline__ double2 ld2cg(const double2* p) { return __ldcg(p); }

// Pivot step p on matrix b, executed by a single block after every elimination of step p-1
// is visible: choose the row r >= p with the largest |Y[r][p]|, swap rows p and r, scale row p
// so that its pivot entry holds 1/piv (in-place inverse), store the column-p multipliers in F
// and clear column p below/above the pivot.
__device__ void nt_pivot(const NewtonArgs& a, int b, int p) {
    __shared__ double sval[kNtThreads];
    __shared__ int sidx[kNtThreads];
    __shared__ double2 spiv;
    const int k = a.k, ld = a.ld;
    double2* Y = a.Y + (size_t)b * ld * ld;
    double2* F = a.F + (size_t)b * ld;
    double best = -1.0;
    int bi = p;
    for (int i = p + threadIdx.x; i < k; i += blockDim.x) {
        double2 v = ld2cg(Y + (size_t)i * ld + p);
        double m = v.x * v.x + v.y * v.y;
        if (m > best) { best = m; bi = i; }
    }
    sval[threadIdx.x] = best;
    sidx[threadIdx.x] = bi;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            double o = sval[threadIdx.x + off];
            int oi = sidx[threadIdx.x + off];
            if (o > sval[threadIdx.x] || (o == sval[threadIdx.x] && oi < sidx[threadIdx.x])) {
                sval[threadIdx.x] = o;
                sidx[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const int r = sidx[0];
    if (threadIdx.x == 0) a.perm[(size_t)b * ld + p] = r;
    if (r != p) {
        for (int c = threadIdx.x; c < k; c += blockDim.x) {
            double2 t = ld2cg(Y + (size_t)p * ld + c);
            Y[(size_t)p * ld + c] = ld2cg(Y + (size_t)r * ld + c);
            Y[(size_t)r * ld + c] = t;
        }
    }
    __threadfence_block();
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 piv = ld2cg(Y + (size_t)p * ld + p);
        double n = piv.x * piv.x + piv.y * piv.y;
        if (!(n > 0.0) || !isfinite(n)) {
            a.scal[b * 16 + NS_STATUS] = (double)LQ_ERR_NEWTON;
            spiv = make_double2(1.0, 0.0);
        } else {
            spiv = make_double2(piv.x / n, -piv.y / n);   // 1/piv
        }
    }
    __syncthreads();
    const double2 inv = spiv;
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double2 v = (c == p) ? make_double2(1.0, 0.0) : ld2cg(Y + (size_t)p * ld + c);
        Y[(size_t)p * ld + c] = cmul(v, inv);
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        if (i == p) { F[i] = make_double2(0.0, 0.0); continue; }
        F[i] = ld2cg(Y + (size_t)i * ld + p);
        Y[(size_t)i * ld + p] = make_double2(0.0, 0.0);
    }
}

__device__ __forceinline__ bool nt_done(const NewtonArgs& a, int b) { return a.scal[b * 16 + NS_DONE] != 0.0; }

// X_0 = T_k from the Lanczos coefficients (identity padding beyond k_eff).
__global__ void k_nt_init_tridiag(NewtonArgs a) {
    const int b = blockIdx.y;
    const int k = a.k, ld = a.ld;
    const int keff = a.state[b].k_eff;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e == 0) {
        double* s = a.scal + b * 16;
        for (int i = 0; i < 16; ++i) s[i] = 0.0;
        s[NS_SCALING] = 1.0;
        s[NS_PREVCHANGE] = 1e300;
        s[NS_KEFF] = keff;
        if (keff <= 0) { s[NS_DONE] = 1.0; s[NS_STATUS] = (double)LQ_ERR_NOT_READY; }
    }
    if (e >= (size_t)k * k) return;
    const int i = (int)(e / k), c = (int)(e % k);
    double2 v = make_double2(0.0, 0.0);
    if (i < keff && c < keff) {
        if (i == c) v = a.alpha[(size_t)b * a.kmax + i];
        else if (c == i + 1) v = a.beta[(size_t)b * a.kmax + i];
        else if (i == c + 1) v = make_double2(a.delta[(size_t)b * a.kmax + c], 0.0);
    } else if (i == c) {
        v = make_double2(1.0, 0.0);
    }
    a.X[(size_t)b * ld * ld + (size_t)i * ld + c] = v;
}

__global__ void k_nt_init_dense(NewtonArgs a, const double2* __restrict__ Xin) {
    const int b = blockIdx.y;
    const int k = a.k, ld = a.ld;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e == 0) {
        double* s = a.scal + b * 16;
        for (int i = 0; i < 16; ++i) s[i] = 0.0;
        s[NS_SCALING] = 1.0;
        s[NS_PREVCHANGE] = 1e300;
        s[NS_KEFF] = k;
    }
    if (e >= (size_t)k * k) return;
    const int i = (int)(e / k), c = (int)(e % k);
    a.X[(size_t)b * ld * ld + (size_t)i * ld + c] = Xin[(size_t)b * k * k + e];
}

// Y = X, ||X||_F^2; last block pivots step 0.
__global__ void __launch_bounds__(kNtThreads) k_nt_copy(NewtonArgs a) {
    __shared__ CSum smem[32];
    const int b = blockIdx.y;
    if (nt_done(a, b)) return;
    const int k = a.k, ld = a.ld;
    CSum acc{0.0, 0.0};
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (size_t)k * k) {
        const size_t o = (size_t)b * ld * ld + (e / k) * ld + (e % k);
        double2 v = a.X[o];
        a.Y[o] = v;
        cs_add_prod(acc, v.x, v.x);
        cs_add_prod(acc, v.y, v.y);
    }
    CSum v1[1] = {acc};
    block_reduce_cs<1>(v1, smem);
    double* part = a.partials + ((size_t)b * a.partial_stride + blockIdx.x) * 2;
    if (threadIdx.x == 0) { part[0] = v1[0].s; part[1] = v1[0].e; }
    if (nt_last_block(a.counters + b, gridDim.x)) {
        CSum t{0.0, 0.0};
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
            CSum p; p.s = __ldcg(a.partials + ((size_t)b * a.partial_stride + i) * 2); p.e = __ldcg(a.partials + ((size_t)b * a.partial_stride + i) * 2 + 1);
            t = cs_merge(t, p);
        }
        CSum tv[1] = {t};
        block_reduce_cs<1>(tv, smem);
        if (threadIdx.x == 0) a.scal[b * 16 + NS_NORMX] = sqrt(tv[0].s + tv[0].e);
        __syncthreads();
        nt_pivot(a, b, 0);
    }
}

// Eliminate column p from every row i != p: Y[i][c] -= F[i] * Y[p][c].  Last block pivots p+1.
__global__ void __launch_bounds__(kNtThreads) k_nt_elim(NewtonArgs a, int p) {
    const int b = blockIdx.y;
    if (nt_done(a, b)) return;
    const int k = a.k, ld = a.ld;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (size_t)k * k) {
        const int i = (int)(e / k), c = (int)(e % k);
        if (i != p) {
            double2* Y = a.Y + (size_t)b * ld * ld;
            const double2 f = a.F[(size_t)b * ld + i];
            const double2 pr = Y[(size_t)p * ld + c];
            double2 y = Y[(size_t)i * ld + c];
            y.x = fma(-f.x, pr.x, y.x); y.x = fma(f.y, pr.y, y.x);
            y.y = fma(-f.x, pr.y, y.y); y.y = fma(-f.y, pr.x, y.y);
            Y[(size_t)i * ld + c] = y;
        }
    }
    if (p + 1 < k && nt_last_block(a.counters + b, gridDim.x)) nt_pivot(a, b, p + 1);
}

// Undo the row interchanges (column swaps in reverse order, one thread per row) and
// accumulate ||X^{-1}||_F^2; the last block sets the scaling m.
__global__ void __launch_bounds__(kNtThreads) k_nt_unscramble(NewtonArgs a) {
    __shared__ CSum smem[32];
    const int b = blockIdx.y;
    if (nt_done(a, b)) return;
    const int k = a.k, ld = a.ld;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    CSum acc{0.0, 0.0};
    if (i < k) {
        double2* row = a.Y + (size_t)b * ld * ld + (size_t)i * ld;
        const int* perm = a.perm + (size_t)b * ld;
        for (int p = k - 1; p >= 0; --p) {
            int r = perm[p];
            if (r != p) { double2 t = row[p]; row[p] = row[r]; row[r] = t; }
        }
        for (int c = 0; c < k; ++c) { double2 v = row[c]; cs_add_prod(acc, v.x, v.x); cs_add_prod(acc, v.y, v.y); }
    }
    CSum v1[1] = {acc};
    block_reduce_cs<1>(v1, smem);
    double* part = a.partials + ((size_t)b * a.partial_stride + blockIdx.x) * 2;
    if (threadIdx.x == 0) { part[0] = v1[0].s; part[1] = v1[0].e; }
    if (nt_last_block(a.counters + a.nb + b, gridDim.x)) {
        CSum t{0.0, 0.0};
        for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) {
            CSum p; p.s = __ldcg(a.partials + ((size_t)b * a.partial_stride + q) * 2); p.e = __ldcg(a.partials + ((size_t)b * a.partial_stride + q) * 2 + 1);
            t = cs_merge(t, p);
        }
        CSum tv[1] = {t};
        block_reduce_cs<1>(tv, smem);
        if (threadIdx.x == 0) {
            double* s = a.scal + b * 16;
            const double ny = sqrt(tv[0].s + tv[0].e);
            s[NS_NORMY] = ny;
            s[NS_MU] = (s[NS_SCALING] != 0.0) ? sqrt(ny / s[NS_NORMX]) : 1.0;
        }
    }
}

// X_{i+1} = (m X + Y / m) / 2 with change / norm partials; last block updates the state.
__global__ void __launch_bounds__(kNtThreads) k_nt_combine(NewtonArgs a) {
    __shared__ CSum smem[32 * 2];
    const int b = blockIdx.y;
    if (nt_done(a, b)) return;
    const int k = a.k, ld = a.ld;
    const double m = a.scal[b * 16 + NS_MU];
    const double h1 = 0.5 * m, h2 = 0.5 / m;
    CSum acc[2] = {{0.0, 0.0}, {0.0, 0.0}};
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (size_t)k * k) {
        const size_t o = (size_t)b * ld * ld + (e / k) * ld + (e % k);
        const double2 x = a.X[o], y = a.Y[o];
        const double2 xn = make_double2(h1 * x.x + h2 * y.x, h1 * x.y + h2 * y.y);
        a.X[o] = xn;
        const double dx = xn.x - x.x, dy = xn.y - x.y;
        cs_add_prod(acc[0], dx, dx); cs_add_prod(acc[0], dy, dy);
        cs_add_prod(acc[1], xn.x, xn.x); cs_add_prod(acc[1], xn.y, xn.y);
    }
    block_reduce_cs<2>(acc, smem);
    double* part = a.partials + ((size_t)b * a.partial_stride + blockIdx.x) * 4;
    if (threadIdx.x == 0) { part[0] = acc[0].s; part[1] = acc[0].e; part[2] = acc[1].s; part[3] = acc[1].e; }
    if (nt_last_block(a.counters + 2 * a.nb + b, gridDim.x)) {
        CSum t[2] = {{0.0, 0.0}, {0.0, 0.0}};
        for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x)
            for (int v = 0; v < 2; ++v) {
                CSum p; p.s = __ldcg(a.partials + ((size_t)b * a.partial_stride + q) * 4 + 2 * v); p.e = __ldcg(a.partials + ((size_t)b * a.partial_stride + q) * 4 + 2 * v + 1);
                t[v] = cs_merge(t[v], p);
            }
        block_reduce_cs<2>(t, smem);
        if (threadIdx.x == 0) {
            double* s = a.scal + b * 16;
            const double ch = sqrt(t[0].s + t[0].e) / sqrt(t[1].s + t[1].e);
            const double prev = s[NS_PREVCHANGE];
            s[NS_ITERS] += 1.0;
            s[NS_CHANGE] = ch;
            const bool scaled = s[NS_SCALING] != 0.0;
            bool done = false;
            if (!isfinite(ch)) { s[NS_STATUS] = (double)LQ_ERR_NONFINITE; done = true; }
            else if (ch <= a.tol) done = true;
            else if (!scaled && ch < 1e-6 && ch > 0.5 * prev) done = true;   // rounding floor
            if (scaled && ch < 1e-2) s[NS_SCALING] = 0.0;
            s[NS_PREVCHANGE] = ch;
            if (!done && s[NS_ITERS] >= a.max_iter) { s[NS_STATUS] = (double)LQ_ERR_NEWTON; done = true; }
            if (s[NS_STATUS] != 0.0) done = true;
            if (done) s[NS_DONE] = 1.0;
        }
    }
}

__global__ void k_nt_copy_out(NewtonArgs a, double2* __restrict__ S) {
    const int b = blockIdx.y;
    const int k = a.k, ld = a.ld;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)k * k) return;
    S[(size_t)b * k * k + e] = a.X[(size_t)b * ld * ld + (e / k) * ld + (e % k)];
}

// ---------------------------------------------------------------------------------------------
// Projected sign by quadrature (an alternative to Newton, checked by the involution residual).
// For T without eigenvalues on the imaginary axis,
//     sgn(T) = (2/pi) T int_0^inf (t^2 + T^2)^{-1} dt,
// and with t = c tan(theta) the integrand becomes pi-periodic and analytic in theta, so the
// midpoint rule with N nodes theta_j = (j + 1/2) pi / (2N) converges geometrically:
//     sgn(T) b ~ (c / 2N) sum_j cos(theta_j)^{-2} [ (T + i tau_j)^{-1} + (T - i tau_j)^{-1} ] b,
//     tau_j = c tan(theta_j).
// Each term is one complex tridiagonal solve (Gaussian elimination with partial pivoting,
// O(k)).  One thread per (node, sign), kQuadBlk of them per block and as many blocks per source
// as the node count needs, so that the FP64 work of a batch spreads over the whole GPU; the U
// factors live in a [row][term] scratch so that a warp's accesses at one row are contiguous.
// Each block sums its terms row by row; a second kernel adds the blocks in a fixed order.
// ---------------------------------------------------------------------------------------------
// Solve (T + shift) x = b for the tridiagonal T (sub-diagonal de real, diagonal al, super-
// diagonal be) by Gaussian elimination with partial pivoting (row interchanges create a second
// super-diagonal).  b(i) is read in row order, so the right-hand side may alias sx.  Per row the
// reciprocal of the pivot goes to sd, the U entries right of it to s1/s2 and the eliminated
// right-hand side to sx; w * x overwrites sx, all at stride ld.  One real division per row.
template <class RHS>
__device__ __forceinline__ void tri_solve(const double2* __restrict__ al, const double2* __restrict__ be,
                                          const double* __restrict__ de, int n, double2 shift, RHS b,
                                          double2* sd, double2* s1, double2* s2, double2* sx, size_t ld, double w) {
    auto D = [&](int i) -> double2 { double2 v = al[i]; v.x += shift.x; v.y += shift.y; return v; };
    auto recip = [](double2 z) -> double2 { const double r = 1.0 / (z.x * z.x + z.y * z.y); return make_double2(z.x * r, -z.y * r); };
    double2 cd = D(0), cu = (n > 1) ? be[0] : make_double2(0.0, 0.0), cx = b(0);
    for (int i = 0; i < n - 1; ++i) {
        const double l = de[i];
        const double2 nd = D(i + 1);
        const double2 nu = (i + 1 < n - 1) ? be[i + 1] : make_double2(0.0, 0.0);
        const double2 nx = b(i + 1);
        const size_t o = (size_t)i * ld;
        if (l * l > cd.x * cd.x + cd.y * cd.y) {
            // pivot on the sub-diagonal row: stored row i = (l, nd, nu | nx)
            const double rl = 1.0 / l;
            const double2 f = cscale(cd, rl);
            sd[o] = make_double2(rl, 0.0); s1[o] = nd; s2[o] = nu; sx[o] = nx;
            const double2 ncd = csub(cu, cmul(f, nd));
            const double2 ncu = make_double2(-(f.x * nu.x - f.y * nu.y), -(f.x * nu.y + f.y * nu.x));
            cx = csub(cx, cmul(f, nx));
            cd = ncd;
            cu = ncu;
        } else {
            const double2 rc = recip(cd);
            const double2 f = cscale(rc, l);
            sd[o] = rc; s1[o] = cu; s2[o] = make_double2(0.0, 0.0); sx[o] = cx;
            cd = csub(nd, cmul(f, cu));
            cu = nu;
            cx = csub(nx, cmul(f, cx));
        }
    }
    double2 x1 = cmul(cx, recip(cd)), x2 = make_double2(0.0, 0.0);
    sx[(size_t)(n - 1) * ld] = cscale(x1, w);
    if (n < 2) return;
    // back substitution, the next row's factors loaded one row ahead (they do not depend on x)
    size_t o = (size_t)(n - 2) * ld;
    double2 px = sx[o], p1 = s1[o], p2 = s2[o], pd = sd[o];
    for (int i = n - 2; i >= 0; --i) {
        const double2 cxr = px, c1 = p1, c2 = p2, cdr = pd;
        const size_t oi = o;
        if (i > 0) { o -= ld; px = sx[o]; p1 = s1[o]; p2 = s2[o]; pd = sd[o]; }
        double2 v = csub(cxr, cmul(c1, x1));
        v = csub(v, cmul(c2, x2));
        v = cmul(v, cdr);
        sx[oi] = cscale(v, w);
        x2 = x1;
        x1 = v;
    }
}

// The right-hand side of a quadrature pass: e_1 (pass 0) or the pass-0 result (pass 1, for the
// involution check Q(T) Q(T) e_1).
struct QuadRhs {
    const double2* rhs;
    __device__ double2 operator()(int i) const { return rhs ? rhs[i] : make_double2(i == 0 ? 1.0 : 0.0, 0.0); }
};

// Terms [blockIdx.x * kQuadBlk, +kQuadBlk) of source blockIdx.y: solve, then the block's row sums
// into part[src][blockIdx.x][row].
__global__ void __launch_bounds__(kQuadBlk) k_quad_solve(QuadArgs a, int pass) {
    const int src = blockIdx.y;
    const int N = a.nodes[src];          // nodes for this source; 0: already accepted, skip
    const int term0 = blockIdx.x * kQuadBlk;
    if (N <= 0 || term0 >= 2 * N) return;
    const int n = a.state[src].k_eff;    // rows beyond k_eff are the identity padding (finish kernel)
    if (n <= 0) return;
    const int t = threadIdx.x;
    const int width = min(kQuadBlk, 2 * N - term0);
    const double2* al = a.alpha + (size_t)src * a.kmax;
    const double2* be = a.beta + (size_t)src * a.kmax;
    const double* de = a.delta + (size_t)src * a.kmax;
    double2* sd = a.work + (size_t)src * a.kmax * 4 * a.nth_max;   // [row][term] x 4 arrays
    double2* s1 = sd + (size_t)a.kmax * a.nth_max;
    double2* s2 = s1 + (size_t)a.kmax * a.nth_max;
    double2* sx = s2 + (size_t)a.kmax * a.nth_max;
    const QuadRhs B{pass == 0 ? nullptr : a.s + (size_t)src * a.kmax};
    if (t < width) {
        const int term = term0 + t;
        const int j = term >> 1;
        const double sg = (term & 1) ? -1.0 : 1.0;
        const double c = a.c[src];
        const double th = (j + 0.5) * 3.14159265358979323846 / (2.0 * N);
        const double ct = cos(th);
        const double tau = sg * c * tan(th);
        const double w = c / (2.0 * N) / (ct * ct);
        tri_solve(al, be, de, n, make_double2(0.0, tau), B, sd + term, s1 + term, s2 + term, sx + term, a.nth_max, w);
    }
    __syncthreads();
    double2* part = a.part + ((size_t)src * a.part_blocks + blockIdx.x) * a.kmax;
    for (int i = t; i < n; i += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int q = 0; q < width; ++q) acc = cadd(acc, sx[(size_t)i * a.nth_max + term0 + q]);
        part[i] = acc;
    }
}

// out = sum of the block sums (fixed order: deterministic), identity padding beyond k_eff; the
// involution residual ||out - e_1|| after pass 1.
__global__ void __launch_bounds__(kQuadFinish) k_quad_finish(QuadArgs a, int pass) {
    const int src = blockIdx.x;
    const int N = a.nodes[src];
    if (N <= 0) return;
    const int n = a.state[src].k_eff;
    if (n <= 0) return;
    const int t = threadIdx.x;
    const int nbk = (2 * N + kQuadBlk - 1) / kQuadBlk;
    const QuadRhs B{pass == 0 ? nullptr : a.s + (size_t)src * a.kmax};
    double2* out = (pass == 0 ? a.s : a.q) + (size_t)src * a.kmax;
    const double2* part = a.part + (size_t)src * a.part_blocks * a.kmax;
    double loc = 0.0;
    for (int i = t; i < a.k; i += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        if (i < n) {
            for (int b = 0; b < nbk; ++b) acc = cadd(acc, part[(size_t)b * a.kmax + i]);
        } else {
            acc = B(i);          // identity padding: sgn(1) = 1
        }
        if (pass == 1) {
            const double ex = (i == 0) ? 1.0 : 0.0;
            loc += (acc.x - ex) * (acc.x - ex) + acc.y * acc.y;
        }
        out[i] = acc;            // pass 1 writes q, never the rhs s it reads
    }
    if (pass == 1) {
        __shared__ double red[kQuadFinish];
        red[t] = loc;
        __syncthreads();
        for (int off = blockDim.x / 2; off > 0; off >>= 1) {
            if (t < off) red[t] += red[t + off];
            __syncthreads();
        }
        if (t == 0) a.check[src] = sqrt(red[0]);
    }
}

// Contour scale c = sqrt(lambda_lo * lambda_hi): the midpoint error for an eigenvalue lambda
// decays like exp(-4 N atanh(min(|lambda|/c, c/|lambda|))), so c is placed at the geometric
// centre of the spectrum.  lambda_hi: ||T x|| after four power-iteration steps; lambda_lo:
// 1 / ||T^{-1} x|| after three inverse-iteration steps (tridiagonal solves).  Only the scale
// matters (a factor 2 costs little): on the 14^4, k = 400 projected matrices four and three
// steps need the same node counts as six and six for all but one of 16 sources.  One block (one working thread) per source, in the
// first column of the quadrature workspace.
__global__ void k_quad_scale(QuadArgs a) {
    const int src = blockIdx.x;              // one source per block (spread over the SMs)
    if (threadIdx.x != 0) return;
    if (src >= a.nb) return;
    const int n = a.state[src].k_eff;
    if (n <= 0) { a.c[src] = 1.0; return; }
    const double2* al = a.alpha + (size_t)src * a.kmax;
    const double2* be = a.beta + (size_t)src * a.kmax;
    const double* de = a.delta + (size_t)src * a.kmax;
    double2* sd = a.work + (size_t)src * a.kmax * 4 * a.nth_max;
    double2* s1 = sd + (size_t)a.kmax * a.nth_max;
    double2* s2 = s1 + (size_t)a.kmax * a.nth_max;
    double2* sx = s2 + (size_t)a.kmax * a.nth_max;
    const size_t ld = a.nth_max;
    const double x0 = 1.0 / sqrt((double)n);
    // lambda_hi: power iteration with T (x in sx, T x into s1)
    for (int i = 0; i < n; ++i) sx[(size_t)i * ld] = make_double2(x0, (i & 1) ? x0 : -x0);
    double hi = 1.0, nx = sqrt(2.0);
    for (int it = 0; it < 4; ++it) {
        double ny = 0.0;
        for (int i = 0; i < n; ++i) {
            double2 v = cmul(al[i], sx[(size_t)i * ld]);
            if (i + 1 < n) v = cadd(v, cmul(be[i], sx[(size_t)(i + 1) * ld]));
            if (i > 0) v = cadd(v, cscale(sx[(size_t)(i - 1) * ld], de[i - 1]));
            s1[(size_t)i * ld] = v;
            ny += v.x * v.x + v.y * v.y;
        }
        ny = sqrt(ny);
        if (!(ny > 0.0) || !isfinite(ny)) break;
        hi = ny / nx;
        for (int i = 0; i < n; ++i) sx[(size_t)i * ld] = cscale(s1[(size_t)i * ld], 1.0 / ny);
        nx = 1.0;
    }
    // lambda_lo: inverse iteration (tridiagonal solves in place)
    for (int i = 0; i < n; ++i) sx[(size_t)i * ld] = make_double2(x0, (i & 1) ? x0 : -x0);
    double lo = hi;
    nx = sqrt(2.0);
    for (int it = 0; it < 3; ++it) {
        auto B = [&](int i) -> double2 { return sx[(size_t)i * ld]; };
        tri_solve(al, be, de, n, make_double2(0.0, 0.0), B, sd, s1, s2, sx, ld, 1.0);
        double ny = 0.0;
        for (int i = 0; i < n; ++i) { double2 v = sx[(size_t)i * ld]; ny += v.x * v.x + v.y * v.y; }
        ny = sqrt(ny);
        if (!(ny > 0.0) || !isfinite(ny)) break;
        lo = nx / ny;
        for (int i = 0; i < n; ++i) sx[(size_t)i * ld] = cscale(sx[(size_t)i * ld], 1.0 / ny);
        nx = 1.0;
    }
    lo = fmin(lo, hi);
    const double c = sqrt(lo * hi);
    a.c[src] = (c > 0.0 && isfinite(c)) ? c : 1.0;
}

// Projected resolvent c = (sigma - T)^{-1} e_1 = -(T - sigma)^{-1} e_1: the two-sided Lanczos
// approximation of (sigma - A)^{-1} b (Sec. 2 applied to f(a) = 1/(sigma - a)).  One thread per
// source; rows beyond k_eff are zero.
__global__ void k_proj_resolvent(QuadArgs a, const double2* __restrict__ shifts) {
    const int src = blockIdx.x;              // one source per block (spread over the SMs)
    if (threadIdx.x != 0) return;
    if (src >= a.nb) return;
    const int n = a.state[src].k_eff;
    double2* out = a.s + (size_t)src * a.kmax;
    for (int i = 0; i < a.k; ++i) out[i] = make_double2(0.0, 0.0);
    if (n <= 0) { a.check[src] = 0.0; return; }
    const double2* al = a.alpha + (size_t)src * a.kmax;
    const double2* be = a.beta + (size_t)src * a.kmax;
    const double* de = a.delta + (size_t)src * a.kmax;
    double2* sd = a.work + (size_t)src * a.kmax * 4 * a.nth_max;
    double2* s1 = sd + (size_t)a.kmax * a.nth_max;
    double2* s2 = s1 + (size_t)a.kmax * a.nth_max;
    double2* sx = s2 + (size_t)a.kmax * a.nth_max;
    const double2 sg = shifts[src];
    auto B = [&](int i) -> double2 { return make_double2(i == 0 ? 1.0 : 0.0, 0.0); };
    tri_solve(al, be, de, n, make_double2(-sg.x, -sg.y), B, sd, s1, s2, sx, a.nth_max, -1.0);
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) { double2 v = sx[(size_t)i * a.nth_max]; out[i] = v; nrm += v.x * v.x + v.y * v.y; }
    a.check[src] = isfinite(nrm) ? 0.0 : 1.0;
}

cudaError_t proj_resolvent(const QuadArgs& a, const double2* shifts, cudaStream_t st) {
    k_proj_resolvent<<<a.nb, 32, 0, st>>>(a, shifts);
    return cudaGetLastError();
}

// Newton result -> projected coefficient vector: first column of X.
__global__ void k_nt_first_column(NewtonArgs a, double2* __restrict__ out, int ldo, const int* __restrict__ sel) {
    const int b = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.k || (sel && !sel[b])) return;
    out[(size_t)b * ldo + i] = a.X[(size_t)b * a.ld * a.ld + (size_t)i * a.ld];
}

cudaError_t quad_sign_e1(const QuadArgs& a, int max_nodes, bool scale, cudaStream_t st) {
    if (max_nodes < 1 || 2 * max_nodes > a.nth_max || (2 * max_nodes + kQuadBlk - 1) / kQuadBlk > a.part_blocks)
        return cudaErrorInvalidValue;
    if (scale) k_quad_scale<<<a.nb, 32, 0, st>>>(a);
    const dim3 grid((unsigned)((2 * max_nodes + kQuadBlk - 1) / kQuadBlk), (unsigned)a.nb);
    for (int pass = 0; pass < 2; ++pass) {
        k_quad_solve<<<grid, kQuadBlk, 0, st>>>(a, pass);
        k_quad_finish<<<a.nb, kQuadFinish, 0, st>>>(a, pass);
    }
    return cudaGetLastError();
}

cudaError_t quad_scale(const QuadArgs& a, cudaStream_t st) {
    k_quad_scale<<<a.nb, 32, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t newton_first_column(const NewtonArgs& a, double2* out, int ldo, cudaStream_t st, const int* sel) {
    k_nt_first_column<<<dim3((unsigned)((a.k + 127) / 128), (unsigned)a.nb), 128, 0, st>>>(a, out, ldo, sel);
    return cudaGetLastError();
}

static inline dim3 nt_grid_elems(const NewtonArgs& a) {
    return dim3((unsigned)(((size_t)a.k * a.k + kNtThreads - 1) / kNtThreads), (unsigned)a.nb);
}

cudaError_t newton_init_tridiag(const NewtonArgs& a, cudaStream_t st) {
    k_nt_init_tridiag<<<nt_grid_elems(a), kNtThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t newton_init_dense(const NewtonArgs& a, const double2* Xin, cudaStream_t st) {
    k_nt_init_dense<<<nt_grid_elems(a), kNtThreads, 0, st>>>(a, Xin);
    return cudaGetLastError();
}

cudaError_t newton_iteration(const NewtonArgs& a, cudaStream_t st) {
    const dim3 ge = nt_grid_elems(a);
    k_nt_copy<<<ge, kNtThreads, 0, st>>>(a);
    for (int p = 0; p < a.k; ++p) k_nt_elim<<<ge, kNtThreads, 0, st>>>(a, p);
    k_nt_unscramble<<<dim3((unsigned)((a.k + kNtThreads - 1) / kNtThreads), (unsigned)a.nb), kNtThreads, 0, st>>>(a);
    k_nt_combine<<<ge, kNtThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t newton_copy_out(const NewtonArgs& a, double2* Sout, cudaStream_t st) {
    k_nt_copy_out<<<nt_grid_elems(a), kNtThreads, 0, st>>>(a, Sout);
    return cudaGetLastError();
}

}  // namespace lq

// ---------------------------------------------------------------------------------------------
// Allocation-free variant of the batched Newton sign (lq_newton_sign_noalloc, include/lq.h).
// Its workspace is one file-scope device array; host code reaches it through the address that
// cudaGetSymbolAddress returns for the current device (the array's name in host code is only a
// host-side stand-in and must never be passed to a kernel).
// ---------------------------------------------------------------------------------------------
#include <mutex>

namespace lq {
namespace {

constexpr int kNaMaxK = 128;     // largest matrix dimension
constexpr int kNaMaxNb = 8;      // largest batch
constexpr size_t kNaPartBlocks = ((size_t)kNaMaxK * kNaMaxK + kNtThreads - 1) / kNtThreads;

struct NaLayout {
    double2 X[kNaMaxNb * kNaMaxK * kNaMaxK];
    double2 Y[kNaMaxNb * kNaMaxK * kNaMaxK];
    double2 F[kNaMaxNb * kNaMaxK];
    double scal[kNaMaxNb * 16];
    double partials[kNaMaxNb * kNaPartBlocks * 4];
    int perm[kNaMaxNb * kNaMaxK];
    int counters[3 * kNaMaxNb];
};

// ~4.2 MB per device, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_na_scratch[sizeof(NaLayout)];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
NaLayout* g_na_ptr[kNaMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t na_scratch(NaLayout** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = reinterpret_cast<NaLayout*>(p);
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

// True when p is device (or managed) memory that kernels on the current device can address.
// cudaPointerGetAttributes allocates nothing.
bool na_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace lq

extern "C" int lq_newton_sign_noalloc(const double* X, double* S, int k, int nb, int max_iter, double tol,
                                      int* iters, void* stream) {
    using namespace lq;
    if (!X || !S || k < 1 || nb < 1 || max_iter < 1 || !(tol > 0.0)) return LQ_ERR_ARG;
    if (k > kNaMaxK || nb > kNaMaxNb) return LQ_ERR_ARG;   // beyond the static workspace
    // a host or stale pointer must come back as an error code, never reach a kernel
    if (!na_device_ptr(X) || !na_device_ptr(S)) return LQ_ERR_LAYOUT;
    cudaStream_t st = (cudaStream_t)stream;
    NaLayout* w = nullptr;
    if (na_scratch(&w) != cudaSuccess) { cudaGetLastError(); return LQ_ERR_CUDA; }
    NewtonArgs a;
    std::memset(&a, 0, sizeof(a));
    a.k = k;
    a.nb = nb;
    a.ld = k;
    a.X = w->X;
    a.Y = w->Y;
    a.F = w->F;
    a.perm = w->perm;
    a.scal = w->scal;
    a.partials = w->partials;
    a.partial_stride = kNaPartBlocks;
    a.counters = w->counters;
    a.tol = tol;
    a.max_iter = max_iter;
    // the array keeps the previous call's contents: the block counters must start at zero
    if (cudaMemsetAsync(w->counters, 0, sizeof(w->counters), st) != cudaSuccess) { cudaGetLastError(); return LQ_ERR_CUDA; }
    if (newton_init_dense(a, reinterpret_cast<const double2*>(X), st) != cudaSuccess) return LQ_ERR_CUDA;
    double scal[kNaMaxNb * 16];
    for (int it = 0; it < max_iter; ++it) {
        if (newton_iteration(a, st) != cudaSuccess) return LQ_ERR_CUDA;
        if (cudaMemcpyAsync(scal, w->scal, sizeof(double) * 16 * nb, cudaMemcpyDeviceToHost, st) != cudaSuccess) return LQ_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return LQ_ERR_CUDA;
        bool all = true;
        for (int b = 0; b < nb; ++b) all = all && scal[b * 16 + NS_DONE] != 0.0;
        if (all) break;
    }
    if (newton_copy_out(a, reinterpret_cast<double2*>(S), st) != cudaSuccess) return LQ_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LQ_ERR_CUDA;
    int bad = 0;
    for (int b = 0; b < nb; ++b) {
        if (iters) iters[b] = (int)scal[b * 16 + NS_ITERS];
        if (scal[b * 16 + NS_STATUS] != 0.0) bad = 1;
    }
    return bad ? LQ_ERR_NEWTON : LQ_OK;
}
