// Kernel templates of the two-sided Lanczos path shared by the translation units that instantiate
// them: the block stencil (Eqs. (1.1), (2.5)), the update step of the recurrences (Sec. 2), start
// vectors, recombination and layout conversions.  lq_kernels.cu instantiates them for FP64 and
// FP32, lq_ff_*.cu for float-float (compiled in parallel: the float-float stencil is large).
#pragma once
#include "lq_internal.cuh"
#include "lq_launch.h"
#include "lq_stencil.cuh"

namespace lq {

// One hop direction (NU, SP = -1 forward / +1 backward) for NF fields per side.
// EMODE 0: no derivative term; 1: d/dmu (time hops, links U); 2: link direction (links Y).
// Right side (side 0): out0 = A in0 + E in1, out1 = A in1.
// Left side  (side 1): out0 = A^dag in0,     out1 = A^dag in1 + E^dag in0.
template <typename R, int NF, int EMODE, int NU, int SP>
__device__ __forceinline__ void do_hop(const HopArgs& a, int side, size_t V, size_t nb, size_t lsite, R bsign,
                                       const typename Tr<R>::Chunk* __restrict__ in0,
                                       const typename Tr<R>::Chunk* __restrict__ in1,
                                       typename Tr<R>::C (&acc0)[12], typename Tr<R>::C (&acc1)[12]) {
    using C = typename Tr<R>::C;
    constexpr bool DAG = SP > 0;   // backward hop uses the adjoint link at x - nu
    const R fa = fac_a<R>(a, side, NU, SP < 0) * bsign;
    const R fe = fac_e<R>(a, side, NU, SP < 0) * bsign;
    C u[9];
    load_gauge(a, V, NU, lsite, u);
    C psi[12], h0[6], g[6];
    load_spinor(in0, V, nb, psi);
    project<C, NU, SP>(psi, h0);
    if (NF == 1) {
        hscale(h0, fa);
        su3_mul<C, DAG>(u, h0, g);
        reconstruct_add<C, NU, SP>(g, acc0);
        return;
    } else {
        C h1[6];
        load_spinor(in1, V, nb, psi);
        project<C, NU, SP>(psi, h1);
        const bool emu = (EMODE == 1) && (NU == 3);
        if (side == 0) {
            // out1 += U (fa h1);  out0 += U (fa h0 [+ fe h1 for d/dmu]) [+ Y (fe h1)]
            C t0[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) t0[i] = cscale(h0[i], fa);
            if (emu) haxpy(t0, fe, h1);
            su3_mul<C, DAG>(u, t0, g);
            reconstruct_add<C, NU, SP>(g, acc0);
            if (EMODE == 2) {
                C y[9], t1[6];
                load_link(reinterpret_cast<const C*>(a.Y), V, NU, lsite, y);
#pragma unroll
                for (int i = 0; i < 6; ++i) t1[i] = cscale(h1[i], fe);
                su3_mul<C, DAG>(y, t1, g);
                reconstruct_add<C, NU, SP>(g, acc0);
            }
            hscale(h1, fa);
            su3_mul<C, DAG>(u, h1, g);
            reconstruct_add<C, NU, SP>(g, acc1);
        } else {
            // out0 += U (fa h0);  out1 += U (fa h1 [+ fe h0]) [+ Y (fe h0)]
            C t1[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) t1[i] = cscale(h1[i], fa);
            if (emu) haxpy(t1, fe, h0);
            su3_mul<C, DAG>(u, t1, g);
            reconstruct_add<C, NU, SP>(g, acc1);
            if (EMODE == 2) {
                C y[9], t0[6];
                load_link(reinterpret_cast<const C*>(a.Y), V, NU, lsite, y);
#pragma unroll
                for (int i = 0; i < 6; ++i) t0[i] = cscale(h0[i], fe);
                su3_mul<C, DAG>(y, t0, g);
                reconstruct_add<C, NU, SP>(g, acc1);
            }
            hscale(h0, fa);
            su3_mul<C, DAG>(u, h0, g);
            reconstruct_add<C, NU, SP>(g, acc0);
        }
    }
}

template <typename R, int NF, int EMODE, int NU>
__device__ __forceinline__ void do_dir(const HopArgs& a, int side, size_t V, size_t s, const int (&x)[4],
                                       const typename Tr<R>::Chunk* in0, const typename Tr<R>::Chunk* in1,
                                       typename Tr<R>::C (&acc0)[12], typename Tr<R>::C (&acc1)[12]) {
    const int ext = a.dims[NU];
    const size_t stride = a.strides[NU];
    // forward neighbour
    size_t sf = (x[NU] == ext - 1) ? s - (size_t)(ext - 1) * stride : s + stride;
    R bf = (NU == 3 && a.apbc && x[NU] == ext - 1) ? (R)-1 : (R)1;
    do_hop<R, NF, EMODE, NU, -1>(a, side, V, sf, s, bf, in0, in1, acc0, acc1);
    // backward neighbour (link at x - nu)
    size_t sb = (x[NU] == 0) ? s + (size_t)(ext - 1) * stride : s - stride;
    R bb = (NU == 3 && a.apbc && x[NU] == 0) ? (R)-1 : (R)1;
    do_hop<R, NF, EMODE, NU, +1>(a, side, V, sb, sb, bb, in0, in1, acc0, acc1);
}


// One (site block, side, source) of the block stencil: one thread per site.
template <typename R, int NF, int EMODE, bool DOT, bool PAIR>
__device__ __forceinline__ void hop_block(const HopArgs& a, int side, int src, unsigned bx, CSum* smem) {
    using C = typename Tr<R>::C;
    using Chunk = typename Tr<R>::Chunk;
    constexpr int kHalf = kHopThreads / 2;
    const size_t V = a.V;
    const size_t s = PAIR ? (size_t)bx * kHalf + threadIdx.x % kHalf : (size_t)bx * blockDim.x + threadIdx.x;
    const bool active = s < V;
    const Chunk* in0 = reinterpret_cast<const Chunk*>(a.in[side]) + (size_t)src * a.src_stride_in[side];
    const Chunk* in1 = in0 + field_elems<R>(V);
    Chunk* out0 = reinterpret_cast<Chunk*>(a.out[side]) + (size_t)src * a.src_stride_out[side];
    Chunk* out1 = out0 + field_elems<R>(V);

    C acc0[12], acc1[12];
    DotAcc<R> d[2];
    d[0].zero(); d[1].zero();
    if (active) {
#pragma unroll
        for (int c = 0; c < 12; ++c) { acc0[c] = cmk<C>(0, 0); acc1[c] = cmk<C>(0, 0); }
        int x[4];
        site_coords(a, s, x);
        do_dir<R, NF, EMODE, 0>(a, side, V, s, x, in0, in1, acc0, acc1);
        do_dir<R, NF, EMODE, 1>(a, side, V, s, x, in0, in1, acc0, acc1);
        do_dir<R, NF, EMODE, 2>(a, side, V, s, x, in0, in1, acc0, acc1);
        do_dir<R, NF, EMODE, 3>(a, side, V, s, x, in0, in1, acc0, acc1);
        const R diag = fac_diag<R>(a);
        C psi[12];
        load_spinor(in0, V, s, psi);
        finish(psi, diag, acc0);
        store_spinor(out0, V, s, acc0);
        if (NF == 2) {
            load_spinor(in1, V, s, psi);
            finish(psi, diag, acc1);
            store_spinor(out1, V, s, acc1);
        }
        if (DOT && side == 0) {
            // <w_j, B vh_j> restricted to this site: left inputs at s (conj) times outputs
            const Chunk* l0 = reinterpret_cast<const Chunk*>(a.in[1]) + (size_t)src * a.src_stride_in[1];
            C w[12];
            load_spinor(l0, V, s, w);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                add_cdot(d[0], d[1], w[c], acc0[c]);
            }
            if (NF == 2) {
                load_spinor(l0 + field_elems<R>(V), V, s, w);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    add_cdot(d[0], d[1], w[c], acc1[c]);
                }
            }
        }
    }
    if (DOT && (PAIR || side == 0)) {   // (block-uniform; with PAIR the left warps add zeros)
        const int nbx = (int)gridDim.x;
        CSum tot[2];
        block_total<R, 2>(d, tot, smem);
        double* part = a.partials + ((size_t)src * a.partial_stride + bx) * 4;
        if (threadIdx.x == 0) { part[0] = tot[0].s; part[1] = tot[0].e; part[2] = tot[1].s; part[3] = tot[1].e; }
        if (last_block(a.counters + src, nbx)) {
            double res[2];
            reduce_partials<2>(a.partials + (size_t)src * a.partial_stride * 4, nbx, res, smem);
            if (threadIdx.x == 0) tsl_alpha_step(a, src, res[0], res[1]);
        }
    }
}

// The block stencil.  Grid (site blocks, sides, sources): the two sides of one source run close
// together in launch order, so that the right side's alpha dot finds the left vectors in L2.
// PAIR (schedule 9): a block holds both sides of kHopThreads / 2 sites instead, warps 0-1 the
// right and 2-3 the left side, so that the second load of each link hits L1.
template <typename R, int NF, int EMODE, bool DOT, int MINB, bool PAIR = false>
__global__ void __launch_bounds__(kHopThreads, MINB) k_hop(HopArgs a) {
    __shared__ CSum smem[32 * 2];
    constexpr int kHalf = kHopThreads / 2;
    const int side = PAIR ? (int)(threadIdx.x / kHalf) : (int)blockIdx.y + a.side0;
    const int src = blockIdx.z;
    if (a.state != nullptr && a.state[src].status != 0) return;   // source finished / failed
    hop_block<R, NF, EMODE, DOT, PAIR>(a, side, src, blockIdx.x, smem);
}

// ---------------------------------------------------------------------------------------
// Update: new right/left vectors and the omega dot, |vh|^2, |wh|^2.
// ---------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kUpdThreads, 3) k_update(UpdArgs a) {
    using C = typename Tr<R>::C;
    using Chunk = typename Tr<R>::Chunk;
    __shared__ CSum smem[32 * 6];
    const int src = blockIdx.y;
    TslState& st = a.state[src];
    if (st.status != 0) return;
    C cv[3], cw[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        cv[i] = cmk<C>((R)st.cv[i].x, (R)st.cv[i].y);
        cw[i] = cmk<C>((R)st.cw[i].x, (R)st.cw[i].y);
    }
    const bool has_prev = a.j > 0;
    const size_t N = a.nelem;
    const Chunk* r = reinterpret_cast<const Chunk*>(a.rout) + (size_t)src * a.src_stride_io;
    const Chunk* l = reinterpret_cast<const Chunk*>(a.lout) + (size_t)src * a.src_stride_io;
    const Chunk* v = reinterpret_cast<const Chunk*>(a.v_cur) + (size_t)src * a.src_stride_basis;
    const Chunk* vp = reinterpret_cast<const Chunk*>(a.v_prev) + (size_t)src * a.src_stride_basis;
    Chunk* vn = reinterpret_cast<Chunk*>(a.v_next) + (size_t)src * a.src_stride_basis;
    const Chunk* w = reinterpret_cast<const Chunk*>(a.w_cur) + (size_t)src * a.src_stride_left;
    const Chunk* wp = reinterpret_cast<const Chunk*>(a.w_prev) + (size_t)src * a.src_stride_left;
    Chunk* wn = reinterpret_cast<Chunk*>(a.w_next) + (size_t)src * a.src_stride_left;
    Chunk* ws = a.w_store ? reinterpret_cast<Chunk*>(a.w_store) + (size_t)src * a.src_stride_store : nullptr;
    DotAcc<R> d[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i].zero();
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const Chunk zero{};
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e + stride < N; e += 2 * stride) {     // two chunks in flight per thread
        const size_t e2 = e + stride;
        const Chunk r0 = __ldg(r + e), r1 = __ldg(r + e2), v0 = __ldg(v + e), v1 = __ldg(v + e2);
        const Chunk p0 = has_prev ? __ldg(vp + e) : zero, p1 = has_prev ? __ldg(vp + e2) : zero;
        const Chunk l0 = __ldg(l + e), l1 = __ldg(l + e2), w0 = __ldg(w + e), w1 = __ldg(w + e2);
        const Chunk q0 = has_prev ? __ldg(wp + e) : zero, q1 = has_prev ? __ldg(wp + e2) : zero;
        const Chunk nv0 = axpy3<R>(r0, v0, p0, cv, has_prev), nv1 = axpy3<R>(r1, v1, p1, cv, has_prev);
        const Chunk nw0 = axpy3<R>(l0, w0, q0, cw, has_prev), nw1 = axpy3<R>(l1, w1, q1, cw, has_prev);
        vn[e] = nv0; vn[e2] = nv1;
        wn[e] = nw0; wn[e2] = nw1;
        if (ws) { ws[e] = nw0; ws[e2] = nw1; }
        dot_chunk<R>(d, nw0, nv0);
        dot_chunk<R>(d, nw1, nv1);
        norm_chunk(d, r0, l0);
        norm_chunk(d, r1, l1);
    }
    if (e < N) {
        const Chunk re = __ldg(r + e), le = __ldg(l + e);
        const Chunk nv = axpy3<R>(re, __ldg(v + e), has_prev ? __ldg(vp + e) : zero, cv, has_prev);
        const Chunk nw = axpy3<R>(le, __ldg(w + e), has_prev ? __ldg(wp + e) : zero, cw, has_prev);
        vn[e] = nv;
        wn[e] = nw;
        if (ws) ws[e] = nw;
        dot_chunk<R>(d, nw, nv);
        norm_chunk(d, re, le);
    }
    CSum tot[6];
    block_total<R, 6>(d, tot, smem);
    double* part = a.partials + ((size_t)src * a.partial_stride + blockIdx.x) * 12;
    if (threadIdx.x == 0)
        for (int i = 0; i < 6; ++i) { part[2 * i] = tot[i].s; part[2 * i + 1] = tot[i].e; }
    if (last_block(a.counters + a.nsrc + src, gridDim.x)) {
        double res[6];
        reduce_partials<6>(a.partials + (size_t)src * a.partial_stride * 12, gridDim.x, res, smem);
        if (threadIdx.x == 0) {
            if (a.defer) { st.rb_nr = res[4]; st.rb_nl = res[5]; }
            else update_scalars<R>(a, src, res);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Start vectors.  Plain:  vh_1 = wh_1 = x.   Block: vh_1 = (0, x), wh_1 = (x, x).
// s_1 = u_1 = 1/|x| so that v_1 = x/|x| (or (0,x)/|x|) and <w_1, v_1> = 1.
// x arrives in the boundary layout (complex128 [nsrc][V][12]).
// ---------------------------------------------------------------------------------------
template <typename R, int NF>
__global__ void __launch_bounds__(kUpdThreads) k_tsl_init(InitArgs a) {
    using C = typename Tr<R>::C;
    using Chunk = typename Tr<R>::Chunk;
    __shared__ CSum smem[32 * 4];
    const int src = blockIdx.y;
    const size_t V = a.V;
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    // sums of the stored (rounded) values: |t|^2, |b|^2, Re <b,t>, Im <b,t>
    CSum acc[4] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    if (s < V) {
        const double2* x = reinterpret_cast<const double2*>(a.x) + ((size_t)src * V + s) * 12;
        C psi[12], top[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            double2 z = x[c];
            psi[c] = cmk<C>((R)z.x, (R)z.y);
            cs_add_prod(acc[1], (double)psi[c].x, (double)psi[c].x);
            cs_add_prod(acc[1], (double)psi[c].y, (double)psi[c].y);
        }
        Chunk* v = reinterpret_cast<Chunk*>(a.v1) + (size_t)src * a.src_stride_basis;
        Chunk* w = reinterpret_cast<Chunk*>(a.w1) + (size_t)src * a.src_stride_left;
        if (NF == 1) {
            store_spinor(v, V, s, psi);
            store_spinor(w, V, s, psi);
            if (a.w1_store) store_spinor(reinterpret_cast<Chunk*>(a.w1_store) + (size_t)src * a.src_stride_store, V, s, psi);
        } else {
            const double2* xt = a.xt ? reinterpret_cast<const double2*>(a.xt) + ((size_t)src * V + s) * 12 : nullptr;
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                double2 z = xt ? xt[c] : make_double2(0.0, 0.0);
                top[c] = cmk<C>((R)z.x, (R)z.y);
                const double tx = (double)top[c].x, ty = (double)top[c].y;
                const double bx = (double)psi[c].x, by = (double)psi[c].y;
                cs_add_prod(acc[0], tx, tx); cs_add_prod(acc[0], ty, ty);
                cs_add_prod(acc[2], bx, tx); cs_add_prod(acc[2], by, ty);     // Re conj(b) t
                cs_add_prod(acc[3], bx, ty); cs_add_prod(acc[3], -by, tx);    // Im conj(b) t
            }
            store_spinor(v, V, s, top);
            store_spinor(v + field_elems<R>(V), V, s, psi);
            store_spinor(w, V, s, psi);
            store_spinor(w + field_elems<R>(V), V, s, psi);
        }
    }
    block_reduce_cs<4>(acc, smem);
    double* part = a.partials + ((size_t)src * a.partial_stride + blockIdx.x) * 8;
    if (threadIdx.x == 0)
        for (int i = 0; i < 4; ++i) { part[2 * i] = acc[i].s; part[2 * i + 1] = acc[i].e; }
    if (last_block(a.counters + 2 * a.nsrc + src, gridDim.x)) {
        double res[4];
        reduce_partials<4>(a.partials + (size_t)src * a.partial_stride * 8, gridDim.x, res, smem);
        if (threadIdx.x == 0) {
            // v_1 = s_1 vh_1 with |v_1| = 1;  <w_1, v_1> = 1 with w_1 = u_1 wh_1, wh_1 = (b, b) or b
            TslState& st = a.state[src];
            const double nt = res[0], nb = res[1];
            const double vn = sqrt(nt + nb);
            st.xnorm = vn;
            st.k_eff = 0;
            st.breakdown_tol = a.breakdown_tol;
            if (!isfinite(vn)) { st.status = LQ_ERR_NONFINITE; return; }   // NaN / Inf in the source
            if (!(vn > 0.0)) { st.status = LQ_ERR_ARG; return; }              // zero source
            const double s1 = 1.0 / vn;
            double2 wv = make_double2(nb, 0.0);                  // <wh_1, vh_1>
            if (NF == 2) { wv.x += res[2]; wv.y += res[3]; }
            // u_1 = 1 / conj(s_1 <wh_1, vh_1>)
            const double2 q = make_double2(s1 * wv.x, -s1 * wv.y);
            const double qn = q.x * q.x + q.y * q.y;
            if (!(qn > 0.0) || !isfinite(qn)) { st.status = LQ_ERR_BREAKDOWN; return; }
            st.status = 0;
            st.s_cur = s1;
            st.s_prev = 0.0;
            st.u_cur = make_double2(q.x / qn, -q.y / qn);
            st.u_prev = make_double2(0.0, 0.0);
            st.beta_prev = make_double2(0.0, 0.0);
            st.delta_prev = 0.0;
            for (int i = 0; i < 3; ++i) { st.cv[i] = make_double2(0.0, 0.0); st.cw[i] = make_double2(0.0, 0.0); }
        }
    }
}

// ---------------------------------------------------------------------------------------
// Recombination y = |x| sum_j c_j s_j vh_j for each field, written in the boundary layout.
// c = sgn(T_k) e_1 (from the Newton iteration or the quadrature), one row per source.
// FP64 basis: FP64 accumulation.  Float-float basis: unnormalised float-float sums of exact
// products.  FP32 basis: groups of four terms in FP32, the group sums in float-float.
// ---------------------------------------------------------------------------------------
template <typename R, int NF>
__global__ void __launch_bounds__(kRecThreads) k_recombine(RecArgs a) {
    using C = typename Tr<R>::C;
    using Chunk = typename Tr<R>::Chunk;
    extern __shared__ double2 coef[];   // [keff] (double) or [keff] float4 (hi.x, hi.y, lo.x, lo.y)
    const int src = blockIdx.y;
    const int f = blockIdx.z;           // field index (0 top / 1 bottom)
    const TslState& st = a.state[src];
    const int keff = st.k_eff;
    const size_t V = a.V;
    const double xn = st.xnorm;
    const int j0 = a.j0, j1 = (a.j1 > 0 && a.j1 < keff) ? a.j1 : keff;   // window [j0, j1)
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        double2 c = a.coef[(size_t)src * a.kmax + j];
        double sc = a.scale[(size_t)src * a.kmax + j] * xn;
        double2 cs = make_double2(c.x * sc, c.y * sc);
        if (Tr<R>::kKind == 0) coef[j - j0] = cs;
        else {
            // split once per block: no FP64 arithmetic is left in the k-loop below
            const float hx = (float)cs.x, hy = (float)cs.y;
            reinterpret_cast<float4*>(coef)[j - j0] = make_float4(hx, hy, (float)(cs.x - (double)hx), (float)(cs.y - (double)hy));
        }
    }
    __syncthreads();
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    double2* y = reinterpret_cast<double2*>(f == 0 ? a.y0 : a.y1) + ((size_t)src * V + s) * 12;
    if (j1 <= j0) {
        if (!a.accumulate)
#pragma unroll
            for (int c = 0; c < 12; ++c) y[c] = make_double2(0.0, 0.0);
        return;
    }
    auto slot = [&](int j) -> size_t { return (size_t)(a.ring > 0 ? j % a.ring : j); };
    const Chunk* base = reinterpret_cast<const Chunk*>(a.basis) + (size_t)src * a.src_stride_basis + (size_t)f * field_elems<R>(V);
    if constexpr (Tr<R>::kKind == 2) {
        // float-float basis: each component an unnormalised float-float sum of the exact
        // products with the float-float coefficient (FP32 operations only), converted at the end
        FFSum ar[12], ai[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) { ar[c] = FFSum{0.f, 0.f}; ai[c] = FFSum{0.f, 0.f}; }
        for (int j = j0; j < j1; ++j) {
            const float4* vj = reinterpret_cast<const float4*>(base + slot(j) * a.vec_stride);
            const float4 cf = reinterpret_cast<const float4*>(coef)[j - j0];
            const ff cr(cf.x, cf.z), ci(cf.y, cf.w);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                const float4 q = __ldg(vj + (size_t)c * V + s);
                const ff vr(q.x, q.y), vi(q.z, q.w);
                ffsum_add_prod<false>(ar[c], cr, vr);
                ffsum_add_prod<true>(ar[c], ci, vi);
                ffsum_add_prod<false>(ai[c], cr, vi);
                ffsum_add_prod<false>(ai[c], ci, vr);
            }
        }
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const double2 w = make_double2((double)ar[c].s + (double)ar[c].e, (double)ai[c].s + (double)ai[c].e);
            y[c] = a.accumulate ? cadd(y[c], w) : w;
        }
    } else if (Tr<R>::kKind == 0) {
        // FP64 accumulation
        double2 acc[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = make_double2(0.0, 0.0);
        for (int j = j0; j < j1; ++j) {
            const Chunk* vj = base + slot(j) * a.vec_stride;
            const double2 cj = coef[j - j0];
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[c] = cfma(cj, __ldg(reinterpret_cast<const double2*>(vj) + (size_t)c * V + s), acc[c]);
        }
#pragma unroll
        for (int c = 0; c < 12; ++c) y[c] = a.accumulate ? cadd(y[c], acc[c]) : acc[c];
    } else {
        // groups of kRecGroup terms summed in FP32 (the coefficient rounded to FP32), the group
        // sums added into float-float accumulators: the result carries about the error of the
        // FP32 storage of the basis itself (4 products per group in one FMA chain), at a sixth
        // of the instructions of exact products per term
        constexpr int kRecGroup = 4;
        FF ar[12], ai[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) { ar[c] = FF{0.f, 0.f}; ai[c] = FF{0.f, 0.f}; }
        for (int jg = j0; jg < j1; jg += kRecGroup) {
            float2 g[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) g[c] = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < kRecGroup; ++t) {
                const int j = jg + t;
                if (j < j1) {
                    const float4* vj = reinterpret_cast<const float4*>(base + slot(j) * a.vec_stride);
                    const float4 cf = reinterpret_cast<const float4*>(coef)[j - j0];
                    const float cr = cf.x, ci = cf.y;
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        const float4 v4 = __ldg(vj + (size_t)q * V + s);
                        g[2 * q].x = fmaf(cr, v4.x, fmaf(-ci, v4.y, g[2 * q].x));
                        g[2 * q].y = fmaf(cr, v4.y, fmaf(ci, v4.x, g[2 * q].y));
                        g[2 * q + 1].x = fmaf(cr, v4.z, fmaf(-ci, v4.w, g[2 * q + 1].x));
                        g[2 * q + 1].y = fmaf(cr, v4.w, fmaf(ci, v4.z, g[2 * q + 1].y));
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                float sh, st;
                two_sum_f(ar[c].h, g[c].x, sh, st); ar[c].h = sh; ar[c].l += st;
                two_sum_f(ai[c].h, g[c].y, sh, st); ai[c].h = sh; ai[c].l += st;
            }
        }
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const double2 w = make_double2((double)ar[c].h + (double)ar[c].l, (double)ai[c].h + (double)ai[c].l);
            y[c] = a.accumulate ? cadd(y[c], w) : w;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Layout conversions
// ---------------------------------------------------------------------------------------
template <typename R>
__global__ void k_to_internal(const double2* __restrict__ x, typename Tr<R>::Chunk* __restrict__ f, size_t V, int nfields) {
    using C = typename Tr<R>::C;
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int fld = blockIdx.y;
    if (s >= V || fld >= nfields) return;
    C psi[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        double2 z = x[((size_t)fld * V + s) * 12 + c];
        psi[c] = cmk<C>((R)z.x, (R)z.y);
    }
    store_spinor(f + (size_t)fld * field_elems<R>(V), V, s, psi);
}

template <typename R>
__global__ void k_to_boundary(const typename Tr<R>::Chunk* __restrict__ f, double2* __restrict__ x, size_t V, int nfields) {
    using C = typename Tr<R>::C;
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int fld = blockIdx.y;
    if (s >= V || fld >= nfields) return;
    C psi[12];
    load_spinor(f + (size_t)fld * field_elems<R>(V), V, s, psi);
#pragma unroll
    for (int c = 0; c < 12; ++c) x[((size_t)fld * V + s) * 12 + c] = make_double2((double)psi[c].x, (double)psi[c].y);
}

// links: boundary [4][V][3][3] complex128 -> internal [4][9][V]
template <typename R>
__global__ void k_links_internal(const double2* __restrict__ U, typename Tr<R>::C* __restrict__ L, size_t V) {
    using C = typename Tr<R>::C;
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nu = blockIdx.y;
    if (s >= V) return;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        double2 z = U[((size_t)nu * V + s) * 9 + e];
        L[((size_t)nu * 9 + e) * V + s] = cmk<C>((R)z.x, (R)z.y);
    }
}

// dU/dt = i Omega U with Omega = sum_a w^a lambda_a / 2 (su(3)) or theta * 1 (U(1)).
// U (FP64 boundary copy), w: [4][V][8] or [4][V]; output Y internal.
template <typename R>
__global__ void k_direction(const double2* __restrict__ U, const double* __restrict__ w, int kind,
                            typename Tr<R>::C* __restrict__ Y, size_t V) {
    using C = typename Tr<R>::C;
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nu = blockIdx.y;
    if (s >= V) return;
    // M = i Omega (3x3)
    double2 M[9];
    if (kind == LQ_DIR_SU3) {
        const double* c = w + ((size_t)nu * V + s) * 8;
        const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
        // Omega = 1/2 sum_a c_a lambda_a (Gell-Mann), written element by element
        double2 O[9];
        O[0] = make_double2(0.5 * (c[2] + r3 * c[7]), 0.0);
        O[4] = make_double2(0.5 * (-c[2] + r3 * c[7]), 0.0);
        O[8] = make_double2(0.5 * (-2.0 * r3 * c[7]), 0.0);
        O[1] = make_double2(0.5 * c[0], -0.5 * c[1]);
        O[3] = make_double2(0.5 * c[0], 0.5 * c[1]);
        O[2] = make_double2(0.5 * c[3], -0.5 * c[4]);
        O[6] = make_double2(0.5 * c[3], 0.5 * c[4]);
        O[5] = make_double2(0.5 * c[5], -0.5 * c[6]);
        O[7] = make_double2(0.5 * c[5], 0.5 * c[6]);
        for (int e = 0; e < 9; ++e) M[e] = make_double2(-O[e].y, O[e].x);
    } else {
        const double th = w[(size_t)nu * V + s];
        for (int e = 0; e < 9; ++e) M[e] = make_double2(0.0, (e % 4 == 0) ? th : 0.0);
    }
    const double2* u = U + ((size_t)nu * V + s) * 9;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double2 acc = make_double2(0.0, 0.0);
            for (int k = 0; k < 3; ++k) acc = cfma(M[r * 3 + k], u[k * 3 + c], acc);
            Y[((size_t)nu * 9 + r * 3 + c) * V + s] = cmk<C>((R)acc.x, (R)acc.y);
        }
}

// ---------------------------------------------------------------------------------------
// Role-split block stencil: one thread per (site, output field, source).  The four outputs
// of a site for the block operator of Eq. (2.5) are
//   role 0: A t + E b      role 1: A b          (right side, operator A = H(mu))
//   role 2: A^dag p        role 3: A^dag q + E^dag p   (left side, A^dag = H(-mu))
// A block holds RS sites x 4 roles (RS / 32 warps per role), so the four roles read the
// same links and neighbour sites and share them in L1.  The alpha dot is accumulated by the
// right-side roles: conj(p(x)) . (A t + E b)(x) + conj(q(x)) . (A b)(x).
// ---------------------------------------------------------------------------------------
constexpr int kRoleSites = 32;

template <typename R, int EMODE, int NU, int SP>
__device__ __forceinline__ void role_hop(const HopArgs& a, int side, bool with_e, size_t V, size_t nb, size_t lsite, R bsign,
                                         const typename Tr<R>::Chunk* __restrict__ fa_in,
                                         const typename Tr<R>::Chunk* __restrict__ fe_in,
                                         typename Tr<R>::C (&acc)[12]) {
    using C = typename Tr<R>::C;
    constexpr bool DAG = SP > 0;
    const R fa = fac_a<R>(a, side, NU, SP < 0) * bsign;
    const bool ehop = with_e && (EMODE == 2 || (EMODE == 1 && NU == 3));
    C u[9], psi[12], h[6], g[6];
    load_gauge(a, V, NU, lsite, u);
    load_spinor(fa_in, V, nb, psi);
    project<C, NU, SP>(psi, h);
    hscale(h, fa);
    if (ehop) {
        const R fe = fac_e<R>(a, side, NU, SP < 0) * bsign;
        C he[6];
        load_spinor(fe_in, V, nb, psi);
        project<C, NU, SP>(psi, he);
        if (EMODE == 1) {
            haxpy(h, fe, he);                 // same link: combine before the multiply
        } else {
            C y[9];
            load_link(reinterpret_cast<const C*>(a.Y), V, NU, lsite, y);
            hscale(he, fe);
            su3_mul<C, DAG>(y, he, g);
            reconstruct_add<C, NU, SP>(g, acc);
        }
    }
    su3_mul<C, DAG>(u, h, g);
    reconstruct_add<C, NU, SP>(g, acc);
}

template <typename R, int EMODE, int NU>
__device__ __forceinline__ void role_dir(const HopArgs& a, int side, bool with_e, size_t V, size_t s, const int (&x)[4],
                                         const typename Tr<R>::Chunk* fa_in, const typename Tr<R>::Chunk* fe_in,
                                         typename Tr<R>::C (&acc)[12]) {
    const int ext = a.dims[NU];
    const size_t stride = a.strides[NU];
    const size_t sf = (x[NU] == ext - 1) ? s - (size_t)(ext - 1) * stride : s + stride;
    const R bf = (NU == 3 && a.apbc && x[NU] == ext - 1) ? (R)-1 : (R)1;
    role_hop<R, EMODE, NU, -1>(a, side, with_e, V, sf, s, bf, fa_in, fe_in, acc);
    const size_t sb = (x[NU] == 0) ? s + (size_t)(ext - 1) * stride : s - stride;
    const R bb = (NU == 3 && a.apbc && x[NU] == 0) ? (R)-1 : (R)1;
    role_hop<R, EMODE, NU, +1>(a, side, with_e, V, sb, sb, bb, fa_in, fe_in, acc);
}

template <typename R, int EMODE, bool DOT, int RS, int MINB>
__global__ void __launch_bounds__(4 * RS, MINB) k_hop_roles(HopArgs a) {
    using C = typename Tr<R>::C;
    using Chunk = typename Tr<R>::Chunk;
    __shared__ CSum smem[32 * 2];
    const int src = blockIdx.y;
    if (a.state != nullptr && a.state[src].status != 0) return;
    const int role = threadIdx.x / RS;                // warp-uniform
    const int side = role >> 1;                       // 0 right, 1 left
    const int fld = role & 1;                         // output field within the side
    const size_t V = a.V;
    const size_t s = (size_t)blockIdx.x * RS + (threadIdx.x % RS);
    const bool active = s < V;
    const size_t F = field_elems<R>(V);
    const Chunk* in0 = reinterpret_cast<const Chunk*>(a.in[side]) + (size_t)src * a.src_stride_in[side];
    Chunk* out = reinterpret_cast<Chunk*>(a.out[side]) + (size_t)src * a.src_stride_out[side] + (size_t)fld * F;
    // operator input and derivative input of this role
    const Chunk* fa_in = in0 + (size_t)fld * F;
    const bool with_e = (EMODE != 0) && ((side == 0 && fld == 0) || (side == 1 && fld == 1));
    const Chunk* fe_in = (side == 0) ? in0 + F : in0;   // right: E acts on the bottom; left: E^dag on the top
    DotAcc<R> d[2];
    d[0].zero(); d[1].zero();
    if (active) {
        C acc[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = cmk<C>(0, 0);
        int x[4];
        site_coords(a, s, x);
        role_dir<R, EMODE, 0>(a, side, with_e, V, s, x, fa_in, fe_in, acc);
        role_dir<R, EMODE, 1>(a, side, with_e, V, s, x, fa_in, fe_in, acc);
        role_dir<R, EMODE, 2>(a, side, with_e, V, s, x, fa_in, fe_in, acc);
        role_dir<R, EMODE, 3>(a, side, with_e, V, s, x, fa_in, fe_in, acc);
        C psi[12];
        load_spinor(fa_in, V, s, psi);
        finish(psi, fac_diag<R>(a), acc);
        store_spinor(out, V, s, acc);
        if (DOT && side == 0) {
            const Chunk* w = reinterpret_cast<const Chunk*>(a.in[1]) + (size_t)src * a.src_stride_in[1] + (size_t)fld * F;
            load_spinor(w, V, s, psi);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                add_cdot(d[0], d[1], psi[c], acc[c]);
            }
        }
    }
    if (DOT) {
        CSum tot[2];
        block_total<R, 2>(d, tot, smem);
        double* part = a.partials + ((size_t)src * a.partial_stride + blockIdx.x) * 4;
        if (threadIdx.x == 0) { part[0] = tot[0].s; part[1] = tot[0].e; part[2] = tot[1].s; part[3] = tot[1].e; }
        if (last_block(a.counters + src, gridDim.x)) {
            double res[2];
            reduce_partials<2>(a.partials + (size_t)src * a.partial_stride * 4, gridDim.x, res, smem);
            if (threadIdx.x == 0) tsl_alpha_step(a, src, res[0], res[1]);
        }
    }
}

}  // namespace lq
