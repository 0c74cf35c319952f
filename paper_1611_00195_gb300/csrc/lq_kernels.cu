// Device kernels of the two-sided Lanczos path:
//   * k_hop      -- the Wilson kernel H(mu) = gamma5 Dw(mu) (Eq. (1.1)), its adjoint H(-mu), and
//                   the block operator B = [[A, dA], [0, A]] / B^dag of Eq. (2.5), for a batch of
//                   sources, with the Lanczos alpha dot fused into the epilogue;
//   * k_update   -- the three-term Lanczos recurrences (Sec. 2) with the omega dot and norms;
//   * k_tsl_init -- boundary -> internal layout, start vectors and |x|;
//   * k_recombine-- y = |x| V_k c (+ internal -> boundary layout);
//   * layout / precision conversion of spinors, links and the derivative direction dU/dt.
#include "lq_internal.cuh"
#include "lq_kernels.cuh"
#include "lq_launch.h"
#include "lq_stencil.cuh"

#include <algorithm>
#include <cstdio>

namespace lq {

// ---------------------------------------------------------------------------------------
// Shared-memory tiled block stencil (schedule 6, FP32).  A block takes a tile of whole x rows,
// kTileY x kTileZ x kTileT in (y, z, t), for one side of one source.  It copies into shared
// memory, each site once and with all loads in flight together: the links of the tile (forward
// links of every tile site, and the backward links that sit on the -y, -z, -t faces), then one
// input field on the tile and its six faces; it applies that field's hops from shared memory,
// then does the same with the other field.  The field whose output has no derivative term is
// processed first, so that one accumulator is finished (gamma5, centre term, store) after each
// phase.  Right side: out1 = A b, out0 = A t + E b (b first); left side: out0 = A^dag p,
// out1 = A^dag q + E^dag p (p first).  On d/dmu hops A and E share the link and the projected
// spinor: one SU(3) product feeds both accumulators.
// ---------------------------------------------------------------------------------------
constexpr int kTileY = 2, kTileZ = 2, kTileT = 2;

struct TileGeom {
    int nx, ny, nz, nt;          // lattice extents
    int ns;                      // tile sites nx * kTileY * kTileZ * kTileT
    int fy, fz, ft;              // sites on one face normal to y, z, t
    int ntot;                    // tile + six faces
    size_t smem;                 // dynamic shared memory bytes
};

__host__ __device__ inline TileGeom tile_geom(const int (&dims)[4]) {
    TileGeom g;
    g.nx = dims[0]; g.ny = dims[1]; g.nz = dims[2]; g.nt = dims[3];
    g.ns = g.nx * kTileY * kTileZ * kTileT;
    g.fy = g.nx * kTileZ * kTileT;
    g.fz = g.nx * kTileY * kTileT;
    g.ft = g.nx * kTileY * kTileZ;
    g.ntot = g.ns + 2 * (g.fy + g.fz + g.ft);
    // site map (int) | forward links [4][9][ns] + backward face links [9][fy + fz + ft] (float2)
    // | one field [6][ntot] (float4)
    const size_t map_b = ((size_t)g.ntot * sizeof(int) + 15) / 16 * 16;
    const size_t link_b = ((size_t)36 * g.ns + (size_t)9 * (g.fy + g.fz + g.ft)) * sizeof(float2);
    g.smem = map_b + (link_b + 15) / 16 * 16 + (size_t)6 * g.ntot * sizeof(float4);
    return g;
}

// Schedule 6 applies when the tiles cover the lattice and fit a block and shared memory.
bool tile_ok(const int (&dims)[4]) {
    if (dims[1] % kTileY || dims[2] % kTileZ || dims[3] % kTileT) return false;
    const TileGeom g = tile_geom(dims);
    // at least one warp (the alpha-dot partials hold one slot per 32 sites) and at most the
    // kernel's launch bound
    return g.ns >= 32 && g.ns <= 256 && g.smem <= 200 * 1024;
}

// Local tile coordinates (x, ly, lz, lt; -1 or the tile extent on a face) of entry r of the
// tile-plus-faces list: the tile sites x-fastest, then the -y, +y, -z, +z, -t, +t faces.
__device__ __forceinline__ void tile_decode(const TileGeom& g, int r, int& x, int& ly, int& lz, int& lt) {
    if (r < g.ns) {
        x = r % g.nx; int q = r / g.nx;
        ly = q % kTileY; q /= kTileY; lz = q % kTileZ; lt = q / kTileZ;
        return;
    }
    r -= g.ns;
    if (r < 2 * g.fy) {
        const int f = r / g.fy, u = r % g.fy;
        x = u % g.nx; const int q = u / g.nx; lz = q % kTileZ; lt = q / kTileZ; ly = f ? kTileY : -1;
        return;
    }
    r -= 2 * g.fy;
    if (r < 2 * g.fz) {
        const int f = r / g.fz, u = r % g.fz;
        x = u % g.nx; const int q = u / g.nx; ly = q % kTileY; lt = q / kTileY; lz = f ? kTileZ : -1;
        return;
    }
    r -= 2 * g.fz;
    const int f = r / g.ft, u = r % g.ft;
    x = u % g.nx; const int q = u / g.nx; ly = q % kTileY; lz = q / kTileY; lt = f ? kTileT : -1;
}

// Shared-memory index of the neighbour of tile site (x, ly, lz, lt) in direction NU, +1 / -1.
template <int NU, int DIR>
__device__ __forceinline__ int tile_nb(const TileGeom& g, int x, int ly, int lz, int lt) {
    const int c = x + g.nx * (ly + kTileY * (lz + kTileZ * lt));
    if (NU == 0) {
        const int xn = DIR > 0 ? (x + 1 == g.nx ? 0 : x + 1) : (x == 0 ? g.nx - 1 : x - 1);
        return c - x + xn;
    }
    if (NU == 1) {
        const int l = ly + DIR;
        if (l >= 0 && l < kTileY) return c + DIR * g.nx;
        return g.ns + (DIR > 0 ? g.fy : 0) + x + g.nx * (lz + kTileZ * lt);
    }
    if (NU == 2) {
        const int l = lz + DIR;
        if (l >= 0 && l < kTileZ) return c + DIR * g.nx * kTileY;
        return g.ns + 2 * g.fy + (DIR > 0 ? g.fz : 0) + x + g.nx * (ly + kTileY * lt);
    }
    const int l = lt + DIR;
    if (l >= 0 && l < kTileT) return c + DIR * g.nx * kTileY * kTileZ;
    return g.ns + 2 * g.fy + 2 * g.fz + (DIR > 0 ? g.ft : 0) + x + g.nx * (ly + kTileY * lz);
}

// Backward link U_NU(s - NU) of tile site (x, ly, lz, lt): the forward link of the tile site
// behind it, or the face copy; element e at lf[(NU * 9 + e) * ns + ...] / lb[e * nb + ...].
template <int NU>
__device__ __forceinline__ void tile_back_link(const TileGeom& g, const float2* lf, const float2* lb, int x, int ly,
                                               int lz, int lt, float2 (&u)[9]) {
    const int c = x + g.nx * (ly + kTileY * (lz + kTileZ * lt));
    const int nbk = g.fy + g.fz + g.ft;
    int idx = -1, fidx = 0;
    if (NU == 0) idx = c - x + (x == 0 ? g.nx - 1 : x - 1);
    else if (NU == 1) { if (ly > 0) idx = c - g.nx; else fidx = x + g.nx * (lz + kTileZ * lt); }
    else if (NU == 2) { if (lz > 0) idx = c - g.nx * kTileY; else fidx = g.fy + x + g.nx * (ly + kTileY * lt); }
    else { if (lt > 0) idx = c - g.nx * kTileY * kTileZ; else fidx = g.fy + g.fz + x + g.nx * (ly + kTileY * lz); }
#pragma unroll
    for (int e = 0; e < 9; ++e) u[e] = idx >= 0 ? lf[(NU * 9 + e) * g.ns + idx] : lb[e * nbk + fidx];
}

// Asynchronous global -> shared copies (cp.async): the copies of a fill are all in flight at
// once and no register holds the data; completed by cp_async_wait_all() + __syncthreads().
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void tile_spinor(const float4* f, int ntot, int i, float2 (&o)[12]) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float4 v = f[q * ntot + i];
        o[2 * q] = make_float2(v.x, v.y);
        o[2 * q + 1] = make_float2(v.z, v.w);
    }
}

constexpr int kTileThreadsMax = 256;

// One hop of one field from shared memory.  The unscaled SU(3) product feeds the operator term
// (factor fa, into accA) and, where this field carries the derivative, the E term (factor fe,
// into accE; EMODE 2 multiplies by the direction links Y instead, read from global memory).
template <int EMODE, bool WITH_E, int NU, int SP>
__device__ __forceinline__ void tile_hop(const HopArgs& a, const TileGeom& g, int side, const float4* fs, int nb,
                                         const float2 (&u)[9], size_t lsite, float bsign, float2 (&accA)[12],
                                         float2 (&accE)[12]) {
    constexpr bool DAG = SP > 0;
    float2 psi[12], h[6], gv[6], tv[6];
    tile_spinor(fs, g.ntot, nb, psi);
    project<float2, NU, SP>(psi, h);
    su3_mul<float2, DAG>(u, h, gv);
    const float fa = fac_a<float>(a, side, NU, SP < 0) * bsign;
#pragma unroll
    for (int i = 0; i < 6; ++i) tv[i] = cscale(gv[i], fa);
    reconstruct_add<float2, NU, SP>(tv, accA);
    if (WITH_E) {
        const float fe = fac_e<float>(a, side, NU, SP < 0) * bsign;
        if (EMODE == 1 && NU == 3) {
#pragma unroll
            for (int i = 0; i < 6; ++i) tv[i] = cscale(gv[i], fe);
            reconstruct_add<float2, NU, SP>(tv, accE);
        } else if (EMODE == 2) {
            float2 y[9];
            load_link(reinterpret_cast<const float2*>(a.Y), a.V, NU, lsite, y);
            su3_mul<float2, DAG>(y, h, gv);
#pragma unroll
            for (int i = 0; i < 6; ++i) tv[i] = cscale(gv[i], fe);
            reconstruct_add<float2, NU, SP>(tv, accE);
        }
    }
}

template <int EMODE, bool WITH_E, int NU>
__device__ __forceinline__ void tile_dir(const HopArgs& a, const TileGeom& g, int side, const float4* fs, const float2* lf,
                                         const float2* lb, const int* map, int x, int ly, int lz, int lt, int gt, size_t s,
                                         float2 (&accA)[12], float2 (&accE)[12]) {
    const int c = x + g.nx * (ly + kTileY * (lz + kTileZ * lt));
    float2 u[9];
    // forward: psi(s + nu) through U_nu(s)
#pragma unroll
    for (int e = 0; e < 9; ++e) u[e] = lf[(NU * 9 + e) * g.ns + c];
    const float bf = (NU == 3 && a.apbc && gt == g.nt - 1) ? -1.f : 1.f;
    tile_hop<EMODE, WITH_E, NU, -1>(a, g, side, fs, tile_nb<NU, +1>(g, x, ly, lz, lt), u, s, bf, accA, accE);
    // backward: psi(s - nu) through U_nu(s - nu)^dag
    tile_back_link<NU>(g, lf, lb, x, ly, lz, lt, u);
    const int nbb = tile_nb<NU, -1>(g, x, ly, lz, lt);
    const float bb = (NU == 3 && a.apbc && gt == 0) ? -1.f : 1.f;
    tile_hop<EMODE, WITH_E, NU, +1>(a, g, side, fs, nbb, u, (size_t)map[nbb], bb, accA, accE);
}

template <int EMODE, bool WITH_E>
__device__ __forceinline__ void tile_phase(const HopArgs& a, const TileGeom& g, int side, const float4* fs, const float2* lf,
                                           const float2* lb, const int* map, int x, int ly, int lz, int lt, int gt, size_t s,
                                           float2 (&accA)[12], float2 (&accE)[12]) {
    tile_dir<EMODE, WITH_E, 0>(a, g, side, fs, lf, lb, map, x, ly, lz, lt, gt, s, accA, accE);
    tile_dir<EMODE, WITH_E, 1>(a, g, side, fs, lf, lb, map, x, ly, lz, lt, gt, s, accA, accE);
    tile_dir<EMODE, WITH_E, 2>(a, g, side, fs, lf, lb, map, x, ly, lz, lt, gt, s, accA, accE);
    tile_dir<EMODE, WITH_E, 3>(a, g, side, fs, lf, lb, map, x, ly, lz, lt, gt, s, accA, accE);
}

template <int EMODE, bool DOT>
__global__ void __launch_bounds__(kTileThreadsMax) k_hop_tiled(HopArgs a) {
    using C = float2;
    using Chunk = float4;
    extern __shared__ float4 tile_smem[];
    __shared__ CSum smem[32 * 2];
    const TileGeom g = tile_geom(a.dims);
    const int side = blockIdx.y + a.side0;
    const int src = blockIdx.z;
    if (a.state != nullptr && a.state[src].status != 0) return;   // source finished / failed
    char* base = reinterpret_cast<char*>(tile_smem);
    const size_t map_b = ((size_t)g.ntot * sizeof(int) + 15) / 16 * 16;
    const int nbk = g.fy + g.fz + g.ft;
    const size_t link_b = ((size_t)36 * g.ns + (size_t)9 * nbk) * sizeof(float2);
    int* map = reinterpret_cast<int*>(base);
    float2* lf = reinterpret_cast<float2*>(base + map_b);
    float2* lb = lf + (size_t)36 * g.ns;
    float4* fs = reinterpret_cast<float4*>(base + map_b + (link_b + 15) / 16 * 16);
    const int my = g.ny / kTileY, mz = g.nz / kTileZ;
    const int y0 = (int)(blockIdx.x % my) * kTileY;
    const int z0 = (int)((blockIdx.x / my) % mz) * kTileZ;
    const int t0 = (int)(blockIdx.x / (my * mz)) * kTileT;
    const size_t V = a.V;
    // global site of every tile and face entry
    for (int r = threadIdx.x; r < g.ntot; r += blockDim.x) {
        int x, ly, lz, lt;
        tile_decode(g, r, x, ly, lz, lt);
        const int gy = (y0 + ly + g.ny) % g.ny, gz = (z0 + lz + g.nz) % g.nz, gtt = (t0 + lt + g.nt) % g.nt;
        map[r] = x + g.nx * (gy + g.ny * (gz + g.nz * gtt));
    }
    __syncthreads();
    // links: forward links of the tile sites, backward links on the -y, -z, -t faces
    const float2* U = reinterpret_cast<const float2*>(a.U);
    for (int c = threadIdx.x; c < g.ns; c += blockDim.x) {
        const size_t sc = (size_t)map[c];
#pragma unroll 4
        for (int ne = 0; ne < 36; ++ne) cp_async8(lf + (size_t)ne * g.ns + c, U + (size_t)ne * V + sc);
    }
    for (int u = threadIdx.x; u < nbk; u += blockDim.x) {
        int nu, r;
        if (u < g.fy) { nu = 1; r = g.ns + u; }
        else if (u < g.fy + g.fz) { nu = 2; r = g.ns + 2 * g.fy + (u - g.fy); }
        else { nu = 3; r = g.ns + 2 * g.fy + 2 * g.fz + (u - g.fy - g.fz); }
        const size_t sr = (size_t)map[r];
#pragma unroll
        for (int e = 0; e < 9; ++e) cp_async8(lb + (size_t)e * nbk + u, U + (size_t)(nu * 9 + e) * V + sr);
    }
    const int t = threadIdx.x;
    const bool active = t < g.ns;
    int x = 0, ly = 0, lz = 0, lt = 0;
    size_t s = 0;
    if (active) { tile_decode(g, t, x, ly, lz, lt); s = (size_t)map[t]; }
    const int gt = t0 + lt;
    const size_t F = field_elems<float>(V);
    const Chunk* in = reinterpret_cast<const Chunk*>(a.in[side]) + (size_t)src * a.src_stride_in[side];
    Chunk* out = reinterpret_cast<Chunk*>(a.out[side]) + (size_t)src * a.src_stride_out[side];
    const Chunk* wl = reinterpret_cast<const Chunk*>(a.in[1]) + (size_t)src * a.src_stride_in[1];
    const float diag = fac_diag<float>(a);
    // the field without a derivative term in its own output goes first (see above)
    const int f1 = (side == 0) ? 1 : 0, f2 = 1 - f1;
    C acc1[12], acc2[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) { acc1[c] = cmk<C>(0.f, 0.f); acc2[c] = cmk<C>(0.f, 0.f); }
    DotAcc<float> d[2];
    d[0].zero(); d[1].zero();
    auto load_field = [&](int f) {   // asynchronous; completed by cp_async_wait_all + barrier
        const Chunk* inf = in + (size_t)f * F;
        for (int r = threadIdx.x; r < g.ntot; r += blockDim.x) {
            const size_t sr = (size_t)map[r];
#pragma unroll
            for (int q = 0; q < 6; ++q) cp_async16(fs + (size_t)q * g.ntot + r, inf + (size_t)q * V + sr);
        }
    };
    auto finish_field = [&](int f, C (&acc)[12]) {   // gamma5 (diag psi + hops), store, alpha dot
        C psi[12];
        tile_spinor(fs, g.ntot, t, psi);
        finish(psi, diag, acc);
        store_spinor(out + (size_t)f * F, V, s, acc);
        if (DOT && side == 0) {
            load_spinor(wl + (size_t)f * F, V, s, psi);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                add_cdot(d[0], d[1], psi[c], acc[c]);
            }
        }
    };
    load_field(f1);
    cp_async_wait_all();   // links and the first field
    __syncthreads();
    if (active) {
        tile_phase<EMODE, EMODE != 0>(a, g, side, fs, lf, lb, map, x, ly, lz, lt, gt, s, acc1, acc2);
        finish_field(f1, acc1);
    }
    __syncthreads();
    load_field(f2);
    cp_async_wait_all();
    __syncthreads();
    if (active) {
        tile_phase<EMODE, false>(a, g, side, fs, lf, lb, map, x, ly, lz, lt, gt, s, acc2, acc2);
        finish_field(f2, acc2);
    }
    if (DOT && side == 0) {
        CSum tot[2];
        block_total<float, 2>(d, tot, smem);
        double* part = a.partials + ((size_t)src * a.partial_stride + blockIdx.x) * 4;
        if (threadIdx.x == 0) { part[0] = tot[0].s; part[1] = tot[0].e; part[2] = tot[1].s; part[3] = tot[1].e; }
        if (last_block(a.counters + src, gridDim.x)) {
            double res[2];
            reduce_partials<2>(a.partials + (size_t)src * a.partial_stride * 4, gridDim.x, res, smem);
            if (threadIdx.x == 0) tsl_alpha_step(a, src, res[0], res[1]);
        }
    }
}

// ---------------------------------------------------------------------------------------
// out[src] = || a + sigma b ||^2 over one boundary-layout field per source (b may be null),
// compensated FP64.  One block per source.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_norm2(const double2* __restrict__ a, const double2* __restrict__ b, double sigma,
                                                size_t n, double* __restrict__ out) {
    __shared__ CSum smem[32];
    const int src = blockIdx.x;
    const double2* pa = a + (size_t)src * n;
    const double2* pb = b ? b + (size_t)src * n : nullptr;
    CSum acc{0.0, 0.0};
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
        double2 v = pa[i];
        if (pb) { double2 w = pb[i]; v.x += sigma * w.x; v.y += sigma * w.y; }
        cs_add_prod(acc, v.x, v.x);
        cs_add_prod(acc, v.y, v.y);
    }
    CSum v1[1] = {acc};
    block_reduce_cs<1>(v1, smem);
    if (threadIdx.x == 0) out[src] = v1[0].s + v1[0].e;
}

cudaError_t launch_norm2(const double* a, const double* b, double sigma, size_t n, int nsrc, double* out, cudaStream_t st) {
    k_norm2<<<nsrc, 1024, 0, st>>>(reinterpret_cast<const double2*>(a), reinterpret_cast<const double2*>(b), sigma, n, out);
    return cudaGetLastError();
}

// BF16 link storage: the FP64 boundary links are rounded in place (FP64 -> FP32 nearest -> BF16
// nearest even -> exact back to FP64), so that every FP64 user of them sees the stored values;
// the internal copy holds the BF16 pairs.
__global__ void k_links_bf16(double2* __restrict__ U, __nv_bfloat162* __restrict__ L, size_t V) {
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nu = blockIdx.y;
    if (s >= V) return;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        double2* p = U + ((size_t)nu * V + s) * 9 + e;
        const double2 z = *p;
        const __nv_bfloat162 b = __floats2bfloat162_rn((float)z.x, (float)z.y);
        const float2 r = __bfloat1622float2(b);
        *p = make_double2((double)r.x, (double)r.y);
        L[((size_t)nu * 9 + e) * V + s] = b;
    }
}

// ---------------------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------------------
template <typename R, int MINB>
static cudaError_t launch_hop_t(const HopArgs& a, int nf, int emode, bool dot, cudaStream_t st) {
    dim3 grid((unsigned)((a.V + kHopThreads - 1) / kHopThreads), (unsigned)a.nsides, (unsigned)a.nsrc);
    dim3 block(kHopThreads);
#define LQ_HOP(NF, EM, D) k_hop<R, NF, EM, D, MINB><<<grid, block, 0, st>>>(a)
    if (nf == 1) {
        if (dot) LQ_HOP(1, 0, true); else LQ_HOP(1, 0, false);
    } else {
        if (emode == 0) { if (dot) LQ_HOP(2, 0, true); else LQ_HOP(2, 0, false); }
        else if (emode == 1) { if (dot) LQ_HOP(2, 1, true); else LQ_HOP(2, 1, false); }
        else { if (dot) LQ_HOP(2, 2, true); else LQ_HOP(2, 2, false); }
    }
#undef LQ_HOP
    return cudaGetLastError();
}

template <typename R, int RS, int MINB>
static cudaError_t launch_roles_t(const HopArgs& a, int emode, bool dot, cudaStream_t st) {
    dim3 grid((unsigned)((a.V + RS - 1) / RS), (unsigned)a.nsrc, 1);
    dim3 block(4 * RS);
#define LQ_ROLE(EM, D) k_hop_roles<R, EM, D, RS, MINB><<<grid, block, 0, st>>>(a)
    if (emode == 0) { if (dot) LQ_ROLE(0, true); else LQ_ROLE(0, false); }
    else if (emode == 1) { if (dot) LQ_ROLE(1, true); else LQ_ROLE(1, false); }
    else { if (dot) LQ_ROLE(2, true); else LQ_ROLE(2, false); }
#undef LQ_ROLE
    return cudaGetLastError();
}

template <int EMODE, bool DOT>
static cudaError_t launch_tiled_k(const HopArgs& a, const TileGeom& g, dim3 grid, dim3 block, cudaStream_t st) {
    static bool attr = false;   // opt in to more than 48 KB of dynamic shared memory, once
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_hop_tiled<EMODE, DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_hop_tiled<EMODE, DOT><<<grid, block, g.smem, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_tiled_t(const HopArgs& a, int emode, bool dot, cudaStream_t st) {
    const TileGeom g = tile_geom(a.dims);
    const dim3 grid((unsigned)(a.V / (size_t)g.ns), (unsigned)a.nsides, (unsigned)a.nsrc);
    const dim3 block((unsigned)((g.ns + 31) / 32 * 32));
    if (emode == 0) return dot ? launch_tiled_k<0, true>(a, g, grid, block, st) : launch_tiled_k<0, false>(a, g, grid, block, st);
    if (emode == 1) return dot ? launch_tiled_k<1, true>(a, g, grid, block, st) : launch_tiled_k<1, false>(a, g, grid, block, st);
    return dot ? launch_tiled_k<2, true>(a, g, grid, block, st) : launch_tiled_k<2, false>(a, g, grid, block, st);
}

// Stencil schedules (chosen by the autotuner in the Lanczos driver):
//   0: one thread per (site, side), registers unconstrained
//   1: one thread per (site, output field), four roles of 32 sites per block
//   2: as 0 with at least 5 resident blocks per SM (register cap ~100)
//   3: as 0 with at least 4 resident blocks per SM (register cap 128)
//   4: as 1 with 64 sites per block and at least 2 resident blocks per SM (FP32)
//   5: as 1 with at least 5 resident blocks per SM (FP32)
//   6: shared-memory tiles of whole x rows x 2 x 2 x 2 (FP32; lattices with even y, z, t extents;
//      schedule 3 otherwise)
//   7: as 3 with packed FP32 pair arithmetic (lq_hop_x2.cu; identical results)
//   8: as 7 with the next hop's neighbour spinors prefetched into shared memory
//   9: as 3 with both sides of 64 sites in a block (the second load of a link hits L1)
cudaError_t launch_hop(int prec, const HopArgs& a, int nf, int emode, bool dot, cudaStream_t st) {
    if (prec == LQ_FLOAT_FLOAT) {   // schedules 0, 1 and 2
        if (nf == 2 && a.nsides == 2 && a.side0 == 0 && (a.variant == 1 || a.variant == 2))
            return emode == 0 ? launch_roles_ff0(a, dot, st) : emode == 1 ? launch_roles_ff1(a, dot, st) : launch_roles_ff2(a, dot, st);
        if (nf == 1 || emode == 0) return launch_hop_ff0(a, nf, dot, st);
        return emode == 1 ? launch_hop_ff1(a, dot, st) : launch_hop_ff2(a, dot, st);
    }
    const bool lanczos_block = nf == 2 && a.nsides == 2 && a.side0 == 0;
    if (a.link_bf16 && a.variant >= 6 && a.variant <= 8) {     // schedules 6-8 read FP32 links: BF16 links run 3
        HopArgs b = a;
        b.variant = 3;
        return launch_hop(prec, b, nf, emode, dot, st);
    }
    if (lanczos_block && prec != LQ_FP64 && (a.variant == 7 || a.variant == 8))
        return launch_hop_x2(a, emode, dot, a.variant == 8, st);
    if (lanczos_block && prec != LQ_FP64 && a.variant == 6) {
        if (tile_ok(a.dims)) return launch_tiled_t(a, emode, dot, st);
        return launch_hop_t<float, 4>(a, nf, emode, dot, st);
    }
    if (lanczos_block && a.variant == 1)
        return prec == LQ_FP64 ? launch_roles_t<double, kRoleSites, 1>(a, emode, dot, st)
                               : launch_roles_t<float, kRoleSites, 1>(a, emode, dot, st);
    if (lanczos_block && prec != LQ_FP64 && a.variant == 2) return launch_hop_t<float, 5>(a, nf, emode, dot, st);
    if (lanczos_block && prec != LQ_FP64 && a.variant == 3) return launch_hop_t<float, 4>(a, nf, emode, dot, st);
    if (lanczos_block && prec != LQ_FP64 && a.variant == 9) {
        const dim3 grid((unsigned)((a.V + kHopThreads / 2 - 1) / (kHopThreads / 2)), 1, (unsigned)a.nsrc);
#define LQ_HOP_P(EM, D) k_hop<float, 2, EM, D, 4, true><<<grid, kHopThreads, 0, st>>>(a)
        if (emode == 0) { if (dot) LQ_HOP_P(0, true); else LQ_HOP_P(0, false); }
        else if (emode == 1) { if (dot) LQ_HOP_P(1, true); else LQ_HOP_P(1, false); }
        else { if (dot) LQ_HOP_P(2, true); else LQ_HOP_P(2, false); }
#undef LQ_HOP_P
        return cudaGetLastError();
    }
    if (lanczos_block && prec != LQ_FP64 && a.variant == 4) return launch_roles_t<float, 2 * kRoleSites, 2>(a, emode, dot, st);
    if (lanczos_block && prec != LQ_FP64 && a.variant == 5) return launch_roles_t<float, kRoleSites, 5>(a, emode, dot, st);
    return prec == LQ_FP64 ? launch_hop_t<double, 1>(a, nf, emode, dot, st) : launch_hop_t<float, 1>(a, nf, emode, dot, st);
}

// Blocks per source of the grid-stride update: enough for exactly one resident wave over all
// sources (no partial last wave), at most one per 256 chunks and at most `cap` (the partials).
unsigned update_grid(size_t nelem, int nsrc, size_t cap) {
    static int resident = 0;   // blocks of k_update<float> resident on the whole GPU
    if (resident == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update<float>, kUpdThreads, 0);
        resident = std::max(1, sms * std::max(1, per_sm));
    }
    size_t b = std::max(1, resident / std::max(1, nsrc));
    b = std::min(b, std::max<size_t>(1, (nelem + kUpdThreads - 1) / kUpdThreads));
    b = std::min(b, std::max<size_t>(1, cap));
    return (unsigned)b;
}

cudaError_t launch_update(int prec, const UpdArgs& a, cudaStream_t st) {
    if (prec == LQ_MIXED && a.bulk && !a.defer && update_bulk_ready()) return launch_update_bulk(a, st);
    dim3 grid(update_grid(a.nelem, a.nsrc, a.partial_stride), (unsigned)a.nsrc);
    if (prec == LQ_FP64) k_update<double><<<grid, kUpdThreads, 0, st>>>(a);
    else if (prec == LQ_FLOAT_FLOAT) return launch_update_ff(a, grid, st);
    else k_update<float><<<grid, kUpdThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tsl_init(int prec, int nf, const InitArgs& a, cudaStream_t st) {
    dim3 grid((unsigned)((a.V + kUpdThreads - 1) / kUpdThreads), (unsigned)a.nsrc);
    if (prec == LQ_FP64) { if (nf == 1) k_tsl_init<double, 1><<<grid, kUpdThreads, 0, st>>>(a); else k_tsl_init<double, 2><<<grid, kUpdThreads, 0, st>>>(a); }
    else if (prec == LQ_FLOAT_FLOAT) return launch_tsl_init_ff(nf, a, grid, st);
    else { if (nf == 1) k_tsl_init<float, 1><<<grid, kUpdThreads, 0, st>>>(a); else k_tsl_init<float, 2><<<grid, kUpdThreads, 0, st>>>(a); }
    return cudaGetLastError();
}

cudaError_t launch_recombine(int prec, int nf, const RecArgs& a, cudaStream_t st) {
    dim3 grid((unsigned)((a.V + kRecThreads - 1) / kRecThreads), (unsigned)a.nsrc, (unsigned)nf);
    const size_t sm = (size_t)a.kmax * 16;   // one double2 (FP64) or float4 (FP32 hi/lo) per coefficient
    if (prec == LQ_FP64) {
        if (nf == 1) { cudaFuncSetAttribute(k_recombine<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); k_recombine<double, 1><<<grid, kRecThreads, sm, st>>>(a); }
        else { cudaFuncSetAttribute(k_recombine<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); k_recombine<double, 2><<<grid, kRecThreads, sm, st>>>(a); }
    } else if (prec == LQ_FLOAT_FLOAT) {
        return launch_recombine_ff(nf, a, grid, sm, st);
    } else {
        if (nf == 1) { cudaFuncSetAttribute(k_recombine<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); k_recombine<float, 1><<<grid, kRecThreads, sm, st>>>(a); }
        else { cudaFuncSetAttribute(k_recombine<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); k_recombine<float, 2><<<grid, kRecThreads, sm, st>>>(a); }
    }
    return cudaGetLastError();
}

cudaError_t launch_to_internal(int prec, const double* x, void* f, size_t V, int nfields, cudaStream_t st) {
    dim3 grid((unsigned)((V + 127) / 128), (unsigned)nfields);
    if (prec == LQ_FP64) k_to_internal<double><<<grid, 128, 0, st>>>(reinterpret_cast<const double2*>(x), reinterpret_cast<double2*>(f), V, nfields);
    else if (prec == LQ_FLOAT_FLOAT) return launch_to_internal_ff(x, f, V, nfields, grid, st);
    else k_to_internal<float><<<grid, 128, 0, st>>>(reinterpret_cast<const double2*>(x), reinterpret_cast<float4*>(f), V, nfields);
    return cudaGetLastError();
}

cudaError_t launch_to_boundary(int prec, const void* f, double* x, size_t V, int nfields, cudaStream_t st) {
    dim3 grid((unsigned)((V + 127) / 128), (unsigned)nfields);
    if (prec == LQ_FP64) k_to_boundary<double><<<grid, 128, 0, st>>>(reinterpret_cast<const double2*>(f), reinterpret_cast<double2*>(x), V, nfields);
    else if (prec == LQ_FLOAT_FLOAT) return launch_to_boundary_ff(f, x, V, nfields, grid, st);
    else k_to_boundary<float><<<grid, 128, 0, st>>>(reinterpret_cast<const float4*>(f), reinterpret_cast<double2*>(x), V, nfields);
    return cudaGetLastError();
}

cudaError_t launch_links_bf16(double* U, void* L, size_t V, cudaStream_t st) {
    dim3 grid((unsigned)((V + 127) / 128), 4);
    k_links_bf16<<<grid, 128, 0, st>>>(reinterpret_cast<double2*>(U), reinterpret_cast<__nv_bfloat162*>(L), V);
    return cudaGetLastError();
}

cudaError_t launch_links_internal(int prec, const double* U, void* L, size_t V, cudaStream_t st) {
    dim3 grid((unsigned)((V + 127) / 128), 4);
    if (prec == LQ_FP64) k_links_internal<double><<<grid, 128, 0, st>>>(reinterpret_cast<const double2*>(U), reinterpret_cast<double2*>(L), V);
    else if (prec == LQ_FLOAT_FLOAT) return launch_links_internal_ff(U, L, V, grid, st);
    else k_links_internal<float><<<grid, 128, 0, st>>>(reinterpret_cast<const double2*>(U), reinterpret_cast<float2*>(L), V);
    return cudaGetLastError();
}

cudaError_t launch_direction(int prec, const double* U, const double* w, int kind, void* Y, size_t V, cudaStream_t st) {
    dim3 grid((unsigned)((V + 127) / 128), 4);
    if (prec == LQ_FP64) k_direction<double><<<grid, 128, 0, st>>>(reinterpret_cast<const double2*>(U), w, kind, reinterpret_cast<double2*>(Y), V);
    else if (prec == LQ_FLOAT_FLOAT) return launch_direction_ff(U, w, kind, Y, V, grid, st);
    else k_direction<float><<<grid, 128, 0, st>>>(reinterpret_cast<const double2*>(U), w, kind, reinterpret_cast<float2*>(Y), V);
    return cudaGetLastError();
}

}  // namespace lq
