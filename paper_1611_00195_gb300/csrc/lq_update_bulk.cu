// FP32 update step of the two-sided Lanczos recurrences (Sec. 2) with its inputs staged by the
// copy engine: for each tile of kBuTile chunks the six input streams (B vh_j, vh_j, vh_{j-1} and
// B^dag wh_j, wh_j, wh_{j-1}) are fetched into shared memory by bulk asynchronous copies
// (cp.async.bulk, completion counted on an mbarrier), kBuStages tiles ahead of the threads that
// combine them.  The loads in flight live in shared memory, not in registers: a block of four
// warps keeps ~72 KB of HBM reads outstanding with 8 K registers.  Alone it moves the update's
// bytes at 0.78 of the measured HBM copy rate against 0.75 for the register-streaming k_update;
// beside the stencil (the split Krylov loop) its shared memory would take the L1 the stencil
// reuses its neighbour rows from, so that loop keeps k_update.  The arithmetic per element, the
// compensated dots and the scalar step are those of k_update (lq_stencil.cuh); the vectors are
// bitwise the same, the dots differ by the order of their (compensated) partial sums.
#include "lq_internal.cuh"
#include "lq_launch.h"
#include "lq_stencil.cuh"

#include <algorithm>

namespace lq {
namespace {

constexpr int kBuThreads = 128;
constexpr int kBuTile = 256;       // chunks (float4) per stream and tile: 4 KB
constexpr int kBuStages = 4;
constexpr int kBuStreams = 6;      // r, v, l, w, v_prev, w_prev
constexpr size_t kBuBufBytes = (size_t)kBuStages * kBuStreams * kBuTile * sizeof(float4);   // 96 KB
constexpr size_t kBuSmem = kBuBufBytes + kBuStages * sizeof(unsigned long long);
// polls of an mbarrier before a wait gives up (each poll may suspend the thread for a while in
// hardware); far beyond the microseconds a tile's copies take
constexpr long kBuWaitPolls = 1L << 22;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ size_t min_sz(size_t x, size_t y) { return x < y ? x : y; }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// one arrival that also announces `bytes` of copies to be counted on the barrier
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the completion of the barrier's phase with the given parity
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    for (long i = 0; i < kBuWaitPolls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__global__ void __launch_bounds__(kBuThreads, 8) k_update_bulk(UpdArgs a) {
    extern __shared__ __align__(128) unsigned char dsm[];
    float4* buf = reinterpret_cast<float4*>(dsm);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(dsm + kBuBufBytes);
    __shared__ CSum smem[32 * 6];
    const int src = blockIdx.y;
    TslState& st = a.state[src];
    if (st.status != 0) return;   // block-uniform, before any barrier or copy
    float2 cv[3], cw[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        cv[i] = make_float2((float)st.cv[i].x, (float)st.cv[i].y);
        cw[i] = make_float2((float)st.cw[i].x, (float)st.cw[i].y);
    }
    const bool has_prev = a.j > 0;
    const int nstream = has_prev ? 6 : 4;
    const size_t N = a.nelem;
    const float4* r = reinterpret_cast<const float4*>(a.rout) + (size_t)src * a.src_stride_io;
    const float4* l = reinterpret_cast<const float4*>(a.lout) + (size_t)src * a.src_stride_io;
    const float4* v = reinterpret_cast<const float4*>(a.v_cur) + (size_t)src * a.src_stride_basis;
    const float4* vp = reinterpret_cast<const float4*>(a.v_prev) + (size_t)src * a.src_stride_basis;
    float4* vn = reinterpret_cast<float4*>(a.v_next) + (size_t)src * a.src_stride_basis;
    const float4* w = reinterpret_cast<const float4*>(a.w_cur) + (size_t)src * a.src_stride_left;
    const float4* wp = reinterpret_cast<const float4*>(a.w_prev) + (size_t)src * a.src_stride_left;
    float4* wn = reinterpret_cast<float4*>(a.w_next) + (size_t)src * a.src_stride_left;
    float4* ws = a.w_store ? reinterpret_cast<float4*>(a.w_store) + (size_t)src * a.src_stride_store : nullptr;

    // tiles t = b, b + nb, ... of this source
    const size_t nb = gridDim.x, b = blockIdx.x;
    const size_t ntiles = (N + kBuTile - 1) / kBuTile;
    const long nmine = b < ntiles ? (long)((ntiles - b + nb - 1) / nb) : 0;
    if (threadIdx.x == 0) {
        for (int q = 0; q < kBuStages; ++q) mbar_init(&bar[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    long issued = 0;   // thread 0: tiles whose copies were started
    auto issue = [&](long i) {
        const size_t e0 = (b + (size_t)i * nb) * kBuTile;
        const unsigned bytes = (unsigned)(min_sz((size_t)kBuTile, N - e0) * sizeof(float4));
        float4* sb = buf + (size_t)(i % kBuStages) * kBuStreams * kBuTile;
        unsigned long long* br = &bar[i % kBuStages];
        mbar_arrive_expect_tx(br, bytes * (unsigned)nstream);
        bulk_load(sb, r + e0, bytes, br);
        bulk_load(sb + kBuTile, v + e0, bytes, br);
        bulk_load(sb + 2 * kBuTile, l + e0, bytes, br);
        bulk_load(sb + 3 * kBuTile, w + e0, bytes, br);
        if (has_prev) {
            bulk_load(sb + 4 * kBuTile, vp + e0, bytes, br);
            bulk_load(sb + 5 * kBuTile, wp + e0, bytes, br);
        }
    };
    if (threadIdx.x == 0)
        for (; issued < nmine && issued < kBuStages; ++issued) issue(issued);

    DotAcc<float> d[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i].zero();
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    long i = 0;
    for (; i < nmine; ++i) {
        const int sg = (int)(i % kBuStages);
        const bool got = mbar_wait(&bar[sg], (unsigned)((i / kBuStages) & 1));
        if (__syncthreads_or(!got)) break;   // a copy did not land: give up (block-uniform)
        const size_t e0 = (b + (size_t)i * nb) * kBuTile;
        const int n = (int)min_sz((size_t)kBuTile, N - e0);
        const float4* sb = buf + (size_t)sg * kBuStreams * kBuTile;
        for (int q = threadIdx.x; q < n; q += kBuThreads) {
            const float4 r0 = sb[q], v0 = sb[kBuTile + q], l0 = sb[2 * kBuTile + q], w0 = sb[3 * kBuTile + q];
            const float4 p0 = has_prev ? sb[4 * kBuTile + q] : zero, q0 = has_prev ? sb[5 * kBuTile + q] : zero;
            const float4 nv = axpy3<float>(r0, v0, p0, cv, has_prev);
            const float4 nw = axpy3<float>(l0, w0, q0, cw, has_prev);
            vn[e0 + q] = nv;
            wn[e0 + q] = nw;
            if (ws) ws[e0 + q] = nw;
            dot_chunk<float>(d, nw, nv);
            norm_chunk(d, r0, l0);
        }
        __syncthreads();   // the stage is read: it may be refilled
        if (threadIdx.x == 0 && issued < nmine) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(issued);
            ++issued;
        }
    }
    if (i < nmine && threadIdx.x == 0) {
        // gave up: flag the source, then let the copies still in flight land before the block's
        // shared memory is released (again with a bounded wait)
        st.status = LQ_ERR_TIMEOUT;
        for (long q = i; q < issued; ++q) (void)mbar_wait(&bar[q % kBuStages], (unsigned)((q / kBuStages) & 1));
    }
    CSum tot[6];
    block_total<float, 6>(d, tot, smem);
    double* part = a.partials + ((size_t)src * a.partial_stride + blockIdx.x) * 12;
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) { part[2 * k] = tot[k].s; part[2 * k + 1] = tot[k].e; }
    if (last_block(a.counters + a.nsrc + src, gridDim.x)) {
        double res[6];
        reduce_partials<6>(a.partials + (size_t)src * a.partial_stride * 12, gridDim.x, res, smem);
        if (threadIdx.x == 0 && st.status == 0) update_scalars<float>(a, src, res);
    }
}

}  // namespace

size_t update_bulk_smem() { return kBuSmem; }

// Blocks per source: two resident blocks per SM over all sources (at most `cap`, the partials;
// at most one per tile).
unsigned update_bulk_grid(size_t nelem, int nsrc, size_t cap) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        sms = std::max(1, sms);
    }
    size_t g = std::max<size_t>(1, (size_t)(2 * sms) / (size_t)std::max(1, nsrc));
    g = std::min(g, std::max<size_t>(1, (nelem + kBuTile - 1) / kBuTile));
    g = std::min(g, std::max<size_t>(1, cap));
    return (unsigned)g;
}

// One-time opt-in to the kernel's dynamic shared memory (above the 48 KB default).
bool update_bulk_ready() {
    static int ok = -1;
    if (ok < 0) {
        ok = cudaFuncSetAttribute(k_update_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBuSmem) == cudaSuccess;
        if (!ok) cudaGetLastError();
    }
    return ok == 1;
}

void update_bulk_prepare() {
    (void)update_bulk_ready();
    (void)update_bulk_grid(1, 1, 1);
}

cudaError_t launch_update_bulk(const UpdArgs& a, cudaStream_t st) {
    const dim3 grid(update_bulk_grid(a.nelem, a.nsrc, a.partial_stride), (unsigned)a.nsrc);
    k_update_bulk<<<grid, kBuThreads, kBuSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace lq
