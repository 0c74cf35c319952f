// Host implementation of the C ABI declared in include/lq.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <complex>
#include <cstring>
#include <functional>
#include <mutex>
#include <numeric>
#include <new>
#include <string>
#include <vector>

#include "lq_internal.cuh"
#include "lq_launch.h"
#include "lq_dense.h"

using namespace lq;

namespace {

int set_err(lq_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define LQ_CUDA(ctx, call)                                                                  \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return set_err(ctx, LQ_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// ---- opt-in kernel timing ---------------------------------------------------------------
enum { PC_HOP = 0, PC_UPDATE = 1, PC_NEWTON = 2, PC_OTHER = 3 };

cudaEvent_t prof_event(lq_ctx* c) {
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

// Mark the start of a timed region of class `cls`; returns the start event (or null).
cudaEvent_t prof_begin(lq_ctx* c, cudaStream_t st) {
    if (!c->prof_on) return nullptr;
    cudaEvent_t a = prof_event(c);
    if (a) cudaEventRecord(a, st);
    return a;
}
void prof_end(lq_ctx* c, int cls, cudaEvent_t a, cudaStream_t st, long long count = 1) {
    c->prof_n[cls] += count;
    if (!c->prof_on || !a) return;
    cudaEvent_t b = prof_event(c);
    if (!b) return;
    cudaEventRecord(b, st);
    c->pending.push_back({cls, a, b});
}
// After a stream synchronisation: fold the recorded pairs into the totals.
void prof_collect(lq_ctx* c) {
    for (auto& p : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) c->prof_ms[p.cls] += ms;
        else cudaGetLastError();
    }
    c->pending.clear();
    c->ev_used = 0;
}

// 1 = device (or managed) memory of this process, 0 = host memory, -1 = unusable.
int is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) { cudaGetLastError(); return 0; }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return 1;
    return 0;
}

template <typename T>
int dalloc(lq_ctx* c, T** p, size_t count) {
    if (*p) { cudaFree(*p); *p = nullptr; }
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_err(c, LQ_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed: " + cudaGetErrorString(e));
    }
    return LQ_OK;
}

void dfree(void* p) { if (p) cudaFree(p); }

// Chunk elements / bytes of one field in the internal layout of precision prec (FP64 and
// float-float: 12 chunks of 16 bytes per site; FP32: 6)
size_t field_elems_of(int prec, size_t V) { return prec == LQ_MIXED ? field_elems<float>(V) : field_elems<double>(V); }
size_t field_bytes_of(int prec, size_t V) { return prec == LQ_MIXED ? field_bytes<float>(V) : field_bytes<double>(V); }
size_t fe(const lq_ctx* c) { return field_elems_of(c->prec, c->V); }   // Chunk elements of one field
size_t fb(const lq_ctx* c) { return field_bytes_of(c->prec, c->V); }   // bytes of one field
size_t chunk_bytes(const lq_ctx* c) { return c->prec == LQ_FP64 ? sizeof(double2) : sizeof(float4); }
// bytes of one complex link entry in the internal layout (BF16: two bfloat16)
size_t link_entry_bytes(const lq_ctx* c) {
    if (c->prec == LQ_MIXED) return c->link_bf16 ? (size_t)4 : sizeof(float2);
    return 16;   // double2, or float-float (hi, lo) x (re, im)
}


// Copy n doubles from a caller buffer (host or device) into device memory.
int stage_in(lq_ctx* c, double* dst, const double* src, size_t n, cudaStream_t st) {
    LQ_CUDA(c, cudaMemcpyAsync(dst, src, n * sizeof(double), is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    return LQ_OK;
}
int stage_out(lq_ctx* c, double* dst, const double* src, size_t n, cudaStream_t st) {
    LQ_CUDA(c, cudaMemcpyAsync(dst, src, n * sizeof(double), is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    return LQ_OK;
}

// Hop factors (-1/2 of Dw included).  dagger = 0: H(mu); 1: H(mu)^dag = H(-mu).
void op_factors(double mu, int dagger, double (&f)[4], double (&b)[4]) {
    for (int nu = 0; nu < 3; ++nu) { f[nu] = -0.5; b[nu] = -0.5; }
    const double m = dagger ? -mu : mu;
    f[3] = -0.5 * std::exp(m);
    b[3] = -0.5 * std::exp(-m);
}
// Derivative factors.  emode 1 (d/dmu): E = dH/dmu has f+ = e^mu, f- = -e^-mu on time hops;
// E^dag = gamma5 W(conj f-, conj f+).  emode 2 (links Y): same factors as the operator.
void der_factors(double mu, int emode, int dagger, double (&f)[4], double (&b)[4]) {
    for (int nu = 0; nu < 4; ++nu) { f[nu] = 0.0; b[nu] = 0.0; }
    if (emode == 1) {
        if (!dagger) { f[3] = -0.5 * std::exp(mu); b[3] = 0.5 * std::exp(-mu); }
        else { f[3] = 0.5 * std::exp(-mu); b[3] = -0.5 * std::exp(mu); }
    } else if (emode == 2) {
        op_factors(mu, dagger, f, b);
    }
}

HopArgs base_hop(const lq_ctx* c) {
    HopArgs a;
    std::memset(&a, 0, sizeof(a));
    for (int i = 0; i < 4; ++i) a.dims[i] = c->dims[i];
    a.strides[0] = 1;
    a.strides[1] = (size_t)c->dims[0];
    a.strides[2] = (size_t)c->dims[0] * c->dims[1];
    a.strides[3] = (size_t)c->dims[0] * c->dims[1] * c->dims[2];
    a.V = c->V;
    a.apbc = c->desc.t_antiperiodic ? 1 : 0;
    a.diag = 4.0 * c->desc.r + c->desc.m_w;
    a.diag_f = (float)a.diag;
    a.U = c->U;
    a.link_bf16 = c->link_bf16 ? 1 : 0;
    a.Y = c->Y;
    a.Up = c->Up;
    a.Yp = c->Yp;
    return a;
}

void set_side(HopArgs& a, int side, const lq_ctx* c, int dagger, int emode) {
    op_factors(c->desc.mu, dagger, a.a_fwd[side], a.a_bwd[side]);
    der_factors(c->desc.mu, emode, dagger, a.e_fwd[side], a.e_bwd[side]);
    for (int nu = 0; nu < 4; ++nu) {
        a.af_fwd[side][nu] = (float)a.a_fwd[side][nu];
        a.af_bwd[side][nu] = (float)a.a_bwd[side][nu];
        a.ef_fwd[side][nu] = (float)a.e_fwd[side][nu];
        a.ef_bwd[side][nu] = (float)a.e_bwd[side][nu];
    }
}

int check_ready(lq_ctx* c, int nsrc, int need_block) {
    if (!c) return LQ_ERR_ARG;
    if (!c->gauge_ready) return set_err(c, LQ_ERR_NOT_READY, "gauge field not uploaded");
    if (!c->basis) return set_err(c, LQ_ERR_NOT_READY, "workspace not reserved (lq_reserve)");
    if (nsrc < 1 || nsrc > c->nsrc) return set_err(c, LQ_ERR_ARG, "nsrc must be in [1, reserved nsrc]");
    if (need_block && !c->block) return set_err(c, LQ_ERR_NOT_READY, "workspace reserved without block = 1");
    return LQ_OK;
}

int emode_of(const lq_ctx* c) {
    if (c->dir_kind == LQ_DIR_MU) return 1;
    if (c->dir_kind == LQ_DIR_SU3 || c->dir_kind == LQ_DIR_U1) return 2;
    return 0;
}

// Run the Newton iteration to convergence on the batch in `a` (already initialised).
int run_newton(lq_ctx* c, const NewtonArgs& a, cudaStream_t st, std::vector<double>& scal) {
    scal.assign((size_t)a.nb * 16, 0.0);
    for (int it = 0; it < a.max_iter; ++it) {
        cudaEvent_t e = prof_begin(c, st);
        LQ_CUDA(c, newton_iteration(a, st));
        prof_end(c, PC_NEWTON, e, st);
        c->launches += a.k + 3;
        LQ_CUDA(c, cudaMemcpyAsync(scal.data(), a.scal, scal.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        LQ_CUDA(c, cudaStreamSynchronize(st));
        bool all = true;
        for (int b = 0; b < a.nb; ++b) all = all && scal[(size_t)b * 16 + NS_DONE] != 0.0;
        if (all) break;
    }
    return LQ_OK;
}

NewtonArgs newton_args(lq_ctx* c, int k, int nb, int max_iter, double tol) {
    NewtonArgs a;
    std::memset(&a, 0, sizeof(a));
    a.k = k;
    a.nb = nb;
    a.ld = c->kmax;
    a.X = c->nx_X;
    a.Y = c->nx_Y;
    a.F = c->nx_F;
    a.perm = c->nx_perm;
    a.scal = c->nx_scal;
    a.partials = c->nx_partials;
    a.partial_stride = c->nx_partial_blocks;
    a.counters = c->nx_counters;
    a.tol = tol;
    a.max_iter = max_iter;
    a.state = c->state;
    a.alpha = c->alpha;
    a.beta = c->beta;
    a.delta = c->delta;
    a.kmax = c->kmax;
    return a;
}

// CUDA graphs of ragged batches (lq_batch_apply): one per batch configuration, keyed by each
// member context and the configuration of its run; shared by all contexts of the process.
struct BatchGraph {
    std::vector<std::pair<lq_ctx*, lq_ctx::GraphKey>> key;
    cudaGraphExec_t exec;
};
std::mutex g_batch_mu;
std::vector<BatchGraph> g_batch_graphs;

// Drop every batch graph that launches kernels on c's workspace.
void clear_batch_graphs(const lq_ctx* c) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t i = 0; i < g_batch_graphs.size();) {
        bool hit = false;
        for (auto& kv : g_batch_graphs[i].key) hit = hit || kv.first == c;
        if (hit) {
            cudaGraphExecDestroy(g_batch_graphs[i].exec);
            g_batch_graphs.erase(g_batch_graphs.begin() + (long)i);
        } else {
            ++i;
        }
    }
}

void clear_graphs(lq_ctx* c) {
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
    clear_batch_graphs(c);
}

void free_workspace(lq_ctx* c) {
    clear_graphs(c);
    void** ps[] = {&c->basis, &c->left, &c->rout, &c->lout, (void**)&c->io, (void**)&c->norms, (void**)&c->partials, (void**)&c->counters,
                   (void**)&c->state, (void**)&c->alpha, (void**)&c->beta, (void**)&c->delta, (void**)&c->scale,
                   (void**)&c->nx_X, (void**)&c->nx_Y, (void**)&c->nx_F, (void**)&c->nx_perm, (void**)&c->nx_scal,
                   (void**)&c->nx_partials, (void**)&c->nx_counters, (void**)&c->proj_c, (void**)&c->quad_q,
                   (void**)&c->quad_work, (void**)&c->quad_c, (void**)&c->quad_check, (void**)&c->quad_nodes, (void**)&c->quad_part, (void**)&c->proj_sel,
                   (void**)&c->nest_state, (void**)&c->nest_alpha, (void**)&c->nest_beta, (void**)&c->nest_delta, (void**)&c->nest_s,
                   (void**)&c->nest_q, (void**)&c->nest_norm, (void**)&c->nest_check, (void**)&c->nest_c,
                   &c->lbasis, (void**)&c->uscale, (void**)&c->adj_coef, &c->adj_nu, &c->adj_om,
                   (void**)&c->adj_force, (void**)&c->adj_dmu, (void**)&c->gen_scr, (void**)&c->solve_ws,
                   (void**)&c->rb_part, (void**)&c->rb_coef, (void**)&c->rb_coef_f};
    for (void** p : ps) { dfree(*p); *p = nullptr; }
    c->kmax = c->nsrc = c->block = c->ring = 0;
    c->lbasis_nf = 0;
    c->adjoint = false;
    c->rebiorth = false;
}

// Choose the stencil schedule for the Lanczos step: time each variant on the caller's data with
// the launch the loop makes (alpha dot included), twice round, and keep the fastest for this
// context and batch size.  The launches run step j = 0 on the freshly initialised state; the
// loop's own first step recomputes everything they write (outputs, alpha_0, the step's
// coefficients), so the tuning leaves no trace in the results.
int tune_hop(lq_ctx* c, HopArgs h, int nf, int emode, cudaStream_t st, int* variant) {
    if (nf != 2) { *variant = 0; return LQ_OK; }
    const int nvar = c->prec == LQ_FP64 ? 2 : (c->prec == LQ_FLOAT_FLOAT ? 3 : kHopSchedules);
    // candidates: FP64 0-1; FP32 all but the packed schedules 7 and 8 (bitwise the same as 3 and
    // measured slower on every lattice tried: they remain selectable through opts.hop_variant);
    // BF16 links without 6 (it reads FP32 links)
    auto candidate = [&](int v) { return !(v == 6 && (!tile_ok(h.dims) || c->link_bf16)) && v != 7 && v != 8; };
    for (const auto& t : c->tuned)
        if (t.nsrc == h.nsrc && t.nf == nf && t.emode == emode) { *variant = t.variant; return LQ_OK; }
    h.j = 0;
    h.kmax_run = std::max(h.kmax_run, 2);   // never mark a source finished while tuning
    cudaEvent_t e0, e1;
    LQ_CUDA(c, cudaEventCreate(&e0));
    LQ_CUDA(c, cudaEventCreate(&e1));
    std::vector<float> best(nvar, 1e30f);
    // three rounds over the candidates, six timed launches each after a warm-up: the minimum
    // over the rounds is robust to the noise of a shared machine
    for (int round = 0; round < 3; ++round)
        for (int v = 0; v < nvar; ++v) {
            if (!candidate(v)) continue;
            h.variant = v;
            LQ_CUDA(c, launch_hop(c->prec, h, nf, emode, true, st));   // warm-up
            LQ_CUDA(c, cudaEventRecord(e0, st));
            for (int i = 0; i < 6; ++i) LQ_CUDA(c, launch_hop(c->prec, h, nf, emode, true, st));
            LQ_CUDA(c, cudaEventRecord(e1, st));
            LQ_CUDA(c, cudaEventSynchronize(e1));
            float ms = 0.f;
            LQ_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
            c->launches += 7;
            best[v] = std::min(best[v], ms);
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int bestv = (int)(std::min_element(best.begin(), best.end()) - best.begin());
    c->tuned.push_back({h.nsrc, nf, emode, bestv});
    *variant = bestv;
    return LQ_OK;
}

// The nested two-sided Lanczos projected sign (lq_nested.cu, Sec. 4) for the sources with
// sel[s] != 0: sgn(T) e_1 into out [nb][kmax] from the context's coefficient arrays (k_eff from
// `state`, or kfix for every source when state is null), with scales cscale [nb] (device); the
// involution residual of the second pass into check (host; +inf where an inner Newton iteration
// failed).  Pass 1 starts at e_1, pass 2 at the result of pass 1.
int nested_run(lq_ctx* c, const TslState* state, int kfix, int nb, int m, const double* cscale, const std::vector<int>& sel,
               double2* out, std::vector<double>& check, int newton_max_iter, double newton_tol, cudaStream_t st) {
    NestArgs na;
    std::memset(&na, 0, sizeof(na));
    na.nb = nb; na.kmax = c->kmax; na.kfix = kfix; na.m = m; na.state = state;
    na.alpha = c->alpha; na.beta = c->beta; na.delta = c->delta; na.cscale = cscale;
    na.work = c->quad_work; na.work_stride = (size_t)4 * c->kmax * 2 * kQuadRetryMaxNodes;
    if (nest_work_entries(c->kmax, m) > na.work_stride) return set_err(c, LQ_ERR_ARG, "nested inner size too large for the workspace");
    na.istate = c->nest_state; na.ialpha = c->nest_alpha; na.ibeta = c->nest_beta; na.idelta = c->nest_delta;
    na.snorm = c->nest_norm; na.sel = c->proj_sel;
    LQ_CUDA(c, cudaMemcpyAsync(c->proj_sel, sel.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
    LQ_CUDA(c, nest_factor(na, st));
    c->launches += 1;
    std::vector<int> bad(nb, 0);
    std::vector<double> scal;
    const double one = 1.0;
    for (int pass = 0; pass < 2; ++pass) {
        na.start = pass ? out : nullptr;
        cudaEvent_t e = prof_begin(c, st);
        LQ_CUDA(c, nest_lanczos(na, st));
        prof_end(c, PC_NEWTON, e, st, 0);
        NewtonArgs nw = newton_args(c, m, nb, newton_max_iter, newton_tol);
        nw.state = c->nest_state; nw.alpha = c->nest_alpha; nw.beta = c->nest_beta; nw.delta = c->nest_delta;
        LQ_CUDA(c, newton_init_tridiag(nw, st));
        for (int s = 0; s < nb; ++s)
            if (!sel[s]) LQ_CUDA(c, cudaMemcpyAsync(c->nx_scal + (size_t)s * 16 + NS_DONE, &one, sizeof(double), cudaMemcpyHostToDevice, st));
        c->launches += 2;
        int r = run_newton(c, nw, st, scal);
        if (r) return r;
        for (int s = 0; s < nb; ++s) if (sel[s] && scal[(size_t)s * 16 + NS_STATUS] != 0.0) bad[s] = 1;
        LQ_CUDA(c, newton_first_column(nw, c->nest_s, c->kmax, st, c->proj_sel));
        LQ_CUDA(c, nest_combine(na, c->nest_s, pass ? c->nest_q : out, st));
        c->launches += 2;
    }
    LQ_CUDA(c, nest_check(na, c->nest_q, c->nest_check, st));
    c->launches += 1;
    check.assign(nb, 0.0);
    LQ_CUDA(c, cudaMemcpyAsync(check.data(), c->nest_check, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    LQ_CUDA(c, cudaStreamSynchronize(st));
    for (int s = 0; s < nb; ++s) if (bad[s]) check[s] = INFINITY;
    return LQ_OK;
}

// The Lanczos driver shared by lq_sign_apply (nf = 1), lq_sign_derivative_apply (nf = 2) and
// lq_batch_apply.  The source is staged in c->io (region 0, boundary layout) unless x_dev names
// another device buffer; results go to the device boundary-layout buffers y0 (field 0: sign, or
// top = derivative) and y1 (field 1: bottom = sign).  A run goes through phases so that a batch
// of contexts can interleave them on separate streams: setup (launch arguments, start vectors,
// stencil schedule), the Krylov loop, the projected sign (enqueued, then completed on the host),
// and the recombination with the reports (enqueued, then completed).
enum { FN_SIGN = 0, FN_RESOLVENT = 1 };

// lq_opts.rebiorth = p: the pair made by the update of step j (v_{j+1}, w_{j+1}, counting from
// v_0) is re-biorthogonalised when j + 1 or j is a multiple of p (j > 0): two consecutive pairs
// per period, since the recurrence forms each new pair from the last two and a lone corrected
// pair would hand the lost biorthogonality straight to the next one
inline bool rb_corrects(int p, int j) { return p > 0 && ((j + 1) % p == 0 || (j > 0 && j % p == 0)); }

struct TslRun {
    lq_ctx* c = nullptr;
    int nf = 1, emode = 0, nsrc = 0, fn = FN_SIGN;
    const lq_opts* o = nullptr;
    lq_report* rep = nullptr;
    double* y0 = nullptr;
    double* y1 = nullptr;
    const double2* shifts = nullptr;
    bool store_left = false;
    int s0 = 0;                // first source of this run in the context's per-source arrays
    bool args_only = false;    // build the launch arguments only (no start vectors, no tuning)

    int k = 0, ring = 0;
    bool two = false;
    int rb = 0;                // re-biorthogonalisation period (0: none)
    bool keep_left = false;    // the left vectors are stored in c->lbasis (adjoint or re-biorthogonalisation)
    size_t F = 0, vstride = 0, sst = 0, cb = 0, sb = 0, sl = 0, sio = 0;
    InitArgs ia;
    HopArgs h;
    UpdArgs u;
    RecArgs ra;
    QuadArgs qa;
    std::vector<double> scal, check;
    std::vector<int> used, nodes;
    int quad_attempt = -1;   // quadrature passes enqueued so far - 1; -1: no quadrature
    // second pass of a two-pass run: called after each window [j0, j1) is recombined, while its
    // right and left vectors are still in the rings (the adjoint accumulates its pair vectors)
    std::function<int(int, int, cudaStream_t)> on_window;

    void* bvec(int j) const {
        return reinterpret_cast<char*>(c->basis) + ((size_t)s0 * sb + (size_t)(ring ? j % ring : j) * vstride) * cb;
    }
    void* lvec(int j) const { return reinterpret_cast<char*>(c->left) + ((size_t)s0 * sl + (size_t)(j % 3) * vstride) * cb; }
    void* ofs(void* base, size_t chunks) const { return reinterpret_cast<char*>(base) + (size_t)s0 * chunks * cb; }

    int init(cudaStream_t st) {
        cudaEvent_t e0 = prof_begin(c, st);
        LQ_CUDA(c, launch_tsl_init(c->prec, nf, ia, st));
        prof_end(c, PC_OTHER, e0, st);
        c->launches += 1;
        return LQ_OK;
    }

    // Launch arguments and start vectors (on st); the stencil schedule (the autotuner launches
    // on st and synchronises it the first time a configuration is met).
    int setup(cudaStream_t st, const double* x_dev, const double* x_top) {
        k = o->kmax;
        F = fe(c);
        vstride = (size_t)nf * F;                    // Chunk elements per Krylov vector
        const int slots = c->ring > 0 ? c->ring : c->kmax;   // basis vectors held per source
        sb = (size_t)slots * vstride;                // per source: basis
        sl = 3 * vstride;                            // per source: left ring
        sio = vstride;                               // per source: operator outputs
        cb = chunk_bytes(c);
        // Two-pass run (lq_opts.two_pass): the first pass keeps only a ring of basis vectors and
        // yields T_k; the second reruns the same (deterministic) process and recombines windows
        // of kTwoPassWindow vectors into y while they are still in the ring.
        two = o->two_pass != 0 && k > 1;
        ring = two ? std::min(slots, kTwoPassRing) : 0;
        // lq_opts.rebiorth: the new pair is re-biorthogonalised every rb steps against the whole
        // right basis and the stored left basis (sign and derivative solves; not the adjoint)
        rb = (o->rebiorth > 0 && fn == FN_SIGN && !store_left && !two) ? o->rebiorth : 0;
        keep_left = store_left || rb > 0;
        sst = (size_t)slots * vstride;               // per source: stored left basis, ring or full

        // per-source arrays from source s0 on (a source group of a split run); the group's
        // last-block counters are a block of 3 nsrc from 3 s0 on
        const size_t xs = (size_t)s0 * c->V * 24;
        TslState* state = c->state + s0;
        double* partials = c->partials + (size_t)s0 * c->partial_blocks * 12;   // 12 doubles per block and source
        int* counters = c->counters + (size_t)3 * s0;
        const size_t ks = (size_t)s0 * c->kmax;
        std::memset(&ia, 0, sizeof(ia));
        ia.V = c->V; ia.nsrc = nsrc; ia.x = (x_dev ? x_dev : c->io) + xs; ia.xt = x_top ? x_top + xs : nullptr;
        ia.v1 = bvec(0); ia.w1 = lvec(0);
        ia.src_stride_basis = sb; ia.src_stride_left = sl; ia.state = state;
        ia.partials = partials; ia.partial_stride = c->partial_blocks; ia.counters = counters;
        ia.breakdown_tol = o->breakdown_tol;
        if (keep_left) { ia.w1_store = reinterpret_cast<char*>(c->lbasis) + (size_t)s0 * sst * cb; ia.src_stride_store = sst; }
        int r = args_only ? LQ_OK : init(st);
        if (r) return r;

        h = base_hop(c);
        h.nsrc = nsrc; h.nsides = 2; h.side0 = 0;
        set_side(h, 0, c, 0, emode);
        set_side(h, 1, c, 1, emode);
        h.state = state; h.partials = partials; h.partial_stride = c->partial_blocks; h.counters = counters;
        h.alpha = c->alpha + ks; h.scale = c->scale + ks; h.kmax = c->kmax; h.kmax_run = k;
        h.uscale = keep_left ? c->uscale + ks : nullptr;
        h.src_stride_in[0] = sb; h.src_stride_in[1] = sl;
        h.src_stride_out[0] = sio; h.src_stride_out[1] = sio;
        h.out[0] = ofs(c->rout, sio); h.out[1] = ofs(c->lout, sio);
        if (args_only) {
            h.variant = 0;
        } else if (o->hop_variant >= 0) {
            // the schedule that actually runs (and is reported): FP64 has schedules 0 and 1 only,
            // the plain operator 0 only, and schedule 6 needs tiles that cover the lattice
            int v = (nf == 2) ? o->hop_variant : 0;
            if (c->prec == LQ_FP64 && v > 1) v = 0;
            if (c->prec == LQ_FLOAT_FLOAT && v > 2) v = 0;
            if (v == 6 && !tile_ok(h.dims)) v = 3;
            if (c->link_bf16 && v >= 6 && v <= 8) v = 3;
            h.variant = v;
        } else {
            h.in[0] = bvec(0);
            h.in[1] = lvec(0);
            int v = 0;
            if ((r = tune_hop(c, h, nf, emode, st, &v))) return r;
            h.variant = v;
        }

        std::memset(&u, 0, sizeof(u));
        u.nelem = vstride; u.nsrc = nsrc; u.rout = ofs(c->rout, sio); u.lout = ofs(c->lout, sio);
        u.src_stride_io = sio; u.src_stride_basis = sb; u.src_stride_left = sl;
        u.state = state; u.partials = partials; u.partial_stride = c->partial_blocks; u.counters = counters;
        u.beta = c->beta + ks; u.delta = c->delta + ks; u.kmax = c->kmax;
        u.bulk = o->update_variant != 0 ? 1 : 0;
        if (keep_left) u.src_stride_store = sst;

        std::memset(&ra, 0, sizeof(ra));
        ra.V = c->V; ra.nsrc = nsrc; ra.basis = c->basis; ra.src_stride_basis = sb; ra.vec_stride = vstride;
        ra.state = c->state; ra.scale = c->scale; ra.kmax = c->kmax; ra.coef = c->proj_c;
        ra.y0 = y0; ra.y1 = y1; ra.ring = ring;

        scal.assign((size_t)nsrc * 16, 0.0);
        check.assign(nsrc, 0.0);   // stays 0 when the quadrature is not attempted
        used.assign(nsrc, LQ_PROJ_NEWTON);
        quad_attempt = -1;
        return LQ_OK;
    }

    int recombine(int j0, int j1, cudaStream_t st) {   // y (+)= |x| sum_{j0 <= j < j1} c_j s_j vh_j
        ra.j0 = j0; ra.j1 = j1; ra.accumulate = j0 > 0 ? 1 : 0;
        cudaEvent_t er = prof_begin(c, st);
        LQ_CUDA(c, launch_recombine(c->prec, nf, ra, st));
        prof_end(c, PC_OTHER, er, st);
        c->launches += 1;
        return LQ_OK;
    }

    // The Lanczos loop on stream ls; with `windows` the second pass of a two-pass run.
    int lanczos(bool windows, cudaStream_t ls) {
        int j0 = 0;
        for (int j = 0; j < k; ++j) {
            h.j = j;
            h.in[0] = bvec(j);
            h.in[1] = lvec(j);
            cudaEvent_t eh = prof_begin(c, ls);
            LQ_CUDA(c, launch_hop(c->prec, h, nf, emode, true, ls));
            prof_end(c, PC_HOP, eh, ls);
            c->launches += 1;
            // vh_0 .. vh_j are in the ring and the update below overwrites slot j + 1
            if (windows && (j + 1 - j0 == kTwoPassWindow || j == k - 1)) {
                int rr = recombine(j0, j + 1, ls);
                if (!rr && on_window) rr = on_window(j0, j + 1, ls);
                if (rr) return rr;
                j0 = j + 1;
            }
            if (j < k - 1) {
                u.j = j;
                u.v_cur = bvec(j); u.v_prev = bvec(j > 0 ? j - 1 : j); u.v_next = bvec(j + 1);
                u.w_cur = lvec(j); u.w_prev = lvec(j > 0 ? j - 1 : j); u.w_next = lvec(j + 1);
                if (keep_left)
                    u.w_store = reinterpret_cast<char*>(c->lbasis) + ((size_t)s0 * sst + (size_t)(ring ? (j + 1) % ring : j + 1) * vstride) * cb;
                const bool rb_step = rb_corrects(rb, j);
                u.defer = rb_step ? 1 : 0;
                cudaEvent_t eu = prof_begin(c, ls);
                LQ_CUDA(c, launch_update(c->prec, u, ls));
                prof_end(c, PC_UPDATE, eu, ls);
                c->launches += 1;
                if (rb_step) {
                    RbArgs b;
                    std::memset(&b, 0, sizeof(b));
                    b.u = u;
                    b.m = j + 1;
                    b.vbasis = bvec(0);
                    b.wbasis = reinterpret_cast<char*>(c->lbasis) + (size_t)s0 * sst * cb;
                    b.vec_stride = vstride;
                    b.scale = c->scale + (size_t)s0 * c->kmax;
                    b.uscale = c->uscale + (size_t)s0 * c->kmax;
                    b.dot_blocks = rb_dot_blocks(vstride);
                    b.part = c->rb_part + (size_t)s0 * c->kmax * b.dot_blocks * 8;
                    b.coef = c->rb_coef + (size_t)s0 * 2 * c->kmax;
                    b.coef_f = c->rb_coef_f + (size_t)s0 * 2 * c->kmax;
                    cudaEvent_t eb = prof_begin(c, ls);
                    LQ_CUDA(c, launch_rebiorth(c->prec, b, ls));
                    prof_end(c, PC_UPDATE, eb, ls);
                    c->launches += 3;
                }
            }
        }
        return LQ_OK;
    }

    lq_ctx::GraphKey key(int groups = 1) const {
        return {k, nsrc, nf, emode, h.variant, store_left ? 1 : 0, ring, c->desc.mu, groups, u.bulk, rb};
    }
    bool graphed() const { return o->graph != 0 && !c->prof_on; }
    long long loop_launches() const {
        long long n = 2 * (long long)k - 1;
        for (int j = 0; j + 1 < k; ++j) n += rb_corrects(rb, j) ? 3 : 0;
        return n;
    }

    int quad_pass(cudaStream_t st) {
        LQ_CUDA(c, cudaMemcpyAsync(c->quad_nodes, nodes.data(), sizeof(int) * nsrc, cudaMemcpyHostToDevice, st));
        cudaEvent_t eq = prof_begin(c, st);
        const int maxn = *std::max_element(nodes.begin(), nodes.end());
        LQ_CUDA(c, quad_sign_e1(qa, maxn, quad_attempt == 0, st));
        prof_end(c, PC_NEWTON, eq, st, 0);
        c->launches += quad_attempt == 0 ? 5 : 4;
        return LQ_OK;
    }

    // Projected step, the part that needs no host decision: the resolvent, or the first
    // quadrature pass (the Newton iteration of LQ_PROJ_NEWTON runs in proj_complete).
    int proj_enqueue(cudaStream_t st) {
        if (fn == FN_RESOLVENT) {
            QuadArgs q;
            std::memset(&q, 0, sizeof(q));
            q.k = k; q.nb = nsrc; q.kmax = c->kmax; q.nth_max = 2 * kQuadMaxNodes; q.state = c->state;
            q.alpha = c->alpha; q.beta = c->beta; q.delta = c->delta; q.work = c->quad_work;
            q.s = c->proj_c; q.check = c->quad_check;
            LQ_CUDA(c, proj_resolvent(q, shifts, st));
            c->launches += 1;
            for (int s = 0; s < nsrc; ++s) used[s] = -1;   // not a reported solver
            return LQ_OK;
        }
        if (o->projected == LQ_PROJ_NEWTON) return LQ_OK;
        std::memset(&qa, 0, sizeof(qa));
        qa.k = k; qa.nb = nsrc; qa.kmax = c->kmax; qa.state = c->state;
        qa.alpha = c->alpha; qa.beta = c->beta; qa.delta = c->delta; qa.c = c->quad_c; qa.work = c->quad_work;
        qa.s = c->proj_c; qa.q = c->quad_q; qa.check = c->quad_check; qa.nodes = c->quad_nodes;
        qa.nth_max = 2 * kQuadRetryMaxNodes; qa.part = c->quad_part; qa.part_blocks = 2 * kQuadRetryMaxNodes / kQuadBlk;
        if (o->projected == LQ_PROJ_NESTED) {      // the scales c only; the nested passes need host decisions
            LQ_CUDA(c, quad_scale(qa, st));
            c->launches += 1;
            return LQ_OK;
        }
        nodes.assign(nsrc, o->quad_nodes);
        quad_attempt = 0;
        return quad_pass(st);
    }

    // The nested rung for the sources with sel[s] != 0; accepted ones leave sel and report the
    // nested solver and its residual.  Returns whether any source is left.
    int nested_rung(std::vector<int>& sel, cudaStream_t st, bool* left) {
        *left = false;
        bool any = false;
        for (int s = 0; s < nsrc; ++s) any = any || sel[s];
        if (!any) return LQ_OK;
        const int m = std::max(1, std::min({o->nested_m > 0 ? o->nested_m : 100, k, c->kmax}));
        std::vector<double> chk;
        int r = nested_run(c, c->state, k, nsrc, m, c->quad_c, sel, c->proj_c, chk, o->newton_max_iter, o->newton_tol, st);
        if (r) return r;
        for (int s = 0; s < nsrc; ++s) {
            if (!sel[s]) continue;
            used[s] = LQ_PROJ_NESTED;
            check[s] = chk[s];
            if (std::isfinite(chk[s]) && chk[s] <= o->proj_tol) sel[s] = 0;
            else *left = true;
        }
        return LQ_OK;
    }

    // LQ_PROJ_QUAD: one pass with opts.quad_nodes.  LQ_PROJ_AUTO: a source whose involution
    // residual exceeds proj_tol is retried once with kQuadRetryMaxNodes nodes (a pass costs the
    // latency of one sequential tridiagonal solve whatever the node count, so one large retry
    // beats a ladder of doublings); the others keep their result; what still fails goes to the
    // Newton iteration.  Synchronises st.
    int proj_complete(cudaStream_t st) {
        bool need_newton = o->projected == LQ_PROJ_NEWTON && fn == FN_SIGN;
        if (quad_attempt >= 0) {
            bool ok = false;
            for (;;) {
                LQ_CUDA(c, cudaMemcpyAsync(check.data(), c->quad_check, sizeof(double) * nsrc, cudaMemcpyDeviceToHost, st));
                LQ_CUDA(c, cudaStreamSynchronize(st));   // nodes and check are host memory
                ok = true;
                bool retry = false;
                for (int s = 0; s < nsrc; ++s) {
                    const bool pass = std::isfinite(check[s]) && check[s] <= o->proj_tol;
                    ok = ok && pass;
                    if (pass || nodes[s] == 0) { nodes[s] = 0; continue; }
                    if (o->projected == LQ_PROJ_AUTO && nodes[s] < kQuadRetryMaxNodes) { nodes[s] = kQuadRetryMaxNodes; retry = true; }
                    else nodes[s] = 0;
                }
                if (ok || !retry) break;
                ++quad_attempt;
                int r = quad_pass(st);
                if (r) return r;
            }
            need_newton = !ok && o->projected == LQ_PROJ_AUTO;
            for (int s = 0; s < nsrc; ++s) used[s] = LQ_PROJ_QUAD;
        }
        std::vector<int> sel(nsrc, 1);
        if (o->projected == LQ_PROJ_AUTO && need_newton) {
            // the nested rung for what the quadrature left, Newton for what it leaves
            for (int s = 0; s < nsrc; ++s) sel[s] = !(std::isfinite(check[s]) && check[s] <= o->proj_tol);
            bool left = false;
            int r = nested_rung(sel, st, &left);
            if (r) return r;
            need_newton = left;
        } else if (o->projected == LQ_PROJ_NESTED && fn == FN_SIGN) {
            bool left = false;
            int r = nested_rung(sel, st, &left);
            if (r) return r;
            need_newton = false;
        }
        if (need_newton) {
            // Newton for every source (LQ_PROJ_NEWTON) or only for those the other rungs left
            NewtonArgs na = newton_args(c, k, nsrc, o->newton_max_iter, o->newton_tol);
            LQ_CUDA(c, newton_init_tridiag(na, st));
            c->launches += 1;
            const double one = 1.0;
            for (int s = 0; s < nsrc; ++s)
                if (!sel[s]) LQ_CUDA(c, cudaMemcpyAsync(c->nx_scal + (size_t)s * 16 + NS_DONE, &one, sizeof(double), cudaMemcpyHostToDevice, st));
            LQ_CUDA(c, cudaMemcpyAsync(c->proj_sel, sel.data(), sizeof(int) * nsrc, cudaMemcpyHostToDevice, st));
            int r = run_newton(c, na, st, scal);
            if (r) return r;
            LQ_CUDA(c, newton_first_column(na, c->proj_c, c->kmax, st, c->proj_sel));
            c->launches += 1;
            for (int s = 0; s < nsrc; ++s) if (sel[s]) used[s] = LQ_PROJ_NEWTON;
            LQ_CUDA(c, cudaStreamSynchronize(st));   // sel is host memory
        }
        return LQ_OK;
    }

    // y = |x| V_k sgn(T_k) e_1, or the second pass of a two-pass run (the same process from the
    // same start, recombining as it goes).
    int finish_enqueue(cudaStream_t st) {
        if (!two) return recombine(0, 0, st);
        int r = init(st);
        return r ? r : lanczos(true, st);
    }

    // Reports (host); synchronises st.
    int finish_complete(cudaStream_t st) {
        std::vector<TslState> hs(nsrc);
        LQ_CUDA(c, cudaMemcpyAsync(hs.data(), c->state, sizeof(TslState) * nsrc, cudaMemcpyDeviceToHost, st));
        LQ_CUDA(c, cudaStreamSynchronize(st));
        prof_collect(c);
        if (!rep) return LQ_OK;
        for (int s = 0; s < nsrc; ++s) {
            lq_report& R = rep[s];
            std::memset(&R, 0, sizeof(R));
            R.k_eff = hs[s].k_eff;
            R.x_norm = hs[s].xnorm;
            R.newton_iters = (int)scal[(size_t)s * 16 + NS_ITERS];
            R.newton_change = scal[(size_t)s * 16 + NS_CHANGE];
            R.projected = used[s];
            R.hop_variant = h.variant;
            R.proj_check = check[s];   // involution residual of the quadrature when it was attempted
            const int ts = hs[s].status;
            int ns = (int)scal[(size_t)s * 16 + NS_STATUS];
            if ((used[s] == LQ_PROJ_QUAD || used[s] == LQ_PROJ_NESTED) && !(std::isfinite(check[s]) && check[s] <= o->proj_tol))
                ns = LQ_ERR_NEWTON;
            R.status = ts < 0 ? ts : (ns != 0 ? ns : LQ_OK);
        }
        return LQ_OK;
    }
};

bool ensure_cap_stream(lq_ctx* c, bool second = false) {
    cudaStream_t& s = second ? c->cap_stream2 : c->cap_stream;
    if (s) return true;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess) return true;
    cudaGetLastError();
    s = nullptr;
    return false;
}

// fork: each stream of `to` waits for the work enqueued on `from` so far; join: `into` waits for
// the work enqueued on each stream of `from` so far.
int fork_streams(lq_ctx* c0, cudaStream_t from, const std::vector<cudaStream_t>& to) {
    cudaEvent_t e = nullptr;
    LQ_CUDA(c0, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaError_t err = cudaEventRecord(e, from);
    for (cudaStream_t s : to) if (err == cudaSuccess) err = cudaStreamWaitEvent(s, e, 0);
    cudaEventDestroy(e);
    LQ_CUDA(c0, err);
    return LQ_OK;
}
int join_streams(lq_ctx* c0, const std::vector<cudaStream_t>& from, cudaStream_t into) {
    for (cudaStream_t s : from) {
        cudaEvent_t e = nullptr;
        LQ_CUDA(c0, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        cudaError_t err = cudaEventRecord(e, s);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(into, e, 0);
        cudaEventDestroy(e);
        LQ_CUDA(c0, err);
    }
    return LQ_OK;
}


// First pass (or the only one): replayed from a CUDA graph of the whole loop when graphs are on
// and the kernels are not being timed one by one (lq_profile_enable); the graph is captured on
// the first call with this configuration.  Any capture failure falls back to plain launches.
int lanczos_graph(TslRun& t, cudaStream_t st) {
    lq_ctx* c = t.c;
    const lq_ctx::GraphKey key = t.key();
    cudaGraphExec_t exec = nullptr;
    for (auto& g : c->graphs) if (g.key == key) exec = g.exec;
    if (!exec) {
        if (!ensure_cap_stream(c)) return t.lanczos(false, st);
        (void)update_grid(t.u.nelem, t.u.nsrc, t.u.partial_stride);   // one-time device queries, before capture
        update_bulk_prepare();
        const long long launches0 = c->launches;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return t.lanczos(false, st);
        }
        const int rr = t.lanczos(false, c->cap_stream);
        const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        c->launches = launches0;
        cudaError_t ei = cudaErrorUnknown;
        if (!rr && e == cudaSuccess && g) ei = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            cudaGetLastError();
            c->err.clear();
            return t.lanczos(false, st);
        }
        if (c->graphs.size() >= 8) { cudaGraphExecDestroy(c->graphs.front().exec); c->graphs.erase(c->graphs.begin()); }
        c->graphs.push_back({key, exec});
    }
    LQ_CUDA(c, cudaGraphLaunch(exec, st));
    c->launches += t.loop_launches();
    return LQ_OK;
}

// The Krylov loops of the two source halves g[0], g[1] of a split run as concurrent branches on
// the context's two capture streams, forked from and joined into st: replayed from one CUDA graph
// when graphs are on (captured on the first call of the configuration), else plain launches.
int lanczos_split(TslRun (&g)[2], cudaStream_t st, bool graphed) {
    lq_ctx* c = g[0].c;
    const std::vector<cudaStream_t> br{c->cap_stream, c->cap_stream2};
    auto branches = [&]() -> int {
        int r = g[0].lanczos(false, br[0]);
        if (!r) r = g[1].lanczos(false, br[1]);
        return r;
    };
    auto plain = [&]() -> int {
        int r = fork_streams(c, st, br);
        if (r) return r;
        r = branches();
        const int rj = join_streams(c, br, st);
        return r ? r : rj;
    };
    if (!graphed) return plain();
    const lq_ctx::GraphKey key = g[0].key(2);
    cudaGraphExec_t exec = nullptr;
    for (auto& e : c->graphs) if (e.key == key) exec = e.exec;
    if (!exec) {
        for (auto& t : g) (void)update_grid(t.u.nelem, t.u.nsrc, t.u.partial_stride);   // device queries, before capture
        update_bulk_prepare();
        const long long launches0 = c->launches;
        cudaEvent_t ev[2] = {nullptr, nullptr};   // fork, join
        bool ok = cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) == cudaSuccess;
        cudaError_t ei = cudaErrorUnknown;
        if (ok && cudaStreamBeginCapture(br[0], cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            int rr = (cudaEventRecord(ev[0], br[0]) == cudaSuccess && cudaStreamWaitEvent(br[1], ev[0], 0) == cudaSuccess)
                         ? LQ_OK : LQ_ERR_CUDA;
            if (!rr) {
                rr = branches();
                // join even after a failed launch, so that the capture ends on the origin stream
                if (cudaEventRecord(ev[1], br[1]) != cudaSuccess || cudaStreamWaitEvent(br[0], ev[1], 0) != cudaSuccess)
                    rr = rr ? rr : LQ_ERR_CUDA;
            }
            cudaGraph_t gr = nullptr;
            const cudaError_t e = cudaStreamEndCapture(br[0], &gr);
            if (!rr && e == cudaSuccess && gr) ei = cudaGraphInstantiate(&exec, gr, 0);
            if (gr) cudaGraphDestroy(gr);
        }
        for (cudaEvent_t e : ev) if (e) cudaEventDestroy(e);
        c->launches = launches0;
        if (ei != cudaSuccess) {
            cudaGetLastError();
            c->err.clear();
            return plain();
        }
        if (c->graphs.size() >= 8) { cudaGraphExecDestroy(c->graphs.front().exec); c->graphs.erase(c->graphs.begin()); }
        c->graphs.push_back({key, exec});
    }
    LQ_CUDA(c, cudaGraphLaunch(exec, st));
    c->launches += g[0].loop_launches() + g[1].loop_launches();
    return LQ_OK;
}

int run_tsl(lq_ctx* c, int nf, int emode, int nsrc, const lq_opts* o, lq_report* rep,
            double* y0, double* y1, cudaStream_t st, const double* x_dev = nullptr,
            const double* x_top = nullptr, int fn = FN_SIGN, const double2* shifts = nullptr,
            bool store_left = false) {
    TslRun t;
    t.c = c; t.nf = nf; t.emode = emode; t.nsrc = nsrc; t.o = o; t.rep = rep;
    t.y0 = y0; t.y1 = y1; t.fn = fn; t.shifts = shifts; t.store_left = store_left;
    // lq_opts.split: the two source halves' Krylov loops as concurrent branches (the update of one
    // half, bandwidth-bound, overlaps the stencil of the other, issue-bound)
    if (o->rebiorth > 0 && fn == FN_SIGN && !store_left && !(c->rebiorth && c->lbasis_nf >= nf))
        return set_err(c, LQ_ERR_NOT_READY, "opts.rebiorth needs a workspace reserved with LQ_RESERVE_REBIORTH"
                                            " (with LQ_RESERVE_BLOCK for the derivative)");
    const bool split = o->split != 0 && !c->prof_on && c->prec == LQ_MIXED && nf == 2 && fn == FN_SIGN && !store_left &&
                       !(o->two_pass != 0 && o->kmax > 1) && o->rebiorth <= 0 && nsrc >= 8 && nsrc % 2 == 0 &&
                       ensure_cap_stream(c) && ensure_cap_stream(c, true);
    int r;
    if (!split) {
        if ((r = t.setup(st, x_dev, x_top))) return r;
        if ((r = t.graphed() ? lanczos_graph(t, st) : t.lanczos(false, st))) return r;
    } else {
        TslRun g[2] = {t, t};
        for (int i = 0; i < 2; ++i) {
            g[i].nsrc = nsrc / 2;
            g[i].s0 = i * (nsrc / 2);
            g[i].rep = nullptr;
            if ((r = g[i].setup(st, x_dev, x_top))) return r;
            // the bulk-copy update needs ~200 KB of shared memory per SM, which leaves the other
            // half's stencil, running beside it, almost no L1: the split loop takes the register
            // kernel unless the caller asks for the bulk one (measured at 14^4, 16 sources:
            // 162.5 ms against 179.6 ms per call)
            g[i].u.bulk = o->update_variant == 1 ? 1 : 0;
        }
        t.args_only = true;
        if ((r = t.setup(st, x_dev, x_top))) return r;
        t.h.variant = g[0].h.variant;   // reported schedule
        if ((r = lanczos_split(g, st, t.graphed()))) return r;
    }
    if ((r = t.proj_enqueue(st)) || (r = t.proj_complete(st))) return r;
    if ((r = t.finish_enqueue(st))) return r;
    return t.finish_complete(st);
}

// ---- ragged batches (lq_batch_apply) --------------------------------------------------------
// Every member of a batch runs on its own context; the branch of member i is its context's
// capture stream.
// The Krylov loops of all members as plain launches, each on its branch, between a fork from
// and a join into st.
int batch_lanczos_plain(std::vector<TslRun>& runs, cudaStream_t st) {
    std::vector<cudaStream_t> br;
    for (auto& t : runs) br.push_back(t.c->cap_stream);
    int r = fork_streams(runs[0].c, st, br);
    if (r) return r;
    for (size_t i = 0; i < runs.size() && !r; ++i) r = runs[i].lanczos(false, br[i]);
    const int rj = join_streams(runs[0].c, br, st);
    return r ? r : rj;
}

// The Krylov loops of all members as one CUDA graph with one branch per member, captured the
// first time this batch configuration is met and replayed with a single launch on st; the
// branches are independent, so the GPU runs the members' kernels side by side.  Any capture
// failure falls back to batch_lanczos_plain.
int batch_lanczos_graph(std::vector<TslRun>& runs, cudaStream_t st) {
    const size_t n = runs.size();
    lq_ctx* c0 = runs[0].c;
    std::vector<std::pair<lq_ctx*, lq_ctx::GraphKey>> key;
    for (auto& t : runs) key.push_back({t.c, t.key()});
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_batch_mu);
        for (auto& g : g_batch_graphs) if (g.key == key) exec = g.exec;
    }
    if (!exec) {
        for (auto& t : runs) (void)update_grid(t.u.nelem, t.u.nsrc, t.u.partial_stride);   // device queries, before capture
        update_bulk_prepare();
        std::vector<long long> launches0;
        for (auto& t : runs) launches0.push_back(t.c->launches);
        std::vector<cudaEvent_t> ev(n, nullptr);   // ev[0]: the fork; ev[i], i > 0: the join of member i
        bool ok = true;
        for (auto& e : ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        const cudaStream_t origin = c0->cap_stream;
        cudaError_t ei = cudaErrorUnknown;
        if (ok && cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            int rr = cudaEventRecord(ev[0], origin) == cudaSuccess ? LQ_OK : LQ_ERR_CUDA;
            if (!rr) rr = runs[0].lanczos(false, origin);
            for (size_t i = 1; i < n && !rr; ++i) {
                const cudaStream_t b = runs[i].c->cap_stream;
                if (cudaStreamWaitEvent(b, ev[0], 0) != cudaSuccess) { rr = LQ_ERR_CUDA; break; }
                rr = runs[i].lanczos(false, b);
                // join even after a failed launch, so that the capture ends on the origin stream
                if (cudaEventRecord(ev[i], b) != cudaSuccess || cudaStreamWaitEvent(origin, ev[i], 0) != cudaSuccess)
                    rr = rr ? rr : LQ_ERR_CUDA;
            }
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(origin, &g);
            if (!rr && e == cudaSuccess && g) ei = cudaGraphInstantiate(&exec, g, 0);
            if (g) cudaGraphDestroy(g);
        }
        for (cudaEvent_t e : ev) if (e) cudaEventDestroy(e);
        for (size_t i = 0; i < n; ++i) runs[i].c->launches = launches0[i];
        if (ei != cudaSuccess) {
            cudaGetLastError();
            for (auto& t : runs) t.c->err.clear();
            return batch_lanczos_plain(runs, st);
        }
        std::lock_guard<std::mutex> lk(g_batch_mu);
        if (g_batch_graphs.size() >= 8) {
            cudaGraphExecDestroy(g_batch_graphs.front().exec);
            g_batch_graphs.erase(g_batch_graphs.begin());
        }
        g_batch_graphs.push_back({key, exec});
    }
    LQ_CUDA(c0, cudaGraphLaunch(exec, st));
    for (auto& t : runs) t.c->launches += t.loop_launches();
    return LQ_OK;
}

int check_opts(lq_ctx* c, const lq_opts* o, bool allow_deflate = false) {
    if (!o) return set_err(c, LQ_ERR_ARG, "null opts");
    if (o->kmax < 1 || o->kmax > c->kmax) return set_err(c, LQ_ERR_ARG, "opts.kmax must be in [1, reserved kmax]");
    if (o->newton_max_iter < 1 || !(o->newton_tol > 0.0) || !(o->breakdown_tol >= 0.0)) return set_err(c, LQ_ERR_ARG, "invalid Newton / breakdown options");
    if (o->deflate != 0 && !allow_deflate) return set_err(c, LQ_ERR_ARG, "deflation is not available in this entry point");
    if (o->deflate != 0 && c->defl_l <= 0) return set_err(c, LQ_ERR_NOT_READY, "deflate = 1 but no deflation space uploaded");
    if (o->projected < LQ_PROJ_AUTO || o->projected > LQ_PROJ_NESTED) return set_err(c, LQ_ERR_ARG, "unknown projected-sign solver");
    if (o->nested_m < 0) return set_err(c, LQ_ERR_ARG, "nested_m must be >= 0");
    if (o->projected != LQ_PROJ_NEWTON && (o->quad_nodes < 1 || o->quad_nodes > kQuadMaxNodes || !(o->proj_tol > 0.0)))
        return set_err(c, LQ_ERR_ARG, "quad_nodes must be in [1, 128] and proj_tol > 0");
    if (o->hop_variant < -1 || o->hop_variant >= kHopSchedules)
        return set_err(c, LQ_ERR_ARG, "hop_variant must be in [-1, " + std::to_string(kHopSchedules - 1) + "]");
    if (o->defl_kmax < 0 || o->defl_kmax > c->kmax) return set_err(c, LQ_ERR_ARG, "defl_kmax must be in [0, reserved kmax]");
    if (o->defl_nderiv < 0) return set_err(c, LQ_ERR_ARG, "defl_nderiv must be >= 0");
    if (o->two_pass != 0 && o->two_pass != 1) return set_err(c, LQ_ERR_ARG, "two_pass must be 0 or 1");
    if (o->graph < -1 || o->graph > 1) return set_err(c, LQ_ERR_ARG, "graph must be -1, 0 or 1");
    if (o->split < -1 || o->split > 1) return set_err(c, LQ_ERR_ARG, "split must be -1, 0 or 1");
    if (o->update_variant < -1 || o->update_variant > 1) return set_err(c, LQ_ERR_ARG, "update_variant must be -1, 0 or 1");
    if (o->rebiorth < 0) return set_err(c, LQ_ERR_ARG, "rebiorth must be >= 0");
    if (o->rebiorth > 0 && o->two_pass) return set_err(c, LQ_ERR_ARG, "re-biorthogonalisation needs the whole bases: not with two_pass");
    if (c->ring > 0 && !o->two_pass && o->kmax > c->ring)
        return set_err(c, LQ_ERR_ARG, "workspace reserved for two-pass runs: set opts.two_pass = 1 or kmax <= " + std::to_string(c->ring));
    return LQ_OK;
}


// ---- deflation (Sec. 3) -------------------------------------------------------------------
size_t nvec(const lq_ctx* c) { return c->V * 24; }   // doubles per boundary-layout field

// <X_a|Y_b> for a < nx, b < ny (device vectors, stride nvec) -> host out[a * ny + b]
int bdots_host(lq_ctx* c, const double* X, int nx, const double* Y, int ny, std::vector<double2>& out, cudaStream_t st) {
    out.assign((size_t)nx * ny, make_double2(0.0, 0.0));
    if (nx == 0 || ny == 0) return LQ_OK;
    const size_t need = bdots_partial_doubles(nx * ny) + 2 * (size_t)nx * ny;
    double* scr = (c->defl_scr && need <= c->defl_scr_doubles) ? c->defl_scr
                : ((c->gen_scr && need <= c->gen_scr_doubles) ? c->gen_scr : nullptr);
    if (!scr) return set_err(c, LQ_ERR_ARG, "reduction scratch too small for " + std::to_string(nx) + " x " + std::to_string(ny) + " dots");
    double* part = scr;
    double* res = scr + bdots_partial_doubles(nx * ny);
    LQ_CUDA(c, launch_bdots(X, nvec(c), nx, Y, nvec(c), ny, nvec(c), part, res, st));
    c->launches += 2;
    LQ_CUDA(c, cudaMemcpyAsync(out.data(), res, sizeof(double2) * nx * ny, cudaMemcpyDeviceToHost, st));
    LQ_CUDA(c, cudaStreamSynchronize(st));
    return LQ_OK;
}

// Z_b = W_b + sum_a coef[b * nx + a] X_a with host coefficients
int bcombine_host(lq_ctx* c, double* Z, const double* W, int nz, const double* X, int nx,
                  const std::vector<double2>& coef, cudaStream_t st) {
    if (nz == 0) return LQ_OK;
    const size_t need = (size_t)nz * nx * 2;
    double* dc = (c->defl_scr && need <= c->defl_scr_doubles) ? c->defl_scr
               : ((c->gen_scr && need <= c->gen_scr_doubles) ? c->gen_scr : nullptr);
    if (!dc) return set_err(c, LQ_ERR_ARG, "coefficient scratch too small");
    LQ_CUDA(c, cudaMemcpyAsync(dc, coef.data(), sizeof(double2) * nz * nx, cudaMemcpyHostToDevice, st));
    LQ_CUDA(c, launch_bcombine(Z, W, nvec(c), nz, X, nvec(c), nx, dc, nvec(c), st));
    c->launches += 1;
    LQ_CUDA(c, cudaStreamSynchronize(st));   // the coefficient buffer is reused by the next call
    return LQ_OK;
}

// out_j = E in_j (dagger = 0) or E^dag in_j (dagger = 1) for `count` boundary fields on the
// device, along the current direction: the block stencil with the operator part switched off.
int apply_E(lq_ctx* c, const double* in, double* out, int count, int dagger, cudaStream_t st) {
    const int em = emode_of(c);
    if (em == 0) return set_err(c, LQ_ERR_NOT_READY, "no derivative direction set");
    for (int b0 = 0; b0 < count; b0 += c->nsrc) {
        const int nb = std::min(c->nsrc, count - b0);
        // fields [src][2]: both halves hold the input, so side 0 gives E in (top) and side 1 E^dag in (bottom)
        for (int s = 0; s < nb; ++s) {
            LQ_CUDA(c, launch_to_internal(c->prec, in + (size_t)(b0 + s) * nvec(c),
                                          reinterpret_cast<char*>(c->rout) + (size_t)(2 * s) * fb(c), c->V, 1, st));
            LQ_CUDA(c, launch_to_internal(c->prec, in + (size_t)(b0 + s) * nvec(c),
                                          reinterpret_cast<char*>(c->rout) + (size_t)(2 * s + 1) * fb(c), c->V, 1, st));
        }
        HopArgs a = base_hop(c);
        a.nsrc = nb;
        a.nsides = 1;
        a.side0 = dagger ? 1 : 0;
        set_side(a, a.side0, c, dagger ? 1 : 0, em);
        for (int nu = 0; nu < 4; ++nu) {
            a.a_fwd[a.side0][nu] = a.a_bwd[a.side0][nu] = 0.0;
            a.af_fwd[a.side0][nu] = a.af_bwd[a.side0][nu] = 0.0f;
        }
        a.diag = 0.0;
        a.diag_f = 0.0f;
        a.in[a.side0] = c->rout;
        a.out[a.side0] = c->lout;
        a.src_stride_in[a.side0] = 2 * fe(c);
        a.src_stride_out[a.side0] = 2 * fe(c);
        LQ_CUDA(c, launch_hop(c->prec, a, 2, em, false, st));
        for (int s = 0; s < nb; ++s)
            LQ_CUDA(c, launch_to_boundary(c->prec, reinterpret_cast<char*>(c->lout) + (size_t)(2 * s + (dagger ? 1 : 0)) * fb(c),
                                          out + (size_t)(b0 + s) * nvec(c), c->V, 1, st));
        c->launches += 3 * nb + 1;
    }
    return LQ_OK;
}

double sgn_re(double2 z) { return z.x > 0 ? 1.0 : (z.x < 0 ? -1.0 : 0.0); }
double2 cdivh(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
double2 conjh(double2 a) { return make_double2(a.x, -a.y); }

// dlambda_i, dR_i, dL_i for the current direction (end of Sec. 3):
//   dR_j = sum_{i != j} R_i (L_i E R_j)/(lambda_j - lambda_i) + Pbar (lambda_j - A)^{-1} Pbar E R_j
//   dLk_j = sum_{i != j} conj((L_j E R_i)/(lambda_j - lambda_i)) Lk_i
//           + Pbar^dag (conj lambda_j - A^dag)^{-1} Pbar^dag E^dag Lk_j
// The shifted solves are two-sided Lanczos approximations of the resolvent at depth opts->kmax
// (the projected function (sigma - T)^{-1} e_1), started from deflated right-hand sides.
int nderiv_of(const lq_ctx* c, const lq_opts* o) {
    return (o->defl_nderiv > 0 && o->defl_nderiv < c->defl_l) ? o->defl_nderiv : c->defl_l;
}

int prepare_deflation_derivative(lq_ctx* c, const lq_opts* o, cudaStream_t st) {
    const int l = c->defl_l;          // pairs projected out of the shifted solves
    const int ld = nderiv_of(c, o);   // pairs whose derivatives are built (Jordan blocks)
    const size_t nv = nvec(c);
    double* R = c->defl_V;
    double* dR = c->defl_V + (size_t)l * nv;
    double* Lk = c->defl_W;
    double* dLk = c->defl_W + (size_t)l * nv;
    double* ER = c->defl_work;
    double* ELk = ER + (size_t)l * nv;
    double* bR = ELk + (size_t)l * nv;
    double* bL = bR + (size_t)l * nv;
    double* zR = bL + (size_t)l * nv;
    double* zL = zR + (size_t)l * nv;
    int r;
    if ((r = apply_E(c, R, ER, ld, 0, st))) return r;
    if ((r = apply_E(c, Lk, ELk, ld, 1, st))) return r;
    std::vector<double2> C, D, coef;
    if ((r = bdots_host(c, Lk, l, ER, ld, C, st))) return r;          // C[i*ld+j] = <Lk_i|E R_j> = L_i E R_j
    if ((r = bdots_host(c, R, l, ELk, ld, D, st))) return r;          // D[i*ld+j] = <R_i|E^dag Lk_j> = conj(L_j E R_i)
    c->defl_dlam.assign(l, make_double2(0.0, 0.0));
    for (int j = 0; j < ld; ++j) c->defl_dlam[j] = C[(size_t)j * ld + j];
    // deflated right-hand sides b_j = Pbar E R_j, b'_j = Pbar^dag E^dag Lk_j (projection with all l pairs)
    coef.assign((size_t)ld * l, make_double2(0.0, 0.0));
    for (int j = 0; j < ld; ++j) for (int i = 0; i < l; ++i) coef[(size_t)j * l + i] = make_double2(-C[(size_t)i * ld + j].x, -C[(size_t)i * ld + j].y);
    if ((r = bcombine_host(c, bR, ER, ld, R, l, coef, st))) return r;
    for (int j = 0; j < ld; ++j) for (int i = 0; i < l; ++i) coef[(size_t)j * l + i] = make_double2(-D[(size_t)i * ld + j].x, -D[(size_t)i * ld + j].y);
    if ((r = bcombine_host(c, bL, ELk, ld, Lk, l, coef, st))) return r;
    // shifted solves, in batches of the reserved number of sources
    lq_opts so = *o;
    so.projected = LQ_PROJ_NEWTON;   // unused by the resolvent; keeps the sign solvers idle
    so.kmax = o->defl_kmax > 0 ? o->defl_kmax : c->kmax;
    const double mu0 = c->desc.mu;
    for (int side = 0; side < 2; ++side) {
        const double* bin = side == 0 ? bR : bL;
        double* zout = side == 0 ? zR : zL;
        if (side == 1) c->desc.mu = -mu0;             // A^dag = H(-mu)
        for (int b0 = 0; b0 < ld; b0 += c->nsrc) {
            const int nb = std::min(c->nsrc, ld - b0);
            std::vector<double2> sh(nb);
            for (int q = 0; q < nb; ++q) sh[q] = side == 0 ? c->defl_lam[b0 + q] : conjh(c->defl_lam[b0 + q]);
            cudaError_t e = cudaMemcpyAsync(c->defl_shift, sh.data(), sizeof(double2) * nb, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) { c->desc.mu = mu0; return set_err(c, LQ_ERR_CUDA, cudaGetErrorString(e)); }
            r = run_tsl(c, 1, 0, nb, &so, nullptr, zout + (size_t)b0 * nv, nullptr, st, bin + (size_t)b0 * nv,
                        nullptr, FN_RESOLVENT, c->defl_shift);
            if (r) { c->desc.mu = mu0; return r; }
        }
        c->desc.mu = mu0;
    }
    // project the solutions and add the sums over the deflated eigenvectors
    std::vector<double2> PZ, PZL;
    if ((r = bdots_host(c, Lk, l, zR, ld, PZ, st))) return r;          // <Lk_i|z_j>
    if ((r = bdots_host(c, R, l, zL, ld, PZL, st))) return r;          // <R_i|z'_j>
    for (int j = 0; j < ld; ++j)
        for (int i = 0; i < l; ++i) {
            double2 v = make_double2(-PZ[(size_t)i * ld + j].x, -PZ[(size_t)i * ld + j].y);
            if (i != j) {
                const double2 q = cdivh(C[(size_t)i * ld + j], make_double2(c->defl_lam[j].x - c->defl_lam[i].x, c->defl_lam[j].y - c->defl_lam[i].y));
                v.x += q.x; v.y += q.y;
            }
            coef[(size_t)j * l + i] = v;
        }
    if ((r = bcombine_host(c, dR, zR, ld, R, l, coef, st))) return r;
    for (int j = 0; j < ld; ++j)
        for (int i = 0; i < l; ++i) {
            double2 v = make_double2(-PZL[(size_t)i * ld + j].x, -PZL[(size_t)i * ld + j].y);
            if (i != j) {
                // conj((L_j E R_i) / (lambda_j - lambda_i)) with L_j E R_i = conj(D[i][j])
                const double2 q = conjh(cdivh(conjh(D[(size_t)i * ld + j]), make_double2(c->defl_lam[j].x - c->defl_lam[i].x, c->defl_lam[j].y - c->defl_lam[i].y)));
                v.x += q.x; v.y += q.y;
            }
            coef[(size_t)j * l + i] = v;
        }
    if ((r = bcombine_host(c, dLk, zL, ld, Lk, l, coef, st))) return r;
    // derivatives beyond ld stay zero
    if (ld < l) {
        LQ_CUDA(c, cudaMemsetAsync(dR + (size_t)ld * nv, 0, sizeof(double) * (l - ld) * nv, st));
        LQ_CUDA(c, cudaMemsetAsync(dLk + (size_t)ld * nv, 0, sizeof(double) * (l - ld) * nv, st));
    }
    return LQ_OK;
}
// ---- deflation-space eigensolver --------------------------------------------------------------
using cplx = std::complex<double>;

// out_b = H x_b (dagger = 0) or H^dag x_b for `count` boundary FP64 vectors on the device, with
// the stencil in precision `prec` on the internal links `links` (the eigensolver always passes
// FP64: the deflation space must be accurate whatever precision the Lanczos path runs in).
int apply_H_batch(lq_ctx* c, const double* in, double* out, int count, int dagger, cudaStream_t st,
                  int prec, const void* links) {
    const size_t fb_ctx = fb(c);
    const size_t fb_op = field_bytes_of(prec, c->V);
    const int cap = std::max(1, (int)((size_t)c->nsrc * (c->block ? 2 : 1) * fb_ctx / fb_op));
    const size_t nv = nvec(c);
    const size_t fe_op = field_elems_of(prec, c->V);
    for (int b0 = 0; b0 < count; b0 += cap) {
        const int nb = std::min(cap, count - b0);
        LQ_CUDA(c, launch_to_internal(prec, in + (size_t)b0 * nv, c->rout, c->V, nb, st));
        HopArgs a = base_hop(c);
        a.U = links;
        a.link_bf16 = (links == c->U && c->link_bf16) ? 1 : 0;
        a.nsrc = nb;
        a.nsides = 1;
        a.side0 = 0;
        set_side(a, 0, c, dagger ? 1 : 0, 0);
        a.in[0] = c->rout;
        a.out[0] = c->lout;
        a.src_stride_in[0] = fe_op;
        a.src_stride_out[0] = fe_op;
        LQ_CUDA(c, launch_hop(prec, a, 1, 0, false, st));
        LQ_CUDA(c, launch_to_boundary(prec, c->lout, out + (size_t)b0 * nv, c->V, nb, st));
        c->launches += 3;
    }
    return LQ_OK;
}

// X <- X L^{-H} with G = X^H X = L L^H (Cholesky QR), twice for stability.  tmp: m vectors.
int orthonormalise(lq_ctx* c, double* X, double* tmp, int m, cudaStream_t st) {
    const size_t nv = nvec(c);
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<double2> G;
        int r;
        if ((r = bdots_host(c, X, m, X, m, G, st))) return r;
        std::vector<cplx> L(m * m);
        for (int i = 0; i < m * m; ++i) L[i] = cplx(G[i].x, G[i].y);
        // G[a*m+b] = <X_a|X_b>; Cholesky of the Hermitian G (row-major a, b)
        if (dense_cholesky(m, L.data()) != LQ_OK) return set_err(c, LQ_ERR_BREAKDOWN, "subspace lost rank in the eigensolver");
        // C = L^{-H} (upper triangular): solve L^H C = I column by column
        std::vector<cplx> Cm(m * m, 0.0);
        for (int col = 0; col < m; ++col) {
            for (int i = m - 1; i >= 0; --i) {
                cplx s = (i == col) ? 1.0 : 0.0;
                for (int k = i + 1; k < m; ++k) s -= std::conj(L[k * m + i]) * Cm[k * m + col];
                Cm[i * m + col] = s / std::conj(L[i * m + i]);
            }
        }
        std::vector<double2> coef(m * m);
        for (int b = 0; b < m; ++b) for (int a = 0; a < m; ++a) coef[b * m + a] = make_double2(Cm[a * m + b].real(), Cm[a * m + b].imag());
        if ((r = bcombine_host(c, tmp, nullptr, m, X, m, coef, st))) return r;
        LQ_CUDA(c, cudaMemcpyAsync(X, tmp, sizeof(double) * nv * m, cudaMemcpyDeviceToDevice, st));
    }
    return LQ_OK;
}

// Chebyshev-filtered subspace iteration on H^2 (dagger selects H^dag) for the nev eigenpairs
// of smallest modulus; returns Ritz values (sorted by modulus) and Ritz vectors in Z.
int eig_subspace(lq_ctx* c, const lq_eig_opts* eo, const double* X0, int dagger, double* W, std::vector<cplx>& theta,
                 std::vector<double>& res, double* Z, cudaStream_t st, const void* links64) {
    auto applyH = [&](const double* in, double* out, int count) { return apply_H_batch(c, in, out, count, dagger, st, LQ_FP64, links64); };
    const int m = eo->nsub, nev = eo->nev;
    const size_t nv = nvec(c);
    double* X = W;
    double* Y0 = W + (size_t)m * nv;
    double* Y1 = Y0 + (size_t)m * nv;
    double* H1 = Y1 + (size_t)m * nv;
    double* H2 = H1 + (size_t)m * nv;
    int r;
    LQ_CUDA(c, cudaMemcpyAsync(X, X0, sizeof(double) * nv * m, cudaMemcpyDeviceToDevice, st));
    if ((r = orthonormalise(c, X, Y0, m, st))) return r;
    // b^2: power iteration with H^2 on the first start vector
    double b2 = 0.0;
    {
        LQ_CUDA(c, cudaMemcpyAsync(Y1, X, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
        for (int it = 0; it < 12; ++it) {
            if ((r = applyH(Y1, H1, 1))) return r;
            if ((r = applyH(H1, H2, 1))) return r;
            std::vector<double2> nn;
            if ((r = bdots_host(c, H2, 1, H2, 1, nn, st))) return r;
            std::vector<double2> n1;
            if ((r = bdots_host(c, Y1, 1, Y1, 1, n1, st))) return r;
            b2 = std::sqrt(nn[0].x / n1[0].x);
            std::vector<double2> sc(1, make_double2(1.0 / std::sqrt(nn[0].x), 0.0));
            if ((r = bcombine_host(c, Y1, nullptr, 1, H2, 1, sc, st))) return r;
        }
        b2 *= 1.15;
    }
    double a2 = b2 / 25.0;
    theta.assign(m, 0.0);
    res.assign(m, 1.0);
    const double hn = std::sqrt(b2);
    for (int it = 0; it <= eo->max_iter; ++it) {
        if (it > 0) {
            // Y = T_d((H^2 - cen) / e) X, three-term recurrence; eigenvalues of H^2 below a2 are amplified
            const double cen = 0.5 * (b2 + a2), e = 0.5 * (b2 - a2);
            if ((r = applyH(X, H1, m))) return r;
            if ((r = applyH(H1, H2, m))) return r;
            LQ_CUDA(c, launch_axpby3(Y1, 1.0 / e, H2, -cen / e, X, 0.0, nullptr, nv * m, st));
            LQ_CUDA(c, cudaMemcpyAsync(Y0, X, sizeof(double) * nv * m, cudaMemcpyDeviceToDevice, st));
            for (int d = 2; d <= eo->degree; ++d) {
                if ((r = applyH(Y1, H1, m))) return r;
                if ((r = applyH(H1, H2, m))) return r;
                // Y2 = 2 (H^2 Y1 - cen Y1)/e - Y0, written over Y0
                LQ_CUDA(c, launch_axpby3(Y0, 2.0 / e, H2, -2.0 * cen / e, Y1, -1.0, Y0, nv * m, st));
                std::swap(Y0, Y1);
                c->launches += 1;
            }
            LQ_CUDA(c, cudaMemcpyAsync(X, Y1, sizeof(double) * nv * m, cudaMemcpyDeviceToDevice, st));
            if ((r = orthonormalise(c, X, Y0, m, st))) return r;
        }
        // Rayleigh-Ritz with H (or H^dag)
        if ((r = applyH(X, H1, m))) return r;
        std::vector<double2> M;
        if ((r = bdots_host(c, X, m, H1, m, M, st))) return r;      // M[a*m+b] = <X_a|H X_b>
        std::vector<cplx> Mc(m * m), w(m), Vr(m * m);
        for (int i = 0; i < m * m; ++i) Mc[i] = cplx(M[i].x, M[i].y);
        if (dense_eig(m, Mc.data(), w.data(), Vr.data()) != LQ_OK) return set_err(c, LQ_ERR_NEWTON, "Rayleigh-Ritz eigensolver failed");
        std::vector<int> ord(m);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int i, int j) { return std::abs(w[i]) < std::abs(w[j]); });
        std::vector<double2> coef(m * m), coefr(m * m);
        for (int b = 0; b < m; ++b)
            for (int a = 0; a < m; ++a) {
                const cplx y = Vr[a * m + ord[b]];
                coef[b * m + a] = make_double2(y.real(), y.imag());
                const cplx yl = -w[ord[b]] * y;
                coefr[b * m + a] = make_double2(yl.real(), yl.imag());
            }
        // Z = X Y (Ritz vectors), residual vectors H X Y - theta X Y in Y0
        if ((r = bcombine_host(c, Z, nullptr, m, X, m, coef, st))) return r;
        if ((r = bcombine_host(c, Y0, nullptr, m, H1, m, coef, st))) return r;
        if ((r = bcombine_host(c, Y0, Y0, m, X, m, coefr, st))) return r;
        LQ_CUDA(c, launch_norm2(Y0, nullptr, 0.0, nv / 2, m, c->gen_scr, st));
        std::vector<double> rn(m);
        LQ_CUDA(c, cudaMemcpyAsync(rn.data(), c->gen_scr, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
        LQ_CUDA(c, cudaStreamSynchronize(st));
        double worst = 0.0;
        for (int b = 0; b < m; ++b) {
            theta[b] = w[ord[b]];
            res[b] = std::sqrt(rn[b]) / hn;
            if (b < nev) worst = std::max(worst, res[b]);
        }
        LQ_CUDA(c, cudaMemcpyAsync(X, Z, sizeof(double) * nv * m, cudaMemcpyDeviceToDevice, st));
        if (worst <= eo->tol) break;
        a2 = std::norm(theta[m - 1]) * 1.02;         // largest Ritz value bounds the damped interval
        if (!(a2 < b2)) a2 = b2 / 25.0;
    }
    return LQ_OK;
}

// ---- shift-and-invert eigensolver ---------------------------------------------------------------
// The l eigenpairs of H(mu) nearest zero (Sec. 3; the paper computes them with ARPACK's Arnoldi
// method) as the largest-modulus eigenvalues 1/lambda of OP = H^{-1}: ARPACK's implicitly restarted
// Arnoldi method with exact shifts (Sorensen, SIAM J. Matrix Anal. Appl. 13 (1992) 357; Lehoucq &
// Sorensen, ibid. 17 (1996) 789) on OP, and on (H^dag)^{-1} = H(-mu)^{-1} for the left eigenvectors.
// The two processes run in lockstep so that their inner solves share every launch: system 0 holds
// the right process (A_0 = H), system 1 the left one (A_1 = H^dag).  Each OP application is an
// FP64 solve by defect correction around FP32 CGNR (lq_eig.cu).

struct SiWork {
    lq_ctx* c = nullptr;
    cudaStream_t st = nullptr;
    size_t V = 0, ne = 0, nv = 0;
    const void* links32 = nullptr;
    const void* links64 = nullptr;
    float4 *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr;   // [2][ne] each
    double* scal = nullptr;                      // [2][kCgNs]
    double* part = nullptr;
    int* counters = nullptr;
    double* res64 = nullptr;                     // [2][nv]
    double* tmp64 = nullptr;                     // [2][nv]
    double* nrm = nullptr;                       // [2]
    long long iters = 0, solves = 0, refinements = 0;
    int inner_max = 20000;
};

// out_s = A_s in_s, or A_s^dag in_s with adjoint (FP32 internal layout, both systems in one launch:
// side 0 of the stencil applies H, side 1 applies H^dag).
int si_apply32(SiWork& w, const float4* in, float4* out, bool adjoint) {
    lq_ctx* c = w.c;
    HopArgs a = base_hop(c);
    a.U = w.links32;             // always FP32 entries (a BF16 context gets an FP32 copy)
    a.link_bf16 = 0;
    a.Up = nullptr; a.Y = nullptr; a.Yp = nullptr;
    a.nsrc = 1; a.nsides = 2; a.side0 = 0;
    set_side(a, 0, c, 0, 0);
    set_side(a, 1, c, 1, 0);
    a.in[0] = adjoint ? in + w.ne : in;           // fed to H: system 0 (A_0 = H), or system 1 (A_1^dag = H)
    a.out[0] = adjoint ? out + w.ne : out;
    a.in[1] = adjoint ? in : in + w.ne;           // fed to H^dag
    a.out[1] = adjoint ? out : out + w.ne;
    a.src_stride_in[0] = a.src_stride_in[1] = w.ne;
    a.src_stride_out[0] = a.src_stride_out[1] = w.ne;
    LQ_CUDA(c, launch_hop(LQ_MIXED, a, 1, 0, false, w.st));
    c->launches += 1;
    return LQ_OK;
}

// The same in FP64 on boundary-layout fields [2][nv].
int si_apply64(SiWork& w, const double* in, double* out) {
    for (int s = 0; s < 2; ++s) {
        int r = apply_H_batch(w.c, in + (size_t)s * w.nv, out + (size_t)s * w.nv, 1, s, w.st, LQ_FP64, w.links64);
        if (r) return r;
    }
    return LQ_OK;
}

// CGNR on A_s e_s = rhs_s (FP32, rhs in w.z, solution in w.x) until |r_s| <= tol |rhs_s|.
int si_cgnr(SiWork& w, double tol) {
    lq_ctx* c = w.c;
    cudaStream_t st = w.st;
    const size_t bytes = sizeof(float4) * 2 * w.ne;
    LQ_CUDA(c, cudaMemsetAsync(w.x, 0, bytes, st));
    LQ_CUDA(c, cudaMemcpyAsync(w.r, w.z, bytes, cudaMemcpyDeviceToDevice, st));
    LQ_CUDA(c, cudaMemsetAsync(w.scal, 0, sizeof(double) * 2 * kCgNs, st));
    CgArgs a;
    a.ne = w.ne; a.nb = 2; a.it = 0;
    a.x = w.x; a.r = w.r; a.p = w.p; a.q = w.q; a.z = w.z;
    a.scal = w.scal; a.part = w.part; a.counters = w.counters;
    LQ_CUDA(c, launch_cg_norm(a, w.r, CG_BB, st));
    int r;
    if ((r = si_apply32(w, w.r, w.z, true))) return r;                // z = A^dag r
    LQ_CUDA(c, launch_cg_norm(a, w.z, CG_G0, st));
    LQ_CUDA(c, cudaMemcpyAsync(w.p, w.z, bytes, cudaMemcpyDeviceToDevice, st));
    c->launches += 2;
    double h[2 * kCgNs];
    int it = 0;
    for (; it < w.inner_max; ++it) {
        a.it = it;
        if ((r = si_apply32(w, w.p, w.q, false))) return r;          // q = A p
        LQ_CUDA(c, launch_cg_norm(a, w.q, CG_QQ, st));
        LQ_CUDA(c, launch_cg_xr(a, st));                            // x += alpha p, r -= alpha q
        if ((r = si_apply32(w, w.r, w.z, true))) return r;          // z = A^dag r
        LQ_CUDA(c, launch_cg_norm(a, w.z, CG_G0 + ((it + 1) & 1), st));
        LQ_CUDA(c, launch_cg_p(a, st));                             // p = z + beta p
        c->launches += 4;
        if ((it + 1) % 16 == 0 || it + 1 == w.inner_max) {
            LQ_CUDA(c, cudaMemcpyAsync(h, w.scal, sizeof(h), cudaMemcpyDeviceToHost, st));
            LQ_CUDA(c, cudaStreamSynchronize(st));
            bool all = true;
            for (int s = 0; s < 2; ++s) {
                double* hs = h + s * kCgNs;
                if (hs[CG_DONE] != 0.0) continue;
                if (!std::isfinite(hs[CG_RR])) return set_err(c, LQ_ERR_NONFINITE, "non-finite residual in an inner solve");
                if (hs[CG_RR] <= tol * tol * hs[CG_BB]) {
                    const double one = 1.0;
                    LQ_CUDA(c, cudaMemcpyAsync(w.scal + s * kCgNs + CG_DONE, &one, sizeof(double), cudaMemcpyHostToDevice, st));
                    LQ_CUDA(c, cudaStreamSynchronize(st));
                } else {
                    all = false;
                }
            }
            if (all) { ++it; break; }
        }
    }
    w.iters += it;
    return LQ_OK;
}

// x_s = A_s^{-1} b_s to relative residual tol (FP64, boundary layout [2][nv]): defect correction,
// each correction an FP32 CGNR solve of the current residual to 1e-5.
int si_solve(SiWork& w, const double* b, double* xout, double tol) {
    lq_ctx* c = w.c;
    cudaStream_t st = w.st;
    const size_t n2 = 2 * w.nv;
    LQ_CUDA(c, cudaMemsetAsync(xout, 0, sizeof(double) * n2, st));
    LQ_CUDA(c, cudaMemcpyAsync(w.res64, b, sizeof(double) * n2, cudaMemcpyDeviceToDevice, st));
    double bn[2], rn[2];
    LQ_CUDA(c, launch_norm2(b, nullptr, 0.0, w.V * 12, 2, w.nrm, st));
    LQ_CUDA(c, cudaMemcpyAsync(bn, w.nrm, sizeof(bn), cudaMemcpyDeviceToHost, st));
    LQ_CUDA(c, cudaStreamSynchronize(st));
    int r;
    for (int outer = 0;; ++outer) {
        if (outer > 0) {
            if ((r = si_apply64(w, xout, w.tmp64))) return r;           // res = b - A x
            LQ_CUDA(c, launch_axpby3(w.res64, 1.0, b, -1.0, w.tmp64, 0.0, nullptr, n2, st));
        }
        LQ_CUDA(c, launch_norm2(w.res64, nullptr, 0.0, w.V * 12, 2, w.nrm, st));
        LQ_CUDA(c, cudaMemcpyAsync(rn, w.nrm, sizeof(rn), cudaMemcpyDeviceToHost, st));
        LQ_CUDA(c, cudaStreamSynchronize(st));
        c->launches += 2;
        bool done = true;
        for (int s = 0; s < 2; ++s) {
            if (!std::isfinite(rn[s])) return set_err(c, LQ_ERR_NONFINITE, "non-finite residual in a shifted solve");
            if (rn[s] > tol * tol * bn[s]) done = false;
        }
        if (done) break;
        if (outer >= 12) return set_err(c, LQ_ERR_NOT_CONVERGED, "inner solve of the eigensolver did not converge");
        // converged systems get a zero right-hand side (their CG then stops at once)
        for (int s = 0; s < 2; ++s)
            if (rn[s] <= tol * tol * bn[s]) LQ_CUDA(c, cudaMemsetAsync(w.res64 + (size_t)s * w.nv, 0, sizeof(double) * w.nv, st));
        LQ_CUDA(c, launch_to_internal(LQ_MIXED, w.res64, w.z, w.V, 2, st));
        if ((r = si_cgnr(w, 1e-5))) return r;
        LQ_CUDA(c, launch_to_boundary(LQ_MIXED, w.x, w.tmp64, w.V, 2, st));
        LQ_CUDA(c, launch_axpby3(xout, 1.0, xout, 1.0, w.tmp64, 0.0, nullptr, n2, st));
        c->launches += 3;
        ++w.refinements;
    }
    ++w.solves;
    return LQ_OK;
}

// One implicitly shifted QR step of the m x m upper Hessenberg H (row-major) with shift mu, by
// Givens rotations; Q <- Q G_0^H G_1^H ... (Golub & Van Loan, "Matrix Computations", Sec. 7.5).
void hess_qr_step(int m, std::vector<cplx>& H, std::vector<cplx>& Q, cplx mu) {
    for (int i = 0; i < m; ++i) H[i * m + i] -= mu;
    std::vector<double> cc(m, 1.0);
    std::vector<cplx> sn(m, 0.0);
    for (int i = 0; i + 1 < m; ++i) {               // R = G_{m-2} ... G_0 (H - mu)
        const cplx a = H[i * m + i], b = H[(i + 1) * m + i];
        const double aa = std::abs(a), ab = std::abs(b), rr = std::hypot(aa, ab);
        double c_ = 1.0;
        cplx s_ = 0.0;
        if (rr > 0.0) {
            if (aa == 0.0) { c_ = 0.0; s_ = std::conj(b) / ab; }
            else { c_ = aa / rr; s_ = (a / aa) * std::conj(b) / rr; }
        }
        cc[i] = c_; sn[i] = s_;
        for (int j = 0; j < m; ++j) {
            const cplx x = H[i * m + j], y = H[(i + 1) * m + j];
            H[i * m + j] = c_ * x + s_ * y;
            H[(i + 1) * m + j] = -std::conj(s_) * x + c_ * y;
        }
    }
    for (int i = 0; i + 1 < m; ++i) {               // R Q: columns times G_i^H
        const double c_ = cc[i];
        const cplx s_ = sn[i];
        for (int r = 0; r < m; ++r) {
            const cplx u = H[r * m + i], v = H[r * m + i + 1];
            H[r * m + i] = c_ * u + std::conj(s_) * v;
            H[r * m + i + 1] = -s_ * u + c_ * v;
            const cplx qu = Q[r * m + i], qv = Q[r * m + i + 1];
            Q[r * m + i] = c_ * qu + std::conj(s_) * qv;
            Q[r * m + i + 1] = -s_ * qu + c_ * qv;
        }
    }
    for (int i = 0; i < m; ++i) H[i * m + i] += mu;
}

// Ritz values of the m x m leading block of Hm ((m + 1) x m, row-major), sorted by decreasing
// modulus, with unit eigenvectors Y (columns, in the same order) and their residual estimates
// |h_{m+1,m}| |e_m^T y| / |theta|.
int ritz(int m, const std::vector<cplx>& Hm, std::vector<cplx>& th, std::vector<cplx>& Y, std::vector<double>& est) {
    std::vector<cplx> A(m * m), w(m), Vr(m * m);
    for (int i = 0; i < m; ++i) for (int j = 0; j < m; ++j) A[i * m + j] = Hm[i * m + j];
    if (dense_eig(m, A.data(), w.data(), Vr.data()) != LQ_OK) return LQ_ERR_NEWTON;
    std::vector<int> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return std::abs(w[a]) > std::abs(w[b]); });
    th.assign(m, 0.0); Y.assign(m * m, 0.0); est.assign(m, 0.0);
    const double f = std::abs(Hm[m * m + (m - 1)]);
    for (int b = 0; b < m; ++b) {
        double nn = 0.0;
        for (int a = 0; a < m; ++a) nn += std::norm(Vr[a * m + ord[b]]);
        nn = std::sqrt(nn);
        for (int a = 0; a < m; ++a) Y[a * m + b] = Vr[a * m + ord[b]] / nn;
        th[b] = w[ord[b]];
        est[b] = f * std::abs(Y[(m - 1) * m + b]) / std::max(std::abs(th[b]), 1e-300);
    }
    return LQ_OK;
}

struct SiResult {
    std::vector<cplx> lam[2];       // eigenvalues of A_0 = H and of A_1 = H^dag
    std::vector<double> res[2];     // true residuals ||A z - lambda z|| / ||H|| (unit z)
    int restarts = 0;
};

// The implicitly restarted Arnoldi process on OP_s = A_s^{-1} for both systems.  Vb: [2][m + 1][nv]
// basis, Zs: [2][kk + 1][nv] scratch, Z: [2][nev][nv] output Ritz vectors; X0: two start fields.
int eig_shift_invert(SiWork& w, const lq_eig_opts& eo, const double* X0, double* Vb, double* Zs, double* Z,
                     double hn, SiResult& out) {
    lq_ctx* c = w.c;
    cudaStream_t st = w.st;
    const int m = eo.nsub, nev = eo.nev;
    const int kk = std::min(m - 2, nev + std::max(2, (m - nev) / 2));   // kept at a restart
    const size_t nv = w.nv;
    const double tol_in = std::max(1e-13, 0.1 * eo.tol);
    auto Vs = [&](int s, int j) { return Vb + ((size_t)s * (m + 1) + j) * nv; };
    std::vector<cplx> Hm[2];
    for (int s = 0; s < 2; ++s) Hm[s].assign((size_t)(m + 1) * m, 0.0);
    double* rhs = Zs + (size_t)2 * (kk + 1) * nv;     // [2][nv]
    double* sol = rhs + 2 * nv;                        // [2][nv]
    int r;
    // start vectors, normalised
    for (int s = 0; s < 2; ++s) {
        std::vector<double2> nn;
        if ((r = bdots_host(c, X0 + (size_t)s * nv, 1, X0 + (size_t)s * nv, 1, nn, st))) return r;
        if (!(nn[0].x > 0.0)) return set_err(c, LQ_ERR_ARG, "zero start vector for the eigensolver");
        std::vector<double2> sc(1, make_double2(1.0 / std::sqrt(nn[0].x), 0.0));
        if ((r = bcombine_host(c, Vs(s, 0), nullptr, 1, X0 + (size_t)s * nv, 1, sc, st))) return r;
    }
    int j0 = 0;
    std::vector<cplx> th[2], Y[2];
    std::vector<double> est[2];
    for (int restart = 0;; ++restart) {
        // Arnoldi steps j0 .. m-1
        for (int j = j0; j < m; ++j) {
            for (int s = 0; s < 2; ++s)
                LQ_CUDA(c, cudaMemcpyAsync(rhs + (size_t)s * nv, Vs(s, j), sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
            if ((r = si_solve(w, rhs, sol, tol_in))) return r;
            for (int s = 0; s < 2; ++s) {
                double* wv = sol + (size_t)s * nv;
                for (int pass = 0; pass < 2; ++pass) {             // classical Gram-Schmidt, twice
                    std::vector<double2> h;
                    if ((r = bdots_host(c, Vs(s, 0), j + 1, wv, 1, h, st))) return r;
                    std::vector<double2> co(j + 1);
                    for (int i = 0; i <= j; ++i) {
                        Hm[s][(size_t)i * m + j] += cplx(h[i].x, h[i].y);
                        co[i] = make_double2(-h[i].x, -h[i].y);
                    }
                    if ((r = bcombine_host(c, wv, wv, 1, Vs(s, 0), j + 1, co, st))) return r;
                }
                std::vector<double2> nn;
                if ((r = bdots_host(c, wv, 1, wv, 1, nn, st))) return r;
                const double beta = std::sqrt(std::max(nn[0].x, 0.0));
                if (!(beta > 0.0) || !std::isfinite(beta)) return set_err(c, LQ_ERR_BREAKDOWN, "Arnoldi breakdown in the eigensolver");
                Hm[s][(size_t)(j + 1) * m + j] = beta;
                std::vector<double2> sc(1, make_double2(1.0 / beta, 0.0));
                if ((r = bcombine_host(c, Vs(s, j + 1), nullptr, 1, wv, 1, sc, st))) return r;
            }
        }
        // convergence of the nev wanted Ritz pairs of both processes.  With OP z = theta z + f and
        // |f| = est |theta|: ||H z - z / theta|| = ||H f|| / |theta| <= ||H|| est, so est bounds the
        // residual relative to ||H|| that the call reports
        bool conv = true;
        for (int s = 0; s < 2; ++s) {
            if (ritz(m, Hm[s], th[s], Y[s], est[s]) != LQ_OK) return set_err(c, LQ_ERR_NEWTON, "Hessenberg eigensolver failed");
            for (int i = 0; i < nev; ++i) conv = conv && est[s][i] <= 0.5 * eo.tol;
        }
        out.restarts = restart;
        if (conv || restart >= eo.max_iter) break;
        // restart: exact shifts = the m - kk unwanted Ritz values; keep kk vectors
        for (int s = 0; s < 2; ++s) {
            std::vector<cplx> H((size_t)m * m), Q((size_t)m * m, 0.0);
            for (int i = 0; i < m; ++i) for (int jj = 0; jj < m; ++jj) H[i * m + jj] = Hm[s][(size_t)i * m + jj];
            for (int i = 0; i < m; ++i) Q[i * m + i] = 1.0;
            for (int i = kk; i < m; ++i) hess_qr_step(m, H, Q, th[s][i]);
            const cplx bk = H[(size_t)kk * m + (kk - 1)];
            const cplx sg = Q[(size_t)(m - 1) * m + (kk - 1)];
            const cplx fm = Hm[s][(size_t)m * m + (m - 1)];
            // Zs_b = sum_a V_a Q[a][b] (b < kk);  Zs_kk = bk V Q[:, kk] + fm sg v_{m+1}
            std::vector<double2> co((size_t)(kk + 1) * (m + 1), make_double2(0.0, 0.0));
            for (int b = 0; b < kk; ++b)
                for (int a = 0; a < m; ++a) co[(size_t)b * (m + 1) + a] = make_double2(Q[a * m + b].real(), Q[a * m + b].imag());
            for (int a = 0; a < m; ++a) {
                const cplx v = bk * Q[a * m + kk];
                co[(size_t)kk * (m + 1) + a] = make_double2(v.real(), v.imag());
            }
            const cplx tail = fm * sg;
            co[(size_t)kk * (m + 1) + m] = make_double2(tail.real(), tail.imag());
            double* Zb = Zs + (size_t)s * (kk + 1) * nv;
            if ((r = bcombine_host(c, Zb, nullptr, kk + 1, Vs(s, 0), m + 1, co, st))) return r;
            std::vector<double2> nn;
            if ((r = bdots_host(c, Zb + (size_t)kk * nv, 1, Zb + (size_t)kk * nv, 1, nn, st))) return r;
            const double fn = std::sqrt(std::max(nn[0].x, 0.0));
            if (!(fn > 0.0) || !std::isfinite(fn)) return set_err(c, LQ_ERR_BREAKDOWN, "invariant subspace at a restart of the eigensolver");
            LQ_CUDA(c, cudaMemcpyAsync(Vs(s, 0), Zb, sizeof(double) * nv * kk, cudaMemcpyDeviceToDevice, st));
            std::vector<double2> sc(1, make_double2(1.0 / fn, 0.0));
            if ((r = bcombine_host(c, Vs(s, kk), nullptr, 1, Zb + (size_t)kk * nv, 1, sc, st))) return r;
            std::fill(Hm[s].begin(), Hm[s].end(), cplx(0.0));
            for (int i = 0; i < kk; ++i) for (int jj = 0; jj < kk; ++jj) Hm[s][(size_t)i * m + jj] = H[i * m + jj];
            Hm[s][(size_t)kk * m + (kk - 1)] = fn;
        }
        j0 = kk;
    }
    // Ritz vectors z = V y of the nev wanted pairs, lambda = 1 / theta, and their true residuals
    for (int s = 0; s < 2; ++s) {
        std::vector<double2> co((size_t)nev * m);
        for (int b = 0; b < nev; ++b)
            for (int a = 0; a < m; ++a) co[(size_t)b * m + a] = make_double2(Y[s][a * m + b].real(), Y[s][a * m + b].imag());
        double* Zo = Z + (size_t)s * nev * nv;
        if ((r = bcombine_host(c, Zo, nullptr, nev, Vs(s, 0), m, co, st))) return r;
        out.lam[s].resize(nev);
        for (int i = 0; i < nev; ++i) out.lam[s][i] = 1.0 / th[s][i];
        double* HZ = Zs;                                   // nev <= kk + 1 vectors of scratch
        if ((r = apply_H_batch(c, Zo, HZ, nev, s, st, LQ_FP64, w.links64))) return r;
        std::vector<double2> cr((size_t)nev * nev, make_double2(0.0, 0.0));
        for (int i = 0; i < nev; ++i) cr[(size_t)i * nev + i] = make_double2(-out.lam[s][i].real(), -out.lam[s][i].imag());
        if ((r = bcombine_host(c, HZ, HZ, nev, Zo, nev, cr, st))) return r;
        std::vector<double2> rr, zz;
        out.res[s].assign(nev, 0.0);
        for (int i = 0; i < nev; ++i) {
            if ((r = bdots_host(c, HZ + (size_t)i * nv, 1, HZ + (size_t)i * nv, 1, rr, st))) return r;
            if ((r = bdots_host(c, Zo + (size_t)i * nv, 1, Zo + (size_t)i * nv, 1, zz, st))) return r;
            out.res[s][i] = std::sqrt(rr[0].x / zz[0].x) / hn;
        }
    }
    return LQ_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
extern "C" {

void lq_default_opts(lq_opts* o) {
    if (!o) return;
    o->kmax = 0;
    o->breakdown_tol = 1e-14;
    o->newton_max_iter = 50;
    o->newton_tol = 1e-13;
    o->deflate = 0;
    o->projected = LQ_PROJ_AUTO;
    o->quad_nodes = 64;
    o->proj_tol = 1e-11;
    o->hop_variant = -1;
    o->defl_kmax = 0;
    o->defl_nderiv = 0;
    o->two_pass = 0;
    o->graph = -1;
    o->split = -1;
    o->update_variant = -1;
    o->nested_m = 100;
    o->rebiorth = 0;
}

int lq_create(const lq_lattice_desc* d, lq_ctx** out) {
    if (!d || !out) return LQ_ERR_ARG;
    *out = nullptr;
    if (d->nt < 1 || d->nx < 1 || d->ny < 1 || d->nz < 1) return LQ_ERR_ARG;
    if (d->r != 1.0) return LQ_ERR_ARG;
    if (d->precision != LQ_FP64 && d->precision != LQ_MIXED && d->precision != LQ_MIXED_BF16 &&
        d->precision != LQ_FLOAT_FLOAT)
        return LQ_ERR_ARG;
    if (!std::isfinite(d->mu) || !std::isfinite(d->m_w)) return LQ_ERR_ARG;
    const double vol = (double)d->nt * d->nx * d->ny * d->nz;
    if (vol * 12.0 > 4.0e9) return LQ_ERR_ARG;
    lq_ctx* c = new (std::nothrow) lq_ctx();
    if (!c) return LQ_ERR_OOM;
    c->desc = *d;
    c->dims[0] = d->nx; c->dims[1] = d->ny; c->dims[2] = d->nz; c->dims[3] = d->nt;
    c->V = (size_t)d->nt * d->nx * d->ny * d->nz;
    c->prec = d->precision == LQ_MIXED_BF16 ? LQ_MIXED : d->precision;
    c->link_bf16 = d->precision == LQ_MIXED_BF16;
    cudaGetDevice(&c->device);
    *out = c;
    return LQ_OK;
}

void lq_destroy(lq_ctx* c) {
    if (!c) return;
    free_workspace(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->cap_stream2) cudaStreamDestroy(c->cap_stream2);
    dfree(c->U);
    dfree(c->Ub);
    dfree(c->Y);
    dfree(c->Up);
    dfree(c->Yp);
    dfree(c->dir_scratch);
    dfree(c->defl_V); dfree(c->defl_W); dfree(c->defl_work); dfree(c->defl_scr); dfree(c->defl_shift);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
}

const char* lq_last_error(const lq_ctx* c) { return c ? c->err.c_str() : "null context"; }

int lq_upload_gauge(lq_ctx* c, const double* U, void* stream) {
    if (!c || !U) return set_err(c, LQ_ERR_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = c->V * 4 * 9 * 2;
    if (!c->Ub) { int r = dalloc(c, &c->Ub, n); if (r) return r; }
    if (!c->U) {
        // FP64: double2, FP32: float2, BF16: two bfloat16 (4 bytes), float-float: 16 bytes per entry
        size_t cb = link_entry_bytes(c) * c->V * 36;
        void* p = nullptr;
        if (cudaMalloc(&p, cb) != cudaSuccess) { cudaGetLastError(); return set_err(c, LQ_ERR_OOM, "gauge allocation failed"); }
        c->U = p;
    }
    int r = stage_in(c, c->Ub, U, n, st);
    if (r) return r;
    if (c->link_bf16) {
        // round the FP64 copy to the stored BF16 values: every operator of the context uses them
        LQ_CUDA(c, launch_links_bf16(c->Ub, c->U, c->V, st));
    } else {
        LQ_CUDA(c, launch_links_internal(c->prec, c->Ub, c->U, c->V, st));
    }
    c->launches += 1;
    if (c->prec == LQ_MIXED && !c->link_bf16) {   // the packed stencil's copy of the FP32 links
        if (!c->Up && cudaMalloc(&c->Up, sizeof(float4) * c->V * 36) != cudaSuccess) {
            cudaGetLastError();
            c->Up = nullptr;
            return set_err(c, LQ_ERR_OOM, "packed gauge allocation failed");
        }
        LQ_CUDA(c, launch_links_packed(c->U, c->Up, c->V, st));
        c->launches += 1;
    }
    c->gauge_ready = true;
    ++c->defl_version;
    if (c->dir_kind == LQ_DIR_SU3 || c->dir_kind == LQ_DIR_U1) c->dir_kind = -1;   // Y is stale
    return LQ_OK;
}

int lq_set_mu(lq_ctx* c, double mu) {
    if (!c || !std::isfinite(mu)) return set_err(c, LQ_ERR_ARG, "invalid mu");
    c->desc.mu = mu;
    return LQ_OK;
}

int lq_reserve(lq_ctx* c, int kmax, int nsrc, int flags) {
    if (c) c->defl_prep_ok = false;
    if (!c || kmax < 1 || nsrc < 1 ||
        (flags & ~(LQ_RESERVE_BLOCK | LQ_RESERVE_ADJOINT | LQ_RESERVE_TWO_PASS | LQ_RESERVE_SOLVE | LQ_RESERVE_REBIORTH)))
        return set_err(c, LQ_ERR_ARG, "invalid reserve arguments");
    free_workspace(c);
    const int block = (flags & LQ_RESERVE_BLOCK) ? 1 : 0;
    const int nf = block ? 2 : 1;
    const size_t fbytes = fb(c);
    int r;
    auto alloc_fields = [&](void** p, size_t nfields) -> int {
        size_t bytes = nfields * fbytes;
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return set_err(c, LQ_ERR_OOM, "workspace allocation of " + std::to_string(bytes) + " bytes failed");
        }
        return LQ_OK;
    };
    // the Krylov basis: kmax vectors per source, or a ring of kTwoPassRing for two-pass runs
    const int ring = ((flags & LQ_RESERVE_TWO_PASS) && kmax > kTwoPassRing) ? kTwoPassRing : 0;
    const bool rbw = (flags & LQ_RESERVE_REBIORTH) != 0;
    if (rbw && ring) return set_err(c, LQ_ERR_ARG, "LQ_RESERVE_REBIORTH needs the whole basis: not with a two-pass ring");
    if ((r = alloc_fields(&c->basis, (size_t)nsrc * (ring ? ring : kmax) * nf))) { free_workspace(c); return r; }
    if ((r = alloc_fields(&c->left, (size_t)nsrc * 3 * nf))) { free_workspace(c); return r; }
    if ((r = alloc_fields(&c->rout, (size_t)nsrc * nf))) { free_workspace(c); return r; }
    if ((r = alloc_fields(&c->lout, (size_t)nsrc * nf))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->io, (size_t)6 * nsrc * c->V * 24))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->norms, (size_t)3 * nsrc))) { free_workspace(c); return r; }
    size_t pb = (c->V + 31) / 32;   // finest stencil grid (32 sites per block)
    pb = std::max(pb, (size_t)64);   // update grid (one resident wave over all sources, capped here)
    pb = std::max(pb, (c->V + kUpdThreads - 1) / kUpdThreads);
    c->partial_blocks = pb;
    if ((r = dalloc(c, &c->partials, (size_t)nsrc * pb * 12))) { free_workspace(c); return r; }   // 6 sums per block
    if ((r = dalloc(c, &c->counters, (size_t)4 * nsrc))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->state, (size_t)nsrc))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->alpha, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->beta, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->delta, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->scale, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    const size_t kk = (size_t)kmax * kmax;
    if ((r = dalloc(c, &c->nx_X, (size_t)nsrc * kk))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nx_Y, (size_t)nsrc * kk))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nx_F, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nx_perm, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nx_scal, (size_t)nsrc * 16))) { free_workspace(c); return r; }
    c->nx_partial_blocks = (kk + 255) / 256;
    if ((r = dalloc(c, &c->nx_partials, (size_t)nsrc * c->nx_partial_blocks * 4))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nx_counters, (size_t)3 * nsrc))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->proj_c, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->quad_q, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->quad_work, (size_t)nsrc * kmax * 4 * 2 * kQuadRetryMaxNodes))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->quad_c, (size_t)nsrc))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->quad_check, (size_t)nsrc))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->quad_nodes, (size_t)nsrc))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->quad_part, (size_t)nsrc * (2 * kQuadRetryMaxNodes / kQuadBlk) * kmax))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->proj_sel, (size_t)nsrc))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nest_state, (size_t)nsrc))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nest_alpha, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nest_beta, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nest_delta, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nest_s, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nest_q, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nest_norm, (size_t)nsrc))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nest_check, (size_t)nsrc))) { free_workspace(c); return r; }
    if ((r = dalloc(c, &c->nest_c, (size_t)nsrc))) { free_workspace(c); return r; }
    {
        const int m = std::max(2 * nsrc, 64);   // dots among up to m x m vectors
        c->gen_scr_doubles = bdots_partial_doubles(m * m) + (size_t)2 * m * m;
        if ((r = dalloc(c, &c->gen_scr, c->gen_scr_doubles))) { free_workspace(c); return r; }
    }
    if ((flags & LQ_RESERVE_SOLVE) && (r = dalloc(c, &c->solve_ws, (size_t)9 * nsrc * c->V * 24))) { free_workspace(c); return r; }
    if ((flags & LQ_RESERVE_ADJOINT) || rbw) {
        // stored left basis: one field per vector for the adjoint, NF for the re-biorthogonalisation
        c->lbasis_nf = rbw ? nf : 1;
        if ((r = alloc_fields(&c->lbasis, (size_t)nsrc * (ring ? ring : kmax) * c->lbasis_nf))) { free_workspace(c); return r; }
        if ((r = dalloc(c, &c->uscale, (size_t)nsrc * kmax))) { free_workspace(c); return r; }
    }
    if (rbw) {
        const size_t nelem = (size_t)nf * fe(c);
        if ((r = dalloc(c, &c->rb_part, (size_t)nsrc * kmax * rb_dot_blocks(nelem) * 8))) { free_workspace(c); return r; }
        if ((r = dalloc(c, &c->rb_coef, (size_t)nsrc * 2 * kmax))) { free_workspace(c); return r; }
        if ((r = dalloc(c, &c->rb_coef_f, (size_t)nsrc * 2 * kmax))) { free_workspace(c); return r; }
        c->rebiorth = true;
    }
    if (flags & LQ_RESERVE_ADJOINT) {
        const int np = 2 * kQuadMaxNodes;
        if ((r = dalloc(c, &c->adj_coef, (size_t)2 * np * kmax))) { free_workspace(c); return r; }
        if ((r = alloc_fields(&c->adj_nu, (size_t)np))) { free_workspace(c); return r; }
        if ((r = alloc_fields(&c->adj_om, (size_t)np))) { free_workspace(c); return r; }
        if ((r = dalloc(c, &c->adj_force, c->V * 32))) { free_workspace(c); return r; }
        if ((r = dalloc(c, &c->adj_dmu, c->V / 128 + 1))) { free_workspace(c); return r; }
        c->adjoint = true;
    }
    LQ_CUDA(c, cudaMemset(c->counters, 0, sizeof(int) * 4 * nsrc));
    LQ_CUDA(c, cudaMemset(c->nx_counters, 0, sizeof(int) * 3 * nsrc));
    LQ_CUDA(c, cudaMemset(c->nx_scal, 0, sizeof(double) * 16 * nsrc));
    LQ_CUDA(c, cudaMemset(c->state, 0, sizeof(TslState) * nsrc));
    LQ_CUDA(c, cudaMemset(c->nest_state, 0, sizeof(TslState) * nsrc));
    c->kmax = kmax;
    c->nsrc = nsrc;
    c->block = block;
    c->ring = ring;
    return LQ_OK;
}

int lq_apply_H(lq_ctx* c, const double* x, double* y, int nsrc, int dagger, void* stream) {
    if (!c || !x || !y) return set_err(c, LQ_ERR_ARG, "null argument");
    int r = check_ready(c, nsrc, 0);
    if (r) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)nsrc * c->V * 24;
    double* io = c->io;
    if ((r = stage_in(c, io, x, n, st))) return r;
    LQ_CUDA(c, launch_to_internal(c->prec, io, c->rout, c->V, nsrc, st));
    c->launches += 3;
    HopArgs a = base_hop(c);
    a.nsrc = nsrc;
    a.nsides = 1;
    a.side0 = 0;
    set_side(a, 0, c, dagger ? 1 : 0, 0);
    a.in[0] = c->rout;
    a.out[0] = c->lout;
    a.src_stride_in[0] = fe(c);
    a.src_stride_out[0] = fe(c);
    LQ_CUDA(c, launch_hop(c->prec, a, 1, 0, false, st));
    LQ_CUDA(c, launch_to_boundary(c->prec, c->lout, io, c->V, nsrc, st));
    return stage_out(c, y, io, n, st);
}

int lq_set_direction(lq_ctx* c, const lq_direction* d, void* stream) {
    if (!c || !d) return set_err(c, LQ_ERR_ARG, "null argument");
    if (d->kind == LQ_DIR_MU) { c->dir_kind = LQ_DIR_MU; return LQ_OK; }
    if (d->kind != LQ_DIR_SU3 && d->kind != LQ_DIR_U1) return set_err(c, LQ_ERR_ARG, "unknown direction kind");
    if (!d->field) return set_err(c, LQ_ERR_ARG, "direction field is null");
    if (!c->gauge_ready) return set_err(c, LQ_ERR_NOT_READY, "gauge field not uploaded");
    cudaStream_t st = (cudaStream_t)stream;
    int r;
    if (!c->dir_scratch && (r = dalloc(c, &c->dir_scratch, c->V * 4 * 8))) return r;
    if (!c->Y) {
        size_t cb = (c->prec == LQ_MIXED ? sizeof(float2) : (size_t)16) * c->V * 36;
        void* p = nullptr;
        if (cudaMalloc(&p, cb) != cudaSuccess) { cudaGetLastError(); return set_err(c, LQ_ERR_OOM, "direction allocation failed"); }
        c->Y = p;
    }
    const size_t n = c->V * 4 * (d->kind == LQ_DIR_SU3 ? 8 : 1);
    if ((r = stage_in(c, c->dir_scratch, d->field, n, st))) return r;
    LQ_CUDA(c, launch_direction(c->prec, c->Ub, c->dir_scratch, d->kind, c->Y, c->V, st));
    c->launches += 1;
    if (c->prec == LQ_MIXED) {
        if (!c->Yp && cudaMalloc(&c->Yp, sizeof(float4) * c->V * 36) != cudaSuccess) {
            cudaGetLastError();
            c->Yp = nullptr;
            return set_err(c, LQ_ERR_OOM, "packed direction allocation failed");
        }
        LQ_CUDA(c, launch_links_packed(c->Y, c->Yp, c->V, st));
        c->launches += 1;
    }
    c->dir_kind = d->kind;
    return LQ_OK;
}

int lq_apply_block(lq_ctx* c, const double* xt, const double* xb, double* yt, double* yb, int nsrc, int dagger, void* stream) {
    if (!c || !xt || !xb || !yt || !yb) return set_err(c, LQ_ERR_ARG, "null argument");
    int r = check_ready(c, nsrc, 1);
    if (r) return r;
    if (c->dir_kind < 0) return set_err(c, LQ_ERR_NOT_READY, "no derivative direction set");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)c->V * 24;
    double* io = c->io;
    // stage as [src][2][V][12]: top, bottom
    for (int s = 0; s < nsrc; ++s) {
        if ((r = stage_in(c, io + (2 * (size_t)s) * n, xt + (size_t)s * n, n, st))) return r;
        if ((r = stage_in(c, io + (2 * (size_t)s + 1) * n, xb + (size_t)s * n, n, st))) return r;
    }
    LQ_CUDA(c, launch_to_internal(c->prec, io, c->rout, c->V, 2 * nsrc, st));
    c->launches += 3;
    const int em = emode_of(c);
    HopArgs a = base_hop(c);
    a.nsrc = nsrc;
    a.nsides = 1;
    a.side0 = dagger ? 1 : 0;
    set_side(a, a.side0, c, dagger ? 1 : 0, em);
    a.in[a.side0] = c->rout;
    a.out[a.side0] = c->lout;
    a.src_stride_in[a.side0] = 2 * fe(c);
    a.src_stride_out[a.side0] = 2 * fe(c);
    LQ_CUDA(c, launch_hop(c->prec, a, 2, em, false, st));
    LQ_CUDA(c, launch_to_boundary(c->prec, c->lout, io, c->V, 2 * nsrc, st));
    for (int s = 0; s < nsrc; ++s) {
        if ((r = stage_out(c, yt + (size_t)s * n, io + (2 * (size_t)s) * n, n, st))) return r;
        if ((r = stage_out(c, yb + (size_t)s * n, io + (2 * (size_t)s + 1) * n, n, st))) return r;
    }
    return LQ_OK;
}

}  // extern "C"

namespace {

// sgn(H) x (Eq. (3.1) deflation when opts ask for it) into staging region 1; x is staged into
// region 0 (and deflated there).
int sign_core(lq_ctx* c, const double* x, int nsrc, const lq_opts* o, lq_report* rep, cudaStream_t st) {
    int r = check_ready(c, nsrc, 0);
    if (r || (r = check_opts(c, o, true))) return r;
    const size_t n = (size_t)nsrc * c->V * 24;
    double* y0 = c->io + (size_t)c->nsrc * c->V * 24;
    if ((r = stage_in(c, c->io, x, n, st))) return r;
    const int l = o->deflate ? c->defl_l : 0;
    std::vector<double2> cx, coef;
    if (l > 0) {
        // Eq. (3.1): x' = Pbar x = x - sum_i R_i <Lk_i|x>
        if ((r = bdots_host(c, c->defl_W, l, c->io, nsrc, cx, st))) return r;
        coef.assign((size_t)nsrc * l, make_double2(0.0, 0.0));
        for (int s = 0; s < nsrc; ++s) for (int i = 0; i < l; ++i) coef[(size_t)s * l + i] = make_double2(-cx[(size_t)i * nsrc + s].x, -cx[(size_t)i * nsrc + s].y);
        if ((r = bcombine_host(c, c->io, c->io, nsrc, c->defl_V, l, coef, st))) return r;
    }
    if ((r = run_tsl(c, 1, 0, nsrc, o, rep, y0, nullptr, st, c->io))) return r;
    if (l > 0) {
        // + sum_i sgn(lambda_i) R_i <Lk_i|x>
        for (int s = 0; s < nsrc; ++s) for (int i = 0; i < l; ++i) {
            const double sg = sgn_re(c->defl_lam[i]);
            coef[(size_t)s * l + i] = make_double2(sg * cx[(size_t)i * nsrc + s].x, sg * cx[(size_t)i * nsrc + s].y);
        }
        if ((r = bcombine_host(c, y0, y0, nsrc, c->defl_V, l, coef, st))) return r;
    }
    return LQ_OK;
}

// (d sgn(H) x, sgn(H) x) into staging regions 1 and 2 (generalised deflation, Eqs. (3.2)-(3.4),
// when opts ask for it); x is staged into region 0.
int sign_derivative_core(lq_ctx* c, const lq_direction* dir, const double* x, int nsrc, const lq_opts* o,
                         lq_report* rep, cudaStream_t st) {
    int r = check_ready(c, nsrc, 1);
    if (r || (r = check_opts(c, o, true))) return r;
    if ((r = lq_set_direction(c, dir, st))) return r;
    const size_t n = (size_t)nsrc * c->V * 24;
    const size_t reg = (size_t)c->nsrc * c->V * 24;
    double* y0 = c->io + reg;
    double* y1 = c->io + 2 * reg;
    if ((r = stage_in(c, c->io, x, n, st))) return r;
    const int l = o->deflate ? c->defl_l : 0;
    if (l == 0) {
        if ((r = run_tsl(c, 2, emode_of(c), nsrc, o, rep, y0, y1, st))) return r;
    } else {
        // generalised deflation, Eqs. (3.2)-(3.4), for psi = (0, x):
        //   Pbar psi = (-sum_i [R_i <dLk_i|x> + dR_i <Lk_i|x>],  x - sum_i R_i <Lk_i|x>)
        //   exact    = ( sum_i sgn_i [R_i <dLk_i|x> + dR_i <Lk_i|x>],  sum_i sgn_i R_i <Lk_i|x>)
        const int ld = nderiv_of(c, o);   // Jordan blocks used (coefficients of the other pairs stay 0)
        const int kd = o->defl_kmax > 0 ? o->defl_kmax : c->kmax;
        const bool cached = c->dir_kind == LQ_DIR_MU && c->defl_prep_ok && c->defl_prep_version == c->defl_version &&
                            c->defl_prep_mu == c->desc.mu && c->defl_prep_ld == ld && c->defl_prep_kd == kd;
        if (!cached) {
            c->defl_prep_ok = false;
            if ((r = prepare_deflation_derivative(c, o, st))) return r;
            if (c->dir_kind == LQ_DIR_MU) {
                c->defl_prep_ok = true;
                c->defl_prep_version = c->defl_version;
                c->defl_prep_mu = c->desc.mu;
                c->defl_prep_ld = ld;
                c->defl_prep_kd = kd;
            }
        }
        std::vector<double2> cd;   // [2l][nsrc]: <Lk_i|x>, then <dLk_i|x>
        if ((r = bdots_host(c, c->defl_W, 2 * l, c->io, nsrc, cd, st))) return r;
        double* xt = c->io + 3 * reg;
        double* xb = c->io + 4 * reg;
        std::vector<double2> ct((size_t)nsrc * 2 * l), cb((size_t)nsrc * 2 * l);
        for (int s = 0; s < nsrc; ++s)
            for (int i = 0; i < ld; ++i) {
                const double2 a = cd[(size_t)i * nsrc + s], b = cd[(size_t)(l + i) * nsrc + s];
                ct[(size_t)s * 2 * l + i] = make_double2(-b.x, -b.y);        // R_i <dLk_i|x>
                ct[(size_t)s * 2 * l + l + i] = make_double2(-a.x, -a.y);    // dR_i <Lk_i|x>
                cb[(size_t)s * 2 * l + i] = make_double2(-a.x, -a.y);
                cb[(size_t)s * 2 * l + l + i] = make_double2(0.0, 0.0);
            }
        if ((r = bcombine_host(c, xt, nullptr, nsrc, c->defl_V, 2 * l, ct, st))) return r;
        if ((r = bcombine_host(c, xb, c->io, nsrc, c->defl_V, 2 * l, cb, st))) return r;
        if ((r = run_tsl(c, 2, emode_of(c), nsrc, o, rep, y0, y1, st, xb, xt))) return r;
        for (auto& v : ct) v = make_double2(-v.x, -v.y);
        for (auto& v : cb) v = make_double2(-v.x, -v.y);
        for (int s = 0; s < nsrc; ++s)
            for (int i = 0; i < ld; ++i) {
                const double sg = sgn_re(c->defl_lam[i]);
                for (int h = 0; h < 2; ++h) {
                    double2& u = ct[(size_t)s * 2 * l + h * l + i];
                    u = make_double2(sg * u.x, sg * u.y);
                }
                double2& u = cb[(size_t)s * 2 * l + i];
                u = make_double2(sg * u.x, sg * u.y);
            }
        if ((r = bcombine_host(c, y0, y0, nsrc, c->defl_V, 2 * l, ct, st))) return r;
        if ((r = bcombine_host(c, y1, y1, nsrc, c->defl_V, 2 * l, cb, st))) return r;
    }
    return LQ_OK;
}


// ---- overlap solver (lq_overlap_solve, lq_axial_current) -----------------------------------
// Per-source inner products <X_s|Y_s> over the first nsrc fields of two device sets.
int sdots_host(lq_ctx* c, const double* X, const double* Y, int nsrc, std::vector<cplx>& out, cudaStream_t st) {
    const size_t nv = nvec(c);
    double* part = c->gen_scr;
    double* res = part + bdots_partial_doubles(nsrc);
    LQ_CUDA(c, launch_sdots(X, Y, nv, nv, nsrc, part, res, st));
    std::vector<double2> h(nsrc);
    LQ_CUDA(c, cudaMemcpyAsync(h.data(), res, sizeof(double2) * nsrc, cudaMemcpyDeviceToHost, st));
    LQ_CUDA(c, cudaStreamSynchronize(st));
    c->launches += 2;
    out.resize(nsrc);
    for (int s = 0; s < nsrc; ++s) out[s] = cplx(h[s].x, h[s].y);
    return LQ_OK;
}

// Z_s = a_s X0_s + b_s X1_s + c_s X2_s with per-source complex coefficients (host values)
int scomb_host(lq_ctx* c, double* Z, const double* X0, const double* X1, const double* X2, const std::vector<cplx>& a,
               const std::vector<cplx>& b, const std::vector<cplx>& cc, int nsrc, cudaStream_t st) {
    const size_t nv = nvec(c);
    std::vector<double2> coef((size_t)3 * nsrc);
    for (int s = 0; s < nsrc; ++s) {
        coef[3 * s] = make_double2(a[s].real(), a[s].imag());
        coef[3 * s + 1] = make_double2(b.empty() ? 0.0 : b[s].real(), b.empty() ? 0.0 : b[s].imag());
        coef[3 * s + 2] = make_double2(cc.empty() ? 0.0 : cc[s].real(), cc.empty() ? 0.0 : cc[s].imag());
    }
    double* dcoef = c->gen_scr + bdots_partial_doubles(nsrc) + 2 * (size_t)nsrc;
    LQ_CUDA(c, cudaMemcpyAsync(dcoef, coef.data(), sizeof(double2) * coef.size(), cudaMemcpyHostToDevice, st));
    LQ_CUDA(c, launch_scomb(Z, X0, X1, X2, dcoef, nv, nv, nsrc, st));
    c->launches += 1;
    return LQ_OK;
}

// out = D(m) x = (1 - m/2)(x + gamma5 sgn(H) x) + m x = (1 + m/2) x + (1 - m/2) gamma5 sgn(H) x for
// nsrc device fields; sgn(H) x by the two-sided Lanczos process with opts (into staging region 1).
// worst[s] keeps the worst status of the sign solves of a source still running (done[s] == 0: a
// finished source is applied to a zero vector, whose solve reports an empty source).
int apply_Dm(lq_ctx* c, const double* x, double* out, int nsrc, double mass, const lq_opts* o, std::vector<int>& worst,
             const std::vector<int>& done, cudaStream_t st) {
    std::vector<lq_report> rep(nsrc);
    int r = sign_core(c, x, nsrc, o, rep.data(), st);
    if (r) return r;
    for (int s = 0; s < nsrc; ++s) if (!done[s] && rep[s].status < 0 && worst[s] == LQ_OK) worst[s] = rep[s].status;
    LQ_CUDA(c, launch_g5axpy(out, x, 1.0 + 0.5 * mass, c->io + (size_t)c->nsrc * c->V * 24, 1.0 - 0.5 * mass,
                             (size_t)nsrc * c->V, st));
    c->launches += 1;
    return LQ_OK;
}

// BiCGStab for D(m) Z = B, nsrc sources at once with their own scalars (van der Vorst, SIAM J.
// Sci. Stat. Comput. 13 (1992)).  B and Z are fields of the solver workspace (device); the six
// others hold the recurrence vectors.  A source stops when its recursive residual is below
// tol ||b||; its scalars are then zero, so its vectors no longer change.  The reported residual
// is recomputed as ||B - D(m) Z|| at the end.
int overlap_bicgstab(lq_ctx* c, const double* B, double* Z, int nsrc, double mass, double tol, int max_iter,
                     const lq_opts* o, lq_solve_report* rep, cudaStream_t st) {
    const size_t nv = nvec(c), reg = (size_t)c->nsrc * nv;
    double* R = c->solve_ws;
    double* RH = R + reg;
    double* P = RH + reg;
    double* Vv = P + reg;
    double* S = Vv + reg;
    double* T = S + reg;
    const size_t bytes = sizeof(double) * nv * nsrc;
    LQ_CUDA(c, cudaMemsetAsync(Z, 0, bytes, st));
    LQ_CUDA(c, cudaMemcpyAsync(R, B, bytes, cudaMemcpyDeviceToDevice, st));
    LQ_CUDA(c, cudaMemcpyAsync(RH, B, bytes, cudaMemcpyDeviceToDevice, st));
    LQ_CUDA(c, cudaMemsetAsync(P, 0, bytes, st));
    LQ_CUDA(c, cudaMemsetAsync(Vv, 0, bytes, st));
    std::vector<cplx> bb, rho1, d, ts, tt, rr;
    int r = sdots_host(c, B, B, nsrc, bb, st);
    if (r) return r;
    std::vector<double> bn(nsrc);
    std::vector<cplx> rho(nsrc, 1.0), alpha(nsrc, 1.0), omega(nsrc, 1.0), one(nsrc, 1.0);
    std::vector<int> done(nsrc, 0), conv(nsrc, 0), status(nsrc, LQ_OK), iters(nsrc, 0), worst(nsrc, LQ_OK);
    for (int s = 0; s < nsrc; ++s) {
        bn[s] = std::sqrt(std::max(bb[s].real(), 0.0));
        if (!(bn[s] > 0.0)) done[s] = conv[s] = 1;
    }
    const std::vector<cplx> nocoef;   // an absent third term of scomb_host
    auto all_done = [&]() { return std::all_of(done.begin(), done.end(), [](int v) { return v != 0; }); };
    auto tiny = [](cplx v, double scale) { return !(std::abs(v) > 1e-300 * scale) || !std::isfinite(std::abs(v)); };
    for (int it = 0; it < max_iter && !all_done(); ++it) {
        if ((r = sdots_host(c, RH, R, nsrc, rho1, st))) return r;
        std::vector<cplx> beta(nsrc, 0.0), mbo(nsrc, 0.0);
        for (int s = 0; s < nsrc; ++s) {
            if (done[s]) continue;
            if (tiny(rho1[s], bn[s] * bn[s] * 1e-30) || tiny(omega[s], 1.0)) { status[s] = LQ_ERR_BREAKDOWN; done[s] = 1; continue; }
            beta[s] = (rho1[s] / rho[s]) * (alpha[s] / omega[s]);
            mbo[s] = -beta[s] * omega[s];
        }
        std::vector<cplx> keep(nsrc);
        for (int s = 0; s < nsrc; ++s) keep[s] = done[s] ? cplx(0.0) : cplx(1.0);
        // P = R + beta (P - omega V) for running sources; a finished source keeps P = 0
        if ((r = scomb_host(c, P, R, P, Vv, keep, beta, mbo, nsrc, st))) return r;
        if ((r = apply_Dm(c, P, Vv, nsrc, mass, o, worst, done, st))) return r;
        if ((r = sdots_host(c, RH, Vv, nsrc, d, st))) return r;
        std::vector<cplx> malpha(nsrc, 0.0);
        for (int s = 0; s < nsrc; ++s) {
            if (done[s]) { alpha[s] = 0.0; continue; }
            if (tiny(d[s], bn[s] * bn[s] * 1e-30)) { status[s] = LQ_ERR_BREAKDOWN; done[s] = 1; alpha[s] = 0.0; continue; }
            alpha[s] = rho1[s] / d[s];
            malpha[s] = -alpha[s];
        }
        if ((r = scomb_host(c, S, R, Vv, nullptr, one, malpha, nocoef, nsrc, st))) return r;   // S = R - alpha V
        if ((r = apply_Dm(c, S, T, nsrc, mass, o, worst, done, st))) return r;
        if ((r = sdots_host(c, T, S, nsrc, ts, st))) return r;
        if ((r = sdots_host(c, T, T, nsrc, tt, st))) return r;
        std::vector<cplx> momega(nsrc, 0.0);
        for (int s = 0; s < nsrc; ++s) {
            if (done[s]) { omega[s] = 0.0; continue; }
            omega[s] = tt[s].real() > 0.0 ? ts[s] / tt[s].real() : cplx(0.0);
            momega[s] = -omega[s];
        }
        if ((r = scomb_host(c, Z, Z, P, S, one, alpha, omega, nsrc, st))) return r;         // Z += alpha P + omega S
        if ((r = scomb_host(c, R, S, T, nullptr, one, momega, nocoef, nsrc, st))) return r;     // R = S - omega T
        if ((r = sdots_host(c, R, R, nsrc, rr, st))) return r;
        for (int s = 0; s < nsrc; ++s) {
            if (done[s]) continue;
            iters[s] = it + 1;
            rho[s] = rho1[s];
            if (std::sqrt(std::max(rr[s].real(), 0.0)) <= tol * bn[s]) done[s] = conv[s] = 1;
            else if (tiny(omega[s], 1.0)) { status[s] = LQ_ERR_BREAKDOWN; done[s] = 1; }
        }
    }
    // true residual
    const std::vector<int> none(nsrc, 0);
    if ((r = apply_Dm(c, Z, T, nsrc, mass, o, worst, none, st))) return r;
    std::vector<cplx> mone(nsrc, -1.0);
    if ((r = scomb_host(c, R, B, T, nullptr, one, mone, nocoef, nsrc, st))) return r;
    if ((r = sdots_host(c, R, R, nsrc, rr, st))) return r;
    if (rep) {
        for (int s = 0; s < nsrc; ++s) {
            lq_solve_report& q = rep[s];
            q.iterations = iters[s];
            q.residual = bn[s] > 0.0 ? std::sqrt(std::max(rr[s].real(), 0.0)) / bn[s] : 0.0;
            // converged: the recursive residual met tol (the recomputed one is reported as is)
            q.status = status[s] != LQ_OK ? status[s] : worst[s] != LQ_OK ? worst[s] : conv[s] ? LQ_OK : LQ_ERR_NOT_CONVERGED;
        }
    }
    return LQ_OK;
}

int solve_ready(lq_ctx* c, int nsrc, int need_block, double mass, double tol, int max_iter, const lq_opts* o) {
    int r = check_ready(c, nsrc, need_block);
    if (r || (r = check_opts(c, o, true))) return r;
    if (!c->solve_ws) return set_err(c, LQ_ERR_NOT_READY, "workspace reserved without LQ_RESERVE_SOLVE");
    if (!(tol > 0.0) || max_iter < 1 || !std::isfinite(mass)) return set_err(c, LQ_ERR_ARG, "need tol > 0, max_iter >= 1, finite mass");
    return LQ_OK;
}

}  // namespace

extern "C" {

int lq_sign_apply(lq_ctx* c, const double* x, double* y, int nsrc, const lq_opts* o, lq_report* rep, void* stream) {
    if (!c || !x || !y) return set_err(c, LQ_ERR_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    int r = sign_core(c, x, nsrc, o, rep, st);
    if (r) return r;
    if ((r = stage_out(c, y, c->io + (size_t)c->nsrc * c->V * 24, (size_t)nsrc * c->V * 24, st))) return r;
    LQ_CUDA(c, cudaStreamSynchronize(st));
    return LQ_OK;
}

int lq_sign_derivative_apply(lq_ctx* c, const lq_direction* dir, const double* x, double* ys, double* yd, int nsrc,
                              const lq_opts* o, lq_report* rep, void* stream) {
    if (!c || !dir || !x || !ys || !yd) return set_err(c, LQ_ERR_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    int r = sign_derivative_core(c, dir, x, nsrc, o, rep, st);
    if (r) return r;
    const size_t reg = (size_t)c->nsrc * c->V * 24, n = (size_t)nsrc * c->V * 24;
    if ((r = stage_out(c, yd, c->io + reg, n, st))) return r;
    if ((r = stage_out(c, ys, c->io + 2 * reg, n, st))) return r;
    LQ_CUDA(c, cudaStreamSynchronize(st));
    return LQ_OK;
}

int lq_overlap_apply(lq_ctx* c, const lq_direction* dir, const double* x, double* y, double* dy, int nsrc,
                     const lq_opts* o, lq_report* rep, void* stream) {
    if (!c || !x || !y || (dy && !dir)) return set_err(c, LQ_ERR_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    int r = check_ready(c, nsrc, dy ? 1 : 0);
    if (r) return r;
    const size_t reg = (size_t)c->nsrc * c->V * 24, n = (size_t)nsrc * c->V * 24;
    double* xk = c->io + 5 * reg;   // the undeflated source, kept for the "1" of Eq. (1.1)
    if ((r = stage_in(c, xk, x, n, st))) return r;
    if (dy) {
        if ((r = sign_derivative_core(c, dir, xk, nsrc, o, rep, st))) return r;
        LQ_CUDA(c, launch_overlap(xk, c->io + 2 * reg, c->io + reg, (size_t)nsrc * c->V, st));
        c->launches += 1;
        if ((r = stage_out(c, dy, c->io + reg, n, st))) return r;
        if ((r = stage_out(c, y, c->io + 2 * reg, n, st))) return r;
    } else {
        if ((r = sign_core(c, xk, nsrc, o, rep, st))) return r;
        LQ_CUDA(c, launch_overlap(xk, c->io + reg, nullptr, (size_t)nsrc * c->V, st));
        c->launches += 1;
        if ((r = stage_out(c, y, c->io + reg, n, st))) return r;
    }
    LQ_CUDA(c, cudaStreamSynchronize(st));
    return LQ_OK;
}

int lq_batch_apply(const lq_batch_item* items, int n, void* stream) {
    if (!items || n < 1 || n > LQ_BATCH_MAX) return LQ_ERR_ARG;
    lq_ctx* c0 = items[0].ctx;
    if (!c0) return LQ_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        const lq_batch_item& it = items[i];
        lq_ctx* c = it.ctx;
        if (!c) return set_err(c0, LQ_ERR_ARG, "batch member " + std::to_string(i) + ": null context");
        for (int j = 0; j < i; ++j)
            if (items[j].ctx == c) return set_err(c, LQ_ERR_ARG, "a context appears twice in the batch");
        if (c->device != c0->device) return set_err(c, LQ_ERR_ARG, "batch members on different devices");
        if (!it.x || !it.y_sign || (it.dir && !it.y_deriv)) return set_err(c, LQ_ERR_ARG, "null argument");
        int r = check_ready(c, it.nsrc, it.dir ? 1 : 0);
        if (r || (r = check_opts(c, it.opts))) return r;
        if (it.opts->two_pass) return set_err(c, LQ_ERR_ARG, "two-pass runs are not batched");
        if (it.opts->rebiorth > 0) return set_err(c, LQ_ERR_ARG, "re-biorthogonalised runs are not batched");
        if (!ensure_cap_stream(c)) return set_err(c, LQ_ERR_CUDA, "cannot create the member's stream");
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<TslRun> runs((size_t)n);
    std::vector<cudaStream_t> br((size_t)n);
    int r = LQ_OK;
    // direction, source and start vectors of every member on st (and its schedule, tuned there
    // on first use)
    for (int i = 0; i < n; ++i) {
        const lq_batch_item& it = items[i];
        lq_ctx* c = it.ctx;
        const size_t reg = (size_t)c->nsrc * c->V * 24;
        if (it.dir && (r = lq_set_direction(c, it.dir, st))) return r;
        if ((r = stage_in(c, c->io, it.x, (size_t)it.nsrc * c->V * 24, st))) return r;
        TslRun& t = runs[(size_t)i];
        t.c = c; t.nsrc = it.nsrc; t.o = it.opts; t.rep = it.report;
        t.nf = it.dir ? 2 : 1;
        t.emode = it.dir ? emode_of(c) : 0;
        t.y0 = c->io + reg;
        t.y1 = it.dir ? c->io + 2 * reg : nullptr;
        if ((r = t.setup(st, c->io, nullptr))) return r;
        br[(size_t)i] = c->cap_stream;
    }
    bool graphed = true;
    for (auto& t : runs) graphed = graphed && t.graphed();
    if ((r = graphed ? batch_lanczos_graph(runs, st) : batch_lanczos_plain(runs, st))) return r;
    // projected signs, recombinations and outputs on the members' branches
    if ((r = fork_streams(c0, st, br))) return r;
    for (int i = 0; i < n && !r; ++i) r = runs[(size_t)i].proj_enqueue(br[(size_t)i]);
    for (int i = 0; i < n && !r; ++i) r = runs[(size_t)i].proj_complete(br[(size_t)i]);
    for (int i = 0; i < n && !r; ++i) r = runs[(size_t)i].finish_enqueue(br[(size_t)i]);
    for (int i = 0; i < n && !r; ++i) {
        const lq_batch_item& it = items[i];
        lq_ctx* c = it.ctx;
        const size_t reg = (size_t)c->nsrc * c->V * 24, cnt = (size_t)it.nsrc * c->V * 24;
        if (it.dir) {
            if ((r = stage_out(c, it.y_deriv, c->io + reg, cnt, br[(size_t)i]))) break;
            r = stage_out(c, it.y_sign, c->io + 2 * reg, cnt, br[(size_t)i]);
        } else {
            r = stage_out(c, it.y_sign, c->io + reg, cnt, br[(size_t)i]);
        }
    }
    for (int i = 0; i < n && !r; ++i) r = runs[(size_t)i].finish_complete(br[(size_t)i]);
    const int rj = join_streams(c0, br, st);
    if (r || (r = rj)) return r;
    LQ_CUDA(c0, cudaStreamSynchronize(st));
    return LQ_OK;
}

int lq_overlap_solve(lq_ctx* c, const double* b, double* z, int nsrc, double mass, double tol, int max_iter,
                     const lq_opts* o, lq_solve_report* rep, void* stream) {
    if (!c || !b || !z) return set_err(c, LQ_ERR_ARG, "null argument");
    int r = solve_ready(c, nsrc, 0, mass, tol, max_iter, o);
    if (r) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t reg = (size_t)c->nsrc * nvec(c), n = (size_t)nsrc * nvec(c);
    double* B = c->solve_ws + 6 * reg;
    double* Z = c->solve_ws + 7 * reg;
    if ((r = stage_in(c, B, b, n, st))) return r;
    if ((r = overlap_bicgstab(c, B, Z, nsrc, mass, tol, max_iter, o, rep, st))) return r;
    if ((r = stage_out(c, z, Z, n, st))) return r;
    LQ_CUDA(c, cudaStreamSynchronize(st));
    return LQ_OK;
}

int lq_axial_current(lq_ctx* c, const lq_direction* dir, const double* eta, int nsrc, double mass, double tol,
                     int max_iter, const lq_opts* o, double* out, lq_solve_report* rep, void* stream) {
    if (!c || !dir || !eta || !out) return set_err(c, LQ_ERR_ARG, "null argument");
    int r = solve_ready(c, nsrc, 1, mass, tol, max_iter, o);
    if (r) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t reg = (size_t)c->nsrc * nvec(c), n = (size_t)nsrc * nvec(c);
    double* B = c->solve_ws + 6 * reg;
    double* Z = c->solve_ws + 7 * reg;
    double* E = c->solve_ws + 8 * reg;
    double* A = c->solve_ws + 2 * reg;   // gamma5 eta (the recurrence vectors are not in use yet)
    if ((r = stage_in(c, E, eta, n, st))) return r;
    LQ_CUDA(c, launch_g5axpy(A, nullptr, 0.0, E, 1.0, (size_t)nsrc * c->V, st));
    std::vector<lq_report> drep(nsrc);
    if ((r = sign_derivative_core(c, dir, A, nsrc, o, drep.data(), st))) return r;
    // B = dD(m) gamma5 eta = (1 - m/2) gamma5 d sgn(H) gamma5 eta (the derivative is staging region 1)
    LQ_CUDA(c, launch_g5axpy(B, nullptr, 0.0, c->io + reg, 1.0 - 0.5 * mass, (size_t)nsrc * c->V, st));
    c->launches += 2;
    if ((r = overlap_bicgstab(c, B, Z, nsrc, mass, tol, max_iter, o, rep, st))) return r;
    std::vector<cplx> j;
    if ((r = sdots_host(c, E, Z, nsrc, j, st))) return r;
    for (int s = 0; s < nsrc; ++s) {
        out[2 * s] = j[s].real();
        out[2 * s + 1] = j[s].imag();
        if (rep && drep[s].status < 0 && rep[s].status == LQ_OK) rep[s].status = drep[s].status;
    }
    return LQ_OK;
}

int lq_profile_enable(lq_ctx* c, int enable) {
    if (!c) return LQ_ERR_ARG;
    c->prof_on = enable ? 1 : 0;
    c->launches = 0;
    for (int i = 0; i < 4; ++i) { c->prof_ms[i] = 0.0; c->prof_n[i] = 0; }
    c->pending.clear();
    c->ev_used = 0;
    return LQ_OK;
}

int lq_profile_read(lq_ctx* c, lq_profile* o) {
    if (!c || !o) return set_err(c, LQ_ERR_ARG, "null argument");
    std::memset(o, 0, sizeof(*o));
    o->enabled = c->prof_on;
    o->launches = c->launches;
    o->hop_ms = c->prof_ms[PC_HOP];
    o->hop_launches = c->prof_n[PC_HOP];
    o->update_ms = c->prof_ms[PC_UPDATE];
    o->update_launches = c->prof_n[PC_UPDATE];
    o->newton_ms = c->prof_ms[PC_NEWTON];
    o->newton_iterations = c->prof_n[PC_NEWTON];
    o->other_ms = c->prof_ms[PC_OTHER];
    o->other_launches = c->prof_n[PC_OTHER];
    return LQ_OK;
}

int lq_upload_deflation(lq_ctx* c, int l, const double* lambda, const double* R, const double* L, void* stream) {
    if (c) { ++c->defl_version; c->defl_prep_ok = false; }
    if (!c || l < 0) return set_err(c, LQ_ERR_ARG, "invalid deflation arguments");
    if (l == 0) { c->defl_l = 0; return LQ_OK; }
    if (!lambda || !R || !L) return set_err(c, LQ_ERR_ARG, "null deflation data");
    if (!c->basis) return set_err(c, LQ_ERR_NOT_READY, "workspace not reserved (lq_reserve)");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nv = nvec(c);
    int r;
    if (l > c->defl_cap) {
        if ((r = dalloc(c, &c->defl_V, (size_t)2 * l * nv))) return r;
        if ((r = dalloc(c, &c->defl_W, (size_t)2 * l * nv))) return r;
        if ((r = dalloc(c, &c->defl_work, (size_t)6 * l * nv))) return r;
        c->defl_scr_doubles = std::max(bdots_partial_doubles(l * std::max(l, c->nsrc) * 2) + (size_t)8 * l * std::max(l, c->nsrc),
                                       (size_t)2 * 2 * l * std::max(l, c->nsrc));
        if ((r = dalloc(c, &c->defl_scr, c->defl_scr_doubles))) return r;
        if ((r = dalloc(c, &c->defl_shift, (size_t)std::max(c->nsrc, l)))) return r;
        c->defl_cap = l;
    }
    if ((r = stage_in(c, c->defl_V, R, (size_t)l * nv, st))) return r;
    if ((r = stage_in(c, c->defl_W, L, (size_t)l * nv, st))) return r;
    LQ_CUDA(c, cudaMemsetAsync(c->defl_V + (size_t)l * nv, 0, sizeof(double) * l * nv, st));
    LQ_CUDA(c, cudaMemsetAsync(c->defl_W + (size_t)l * nv, 0, sizeof(double) * l * nv, st));
    c->defl_lam.resize(l);
    for (int i = 0; i < l; ++i) c->defl_lam[i] = make_double2(lambda[2 * i], lambda[2 * i + 1]);
    c->defl_dlam.assign(l, make_double2(0.0, 0.0));
    c->defl_l = l;
    LQ_CUDA(c, cudaStreamSynchronize(st));
    return LQ_OK;
}

int lq_compute_deflation(lq_ctx* c, const lq_eig_opts* eo_in, const double* X0, double* lambda, double* resid, void* stream) {
    if (c) { ++c->defl_version; c->defl_prep_ok = false; }
    if (!c || !eo_in || !X0) return set_err(c, LQ_ERR_ARG, "null argument");
    lq_eig_opts eo = *eo_in;
    const bool si = eo.method == LQ_EIG_SHIFT_INVERT;
    if (eo.method != LQ_EIG_SHIFT_INVERT && eo.method != LQ_EIG_CHEBYSHEV) return set_err(c, LQ_ERR_ARG, "unknown eigensolver method");
    if (eo.nsub <= 0) eo.nsub = si ? std::min(2 * eo.nev + 10, 63) : std::min(eo.nev + 12, 64);
    if (eo.degree <= 0) eo.degree = 40;
    if (eo.max_iter <= 0) eo.max_iter = si ? 300 : 60;
    if (!(eo.tol > 0.0)) eo.tol = 1e-10;
    if (si) {
        if (eo.nev < 1 || eo.nsub < eo.nev + 4 || eo.nsub > 63) return set_err(c, LQ_ERR_ARG, "need 1 <= nev and nev + 4 <= nsub <= 63");
    } else if (eo.nev < 1 || eo.nsub < eo.nev + 2 || eo.nsub > 64) {
        return set_err(c, LQ_ERR_ARG, "need 1 <= nev and nev + 2 <= nsub <= 64");
    }
    int r = check_ready(c, 1, 0);
    if (r) return r;
    if ((size_t)(eo.nsub + 1) * (eo.nsub + 1) > (size_t)std::max(2 * c->nsrc, 64) * std::max(2 * c->nsrc, 64))
        return set_err(c, LQ_ERR_ARG, "nsub too large for the reserved reduction scratch");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nv = nvec(c);
    const int m = eo.nsub, nev = eo.nev;
    c->eig_stats = lq_eig_stats();
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (cudaEventCreate(&t0) == cudaSuccess && cudaEventCreate(&t1) == cudaSuccess) cudaEventRecord(t0, st);
    else cudaGetLastError();
    // workspace (a set-up call): Chebyshev: X, Y0, Y1, H1, H2 | ZR, ZL | X0 copy (m fields each);
    // shift-and-invert: basis [2][m+1] | restart scratch [2][kk+1] + [4] | Ritz vectors [2][nev] |
    // residuals [4] | start fields [2] | the FP32 CG vectors and scalars
    const int kk_max = m;   // bound on the vectors kept at a restart
    const size_t doubles = si ? nv * ((size_t)2 * (m + 1) + 2 * (kk_max + 1) + 4 + 2 * nev + 4 + 2) : nv * (size_t)m * 8;
    const size_t cg_bytes = si ? sizeof(float4) * 5 * 2 * (size_t)c->V * 6 + sizeof(double) * (2 * kCgNs + cg_partial_doubles(2) + 2) + sizeof(int) * 8 : 0;
    char* W = nullptr;
    if (cudaMalloc(&W, sizeof(double) * doubles + cg_bytes + 256) != cudaSuccess) { cudaGetLastError(); return set_err(c, LQ_ERR_OOM, "eigensolver workspace"); }
    // the eigensolver's FP64 stencil: a mixed-precision context gets a temporary FP64 copy of the
    // links; its FP32 stencil (shift-and-invert inner solves): an FP64 context gets an FP32 copy
    void* U64 = nullptr;
    void* U32 = nullptr;
    auto fail = [&](int code) { cudaFree(W); if (U64) cudaFree(U64); if (U32) cudaFree(U32); if (t0) cudaEventDestroy(t0); if (t1) cudaEventDestroy(t1); return code; };
    if (c->prec != LQ_FP64) {
        if (cudaMalloc(&U64, sizeof(double2) * c->V * 36) != cudaSuccess) { cudaGetLastError(); U64 = nullptr; return fail(set_err(c, LQ_ERR_OOM, "eigensolver links")); }
        cudaError_t e = launch_links_internal(LQ_FP64, c->Ub, U64, c->V, st);
        if (e != cudaSuccess) return fail(set_err(c, LQ_ERR_CUDA, cudaGetErrorString(e)));
    }
    if (si && (c->prec != LQ_MIXED || c->link_bf16)) {   // FP32 links for the inner solves
        if (cudaMalloc(&U32, sizeof(float2) * c->V * 36) != cudaSuccess) { cudaGetLastError(); U32 = nullptr; return fail(set_err(c, LQ_ERR_OOM, "eigensolver links")); }
        cudaError_t e = launch_links_internal(LQ_MIXED, c->Ub, U32, c->V, st);
        if (e != cudaSuccess) return fail(set_err(c, LQ_ERR_CUDA, cudaGetErrorString(e)));
    }
    const void* links64 = U64 ? U64 : c->U;
    const void* links32 = U32 ? U32 : c->U;
    double* Wd = reinterpret_cast<double*>(W);
    std::vector<cplx> thR, thL;
    std::vector<double> resR, resL;
    double* ZR = nullptr;
    double* ZL = nullptr;
    int ncand = m;       // left candidates for the pairing
    if (!si) {
        ZR = Wd + (size_t)5 * m * nv;
        ZL = ZR + (size_t)m * nv;
        double* X0d = ZL + (size_t)m * nv;
        if ((r = stage_in(c, X0d, X0, nv * m, st))) return fail(r);
        if ((r = eig_subspace(c, &eo, X0d, 0, Wd, thR, resR, ZR, st, links64))) return fail(r);
        if ((r = eig_subspace(c, &eo, X0d, 1, Wd, thL, resL, ZL, st, links64))) return fail(r);
    } else {
        double* Vb = Wd;
        double* Zs = Vb + (size_t)2 * (m + 1) * nv;
        double* Z = Zs + ((size_t)2 * (kk_max + 1) + 4) * nv;
        double* R4 = Z + (size_t)2 * nev * nv;
        double* X0d = R4 + (size_t)4 * nv;
        char* g = reinterpret_cast<char*>(X0d + 2 * nv);
        SiWork w;
        w.c = c; w.st = st; w.V = c->V; w.ne = (size_t)6 * c->V; w.nv = nv;
        w.links32 = links32; w.links64 = links64;
        float4* f = reinterpret_cast<float4*>(g);
        w.x = f; w.r = f + 2 * w.ne; w.p = f + 4 * w.ne; w.q = f + 6 * w.ne; w.z = f + 8 * w.ne;
        double* dd = reinterpret_cast<double*>(f + 10 * w.ne);
        w.scal = dd; w.part = dd + 2 * kCgNs; w.nrm = w.part + cg_partial_doubles(2);
        w.counters = reinterpret_cast<int*>(w.nrm + 2);
        w.res64 = R4; w.tmp64 = R4 + 2 * nv;
        if (eo.inner_max > 0) w.inner_max = eo.inner_max;
        LQ_CUDA(c, cudaMemsetAsync(w.counters, 0, sizeof(int) * 8, st));
        if ((r = stage_in(c, X0d, X0, nv * 2, st))) return fail(r);
        // ||H|| estimate (power iteration with H^dag H on the first start field): the residual scale
        double hn = 0.0;
        {
            double* y = R4;
            double* t = R4 + nv;
            LQ_CUDA(c, cudaMemcpyAsync(y, X0d, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
            for (int it = 0; it < 12; ++it) {
                std::vector<double2> n0, n1;
                if ((r = bdots_host(c, y, 1, y, 1, n0, st))) return fail(r);
                if ((r = apply_H_batch(c, y, t, 1, 0, st, LQ_FP64, links64))) return fail(r);
                if ((r = apply_H_batch(c, t, y, 1, 1, st, LQ_FP64, links64))) return fail(r);
                if ((r = bdots_host(c, y, 1, y, 1, n1, st))) return fail(r);
                hn = std::sqrt(std::sqrt(n1[0].x / n0[0].x));
                std::vector<double2> sc(1, make_double2(1.0 / std::sqrt(n1[0].x), 0.0));
                if ((r = bcombine_host(c, t, nullptr, 1, y, 1, sc, st))) return fail(r);
                LQ_CUDA(c, cudaMemcpyAsync(y, t, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
            }
            hn *= 1.05;
        }
        SiResult res;
        if ((r = eig_shift_invert(w, eo, X0d, Vb, Zs, Z, hn, res))) return fail(r);
        thR = res.lam[0]; thL = res.lam[1];
        resR = res.res[0]; resL = res.res[1];
        ZR = Z; ZL = Z + (size_t)nev * nv;
        ncand = nev;
        c->eig_stats.restarts = res.restarts;
        c->eig_stats.solves = w.solves;
        c->eig_stats.inner_iterations = w.iters;
        c->eig_stats.refinements = w.refinements;
        c->eig_stats.norm_estimate = hn;
    }
    // pair right eigenvalue lambda_i with the left eigenvalue conj(theta_j) closest to it
    std::vector<int> pick(nev, -1);
    std::vector<char> used(ncand, 0);
    for (int i = 0; i < nev; ++i) {
        double best = 1e300;
        for (int j = 0; j < ncand; ++j) {
            if (used[j]) continue;
            const double d = std::abs(thR[i] - std::conj(thL[j]));
            if (d < best) { best = d; pick[i] = j; }
        }
        used[pick[i]] = 1;
        c->eig_stats.pair_mismatch = std::max(c->eig_stats.pair_mismatch, best / std::max(std::abs(thR[i]), 1e-300));
    }
    // install: defl_V = R (first nev right Ritz vectors), defl_W = the paired left vectors
    if (nev > c->defl_cap) {
        if ((r = dalloc(c, &c->defl_V, (size_t)2 * nev * nv))) return fail(r);
        if ((r = dalloc(c, &c->defl_W, (size_t)2 * nev * nv))) return fail(r);
        if ((r = dalloc(c, &c->defl_work, (size_t)6 * nev * nv))) return fail(r);
        c->defl_scr_doubles = std::max(bdots_partial_doubles(nev * std::max(nev, c->nsrc) * 2) + (size_t)8 * nev * std::max(nev, c->nsrc),
                                       (size_t)2 * 2 * nev * std::max(nev, c->nsrc));
        if ((r = dalloc(c, &c->defl_scr, c->defl_scr_doubles))) return fail(r);
        if ((r = dalloc(c, &c->defl_shift, (size_t)std::max(c->nsrc, nev)))) return fail(r);
        c->defl_cap = nev;
    }
    LQ_CUDA(c, cudaMemcpyAsync(c->defl_V, ZR, sizeof(double) * nv * nev, cudaMemcpyDeviceToDevice, st));
    for (int i = 0; i < nev; ++i)
        LQ_CUDA(c, cudaMemcpyAsync(c->defl_W + (size_t)i * nv, ZL + (size_t)pick[i] * nv, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
    // biorthonormalise: Lk <- Lk G^{-H} with G = Lk^H R
    std::vector<double2> G;
    if ((r = bdots_host(c, c->defl_W, nev, c->defl_V, nev, G, st))) return fail(r);
    std::vector<cplx> Gi(nev * nev);
    for (int i = 0; i < nev * nev; ++i) Gi[i] = cplx(G[i].x, G[i].y);
    if (dense_inverse(nev, Gi.data()) != LQ_OK) return fail(set_err(c, LQ_ERR_BREAKDOWN, "left and right eigenvectors are not biorthogonal"));
    std::vector<double2> coef(nev * nev);
    for (int j = 0; j < nev; ++j) for (int i = 0; i < nev; ++i) coef[j * nev + i] = make_double2(Gi[j * nev + i].real(), -Gi[j * nev + i].imag());
    if ((r = bcombine_host(c, ZL, nullptr, nev, c->defl_W, nev, coef, st))) return fail(r);
    LQ_CUDA(c, cudaMemcpyAsync(c->defl_W, ZL, sizeof(double) * nv * nev, cudaMemcpyDeviceToDevice, st));
    LQ_CUDA(c, cudaMemsetAsync(c->defl_V + (size_t)nev * nv, 0, sizeof(double) * nev * nv, st));
    LQ_CUDA(c, cudaMemsetAsync(c->defl_W + (size_t)nev * nv, 0, sizeof(double) * nev * nv, st));
    LQ_CUDA(c, cudaStreamSynchronize(st));
    c->defl_lam.resize(nev);
    for (int i = 0; i < nev; ++i) c->defl_lam[i] = make_double2(thR[i].real(), thR[i].imag());
    c->defl_dlam.assign(nev, make_double2(0.0, 0.0));
    c->defl_l = nev;
    if (lambda) for (int i = 0; i < nev; ++i) { lambda[2 * i] = thR[i].real(); lambda[2 * i + 1] = thR[i].imag(); }
    for (int i = 0; i < nev; ++i) c->eig_stats.max_residual = std::max(c->eig_stats.max_residual, std::max(resR[i], resL[pick[i]]));
    if (resid) for (int i = 0; i < nev; ++i) resid[i] = std::max(resR[i], resL[pick[i]]);
    if (t0 && t1) {
        cudaEventRecord(t1, st);
        cudaEventSynchronize(t1);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess) c->eig_stats.seconds = ms * 1e-3;
        else cudaGetLastError();
    }
    c->eig_stats.method = eo.method;
    return fail(LQ_OK);
}

int lq_eig_stats_read(const lq_ctx* c, lq_eig_stats* out) {
    if (!c || !out) return LQ_ERR_ARG;
    *out = c->eig_stats;
    return LQ_OK;
}

int lq_deflation_derivatives(lq_ctx* c, const lq_direction* dir, const lq_opts* o, double* dlambda, double* dR,
                             double* dL, void* stream) {
    if (c) c->defl_prep_ok = false;   // the derivatives below are along its own direction
    if (!c || !dir) return set_err(c, LQ_ERR_ARG, "null argument");
    if (c->defl_l <= 0) return set_err(c, LQ_ERR_NOT_READY, "no deflation space uploaded");
    int r = check_ready(c, 1, 1);
    if (r || (r = check_opts(c, o, true))) return r;
    cudaStream_t st = (cudaStream_t)stream;
    if ((r = lq_set_direction(c, dir, stream))) return r;
    if ((r = prepare_deflation_derivative(c, o, st))) return r;
    const int l = c->defl_l;
    if (dlambda) for (int i = 0; i < l; ++i) { dlambda[2 * i] = c->defl_dlam[i].x; dlambda[2 * i + 1] = c->defl_dlam[i].y; }
    if (dR && (r = stage_out(c, dR, c->defl_V + (size_t)l * nvec(c), (size_t)l * nvec(c), st))) return r;
    if (dL && (r = stage_out(c, dL, c->defl_W + (size_t)l * nvec(c), (size_t)l * nvec(c), st))) return r;
    LQ_CUDA(c, cudaStreamSynchronize(st));
    return LQ_OK;
}

int lq_sign_bilinear_grad(lq_ctx* c, const double* x, const double* y, const lq_opts* o, double* S, double* force,
                          double* dS_dmu, void* stream) {
    if (!c || !x || !y) return set_err(c, LQ_ERR_ARG, "null argument");
    if (!c->adjoint) return set_err(c, LQ_ERR_NOT_READY, "workspace reserved without LQ_RESERVE_ADJOINT");
    int r = check_ready(c, 2, 0);
    if (r || (r = check_opts(c, o, true))) return r;
    if (o->rebiorth > 0) return set_err(c, LQ_ERR_ARG, "re-biorthogonalisation is not available for the adjoint");
    const int l = o->deflate ? c->defl_l : 0;
    const bool two = o->two_pass != 0 && o->kmax > 1;
    if (two && l > 0) return set_err(c, LQ_ERR_ARG, "the two-pass adjoint runs without deflation");
    if (l > 0 && 2 * o->quad_nodes + 3 * l > 2 * kQuadMaxNodes)
        return set_err(c, LQ_ERR_ARG, "deflated adjoint: 2 quad_nodes + 3 l must not exceed " + std::to_string(2 * kQuadMaxNodes));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nv = nvec(c);
    const size_t reg = (size_t)c->nsrc * nv;
    double* io0 = c->io;            // sources: 0 = x, 1 = y (deflated: x' = Pbar x, y' = Pbar^H y)
    double* io1 = c->io + reg;      // results: 0 = sgn(H) x'
    double* io2 = c->io + 2 * reg;  // the caller's x and y
    if ((r = stage_in(c, io2, x, nv, st))) return r;
    if ((r = stage_in(c, io2 + nv, y, nv, st))) return r;
    LQ_CUDA(c, cudaMemcpyAsync(io0, io2, sizeof(double) * 2 * nv, cudaMemcpyDeviceToDevice, st));
    // deflation (Sec. 3): c_j = <Lk_j|x>, d_j = y^H R_j = conj(<R_j|y>); x' = x - sum_j R_j c_j,
    // y' = y - sum_j Lk_j <R_j|y>
    std::vector<double2> cx, ry;
    if (l > 0) {
        if ((r = bdots_host(c, c->defl_W, l, io2, 1, cx, st))) return r;
        if ((r = bdots_host(c, c->defl_V, l, io2 + nv, 1, ry, st))) return r;
        std::vector<double2> m1(l), m2(l);
        for (int j = 0; j < l; ++j) { m1[j] = make_double2(-cx[j].x, -cx[j].y); m2[j] = make_double2(-ry[j].x, -ry[j].y); }
        if ((r = bcombine_host(c, io0, io0, 1, c->defl_V, l, m1, st))) return r;
        if ((r = bcombine_host(c, io0 + nv, io0 + nv, 1, c->defl_W, l, m2, st))) return r;
    }
    lq_opts so = *o;
    if (so.projected == LQ_PROJ_NEWTON) so.projected = LQ_PROJ_AUTO;   // the adjoint uses the quadrature
    std::vector<lq_report> rep(2);
    const size_t F = fe(c);
    // right basis of source 0 (x) and stored left basis of source 1 (y): full, or rings of a
    // two-pass workspace
    const size_t lslots = (size_t)(c->ring > 0 ? c->ring : c->kmax);
    const void* lb1 = reinterpret_cast<const char*>(c->lbasis) + lslots * F * chunk_bytes(c);
    double cscale = 1.0;
    AdjArgs a;
    auto make_adj = [&]() {
        std::memset(&a, 0, sizeof(a));
        a.npairs = 2 * o->quad_nodes;
        a.kmax = c->kmax;
        a.nth_max = 2 * kQuadMaxNodes;
        a.c = cscale;
        a.state = c->state;
        a.alpha = c->alpha; a.beta = c->beta; a.delta = c->delta;
        a.scale = c->scale; a.uscale = c->uscale;
        a.work = c->quad_work;
        a.cnu = c->adj_coef;
        a.com = c->adj_coef + (size_t)2 * kQuadMaxNodes * c->kmax;
        a.nu = c->adj_nu; a.om = c->adj_om;
        a.V = c->V;
        for (int i = 0; i < 4; ++i) a.dims[i] = c->dims[i];
        a.strides[0] = 1;
        a.strides[1] = (size_t)c->dims[0];
        a.strides[2] = (size_t)c->dims[0] * c->dims[1];
        a.strides[3] = (size_t)c->dims[0] * c->dims[1] * c->dims[2];
        a.apbc = c->desc.t_antiperiodic ? 1 : 0;
        a.efwd = std::exp(c->desc.mu);
        a.ebwd = std::exp(-c->desc.mu);
        a.Ub = reinterpret_cast<const double2*>(c->Ub);
        a.force = c->adj_force;
        a.dmu_part = c->adj_dmu;
    };
    if (!two) {
        if ((r = run_tsl(c, 1, 0, 2, &so, rep.data(), io1, nullptr, st, io0, nullptr, FN_SIGN, nullptr, true))) return r;
        LQ_CUDA(c, cudaMemcpy(&cscale, c->quad_c, sizeof(double), cudaMemcpyDeviceToHost));
        make_adj();
    } else {
        // two-pass adjoint: the first pass (rings only) yields T_1, T_2 and the projected sign; the
        // pair coefficients follow from them; the second pass reruns both processes and, window by
        // window, recombines sgn(H) x' and accumulates the 2N pair vectors from the rings
        so.two_pass = 1;
        TslRun t;
        t.c = c; t.nf = 1; t.emode = 0; t.nsrc = 2; t.o = &so; t.rep = rep.data();
        t.y0 = io1; t.y1 = nullptr; t.fn = FN_SIGN; t.store_left = true;
        if ((r = t.setup(st, io0, nullptr)) || (r = t.lanczos(false, st))) return r;
        if ((r = t.proj_enqueue(st)) || (r = t.proj_complete(st))) return r;
        LQ_CUDA(c, cudaMemcpy(&cscale, c->quad_c, sizeof(double), cudaMemcpyDeviceToHost));
        make_adj();
        LQ_CUDA(c, launch_adj_pairs(a, st));
        c->launches += 1;
        const int ring = t.ring;
        t.on_window = [&](int j0, int j1, cudaStream_t ls) -> int {
            cudaError_t e = launch_adj_window(c->prec, a, c->basis, F, lb1, F, j0, j1, ring, ls);
            c->launches += 2;
            return e == cudaSuccess ? LQ_OK : set_err(c, LQ_ERR_CUDA, cudaGetErrorString(e));
        };
        if ((r = t.finish_enqueue(st)) || (r = t.finish_complete(st))) return r;
    }
    for (int s = 0; s < 2; ++s)
        if (rep[s].status != LQ_OK) return set_err(c, rep[s].status, "Lanczos process failed for the bilinear");
    // S = Re <y | sgn(H) x'> (+ Re sum_j sgn(lambda_j) c_j d_j with deflation)
    std::vector<double2> d;
    if ((r = bdots_host(c, io2 + nv, 1, io1, 1, d, st))) return r;
    double Sdefl = 0.0;
    for (int j = 0; j < l; ++j) {
        const cplx cj(cx[j].x, cx[j].y), dj(ry[j].x, -ry[j].y);
        Sdefl += sgn_re(c->defl_lam[j]) * (cj * dj).real();
    }
    const int k = o->kmax;
    if (l > 0) {
        // the 3 l deflation pairs after the 2N Krylov pairs, from the four-block split of G by the
        // spectral projectors (lq_adjoint.cu, k_defl_coef): (R_i, b_i) with b_i = sum_j conj(F_ij c_i
        // d_j) Lk_j and the divided differences F_ij = (sgn l_i - sgn l_j) / (l_i - l_j) (the
        // deflated block); (R_i, conj(c_i) u_i) and (d_j v_j, Lk_j) (the two mixed blocks)
        const int nq = a.npairs;
        std::vector<double2> bc((size_t)l * l);
        for (int i = 0; i < l; ++i)
            for (int j = 0; j < l; ++j) {
                const cplx li(c->defl_lam[i].x, c->defl_lam[i].y), lj(c->defl_lam[j].x, c->defl_lam[j].y);
                const double si = sgn_re(c->defl_lam[i]), sj = sgn_re(c->defl_lam[j]);
                const cplx F_ij = si != sj ? cplx(si - sj) / (li - lj) : cplx(0.0);
                const cplx m = std::conj(F_ij * cplx(cx[i].x, cx[i].y) * cplx(ry[j].x, -ry[j].y));
                bc[(size_t)i * l + j] = make_double2(m.real(), m.imag());
            }
        double* bvec = c->defl_work;   // l FP64 fields
        if ((r = bcombine_host(c, bvec, nullptr, l, c->defl_W, l, bc, st))) return r;
        const size_t fbytes = fb(c);
        auto slot = [&](void* base, int q) { return reinterpret_cast<char*>(base) + (size_t)q * fbytes; };
        LQ_CUDA(c, launch_to_internal(c->prec, c->defl_V, slot(c->adj_nu, nq), c->V, l, st));
        LQ_CUDA(c, launch_to_internal(c->prec, bvec, slot(c->adj_om, nq), c->V, l, st));
        LQ_CUDA(c, launch_to_internal(c->prec, c->defl_V, slot(c->adj_nu, nq + l), c->V, l, st));
        LQ_CUDA(c, launch_to_internal(c->prec, c->defl_W, slot(c->adj_om, nq + 2 * l), c->V, l, st));
        c->launches += 4;
        std::vector<double2> small((size_t)3 * l);
        for (int j = 0; j < l; ++j) {
            small[j] = c->defl_lam[j];
            small[(size_t)l + j] = cx[j];
            small[(size_t)2 * l + j] = make_double2(ry[j].x, -ry[j].y);
        }
        double2* dsmall = reinterpret_cast<double2*>(c->gen_scr + c->gen_scr_doubles) - 3 * (size_t)l;
        LQ_CUDA(c, cudaMemcpyAsync(dsmall, small.data(), sizeof(double2) * small.size(), cudaMemcpyHostToDevice, st));
        a.ndefl = l;
        a.npairs_force = nq + 3 * l;
        a.dlam = dsmall;
        a.dcx = dsmall + l;
        a.ddy = dsmall + 2 * l;
    }
    if (!two) {
        LQ_CUDA(c, launch_adjoint(c->prec, a, c->basis, F, lb1, F, std::max(k, 1), st));
        c->launches += 4;
    } else {
        LQ_CUDA(c, launch_adj_force(c->prec, a, st));
        c->launches += 1;
    }
    const size_t nblk = (c->V + 127) / 128;
    std::vector<double> dmu(nblk);
    LQ_CUDA(c, cudaMemcpyAsync(dmu.data(), c->adj_dmu, sizeof(double) * nblk, cudaMemcpyDeviceToHost, st));
    if (force && (r = stage_out(c, force, c->adj_force, c->V * 32, st))) return r;
    LQ_CUDA(c, cudaStreamSynchronize(st));
    if (S) *S = d[0].x + Sdefl;
    if (dS_dmu) { double t = 0.0; for (double v : dmu) t += v; *dS_dmu = t; }
    return LQ_OK;
}

int lq_tsl_coefficients(lq_ctx* c, int src, int k, double* alpha, double* beta, double* delta) {
    if (!c || !alpha || !beta || !delta) return set_err(c, LQ_ERR_ARG, "null argument");
    if (!c->alpha) return set_err(c, LQ_ERR_NOT_READY, "workspace not reserved (lq_reserve)");
    if (src < 0 || src >= c->nsrc || k < 1 || k > c->kmax) return set_err(c, LQ_ERR_ARG, "src / k outside the reserved workspace");
    TslState st;
    LQ_CUDA(c, cudaMemcpy(&st, c->state + src, sizeof(st), cudaMemcpyDeviceToHost));
    LQ_CUDA(c, cudaMemcpy(alpha, c->alpha + (size_t)src * c->kmax, sizeof(double2) * k, cudaMemcpyDeviceToHost));
    LQ_CUDA(c, cudaMemcpy(beta, c->beta + (size_t)src * c->kmax, sizeof(double2) * k, cudaMemcpyDeviceToHost));
    LQ_CUDA(c, cudaMemcpy(delta, c->delta + (size_t)src * c->kmax, sizeof(double) * k, cudaMemcpyDeviceToHost));
    for (int j = 0; j < k; ++j) {
        if (j >= st.k_eff) { alpha[2 * j] = alpha[2 * j + 1] = 0.0; }
        if (j >= st.k_eff - 1) { beta[2 * j] = beta[2 * j + 1] = 0.0; delta[j] = 0.0; }
    }
    return LQ_OK;
}

int lq_error_estimate(lq_ctx* c, const lq_direction* dir, const double* x, int nsrc, const lq_opts* o, double* eps,
                      void* stream) {
    if (!c || !x || !eps) return set_err(c, LQ_ERR_ARG, "null argument");
    int r = check_ready(c, nsrc, dir ? 1 : 0);
    if (r || (r = check_opts(c, o))) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)c->V * 12;              // complex entries per field
    const size_t reg = (size_t)c->nsrc * n * 2;      // doubles per staging region
    double* io[6];
    for (int i = 0; i < 6; ++i) io[i] = c->io + (size_t)i * reg;
    if ((r = stage_in(c, io[0], x, (size_t)nsrc * n * 2, st))) return r;
    std::vector<double> num(nsrc), num2(nsrc), den(nsrc);
    if (!dir) {
        if ((r = run_tsl(c, 1, 0, nsrc, o, nullptr, io[1], nullptr, st, io[0]))) return r;
        if ((r = run_tsl(c, 1, 0, nsrc, o, nullptr, io[2], nullptr, st, io[1]))) return r;
        LQ_CUDA(c, launch_norm2(io[2], io[0], -1.0, n, nsrc, c->norms, st));
        LQ_CUDA(c, launch_norm2(io[0], nullptr, 0.0, n, nsrc, c->norms + c->nsrc, st));
        c->launches += 2;
        LQ_CUDA(c, cudaMemcpyAsync(num.data(), c->norms, sizeof(double) * nsrc, cudaMemcpyDeviceToHost, st));
        LQ_CUDA(c, cudaMemcpyAsync(den.data(), c->norms + c->nsrc, sizeof(double) * nsrc, cudaMemcpyDeviceToHost, st));
        LQ_CUDA(c, cudaStreamSynchronize(st));
        for (int s = 0; s < nsrc; ++s) eps[s] = std::sqrt(num[s]) / (2.0 * std::sqrt(den[s]));
        return LQ_OK;
    }
    if ((r = lq_set_direction(c, dir, stream))) return r;
    const int em = emode_of(c);
    // (y_d, y_s) = sgn(B)(0, x);  (z_d, z_s) = sgn(B)(0, y_s);  s_d = sgn(A) y_d
    if ((r = run_tsl(c, 2, em, nsrc, o, nullptr, io[1], io[2], st, io[0]))) return r;
    if ((r = run_tsl(c, 2, em, nsrc, o, nullptr, io[3], io[4], st, io[2]))) return r;
    if ((r = run_tsl(c, 1, 0, nsrc, o, nullptr, io[5], nullptr, st, io[1]))) return r;
    LQ_CUDA(c, launch_norm2(io[5], io[3], 1.0, n, nsrc, c->norms, st));              // top: s_d + z_d
    LQ_CUDA(c, launch_norm2(io[4], io[0], -1.0, n, nsrc, c->norms + c->nsrc, st));   // bottom: z_s - x
    LQ_CUDA(c, launch_norm2(io[0], nullptr, 0.0, n, nsrc, c->norms + 2 * c->nsrc, st));
    c->launches += 3;
    LQ_CUDA(c, cudaMemcpyAsync(num.data(), c->norms, sizeof(double) * nsrc, cudaMemcpyDeviceToHost, st));
    LQ_CUDA(c, cudaMemcpyAsync(num2.data(), c->norms + c->nsrc, sizeof(double) * nsrc, cudaMemcpyDeviceToHost, st));
    LQ_CUDA(c, cudaMemcpyAsync(den.data(), c->norms + 2 * c->nsrc, sizeof(double) * nsrc, cudaMemcpyDeviceToHost, st));
    LQ_CUDA(c, cudaStreamSynchronize(st));
    for (int s = 0; s < nsrc; ++s) eps[s] = std::sqrt(num[s] + num2[s]) / (2.0 * std::sqrt(den[s]));
    return LQ_OK;
}

int lq_newton_sign(lq_ctx* c, const double* X, double* S, int k, int nb, int max_iter, double tol, int* iters, void* stream) {
    if (!c || !X || !S) return set_err(c, LQ_ERR_ARG, "null argument");
    if (!c->nx_X) return set_err(c, LQ_ERR_NOT_READY, "workspace not reserved (lq_reserve)");
    if (k < 1 || k > c->kmax || nb < 1 || nb > c->nsrc || max_iter < 1 || !(tol > 0.0))
        return set_err(c, LQ_ERR_ARG, "k / nb outside the reserved workspace, or bad iteration limits");
    if (!is_device_ptr(X) || !is_device_ptr(S)) return set_err(c, LQ_ERR_LAYOUT, "X and S must be device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    NewtonArgs a = newton_args(c, k, nb, max_iter, tol);
    LQ_CUDA(c, newton_init_dense(a, reinterpret_cast<const double2*>(X), st));
    c->launches += 2;
    std::vector<double> scal;
    int r = run_newton(c, a, st, scal);
    if (r) return r;
    LQ_CUDA(c, newton_copy_out(a, reinterpret_cast<double2*>(S), st));
    LQ_CUDA(c, cudaStreamSynchronize(st));
    prof_collect(c);
    int bad = 0;
    for (int b = 0; b < nb; ++b) {
        if (iters) iters[b] = (int)scal[(size_t)b * 16 + NS_ITERS];
        if (scal[(size_t)b * 16 + NS_STATUS] != 0.0) bad = 1;
    }
    return bad ? set_err(c, LQ_ERR_NEWTON, "Newton iteration did not converge for at least one matrix") : LQ_OK;
}

int lq_nested_sign(lq_ctx* c, const double* alpha, const double* beta, const double* delta, const double* scale, int k, int nb,
                   int m, double* out, double* check, void* stream) {
    if (!c || !alpha || (k > 1 && (!beta || !delta)) || !out) return set_err(c, LQ_ERR_ARG, "null argument");
    if (!c->nest_state) return set_err(c, LQ_ERR_NOT_READY, "workspace not reserved (lq_reserve)");
    if (k < 1 || k > c->kmax || nb < 1 || nb > c->nsrc || m < 1 || m > c->kmax)
        return set_err(c, LQ_ERR_ARG, "k, nb or m outside the reserved workspace");
    cudaStream_t st = (cudaStream_t)stream;
    // the coefficients go to the context's rows (stride kmax); rows beyond k are not read
    for (int b = 0; b < nb; ++b) {
        const size_t o = (size_t)b * c->kmax;
        auto kind = [](const void* p) { return is_device_ptr(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; };
        LQ_CUDA(c, cudaMemcpyAsync(c->alpha + o, alpha + (size_t)b * k * 2, sizeof(double2) * k, kind(alpha), st));
        if (k > 1) {
            LQ_CUDA(c, cudaMemcpyAsync(c->beta + o, beta + (size_t)b * (k - 1) * 2, sizeof(double2) * (k - 1), kind(beta), st));
            LQ_CUDA(c, cudaMemcpyAsync(c->delta + o, delta + (size_t)b * (k - 1), sizeof(double) * (k - 1), kind(delta), st));
        }
    }
    if (scale) {
        LQ_CUDA(c, cudaMemcpyAsync(c->nest_c, scale, sizeof(double) * nb, is_device_ptr(scale) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else {
        // the quadrature's estimate, from per-source states of dimension k
        std::vector<TslState> hs(nb);
        std::memset(hs.data(), 0, sizeof(TslState) * nb);
        for (auto& s : hs) s.k_eff = k;
        LQ_CUDA(c, cudaMemcpyAsync(c->state, hs.data(), sizeof(TslState) * nb, cudaMemcpyHostToDevice, st));
        QuadArgs qa;
        std::memset(&qa, 0, sizeof(qa));
        qa.k = k; qa.nb = nb; qa.kmax = c->kmax; qa.state = c->state;
        qa.alpha = c->alpha; qa.beta = c->beta; qa.delta = c->delta; qa.c = c->nest_c; qa.work = c->quad_work;
        qa.nth_max = 2 * kQuadRetryMaxNodes;
        LQ_CUDA(c, quad_scale(qa, st));
        LQ_CUDA(c, cudaStreamSynchronize(st));   // hs is host memory
    }
    std::vector<int> sel(nb, 1);
    std::vector<double> chk;
    int r = nested_run(c, nullptr, k, nb, m, c->nest_c, sel, c->proj_c, chk, 50, 1e-13, st);
    if (r) return r;
    for (int b = 0; b < nb; ++b) {
        const size_t o = (size_t)b * c->kmax;
        LQ_CUDA(c, cudaMemcpyAsync(out + (size_t)b * k * 2, c->proj_c + o, sizeof(double2) * k,
                                   is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    LQ_CUDA(c, cudaStreamSynchronize(st));
    bool bad = false;
    for (int b = 0; b < nb; ++b) {
        if (check) check[b] = chk[b];
        bad = bad || !std::isfinite(chk[b]);
    }
    return bad ? set_err(c, LQ_ERR_NEWTON, "an inner Newton iteration of the nested process did not converge") : LQ_OK;
}

}  // extern "C"
