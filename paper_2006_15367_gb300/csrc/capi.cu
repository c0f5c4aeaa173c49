// C ABI of the MLFMA library: argument checks, plan lifetime, host/device staging.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "common.cuh"

namespace mlfma {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

void fail(mlfma_status st, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    throw Failure{st};
}

void* Allocator::get(size_t n) {
    if (n == 0) n = 16;
    n = (n + 255) & ~(size_t)255;
    void* ptr = nullptr;
    if (alloc) {
        ptr = alloc(n, (void*)stream, ctx);
        if (!ptr) fail(MLFMA_ERR_OUT_OF_MEMORY, "allocator callback returned NULL for %zu bytes", n);
        if ((uintptr_t)ptr & 255) {
            if (free) free(ptr, (void*)stream, ctx);
            fail(MLFMA_ERR_INVALID_ARG, "allocator callback returned %p, not 256-byte aligned", ptr);
        }
    } else {
        cudaError_t e = cudaMalloc(&ptr, n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(MLFMA_ERR_OUT_OF_MEMORY, "cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
        }
    }
    live.emplace_back(ptr, n);
    bytes += n;
    return ptr;
}

void Allocator::drop(void* ptr) {
    if (!ptr) return;
    for (size_t i = 0; i < live.size(); ++i)
        if (live[i].first == ptr) {
            if (free) free(ptr, (void*)stream, ctx);
            else cudaFree(ptr);
            bytes -= live[i].second;
            live[i] = live.back();
            live.pop_back();
            return;
        }
}

void Allocator::release_all() {
    for (auto& a : live) {
        if (free) free(a.first, (void*)stream, ctx);
        else cudaFree(a.first);
    }
    live.clear();
    bytes = 0;
}

size_t csize(const Plan& p) { return p.prec == MLFMA_PREC_FP64 ? 16 : 8; }

// A pointer the current device's kernels can dereference: managed memory, or device memory of
// the current device (another GPU's memory would need peer access; such pointers are refused).
static bool is_device_ptr(const void* ptr) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    if (a.type != cudaMemoryTypeDevice) return false;
    int dev = 0;
    MLFMA_CUDA(cudaGetDevice(&dev));
    if (a.device != dev)
        fail(MLFMA_ERR_INVALID_ARG, "pointer %p is memory of device %d, not of the current device %d", ptr, a.device, dev);
    return true;
}

static void drop_graphs(Plan& p) {
    for (auto& g : p.graphs) cudaGraphExecDestroy(g.second);
    p.graphs.clear();
}

// Signatures F and G of every far level with room for nr right-hand sides (layout
// [r][nbox][K], slice 0 first).  The old buffers are released, so the plan is marked: run()
// drops every captured graph (a batched plan's graphs belong to its parent) before it
// captures again.
static void ensure_far_rhs(Plan& p, int nr) {
    if (nr <= p.far_nr || !p.top) return;
    MLFMA_CUDA(cudaDeviceSynchronize());           // no graph in flight still uses the old buffers
    for (int l = p.top; l <= p.nlev; ++l) {
        FarLevel& F = p.far[l];
        const size_t bytes = (size_t)nr * p.lev[l].nbox * F.K * csize(p);
        p.mem.drop(F.F);
        p.mem.drop(F.G);
        F.F = p.mem.get(bytes);
        F.G = p.mem.get(bytes);
        MLFMA_CUDA(cudaMemsetAsync(F.G, 0, bytes, p.stream));    // boxes M2L never writes stay zero
    }
    p.far_nr = nr;
    p.graphs_stale = true;
}

// Morton-order work buffers of one plan (grown only; growth invalidates captured graphs)
static void ensure_apply_buffers(Plan& p, int nrhs) {
    if (nrhs >= kMaxNR) ensure_far_rhs(p, kMaxNR);
    if (nrhs <= p.nrhs_cap) return;
    p.qs = p.mem.get((size_t)nrhs * p.n * csize(p));
    p.phis = p.mem.get((size_t)nrhs * p.n * csize(p));
    p.nrhs_cap = nrhs;
    drop_graphs(p);
}

static void ensure_grad_buffers(Plan& p, int nrhs) {
    if (nrhs <= p.nrhs_grad) return;
    p.grads = p.mem.get((size_t)3 * nrhs * p.n * csize(p));
    p.nrhs_grad = nrhs;
    drop_graphs(p);
}

// caller-order staging of the (top-level) plan
static void ensure_io_buffers(Plan& P, int nrhs, bool grad) {
    if (nrhs > P.nrhs_io) {
        P.qin = P.mem.get((size_t)nrhs * P.ntot * csize(P));
        P.phiout = P.mem.get((size_t)nrhs * P.ntot * csize(P));
        P.gout = nullptr;
        P.nrhs_io = nrhs;
        drop_graphs(P);
    }
    if (grad && !P.gout) {
        P.gout = P.mem.get((size_t)3 * P.nrhs_io * P.ntot * csize(P));
        drop_graphs(P);
    }
}

// One plan's share of an apply on p.stream: permute the rows of qin (stride ld) into
// Morton order, run the sweep per right-hand side, permute back into phiout / gout.
static void sweep(Plan& p, const void* qin, void* phiout, void* gout, int64_t ld, int nrhs, bool adjoint, bool grad) {
    ensure_apply_buffers(p, nrhs);
    if (grad) ensure_grad_buffers(p, nrhs);
    const size_t cs = csize(p);
    {
        StageTimer st(p, MLFMA_STAGE_PERMUTE, 0, 1);
        permute_in(p, qin, p.qs, nrhs, adjoint, ld);
    }
    // passes of kMaxNR right-hand sides while that many remain (not for gradients), then single ones
    for (int r = 0; r < nrhs;) {
        const int nr = (!grad && nrhs - r >= kMaxNR) ? kMaxNR : 1;
        apply_pipeline(p, (const char*)p.qs + (size_t)r * p.n * cs, (char*)p.phis + (size_t)r * p.n * cs,
                       grad ? (char*)p.grads + (size_t)3 * r * p.n * cs : nullptr, nr);
        r += nr;
    }
    {
        StageTimer st(p, MLFMA_STAGE_PERMUTE, 0, 1);
        permute_out(p, p.phis, phiout, nrhs, adjoint, ld);
        if (grad) permute_out3(p, p.grads, gout, nrhs, ld);
    }
}

// The whole apply of P from P.qin to P.phiout on stream s (batched plans fork their
// geometries over the sub-streams and join back).
static void sweep_all(Plan& P, cudaStream_t s, int nrhs, bool adjoint, bool grad) {
    if (P.subs.empty() || P.forest) {
        cudaStream_t keep = P.stream;
        P.stream = s;
        try {
            sweep(P, P.qin, P.phiout, P.gout, P.ntot, nrhs, adjoint, grad);
        } catch (...) {
            P.stream = keep;
            throw;
        }
        P.stream = keep;
        return;
    }
    const size_t cs = csize(P);
    MLFMA_CUDA(cudaEventRecord(P.ev_fork, s));
    for (size_t w = 0; w < P.sub_streams.size(); ++w) MLFMA_CUDA(cudaStreamWaitEvent(P.sub_streams[w], P.ev_fork, 0));
    for (size_t g = 0; g < P.subs.size(); ++g) {
        Plan& sp = *P.subs[g];
        sp.stream = P.sub_streams[g % P.sub_streams.size()];
        const int64_t o = P.sub_off[g];
        sweep(sp, (const char*)P.qin + o * cs, (char*)P.phiout + o * cs, grad ? (char*)P.gout + 3 * o * cs : nullptr,
              P.ntot, nrhs, adjoint, grad);
    }
    for (size_t w = 0; w < P.sub_streams.size(); ++w) {
        MLFMA_CUDA(cudaEventRecord(P.sub_events[w], P.sub_streams[w]));
        MLFMA_CUDA(cudaStreamWaitEvent(s, P.sub_events[w], 0));
    }
}

static void run(Plan& P, int nrhs, bool adjoint, bool grad) {
    const bool graphs = P.use_graphs && !P.profiling;
    if (!graphs) {
        sweep_all(P, P.stream, nrhs, adjoint, grad);
        return;
    }
    const int64_t key = (int64_t)nrhs * 4 + (adjoint ? 2 : 0) + (grad ? 1 : 0);
    auto it = P.graphs.find(key);
    if (it == P.graphs.end()) {
        // first call with this shape: run eagerly (this also sizes every buffer), then capture
        sweep_all(P, P.stream, nrhs, adjoint, grad);
        bool stale = P.graphs_stale;
        for (Plan* sp : P.subs) stale = stale || sp->graphs_stale;
        if (stale) {                                   // buffers the other graphs captured were replaced
            drop_graphs(P);
            P.graphs_stale = false;
            for (Plan* sp : P.subs) sp->graphs_stale = false;
        }
        MLFMA_CUDA(cudaEventRecord(P.ev_fork, P.stream));
        MLFMA_CUDA(cudaStreamWaitEvent(P.gstream, P.ev_fork, 0));
        MLFMA_CUDA(cudaStreamBeginCapture(P.gstream, cudaStreamCaptureModeThreadLocal));
        cudaGraph_t graph = nullptr;
        try {
            sweep_all(P, P.gstream, nrhs, adjoint, grad);
        } catch (...) {
            cudaStreamEndCapture(P.gstream, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        MLFMA_CUDA(cudaStreamEndCapture(P.gstream, &graph));
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        MLFMA_CUDA(e);
        P.graphs[key] = exec;
        return;
    }
    MLFMA_CUDA(cudaEventRecord(P.ev_fork, P.stream));
    MLFMA_CUDA(cudaStreamWaitEvent(P.gstream, P.ev_fork, 0));
    MLFMA_CUDA(cudaGraphLaunch(it->second, P.gstream));
    MLFMA_CUDA(cudaEventRecord(P.ev_join, P.gstream));
    MLFMA_CUDA(cudaStreamWaitEvent(P.stream, P.ev_join, 0));
}

// Error flags raised by kernels that gave up a bounded wait (this plan and its sub-plans):
// synchronises the streams, reports a raised flag as MLFMA_ERR_TIMEOUT and clears it.
// Flag values: 1 = a tensor-core MMA did not complete, 2 = the M2L operator-slice copy did not land.
static void check_device_errors(const Plan& p) {
    auto one = [](const Plan& q) {
        if (!q.dev_err) return;
        int e = 0;
        MLFMA_CUDA(cudaStreamSynchronize(q.stream));
        MLFMA_CUDA(cudaMemcpy(&e, q.dev_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) {
            MLFMA_CUDA(cudaMemset(q.dev_err, 0, sizeof(int)));
            fail(MLFMA_ERR_TIMEOUT, "a bounded device wait ran out (%s)",
                 e == 1 ? "tensor-core MMA completion" : e == 2 ? "M2L operator-slice copy" : "unknown wait");
        }
    };
    one(p);
    if (p.gstream) MLFMA_CUDA(cudaStreamSynchronize(p.gstream));
    for (const Plan* sp : p.subs) one(*sp);
}

static void apply_impl(Plan& P, const void* q, void* phi, int nrhs, bool adjoint, void* grad = nullptr) {
    if (!q || (!phi && !grad)) fail(MLFMA_ERR_INVALID_ARG, "null q or phi");
    if (nrhs < 1) fail(MLFMA_ERR_INVALID_ARG, "nrhs must be >= 1 (got %d)", nrhs);
    const size_t bytes = (size_t)nrhs * P.ntot * csize(P);
    const bool dq = is_device_ptr(q), dphi = phi ? is_device_ptr(phi) : true;
    if (grad && (!dq || !dphi || !is_device_ptr(grad)))
        fail(MLFMA_ERR_INVALID_ARG, "mlfma_apply_grad takes device pointers only");
    ensure_io_buffers(P, nrhs, grad != nullptr);
    MLFMA_CUDA(cudaMemcpyAsync(P.qin, q, bytes, dq ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, P.stream));
    run(P, nrhs, adjoint, grad != nullptr);
    if (phi)
        MLFMA_CUDA(cudaMemcpyAsync(phi, P.phiout, bytes, dphi ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, P.stream));
    if (grad) MLFMA_CUDA(cudaMemcpyAsync(grad, P.gout, 3 * bytes, cudaMemcpyDeviceToDevice, P.stream));
    if (P.profiling) P.acc.applies += nrhs;
    if (!dphi || !dq) {
        MLFMA_CUDA(cudaStreamSynchronize(P.stream));
        check_device_errors(P);
    }
}

// Reverse mode (see mlfma_apply_vjp): psi = A conj(g) and grad psi by one adjoint gradient sweep
// (phiout = conj(psi) = A^H g), grad phi from the caller or from a second gradient sweep, and
// the position gradient assembled by one kernel.
static void vjp_impl(Plan& P, const void* q, const void* g, const void* gphi, void* grad_q, double* grad_r, int nrhs) {
    if (!q || !g) fail(MLFMA_ERR_INVALID_ARG, "null q or g");
    if (!grad_q && !grad_r) fail(MLFMA_ERR_INVALID_ARG, "grad_q and grad_r are both NULL");
    if (nrhs < 1) fail(MLFMA_ERR_INVALID_ARG, "nrhs must be >= 1 (got %d)", nrhs);
    if (!is_device_ptr(q) || !is_device_ptr(g) || (gphi && !is_device_ptr(gphi)) || (grad_q && !is_device_ptr(grad_q)) ||
        (grad_r && !is_device_ptr(grad_r)))
        fail(MLFMA_ERR_INVALID_ARG, "mlfma_apply_vjp takes device pointers only");
    const size_t bytes = (size_t)nrhs * P.ntot * csize(P);
    const bool want_r = grad_r != nullptr;
    ensure_io_buffers(P, nrhs, want_r);
    const void* gphi_use = gphi;
    if (want_r && !gphi) {
        // recompute grad phi of the forward charges and keep it while the adjoint sweep runs
        if (nrhs > P.nrhs_vjp) {
            P.mem.drop(P.vjp_buf);
            P.vjp_buf = nullptr;
            P.vjp_buf = P.mem.get(3 * bytes);
            P.nrhs_vjp = nrhs;
        }
        MLFMA_CUDA(cudaMemcpyAsync(P.qin, q, bytes, cudaMemcpyDeviceToDevice, P.stream));
        run(P, nrhs, false, true);
        MLFMA_CUDA(cudaMemcpyAsync(P.vjp_buf, P.gout, 3 * bytes, cudaMemcpyDeviceToDevice, P.stream));
        gphi_use = P.vjp_buf;
    }
    MLFMA_CUDA(cudaMemcpyAsync(P.qin, g, bytes, cudaMemcpyDeviceToDevice, P.stream));
    run(P, nrhs, true, want_r);
    if (grad_q) MLFMA_CUDA(cudaMemcpyAsync(grad_q, P.phiout, bytes, cudaMemcpyDeviceToDevice, P.stream));
    if (want_r) position_grad(P, P.ntot, nrhs, q, g, gphi_use, P.gout, grad_r, P.stream);
    if (P.profiling) P.acc.applies += nrhs * (want_r && !gphi ? 2 : 1);
    MLFMA_CUDA(cudaStreamSynchronize(P.stream));
    check_device_errors(P);
}

void apply_device(Plan& P, const void* q) {
    ensure_io_buffers(P, 1, false);
    MLFMA_CUDA(cudaMemcpyAsync(P.qin, q, (size_t)P.ntot * csize(P), cudaMemcpyDeviceToDevice, P.stream));
    run(P, 1, false, false);
    if (P.profiling) P.acc.applies += 1;
}

// Plan-time choice of the interpolation tile budgets (row tiles, per-parent tiles, fused level
// pairs).  Each candidate runs the apply sweep eagerly on a zero charge vector (the instruction
// stream does not depend on the values): once to warm up, then three times timed by CUDA events
// on the plan stream; the smallest median wins.  Captured graphs are dropped afterwards.
static void set_tiles(Plan& P, const int* t) {
    P.tile_fft = t[0];
    P.tile_parent = t[1];
    P.tile_fused = t[2];
    for (Plan* sp : P.subs) set_tiles(*sp, t);
}

static void autotune_tiles(Plan& P) {
    static const int cand[4][3] = {{20 << 10, 32 << 10, 40 << 10},
                                   {16 << 10, 24 << 10, 32 << 10},
                                   {32 << 10, 64 << 10, 64 << 10},
                                   {12 << 10, 16 << 10, 24 << 10}};
    ensure_io_buffers(P, 1, false);
    MLFMA_CUDA(cudaMemsetAsync(P.qin, 0, (size_t)P.ntot * csize(P), P.stream));
    cudaEvent_t a = nullptr, b = nullptr;
    MLFMA_CUDA(cudaEventCreate(&a));
    MLFMA_CUDA(cudaEventCreate(&b));
    const bool graphs = P.use_graphs;
    P.use_graphs = false;
    int best = 0;
    float best_ms = 0;
    try {
        for (int c = 0; c < 4; ++c) {
            set_tiles(P, cand[c]);
            run(P, 1, false, false);
            float t[3];
            for (int r = 0; r < 3; ++r) {
                MLFMA_CUDA(cudaEventRecord(a, P.stream));
                run(P, 1, false, false);
                MLFMA_CUDA(cudaEventRecord(b, P.stream));
                MLFMA_CUDA(cudaEventSynchronize(b));
                MLFMA_CUDA(cudaEventElapsedTime(&t[r], a, b));
            }
            std::sort(t, t + 3);
            if (c == 0 || t[1] < best_ms) {
                best_ms = t[1];
                best = c;
            }
        }
    } catch (...) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        P.use_graphs = graphs;
        throw;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    set_tiles(P, cand[best]);
    P.use_graphs = graphs;
    drop_graphs(P);
}

static void init_streams(Plan& P, int nsub) {
    MLFMA_CUDA(cudaStreamCreateWithFlags(&P.gstream, cudaStreamNonBlocking));
    MLFMA_CUDA(cudaEventCreateWithFlags(&P.ev_fork, cudaEventDisableTiming));
    MLFMA_CUDA(cudaEventCreateWithFlags(&P.ev_join, cudaEventDisableTiming));
    MLFMA_CUDA(cudaStreamCreateWithFlags(&P.nstream, cudaStreamNonBlocking));
    MLFMA_CUDA(cudaEventCreateWithFlags(&P.ev_nfork, cudaEventDisableTiming));
    MLFMA_CUDA(cudaEventCreateWithFlags(&P.ev_near, cudaEventDisableTiming));
    MLFMA_CUDA(cudaStreamCreateWithFlags(&P.mstream, cudaStreamNonBlocking));
    MLFMA_CUDA(cudaEventCreateWithFlags(&P.ev_mfork, cudaEventDisableTiming));
    MLFMA_CUDA(cudaEventCreateWithFlags(&P.ev_mdone, cudaEventDisableTiming));
    MLFMA_CUDA(cudaStreamCreateWithFlags(&P.sstream, cudaStreamNonBlocking));
    MLFMA_CUDA(cudaEventCreateWithFlags(&P.ev_sfork, cudaEventDisableTiming));
    MLFMA_CUDA(cudaEventCreateWithFlags(&P.ev_sdone, cudaEventDisableTiming));
    for (int w = 0; w < nsub; ++w) {
        cudaStream_t st;
        cudaEvent_t ev;
        MLFMA_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        P.sub_streams.push_back(st);
        MLFMA_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        P.sub_events.push_back(ev);
    }
}

static void release_plan(Plan& P) {
    if (P.stream) cudaStreamSynchronize(P.stream);
    if (P.gstream) cudaStreamSynchronize(P.gstream);
    if (P.nstream) cudaStreamSynchronize(P.nstream);
    if (P.mstream) cudaStreamSynchronize(P.mstream);
    if (P.sstream) cudaStreamSynchronize(P.sstream);
    for (auto s : P.sub_streams) cudaStreamSynchronize(s);
    drop_graphs(P);
    for (auto* sp : P.subs) {
        release_plan(*sp);
        delete sp;
    }
    P.subs.clear();
    for (auto& r : P.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    P.recs.clear();
    for (auto e : P.pool) cudaEventDestroy(e);
    P.pool.clear();
    for (auto s : P.sub_streams) cudaStreamDestroy(s);
    for (auto e : P.sub_events) cudaEventDestroy(e);
    P.sub_streams.clear();
    P.sub_events.clear();
    if (P.ev_fork) cudaEventDestroy(P.ev_fork);
    if (P.ev_join) cudaEventDestroy(P.ev_join);
    if (P.gstream) cudaStreamDestroy(P.gstream);
    if (P.ev_nfork) cudaEventDestroy(P.ev_nfork);
    if (P.ev_near) cudaEventDestroy(P.ev_near);
    if (P.nstream) cudaStreamDestroy(P.nstream);
    if (P.ev_mfork) cudaEventDestroy(P.ev_mfork);
    if (P.ev_mdone) cudaEventDestroy(P.ev_mdone);
    if (P.mstream) cudaStreamDestroy(P.mstream);
    if (P.ev_sfork) cudaEventDestroy(P.ev_sfork);
    if (P.ev_sdone) cudaEventDestroy(P.ev_sdone);
    if (P.sstream) cudaStreamDestroy(P.sstream);
    P.ev_fork = P.ev_join = P.ev_nfork = P.ev_near = P.ev_mfork = P.ev_mdone = P.ev_sfork = P.ev_sdone = nullptr;
    P.gstream = P.nstream = P.mstream = P.sstream = nullptr;
    P.mem.release_all();
}

}  // namespace mlfma

using namespace mlfma;

template <typename F>
static mlfma_status guarded(F f) {
    try {
        mlfma::set_error("%s", "");
        f();
        return MLFMA_OK;
    } catch (const Failure& e) {
        return e.status;
    } catch (const std::bad_alloc&) {
        mlfma::set_error("host allocation failed");
        return MLFMA_ERR_OUT_OF_MEMORY;
    }
}

extern "C" {

void mlfma_options_init(mlfma_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->struct_size = sizeof(*opt);
    opt->precision = MLFMA_PREC_FP32;
    opt->leaf_edge = 0.0;
    opt->max_depth = 12;
    opt->digit_margin = -1;
}

static mlfma_options checked_options(const mlfma_options* opt, double k, int digits, int leaf_max) {
    if (!(k > 0.0) || !std::isfinite(k)) fail(MLFMA_ERR_INVALID_ARG, "k must be finite and > 0");
    if (digits < 1 || digits > 12) fail(MLFMA_ERR_INVALID_ARG, "digits must be in [1, 12] (got %d)", digits);
    if (leaf_max < 0) fail(MLFMA_ERR_INVALID_ARG, "leaf_max must be >= 0");
    mlfma_options o;
    mlfma_options_init(&o);
    if (opt) {
        // callers built against an older header pass a shorter struct: the fields they know are
        // taken, the newer ones keep their defaults
        constexpr size_t kOldest = offsetof(mlfma_options, autotune) + sizeof(int);
        if (opt->struct_size < kOldest) fail(MLFMA_ERR_INVALID_ARG, "options.struct_size too small");
        memcpy(&o, opt, std::min(opt->struct_size, sizeof(mlfma_options)));
        o.struct_size = sizeof(mlfma_options);
    }
    if (o.precision != MLFMA_PREC_FP64 && o.precision != MLFMA_PREC_FP32 && o.precision != MLFMA_PREC_FP32_TF32X3 &&
        o.precision != MLFMA_PREC_FP32_BF16X3)
        fail(MLFMA_ERR_INVALID_ARG, "unknown precision %d", (int)o.precision);
    if (o.max_depth < 1 || o.max_depth > kMaxLev) fail(MLFMA_ERR_INVALID_ARG, "max_depth must be in [1, %d]", kMaxLev);
    if (o.digit_margin < -1 || o.digit_margin > 8) fail(MLFMA_ERR_INVALID_ARG, "digit_margin must be in [-1, 8]");
    if (!std::isfinite(o.leaf_edge)) fail(MLFMA_ERR_INVALID_ARG, "leaf_edge must be finite");
    if ((o.alloc == nullptr) != (o.free == nullptr)) fail(MLFMA_ERR_INVALID_ARG, "alloc and free must be given together");
    if (o.recompute_signatures != 0 && o.recompute_signatures != 1)
        fail(MLFMA_ERR_INVALID_ARG, "recompute_signatures must be 0 or 1");
    if (o.test_fail_waits != 0 && o.test_fail_waits != 1) fail(MLFMA_ERR_INVALID_ARG, "test_fail_waits must be 0 or 1");
    if (o.dense_samples < -1) fail(MLFMA_ERR_INVALID_ARG, "dense_samples must be >= -1");
    if (o.sampled_operators != 0 && (o.sampled_operators < 3 || o.sampled_operators > 32))
        fail(MLFMA_ERR_INVALID_ARG, "sampled_operators must be 0 or in [3, 32] (got %d)", o.sampled_operators);
    return o;
}

static void configure(Plan& p, int64_t n, double k, int digits, int leaf_max, const mlfma_options& o) {
    p.n = n;
    p.ntot = n;
    p.k = k;
    p.digits = digits;
    p.leaf_max = leaf_max;
    p.max_depth = o.max_depth;
    p.margin = o.digit_margin >= 0 ? o.digit_margin : (o.precision == MLFMA_PREC_FP64 ? 1 : 0);
    p.prec = o.precision;
    p.leaf_edge = o.leaf_edge > 0 ? o.leaf_edge : (digits <= 4 ? 0.5 * M_PI / k : M_PI / k);
    p.stream = (cudaStream_t)o.stream;
    p.use_graphs = !o.disable_graphs;
    p.mem.alloc = o.alloc;
    p.mem.free = o.free;
    p.mem.ctx = o.alloc_ctx;
    p.mem.stream = p.stream;
    p.wait_first = o.test_fail_waits ? 0 : (1ll << 22);
    p.recompute = o.recompute_signatures ? 1 : 0;
    p.dense_kc = o.dense_samples > 0 ? o.dense_samples : 0;
    p.op_s = o.sampled_operators;
}

// tree, lists, grids and operators of one point set (device points)
static void build_plan(Plan& p, const double* pts) {
    build_tree(p, pts);
    build_lists(p);
    build_far_levels(p);
    build_m2l_lists(p);
    build_p2p_work(p);
    p.dev_err = p.mem.make<int>(1);
    MLFMA_CUDA(cudaMemsetAsync(p.dev_err, 0, sizeof(int), p.stream));
    prepare_kernels(p);
    p.near_dump = p.mem.get(p.n * csize(p));
    ensure_apply_buffers(p, 1);
    MLFMA_CUDA(cudaStreamSynchronize(p.stream));
}

mlfma_status mlfma_plan_create(const double* points, int64_t n, double k, int digits, int leaf_max, const mlfma_options* opt,
                               mlfma_plan** out) {
    if (out) *out = nullptr;
    mlfma_plan* h = nullptr;
    mlfma_status st = guarded([&] {
        auto t0 = std::chrono::steady_clock::now();
        if (!points || !out) fail(MLFMA_ERR_INVALID_ARG, "null points or out");
        if (n < 1) fail(MLFMA_ERR_INVALID_ARG, "n must be >= 1 (got %lld)", (long long)n);
        if (n > (int64_t)INT32_MAX / 4) fail(MLFMA_ERR_UNSUPPORTED, "n = %lld exceeds the 32-bit index range", (long long)n);
        const mlfma_options o = checked_options(opt, k, digits, leaf_max);
        h = new mlfma_plan();
        Plan& p = h->p;
        configure(p, n, k, digits, leaf_max, o);
        init_streams(p, 0);
        const double* pts = points;
        if (!is_device_ptr(points)) {
            double* d = p.mem.make<double>(3 * n);
            MLFMA_CUDA(cudaMemcpyAsync(d, points, 3 * n * sizeof(double), cudaMemcpyHostToDevice, p.stream));
            pts = d;
        }
        build_plan(p, pts);
        if (o.autotune) autotune_tiles(p);
        p.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        *out = h;
    });
    if (st != MLFMA_OK && h) {
        release_plan(h->p);
        delete h;
    }
    return st;
}

mlfma_status mlfma_plan_create_batched(const double* points, const int64_t* offsets, int n_geom, double k, int digits,
                                       int leaf_max, const mlfma_options* opt, mlfma_plan** out) {
    if (out) *out = nullptr;
    mlfma_plan* h = nullptr;
    mlfma_status st = guarded([&] {
        auto t0 = std::chrono::steady_clock::now();
        if (!points || !offsets || !out) fail(MLFMA_ERR_INVALID_ARG, "null points, offsets or out");
        if (n_geom < 1) fail(MLFMA_ERR_INVALID_ARG, "n_geom must be >= 1");
        if (offsets[0] != 0) fail(MLFMA_ERR_INVALID_ARG, "offsets[0] must be 0");
        for (int g = 0; g < n_geom; ++g)
            if (offsets[g + 1] <= offsets[g]) fail(MLFMA_ERR_INVALID_ARG, "geometry %d has no points", g);
        const int64_t ntot = offsets[n_geom];
        if (ntot > (int64_t)INT32_MAX / 4) fail(MLFMA_ERR_UNSUPPORTED, "total n exceeds the 32-bit index range");
        const mlfma_options o = checked_options(opt, k, digits, leaf_max);
        h = new mlfma_plan();
        Plan& P = h->p;
        configure(P, ntot, k, digits, leaf_max, o);
        init_streams(P, std::min(n_geom, 16));
        const double* pts = points;
        if (!is_device_ptr(points)) {
            double* d = P.mem.make<double>(3 * ntot);
            MLFMA_CUDA(cudaMemcpyAsync(d, points, 3 * ntot * sizeof(double), cudaMemcpyHostToDevice, P.stream));
            pts = d;
        }
        P.sub_off.assign(offsets, offsets + n_geom + 1);
        for (int g = 0; g < n_geom; ++g) {
            Plan* sp = new Plan();
            P.subs.push_back(sp);
            configure(*sp, offsets[g + 1] - offsets[g], k, digits, leaf_max, o);
            build_plan(*sp, pts + 3 * offsets[g]);
        }
        if (forest_possible(P.subs)) {
            build_forest(P);
            P.forest = true;
        }
        MLFMA_CUDA(cudaStreamSynchronize(P.stream));
        if (o.autotune) autotune_tiles(P);
        P.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        *out = h;
    });
    if (st != MLFMA_OK && h) {
        release_plan(h->p);
        delete h;
    }
    return st;
}

mlfma_status mlfma_apply(mlfma_plan* plan, const void* q, void* phi, int nrhs) {
    return guarded([&] {
        if (!plan) fail(MLFMA_ERR_INVALID_ARG, "null plan");
        apply_impl(plan->p, q, phi, nrhs, false);
    });
}

mlfma_status mlfma_apply_adjoint(mlfma_plan* plan, const void* r, void* g, int nrhs) {
    return guarded([&] {
        if (!plan) fail(MLFMA_ERR_INVALID_ARG, "null plan");
        apply_impl(plan->p, r, g, nrhs, true);
    });
}

mlfma_status mlfma_apply_grad(mlfma_plan* plan, const void* q, void* phi, void* grad, int nrhs) {
    return guarded([&] {
        if (!plan) fail(MLFMA_ERR_INVALID_ARG, "null plan");
        if (!grad) fail(MLFMA_ERR_INVALID_ARG, "null grad");
        apply_impl(plan->p, q, phi, nrhs, false, grad);
    });
}

mlfma_status mlfma_apply_vjp(mlfma_plan* plan, const void* q, const void* g, const void* gphi, void* grad_q,
                             double* grad_r, int nrhs) {
    return guarded([&] {
        if (!plan) fail(MLFMA_ERR_INVALID_ARG, "null plan");
        vjp_impl(plan->p, q, g, gphi, grad_q, grad_r, nrhs);
    });
}

mlfma_status mlfma_solve_gmres(mlfma_plan* plan, const void* b, void* x, double sigma_re, double sigma_im, double tol,
                               int restart, int max_iter, mlfma_solve_info* info) {
    return guarded([&] {
        if (!plan || !b || !x || !info) fail(MLFMA_ERR_INVALID_ARG, "null plan, b, x or info");
        if (!is_device_ptr(b) || !is_device_ptr(x)) fail(MLFMA_ERR_INVALID_ARG, "b and x must be device pointers");
        if (!(tol > 0 && tol < 1)) fail(MLFMA_ERR_INVALID_ARG, "tol must be in (0, 1) (got %g)", tol);
        if (restart < 1 || restart > 256) fail(MLFMA_ERR_INVALID_ARG, "restart must be in [1, 256] (got %d)", restart);
        if (max_iter < 1) fail(MLFMA_ERR_INVALID_ARG, "max_iter must be >= 1 (got %d)", max_iter);
        if (!std::isfinite(sigma_re) || !std::isfinite(sigma_im)) fail(MLFMA_ERR_INVALID_ARG, "sigma must be finite");
        gmres_solve(plan->p, b, x, sigma_re, sigma_im, tol, restart, max_iter, info);
        check_device_errors(plan->p);
    });
}

mlfma_status mlfma_plan_info(const mlfma_plan* plan, mlfma_info* info) {
    return guarded([&] {
        if (!plan || !info) fail(MLFMA_ERR_INVALID_ARG, "null plan or info");
        const Plan& p = plan->p;
        check_device_errors(p);
        memset(info, 0, sizeof(*info));
        info->n = p.n;
        info->nlev = p.nlev;
        info->top = p.top;
        info->precision = (int)p.prec;
        info->k = p.k;
        info->leaf_edge = p.leaf_edge;
        info->root_edge = p.a1;
        for (int a = 0; a < 3; ++a) info->root_corner[a] = p.x0[a];
        for (int l = 1; l <= p.nlev; ++l) {
            info->nbox[l] = p.lev[l].nbox;
            info->nleaf[l] = p.lev[l].nleaf;
            info->nv[l] = p.lev[l].nv;
            if (p.top && l >= p.top) {
                info->L[l] = p.far[l].L;
                info->K[l] = p.far[l].K;
            }
        }
        info->near_pairs = p.near_pairs;
        info->device_bytes = (int64_t)p.mem.bytes;
        info->setup_ms = p.setup_ms;
        info->tile_bytes[0] = p.tile_fft;
        info->tile_bytes[1] = p.tile_parent;
        info->tile_bytes[2] = p.tile_fused;
        info->n_geom = p.subs.empty() ? 1 : (int)p.subs.size();
        info->recompute_signatures = p.recompute;
        for (int l = 0; l <= kMaxLev; ++l) info->dense[l] = p.far[l].dense;
        info->sampled_operators = p.op_s;
        for (int l = 0; l <= kMaxLev; ++l) info->sampled[l] = p.far[l].T1 != nullptr;
        if (p.forest) {                                // the merged levels (height above the leaves)
            for (const Plan* sp : p.subs) info->device_bytes += (int64_t)sp->mem.bytes;
        } else if (!p.subs.empty()) {
            const Plan& s0 = *p.subs[0];
            info->nlev = s0.nlev;
            info->top = s0.top;
            info->leaf_edge = s0.leaf_edge;
            info->root_edge = s0.a1;
            for (int l = 1; l <= s0.nlev; ++l) {
                info->nbox[l] = s0.lev[l].nbox;
                info->nleaf[l] = s0.lev[l].nleaf;
                info->nv[l] = s0.lev[l].nv;
                if (s0.top && l >= s0.top) { info->L[l] = s0.far[l].L; info->K[l] = s0.far[l].K; }
            }
            for (const Plan* sp : p.subs) {
                info->device_bytes += (int64_t)sp->mem.bytes;
                info->near_pairs += sp->near_pairs;
            }
        }
    });
}

mlfma_status mlfma_plan_export(const mlfma_plan* plan, int item, int level, void* dst, size_t bytes, size_t* needed) {
    return guarded([&] {
        if (!plan) fail(MLFMA_ERR_INVALID_ARG, "null plan");
        const Plan& p = plan->p;
        if (!p.subs.empty()) fail(MLFMA_ERR_INVALID_ARG, "export is not available for batched plans");
        const bool per_level = item >= MLFMA_EXPORT_BOX_KEY && item != MLFMA_EXPORT_NEAR_OFFSETS &&
                               item != MLFMA_EXPORT_NEAR_SOURCES && item != MLFMA_EXPORT_NEAR_PHI;
        if (per_level && (level < 1 || level > p.nlev)) fail(MLFMA_ERR_INVALID_ARG, "level %d outside 1..%d", level, p.nlev);
        const TreeLevel* L = per_level ? &p.lev[level] : nullptr;
        const bool far_item = item == MLFMA_EXPORT_F || item == MLFMA_EXPORT_G || item == MLFMA_EXPORT_TRANSLATION ||
                              item == MLFMA_EXPORT_OPERATOR_SAMPLES;
        if (far_item && (!p.top || level < p.top)) fail(MLFMA_ERR_INVALID_ARG, "level %d has no far-field data", level);
        std::vector<std::pair<const void*, size_t>> parts;
        switch (item) {
            case MLFMA_EXPORT_PERM: parts.push_back({p.perm, p.n * sizeof(int)}); break;
            case MLFMA_EXPORT_KEYS: parts.push_back({p.keys, p.n * sizeof(uint64_t)}); break;
            case MLFMA_EXPORT_BOX_KEY: parts.push_back({L->key, L->nbox * sizeof(uint64_t)}); break;
            case MLFMA_EXPORT_BOX_BEGIN: parts.push_back({L->begin, L->nbox * sizeof(int)}); break;
            case MLFMA_EXPORT_BOX_END: parts.push_back({L->end, L->nbox * sizeof(int)}); break;
            case MLFMA_EXPORT_BOX_PARENT: parts.push_back({L->parent, L->nbox * sizeof(int)}); break;
            case MLFMA_EXPORT_BOX_LEAF: parts.push_back({L->leaf, L->nbox * sizeof(uint8_t)}); break;
            case MLFMA_EXPORT_V_OFFSETS:
                if (level < 2) fail(MLFMA_ERR_INVALID_ARG, "V lists start at level 2");
                parts.push_back({L->v_off, (L->nbox + 1) * sizeof(int)});
                break;
            case MLFMA_EXPORT_V_SOURCES:
                if (level < 2) fail(MLFMA_ERR_INVALID_ARG, "V lists start at level 2");
                parts.push_back({L->v_src, L->nv * sizeof(int)});
                break;
            case MLFMA_EXPORT_NEAR_OFFSETS: parts.push_back({p.near_off, (p.nleaf_total + 1) * sizeof(int)}); break;
            case MLFMA_EXPORT_NEAR_SOURCES:
                parts.push_back({p.near_lev, p.nnear * sizeof(int)});
                parts.push_back({p.near_box, p.nnear * sizeof(int)});
                break;
            case MLFMA_EXPORT_F: parts.push_back({p.far[level].F, L->nbox * p.far[level].K * csize(p)}); break;
            case MLFMA_EXPORT_G: parts.push_back({p.far[level].G, L->nbox * p.far[level].K * csize(p)}); break;
            case MLFMA_EXPORT_NEAR_PHI: parts.push_back({p.near_dump, p.n * csize(p)}); break;
            case MLFMA_EXPORT_TRANSLATION: {   // the 316 far rows of the 7^3 cube in raster order
                if (!p.far[level].T) fail(MLFMA_ERR_UNSUPPORTED, "level %d keeps sampled operators", level);
                const size_t row = p.far[level].K * csize(p);
                for (int dz = -3; dz <= 3; ++dz)
                    for (int dy = -3; dy <= 3; ++dy)
                        for (int dx = -3; dx <= 3; ++dx) {
                            if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) <= 1) continue;
                            const int r = (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3);
                            parts.push_back({(const char*)p.far[level].T + r * row, row});
                        }
                break;
            }
            case MLFMA_EXPORT_OPERATOR_SAMPLES:
                if (!p.far[level].T1) fail(MLFMA_ERR_UNSUPPORTED, "level %d keeps full operator tables", level);
                parts.push_back({p.far[level].T1, (size_t)kOpRows * p.far[level].T1n * csize(p)});
                break;
            default: fail(MLFMA_ERR_INVALID_ARG, "unknown export item %d", item);
        }
        size_t tot = 0;
        for (auto& x : parts) tot += x.second;
        if (needed) *needed = tot;
        if (!dst) return;
        if (bytes < tot) fail(MLFMA_ERR_INVALID_ARG, "buffer of %zu bytes < %zu needed", bytes, tot);
        check_device_errors(p);
        size_t off = 0;
        for (auto& x : parts) {
            if (x.second) MLFMA_CUDA(cudaMemcpy((char*)dst + off, x.first, x.second, cudaMemcpyDefault));
            off += x.second;
        }
    });
}

mlfma_status mlfma_direct_fp64(const double* points, int64_t n, const void* q, double k, const int64_t* targets, int64_t nt,
                               void* phi, void* stream) {
    return guarded([&] {
        if (!points || !q || !targets || !phi) fail(MLFMA_ERR_INVALID_ARG, "null pointer");
        if (n < 1 || nt < 0) fail(MLFMA_ERR_INVALID_ARG, "bad sizes");
        if (!(k > 0.0) || !std::isfinite(k)) fail(MLFMA_ERR_INVALID_ARG, "k must be finite and > 0");
        direct_fp64(points, n, q, k, targets, nt, phi, (cudaStream_t)stream);
    });
}

void mlfma_destroy(mlfma_plan* plan) {
    if (!plan) return;
    release_plan(plan->p);
    delete plan;
}

const char* mlfma_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace mlfma {

static cudaEvent_t take_event(Plan& p) {
    if (!p.pool.empty()) {
        cudaEvent_t e = p.pool.back();
        p.pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    MLFMA_CUDA(cudaEventCreate(&e));
    return e;
}

StageTimer::StageTimer(Plan& plan, int stage, int level, int launches, bool on) : p(plan) {
    if (!p.profiling || !on) return;
    Plan::EventRec r{stage, level, launches, take_event(p), take_event(p)};
    MLFMA_CUDA(cudaEventRecord(r.a, p.stream));
    p.recs.push_back(r);
    idx = (int)p.recs.size() - 1;
}

StageTimer::~StageTimer() {
    if (idx >= 0) cudaEventRecord(p.recs[idx].b, p.stream);
}

void collect_timings(Plan& p) {
    MLFMA_CUDA(cudaStreamSynchronize(p.stream));
    for (auto& r : p.recs) {
        float ms = 0;
        MLFMA_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        p.acc.ms[r.stage] += ms;
        p.acc.launches[r.stage] += r.launches;
        if (r.stage == MLFMA_STAGE_M2L && r.level >= 0 && r.level <= kMaxLev) p.acc.m2l_ms[r.level] += ms;
        p.pool.push_back(r.a);
        p.pool.push_back(r.b);
    }
    p.recs.clear();
}

}  // namespace mlfma

extern "C" {

mlfma_status mlfma_plan_profile(mlfma_plan* plan, int enable) {
    return guarded([&] {
        if (!plan) fail(MLFMA_ERR_INVALID_ARG, "null plan");
        plan->p.profiling = enable != 0;
        for (Plan* sp : plan->p.subs) sp->profiling = enable != 0;
    });
}

mlfma_status mlfma_plan_timings(mlfma_plan* plan, mlfma_timings* out, int reset) {
    return guarded([&] {
        if (!plan || !out) fail(MLFMA_ERR_INVALID_ARG, "null plan or out");
        Plan& P = plan->p;
        check_device_errors(P);
        collect_timings(P);
        for (Plan* sp : P.subs) {
            collect_timings(*sp);
            for (int s = 0; s < MLFMA_STAGE_COUNT; ++s) {
                P.acc.ms[s] += sp->acc.ms[s];
                P.acc.launches[s] += sp->acc.launches[s];
            }
            for (int l = 0; l <= kMaxLev; ++l) P.acc.m2l_ms[l] += sp->acc.m2l_ms[l];
            memset(&sp->acc, 0, sizeof(sp->acc));
        }
        *out = P.acc;
        if (reset) memset(&P.acc, 0, sizeof(P.acc));
    });
}

}  // extern "C"
