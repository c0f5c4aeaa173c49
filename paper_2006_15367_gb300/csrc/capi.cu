// C ABI of the MLFMA library: argument checks, plan lifetime, host/device staging.
#include <chrono>
#include <cmath>
#include <cstdarg>
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

void Allocator::release_all() {
    for (auto& a : live) {
        if (free) free(a.first, (void*)stream, ctx);
        else cudaFree(a.first);
    }
    live.clear();
    bytes = 0;
}

size_t csize(const Plan& p) { return p.prec == MLFMA_PREC_FP64 ? 16 : 8; }

static bool is_device_ptr(const void* ptr) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void ensure_apply_buffers(Plan& p, int nrhs) {
    if (nrhs <= p.nrhs_cap) return;
    // buffers are only ever grown; old ones stay owned by the plan until destroy
    p.qs = p.mem.get((size_t)nrhs * p.n * csize(p));
    p.phis = p.mem.get((size_t)nrhs * p.n * csize(p));
    p.nrhs_cap = nrhs;
}

static void apply_impl(Plan& p, const void* q, void* phi, int nrhs, bool adjoint, void* grad = nullptr) {
    if (!q || (!phi && !grad)) fail(MLFMA_ERR_INVALID_ARG, "null q or phi");
    if (nrhs < 1) fail(MLFMA_ERR_INVALID_ARG, "nrhs must be >= 1 (got %d)", nrhs);
    const size_t bytes = (size_t)nrhs * p.n * csize(p);
    const bool dq = is_device_ptr(q), dphi = phi ? is_device_ptr(phi) : true;
    if (grad && (!dq || !dphi || !is_device_ptr(grad)))
        fail(MLFMA_ERR_INVALID_ARG, "mlfma_apply_grad takes device pointers only");
    ensure_apply_buffers(p, nrhs);
    if (grad && p.nrhs_grad < nrhs) {
        p.grads = p.mem.get((size_t)3 * nrhs * p.n * csize(p));
        p.nrhs_grad = nrhs;
    }
    const void* qd = q;
    void* phid = phi;
    if (!dq || !dphi) {
        if (p.nrhs_stage < nrhs) {
            p.host_stage = p.mem.get(2 * bytes);
            p.nrhs_stage = nrhs;
        }
        if (!dq) {
            MLFMA_CUDA(cudaMemcpyAsync(p.host_stage, q, bytes, cudaMemcpyHostToDevice, p.stream));
            qd = p.host_stage;
        }
        if (!dphi) phid = (char*)p.host_stage + bytes;
    }
    {
        StageTimer st(p, MLFMA_STAGE_PERMUTE, 0, 1);
        permute_in(p, qd, p.qs, nrhs, adjoint);
    }
    for (int r = 0; r < nrhs; ++r)
        apply_pipeline(p, (const char*)p.qs + (size_t)r * p.n * csize(p), (char*)p.phis + (size_t)r * p.n * csize(p),
                       grad ? (char*)p.grads + (size_t)3 * r * p.n * csize(p) : nullptr);
    {
        StageTimer st(p, MLFMA_STAGE_PERMUTE, 0, 1);
        if (phid) permute_out(p, p.phis, phid, nrhs, adjoint);
        if (grad) permute_out3(p, p.grads, grad, nrhs);
    }
    if (p.profiling) p.acc.applies += nrhs;
    if (!dphi) {
        MLFMA_CUDA(cudaMemcpyAsync(phi, phid, bytes, cudaMemcpyDeviceToHost, p.stream));
        MLFMA_CUDA(cudaStreamSynchronize(p.stream));
    } else if (!dq) {
        MLFMA_CUDA(cudaStreamSynchronize(p.stream));
    }
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
    opt->digit_margin = 1;
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
        if (!(k > 0.0) || !std::isfinite(k)) fail(MLFMA_ERR_INVALID_ARG, "k must be finite and > 0");
        if (digits < 1 || digits > 12) fail(MLFMA_ERR_INVALID_ARG, "digits must be in [1, 12] (got %d)", digits);
        if (leaf_max < 0) fail(MLFMA_ERR_INVALID_ARG, "leaf_max must be >= 0");
        mlfma_options o;
        mlfma_options_init(&o);
        if (opt) {
            if (opt->struct_size < sizeof(mlfma_options)) fail(MLFMA_ERR_INVALID_ARG, "options.struct_size too small");
            o = *opt;
        }
        if (o.precision != MLFMA_PREC_FP64 && o.precision != MLFMA_PREC_FP32)
            fail(MLFMA_ERR_INVALID_ARG, "unknown precision %d", (int)o.precision);
        if (o.max_depth < 1 || o.max_depth > kMaxLev) fail(MLFMA_ERR_INVALID_ARG, "max_depth must be in [1, %d]", kMaxLev);
        if (o.digit_margin < 0 || o.digit_margin > 8) fail(MLFMA_ERR_INVALID_ARG, "digit_margin must be in [0, 8]");
        if (!std::isfinite(o.leaf_edge)) fail(MLFMA_ERR_INVALID_ARG, "leaf_edge must be finite");
        if ((o.alloc == nullptr) != (o.free == nullptr)) fail(MLFMA_ERR_INVALID_ARG, "alloc and free must be given together");
        h = new mlfma_plan();
        Plan& p = h->p;
        p.n = n;
        p.k = k;
        p.digits = digits;
        p.leaf_max = leaf_max;
        p.max_depth = o.max_depth;
        p.margin = o.digit_margin;
        p.prec = o.precision;
        p.leaf_edge = o.leaf_edge > 0 ? o.leaf_edge : (digits <= 4 ? 0.5 * M_PI / k : M_PI / k);
        p.stream = (cudaStream_t)o.stream;
        p.mem.alloc = o.alloc;
        p.mem.free = o.free;
        p.mem.ctx = o.alloc_ctx;
        p.mem.stream = p.stream;
        const double* pts = points;
        if (!is_device_ptr(points)) {
            double* d = p.mem.make<double>(3 * n);
            MLFMA_CUDA(cudaMemcpyAsync(d, points, 3 * n * sizeof(double), cudaMemcpyHostToDevice, p.stream));
            pts = d;
        }
        build_tree(p, pts);
        build_lists(p);
        build_far_levels(p);
        build_m2l_lists(p);
        p.near_dump = p.mem.get(p.n * csize(p));
        ensure_apply_buffers(p, 1);
        MLFMA_CUDA(cudaStreamSynchronize(p.stream));
        p.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        *out = h;
    });
    if (st != MLFMA_OK && h) {
        cudaStreamSynchronize(h->p.stream);
        h->p.mem.release_all();
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

mlfma_status mlfma_plan_info(const mlfma_plan* plan, mlfma_info* info) {
    return guarded([&] {
        if (!plan || !info) fail(MLFMA_ERR_INVALID_ARG, "null plan or info");
        const Plan& p = plan->p;
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
    });
}

mlfma_status mlfma_plan_export(const mlfma_plan* plan, int item, int level, void* dst, size_t bytes, size_t* needed) {
    return guarded([&] {
        if (!plan) fail(MLFMA_ERR_INVALID_ARG, "null plan");
        const Plan& p = plan->p;
        const bool per_level = item >= MLFMA_EXPORT_BOX_KEY && item != MLFMA_EXPORT_NEAR_OFFSETS &&
                               item != MLFMA_EXPORT_NEAR_SOURCES && item != MLFMA_EXPORT_NEAR_PHI;
        if (per_level && (level < 1 || level > p.nlev)) fail(MLFMA_ERR_INVALID_ARG, "level %d outside 1..%d", level, p.nlev);
        const TreeLevel* L = per_level ? &p.lev[level] : nullptr;
        const bool far_item = item == MLFMA_EXPORT_F || item == MLFMA_EXPORT_G || item == MLFMA_EXPORT_TRANSLATION;
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
            case MLFMA_EXPORT_TRANSLATION: parts.push_back({p.far[level].T, kNumOffsets * p.far[level].K * csize(p)}); break;
            default: fail(MLFMA_ERR_INVALID_ARG, "unknown export item %d", item);
        }
        size_t tot = 0;
        for (auto& x : parts) tot += x.second;
        if (needed) *needed = tot;
        if (!dst) return;
        if (bytes < tot) fail(MLFMA_ERR_INVALID_ARG, "buffer of %zu bytes < %zu needed", bytes, tot);
        MLFMA_CUDA(cudaStreamSynchronize(p.stream));
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
    cudaStreamSynchronize(plan->p.stream);
    for (auto& r : plan->p.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : plan->p.pool) cudaEventDestroy(e);
    plan->p.mem.release_all();
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

StageTimer::StageTimer(Plan& plan, int stage, int level, int launches) : p(plan) {
    if (!p.profiling) return;
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
    });
}

mlfma_status mlfma_plan_timings(mlfma_plan* plan, mlfma_timings* out, int reset) {
    return guarded([&] {
        if (!plan || !out) fail(MLFMA_ERR_INVALID_ARG, "null plan or out");
        collect_timings(plan->p);
        *out = plan->p.acc;
        if (reset) memset(&plan->p.acc, 0, sizeof(plan->p.acc));
    });
}

}  // extern "C"
