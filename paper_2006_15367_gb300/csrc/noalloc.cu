// Near-field potential for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc once they are running: code inside a
// real-time loop or another library's callback where an allocation would stall or
// is not permitted, or a process whose memory budget was fixed at start-up.  They
// create their plan during set-up and then need every later call to allocate
// nothing.  mlfma_apply may allocate on a first call or when given host pointers;
// this entry point never does.  Its scratch (the charges and potentials in the
// plan's Morton order) lives in a file-scope __device__ array of fixed size that
// every GPU loading this library holds until the process exits.
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB: 2 * n complex values
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
// device address of the array per device, with the context it was looked up in
struct ScratchAddr {
    CUcontext ctx = nullptr;
    void* ptr = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];

using CtxGetCurrent = CUresult (*)(CUcontext*);

CUcontext current_context() {
    static CtxGetCurrent get = nullptr;
    if (!get) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        MLFMA_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn) mlfma::fail(MLFMA_ERR_CUDA, "cuCtxGetCurrent is not available");
        get = (CtxGetCurrent)fn;
    }
    CUcontext ctx = nullptr;
    if (get(&ctx) != CUDA_SUCCESS || !ctx) mlfma::fail(MLFMA_ERR_CUDA, "no current CUDA context");
    return ctx;
}

// A device pointer of the current device.  A pointer into another GPU's memory is refused:
// this device's kernels would dereference it, which needs peer access.
bool device_pointer(const void* ptr, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

// The array's name is only a host-side stand-in.  Its device address is looked up with the
// device current on the first call in each context: the first call on a device, and again
// after that device's context was destroyed and re-created (cudaDeviceReset).
void* scratch_on_current_device(int dev) {
    if (dev < 0 || dev >= kMaxDevices) mlfma::fail(MLFMA_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    const CUcontext ctx = current_context();
    std::lock_guard<std::mutex> lock(g_mu);
    ScratchAddr& a = g_scratch_addr[dev];
    if (!a.ptr || a.ctx != ctx) {
        void* ptr = nullptr;
        MLFMA_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        a.ctx = ctx;
        a.ptr = ptr;
    }
    return a.ptr;
}

}  // namespace

extern "C" mlfma_status mlfma_apply_near_noalloc(mlfma_plan* plan, const void* q, void* phi) {
    try {
        mlfma::set_error("%s", "");
        if (!plan || !q || !phi) mlfma::fail(MLFMA_ERR_INVALID_ARG, "null plan, q or phi");
        mlfma::Plan& p = plan->p;
        if (!p.subs.empty()) mlfma::fail(MLFMA_ERR_INVALID_ARG, "batched plans are not supported here");
        int dev = 0;
        MLFMA_CUDA(cudaGetDevice(&dev));
        if (!device_pointer(q, dev) || !device_pointer(phi, dev))
            mlfma::fail(MLFMA_ERR_INVALID_ARG,
                        "q and phi must be device pointers of the current device (host staging would allocate)");
        const size_t half = (size_t)p.n * mlfma::csize(p);
        if (2 * half > kNoAllocScratchBytes)
            mlfma::fail(MLFMA_ERR_INVALID_ARG, "n = %lld needs %zu bytes of scratch; the maximum is %zu bytes",
                        (long long)p.n, 2 * half, kNoAllocScratchBytes);
        unsigned char* scratch = static_cast<unsigned char*>(scratch_on_current_device(dev));
        void* qs = scratch;
        void* phis = scratch + half;
        // every sorted slot of qs and phis is written before it is read: nothing needs clearing
        mlfma::permute_in(p, q, qs, 1, false);
        // no stage events: a profiled plan's timings cover its applies only
        mlfma::near_only(p, qs, phis, false);
        mlfma::permute_out(p, phis, phi, 1, false);
        return MLFMA_OK;
    } catch (const mlfma::Failure& e) {
        return e.status;
    }
}
