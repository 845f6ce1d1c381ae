// CUDA runtime backend and the recording fake.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <string>

#include "backend.h"

namespace gdag {
namespace {

// Sticky errors leave the CUDA context unusable; everything else is local to
// the failing call.
bool is_sticky(cudaError_t e)
{
    switch (e) {
    case cudaErrorIllegalAddress:
    case cudaErrorLaunchFailure:
    case cudaErrorIllegalInstruction:
    case cudaErrorMisalignedAddress:
    case cudaErrorInvalidAddressSpace:
    case cudaErrorInvalidPc:
    case cudaErrorHardwareStackError:
    case cudaErrorAssert:
    case cudaErrorLaunchTimeout:
    case cudaErrorECCUncorrectable:
    case cudaErrorContextIsDestroyed:
        return true;
    default:
        return false;
    }
}

class CudaBackend final : public Backend {
  public:
    int chk(cudaError_t e, const char *what)
    {
        if (e == cudaSuccess) return BE_OK;
        err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
        if (is_sticky(e)) return BE_STICKY;
        (void)cudaGetLastError();  // clear a non-sticky error
        return BE_ERROR;
    }
    int init(int device) override
    {
        int n = 0;
        int r = chk(cudaGetDeviceCount(&n), "cudaGetDeviceCount");
        if (r) return r;
        if (device < 0 || device >= n) {
            err = "device ordinal out of range";
            return BE_ERROR;
        }
        return chk(cudaSetDevice(device), "cudaSetDevice");
    }
    int stream_create(void **s, int priority) override
    {
        // blocking streams: device work the caller put on the legacy default
        // stream (allocation fills, copies by the framework that owns the
        // memory) is ordered before anything issued here afterwards
        cudaStream_t st;
        int r = chk(cudaStreamCreateWithPriority(&st, cudaStreamDefault, priority), "cudaStreamCreate");
        if (!r) *s = st;
        return r;
    }
    int stream_destroy(void *s) override { return chk(cudaStreamDestroy((cudaStream_t)s), "cudaStreamDestroy"); }
    int event_create(void **e, bool timing) override
    {
        cudaEvent_t ev;
        int r = chk(cudaEventCreateWithFlags(&ev, timing ? cudaEventDefault : cudaEventDisableTiming),
                    "cudaEventCreate");
        if (!r) *e = ev;
        return r;
    }
    int event_destroy(void *e) override { return chk(cudaEventDestroy((cudaEvent_t)e), "cudaEventDestroy"); }
    int event_record(void *e, void *s) override
    {
        return chk(cudaEventRecord((cudaEvent_t)e, (cudaStream_t)s), "cudaEventRecord");
    }
    int stream_wait(void *s, void *e) override
    {
        return chk(cudaStreamWaitEvent((cudaStream_t)s, (cudaEvent_t)e, 0), "cudaStreamWaitEvent");
    }
    int event_query(void *e) override
    {
        cudaError_t r = cudaEventQuery((cudaEvent_t)e);
        if (r == cudaErrorNotReady) return BE_NOT_READY;
        return chk(r, "cudaEventQuery");
    }
    int event_elapsed_ms(void *e0, void *e1, float *ms) override
    {
        return chk(cudaEventElapsedTime(ms, (cudaEvent_t)e0, (cudaEvent_t)e1), "cudaEventElapsedTime");
    }
    int stream_query(void *s) override
    {
        cudaError_t r = cudaStreamQuery((cudaStream_t)s);
        if (r == cudaErrorNotReady) return BE_NOT_READY;
        return chk(r, "cudaStreamQuery");
    }
    int launch(const KernelEntry &k, const LaunchArgs &a, void *s) override
    {
        if (k.launcher) {
            cudaError_t e = (cudaError_t)k.launcher(a, s);
            if (e == cudaSuccess) e = cudaGetLastError();
            return chk(e, k.name.c_str());
        }
        void *argp[kMaxArgs];
        for (int i = 0; i < a.nargs; ++i) {
            if (k.spec[i].kind == GDAG_ARG_ARRAY)
                argp[i] = (void *)&a.ptr[i];
            else
                argp[i] = (void *)&a.val[i];
        }
        dim3 g(a.grid[0], a.grid[1], a.grid[2]), b(a.block[0], a.block[1], a.block[2]);
        return chk(cudaLaunchKernel(k.fn, g, b, argp, a.smem, (cudaStream_t)s), k.name.c_str());
    }
    int launch_fused(const KernelEntry &k, const LaunchArgs *a, int count, void *s) override
    {
        cudaError_t e = (cudaError_t)k.fused(a, count, s);
        if (e == cudaSuccess) e = cudaGetLastError();
        return chk(e, k.name.c_str());
    }
    int copy_h2d(void *dst, const void *src, size_t bytes, void *s) override
    {
        return chk(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, (cudaStream_t)s), "cudaMemcpyAsync H2D");
    }
    int copy_d2h(void *dst, const void *src, size_t bytes, void *s) override
    {
        return chk(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, (cudaStream_t)s), "cudaMemcpyAsync D2H");
    }
    int external(void (*fn)(void *, void *), void *user, void *s) override
    {
        fn(s, user);
        return chk(cudaGetLastError(), "external call");
    }
    int capture_begin(void *s) override
    {
        return chk(cudaStreamBeginCapture((cudaStream_t)s, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    }
    int capture_end(void *s, void **exec) override
    {
        cudaGraph_t g = nullptr;
        int r = chk(cudaStreamEndCapture((cudaStream_t)s, &g), "cudaStreamEndCapture");
        if (r) return r;
        cudaGraphExec_t ge = nullptr;
        r = chk(cudaGraphInstantiate(&ge, g, 0), "cudaGraphInstantiate");
        cudaGraphDestroy(g);
        if (!r) *exec = ge;
        return r;
    }
    int graph_launch(void *exec, void *s) override
    {
        return chk(cudaGraphLaunch((cudaGraphExec_t)exec, (cudaStream_t)s), "cudaGraphLaunch");
    }
    int graph_destroy(void *exec) override { return chk(cudaGraphExecDestroy((cudaGraphExec_t)exec), "cudaGraphExecDestroy"); }
    int host_alloc(void **p, size_t bytes) override
    {
        return chk(cudaHostAlloc(p, bytes ? bytes : 1, cudaHostAllocPortable), "cudaHostAlloc");
    }
    int host_free(void *p) override { return chk(cudaFreeHost(p), "cudaFreeHost"); }
    bool is_fake() const override { return false; }
};

// Records nothing itself (the runtime keeps the op log); hands out distinct
// fake handles, counts operations and fails the configured one.
class FakeBackend final : public Backend {
  public:
    FakeBackend(int complete, int64_t fail_op, int sticky)
        : complete_(complete), fail_op_(fail_op), sticky_(sticky) {}
    int op()
    {
        int64_t i = count_++;
        if (i == fail_op_) {
            err = "injected failure at op " + std::to_string(i);
            return sticky_ ? BE_STICKY : BE_ERROR;
        }
        return BE_OK;
    }
    int init(int) override { return BE_OK; }
    int stream_create(void **s, int) override
    {
        *s = (void *)(uintptr_t)(0x1000 + next_++);
        return BE_OK;
    }
    int stream_destroy(void *) override { return BE_OK; }
    int event_create(void **e, bool) override
    {
        *e = (void *)(uintptr_t)(0x100000 + next_++);
        return BE_OK;
    }
    int event_destroy(void *) override { return BE_OK; }
    int event_record(void *, void *) override { return op(); }
    int stream_wait(void *, void *) override { return op(); }
    // complete_: 1 = every event reports done when queried; 0 = only a host
    // wait completes it; 2 = nothing ever completes (a hung device).
    int event_query(void *) override { return complete_ == 1 ? BE_OK : BE_NOT_READY; }
    int wait_query_event(void *) override { return complete_ == 2 ? BE_NOT_READY : BE_OK; }
    int wait_query_stream(void *) override { return complete_ == 2 ? BE_NOT_READY : BE_OK; }
    int event_elapsed_ms(void *, void *, float *ms) override
    {
        *ms = 0.f;
        return BE_OK;
    }
    int stream_query(void *) override { return complete_ == 1 ? BE_OK : BE_NOT_READY; }
    int launch(const KernelEntry &, const LaunchArgs &, void *) override { return op(); }
    int launch_fused(const KernelEntry &, const LaunchArgs *, int, void *) override { return op(); }
    int copy_h2d(void *, const void *, size_t, void *) override { return op(); }
    int copy_d2h(void *, const void *, size_t, void *) override { return op(); }
    int external(void (*fn)(void *, void *), void *user, void *s) override
    {
        fn(s, user);  // as the CUDA backend does: the caller enqueues nothing real here
        return op();
    }
    int capture_begin(void *) override { return BE_OK; }
    int capture_end(void *, void **exec) override
    {
        *exec = (void *)(uintptr_t)(0x200000 + next_++);
        return BE_OK;
    }
    int graph_launch(void *, void *) override { return op(); }
    int graph_destroy(void *) override { return BE_OK; }
    int host_alloc(void **p, size_t bytes) override
    {
        *p = std::malloc(bytes ? bytes : 1);
        if (!*p) {
            err = "malloc failed";
            return BE_ERROR;
        }
        return BE_OK;
    }
    int host_free(void *p) override
    {
        std::free(p);
        return BE_OK;
    }
    bool is_fake() const override { return true; }

  private:
    int complete_;
    int64_t fail_op_;
    int sticky_;
    int64_t count_ = 0;
    uintptr_t next_ = 0;
};

}  // namespace

Backend *make_cuda_backend() { return new CudaBackend(); }
Backend *make_fake_backend(int complete, int64_t fail_op, int sticky)
{
    return new FakeBackend(complete, fail_op, sticky);
}

}  // namespace gdag
