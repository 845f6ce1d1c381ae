// The runtime's only view of the device: the "intermediate layer exposing the
// CUDA API" of Section III-B.  Two implementations: CUDA (real device) and a
// recording fake that computes nothing (scheduler tests without a GPU).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include "catalog.h"

namespace gdag {

// Result of a backend call.
enum BeStatus : int {
    BE_OK = 0,
    BE_NOT_READY = 1,   // event_query: still running
    BE_ERROR = -1,      // failed, context still usable
    BE_STICKY = -2,     // failed, device context lost
};

class Backend {
  public:
    virtual ~Backend() {}
    virtual int init(int device) = 0;
    virtual int stream_create(void **s, int priority) = 0;
    virtual int stream_destroy(void *s) = 0;
    virtual int event_create(void **e, bool timing) = 0;
    virtual int event_destroy(void *e) = 0;
    virtual int event_record(void *e, void *s) = 0;
    virtual int stream_wait(void *s, void *e) = 0;
    virtual int event_query(void *e) = 0;
    virtual int event_elapsed_ms(void *e0, void *e1, float *ms) = 0;
    virtual int stream_query(void *s) = 0;
    // Completion as seen by a blocking host wait (the fake completes its work
    // when the host waits, unless it models a hang).
    virtual int wait_query_event(void *e) { return event_query(e); }
    virtual int wait_query_stream(void *s) { return stream_query(s); }
    virtual int launch(const KernelEntry &k, const LaunchArgs &a, void *s) = 0;
    virtual int launch_fused(const KernelEntry &k, const LaunchArgs *a, int count, void *s) = 0;
    virtual int copy_h2d(void *dst, const void *src, size_t bytes, void *s) = 0;
    virtual int copy_d2h(void *dst, const void *src, size_t bytes, void *s) = 0;
    virtual int external(void (*fn)(void *, void *), void *user, void *s) = 0;
    // Stream capture into a CUDA graph and its replay.
    virtual int capture_begin(void *s) = 0;
    virtual int capture_end(void *s, void **exec) = 0;  // instantiated graph
    virtual int graph_launch(void *exec, void *s) = 0;
    virtual int graph_destroy(void *exec) = 0;
    virtual int host_alloc(void **p, size_t bytes) = 0;
    virtual int host_free(void *p) = 0;
    virtual bool is_fake() const = 0;
    // Message of the last failure.
    std::string err;
};

Backend *make_cuda_backend();
Backend *make_fake_backend(int complete_on_query, int64_t fail_op, int fail_sticky);

}  // namespace gdag
