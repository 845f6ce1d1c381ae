/*
 * gdag.h -- run-time DAG scheduling of GPU kernel launches (C ABI).
 *
 * A program issues a plain sequence of kernel launches, host writes and host
 * reads on registered arrays.  The library infers the dependency DAG from each
 * element's per-argument access modes as the elements arrive (Section III-A,
 * "Computation DAG and Dependency Sets"), runs independent elements on
 * separate CUDA streams with event waits only along DAG edges, and issues
 * host-to-device copies as DAG nodes so they overlap computation (Section
 * III-B "System Architecture", Section III-C "Scheduling Policies and Stream
 * Management").  Argument annotations follow Section III-D ("Language Design
 * and Integration").
 *
 * Conventions for every call:
 *   - returns GDAG_OK (0) or a negative GDAG_ERR_* code; gdag_last_error()
 *     gives a message for the last failing call on that context;
 *   - pointers named dev* are CUDA device pointers, host* are host pointers;
 *   - a context belongs to one host thread and is not thread-safe;
 *   - after a CUDA error that poisons the device context (a sticky error) the
 *     gdag context is poisoned and every later call returns
 *     GDAG_ERR_POISONED; gdag_destroy() still releases host resources;
 *   - host waits poll for completion against options.timeout_ms and return
 *     GDAG_ERR_TIMEOUT instead of blocking forever;
 *   - an element whose stream wait, launch, copy or event record fails with
 *     a non-sticky error still gets its node id and its edges, but is
 *     retired at once.  Before the call returns, the host waits for the
 *     element's active parents (or, when its work was issued but its event
 *     could not be recorded, for its stream), so that later elements stay
 *     ordered after them.
 */
#ifndef GDAG_H
#define GDAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define GDAG_OK             0
#define GDAG_ERR_INVALID   -1  /* bad argument, unknown handle, size error   */
#define GDAG_ERR_CUDA      -2  /* a CUDA runtime call failed (not sticky)    */
#define GDAG_ERR_TIMEOUT   -3  /* a host wait passed options.timeout_ms      */
#define GDAG_ERR_OOM       -4  /* host or pinned allocation failed           */
#define GDAG_ERR_POISONED  -5  /* an earlier sticky CUDA error               */
#define GDAG_ERR_BUSY      -6  /* array still referenced by active nodes     */
#define GDAG_ERR_NOT_FOUND -7  /* no built-in kernel of that name            */

/* ------------------------------------------------------------- policies
 * Section III-C: a serial scheduler runs elements one after the other with
 * no overlap; a parallel one lets dependencies alone order them.  A
 * synchronous one makes the host wait for every GPU element; an asynchronous
 * one does not.  The paper's baseline is serial+synchronous, its method
 * parallel+asynchronous.                                                   */
#define GDAG_POLICY_SERIAL_SYNC  0  /* one stream, host waits after each op  */
#define GDAG_POLICY_SERIAL_ASYNC 1  /* one stream, no host waits             */
#define GDAG_POLICY_PARALLEL     2  /* DAG-driven multi-stream (default)     */

#define GDAG_BACKEND_CUDA 0  /* real device                                  */
#define GDAG_BACKEND_FAKE 1  /* records operations only; runs and computes
                                nothing (scheduler tests without a GPU)      */

/* ------------------------------------------------------- access modes
 * Section III-D: "input" and "const" arguments are read-only; "output" and
 * unannotated arguments are treated as modified.  OUT is write-only for edge
 * labelling; INOUT and DEFAULT read and write.                             */
#define GDAG_MODE_DEFAULT 0
#define GDAG_MODE_IN      1
#define GDAG_MODE_CONST   2
#define GDAG_MODE_OUT     3
#define GDAG_MODE_INOUT   4
#define GDAG_MODE_SIGNATURE -1  /* gdag_arg.mode: keep the signature's mode */

/* ----------------------------------------------------------- edge kinds */
#define GDAG_EDGE_RAW 0
#define GDAG_EDGE_WAR 1
#define GDAG_EDGE_WAW 2

/* ----------------------------------------------------------- node kinds */
#define GDAG_NODE_KERNEL     0
#define GDAG_NODE_HOST_WRITE 1  /* host-to-device copy of a host write      */
#define GDAG_NODE_HOST_READ  2  /* host read (device-to-host copy if needed) */
#define GDAG_NODE_EXTERNAL   3  /* library call given the chosen stream     */
#define GDAG_NODE_HOST_PREFETCH 4 /* device-to-host copy ahead of a read    */
#define GDAG_NODE_GRAPH      5  /* replay of a captured CUDA graph          */

typedef struct gdag_ctx gdag_ctx;
typedef int32_t gdag_array;   /* array handle, >= 0                          */
typedef int32_t gdag_kernel;  /* kernel handle, >= 0                         */
typedef int32_t gdag_graph;   /* captured graph handle, >= 0                 */

typedef struct {
    uint32_t x, y, z;
} gdag_dim3;

typedef struct {
    int32_t policy;          /* GDAG_POLICY_*; default PARALLEL              */
    int32_t backend;         /* GDAG_BACKEND_*; default CUDA                 */
    int32_t device;          /* CUDA device ordinal; default 0               */
    int32_t max_streams;     /* stream pool cap; default 16                  */
    int32_t prefetch;        /* 1: host writes become asynchronous copy
                                nodes that overlap compute; 0: each host
                                write's copy completes before the call
                                returns; default 1                           */
    int32_t retire_by_query; /* 1: at each new element, parents whose event
                                has completed are retired without a host
                                wait; default 0 (the paper retires on host
                                access only)                                  */
    int32_t record_log;      /* 1: keep element, edge and op logs for the
                                export calls; 2: keep the op log only (for
                                long programs: retired readers may then be
                                dropped, see trim_nodes); default 0          */
    int32_t trace;           /* 1: timing events around every node for
                                gdag_trace_export, and an NVTX range around
                                each element's host-side issue; default 0    */
    int32_t timeout_ms;      /* host-wait deadline; default 60000            */
    int32_t trim_nodes;      /* node-table size at which retired elements
                                are dropped, so that a long-running program
                                (a serving loop that never calls gdag_sync)
                                holds memory for its active window only:
                                once the table holds this many elements, the
                                retired ones issued before the oldest active
                                element are dropped, and unless record_log
                                is 1 so are retired readers in each array's
                                reader set.  A dropped element counts as
                                retired everywhere (gdag_node_query reports
                                it done).  Scheduling is unchanged: retired
                                elements cause no waits and pick no
                                streams.  0 = 65536; ignored when trace = 1
                                (the trace keeps every element)              */
    int32_t fake_complete;   /* FAKE backend: 1 = an event reports complete
                                when queried; 0 = only after a host wait;
                                2 = never (host waits time out)              */
    int32_t fake_fail_sticky;/* FAKE backend: 1 = the injected failure is a
                                sticky (context-losing) error                */
    int64_t fake_fail_op;    /* FAKE backend: index of the backend operation
                                (launch, copy, record, wait, external) that
                                fails, -1 = none                              */
    int32_t stream_priority; /* CUDA priority of the streams the library
                                creates (lower is more urgent; CUDA clamps it
                                into the device's range): the block scheduler
                                then prefers this context's pending work, e.g.
                                a context serving short requests beside one
                                serving long ones; default 0                  */
    int32_t auto_graph;      /* N > 0: gdag_issue captures a sequence it has
                                been given N times (the same elements, arrays,
                                scalar values and copy ranges) into a CUDA
                                graph and replays it from then on; see
                                gdag_issue.  0 = off (default)               */
} gdag_options;

/* Array argument or scalar argument of a launch. */
#define GDAG_ARG_ARRAY  0
#define GDAG_ARG_SCALAR 1

typedef struct {
    int32_t kind;    /* GDAG_ARG_ARRAY or GDAG_ARG_SCALAR                    */
    int32_t mode;    /* arrays: GDAG_MODE_SIGNATURE or a GDAG_MODE_* override */
    int32_t array;   /* arrays: handle                                       */
    int32_t size;    /* scalars: bytes, 1..8 (must match the signature)      */
    uint64_t value;  /* scalars: the value's bytes, little-endian            */
} gdag_arg;

typedef struct {
    int32_t kind;    /* GDAG_ARG_ARRAY or GDAG_ARG_SCALAR                    */
    int32_t mode;    /* arrays: GDAG_MODE_*                                  */
    int32_t size;    /* scalars: bytes                                       */
    int32_t reserved;
} gdag_argspec;

/* One logical DAG edge src -> dst caused by `array`. */
typedef struct {
    int64_t src, dst;
    int32_t array;
    int32_t kind;    /* GDAG_EDGE_*                                          */
} gdag_edge;

/* One element of the program, in issue order (node ids are consecutive). */
typedef struct {
    int64_t id;
    int32_t kind;    /* GDAG_NODE_*                                          */
    int32_t stream;  /* pool index of the stream it ran on, -1 = host only   */
} gdag_node_info;

/* One recorded runtime operation (issue order). */
#define GDAG_OP_LAUNCH      0
#define GDAG_OP_COPY_H2D    1
#define GDAG_OP_COPY_D2H    2
#define GDAG_OP_EXTERNAL    3
#define GDAG_OP_RECORD      4
#define GDAG_OP_WAIT        5
#define GDAG_OP_HOST_WAIT   6
#define GDAG_OP_STREAM_SYNC 7
#define GDAG_OP_HOST_NODE   8  /* host-only element (read from the view)  */
#define GDAG_OP_QUERY_DONE  9  /* an event query found the node complete  */
typedef struct {
    int32_t type;    /* GDAG_OP_*                                            */
    int32_t stream;  /* pool index, -1 for host ops                          */
    int32_t event;   /* event slot for RECORD/WAIT/HOST_WAIT, else -1        */
    int32_t reserved;
    int64_t node;    /* node the op belongs to, -1 if none                   */
} gdag_op;

/* Timing of one node when options.trace = 1 (ms from context creation). */
typedef struct {
    int64_t node;
    int32_t kind;
    int32_t stream;
    double start_ms, end_ms;
} gdag_trace_rec;

typedef struct {
    int64_t nodes;          /* elements issued                               */
    int64_t edges;          /* logical edges inferred (a reader dropped from
                               its array's reader set gives none)           */
    int64_t waits;          /* cudaStreamWaitEvent calls issued              */
    int64_t launches;       /* kernel launches issued (all nodes)            */
    int64_t copies;         /* host<->device copies issued                   */
    int64_t host_waits;     /* host blocking waits                           */
    int32_t streams;        /* streams in the pool                           */
    int32_t active;         /* nodes currently active                        */
    int64_t fused_members;  /* launches folded into gdag_launch_fused calls  */
    int64_t held_nodes;     /* elements held in the node table               */
    int64_t held_readers;   /* reader-set entries held over all arrays       */
} gdag_stats;

/* ------------------------------------------------------------ lifetime */

/* Fill *o with the defaults listed in gdag_options, then apply environment
 * overrides where set to an integer: GDAG_POLICY, GDAG_MAX_STREAMS,
 * GDAG_PREFETCH, GDAG_RETIRE_BY_QUERY, GDAG_RECORD_LOG, GDAG_TRACE,
 * GDAG_TIMEOUT_MS, GDAG_DEVICE, GDAG_TRIM_NODES, GDAG_STREAM_PRIORITY,
 * GDAG_AUTO_GRAPH (a caller may still change any field before gdag_create,
 * which validates them). */
void gdag_options_default(gdag_options *o);

/* Create a context.  opts may be NULL (defaults).  With the CUDA backend the
 * device is made current; streams are created lazily and owned by the
 * library.  They are ordinary (blocking) streams, so device work the caller
 * issued on the legacy default stream before an element (for example a fill
 * of a freshly allocated scratch array) is ordered before it.  Errors:
 * INVALID, CUDA, OOM. */
int gdag_create(gdag_ctx **out, const gdag_options *opts);
/* Concurrency note: CUDA maps streams onto CUDA_DEVICE_MAX_CONNECTIONS
 * hardware work queues (8 unless the environment sets it).  Streams that
 * share a queue are serialised behind each other's cross-stream waits when
 * the host issues far ahead of the device, so a process using more than 8
 * pool streams should set CUDA_DEVICE_MAX_CONNECTIONS=32 before it creates
 * its CUDA context (the Python binding does so at import). */

/* Wait for all work (bounded by timeout_ms), then free every library-owned
 * stream, event and pinned buffer.  Caller-owned memory is not touched. */
int gdag_destroy(gdag_ctx *ctx);

/* Message of the last failing call on ctx ("" if none).  Owned by ctx. */
const char *gdag_last_error(gdag_ctx *ctx);

/* Add a caller-owned CUDA stream (cudaStream_t) to the pool; the library
 * uses it like its own but never destroys it.  INVALID past max_streams. */
int gdag_add_stream(gdag_ctx *ctx, void *stream);

/* --------------------------------------------------------------- arrays
 * Section III-A: arrays are managed objects, so dependency identity is array
 * identity (no aliasing between distinct handles).
 *
 * Register `bytes` of device memory at dev (non-owning; the caller keeps it
 * alive until unregister).  host is an optional caller-owned pinned host
 * buffer of the same size used as the array's host view; if NULL, the library
 * allocates one (cudaHostAlloc) on the first host access.  Errors: INVALID
 * (dev NULL with bytes > 0). */
int gdag_array_register(gdag_ctx *ctx, void *dev, size_t bytes, void *host,
                        gdag_array *out);

/* Wait (bounded) for every active element that uses the array, then forget
 * it; frees the library-owned host view. */
int gdag_array_unregister(gdag_ctx *ctx, gdag_array a);

/* Host view of the array (allocating it if needed).  mode GDAG_MODE_IN:
 * waits until the view holds the array's current contents (a host read of
 * the whole array).  mode GDAG_MODE_OUT: waits until no copy in flight reads
 * the view, so the caller may overwrite it and then call gdag_array_write
 * with src = NULL.  Section III-A: a host access that conflicts with active
 * GPU work waits for it. */
int gdag_array_host(gdag_ctx *ctx, gdag_array a, int32_t mode, void **out);

/* Host write of [off, off+bytes) (Sections III-A and III-C).  src == NULL, or
 * src equal to the host view + off: the caller already wrote the view.
 * Otherwise src is copied into the view first (after any copy in flight from
 * that region completes); src may be reused when the call returns.  The
 * device copy is a DAG node that writes the array: it waits on the GPU for
 * the array's active readers (WAR) or writer (WAW), never on the host.
 * Errors: INVALID (range), TIMEOUT, CUDA. */
int gdag_array_write(gdag_ctx *ctx, gdag_array a, const void *src, size_t off,
                     size_t bytes);

/* Host read of [off, off+bytes) into dst (dst == NULL or equal to host view
 * + off: leave it in the view).  If the device holds newer data than the
 * view, a device-to-host copy runs after the array's last writer and the
 * host waits for it; that node and all its ancestors become inactive
 * (Section III-B: computations stay active until the host needs their result
 * or a child's).  Errors: INVALID, TIMEOUT, CUDA. */
int gdag_array_read(gdag_ctx *ctx, gdag_array a, void *dst, size_t off,
                    size_t bytes);

/* Start copying [off, off+bytes) of the array to its host view without
 * waiting (a DAG element that reads the array, placed like a kernel: after
 * the array's last writer, as the first child on the writer's stream when it
 * can be).  A later gdag_array_read inside that range, with no GPU write to
 * the array in between, waits for this copy instead of issuing its own.  The
 * device-to-host counterpart of the automatic host-to-device prefetch of
 * Section III-C; on a full-duplex host link, result copies then overlap the
 * input copies of other branches.  The caller must not touch the host view
 * until a read (or gdag_array_host) returns.  Errors: INVALID, CUDA. */
int gdag_array_prefetch_host(gdag_ctx *ctx, gdag_array a, size_t off,
                             size_t bytes);

/* -------------------------------------------------------------- kernels
 * Built-in sm_103a kernels (the DAG nodes of the Section IV-B benchmarks).
 * Arguments in order; modes IN / OUT / INOUT as in Section III-D; scalars
 * i32 (4 bytes), i64 or f32 as given; arrays are device buffers of the
 * stated element type, row-major.  A launch whose sizes do not fit its
 * buffers fails with INVALID before anything is queued.
 *
 *  VEC   vec_square      (x INOUT f32[n], n i64)                 x := x*x
 *        vec_reduce_diff (x IN f32[n], y IN f32[n], z OUT f32[1],
 *                         scratch INOUT, n i64)                  z = sum(x-y)
 *  B&S   bs_call         (S IN f32[n], C OUT f32[n], n i64, K f32, r f32,
 *                         sigma f32, T f32)                      call prices
 *                         K, sigma, T > 0; an explicit launch shape takes
 *                         blocks of at most 256 threads
 *  IMG   gauss_blur      (img IN f32[rows*cols], out OUT, w IN f32[2R+1],
 *                         rows i32, cols i32, R i32)    separable, clamped
 *                         rows, cols >= 1; R 1..8
 *        sobel           (in IN, out OUT, rows i32, cols i32)    magnitude
 *                         rows, cols >= 1
 *        minmax          (x IN f32[n], mm OUT f32[2], scratch INOUT, n i64)
 *                         n >= 1
 *        extend          (x INOUT f32[n], mm IN f32[2], n i64)
 *                                               x := (x-min)/(max-min) or 0
 *        unsharp         (img IN, blur IN, out OUT, alpha f32, n i64)
 *        combine         (s IN, b5 IN, b9 IN, e5 IN, e9 IN, out OUT, n i64)
 *  ML    dense_scores    (X IN i32[rows*feats], table IN f32[feats*classes],
 *                         bias IN f32[classes], S OUT f32[rows*classes],
 *                         rows i32, feats i32, classes i32)  S = X table + b
 *                         classes 1..16, feats a multiple of 32 with
 *                         feats * ceil(classes/4) <= 12796 (the table is
 *                         held in shared memory), X 16-byte
 *                         aligned; feats a multiple of 64 up to 1024 runs on
 *                         the tensor cores (exact products: X in bf16, the
 *                         table as three bf16 pieces; 128-row tiles holding
 *                         any |x| > 256 are recomputed on CUDA cores)
 *        row_softmax     (S INOUT f32[rows*classes], rows i32, classes i32)
 *                         classes 1..32
 *        argmax_combine  (P1 IN, P2 IN, labels OUT i32[rows], rows i32,
 *                         classes i32)                 argmax(P1+P2), lowest
 *                         classes >= 1
 *  HITS  spmv_partition  (rowptr IN i32[n+1], part OUT, n i32, nnz i32)
 *        spmv_csr        (rowptr IN, col IN i32[nnz], val IN f32[nnz],
 *                         x IN f32[n], part IN, y OUT f32[n], carry INOUT,
 *                         n i32, nnz i32)                         y = A x
 *                         The index data is not checked (only sizes are):
 *                         rowptr must rise from 0 to nnz, every col entry
 *                         must lie in [0, n), and part must come from
 *                         spmv_partition of the same rowptr; a col entry
 *                         outside x is an out-of-bounds device read
 *        l2norm          (x IN f32[n], norm OUT f32[1], scratch INOUT, n i64)
 *        scale           (x INOUT f32[n], norm IN f32[1], n i64)
 *                                                x := x/norm (norm 0: kept)
 *        seg_l2norm      (x IN f32[n], seg IN i32[G+1], norms OUT f32[G],
 *                         scratch INOUT, G i32, n i32)
 *                         norms[g] = ||x[seg[g] .. seg[g+1])||, for a batch
 *                         of graphs stored block-diagonally; G <= 65535,
 *                         x 16-byte aligned (also for seg_scale)
 *        seg_scale       (x INOUT f32[n], seg IN i32[G+1], norms IN f32[G],
 *                         G i32, n i32)  x := x/norms[g] on segment g
 *                         (norm 0: kept); segment bounds are clamped to n
 *  DL    conv3x3_relu_pool (x IN bf16[n*3*h*w], wt IN bf16[64*3*3*3],
 *                         bias IN f32[64], out OUT bf16[n*64*(h/2)*(w/2)],
 *                         status INOUT i32[1], n i32, h i32, w i32)
 *                         3x3 conv (zero pad 1) + bias + ReLU + 2x2 max-pool
 *                         on the tensor cores; n >= 1, h >= 2 even, w >= 8
 *                         a multiple of 8, x
 *                         and out 16-byte aligned; status := 1 if a tensor-core
 *                         or copy wait timed out (the output is then
 *                         incomplete), 2 if the kernel's shared-memory window
 *                         was not 128-byte aligned (nothing computed)
 *        avgpool_global  (p IN bf16[planes*hw], e OUT f32[planes],
 *                         planes i32, hw i32)               plane means
 *                         planes, hw >= 1
 *        concat_dense    (e1 IN f32[n*c], e2 IN f32[n*c],
 *                         wd IN f32[2c*classes], bd IN f32[classes],
 *                         out OUT f32[n*classes], n i32, c i32, classes i32)
 *                                                  out = [e1 e2] wd + bd
 *                         n, c, classes >= 1
 * Scratch and part/carry sizes come from gdag_scratch_bytes.
 * Errors: NOT_FOUND. */
int gdag_kernel_lookup(gdag_ctx *ctx, const char *name, gdag_kernel *out);

/* Number of arguments of kernel k and its signature (spec may be NULL). */
int gdag_kernel_signature(gdag_ctx *ctx, gdag_kernel k, int32_t *nargs,
                          gdag_argspec *spec, int32_t cap);

/* Register a user kernel: fn is a __global__ function's host handle usable
 * with cudaLaunchKernel; spec gives each argument's kind, access mode
 * (Section III-D annotations) and scalar size.  nargs <= 16. */
int gdag_kernel_register(gdag_ctx *ctx, const char *name, const void *fn,
                         int32_t nargs, const gdag_argspec *spec,
                         gdag_kernel *out);

/* Launch kernel k as a DAG element (Section III-A, III-B).  grid = {0,0,0}
 * lets a built-in kernel pick its own launch shape (block and smem are then
 * ignored).  For every array argument the dependency sets are updated and
 * edges inferred; the stream is chosen by the policy (first child on its
 * parent's stream, else the oldest empty stream, else a new one up to
 * max_streams, else the least recently used); the stream waits on the events
 * of active parents on other streams; the node records its own event.
 * Never blocks the host except under GDAG_POLICY_SERIAL_SYNC.  *node_out
 * (may be NULL) receives the node id.  Errors: INVALID (unknown array or
 * kernel, argument count or kind mismatch), CUDA. */
int gdag_launch(gdag_ctx *ctx, gdag_kernel k, gdag_dim3 grid, gdag_dim3 block,
                size_t smem, const gdag_arg *args, int32_t nargs,
                int64_t *node_out);

/* Fused launch (kernel consolidation, Section II: merging independent
 * kernels into one launch raises utilization).  `count` launches of built-in
 * kernel k, given as count consecutive argument lists of nargs arguments
 * each (args[m*nargs .. m*nargs+nargs-1] is member m, exactly as it would be
 * passed to gdag_launch), become ONE DAG element and one persistent kernel
 * launch that walks every member's work.  The element's accesses are the
 * union of the members' (a write dominates), so it gets every edge any
 * member would get and each member's result is what its own gdag_launch
 * would give, bit for bit (elementwise members trivially; reductions keep
 * the member's own block partition and combine order).  Members use the
 * kernel's automatic launch shape.  Kernels with a fused form: vec_square,
 * vec_reduce_diff, bs_call.  1 <= count <= GDAG_FUSED_MAX; members beyond the
 * kernel's per-launch table (GDAG_FUSED_TABLE) go to further launches of the
 * same element, back to back on its stream.  Errors: INVALID (kernel without
 * a fused form, a member that gdag_launch would reject, or an array written
 * by one member and used by another), CUDA. */
#define GDAG_FUSED_MAX   4096
#define GDAG_FUSED_TABLE 128
int gdag_launch_fused(gdag_ctx *ctx, gdag_kernel k, const gdag_arg *args,
                      int32_t nargs, int32_t count, int64_t *node_out);

/* Launch kernel k on the caller's CUDA stream with no dependency tracking
 * (hand-scheduled baselines and graph capture).  Arrays are resolved to their
 * device pointers only. */
int gdag_launch_raw(gdag_ctx *ctx, gdag_kernel k, gdag_dim3 grid,
                    gdag_dim3 block, size_t smem, const gdag_arg *args,
                    int32_t nargs, void *stream);

/* A library call as a DAG element (Section III-A: pre-registered library
 * functions are scheduled asynchronously when they take a stream).  fn is
 * called once on the host with the chosen cudaStream_t and user, before this
 * call returns (the library keeps neither afterwards); it must only enqueue
 * work on that stream.  arrays/modes give its accesses. */
int gdag_launch_external(gdag_ctx *ctx, void (*fn)(void *stream, void *user),
                         void *user, const gdag_array *arrays,
                         const int32_t *modes, int32_t n, int64_t *node_out);

/* ------------------------------------------------------ batched issue
 * Section III-B: the runtime sees a program as a stream of element
 * requests, and the host-side cost of each sits on the critical path of
 * short DAGs (the comparison with CUDA Graphs, Section IV-D, finds the
 * runtime's overhead negligible only for computations longer than a few
 * milliseconds).  gdag_issue takes several consecutive
 * non-blocking elements of a program in one call; element i is inferred,
 * placed and issued exactly as its own call would be (gdag_launch,
 * gdag_launch_fused, gdag_array_write with src NULL, or
 * gdag_array_prefetch_host), in order, so the DAG, the streams, the waits
 * and the results are those of the single calls.                         */
#define GDAG_ELEM_LAUNCH        0  /* gdag_launch                            */
#define GDAG_ELEM_LAUNCH_FUSED  1  /* gdag_launch_fused                      */
#define GDAG_ELEM_WRITE         2  /* gdag_array_write(a, NULL, off, bytes):
                                      the host view already holds the data  */
#define GDAG_ELEM_PREFETCH_HOST 3  /* gdag_array_prefetch_host(a, off, bytes) */
typedef struct {
    int32_t type;     /* GDAG_ELEM_*                                         */
    int32_t kernel;   /* LAUNCH, LAUNCH_FUSED: kernel handle                 */
    int32_t array;    /* WRITE, PREFETCH_HOST: array handle                  */
    int32_t nargs;    /* LAUNCH: arguments; LAUNCH_FUSED: arguments per member */
    int32_t count;    /* LAUNCH_FUSED: members (args holds count * nargs)    */
    uint32_t smem;    /* LAUNCH: dynamic shared memory, bytes                */
    int64_t arg0;     /* LAUNCH, LAUNCH_FUSED: index in args of the first one */
    uint64_t off;     /* WRITE, PREFETCH_HOST: byte offset                   */
    uint64_t bytes;   /* WRITE, PREFETCH_HOST: byte count                    */
    gdag_dim3 grid;   /* LAUNCH: {0,0,0} = the kernel's automatic shape      */
    gdag_dim3 block;  /* LAUNCH                                              */
} gdag_elem;

/* Issue elems[0..n) in order.  args holds nargs_total gdag_arg entries that
 * the launch elements index (arg0 .. arg0 + nargs*count - 1 must lie inside
 * it).  nodes_out (may be NULL) receives each element's node id, or -1 for
 * an element that made no node (a prefetch of a view that is already
 * current, or an element not issued).  *issued (may be NULL) receives the
 * number of elements handled before the first failure (n on success).  On
 * a failure the call returns that element's error at once: the elements
 * before it stay issued, the failing one behaves as its single call does
 * on that error, and the ones after it are not issued.  Never blocks the
 * host except where a single call would (policy SERIAL_SYNC, prefetch = 0,
 * both staging uses of a view in flight).  Errors: INVALID (an element
 * type, index range, or anything its single call rejects), CUDA, TIMEOUT,
 * POISONED. */
/* Automatic capture of repeated sequences (options.auto_graph = N > 0; the
 * repeated DAG shapes of Section IV-D's CUDA-graph comparison, captured and
 * replayed without the caller marking them).  gdag_issue keys each sequence
 * by its elements and the argument entries they use (arg0 itself excluded):
 *   - the first N - 1 successful issues of a key run as described above;
 *   - the N-th issue waits for all work (as gdag_capture_begin does), records
 *     the sequence into a graph (nothing runs) and replays it; every later
 *     issue of the key replays the graph (gdag_graph_launch: one DAG element
 *     whose accesses are the union of the sequence's, so a later element
 *     that touches any array of the sequence waits for the whole replay);
 *     nodes_out then receives the replay's node for every element, and
 *     *issued is n on success, 0 on failure;
 *   - host writes in a replay copy what the array's host view holds when the
 *     copy runs, as their single calls do;
 *   - a graph whose arrays were registered again at another address or size
 *     is dropped (after a wait for all work) and its key starts over; a
 *     sequence that fails inside its capture is issued as above, now and
 *     from then on;
 *   - at most GDAG_AUTO_GRAPH_SEQS keys are kept: a new key beyond that
 *     drops the least recently used one and its graph (after a wait for all
 *     work);
 *   - never captured: sequences holding a prefetch to the host, issues under
 *     SERIAL_SYNC, with trace = 1, or inside an open gdag_capture_begin. */
#define GDAG_AUTO_GRAPH_SEQS 64
int gdag_issue(gdag_ctx *ctx, const gdag_elem *elems, int32_t n,
               const gdag_arg *args, int64_t nargs_total, int64_t *nodes_out,
               int32_t *issued);

/* ----------------------------------------------------------------- sync */

/* Wait for every stream (bounded) and retire every node; the retired nodes
 * then leave the node table (unless options.trace = 1) as under trim_nodes,
 * which changes no later dependency or wait.  Errors: TIMEOUT (a stream did
 * not finish within timeout_ms), POISONED, INVALID while capturing. */
int gdag_sync(gdag_ctx *ctx);

/* Non-blocking: *done = 1 if node's work has completed (it and its
 * ancestors are then retired, as after a host wait), 0 if it is still
 * running.  Lets a dispatcher poll many in-flight DAGs without blocking on
 * any (Section III-B: results become available when the host asks).
 * Errors: INVALID (unknown node, or while capturing), CUDA. */
int gdag_node_query(gdag_ctx *ctx, int64_t node, int32_t *done);

/* gdag_node_query for nodes[0..n): done[i] receives node i's completion
 * flag.  One call lets a dispatcher poll every in-flight DAG without a host
 * round trip per node.  Errors: as gdag_node_query, for the first failing
 * node (later flags are then unset). */
int gdag_nodes_query(gdag_ctx *ctx, const int64_t *nodes, int32_t n,
                     int32_t *done);

/* Make the caller's CUDA stream wait for all work issued so far, without
 * blocking the host (a join for timing events or stream capture). */
int gdag_stream_wait_all(gdag_ctx *ctx, void *stream);

/* Make every pool stream wait for the caller's stream's work issued so far
 * (a fork: later nodes run after it). */
int gdag_stream_fork(gdag_ctx *ctx, void *stream);

/* ------------------------------------------------ captured DAG shapes
 * A program that repeats the same sequence of elements can record it once
 * as a CUDA graph and replay it; the replay is one DAG element, so it mixes
 * with dynamically scheduled elements.  (Section II names the up-front,
 * static DAG of CUDA Graphs as the alternative the paper's scheduler avoids;
 * this keeps the dynamic inference and adds replay of a shape that is known
 * to repeat.)
 *
 * gdag_capture_begin waits for all work (as gdag_sync), then records instead
 * of executing: every element issued until gdag_capture_end is inferred and
 * placed on streams as usual, and its launches, copies, event records and
 * waits become the nodes and edges of one graph.  While capturing, host
 * reads, prefetches, waits, syncs and unregistering return GDAG_ERR_INVALID,
 * and host writes must copy from the array's host view (src NULL): a replay
 * copies whatever the view holds at replay time.  Needs an asynchronous
 * policy.  gdag_capture_end instantiates the graph; nothing captured has
 * run.  Errors: INVALID, CUDA. */
int gdag_capture_begin(gdag_ctx *ctx);
int gdag_capture_end(gdag_ctx *ctx, gdag_graph *out);

/* Replay graph g as one DAG element whose accesses are the union of the
 * captured elements' accesses (edges, stream choice and waits as for a
 * kernel).  The arrays must still be registered, at the device address,
 * size and (where the array had one at capture) host view they had at
 * capture, since the graph holds those addresses; otherwise
 * GDAG_ERR_INVALID. */
int gdag_graph_launch(gdag_ctx *ctx, gdag_graph g, int64_t *node_out);

/* Wait for all work, then free graph g. */
int gdag_graph_destroy(gdag_ctx *ctx, gdag_graph g);

/* ---------------------------------------------------------- inspection */

/* Copy up to cap records; *n receives the total available.  The edge and
 * element logs need options.record_log = 1, the op log record_log = 1 or 2
 * (INVALID otherwise). */
int gdag_dag_export(gdag_ctx *ctx, gdag_edge *buf, size_t cap, size_t *n);
int gdag_nodes_export(gdag_ctx *ctx, gdag_node_info *buf, size_t cap,
                      size_t *n);
int gdag_ops_export(gdag_ctx *ctx, gdag_op *buf, size_t cap, size_t *n);

/* Timing records (options.trace = 1); waits for completion first. */
int gdag_trace_export(gdag_ctx *ctx, gdag_trace_rec *buf, size_t cap,
                      size_t *n);

/* Write the timing records (options.trace = 1; waits for completion first)
 * to the file at path as a Chrome trace (JSON, for chrome://tracing or
 * Perfetto): one complete event per node, named after its kernel or its
 * kind, on one track per pool stream, in microseconds from context
 * creation.  The trace of Section IV-F's overlap analysis.  Errors: INVALID
 * (tracing off, or the file cannot be written), CUDA. */
int gdag_trace_write(gdag_ctx *ctx, const char *path);

int gdag_stats_get(gdag_ctx *ctx, gdag_stats *out);

/* Bytes of scratch the built-in reductions (vec_reduce_diff, minmax, l2norm)
 * and spmv_csr need for `n` elements (for seg_l2norm, n is the number of
 * segments G); the scratch array must be zeroed once before its first use
 * and is left zeroed-counter by every launch. */
size_t gdag_scratch_bytes(const char *kernel, int64_t n);

/* ------------------------------------------------- allocation-free entry
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory: plug-ins whose host application owns every
 * device allocation, processes whose device memory is budgeted by an
 * allocator they must not bypass, and latency-critical loops that cannot
 * afford cudaMalloc/cudaFree (which may synchronize the device).
 *
 * gdag_vec_reduce_diff_noalloc computes *dev_z = sum_i (dev_x[i] - dev_y[i])
 * over n floats (the VEC reduction, same kernel and same result as launching
 * "vec_reduce_diff" through gdag_launch) on the caller's CUDA stream, without
 * a context and without allocating: the caller passes the inputs and the
 * one-float output, and the kernel's scratch (per-block partial sums and an
 * arrival counter) is a fixed file-scope device array of
 * GDAG_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  No cudaMalloc, cudaFree or allocating library routine
 * is called.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address and keeps it for the life of the process; make
 *     that first call before any stream capture on the device.  It issues no
 *     GPU work: every call enqueues only on the caller's stream (a clear of
 *     the arrival counter, then the kernel), so the first call is ordered
 *     like any other, on blocking and non-blocking streams alike.
 *   - The cached address is not refreshed: do not call this entry point on a
 *     device after cudaDeviceReset() on it in the same process.
 *   - Every call shares the one array per device and leaves the last call's
 *     partial sums in it; each call clears the counter it needs on its own
 *     stream first, and every partial sum is written before it is read.
 *     Calls whose kernels overlap on the GPU (different streams, or
 *     different host threads, without ordering) race on the array: order
 *     them on one stream or with events.
 *   - The array holds 1024 partial sums and the counter, the most any launch
 *     of this reduction uses: its grid is capped at 1024 blocks whatever n
 *     is, and a compile-time check ties the array's size to that cap, so no
 *     size is too large.  A negative n, or a NULL pointer, is rejected with
 *     GDAG_ERR_INVALID before anything is enqueued.
 *   - Returns GDAG_ERR_CUDA if the set-up or the launch fails. */
#define GDAG_NOALLOC_SCRATCH_BYTES 16384
int gdag_vec_reduce_diff_noalloc(const void *dev_x, const void *dev_y,
                                 void *dev_z, int64_t n, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GDAG_H */
