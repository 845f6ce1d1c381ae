// Dependency tracker, stream manager and C ABI of libgdag.
//
// Section III-A (Computation DAG and dependency sets): every kernel launch,
// host array access and library call is a computational element.  For each
// array the tracker keeps the last writer W and the readers R since W; a
// reader gets an edge from W; a writer gets edges from every reader in R, or
// from W when R is empty, and then becomes the new W with R emptied.  This is
// the paper's dependency-set rule (a read-only use adds an edge but does not
// remove the argument from the parent's set; a later writer depends on all
// readers, not on the writer).
//
// Section III-B (System Architecture): elements stay active until the host
// needs their result or a child's; only active parents cause waits.
//
// Section III-C (Scheduling Policies and Stream Management): the first child
// of a parent runs on the parent's stream; otherwise the oldest empty stream
// is reused (FIFO), a new stream is created only if none is empty, and one
// event per element provides the cross-stream synchronization.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "backend.h"
#include "catalog.h"
#include "gdag.h"

namespace gdag {
namespace {

constexpr int R_BIT = 1, W_BIT = 2;

int mode_bits(int mode)
{
    switch (mode) {
    case GDAG_MODE_IN:
    case GDAG_MODE_CONST:
        return R_BIT;
    case GDAG_MODE_OUT:
        return W_BIT;
    default:  // INOUT and unannotated: read and modified
        return R_BIT | W_BIT;
    }
}

struct Node {
    int32_t kind = 0;
    int32_t stream = -1;
    int32_t event = -1;       // pooled event slot (active nodes only)
    int32_t tev0 = -1, tev1 = -1;  // timing events (trace)
    int32_t label = -1;       // kernel handle of a kernel node (trace names)
    bool active = false;
    bool first_child_taken = false;
    uint32_t parent_off = 0, parent_cnt = 0;
    int64_t parent_of = -1;   // last element that took this node as a parent
};

struct ArrayState {
    void *dev = nullptr;
    size_t bytes = 0;
    void *host = nullptr;
    bool host_owned = false;
    bool live = false;
    bool host_valid = false;  // host view holds the current contents
    int64_t writer = -1;
    std::vector<int64_t> readers;
    int64_t view_copy = -1;   // last copy node reading or writing the view
    int64_t prefetch = -1;    // pending device-to-host prefetch node
    int64_t pf_writer = -1;   // the array's writer when it was issued
    size_t pf_off = 0, pf_bytes = 0;
};

struct StreamState {
    void *handle = nullptr;
    bool owned = true;
    int64_t tail = -1;
    int32_t active = 0;
    uint64_t last_use = 0;
    bool queued = false;
};

struct Access {
    int32_t array;
    int32_t bits;
};

}  // namespace

struct Ctx {
    gdag_options opt;
    std::unique_ptr<Backend> be;
    std::string last_error;
    bool poisoned = false;

    std::vector<KernelEntry> kernels;
    std::vector<ArrayState> arrays;
    std::vector<int32_t> free_arrays;

    // node table: ids [base, base + nodes.size())
    int64_t base = 0;
    std::deque<Node> nodes;
    std::vector<int64_t> parent_arena;
    int64_t active_count = 0;
    size_t trim_at = 0;  // node-table size of the next trim check
    int64_t reader_entries = 0;  // sum of the arrays' reader-set sizes

    std::vector<StreamState> streams;
    std::deque<int32_t> free_streams;  // empty streams, oldest first
    uint64_t tick = 0;

    std::vector<void *> events;      // pooled (non-timing)
    std::vector<int32_t> free_events;
    std::vector<void *> tevents;     // timing events (trace), never reused
    void *t0 = nullptr;              // trace time base

    // logs
    std::vector<gdag_edge> edge_log;
    std::vector<gdag_node_info> node_log;
    std::vector<gdag_op> op_log;
    gdag_stats st{};

    // scratch for one element
    std::vector<int64_t> par;

    // stream capture (CUDA graphs of a repeated DAG shape)
    bool capturing = false;
    void *cap_stream = nullptr;
    std::vector<Access> cap_access;  // union of the captured elements' accesses
    struct Graph {
        void *exec = nullptr;
        std::vector<Access> access;
        // each accessed array's device and host pointers and size at capture
        // time: the graph's copies and launches hold these addresses
        std::vector<const void *> dev, host;
        std::vector<size_t> bytes;
        bool live = false;
    };
    std::vector<Graph> graphs;

    // automatic capture of repeated gdag_issue sequences (options.auto_graph)
    struct AutoSeq {
        uint64_t hash = 0;
        std::vector<uint64_t> key;  // the sequence's elements and the arguments they use
        int32_t seen = 0;           // dynamic issues of it so far
        int32_t graph = -1;         // its graph, once captured
        bool never = false;         // its capture failed: always issued dynamically
        uint64_t used = 0;          // last use, for least-recently-used eviction
    };
    std::vector<AutoSeq> auto_seqs;
    uint64_t auto_clock = 0;

    // the graph still holds the addresses and sizes its arrays have now
    bool graph_current(int32_t g) const
    {
        if (g < 0 || (size_t)g >= graphs.size() || !graphs[(size_t)g].live) return false;
        const Graph &gr = graphs[(size_t)g];
        for (size_t i = 0; i < gr.access.size(); ++i) {
            const int32_t a = gr.access[i].array;
            if (a < 0 || (size_t)a >= arrays.size() || !arrays[(size_t)a].live) return false;
            const ArrayState &st = arrays[(size_t)a];
            if (st.dev != gr.dev[i] || (gr.host[i] && st.host != gr.host[i]) || st.bytes != gr.bytes[i]) return false;
        }
        return true;
    }

    void capture_note(const Access *acc, int n)
    {
        if (!capturing) return;
        for (int i = 0; i < n; ++i) {
            size_t j = 0;
            while (j < cap_access.size() && cap_access[j].array != acc[i].array) ++j;
            if (j == cap_access.size()) cap_access.push_back(acc[i]);
            else cap_access[j].bits |= acc[i].bits;
        }
    }

    // ------------------------------------------------------------- errors
    int fail(int code, const char *fmt, ...)
    {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        last_error = buf;
        return code;
    }
    int be_fail(int r, const char *what)
    {
        if (r == BE_STICKY) poisoned = true;
        return fail(r == BE_STICKY ? GDAG_ERR_POISONED : GDAG_ERR_CUDA, "%s: %s", what, be->err.c_str());
    }

    void log_op(int type, int stream, int event, int64_t node)
    {
        if (opt.record_log && !capturing) op_log.push_back(gdag_op{type, stream, event, 0, node});
    }

    // ------------------------------------------------------------- nodes
    Node *node(int64_t id)
    {
        if (id < base || id >= base + (int64_t)nodes.size()) return nullptr;
        return &nodes[(size_t)(id - base)];
    }
    int64_t next_id() const { return base + (int64_t)nodes.size(); }

    int acquire_event(int32_t *slot)
    {
        if (!free_events.empty()) {
            *slot = free_events.back();
            free_events.pop_back();
            return GDAG_OK;
        }
        void *e;
        int r = be->event_create(&e, false);
        if (r) return be_fail(r, "event create");
        events.push_back(e);
        *slot = (int32_t)events.size() - 1;
        return GDAG_OK;
    }

    // Mark one active node inactive: its event slot and its stream's share
    // are released.  Returns false if it was not active.
    bool deactivate(Node *n)
    {
        if (!n || !n->active) return false;
        n->active = false;
        --active_count;
        if (n->event >= 0) {
            free_events.push_back(n->event);
            n->event = -1;
        }
        if (n->stream >= 0) {
            StreamState &s = streams[(size_t)n->stream];
            if (--s.active == 0 && !s.queued) {
                s.queued = true;
                free_streams.push_back(n->stream);
            }
        }
        return true;
    }

    // Retire node id and all its active ancestors (their results are
    // complete once the host has observed id's completion).
    void retire(int64_t id)
    {
        std::vector<int64_t> stack{id};
        while (!stack.empty()) {
            int64_t v = stack.back();
            stack.pop_back();
            Node *n = node(v);
            if (!deactivate(n)) continue;
            for (uint32_t k = 0; k < n->parent_cnt; ++k) stack.push_back(parent_arena[n->parent_off + k]);
        }
    }

    void retire_all()
    {
        for (size_t i = 0; i < nodes.size(); ++i)
            if (nodes[i].active) retire(base + (int64_t)i);
    }

    // Host wait for node id (bounded); retires it and its ancestors.
    int host_wait(int64_t id)
    {
        Node *n = node(id);
        if (!n || !n->active) return GDAG_OK;
        if (capturing) return fail(GDAG_ERR_INVALID, "a host wait is not possible while capturing");
        if (n->event < 0) {
            retire(id);
            return GDAG_OK;
        }
        log_op(GDAG_OP_HOST_WAIT, n->stream, n->event, id);
        ++st.host_waits;
        int r = poll_event(events[(size_t)n->event]);
        if (r) return r;
        retire(id);
        return GDAG_OK;
    }

    int poll_event(void *ev)
    {
        auto t_end = std::chrono::steady_clock::now() + std::chrono::milliseconds(opt.timeout_ms);
        unsigned spins = 0;
        for (;;) {
            int q = be->wait_query_event(ev);
            if (q == BE_OK) return GDAG_OK;
            if (q != BE_NOT_READY) return be_fail(q, "event query");
            if (++spins > 64) {
                if (std::chrono::steady_clock::now() > t_end)
                    return fail(GDAG_ERR_TIMEOUT, "host wait exceeded %d ms", opt.timeout_ms);
                std::this_thread::yield();
            }
        }
    }

    int poll_stream(int32_t s)
    {
        auto t_end = std::chrono::steady_clock::now() + std::chrono::milliseconds(opt.timeout_ms);
        unsigned spins = 0;
        for (;;) {
            int q = be->wait_query_stream(streams[(size_t)s].handle);
            if (q == BE_OK) return GDAG_OK;
            if (q != BE_NOT_READY) return be_fail(q, "stream query");
            if (++spins > 64) {
                if (std::chrono::steady_clock::now() > t_end)
                    return fail(GDAG_ERR_TIMEOUT, "stream sync exceeded %d ms", opt.timeout_ms);
                std::this_thread::yield();
            }
        }
    }

    // ------------------------------------------------------------ streams
    int new_stream(int32_t *out)
    {
        void *h;
        int r = be->stream_create(&h, opt.stream_priority);
        if (r) return be_fail(r, "stream create");
        StreamState s;
        s.handle = h;
        streams.push_back(s);
        *out = (int32_t)streams.size() - 1;
        if (capturing) {  // a stream created during capture joins it
            int rr = fork_from(cap_stream, h);
            if (rr) return rr;
        }
        if (opt.trace && !t0) {
            int rr = be->event_create(&t0, true);
            if (rr) return be_fail(rr, "event create");
            rr = be->event_record(t0, h);
            if (rr) return be_fail(rr, "event record");
        }
        return GDAG_OK;
    }

    // Section III-C stream choice for a new element with parents `par`.
    int pick_stream(int32_t *out)
    {
        if (opt.policy != GDAG_POLICY_PARALLEL) {
            if (streams.empty()) {
                int r = new_stream(out);
                if (r) return r;
            }
            *out = 0;
            return GDAG_OK;
        }
        // first child on a parent's stream: the parent must be active, be
        // the last work issued on its stream, and have no child there yet
        for (int64_t p : par) {
            Node *n = node(p);
            if (!n || !n->active || n->stream < 0) continue;
            if (streams[(size_t)n->stream].tail == p && !n->first_child_taken) {
                n->first_child_taken = true;
                *out = n->stream;
                return GDAG_OK;
            }
        }
        // oldest empty stream
        while (!free_streams.empty()) {
            int32_t s = free_streams.front();
            free_streams.pop_front();
            streams[(size_t)s].queued = false;
            if (streams[(size_t)s].active == 0) {
                *out = s;
                return GDAG_OK;
            }
        }
        if ((int)streams.size() < opt.max_streams) return new_stream(out);
        // cap reached: least recently used stream
        int32_t best = 0;
        for (size_t i = 1; i < streams.size(); ++i)
            if (streams[i].last_use < streams[(size_t)best].last_use) best = (int32_t)i;
        *out = best;
        return GDAG_OK;
    }

    // --------------------------------------------------------- tracking
    // Every edge is logged; only an active source becomes a parent of dst.
    // A retired one is complete and observed: it needs no wait, picks no
    // stream and ends the retirement walk, so leaving it out of the parent
    // list changes nothing but the list's length (which, for a writer after
    // many readers, would otherwise grow with every read ever issued).
    void add_edge(int64_t src, int64_t dst, int32_t a, int32_t kind)
    {
        ++st.edges;
        if (opt.record_log == 1) edge_log.push_back(gdag_edge{src, dst, a, kind});
        Node *n = node(src);
        if (n && n->active && n->parent_of != dst) {
            n->parent_of = dst;
            par.push_back(src);
        }
    }

    // Section III-A dependency rule for element `id` with accesses acc.
    void infer(int64_t id, const Access *acc, int n)
    {
        par.clear();
        for (int i = 0; i < n; ++i) {
            ArrayState &s = arrays[(size_t)acc[i].array];
            int bits = acc[i].bits;
            if (!(bits & W_BIT)) {
                if (s.writer >= 0) add_edge(s.writer, id, acc[i].array, GDAG_EDGE_RAW);
                s.readers.push_back(id);
                ++reader_entries;
            } else {
                if (!s.readers.empty()) {
                    for (int64_t r : s.readers) add_edge(r, id, acc[i].array, GDAG_EDGE_WAR);
                } else if (s.writer >= 0) {
                    add_edge(s.writer, id, acc[i].array, (bits & R_BIT) ? GDAG_EDGE_RAW : GDAG_EDGE_WAW);
                }
                s.writer = id;
                reader_entries -= (int64_t)s.readers.size();
                s.readers.clear();
            }
        }
        std::sort(par.begin(), par.end());
    }

    // Append the node for element `id` (after infer()).
    void push_node(int32_t kind)
    {
        trim();
        Node nd;
        nd.kind = kind;
        nd.parent_off = (uint32_t)parent_arena.size();
        nd.parent_cnt = (uint32_t)par.size();
        parent_arena.insert(parent_arena.end(), par.begin(), par.end());
        nodes.push_back(nd);
        ++st.nodes;
        if (opt.record_log == 1) node_log.push_back(gdag_node_info{next_id() - 1, kind, -1});
    }

    // Drop the retired elements issued before the oldest active one, once
    // the node table holds opt.trim_nodes elements.  Nothing needs them:
    // node() of a dropped id is null, which every lookup reads as retired
    // (complete), and the parent lists hold active nodes only.  Unless the
    // edge log is kept, the dropped ids also leave the reader sets (each
    // sorted by id), where they would only have produced edges to retired
    // elements.  The next check comes when the table has grown to twice
    // what is left, so the scans cost O(1) per element.
    void trim(bool now = false)
    {
        if (opt.trace || (!now && nodes.size() < trim_at)) return;
        size_t f = 0;
        while (f < nodes.size() && !nodes[f].active) ++f;
        if (f > 0) {
            const size_t keep = f < nodes.size() ? nodes[f].parent_off : parent_arena.size();
            parent_arena.erase(parent_arena.begin(), parent_arena.begin() + (std::ptrdiff_t)keep);
            for (size_t i = f; i < nodes.size(); ++i) nodes[i].parent_off -= (uint32_t)keep;
            nodes.erase(nodes.begin(), nodes.begin() + (std::ptrdiff_t)f);
            base += (int64_t)f;
            if (opt.record_log != 1)
                for (auto &a : arrays) {
                    auto keep = std::lower_bound(a.readers.begin(), a.readers.end(), base);
                    reader_entries -= (int64_t)(keep - a.readers.begin());
                    a.readers.erase(a.readers.begin(), keep);
                }
        }
        trim_at = std::max((size_t)opt.trim_nodes, 2 * nodes.size());
    }

    // Make stream `to` wait for the work issued so far on `from`.
    int fork_from(void *from, void *to)
    {
        void *e;
        int r = be->event_create(&e, false);
        if (r) return be_fail(r, "event create");
        r = be->event_record(e, from);
        if (!r) r = be->stream_wait(to, e);
        be->event_destroy(e);
        if (r) return be_fail(r, "fork");
        return GDAG_OK;
    }

    // Optionally retire completed parents without a host wait.
    int retire_done_parents()
    {
        if (!opt.retire_by_query || capturing) return GDAG_OK;
        for (int64_t p : par) {
            Node *n = node(p);
            if (!n || !n->active || n->event < 0) continue;
            int q = be->event_query(events[(size_t)n->event]);
            if (q == BE_OK) {
                log_op(GDAG_OP_QUERY_DONE, n->stream, n->event, p);
                retire(p);
            }
            else if (q != BE_NOT_READY)
                return be_fail(q, "event query");
        }
        return GDAG_OK;
    }

    // Choose the stream, issue waits on active parents of other streams
    // (only the latest parent per stream), mark the node active there.
    int place(int64_t id, int32_t *stream_out)
    {
        int r = retire_done_parents();
        if (r) return r;
        int32_t s;
        r = pick_stream(&s);
        if (r) return r;
        // waits: latest active parent per other stream
        int64_t latest[64];
        int nl = 0;
        int32_t lstream[64];
        for (int64_t p : par) {
            Node *n = node(p);
            if (!n || !n->active || n->stream < 0 || n->stream == s || n->event < 0) continue;
            int k = 0;
            while (k < nl && lstream[k] != n->stream) ++k;
            if (k == nl) {
                if (nl == 64) {  // more streams than the table: wait directly
                    int rr = wait_on(s, p);
                    if (rr) return rr;
                    continue;
                }
                lstream[nl] = n->stream;
                latest[nl++] = p;
            } else if (p > latest[k]) {
                latest[k] = p;
            }
        }
        for (int k = 0; k < nl; ++k) {
            r = wait_on(s, latest[k]);
            if (r) return r;
        }
        Node *me = node(id);
        me->stream = s;
        me->active = true;
        ++active_count;
        StreamState &ss = streams[(size_t)s];
        if (ss.queued) {  // taken from the FIFO by the LRU path: drop it
            ss.queued = false;
            free_streams.erase(std::find(free_streams.begin(), free_streams.end(), s));
        }
        ss.active++;
        ss.tail = id;
        ss.last_use = ++tick;
        if (opt.record_log == 1) node_log.back().stream = s;
        *stream_out = s;
        if (opt.trace) {
            void *e;
            r = be->event_create(&e, true);
            if (r) return be_fail(r, "event create");
            tevents.push_back(e);
            me->tev0 = (int32_t)tevents.size() - 1;
            r = be->event_record(e, ss.handle);
            if (r) return be_fail(r, "event record");
        }
        return GDAG_OK;
    }

    int wait_on(int32_t s, int64_t p)
    {
        Node *n = node(p);
        log_op(GDAG_OP_WAIT, s, n->event, p);
        ++st.waits;
        int r = be->stream_wait(streams[(size_t)s].handle, events[(size_t)n->event]);
        if (r) return be_fail(r, "stream wait");
        return GDAG_OK;
    }

    // After the node's work op: record its event; under SERIAL_SYNC wait.
    int finish(int64_t id, int32_t s)
    {
        int r = record_end(id, s);
        if (r) return unrecorded(id, s, r);
        if (opt.policy == GDAG_POLICY_SERIAL_SYNC) return host_wait(id);
        return GDAG_OK;
    }

    int record_end(int64_t id, int32_t s)
    {
        int r;
        if (opt.trace) {
            void *e;
            r = be->event_create(&e, true);
            if (r) return be_fail(r, "event create");
            tevents.push_back(e);
            node(id)->tev1 = (int32_t)tevents.size() - 1;
            r = be->event_record(e, streams[(size_t)s].handle);
            if (r) return be_fail(r, "event record");
        }
        int32_t slot;
        r = acquire_event(&slot);
        if (r) return r;
        node(id)->event = slot;
        log_op(GDAG_OP_RECORD, s, slot, id);
        r = be->event_record(events[(size_t)slot], streams[(size_t)s].handle);
        if (r) return be_fail(r, "event record");
        return GDAG_OK;
    }

    // The node's work was issued but its event was not recorded, so no
    // later element could wait for it.  The host waits for its stream
    // instead (the work and, through the stream's waits, the node's
    // parents) and retires it; if that wait fails too, only the node is
    // retired.  The error `rc` and its message are kept.
    int unrecorded(int64_t id, int32_t s, int rc)
    {
        const std::string msg = last_error;
        bool done = capturing || poisoned;
        if (!done) {
            log_op(GDAG_OP_STREAM_SYNC, s, -1, -1);
            ++st.host_waits;
            done = poll_stream(s) == GDAG_OK;
        }
        if (done) retire(id);
        else deactivate(node(id));
        last_error = msg;
        return rc;
    }

    // An element whose placement or work op failed stays in the DAG as a
    // retired element.  Its work never ran, so nothing it would have ordered
    // is known to be complete: later elements that conflict with its
    // parents only through it (a reader of an array it was to overwrite,
    // say) would get no wait.  So the host first waits for its active
    // parents (`par` still holds them), which retires them truthfully, and
    // only then retires the element itself.  If such a wait fails, only the
    // element is retired.  The error `rc` and its message are kept.
    int drop_failed(int64_t id, int rc)
    {
        const std::string msg = last_error;
        bool waited = true;
        if (!capturing && !poisoned) {
            const std::vector<int64_t> ps(par);
            for (size_t i = 0; i < ps.size() && waited; ++i) waited = host_wait(ps[i]) == GDAG_OK;
        }
        if (waited) retire(id);
        else deactivate(node(id));
        last_error = msg;
        return rc;
    }
    int abort_node(int64_t id, int r, const char *what) { return drop_failed(id, be_fail(r, what)); }

    // ------------------------------------------------------------ arrays
    ArrayState *arr(int32_t a)
    {
        if (a < 0 || (size_t)a >= arrays.size() || !arrays[(size_t)a].live) return nullptr;
        return &arrays[(size_t)a];
    }

    int ensure_host(ArrayState &s)
    {
        if (s.host) return GDAG_OK;
        int r = be->host_alloc(&s.host, s.bytes);
        if (r) return fail(GDAG_ERR_OOM, "pinned host allocation of %zu bytes failed: %s", s.bytes, be->err.c_str());
        s.host_owned = true;
        return GDAG_OK;
    }

    // Wait until no copy in flight reads or writes the host view.
    int release_view(ArrayState &s)
    {
        if (s.view_copy >= 0) {
            Node *n = node(s.view_copy);
            if (n && n->active) {
                int r = host_wait(s.view_copy);
                if (r) return r;
            }
            s.view_copy = -1;
        }
        return GDAG_OK;
    }

    int guard()
    {
        if (poisoned) return fail(GDAG_ERR_POISONED, "context poisoned by an earlier sticky CUDA error");
        return GDAG_OK;
    }
};

}  // namespace gdag

// With options.trace set, an NVTX range marks the host-side issue of each
// element (named after its kernel or its kind), so a system profiler shows
// the library's issue timeline next to the device work.
struct IssueRange {
    bool on;
    IssueRange(const gdag::Ctx *c, const char *name) : on(c && c->opt.trace)
    {
        if (on) nvtxRangePushA(name);
    }
    ~IssueRange()
    {
        if (on) nvtxRangePop();
    }
};

using gdag::Access;
using gdag::ArrayState;
using gdag::Ctx;
using gdag::KernelEntry;
using gdag::LaunchArgs;

struct gdag_ctx : Ctx {};

template <class T>
static int export_vec(gdag_ctx *c, const std::vector<T> &v, T *buf, size_t cap, size_t *n, bool op_log = false)
{
    if (!c || !n) return GDAG_ERR_INVALID;
    if (!(c->opt.record_log == 1 || (op_log && c->opt.record_log == 2)))
        return c->fail(GDAG_ERR_INVALID, op_log ? "the op log needs options.record_log = 1 or 2"
                                                : "edge and element logs need options.record_log = 1");
    *n = v.size();
    if (buf)
        for (size_t i = 0; i < v.size() && i < cap; ++i) buf[i] = v[i];
    return GDAG_OK;
}

extern "C" {

void gdag_options_default(gdag_options *o)
{
    std::memset(o, 0, sizeof *o);
    o->policy = GDAG_POLICY_PARALLEL;
    o->backend = GDAG_BACKEND_CUDA;
    o->device = 0;
    o->max_streams = 16;
    o->prefetch = 1;
    o->retire_by_query = 0;
    o->record_log = 0;
    o->trace = 0;
    o->timeout_ms = 60000;
    o->trim_nodes = 0;
    o->fake_complete = 0;
    o->fake_fail_sticky = 0;
    o->fake_fail_op = -1;
    // environment overrides of the defaults (an unset or unparsable value
    // keeps the default)
    struct {
        const char *name;
        int32_t *field;
    } env[] = {{"GDAG_POLICY", &o->policy},           {"GDAG_MAX_STREAMS", &o->max_streams},
               {"GDAG_PREFETCH", &o->prefetch},       {"GDAG_RETIRE_BY_QUERY", &o->retire_by_query},
               {"GDAG_RECORD_LOG", &o->record_log},   {"GDAG_TRACE", &o->trace},
               {"GDAG_TIMEOUT_MS", &o->timeout_ms}, {"GDAG_DEVICE", &o->device},
               {"GDAG_TRIM_NODES", &o->trim_nodes}, {"GDAG_STREAM_PRIORITY", &o->stream_priority},
               {"GDAG_AUTO_GRAPH", &o->auto_graph}};
    for (const auto &e : env) {
        const char *v = std::getenv(e.name);
        if (!v || !*v) continue;
        char *end = nullptr;
        const long x = std::strtol(v, &end, 10);
        if (end && *end == '\0' && x >= INT32_MIN && x <= INT32_MAX) *e.field = (int32_t)x;
    }
}

int gdag_create(gdag_ctx **out, const gdag_options *opts)
{
    if (!out) return GDAG_ERR_INVALID;
    *out = nullptr;
    gdag_options o;
    if (opts)
        o = *opts;
    else
        gdag_options_default(&o);
    if (o.policy < 0 || o.policy > 2 || o.max_streams < 1 || o.max_streams > 1024 || o.timeout_ms <= 0 ||
        o.record_log < 0 || o.record_log > 2 || o.trim_nodes < 0 || o.auto_graph < 0 ||
        (o.backend != GDAG_BACKEND_CUDA && o.backend != GDAG_BACKEND_FAKE))
        return GDAG_ERR_INVALID;
    gdag_ctx *c = new (std::nothrow) gdag_ctx();
    if (!c) return GDAG_ERR_OOM;
    c->opt = o;
    if (c->opt.trim_nodes == 0) c->opt.trim_nodes = 65536;
    c->trim_at = (size_t)c->opt.trim_nodes;
    c->be.reset(o.backend == GDAG_BACKEND_FAKE
                    ? gdag::make_fake_backend(o.fake_complete, o.fake_fail_op, o.fake_fail_sticky)
                    : gdag::make_cuda_backend());
    int r = c->be->init(o.device);
    if (r) {
        delete c;
        return r == gdag::BE_STICKY ? GDAG_ERR_POISONED : GDAG_ERR_CUDA;
    }
    for (int i = 0; i < gdag::builtin_count(); ++i) c->kernels.push_back(gdag::builtin(i));
    *out = c;
    return GDAG_OK;
}

int gdag_destroy(gdag_ctx *c)
{
    if (!c) return GDAG_ERR_INVALID;
    int rc = GDAG_OK;
    if (!c->poisoned) {
        for (size_t s = 0; s < c->streams.size(); ++s) {
            int r = c->poll_stream((int32_t)s);
            if (r && !rc) rc = r;
        }
    }
    if (c->capturing) {
        void *exec = nullptr;
        if (!c->be->capture_end(c->cap_stream, &exec) && exec) c->be->graph_destroy(exec);
    }
    for (auto &g : c->graphs)
        if (g.live) c->be->graph_destroy(g.exec);
    if (c->cap_stream) c->be->stream_destroy(c->cap_stream);
    for (auto &a : c->arrays)
        if (a.live && a.host_owned) c->be->host_free(a.host);
    for (void *e : c->events) c->be->event_destroy(e);
    for (void *e : c->tevents) c->be->event_destroy(e);
    if (c->t0) c->be->event_destroy(c->t0);
    for (auto &s : c->streams)
        if (s.owned) c->be->stream_destroy(s.handle);
    delete c;
    return rc;
}

const char *gdag_last_error(gdag_ctx *c) { return c ? c->last_error.c_str() : "null context"; }

int gdag_add_stream(gdag_ctx *c, void *stream)
{
    if (!c) return GDAG_ERR_INVALID;
    if ((int)c->streams.size() >= c->opt.max_streams) return c->fail(GDAG_ERR_INVALID, "stream pool full");
    gdag::StreamState s;
    s.handle = stream;
    s.owned = false;
    s.queued = true;
    c->streams.push_back(s);
    c->free_streams.push_back((int32_t)c->streams.size() - 1);
    return GDAG_OK;
}

int gdag_array_register(gdag_ctx *c, void *dev, size_t bytes, void *host, gdag_array *out)
{
    if (!c || !out) return GDAG_ERR_INVALID;
    if (!dev && bytes) return c->fail(GDAG_ERR_INVALID, "null device pointer");
    int32_t id;
    if (!c->free_arrays.empty()) {
        id = c->free_arrays.back();
        c->free_arrays.pop_back();
    } else {
        c->arrays.emplace_back();
        id = (int32_t)c->arrays.size() - 1;
    }
    ArrayState &s = c->arrays[(size_t)id];
    s = ArrayState();
    s.dev = dev;
    s.bytes = bytes;
    s.host = host;
    s.live = true;
    *out = id;
    return GDAG_OK;
}

int gdag_array_unregister(gdag_ctx *c, gdag_array a)
{
    if (!c) return GDAG_ERR_INVALID;
    ArrayState *s = c->arr(a);
    if (!s) return c->fail(GDAG_ERR_INVALID, "unknown array %d", a);
    if (c->capturing) return c->fail(GDAG_ERR_INVALID, "not allowed while capturing");
    if (!c->poisoned) {
        std::vector<int64_t> users = s->readers;
        if (s->writer >= 0) users.push_back(s->writer);
        for (int64_t u : users) {
            int r = c->host_wait(u);
            if (r) return r;
        }
        int r = c->release_view(*s);
        if (r) return r;
    }
    if (s->host_owned) c->be->host_free(s->host);
    c->reader_entries -= (int64_t)s->readers.size();
    *s = ArrayState();
    c->free_arrays.push_back(a);
    return GDAG_OK;
}

int gdag_kernel_lookup(gdag_ctx *c, const char *name, gdag_kernel *out)
{
    if (!c || !name || !out) return GDAG_ERR_INVALID;
    for (size_t i = 0; i < c->kernels.size(); ++i)
        if (c->kernels[i].name == name) {
            *out = (gdag_kernel)i;
            return GDAG_OK;
        }
    return c->fail(GDAG_ERR_NOT_FOUND, "no kernel named '%s'", name);
}

int gdag_kernel_signature(gdag_ctx *c, gdag_kernel k, int32_t *nargs, gdag_argspec *spec, int32_t cap)
{
    if (!c || k < 0 || (size_t)k >= c->kernels.size() || !nargs) return GDAG_ERR_INVALID;
    const KernelEntry &e = c->kernels[(size_t)k];
    *nargs = e.nargs;
    if (spec)
        for (int i = 0; i < e.nargs && i < cap; ++i) spec[i] = e.spec[i];
    return GDAG_OK;
}

int gdag_kernel_register(gdag_ctx *c, const char *name, const void *fn, int32_t nargs, const gdag_argspec *spec,
                         gdag_kernel *out)
{
    if (!c || !name || !out || (!fn && c->opt.backend == GDAG_BACKEND_CUDA)) return GDAG_ERR_INVALID;
    if (nargs < 0 || nargs > gdag::kMaxArgs || (nargs && !spec))
        return c->fail(GDAG_ERR_INVALID, "bad argument count %d", nargs);
    KernelEntry e;
    e.name = name;
    e.fn = fn;
    e.nargs = nargs;
    for (int i = 0; i < nargs; ++i) {
        if (spec[i].kind == GDAG_ARG_SCALAR && (spec[i].size < 1 || spec[i].size > 8))
            return c->fail(GDAG_ERR_INVALID, "scalar argument %d: size %d not in 1..8", i, spec[i].size);
        if (spec[i].kind != GDAG_ARG_SCALAR && spec[i].kind != GDAG_ARG_ARRAY)
            return c->fail(GDAG_ERR_INVALID, "argument %d: bad kind", i);
        e.spec[i] = spec[i];
    }
    c->kernels.push_back(e);
    *out = (gdag_kernel)c->kernels.size() - 1;
    return GDAG_OK;
}

// Resolve and validate arguments; fills acc (merged per array) and la.
static int resolve(gdag_ctx *c, gdag_kernel k, gdag_dim3 grid, gdag_dim3 block, size_t smem, const gdag_arg *args,
                   int32_t nargs, LaunchArgs &la, Access *acc, int *nacc)
{
    if (k < 0 || (size_t)k >= c->kernels.size()) return c->fail(GDAG_ERR_INVALID, "unknown kernel %d", k);
    const KernelEntry &e = c->kernels[(size_t)k];
    if (nargs != e.nargs)
        return c->fail(GDAG_ERR_INVALID, "%s takes %d arguments, got %d", e.name.c_str(), e.nargs, nargs);
    if (nargs && !args) return c->fail(GDAG_ERR_INVALID, "null argument list");
    la.nargs = nargs;
    *nacc = 0;
    for (int i = 0; i < nargs; ++i) {
        const gdag_arg &a = args[i];
        if (a.kind != e.spec[i].kind)
            return c->fail(GDAG_ERR_INVALID, "%s argument %d: expected %s", e.name.c_str(), i,
                           e.spec[i].kind == GDAG_ARG_ARRAY ? "an array" : "a scalar");
        la.ptr[i] = nullptr;
        la.bytes[i] = 0;
        la.val[i] = 0;
        if (a.kind == GDAG_ARG_SCALAR) {
            if (a.size != e.spec[i].size)
                return c->fail(GDAG_ERR_INVALID, "%s argument %d: scalar of %d bytes, expected %d", e.name.c_str(), i,
                               a.size, e.spec[i].size);
            la.val[i] = a.value;
            continue;
        }
        ArrayState *s = c->arr(a.array);
        if (!s) return c->fail(GDAG_ERR_INVALID, "%s argument %d: unknown array %d", e.name.c_str(), i, a.array);
        la.ptr[i] = s->dev;
        la.bytes[i] = s->bytes;
        int mode = a.mode == GDAG_MODE_SIGNATURE ? e.spec[i].mode : a.mode;
        if (mode < GDAG_MODE_DEFAULT || mode > GDAG_MODE_INOUT)
            return c->fail(GDAG_ERR_INVALID, "%s argument %d: bad mode %d", e.name.c_str(), i, mode);
        int bits = gdag::mode_bits(mode);
        int j = 0;
        while (j < *nacc && acc[j].array != a.array) ++j;
        if (j == *nacc) acc[(*nacc)++] = Access{a.array, bits};
        else acc[j].bits |= bits;  // the same array twice: write dominates
    }
    bool autocfg = grid.x == 0 && grid.y == 0 && grid.z == 0;
    if (autocfg && !e.launcher)
        return c->fail(GDAG_ERR_INVALID, "%s: user kernels need an explicit grid", e.name.c_str());
    if (!autocfg && (grid.x == 0 || grid.y == 0 || grid.z == 0 || block.x == 0 || block.y == 0 || block.z == 0))
        return c->fail(GDAG_ERR_INVALID, "%s: zero grid or block dimension", e.name.c_str());
    la.auto_cfg = autocfg;
    la.grid[0] = grid.x; la.grid[1] = grid.y; la.grid[2] = grid.z;
    la.block[0] = block.x; la.block[1] = block.y; la.block[2] = block.z;
    la.smem = smem;
    if (e.validate) {
        const char *msg = e.validate(la);
        if (msg) return c->fail(GDAG_ERR_INVALID, "%s: %s", e.name.c_str(), msg);
    }
    return GDAG_OK;
}

int gdag_launch(gdag_ctx *c, gdag_kernel k, gdag_dim3 grid, gdag_dim3 block, size_t smem, const gdag_arg *args,
                int32_t nargs, int64_t *node_out)
{
    if (!c) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    IssueRange nvtx(c, (k >= 0 && (size_t)k < c->kernels.size()) ? c->kernels[(size_t)k].name.c_str() : "launch");
    LaunchArgs la;
    Access acc[gdag::kMaxArgs];
    int nacc;
    r = resolve(c, k, grid, block, smem, args, nargs, la, acc, &nacc);
    if (r) return r;
    c->capture_note(acc, nacc);
    int64_t id = c->next_id();
    c->infer(id, acc, nacc);
    for (int i = 0; i < nacc; ++i)
        if (acc[i].bits & gdag::W_BIT) c->arrays[(size_t)acc[i].array].host_valid = false;
    c->push_node(GDAG_NODE_KERNEL);
    c->node(id)->label = k;
    if (node_out) *node_out = id;
    int32_t s;
    r = c->place(id, &s);
    if (r) return c->drop_failed(id, r);
    c->log_op(GDAG_OP_LAUNCH, s, -1, id);
    ++c->st.launches;
    r = c->be->launch(c->kernels[(size_t)k], la, c->streams[(size_t)s].handle);
    if (r) return c->abort_node(id, r, "launch");
    return c->finish(id, s);
}

int gdag_launch_fused(gdag_ctx *c, gdag_kernel k, const gdag_arg *args, int32_t nargs, int32_t count,
                      int64_t *node_out)
{
    if (!c) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    IssueRange nvtx(c, (k >= 0 && (size_t)k < c->kernels.size()) ? c->kernels[(size_t)k].name.c_str() : "fused launch");
    if (k < 0 || (size_t)k >= c->kernels.size()) return c->fail(GDAG_ERR_INVALID, "unknown kernel %d", k);
    const KernelEntry &e = c->kernels[(size_t)k];
    if (!e.fused) return c->fail(GDAG_ERR_INVALID, "%s has no fused form", e.name.c_str());
    if (count < 1 || count > GDAG_FUSED_MAX)
        return c->fail(GDAG_ERR_INVALID, "fused launch of %d members (1..%d)", count, GDAG_FUSED_MAX);
    if (nargs != e.nargs)
        return c->fail(GDAG_ERR_INVALID, "%s takes %d arguments, got %d", e.name.c_str(), e.nargs, nargs);
    if (!args) return c->fail(GDAG_ERR_INVALID, "null argument list");
    const gdag_dim3 autocfg{0, 0, 0};
    std::vector<LaunchArgs> la((size_t)count);
    std::vector<Access> acc;
    for (int32_t m = 0; m < count; ++m) {
        Access one[gdag::kMaxArgs];
        int n1;
        r = resolve(c, k, autocfg, autocfg, 0, args + (size_t)m * (size_t)nargs, nargs, la[(size_t)m], one, &n1);
        if (r) return r;
        // the element's accesses: the union of its members' (write dominates)
        for (int i = 0; i < n1; ++i) {
            size_t j = 0;
            while (j < acc.size() && acc[j].array != one[i].array) ++j;
            if (j == acc.size()) acc.push_back(one[i]);
            else acc[j].bits |= one[i].bits;
        }
    }
    // an array that a member writes is touched by no other member: inside
    // one launch the members' order is undefined
    for (size_t j = 0; j < acc.size(); ++j) {
        if (!(acc[j].bits & gdag::W_BIT)) continue;
        int users = 0;
        for (int32_t m = 0; m < count; ++m) {
            const gdag_arg *a = args + (size_t)m * (size_t)nargs;
            bool uses = false;
            for (int i = 0; i < nargs; ++i) uses = uses || (a[i].kind == GDAG_ARG_ARRAY && a[i].array == acc[j].array);
            users += uses;
        }
        if (users > 1)
            return c->fail(GDAG_ERR_INVALID, "%s: array %d is written by one member of a fused launch and used by %d",
                           e.name.c_str(), acc[j].array, users);
    }
    c->capture_note(acc.data(), (int)acc.size());
    int64_t id = c->next_id();
    c->infer(id, acc.data(), (int)acc.size());
    for (const Access &x : acc)
        if (x.bits & gdag::W_BIT) c->arrays[(size_t)x.array].host_valid = false;
    c->push_node(GDAG_NODE_KERNEL);
    c->node(id)->label = k;
    if (node_out) *node_out = id;
    int32_t s;
    r = c->place(id, &s);
    if (r) return c->drop_failed(id, r);
    c->log_op(GDAG_OP_LAUNCH, s, -1, id);
    ++c->st.launches;
    c->st.fused_members += count;
    r = c->be->launch_fused(c->kernels[(size_t)k], la.data(), count, c->streams[(size_t)s].handle);
    if (r) return c->abort_node(id, r, "fused launch");
    return c->finish(id, s);
}

int gdag_launch_raw(gdag_ctx *c, gdag_kernel k, gdag_dim3 grid, gdag_dim3 block, size_t smem, const gdag_arg *args,
                    int32_t nargs, void *stream)
{
    if (!c) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    LaunchArgs la;
    Access acc[gdag::kMaxArgs];
    int nacc;
    r = resolve(c, k, grid, block, smem, args, nargs, la, acc, &nacc);
    if (r) return r;
    ++c->st.launches;
    r = c->be->launch(c->kernels[(size_t)k], la, stream);
    if (r) return c->be_fail(r, "raw launch");
    return GDAG_OK;
}

int gdag_launch_external(gdag_ctx *c, void (*fn)(void *, void *), void *user, const gdag_array *arrays,
                         const int32_t *modes, int32_t n, int64_t *node_out)
{
    if (!c || !fn || n < 0 || n > gdag::kMaxArgs || (n && (!arrays || !modes))) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    IssueRange nvtx(c, "external");
    Access acc[gdag::kMaxArgs];
    int nacc = 0;
    for (int i = 0; i < n; ++i) {
        if (!c->arr(arrays[i])) return c->fail(GDAG_ERR_INVALID, "unknown array %d", arrays[i]);
        if (modes[i] < GDAG_MODE_DEFAULT || modes[i] > GDAG_MODE_INOUT)
            return c->fail(GDAG_ERR_INVALID, "bad mode %d", modes[i]);
        int bits = gdag::mode_bits(modes[i]);
        int j = 0;
        while (j < nacc && acc[j].array != arrays[i]) ++j;
        if (j == nacc) acc[nacc++] = Access{arrays[i], bits};
        else acc[j].bits |= bits;
    }
    c->capture_note(acc, nacc);
    int64_t id = c->next_id();
    c->infer(id, acc, nacc);
    for (int i = 0; i < nacc; ++i)
        if (acc[i].bits & gdag::W_BIT) c->arrays[(size_t)acc[i].array].host_valid = false;
    c->push_node(GDAG_NODE_EXTERNAL);
    if (node_out) *node_out = id;
    int32_t s;
    r = c->place(id, &s);
    if (r) return c->drop_failed(id, r);
    c->log_op(GDAG_OP_EXTERNAL, s, -1, id);
    r = c->be->external(fn, user, c->streams[(size_t)s].handle);
    if (r) return c->abort_node(id, r, "external call");
    return c->finish(id, s);
}

int gdag_array_host(gdag_ctx *c, gdag_array a, int32_t mode, void **out)
{
    if (!c || !out) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    if (c->capturing) return c->fail(GDAG_ERR_INVALID, "not allowed while capturing");
    ArrayState *s = c->arr(a);
    if (!s) return c->fail(GDAG_ERR_INVALID, "unknown array %d", a);
    r = c->ensure_host(*s);
    if (r) return r;
    if (mode == GDAG_MODE_IN) {
        r = gdag_array_read(c, a, nullptr, 0, s->bytes);
        if (r) return r;
    } else if (mode == GDAG_MODE_OUT) {
        r = c->release_view(*s);
        if (r) return r;
    } else {
        return c->fail(GDAG_ERR_INVALID, "mode must be GDAG_MODE_IN or GDAG_MODE_OUT");
    }
    *out = s->host;
    return GDAG_OK;
}

int gdag_array_write(gdag_ctx *c, gdag_array a, const void *src, size_t off, size_t bytes)
{
    if (!c) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    IssueRange nvtx(c, "host write");
    ArrayState *s = c->arr(a);
    if (!s) return c->fail(GDAG_ERR_INVALID, "unknown array %d", a);
    if (off > s->bytes || bytes > s->bytes - off)
        return c->fail(GDAG_ERR_INVALID, "write of [%zu, %zu) outside %zu bytes", off, off + bytes, s->bytes);
    r = c->ensure_host(*s);
    if (r) return r;
    char *view = static_cast<char *>(s->host) + off;
    if (src && src != view) {
        if (c->capturing)
            return c->fail(GDAG_ERR_INVALID, "while capturing, a host write copies from the host view (src NULL)");
        r = c->release_view(*s);
        if (r) return r;
        std::memcpy(view, src, bytes);
    }
    Access acc{a, gdag::W_BIT};
    c->capture_note(&acc, 1);
    int64_t id = c->next_id();
    c->infer(id, &acc, 1);
    bool full = off == 0 && bytes == s->bytes;
    s->host_valid = s->host_valid || full;
    c->push_node(GDAG_NODE_HOST_WRITE);
    int32_t st;
    r = c->place(id, &st);
    if (r) return c->drop_failed(id, r);
    c->log_op(GDAG_OP_COPY_H2D, st, -1, id);
    ++c->st.copies;
    r = c->be->copy_h2d(static_cast<char *>(s->dev) + off, view, bytes, c->streams[(size_t)st].handle);
    if (r) return c->abort_node(id, r, "host-to-device copy");
    s->view_copy = id;
    s->prefetch = -1;  // the view now holds the host's data
    r = c->finish(id, st);
    if (r) return r;
    if (!c->opt.prefetch) return c->host_wait(id);
    return GDAG_OK;
}

int gdag_array_read(gdag_ctx *c, gdag_array a, void *dst, size_t off, size_t bytes)
{
    if (!c) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    IssueRange nvtx(c, "host read");
    if (c->capturing) return c->fail(GDAG_ERR_INVALID, "not allowed while capturing");
    ArrayState *s = c->arr(a);
    if (!s) return c->fail(GDAG_ERR_INVALID, "unknown array %d", a);
    if (off > s->bytes || bytes > s->bytes - off)
        return c->fail(GDAG_ERR_INVALID, "read of [%zu, %zu) outside %zu bytes", off, off + bytes, s->bytes);
    r = c->ensure_host(*s);
    if (r) return r;
    char *view = static_cast<char *>(s->host) + off;
    const bool covered = s->prefetch >= 0 && s->pf_writer == s->writer && off >= s->pf_off &&
                         off + bytes <= s->pf_off + s->pf_bytes;
    Access acc{a, gdag::R_BIT};
    int64_t id = c->next_id();
    c->infer(id, &acc, 1);
    c->push_node(GDAG_NODE_HOST_READ);
    if (!s->host_valid && covered) {
        // a device-to-host prefetch of this range is in flight or done
        int64_t pf = s->prefetch;
        r = c->host_wait(pf);
        if (r) return r;
        c->log_op(GDAG_OP_HOST_NODE, -1, -1, id);
        if (s->pf_off == 0 && s->pf_bytes == s->bytes) s->host_valid = true;
    } else if (!s->host_valid) {
        int32_t st;
        r = c->place(id, &st);
        if (r) return c->drop_failed(id, r);
        c->log_op(GDAG_OP_COPY_D2H, st, -1, id);
        ++c->st.copies;
        r = c->be->copy_d2h(view, static_cast<char *>(s->dev) + off, bytes, c->streams[(size_t)st].handle);
        if (r) return c->abort_node(id, r, "device-to-host copy");
        r = c->finish(id, st);
        if (r) return r;
        r = c->host_wait(id);
        if (r) return r;
        if (off == 0 && bytes == s->bytes) s->host_valid = true;
    } else {
        // The view already holds the data: a host-only element.  A later
        // writer of the array takes its edges from the readers alone, so
        // this element must not complete before its writer: when that is a
        // host write whose copy to the device is still in flight, the host
        // waits for the copy first (a writer that races it would otherwise
        // be overwritten by it).
        for (int64_t p : c->par) {
            r = c->host_wait(p);
            if (r) return r;
        }
        c->log_op(GDAG_OP_HOST_NODE, -1, -1, id);
    }
    if (dst && dst != view) std::memcpy(dst, view, bytes);
    return GDAG_OK;
}

int gdag_array_prefetch_host(gdag_ctx *c, gdag_array a, size_t off, size_t bytes)
{
    if (!c) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    IssueRange nvtx(c, "prefetch to host");
    if (c->capturing) return c->fail(GDAG_ERR_INVALID, "not allowed while capturing");
    ArrayState *s = c->arr(a);
    if (!s) return c->fail(GDAG_ERR_INVALID, "unknown array %d", a);
    if (off > s->bytes || bytes > s->bytes - off)
        return c->fail(GDAG_ERR_INVALID, "prefetch of [%zu, %zu) outside %zu bytes", off, off + bytes, s->bytes);
    if (s->host_valid) return GDAG_OK;  // the view is already current
    r = c->ensure_host(*s);
    if (r) return r;
    r = c->release_view(*s);  // an earlier copy still using the view
    if (r) return r;
    Access acc{a, gdag::R_BIT};
    int64_t id = c->next_id();
    c->infer(id, &acc, 1);
    c->push_node(GDAG_NODE_HOST_PREFETCH);
    int32_t st;
    r = c->place(id, &st);
    if (r) return c->drop_failed(id, r);
    c->log_op(GDAG_OP_COPY_D2H, st, -1, id);
    ++c->st.copies;
    r = c->be->copy_d2h(static_cast<char *>(s->host) + off, static_cast<char *>(s->dev) + off, bytes,
                        c->streams[(size_t)st].handle);
    if (r) return c->abort_node(id, r, "device-to-host prefetch");
    s->prefetch = id;
    s->pf_writer = s->writer;
    s->pf_off = off;
    s->pf_bytes = bytes;
    s->view_copy = id;
    return c->finish(id, st);
}

// gdag_issue without the automatic capture: each element as its own call
static int issue_each(gdag_ctx *c, const gdag_elem *elems, int32_t n, const gdag_arg *args, int64_t nargs_total,
                      int64_t *nodes_out, int32_t *issued)
{
    if (issued) *issued = 0;
    if (nodes_out)
        for (int32_t i = 0; i < n; ++i) nodes_out[i] = -1;
    for (int32_t i = 0; i < n; ++i) {
        const gdag_elem &e = elems[i];
        const int64_t before = c->next_id();
        int64_t node = -1;
        int r;
        switch (e.type) {
        case GDAG_ELEM_LAUNCH:
        case GDAG_ELEM_LAUNCH_FUSED: {
            const int64_t count = e.type == GDAG_ELEM_LAUNCH ? 1 : (int64_t)e.count;
            if (e.nargs < 0 || count < 1 || e.arg0 < 0 || e.arg0 > nargs_total ||
                (int64_t)e.nargs * count > nargs_total - e.arg0) {
                r = c->fail(GDAG_ERR_INVALID, "element %d: arguments [%lld, +%lld) outside the %lld given", i,
                            (long long)e.arg0, (long long)e.nargs * count, (long long)nargs_total);
                break;
            }
            const gdag_arg *a = e.nargs ? args + e.arg0 : nullptr;
            if (e.type == GDAG_ELEM_LAUNCH)
                r = gdag_launch(c, e.kernel, e.grid, e.block, (size_t)e.smem, a, e.nargs, &node);
            else
                r = gdag_launch_fused(c, e.kernel, a, e.nargs, e.count, &node);
            break;
        }
        case GDAG_ELEM_WRITE:
            r = gdag_array_write(c, e.array, nullptr, (size_t)e.off, (size_t)e.bytes);
            break;
        case GDAG_ELEM_PREFETCH_HOST:
            r = gdag_array_prefetch_host(c, e.array, (size_t)e.off, (size_t)e.bytes);
            break;
        default:
            r = c->fail(GDAG_ERR_INVALID, "element %d: unknown type %d", i, e.type);
        }
        // the element's node, when it made one (a write or prefetch made the
        // last node; a failed element may still have one)
        if (c->next_id() > before) node = c->next_id() - 1;
        if (nodes_out) nodes_out[i] = node;
        if (r) return r;
        if (issued) *issued = i + 1;
    }
    return GDAG_OK;
}

// The key of a sequence for the automatic capture: every field of every
// element but arg0, then the argument entries each launch element uses (so
// that the same elements with other scalar values or arrays make another
// key).  False for a sequence that is never captured: one holding a
// prefetch to the host (not allowed in a capture) or an argument range
// outside the list (the dynamic issue reports it).
static bool auto_key(const gdag_elem *elems, int32_t n, const gdag_arg *args, int64_t nargs_total,
                     std::vector<uint64_t> &key, uint64_t &hash)
{
    key.clear();
    auto u = [](int32_t a, int32_t b) { return ((uint64_t)(uint32_t)a << 32) | (uint32_t)b; };
    for (int32_t i = 0; i < n; ++i) {
        const gdag_elem &e = elems[i];
        if (e.type != GDAG_ELEM_LAUNCH && e.type != GDAG_ELEM_LAUNCH_FUSED && e.type != GDAG_ELEM_WRITE) return false;
        key.push_back(u(e.type, e.kernel));
        key.push_back(u(e.array, e.nargs));
        key.push_back(u(e.count, (int32_t)e.smem));
        key.push_back(e.off);
        key.push_back(e.bytes);
        key.push_back(u((int32_t)e.grid.x, (int32_t)e.grid.y));
        key.push_back(u((int32_t)e.grid.z, (int32_t)e.block.x));
        key.push_back(u((int32_t)e.block.y, (int32_t)e.block.z));
        if (e.type == GDAG_ELEM_WRITE) continue;
        const int64_t count = e.type == GDAG_ELEM_LAUNCH ? 1 : (int64_t)e.count;
        if (e.nargs < 0 || count < 1 || e.arg0 < 0 || e.arg0 > nargs_total ||
            (int64_t)e.nargs * count > nargs_total - e.arg0)
            return false;
        for (int64_t j = 0; j < (int64_t)e.nargs * count; ++j) {
            const gdag_arg &a = args[e.arg0 + j];
            key.push_back(u(a.kind, a.mode));
            key.push_back(u(a.array, a.size));
            key.push_back(a.value);
        }
    }
    hash = 1469598103934665603ull;  // FNV-1a over the words
    for (uint64_t w : key) hash = (hash ^ w) * 1099511628211ull;
    return true;
}

// Replay graph g as the whole sequence: every element's node is the graph's.
static int auto_replay(gdag_ctx *c, int32_t g, int32_t n, int64_t *nodes_out, int32_t *issued)
{
    const int64_t before = c->next_id();
    int64_t node = -1;
    const int r = gdag_graph_launch(c, g, &node);
    if (c->next_id() == before) node = -1;
    if (nodes_out)
        for (int32_t i = 0; i < n; ++i) nodes_out[i] = node;
    if (issued) *issued = r ? 0 : n;
    return r;
}

int gdag_issue(gdag_ctx *c, const gdag_elem *elems, int32_t n, const gdag_arg *args, int64_t nargs_total,
               int64_t *nodes_out, int32_t *issued)
{
    if (issued) *issued = 0;
    if (!c) return GDAG_ERR_INVALID;
    if (n < 0 || (n && !elems) || nargs_total < 0 || (nargs_total && !args))
        return c->fail(GDAG_ERR_INVALID, "bad element or argument list");
    if (c->opt.auto_graph <= 0 || c->capturing || c->opt.trace || c->opt.policy == GDAG_POLICY_SERIAL_SYNC ||
        n == 0 || c->poisoned)
        return issue_each(c, elems, n, args, nargs_total, nodes_out, issued);
    std::vector<uint64_t> key;
    uint64_t hash = 0;
    if (!auto_key(elems, n, args, nargs_total, key, hash))
        return issue_each(c, elems, n, args, nargs_total, nodes_out, issued);
    size_t i = 0;
    while (i < c->auto_seqs.size() && !(c->auto_seqs[i].hash == hash && c->auto_seqs[i].key == key)) ++i;
    if (i == c->auto_seqs.size()) {
        if (c->auto_seqs.size() >= (size_t)GDAG_AUTO_GRAPH_SEQS) {
            // the least recently used sequence leaves, with its graph
            size_t lru = 0;
            for (size_t j = 1; j < c->auto_seqs.size(); ++j)
                if (c->auto_seqs[j].used < c->auto_seqs[lru].used) lru = j;
            if (c->auto_seqs[lru].graph >= 0) {
                const int r = gdag_graph_destroy(c, c->auto_seqs[lru].graph);
                if (r) return r;
            }
            c->auto_seqs.erase(c->auto_seqs.begin() + (std::ptrdiff_t)lru);
            i = c->auto_seqs.size();
        }
        Ctx::AutoSeq q;
        q.hash = hash;
        q.key.swap(key);
        c->auto_seqs.push_back(std::move(q));
    }
    c->auto_seqs[i].used = ++c->auto_clock;
    if (c->auto_seqs[i].graph >= 0) {
        if (c->graph_current(c->auto_seqs[i].graph)) return auto_replay(c, c->auto_seqs[i].graph, n, nodes_out, issued);
        // an array moved since the capture: drop the graph and start over
        const int r = gdag_graph_destroy(c, c->auto_seqs[i].graph);
        c->auto_seqs[i].graph = -1;
        c->auto_seqs[i].seen = 0;
        if (r) return r;
    }
    if (c->auto_seqs[i].never || c->auto_seqs[i].seen + 1 < c->opt.auto_graph) {
        const int r = issue_each(c, elems, n, args, nargs_total, nodes_out, issued);
        if (!r) ++c->auto_seqs[i].seen;
        return r;
    }
    // the auto_graph-th issue: capture the sequence (nothing runs), then
    // replay it; a sequence that fails inside the capture is issued
    // dynamically now and from then on, where it succeeds or fails as its
    // single calls would
    int r = gdag_capture_begin(c);
    if (r) return r;
    int32_t cap_issued = 0;
    const int rc = issue_each(c, elems, n, args, nargs_total, nullptr, &cap_issued);
    gdag_graph g = -1;
    const int re = gdag_capture_end(c, &g);
    if (rc || re) {
        if (!re && g >= 0) gdag_graph_destroy(c, g);
        if (c->poisoned) return re ? re : rc;
        c->auto_seqs[i].never = true;
        return issue_each(c, elems, n, args, nargs_total, nodes_out, issued);
    }
    c->auto_seqs[i].graph = g;
    return auto_replay(c, g, n, nodes_out, issued);
}

int gdag_sync(gdag_ctx *c)
{
    if (!c) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    if (c->capturing) return c->fail(GDAG_ERR_INVALID, "not allowed while capturing");
    for (size_t s = 0; s < c->streams.size(); ++s) {
        if (c->streams[s].active == 0) continue;
        c->log_op(GDAG_OP_STREAM_SYNC, (int)s, -1, -1);
        ++c->st.host_waits;
        r = c->poll_stream((int32_t)s);
        if (r) return r;
    }
    c->retire_all();
    c->trim(true);  // every element is retired now
    return GDAG_OK;
}

int gdag_stream_wait_all(gdag_ctx *c, void *stream)
{
    if (!c) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    if (c->capturing) return c->fail(GDAG_ERR_INVALID, "not allowed while capturing");
    for (size_t s = 0; s < c->streams.size(); ++s) {
        gdag::Node *n = c->node(c->streams[s].tail);
        if (!n || !n->active || n->event < 0) continue;
        r = c->be->stream_wait(stream, c->events[(size_t)n->event]);
        if (r) return c->be_fail(r, "stream wait");
    }
    return GDAG_OK;
}

int gdag_stream_fork(gdag_ctx *c, void *stream)
{
    if (!c) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    if (c->capturing) return c->fail(GDAG_ERR_INVALID, "not allowed while capturing");
    if (c->streams.empty()) return GDAG_OK;
    void *e;
    r = c->be->event_create(&e, false);
    if (r) return c->be_fail(r, "event create");
    r = c->be->event_record(e, stream);
    for (size_t s = 0; !r && s < c->streams.size(); ++s) r = c->be->stream_wait(c->streams[s].handle, e);
    c->be->event_destroy(e);
    if (r) return c->be_fail(r, "fork");
    return GDAG_OK;
}

int gdag_dag_export(gdag_ctx *c, gdag_edge *buf, size_t cap, size_t *n) { return export_vec(c, c->edge_log, buf, cap, n); }
int gdag_nodes_export(gdag_ctx *c, gdag_node_info *buf, size_t cap, size_t *n)
{
    return export_vec(c, c->node_log, buf, cap, n);
}
int gdag_ops_export(gdag_ctx *c, gdag_op *buf, size_t cap, size_t *n)
{
    return export_vec(c, c->op_log, buf, cap, n, true);
}

int gdag_trace_export(gdag_ctx *c, gdag_trace_rec *buf, size_t cap, size_t *n)
{
    if (!c || !n) return GDAG_ERR_INVALID;
    if (!c->opt.trace) return c->fail(GDAG_ERR_INVALID, "tracing needs options.trace = 1");
    int r = c->guard();
    if (r) return r;
    for (size_t s = 0; s < c->streams.size(); ++s) {
        r = c->poll_stream((int32_t)s);
        if (r) return r;
    }
    size_t k = 0;
    for (size_t i = 0; i < c->nodes.size(); ++i) {
        const gdag::Node &nd = c->nodes[i];
        if (nd.tev0 < 0 || nd.tev1 < 0) continue;
        if (buf && k < cap) {
            float a = 0.f, b = 0.f;
            r = c->be->event_elapsed_ms(c->t0, c->tevents[(size_t)nd.tev0], &a);
            if (!r) r = c->be->event_elapsed_ms(c->t0, c->tevents[(size_t)nd.tev1], &b);
            if (r) return c->be_fail(r, "elapsed time");
            buf[k] = gdag_trace_rec{c->base + (int64_t)i, nd.kind, nd.stream, (double)a, (double)b};
        }
        ++k;
    }
    *n = k;
    return GDAG_OK;
}



static void json_string(FILE *f, const char *s)
{
    std::fputc('"', f);
    for (; *s; ++s) {
        const unsigned char ch = (unsigned char)*s;
        if (ch == '"' || ch == '\\') std::fprintf(f, "\\%c", ch);
        else if (ch < 0x20) std::fprintf(f, "\\u%04x", ch);
        else std::fputc(ch, f);
    }
    std::fputc('"', f);
}

int gdag_trace_write(gdag_ctx *c, const char *path)
{
    if (!c || !path) return GDAG_ERR_INVALID;
    size_t n = 0;
    int r = gdag_trace_export(c, nullptr, 0, &n);
    if (r) return r;
    std::vector<gdag_trace_rec> recs(n);
    r = gdag_trace_export(c, recs.data(), n, &n);
    if (r) return r;
    FILE *f = std::fopen(path, "w");
    if (!f) return c->fail(GDAG_ERR_INVALID, "cannot open %s for writing", path);
    static const char *kinds[] = {"kernel", "h2d", "read", "external", "d2h", "graph"};
    std::fprintf(f, "{\"displayTimeUnit\": \"ms\", \"traceEvents\": [");
    for (size_t i = 0; i < recs.size(); ++i) {
        const gdag_trace_rec &t = recs[i];
        const char *cat = (t.kind >= 0 && t.kind <= 5) ? kinds[t.kind] : "node";
        const gdag::Node *nd = c->node(t.node);
        const int32_t lab = nd ? nd->label : -1;
        const char *name = (lab >= 0 && (size_t)lab < c->kernels.size()) ? c->kernels[(size_t)lab].name.c_str() : cat;
        std::fprintf(f, "%s\n{\"name\": ", i ? "," : "");
        json_string(f, name);
        std::fprintf(f, ", \"cat\": \"%s\", \"ph\": \"X\", \"ts\": %.3f, \"dur\": %.3f, \"pid\": 0, ", cat,
                     t.start_ms * 1e3, (t.end_ms > t.start_ms ? t.end_ms - t.start_ms : 0.0) * 1e3);
        if (t.stream >= 0) std::fprintf(f, "\"tid\": \"stream %d\", ", t.stream);
        else std::fprintf(f, "\"tid\": \"host\", ");
        std::fprintf(f, "\"args\": {\"node\": %lld}}", (long long)t.node);
    }
    std::fprintf(f, "\n]}\n");
    const bool bad = std::ferror(f) != 0;
    if (std::fclose(f) != 0 || bad) return c->fail(GDAG_ERR_INVALID, "writing %s failed", path);
    return GDAG_OK;
}

int gdag_node_query(gdag_ctx *c, int64_t node, int32_t *done)
{
    if (!c || !done) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    if (c->capturing) return c->fail(GDAG_ERR_INVALID, "not allowed while capturing");
    if (node < 0 || node >= c->next_id()) return c->fail(GDAG_ERR_INVALID, "unknown node %lld", (long long)node);
    gdag::Node *n = c->node(node);
    if (!n || !n->active) {  // retired, or dropped after a sync
        *done = 1;
        return GDAG_OK;
    }
    if (n->event < 0) {
        *done = 0;
        return GDAG_OK;
    }
    const int q = c->be->event_query(c->events[(size_t)n->event]);
    if (q == gdag::BE_NOT_READY) {
        *done = 0;
        return GDAG_OK;
    }
    if (q != gdag::BE_OK) return c->be_fail(q, "event query");
    c->log_op(GDAG_OP_QUERY_DONE, n->stream, n->event, node);
    c->retire(node);
    *done = 1;
    return GDAG_OK;
}

int gdag_nodes_query(gdag_ctx *c, const int64_t *nodes, int32_t n, int32_t *done)
{
    if (!c || n < 0 || (n && (!nodes || !done))) return GDAG_ERR_INVALID;
    for (int32_t i = 0; i < n; ++i) {
        int r = gdag_node_query(c, nodes[i], &done[i]);
        if (r) return r;
    }
    return GDAG_OK;
}

int gdag_capture_begin(gdag_ctx *c)
{
    if (!c) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    if (c->capturing) return c->fail(GDAG_ERR_INVALID, "a capture is already open");
    if (c->opt.policy == GDAG_POLICY_SERIAL_SYNC)
        return c->fail(GDAG_ERR_INVALID, "capture needs an asynchronous policy");
    r = gdag_sync(c);  // no parent from before the capture can remain active
    if (r) return r;
    if (!c->cap_stream) {
        r = c->be->stream_create(&c->cap_stream, c->opt.stream_priority);
        if (r) return c->be_fail(r, "stream create");
    }
    r = c->be->capture_begin(c->cap_stream);
    if (r) return c->be_fail(r, "capture begin");
    c->capturing = true;
    c->cap_access.clear();
    for (auto &st : c->streams) {
        r = c->fork_from(c->cap_stream, st.handle);
        if (r) return r;
    }
    return GDAG_OK;
}

int gdag_capture_end(gdag_ctx *c, gdag_graph *out)
{
    if (!c || !out) return GDAG_ERR_INVALID;
    if (!c->capturing) return c->fail(GDAG_ERR_INVALID, "no capture is open");
    int r = GDAG_OK;
    for (auto &st : c->streams) {  // every stream joins back into the origin
        r = c->fork_from(st.handle, c->cap_stream);
        if (r) break;
    }
    void *exec = nullptr;
    int rr = c->be->capture_end(c->cap_stream, &exec);
    c->capturing = false;
    // nothing captured has run: the captured nodes leave the frontier (the
    // capture began with a sync, so every element is retired now)
    c->retire_all();
    c->trim(true);
    if (r) return r;
    if (rr) return c->be_fail(rr, "capture end");
    Ctx::Graph g;
    g.exec = exec;
    g.access = c->cap_access;
    for (const Access &a : g.access) {
        const ArrayState &st = c->arrays[(size_t)a.array];
        g.dev.push_back(st.dev);
        g.host.push_back(st.host);
        g.bytes.push_back(st.bytes);
    }
    g.live = true;
    c->graphs.push_back(g);
    *out = (gdag_graph)c->graphs.size() - 1;
    return GDAG_OK;
}

int gdag_graph_launch(gdag_ctx *c, gdag_graph g, int64_t *node_out)
{
    if (!c) return GDAG_ERR_INVALID;
    int r = c->guard();
    if (r) return r;
    IssueRange nvtx(c, "graph replay");
    if (c->capturing) return c->fail(GDAG_ERR_INVALID, "not allowed while capturing");
    if (g < 0 || (size_t)g >= c->graphs.size() || !c->graphs[(size_t)g].live)
        return c->fail(GDAG_ERR_INVALID, "unknown graph %d", g);
    const Ctx::Graph &gr = c->graphs[(size_t)g];
    for (size_t i = 0; i < gr.access.size(); ++i) {
        const int32_t a = gr.access[i].array;
        const ArrayState *st = c->arr(a);
        if (!st) return c->fail(GDAG_ERR_INVALID, "graph uses unregistered array %d", a);
        // (an array without a host view at capture had no host copy in it;
        // its view may have been allocated since)
        if (st->dev != gr.dev[i] || (gr.host[i] && st->host != gr.host[i]) || st->bytes != gr.bytes[i])
            return c->fail(GDAG_ERR_INVALID, "array %d was registered again at another address since graph %d was captured",
                           a, g);
    }
    int64_t id = c->next_id();
    c->infer(id, gr.access.data(), (int)gr.access.size());
    for (const auto &a : gr.access)
        if (a.bits & gdag::W_BIT) c->arrays[(size_t)a.array].host_valid = false;
    c->push_node(GDAG_NODE_GRAPH);
    if (node_out) *node_out = id;
    int32_t s;
    r = c->place(id, &s);
    if (r) return c->drop_failed(id, r);
    c->log_op(GDAG_OP_LAUNCH, s, -1, id);
    r = c->be->graph_launch(gr.exec, c->streams[(size_t)s].handle);
    if (r) return c->abort_node(id, r, "graph launch");
    return c->finish(id, s);
}

int gdag_graph_destroy(gdag_ctx *c, gdag_graph g)
{
    if (!c) return GDAG_ERR_INVALID;
    if (g < 0 || (size_t)g >= c->graphs.size() || !c->graphs[(size_t)g].live)
        return c->fail(GDAG_ERR_INVALID, "unknown graph %d", g);
    // a launched replay may still run: wait for every stream first
    if (!c->poisoned) {
        int r = gdag_sync(c);
        if (r) return r;
    }
    c->be->graph_destroy(c->graphs[(size_t)g].exec);
    c->graphs[(size_t)g] = Ctx::Graph();
    return GDAG_OK;
}

int gdag_stats_get(gdag_ctx *c, gdag_stats *out)
{
    if (!c || !out) return GDAG_ERR_INVALID;
    *out = c->st;
    out->streams = (int32_t)c->streams.size();
    out->active = (int32_t)c->active_count;
    out->held_nodes = (int64_t)c->nodes.size();
    out->held_readers = c->reader_entries;
    return GDAG_OK;
}

size_t gdag_scratch_bytes(const char *kernel, int64_t n) { return kernel ? gdag::scratch_bytes(kernel, n) : 0; }

}  // extern "C"
