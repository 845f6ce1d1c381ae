/* Random programs of every element kind, driven through the C ABI on the
 * recording fake backend.  Built against an AddressSanitizer/UBSan build of
 * the library by tests/test_runtime_sanitized.py: any memory or undefined-
 * behaviour error in the tracker aborts the run.  Calls may fail (injected
 * backend failures, refused arguments); only the process's health and the
 * end state are checked.  Usage: random_programs <programs> <steps> <seed>. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>
#include <stdlib.h>

#include "gdag.h"

static uint64_t rng_state;

static uint32_t rnd(uint32_t n) /* xorshift64*, uniform enough for choices */
{
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return (uint32_t)((rng_state * 2685821657736338717ULL) >> 33) % n;
}

static void external_fn(void *stream, void *user)
{
    (void)stream;
    ++*(int *)user;
}

#define MAXA 6
#define NB 64

int main(int argc, char **argv)
{
    const int programs = argc > 1 ? atoi(argv[1]) : 100;
    const int steps = argc > 2 ? atoi(argv[2]) : 200;
    rng_state = argc > 3 ? strtoull(argv[3], NULL, 10) * 0x9E3779B97F4A7C15ULL + 1 : 1;
    int calls = 0, external_calls = 0;
    for (int p = 0; p < programs; ++p) {
        gdag_options o;
        gdag_options_default(&o);
        o.backend = GDAG_BACKEND_FAKE;
        o.policy = (int32_t)rnd(3);
        o.max_streams = 1 + (int32_t)rnd(6);
        o.prefetch = (int32_t)rnd(2);
        o.retire_by_query = (int32_t)rnd(2);
        o.fake_complete = (int32_t)rnd(2);
        o.record_log = (int32_t)rnd(3);
        o.trace = rnd(5) == 0;
        const int32_t trims[] = {0, 1, 2, 3, 8, 64};
        o.trim_nodes = trims[rnd(6)];
        o.fake_fail_op = rnd(3) == 0 ? (int64_t)rnd(400) : -1;
        o.fake_fail_sticky = rnd(4) == 0;
        o.auto_graph = (int32_t)rnd(3);
        gdag_ctx *c = NULL;
        if (gdag_create(&c, &o)) {
            printf("create failed\n");
            return 1;
        }
        const int na = 1 + (int)rnd(MAXA);
        gdag_array arr[MAXA];
        uintptr_t next_dev = 0x100000;
        for (int i = 0; i < na; ++i, next_dev += 0x10000)
            if (gdag_array_register(c, (void *)next_dev, NB, NULL, &arr[i])) return 2;
        gdag_argspec spec[4];
        for (int i = 0; i < 4; ++i) {
            spec[i].kind = GDAG_ARG_ARRAY;
            spec[i].mode = GDAG_MODE_DEFAULT;
            spec[i].size = 0;
            spec[i].reserved = 0;
        }
        gdag_kernel kern[5], bs;
        for (int n = 1; n <= 4; ++n) {
            char name[16];
            snprintf(name, sizeof name, "k%d", n);
            if (gdag_kernel_register(c, name, NULL, n, spec, &kern[n])) return 3;
        }
        if (gdag_kernel_lookup(c, "bs_call", &bs)) return 4;
        gdag_graph graph = -1;
        const gdag_dim3 one = {1, 1, 1}, warp = {32, 1, 1}, autoshape = {0, 0, 0};
        for (int s = 0; s < steps; ++s) {
            const int a = (int)rnd((uint32_t)na);
            const size_t off = rnd(3) == 0 ? 16 : 0, bytes = rnd(4) == 0 ? 16 : NB - off;
            const uint32_t r = rnd(100);
            int64_t node = -1;
            ++calls;
            unsigned char hostbuf[NB];  /* a caller buffer of exactly `bytes` bytes is enough */
            for (size_t k = 0; k < bytes; ++k) hostbuf[k] = (unsigned char)(s + k);
            if (r < 10) {
                gdag_array_write(c, arr[a], rnd(2) ? hostbuf : NULL, off, bytes);
            } else if (r < 18) {
                gdag_array_read(c, arr[a], rnd(2) ? hostbuf : NULL, off, bytes);
            } else if (r < 23) {
                gdag_array_prefetch_host(c, arr[a], off, bytes);
            } else if (r < 28 && na > 1) {
                /* fused bs_call: every member reads array `a` and writes its own output */
                gdag_arg m[3 * 7];
                int count = 0;
                for (int b = 0; b < na && count < 3; ++b) {
                    if (b == a) continue;
                    gdag_arg *q = &m[7 * count++];
                    q[0].kind = GDAG_ARG_ARRAY; q[0].mode = GDAG_MODE_SIGNATURE; q[0].array = arr[a];
                    q[0].size = 0; q[0].value = 0;
                    q[1] = q[0];
                    q[1].array = arr[b];
                    q[2].kind = GDAG_ARG_SCALAR; q[2].mode = 0; q[2].array = 0; q[2].size = 8; q[2].value = 16;
                    const float vals[4] = {60.0f, 0.1f, 0.2f, 1.0f};
                    for (int k = 0; k < 4; ++k) {
                        union { float f; uint32_t u; } u;
                        u.f = vals[k];
                        q[3 + k].kind = GDAG_ARG_SCALAR; q[3 + k].mode = 0; q[3 + k].array = 0;
                        q[3 + k].size = 4; q[3 + k].value = u.u;
                    }
                }
                gdag_launch_fused(c, bs, m, 7, count, &node);
            } else if (r < 32) {
                gdag_array xs[2] = {arr[a], arr[(a + 1) % na]};
                int32_t modes[2] = {GDAG_MODE_IN, GDAG_MODE_INOUT};
                gdag_launch_external(c, external_fn, &external_calls, xs, modes, na > 1 ? 2 : 1, &node);
            } else if (r < 35) {
                if (gdag_capture_begin(c) == GDAG_OK) {
                    gdag_arg g[1];
                    g[0].kind = GDAG_ARG_ARRAY; g[0].mode = GDAG_MODE_INOUT; g[0].array = arr[a];
                    g[0].size = 0; g[0].value = 0;
                    gdag_launch(c, kern[1], one, warp, 0, g, 1, &node);
                    gdag_graph gg;
                    if (gdag_capture_end(c, &gg) == GDAG_OK) graph = gg;
                }
            } else if (r < 40) {
                if (graph >= 0) gdag_graph_launch(c, graph, &node);
            } else if (r < 42) {
                if (gdag_array_unregister(c, arr[a]) == GDAG_OK) {
                    next_dev += 0x10000;
                    if (gdag_array_register(c, (void *)next_dev, NB, NULL, &arr[a])) return 5;
                }
            } else if (r < 44) {
                gdag_sync(c);
            } else if (r < 48) {
                /* a two-element sequence through gdag_issue: repeated keys are
                   captured and replayed under auto_graph, many keys evict */
                gdag_elem e[2];
                memset(e, 0, sizeof e);
                gdag_arg g[2];
                e[0].type = GDAG_ELEM_WRITE;
                e[0].array = arr[a];
                e[0].off = off;
                e[0].bytes = bytes;
                e[1].type = GDAG_ELEM_LAUNCH;
                e[1].kernel = kern[2];
                e[1].nargs = 2;
                e[1].arg0 = 0;
                e[1].grid = one;
                e[1].block = warp;
                for (int i = 0; i < 2; ++i) {
                    const int32_t modes[4] = {GDAG_MODE_IN, GDAG_MODE_IN, GDAG_MODE_OUT, GDAG_MODE_INOUT};
                    g[i].kind = GDAG_ARG_ARRAY;
                    g[i].mode = modes[rnd(4)];
                    g[i].array = arr[(a + i) % na];
                    g[i].size = 0;
                    g[i].value = 0;
                }
                int64_t nodes[2];
                int32_t issued = 0;
                gdag_issue(c, e, 2, g, 2, nodes, &issued);
            } else if (r < 52) {
                gdag_stats st;
                gdag_stats_get(c, &st);
                int32_t done = 0;
                if (st.nodes > 0) gdag_node_query(c, (int64_t)rnd((uint32_t)st.nodes), &done);
            } else {
                const int n = 1 + (int)rnd(na < 4 ? (uint32_t)na : 4u);
                gdag_arg g[4];
                for (int i = 0; i < n; ++i) {
                    const int32_t modes[4] = {GDAG_MODE_IN, GDAG_MODE_IN, GDAG_MODE_OUT, GDAG_MODE_INOUT};
                    g[i].kind = GDAG_ARG_ARRAY;
                    g[i].mode = modes[rnd(4)];
                    g[i].array = arr[(a + i) % na];
                    g[i].size = 0;
                    g[i].value = 0;
                }
                gdag_launch(c, kern[n], rnd(2) ? one : autoshape, warp, 0, g, n, &node);
            }
        }
        /* exports in whatever form the options allow (errors expected) */
        size_t n = 0;
        gdag_dag_export(c, NULL, 0, &n);
        gdag_ops_export(c, NULL, 0, &n);
        gdag_nodes_export(c, NULL, 0, &n);
        if (o.trace) gdag_trace_export(c, NULL, 0, &n);
        const int rs = gdag_sync(c);
        gdag_stats st;
        gdag_stats_get(c, &st);
        if (rs == GDAG_OK && (st.active != 0 || st.held_readers < 0 || (!o.trace && st.held_nodes != 0))) {
            printf("program %d: active %d held_nodes %lld held_readers %lld after sync\n", p, st.active,
                   (long long)st.held_nodes, (long long)st.held_readers);
            return 6;
        }
        if (graph >= 0) gdag_graph_destroy(c, graph);
        gdag_destroy(c);
    }
    printf("ok %d programs %d calls %d external\n", programs, calls, external_calls);
    return 0;
}
