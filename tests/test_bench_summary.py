"""The bench line's compact summary: the last key of the line, short enough
that the line's last 1500 characters hold it whole, with every DAG, every
served rate and every kernel's cold fraction of HBM taken from the detailed
keys unchanged (rounded)."""
import json

import bench


def fake_line():
    dag = lambda ms: {"makespan_ms": {"parallel": ms}, "speedup_vs_serial_sync": 1.5, "vs_hand_cuda_graph": 1.01,
                      "auto_graph_vs_hand_cuda_graph": 1.02, "frac_of_cp_bound": 0.5,
                      "frac_of_resource_bound": 0.9,
                      "per_kernel_solo": {"k%d" % i: {"frac_of_hbm_peak": 0.1 * i} for i in range(1, 4)}}
    names = ["B&S", "VEC", "IMG", "ML", "HITS", "DL", "HITS-batch"]
    out = {"metric": "m", "value": 1.0, "roofline": {"frac": 0.7471}, "e2e": {"ms_per_step": 2.6601},
           "dags": {n: dag(0.1 * (i + 1)) for i, n in enumerate(names)},
           "serve": {"runs": [{"offered_req_s": r, "fusion": f, "window_ms": w, "throughput_req_s": r - 1,
                               "p50_ms": 0.3, "p99_ms": 19.0} for r, f, w in
                              ((2000.0, True, 1.0), (2000.0, False, 1.0), (1000.0, True, 1.0), (2000.0, True, None))]}}
    # a real line carries 19 kernels and long detailed keys before the summary
    for i in range(20):
        out["dags"]["HITS"]["per_kernel_solo"]["kernel_with_a_long_name_%02d" % i] = {"frac_of_hbm_peak": 0.01 * i}
    out["padding"] = "x" * 5000
    out["summary"] = bench.compact_summary(out)
    return out


def test_summary_is_last_and_fits_the_tail():
    out = fake_line()
    line = json.dumps(out)
    assert list(out)[-1] == "summary"
    tail = line[-1500:]
    assert json.dumps(out["summary"]) in tail


def test_summary_values_come_from_the_detailed_keys():
    out = fake_line()
    s = out["summary"]
    assert s["dags"]["DL"] == [0.6, 1.5, 1.01, 1.02, 0.5, 0.9]
    assert [r[:3] for r in s["serve"]] == [[2000.0, 1, 1], [2000.0, 0, 1], [1000.0, 1, 1], [2000.0, 1, 0]]
    assert s["serve"][0][3:] == [1999.0, 0.3, 19.0]
    assert s["kernel_cold_frac_of_hbm"]["k3"] == 0.3
    assert s["bs_call_frac"] == 0.747 and s["e2e_ms"] == 2.66
