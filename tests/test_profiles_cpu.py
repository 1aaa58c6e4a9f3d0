"""The DRAM traffic that bench.py reports for a kernel is the one in the committed ncu summary of it."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SUMMARIES = {("c3", "flux"): "flux_mixed_c3_population.md", ("c3", "grad"): "grad_mixed_c3_population.md",
             ("c4", "flux"): "flux_mixed_c4_heterogeneous.md"}


def summary_bytes(name):
    text = open(os.path.join(ROOT, "profiles", name)).read()
    total = 0.0
    for metric in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
        m = re.search(r"`" + re.escape(metric) + r"`\) \| ([0-9.]+) (Kbyte|Mbyte|Gbyte|byte)", text)
        assert m, f"{metric} missing from {name}"
        total += float(m.group(1)) * {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}[m.group(2)]
    return total


def test_bench_traffic_matches_the_ncu_summaries():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for key, value in bench.TRAFFIC.items():
        assert key in SUMMARIES, f"traffic for {key} has no ncu summary"
        assert abs(value - summary_bytes(SUMMARIES[key])) <= 1e3, (key, value, summary_bytes(SUMMARIES[key]))
