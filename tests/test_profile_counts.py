"""The per-unit counts behind bench.py's roofline come from a committed ncu summary that records a
hash of the kernel sources it was measured on; they must belong to the sources as they stand."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_flux_kernel_counts_belong_to_the_current_sources():
    bench = _bench()
    counts, why = bench.profile_counts()
    assert counts is not None, why + ": re-capture the counts with the commands in " + bench.FLUX_PROFILE
    assert 500.0 < counts["flops_per_unit"] < 5000.0
    assert counts["fp64_inst_per_unit"] <= counts["flops_per_unit"] <= 2.0 * counts["fp64_inst_per_unit"]
    assert counts["traffic_bytes_per_launch"] > 0


def test_stale_counts_are_not_used(tmp_path):
    bench = _bench()
    src = open(bench.FLUX_PROFILE).read().replace('"source_hash": "', '"source_hash": "0')
    p = tmp_path / "stale.txt"
    p.write_text(src)
    counts, why = bench.profile_counts(str(p))
    assert counts is None and "changed" in why
