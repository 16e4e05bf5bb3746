"""Host logic of the benchmark's ncu records: the kernel-source hash ignores
comments but not code, and a recorded DRAM traffic figure is used only for
the sources and kernel variant it was captured with."""
import importlib.util
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(root):
    spec = importlib.util.spec_from_file_location("bench_records_under_test", os.path.join(root, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _copy_tree(tmp_path):
    root = tmp_path / "repo"
    (root / "paper_2209_15333_gb300").mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, "bench.py"), root / "bench.py")
    shutil.copytree(os.path.join(ROOT, "paper_2209_15333_gb300", "csrc"), root / "paper_2209_15333_gb300" / "csrc")
    return root


def test_source_hash_ignores_comments_only(tmp_path):
    root = _copy_tree(tmp_path)
    kern = root / "paper_2209_15333_gb300" / "csrc" / "cfd_kernels.cuh"
    h0 = _bench(str(root)).kernel_src_hash()
    text = kern.read_text(encoding="utf-8")
    kern.write_text(text + "\n// a remark\n/* a block\n   remark */\n", encoding="utf-8")
    assert _bench(str(root)).kernel_src_hash() == h0
    kern.write_text(text + "\nstatic const int cfd_probe_constant = 1;\n", encoding="utf-8")
    assert _bench(str(root)).kernel_src_hash() != h0


def test_traffic_record_needs_matching_sources_and_variant():
    b = _bench(ROOT)
    tr = b.NCU_TRAFFIC
    N = tr["nodes"]
    rec = tr["fp64"]["sweep_zeta"][0]
    assert b.kernel_traffic("fp64", "sweep_zeta", rec["variant"], N, tr["src"]) == rec["bytes_per_launch"]
    # twice the nodes, twice the bytes
    assert b.kernel_traffic("fp64", "sweep_zeta", rec["variant"], 2 * N, tr["src"]) == 2 * rec["bytes_per_launch"]
    assert b.kernel_traffic("fp64", "sweep_zeta", rec["variant"], N, "000000000000") is None
    assert b.kernel_traffic("fp64", "sweep_zeta", [9, 9], N, tr["src"]) is None
    # the learned form takes its own sensor record and the plain form's sweeps
    assert b.kernel_traffic("mixed_learned", "sensor", None, N, tr["src"]) == \
        tr["mixed_learned"]["sensor"][0]["bytes_per_launch"]
    z = tr["mixed"]["sweep_zeta"][0]
    assert b.kernel_traffic("mixed_learned", "sweep_zeta", z["variant"], N, tr["src"]) == z["bytes_per_launch"]
