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


def test_rooflines_follow_their_definitions():
    """The bench line's roofline objects from synthetic kernel times: FP64 by
    counted flops of the dominant kernel against the FMA probe; FP32 by the
    stage's algorithmic bytes against the HBM peak, with the dominant kernel's
    compulsory bytes beside it (plus the sensor's where the viscous kernel
    forms the classes)."""
    b = _bench(ROOT)
    N = 256 ** 3
    peaks = {"hbm_gbs": 6800.0}
    fma = {"fp64": 1.25, "fp32": 76.0}
    prof = {"prim": 0.9, "sensor": 0.8, "visc_flux": 4.7, "sweep_xi": 5.2, "sweep_eta": 5.5, "sweep_zeta": 5.6}
    var = {"visc": [0, 0], "xi": [1, 0], "eta": [2, 0], "zeta": [2, 64]}
    r = {"prof": prof, "variants": var, "value": 7.0e8}
    roof, stage = b.rooflines("fp64", r, N, peaks, fma, "none", 1)
    assert roof["bound"] == "alu" and roof["kernel"] == "sweep_zeta"
    ach = b.FP64_FLOPS["sweep_zeta"] * N / (5.6e-3) / 1e12
    assert abs(roof["achieved"] - ach) < 1e-12 * ach and abs(roof["frac"] - ach / 1.25) < 1e-12
    assert roof["traffic"] is None  # sources other than the recorded ones
    flops = sum(b.FP64_FLOPS.values())
    assert abs(stage["fp64_frac"] - flops * 7.0e8 / 1e12 / 1.25) < 1e-12
    assert abs(stage["hbm_frac"] - b.ALG_BYTES_PER_POINT_STAGE * 7.0e8 / 1e9 / 6800.0) < 1e-12
    # FP32 bulk, the viscous kernel dominant and forming the plain sensor's classes
    prof32 = {"prim": 0.17, "sensor": 0.002, "visc_flux": 0.64, "sweep_xi": 0.41, "sweep_eta": 0.52,
              "sweep_zeta": 0.61}
    r32 = {"prof": prof32, "variants": {"visc": [0, 0], "xi": [0, 0], "eta": [1, 16], "zeta": [1, 16]},
           "value": 6.4e9}
    roof, _ = b.rooflines("mixed", r32, N, peaks, fma, "none", 1)
    assert roof["bound"] == "hbm" and roof["traffic_kernel"] == "visc_flux"
    assert abs(roof["achieved"] - b.ALG_BYTES_PER_POINT_STAGE * N / (sum(prof32.values()) * 1e-3) / 1e9) < 1e-6
    kc = roof["kernel_compulsory"]
    assert kc["bytes_per_node"] == b.MIXED_BYTES["visc_flux"] + b.MIXED_BYTES["sensor"]
    # the 2.5-D viscous kernel leaves the classes to the sensor kernel
    r32["variants"]["visc"] = [2, 32]
    roof, _ = b.rooflines("mixed", r32, N, peaks, fma, "none", 1)
    assert roof["kernel_compulsory"]["bytes_per_node"] == b.MIXED_BYTES["visc_flux"]
