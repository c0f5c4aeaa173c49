"""Host logic of bench.py on CPU: the roofline traffic is read from the committed ncu summary only
while the kernel sources hash to the value recorded there."""
import bench


def _recorded_hash():
    import os
    for ln in open(os.path.join(bench.ROOT, "profiles", "k_m2l_sphere1m.md")):
        if ln.startswith("- source_sha256_16:"):
            return ln.split(":", 1)[1].strip().strip("`")
    return None


def test_traffic_applies_exactly_when_the_sources_match_the_summary():
    t = bench.measured_traffic("sphere1m", "fp32", 1, "apply")
    if _recorded_hash() == bench.source_hash():
        assert t is not None and t["bytes_per_step"] > 1e9
        assert t["source"] == "profiles/k_m2l_sphere1m.md"
    else:
        assert t is None


def test_traffic_is_none_for_other_workloads_and_changed_sources(monkeypatch, tmp_path):
    assert bench.measured_traffic("sphere256k", "fp32", 1, "apply") is None
    assert bench.measured_traffic("sphere1m", "fp64", 1, "apply") is None
    assert bench.measured_traffic("sphere1m", "fp32", 4, "apply") is None
    # a kernel source that differs from the profiled one: the summary no longer applies
    changed = tmp_path / "far.cu"
    changed.write_text("// changed\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCES", (str(changed),))
    assert bench.measured_traffic("sphere1m", "fp32", 1, "apply") is None


def test_oracle_mlfma_cpu_reference_runs():
    r = bench.oracle_mlfma_rate("sphere4k")
    assert "error" not in r, r
    assert r["value"] > 0 and r["unit"] == "points/s" and r["apply_s"] > 0


def test_config_names_the_sampled_operator_form():
    import argparse
    prm = {"digits": 3}
    base = dict(workload=bench.WORKLOAD, digits=0, precision="fp32", nrhs=1, mode="apply")
    plain = bench.config_dict(argparse.Namespace(**base, sampled_operators=0), 1 << 20, prm)
    smp = bench.config_dict(argparse.Namespace(**base, sampled_operators=6), 1 << 20, prm)
    assert "sampled operators" not in plain["workload"]
    assert smp["workload"].endswith("sampled operators (oversampling 6)")
