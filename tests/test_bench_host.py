"""bench.py's host-side bookkeeping of the recorded ncu traffic: the source hash ignores
comments and whitespace but not code, and a record taken on other kernel code is reported
as null rather than as a stale figure."""
import bench


def test_code_sha_ignores_comments_and_whitespace_not_code(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("int f(int x) { return x + 1; }  // one\n")
    b.write_text("/* header */\nint f(int x)\n{\n    return x + 1;   // other words\n}\n")
    c.write_text("int f(int x) { return x + 2; }\n")
    assert bench.code_sha(str(a)) == bench.code_sha(str(b))
    assert bench.code_sha(str(a)) != bench.code_sha(str(c))
    assert bench.code_sha(str(a), str(c)) != bench.code_sha(str(a))


def test_ncu_traffic_scales_the_record_and_drops_stale_ones(monkeypatch):
    import os
    csrc = os.path.join(bench.ROOT, "paper_2407_21552_gb300", "csrc")
    sha = bench.code_sha(*bench.update_kernel_sources(csrc))
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {
        "cur": {"source_sha": sha, "read_per_loaded_byte": 1.25, "write_per_block": 0.5},
        "old": {"source_sha": "0" * 16, "read_per_loaded_byte": 1.25, "write_per_block": 0.5}})
    # 2000 blocks, 4000 PDM bytes loaded: 1.25 * 4000 + 0.5 * 2000
    assert bench.ncu_traffic("cur", 2000, 4000.0) == 6000.0
    assert bench.ncu_traffic("old", 2000, 4000.0) is None
    assert bench.ncu_traffic("none", 2000, 4000.0) is None


def test_precompute_alu_roofline_uses_the_record_of_the_current_code(monkeypatch):
    import os
    csrc = os.path.join(bench.ROOT, "paper_2407_21552_gb300", "csrc")
    sha = bench.code_sha(*bench.precompute_kernel_sources(csrc))
    monkeypatch.setattr(bench, "NCU_PRECOMPUTE_INST", {
        "cur": {"source_sha": sha, "warp_instructions": 1.0e9},
        "old": {"source_sha": "0" * 16, "warp_instructions": 1.0e9}})
    r = bench.precompute_alu("cur", 2.0, {"sm_mhz": 2000.0}, 100)
    # 1e9 warp instructions in 2 ms against 4 x 100 SMs x 2 GHz = 8e11 per second
    assert r["achieved"] == 5.0e11 and r["peak"] == 8.0e11 and abs(r["frac"] - 0.625) < 1e-12
    assert bench.precompute_alu("old", 2.0, {"sm_mhz": 2000.0}, 100) is None
    assert bench.precompute_alu("none", 2.0, {"sm_mhz": 2000.0}, 100) is None
