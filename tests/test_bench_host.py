"""Host logic of the benchmark (no GPU): the kernel-source fingerprint that
ties a committed DRAM-traffic capture to the code it was taken on, and the
whole-job rate."""
import bench


def _write(tmp_path, name, text):
    p = tmp_path / name
    p.write_text(text)
    return str(p)


def test_source_hash_ignores_comments_and_whitespace(tmp_path, monkeypatch):
    a = _write(tmp_path, "a.cu", "int f(int x) {\n  return x + 1;  // add one\n}\n/* block\ncomment */\n")
    b = _write(tmp_path, "b.cu", "int f(int x){return x+1;}")
    c = _write(tmp_path, "c.cu", "int f(int x){return x+2;}")
    monkeypatch.setattr(bench, "KERNEL_SOURCES", [a])
    ha = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "KERNEL_SOURCES", [b])
    assert bench.kernel_source_hash() == ha
    monkeypatch.setattr(bench, "KERNEL_SOURCES", [c])
    assert bench.kernel_source_hash() != ha


def test_profiled_traffic_only_for_the_current_source(tmp_path, monkeypatch):
    src = _write(tmp_path, "k.cu", "__global__ void k() {}")
    monkeypatch.setattr(bench, "KERNEL_SOURCES", [src])
    h = bench.kernel_source_hash()
    good = _write(tmp_path, "good.md", f"- kernel source sha256[:16]: `{h}`\n"
                                       "- dram bytes per launch (read+write): 6544248320\n")
    stale = _write(tmp_path, "stale.md", "- kernel source sha256[:16]: `0123456789abcdef`\n"
                                         "- dram bytes per launch (read+write): 6544248320\n")
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", good)
    assert bench.profiled_traffic() == 6544248320.0
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", stale)
    assert bench.profiled_traffic() is None
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(tmp_path / "missing.md"))
    assert bench.profiled_traffic() is None


def test_committed_profile_is_parseable():
    """The committed summary carries both fields the benchmark reads."""
    text = open(bench.PROFILE_SUMMARY).read()
    assert "kernel source sha256[:16]:" in text and "dram bytes per launch (read+write):" in text


def test_whole_job_rate_is_all_ranks_over_the_slowest():
    assert bench.whole_job_rate(100, 4, 2.0) == 200.0
    assert bench.whole_job_rate(100, 1, 0.5) == 200.0


def test_clock_summary_keeps_the_worst_region():
    """Several timed regions report one clock record: the lowest median SM
    clock, the highest maximum and every throttle reason any region saw."""
    recs = [{"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5},
            {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4}]
    s = bench.timed_clocks_summary(recs)
    assert s == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 9, "regions": 2}
    assert bench.timed_clocks_summary([]) is None
