"""Host logic of bench.py that its JSON line depends on (CPU only): the DRAM traffic taken from
a committed ncu summary only while the kernel sources still hash to the profiled version, and the
summary of nvidia-smi clock samples (median SM clock, maximum, active throttle reasons)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_host_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_committed_profiles_carry_hash_and_traffic(bench):
    """Every committed summary names the source hash it was taken on and the DRAM bytes of one
    full-size launch: at least the algorithmic reads (16 B x 1e7 points); up to the L2's 129 MB of
    the 16 B x 1e7 output bytes can still sit in L2 when the kernel ends and go uncounted."""
    import re
    for which, (path, files) in bench.PROFILES.items():
        text = open(path).read()
        assert re.search(r"kernel_source_hash:\s*[0-9a-f]{16}", text), which
        m = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
        assert m and float(m.group(1)) >= 1.6e8, which


def _stamped(bench, which, tmp_path, name):
    """The committed summary of `which`, re-stamped with the hash of the current sources."""
    import re
    path, files = bench.PROFILES[which]
    text = re.sub(r"(kernel_source_hash:\s*)[0-9a-f]+", lambda m: m.group(1) + bench.kernel_hash(files),
                  open(path).read())
    p = tmp_path / name
    p.write_text(text)
    return p, text, files


def test_traffic_is_dropped_once_the_kernel_changes(bench, tmp_path, monkeypatch):
    _, text, files = _stamped(bench, "f64", tmp_path, "stamped.md")
    good = bench.kernel_hash(files)
    stale = tmp_path / "stale.md"
    stale.write_text(text.replace(good, "0" * len(good)))
    monkeypatch.setitem(bench.PROFILES, "f64", (str(stale), files))
    assert bench.profiled_traffic("f64") is None
    fresh = tmp_path / "fresh.md"
    fresh.write_text(text)
    monkeypatch.setitem(bench.PROFILES, "f64", (str(fresh), files))
    assert bench.profiled_traffic("f64") is not None
    monkeypatch.setitem(bench.PROFILES, "f64", (str(tmp_path / "absent.md"), files))
    assert bench.profiled_traffic("f64") is None


def test_profiled_counters_follow_the_same_rule(bench, tmp_path, monkeypatch):
    """The pipe-utilisation counters reported beside each roofline come from the same summaries,
    as fractions, under the same source-hash rule."""
    expect = {"f64": "fp64_pipe_active_pct", "mixed": "issue_active_pct"}
    for which, key in expect.items():
        fresh, text, files = _stamped(bench, which, tmp_path, "fresh_%s.md" % which)
        assert key + ":" in text, which
        monkeypatch.setitem(bench.PROFILES, which, (str(fresh), files))
        v = bench.profiled_fraction(which, key)
        assert v is not None and 0.0 < v <= 1.0, which
        stale = tmp_path / ("stale_%s.md" % which)
        stale.write_text(text.replace(bench.kernel_hash(files), "f" * 16))
        monkeypatch.setitem(bench.PROFILES, which, (str(stale), files))
        assert bench.profiled_fraction(which, key) is None
        monkeypatch.setitem(bench.PROFILES, which, (str(fresh), files))
        assert bench.profiled_field(which, "no_such_counter") is None


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def test_clock_samples_summary(bench, tmp_path):
    rows = [
        "0, 2070, 2070, 910.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.4, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1402.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(rows) + "\n")
    c = bench.Clocks(0)
    c.proc, c.path = _Done(), str(p)
    out = c.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not p.exists()  # the sample file is removed


def test_clock_summary_without_sampler(bench):
    c = bench.Clocks(0)
    assert c.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
