"""Host-side logic that needs no GPU: the tuning cache, workload naming and
the benchmark's host description."""
import json

import pytest

import bench
from paper_1903_11749_gb300 import tune


class _Info:
    n, m, instances = 1000, 12000, 0


class _FakeGraph:
    """Stands in for a loaded graph: counts the tuner calls."""

    def __init__(self):
        self.calls = 0

    def info(self):
        return _Info()

    def autotune(self, sample_sources=0, **run):
        self.calls += 1
        return {"chunk_sources": 4, "large_degree": 0, "warps_per_block": 8, "refill_lanes": 16, "ms": 1.5,
                "candidates": 33, "sample_sources": sample_sources}


def test_tuning_cache_hits_and_keys(tmp_path, monkeypatch):
    monkeypatch.setenv("PPR_TUNE_CACHE", str(tmp_path / "tune.json"))
    G = _FakeGraph()
    run = dict(alpha=0.15, R=200, seed=1, topk=32)
    t1 = tune.tuned(G, "GB300", sample_sources=1000, **run)
    t2 = tune.tuned(G, "GB300", sample_sources=1000, **run)
    assert G.calls == 1 and not t1["cached"] and t2["cached"]
    # another sampler, R or device is another entry
    tune.tuned(G, "GB300", sample_sources=1000, sampler=1, **run)
    tune.tuned(G, "other", sample_sources=1000, **run)
    tune.tuned(G, "GB300", sample_sources=1000, **dict(run, R=100))
    assert G.calls == 4
    assert len(json.load(open(tmp_path / "tune.json"))) == 4
    tune.tuned(G, "GB300", sample_sources=1000, refresh=True, **run)
    assert G.calls == 5
    assert tune.launch_kwargs(t1) == {"chunk_sources": 4, "large_degree": 0, "warps_per_block": 8, "refill_lanes": 16}
    # entries cached before the refill threshold existed default to refilling at once
    assert tune.launch_kwargs({"chunk_sources": 2, "large_degree": 0, "warps_per_block": 4})["refill_lanes"] == 0


def test_tuning_cache_survives_a_corrupt_file(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    monkeypatch.setenv("PPR_TUNE_CACHE", str(path))
    G = _FakeGraph()
    t = tune.tuned(G, "GB300", R=10, alpha=0.2)
    assert not t["cached"] and G.calls == 1
    assert len(json.load(open(path))) == 1


@pytest.mark.parametrize("name,graph", [("rmat20", "rmat20"), ("rmat20alias", "rmat20"), ("rmat24plain", "rmat24"),
                                        ("rmat24alias", "rmat24"), ("er1k", "er1k")])
def test_workload_variants_share_their_graph(name, graph):
    assert bench.base_graph(name) == graph
    assert name in bench.WORKLOADS


def test_every_workload_is_described():
    for name, wl in bench.WORKLOADS.items():
        assert {"alpha", "R", "seed", "topk", "segments", "desc"} <= set(wl), name
        assert wl.get("sampler", 0) in (0, 1)
        assert not (wl["segments"] and wl.get("sampler", 0) == 1), name  # segment tables use the prefix rule


def test_replica_workload_and_host_description():
    assert bench.rank_workload(1000, 3, 8) == (0, 1000, 3)  # every source, the rank as the tag
    h = bench.host_cpu()
    assert h["nproc"] >= 1 and h["model"] and h["machine"]


def test_recorded_traffic_needs_the_same_kernel_and_launch(tmp_path, monkeypatch):
    """The recorded DRAM traffic of a walker launch is reported only for the
    kernel source and the launch shape it was captured with."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    entry = {"kernel_hash": bench.kernel_source_hash(), "launch": {"refill_lanes": 24},
             "dram_bytes_per_draw": 123.0}
    (prof / "walker_traffic.json").write_text(json.dumps({"w": entry, "old": dict(entry, kernel_hash="0" * 16)}))
    h = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    shape = {"warps_per_block": 0, "chunk_sources": 0, "large_degree": 0, "l2_persist": 0, "refill_lanes": 24}
    assert bench.recorded_traffic("w", shape)["dram_bytes_per_draw"] == 123.0
    assert bench.recorded_traffic("w", dict(shape, refill_lanes=0)) is None  # another launch shape
    assert bench.recorded_traffic("old", shape) is None  # another kernel source
    assert bench.recorded_traffic("missing", shape) is None
    # the roofline scales the per-draw figure to the launch and reports it as the DRAM fraction
    r = bench.walker_roofline("w", shape, False, draws=1000, sectors=2500, model_sectors=4000, kernel_ms=1.0,
                              peak=1000.0, peak_kind="measured")
    assert r["traffic"] == 123000.0 and abs(r["achieved"] - 123000.0 / 1e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1000.0) < 1e-12 and r["basis"].startswith("ncu DRAM")
    assert abs(r["counted_sector_frac"] - 2500 * 32 / 1e-3 / 1e9 / 1000.0) < 1e-12
    assert abs(r["flat_csr_model"]["frac"] - 4000 * 32 / 1e-3 / 1e9 / 1000.0) < 1e-12
    r = bench.walker_roofline("old", shape, False, 1000, 2500, 4000, 1.0, 1000.0, "measured")
    assert r["traffic"] is None and r["frac"] == r["counted_sector_frac"] and "no current ncu" in r["basis"]

def test_kernel_hash_ignores_comments_only(tmp_path):
    """The traffic records stay valid across comment edits of the walker
    sources and lapse on any code change."""
    src = tmp_path / "paper_1903_11749_gb300" / "csrc"
    src.mkdir(parents=True)
    files = ("walk.cu", "walk_step.cuh", "ppr_internal.cuh", "renumber.cu", "graph.cu")
    for f in files:
        (src / f).write_text("// header\nint f_%s(int x) { return x + 1; }  // trailing\n/* block\n comment */\n" % f[0])
    h0 = bench.kernel_source_hash(str(tmp_path))
    (src / "walk.cu").write_text("// another header\n\nint f_w(int x) { return x + 1; }\n")
    assert bench.kernel_source_hash(str(tmp_path)) == h0
    (src / "walk.cu").write_text("int f_w(int x) { return x + 2; }\n")
    assert bench.kernel_source_hash(str(tmp_path)) != h0


def test_committed_traffic_records_belong_to_the_committed_walker():
    """Every DRAM traffic record under profiles/ was taken on the walker
    sources as they stand (the benchmark reports no DRAM fraction otherwise),
    with a positive figure per draw and the launch shape of its workload."""
    d = json.load(open(bench.os.path.join(bench.ROOT, "profiles", "walker_traffic.json")))
    h = bench.kernel_source_hash()
    for name, e in d.items():
        if name.startswith("_"):
            continue
        assert e["kernel_hash"] == h, name
        assert e["dram_bytes_per_draw"] > 0, name
        assert e["launch"] == {k: v for k, v in bench.WORKLOADS[name].get("launch", {}).items() if v}, name


def test_clock_samples_give_median_max_and_reasons(tmp_path):
    """The sampler's CSV (nvidia-smi query fields) becomes the median SM clock
    under load, the highest maximum clock and the throttle reasons seen."""
    path = tmp_path / "clocks.csv"
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbled line"]
    path.write_text("\n".join(rows) + "\n")

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = bench.Clocks(0, str(path))
    c.proc, c.f = _Done(), open(tmp_path / "unused", "w")
    out = c.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_collector_paused_over_timed_regions():
    import gc
    was = gc.isenabled()
    bench.gc_pause()
    assert not gc.isenabled()
    bench.gc_resume()
    assert gc.isenabled()
    if not was:
        gc.disable()
