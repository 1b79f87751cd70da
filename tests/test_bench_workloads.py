"""Host logic of bench.py's workload definitions (CPU): the Delaunay graph workload colours by
Jones-Plassmann with random 32-bit priorities as the workload is stated, its _ldf variant with
the sampler's default largest-degree-first order, and the oracle's CPU baseline colours each
the same way the sampler does."""
import numpy as np

import bench
import oracle
from paper_1702_05518_gb300 import gmrf as g


def _colours(spec, ldf):
    f = spec["fields"][0]
    colors, k = oracle.color_graph(f["row_ptr"], f["col_idx"], f.get("color_seed", 0), ldf=ldf)
    return np.asarray(colors), int(k)


def test_delaunay_workload_takes_random_priorities():
    spec = bench.workload_spec("delaunay16k")
    assert spec["color_random"] is True
    assert "random 32-bit priorities" in spec["name"]
    kw = bench.sampler_kwargs(spec, g, spec["seed"])
    assert kw["flags"] == g.FLAG_COLOR_RANDOM
    # an override (the profile case turns graphs off) keeps the colouring flag
    assert bench.sampler_kwargs(spec, g, spec["seed"], graph_sweeps=0)["flags"] == g.FLAG_COLOR_RANDOM


def test_delaunay_ldf_variant_takes_the_default_order():
    spec = bench.workload_spec("delaunay16k_ldf")
    assert not spec["color_random"]
    assert "largest-degree-first" in spec["name"]
    assert "flags" not in bench.sampler_kwargs(spec, g, spec["seed"])


def test_delaunay_colour_counts_of_the_two_orders():
    # one colour step per colour: the random-priority order needs 7 on this graph, largest
    # degree first 6; both colourings are proper
    spec = bench.workload_spec("delaunay16k")
    f = spec["fields"][0]
    rp, ci = np.asarray(f["row_ptr"]), np.asarray(f["col_idx"])
    src = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    for ldf, want in ((False, 7), (True, 6)):
        colors, k = _colours(spec, ldf)
        assert k == want
        assert not np.any(colors[src] == colors[ci])


def test_other_workloads_keep_the_default_colouring():
    for name in ("image64", "paper50"):
        spec = bench.workload_spec(name)
        assert not spec.get("color_random")
        assert "flags" not in bench.sampler_kwargs(spec, g, spec["seed"])
