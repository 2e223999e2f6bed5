"""Host-side pieces of bench.py that shape its JSON line (no GPU): the
roofline object's traffic rule and the workload config's weights statement."""
import bench


def test_roofline_traffic_rule():
    # gridding dominant, region schedule: the capture predates the kernel, so
    # traffic is null and the previous figure stands beside it
    r = bench.roofline_entry("aw_grid (grid_region_kernel + grid_offset_kernel)", 29.1, 80.5, "derived",
                             4.47e12, 153.5, 115.9, region=True, nvalid=63851035, subset=False)
    assert r["traffic"] is None and r["traffic_source"] is None
    prev = r["traffic_previous_region_kernel"]
    assert abs(prev["bytes"] - bench.TRAFFIC_PER_VIS["region"] * 63851035) < 1.0
    assert r["frac"] == 29.1 / 80.5 and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    # degridding dominant: its capture still describes the kernel
    r = bench.roofline_entry("aw_degrid (degrid_items_kernel)", 38.5, 80.5, "derived", 4.47e12, 100.0, 115.9,
                             region=True, nvalid=1000, subset=False)
    assert r["traffic"] == bench.TRAFFIC_PER_VIS["degrid_items_kernel"] * 1000
    assert "traffic_previous_region_kernel" not in r and r["traffic_source"]
    # other schedules and the subset scale: no figure
    r = bench.roofline_entry("aw_grid (grid_offset_kernel)", 20.0, 80.5, "derived", 1.0, 200.0, 100.0,
                             region=False, nvalid=1000, subset=False)
    assert r["traffic"] is None and "traffic_previous_region_kernel" not in r
    r = bench.roofline_entry("aw_grid (grid_region_kernel + grid_offset_kernel)", 20.0, 80.5, "derived", 1.0,
                             200.0, 100.0, region=True, nvalid=1000, subset=True)
    assert r["traffic"] is None and "traffic_previous_region_kernel" not in r


def test_workload_config_states_natural_weights():
    class Ob:
        nvis = 10
        pa_centres = [0.0]
        fbin_freqs = [1.4e9]

    kw = {"N": 64, "OS": 8, "supports": [16], "pa": [0.0], "fbin_freqs": [1.4e9]}
    cfg = bench.workload_config(Ob(), kw, None)
    assert "natural" in cfg["weights"] and "weighted_grid" in cfg["weights"]
