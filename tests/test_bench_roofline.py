"""The roofline's DRAM traffic in the benchmark line: a stored ncu figure, reported only for the
workload and settings it was captured at, and labelled as stored (checked on the CPU)."""
import bench

TUNED = {"bucket": 16, "group": 64, "list_chunk": 128, "tuned": True}


def test_nfw_box_reports_the_stored_launch_bytes():
    t, src = bench.stored_traffic("nfw2m", None, TUNED, "k_pc", {"n_pc_pairs": 412271101})
    assert t == bench.NCU_TRAFFIC["k_pc"] and "stored" in src


def test_large_box_scales_the_stored_rate_by_its_own_pairs():
    pc = 13654331836
    t, src = bench.stored_traffic("learned134m", None, TUNED, "k_pc", {"n_pc_pairs": pc, "n_pp_pairs": 1})
    assert abs(t - bench.NCU_TRAFFIC_PER_PAIR_512["k_pc"] * pc) < 1.0 and "stored" in src and "pairs" in src
    # the fixed-theta solve the rate came from gives back the captured bytes
    t, _ = bench.stored_traffic("learned134m", None, TUNED, "k_pc", {"n_pc_pairs": 31659347808})
    assert abs(t - 54254844416) < 1e3
    t, _ = bench.stored_traffic("learned134m", None, TUNED, "k_pp", {"n_pp_pairs": 128335887451})
    assert abs(t - 18396550144) < 1e3


def test_other_settings_sizes_and_workloads_report_none():
    other = dict(TUNED, group=48)
    for args in (("nfw2m", None, other, "k_pc", {}), ("nfw2m", 262144, TUNED, "k_pc", {}),
                 ("batch64", None, TUNED, "k_pc", {}), ("learned134m", None, TUNED, "k_pc", {}),
                 ("learned134m", None, None, "k_pc", {"n_pc_pairs": 5})):
        t, src = bench.stored_traffic(*args)
        assert t is None and "no ncu capture" in src
