"""The autotuner's search on the CPU, with a made-up cost in place of GPU timings."""
import json


def test_coordinate_descent_finds_a_separable_optimum():
    from paper_2301_01356_gb300 import autotune as A
    want = dict(cc_local=16384, cc_sample=0, ruler_stride=32, lcc_sample=2, chase_chains=2, rank_variant=1,
                grid_ctas=-4, cc_order=1, hub_deg=-1, cc_ldd=0)
    calls = []

    def measure(cfg, reps):
        calls.append((json.dumps(cfg, sort_keys=True), reps))
        return 1.0 + sum(cfg[k] != v for k, v in want.items()) + 0.001 * (reps == 30)

    best, ms, times = A._search(measure, 8, 30)
    assert best == want
    assert abs(ms - 1.001) < 1e-9
    # every knob value is tried once from the running best, then three finalists again
    n_values = sum(len(ch) for _, ch in A.KNOBS)
    assert len([c for c in calls if c[1] == 8]) <= n_values
    assert len([c for c in calls if c[1] == 30]) == 3
    assert set(json.loads(k)["ruler_stride"] for k in times) == {8, 16, 32, 64}


def test_knob_values_are_valid_configurations():
    """Every value the tuner tries is one the library accepts (checked by its rules)."""
    from paper_2301_01356_gb300 import autotune as A
    for _, choices in A.KNOBS:
        for ch in choices:
            cfg = {**A.DEFAULT, **ch}
            assert cfg["ruler_stride"] >= 8 and cfg["ruler_stride"] & (cfg["ruler_stride"] - 1) == 0
            assert cfg["cc_local"] == 0 or 1024 <= cfg["cc_local"] <= 16384
            assert cfg["chase_chains"] in (1, 2, 4) and cfg["rank_variant"] in (0, 1) and cfg["cc_order"] in (0, 1)
            assert -64 <= cfg["grid_ctas"] <= 0 and 0 <= cfg["lcc_sample"] <= 4
            assert cfg["hub_deg"] in (-1, 0) or cfg["hub_deg"] >= 32
            assert 0 <= cfg["cc_ldd"] <= 64 and (cfg["cc_ldd"] == 0 or cfg["cc_local"] == cfg["cc_sample"] == 0)
