"""Autotuner host logic (no GPU): the choice among timed trials."""


def test_autotune_pick_prefers_the_smaller_index_within_noise():
    from paper_1811_06127_gb300 import autotune
    trials = [{"interval": 32, "warps_per_block": 8, "ms_search": 100.0},
              {"interval": 64, "warps_per_block": 8, "ms_search": 101.5},
              {"interval": 64, "warps_per_block": 4, "ms_search": 101.0},
              {"interval": 128, "warps_per_block": 8, "ms_search": 103.0}]
    got = autotune.pick(trials)
    assert (got["interval"], got["warps_per_block"]) == (64, 4)   # within 2%, fastest of I=64
    assert autotune.pick(trials, tolerance=0.0)["interval"] == 32
    assert autotune.pick([{"interval": 32, "ms_search": 50.0},
                          {"interval": 64, "ms_search": 60.0}])["interval"] == 32
