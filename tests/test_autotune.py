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


def test_autotune_table_stage_prefers_less_memory_within_noise():
    from paper_1811_06127_gb300 import autotune
    trials = [{"kmer_depth": 13, "pair_steps": 1, "ms_search": 100.0},
              {"kmer_depth": 12, "pair_steps": 1, "ms_search": 101.0},
              {"kmer_depth": 12, "pair_steps": 2, "ms_search": 103.0},
              {"kmer_depth": 14, "pair_steps": 1, "ms_search": 99.5}]
    got = autotune.pick_tables(trials)
    assert (got["kmer_depth"], got["pair_steps"]) == (12, 1)
    assert autotune.pick_tables(trials, tolerance=0.0)["kmer_depth"] == 14


def test_autotune_points_cover_both_stages():
    from paper_1811_06127_gb300 import autotune
    # the library's automatic depth: floor(log4(n+1)) - 1
    assert autotune.auto_kmer_depth(2_000_000_000) == 14
    assert autotune.auto_kmer_depth(256_000_000) == 12
    assert autotune.auto_kmer_depth(8_000_000) == 10
    assert autotune.auto_kmer_depth(10) == 0
    assert autotune.kmer_depth_of(10, 1) == 1
    pts = autotune.points(2_000_000_000)
    assert len(pts) == 3 * 2 * 3 * 3 * 3 * 2
    assert {p["kmer_depth"] for p in pts} == {13, 14, 15}
    assert {p["pair_steps"] for p in pts} == {1, 2}
    assert {(p["interval"], p["chunk"]) for p in pts} == {(i, c) for i in (32, 64, 128)
                                                          for c in (8, 16, 32)}
