"""Host logic of the batched-form autotuner: K1 choice at equal success,
problem classes, schedule lookup and its JSON form."""
from paper_2507_01439_gb300 import autotune


def test_choose_k1_takes_cheapest_at_best_success():
    assert autotune.choose_k1({100: 20, 250: 24, 500: 24, 1000: 24}) == 250
    assert autotune.choose_k1({100: 24, 250: 24}) == 100
    assert autotune.choose_k1({100: 3, 250: 2, 500: 1}) == 100
    assert autotune.choose_k1({2000: 7}) == 2000


def test_class_key_buckets():
    edges = (1500, 3000, 5000)
    assert autotune.class_key(0.1, 500, edges) == (0.1, 1500)
    assert autotune.class_key(0.1, 1500, edges) == (0.1, 1500)
    assert autotune.class_key(0.6, 1501, edges) == (0.6, 3000)
    assert autotune.class_key(0.6, 9000, edges) == (0.6, 5000)


def test_schedule_lookup_and_json():
    s = autotune.Schedule(flags=0x8, tile="sc2_single+verify256",
                          k1_rules=[[0.1, 1500, 250], [0.1, 5000, 1000], [0.6, 3000, 500]], default_k1=2000)
    assert s.k1_for(1000, 0.1) == 250
    assert s.k1_for(4000, 0.1) == 1000
    assert s.k1_for(9000, 0.1) == 1000          # beyond the last bucket: its K1
    assert s.k1_for(2000, 0.6) == 500
    assert s.k1_for(2000, 0.3) == 2000          # unknown class: the default
    t = autotune.Schedule.from_json(s.to_json())
    assert t == s


def test_tile_candidates_are_distinct_flag_sets():
    vals = list(autotune.TILE_CANDIDATES.values())
    assert len(set(vals)) == len(vals) == 6
