"""Host logic of the tile-width and sort-interval autotuner (CPU; the GPU probe is faked).

The probe itself (copies of a run stepping concurrently, CUDA events around whole
periods) runs in the GPU ensemble tests; here: the density classes, the candidate pairs,
the number of concurrent copies, and that the pair with the least time is kept and cached
per key.
"""
import pytest

from paper_2410_18414_gb300 import autotune, pic


def test_density_class_is_the_nearest_class():
    assert autotune.density_class(16) == 16
    assert autotune.density_class(20) == 16
    assert autotune.density_class(30) == 32
    assert autotune.density_class(50) == 64
    assert autotune.density_class(100) == 64
    assert autotune.density_class(24) == 16  # a tie goes to the smaller class


def test_candidates_keep_tiles_of_at_most_half_the_grid():
    pairs = autotune.candidates(16)
    assert {t for t, _ in pairs} == {4, 8}
    assert len(pairs) == 2 * len(autotune.SORT_INTERVALS)
    assert {t for t, _ in autotune.candidates(32)} == {4, 8, 16}
    assert autotune.candidates(4) == []


def test_copies_fill_about_four_million_particles_up_to_sixteen():
    assert autotune.copies_for(1 << 20) == 4
    assert autotune.copies_for(3 << 20) == 2     # rounded up
    assert autotune.copies_for(16384) == 16      # capped
    assert autotune.copies_for(10 ** 8) == 1
    assert autotune.copies_for(0) == 16


def test_tune_keeps_the_fastest_pair_and_caches_it_per_key(monkeypatch):
    calls = []

    def fake_probe(n_axis, ppc, tile, s, p, precision, stepper, bdf_order, periods):
        calls.append((n_axis, ppc, tile, s))
        return 1.0 + abs(tile - 8) + 0.1 * abs(s - 4)  # fastest at (8, 4)

    monkeypatch.setattr(autotune, "probe_ms", fake_probe)
    monkeypatch.setattr(autotune, "_cache", {})
    t, s, ms = autotune.tune(64, 60)
    assert (t, s) == (8, 4)
    assert len(ms) == len(autotune.candidates(64)) == len(calls)
    assert all(c[1] == 64 for c in calls)  # probed at the density class, not the raw ppc
    n = len(calls)
    t2, s2, ms2 = autotune.tune(64, 70)   # same key: grid, class 64, order, form
    assert (t2, s2) == (8, 4) and ms2 == {} and len(calls) == n
    autotune.tune(64, 20)                  # another density class probes again
    assert len(calls) == 2 * n
    autotune.tune(64, 60, precision=pic.FP64)  # another form probes again
    assert len(calls) == 3 * n


@pytest.mark.parametrize("n_axis", [8, 48, 128])
def test_candidate_tiles_are_at_most_half_the_grid(n_axis):
    for t, s in autotune.candidates(n_axis):
        assert 2 * t <= n_axis and s in autotune.SORT_INTERVALS
