"""The seeded input generators shared by the GPU tests, the benchmark and the
oracle checks (CPU only): the counter-based generator against the published
SplitMix64 sequence, window extraction, densities and reproducibility."""
import numpy as np
import pytest

from paper_2406_17284_gb300 import inputs

_MASK = (1 << 64) - 1


def splitmix64_int(seed: int, i: int) -> int:
    """The generator's definition in plain Python integers (mod 2^64)."""
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def test_splitmix64_matches_published_sequence():
    # SplitMix64 from state 0: the first three outputs of the reference generator
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = inputs.splitmix64(np.arange(3, dtype=np.uint64), 0)
    assert [int(v) for v in got] == want


@pytest.mark.parametrize("seed", [0, 1, 2024, (1 << 63) + 12345])
def test_splitmix64_vectorised_equals_integer_definition(seed):
    counters = np.array([0, 1, 2, 1000, 123456789, (1 << 40) + 7], dtype=np.uint64)
    got = inputs.splitmix64(counters, seed)
    assert [int(v) for v in got] == [splitmix64_int(seed, int(i)) for i in counters]


@pytest.mark.parametrize("y0,x0,h,w", [(0, 0, 37, 51), (100, 200, 64, 64), (-5, -7, 20, 30),
                                       (250, 390, 40, 60), (-3, 420, 10, 30)])
def test_windows_are_slices_of_the_grid(y0, x0, h, w):
    H, W = 300, 437
    full_b = inputs.bernoulli(H, W, 0.37, 99)
    full_u = inputs.uniform_states(H, W, 16, 98)
    wb = inputs.bernoulli_window(H, W, 0.37, 99, y0, x0, h, w)
    wu = inputs.uniform_states_window(H, W, 16, 98, y0, x0, h, w)
    ref_b = np.zeros((h, w), np.uint8)
    ref_u = np.zeros((h, w), np.uint8)
    ya, yb, xa, xb = max(y0, 0), min(y0 + h, H), max(x0, 0), min(x0 + w, W)
    ref_b[ya - y0:yb - y0, xa - x0:xb - x0] = full_b[ya:yb, xa:xb]
    ref_u[ya - y0:yb - y0, xa - x0:xb - x0] = full_u[ya:yb, xa:xb]
    assert np.array_equal(wb, ref_b) and np.array_equal(wu, ref_u)


def test_bernoulli_cells_follow_the_threshold_rule():
    H, W, p, seed = 64, 80, 0.3, 5
    g = inputs.bernoulli(H, W, p, seed)
    t = int(np.floor(p * 2.0 ** 64))
    want = np.array([[1 if splitmix64_int(seed, y * W + x) < t else 0 for x in range(W)] for y in range(H)], np.uint8)
    assert np.array_equal(g, want)


def test_uniform_states_follow_the_multiply_shift_rule():
    H, W, C, seed = 40, 50, 16, 7
    g = inputs.uniform_states(H, W, C, seed)
    want = np.array([[((splitmix64_int(seed, y * W + x) >> 32) * C) >> 32 for x in range(W)] for y in range(H)], np.uint8)
    assert np.array_equal(g, want)


@pytest.mark.parametrize("p", [0.0, 0.2, 0.5, 0.9, 1.0])
def test_bernoulli_density(p):
    g = inputs.bernoulli(1024, 1024, p, 11)
    n = g.size
    assert abs(g.mean() - p) <= 6 * np.sqrt(max(p * (1 - p), 1e-12) / n) + 1e-12
    assert set(np.unique(g)) <= {0, 1}


def test_uniform_states_cover_all_states_evenly():
    C = 16
    g = inputs.uniform_states(512, 512, C, 3)
    counts = np.bincount(g.ravel(), minlength=C)
    assert counts.size == C and counts.min() > 0
    expect = g.size / C
    assert np.all(np.abs(counts - expect) < 6 * np.sqrt(expect))


def test_seeds_are_reproducible_and_distinct():
    a = inputs.bernoulli(200, 300, 0.5, 1)
    assert np.array_equal(a, inputs.bernoulli(200, 300, 0.5, 1))
    assert not np.array_equal(a, inputs.bernoulli(200, 300, 0.5, 2))


def test_batch_instances_workload_ranges():
    specs = inputs.batch_instances(256, seed=2024)
    assert specs == inputs.batch_instances(256, seed=2024)
    for d in specs:
        assert 64 <= d["H"] <= 2048 and 64 <= d["W"] <= 2048
        assert 1 <= d["rule"]["r"] <= 16 and d["rule"]["M"] in (0, 1) and d["rule"]["C"] == 2
        assert 0.2 <= d["p"] <= 0.6
    assert len({d["seed"] for d in specs}) == len(specs)


def test_patterns_are_the_textbook_shapes():
    g = np.zeros((8, 8), np.uint8)
    inputs.place(g, "glider", 1, 1)
    assert int(g.sum()) == 5
    for name, cells in (("blinker", 3), ("block", 4)):
        h = np.zeros((8, 8), np.uint8)
        inputs.place(h, name, 2, 2)
        assert int(h.sum()) == cells
