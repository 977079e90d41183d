"""The seeded input generators shared by the oracle and the GPU tests: the
counter-based SplitMix64 against its published outputs, and the uniform
samples built on it."""
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "splitmix64_seed0.txt")
GAMMA = 0x9E3779B97F4A7C15


def test_splitmix64_matches_the_published_sequence():
    want = [int(l, 16) for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    # synth.splitmix64(x) mixes x + gamma: the generator's output from state x
    states = np.array([(k * GAMMA) & ((1 << 64) - 1) for k in range(len(want))], dtype=np.uint64)
    got = [int(v) for v in synth.splitmix64(states)]
    assert got == want


def test_uniform01_is_deterministic_in_range_and_uniform():
    a = synth.uniform01(7, 1, 200_000)
    assert np.array_equal(a, synth.uniform01(7, 1, 200_000))
    assert a.min() >= 0.0 and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 5 * (1 / 12) ** 0.5 / len(a) ** 0.5
    hist = np.histogram(a, bins=20, range=(0, 1))[0]
    e = len(a) / 20
    assert ((hist - e) ** 2 / e).sum() < 45          # chi-square, 19 dof, p ~ 1e-3
    b = synth.uniform01(7, 2, 200_000)               # another component: another stream
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.02
    assert not np.array_equal(a[:100], synth.uniform01(8, 1, 100))
