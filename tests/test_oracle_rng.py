"""Pins of the oracle's Philox4x32-10 and of the Gaussian draws built on it (no GPU)."""
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(v, 16) for v in r]
        out = philox.philox4x32_10(np.array(w[:4], dtype=np.uint64).reshape(4, 1), w[4:6])
        assert [int(v) for v in out[:, 0]] == w[6:10]


def test_momenta_and_pseudofermion_moments():
    L, N = 8, 40
    p = philox.draw_momenta(seed=7, traj_counter=3, L=L, Ntau=N)
    R = philox.draw_pseudofermion(seed=7, traj_counter=3, L=L, Ntau=N)
    n = p.size
    assert abs(p.mean()) < 5 * np.sqrt(0.5 / n)
    assert abs(p.var() - 0.5) < 5 * 0.5 * np.sqrt(2.0 / n)
    assert abs(np.mean(np.abs(R) ** 2) - 1.0) < 5 * np.sqrt(1.0 / R.size)
    assert abs(np.mean(R.real * R.imag)) < 5 * 0.5 / np.sqrt(R.size)
    # distinct streams and counters give distinct draws; same inputs repeat exactly
    assert not np.allclose(p, philox.draw_momenta(7, 4, L, N))
    assert np.array_equal(p, philox.draw_momenta(7, 3, L, N))
    u = philox.draw_metropolis(7, 3)
    assert 0.0 <= u < 1.0 and u == philox.draw_metropolis(7, 3)
