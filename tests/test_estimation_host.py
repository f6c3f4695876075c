"""Host logic of the estimation study (Sec. 6, Experiment 2) in bench.py: the
DST band for a kept share of tiles, the simplex stopping rule and the
parameter-error summary.  CPU only."""
import math
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2008_07437_gb300 import inputs  # noqa: E402


def kept_share(T, d):
    # count the tiles (i, j) of the T x T tile grid with |i - j| < d directly
    return sum(1 for i in range(T) for j in range(T) if abs(i - j) < d) / T / T


@pytest.mark.parametrize("T", [4, 7, 10, 16, 25])
@pytest.mark.parametrize("keep", [0.4, 0.7])
def test_dst_band_is_the_closest_share(T, keep):
    d = bench.dst_band(T, keep)
    best = min(range(1, T + 1), key=lambda e: (abs(kept_share(T, e) - keep), e))
    assert d == best


def test_dst_band_ten_tiles():
    assert bench.dst_band(10, 0.4) == 3 and kept_share(10, 3) == pytest.approx(0.44)
    assert bench.dst_band(10, 0.7) == 5 and kept_share(10, 5) == pytest.approx(0.70)


def _state(f, x):
    q = len(x[0])
    return SimpleNamespace(q=q, initialized=1, f=f, x=x)


def test_nm_converged_rule():
    x = [[0.1, 0.2], [0.1 + 1e-6, 0.2], [0.1, 0.2 - 1e-6]]
    assert bench.nm_converged(_state([1.0, 1.0 + 1e-7, 1.0 + 5e-7], x))
    assert not bench.nm_converged(_state([1.0, 1.0, 1.0 + 2e-6], x))                 # f spread
    assert not bench.nm_converged(_state([1.0, 1.0, 1.0], [[0.1, 0.2], [0.1, 0.2 + 1e-4], [0.1, 0.2]]))
    assert not bench.nm_converged(_state([1.0, 1.0, math.inf], x))
    assert not bench.nm_converged(SimpleNamespace(q=2, initialized=0, f=[0, 0, 0], x=x))


def test_theta_rel_error():
    spec = inputs.ThetaSpec((1.0, 2.0), 0.1, (0.5, 1.0), (0.5,))
    best = SimpleNamespace(sigma2=(1.1, 1.0), a=0.12, nu=(0.5, 1.5), beta=[[1.0, 0.4], [0.4, 1.0]])
    e = bench.theta_rel_error(best, spec)
    assert e["sigma2"] == pytest.approx([0.1, 0.5])
    assert e["a"] == pytest.approx(0.2)
    assert e["nu"] == pytest.approx([0.0, 0.5])
    assert e["beta_abs"] == pytest.approx([0.1])
