"""Pins for the oracle's running estimators (App. D, Eqs. running mean / running median).

Interior bins must equal numpy's sliding-window mean and median (a library
special case); bins near the band edges use the window cut to the band, checked
against a brute force with math.fsum and sorted().
"""
import math

import numpy as np
import pytest
from numpy.lib.stride_tricks import sliding_window_view

import oracle

C = 729.0 / 512.0


def _brute(est, W, P):
    n = len(P)
    out = []

    def bounds(j):
        s = j - W // 2
        return max(0, s), min(n - 1, s + W - 1)

    def med(vals):
        v = sorted(vals)
        c = len(v)
        return v[c // 2] if c % 2 else 0.5 * (v[c // 2 - 1] + v[c // 2])

    meds = [C * med(P[a:b + 1]) for a, b in map(bounds, range(n))]
    for j in range(n):
        a, b = bounds(j)
        if est == oracle.MEAN:
            out.append(math.fsum(P[a:b + 1]) / (b - a + 1))
        elif est == oracle.MEDIAN:
            out.append(meds[j])
        else:
            out.append(math.fsum(meds[a:b + 1]) / (b - a + 1))
    return np.array(out)


def _spectrum(n, seed):
    rng = np.random.default_rng(seed)
    # chi^2_2-like positive values over many decades, some exact zeros and ties
    P = rng.exponential(1.0, n) * 10 ** rng.uniform(-50, -40, n)
    P[rng.random(n) < 0.1] = 0.0
    P[rng.random(n) < 0.05] = P[0]
    return P


@pytest.mark.parametrize("W", [1, 2, 3, 10, 11, 64])
@pytest.mark.parametrize("est", [oracle.MEAN, oracle.MEDIAN, oracle.MEDIAN_MEAN])
def test_estimators_brute_force(est, W):
    P = _spectrum(157, W)
    got = oracle.smooth(est, W, P)
    np.testing.assert_allclose(got, _brute(est, W, list(P)), rtol=1e-14, atol=0)


@pytest.mark.parametrize("W", [999, 1000])
def test_interior_matches_numpy_sliding_window(W):
    n = 6000
    P = _spectrum(n, 3)
    h = W // 2
    win = sliding_window_view(P, W)          # window i covers P[i .. i+W-1] -> output i+h
    out_idx = np.arange(h, h + win.shape[0])
    mean = oracle.smooth(oracle.MEAN, W, P)
    np.testing.assert_allclose(mean[out_idx], win.mean(axis=1), rtol=1e-12)
    med = oracle.smooth(oracle.MEDIAN, W, P)
    np.testing.assert_array_equal(med[out_idx], C * np.median(win, axis=1))
    mm = oracle.smooth(oracle.MEDIAN_MEAN, W, P)
    inner = out_idx[(out_idx >= 2 * h) & (out_idx < n - W + h)]
    mwin = sliding_window_view(med, W)
    np.testing.assert_allclose(mm[inner], mwin[inner - h].mean(axis=1), rtol=1e-12)


def test_window_larger_than_band_is_global():
    P = _spectrum(40, 9)
    W = 1000
    for j, v in enumerate(oracle.smooth(oracle.MEAN, W, P)):
        s, e = max(0, j - W // 2), min(39, j - W // 2 + W - 1)
        assert v == pytest.approx(np.mean(P[s:e + 1]), rel=1e-14)


def test_smooth_at_matches_full():
    P = _spectrum(3000, 4)
    idx = np.array([0, 1, 17, 500, 1499, 2999, 2500])
    for est in (oracle.MEAN, oracle.MEDIAN, oracle.MEDIAN_MEAN):
        full = oracle.smooth(est, 301, P)
        np.testing.assert_array_equal(oracle.smooth_at(est, 301, P, idx), full[idx])


def test_estimators_are_monotone_and_scale():
    P = _spectrum(2000, 5)
    Q = P * np.random.default_rng(1).uniform(0, 1, P.size)  # pointwise smaller
    for est in (oracle.MEAN, oracle.MEDIAN, oracle.MEDIAN_MEAN):
        a, b = oracle.smooth(est, 100, P), oracle.smooth(est, 100, Q)
        assert np.all(b <= a)
        np.testing.assert_allclose(oracle.smooth(est, 100, 4.0 * P), 4.0 * a, rtol=1e-15)
