"""Pins of the oracle's coarse-graining (Sec. "Coarse-graining of the data": bin averages of
the spectrum and of the frequencies over logarithmically spaced bins), against the partition
computed independently with numpy, closed forms of arithmetic means, and conservation."""
import numpy as np
import pytest

import oracle

YEAR = oracle.YEAR


def bounds(c):
    """First grid index of every bin and the end of the last one."""
    return np.concatenate([[0], np.cumsum(c)])


@pytest.mark.parametrize("T,nb", [(YEAR, 100), (4 * YEAR, 100), (2 * YEAR, 37), (YEAR, 1)])
def test_partition_follows_the_log_edges(T, nb):
    k_lo, n = oracle.grid(T)
    _, _, c = oracle.coarse_grain(T, 1e-4, 1e-2, k_lo, np.zeros(n), nb)
    assert c.sum() == n and np.all(c >= 0)
    e = np.logspace(np.log10(1e-4), np.log10(1e-2), nb + 1)
    b = bounds(c)
    f = (k_lo + np.arange(n)) / T
    for k in range(1, nb):
        # the first frequency of bin k is at or above its lower edge, the one before below
        assert f[b[k]] >= e[k] * (1 - 1e-12)
        assert f[b[k] - 1] < e[k] * (1 + 1e-12)


@pytest.mark.parametrize("T", [YEAR, 4 * YEAR])
def test_means_of_arithmetic_sequences_are_the_midpoints(T):
    k_lo, n = oracle.grid(T)
    a, slope = 3.0e-41, 7.0e-47
    x = a + slope * np.arange(n)
    S, fk, c = oracle.coarse_grain(T, 1e-4, 1e-2, k_lo, x, 100)
    b = bounds(c)
    first, last = b[:-1], b[1:] - 1
    np.testing.assert_allclose(fk, (k_lo + (first + last) / 2.0) / T, rtol=1e-14)
    np.testing.assert_allclose(S, a + slope * (first + last) / 2.0, rtol=1e-12)


def test_totals_are_conserved_and_constants_kept():
    T = 2 * YEAR
    k_lo, n = oracle.grid(T)
    x = np.random.default_rng(4).exponential(1.0, n) * 1e-40
    S, _, c = oracle.coarse_grain(T, 1e-4, 1e-2, k_lo, x, 100)
    assert abs(np.sum(S * c) - np.sum(x)) <= 1e-12 * np.sum(x)
    S1, _, _ = oracle.coarse_grain(T, 1e-4, 1e-2, k_lo, np.full(n, 0.25), 100)
    assert np.all(S1 == 0.25)


def test_empty_bins_give_nan_and_zero_count():
    T = 1.0e5  # a short observation: some low bins hold no grid frequency
    k_lo, n = oracle.grid(T)
    S, fk, c = oracle.coarse_grain(T, 1e-4, 1e-2, k_lo, np.ones(n), 100)
    empty = c == 0
    assert empty.any() and c.sum() == n
    assert np.all(np.isnan(S[empty])) and np.all(np.isnan(fk[empty]))
    assert np.all(S[~empty] == 1.0)
