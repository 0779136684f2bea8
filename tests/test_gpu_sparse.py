"""The shortcuts for empty and sparse chunks (App. D, Eqs. running median / running mean),
through the C ABI (sub_estimate), against the FP64 oracle at their thresholds.

A chunk with no nonzero bin is sorted without the network, and one with at most 128 by
merging them into the all-zero order; a median tile whose span holds fewer nonzero bins
than half its smallest window writes zeros.  Here spectra are zero except for m nonzero
bins placed in one tile's span, with m on both sides of each threshold: 128/129 nonzero
bins in one chunk, and around ceil(c/2) in the span of an interior tile (c = W) and of the
first tile (whose smallest window is cut by the band edge).  The median is a selection, so
its values must equal the oracle's bit for bit; the mean and median-then-mean within 1e-12.
"""
import numpy as np
import pytest

import oracle
from paper_2602_18560_gb300 import gbsub, synth

pytestmark = pytest.mark.gpu

T = synth.YEAR
W = 1000
KC = 1024          # chunk length for W = 1000 (32 * ceil(W / 32))
N = 6 * KC + 321   # six whole chunks and a ragged one


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    gbsub.lib()


def _f_max(n):
    k_lo, _ = oracle.grid(T, 1e-4, 1e-2)
    return (k_lo + n - 1 + 0.25) / T


def _spectrum(lo, hi, m, seed):
    """Zeros, with m nonzero values (distinct, some tied) at distinct positions in [lo, hi)."""
    rng = np.random.default_rng(seed)
    P = np.zeros(N)
    pos = rng.choice(np.arange(lo, hi), size=m, replace=False)
    v = rng.exponential(1.0, m) * 1e-42
    if m > 4:
        v[: m // 4] = v[0]  # ties
    P[pos] = v
    return P


def _rel(got, ref):
    nz = ref != 0
    assert np.all(got[~nz] == 0)
    return float(np.max(np.abs(got[nz] / ref[nz] - 1.0))) if nz.any() else 0.0


# (span lo, span hi, counts): chunk 3 alone (the sort's 128 cut); chunks 2-3, the span of
# interior tile 3 (smallest window W: 500 nonzero bins are the cut); chunk 0, the first
# tile's span (its first window holds W - W/2 = 500 bins: 250 is the cut)
CASES = [
    (3 * KC, 4 * KC, [1, 127, 128, 129, 130]),
    (2 * KC, 4 * KC, [498, 499, 500, 501, 502]),
    (0, KC, [248, 249, 250, 251, 252]),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_sparse_spans_match_the_oracle(case):
    lo, hi, counts = CASES[case]
    for m in counts:
        P = _spectrum(lo, hi, m, 1000 * case + m)
        for est in (gbsub.MEDIAN, gbsub.MEDIAN_MEAN, gbsub.MEAN):
            with gbsub.Subtraction(T_obs=T, window=W, estimator=est, f_max=_f_max(N)) as s:
                assert s.grid[0] == N
                got = s.estimate(P)
            ref = oracle.smooth(est, W, P)
            if est == gbsub.MEDIAN:
                np.testing.assert_array_equal(got, ref)
            else:
                assert _rel(got, ref) <= 1e-12, (m, est)


@pytest.mark.parametrize("lo,m", [(3 * KC - 250, 500), (3 * KC - 250, 499), (0, 250), (0, 249)])
def test_packed_spans_at_the_median_cut(lo, m):
    # m nonzero bins packed into one window: at the cut (500 in an interior window, 250 in
    # the first window, which the band edge cuts to 500 bins) that window's median is
    # nonzero, so the tile must not take the shortcut; one fewer, and every median is zero
    P = np.zeros(N)
    P[lo: lo + m] = np.linspace(1.0, 2.0, m) * 1e-42
    ref = oracle.smooth(gbsub.MEDIAN, W, P)
    at_cut = m in (250, 500)
    assert np.any(ref != 0) == at_cut
    for est in (gbsub.MEDIAN, gbsub.MEDIAN_MEAN):
        with gbsub.Subtraction(T_obs=T, window=W, estimator=est, f_max=_f_max(N)) as s:
            got = s.estimate(P)
        ref = oracle.smooth(est, W, P)
        if est == gbsub.MEDIAN:
            np.testing.assert_array_equal(got, ref)
        else:
            assert _rel(got, ref) <= 1e-12
