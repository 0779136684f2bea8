"""Pins for the oracle's source model: bins swept by a chirp, their weights,
the power normalisation K = 1/5 and the SNR of a single-bin source.

Independent references used here:
  * the instantaneous frequency of the phase Taylor expansion (Sec. II.A),
    sampled finely in time, gives the time fraction spent in each bin;
  * numerical quadrature of the waveform Eq. (GB waveform) over inclination and
    phase gives <h+^2 + hx^2> = (2/5) A^2;
  * a library FFT of a sampled tone gives the one-sided periodogram
    2 df |h~|^2 = T x (mean square), and 4 df |h~|^2 / S per channel for the
    discretised inner product.
"""
import math

import numpy as np
import pytest

import oracle

T1 = oracle.YEAR


def _time_fractions(T, f, fdot, k_lo, n, m=400_000):
    """Fraction of [0, T] during which f + fdot t lies in cell [k-1/2, k+1/2)/T."""
    t = (np.arange(m) + 0.5) / m * T
    u = (f + fdot * t) * T
    k = np.floor(u + 0.5).astype(np.int64)
    inb = (k >= k_lo) & (k < k_lo + n)
    ks, cnt = np.unique(k[inb], return_counts=True)
    return dict(zip((ks - k_lo).tolist(), (cnt / m).tolist()))


@pytest.mark.parametrize("sweep_bins, offset", [
    (0.0, 0.3), (0.01, 0.2), (0.4, 0.45), (1.0, -0.2), (3.7, 0.1), (25.5, 0.33), (-2.6, 0.0),
])
def test_weights_equal_time_fraction_in_bin(sweep_bins, offset):
    T = T1
    k_lo, n = oracle.grid(T)
    k0 = k_lo + 5000
    f = (k0 + offset) / T
    fdot = sweep_bins / (T * T)
    j, w = oracle.source_pieces(T, k_lo, n, f, fdot)
    ref = _time_fractions(T, f, fdot, k_lo, n)
    got = dict(zip(j.tolist(), w.tolist()))
    assert set(ref) <= set(got)
    tol = 4.0 / 400_000 * max(1.0, 1.0)
    for key, val in got.items():
        assert val == pytest.approx(ref.get(key, 0.0), abs=tol)
    assert math.fsum(w) == pytest.approx(1.0, abs=1e-14)


def test_zero_sweep_goes_to_nearest_bin_and_ties_go_up():
    T = T1
    k_lo, n = oracle.grid(T)
    k0 = k_lo + 100
    for off, expect in ((0.49, 0), (-0.5, 0), (0.5, 1), (-0.51, -1)):
        f = (k0 + off) / T
        j, w = oracle.source_pieces(T, k_lo, n, f, 0.0)
        # f T may round away from the exact half; compare with the rounded value itself
        u = f * T
        assert j.tolist() == [int(math.floor(u + 0.5)) - k_lo]
        assert w.tolist() == [1.0]
        if off not in (-0.5, 0.5):
            assert j[0] == 100 + expect


def test_band_edges_drop_weight_outside():
    T = T1
    k_lo, n = oracle.grid(T)
    # sweep of 10 bins starting 3 bins below the band: 7 bins inside
    f = (k_lo - 3.0 - 0.5) / T
    fdot = 10.0 / T**2
    j, w = oracle.source_pieces(T, k_lo, n, f, fdot)
    assert j.min() == 0
    assert math.fsum(w) == pytest.approx(0.7, abs=1e-12)
    # entirely outside: nothing
    j, w = oracle.source_pieces(T, k_lo, n, (k_lo + n + 5) / T, 1.0 / T**2)
    assert j.size == 0
    # the top edge
    f = (k_lo + n - 1 - 0.5) / T
    j, w = oracle.source_pieces(T, k_lo, n, f, 4.0 / T**2)
    assert j.max() == n - 1
    assert math.fsum(w) == pytest.approx(0.25, abs=1e-12)


def test_waveform_average_gives_two_fifths():
    # <h+^2 + hx^2> over isotropic inclination (cos i uniform) and phase, per unit A^2,
    # from Eq. (GB waveform): h+ = A (1 + cos^2 i)/2 cos phi, hx = A cos i sin phi.
    ci, wi = np.polynomial.legendre.leggauss(64)          # cos(iota) on [-1, 1]
    phi = (np.arange(256) + 0.5) / 256 * 2 * np.pi
    hp = 0.5 * (1 + ci[:, None] ** 2) * np.cos(phi[None, :])
    hx = ci[:, None] * np.sin(phi[None, :])
    avg = np.sum(wi[:, None] * (hp**2 + hx**2)) / 2.0 / phi.size
    assert avg == pytest.approx(0.4, rel=1e-13)
    # The oracle's channel power of a single-bin source is T * (R/2) * avg * A^2
    # (sky/polarisation average of F+^2 and Fx^2 is R/2 each).
    T = T1
    k_lo, n = oracle.grid(T)
    S, R = oracle.tables(T, k_lo, n, True)
    j0 = 7777
    f = (k_lo + j0) / T
    A = 3e-22
    D = oracle.deposit(T, k_lo, n, [A], [f], [0.0])
    P = oracle.power(T, R, D)
    assert P[j0] == pytest.approx(T * (R[j0] / 2.0) * avg * A * A, rel=1e-13)
    assert np.count_nonzero(P) == 1


def test_periodogram_of_tone_is_T_times_mean_square():
    # One-sided periodogram 2 df |h~(f_k)|^2 with h~ = dt * DFT, for a tone centred on a bin.
    T = 4096.0
    fs = 8.0
    N = int(T * fs)
    t = np.arange(N) / fs
    a = 1.7
    k = 300
    x = a * np.cos(2 * np.pi * (k / T) * t + 0.3)
    X = np.fft.rfft(x) / fs
    df = 1.0 / T
    P = 2 * df * np.abs(X) ** 2
    assert P[k] == pytest.approx(T * a * a / 2.0, rel=1e-10)
    # and the discretised inner product 4 df sum |h~|^2 / S equals 2 P / S per channel
    S = 2.5
    inner = 4 * df * np.sum(np.abs(X) ** 2) / S
    assert inner == pytest.approx(2 * P[k] / S, rel=1e-9)


def test_snr_single_bin_source_against_instrument_noise():
    # rho^2 = sum over A, E of 2 P/S with P = T R A^2 / 5 (two equal channels).
    T = 4 * oracle.YEAR
    k_lo, n = oracle.grid(T)
    S, R = oracle.tables(T, k_lo, n, True)
    rng = np.random.default_rng(5)
    js = rng.integers(0, n, 50)
    A = 10 ** rng.uniform(-23, -21, 50)
    f = (k_lo + js) / T
    r2 = oracle.snr2(T, k_lo, n, S, R, None, A, f, np.zeros(50))
    per_channel = 2 * (T * R[js] * A * A / 5.0) / S[js]
    np.testing.assert_allclose(r2, 2 * per_channel, rtol=1e-13)
    # a multi-bin source sums its pieces
    f1 = (k_lo + 1000.2) / T
    fdot = 17.3 / T**2
    j, w = oracle.source_pieces(T, k_lo, n, f1, fdot)
    expect = math.fsum(4 * T * R[j] * w * 1e-44 / 5 / S[j] for j, w in zip(j, w))
    got = oracle.snr2(T, k_lo, n, S, R, None, [1e-22], [f1], [fdot])[0]
    assert got == pytest.approx(expect, rel=1e-13)
    # a larger S_n lowers rho
    Sg = np.full(n, 1e-40)
    assert oracle.snr2(T, k_lo, n, S, R, Sg, [1e-22], [f1], [fdot])[0] < got


def test_deposit_energy_conservation():
    # sum_k D_k = sum_s A_s^2 x (in-band fraction of the sweep)
    from paper_2602_18560_gb300 import synth
    T = oracle.YEAR
    k_lo, n = oracle.grid(T)
    A, f, fdot = synth.catalog(20000, 11, synth.Population(2.0, 2.0))
    fdot = fdot * 1e3  # stretch sweeps so that many sources span several bins
    D = oracle.deposit(T, k_lo, n, A, f, fdot)
    frac = np.array([math.fsum(oracle.source_pieces(T, k_lo, n, a, b)[1]) for a, b in zip(f, fdot)])
    assert np.sum(D) == pytest.approx(math.fsum(A * A * frac), rel=1e-12)
    assert np.mean(frac < 1.0) > 0.0  # some sweeps cross the top edge
    # excluding sources removes exactly their share
    ex = np.zeros(A.size, np.uint8)
    ex[::3] = 1
    D2 = oracle.deposit(T, k_lo, n, A, f, fdot, ex)
    assert np.sum(D2) == pytest.approx(math.fsum((A * A * frac)[ex == 0]), rel=1e-12)
    assert np.all(D2 <= D)
