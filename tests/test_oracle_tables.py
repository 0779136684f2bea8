"""Pins for the oracle's tables: S_instr (App. C), R (App. B), f*, the TDI-2 factor, the grid.

Each check compares against something other than the oracle's own formula:
the SciRDv1 numbers the paper prints, trigonometric special points where the
A-channel expression reduces to known numbers, the low-frequency limit derived
by hand, and the textbook LISA sensitivity curve of Robson, Cornish & Liu
(2019, CQG 36 105011, Eq. 13), whose low-frequency limit S_AA / R_AA must reach.
"""
import math

import numpy as np
import pytest

import oracle

C_LIGHT = 299792458.0


def test_fstar_is_first_null_of_response(golden):
    # sin^2(f/f*) vanishes at f = pi f* = c / (2 L): the arm transfer frequency.
    L = golden["arm_length_m"]["value"]
    f_null = C_LIGHT / (2.0 * L)
    assert oracle.fstar() == pytest.approx(f_null / math.pi, rel=1e-15)
    assert oracle.response(f_null, tdi2=False) < 1e-25
    assert oracle.s_instr(f_null, tdi2=False) / oracle.s_instr(f_null * 0.9, tdi2=False) < 1e-25


def test_oms_noise_level_and_corner(golden):
    # At f >> 2 mHz the OMS noise is P pm/sqrt(Hz) of displacement, converted to
    # fractional frequency by (2 pi f / c)^2; at f = 2 mHz the bracket doubles it.
    pm = golden["oms_pm"]["value"] * 1e-12
    fc = golden["oms_corner_hz"]["value"]
    for f in (1.0, 3.0):
        disp = math.sqrt(oracle.p_oms(f)) * C_LIGHT / (2 * math.pi * f)
        assert disp == pytest.approx(pm, rel=1e-10)
    ratio = oracle.p_oms(fc) / (pm**2 * (2 * math.pi * fc / C_LIGHT) ** 2)
    assert ratio == pytest.approx(2.0, rel=1e-14)


def test_tm_noise_level_and_corners(golden):
    fm = golden["tm_fm"]["value"] * 1e-15
    lo = golden["tm_corner_low_hz"]["value"]
    hi = golden["tm_corner_high_hz"]["value"]

    def accel(f):  # back to acceleration noise in m/s^2/sqrt(Hz)
        w = 2 * math.pi * f
        return math.sqrt(oracle.p_tm(f) * w**4 / (w / C_LIGHT) ** 2)

    f_mid = math.sqrt(lo * hi)  # both brackets close to 1 here
    b_mid = (1 + (lo / f_mid) ** 2) * (1 + (f_mid / hi) ** 4)
    assert accel(f_mid) == pytest.approx(fm * math.sqrt(b_mid), rel=1e-12)
    # At each corner its own bracket is exactly 2.
    assert (accel(lo) / fm) ** 2 / (1 + (lo / hi) ** 4) == pytest.approx(2.0, rel=1e-12)
    assert (accel(hi) / fm) ** 2 / (1 + (lo / hi) ** 2) == pytest.approx(2.0, rel=1e-12)


@pytest.mark.parametrize("x, sin2, cosx", [
    (math.pi / 2, 1.0, 0.0),
    (2 * math.pi / 3, 0.75, -0.5),
    (math.pi / 3, 0.75, 0.5),
])
def test_s_instr_at_trig_special_points(x, sin2, cosx):
    # App. C A-channel PSD at points where sin and cos are known exactly:
    # 8 sin^2 { 4 [1 + cos + cos^2] P_TM + [2 + cos] P_OMS }.
    f = x * oracle.fstar()
    expect = 8 * sin2 * (4 * (1 + cosx + cosx * cosx) * oracle.p_tm(f) + (2 + cosx) * oracle.p_oms(f))
    assert oracle.s_instr(f, tdi2=False) == pytest.approx(expect, rel=1e-13)


def test_s_instr_low_frequency_limit():
    # x -> 0: sin x ~ x, cos x ~ 1  =>  S_AA ~ 8 x^2 (12 P_TM + 3 P_OMS).
    for f in (1e-6, 1e-5):
        x = f / oracle.fstar()
        lim = 8 * x * x * (12 * oracle.p_tm(f) + 3 * oracle.p_oms(f))
        assert oracle.s_instr(f, tdi2=False) == pytest.approx(lim, rel=5 * x * x)


def test_tdi2_factor(golden):
    fs = oracle.fstar()
    pre = golden["tdi2_factor_prefactor"]["value"]
    # 4 sin^2(2x): equals 4 at x = pi/4 and 2 at x = pi/8; ~16 x^2 as x -> 0.
    for x, expect in ((math.pi / 4, pre * 1.0), (math.pi / 8, pre * 0.5)):
        f = x * fs
        assert oracle.s_instr(f, True) / oracle.s_instr(f, False) == pytest.approx(expect, rel=1e-13)
        assert oracle.response(f, True) / oracle.response(f, False) == pytest.approx(expect, rel=1e-13)
    f = 1e-6
    x = f / fs
    assert oracle.s_instr(f, True) / oracle.s_instr(f, False) == pytest.approx(16 * x * x, rel=1e-8)


def test_response_limits_and_special_points(golden):
    fs = oracle.fstar()
    a16 = golden["R_prefactor"]["value"]
    rt = golden["R_tilde_AA_low_f"]["value"]
    # low f: R ~ 16 x^4 (9/20)
    x = 1e-5
    assert oracle.response(x * fs, False) == pytest.approx(a16 * rt * x**4, rel=1e-8)
    # at 0.7 x^2 = 1 the Lorentzian halves R~: R = 16 sin^2 x x^2 (9/40)
    x = 1 / math.sqrt(0.7)
    assert oracle.response(x * fs, False) == pytest.approx(a16 * math.sin(x) ** 2 * x * x * rt / 2, rel=1e-13)
    # at x = pi/2 sin^2 = 1
    x = math.pi / 2
    assert oracle.response(x * fs, False) == pytest.approx(a16 * x * x * rt / (1 + 0.7 * x * x), rel=1e-13)


def _rcl_sensitivity(f, L=2.5e9):
    """Robson, Cornish & Liu (2019) Eq. 13, sky-averaged LISA sensitivity (strain / Hz)."""
    fstar = C_LIGHT / (2 * math.pi * L)
    p_oms = (1.5e-11) ** 2 * (1 + (2e-3 / f) ** 4)
    p_acc = (3e-15) ** 2 * (1 + (4e-4 / f) ** 2) * (1 + (f / 8e-3) ** 4)
    return (10.0 / (3.0 * L * L)) * (p_oms + 2 * (1 + math.cos(f / fstar) ** 2) * p_acc
                                     / (2 * math.pi * f) ** 4) * (1 + 0.6 * (f / fstar) ** 2)


@pytest.mark.parametrize("f", [1e-5, 3e-5, 1e-4, 3e-4])
@pytest.mark.parametrize("tdi2", [False, True])
def test_strain_sensitivity_matches_textbook_curve_at_low_f(f, tdi2):
    # S_AA / R_AA is the strain sensitivity of one channel; at f << f* it must
    # reduce to the textbook curve (both are 10/(3L^2) (P_OMS + 4 P_acc/(2 pi f)^4)).
    x = f / oracle.fstar()
    ours = oracle.s_instr(f, tdi2) / oracle.response(f, tdi2)
    assert ours == pytest.approx(_rcl_sensitivity(f), rel=3 * x * x + 1e-12)


def test_grid_counts():
    # Bins k / T_obs inside [0.1, 10] mHz for 1, 2 and 4 (Julian) years.
    for years, n_expect in ((1, 312421), (2, 624841), (4, 1249681)):
        k_lo, n = oracle.grid(years * oracle.YEAR)
        assert n == n_expect
        assert k_lo / (years * oracle.YEAR) >= 1e-4
        assert (k_lo - 1) / (years * oracle.YEAR) < 1e-4
        assert (k_lo + n - 1) / (years * oracle.YEAR) <= 1e-2


def test_tables_are_the_pointwise_functions():
    T = oracle.YEAR
    k_lo, n = oracle.grid(T)
    S, R = oracle.tables(T, k_lo, n, True)
    for j in (0, 1, n // 3, n - 1):
        f = (k_lo + j) / T
        assert S[j] == oracle.s_instr(f, True)
        assert R[j] == oracle.response(f, True)
    assert np.all(S > 0) and np.all(R > 0)


def test_median_bias_constant(golden):
    from fractions import Fraction
    nu = golden["median_bias_nu"]["value"]
    exact = float((1 - Fraction(2, 9 * nu)) ** -3)  # (8/9)^-3 = 729/512
    assert oracle.median_bias() == exact == 729 / 512
    # The paper prints ~1.4237; the exact value 1.423828125 rounds to 1.4238.
    assert abs(oracle.median_bias() - golden["median_bias_printed"]["value"]) < 2e-4
    # It is the Wilson-Hilferty estimate of mean/median of chi^2_2, whose exact value is 1/ln 2.
    assert abs(oracle.median_bias() - 1 / math.log(2)) < 0.02
