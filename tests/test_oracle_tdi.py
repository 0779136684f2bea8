"""An independent pin of the oracle's S_instr (App. C, the A-channel noise PSD, with and without
the TDI-2 factor) at every frequency of the band and beyond, not only at its limits and
trigonometric special points.

The App. C expression is the closed form of a time-delay-interferometry combination.  Here
the combination is built from its definition instead, with complex transfer functions and no
closed form: six single-link measurements y_ij (received on spacecraft i from j) of an equal-
arm constellation, each carrying its own optical-metrology noise O_ij and the noise of the
two test masses it bounces off, the local one and the distant one one light travel time
earlier (one-arm delay D = exp(-i f/f*)):

    y_ij = O_ij - T_ij - D T_ji
    X = (1 - D^2) [(y_13 + D y_31) - (y_12 + D y_21)],  Y, Z by cyclic relabelling,
    A = (Z - X) / sqrt(2),  and the second-generation combinations carry (1 - D^4) more.

With every O of PSD P_OMS and every T of PSD P_TM (the App. C single-link levels, in
fractional frequency), the PSD of A is the sum over the twelve independent noises of
|coefficient|^2 times their PSD.  A dropped or wrong cos(f/f*) term of the closed form
changes S_instr by tens of percent somewhere in 1-60 mHz and fails here.
"""
import math

import numpy as np
import pytest

import oracle

def y_link(i, j, D):
    """Noise content of y_ij as {noise name: complex coefficient}."""
    return {("O", i, j): 1.0, ("T", i, j): -1.0, ("T", j, i): -D}


def add(acc, terms, c):
    for k, v in terms.items():
        acc[k] = acc.get(k, 0.0) + c * v


def michelson(a, b, c, D):
    """First-generation Michelson combination of spacecraft a with arms to b and c:
    (1 - D^2) [(y_ac + D y_ca) - (y_ab + D y_ba)]."""
    out = {}
    add(out, y_link(a, c, D), 1.0)
    add(out, y_link(c, a, D), D)
    add(out, y_link(a, b, D), -1.0)
    add(out, y_link(b, a, D), -D)
    return {k: (1.0 - D * D) * v for k, v in out.items()}


def s_a_from_transfer(f, tdi2):
    x = f / oracle.fstar()
    D = complex(math.cos(x), -math.sin(x))
    X = michelson(1, 2, 3, D)
    Z = michelson(3, 1, 2, D)
    A = {}
    add(A, Z, 1.0 / math.sqrt(2.0))
    add(A, X, -1.0 / math.sqrt(2.0))
    g = (1.0 - D**4) if tdi2 else 1.0
    p_oms, p_tm = oracle.p_oms(f), oracle.p_tm(f)
    s = 0.0
    for (kind, _, _), c in A.items():
        s += abs(g * c) ** 2 * (p_oms if kind == "O" else p_tm)
    return s


def test_every_noise_enters_once():
    D = complex(math.cos(0.3), -math.sin(0.3))
    X = michelson(1, 2, 3, D)
    # the Michelson X of spacecraft 1 sees the four links of its two arms, and all four
    # test masses on them
    assert {k for k in X if k[0] == "O"} == {("O", 1, 2), ("O", 2, 1), ("O", 1, 3), ("O", 3, 1)}
    assert {k for k in X if k[0] == "T"} == {("T", 1, 2), ("T", 2, 1), ("T", 1, 3), ("T", 3, 1)}


@pytest.mark.parametrize("tdi2", [False, True])
def test_s_instr_equals_the_tdi_transfer_function_sum(tdi2):
    fs = np.geomspace(1e-4, 6e-2, 241)
    got = np.array([oracle.s_instr(f, tdi2) for f in fs])
    ref = np.array([s_a_from_transfer(f, tdi2) for f in fs])
    # away from the nulls of the response (sin x = 0, and sin 2x = 0 with TDI-2) both are
    # evaluated to double precision; near a null the relative error of either can grow
    x = fs / oracle.fstar()
    far = (np.abs(np.sin(x)) > 1e-3) & ((not tdi2) | (np.abs(np.sin(2 * x)) > 1e-3))
    assert far.sum() > 200
    rel = np.abs(got[far] / ref[far] - 1.0)
    assert rel.max() < 1e-12, rel.max()


def test_a_wrong_cos_coefficient_would_be_caught():
    # the check above distinguishes the App. C form from near misses: e.g. (2 - cos x) in
    # place of (2 + cos x) for the OMS term differs by far more than its tolerance
    worst = 0.0
    for f in np.geomspace(1e-3, 6e-2, 50):
        x = f / oracle.fstar()
        wrong = 8 * math.sin(x) ** 2 * (4 * (1 + math.cos(x) + math.cos(x) ** 2) * oracle.p_tm(f)
                                        + (2 - math.cos(x)) * oracle.p_oms(f))
        worst = max(worst, abs(wrong / s_a_from_transfer(f, False) - 1.0))
    assert worst > 0.1
