"""Pins of the oracle's forward model (Eqs. 1, 3 and 26 of the paper).

The closed-form SPGR/MT signal is checked against things it does not compute
itself: a pulse-by-pulse Bloch simulation of the spoiled sequence run to its
steady state, the Ernst angle, and the DESPOT1 straight line.
"""
import math

import numpy as np
import pytest


def _rot_x(theta):
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, s], [0.0, -s, c]])


def bloch_spgr(a, r1, r2, delta, alpha, tr, te, mt, b1p=1.0, b1m=1.0, tol=1e-14):
    """Spoiled gradient echo simulated pulse by pulse on the magnetisation
    vector: (MT saturation pulse of angle acos(1 - delta) immediately before the
    excitation, i.e. TR2 = 0, Eq. 2), excitation about x, ideal spoiling of
    the transverse part, T1 recovery over TR, repeated until the longitudinal
    magnetisation stops changing.  Returns the magnitude at echo time te."""
    m0 = a
    mz = m0
    rx = _rot_x(alpha * b1p)
    rmt = _rot_x(math.acos(1.0 - delta)) if mt else None
    e1 = math.exp(-r1 * tr)
    for _ in range(2_000_000):
        v = np.array([0.0, 0.0, mz])
        if mt:
            v = rmt @ v
            v[:2] = 0.0                      # the saturated part is spoiled
        v = rx @ v
        transverse = math.hypot(v[0], v[1])
        mz_new = m0 + (v[2] - m0) * e1       # recovery; transverse spoiled
        if abs(mz_new - mz) <= tol * m0:
            mz = mz_new
            break
        mz = mz_new
    v = np.array([0.0, 0.0, mz])
    if mt:
        v = rmt @ v
        v[:2] = 0.0
    v = rx @ v
    transverse = math.hypot(v[0], v[1])
    return b1m * transverse * math.exp(-r2 * te)


CASES = [
    # (A, R1, R2*, delta, alpha_deg, TR, TE, mt, b1p, b1m)
    (3000.0, 1.0, 20.0, 0.01, 6.0, 0.025, 0.0023, 1, 1.0, 1.0),
    (2500.0, 0.7, 15.0, 0.02, 6.0, 0.025, 0.0161, 1, 1.13, 0.95),
    (3500.0, 1.4, 35.0, 0.0, 21.0, 0.025, 0.0069, 0, 0.85, 1.07),
    (2000.0, 0.5, 10.0, 0.0, 6.0, 0.025, 0.0184, 0, 1.2, 0.9),
    (1.5, 3.0, 2.0, 0.3, 40.0, 0.5, 0.1, 1, 1.0, 1.0),
    (10.0, 0.2, 50.0, 0.0, 70.0, 0.01, 0.001, 0, 1.0, 1.0),
]


@pytest.mark.parametrize("case", CASES)
def test_signal_matches_bloch_steady_state(orc, case):
    a, r1, r2, delta, adeg, tr, te, mt, bp, bm = case
    y = [math.log(a), math.log(r1), math.log(r2),
         math.log(delta / (1 - delta)) if delta > 0 else -50.0]
    s_closed = orc.signal(y, math.radians(adeg), tr, te, mt, bp, bm)
    s_sim = bloch_spgr(a, r1, r2, delta, math.radians(adeg), tr, te, mt, bp, bm)
    assert s_closed == pytest.approx(s_sim, rel=1e-11)


def test_mt_signal_reduces_to_ernst_when_saturation_vanishes(orc):
    y_mt = [math.log(3000.0), math.log(1.0), math.log(20.0), -60.0]
    s_mt = orc.signal(y_mt, math.radians(6), 0.025, 0.003, 1)
    s_plain = orc.signal(y_mt, math.radians(6), 0.025, 0.003, 0)
    assert s_mt == pytest.approx(s_plain, rel=1e-14)


@pytest.mark.parametrize("r1,tr", [(1.0, 0.025), (0.6, 0.015), (2.0, 0.1)])
def test_ernst_angle_maximises_signal(orc, r1, tr):
    from scipy.optimize import minimize_scalar
    y = [math.log(1000.0), math.log(r1), math.log(20.0), 0.0]
    res = minimize_scalar(lambda al: -orc.signal(y, al, tr, 0.0, 0),
                          bounds=(1e-4, math.pi / 2), method="bounded",
                          options={"xatol": 1e-12})
    assert res.x == pytest.approx(math.acos(math.exp(-r1 * tr)), rel=1e-6)


def test_despot1_line(orc):
    """Without MT, S/sin(a) = E S/tan(a) + A (1 - E) exp(-R2* TE) for every a."""
    a, r1, r2, tr, te, bm = 2700.0, 0.9, 25.0, 0.025, 0.004, 1.05
    y = [math.log(a), math.log(r1), math.log(r2), 0.0]
    angles = np.radians([2, 5, 9, 14, 21, 30, 45])
    S = np.array([orc.signal(y, al, tr, te, 0, 1.0, bm) for al in angles])
    X, Y = S / np.tan(angles), S / np.sin(angles)
    slope, icpt = np.polyfit(X, Y, 1)
    E = math.exp(-r1 * tr)
    assert slope == pytest.approx(E, rel=1e-10)
    assert icpt == pytest.approx(bm * a * (1 - E) * math.exp(-r2 * te), rel=1e-8)


def test_forward_layout_matches_signal(orc):
    from paper_2102_01604_gb300 import phantom
    prot = phantom.protocol()
    ph = phantom.phantom((5, 3, 2), seed=3)
    p = orc.make_problem(prot, (5, 3, 2))
    s = orc.forward(p, ph["y"], ph["b1p"], ph["b1m"])
    N = 30
    i = 0
    for c in range(3):
        for e in range(prot["n_echoes"][c]):
            for n in (0, 7, 29):
                ref = orc.signal(ph["y"][:, n], prot["alpha"][c], prot["tr"][c], prot["te"][i],
                                 prot["mt"][c], ph["b1p"][n], ph["b1m"][c, n])
                assert s[i, n] == ref
            i += 1
    assert s.shape == (22, N)
