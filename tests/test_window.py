"""Pins for the oracle's elliptical concentration window generator
(oracle/window.py, Sec. III-D), and for the stored windows of workloads 2
and 5 that the seeded-input module hands to both sides."""
import json
import os
from math import pi

import numpy as np

import synth
from oracle import window as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_printed_ninety_percent_concentration():
    """Sec. V: the eigenfunction window with L_h = 18 in R_(pi/6, pi/6+pi/240)
    has 90% concentration.  Reading: L_h = 18 is the exclusive band limit
    (degrees l < 18, the convention of the SSHT code the paper used); it gives
    0.897, while degrees l <= 18 give 0.914."""
    ex = GOLDEN["window_example1"]
    h, lam = W.window_ellipse(ex["L"], pi / 6, pi / 6 + pi / 240)
    assert abs(lam - ex["concentration"]) < 0.005
    h2, lam2 = W.window_ellipse(ex["L"] + 1, pi / 6, pi / 6 + pi / 240)
    assert lam2 > lam


def test_shannon_number_and_eigen_range():
    """trace D = L^2 Area(R)/(4 pi) (addition theorem) and 0 <= lambda <= 1."""
    L = 8
    tc, a = synth.ellipse_from_axes(20.0, 10.0)
    D = W.concentration_matrix(tc, a, L)
    th, ph, w = W.region_rule(tc, a, L)
    assert abs(np.trace(D).real - L * L * w.sum() / (4 * pi)) < 1e-12
    lam = np.linalg.eigvalsh(D)
    assert lam.min() > -1e-12 and lam.max() < 1 + 1e-12
    assert np.max(np.abs(D - D.conj().T)) < 1e-14


def test_region_limits_are_polar_caps():
    """theta_c = 0 and a = pi/2 both give polar caps (remark after Eq. region_def):
    the area is 2 pi (1 - cos a) and D decouples the orders m."""
    L = 6
    for tc, a in [(0.0, 0.5), (0.3, pi / 2)]:
        th, ph, w = W.region_rule(tc, a, L)
        cap = a if tc == 0.0 else pi / 2
        assert abs(w.sum() - 2 * pi * (1 - np.cos(cap))) < 1e-12
        D = W.concentration_matrix(tc, a, L)
        ms = np.array([m for l in range(L) for m in range(-l, l + 1)])
        off = np.abs(D[ms[:, None] != ms[None, :]]).max()
        assert off < 1e-13


def test_axes_to_focus():
    tc, a = synth.ellipse_from_axes(20.0, 10.0)
    assert abs(np.rad2deg(tc) - 17.4099) < 1e-3 and abs(np.rad2deg(a) - 20.0) < 1e-12
    # boundary along the minor axis is the semi-minor arc
    b = W.boundary(tc, a, np.array([pi / 2, 0.0]))
    assert abs(b[0] - np.deg2rad(10.0)) < 1e-12 and abs(b[1] - a) < 1e-12


def test_window_is_real_unit_energy_positive_dc():
    L = 8
    h, lam = W.window_ellipse(L, *synth.ellipse_from_axes(20.0, 10.0))
    assert abs(np.linalg.norm(h) - 1) < 1e-14
    assert h[0].real > 0 and abs(h[0].imag) < 1e-14
    for l in range(L):
        for m in range(-l, l + 1):
            assert abs(h[l * l + l - m] - (-1) ** (m % 2) * np.conj(h[l * l + l + m])) < 1e-13
    assert 0.3 < lam < 1.0


def test_stored_windows_are_the_oracle_windows():
    """The stored workload-2 window is the oracle's eigenfunction (recomputed
    here); both stored windows are unit-energy real fields with h00 > 0 and
    the concentration the file records lies in (0, 1]."""
    h2, lam2 = synth.stored_window(2)
    h, lam = W.window_ellipse(8, *synth.ellipse_from_axes(20.0, 10.0))
    assert np.linalg.norm(h2 - h) < 1e-13 and abs(lam2 - lam) < 1e-14
    for w, L in ((2, 8), (5, 64)):
        hw, lw = synth.stored_window(w)
        assert hw.shape == (L * L,) and abs(np.linalg.norm(hw) - 1) < 1e-13 and hw[0].real > 0
        assert np.max(np.abs(hw - W.mirror(hw, L))) < 1e-12
        assert 0.0 < lw <= 1.0
