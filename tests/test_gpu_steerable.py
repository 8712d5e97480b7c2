"""Steerable windows (Sec. IV-B, the closing remarks on steerability): a
window whose coefficients vanish for |q'| >= N < L_h, azimuthally
band-limited.  With SLSHT_OPT_WINDOW_ORDERS the rotated window sums only over
the window's active orders; the terms left out are exactly zero, so g must be
bit for bit the full computation's, and equal to the oracle within the
path's tolerance, for every engine that reads the rotated window.  A window
with only even orders (the concentration window of an ellipse centred on the
pole has odd orders at the rounding level) is checked against the oracle."""
import numpy as np
import pytest

import synth
from oracle import slsht as O

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1207_5558_gb300 as pkg
    from paper_1207_5558_gb300 import build
    build.build()
    c = pkg.Context(0)
    yield c
    c.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def steerable_window(Lh, N, seed):
    """CN(0,1)/(p+1) coefficients with h_p^q' = 0 for |q'| >= N, unit energy."""
    h = synth.window_cn(Lh, seed, decay=1.0)
    for p in range(Lh):
        for q in range(-p, p + 1):
            if abs(q) >= N:
                h[p * p + p + q] = 0.0
    return h / np.linalg.norm(h)


@pytest.mark.parametrize("prec,Lh,arith", [(0, 12, 0), (0, 12, 1), (0, 20, 0), (1, 12, 0), (1, 24, 0)])
def test_steerable_window_skips_zero_orders(ctx, prec, Lh, arith):
    import torch
    import paper_1207_5558_gb300 as pkg
    Lf, N = 18, 3
    grid = (2 * Lf - 1, Lf, 2 * Lh + 1)
    f = synth.signal_powerlaw(Lf, 301)
    h = steerable_window(Lh, N, 302)
    pairs = synth.pairs_bands([0, 7, 17, Lf + Lh - 2])
    ctx.set_option(pkg.SLSHT_OPT_FP64_ARITH, arith)
    try:
        full = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=prec).cpu().numpy()
        ctx.set_option(pkg.SLSHT_OPT_WINDOW_ORDERS, 1)
        steer = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=prec).cpu().numpy()
        torch.cuda.synchronize()
    finally:
        ctx.set_option(pkg.SLSHT_OPT_WINDOW_ORDERS, 0)
        ctx.set_option(pkg.SLSHT_OPT_FP64_ARITH, 0)
    assert np.array_equal(steer, full)
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    assert _rel(steer, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_even_order_window(ctx, prec):
    """The workload-2 window (L_h = 8, 20 x 10 degree ellipse) has its odd
    orders at the rounding level only (about 1e-15 of its largest
    coefficient): with the option at 2 (the FP32_BULK threshold leaves them
    out), g stays within the path's tolerance of the oracle."""
    import paper_1207_5558_gb300 as pkg
    Lf, Lh, grid = 24, 8, (47, 24, 15)
    f = synth.signal_powerlaw(Lf, 311)
    h = synth.stored_window(2)[0]
    pairs = synth.pairs_bands([3, 23, 30])
    ctx.set_option(pkg.SLSHT_OPT_WINDOW_ORDERS, 2)
    try:
        g = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=prec).cpu().numpy()
    finally:
        ctx.set_option(pkg.SLSHT_OPT_WINDOW_ORDERS, 0)
    assert _rel(g, O.forward_coeff(f, h, Lf, Lh, pairs, grid)) < TOL[prec]
