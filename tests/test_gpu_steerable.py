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


@pytest.mark.parametrize("prec,Lh,arith,rot", [(0, 12, 0, 0), (0, 12, 1, 0), (0, 20, 0, 0), (1, 12, 0, 0),
                                               (1, 24, 0, 1), (1, 24, 0, 2)])
def test_steerable_window_skips_zero_orders(ctx, prec, Lh, arith, rot):
    """SLSHT_OPT_WINDOW_ORDERS 1 leaves the window's vanishing orders out of
    the rotated window (CUDA cores: skipped; tensor cores, rot 2: zero columns
    of K) with the same bits as the full sum, and matches the oracle."""
    import torch
    import paper_1207_5558_gb300 as pkg
    Lf, N = 18, 3
    grid = (2 * Lf - 1, Lf, 2 * Lh + 1)
    f = synth.signal_powerlaw(Lf, 301)
    h = steerable_window(Lh, N, 302)
    pairs = synth.pairs_bands([0, 7, 17, Lf + Lh - 2])
    ctx.set_option(pkg.SLSHT_OPT_FP64_ARITH, arith)
    ctx.set_option(pkg.SLSHT_OPT_ROTWIN_ENGINE, rot)
    try:
        full = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=prec).cpu().numpy()
        ctx.set_option(pkg.SLSHT_OPT_WINDOW_ORDERS, 1)
        steer = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=prec).cpu().numpy()
        torch.cuda.synchronize()
    finally:
        ctx.set_option(pkg.SLSHT_OPT_WINDOW_ORDERS, 0)
        ctx.set_option(pkg.SLSHT_OPT_FP64_ARITH, 0)
        ctx.set_option(pkg.SLSHT_OPT_ROTWIN_ENGINE, 0)
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


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("N", [3, None])
def test_steer_gamma_from_basis_orientations(ctx, prec, N):
    """g at orientations between the grid's gamma samples (Sec. IV-B, the
    linearity remark): a steerable window (|q'| < N) evaluated on 2N - 1 basis
    orientations, and a general window on 2 L_h - 1, interpolated to 13
    orientations and compared with the oracle's g computed there directly."""
    import torch
    import paper_1207_5558_gb300 as pkg
    Lf, Lh = 14, 10
    f = synth.signal_powerlaw(Lf, 321)
    h = steerable_window(Lh, N, 322) if N else synth.window_cn(Lh, 322, decay=1.0)
    Q = (N - 1) if N else Lh - 1
    coarse = (2 * Lf - 1, Lf, 2 * Q + 1)
    fine = (2 * Lf - 1, Lf, 13 if N else 29)
    pairs = synth.pairs_bands([2, 9, 13, 20])
    g = ctx.forward(Lf, Lh, coarse, f, h, pairs, prec=prec)
    gam = 2 * np.pi * np.arange(fine[2]) / fine[2]
    dt = torch.complex128 if prec == 0 else torch.complex64
    out = torch.empty((len(pairs), coarse[0], coarse[1], fine[2]), dtype=dt, device="cuda")
    pkg.slsht_steer_gamma(ctx.h, pkg.make_desc(Lf, Lh, coarse, prec), g, len(pairs), gam, len(gam), Q, out)
    torch.cuda.synchronize()
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, fine)
    assert _rel(out.cpu().numpy(), ref) < TOL[prec]
    with pytest.raises(pkg.SlshtError):            # too few orientations for the band
        pkg.slsht_steer_gamma(ctx.h, pkg.make_desc(Lf, Lh, coarse, prec), g, len(pairs), gam, len(gam), Q + 1, out)


@pytest.mark.parametrize("Lh,grid,orders", [
    (16, (35, 18, 31), 0),
    (24, (47, 24, 47), 0),
    (40, (81, 20, 127), 0),          # two K chunks, 127 gamma samples on the 128 TMEM lanes
    (24, (47, 24, 47), 1),           # a steerable window: the inactive orders are zero columns of K
    (5, (130, 10, 9), 0),            # ragged row tiles, short K
    (64, (129, 33, 128), 0),         # L_h = 64: K = 127 in two chunks, all 128 lanes, 33 beta rows
    (64, (129, 7, 65), 2),           # few beta rows: tiles that span several betas; rounding-level orders
    (20, (41, 1, 1), 0),             # one beta row, one gamma sample: a tile per degree, most rows padding
    (17, (35, 3, 2), 0),             # the smallest window on the default path (L_h > 16), two gamma samples
    (64, (9, 41, 127), 0),           # 41 tiles x 127 orders: the wide producer's first pass on the tensor cores, ragged last tile
    (24, (9, 104, 128), 1),          # the same at L_h = 24 (one 32-degree chunk an order), steerable window
])
def test_rotated_window_on_tensor_cores(ctx, Lh, grid, orders):
    """The rotated window on the tensor cores (SLSHT_OPT_ROTWIN_ENGINE = 2,
    split-FP16 products) against the oracle and the CUDA-core window (1),
    FP32_BULK; the default (0) takes the tensor cores for L_h > 16."""
    import paper_1207_5558_gb300 as pkg
    Lf = 12
    f = synth.signal_powerlaw(Lf, 330 + Lh)
    h = steerable_window(Lh, 4, 331) if orders else synth.window_cn(Lh, 331, decay=1.0)
    pairs = synth.pairs_bands([0, 5, 11, Lf + Lh - 2])
    if Lh > 40 or grid[1] * grid[2] > 8000:
        pairs = pairs[::9]                         # keeps the oracle to seconds at L_h = 64 and on large grids
    ctx.set_option(pkg.SLSHT_OPT_WINDOW_ORDERS, orders)
    try:
        ctx.set_option(pkg.SLSHT_OPT_ROTWIN_ENGINE, 1)
        cc = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=1).cpu().numpy()
        ctx.set_option(pkg.SLSHT_OPT_ROTWIN_ENGINE, 2)
        tc = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=1).cpu().numpy()
        ctx.set_option(pkg.SLSHT_OPT_ROTWIN_ENGINE, 0)
        default = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=1).cpu().numpy()
    finally:
        ctx.set_option(pkg.SLSHT_OPT_ROTWIN_ENGINE, 0)
        ctx.set_option(pkg.SLSHT_OPT_WINDOW_ORDERS, 0)
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    assert _rel(tc, ref) < TOL[1]
    assert _rel(tc, cc) < 5e-6
    assert np.array_equal(default, tc if Lh > 16 else cc)   # the default: the tensor cores for L_h > 16


def _rtab_bytes(Lh, Nb):
    """Bytes of the tensor-core rotated window's d(beta) image: a 32 KB block
    per (degree, tile of 128 (beta, q) rows, 64-wide K chunk) and a float per
    row."""
    tiles = chunks = 0
    for p in range(Lh):
        t = (Nb * (2 * p + 1) + 127) // 128
        tiles += t
        chunks += t * ((2 * p + 1 + 63) // 64)
    return chunks * 32768 + tiles * 128 * 4


def test_rotated_window_engine_falls_back_within_budget():
    """The default engine leaves the tensor cores for the CUDA cores when the
    context's budget cannot hold the d(beta) image (with a quarter of the
    budget to spare); forcing the tensor cores then fails with
    SLSHT_E_NOMEM.  The fallback's g equals the CUDA-core engine's bits."""
    import torch
    import paper_1207_5558_gb300 as pkg
    from paper_1207_5558_gb300 import _abi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Lf, Lh, grid = 12, 40, (81, 64, 127)
    f = synth.signal_powerlaw(Lf, 341)
    h = synth.window_cn(Lh, 342, decay=1.0)
    pairs = synth.pairs_bands([5])
    big = pkg.Context(0, 4 << 30)
    try:
        big.set_option(pkg.SLSHT_OPT_ROTWIN_ENGINE, 1)
        cc = big.forward(Lf, Lh, grid, f, h, pairs, prec=1).cpu().numpy()
        need = pkg.slsht_mem_used(big.h)
    finally:
        big.close()
    small = pkg.Context(0, need + _rtab_bytes(Lh, grid[1]) // 2)
    try:
        got = small.forward(Lf, Lh, grid, f, h, pairs, prec=1).cpu().numpy()
        assert np.array_equal(got, cc)
        small.set_option(pkg.SLSHT_OPT_ROTWIN_ENGINE, 2)
        with pytest.raises(pkg.SlshtError) as e:
            small.forward(Lf, Lh, grid, f, h, pairs, prec=1)
        assert e.value.code == _abi.SLSHT_E_NOMEM
    finally:
        small.close()

