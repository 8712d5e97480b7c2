"""Batch plans (slsht_batch_*) on the GPU: many analyses of uneven band
limits, grids and precisions in one plan, checked against the FP64 oracle
(relative L2 <= 1e-12 for FP64 items, <= 1e-5 for FP32_BULK items), plus the
plan's own contracts: a relaunch reads the inputs' current contents, an item
gives the same bits alone and in a mix, the graph replay gives the same bits
as the direct launches, and the tuner's choices are cached per shape."""
import numpy as np
import pytest

import synth
from oracle import slsht as O

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1207_5558_gb300 as P
    from paper_1207_5558_gb300 import build
    build.build()
    return P


@pytest.fixture()
def ctx(pkg):
    c = pkg.Context(0)
    yield c
    c.close()


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def _item(Lf, Lh, grid, f, h, pairs, prec):
    return {"L_f": Lf, "L_h": Lh, "grid": grid, "f": f, "h": h, "lm": pairs, "prec": prec}


def _mix():
    """Nine analyses: both precisions, L_h from 1 to 20, prime and composite
    N_alpha (direct sum and split DFT), ragged column counts, a shared signal
    (one coupling for two windows), a shared window over two grids, and FP32
    items the tensor cores can take (narrow and wide windows)."""
    fA = synth.signal_powerlaw(8, 11)
    hA = synth.window_cn(4, 12)
    hF = synth.window_cn(4, 13)
    spec = [
        # Lf, Lh, grid, f, h, pairs, prec
        (8, 4, (15, 8, 7), fA, hA, synth.pairs_random(11, 9, 21), 0),
        (12, 5, (23, 12, 9), synth.signal_powerlaw(12, 14), synth.window_cn(5, 15), synth.pairs_random(16, 7, 22), 1),
        (6, 16, (31, 16, 31), synth.signal_cn_real(6, 16), synth.window_cn(16, 17, decay=1.0),
         synth.pairs_random(21, 3, 23), 0),
        (10, 3, (130, 5, 33), synth.signal_powerlaw(10, 18), synth.window_cn(3, 19), synth.pairs_random(12, 5, 24), 1),
        (5, 1, (3, 2, 1), synth.signal_cn_real(5, 20), synth.window_cn(1, 21), synth.pairs_all(5), 0),
        (8, 4, (15, 8, 7), fA, hF, synth.pairs_random(11, 9, 21), 0),       # same f and pairs as item 0
        (8, 4, (45, 6, 11), fA, hA, synth.pairs_random(11, 4, 25), 0),      # same window as item 0, other grid
        (9, 8, (63, 9, 15), synth.signal_powerlaw(9, 22), synth.window_cn(8, 23), synth.pairs_random(16, 6, 26), 1),
        (7, 20, (40, 7, 39), synth.signal_powerlaw(7, 24), synth.window_cn(20, 25, decay=1.0),
         synth.pairs_random(26, 5, 27), 1),                                   # wide window: K in two chunks
    ]
    return spec


def _build_items(spec, dev_cache=None):
    dev_cache = {} if dev_cache is None else dev_cache
    items, refs = [], []
    for (Lf, Lh, grid, f, h, pairs, prec) in spec:
        fd = dev_cache.setdefault(id(f), _dev(f))
        hd = dev_cache.setdefault(id(h), _dev(h))
        items.append(_item(Lf, Lh, grid, fd, hd, pairs, prec))
        refs.append(O.forward_coeff(f, h, Lf, Lh, pairs, grid))
    return items, refs, dev_cache


def test_mixed_batch_vs_oracle(pkg, ctx):
    spec = _mix()
    items, refs, _ = _build_items(spec)
    b = ctx.batch(items)
    try:
        assert b.query(pkg.SLSHT_BQ_GRAPH) == 1
        assert b.query(pkg.SLSHT_BQ_KERNELS) >= 3
        for i, (it, ref) in enumerate(zip(items, refs)):
            g = b.outputs[i].cpu().numpy()
            assert rel(g, ref) < TOL[it["prec"]], i
            form = b.query(pkg.SLSHT_BQ_ALPHA_FORM, i)
            assert form in (-1, 0, 3, 5, 7, 9)
            if form > 0:
                assert it["grid"][0] % form == 0
            if form == -1:
                assert it["prec"] == 1
        # the creation ran the plan once; a launch recomputes the same values
        for o in b.outputs:
            o.zero_()
        b.launch()
        for i, (it, ref) in enumerate(zip(items, refs)):
            assert rel(b.outputs[i].cpu().numpy(), ref) < TOL[it["prec"]], i
    finally:
        b.close()


def test_relaunch_reads_current_inputs(pkg, ctx):
    import torch
    Lf, Lh, grid = 10, 6, (21, 10, 11)
    pairs = synth.pairs_random(15, 8, 31)
    f1, f2 = synth.signal_powerlaw(Lf, 32), synth.signal_powerlaw(Lf, 33)
    h1, h2 = synth.window_cn(Lh, 34), synth.window_cn(Lh, 35)
    fd, hd = _dev(f1), _dev(h1)
    b = ctx.batch([_item(Lf, Lh, grid, fd, hd, pairs, 0)])
    try:
        assert rel(b.outputs[0].cpu().numpy(), O.forward_coeff(f1, h1, Lf, Lh, pairs, grid)) < 1e-12
        fd.copy_(torch.as_tensor(f2))
        hd.copy_(torch.as_tensor(h2))
        b.launch()
        assert rel(b.outputs[0].cpu().numpy(), O.forward_coeff(f2, h2, Lf, Lh, pairs, grid)) < 1e-12
    finally:
        b.close()


def test_item_alone_equals_item_in_mix(pkg, ctx):
    """The same analysis gives the same bits in a plan of its own and inside
    a mix: its tile shape is a function of its shape only (tuned once, then
    taken from the context's cache) and no tile mixes items."""
    spec = _mix()
    items, _, cache = _build_items(spec[:1])
    alone = ctx.batch(items)
    try:
        assert alone.query(pkg.SLSHT_BQ_TUNED, 0) == 1
        items2, _, _ = _build_items(spec, cache)
        mix = ctx.batch(items2)
        try:
            assert mix.query(pkg.SLSHT_BQ_TUNED, 0) == 2
            assert mix.query(pkg.SLSHT_BQ_TILE_COLS, 0) == alone.query(pkg.SLSHT_BQ_TILE_COLS, 0)
            a = alone.outputs[0].cpu().numpy()
            m = mix.outputs[0].cpu().numpy()
            assert np.array_equal(a.view(np.float64), m.view(np.float64))
        finally:
            mix.close()
    finally:
        alone.close()


def test_graph_replay_equals_direct_launches(pkg, ctx):
    spec = _mix()
    items, refs, cache = _build_items(spec)
    g1 = ctx.batch(items)
    items2, _, _ = _build_items(spec, cache)
    g2 = ctx.batch(items2, flags=pkg.SLSHT_BATCH_NO_GRAPH)
    try:
        assert g2.query(pkg.SLSHT_BQ_GRAPH) == 0
        g1.launch()
        g2.launch()
        for a, b_ in zip(g1.outputs, g2.outputs):
            x, y = a.cpu().numpy(), b_.cpu().numpy()
            w = np.float64 if x.dtype == np.complex128 else np.float32
            assert np.array_equal(x.view(w), y.view(w))
    finally:
        g1.close()
        g2.close()


@pytest.mark.parametrize("flags", ["rule", "cuda_cores"])
def test_rule_and_cuda_core_plans(pkg, ctx, flags):
    f = pkg.SLSHT_BATCH_NO_TUNE if flags == "rule" else pkg.SLSHT_BATCH_NO_TC
    spec = _mix()
    items, refs, _ = _build_items(spec)
    b = ctx.batch(items, flags=f)
    try:
        for i, (it, ref) in enumerate(zip(items, refs)):
            assert rel(b.outputs[i].cpu().numpy(), ref) < TOL[it["prec"]], i
            if flags == "rule":
                assert b.query(pkg.SLSHT_BQ_TUNED, i) == 0
            else:
                assert b.query(pkg.SLSHT_BQ_ALPHA_FORM, i) >= 0
    finally:
        b.close()


def test_batch_matches_per_call_forward(pkg, ctx):
    """FP64: the plan and slsht_forward agree to rounding (the plan forms X per
    tile, the per-call path in a separate kernel; the plan's tuner may pick the
    double-float engine, about 2^-48 per operation)."""
    Lf, Lh, grid = 16, 8, (63, 16, 15)
    f, h = synth.signal_powerlaw(Lf, 41), synth.window_cn(Lh, 42)
    pairs = synth.pairs_random(Lf + Lh - 1, 12, 43)
    b = ctx.batch([_item(Lf, Lh, grid, _dev(f), _dev(h), pairs, 0)])
    try:
        g = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=0).cpu().numpy()
        assert rel(b.outputs[0].cpu().numpy(), g) < 1e-13
    finally:
        b.close()


def test_wide_fp32_window_on_tensor_cores(pkg, ctx):
    """A plan rotates wide FP32 windows (L_h > 16) on the tensor cores by
    default (window-operand kernel + tensor-core kernel in place of the
    CUDA-core launch): it matches the oracle, the per-call forward, and a plan
    made with the CUDA-core window (SLSHT_OPT_ROTWIN_ENGINE 1)."""
    Lf, Lh, grid = 10, 24, (61, 12, 47)
    f, h = synth.signal_powerlaw(Lf, 51), synth.window_cn(Lh, 52, decay=1.0)
    pairs = synth.pairs_random(Lf + Lh - 1, 10, 53)
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    out = {}
    for eng in (0, 1):
        ctx.set_option(pkg.SLSHT_OPT_ROTWIN_ENGINE, eng)
        try:
            b = ctx.batch([_item(Lf, Lh, grid, _dev(f), _dev(h), pairs, 1)])
            try:
                out[eng] = (b.outputs[0].cpu().numpy(), b.query(pkg.SLSHT_BQ_KERNELS))
            finally:
                b.close()
        finally:
            ctx.set_option(pkg.SLSHT_OPT_ROTWIN_ENGINE, 0)
    (tc, k_tc), (cc, k_cc) = out[0], out[1]
    assert rel(tc, ref) < TOL[1] and rel(cc, ref) < TOL[1]
    assert rel(tc, cc) < 5e-6
    assert k_tc == k_cc + 1
    call = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=1).cpu().numpy()
    assert rel(tc, call) < 5e-6


def test_batch_argument_errors(pkg, ctx):
    import torch
    Lf, Lh, grid = 4, 2, (3, 2, 3)
    fd = _dev(synth.signal_cn_real(Lf, 1))
    hd = _dev(synth.window_cn(Lh, 2))
    pairs = synth.pairs_all(Lf)
    with pytest.raises(pkg.SlshtError):                  # host signal
        ctx.batch([_item(Lf, Lh, grid, fd.cpu(), hd, pairs, 0)])
    with pytest.raises(pkg.SlshtError):                  # pair outside the band
        ctx.batch([_item(Lf, Lh, grid, fd, hd, [[Lf + Lh - 1, 0]], 0)])
    g = torch.empty(len(pairs) * 3 * 2 * 3 + 1, dtype=torch.complex64, device="cuda")
    with pytest.raises(pkg.SlshtError):                  # misaligned output
        it = _item(Lf, Lh, grid, fd, hd, pairs, 1)
        it["g_out"] = g[1:]
        ctx.batch([it])
    assert ctx.mem_used() >= 0


@pytest.mark.parametrize("flags", ["double_float", "fp64_only"])
def test_fp64_engines_vs_oracle(pkg, ctx, flags):
    """FP64 items in double-float arithmetic (pairs of floats on the FP32
    pipe, forced) and in FP64 arithmetic (forced): both within the FP64 path's
    1e-12 of the oracle."""
    f = pkg.SLSHT_BATCH_FP64_DD if flags == "double_float" else pkg.SLSHT_BATCH_NO_DD
    spec = _mix()
    items, refs, _ = _build_items(spec)
    b = ctx.batch(items, flags=f)
    try:
        for i, (it, ref) in enumerate(zip(items, refs)):
            err = rel(b.outputs[i].cpu().numpy(), ref)
            assert err < TOL[it["prec"]], (i, err)
            if it["prec"] == 0:
                assert b.query(pkg.SLSHT_BQ_ENGINE, i) == (1 if flags == "double_float" else 0)
    finally:
        b.close()


def test_double_float_engine_extreme_scales(pkg, ctx):
    """The double-float engine scales k and the rotated window by powers of two
    into the float range: signals near 1e-35 and windows near 1e+30 (far
    outside what unscaled float pairs could hold) keep FP64 accuracy."""
    Lf, Lh, grid = 9, 5, (35, 9, 9)
    f = synth.signal_powerlaw(Lf, 51) * 1e-35
    h = synth.window_cn(Lh, 52) * 1e30
    pairs = synth.pairs_random(Lf + Lh - 1, 10, 53)
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    b = ctx.batch([_item(Lf, Lh, grid, _dev(f), _dev(h), pairs, 0)], flags=pkg.SLSHT_BATCH_FP64_DD)
    try:
        assert b.query(pkg.SLSHT_BQ_ENGINE, 0) == 1
        assert rel(b.outputs[0].cpu().numpy(), ref) < 1e-12
    finally:
        b.close()


def test_double_float_matches_fp64_arithmetic(pkg, ctx):
    """The two FP64 engines agree far inside the tolerance on a larger case
    (workload-3 band limits, both alpha forms)."""
    Lf, Lh = 64, 16
    f, h = synth.signal_powerlaw(Lf, 61), synth.window_cn(Lh, 62, decay=1.0)
    pairs = synth.pairs_bands([17, 63])
    for grid in [(127, 20, 31), (105, 12, 31)]:            # direct (prime N_alpha) and split (3, 5, 7)
        b1 = ctx.batch([_item(Lf, Lh, grid, _dev(f), _dev(h), pairs, 0)], flags=pkg.SLSHT_BATCH_FP64_DD)
        b2 = ctx.batch([_item(Lf, Lh, grid, _dev(f), _dev(h), pairs, 0)], flags=pkg.SLSHT_BATCH_NO_DD)
        try:
            x, y = b1.outputs[0].cpu().numpy(), b2.outputs[0].cpu().numpy()
            assert rel(x, y) < 1e-13, grid
        finally:
            b1.close()
            b2.close()


def test_tune_feeds_per_call_fp64(pkg, ctx):
    """slsht_tune measures one FP64 grid shape; the per-call forward then uses
    the cached tile shape and stays within the FP64 tolerance, equal to the
    untuned call to rounding."""
    Lf, Lh, grid = 20, 9, (45, 20, 17)
    f, h = synth.signal_powerlaw(Lf, 71), synth.window_cn(Lh, 72)
    pairs = synth.pairs_random(Lf + Lh - 1, 9, 73)
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    before = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=0).cpu().numpy()
    ctx.tune(Lf, Lh, grid, 0)
    after = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=0).cpu().numpy()
    assert rel(before, ref) < 1e-12
    assert rel(after, ref) < 1e-12
    assert rel(after, before) < 1e-13
