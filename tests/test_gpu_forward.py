"""GPU parity of the forward transform through the C ABI against the FP64
oracle.  Tolerances: relative L2 <= 1e-12 for the FP64 path and <= 1e-5 for
FP32_BULK, per call (the bounds the method's precision targets state)."""
import numpy as np
import pytest

import synth
from oracle import slsht as O

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


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


def _fw(ctx, Lf, Lh, grid, f, h, pairs, prec):
    return ctx.forward(Lf, Lh, grid, f, h, pairs, prec=prec).cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
def test_config1_vs_direct_quadrature(ctx, prec):
    """Workload 1 in full: L_f=16, L_h=4, all l<16, grid 31x16x7, against the
    quadrature of the definition (Eq. stft_spatial)."""
    c = synth.CONFIGS[1]
    f, h, pairs = synth.config_inputs(1)
    ref = O.forward_quadrature(f, h, c["Lf"], c["Lh"], pairs, c["grid"])
    g = _fw(ctx, c["Lf"], c["Lh"], c["grid"], f, h, pairs, prec)
    assert rel(g, ref) < (TOL64 if prec == 0 else TOL32)


@pytest.mark.parametrize("route", [1, 2])
def test_beta_routes_agree_with_oracle(ctx, route):
    """Both beta-stage routes: d(beta) table (separation of variables) and the
    factoring of rotations (C tensor + DFT in q'')."""
    import paper_1207_5558_gb300 as pkg
    Lf, Lh, grid = 12, 5, (23, 12, 9)
    f = synth.signal_powerlaw(Lf, 3)
    h = synth.window_cn(Lh, 4)
    pairs = synth.pairs_all(Lf + Lh - 1)
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    ctx.set_option(pkg.SLSHT_OPT_BETA_ROUTE, route)
    try:
        for prec, tol in [(0, TOL64), (1, TOL32)]:
            g = _fw(ctx, Lf, Lh, grid, f, h, pairs, prec)
            assert rel(g, ref) < tol, (route, prec)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_BETA_ROUTE, 0)


@pytest.mark.parametrize("Lf,Lh,grid", [
    (1, 1, (1, 1, 1)),        # K = 1, one sample
    (5, 1, (3, 2, 1)),        # window = constant
    (4, 2, (5, 3, 1)),        # N_gamma = 1
    (6, 6, (11, 6, 11)),      # L_h = L_f, native grid
    (3, 7, (13, 7, 13)),      # L_h > L_f
    (9, 4, (2, 1, 3)),        # fewer samples than the band limit
    (7, 3, (130, 5, 33)),     # ragged: several alpha tiles, columns not a multiple of a warp
    (5, 2, (257, 3, 45)),     # columns not a multiple of the 128-column tensor-core tile
])
def test_edge_shapes(ctx, Lf, Lh, grid):
    f = synth.signal_cn_real(Lf, Lf * 100 + Lh)
    h = synth.window_cn(Lh, Lh * 7 + 1)
    pairs = synth.pairs_all(Lf + Lh - 1)        # includes l > Lf - 1 and |m| = l
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    for prec, tol in [(0, TOL64), (1, TOL32)]:
        g = _fw(ctx, Lf, Lh, grid, f, h, pairs, prec)
        assert rel(g, ref) < tol, (prec, rel(g, ref))


def test_vanishing_and_window_y00(ctx):
    Lf, Lh, grid = 6, 1, (4, 3, 2)
    f = synth.signal_cn_real(Lf, 2)
    h = np.ones(1, complex)
    pairs = synth.pairs_all(Lf)
    g = _fw(ctx, Lf, Lh, grid, f, h, pairs, 0)
    ref = f[:, None, None, None] / np.sqrt(4 * np.pi) * np.ones((1,) + grid)
    assert np.max(np.abs(g - ref)) < 1e-14


def test_config2_sampled_pairs(ctx):
    """Workload 2 (power-law f, 20x10 deg elliptical window, grid 127x64x15):
    the whole map in the bench's launch configuration, sampled pairs checked."""
    c = synth.CONFIGS[2]
    f, h, pairs = synth.config_inputs(2)
    g = ctx.forward(c["Lf"], c["Lh"], c["grid"], f, h, pairs, prec=0)
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, len(pairs) - 1, len(pairs) // 2], rng.choice(len(pairs), 20, replace=False)]))
    ref = O.forward_coeff(f, h, c["Lf"], c["Lh"], pairs[idx], c["grid"])
    got = g[idx].cpu().numpy()
    assert rel(got, ref) < TOL64


def test_config3_sampled_pairs_full_grid(ctx):
    """Workload 3 (L_f=256, L_h=16, grid 511x256x31): one whole map computed
    in the bench's launch configuration, seeded sampled pairs (including the
    extreme orders of l = 255) compared with the oracle over their full grid."""
    import torch
    c = synth.CONFIGS[3]
    f, h, pairs = synth.config_inputs(3, map_index=1)
    sel = [0, 32, 33, 161, 929, 928, 673]
    ref = O.forward_coeff(f, h, c["Lf"], c["Lh"], pairs[sel], c["grid"])
    for prec, tol in [(0, TOL64), (1, TOL32)]:
        g = ctx.forward(c["Lf"], c["Lh"], c["grid"], f, h, pairs, prec=prec)
        got = g[sel].cpu().numpy()
        del g
        torch.cuda.empty_cache()
        assert rel(got, ref) < tol, prec
        for i in range(len(sel)):
            assert rel(got[i], ref[i]) < tol * 10, (prec, sel[i])


def test_host_output_buffer(ctx):
    """g_out in host memory: the library stages chunks and copies them back."""
    import torch
    import paper_1207_5558_gb300 as pkg
    Lf, Lh, grid = 10, 4, (19, 10, 7)
    f = synth.signal_powerlaw(Lf, 5)
    h = synth.window_cn(Lh, 6)
    pairs = synth.pairs_all(Lf)
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    ctx.set_option(pkg.SLSHT_OPT_CHUNK_PAIRS, 7)
    try:
        for prec, tol, dt in [(0, TOL64, np.complex128), (1, TOL32, np.complex64)]:
            host = np.zeros((len(pairs),) + grid, dtype=dt)
            pkg.slsht_forward(ctx.h, pkg.make_desc(Lf, Lh, grid, prec), f, h, pairs, len(pairs), host)
            torch.cuda.synchronize()
            assert rel(host, ref) < tol
    finally:
        ctx.set_option(pkg.SLSHT_OPT_CHUNK_PAIRS, 0)


def test_device_inputs_and_chunking(ctx):
    import torch
    import paper_1207_5558_gb300 as pkg
    Lf, Lh, grid = 9, 3, (17, 9, 5)
    f = synth.signal_cn_real(Lf, 8)
    h = synth.window_cn(Lh, 9)
    pairs = synth.pairs_all(Lf + Lh - 1)
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    fd = torch.from_numpy(f).cuda()
    hd = torch.from_numpy(h).cuda()
    lmd = torch.from_numpy(pairs).cuda()
    for chunk in (1, 5, 0):
        ctx.set_option(pkg.SLSHT_OPT_CHUNK_PAIRS, chunk)
        g = torch.empty((len(pairs),) + grid, dtype=torch.complex128, device="cuda")
        pkg.slsht_forward(ctx.h, pkg.make_desc(Lf, Lh, grid, 0), fd, hd, lmd, len(pairs), g)
        assert rel(g.cpu().numpy(), ref) < TOL64
    ctx.set_option(pkg.SLSHT_OPT_CHUNK_PAIRS, 0)


def test_invalid_arguments_rejected(ctx):
    import torch
    import paper_1207_5558_gb300 as pkg
    g = torch.empty((1, 3, 3, 3), dtype=torch.complex128, device="cuda")
    f = np.zeros(16, complex)
    h = np.ones(4, complex)
    with pytest.raises(pkg.SlshtError) as e:
        pkg.slsht_forward(ctx.h, pkg.make_desc(4, 2, (3, 3, 3)), f, h, np.array([[5, 0]], np.int32), 1, g)
    assert e.value.code == -1
    with pytest.raises(pkg.SlshtError):
        pkg.slsht_forward(ctx.h, pkg.make_desc(4, 2, (3, 3, 3)), f, h, np.array([[2, 3]], np.int32), 1, g)
    assert pkg.slsht_forward(ctx.h, pkg.make_desc(4, 2, (3, 3, 3)), f, h, np.zeros((0, 2), np.int32), 0, g) == 0


def test_determinism(ctx):
    Lf, Lh, grid = 12, 6, (23, 12, 11)
    f = synth.signal_powerlaw(Lf, 1)
    h = synth.window_cn(Lh, 2)
    pairs = synth.pairs_all(Lf)
    for prec in (0, 1):
        a = _fw(ctx, Lf, Lh, grid, f, h, pairs, prec)
        b = _fw(ctx, Lf, Lh, grid, f, h, pairs, prec)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("engine", [1, 2, 3])
def test_fp32_alpha_engines(ctx, engine):
    """FP32_BULK with the alpha stage on CUDA cores (1), on tcgen05 fed by the
    separate producer kernel (2) and in the fused producer + tcgen05 kernel (3)."""
    import paper_1207_5558_gb300 as pkg
    Lf, Lh, grid = 20, 16, (300, 9, 31)      # K = 31: the largest single K block; 3 alpha chunks
    f = synth.signal_powerlaw(Lf, 21)
    h = synth.window_cn(Lh, 22, decay=1.0)
    pairs = synth.pairs_bands([0, 7, 19, 33])
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, engine)
    try:
        g = _fw(ctx, Lf, Lh, grid, f, h, pairs, 1)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, 0)
    assert rel(g, ref) < TOL32
    st = ctx.stats()
    assert st is not None


@pytest.mark.parametrize("engine", [2, 3])
@pytest.mark.parametrize("Lf,Lh,grid,chunk", [
    (6, 3, (130, 5, 33), 7),      # 165 columns: a ragged second tile; 2 alpha chunks; 5 launches
    (8, 7, (257, 3, 45), 0),      # 3 alpha chunks, the last one row long
    (10, 12, (140, 11, 23), 5),   # the 16-degree producer bucket with L_h = 12
])
def test_tensor_core_engines_ragged(ctx, engine, Lf, Lh, grid, chunk):
    """Both tensor-core engines on tiles and alpha chunks that do not divide
    the grid, with the pairs split over several launches."""
    import paper_1207_5558_gb300 as pkg
    f = synth.signal_powerlaw(Lf, 40 + Lh)
    h = synth.window_cn(Lh, 50 + Lh, decay=1.0)
    every = synth.pairs_all(Lf + Lh - 1)
    pairs = synth.subsample_pairs(every, 23 / len(every), seed=Lh)
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, engine)
    ctx.set_option(pkg.SLSHT_OPT_CHUNK_PAIRS, chunk)
    try:
        g = _fw(ctx, Lf, Lh, grid, f, h, pairs, 1)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, 0)
        ctx.set_option(pkg.SLSHT_OPT_CHUNK_PAIRS, 0)
    assert rel(g, ref) < TOL32
    assert np.abs(g - ref).max() <= 1e-5 * np.abs(ref).max()


def test_gaunt_table_reuse_and_invalidation(ctx):
    """The per-workspace Gaunt table: a repeated pair list with a new signal,
    then a different pair list, then the first again, each against the path
    that recomputes the 3j chains in the call, and against the oracle."""
    import paper_1207_5558_gb300 as pkg
    Lf, Lh, grid = 24, 6, (47, 24, 11)
    h = synth.window_cn(Lh, 61)
    lists = [synth.pairs_bands([3, 17, 28]), synth.pairs_bands([0, 9, 23]), synth.pairs_bands([3, 17, 28])]
    sigs = [synth.signal_powerlaw(Lf, 62), synth.signal_powerlaw(Lf, 63), synth.signal_powerlaw(Lf, 64)]
    got = []
    for f, pairs in zip(sigs, lists):
        got.append(_fw(ctx, Lf, Lh, grid, f, h, pairs, 0))
    ctx.set_option(pkg.SLSHT_OPT_GAUNT_TABLE, 2)
    try:
        for (f, pairs), g in zip(zip(sigs, lists), got):
            ref_gpu = _fw(ctx, Lf, Lh, grid, f, h, pairs, 0)
            assert rel(g, ref_gpu) < 1e-13
    finally:
        ctx.set_option(pkg.SLSHT_OPT_GAUNT_TABLE, 0)
    for (f, pairs), g in zip(zip(sigs, lists), got):
        assert rel(g, O.forward_coeff(f, h, Lf, Lh, pairs, grid)) < TOL64


def test_gaunt_table_mirror_pairs_with_duplicates(ctx):
    """Mirror pairs (l, m), (l, -m) share one chain in the Gaunt table; lists
    with repeated pairs, unmatched mirrors and m = 0 against the per-call
    chains and the oracle."""
    import paper_1207_5558_gb300 as pkg
    Lf, Lh, grid = 20, 7, (39, 20, 13)
    f = synth.signal_powerlaw(Lf, 71)
    h = synth.window_cn(Lh, 72)
    pairs = np.array([[5, 2], [5, 2], [5, -2], [7, 3], [7, 0], [9, -4], [24, 1], [24, -1], [3, -3]], dtype=np.int32)
    g = _fw(ctx, Lf, Lh, grid, f, h, pairs, 0)
    ctx.set_option(pkg.SLSHT_OPT_GAUNT_TABLE, 2)
    try:
        g2 = _fw(ctx, Lf, Lh, grid, f, h, pairs, 0)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_GAUNT_TABLE, 0)
    assert rel(g, g2) < 1e-13
    assert rel(g, O.forward_coeff(f, h, Lf, Lh, pairs, grid)) < TOL64


@pytest.mark.parametrize("npairs", [3, 7, 37])
def test_wide_engine_pair_group_sizes(ctx, npairs):
    """The wide engine's producer in groups of up to 16 pairs (one launch
    over every group, with the group's sums in registers: 4, 8 or 16 of them
    a thread): 3, 7 and 37 pairs (two full groups and a group of 5), FP32_BULK
    at L_h = 20 and 40, against the oracle and the CUDA-core alpha stage."""
    import paper_1207_5558_gb300 as pkg
    Lf = 14
    for Lh in (20, 40):
        grid = (2 * (Lf + Lh) - 1, 10, 2 * Lh - 1)
        f = synth.signal_powerlaw(Lf, 181 + Lh)
        h = synth.window_cn(Lh, 182 + Lh, decay=1.0)
        pairs = synth.pairs_random(Lf + Lh - 1, npairs, 183 + npairs)
        g = _fw(ctx, Lf, Lh, grid, f, h, pairs, 1)
        assert rel(g, O.forward_coeff(f, h, Lf, Lh, pairs, grid)) < TOL32
        ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, 1)
        try:
            cc = _fw(ctx, Lf, Lh, grid, f, h, pairs, 1)
        finally:
            ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, 0)
        assert rel(g, cc) < 5e-6


@pytest.mark.parametrize("Lh", [7, 24, 40])
def test_coupling_chains_share_mirror_items(ctx, Lh):
    """The 3j chains of the call (SLSHT_OPT_GAUNT_TABLE 2) run once for a
    pair and its mirror (l, -m), and once for the items (p, q), (p, -q) of an
    m = 0 pair: a list with matched and unmatched mirrors, a repeated pair, a
    pair listed before its mirror and after it, against the oracle and the
    Gaunt-table route (every chain length class: L_h <= 16, <= 32, <= 64)."""
    import paper_1207_5558_gb300 as pkg
    Lf = 30
    grid = (2 * (Lf + Lh) - 1, 12, 2 * Lh - 1)
    f = synth.signal_powerlaw(Lf, 171)
    h = synth.window_cn(Lh, 172, decay=1.0)
    pairs = np.concatenate([np.array([[11, 4], [11, 4], [11, -4], [20, 0], [13, -7], [3, 2], [29 + Lh // 2, 5],
                                      [29 + Lh // 2, -5], [8, -3]], dtype=np.int32),
                            synth.pairs_bands([Lf + Lh - 2])[::3]])
    ctx.set_option(pkg.SLSHT_OPT_GAUNT_TABLE, 2)
    try:
        chains = _fw(ctx, Lf, Lh, grid, f, h, pairs, 0)
        ctx.set_option(pkg.SLSHT_OPT_GAUNT_TABLE, 1)
        table = _fw(ctx, Lf, Lh, grid, f, h, pairs, 0)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_GAUNT_TABLE, 0)
    assert rel(chains, table) < 1e-13
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    assert rel(chains, ref) < TOL64
    for i in range(len(pairs)):                      # every pair, mirrors and duplicates included
        assert rel(chains[i], ref[i]) < 1e-11, i


@pytest.mark.parametrize("name,prec,Lh,engine,rot", [
    ("fused", 1, 5, 0, 0),           # k_alpha_fused: producer warps in the alpha kernel
    ("two_kernel", 1, 5, 2, 0),      # k_alpha_tc fed by k_xa_from_h
    ("wide", 1, 20, 0, 0),           # k_alpha_tcw (16 < L_h <= 64)
    ("fp64_digits", 0, 5, 0, 0),     # k_alpha_tc64 (FP64 from exact digit products)
    ("rotated_window", 1, 20, 0, 2), # k_rotwin_tc (the rotated window on the tensor cores)
])
def test_bounded_wait_expiry_reports_and_context_recovers(ctx, name, prec, Lh, engine, rot):
    """The timeout path of every tensor-core kernel: with one internal
    hand-off withheld (SLSHT_OPT_WAIT_TEST: the fused kernel's first A tile is
    never handed to the issuer; the other alpha kernels' first A operand and
    the rotated window's first d chunk are never fetched) the bounded waits
    expire, the kernel leaves cleanly, slsht_get_stats reports
    SLSHT_E_TIMEOUT, and the next call on the same context is correct."""
    import torch
    import paper_1207_5558_gb300 as pkg
    from paper_1207_5558_gb300 import _abi
    Lf, grid = 10, (130, 10, 2 * Lh + 3)
    f = synth.signal_powerlaw(Lf, 81)
    h = synth.window_cn(Lh, 82)
    pairs = synth.pairs_bands([2, 9])
    ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, engine)
    ctx.set_option(pkg.SLSHT_OPT_ROTWIN_ENGINE, rot)
    try:
        ctx.stats(reset=True)
        ctx.set_option(pkg.SLSHT_OPT_WAIT_TEST, 1)
        ctx.forward(Lf, Lh, grid, f, h, pairs, prec=prec)
        torch.cuda.synchronize()
        with pytest.raises(pkg.SlshtError) as e:
            ctx.stats()
        assert e.value.code == _abi.SLSHT_E_TIMEOUT
        ctx.stats()                                    # the error word was cleared
        g = _fw(ctx, Lf, Lh, grid, f, h, pairs, prec)
        assert rel(g, O.forward_coeff(f, h, Lf, Lh, pairs, grid)) < (TOL32 if prec else TOL64)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_WAIT_TEST, 0)
        ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, 0)
        ctx.set_option(pkg.SLSHT_OPT_ROTWIN_ENGINE, 0)


@pytest.mark.parametrize("prec,engine,arith", [(0, 0, 0), (0, 0, 1), (0, 0, 3), (1, 0, 0), (1, 1, 0), (1, 2, 0)])
def test_real_fields_mirror_pairs(ctx, prec, engine, arith):
    """SLSHT_OPT_REAL_FIELDS: for real f and h, g(l, -m) = (-1)^m conj g(l, m)
    (Sec. IV-B; pin (iv) of the oracle tests), so only one of each mirrored
    pair is computed and the alpha stage writes both.  Against the full
    computation and the oracle, with unmatched pairs and m = 0 in the list."""
    import paper_1207_5558_gb300 as pkg
    Lf, Lh, grid = 14, 6, (131, 14, 11)
    f = synth.signal_powerlaw(Lf, 91)
    h = synth.signal_cn_real(Lh, 92)
    pairs = np.concatenate([synth.pairs_bands([3, 13]), np.array([[9, 4], [18, -5]], dtype=np.int32)])
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, engine)
    ctx.set_option(pkg.SLSHT_OPT_FP64_ARITH, arith)
    try:
        full = _fw(ctx, Lf, Lh, grid, f, h, pairs, prec)
        ctx.set_option(pkg.SLSHT_OPT_REAL_FIELDS, 1)
        half = _fw(ctx, Lf, Lh, grid, f, h, pairs, prec)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_REAL_FIELDS, 0)
        ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, 0)
        ctx.set_option(pkg.SLSHT_OPT_FP64_ARITH, 0)
    tol = TOL64 if prec == 0 else TOL32
    assert rel(half, ref) < tol
    assert rel(half, full) < (1e-13 if prec == 0 else 2e-6)


@pytest.mark.parametrize("prec,arith", [(0, 0), (0, 1), (1, 0)])
@pytest.mark.parametrize("Na", [15, 33, 45, 105, 511])
def test_split_dft_alpha_stage(ctx, prec, arith, Na):
    """The CUDA-core alpha stage as a split DFT over a = Q s + t (P = 3, 5, 7
    or 9 dividing N_alpha) against the direct sum (engine 4) and the oracle,
    with mirrored pairs under the real-field option as well; FP64 both in
    double-float (arith 0) and in FP64 arithmetic (arith 1)."""
    import paper_1207_5558_gb300 as pkg
    ctx.set_option(pkg.SLSHT_OPT_FP64_ARITH, arith)
    Lf, Lh = 12, 12
    grid = (Na, 7, 9)
    f = synth.signal_powerlaw(Lf, 100 + Na)
    h = synth.signal_cn_real(Lh, 200 + Na)
    pairs = synth.pairs_bands([4, 15])
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    tol = TOL64 if prec == 0 else TOL32
    try:
        ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, 1)
        split = _fw(ctx, Lf, Lh, grid, f, h, pairs, prec)
        ctx.set_option(pkg.SLSHT_OPT_REAL_FIELDS, 1)
        split_mirror = _fw(ctx, Lf, Lh, grid, f, h, pairs, prec)
        ctx.set_option(pkg.SLSHT_OPT_REAL_FIELDS, 0)
        ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, 4)
        direct = _fw(ctx, Lf, Lh, grid, f, h, pairs, prec)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_REAL_FIELDS, 0)
        ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, 0)
        ctx.set_option(pkg.SLSHT_OPT_FP64_ARITH, 0)
    assert rel(split, ref) < tol
    assert rel(split_mirror, ref) < tol
    assert rel(direct, ref) < tol
    assert rel(split, direct) < (1e-13 if prec == 0 else 2e-6)


@pytest.mark.parametrize("prec", [0, 1])
def test_forward_windows_reuses_coupling(ctx, prec):
    """slsht_forward_windows (Sec. IV-B, several windows over one signal):
    equal to one slsht_forward per window, and to the oracle."""
    Lf, Lh, grid = 16, 7, (61, 16, 13)
    f = synth.signal_powerlaw(Lf, 301)
    hs = np.stack([synth.window_cn(Lh, 302 + i, decay=1.0) for i in range(3)])
    pairs = synth.pairs_bands([2, 11, 19])
    g = ctx.forward_windows(Lf, Lh, grid, f, hs, pairs, prec=prec).cpu().numpy()
    tol = TOL64 if prec == 0 else TOL32
    for i in range(3):
        single = _fw(ctx, Lf, Lh, grid, f, hs[i], pairs, prec)
        assert np.array_equal(g[i], single)
    assert rel(g[1], O.forward_coeff(f, hs[1], Lf, Lh, pairs, grid)) < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_modulated_sht_coupling_route(ctx, prec):
    """SLSHT_OPT_COUPLING 2: k by Gauss-Legendre quadrature of the modulated
    signal's transform (Appendix A) instead of Gaunt coefficients; against the
    oracle and the Gaunt route, including l > L_f - 1 and |m| = l."""
    import paper_1207_5558_gb300 as pkg
    Lf, Lh, grid = 20, 6, (45, 20, 11)
    f = synth.signal_powerlaw(Lf, 401)
    h = synth.window_cn(Lh, 402)
    pairs = synth.subsample_pairs(synth.pairs_all(Lf + Lh - 1), 0.1, seed=403)
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    gaunt = _fw(ctx, Lf, Lh, grid, f, h, pairs, prec)
    ctx.set_option(pkg.SLSHT_OPT_COUPLING, 2)
    try:
        msht = _fw(ctx, Lf, Lh, grid, f, h, pairs, prec)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_COUPLING, 0)
    tol = TOL64 if prec == 0 else TOL32
    assert rel(msht, ref) < tol
    assert rel(msht, gaunt) < (1e-12 if prec == 0 else 2e-6)


def test_modulated_sht_coupling_workload2_size(ctx):
    """Both coupling routes at workload 2's band limits (L_f = 64, L_h = 8),
    FP64, on a seeded 5% of its pairs."""
    import paper_1207_5558_gb300 as pkg
    c = synth.CONFIGS[2]
    f = synth.signal_powerlaw(c["Lf"], 404)
    h = synth.window_cn(c["Lh"], 405, decay=1.0)
    pairs = synth.subsample_pairs(synth.pairs_all(c["Lf"]), 0.05, seed=406)
    grid = (c["grid"][0], 12, c["grid"][2])
    gaunt = _fw(ctx, c["Lf"], c["Lh"], grid, f, h, pairs, 0)
    ctx.set_option(pkg.SLSHT_OPT_COUPLING, 2)
    try:
        msht = _fw(ctx, c["Lf"], c["Lh"], grid, f, h, pairs, 0)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_COUPLING, 0)
    assert rel(msht, gaunt) < 1e-12


@pytest.mark.parametrize("Lf,Lh,grid", [
    (6, 1, (9, 4, 1)),          # L_h = 1: one order, one alpha chunk (9 < 16 rows)
    (12, 4, (31, 5, 9)),        # a ragged alpha chunk (31 = 16 + 15), 45 columns in one tile
    (16, 8, (70, 9, 15)),       # 70 = 4 x 16 + 6 alpha rows, 135 columns: two tiles, the second ragged
    (20, 16, (511, 8, 31)),     # the widest narrow window at workload 3's N_alpha, 248 columns
])
def test_fp64_tensor_core_engine(ctx, Lf, Lh, grid):
    """The FP64 alpha stage from exact base-256 digit products on the tensor
    cores (the FP64 default for L_h <= 16, SLSHT_OPT_FP64_ARITH 0 or 2),
    against the oracle (FP64 bound), the double-float engine (3), and itself
    in chunks of two pairs."""
    import paper_1207_5558_gb300 as pkg
    f = synth.signal_powerlaw(Lf, 810 + Lh)
    h = synth.window_cn(Lh, 820 + Lh, decay=1.0)
    pairs = synth.pairs_random(Lf + Lh - 1, 7, 830 + Lh)
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    g0 = _fw(ctx, Lf, Lh, grid, f, h, pairs, 0)
    ctx.set_option(pkg.SLSHT_OPT_FP64_ARITH, 3)
    try:
        dd = _fw(ctx, Lf, Lh, grid, f, h, pairs, 0)
        ctx.set_option(pkg.SLSHT_OPT_FP64_ARITH, 2)
        g = _fw(ctx, Lf, Lh, grid, f, h, pairs, 0)
        ctx.set_option(pkg.SLSHT_OPT_CHUNK_PAIRS, 2)
        gc = _fw(ctx, Lf, Lh, grid, f, h, pairs, 0)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_CHUNK_PAIRS, 0)
        ctx.set_option(pkg.SLSHT_OPT_FP64_ARITH, 0)
    assert rel(g, ref) < TOL64
    assert rel(g, dd) < 1e-13
    assert np.array_equal(g, g0)           # the default
    if Lh > 1:                             # (L_h = 1: g = X_0 exactly, both ways)
        assert not np.array_equal(g, dd)   # a different arithmetic ran
    assert np.array_equal(g, gc)


@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("Na", [135, 127])
def test_fp64_widest_window_band(ctx, Na, arith):
    """FP64 at the largest window band limit, L_h = 64 (K = 127): the FP64
    alpha stage drops to 64-column CTAs to fit 127 staged coefficients, the
    double-float one to 32; N_alpha = 135 takes the split DFT (P = 9), 127
    the direct sum."""
    import paper_1207_5558_gb300 as pkg
    Lf, Lh = 6, 64
    grid = (Na, 3, 131)
    f = synth.signal_powerlaw(Lf, 500 + Na)
    h = synth.window_cn(Lh, 600 + Na, decay=1.0)
    pairs = np.array([[5, -2], [40, 7], [68, 68]], dtype=np.int32)
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid, kroute="recurrence")
    ctx.set_option(pkg.SLSHT_OPT_FP64_ARITH, arith)
    try:
        g = _fw(ctx, Lf, Lh, grid, f, h, pairs, 0)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_FP64_ARITH, 0)
    assert rel(g, ref) < TOL64


@pytest.mark.parametrize("Lf,Lh,grid", [
    (20, 17, (70, 9, 33)),      # two K-chunks; a ragged alpha chunk (70 = 64 + 6), 297 columns
    (12, 32, (130, 5, 63)),     # two K-chunks at their limit
    (8, 33, (65, 4, 65)),       # four K-chunks from here on
    (6, 64, (127, 3, 131)),     # four K-chunks at the largest window band
])
def test_wide_tensor_core_engine(ctx, Lf, Lh, grid):
    """FP32_BULK with L_h > 16 on the tensor cores (K split into 2 or 4 chunks
    of 64) against the oracle and against the CUDA-core path."""
    import paper_1207_5558_gb300 as pkg
    f = synth.signal_powerlaw(Lf, 700 + Lh)
    h = synth.window_cn(Lh, 800 + Lh, decay=1.0)
    pairs = synth.pairs_random(Lf + Lh - 1, 6, 900 + Lh)
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid, kroute="recurrence" if Lh > 40 else "exact")
    g = _fw(ctx, Lf, Lh, grid, f, h, pairs, 1)
    ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, 1)
    try:
        gc = _fw(ctx, Lf, Lh, grid, f, h, pairs, 1)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_ALPHA_ENGINE, 0)
    assert rel(g, ref) < TOL32
    assert rel(gc, ref) < TOL32
    assert rel(g, gc) < 2e-6


def test_wide_tensor_core_real_fields(ctx):
    """The wide engine's mirror stores: real f and h, SLSHT_OPT_REAL_FIELDS,
    equal to the full computation and the oracle."""
    import paper_1207_5558_gb300 as pkg
    Lf, Lh, grid = 10, 24, (67, 5, 47)
    f = synth.signal_powerlaw(Lf, 951)
    h = synth.signal_cn_real(Lh, 952)
    pairs = np.concatenate([synth.pairs_bands([5, 20]), np.array([[7, 3]], dtype=np.int32)])
    ref = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    full = _fw(ctx, Lf, Lh, grid, f, h, pairs, 1)
    ctx.set_option(pkg.SLSHT_OPT_REAL_FIELDS, 1)
    try:
        half = _fw(ctx, Lf, Lh, grid, f, h, pairs, 1)
    finally:
        ctx.set_option(pkg.SLSHT_OPT_REAL_FIELDS, 0)
    assert rel(half, ref) < TOL32
    assert rel(half, full) < 2e-6
