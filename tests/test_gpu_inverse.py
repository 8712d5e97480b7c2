"""GPU inverse (Eq. inversion_1/2 with the exact SO(3) quadrature) through the
C ABI: against the oracle's inverse on the same g, and the round trip f -> g -> f
(the paper's own accuracy check, Sec. V-A)."""
import numpy as np
import pytest

import synth
from oracle import slsht as O

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("cfg", [1, 2])
def test_round_trip(ctx, cfg):
    c = synth.CONFIGS[cfg]
    f, h, _ = synth.config_inputs(cfg)
    pairs = synth.pairs_all(c["Lf"])
    for prec, tol in [(0, 1e-12), (1, 1e-5)]:
        g = ctx.forward(c["Lf"], c["Lh"], c["grid"], f, h, pairs, prec=prec)
        fr = ctx.inverse(c["Lf"], c["Lh"], c["grid"], g, h[0], pairs, prec=prec)
        err = np.linalg.norm(fr - f) / np.linalg.norm(f)
        assert err < tol, (cfg, prec, err)


def test_inverse_matches_oracle_inverse(ctx):
    import torch
    Lf, Lh, grid = 9, 4, (7, 5, 9)
    f = synth.signal_powerlaw(Lf, 11)
    h = synth.window_cn(Lh, 12)
    pairs = synth.pairs_all(Lf + Lh - 1)
    rng = np.random.default_rng(3)
    g = rng.standard_normal((len(pairs),) + grid) + 1j * rng.standard_normal((len(pairs),) + grid)
    ref = O.inverse(g, h[0], grid)
    gd = torch.from_numpy(g).cuda()
    fr = ctx.inverse(Lf, Lh, grid, gd, h[0], pairs, prec=0)
    assert np.max(np.abs(fr - ref)) / np.max(np.abs(ref)) < 1e-13
    # complex64 g: FP32 block sums feeding FP64 totals, held to the FP32_BULK bound
    g32 = torch.from_numpy(g.astype(np.complex64)).cuda()
    ref32 = O.inverse(g.astype(np.complex64).astype(np.complex128), h[0], grid)
    fr32 = ctx.inverse(Lf, Lh, grid, g32, h[0], pairs, prec=1)
    assert np.max(np.abs(fr32 - ref32)) / np.max(np.abs(ref32)) < 1e-5


def test_inverse_is_bitwise_reproducible(ctx):
    Lf, Lh, grid = 8, 3, (9, 6, 5)
    f = synth.signal_cn_real(Lf, 1)
    h = synth.window_cn(Lh, 2)
    pairs = synth.pairs_all(Lf)
    g = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=0)
    a = ctx.inverse(Lf, Lh, grid, g, h[0], pairs, prec=0)
    b = ctx.inverse(Lf, Lh, grid, g, h[0], pairs, prec=0)
    assert np.array_equal(a, b)


def test_inverse_argument_errors(ctx):
    import paper_1207_5558_gb300 as pkg
    import torch
    g = torch.zeros((1, 4, 4, 4), dtype=torch.complex128, device="cuda")
    out = np.zeros(1, complex)
    with pytest.raises(pkg.SlshtError) as e:
        pkg.slsht_inverse(ctx.h, pkg.make_desc(4, 2, (4, 4, 4)), g, 0.0, np.array([[1, 0]], np.int32), 1, out)
    assert e.value.code == -2
    with pytest.raises(pkg.SlshtError) as e:      # grid coarser than the window band limit
        pkg.slsht_inverse(ctx.h, pkg.make_desc(4, 5, (4, 4, 4)), g, 1.0, np.array([[1, 0]], np.int32), 1, out)
    assert e.value.code == -1
    with pytest.raises(pkg.SlshtError) as e:      # g in host memory
        pkg.slsht_inverse(ctx.h, pkg.make_desc(4, 2, (4, 4, 4)), g.cpu().numpy(), 1.0,
                          np.array([[1, 0]], np.int32), 1, out)
    assert e.value.code == -1


def test_inverse_fp32_long_rows(ctx):
    """complex64 inverse over rows longer than four thread strides (the
    unrolled loop and its tail) and several alpha rows per slab, against the
    oracle's inverse of the same complex64 values."""
    import torch
    Lf, Lh, grid = 6, 3, (37, 41, 29)       # 1189 columns: 4 strides of 256 plus a tail
    h = synth.window_cn(Lh, 21)
    pairs = synth.pairs_all(4)
    rng = np.random.default_rng(9)
    g = (rng.standard_normal((len(pairs),) + grid) + 1j * rng.standard_normal((len(pairs),) + grid)).astype(np.complex64)
    ref = O.inverse(g.astype(np.complex128), h[0], grid)
    fr = ctx.inverse(Lf, Lh, grid, torch.from_numpy(g).cuda(), h[0], pairs, prec=1)
    assert np.max(np.abs(fr - ref)) / np.max(np.abs(ref)) < 1e-5


def _alt_pairs(outs, p):
    return np.array(sorted({(int(L) + p, int(M) + q) for L, M in outs for q in range(-p, p + 1)}), dtype=np.int32)


@pytest.mark.parametrize("Lf,Lh,p,grid", [
    (8, 4, 1, (5, 5, 5)),            # the smallest exact grid: every size L_h + p
    (8, 4, 3, (9, 8, 7)),
    (24, 8, 2, (47, 24, 15)),        # workload-2-like grid (N_beta = L_f)
    (20, 12, 5, (39, 20, 27)),       # orders in two passes of the projection kernel
])
@pytest.mark.parametrize("prec", [0, 1])
def test_inverse_alt_without_dc(ctx, Lf, Lh, p, grid, prec):
    """The inverse of the remark after Eq. inversion_2 for a window with
    h_0^0 = 0: f recovered from g at degrees L + p (round trip), and equal to
    the oracle's inverse_alt on the same g."""
    import torch
    f = synth.signal_powerlaw(Lf, 400 + p)
    h = synth.window_cn(Lh, 401 + p, decay=1.0)
    h[0] = 0.0
    outs = synth.pairs_all(Lf)
    pairs = _alt_pairs(outs, p)
    g = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=prec)
    torch.cuda.synchronize()
    fr = ctx.inverse_alt(Lf, Lh, grid, g, h, pairs, p, outs, prec=prec)
    ft = f[outs[:, 0] ** 2 + outs[:, 0] + outs[:, 1]]
    tol = 1e-12 if prec == 0 else 1e-5
    assert np.linalg.norm(fr - ft) / np.linalg.norm(ft) < tol
    ref = O.inverse_alt(g.cpu().numpy().astype(np.complex128), h, Lh, pairs, grid, p, outs)
    assert np.linalg.norm(fr - ref) / np.linalg.norm(ref) < (1e-13 if prec == 0 else 1e-6)


def test_inverse_alt_device_arguments_and_errors(ctx):
    """Device-resident h, pair lists and output; the argument checks (a
    missing pair, a degree without window energy, a grid below L_h + p)."""
    import torch
    import paper_1207_5558_gb300 as pkg
    Lf, Lh, p, grid = 10, 5, 2, (9, 10, 11)
    f = synth.signal_powerlaw(Lf, 410)
    h = synth.window_cn(Lh, 411)
    h[0] = 0.0
    outs = synth.pairs_all(Lf)
    pairs = _alt_pairs(outs, p)
    g = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=0)
    hd, ind, outd = (torch.from_numpy(h).cuda(), torch.from_numpy(pairs).cuda(), torch.from_numpy(outs).cuda())
    fd = torch.zeros(len(outs), dtype=torch.complex128, device="cuda")
    desc = pkg.make_desc(Lf, Lh, grid, 0)
    pkg.slsht_inverse_alt(ctx.h, desc, g, hd, ind, len(pairs), p, outd, len(outs), fd)
    torch.cuda.synchronize()
    ft = f[outs[:, 0] ** 2 + outs[:, 0] + outs[:, 1]]
    assert np.linalg.norm(fd.cpu().numpy() - ft) / np.linalg.norm(ft) < 1e-12
    with pytest.raises(pkg.SlshtError) as e:                      # (L + p, M + q) missing
        ctx.inverse_alt(Lf, Lh, grid, g[1:], h, pairs[1:], p, outs)
    assert e.value.code == -1
    hz = h.copy()
    hz[p * p:(p + 1) * (p + 1)] = 0.0
    with pytest.raises(pkg.SlshtError) as e:                      # E_p = 0
        ctx.inverse_alt(Lf, Lh, grid, g, hz, pairs, p, outs)
    assert e.value.code == -2
    with pytest.raises(pkg.SlshtError) as e:                      # n_beta < L_h + p
        ctx.inverse_alt(Lf, Lh, (9, 6, 11), g, h, pairs, p, outs)
    assert e.value.code == -1
