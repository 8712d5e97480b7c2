"""Workload 5 at full size through the C ABI: L_f = 2048, L_h = 64 (the
8 x 3 degree elliptical eigenfunction window), 16 seeded pairs, each on the
full 4095 x 2048 x 127 grid (1.7e10 complex64 samples, 136 GB on the device),
FP32_BULK with the FP64 Delta recursion and 3j generation.

Checked: eight seeded beta rows (full alpha and gamma) of four seeded pairs
against the oracle's coefficient-domain route with its coupling from the
order-recursion 3j families (Racah's rational sum is too slow for a whole
pair at l ~ 2000; the families are pinned against it in the oracle tests),
and the inversion round trip of all 16 f_lm (Sec. III-C)."""
import numpy as np
import pytest

import synth
from oracle import slsht as O

pytestmark = pytest.mark.gpu


def _window():
    """The stored L_h = 64 window, written by the oracle (make_windows.py)."""
    return synth.stored_window(5)[0]


def test_workload5_full_grid():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < (150 << 30):
        pytest.skip("workload 5 keeps 136 GB of g on the device")
    import paper_1207_5558_gb300 as pkg
    from paper_1207_5558_gb300 import build
    build.build()
    c = synth.CONFIGS[5]
    Lf, Lh, grid = c["Lf"], c["Lh"], c["grid"]
    h = _window()
    f, _, pairs = synth.config_inputs(5, window_cache=h)
    ctx = pkg.Context(0, mem_budget_bytes=(48 << 30))
    try:
        g = torch.empty((len(pairs),) + grid, dtype=torch.complex64, device="cuda")
        ctx.forward(Lf, Lh, grid, f, h, pairs, prec=pkg.SLSHT_FP32_BULK, g_out=g)
        # inversion round trip of every pair
        fr = ctx.inverse(Lf, Lh, grid, g, h[0], pairs, prec=pkg.SLSHT_FP32_BULK)
        ftrue = f[pairs[:, 0] ** 2 + pairs[:, 0] + pairs[:, 1]]
        assert np.linalg.norm(fr - ftrue) / np.linalg.norm(ftrue) < 1e-5
        # sampled rows against the oracle
        rng = np.random.default_rng(5005)
        sel = np.sort(rng.choice(len(pairs), size=4, replace=False))
        rows = np.sort(rng.choice(grid[1], size=8, replace=False))
        got = g[torch.as_tensor(sel, device="cuda")][:, :, torch.as_tensor(rows, device="cuda"), :].cpu().numpy()
        del g
        ref = O.forward_coeff(f, h, Lf, Lh, pairs[sel], grid, beta_rows=rows, kroute="recurrence")
        for i in range(len(sel)):
            err = np.linalg.norm(got[i] - ref[i]) / np.linalg.norm(ref[i])
            assert err < 1e-5, (tuple(pairs[sel[i]]), err)
    finally:
        ctx.close()
