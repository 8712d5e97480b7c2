"""The concentrated-window generator on the device (slsht_window_ellipse,
Sec. III-D) against the oracle's generator (oracle/window.py, pinned in
test_window.py): the same eigenfunction and concentration."""
import numpy as np
import pytest

import synth
from oracle.window import window_ellipse
from synth import ellipse_from_axes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1207_5558_gb300 as pkg
    from paper_1207_5558_gb300 import build
    build.build()
    c = pkg.Context(0, mem_budget_bytes=(16 << 30))
    yield c
    c.close()


@pytest.mark.parametrize("L,region", [
    (8, ellipse_from_axes(20.0, 10.0)),           # workload 2
    (18, (np.pi / 6, np.pi / 6 + np.pi / 240)),   # Sec. V-B, 90% concentration
    (5, (0.0, 0.4)),                              # theta_c = 0: a polar cap
])
def test_window_matches_host_generator(ctx, L, region):
    h_ref, lam_ref = window_ellipse(L, *region)
    h, lam = ctx.window_ellipse(L, *region)
    assert abs(lam - lam_ref) < 1e-12
    assert np.linalg.norm(h - h_ref) < 1e-9
    assert h[0].real > 0 and abs(np.linalg.norm(h) - 1.0) < 1e-13


def test_window_workload5(ctx):
    """L = 64, 8 x 3 degrees (workload 5) against the oracle's stored result
    (tests/golden/make_windows.py)."""
    h_ref, lam_ref = synth.stored_window(5)
    h, lam = ctx.window_ellipse(64, *ellipse_from_axes(8.0, 3.0))
    assert np.linalg.norm(h - h_ref) < 1e-8
    assert abs(lam - lam_ref) < 1e-12
