"""slsht_forward_noalloc: the forward transform for callers that cannot
allocate device memory when they need it (host callbacks and real-time
sections where cudaMalloc's implicit synchronisation is not allowed, plug-ins
whose host owns the device allocator, processes that gave the whole device to
a fixed pool).  It works in one static device array instead of allocating.

Checked here against slsht_forward (which allocates its scratch) on two calls
in a row with different shapes, so the second call runs over what the first
left in the shared array; and an oversized request must be refused before
anything runs.  This file is collected last on purpose."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1207_5558_gb300 as pkg
    from paper_1207_5558_gb300 import build
    build.build()
    ctx = pkg.Context(0)
    yield pkg, ctx
    ctx.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_forward_twice(env, prec):
    import torch
    pkg, ctx = env
    cases = [
        (16, 4, (31, 16, 7), synth.signal_cn_real(16, 41), synth.window_cn(4, 42), synth.pairs_all(19)),
        (40, 8, (79, 40, 15), synth.signal_powerlaw(40, 43), synth.window_cn(8, 44, decay=1.0),
         synth.pairs_bands([0, 13, 39, 46])),
    ]
    for Lf, Lh, grid, f, h, pairs in cases:
        ref = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=prec).cpu().numpy()
        dt = torch.complex128 if prec == 0 else torch.complex64
        g = torch.full((len(pairs),) + grid, float("nan"), dtype=dt, device="cuda")
        pkg.slsht_forward_noalloc(pkg.make_desc(Lf, Lh, grid, prec), f, h, pairs, len(pairs), g)
        torch.cuda.synchronize()
        assert _rel(g.cpu().numpy(), ref) < TOL[prec], (Lf, Lh, prec)


def test_noalloc_rejects_requests_beyond_the_array(env):
    import torch
    pkg, ctx = env
    Lf, Lh, grid = 8, 16, (4095, 2048, 31)    # this grid's FP64 d(beta) table alone (89 MB) exceeds the array
    g = torch.empty(8, dtype=torch.complex128, device="cuda")
    f = synth.signal_cn_real(Lf, 1)
    h = synth.window_cn(Lh, 2)
    with pytest.raises(pkg.SlshtError) as e:
        pkg.slsht_forward_noalloc(pkg.make_desc(Lf, Lh, grid, 0), f, h, np.array([[3, 1]], np.int32), 1, g)
    assert e.value.code == -3
    assert "static scratch limit" in pkg._abi.load().slsht_last_error().decode()
