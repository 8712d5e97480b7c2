"""Continuous-batching serving path (slsht_submit / slsht_poll / slsht_drain):
requests of different band limits and precisions submitted while others run;
each result must equal the same request run alone (bitwise: every kernel has a
fixed reduction order) and the oracle within the path's tolerance."""
import time

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


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        Lf = int(rng.choice([8, 16, 32]))
        Lh = int(rng.choice([2, 4, 8]))
        grid = synth.grid_native(Lh)
        nb = int(rng.integers(1, 4))
        bands = sorted(rng.choice(Lf, size=nb, replace=False).tolist())
        prec = int(rng.integers(0, 2))
        out.append(dict(Lf=Lf, Lh=Lh, grid=grid, prec=prec, f=synth.signal_powerlaw(Lf, 10 * seed + i),
                        h=synth.window_cn(Lh, 10 * seed + i + 5, decay=1.0), pairs=synth.pairs_bands(bands)))
    return out


def test_mix_equals_alone_and_oracle(ctx):
    import torch
    reqs = _requests(24, 7)
    alone = []
    for r in reqs:
        g = ctx.forward(r["Lf"], r["Lh"], r["grid"], r["f"], r["h"], r["pairs"], prec=r["prec"])
        torch.cuda.synchronize()
        alone.append(g.cpu().numpy())
    outs, tickets = [], []
    for r in reqs:
        dt = torch.complex128 if r["prec"] == 0 else torch.complex64
        g = torch.full((len(r["pairs"]),) + r["grid"], float("nan"), dtype=dt, device="cuda")
        outs.append(g)
        tickets.append(ctx.submit(r["Lf"], r["Lh"], r["grid"], r["f"], r["h"], r["pairs"], g, prec=r["prec"]))
    done = {}
    t0 = time.time()
    while len(done) < len(tickets) and time.time() - t0 < 120:
        for t in tickets:
            if t not in done:
                s = ctx.poll(t)
                if s != 1:
                    done[t] = s
        time.sleep(0.001)
    assert all(done.get(t) == 0 for t in tickets), done
    for r, g, a in zip(reqs, outs, alone):
        got = g.cpu().numpy()
        assert np.array_equal(got, a)
        ref = O.forward_coeff(r["f"], r["h"], r["Lf"], r["Lh"], r["pairs"][:3], r["grid"])
        tol = 1e-12 if r["prec"] == 0 else 1e-5
        assert np.linalg.norm(got[:3] - ref) / np.linalg.norm(ref) < tol
    assert ctx.poll(tickets[0]) == -7          # forgotten after its final status


def test_drain_and_invalid_submit(ctx):
    import paper_1207_5558_gb300 as pkg
    import torch
    r = _requests(1, 3)[0]
    g = torch.empty((len(r["pairs"]),) + r["grid"], dtype=torch.complex128, device="cuda")
    t = ctx.submit(r["Lf"], r["Lh"], r["grid"], r["f"], r["h"], r["pairs"], g, prec=0)
    assert ctx.drain(60000) == 0
    assert ctx.poll(t) == 0
    with pytest.raises(pkg.SlshtError):        # host output is not allowed for requests
        ctx.submit(r["Lf"], r["Lh"], r["grid"], r["f"], r["h"], r["pairs"], g.cpu().numpy(), prec=0)
    with pytest.raises(pkg.SlshtError):
        ctx.submit(r["Lf"], r["Lh"], r["grid"], r["f"], r["h"], np.array([[99, 0]], np.int32), g, prec=0)
