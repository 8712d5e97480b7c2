"""Continuous-batching serving path (slsht_submit / slsht_poll / slsht_drain):
requests of different band limits, window band limits, grids and precisions
submitted while others run, evaluated in ticks of persistent batched kernels
replayed from a captured graph.  Each result must equal the same request
served alone (bitwise: a request's tile shape depends only on its grid
shape, and every kernel has a fixed reduction order), the per-call forward
within the path's tolerance, and the oracle within the path's tolerance on
every pair; a large request is spread over several ticks without holding up
the small ones behind it."""
import time

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
    c = pkg.Context(0, mem_budget_bytes=(16 << 30))
    yield c
    c.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _requests(n, seed, Lfs, Lhs, max_band):
    """Requests with L_f in Lfs, L_h in Lhs, one to three degrees below
    max_band (all orders), FP64 or FP32_BULK, on the window's native grid."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        Lf = int(rng.choice(Lfs))
        Lh = int(rng.choice(Lhs))
        nb = int(rng.integers(1, 4))
        bands = sorted(rng.choice(min(Lf, max_band), size=nb, replace=False).tolist())
        out.append(dict(Lf=Lf, Lh=Lh, grid=synth.grid_native(Lh), prec=int(rng.integers(0, 2)),
                        f=synth.signal_powerlaw(Lf, 10 * seed + i), h=synth.window_cn(Lh, 10 * seed + i + 5, decay=1.0),
                        pairs=synth.pairs_bands(bands)))
    return out


def _serve(ctx, reqs, timeout_s=180):
    """Submit every request at once; returns (outputs, times)."""
    import torch
    outs, tickets = [], []
    for r in reqs:
        dt = torch.complex128 if r["prec"] == 0 else torch.complex64
        g = torch.full((len(r["pairs"]),) + r["grid"], float("nan"), dtype=dt, device="cuda")
        outs.append(g)
        tickets.append(ctx.submit(r["Lf"], r["Lh"], r["grid"], r["f"], r["h"], r["pairs"], g, prec=r["prec"]))
    done, times = {}, {}
    t0 = time.time()
    while len(done) < len(tickets) and time.time() - t0 < timeout_s:
        for t in tickets:
            if t not in done:
                s, tm = ctx.poll_times(t)
                if s != 1:
                    done[t] = s
                    times[t] = tm
        time.sleep(0.001)
    assert all(done.get(t) == 0 for t in tickets), done
    torch.cuda.synchronize()
    return [g.cpu().numpy() for g in outs], [times[t] for t in tickets]


@pytest.mark.parametrize("Lfs,Lhs,max_band", [
    ([8, 16, 32], [2, 4, 8], 32),
    ([128, 256], [16, 32], 8),           # wide windows, large signals; low degrees keep the oracle quick
])
def test_mix_equals_alone_and_oracle(ctx, Lfs, Lhs, max_band):
    reqs = _requests(16 if max_band > 8 else 8, 7 + len(Lfs), Lfs, Lhs, max_band)
    alone = [_serve(ctx, [r])[0][0] for r in reqs]
    mix, times = _serve(ctx, reqs)
    for r, got, a, tm in zip(reqs, mix, alone, times):
        assert np.array_equal(got, a)
        ref = O.forward_coeff(r["f"], r["h"], r["Lf"], r["Lh"], r["pairs"], r["grid"])
        assert _rel(got, ref) < TOL[r["prec"]]
        call = ctx.forward(r["Lf"], r["Lh"], r["grid"], r["f"], r["h"], r["pairs"], prec=r["prec"]).cpu().numpy()
        assert _rel(got, call) < TOL[r["prec"]]
        assert len(tm) == 4 and all(v >= 0 for v in tm) and tm[3] >= tm[0]


def test_large_request_is_split_and_does_not_block(ctx):
    """A request of ~4000 pairs (about 5e8 samples, several ticks) submitted
    first, then small requests: the small ones finish before the large one,
    and every result matches the oracle (sampled pairs of the large one)."""
    big = dict(Lf=128, Lh=32, grid=synth.grid_native(32), prec=1, f=synth.signal_powerlaw(128, 901),
               h=synth.window_cn(32, 902, decay=1.0), pairs=synth.pairs_bands(list(range(100, 118))))
    small = _requests(6, 903, [16, 32], [4, 8], 16)
    outs, times = _serve(ctx, [big] + small)
    for r, got in zip(small, outs[1:]):
        assert _rel(got, O.forward_coeff(r["f"], r["h"], r["Lf"], r["Lh"], r["pairs"], r["grid"])) < TOL[r["prec"]]
    idx = [0, 1234, len(big["pairs"]) - 1]
    ref = O.forward_coeff(big["f"], big["h"], big["Lf"], big["Lh"], big["pairs"][idx], big["grid"])
    assert _rel(outs[0][idx], ref) < TOL[1]
    assert max(t[3] for t in times[1:]) < times[0][3]


def test_drain_and_invalid_submit(ctx):
    import paper_1207_5558_gb300 as pkg
    import torch
    r = _requests(1, 3, [8, 16], [2, 4], 8)[0]
    g = torch.empty((len(r["pairs"]),) + r["grid"], dtype=torch.complex128, device="cuda")
    t = ctx.submit(r["Lf"], r["Lh"], r["grid"], r["f"], r["h"], r["pairs"], g, prec=0)
    assert ctx.drain(60000) == 0
    assert ctx.poll(t) == 0
    assert ctx.poll(t) == -7                   # forgotten after its final status
    with pytest.raises(pkg.SlshtError):        # host output is not allowed for requests
        ctx.submit(r["Lf"], r["Lh"], r["grid"], r["f"], r["h"], r["pairs"], g.cpu().numpy(), prec=0)
    with pytest.raises(pkg.SlshtError):
        ctx.submit(r["Lf"], r["Lh"], r["grid"], r["f"], r["h"], np.array([[99, 0]], np.int32), g, prec=0)
