"""slsht_forward_noalloc: the forward transform for callers that cannot
allocate device memory when they need it (real-time sections where
cudaMalloc's implicit synchronisation is not allowed, plug-ins whose host
owns the device allocator, processes that gave the whole device to a fixed
pool).  It works in one static device array instead of allocating.

Each case runs the entry point twice in a row, so the second call runs over
what the first left in the shared array, and checks both results against
slsht_forward (which allocates its own scratch) and against the FP64 oracle,
at the tolerances of every parity test here (relative L2 1e-12 for FP64,
1e-5 for FP32_BULK).  The cases include pair lists longer than one chunk of
the array (so the chunk loop runs several times), and inputs held in device
memory, with the pair list written on a side stream just before the call.
An oversized request must be refused before anything runs.  This file is
collected last on purpose."""
import numpy as np
import pytest

import synth
from oracle import slsht as O

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}
SCRATCH = 32 << 20          # SLSHT_NOALLOC_SCRATCH_BYTES


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


def _pairs_per_chunk(Lf, Lh, grid, prec, n_pairs):
    """Pairs per chunk of the array for host inputs, by the entry point's
    carving: the staged inputs and the tables first, then per pair its
    couplings and its X scratch."""
    up = lambda n: (n + 255) // 256 * 256  # noqa: E731
    Na, Nb, Ng = grid
    K, el = 2 * Lh - 1, (8 if prec == 0 else 4)
    nd = sum((2 * p + 1) ** 2 for p in range(Lh))
    fixed = up(16 * Lf * Lf) + up(16 * Lh * Lh) + up(8 * n_pairs)
    fixed += up(8 * nd) + up(el * nd * Nb) + up(2 * el * Ng * K) + up(2 * el * Na * Lh)
    per_pair = up(16 * Lh * Lh) + up(2 * el * K * Nb * Ng)
    return (SCRATCH - fixed) // per_pair


CASES = [
    # (L_f, L_h, grid, f, h, pairs): one chunk, then one that needs several
    ("one_chunk", 16, 4, (31, 16, 7), synth.signal_cn_real(16, 41), synth.window_cn(4, 42), synth.pairs_all(19)),
    ("chunked", 40, 16, (127, 64, 31), synth.signal_powerlaw(40, 45), synth.window_cn(16, 46, decay=1.0),
     synth.pairs_random(55, 100, 47)),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_forward_and_oracle_twice(env, prec, case):
    import torch
    pkg, ctx = env
    _, Lf, Lh, grid, f, h, pairs = case
    if case[0] == "chunked":
        assert _pairs_per_chunk(Lf, Lh, grid, prec, len(pairs)) < len(pairs)   # the chunk loop runs again
    ref = ctx.forward(Lf, Lh, grid, f, h, pairs, prec=prec).cpu().numpy()
    orc = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    dt = torch.complex128 if prec == 0 else torch.complex64
    for _ in range(2):
        g = torch.full((len(pairs),) + grid, float("nan"), dtype=dt, device="cuda")
        pkg.slsht_forward_noalloc(pkg.make_desc(Lf, Lh, grid, prec), f, h, pairs, len(pairs), g)
        torch.cuda.synchronize()
        out = g.cpu().numpy()
        assert _rel(out, ref) < TOL[prec], (Lf, Lh, prec)
        assert _rel(out, orc) < TOL[prec], (Lf, Lh, prec)


def test_noalloc_device_inputs_written_on_a_side_stream(env):
    """f, h and the pair list in device memory; the pair list is written on a
    non-blocking stream that the call's stream waits on, so the entry point
    must read it in stream order (a read on another stream could see the old
    contents: here a list of valid but different pairs)."""
    import torch
    pkg, ctx = env
    Lf, Lh, grid, prec = 24, 8, (47, 24, 15), 0
    f, h = synth.signal_powerlaw(Lf, 51), synth.window_cn(Lh, 52, decay=1.0)
    pairs = synth.pairs_random(Lf + Lh - 1, 40, 53)
    stale = np.zeros_like(pairs)
    stale[:, 0] = 1
    fd, hd = torch.from_numpy(f).cuda(), torch.from_numpy(h).cuda()
    lmd = torch.from_numpy(stale).cuda()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    main = torch.cuda.current_stream()
    src = torch.from_numpy(pairs).pin_memory()
    g = torch.full((len(pairs),) + grid, float("nan"), dtype=torch.complex128, device="cuda")
    with torch.cuda.stream(side):
        torch.cuda._sleep(20_000_000)                 # keep the side stream busy before the copy lands
        lmd.copy_(src, non_blocking=True)
    main.wait_stream(side)
    pkg.slsht_forward_noalloc(pkg.make_desc(Lf, Lh, grid, prec), fd, hd, lmd, len(pairs), g, main)
    torch.cuda.synchronize()
    orc = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    assert _rel(g.cpu().numpy(), orc) < TOL[prec]


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
