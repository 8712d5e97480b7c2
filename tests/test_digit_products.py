"""Host checks of the arithmetic behind the FP64 alpha stage on the tensor
cores (csrc/alpha_tc64.cu), replayed operation by operation in FP32 with
numpy: X given as double-float pairs is scaled into [0.5, 1) and cut into
seven base-256 digits (power-of-two scaling, rounding to an integer, exact
subtraction, TwoSum renormalisation); cos/sin of q alpha likewise in FP64;
the digit products of each weight i + j <= 8 are summed as integers, and the
seven sums are combined by TwoSum as the epilogue does.  Pins: the digit
bounds (|d_1| <= 256, |d_i| <= 128), every partial sum below 2^24 (exact in
FP32 in any order), and the result against a 200-bit evaluation of
g = sum_q X_q e^{-i q alpha} (Sec. IV, the alpha sum of Eq. alternative_harmonic_formulation_wigner)
within 1e-14 relative L2."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    v = f32(s - a)
    return s, f32(f32(a - f32(s - v)) + f32(b - v))


def digits_dd(h, l):
    """Seven base-256 digits of h + l (|h + l| < 1), FP32 steps."""
    h, l, out = f32(h), f32(l), []
    for _ in range(7):
        h, l = f32(h * f32(256)), f32(l * f32(256))
        d = f32(np.rint(h))
        h = f32(h - d)
        h, l = two_sum(h, l)
        out.append(int(d))
    return out


def digits_d(v):
    out = []
    for _ in range(7):
        v *= 256.0
        d = float(np.rint(v))
        v -= d
        out.append(int(d))
    return out


def combine(a):
    """The epilogue: sum_w A_w 256^-(w-2) as a double-float (h, l)."""
    af = [f32(x) for x in a]
    tail = f32(af[3] * f32(2.0 ** -24) + f32(af[4] * f32(2.0 ** -32) + f32(af[5] * f32(2.0 ** -40)
                                                                         + f32(af[6] * f32(2.0 ** -48)))))
    s, e1 = two_sum(af[0], f32(af[1] * f32(2.0 ** -8)))
    s2, e2 = two_sum(s, f32(af[2] * f32(2.0 ** -16)))
    return two_sum(s2, f32(f32(e1 + e2) + tail))


@pytest.mark.parametrize("seed", [1, 2])
def test_digit_products_exact_and_accurate(seed):
    mp.mp.prec = 200
    rng = np.random.default_rng(seed)
    Na, K = 511, 31
    errs, refs, peak = [], [], 0
    for _ in range(6):
        X = (rng.standard_normal(K) + 1j * rng.standard_normal(K)) * np.exp(rng.uniform(-4, 4, K))
        xh = [X.real.astype(f32), X.imag.astype(f32)]
        xl = [(X.real - xh[0].astype(float)).astype(f32), (X.imag - xh[1].astype(float)).astype(f32)]
        exact = [[mp.mpf(float(xh[c][u])) + mp.mpf(float(xl[c][u])) for u in range(K)] for c in range(2)]
        ex = int(np.frexp(max(np.abs(xh[0]).max(), np.abs(xh[1]).max()))[1])
        down = f32(2.0 ** -ex)
        A = np.zeros((7, 64), dtype=np.int64)                 # slots: Re X_q at 15 + q, Im at 47 + q
        for u in range(K):
            A[:, u] = digits_dd(f32(xh[0][u] * down), f32(xl[0][u] * down))
            A[:, 32 + u] = digits_dd(f32(xh[1][u] * down), f32(xl[1][u] * down))
        assert np.abs(A[0]).max() <= 256 and np.abs(A[1:]).max() <= 128
        for a in rng.integers(0, Na, 4):
            for comp in (0, 1):                               # rows (cos | sin) and (-sin | cos)
                B = np.zeros((7, 64), dtype=np.int64)
                for u in range(K):
                    th = 2 * np.pi * (((u - 15) * int(a)) % Na) / Na
                    c, s = np.cos(th), np.sin(th)
                    B[:, u] = digits_d(c if comp == 0 else -s)
                    B[:, 32 + u] = digits_d(s if comp == 0 else c)
                acc = np.zeros(7, dtype=np.int64)
                for i in range(7):
                    for j in range(7 - i):
                        acc[i + j] += int(A[i] @ B[j])
                        peak = max(peak, int(np.abs(A[i]) @ np.abs(B[j])) * (i + j + 1))
                h, l = combine(acc)
                got = (mp.mpf(float(h)) + mp.mpf(float(l))) * mp.mpf(2) ** (ex - 16)
                ref = mp.mpf(0)
                for u in range(K):
                    th = 2 * mp.pi * (((u - 15) * int(a)) % Na) / Na
                    if comp == 0:
                        ref += exact[0][u] * mp.cos(th) + exact[1][u] * mp.sin(th)
                    else:
                        ref += exact[1][u] * mp.cos(th) - exact[0][u] * mp.sin(th)
                errs.append(float(got - ref))
                refs.append(float(ref))
    assert peak < 2 ** 24                                     # every partial sum exact in FP32
    assert np.linalg.norm(errs) / np.linalg.norm(refs) < 1e-14


def test_combine_exact_for_integer_sums():
    """A single non-zero weight combines exactly; cancellation between the
    two leading weights leaves an exact result."""
    for a in ([123456, 0, 0, 0, 0, 0, 0], [0, 0, 0, 0, 0, 0, 977], [1000, -256000, 17, 0, 0, 0, 0]):
        h, l = combine(a)
        exact = sum(mp.mpf(v) * mp.mpf(2) ** (-8 * w) for w, v in enumerate(a))
        assert mp.mpf(float(h)) + mp.mpf(float(l)) == exact
