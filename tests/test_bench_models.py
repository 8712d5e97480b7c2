"""The bench's per-sample work models against the values the design notes
quote, and the split-DFT factor rule of the CUDA-core alpha stage (the same
rule as alpha_split_factor in csrc/alpha.cu: the odd P in {9, 7, 5, 3}
dividing N_alpha with the smallest 4K/P + P + 3 below the direct sum's
4(L_h - 1) + 2)."""
import pytest

bench = pytest.importorskip("bench")


@pytest.mark.parametrize("Lh,Na,P", [
    (16, 511, 7),      # workload 3: 511 = 7 x 73
    (64, 4095, 9),     # workload 5: 4095 = 3^2 5 7 13
    (64, 127, 0),      # prime: the direct sum
    (32, 63, 9),       # serving, L_h = 32 native grid
    (8, 15, 5),
    (16, 31, 0),
    (4, 7, 0),         # 4K/P + P + 3 = 14 > 4(L_h - 1) + 2 = 14: no gain, direct
])
def test_split_factor_rule(Lh, Na, P):
    assert bench.alpha_split_factor_py(Lh, Na) == P


def test_fp64_alpha_cost_workload3():
    """(4K + 4H^2 + 10H)/P FP64 instructions a sample: 27.1 (50 flop) at L_h = 16, P = 7."""
    P, instr, flops, _ = bench.alpha_fp64_cost(16, 511)
    assert P == 7
    assert instr == pytest.approx((4 * 31 + 4 * 9 + 30) / 7)
    assert flops == pytest.approx(50.0)


def test_double_float_issue_model_workload3():
    """About 385 FP32/INT instructions a sample for the double-float engine on workload 3."""
    ops, form = bench.alpha_dd_ops(16, 511, 7)
    assert 380 < ops < 390 and "P = 7" in form
