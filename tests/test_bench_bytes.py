"""The algorithmic byte and flop counts behind bench.py's roofline, checked
against a hand count for the benchmark workload (12^4 lattice, nb 48,
81-point stencil, 32 right-hand sides), and the preconditioner launch's count
against the value the benchmark reports."""
import bench
from synth import WORKLOADS

W = WORKLOADS["L12_nb48_81pt_r32"]
V = 12 ** 4
R = 32


def test_operator_bytes_by_hand():
    coef_fp16 = 81 * V * 48 * 48 * 4          # two fp16 codes per complex coefficient
    scales = 8 * V                            # float site scale + float diagonal
    vectors = 2 * V * 48 * R * 8              # complex64 input and output, once each
    assert bench.op_bytes(W, R, "fp16") == coef_fp16 + scales + vectors == 15_989_114_880
    assert bench.op_bytes(W, R, "fp64") == 81 * V * 48 * 48 * 16 + 2 * V * 48 * R * 16
    # TC32: hi and lo fp16 codes, 8 bytes per complex coefficient
    assert bench.op_bytes(W, R, "tc32") - bench.op_bytes(W, R, "fp16") == coef_fp16
    # the digit image: 8 fp16 digits of Re and Im, a double scale and diagonal
    assert bench.op_bytes(W, R, "oz") == 81 * V * 48 * 48 * 32 + 16 * V + 2 * V * 48 * R * 16


def test_operator_flops():
    assert bench.op_flops(W, R) == 8 * 48 * 48 * R * 81 * V == 990_677_827_584


def test_chebyshev_launch_bytes():
    """Degree 8 in the FP16X epilogue: the first step reads the input and writes
    T and P (3 passes), each of the other seven also reads T_prev and P
    (5 passes); averaged over the 8 launches, plus the coefficients once."""
    vec = V * 48 * R * 8
    coef = 81 * V * 48 * 48 * 4 + 8 * V
    expect = coef + (3 + 5 * 7) * vec / 8
    got = bench.cheb_launch_bytes(W, R, "fp16x", 8)
    assert got == expect
    assert int(got) == 16_689_825_792       # the benchmark line's algorithmic_bytes
