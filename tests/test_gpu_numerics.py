"""Device checks of the adaptive kernel's arithmetic building blocks, through the C ABI:
the table-driven sincos against CUDA's sincos, the exact split-precision tensor-core
contraction against a plain FP64 contraction of the same operands, and the two-float kernel
value and sincos of the mixed form against FP64 (lcq_selftest)."""
import pytest

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def test_sincos_table_and_tensor_contraction():
    import __graft_entry__ as g
    g.build()
    from paper_2006_02545_gb300 import lcq
    r = lcq.selftest(0)
    # sin and cos of magnitude <= 1: within 4 ulp(1) = 2^-50 of CUDA's (itself within 1 ulp):
    # table entries and the angle-addition step round, the Taylor tails are below 1.3e-20
    assert 0.0 <= r["sincos_abs_err"] <= 8 * U, r
    # the 8-slice split keeps 56 bits per operand on the row's (kernel) and the column's
    # bound (basis) power-of-two scales and keeps the slice products of diagonals i + j <= 8
    # (the dropped ones are below 2^-60 of the scales): against a double-double reference,
    # at the FP64 rounding level of sum |products| (12 decades of kernel magnitudes within one
    # row, up to 128 nodes)
    assert 0.0 <= r["tc_rel_err_d6"] <= 8 * U, r
    assert 0.0 <= r["tc_rel_err_d10"] <= 8 * U, r
    # two-float arithmetic carries 48 bits (2^-48 = 32 U per stored value); the kernel value
    # chains about 20 products and sums, each within a few 2^-48 relative (products) or of
    # the magnitudes summed (sums), so the difference from the FP64 value stays within
    # 2^-40 of the magnitude of its terms, at every distance (x - X is FP64)
    assert 0.0 <= r["ff_kernel_rel_err"] <= 2.0 ** -40, r
    # sin and cos: the argument's own two-float rounding (2^-48 |th|) plus the table and
    # angle-addition roundings
    assert 0.0 <= r["ff_sincos_err"] <= 2.0 ** -44, r
