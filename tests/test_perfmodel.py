"""The algorithmic counts behind the roofline figures: the residual's flops per element
on the 3-D p = 3 workload (the figure the benchmark divides by), the block solve's bytes,
and the matrix-based smoother's product and solve bytes."""
from paper_2202_09733_gb300 import perfmodel as PM


def test_residual_and_block_solve_counts():
    assert PM.residual_flops(3, 3) == 98720.0
    nd = 5 * 64
    assert PM.block_solve_bytes(3, 3, 4) == 4 * nd * nd + 4 * nd + 2 * 4 * nd
    assert PM.block_solve_flops(3, 3) == 2 * nd * nd


def test_assembled_operator_counts():
    """(2d + 1) blocks of nd^2 per element for the product; a solve with m steps costs at
    least m products and m + 1 block solves, and its vector traffic stays below half of that."""
    nd = 4 * 9                                         # 2-D p = 2
    assert PM.assembled_product_bytes(2, 2) == 8 * (5 * nd * nd + 5 * nd + nd)
    assert PM.assembled_product_flops(2, 2, neighbours=0) == PM.block_solve_flops(2, 2)
    m = 5
    low = m * PM.assembled_product_bytes(2, 2) + (m + 1) * PM.block_solve_bytes(2, 2)
    assert low < PM.mbnk_solve_bytes(2, 2, m) < 1.5 * low
