"""The benchmark's algorithmic work model (the numerators of its roofline fractions) on the 2^20-point
contract workload, against closed forms of the counts: the weights w_j = min(floor(log2(j+1)), 12)
of 1024 columns give tau_I = 2^I columns at levels I <= 9 and one column at level 10; the fine band
expands levels 0-3, whose tree costs sum_{I<4} tau_I 2^-I = 4 multiply-adds per output; every coarse
level I costs 2 n_I tau tau_I flops per shift and piece product (n_I = 2^(20-I) distinct rows, six
piece products in the split tier)."""
import numpy as np
import pytest

import bench
from paper_2305_11645_gb300 import inputs as I

M, TAU, R = 20, 1024, 16
OUTPUTS = (1 << M) * TAU * R


@pytest.fixture(scope="module")
def net20():
    return I.c3()


def tau_of(level):
    return 1 << level if level <= 9 else 1


def test_levels_of_the_workload(net20):
    jf, tau_I, chain = bench.band_of(net20)
    assert jf == 4
    assert [tau_I[l] for l in range(11)] == [tau_of(l) for l in range(11)]
    assert sum(tau_I) == TAU and chain == list(range(4, 11))


def test_fine_band_work(net20):
    # forward: 4 tree multiply-adds and the Gaussian norm's v*v + u per output; adjoint: the tree
    # twice (recomputation, gradient), h'(v) folded into the coefficient, its multiply and the fold
    assert bench.fine_work(net20, "k_fine_fwd_s4") == (OUTPUTS * 5.0, 0)
    assert bench.fine_work(net20, "k_fine_bwd_s4") == (OUTPUTS * 11.0, 0)


def test_coarse_tensor_work(net20):
    def flops(levels):
        return sum(2.0 * (1 << (M - l)) * TAU * tau_of(l) for l in levels) * R * 6
    assert bench.coarse_kernel_levels(net20, "k_level_tc") == list(range(4, 11))
    assert bench.coarse_kernel_levels(net20, "k_fold_grad_tc") == [4, 5, 6]
    assert bench.coarse_kernel_levels(net20, "k_grad_tc") == [7, 8, 9, 10]
    assert bench.coarse_kernel_levels(net20, "k_coarse_grad_tc") == []
    assert bench.coarse_mma_flops(net20, 3) == flops(range(4, 11))
    assert bench.coarse_mma_flops(net20, 3, [4, 5, 6]) == flops([4, 5, 6])
    # six levels of 2 * 2^20 * 1024 * 96 flops each, and level 10's single column
    assert np.isclose(flops(range(4, 11)), 6 * 2.0 * 2**20 * TAU * 16 * 6 + 2.0 * 2**10 * TAU * 16 * 6)
    assert bench.coarse_mma_flops(net20, 1) * 6 == bench.coarse_mma_flops(net20, 3)


def test_roofline_fractions(net20):
    # the dominant kernel at the measured 7.315 ms per step and a 2070 MHz clock: 11 FP32 operations
    # per output against 152 SMs x 128 lanes x clock; a tensor-core kernel against the sustained peak
    mp = {"bf16_tflops_sustained": 1684.4}
    r = bench.roofline_of(net20, "split", "k_fine_bwd_s4", 7.315, 1.0, 2070.0, mp, "measured", "net20")
    assert r["bound"] == "alu" and r["pipe"] == "fp32" and r["unit"] == "Gop/s"
    assert np.isclose(r["peak"], 152 * 128 * 2070e6 / 1e9)
    assert np.isclose(r["frac"], OUTPUTS * 11.0 / (7.315e-3 * 152 * 128 * 2070e6))
    assert np.isclose(r["achieved"] / r["peak"], r["frac"])
    assert r["traffic"] == bench.TRAFFIC_BYTES[("net20", "k_fine_bwd_s4")]
    t = bench.roofline_of(net20, "split", "k_grad_tc", 0.5, 1.0, 2070.0, mp, "measured", "net20")
    fl = sum(2.0 * (1 << (M - l)) * TAU * tau_of(l) for l in (7, 8, 9, 10)) * R * 6
    assert t["bound"] == "tensor" and np.isclose(t["frac"], fl / 0.5e-3 / 1e12 / 1684.4)
    # a kernel without counters of its current code reports no traffic
    f = bench.roofline_of(net20, "split", "k_fine_fwd_s4", 3.2, 1.0, 2070.0, mp, "measured", "net20")
    assert f["traffic"] is None
