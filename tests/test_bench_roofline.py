"""The bench's roofline of the float32 product (host arithmetic only): the
roofline time is the largest ideal pipe time and frac = that time / the
measured launch time."""
import types

import pytest

import bench


def wl(kernel, d, m, N=100_000):
    return types.SimpleNamespace(kernel=kernel, N=N, d=d, m=m)


def test_fma_path_is_the_fp32_pipe():
    r = bench.product_roofline("fma", wl(0, 16, 4), 7.48, 50, 2070.0)
    assert r["pipe"] == "fp32" and r["bound"] == "alu"
    flop = (2 * 16 + 1 + 2 * 4) * 1e10
    assert r["achieved"] == pytest.approx(flop / 7.48e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert "tensor" not in r["pipes"]


def test_tcgen05_path_takes_the_largest_pipe_time():
    # d = 16, m = 4: 4 MMAs (L.H, H.L, H.H, c) = 128 tensor flop, 2m = 8 FP32
    # flop (c_i + c_j folded into the MMAs) and 1 ex2: FP32 and MUFU tie at
    # 1/32 clock per entry per SM, above the tensor time
    r = bench.product_roofline("tensor", wl(0, 16, 4), 2.25, 3, 2070.0)
    times = {k: v["ideal_ms"] for k, v in r["pipes"].items()}
    assert r["pipe"] == max(times, key=times.get)
    assert r["pipe"] in ("fp32", "mufu")
    assert times["fp32"] == pytest.approx(times["mufu"], rel=2e-3)
    assert r["frac"] == pytest.approx(times[r["pipe"]] / 2.25)
    assert r["pipes"]["tensor"]["per_entry"] == 128
    assert r["pipes"]["fp32"]["per_entry"] == 8
    # the c-part rides in a spare block position when d mod 16 is 1..10
    assert bench.tc5_mmas(8) == 3 and bench.tc5_mmas(12) == 4 and bench.tc5_mmas(20) == 6
    # d = 32, m = 1: two coordinate blocks and a c block of MMAs dominate
    r = bench.product_roofline("tensor", wl(0, 32, 1), 3.0, 3, 2070.0)
    assert r["pipe"] == "tensor" and r["bound"] == "tensor"
    assert r["pipes"]["tensor"]["per_entry"] == 2 * 16 * 7
    # Matern: two MUFU operations per entry
    r = bench.product_roofline("tensor", wl(2, 8, 1), 3.0, 3, 2070.0)
    assert r["pipes"]["mufu"]["per_entry"] == 2


def test_mma_sync_path_uses_its_own_tensor_peak():
    # d = 16, m = 4: 96 flop per entry at the measured mma.sync f16 rate
    # (1.58 ms) outweighs the FP32 pipe (1 + 2m = 9 flop, 1.12 ms)
    r = bench.product_roofline("mma_sync", wl(0, 16, 4), 3.39, 50, 2070.0)
    assert r["pipe"] == "tensor" and r["bound"] == "tensor"
    assert r["peak"] == bench.MMA_SYNC_F16_TFLOPS
    assert r["pipes"]["tensor"]["per_entry"] == 96
    assert r["pipes"]["fp32"]["per_entry"] == 9
    assert r["frac"] == pytest.approx(96e10 / 606e12 * 1e3 / 3.39)


def test_laplace_has_no_tensor_path():
    r = bench.product_roofline("tensor", wl(1, 16, 4), 5.0, 50, 2070.0)
    assert r["kernel"].startswith("kmv32_kernel") and "tensor" not in r["pipes"]


def test_traffic_reported_for_captured_tiles_only():
    # the ncu DRAM bytes of the tcgen05 product at the headline shape were
    # captured for the two epilogue variants the autotuner picks there; any
    # other tile or shape reports None
    w = wl(0, 16, 4)
    for tile in (1, 3):
        r = bench.product_roofline("tensor", w, 2.31, tile, 2070.0)
        assert r["traffic"] is not None and 20e6 < r["traffic"] < 25e6
    assert bench.product_roofline("tensor", w, 2.31, 2, 2070.0)["traffic"] is None
    assert bench.product_roofline("tensor", wl(0, 16, 4, N=50_000), 0.6, 3, 2070.0)["traffic"] is None
