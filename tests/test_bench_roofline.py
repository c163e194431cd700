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


def test_tensor_path_takes_the_largest_pipe_time():
    # d = 16, m = 4: FP32 (9 flop) outweighs MUFU (1 ex2) and the MMAs
    r = bench.product_roofline("tensor", wl(0, 16, 4), 3.39, 50, 2070.0)
    times = {k: v["ideal_ms"] for k, v in r["pipes"].items()}
    assert r["pipe"] == max(times, key=times.get) == "fp32"
    assert r["frac"] == pytest.approx(times["fp32"] / 3.39)
    assert r["pipes"]["tensor"]["per_entry"] == 96
    # d = 32, m = 1: two coordinate blocks of MMAs now dominate
    r = bench.product_roofline("tensor", wl(0, 32, 1), 3.0, 50, 2070.0)
    assert r["pipe"] == "tensor" and r["bound"] == "tensor"
    assert r["pipes"]["tensor"]["per_entry"] == 192
    # Matern: two MUFU operations per entry
    r = bench.product_roofline("tensor", wl(2, 8, 1), 3.0, 50, 2070.0)
    assert r["pipes"]["mufu"]["per_entry"] == 2


def test_laplace_has_no_tensor_path():
    r = bench.product_roofline("tensor", wl(1, 16, 4), 5.0, 50, 2070.0)
    assert r["kernel"].startswith("kmv32_kernel") and "tensor" not in r["pipes"]
