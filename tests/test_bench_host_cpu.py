"""Host logic of bench.py that its reported rooflines rest on: the algorithmic
byte counts (checked against counts made independently by enumerating the
kept modes), the pair and step totals, and the lookup of measured DRAM traffic."""
import numpy as np
import pytest

import bench


def _kept_counts(n):
    k = np.where(2 * np.arange(n) < n, np.arange(n), np.arange(n) - n)
    keep_xy = 3 * np.abs(k) < n
    keep_z = 3 * np.arange(n // 2 + 1) < n
    A = int(keep_xy.sum()) ** 2 * int(keep_z.sum())
    Bx = n * int(keep_xy.sum()) * int(keep_z.sum())
    By = n * n * int(keep_z.sum())
    return A, Bx, By


@pytest.mark.parametrize("n", [8, 12, 24, 64, 96, 512, 768, 1024])
def test_kept_mode_counts(n):
    A, Bx, By, M = bench.ns_counts(n)
    assert (A, Bx, By) == _kept_counts(n)
    assert M == n * n * (n // 2 + 1)


def test_pair_bytes_are_eight_r_plus_eighty_m():
    for n in (256, 512, 1024, 2048):
        R, M = n**3, n * n * (n // 2 + 1)
        assert sum(bench.fft_pass_bytes(n).values()) == 8 * R + 80 * M
    assert sum(bench.fft_pass_bytes(1024).values()) == 51_623_493_632


def test_ns_step_bytes_at_512():
    kb = bench.ns_kernel_bytes(512)
    assert kb["ns_z_product"] == 3_227_516_928  # 9 fields x 512^2 x 171 x 8 B
    assert kb["ns_invy"] == 8 * 6 * (512 * 341 * 171 + 512 * 512 * 171)
    pruned, unpruned = bench.ns_step_bytes(512)
    assert pruned == 2 * sum(kb.values())
    assert pruned == pytest.approx(24.85e9, rel=1e-3)
    assert unpruned == 93 * 8 * 512 * 512 * 257


def test_unfused_bytes_grow_with_the_grid():
    b384, b768 = bench.ns_rhs_bytes_unfused(384), bench.ns_rhs_bytes_unfused(768)
    assert 7.5 < b768 / b384 < 8.5
    assert bench.ns_rhs_bytes_unfused(768) == pytest.approx(135.7e9, rel=1e-3)  # per right-hand side


def test_measured_traffic_lookup():
    assert bench.measured_traffic("no_such_kernel", "ns512") is None
    h = bench.source_hash("ns")
    assert h == bench.source_hash("ns") and len(h) == 12
    got = bench.measured_traffic("ns_z_product", "ns512")
    # a record exists; when it matches the sources it is within 10 % of the algorithmic bytes
    if got is not None:
        assert abs(got / bench.ns_kernel_bytes(512)["ns_z_product"] - 1) < 0.1
