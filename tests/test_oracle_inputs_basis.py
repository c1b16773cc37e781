"""Pins of the seeded generators and of the oracle's bases (CPU only)."""
import math
import os

import numpy as np
import pytest

import pf_inputs as pi
from oracle import basis

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vector():
    rows = [l.split() for l in open(os.path.join(GOLD, "splitmix64_seed0.txt")) if not l.startswith("#")]
    for idx, hexv in rows:
        assert int(pi.splitmix64(0, int(idx))) == int(hexv, 16)


def test_uniform_ranges_and_counter_form():
    u = pi.uniform01(7, np.arange(100000))
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    # counter form: element i does not depend on how many were drawn before it
    assert pi.uniform01(7, np.array([12345]))[0] == u[12345]
    n = pi.normals(3, 20000)
    assert abs(n.mean()) < 0.03 and abs(n.std() - 1.0) < 0.03


@pytest.mark.parametrize("L", [2, 4, 6, 8, 10, 12, 14, 16])
def test_xxz_dimension_and_order(L):
    st = basis.xxz_basis(L, L // 2)
    assert len(st) == math.comb(L, L // 2)
    assert np.all(np.diff(st) > 0)
    assert np.all(basis.popcount(st) == L // 2)


def test_sector_dimensions_of_the_workloads():
    assert len(basis.xxz_basis(12, 6)) == 924
    assert math.comb(20, 10) == 184756 and math.comb(22, 11) == 705432
    ups, dns = basis.hubbard_basis(12, 6, 6)
    assert len(ups) * len(dns) == 853776
    assert len(basis.qsun_basis(3, 15)) == 262144


def test_row_of_roundtrip():
    st = basis.xxz_basis(10, 5)
    idx = np.random.default_rng(0).permutation(len(st))
    assert np.array_equal(basis.row_of(st, st[idx]), idx)
