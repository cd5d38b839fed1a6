"""The benchmark's sampled-error reference (bench.sampled_reference, plain
numpy) against the FP64 oracle on every op pair and both layouts, with
padded leading dimensions and non-commuting scalars: it must give the
oracle's entries to rounding."""
import numpy as np
import pytest

import bench
import qsynth
from oracle import oracle as orc

OPS = ("N", "T", "C", "H")


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("opA", OPS)
@pytest.mark.parametrize("opB", OPS)
def test_sampled_reference_matches_oracle(opA, opB, layout):
    m, n, k = 23, 17, 31
    seed = 300 + 4 * OPS.index(opA) + OPS.index(opB)
    ra, ca = qsynth.stored_shape(opA, m, k)
    rb, cb = qsynth.stored_shape(opB, k, n)
    A = qsynth.normal(ra, ca, seed, layout, ld=ra + 3)
    B = qsynth.normal(rb, cb, seed + 1, layout, ld=rb + 2)
    C = qsynth.normal(m, n, seed + 2, layout, ld=m + 1)
    alpha, beta = np.array([0.5, -1.0, 2.0, 0.25]), np.array([-1.0, 0.5, 0.0, 1.5])
    g = np.random.default_rng(seed)
    rows, cols = g.integers(0, m, 40), g.integers(0, n, 40)
    ref = orc.qgemm_entries(opA, opB, m, n, k, alpha, A, B, beta, C, rows, cols, layout=layout)
    got = bench.sampled_reference(opA, opB, m, n, k, alpha, A, B, beta, C, rows, cols, layout)
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_sampled_reference_small_integers_exact_and_beta_zero():
    m, n, k = 9, 11, 50
    A = qsynth.small_int(m, k, 41)
    B = qsynth.small_int(k, n, 42)
    C = qsynth.empty(m, n)            # NaN: not read when beta = 0
    rows, cols = np.arange(m).repeat(n), np.tile(np.arange(n), m)
    ref = orc.qgemm_entries("N", "N", m, n, k, np.array([1.0, 2.0, -1.0, 0.0]), A, B,
                            np.zeros(4), qsynth.empty(m, n, pad=0.0), rows, cols)
    got = bench.sampled_reference("N", "N", m, n, k, np.array([1.0, 2.0, -1.0, 0.0]), A, B,
                                  np.zeros(4), C, rows, cols)
    assert np.array_equal(got, ref)
