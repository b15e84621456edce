"""Pins for the oracle's random MPO (Lemma 5.1) and its SplitMix64 / Box-Muller stream."""

import numpy as np
import pytest

from oracle import mpo, rng
from tests.conftest import golden_path


def test_splitmix64_published_values():
    want = [int(l.strip(), 16) for l in open(golden_path("splitmix64.txt")) if l.strip() and not l.startswith("#")]
    got = [int(x) for x in rng.splitmix64(0, 0, len(want))]
    assert got == want
    # Counter-based: output n does not depend on where the slice starts.
    np.testing.assert_array_equal(rng.splitmix64(7, 5, 3), rng.splitmix64(7, 0, 8)[5:])


def test_uniform_range_and_normal_distribution():
    u = rng.uniforms(1, 0, 200000)
    assert u.min() > 0.0 and u.max() <= 1.0
    g = rng.normals(1, 0, 200000)
    stats = pytest.importorskip("scipy.stats")
    assert stats.kstest(g, "norm").pvalue > 1e-4
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1) < 0.02


def test_omega_lemma_5_1_rank_and_layout():
    J, K = [8, 2, 3], 6
    O = rng.omega(5, J, K)
    assert [c.shape for c in O] == [(1, 8, 6, 1), (1, 2, 1, 1), (1, 3, 1, 1)]
    D = mpo.dense(O)
    assert D.shape == (48, 6)
    assert np.linalg.matrix_rank(D) == K  # Lemma 5.1: rank(Omega) = K
    # Kronecker structure (proof of Lemma 5.1): Omega = w3 (x) w2 (x) Omega1
    ref = np.kron(O[2][0, :, :, 0], np.kron(O[1][0, :, :, 0], O[0][0, :, :, 0]))
    np.testing.assert_allclose(D, ref, atol=1e-15)
    # draw order: Omega1 column-major first, then the site vectors
    g = rng.normals(5, 0, 8 * 6 + 5)
    np.testing.assert_array_equal(O[0][0, :, :, 0].reshape(-1, order="F"), g[:48])
    np.testing.assert_array_equal(O[1].reshape(-1), g[48:50])
    with pytest.raises(ValueError):
        rng.omega(0, [4, 4], 5)  # K > J_1
