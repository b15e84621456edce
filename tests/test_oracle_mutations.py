"""Planted mistakes in the oracle (CPU only): each plausible error must fail at least one pin.

Each case monkeypatches one oracle function with a subtly wrong variant and runs the pin tests
that should catch it, expecting an assertion failure. This shows the pins are not vacuous.
"""

import numpy as np
import pytest

import oracle.convert
import oracle.mpo
import oracle.rng
import oracle.rounding
from tests import test_oracle_basics as tb
from tests import test_oracle_convert as tc
from tests import test_oracle_rng as tr
from tests import test_oracle_rounding as tro
from tests import test_oracle_tnrsvd as tt


def _fails(fn, *args):
    with pytest.raises((AssertionError, ValueError, IndexError)):
        fn(*args)


def test_transposed_operand_in_contract(monkeypatch):
    orig = oracle.mpo.contract

    def bad(A, X, trans=False):
        return orig(A, X, trans=not trans) if A[0].shape[1] == A[0].shape[2] else orig(oracle.mpo.transpose(A), X, trans)

    monkeypatch.setattr(oracle.mpo, "contract", bad)
    _fails(tb.test_contract_equals_dense_product, False)


def test_bond_order_swapped_in_contract(monkeypatch):
    def bad(A, X, trans=False):
        out = []
        for a, x in zip(A, X):
            R, Ia, Ja, R2 = a.shape
            S, Ix, Kx, S2 = x.shape
            y = np.einsum("rijt,sjku->rsikut", a, x).reshape(S * R, Ia, Kx, S2 * R2)  # (r,s) -> s + S r
            out.append(y)
        return out

    monkeypatch.setattr(oracle.mpo, "contract", bad)
    _fails(tb.test_contract_equals_dense_product, False)


def test_dropped_r_absorption(monkeypatch):
    def bad(cores):
        cores = [c.copy() for c in cores]
        for k in range(len(cores) - 1):
            t, I, Kx, t2 = cores[k].shape
            Q, _ = np.linalg.qr(cores[k].reshape(t * I * Kx, t2, order="F"))
            cores[k] = Q.reshape(t, I, Kx, Q.shape[1], order="F")  # R never absorbed
        return cores

    monkeypatch.setattr(oracle.rounding, "_lr_orthogonalize", bad)
    _fails(tro.test_orthogonalize_no_truncation, 0)


def test_wrong_sign_in_site1(monkeypatch):
    orig = oracle.rounding._site1_core

    def bad(M, I1, R2):
        M = M.copy()
        M[0] = -M[0]
        return orig(M, I1, R2)

    monkeypatch.setattr(oracle.rounding, "_site1_core", bad)
    _fails(tro.test_orthogonalize_no_truncation, 0)


def test_omega_kappa_fastest(monkeypatch):
    def bad(seed, J, K):
        g = oracle.rng.normals(seed, 0, J[0] * K + sum(J[1:]))
        cores = [g[: J[0] * K].reshape(J[0], K)[None, :, :, None].copy()]  # kappa fastest
        pos = J[0] * K
        for j in J[1:]:
            cores.append(g[pos:pos + j].reshape(1, j, 1, 1).copy())
            pos += j
        return cores

    monkeypatch.setattr(oracle.rng, "omega", bad)
    _fails(tr.test_omega_lemma_5_1_rank_and_layout)


def test_digits_reversed(monkeypatch):
    orig = oracle.convert.convert

    def bad(*a, **k):
        R, X, digits = orig(*a, **k)
        return R, X, digits[:, ::-1].copy()

    monkeypatch.setattr(oracle.convert, "convert", bad)
    _fails(tc.test_random_sparse_exact_and_lemmas, 0)


def test_keep_rank_off_by_one(monkeypatch):
    orig = oracle.rounding.keep_rank
    monkeypatch.setattr(oracle.rounding, "keep_rank", lambda s, d, m: min(len(s), orig(s, d, m) + 1))
    _fails(tro.test_keep_rank_closed_form)


def test_mpo_svd_w_transposed(monkeypatch):
    orig = oracle.rounding.mpo_svd

    def bad(Z, tol=0.0, max_rank=0):
        W, S, V = orig(Z, tol, max_rank)
        return W.T, S, V

    monkeypatch.setattr(oracle.rounding, "mpo_svd", bad)
    _fails(tro.test_mpo_svd_matches_lapack)


def test_no_power_iteration_transpose(monkeypatch):
    """Using A instead of A^T in the power iteration breaks the dense cross-check (rectangular
    products would not even conform; here the square case gives the wrong subspace)."""
    orig = oracle.mpo.contract
    monkeypatch.setattr(oracle.mpo, "contract", lambda A, X, trans=False: orig(A, X, False))
    _fails(tt.test_dense_rsvd_cross_check, 1)


def _patched_rl_truncate(delta_of):
    """_rl_truncate with a planted mistake in its threshold: delta_of(cores, tol, d) -> delta."""

    def bad(cores, tol, max_rank):
        d = len(cores)
        delta = delta_of(cores, tol, d)
        for k in range(d - 1, 0, -1):
            t, I, Kx, t2 = cores[k].shape
            U, s, Vt = np.linalg.svd(cores[k].reshape(t, I * Kx * t2, order="F"), full_matrices=False)
            r = oracle.rounding.keep_rank(s, delta, max_rank)
            cores[k] = Vt[:r].reshape(r, I, Kx, t2, order="F")
            cores[k - 1] = np.einsum("aijb,bc->aijc", cores[k - 1], U[:, :r] * s[:r])
        return cores

    return bad


def _threshold_pins():
    for tol in (0.02, 0.05, 0.1, 0.2):
        tro.test_round_mpo_threshold_exact_ranks(tol)
        tro.test_orthogonalize_threshold_exact_ranks(tol)


def test_threshold_without_sqrt_d_minus_1(monkeypatch):
    monkeypatch.setattr(oracle.rounding, "_rl_truncate",
                        _patched_rl_truncate(lambda c, tol, d: tol * np.linalg.norm(c[-1])))
    _fails(_threshold_pins)


def test_threshold_from_squared_norm(monkeypatch):
    monkeypatch.setattr(oracle.rounding, "_rl_truncate",
                        _patched_rl_truncate(lambda c, tol, d: tol * np.linalg.norm(c[-1]) ** 2 / np.sqrt(d - 1)))
    _fails(_threshold_pins)


def test_threshold_from_the_wrong_core(monkeypatch):
    monkeypatch.setattr(oracle.rounding, "_rl_truncate",
                        _patched_rl_truncate(lambda c, tol, d: tol * np.linalg.norm(c[0]) / np.sqrt(d - 1)))
    _fails(_threshold_pins)


def test_threshold_pins_pass_with_the_correct_rule(monkeypatch):
    """The patched sweep with the oracle's own rule passes the same pins (the harness is sound)."""
    monkeypatch.setattr(oracle.rounding, "_rl_truncate",
                        _patched_rl_truncate(lambda c, tol, d: tol * np.linalg.norm(c[-1]) / np.sqrt(d - 1)))
    _threshold_pins()


# ---- planted mistakes in the zip-up rounding of a product ----
from tests import test_oracle_zipup as tz  # noqa: E402


def _patched_zipup(carry, delta_of):
    """zipup_product with a planted mistake: carry(U, s, r) -> C, delta_of(s, tol, d) -> delta."""

    def bad(A, X, trans=False, tol=0.0, max_rank=0):
        d = len(A)
        cores = [None] * d
        C = np.ones((1, 1))
        for k in range(d - 1, -1, -1):
            Yk = oracle.mpo.contract([A[k]], [X[k]], trans)[0]
            T = np.einsum("axcb,bt->axct", Yk, C)
            if k == 0:
                cores[0] = T
                break
            rs, n, kx, t = T.shape
            U, s, Vt = np.linalg.svd(T.reshape(rs, n * kx * t, order="F"), full_matrices=False)
            r = oracle.rounding.keep_rank(s, delta_of(s, tol, d), max_rank)
            cores[k] = Vt[:r].reshape(r, n, kx, t, order="F")
            C = carry(U, s, r)
        return cores

    return bad


_GOOD_CARRY = lambda U, s, r: U[:, :r] * s[:r]  # noqa: E731
_GOOD_DELTA = lambda s, tol, d: tol * np.linalg.norm(s) / np.sqrt(d - 1)  # noqa: E731


def _zipup_pins():
    tz.test_zipup_without_truncation_is_the_product(False)
    tz.test_zipup_without_truncation_is_the_product(True)
    for tol in (0.02, 0.05, 0.1, 0.2):
        tz.test_zipup_exact_ranks_on_left_canonical_input(tol, 0)


def test_zipup_carries_u_without_s(monkeypatch):
    monkeypatch.setattr(oracle.rounding, "zipup_product", _patched_zipup(lambda U, s, r: U[:, :r], _GOOD_DELTA))
    _fails(_zipup_pins)


def test_zipup_threshold_without_sqrt_d_minus_1(monkeypatch):
    monkeypatch.setattr(oracle.rounding, "zipup_product",
                        _patched_zipup(_GOOD_CARRY, lambda s, tol, d: tol * np.linalg.norm(s)))
    _fails(_zipup_pins)


def test_zipup_threshold_from_squared_norm(monkeypatch):
    monkeypatch.setattr(oracle.rounding, "zipup_product",
                        _patched_zipup(_GOOD_CARRY, lambda s, tol, d: tol * np.sum(s ** 2) / np.sqrt(d - 1)))
    _fails(_zipup_pins)


def test_zipup_carry_scaled_in_reverse_order(monkeypatch):
    """The carried factor scaled by the singular values in the wrong order: fails on the product."""
    monkeypatch.setattr(oracle.rounding, "zipup_product",
                        _patched_zipup(lambda U, s, r: U[:, :r] * s[:r][::-1], _GOOD_DELTA))
    _fails(_zipup_pins)


def test_zipup_pins_pass_with_the_correct_steps(monkeypatch):
    monkeypatch.setattr(oracle.rounding, "zipup_product", _patched_zipup(_GOOD_CARRY, _GOOD_DELTA))
    _zipup_pins()
