"""Pins for the diagonal estimation rule (Prop. 1, Eq. diag-estimate, Lemma 1).

All checks are exact enumerations over every probe vector, so they hold to
rounding and do not depend on random draws."""
import itertools

import numpy as np
import pytest

from oracle.cofem import diag_estimate, diag_estimate_general


def _spd(D, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((D, D))
    return G @ G.T / D + np.diag(rng.uniform(0.5, 2.0, D))


def _all_signs(D):
    return np.array(list(itertools.product([-1.0, 1.0], repeat=D))).T   # D x 2^D


@pytest.mark.parametrize("D", [3, 8, 12])
def test_prop1_unbiased_by_enumeration(D):
    """Averaging s over all 2^D sign vectors (K = 2^D probes) gives diag(M) exactly."""
    M = _spd(D, D)
    P = _all_signs(D)
    s = diag_estimate(P, M @ P)
    np.testing.assert_allclose(s, np.diag(M), rtol=0, atol=1e-12)


def test_prop1_general_rule_non_rademacher():
    """Prop. 1 for zero-mean iid probes with values {-2,-1,1,2}: the K = 1
    estimator p_j (Mp)_j / p_j^2 averages to M_jj over all 4^D vectors."""
    D = 5
    M = _spd(D, 1)
    vals = [-2.0, -1.0, 1.0, 2.0]
    P = np.array(list(itertools.product(vals, repeat=D))).T
    X = M @ P
    s_each = P * X / (P * P)                      # K = 1 estimator per vector
    np.testing.assert_allclose(s_each.mean(axis=1), np.diag(M), atol=1e-12)
    # and the K-probe general rule, applied to the whole set at once, is exact too
    np.testing.assert_allclose(diag_estimate_general(P, X), np.diag(M), atol=1e-12)


@pytest.mark.parametrize("D", [4, 9])
def test_lemma1_variance_k1(D):
    """Lemma 1 with K = 1: Var[s_j] = sum_{j' != j} M_jj'^2, by enumeration."""
    M = _spd(D, 7 + D)
    P = _all_signs(D)
    X = M @ P
    s_each = np.stack([diag_estimate(P[:, i:i + 1], X[:, i:i + 1]) for i in range(P.shape[1])], axis=1)
    var = s_each.var(axis=1)
    off = (M ** 2).sum(axis=1) - np.diag(M) ** 2
    np.testing.assert_allclose(var, off, rtol=1e-12)


def test_lemma1_variance_k2():
    """Lemma 1 with K = 2 (all ordered pairs of sign vectors, D = 5):
    Var[s_j] = (1/2) sum_{j' != j} M_jj'^2."""
    D = 5
    M = _spd(D, 3)
    S = _all_signs(D)
    n = S.shape[1]
    vals = []
    for a in range(n):
        for b in range(n):
            P = S[:, [a, b]]
            vals.append(diag_estimate(P, M @ P))
    var = np.var(np.array(vals), axis=0)
    off = (M ** 2).sum(axis=1) - np.diag(M) ** 2
    np.testing.assert_allclose(var, off / 2.0, rtol=1e-12)


def _hadamard(n):
    H = np.array([[1.0]])
    while H.shape[0] < n:
        H = np.block([[H, H], [H, -H]])
    return H


@pytest.mark.parametrize("D", [16, 64])
def test_hadamard_probes_give_exact_diagonal(D):
    """With the D columns of a Sylvester-Hadamard matrix as probes,
    sum_k p_kj p_kj' = D delta_jj', so s = diag(M) exactly (Eq. diag-expansion)."""
    M = _spd(D, 11)
    H = _hadamard(D)
    np.testing.assert_allclose(diag_estimate(H, M @ H), np.diag(M), atol=1e-12)


def test_estimator_wrong_scale_would_fail():
    """Guard: the 1/K factor matters (dropping it multiplies s by K)."""
    D = 8
    M = _spd(D, 5)
    P = _all_signs(D)
    s = diag_estimate(P, M @ P)
    assert not np.allclose(s * P.shape[1], np.diag(M))
