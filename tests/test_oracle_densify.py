"""Pins of the densification oracle (paper App. F, Algorithm 2): invariants
the algorithm states (intensity kept by cloning, volume kept by splitting, the
n_max cap, top-k by mean gradient, the pruning rule), the rotation of the
split samples against a rotation built from cos/sin, and a hand-worked case."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import densify as D


def _grid():
    return O.Grid((40, 40, 40), 1.0, (-20.0, -20.0, -20.0))


def _state(n=300, seed=0):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-15, 15, (n, 3))
    s = np.exp(rng.uniform(np.log(0.05), np.log(2.0), (n, 3)))
    q = rng.standard_normal((n, 4))
    rho = rng.uniform(0.05, 1, n)
    acc = rng.exponential(2e-2, n)  # accumulated over 100 iterations: mean ~2e-4
    z = rng.standard_normal((n, 2, 3))
    return mu, s, q, rho, acc, z


def test_hand_worked_case():
    """theta = 0.005 * 40 sqrt(3) = 0.3464; tau = 2e-4; 100 iterations.
    g0: avg 5e-4, sigma 0.1  -> clone (rho halves, a copy follows)
    g1: avg 1e-4, sigma 0.1  -> pruned (avg <= tau)
    g2: avg 9e-4, sigma 0.9  -> split (two children at the end)
    g3: avg 3e-4, sigma 60   -> pruned (sigma > 3 x 17 x h)... but first a split
        candidate: it is large and above tau, so it splits (split wins)
    g4: avg 7e-4, sigma 0.2  -> clone"""
    g = _grid()
    mu = np.array([[0, 0, 0], [1, 1, 1], [2, 2, 2], [3, 3, 3], [4, 4, 4]], float)
    s = np.array([[0.1] * 3, [0.1] * 3, [0.9, 0.5, 0.5], [60.0, 1, 1], [0.2] * 3])
    q = np.tile([1.0, 0, 0, 0], (5, 1))
    rho = np.array([0.8, 0.5, 0.6, 0.7, 0.4])
    acc = np.array([5e-2, 1e-2, 9e-2, 3e-2, 7e-2])
    z = np.zeros((5, 2, 3)); z[2, 0] = [1, 0, 0]; z[2, 1] = [0, -1, 0]; z[3, 0] = [0, 0, 1]
    mu2, s2, q2, rho2, kind, src = D.densify(g, mu, s, q, rho, acc, 100, z)
    assert list(src) == [0, 4, 0, 4, 2, 2, 3, 3]
    assert list(kind) == [0, 0, 1, 1, 2, 2, 2, 2]
    assert np.allclose(rho2, [0.4, 0.2, 0.4, 0.2, 0.6, 0.6, 0.7, 0.7])
    c = 2 ** (-1 / 3)
    assert np.allclose(mu2[4], [2.9, 2, 2]) and np.allclose(mu2[5], [2, 1.5, 2])
    assert np.allclose(mu2[6], [3, 3, 4]) and np.allclose(s2[4], np.array([0.9, 0.5, 0.5]) * c)


def test_clone_keeps_intensity_split_keeps_volume_and_cap():
    g = _grid()
    mu, s, q, rho, acc, z = _state()
    n_max = 330
    mu2, s2, q2, rho2, kind, src = D.densify(g, mu, s, q, rho, acc, 100, z, n_max=n_max)
    assert mu2.shape[0] <= n_max
    for i in np.unique(src[kind == 1]):  # a cloned original and its clone share its intensity
        assert abs(rho2[(src == i) & (kind < 2)].sum() - rho[i]) < 1e-14
    for i in np.unique(src[kind == 2]):
        ch = (src == i) & (kind == 2)
        assert ch.sum() == 2
        assert abs(2 * np.prod(s2[ch][0]) - np.prod(s[i])) < 1e-12 * np.prod(s[i])
        assert np.allclose(rho2[ch], rho[i]) and np.allclose(q2[ch], q[i])


def test_selection_is_top_k_by_mean_gradient():
    g = _grid()
    mu, s, q, rho, acc, z = _state(seed=1)
    avg = acc / 100
    theta = 0.005 * 40 * math.sqrt(3)
    sig = s.max(1)
    n = mu.shape[0]
    n_max = n + 7  # room for 7 clones and no split
    _, _, _, _, kind, src = D.densify(g, mu, s, q, rho, acc, 100, z, n_max=n_max)
    cand = np.flatnonzero((avg >= 2e-4) & (sig <= theta))
    best = sorted(cand, key=lambda i: (-avg[i], i))[:7]
    assert sorted(src[kind == 1]) == sorted(best)
    assert (kind == 2).sum() == 0


def test_pruning_rule_on_survivors():
    g = _grid()
    mu, s, q, rho, acc, z = _state(seed=2)
    s[:10] *= 40  # some beyond 3 x 17 voxels
    avg = acc / 100
    _, _, _, _, kind, src = D.densify(g, mu, s, q, rho, acc, 100, z)
    surv = src[kind == 0]
    assert np.all(avg[surv] > 2e-4)
    assert np.all(s[surv].max(1) <= 3 * 17 * 1.0)


def test_split_samples_use_the_gaussian_rotation():
    """q = (cos a/2, 0, 0, sin a/2) is a rotation by a about z: the child of
    z = (1, 0, 0) sits at mu + s_x (cos a, sin a, 0)."""
    g = _grid()
    a = 0.7
    mu = np.array([[1.0, -2.0, 0.5]]); s = np.array([[3.0, 1.0, 1.0]])
    q = np.array([[math.cos(a / 2), 0, 0, math.sin(a / 2)]]); rho = np.array([0.5])
    z = np.array([[[1.0, 0, 0], [0, 0, 2.0]]])
    mu2, _, _, _, kind, _ = D.densify(g, mu, s, q, rho, np.array([1.0]), 100, z)
    assert list(kind) == [2, 2]
    assert np.allclose(mu2[0], mu[0] + 3.0 * np.array([math.cos(a), math.sin(a), 0]))
    assert np.allclose(mu2[1], mu[0] + np.array([0, 0, 2.0]))
