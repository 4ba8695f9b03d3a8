"""Pins of the network oracle (oracle/net.py) against library routines,
adjoint identities and finite differences."""
import numpy as np
import pytest

from oracle import net as N


def test_conv3_single_channel_is_scipy_correlate():
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((7, 7, 7))
    w = rng.standard_normal((27, 1, 1))
    K = np.zeros((3, 3, 3))
    for t, (dx, dy, dz) in enumerate(N.taps()):
        K[dz + 1, dy + 1, dx + 1] = w[t, 0, 0]
    ref = nd.correlate(x, K, mode="constant", cval=0.0)
    assert np.max(np.abs(N.conv3(x[..., None], w)[..., 0] - ref)) < 1e-12


def test_conv_pool_up_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((6, 6, 6, 3)); w = rng.standard_normal((27, 3, 4))
    g = rng.standard_normal((6, 6, 6, 4))
    lhs = (N.conv3(x, w) * g).sum()
    assert abs(lhs - (x * N.conv3_dgrad(g, w)).sum()) < 1e-10
    assert abs(lhs - (w * N.conv3_wgrad(x, g)).sum()) < 1e-10
    y = rng.standard_normal((3, 3, 3, 3))
    assert abs((N.pool(x) * y).sum() - (x * N.pool_T(y)).sum()) < 1e-12
    z = rng.standard_normal((12, 12, 12, 3))
    assert abs((N.up(x) * z).sum() - (x * N.up_T(z)).sum()) < 1e-10


def test_network_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    P = rng.standard_normal(N.n_params()) * 0.3
    x = rng.uniform(0, 1, (4, 4, 4))
    gy = rng.standard_normal((4, 4, 4, 2))
    g = N.backward(P, x, gy, bf=False)
    L = lambda p: (N.forward(p, x, bf=False)[0] * gy).sum()
    idx = np.concatenate([rng.choice(N.n_params(), 40, replace=False), [0, 432, N.n_params() - 1]])
    for i in idx:
        e = 1e-6
        p1 = P.copy(); p1[i] += e
        p2 = P.copy(); p2[i] -= e
        fd = (L(p1) - L(p2)) / (2 * e)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding_ties_to_even():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.140625], np.float32)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert list(N.bf16(vals)) == [1.0, 1.0, 1.0 + 2 ** -6, -2.5, 3.140625]


def test_ramlak_kernel_sums_to_zero_and_is_linear():
    """The Ram-Lak kernel has zero DC gain: a long constant row filters to ~0
    away from its ends (the truncated kernel tail decays as 1/k)."""
    nu = 4001
    sino = np.ones((1, 1, nu))
    out = N.ramlak_filter(sino, 1.0, 0)
    assert abs(out[0, 0, nu // 2]) < 1e-4
    rng = np.random.default_rng(3)
    a = rng.standard_normal((2, 3, 17)); b = rng.standard_normal((2, 3, 17))
    fa = N.ramlak_filter(a, 0.7, 1, dsd=50.0, pv=1.2)
    fb = N.ramlak_filter(b, 0.7, 1, dsd=50.0, pv=1.2)
    assert np.max(np.abs(N.ramlak_filter(2 * a - b, 0.7, 1, dsd=50.0, pv=1.2) - (2 * fa - fb))) < 1e-12
