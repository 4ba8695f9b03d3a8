"""Adaptive density control on the GPU (paper App. F, Algorithm 2) against the
oracle: the same Gaussians survive, are cloned and are split, in the same
order (integer decisions, bit-exact), with the same parameters (FP32 within
1e-6 relative); the optimiser state of survivors is carried over, new entries
start from zero moments.  Then a short optimisation run with densification
every 20 iterations keeps a finite, decreasing loss."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import densify as D
from paper_2411_04844_b300 import dgr, synth
from tests._common import oracle_geom, oracle_grid

pytestmark = pytest.mark.gpu
DEV = "cuda"


def T(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def H(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("n,n_max", [(3000, 500_000), (3000, 3400), (5000, 5000)])
def test_densify_matches_oracle(n, n_max):
    gs = synth.GridSpec((64, 64, 64), 1.0, (-32.0, -32.0, -32.0))
    grid = dgr.Grid.of(gs)
    rng = np.random.default_rng(n + n_max)
    mu = rng.uniform(-28, 28, (n, 3)).astype(np.float32)
    s = np.exp(rng.uniform(np.log(0.05), np.log(1.5), (n, 3))).astype(np.float32)
    s[:40] *= 60  # beyond 3 x 17 voxels
    q = rng.standard_normal((n, 4)).astype(np.float32)
    rho = rng.uniform(0.05, 1, n).astype(np.float32)
    acc = rng.exponential(2e-2, n).astype(np.float32)
    acc[100:120] = acc[99]  # ties of the mean gradient
    z = rng.standard_normal((n, 2, 3)).astype(np.float32)
    src = dgr.State(T(mu), T(s), T(q), T(rho), accumulate=True)
    src.grad_accum[:n] = T(acc)
    src.theta.copy_(torch.arange(11 * n, device=DEV, dtype=torch.float32))
    src.m.fill_(0.25); src.v.fill_(0.5); src.step.fill_(37)
    dst = dgr.State(T(mu[:1]), T(s[:1]), T(q[:1]), T(rho[:1]), accumulate=True, capacity=n_max)
    ws = dgr.Workspace(dgr.make_plan(grid, n))
    n_out = dgr.dgr_densify(grid, dgr.DensifyCfg.paper(n_max), 100, src, T(z), dst, ws)
    mu2, s2, q2, rho2, kind, srci = D.densify(oracle_grid(gs), mu, s, q, rho, acc, 100, z, n_max=n_max)
    assert n_out == mu2.shape[0] and n_out <= n_max
    gm, gsc, gq, gr = (H(t) for t in dst.view())
    assert np.allclose(gm, mu2, rtol=1e-6, atol=1e-5)
    assert np.allclose(gsc, s2, rtol=1e-6, atol=0)
    assert np.array_equal(gq, q2.astype(np.float32))
    assert np.allclose(gr, rho2, rtol=1e-7, atol=0)
    th = H(dst.theta)
    nk = int((kind == 0).sum())
    # survivors carry their moments; new entries start from zero
    mm = H(dst.m)[:11 * n_out]
    idx = lambda j, o: (3 * o + j if j < 3 else 3 * n_out + 3 * o + j - 3 if j < 6
                        else 6 * n_out + 4 * o + j - 6 if j < 10 else 10 * n_out + o)
    for o in [0, nk // 2, nk - 1] if nk else []:
        assert mm[idx(0, o)] == 0.25 and mm[idx(10, o)] == 0.25
        i = srci[o]
        assert th[idx(4, o)] == float(3 * n + 3 * i + 1)  # theta copied bit for bit
    for o in range(nk, n_out, max(1, (n_out - nk) // 7)):
        assert mm[idx(0, o)] == 0.0 and mm[idx(10, o)] == 0.0
    assert int(H(dst.step)[0]) == 37
    assert np.all(H(dst.grad_accum)[:n_out] == 0)


def test_training_with_densification():
    gs = synth.GridSpec((32, 32, 32), 1.0, (-16.0, -16.0, -16.0))
    geo = synth.cone_geom(24, 48, 48, 1.4, 1.4, 120.0, 180.0)
    grid = dgr.Grid.of(gs)
    ang = T(geo.angles)
    gg = dgr.Geom.of(geo, ang)
    phantom = synth.ellipsoid_phantom(synth.rng_for(1, 41), gs, 6)
    meas = T(O.project(oracle_grid(gs), oracle_geom(geo), phantom).astype(np.float32))
    f = synth.gaussian_field(synth.rng_for(1, 42), 400, gs, ("loguniform", 0.8, 2.5))
    f.rho = np.clip(f.rho * 0.2, 0.01, 1.0).astype(np.float32)
    n_max = 4000
    st = dgr.State(T(f.mu), T(f.s), T(f.q), T(f.rho), accumulate=True, capacity=n_max)
    prob = dgr.make_problem(grid, gg, 3.0, 3e-3, 3e-4, 200)
    dgr.dgr_params_init(prob, st)
    cfg = dgr.DensifyCfg(1e-5, 0.005, 17.0, n_max)
    rng = np.random.default_rng(43)
    losses, counts = [], [st.n]
    other = dgr.State(T(f.mu[:1]), T(f.s[:1]), T(f.q[:1]), T(f.rho[:1]), accumulate=True, capacity=n_max)
    loss = torch.zeros(1, device=DEV)
    for it in range(1, 201):
        if it % 20 == 1:
            ws0 = dgr.Workspace(dgr.make_plan(grid, st.n))
            mu, s, q, _ = st.view()
            pairs, items = dgr.dgr_voxelize_count(grid, mu, s, q, 3.0, ws0)
            ws0.close()
            ws = dgr.Workspace(dgr.make_plan(grid, st.n, 2 * pairs + 1024, 2 * items + 1024, gg, step=True))
        dgr.dgr_step(prob, st, meas, loss, ws)
        losses.append(float(loss))
        if it % 20 == 0 and it < 200:
            z = T(rng.standard_normal((st.n, 2, 3)))
            dws = dgr.Workspace(dgr.make_plan(grid, st.n))
            dgr.dgr_densify(grid, cfg, 20, st, z, other, dws)
            dws.close()
            st, other = other, st
            counts.append(st.n)
    torch.cuda.synchronize()
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.7 * losses[0], (losses[0], losses[-1])
    assert max(counts) > counts[0]  # the density control added Gaussians
