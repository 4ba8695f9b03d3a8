"""Several optimisation iterations (dgr_step) against the FP64 oracle stepped
the same number of times, element by element on theta, m and v.

The step's last link -- the chain from (mu, s, q, rho) gradients to the
optimiser variables ((mu - c)/half, log s, raw q, softplus^-1 rho), the Adam
moments, the bias corrections at t > 1 and the exponential learning-rate decay
(Sec. 5.1: Adam, lr 3e-4 -> 3e-5) -- is checked here:
  * m and v carry the gradients in optimiser variables (m = sum of
    (1 - b1) b1^k g, v likewise with g^2), so a wrong chain factor (half, s,
    sigmoid(theta_rho)) changes them by that factor;
  * every step t draws its own measured projections, so the gradients change
    from step to step and Adam's move m_hat / (sqrt(v_hat) + eps) is not
    saturated at +-lr: theta then depends on the bias corrections and on
    lr(t), which decays from lr0 to lr1 over the n_iters = T steps run here.
The measurement of step t is the oracle's own prediction at step t plus
+-U[0.02, 0.06] per ray, so no L1 residual sits near its kink (the GPU and
the oracle take every sign decision the same way).

Tolerances: loss 1e-5 relative; m and v per kind relative L2 <= 2e-4 (the
gradients' FP32-vs-FP64 bound, doubled for v ~ g^2) and max-abs <= 1e-3 of
the kind's largest entry; theta per element |dtheta_gpu - dtheta_oracle| <=
1e-2 lr0 where the gradient is not negligible (sqrt(v) >= 1e-3 of the kind's
largest: below that Adam's ratio divides FP32 noise by ~eps).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2411_04844_b300 import dgr, synth
from tests._common import (_near_integer, guard_field, margin_measurement, oracle_geom,
                           oracle_grid, rel_l2)

pytestmark = pytest.mark.gpu
DEV = "cuda"
T_STEPS = 6
LR0, LR1 = 1e-4, 1e-5
KINDS = (("mu", 3), ("s", 3), ("q", 4), ("rho", 1))


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def H(t):
    return t.detach().cpu().numpy().astype(np.float64)


def split(flat, n):
    out, o = {}, 0
    for k, w in KINDS:
        out[k] = flat[o:o + w * n].reshape((n, w) if w > 1 else (n,))
        o += w * n
    return out


def _problem(which):
    if which == "cone":
        gs = synth.GridSpec((32, 32, 32), 1.0, (-16.0, -16.0, -16.0))
        geo = synth.cone_geom(10, 48, 40, 1.5, 1.5, 120.0, 180.0)
    else:
        gs = synth.GridSpec((32, 32, 32), 1.0, (-16.0, -16.0, -16.0))
        geo = synth.parallel_geom(12, 40, 32, 1.0, 1.0)
    # a wide guard band: the moves of T_STEPS steps stay far from every
    # footprint-integer edge (checked again at each step)
    f = guard_field(synth.gaussian_field(synth.rng_for(1, 31), 300, gs, ("loguniform", 0.5, 3.0)),
                    gs, band=0.03)
    f.rho = np.clip(f.rho, 0.05, 1.0).astype(np.float32)
    return gs, geo, f


@pytest.mark.parametrize("which,weights", [("parallel3d", (1.0, 0.0, 0.0)),
                                           ("parallel3d", dgr.PAPER_WEIGHTS),
                                           ("cone", (1.0, 0.0, 0.0))])
def test_several_steps_match_oracle_theta_m_v(which, weights):
    gs, geo, f = _problem(which)
    og, oo = oracle_grid(gs), oracle_geom(geo)
    grid = dgr.Grid.of(gs)
    ang = T(geo.angles)
    gg = dgr.Geom.of(geo, ang)
    prob = dgr.make_problem(grid, gg, 3.0, LR0, LR1, T_STEPS, weights=weights)
    mu, s, q, rho = T(f.mu), T(f.s), T(f.q), T(f.rho)
    ws0 = dgr.Workspace(dgr.make_plan(grid, f.n))
    pairs, items = dgr.dgr_voxelize_count(grid, mu, s, q, 3.0, ws0)
    ws0.close()
    ws = dgr.Workspace(dgr.make_plan(grid, f.n, pairs * 2 + 64, items * 2 + 64, gg, step=True))
    st = dgr.State(mu, s, q, rho)
    dgr.dgr_params_init(prob, st)
    loss = torch.zeros(1, device=DEV)

    th = O.to_opt(og, f.mu.astype(np.float64), f.s.astype(np.float64), f.q.astype(np.float64),
                  f.rho.astype(np.float64))
    th0 = {k: a.copy() for k, a in th.items()}
    m = {k: np.zeros_like(a) for k, a in th.items()}
    v = {k: np.zeros_like(a) for k, a in th.items()}
    rng = np.random.default_rng(4242)
    for t in range(1, T_STEPS + 1):
        meas, (mu32, s32, q32, rho32) = margin_measurement(og, oo, th, rng)
        # the oracle's FP32 parameters decide the box integers: keep them off the edges
        assert not _near_integer(synth.Field(mu32, s32, q32, rho32), gs, 3.0, 1e-4).any()
        lo, th, _ = O.step(og, oo, mu32, s32, q32, rho32, th, m, v, t, meas, 3.0, LR0, LR1,
                           T_STEPS, weights=weights)
        dgr.dgr_step(prob, st, T(meas), loss, ws)
        torch.cuda.synchronize()
        assert dgr.dgr_status(ws) == 0
        assert abs(float(loss) - lo) <= 1e-5 * abs(lo), (t, float(loss), lo)
    assert int(H(st.step)[0]) == T_STEPS

    n = f.n
    tg, mg, vg = split(H(st.theta), n), split(H(st.m), n), split(H(st.v), n)
    for k, _ in KINDS:
        for name, a_g, a_o, tol in (("m", mg[k], m[k], 2e-4), ("v", vg[k], v[k], 2e-4)):
            assert rel_l2(a_g, a_o) <= tol, (k, name, rel_l2(a_g, a_o))
            assert np.max(np.abs(a_g - a_o)) <= 1e-3 * np.max(np.abs(a_o)), (k, name)
        live = np.sqrt(v[k]) >= 1e-3 * np.max(np.sqrt(v[k]))
        d = np.abs((tg[k] - th0[k]) - (th[k] - th0[k]))
        assert np.all(d[live] <= 1e-2 * LR0), (k, float(d[live].max()))
        # the moves are not saturated at +-lr: Adam's ratio varies between entries
        mv = np.abs(th[k] - th0[k])[live] / sum(O.lr_at(t, LR0, LR1, T_STEPS)
                                                for t in range(1, T_STEPS + 1))
        assert np.std(mv) > 0.05, (k, float(np.std(mv)))
