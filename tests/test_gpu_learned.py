"""GPU parity of the learned collision operator against the FP64 oracle
through the C ABI: the local Knudsen sensor, the 64-mode Hermite projection,
the application of given network outputs (conservative correction, entropy
check, hard-sphere fallback), the training pairs, and exact special cases
(a zero network leaves f unchanged; a zero threshold is the hard-sphere
update bit for bit)."""
import numpy as np
import pytest

import oracle as O
import paper_1503_00707_gb300 as D
import workloads as W
from tests.gpu_util import bf16_round, pair, random_params, rel_linf, same_start

pytestmark = pytest.mark.gpu

TRIALS, SEED = 64, 20150303


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1503_00707_gb300 import _build
    _build.build()


def _cfg():
    # the bimodal periodic box on a small tree: seeded per-cell states give
    # strong gradients, so the sensor splits the cells
    c = dict(W.CONFIGS["c4_hs_bimodal"])
    c.update(base_level=2, max_level=3, coll=D.COLL_LEARNED)
    return c


def _setup(threshold=None):
    c = _cfg()
    s, o = pair(c, collision=D.COLL_LEARNED)
    s.set_collision_tables(TRIALS, SEED)
    o.hs_tables(TRIALS, SEED)
    same_start(s, o, o.get_f(), "f32")  # both sides start from the same FP32 values
    knl = np.sort(o.kn_local(c["kn"]))
    # half way between the two middle values: no cell's local Kn lies within
    # rounding of the threshold, so both sides split the cells alike
    thr = float(0.5 * (knl[len(knl) // 2 - 1] + knl[len(knl) // 2])) if threshold is None else threshold
    s.learned_configure(thr)
    return c, s, o, thr


def _psi_moments(q, xi, dV):
    ps = np.stack([np.ones(len(xi)), xi[:, 0], xi[:, 1], xi[:, 2], (xi * xi).sum(1)], 1)
    return q @ ps * dV, np.abs(q) @ np.abs(ps) * dV


def test_sensor_and_projection_match_oracle():
    c, s, o, thr = _setup()
    nc = s.ncells
    r = s.learned_collide(1e-5, o=np.zeros((nc, 64), np.float32), want=("knl", "a"))
    knl_o = o.kn_local(c["kn"])
    assert rel_linf(r["knl"], knl_o) < 1e-9
    assert 0 < (knl_o < thr).sum() < nc
    a_o, _ = o.hermite_project()
    assert np.max(np.abs(r["a"] - a_o)) < 2e-5 * np.max(np.abs(a_o))
    assert np.allclose(r["a"][:, 0], 1.0, atol=1e-5)   # sum f dV / rho
    assert np.max(np.abs(r["a"][:, [16, 4, 1]])) < 1e-4  # first moments about u vanish


def test_zero_network_leaves_f_unchanged():
    c, s, o, thr = _setup(threshold=1e30)
    nc = s.ncells
    f0 = s.get_f()
    r = s.learned_collide(1e-5, o=np.zeros((nc, 64), np.float32), want=("used",))
    # o = 0: the reconstructed term is zero, the correction solves A d = 0,
    # the entropy production is 0 <= 0, and every cell keeps f
    assert r["used"].all()
    assert np.array_equal(s.get_f(), f0)


def test_zero_threshold_is_the_hard_sphere_update():
    c, s, o, thr = _setup(threshold=0.0)
    s.set_weights(random_params(1))
    h = D.solver_from_config(c, D.F32, D.COLL_HS)
    h.set_f(s.get_f())
    h.set_collision_tables(TRIALS, SEED)
    dt = 2.5e-5
    s.step(2, dt)
    h.step(2, dt)
    assert s.learned_fallback_count() == s.ncells
    assert np.array_equal(s.get_f(), h.get_f())


def test_apply_given_outputs_matches_oracle():
    c, s, o, thr = _setup()
    nc, nv = s.ncells, s.nv
    a_o, _ = o.hermite_project()
    # a relaxation-like term: o = -k (a - e_0), which pulls the resolved
    # modes of f towards the Maxwellian's
    e0 = np.zeros(64)
    e0[0] = 1.0
    oin = (-2.0 * (a_o - e0)).astype(np.float32)
    dt = 2.5e-5
    r = s.learned_collide(dt, o=oin, want=("used", "q"))
    used_o, q_o = o.learned_apply(dt, c["kn"], o.kn_local(c["kn"]), oin.astype(np.float64), thr, want_q=True)
    assert np.array_equal(r["used"], used_o)
    assert 0 < used_o.sum() < nc
    lm = used_o.astype(bool)
    scale = np.max(np.abs(q_o[lm]))
    assert np.max(np.abs(r["q"][lm] - q_o[lm])) < 1e-4 * scale
    assert np.all(r["q"][~lm] == 0)
    assert rel_linf(s.get_f(), o.get_f()) < 2e-5
    # the applied term carries no mass, momentum or energy (FP32 per node)
    xi, dV = o.xi.reshape(-1, 3), o.dV
    mom, absm = _psi_moments(r["q"][lm].astype(np.float64), xi, dV)
    assert np.all(np.abs(mom) <= 1e-5 * absm + 1e-30)


def test_network_outputs_match_oracle_network():
    c, s, o, thr = _setup()
    params = random_params(5)
    s.set_weights(params)
    r = s.learned_collide(1e-5, want=("o", "used"))
    # the oracle network on the oracle's Hermite coefficients rounded to BF16,
    # as the tensor cores see them (the weights are BF16-exact)
    a_o, _ = o.hermite_project()
    y = O.mlp_forward(params.astype(np.float64), bf16_round(a_o).astype(np.float64))
    assert np.max(np.abs(r["o"] - y)) < 2e-2 * np.max(np.abs(y))


def test_training_pairs_match_oracle():
    c, s, o, thr = _setup()
    a, t = s.learned_pairs()
    a_o, mom = o.hermite_project()
    f_keep = o.get_f()
    I, _, _ = o.hs_collide(0.0, 1.0, want=True)
    o.set_f(f_keep)  # hs_collide with dt = 0 keeps f; restore exactly anyway
    t_o = o.hermite_target(I, mom)
    assert np.max(np.abs(a - a_o)) < 2e-5 * np.max(np.abs(a_o))
    assert np.max(np.abs(t - t_o)) < 1e-3 * np.max(np.abs(t_o))
    # the target has no mass, momentum or energy modes: o_0 = 0 (mass),
    # o for H_1 along each axis (momentum), and the trace of the H_2 modes
    assert np.max(np.abs(t[:, [0, 16, 4, 1]])) < 1e-3 * np.max(np.abs(t_o))


def test_learned_step_matches_oracle_split():
    c, s, o, thr = _setup()
    params = random_params(9, gain=0.3, bias=0.0)
    s.set_weights(params)
    dt = 2.5e-5
    s.step(1, dt)
    # the oracle: transport (Eq. 2), then the learned update with the same
    # network in FP64
    o.step(1, dt, O.COLL_NONE, c["kn"])
    o.learned_collide(dt, c["kn"], params.astype(np.float64), thr)
    rs, us, Ts = s.moments()
    ro, uo, To = o.moments()
    assert rel_linf(rs, ro) < 1e-5 and rel_linf(us, uo) < 1e-5 and rel_linf(Ts, To) < 1e-5
    assert rel_linf(s.get_f(), o.get_f()) < 2e-3
