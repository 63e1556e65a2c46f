"""Pins for the oracle's local Knudsen number, Hermite projections, MLP and
learned collision update.

Pinned against: exact gradients of linear fields on refined trees (centred
differences of area-weighted neighbour means are exact for linear data),
orthonormality of the Hermite modes under the Maxwellian weight (a Maxwellian
projects onto mode 0; a Maxwellian times 1 + eps H_m onto eps at mode m),
reconstruction of known mode coefficients, torch autograd (FP64) for the MLP
forward and backward, finite differences for the gradient, and exact
conservation of the corrected learned collision term.
"""
import math

import numpy as np
import pytest

import oracle as O


def _fine_problem(spec):
    return O.Problem(spec, (24, 24, 24), (-9.0,) * 3, (9.0,) * 3)


def _kn_case(spec, rho_of, T_of, uz_of, kn=0.05):
    p = _fine_problem(spec)
    xyz, h = p.centres()
    nc = p.ncells
    rho, T = rho_of(xyz), T_of(xyz)
    u = np.zeros((nc, 3))
    u[:, 2] = uz_of(xyz)
    p.init_maxwellian(np.ones(nc), rho, u, T)
    return p.kn_local(kn), rho, T


def test_kn_local_linear_fields_exact_on_uniform_tree():
    """rho linear in x, T in y, u_z in z: every gradient is exact, including
    the one-sided differences at the outflow sides."""
    spec = O.make_spec(3, 3, 3, O.PRED_NONE, bc=(2,) * 6)
    got, rho, T = _kn_case(spec, lambda x: 1 + 0.5 * x[:, 0], lambda x: 1 + 0.3 * x[:, 1],
                           lambda x: 0.2 * x[:, 2])
    grads = np.stack([0.5 / rho, 0.3 / T, 0.2 / np.sqrt(T)], axis=1)
    assert np.allclose(got, 0.05 / rho * grads.max(axis=1), rtol=1e-9, atol=0)


def test_kn_local_linear_field_exact_across_hanging_faces():
    """Linear fields are differentiated exactly on a refined tree too: the
    least-squares fit uses the true neighbour offsets, coarse or fine."""
    spec = O.make_spec(3, 2, 4, O.PRED_BALL, (0.4, 0.6, 0.5), 0.15, bc=(2,) * 6)
    got, rho, T = _kn_case(spec, lambda x: 1 + 0.5 * x[:, 0] + 0.1 * x[:, 1],
                           lambda x: 1 + 0.3 * x[:, 1] - 0.2 * x[:, 2], lambda x: 0.2 * x[:, 2])
    gr = np.hypot(0.5, 0.1) / rho
    gT = np.hypot(0.3, 0.2) / T
    gu = 0.2 / np.sqrt(T)
    assert np.allclose(got, 0.05 / rho * np.maximum(np.maximum(gr, gT), gu), rtol=1e-9, atol=0)


def test_hermite_projection_of_maxwellian_and_modes():
    spec = O.make_spec(3, 1, 1, O.PRED_NONE)
    p = O.Problem(spec, (32, 32, 32), (-10.0,) * 3, (10.0,) * 3)
    nc = p.ncells
    rho, u, T = 1.4, np.array([0.3, -0.2, 0.5]), 0.8
    p.init_maxwellian(np.ones(nc), np.full(nc, rho), np.tile(u, (nc, 1)), np.full(nc, T))
    a, mom = p.hermite_project()
    e0 = np.zeros(64)
    e0[0] = 1.0
    assert np.max(np.abs(a - e0)) < 1e-10
    assert np.allclose(mom[:, 0], rho) and np.allclose(mom[:, 4], T)
    # M (1 + eps H_m) for modes that leave rho, u, T unchanged
    f = p.get_f()[0]
    g = (p.xi - u) / math.sqrt(T)

    def h(k, x):
        return [np.ones_like(x), x, (x * x - 1) / math.sqrt(2), (x ** 3 - 3 * x) / math.sqrt(6)][k]
    for m in (16 * 3, 16 + 4, 16 * 2 + 4, 4 * 1 + 3, 16 * 3 + 4 * 3 + 3, 16 * 2 + 4 * 2 + 2):
        Hm = h(m >> 4, g[:, 0]) * h((m >> 2) & 3, g[:, 1]) * h(m & 3, g[:, 2])
        eps = 0.01
        p.set_f(np.tile(f * (1 + eps * Hm), (nc, 1)))
        a, mom = p.hermite_project()
        want = e0.copy()
        want[m] += eps
        assert np.max(np.abs(a[0] - want)) < 1e-9, m


def test_hermite_target_recovers_coefficients():
    spec = O.make_spec(3, 1, 1, O.PRED_NONE)
    p = O.Problem(spec, (32, 32, 32), (-10.0,) * 3, (10.0,) * 3)
    nc = p.ncells
    rho, u, T = 1.2, np.array([0.1, 0.2, -0.3]), 1.1
    p.init_maxwellian(np.ones(nc), np.full(nc, rho), np.tile(u, (nc, 1)), np.full(nc, T))
    M = p.get_f()[0]
    g = (p.xi - u) / math.sqrt(T)

    def h(k, x):
        return [np.ones_like(x), x, (x * x - 1) / math.sqrt(2), (x ** 3 - 3 * x) / math.sqrt(6)][k]
    rng = np.random.default_rng(0)
    o = rng.normal(size=64)
    s = np.zeros(p.nv)
    for m in range(64):
        s += o[m] * h(m >> 4, g[:, 0]) * h((m >> 2) & 3, g[:, 1]) * h(m & 3, g[:, 2])
    I = rho * math.sqrt(T) * M * s
    mom = np.tile([rho, u[0], u[1], u[2], T], (nc, 1))
    got = p.hermite_target(np.tile(I, (nc, 1)), mom)
    assert np.max(np.abs(got[0] - o)) < 1e-9


def _params(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    out = []
    for (r, c), nb in O.MLP_SHAPES:
        out.append(rng.normal(0, scale / math.sqrt(c) * 3, size=(r, c)).ravel())
        out.append(rng.normal(0, 0.1, size=nb))
    p = np.concatenate(out)
    assert p.size == O.MLP_NPARAM
    return p


def test_mlp_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    params = _params(1)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(7, 64))
    t = rng.normal(size=(7, 64))
    y = O.mlp_forward(params, x)
    g, loss = O.mlp_backward(params, x, t)
    # the same network with torch's Linear/SiLU in FP64
    P = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    off = 0
    h = torch.tensor(x, dtype=torch.float64)
    for li, ((r, c), nb) in enumerate(O.MLP_SHAPES):
        W = P[off:off + r * c].view(r, c)
        off += r * c
        b = P[off:off + nb]
        off += nb
        h = torch.nn.functional.linear(h, W, b)
        if li < 3:
            h = torch.nn.functional.silu(h)
    L = torch.mean((h - torch.tensor(t)) ** 2)
    L.backward()
    assert np.allclose(y, h.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert abs(loss - L.item()) < 1e-12 * max(1.0, abs(L.item()))
    assert np.allclose(g, P.grad.numpy(), rtol=1e-9, atol=1e-13)


def test_mlp_gradient_finite_differences():
    params = _params(3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(3, 64))
    t = rng.normal(size=(3, 64))
    g, _ = O.mlp_backward(params, x, t)
    idx = rng.choice(O.MLP_NPARAM, 25, replace=False)
    for k in idx:
        e = 1e-6
        pp = params.copy()
        pp[k] += e
        lp = np.mean((O.mlp_forward(pp, x) - t) ** 2)
        pp[k] -= 2 * e
        lm = np.mean((O.mlp_forward(pp, x) - t) ** 2)
        fd = (lp - lm) / (2 * e)
        assert abs(fd - g[k]) < 1e-6 * max(1.0, abs(g[k])) + 1e-9


def _bimodal_problem():
    spec = O.make_spec(3, 1, 2, O.PRED_BALL, (0.3, 0.3, 0.3), 0.2)
    p = O.Problem(spec, (12, 12, 12), (-6.0,) * 3, (6.0,) * 3)
    nc = p.ncells
    rng = np.random.default_rng(5)
    u = np.zeros((nc, 2, 3))
    u[:, 0, 0] = rng.uniform(1, 2, nc)
    u[:, 1, 0] = -rng.uniform(1, 2, nc)
    p.init_maxwellian(np.tile([0.45, 0.55], (nc, 1)), np.ones((nc, 2)), u, np.full((nc, 2), 0.6))
    return p


def test_learned_collide_conserves_and_falls_back():
    p = _bimodal_problem()
    p.hs_tables(64, 11)
    f0 = p.get_f()
    params = _params(6, scale=0.05)
    used, q = p.learned_collide(1e-5, 0.02, params, threshold=1e9, want_q=True)
    if used.sum() == 0:
        # a random network's term is linear in its output: flipping the last
        # layer flips the sign of the entropy production
        n_last = 64 * 256 + 64
        params[-n_last:] *= -1
        p.set_f(f0)
        used, q = p.learned_collide(1e-5, 0.02, params, threshold=1e9, want_q=True)
    assert used.sum() > 0
    ps = np.stack([np.ones(p.nv), p.xi[:, 0], p.xi[:, 1], p.xi[:, 2], (p.xi ** 2).sum(1)], 1)
    for c in np.nonzero(used)[0]:
        num = np.abs(q[c] @ ps)
        den = (np.abs(q[c])[:, None] * np.abs(ps)).sum(0)
        assert np.max(num / den) < 1e-12
    # threshold 0: every cell takes the plain hard-sphere term
    p.set_f(f0)
    used0, q0 = p.learned_collide(1e-5, 0.02, params, threshold=0.0, want_q=True)
    assert used0.sum() == 0
    p.set_f(f0)
    qhs, _, _ = p.hs_collide(1e-5, 0.02, want=True)
    assert np.max(np.abs(q0 - qhs)) <= 1e-12 * np.max(np.abs(qhs))


def test_learned_collide_zero_network_is_identity():
    p = _bimodal_problem()
    f0 = p.get_f()
    params = np.zeros(O.MLP_NPARAM)
    used, q = p.learned_collide(1e-3, 0.02, params, threshold=1e9, want_q=True)
    assert used.all()
    assert np.max(np.abs(q)) < 1e-12 * np.max(f0)
