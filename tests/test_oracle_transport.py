"""Pins for the oracle's velocity grid, transport (Eq. 2) and moments.

Pinned against: the closed-form discrete Fourier amplification of first-order
upwind on a uniform periodic mesh, exact freestream preservation on refined
trees, conservation of every discrete velocity's mass under periodic sides,
mass/energy conservation at specular walls, the inflow ghost value, the
Gaussian closed form for the discrete moments on a fine velocity mesh, and
first-order convergence of free streaming to the exact translated solution
on uniform and refined trees.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _uniform(dim, lev, bc=(0,) * 6):
    return O.make_spec(dim, lev, lev, O.PRED_NONE, bc=bc)


def test_velocity_grid_order_and_values():
    n, lo, hi = (4, 6, 8), (-2.0, -3.0, -1.0), (2.0, 3.0, 3.0)
    xi, k, dV = O.vgrid(n, lo, hi)
    nv = 4 * 6 * 8
    assert xi.shape == (nv, 3)
    assert dV == pytest.approx(1.0 * 1.0 * 0.5, rel=0, abs=0)
    # every node once
    lin = (k[:, 0] * n[1] + k[:, 1]) * n[2] + k[:, 2]
    assert sorted(lin.tolist()) == list(range(nv))
    # node values: midpoints of the n cells of [lo, hi]
    for d in range(3):
        edges = np.linspace(lo[d], hi[d], n[d] + 1)
        mids = 0.5 * (edges[:-1] + edges[1:])
        assert np.allclose(xi[:, d], mids[k[:, d]], rtol=0, atol=1e-15)
    # sign groups are contiguous blocks, group o = 4[x>0]+2[y>0]+[z>0]
    blk = nv // 8
    # with lo/hi not symmetric in z the sign split is by index half, as for the
    # paper's symmetric meshes; check on a symmetric mesh:
    xs, ks, _ = O.vgrid((6, 4, 8), (-3, -2, -4), (3, 2, 4))
    blk = len(xs) // 8
    for o in range(8):
        sg = xs[o * blk:(o + 1) * blk] > 0
        assert np.all(sg[:, 0] == bool(o & 4)) and np.all(sg[:, 1] == bool(o & 2)) and np.all(sg[:, 2] == bool(o & 1))
        # inside a group: lexicographic in |xi| (x, y, z), z fastest
        mag = np.abs(xs[o * blk:(o + 1) * blk])
        keys = [tuple(r) for r in np.round(mag[:, [0, 1, 2]], 12)]
        assert keys == sorted(keys)
    # |xi| per position is the same in every group (mirror symmetry)
    m0 = np.abs(xs[:blk])
    for o in range(8):
        assert np.array_equal(np.abs(xs[o * blk:(o + 1) * blk]), m0)


def _fourier_case(dim, lev, n, vmax, wav, nsteps=7):
    spec = _uniform(dim, lev)
    p = O.Problem(spec, n, (-vmax,) * 3, (vmax,) * 3)
    xyz, h = p.centres()
    hh = 2.0 ** -lev
    kvec = 2 * np.pi * np.asarray(wav, dtype=float)
    phase = xyz[:, :dim] @ kvec[:dim]
    amp = 0.3 + 0.01 * np.arange(p.nv)  # a different amplitude per velocity
    f0 = 2.0 + np.cos(phase)[:, None] * amp[None, :]
    p.set_f(f0)
    dt = p.dt_cfl(0.45)
    for _ in range(nsteps):
        p.transport(dt)
    # closed form: G_i = 1 - sum_b nu_b (1 - exp(-i s_b k_b h)), nu_b = dt |xi_b| / h
    G = np.ones(p.nv, dtype=complex)
    for b in range(dim):
        nu = dt * np.abs(p.xi[:, b]) / hh
        s = np.sign(p.xi[:, b])
        G -= nu * (1 - np.exp(-1j * s * kvec[b] * hh))
    exact = 2.0 + np.real(np.exp(1j * phase)[:, None] * (G ** nsteps)[None, :]) * amp[None, :]
    return p.get_f(), exact


@pytest.mark.parametrize("dim,lev,n,wav", [(2, 4, (8, 8, 8), (1, 2)), (3, 3, (4, 6, 4), (1, -1, 2))])
def test_transport_fourier_closed_form(dim, lev, n, wav):
    got, exact = _fourier_case(dim, lev, n, 3.0, wav)
    assert np.max(np.abs(got - exact)) < 1e-12


REFINED = [
    O.make_spec(2, 2, 5, O.PRED_BALL, (0.3, 0.6, 0.5), 0.05),
    O.make_spec(3, 1, 4, O.PRED_BALL, (0.3, 0.6, 0.7), 0.05),
]


@pytest.mark.parametrize("spec", REFINED)
def test_transport_freestream_preserved_on_refined_tree(spec):
    p = O.Problem(spec, (4, 4, 4), (-2,) * 3, (2,) * 3)
    rng = np.random.default_rng(1)
    row = rng.uniform(0.5, 1.5, p.nv)
    p.set_f(np.tile(row, (p.ncells, 1)))
    p.transport(p.dt_cfl(0.5))
    assert np.max(np.abs(p.get_f() - row[None, :])) < 1e-14


@pytest.mark.parametrize("spec", REFINED)
def test_transport_conserves_each_velocity_periodic(spec):
    p = O.Problem(spec, (4, 4, 4), (-2,) * 3, (2,) * 3)
    xyz, h = p.centres()
    V = h ** spec.dim
    rng = np.random.default_rng(2)
    f0 = rng.uniform(0.1, 1.0, (p.ncells, p.nv))
    p.set_f(f0)
    p.transport(p.dt_cfl(0.5))
    m0 = V @ f0
    m1 = V @ p.get_f()
    assert np.max(np.abs(m1 - m0) / m0) < 1e-14
    # and something did move
    assert np.max(np.abs(p.get_f() - f0)) > 1e-3


def test_transport_specular_walls_conserve_mass_and_energy():
    spec = O.make_spec(3, 1, 3, O.PRED_BALL, (0.4, 0.4, 0.6), 0.1, bc=(3,) * 6)
    p = O.Problem(spec, (6, 6, 6), (-3,) * 3, (3,) * 3)
    xyz, h = p.centres()
    V = h ** 3
    rng = np.random.default_rng(3)
    p.set_f(rng.uniform(0.1, 1.0, (p.ncells, p.nv)))
    t0 = p.totals()
    for _ in range(3):
        p.transport(p.dt_cfl(0.5))
    t1 = p.totals()
    assert abs(t1[0] - t0[0]) < 1e-14 * t0[0]
    assert abs(t1[4] - t0[4]) < 1e-13 * t0[4]
    # momentum along x is not conserved by walls (they push)
    assert abs(t1[1] - t0[1]) > 1e-6 * abs(t0[4])


def test_transport_specular_symmetric_state_preserved():
    spec = O.make_spec(3, 1, 3, O.PRED_BALL, (0.4, 0.4, 0.6), 0.1, bc=(3,) * 6)
    p = O.Problem(spec, (6, 6, 6), (-3,) * 3, (3,) * 3)
    # an isotropic row: depends on |xi| only, so every reflection maps it to itself
    row = np.exp(-0.3 * (p.xi ** 2).sum(axis=1))
    p.set_f(np.tile(row, (p.ncells, 1)))
    p.transport(p.dt_cfl(0.5))
    assert np.max(np.abs(p.get_f() - row[None, :])) < 1e-15


def test_transport_outflow_preserves_uniform_state():
    spec = O.make_spec(3, 1, 3, O.PRED_BALL, (0.4, 0.4, 0.6), 0.1, bc=(2,) * 6)
    p = O.Problem(spec, (4, 4, 4), (-2,) * 3, (2,) * 3)
    rng = np.random.default_rng(4)
    row = rng.uniform(0.5, 1.5, p.nv)
    p.set_f(np.tile(row, (p.ncells, 1)))
    p.transport(p.dt_cfl(0.5))
    assert np.max(np.abs(p.get_f() - row[None, :])) < 1e-14


def test_transport_inflow_ghost_is_freestream():
    spec = O.make_spec(3, 2, 2, O.PRED_NONE, bc=(1, 2, 2, 2, 2, 2))
    p = O.Problem(spec, (6, 6, 6), (-4,) * 3, (4,) * 3)
    u = (1.2, 0.1, -0.2)
    p.set_freestream(1.0, u, 0.8)
    # the freestream sampled by init_maxwellian
    p.init_maxwellian(np.ones(p.ncells), np.ones(p.ncells), np.tile(u, (p.ncells, 1)), np.full(p.ncells, 0.8))
    fin = p.get_f()[0].copy()
    p.set_f(np.zeros((p.ncells, p.nv)))
    dt = p.dt_cfl(0.4)
    p.transport(dt)
    f = p.get_f()
    xyz, h = p.centres()
    first = np.isclose(xyz[:, 0], 0.125)
    pos = p.xi[:, 0] > 0
    expect = dt * p.xi[pos, 0] / 0.25 * fin[pos]
    assert np.allclose(f[first][:, pos], expect[None, :], rtol=1e-14, atol=0)
    assert np.all(f[first][:, ~pos] == 0) and np.all(f[~first] == 0)


def test_moments_of_maxwellian_closed_form():
    spec = _uniform(3, 1)
    p = O.Problem(spec, (32, 32, 32), (-10,) * 3, (10,) * 3)
    rho, u, T = 1.3, np.array([0.3, -0.2, 0.1]), 0.9
    nc = p.ncells
    p.init_maxwellian(np.ones(nc), np.full(nc, rho), np.tile(u, (nc, 1)), np.full(nc, T))
    r, uu, TT = p.moments()
    assert np.allclose(r, rho, rtol=1e-12)
    assert np.allclose(uu, u[None, :], rtol=0, atol=1e-12)
    assert np.allclose(TT, T, rtol=1e-12)


def test_density_of_a_truncated_maxwellian_closed_form():
    """On a grid that cuts the Maxwellian off (here [-3, 3]^3, 24^3 nodes), the
    discrete density is the midpoint rule of a truncated Gaussian per axis:
    the exact integral (erf) plus the Euler-Maclaurin endpoint terms of the
    midpoint rule, -h^2/24 [g1] + 7 h^4/5760 [g3] (g1, g3 the first and third
    derivatives at the ends), to O(h^6).  This fixes the node positions, the
    cell volume dV and the truncation of the Mach-number flows (R17)."""
    from math import erf, exp, pi, sqrt
    V, n = 3.0, 24
    h = 2 * V / n
    p = O.Problem(_uniform(3, 1), (n,) * 3, (-V,) * 3, (V,) * 3)
    nc = p.ncells

    def axis_sum(u, T):
        def g(x):
            return exp(-(x - u) ** 2 / (2 * T))

        def g1(x):
            return -(x - u) / T * g(x)

        def g3(x):
            z = (x - u) / sqrt(T)
            return -(z ** 3 - 3 * z) / T ** 1.5 * g(x)

        s = sqrt(2 * T)
        integral = sqrt(2 * pi * T) * (erf((V - u) / s) + erf((V + u) / s)) / 2
        return integral - h * h / 24 * (g1(V) - g1(-V)) + 7 * h ** 4 / 5760 * (g3(V) - g3(-V))

    for u0, T in ((0.0, 1.0), (1.0, 1.0), (0.5, 0.7)):
        rho = 1.3
        p.init_maxwellian(np.ones(nc), np.full(nc, rho), np.tile([u0, 0.0, 0.0], (nc, 1)), np.full(nc, T))
        r, _, _ = p.moments()
        want = rho * axis_sum(u0, T) * axis_sum(0.0, T) ** 2 / (2 * pi * T) ** 1.5
        assert abs(r[0] / want - 1) < 5e-8, (u0, T, r[0] / want - 1)


def test_dt_cfl_closed_form():
    def prob(name, n_only=False):
        c = W.CONFIGS[name]
        spec = O.make_spec(c["dim"], c["base_level"], c["max_level"], c["pred"], c["c"], c["r"],
                           c["beta"], c["solid"], c["bc"])
        return O.Problem(spec, c["n"], c["lo"], c["hi"]), c
    p, c = prob("c1_2d_bump")
    assert p.dt_cfl(0.4) == pytest.approx(0.4 / (64 * 7), rel=1e-15)
    p, c = prob("c2_sphere_m3")
    assert p.dt_cfl(0.4) == pytest.approx(0.4 / (64 * 16.875), rel=1e-15)


def test_solver_matches_lapack_and_detects_singular():
    rng = np.random.default_rng(5)
    for _ in range(20):
        A = rng.normal(size=(5, 5)) + 5 * np.eye(5)
        b = rng.normal(size=5)
        assert np.allclose(O.solve(A, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-14)
    # needs pivoting
    A = np.array([[0.0, 1, 0, 0, 0], [1, 0, 0, 0, 0], [0, 0, 1, 0, 0], [0, 0, 0, 1, 0], [0, 0, 0, 0, 1]])
    assert np.allclose(O.solve(A, np.arange(5.0)), [1, 0, 2, 3, 4])
    with pytest.raises(np.linalg.LinAlgError):
        O.solve(np.ones((5, 5)), np.ones(5))


def _streaming_error(spec, T=0.25):
    """L-infinity error of free streaming (no collision) against the exact
    translation f(x - xi t) of a periodic sinusoid, every velocity of a 2^3
    grid (components +-1/2)."""
    p = O.Problem(spec, (2, 2, 2), (-1.0,) * 3, (1.0,) * 3)
    xyz, _ = p.centres()
    k = 2 * np.pi * np.array([1.0, 1.0, 1.0])[:spec.dim]

    def f0(x):
        return 2.0 + np.cos(x[:, :spec.dim] @ k)

    p.set_f(np.stack([f0(xyz)] * p.nv, axis=1))
    nsteps = int(np.ceil(T / p.dt_cfl(0.4)))
    dt = T / nsteps
    for _ in range(nsteps):
        p.transport(dt)
    g = p.get_f()
    return max(np.max(np.abs(g[:, v] - f0(xyz - p.xi[v] * T))) for v in range(p.nv))


@pytest.mark.parametrize("dim,levels,refined", [(2, (4, 5, 6), False), (2, (4, 5, 6), True), (3, (4, 5), True)])
def test_free_streaming_converges_at_first_order(dim, levels, refined):
    """Halving every cell halves the error of free molecular streaming
    against the exact solution, on uniform trees and on trees with a refined
    ball (hanging faces): the scheme of Eq. 2 is consistent, and a wrong
    coarse-fine weight would leave an error that does not shrink."""
    errs = []
    for L in levels:
        if refined:
            spec = O.make_spec(dim, L, L + 1, O.PRED_BALL, (0.5, 0.5, 0.5), 0.25)
        else:
            spec = O.make_spec(dim, L, L, O.PRED_NONE)
        errs.append(_streaming_error(spec))
    ratios = [a / b for a, b in zip(errs, errs[1:])]
    assert all(1.7 < r < 2.2 for r in ratios), (errs, ratios)
