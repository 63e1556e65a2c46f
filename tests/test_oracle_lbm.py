"""Pins of the oracle's lattice Boltzmann (Sec. 4): velocity sets and weights
against the isotropy conditions that fix them, the second-order equilibrium
against its closed-form moments, the BGK relaxation against its closed-form
solution, the finite-volume transport on the lattice velocities against
the Fourier amplification factor of first-order upwind and against exact
conservation and freestream preservation on refined trees, and the whole
scheme against the exact shear-mode damping of the BGK equation (the
viscosity c_s^2 tau)."""
import itertools
import math

import numpy as np
import pytest

import oracle as O

SETS = [(O.D2Q9, 2, 9), (O.D3Q19, 3, 19), (O.D3Q27, 3, 27)]


@pytest.mark.parametrize("kind,dim,q", SETS)
def test_velocity_set_membership_and_order(kind, dim, q):
    c, w = O.lattice(kind)
    assert c.shape == (q, 3) and w.shape == (q,)
    assert np.all(np.isin(c, [-1.0, 0.0, 1.0]))
    if dim == 2:
        assert np.all(c[:, 2] == 0)
    assert len({tuple(x) for x in c}) == q
    r2 = (c ** 2).sum(axis=1)
    # D3Q19 is the 3x3x3 set without the 8 corners
    if kind == O.D3Q19:
        assert r2.max() == 2
    full = [x for x in itertools.product([-1, 0, 1], repeat=3) if (dim == 3 or x[2] == 0)
            and (kind != O.D3Q19 or sum(t * t for t in x) < 3)]
    order = sorted(full, key=lambda x: (sum(t * t for t in x), x))
    assert [tuple(int(t) for t in x) for x in c] == order
    # weights depend on |c|^2 only
    for k in range(4):
        assert len(set(w[r2 == k])) <= 1


@pytest.mark.parametrize("kind,dim,q", SETS)
def test_weights_satisfy_isotropy(kind, dim, q):
    """sum w = 1, odd moments 0, sum w c_a c_b = delta/3, sum w c_a c_b c_c c_d
    = (delta delta + delta delta + delta delta)/9: the conditions that give the
    lattice its speed of sound 1/sqrt(3) and fix the weights uniquely."""
    c, w = O.lattice(kind)
    c = c[:, :dim]
    I = np.eye(dim)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), I / 3, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I) + np.einsum("ad,bc->abcd", I, I)) / 9
    assert np.allclose(m4, iso, atol=1e-15)


def _periodic(dim, base, maxl=None, pred=O.PRED_NONE, r=0.0, kind=None, bc=(0,) * 6):
    spec = O.make_spec(dim, base, maxl if maxl is not None else base, pred, (0.5, 0.5, 0.5), r, 0.0, 0, bc)
    return O.Problem(spec, lattice=kind or (O.D2Q9 if dim == 2 else O.D3Q27))


@pytest.mark.parametrize("kind,dim,q", SETS)
def test_equilibrium_moments(kind, dim, q):
    """sum feq = rho, sum c feq = rho u and sum c c feq = rho (I/3 + u u),
    exactly (up to rounding) for any rho, u."""
    p = _periodic(dim, 1, kind=kind)
    c = p.xi[:, :dim]
    rng = np.random.default_rng(5)
    for _ in range(5):
        rho = rng.uniform(0.5, 2.0)
        u = np.zeros(3)
        u[:dim] = rng.uniform(-0.3, 0.3, dim)
        feq = p.lbm_feq(rho, u)
        assert abs(feq.sum() - rho) < 1e-14
        assert np.allclose(c.T @ feq, rho * u[:dim], atol=1e-15)
        P = np.einsum("i,ia,ib->ab", feq, c, c)
        assert np.allclose(P, rho * (np.eye(dim) / 3 + np.outer(u[:dim], u[:dim])), atol=1e-14)
        # at rest feq is rho w
        assert np.allclose(p.lbm_feq(rho, np.zeros(3)), rho * p.w, atol=1e-16)


@pytest.mark.parametrize("kind,dim,q", SETS)
def test_homogeneous_bgk_relaxation_closed_form(kind, dim, q):
    """Identical cells on a periodic tree (transport leaves them unchanged):
    rho and u are conserved, so feq is fixed and f - feq shrinks by 1 - dt/tau
    per step."""
    p = _periodic(dim, 2, kind=kind)
    rng = np.random.default_rng(7)
    f0 = p.w * rng.uniform(0.5, 1.5, p.nv)
    p.set_f(np.tile(f0, (p.ncells, 1)))
    rho = f0.sum()
    u = np.zeros(3)
    u[:] = p.xi.T @ f0 / rho
    feq = p.lbm_feq(rho, u)
    dt, tau, n = 0.01, 0.04, 7
    p.lbm_step(n, dt, tau)
    want = feq + (1 - dt / tau) ** n * (f0 - feq)
    f = p.get_f()
    assert np.max(np.abs(f - want[None, :])) < 1e-14
    r1, u1 = p.lbm_moments()
    assert np.allclose(r1, rho, rtol=1e-14) and np.allclose(u1, u[None, :], atol=1e-14)


@pytest.mark.parametrize("kind,dim,q", SETS)
def test_transport_fourier_amplification(kind, dim, q):
    """One transport step on a uniform periodic tree: for velocity c the mode
    exp(2 pi i k.x) is multiplied by G = 1 - (dt/h) sum_d |c_d| (1 -
    exp(-2 pi i sign(c_d) k_d h)); a zero component carries no flux."""
    L = 3 if dim == 3 else 4
    p = _periodic(dim, L, kind=kind)
    h = 2.0 ** -L
    xyz, _ = p.centres()
    ks = np.array([[1, 2, 1], [2, 1, 3], [3, 1, 2]])[:, :dim]
    f = np.zeros((p.ncells, p.nv))
    theta = []
    for i in range(p.nv):
        k = ks[i % 3]
        th = 2 * math.pi * (xyz[:, :dim] @ k)
        theta.append(th)
        f[:, i] = 2.0 + np.cos(th)
    p.set_f(f)
    dt = p.dt_cfl(0.5)
    p.transport(dt)
    g = p.get_f()
    for i in range(p.nv):
        k = ks[i % 3]
        c = p.xi[i, :dim]
        G = 1.0 - (dt / h) * sum(abs(c[d]) * (1 - np.exp(-2j * math.pi * np.sign(c[d]) * k[d] * h))
                                 for d in range(dim))
        want = 2.0 + np.real(G * np.exp(1j * theta[i]))
        assert np.max(np.abs(g[:, i] - want)) < 1e-13, i


@pytest.mark.parametrize("kind,dim", [(O.D2Q9, 2), (O.D3Q19, 3)])
def test_conservation_on_refined_periodic_tree(kind, dim):
    """Hanging faces: sum_cells V f_i is unchanged by transport for every
    velocity, and rho, rho u by the whole step."""
    p = _periodic(dim, 2, 4, O.PRED_BALL, 0.2, kind=kind)
    _, hh = p.centres()
    V = hh ** dim
    rng = np.random.default_rng(9)
    f = p.w[None, :] * rng.uniform(0.5, 1.5, (p.ncells, p.nv))
    p.set_f(f)
    tot0 = V @ f
    dt = p.dt_cfl(0.4)
    p.transport(dt)
    tot1 = V @ p.get_f()
    assert np.allclose(tot1, tot0, rtol=1e-13, atol=0)
    m0 = np.array([tot1.sum(), *(tot1 @ p.xi[:, :dim])])
    p.lbm_collide(dt, 0.05)
    tot2 = V @ p.get_f()
    m1 = np.array([tot2.sum(), *(tot2 @ p.xi[:, :dim])])
    assert np.max(np.abs(m1 - m0)) < 1e-14 * tot0.sum()


@pytest.mark.parametrize("kind,dim", [(O.D2Q9, 2), (O.D3Q19, 3), (O.D3Q27, 3)])
def test_freestream_preserved_with_inflow_outflow_walls(kind, dim):
    """A uniform stream parallel to the walls, entering at its own
    equilibrium, stays exactly uniform on a refined tree with a solid
    obstacle-free refinement ball: every flux balance and boundary ghost of
    the scheme cancels."""
    bc = (O.BC_INFLOW, O.BC_OUTFLOW, O.BC_WALL, O.BC_WALL, O.BC_WALL, O.BC_WALL)
    p = _periodic(dim, 2, 4, O.PRED_BALL, 0.2, kind=kind, bc=bc)
    u = np.array([0.12, 0.0, 0.0])
    p.lbm_set_inflow(1.1, u)
    p.lbm_init(np.full(p.ncells, 1.1), np.tile(u, (p.ncells, 1)))
    f0 = p.get_f()
    p.lbm_step(6, p.dt_cfl(0.4), 0.03)
    assert np.max(np.abs(p.get_f() - f0)) < 1e-14


def _shear_mode_decay(tau, k):
    """Damping rate of the shear wave of the D2Q9 discrete-velocity BGK
    equation df/dt + c_x df/dx = -(f - feq)/tau, linearised about rest: the
    slowest eigenvalue of -i k diag(c_x) - (I - P)/tau, with P the linear
    equilibrium map feq_i = w_i (rho + 3 c_i.j).  Its long-wave limit is
    nu k^2 with nu = c_s^2 tau."""
    c, w = O.lattice(O.D2Q9)
    c = c[:, :2]
    P = w[:, None] * (1.0 + 3.0 * (c @ c.T))
    A = -1j * k * np.diag(c[:, 0]) - (np.eye(len(w)) - P) / tau
    ev, V = np.linalg.eig(A)
    jy = np.abs(c[:, 1] @ V) / np.linalg.norm(V, axis=0)
    return -ev[np.argmax(jy)].real


def test_shear_wave_damping_matches_the_bgk_equation():
    """A small shear wave u_y = U sin(2 pi x) on uniform periodic quadtrees
    decays at the rate of the continuous D2Q9 BGK equation: the rate measured
    between t = 0.25 and 0.75 (after the initial transient) at levels 7 and 8,
    extrapolated linearly in h (first-order scheme), matches the exact mode
    to 0.1%.  This fixes the viscosity c_s^2 tau the equilibrium and the
    relaxation produce, not only their moments."""
    tau, k, U = 0.02, 2 * np.pi, 1e-3

    def rate(L):
        p = _periodic(2, L, kind=O.D2Q9)
        xyz, _ = p.centres()
        u = np.zeros((p.ncells, 3))
        u[:, 1] = U * np.sin(k * xyz[:, 0])
        p.lbm_init(np.ones(p.ncells), u)
        dt = p.dt_cfl(0.4)
        n1 = int(round(0.25 / dt))
        dt = 0.25 / n1

        def amp():
            _, uu = p.lbm_moments()
            return 2 * np.mean(uu[:, 1] * np.sin(k * xyz[:, 0]))

        p.lbm_step(n1, dt, tau)
        a1 = amp()
        p.lbm_step(2 * n1, dt, tau)
        return -np.log(amp() / a1) / (2 * n1 * dt)

    r7, r8 = rate(7), rate(8)
    exact = _shear_mode_decay(tau, k)
    assert abs(exact / (tau / 3 * k * k) - 1) < 0.01   # the long-wave limit nu k^2
    assert abs((2 * r8 - r7) / exact - 1) < 1e-3, (r7, r8, exact)
