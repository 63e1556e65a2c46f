"""Pins for the oracle's collision operators: conservative BGK and the
hard-sphere discrete collision integral with its conservative correction
(Eqs. 3-6).

Pinned against: exact conservation of mass, momentum and energy by the
collision term (the property Eq. 6 is built for), the Maxwellian fixed point,
the closed-form geometric relaxation of spatially homogeneous BGK, H-theorem
monotonicity, the hard-sphere mean collision frequency sqrt(8/pi) of a unit
Maxwellian, the published SplitMix64 output sequence, an independent
pure-Python regeneration of the seeded trial tables, the shear-wave
damping of the whole BGK step against the linearised discrete-velocity BGK
equation, and the hard-sphere relaxation towards the Maxwellian as the
trials grow.
"""
import math

import numpy as np
import pytest

import oracle as O


def _homog(n=(12, 12, 12), vmax=6.0):
    """Spatially homogeneous problem: one uniform periodic level-1 tree."""
    spec = O.make_spec(3, 1, 1, O.PRED_NONE)
    return O.Problem(spec, n, (-vmax,) * 3, (vmax,) * 3)


def _bimodal(p, w=0.4, a=1.5, T=0.5):
    nc = p.ncells
    u = np.zeros((nc, 2, 3))
    u[:, 0, 0], u[:, 1, 0] = a, -a
    p.init_maxwellian(np.tile([w, 1 - w], (nc, 1)), np.ones((nc, 2)), u, np.full((nc, 2), T))


def _psi(xi):
    return np.stack([np.ones(len(xi)), xi[:, 0], xi[:, 1], xi[:, 2], (xi ** 2).sum(axis=1)], axis=1)


def _conservation_residual(q, xi, dV):
    ps = _psi(xi)
    num = np.abs(q @ ps) * dV
    den = (np.abs(q)[:, :, None] * np.abs(ps)[None, :, :]).sum(axis=1) * dV
    return np.max(num / den)


# ---------------------------------------------------------------- BGK
def test_bgk_collision_term_conserves():
    p = _homog()
    _bimodal(p)
    rng = np.random.default_rng(7)
    p.set_f(p.get_f() * rng.uniform(0.8, 1.2, (p.ncells, p.nv)))
    q = p.bgk(1e-3, 0.05, want_q=True)
    assert _conservation_residual(q, p.xi, p.dV) < 1e-12


def test_bgk_homogeneous_geometric_relaxation():
    """With conserved moments the target M~ is fixed, so each step scales
    f - M~ by the same factor (1 - nu dt)."""
    p = _homog()
    _bimodal(p)
    f0 = p.get_f()[0].copy()
    rho, u, T = p.moments()
    kn, dt = 0.05, 2e-3
    f = [f0]
    for _ in range(4):
        p.step(1, dt, O.COLL_BGK, kn)
        f.append(p.get_f()[0].copy())
    nu = math.sqrt(8 / math.pi) * rho[0] * math.sqrt(T[0]) / kn
    lam = 1 - nu * dt
    Mt = (f[1] - lam * f[0]) / (1 - lam)
    for n in range(1, 5):
        assert np.max(np.abs(f[n] - (Mt + lam ** n * (f0 - Mt)))) < 1e-13 * np.max(f0)
    # M~ is a fixed point
    p.set_f(np.tile(Mt, (p.ncells, 1)))
    p.step(1, dt, O.COLL_BGK, kn)
    assert np.max(np.abs(p.get_f()[0] - Mt)) < 1e-14 * np.max(Mt)
    # and carries the moments of f0
    ps = _psi(p.xi)
    assert np.allclose(Mt @ ps, f0 @ ps, rtol=1e-13, atol=1e-13)


def test_bgk_h_theorem_homogeneous():
    p = _homog()
    _bimodal(p, w=0.3, a=1.8, T=0.6)
    kn, dt = 0.05, 4e-3
    H = []
    for _ in range(30):
        f = p.get_f()[0]
        H.append(float(np.sum(f * np.log(np.maximum(f, 1e-300))) * p.dV))
        p.step(1, dt, O.COLL_BGK, kn)
    dH = np.diff(H)
    # the polynomial-corrected Maxwellian obeys the H-theorem up to O(d^2)
    assert np.all(dH <= 1e-6 * abs(H[0]))
    assert H[-1] < H[0] - 1e-3


def test_bgk_rejects_bad_state():
    p = _homog(n=(4, 4, 4), vmax=2.0)
    p.set_f(-np.ones((p.ncells, p.nv)))
    with pytest.raises(RuntimeError):
        p.bgk(1e-3, 0.1)


# ---------------------------------------------------------------- HS
SPLITMIX64_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_splitmix64_published_sequence():
    # the first outputs of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014)
    assert [O.splitmix64(0, n) for n in range(4)] == SPLITMIX64_SEED0


def _py_tables(n, lo, hi, M, seed):
    """Trial tables restated in pure Python from the seeded construction."""
    xi, k, dV = O.vgrid(n, lo, hi)
    nv = len(xi)
    mask = (1 << 64) - 1

    def sm(nn):
        z = (seed + (nn + 1) * 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        return z ^ (z >> 31)

    def U(nn):
        return (sm(nn) >> 11) * 2.0 ** -53

    h = [(hi[d] - lo[d]) / n[d] for d in range(3)]
    where = {tuple(k[v]): v for v in range(nv)}
    rows = []
    disc = 0
    for i in range(nv):
        kept = []
        for t in range(M):
            s = i * M + t
            g = int(U(3 * s) * nv)
            z = 2.0 * U(3 * s + 1) - 1.0
            phi = 2.0 * math.pi * U(3 * s + 2)
            st = math.sqrt(max(0.0, 1.0 - z * z))
            w = (st * math.cos(phi), st * math.sin(phi), z)
            gn = math.sqrt(sum((xi[i][d] - xi[g][d]) ** 2 for d in range(3)))
            xp, xq = [], []
            for d in range(3):
                c = 0.5 * (xi[i][d] + xi[g][d])
                xp.append(c + 0.5 * gn * w[d])
                xq.append(c - 0.5 * gn * w[d])

            def near(x):
                out = []
                for d in range(3):
                    tt = (x[d] - lo[d]) / h[d] - 0.5
                    r = math.floor(abs(tt) + 0.5) * (1 if tt >= 0 else -1)
                    if r < 0 or r > n[d] - 1:
                        return None
                    out.append(int(r))
                return tuple(out)
            kp, kq = near(xp), near(xq)
            if kp is None or kq is None:
                disc += 1
                continue
            kept.append((g, where[kp], where[kq], gn))
        rows.append([(g, l, m, nv * dV * gn / (math.sqrt(2.0) * M)) for g, l, m, gn in kept])
    return rows, disc


def test_hs_tables_match_independent_regeneration():
    n, lo, hi, M, seed = (8, 8, 8), (-4.0,) * 3, (4.0,) * 3, 16, 12345
    spec = O.make_spec(3, 1, 1, O.PRED_NONE)
    p = O.Problem(spec, n, lo, hi)
    p.hs_tables(M, seed)
    start, gam, l, m, b, disc = p.hs_get_tables()
    rows, disc_py = _py_tables(n, lo, hi, M, seed)
    assert disc == disc_py and disc > 0
    for i, row in enumerate(rows):
        s, e = start[i], start[i + 1]
        assert e - s == len(row)
        assert gam[s:e].tolist() == [r[0] for r in row]
        assert l[s:e].tolist() == [r[1] for r in row]
        assert m[s:e].tolist() == [r[2] for r in row]
        ref = np.array([r[3] for r in row])
        assert np.all(np.abs(b[s:e] - ref) <= np.spacing(ref))


def test_hs_collision_term_conserves_and_produces_entropy():
    p = _homog(n=(10, 10, 10), vmax=5.0)
    _bimodal(p, w=0.35, a=1.4, T=0.5)
    p.hs_tables(64, 20150303)
    f = p.get_f()[0].copy()
    q, B, Cc = p.hs_collide(1e-4, 0.02, want=True)
    assert _conservation_residual(q, p.xi, p.dV) < 1e-12
    # entropy production sum I ln f dV <= 0 on the bimodal state
    assert float(np.sum(q[0] * np.log(f)) * p.dV) < 0


def test_hs_mean_collision_frequency_of_maxwellian():
    """sum f B / sum f -> sqrt(8/pi) for a unit Maxwellian (rho = T = 1):
    the hard-sphere normalisation that makes the mean free path Kn.  The
    estimate is Monte Carlo over the seeded trials (about 2% noise per seed at
    1024 trials on this mesh), so three seeds are averaged."""
    nus = []
    for seed in (1, 2, 3):
        p = _homog(n=(12, 12, 12), vmax=6.0)
        nc = p.ncells
        p.init_maxwellian(np.ones(nc), np.ones(nc), np.zeros((nc, 3)), np.ones(nc))
        p.hs_tables(1024, seed)
        f = p.get_f()[0].copy()
        q, B, Cc = p.hs_collide(1e-6, 1.0, want=True)
        nus.append(float(np.sum(f * B[0]) / np.sum(f)))
        # the corrected collision term of a Maxwellian is small next to the loss term
        assert np.max(np.abs(q[0])) < 0.5 * np.max(f * B[0])
    assert abs(np.mean(nus) / math.sqrt(8 / math.pi) - 1) < 0.05


def test_bgk_frequency_equals_hs_mean_frequency():
    """The DVM-BGK frequency is the hard-sphere mean collision frequency of the
    local Maxwellian, (1/sqrt 2) <|g|> rho: the relaxation factor measured from
    one homogeneous BGK step must match the pair sum over the discrete
    Maxwellian at rho = 1.7, T = 0.8."""
    p = _homog(n=(16, 16, 16), vmax=8.0)
    nc = p.ncells
    rho, T = 1.7, 0.8
    p.init_maxwellian(np.ones(nc), np.full(nc, rho), np.zeros((nc, 3)), np.full(nc, T))
    M0 = p.get_f()[0].copy()
    xi = p.xi
    pert = M0 * (1 + 0.05 * np.cos(xi[:, 0]))
    # the local Maxwellian of the perturbed state
    p.set_f(np.tile(pert, (nc, 1)))
    r1, u1, T1 = p.moments()
    p.init_maxwellian(np.ones(nc), r1, u1, T1)
    M = p.get_f()[0].copy()
    g = np.sqrt(((xi[:, None, :] - xi[None, :, :]) ** 2).sum(-1))
    nu_pairs = float((M[:, None] * M[None, :] * g).sum() * p.dV / math.sqrt(2.0) / M.sum())
    # two homogeneous steps: f - M~ shrinks by the same factor 1 - nu dt each time
    kn, dt = 1.0, 1e-2
    p.set_f(np.tile(pert, (nc, 1)))
    p.step(1, dt, O.COLL_BGK, kn)
    f1 = p.get_f()[0].copy()
    p.step(1, dt, O.COLL_BGK, kn)
    f2 = p.get_f()[0].copy()
    lam = np.sum((f2 - f1) * (f1 - pert)) / np.sum((f1 - pert) ** 2)
    nu_bgk = (1 - lam) / dt
    assert abs(nu_bgk / nu_pairs - 1) < 0.01


# ---------------------------------------------------------------- HS, lattice trials
def test_korobov_lattice_is_stratified():
    """A rank-1 lattice with generator (1, a, a^2, a^3, a^4) and a odd is, for
    M a power of two, a permutation in every coordinate: the M points of a
    node fall one in each interval [m/M, (m+1)/M) of every axis, whatever
    the node's shift (the shift moves all points by the same amount modulo
    1).  Random trials do not have this property."""
    for M in (32, 64, 256):
        a = O.korobov_a(M)
        assert a % 2 == 1 and 1 <= a < M
        for i in (0, 7, 123):
            u = np.array([O.trial_uniforms(1, 20150303, i, k, M) for k in range(M)])
            shift = u[0]  # point 0 is the shift itself
            for j in range(5):
                cell = np.floor(((u[:, j] - shift[j]) % 1.0) * M + 1e-9).astype(int) % M
                assert sorted(cell.tolist()) == list(range(M)), (M, i, j)
    u = np.array([O.trial_uniforms(0, 20150303, 0, k, 64) for k in range(64)])
    assert len(set(np.floor(u[:, 0] * 64).astype(int).tolist())) < 64


def test_korobov_multiplier_maximises_the_lattice_spacing():
    """The multiplier's defining property, checked by brute force over every
    odd a: no other a gives a larger smallest torus distance between points."""
    M = 64

    def spacing(a):
        z = np.array([pow(a, j, M) for j in range(5)])
        r = (np.arange(1, M)[:, None] * z[None, :]) % M
        r = np.minimum(r, M - r)
        return int((r ** 2).sum(axis=1).min())
    best = max(spacing(a) for a in range(1, M, 2))
    a = O.korobov_a(M)
    assert spacing(a) == best
    assert all(spacing(b) < best for b in range(1, a, 2))


def _nubar(M, seed, lattice):
    p = _homog(n=(12, 12, 12), vmax=6.0)
    nc = p.ncells
    p.init_maxwellian(np.ones(nc), np.ones(nc), np.zeros((nc, 3)), np.ones(nc))
    p.hs_tables(M, seed, lattice=lattice)
    f = p.get_f()[0].copy()
    q, B, Cc = p.hs_collide(1e-6, 1.0, want=True)
    return float(np.sum(f * B[0]) / np.sum(f))


def test_lattice_trials_estimate_the_collision_frequency_better():
    """sum f B / sum f of a unit Maxwellian estimates sqrt(8/pi).  Over six
    lattice shifts the lattice estimate scatters less than six random-trial
    estimates and lies closer to sqrt(8/pi) (the quasi-Monte Carlo gain the
    Korobov construction is for)."""
    target = math.sqrt(8 / math.pi)
    M = 64
    lat = np.array([_nubar(M, s, True) for s in range(1, 7)])
    rnd = np.array([_nubar(M, s, False) for s in range(1, 7)])
    assert lat.std() < 0.7 * rnd.std(), (lat.std(), rnd.std())
    assert abs(lat.mean() - target) < abs(rnd.mean() - target)
    assert abs(lat.mean() / target - 1) < 0.03


def test_lattice_hs_collision_conserves():
    p = _homog(n=(10, 10, 10), vmax=5.0)
    _bimodal(p, w=0.35, a=1.4, T=0.5)
    p.hs_tables(64, 20150303, lattice=True)
    f = p.get_f()[0].copy()
    q, B, Cc = p.hs_collide(1e-4, 0.02, want=True)
    assert _conservation_residual(q, p.xi, p.dV) < 1e-12
    assert float(np.sum(q[0] * np.log(f)) * p.dV) < 0


# ---------------------------------------------------------------- entropic BGK
def _entropy(f, dV):
    return float(np.sum(f * np.log(f)) * dV)


def test_entropic_bgk_conserves_and_is_exponential_of_a_quadratic():
    """The entropic target has the moments of f (conservation of the
    collision term to 1e-12) and its logarithm is a quadratic in xi with an
    isotropic square term, the form of the discrete entropic equilibrium."""
    p = _homog(n=(12, 12, 12), vmax=6.0)
    _bimodal(p, w=0.35, a=1.4, T=0.5)
    f = p.get_f()[0].copy()
    dt, kn = 1e-3, 1.0
    q = p.bgk_entropic(dt, kn, want_q=True)
    assert _conservation_residual(q, p.xi, p.dV) < 1e-12
    # recover E from the step: f1 = f + dt nu (E - f)
    r, u, T = p.moments()
    nu = math.sqrt(8 / math.pi) * r[0] * math.sqrt(T[0]) / kn
    E = f + q[0] / nu
    X = _psi(p.xi)
    coef, res, *_ = np.linalg.lstsq(X, np.log(E), rcond=None)
    assert np.max(np.abs(X @ coef - np.log(E))) < 1e-9
    assert coef[4] < 0


def test_entropic_bgk_fixed_point_and_monotone_entropy():
    """The entropic equilibrium is a fixed point to rounding, and the
    homogeneous relaxation towards it decreases the entropy H = sum f ln f dV
    at every step (exactly: E minimises H under the conserved moments and the
    update is a convex combination), where the polynomial-corrected target
    only keeps it to O(d^2)."""
    p = _homog(n=(12, 12, 12), vmax=6.0)
    _bimodal(p, w=0.3, a=1.6, T=0.4)
    dt, kn = 2e-3, 0.05
    H = [_entropy(p.get_f()[0], p.dV)]
    for _ in range(40):
        p.bgk_entropic(dt, kn)
        H.append(_entropy(p.get_f()[0], p.dV))
    dH = np.diff(H)
    assert np.all(dH <= 1e-13 * abs(H[0])), dH.max()
    assert H[-1] < H[0]
    # at the end f is (nearly) its own equilibrium: one more step moves it
    # only by the remaining distance, and an exact equilibrium not at all
    f = p.get_f()[0].copy()
    q = p.bgk_entropic(dt, kn, want_q=True)
    r, u, T = p.moments()
    nu = math.sqrt(8 / math.pi) * r[0] * math.sqrt(T[0]) / kn
    E = f + q[0] / nu
    p.set_f(np.tile(E, (p.ncells, 1)))
    q2 = p.bgk_entropic(dt, kn, want_q=True)
    assert np.max(np.abs(q2[0])) < 1e-12 * nu * np.max(E)


def test_entropic_equilibrium_has_least_entropy():
    """Among distributions with the same discrete moments, the entropic
    equilibrium has the least H: below the polynomial-corrected discrete
    Maxwellian of the conservative BGK."""
    p = _homog(n=(10, 10, 10), vmax=5.0)
    _bimodal(p, w=0.35, a=1.4, T=0.5)
    f = p.get_f()[0].copy()
    r, u, T = p.moments()
    kn = 1.0
    nu = math.sqrt(8 / math.pi) * r[0] * math.sqrt(T[0]) / kn
    E = f + p.bgk_entropic(1e-6, kn, want_q=True)[0] / nu
    p.set_f(np.tile(f, (p.ncells, 1)))
    Mp = f + p.bgk(1e-6, kn, want_q=True)[0] / nu
    assert np.all(E > 0) and np.all(Mp > 0)
    assert _entropy(E, p.dV) < _entropy(Mp, p.dV)
    X = _psi(p.xi)
    assert np.allclose(E @ X, Mp @ X, rtol=1e-11, atol=1e-14)


def test_bgk_shear_wave_damping_matches_the_discrete_bgk_equation():
    """A small shear wave u_y = U sin(2 pi x) in the whole DVM-BGK step
    (transport of Eq. 2, conservative BGK) on uniform periodic quadtrees: the
    damping rate measured between t = 0.1 and 0.3, extrapolated to h -> 0
    from levels 4-6 (quadratic Richardson, first-order scheme), equals the
    shear mode of the discrete-velocity BGK equation linearised about the
    discrete Maxwellian, -i k diag(xi_x) + nu (Pi - I), with Pi the
    projection onto span{psi_r M} that keeps the five moments (the
    linearised corrected target).  That mode is close to mu k^2 with
    mu = p / nu."""
    n, vmax, kn, k, U = (8, 8, 8), 4.0, 0.02, 2 * math.pi, 1e-3
    p0 = O.Problem(O.make_spec(2, 1, 1, O.PRED_NONE), n, (-vmax,) * 3, (vmax,) * 3)
    xi, dV = p0.xi, p0.dV
    M0 = np.exp(-(xi ** 2).sum(1) / 2) / (2 * math.pi) ** 1.5
    Psi = _psi(xi)
    G = Psi.T @ (M0[:, None] * Psi) * dV
    Pi = (M0[:, None] * Psi) @ np.linalg.solve(G, Psi.T * dV)
    rho = M0.sum() * dV
    T = ((xi ** 2).sum(1) * M0).sum() * dV / rho / 3
    nu = math.sqrt(8 / math.pi) * rho * math.sqrt(T) / kn
    ev, V = np.linalg.eig(-1j * k * np.diag(xi[:, 0]) + nu * (Pi - np.eye(len(xi))))
    exact = -ev[np.argmax(np.abs(xi[:, 1] @ V) / np.linalg.norm(V, axis=0))].real
    assert abs(exact / (k * k / nu) - 1) < 0.02

    def rate(L):
        p = O.Problem(O.make_spec(2, L, L, O.PRED_NONE), n, (-vmax,) * 3, (vmax,) * 3)
        xyz, _ = p.centres()
        nc = p.ncells
        u = np.zeros((nc, 3))
        u[:, 1] = U * np.sin(k * xyz[:, 0])
        p.init_maxwellian(np.ones(nc), np.ones(nc), u, np.ones(nc))
        dt = p.dt_cfl(0.4)
        n1 = int(round(0.1 / dt))
        dt = 0.1 / n1

        def amp():
            return 2 * np.mean(p.moments()[1][:, 1] * np.sin(k * xyz[:, 0]))

        p.step(n1, dt, O.COLL_BGK, kn)
        a1 = amp()
        p.step(2 * n1, dt, O.COLL_BGK, kn)
        return -math.log(amp() / a1) / (2 * n1 * dt)

    r4, r5, r6 = rate(4), rate(5), rate(6)
    extrap = (8 * r6 - 6 * r5 + r4) / 3
    assert abs(extrap / exact - 1) < 0.01, (r4, r5, r6, extrap, exact)


def test_hs_relaxation_approaches_the_maxwellian_as_trials_grow():
    """Homogeneous relaxation of the bimodal state under the hard-sphere
    operator (Eqs. 3-6): H = sum f ln f dV falls at every one of the first 40
    steps, and the state settles near the discrete Maxwellian with its
    moments.  The remaining L1 distance comes from the finite trial set, so
    it shrinks as the trials grow (about as 1/sqrt(M)): a wrong gain term
    would leave a floor that more trials do not lower."""
    def run(M, steps=300, dt=0.05):
        p = _homog(n=(12, 12, 12), vmax=5.0)
        _bimodal(p, w=0.35, a=1.4, T=0.5)
        p.hs_tables(M, 7)
        H = []
        for s in range(steps):
            if s <= 40:
                f = p.get_f()[0]
                H.append(float(np.sum(f * np.log(f)) * p.dV))
            p.hs_collide(dt, 1.0)
        f = p.get_f()[0]
        r, u, T = p.moments()
        q = _homog(n=(12, 12, 12), vmax=5.0)
        q.init_maxwellian(np.ones(q.ncells), np.full(q.ncells, r[0]), np.tile(u[0], (q.ncells, 1)),
                          np.full(q.ncells, T[0]))
        return float(np.abs(f - q.get_f()[0]).sum() * p.dV), np.diff(H)

    d256, dH = run(256)
    d1024, _ = run(1024)
    assert np.all(dH < 0)
    assert d256 < 0.2 and d1024 < 0.6 * d256, (d256, d1024)
