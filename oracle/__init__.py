"""ctypes view of the FP64 CPU oracle (dvm_oracle.c).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously correct CPU
statement of the DVM Boltzmann step (paper Sec. 2.1, Sec. 3, Eqs. 1-6, the BGK
form of Sec. 4).  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import it; the product package never does.

Parity status of each function is recorded in the design notes; every
function here is pinned by a -m "not gpu" test under tests/test_oracle_*.py.
"""
import ctypes as C
import os
import numpy as np

from . import build as _build

BC_PERIODIC, BC_INFLOW, BC_OUTFLOW, BC_WALL = 0, 1, 2, 3
PRED_NONE, PRED_BALL, PRED_SHELL = 0, 1, 2
COLL_NONE, COLL_BGK, COLL_HS = 0, 1, 2
COLL_BGK_ENTROPIC = 4
D2Q9, D3Q19, D3Q27 = 9, 19, 27


class TreeSpec(C.Structure):
    _fields_ = [("dim", C.c_int), ("base_level", C.c_int), ("max_level", C.c_int),
                ("pred", C.c_int), ("c", C.c_double * 3), ("r", C.c_double),
                ("beta", C.c_double), ("solid", C.c_int), ("bc", C.c_int * 6)]


def make_spec(dim, base_level, max_level, pred=PRED_NONE, c=(0.5, 0.5, 0.5),
              r=0.0, beta=0.0, solid=0, bc=(0,) * 6):
    s = TreeSpec()
    s.dim, s.base_level, s.max_level, s.pred = dim, base_level, max_level, pred
    for d in range(3):
        s.c[d] = c[d]
    s.r, s.beta, s.solid = r, beta, int(solid)
    for q in range(6):
        s.bc[q] = bc[q]
    return s


_lib = None


def lib():
    global _lib
    if _lib is None:
        # DVM_ORACLE_LIB: a library built from a deliberately altered copy of
        # the oracle, loaded only by the mutation check of the pins
        path = os.environ.get("DVM_ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        d_p = C.POINTER(C.c_double)
        i64 = C.c_int64
        L.orc_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = None
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_vgrid_size.restype = i64
        L.orc_vgrid.argtypes = [P, P, P, P, P, P]
        L.orc_build_tree.argtypes = [C.POINTER(TreeSpec), i64, C.POINTER(i64), P, P, P]
        L.orc_create.restype = P
        L.orc_create.argtypes = [C.POINTER(TreeSpec), P, P, P]
        L.orc_create_sparse.restype = P
        L.orc_create_sparse.argtypes = [C.POINTER(TreeSpec), P, P, P]
        L.orc_step_inputs.restype = i64
        L.orc_step_inputs.argtypes = [P, i64, P, P]
        L.orc_maxwellian_rows.argtypes = [P, i64, C.c_int, P, P, P, P, P]
        L.orc_step_cells.argtypes = [P, i64, P, i64, P, P, C.c_double, C.c_int, C.c_double, P]
        L.orc_step_cells_learned.argtypes = [P, i64, P, i64, P, P, C.c_double, C.c_double, P, C.c_double, P, P, P]
        L.orc_destroy.argtypes = [P]
        for nm in ("orc_nleaves", "orc_ncells", "orc_nv", "orc_n_faces", "orc_n_bfaces", "orc_hs_nkept"):
            getattr(L, nm).restype = i64
            getattr(L, nm).argtypes = [P]
        L.orc_get_leaves.argtypes = [P, P, P, P]
        L.orc_cell_centres.argtypes = [P, P, P]
        L.orc_get_faces.argtypes = [P, P, P, P, P]
        L.orc_get_bfaces.argtypes = [P, P, P, P, P, P, P]
        L.orc_set_freestream.argtypes = [P, C.c_double, P, C.c_double]
        L.orc_init_maxwellian.argtypes = [P, C.c_int, P, P, P, P]
        L.orc_get_f.argtypes = [P, P]
        L.orc_set_f.argtypes = [P, P]
        L.orc_dt_cfl.restype = C.c_double
        L.orc_dt_cfl.argtypes = [P, C.c_double]
        L.orc_transport.argtypes = [P, C.c_double]
        L.orc_moments.argtypes = [P, P, P, P]
        L.orc_totals.argtypes = [P, P]
        L.orc_bgk.argtypes = [P, C.c_double, C.c_double, P]
        L.orc_bgk_entropic.argtypes = [P, C.c_double, C.c_double, P]
        L.orc_hs_tables.argtypes = [P, C.c_int, C.c_uint64]
        L.orc_hs_tables_lattice.argtypes = [P, C.c_int, C.c_uint64]
        L.orc_korobov_a.argtypes = [C.c_int64]
        L.orc_korobov_a.restype = C.c_int64
        L.orc_trial_uniforms.argtypes = [C.c_int, C.c_uint64, C.c_int64, C.c_int64, C.c_int64, P]
        L.orc_trial_uniforms.restype = None
        L.orc_hs_get_tables.argtypes = [P, P, P, P, P, P, P]
        L.orc_hs_collide.argtypes = [P, C.c_double, C.c_double, P, P, P]
        L.orc_step.argtypes = [P, C.c_int, C.c_double, C.c_int, C.c_double]
        L.orc_solve.argtypes = [C.c_int, P, P, P]
        L.orc_kn_local.argtypes = [P, C.c_double, P]
        L.orc_refine_project.argtypes = [P, P]
        L.orc_coarsen_project.argtypes = [P, P]
        L.orc_hermite_project.argtypes = [P, P, P, P]
        L.orc_hermite_target.argtypes = [P, P, P, P]
        L.orc_mlp_forward.argtypes = [C.c_int64, P, P, P]
        L.orc_mlp_backward.argtypes = [C.c_int64, P, P, P, P, P]
        L.orc_learned_collide.argtypes = [P, C.c_double, C.c_double, P, C.c_double, P, P]
        L.orc_learned_apply.argtypes = [P, C.c_double, C.c_double, P, P, C.c_double, P, P]
        L.orc_lattice_q.argtypes = [C.c_int]
        L.orc_lattice.argtypes = [C.c_int, P, P]
        L.orc_create_lattice.restype = P
        L.orc_create_lattice.argtypes = [C.POINTER(TreeSpec), C.c_int]
        L.orc_lbm_feq.argtypes = [P, C.c_double, P, P]
        L.orc_lbm_set_inflow.argtypes = [P, C.c_double, P]
        L.orc_lbm_init.argtypes = [P, P, P]
        L.orc_lbm_moments.argtypes = [P, P, P]
        L.orc_lbm_collide.argtypes = [P, C.c_double, C.c_double]
        L.orc_lbm_step.argtypes = [P, C.c_int, C.c_double, C.c_double]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def korobov_a(M):
    return int(lib().orc_korobov_a(int(M)))


def trial_uniforms(lattice, seed, i, k, M):
    u = np.zeros(5)
    lib().orc_trial_uniforms(int(lattice), int(seed), int(i), int(k), int(M), _p(u))
    return u


def lattice(kind):
    """(c [Q][3] as floats, w [Q]) of D2Q9 / D3Q19 / D3Q27 (Sec. 4)."""
    q = lib().orc_lattice_q(int(kind))
    if q < 0:
        raise ValueError("unknown lattice")
    c = np.zeros((q, 3))
    w = np.zeros(q)
    lib().orc_lattice(int(kind), _p(c), _p(w))
    return c, w


def threads():
    return int(lib().orc_threads())


def set_threads(n):
    """OpenMP threads of the oracle's later loops (for timing)."""
    lib().orc_set_threads(int(n))


def splitmix64(seed, n):
    return int(lib().orc_splitmix64(seed, n))


def vgrid(n, lo, hi):
    n = np.asarray(n, dtype=np.int32)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    nv = int(np.prod(n.astype(np.int64)))
    xi = np.zeros((nv, 3))
    k = np.zeros((nv, 3), dtype=np.int32)
    dV = np.zeros(1)
    if lib().orc_vgrid(_p(n), _p(lo), _p(hi), _p(xi), _p(k), _p(dV)):
        raise ValueError("bad velocity grid")
    return xi, k, float(dV[0])


def build_tree(spec):
    n = C.c_int64(0)
    rc = lib().orc_build_tree(C.byref(spec), 0, C.byref(n), None, None, None)
    if rc:
        raise ValueError("tree build failed %d" % rc)
    keys = np.zeros(n.value, dtype=np.uint64)
    lev = np.zeros(n.value, dtype=np.uint8)
    sol = np.zeros(n.value, dtype=np.uint8)
    rc = lib().orc_build_tree(C.byref(spec), n.value, C.byref(n), _p(keys), _p(lev), _p(sol))
    if rc:
        raise ValueError("tree build failed %d" % rc)
    return keys, lev, sol


MLP_NPARAM = 164672
MLP_SHAPES = [((256, 64), 256), ((256, 256), 256), ((256, 256), 256), ((64, 256), 64)]


def mlp_forward(params, x):
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 64)
    y = np.zeros_like(x)
    lib().orc_mlp_forward(x.shape[0], _p(params), _p(x), _p(y))
    return y


def mlp_backward(params, x, t):
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 64)
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1, 64)
    g = np.zeros(MLP_NPARAM)
    loss = np.zeros(1)
    lib().orc_mlp_backward(x.shape[0], _p(params), _p(x), _p(t), _p(g), _p(loss))
    return g, float(loss[0])


def solve(A, b):
    A = np.array(A, dtype=np.float64, order="C")
    b = np.array(b, dtype=np.float64)
    x = np.zeros_like(b)
    if lib().orc_solve(len(b), _p(A), _p(b), _p(x)):
        raise np.linalg.LinAlgError("singular")
    return x


class Problem:
    """One tree + velocity grid + state, all in FP64 on the host."""

    def __init__(self, spec, n=None, lo=None, hi=None, lattice=None, store_f=True):
        """store_f=False: no f storage (trees whose f does not fit in host
        memory); only the geometry, dt_cfl, set_freestream and the
        selected-cell calls (step_inputs, maxwellian_rows, step_cells) and
        the hard-sphere tables apply then."""
        self.spec = spec
        self.store_f = bool(store_f) and lattice is None
        if lattice is not None:
            # lattice Boltzmann (Sec. 4): the tree with an LBM velocity set
            self._h = lib().orc_create_lattice(C.byref(spec), int(lattice))
            if not self._h:
                raise ValueError("oracle lattice problem creation failed")
            self.lattice = int(lattice)
            self.nleaves = lib().orc_nleaves(self._h)
            self.ncells = lib().orc_ncells(self._h)
            self.nv = lib().orc_nv(self._h)
            self.xi, self.w = globals()["lattice"](lattice)
            self.dV = 1.0
            return
        self.lattice = None
        n = np.asarray(n, dtype=np.int32)
        lo = np.asarray(lo, dtype=np.float64)
        hi = np.asarray(hi, dtype=np.float64)
        create = lib().orc_create if store_f else lib().orc_create_sparse
        self._h = create(C.byref(spec), _p(n), _p(lo), _p(hi))
        if not self._h:
            raise ValueError("oracle problem creation failed")
        self.nleaves = lib().orc_nleaves(self._h)
        self.ncells = lib().orc_ncells(self._h)
        self.nv = lib().orc_nv(self._h)
        self.xi, self.k, self.dV = vgrid(n, lo, hi)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    def leaves(self):
        keys = np.zeros(self.nleaves, dtype=np.uint64)
        lev = np.zeros(self.nleaves, dtype=np.uint8)
        sol = np.zeros(self.nleaves, dtype=np.uint8)
        lib().orc_get_leaves(self._h, _p(keys), _p(lev), _p(sol))
        return keys, lev, sol

    def centres(self):
        xyz = np.zeros((self.ncells, 3))
        h = np.zeros(self.ncells)
        lib().orc_cell_centres(self._h, _p(xyz), _p(h))
        return xyz, h

    def faces(self):
        nf = lib().orc_n_faces(self._h)
        m = np.zeros(nf, dtype=np.int64)
        p = np.zeros(nf, dtype=np.int64)
        ax = np.zeros(nf, dtype=np.uint8)
        ar = np.zeros(nf)
        lib().orc_get_faces(self._h, _p(m), _p(p), _p(ax), _p(ar))
        return m, p, ax, ar

    def bfaces(self):
        nb = lib().orc_n_bfaces(self._h)
        leaf = np.zeros(nb, dtype=np.int64)
        ax = np.zeros(nb, dtype=np.uint8)
        side = np.zeros(nb, dtype=np.uint8)
        kind = np.zeros(nb, dtype=np.uint8)
        other = np.zeros(nb, dtype=np.int64)
        ar = np.zeros(nb)
        lib().orc_get_bfaces(self._h, _p(leaf), _p(ax), _p(side), _p(kind), _p(other), _p(ar))
        return leaf, ax, side, kind, other, ar

    def set_freestream(self, rho, u, T):
        u = np.asarray(u, dtype=np.float64)
        lib().orc_set_freestream(self._h, rho, _p(u), T)

    def init_maxwellian(self, w, rho, u, T):
        """w, rho, T: [ncells, nmix]; u: [ncells, nmix, 3]."""
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(self.ncells, -1))
        nmix = w.shape[1]
        rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(self.ncells, nmix))
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(self.ncells, nmix, 3))
        T = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(self.ncells, nmix))
        if lib().orc_init_maxwellian(self._h, nmix, _p(w), _p(rho), _p(u), _p(T)):
            raise RuntimeError("this problem holds no f")

    def refine_project(self, flags):
        """Split the flagged leaves, rebalance, carry f over (injection)."""
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        assert flags.size == self.nleaves
        if lib().orc_refine_project(self._h, _p(flags)):
            raise RuntimeError("refinement failed")
        self.nleaves = lib().orc_nleaves(self._h)
        self.ncells = lib().orc_ncells(self._h)

    def coarsen_project(self, flags):
        """Merge flagged sibling groups (2:1 balance kept), carry f over
        (the mean of the fluid children)."""
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        assert flags.size == self.nleaves
        if lib().orc_coarsen_project(self._h, _p(flags)):
            raise RuntimeError("coarsening failed")
        self.nleaves = lib().orc_nleaves(self._h)
        self.ncells = lib().orc_ncells(self._h)

    def get_f(self):
        f = np.zeros((self.ncells, self.nv))
        if lib().orc_get_f(self._h, _p(f)):
            raise RuntimeError("this problem holds no f")
        return f

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.ncells, self.nv)
        if lib().orc_set_f(self._h, _p(f)):
            raise RuntimeError("this problem holds no f")

    def step_inputs(self, cells):
        """The sorted distinct cells whose f one step of `cells` reads."""
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        k = lib().orc_step_inputs(self._h, cells.size, _p(cells), None)
        if k < 0:
            raise IndexError("cell index out of range")
        out = np.zeros(k, dtype=np.int64)
        lib().orc_step_inputs(self._h, cells.size, _p(cells), _p(out))
        return out

    def maxwellian_rows(self, w, rho, u, T):
        """Rows of the mixture init_maxwellian sets, for len(w) cells:
        w, rho, T [n, nmix], u [n, nmix, 3]."""
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
        n, nmix = w.shape
        rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(n, nmix))
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(n, nmix, 3))
        T = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(n, nmix))
        out = np.zeros((n, self.nv))
        lib().orc_maxwellian_rows(self._h, n, nmix, _p(w), _p(rho), _p(u), _p(T), _p(out))
        return out

    def step_cells(self, cells, inputs, fin, dt, coll, kn):
        """One step (transport, then the collision update coll: COLL_BGK, or
        COLL_HS with tables set) of `cells` from the rows fin of `inputs`
        (as step_inputs gives them)."""
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        inputs = np.ascontiguousarray(inputs, dtype=np.int64)
        fin = np.ascontiguousarray(fin, dtype=np.float64).reshape(inputs.size, self.nv)
        out = np.zeros((cells.size, self.nv))
        if lib().orc_step_cells(self._h, cells.size, _p(cells), inputs.size, _p(inputs), _p(fin),
                                float(dt), int(coll), float(kn), _p(out)):
            raise RuntimeError("selected-cell step failed")
        return out

    def step_cells_learned(self, cells, inputs, fin, dt, kn, params, threshold):
        """One learned step (transport, then the learned update with the
        hard-sphere fallback) of `cells` from the rows fin of `inputs`, which
        must cover two rings of face neighbours.  Returns (rows, local Kn,
        used flags) of the cells."""
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        inputs = np.ascontiguousarray(inputs, dtype=np.int64)
        fin = np.ascontiguousarray(fin, dtype=np.float64).reshape(inputs.size, self.nv)
        params = np.ascontiguousarray(params, dtype=np.float64)
        out = np.zeros((cells.size, self.nv))
        knl = np.zeros(cells.size)
        used = np.zeros(cells.size, dtype=np.int32)
        if lib().orc_step_cells_learned(self._h, cells.size, _p(cells), inputs.size, _p(inputs), _p(fin), float(dt),
                                        float(kn), _p(params), float(threshold), _p(knl), _p(used), _p(out)):
            raise RuntimeError("selected-cell learned step failed")
        return out, knl, used

    def dt_cfl(self, cfl):
        return lib().orc_dt_cfl(self._h, cfl)

    def transport(self, dt):
        if lib().orc_transport(self._h, dt):
            raise RuntimeError("transport failed")

    def moments(self):
        rho = np.zeros(self.ncells)
        u = np.zeros((self.ncells, 3))
        T = np.zeros(self.ncells)
        lib().orc_moments(self._h, _p(rho), _p(u), _p(T))
        return rho, u, T

    def totals(self):
        out = np.zeros(5)
        lib().orc_totals(self._h, _p(out))
        return out

    # ---- lattice Boltzmann (Sec. 4)
    def lbm_feq(self, rho, u):
        u = np.asarray(u, dtype=np.float64)
        out = np.zeros(self.nv)
        assert lib().orc_lbm_feq(self._h, float(rho), _p(u), _p(out)) == 0
        return out

    def lbm_set_inflow(self, rho, u):
        u = np.asarray(u, dtype=np.float64)
        assert lib().orc_lbm_set_inflow(self._h, float(rho), _p(u)) == 0

    def lbm_init(self, rho, u):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.ncells)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.ncells, 3)
        assert lib().orc_lbm_init(self._h, _p(rho), _p(u)) == 0

    def lbm_moments(self):
        rho = np.zeros(self.ncells)
        u = np.zeros((self.ncells, 3))
        lib().orc_lbm_moments(self._h, _p(rho), _p(u))
        return rho, u

    def lbm_collide(self, dt, tau):
        if lib().orc_lbm_collide(self._h, dt, tau):
            raise RuntimeError("LBM collision failed (non-positive density)")

    def lbm_step(self, nsteps, dt, tau):
        rc = lib().orc_lbm_step(self._h, int(nsteps), dt, tau)
        if rc:
            raise RuntimeError("LBM step failed (%d)" % rc)

    def bgk(self, dt, kn, want_q=False):
        q = np.zeros((self.ncells, self.nv)) if want_q else None
        if lib().orc_bgk(self._h, dt, kn, _p(q)):
            raise RuntimeError("BGK failed (non-positive moments or singular system)")
        return q

    def bgk_entropic(self, dt, kn, want_q=False):
        q = np.zeros((self.ncells, self.nv)) if want_q else None
        if lib().orc_bgk_entropic(self._h, dt, kn, _p(q)):
            raise RuntimeError("entropic BGK failed (non-positive moments or no Newton convergence)")
        return q

    def hs_tables(self, trials, seed, lattice=False):
        if lattice:
            assert lib().orc_hs_tables_lattice(self._h, trials, seed) == 0
        else:
            lib().orc_hs_tables(self._h, trials, seed)

    def hs_get_tables(self):
        nk = lib().orc_hs_nkept(self._h)
        start = np.zeros(self.nv + 1, dtype=np.int64)
        gam = np.zeros(nk, dtype=np.int32)
        l = np.zeros(nk, dtype=np.int32)
        m = np.zeros(nk, dtype=np.int32)
        b = np.zeros(nk)
        disc = np.zeros(1, dtype=np.int64)
        if lib().orc_hs_get_tables(self._h, _p(start), _p(gam), _p(l), _p(m), _p(b), _p(disc)):
            raise RuntimeError("no tables")
        return start, gam, l, m, b, int(disc[0])

    def hs_collide(self, dt, kn, want=False):
        q = np.zeros((self.ncells, self.nv)) if want else None
        B = np.zeros((self.ncells, self.nv)) if want else None
        Cc = np.zeros((self.ncells, self.nv)) if want else None
        if lib().orc_hs_collide(self._h, dt, kn, _p(q), _p(B), _p(Cc)):
            raise RuntimeError("hard-sphere collision failed")
        return q, B, Cc

    def kn_local(self, kn):
        out = np.zeros(self.ncells)
        lib().orc_kn_local(self._h, kn, _p(out))
        return out

    def hermite_project(self, f=None):
        a = np.zeros((self.ncells, 64))
        mom = np.zeros((self.ncells, 5))
        ff = None if f is None else np.ascontiguousarray(f, dtype=np.float64)
        lib().orc_hermite_project(self._h, _p(ff), _p(a), _p(mom))
        return a, mom

    def hermite_target(self, I, mom):
        o = np.zeros((self.ncells, 64))
        I = np.ascontiguousarray(I, dtype=np.float64)
        mom = np.ascontiguousarray(mom, dtype=np.float64)
        lib().orc_hermite_target(self._h, _p(I), _p(mom), _p(o))
        return o

    def learned_collide(self, dt, kn, params, threshold, want_q=False):
        params = np.ascontiguousarray(params, dtype=np.float64)
        used = np.zeros(self.ncells, dtype=np.int32)
        q = np.zeros((self.ncells, self.nv)) if want_q else None
        if lib().orc_learned_collide(self._h, dt, kn, _p(params), threshold, _p(used), _p(q)):
            raise RuntimeError("learned collision failed")
        return used, q

    def learned_apply(self, dt, kn, knl, o, threshold, want_q=False):
        knl = np.ascontiguousarray(knl, dtype=np.float64)
        o = np.ascontiguousarray(o, dtype=np.float64).reshape(self.ncells, 64)
        used = np.zeros(self.ncells, dtype=np.int32)
        q = np.zeros((self.ncells, self.nv)) if want_q else None
        if lib().orc_learned_apply(self._h, dt, kn, _p(knl), _p(o), threshold, _p(used), _p(q)):
            raise RuntimeError("learned collision failed")
        return used, q

    def step(self, nsteps, dt, coll, kn):
        rc = lib().orc_step(self._h, nsteps, dt, coll, kn)
        if rc:
            raise RuntimeError("oracle step failed %d" % rc)
