"""Python binding of libdvm: argument marshalling over the C ABI in include/dvm.h.

Every step of the DVM path runs in the library's CUDA kernels; this module only
loads libdvm.so (built in-tree by `_build.py`), converts numpy/torch buffers to
pointers and raises on error codes.  There is no CPU fallback: if the shared
library is missing or no CUDA device is present, construction raises.

Paper: Zabelok, Arslanbekov, Kolobov, "Adaptive Kinetic-Fluid Solvers for
Heterogeneous Computing Architectures" (Sec. 2.1 tree mesh, Sec. 3 DVM,
Sec. 3.1 Eq. 2 advection, Sec. 3.2 Eqs. 3-6 collision integral).
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdvm.so")

F64, F32, BF16 = 0, 1, 2
COLL_NONE, COLL_BGK, COLL_HS, COLL_LEARNED, COLL_BGK_ENTROPIC = 0, 1, 2, 3, 4
LBM_D2Q9, LBM_D3Q19, LBM_D3Q27 = 9, 19, 27
BC_PERIODIC, BC_INFLOW, BC_OUTFLOW, BC_WALL = 0, 1, 2, 3
PRED_NONE, PRED_BALL, PRED_SHELL = 0, 1, 2

STATUS = {0: "DVM_OK", -1: "DVM_EINVAL", -2: "DVM_ENOMEM", -3: "DVM_ECUDA", -4: "DVM_ESTATE",
          -5: "DVM_EUNSTABLE", -6: "DVM_EBOUNDS", -7: "DVM_ETIMEOUT", -9: "DVM_ENOTIMPL"}

# every entry point declared in include/dvm.h
EXPORTS = [
    "dvm_create", "dvm_destroy", "dvm_last_error", "dvm_set_stream", "dvm_set_allocator",
    "dvm_build_tree", "dvm_refine", "dvm_get_counts", "dvm_get_leaves", "dvm_get_faces",
    "dvm_get_bfaces", "dvm_cell_centres", "dvm_set_velocity_grid", "dvm_get_velocities",
    "dvm_set_freestream", "dvm_init_maxwellian", "dvm_get_f", "dvm_get_f_rows", "dvm_set_f", "dvm_upload_f",
    "dvm_download_f", "dvm_f_device", "dvm_dt_cfl", "dvm_set_collision_tables", "dvm_step",
    "dvm_moments", "dvm_step_moments", "dvm_launch_count", "dvm_get_collision_tables",
    "dvm_hs_collide_noalloc", "dvm_learned_set_weights", "dvm_learned_get_weights",
    "dvm_mlp_forward", "dvm_mlp_loss_grad", "dvm_learned_train", "dvm_learned_configure",
    "dvm_learned_collide", "dvm_learned_pairs", "dvm_learned_fallback_count",
    "dvm_partition_info", "dvm_step_partitioned", "dvm_set_collision_tables_lattice",
    "dvm_refine_project", "dvm_lbm_set_lattice", "dvm_lbm_get_velocities", "dvm_lbm_info",
    "dvm_lbm_set_inflow", "dvm_lbm_init_equilibrium", "dvm_lbm_set_f", "dvm_lbm_get_f",
    "dvm_lbm_dt_cfl", "dvm_lbm_step", "dvm_lbm_moments", "dvm_lbm_get_codes",
    "dvm_coarsen", "dvm_coarsen_project", "dvm_kn_local", "dvm_flag_kinetic",
    "dvm_partition_weighted", "dvm_lbm_lattice", "dvm_step_residual", "dvm_set_timing",
    "dvm_step_timing", "dvm_rank_create", "dvm_rank_destroy", "dvm_rank_last_error", "dvm_rank_info",
    "dvm_rank_plan", "dvm_rank_set_stream", "dvm_rank_set_velocity_grid", "dvm_rank_set_freestream",
    "dvm_rank_cell_centres", "dvm_rank_init_maxwellian", "dvm_rank_row_bytes", "dvm_rank_pack",
    "dvm_rank_unpack", "dvm_rank_dt_cfl", "dvm_rank_step", "dvm_rank_moments", "dvm_rank_get_f",
    "dvm_rank_totals",
]
MLP_NPARAM = 164672
HS_NOALLOC_SCRATCH_BYTES = 64 << 20


class DvmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class Config(C.Structure):
    _fields_ = [("precision", C.c_int), ("collision", C.c_int), ("kn", C.c_double)]


class TreeSpec(C.Structure):
    _fields_ = [("dim", C.c_int), ("base_level", C.c_int), ("max_level", C.c_int),
                ("pred", C.c_int), ("c", C.c_double * 3), ("r", C.c_double),
                ("beta", C.c_double), ("solid", C.c_int), ("bc", C.c_int * 6)]


def tree_spec(dim, base_level, max_level, pred=PRED_NONE, c=(0.5, 0.5, 0.5), r=0.0,
              beta=0.0, solid=0, bc=(0,) * 6):
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
    """Load libdvm.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libdvm.so not built: run __graft_entry__.build() "
                              "(or python -m paper_1503_00707_gb300._build)")
        L = C.CDLL(LIB_PATH)
        P, i64, d = C.c_void_p, C.c_int64, C.c_double
        sig = {
            "dvm_create": [C.POINTER(P), C.POINTER(Config)],
            "dvm_destroy": [P],
            "dvm_last_error": [P],
            "dvm_set_stream": [P, P],
            "dvm_set_allocator": [P, P, P, P],
            "dvm_build_tree": [P, C.POINTER(TreeSpec)],
            "dvm_refine": [P, P, i64],
            "dvm_get_counts": [P, P, P, P, P, P],
            "dvm_get_leaves": [P, P, P, P],
            "dvm_get_faces": [P, P, P, P, P],
            "dvm_get_bfaces": [P, P, P, P, P, P, P],
            "dvm_cell_centres": [P, P, P],
            "dvm_set_velocity_grid": [P, P, P, P],
            "dvm_get_velocities": [P, P],
            "dvm_set_freestream": [P, d, P, d],
            "dvm_init_maxwellian": [P, C.c_int, P, P, P, P],
            "dvm_get_f": [P, P, i64],
            "dvm_get_f_rows": [P, i64, P, P],
            "dvm_set_f": [P, P, i64],
            "dvm_upload_f": [P, P, i64],
            "dvm_download_f": [P, P, i64],
            "dvm_f_device": [P, P, P],
            "dvm_dt_cfl": [P, d, P],
            "dvm_set_collision_tables": [P, C.c_int, C.c_uint64],
            "dvm_step": [P, C.c_int, d],
            "dvm_moments": [P, P, P, P],
            "dvm_step_moments": [P, P, P, P],
            "dvm_launch_count": [P],
            "dvm_get_collision_tables": [P, P, P, P, P, P],
            "dvm_hs_collide_noalloc": [P, P, i64, d],
            "dvm_learned_set_weights": [P, P],
            "dvm_learned_get_weights": [P, P],
            "dvm_mlp_forward": [P, P, i64, P],
            "dvm_mlp_loss_grad": [P, P, P, i64, P, P],
            "dvm_learned_train": [P, P, P, i64, C.c_int, C.c_int, d, C.c_uint64, P],
            "dvm_learned_configure": [P, d],
            "dvm_learned_collide": [P, d, P, P, P, P, P, P],
            "dvm_learned_pairs": [P, P, P],
            "dvm_learned_fallback_count": [P, P],
            "dvm_partition_info": [P, C.c_int, C.c_int, P, P, P, P, i64],
            "dvm_step_partitioned": [P, C.c_int, C.c_int, d],
            "dvm_set_collision_tables_lattice": [P, C.c_int, C.c_uint64],
            "dvm_refine_project": [P, P, i64],
            "dvm_lbm_set_lattice": [P, C.c_int],
            "dvm_lbm_get_velocities": [P, P, P],
            "dvm_lbm_info": [P, P, P, P],
            "dvm_lbm_set_inflow": [P, d, P],
            "dvm_lbm_init_equilibrium": [P, P, P],
            "dvm_lbm_set_f": [P, P, i64],
            "dvm_lbm_get_f": [P, P, i64],
            "dvm_lbm_dt_cfl": [P, d, P],
            "dvm_lbm_step": [P, C.c_int, d, d],
            "dvm_lbm_moments": [P, P, P],
            "dvm_lbm_get_codes": [P, P, P, P],
            "dvm_coarsen": [P, P, i64],
            "dvm_coarsen_project": [P, P, i64],
            "dvm_kn_local": [P, P],
            "dvm_flag_kinetic": [P, d, P, P],
            "dvm_partition_weighted": [P, C.c_int, P, C.c_int, P, P, P, P, i64],
            "dvm_lbm_lattice": [C.c_int, P, P, P],
            "dvm_step_residual": [P, P],
            "dvm_set_timing": [P, C.c_int],
            "dvm_step_timing": [P, P, P],
            "dvm_rank_create": [C.POINTER(P), C.POINTER(Config), C.POINTER(TreeSpec), C.c_int, C.c_int],
            "dvm_rank_destroy": [P],
            "dvm_rank_last_error": [P],
            "dvm_rank_info": [P, P, P, P, P],
            "dvm_rank_plan": [P, C.c_int, P, P, P, P],
            "dvm_rank_set_stream": [P, P],
            "dvm_rank_set_velocity_grid": [P, P, P, P],
            "dvm_rank_set_freestream": [P, d, P, d],
            "dvm_rank_cell_centres": [P, P, P],
            "dvm_rank_init_maxwellian": [P, C.c_int, P, P, P, P],
            "dvm_rank_row_bytes": [P, P],
            "dvm_rank_pack": [P, C.c_int, P],
            "dvm_rank_unpack": [P, C.c_int, P],
            "dvm_rank_dt_cfl": [P, d, P],
            "dvm_rank_step": [P, d],
            "dvm_rank_moments": [P, P, P, P],
            "dvm_rank_get_f": [P, P, i64],
            "dvm_rank_totals": [P, P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.dvm_destroy.restype = None
        L.dvm_last_error.restype = C.c_char_p
        L.dvm_rank_destroy.restype = None
        L.dvm_rank_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _p(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


class Solver:
    """One DVM problem on the current CUDA device (thin wrapper over dvm_ctx)."""

    def __init__(self, precision=F32, collision=COLL_BGK, kn=0.1, stream=None):
        L = lib()
        cfg = Config(precision, collision, kn)
        h = C.c_void_p()
        rc = L.dvm_create(C.byref(h), C.byref(cfg))
        if rc:
            raise DvmError(rc, "dvm_create failed (bad config)")
        self._h = h
        self.precision = precision
        self.collision = collision
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "_h", None):
            lib().dvm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc):
        if rc:
            msg = lib().dvm_last_error(self._h)
            raise DvmError(rc, msg.decode() if msg else "")

    # ---- setup
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None."""
        handle = getattr(stream, "cuda_stream", stream)
        self._chk(lib().dvm_set_stream(self._h, C.c_void_p(handle or 0)))

    def build_tree(self, spec):
        self._chk(lib().dvm_build_tree(self._h, C.byref(spec)))
        self.dim = spec.dim
        self.counts()

    def coarsen(self, flags):
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        self._chk(lib().dvm_coarsen(self._h, _p(flags), len(flags)))
        self.counts()

    def coarsen_project(self, flags):
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        self._chk(lib().dvm_coarsen_project(self._h, _p(flags), len(flags)))
        self.counts()

    def kn_local(self):
        knl = np.zeros(self.ncells)
        self._chk(lib().dvm_kn_local(self._h, _p(knl)))
        return knl

    def flag_kinetic(self, threshold):
        flags = np.zeros(self.ncells, dtype=np.uint8)
        n = C.c_int64()
        self._chk(lib().dvm_flag_kinetic(self._h, float(threshold), _p(flags), C.byref(n)))
        return flags, n.value

    def refine(self, flags):
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        self._chk(lib().dvm_refine(self._h, _p(flags), len(flags)))
        self.counts()

    def refine_project(self, flags):
        """Refine and carry f over (children take their parent's f)."""
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        self._chk(lib().dvm_refine_project(self._h, _p(flags), len(flags)))
        self.counts()

    def counts(self):
        v = [C.c_int64() for _ in range(5)]
        self._chk(lib().dvm_get_counts(self._h, *[C.byref(x) for x in v]))
        self.nleaves, self.ncells, self.nfaces, self.nbfaces, self.nv = [x.value for x in v]
        return self.nleaves, self.ncells, self.nfaces, self.nbfaces, self.nv

    def leaves(self):
        n = self.nleaves
        keys, lev, sol = np.zeros(n, np.uint64), np.zeros(n, np.uint8), np.zeros(n, np.uint8)
        self._chk(lib().dvm_get_leaves(self._h, _p(keys), _p(lev), _p(sol)))
        return keys, lev, sol

    def faces(self):
        n = self.nfaces
        m, p, ax, ar = np.zeros(n, np.int64), np.zeros(n, np.int64), np.zeros(n, np.uint8), np.zeros(n)
        self._chk(lib().dvm_get_faces(self._h, _p(m), _p(p), _p(ax), _p(ar)))
        return m, p, ax, ar

    def bfaces(self):
        n = self.nbfaces
        leaf, ax, side, kind = np.zeros(n, np.int64), np.zeros(n, np.uint8), np.zeros(n, np.uint8), np.zeros(n, np.uint8)
        other, ar = np.zeros(n, np.int64), np.zeros(n)
        self._chk(lib().dvm_get_bfaces(self._h, _p(leaf), _p(ax), _p(side), _p(kind), _p(other), _p(ar)))
        return leaf, ax, side, kind, other, ar

    def centres(self):
        xyz, h = np.zeros((self.ncells, 3)), np.zeros(self.ncells)
        self._chk(lib().dvm_cell_centres(self._h, _p(xyz), _p(h)))
        return xyz, h

    def set_velocity_grid(self, n, lo, hi):
        n = np.ascontiguousarray(n, dtype=np.int32)
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        self._chk(lib().dvm_set_velocity_grid(self._h, _p(n), _p(lo), _p(hi)))
        self.counts()

    def velocities(self):
        xi = np.zeros((self.nv, 3))
        self._chk(lib().dvm_get_velocities(self._h, _p(xi)))
        return xi

    def set_freestream(self, rho, u, T):
        u = np.ascontiguousarray(u, dtype=np.float64)
        self._chk(lib().dvm_set_freestream(self._h, float(rho), _p(u), float(T)))

    def init_maxwellian(self, w, rho, u, T):
        nc = self.ncells
        w = np.ascontiguousarray(np.asarray(w, np.float64).reshape(nc, -1))
        k = w.shape[1]
        rho = np.ascontiguousarray(np.asarray(rho, np.float64).reshape(nc, k))
        u = np.ascontiguousarray(np.asarray(u, np.float64).reshape(nc, k, 3))
        T = np.ascontiguousarray(np.asarray(T, np.float64).reshape(nc, k))
        self._chk(lib().dvm_init_maxwellian(self._h, k, _p(w), _p(rho), _p(u), _p(T)))

    def set_collision_tables(self, trials, seed, lattice=False):
        fn = lib().dvm_set_collision_tables_lattice if lattice else lib().dvm_set_collision_tables
        self._chk(fn(self._h, int(trials), int(seed)))

    def collision_tables(self, trials):
        n = self.nv * trials
        gam, l, m = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int32)
        b = np.zeros(n, np.float32)
        disc = C.c_int64()
        self._chk(lib().dvm_get_collision_tables(self._h, _p(gam), _p(l), _p(m), _p(b), C.byref(disc)))
        return gam, l, m, b, disc.value

    def hs_collide_noalloc(self, f_dev_ptr, ncells, dt):
        """Collision update of caller-owned device f (FP32) with no device
        allocation; f_dev_ptr is an integer device address."""
        self._chk(lib().dvm_hs_collide_noalloc(self._h, C.c_void_p(f_dev_ptr), int(ncells), float(dt)))

    # ---- learned operator network
    def set_weights(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        assert params.size == MLP_NPARAM
        self._chk(lib().dvm_learned_set_weights(self._h, _p(params)))

    def get_weights(self):
        out = np.zeros(MLP_NPARAM, np.float32)
        self._chk(lib().dvm_learned_get_weights(self._h, _p(out)))
        return out

    def mlp_forward(self, x):
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 64)
        y = np.zeros_like(x)
        self._chk(lib().dvm_mlp_forward(self._h, _p(x), x.shape[0], _p(y)))
        return y

    def mlp_loss_grad(self, x, t, want_grad=True):
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 64)
        t = np.ascontiguousarray(t, dtype=np.float32).reshape(-1, 64)
        g = np.zeros(MLP_NPARAM, np.float32) if want_grad else None
        loss = C.c_double()
        self._chk(lib().dvm_mlp_loss_grad(self._h, _p(x), _p(t), x.shape[0], _p(g), C.byref(loss)))
        return loss.value, g

    def train(self, x, t, epochs, batch, lr, seed=0):
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 64)
        t = np.ascontiguousarray(t, dtype=np.float32).reshape(-1, 64)
        loss = C.c_double()
        self._chk(lib().dvm_learned_train(self._h, _p(x), _p(t), x.shape[0], int(epochs), int(batch),
                                          float(lr), int(seed), C.byref(loss)))
        return loss.value

    # ---- learned collision
    def learned_configure(self, kn_threshold):
        self._chk(lib().dvm_learned_configure(self._h, float(kn_threshold)))

    def learned_collide(self, dt, o=None, want=("knl", "a", "o", "used", "q")):
        """One learned collision update of the stored f; returns the requested
        intermediates (knl, a, o, used, q) as numpy arrays."""
        nc, nv = self.ncells, self.nv
        o_in = None if o is None else np.ascontiguousarray(o, dtype=np.float32).reshape(nc, 64)
        out = {
            "knl": np.zeros(nc) if "knl" in want else None,
            "a": np.zeros((nc, 64), np.float32) if "a" in want else None,
            "o": np.zeros((nc, 64), np.float32) if "o" in want else None,
            "used": np.zeros(nc, np.int32) if "used" in want else None,
            "q": np.zeros((nc, nv), np.float32) if "q" in want else None,
        }
        self._chk(lib().dvm_learned_collide(self._h, float(dt), _p(o_in), _p(out["knl"]), _p(out["a"]),
                                            _p(out["o"]), _p(out["used"]), _p(out["q"])))
        return {k: v for k, v in out.items() if v is not None}

    def learned_pairs(self):
        a = np.zeros((self.ncells, 64), np.float32)
        o = np.zeros((self.ncells, 64), np.float32)
        self._chk(lib().dvm_learned_pairs(self._h, _p(a), _p(o)))
        return a, o

    def learned_fallback_count(self):
        n = C.c_int64()
        self._chk(lib().dvm_learned_fallback_count(self._h, C.byref(n)))
        return n.value

    # ---- Morton-range partition
    def partition_info(self, nparts, part):
        """(c0, c1, ghosts): the owned cell range of `part` and its halo."""
        c0, c1, ng = C.c_int64(), C.c_int64(), C.c_int64()
        self._chk(lib().dvm_partition_info(self._h, int(nparts), int(part), C.byref(c0), C.byref(c1),
                                           C.byref(ng), None, 0))
        g = np.zeros(ng.value, np.int64)
        self._chk(lib().dvm_partition_info(self._h, int(nparts), int(part), None, None, None, _p(g), g.size))
        return c0.value, c1.value, g

    def partition_weighted(self, nparts, part, weights):
        """(c0, c1, ghosts) of `part` for ranges of equal total weight."""
        w = np.ascontiguousarray(weights, dtype=np.float64)
        c0, c1, ng = C.c_int64(), C.c_int64(), C.c_int64()
        self._chk(lib().dvm_partition_weighted(self._h, int(nparts), _p(w), int(part), C.byref(c0), C.byref(c1),
                                               C.byref(ng), None, 0))
        g = np.zeros(ng.value, np.int64)
        self._chk(lib().dvm_partition_weighted(self._h, int(nparts), _p(w), int(part), None, None, None, _p(g),
                                               g.size))
        return c0.value, c1.value, g

    def step_partitioned(self, nparts, nsteps, dt):
        self._chk(lib().dvm_step_partitioned(self._h, int(nparts), int(nsteps), float(dt)))

    # ---- state
    def get_f(self):
        f = np.zeros((self.ncells, self.nv))
        self._chk(lib().dvm_get_f(self._h, _p(f), f.size))
        return f

    def get_f_rows(self, cells):
        """f of the given cells, [len(cells), nv] FP64, gathered on the device."""
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros((cells.size, self.nv))
        self._chk(lib().dvm_get_f_rows(self._h, cells.size, _p(cells), _p(out)))
        return out

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.ncells, self.nv)
        self._chk(lib().dvm_set_f(self._h, _p(f), f.size))

    def f_bytes(self):
        ptr, nb = C.c_void_p(), C.c_int64()
        self._chk(lib().dvm_f_device(self._h, C.byref(ptr), C.byref(nb)))
        return nb.value

    def f_device_ptr(self):
        ptr, nb = C.c_void_p(), C.c_int64()
        self._chk(lib().dvm_f_device(self._h, C.byref(ptr), C.byref(nb)))
        return ptr.value, nb.value

    def upload_f(self, host_ptr, nbytes):
        """host_ptr: integer address of host memory in the storage format."""
        self._chk(lib().dvm_upload_f(self._h, C.c_void_p(host_ptr), int(nbytes)))

    def download_f(self, host_ptr, nbytes):
        self._chk(lib().dvm_download_f(self._h, C.c_void_p(host_ptr), int(nbytes)))

    def dt_cfl(self, cfl):
        dt = C.c_double()
        self._chk(lib().dvm_dt_cfl(self._h, float(cfl), C.byref(dt)))
        return dt.value

    def step(self, nsteps, dt):
        self._chk(lib().dvm_step(self._h, int(nsteps), float(dt)))

    def moments(self):
        rho, u, T = np.zeros(self.ncells), np.zeros((self.ncells, 3)), np.zeros(self.ncells)
        self._chk(lib().dvm_moments(self._h, _p(rho), _p(u), _p(T)))
        return rho, u, T

    def step_moments(self, out=None):
        """Moments of the last step's f*; `out` (optional) is a (rho, u, T) tuple
        of preallocated float64 arrays."""
        if out is None:
            out = (np.zeros(self.ncells), np.zeros((self.ncells, 3)), np.zeros(self.ncells))
        self._chk(lib().dvm_step_moments(self._h, *[_p(a) for a in out]))
        return out

    def step_residual(self):
        """[ncells][5] conservation residual sum_i psi_r q_i dV of the last
        collision update, psi = (1, xi, |xi|^2) (see dvm_step_residual)."""
        out = np.zeros((self.ncells, 5))
        self._chk(lib().dvm_step_residual(self._h, _p(out)))
        return out

    def set_timing(self, enable=True):
        self._chk(lib().dvm_set_timing(self._h, int(bool(enable))))

    def step_timing(self):
        """(ms[3] per phase: transport, collision, fallback; steps), reset after reading."""
        ms = np.zeros(3)
        n = C.c_int64()
        self._chk(lib().dvm_step_timing(self._h, _p(ms), C.byref(n)))
        return ms, n.value

    # ---- lattice Boltzmann (Sec. 4)
    def lbm_set_lattice(self, lattice):
        self._chk(lib().dvm_lbm_set_lattice(self._h, int(lattice)))
        q = C.c_int()
        self._chk(lib().dvm_lbm_info(self._h, C.byref(q), None, None))
        self.q = q.value

    def lbm_codes(self):
        """(codes [2 dim][ncells] uint32, overflow entries) of the current tree
        (host work, no device needed)."""
        no = C.c_int64()
        self._chk(lib().dvm_lbm_get_codes(self._h, None, None, C.byref(no)))
        dim = self.dim
        codes = np.zeros((2 * dim, self.ncells), dtype=np.uint32)
        ovf = np.zeros(max(no.value, 1), dtype=np.uint32)
        self._chk(lib().dvm_lbm_get_codes(self._h, _p(codes), _p(ovf), C.byref(no)))
        return codes, ovf[:no.value]

    def lbm_velocities(self):
        c = np.zeros((self.q, 3), dtype=np.int32)
        w = np.zeros(self.q)
        self._chk(lib().dvm_lbm_get_velocities(self._h, _p(c), _p(w)))
        return c, w

    def lbm_info(self):
        """(q, row stride ld of the device f, overflow upwind entries)"""
        q, ld, no = C.c_int(), C.c_int64(), C.c_int64()
        self._chk(lib().dvm_lbm_info(self._h, C.byref(q), C.byref(ld), C.byref(no)))
        return q.value, ld.value, no.value

    def lbm_set_inflow(self, rho, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        self._chk(lib().dvm_lbm_set_inflow(self._h, float(rho), _p(u)))

    def lbm_init(self, rho, u):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.ncells)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.ncells, 3)
        self._chk(lib().dvm_lbm_init_equilibrium(self._h, _p(rho), _p(u)))

    def lbm_set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.ncells, self.q)
        self._chk(lib().dvm_lbm_set_f(self._h, _p(f), f.size))

    def lbm_get_f(self):
        f = np.zeros((self.ncells, self.q))
        self._chk(lib().dvm_lbm_get_f(self._h, _p(f), f.size))
        return f

    def lbm_dt_cfl(self, cfl):
        dt = C.c_double()
        self._chk(lib().dvm_lbm_dt_cfl(self._h, float(cfl), C.byref(dt)))
        return dt.value

    def lbm_step(self, nsteps, dt, tau):
        self._chk(lib().dvm_lbm_step(self._h, int(nsteps), float(dt), float(tau)))

    def lbm_moments(self):
        rho, u = np.zeros(self.ncells), np.zeros((self.ncells, 3))
        self._chk(lib().dvm_lbm_moments(self._h, _p(rho), _p(u)))
        return rho, u

    @staticmethod
    def launch_count():
        n = C.c_int64()
        rc = lib().dvm_launch_count(C.byref(n))
        if rc:
            raise DvmError(rc, "dvm_launch_count")
        return n.value


class Rank:
    """One rank of the Morton-range partition (dvm_rank_*): the rank's own
    cells, its halo and the inflow ghost on the current device.  Host arrays
    of cells cover the owned cells in order."""

    def __init__(self, cfg, precision, collision, nparts, part, kn=None, device=True, stream=None):
        prec = {"f64": F64, "f32": F32, "bf16": BF16}[precision] if isinstance(precision, str) else precision
        L = lib()
        h = C.c_void_p()
        conf = Config(prec, collision, cfg["kn"] if kn is None else kn)
        spec = tree_spec(cfg["dim"], cfg["base_level"], cfg["max_level"], cfg["pred"], cfg["c"], cfg["r"],
                         cfg["beta"], cfg["solid"], cfg["bc"])
        rc = L.dvm_rank_create(C.byref(h), C.byref(conf), C.byref(spec), int(nparts), int(part))
        if rc:
            raise DvmError(rc, "dvm_rank_create failed")
        self._h = h
        self.nparts, self.part = nparts, part
        v = [C.c_int64() for _ in range(4)]
        self._chk(L.dvm_rank_info(h, *[C.byref(x) for x in v]))
        self.ncells_global, self.c0, self.c1, self.nhalo = [x.value for x in v]
        self.ncells = self.c1 - self.c0
        if stream is not None:
            self._chk(L.dvm_rank_set_stream(h, C.c_void_p(getattr(stream, "cuda_stream", stream) or 0)))
        if device:
            n = np.ascontiguousarray(cfg["n"], dtype=np.int32)
            lo = np.ascontiguousarray(cfg["lo"], dtype=np.float64)
            hi = np.ascontiguousarray(cfg["hi"], dtype=np.float64)
            self._chk(L.dvm_rank_set_velocity_grid(h, _p(n), _p(lo), _p(hi)))
            u = np.ascontiguousarray(cfg["fs_u"], dtype=np.float64)
            self._chk(L.dvm_rank_set_freestream(h, float(cfg["fs_rho"]), _p(u), float(cfg["fs_T"])))
            self.nv = int(n[0]) * int(n[1]) * int(n[2])
            rb = C.c_int64()
            self._chk(L.dvm_rank_row_bytes(h, C.byref(rb)))
            self.row_bytes = rb.value

    def close(self):
        if getattr(self, "_h", None):
            lib().dvm_rank_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc):
        if rc:
            msg = lib().dvm_rank_last_error(self._h)
            raise DvmError(rc, msg.decode() if msg else "")

    def plan(self, peer):
        """(send_cells, recv_cells): ascending global indices exchanged with `peer`."""
        ns, nr = C.c_int64(), C.c_int64()
        self._chk(lib().dvm_rank_plan(self._h, int(peer), C.byref(ns), None, C.byref(nr), None))
        s, r = np.zeros(ns.value, np.int64), np.zeros(nr.value, np.int64)
        self._chk(lib().dvm_rank_plan(self._h, int(peer), None, _p(s), None, _p(r)))
        return s, r

    def centres(self):
        xyz, h = np.zeros((self.ncells, 3)), np.zeros(self.ncells)
        self._chk(lib().dvm_rank_cell_centres(self._h, _p(xyz), _p(h)))
        return xyz, h

    def init_maxwellian(self, w, rho, u, T):
        nc = self.ncells
        w = np.ascontiguousarray(np.asarray(w, np.float64).reshape(nc, -1))
        k = w.shape[1]
        rho = np.ascontiguousarray(np.asarray(rho, np.float64).reshape(nc, k))
        u = np.ascontiguousarray(np.asarray(u, np.float64).reshape(nc, k, 3))
        T = np.ascontiguousarray(np.asarray(T, np.float64).reshape(nc, k))
        self._chk(lib().dvm_rank_init_maxwellian(self._h, k, _p(w), _p(rho), _p(u), _p(T)))

    def pack(self, peer, dev_ptr):
        self._chk(lib().dvm_rank_pack(self._h, int(peer), C.c_void_p(dev_ptr)))

    def unpack(self, peer, dev_ptr):
        self._chk(lib().dvm_rank_unpack(self._h, int(peer), C.c_void_p(dev_ptr)))

    def dt_cfl(self, cfl):
        dt = C.c_double()
        self._chk(lib().dvm_rank_dt_cfl(self._h, float(cfl), C.byref(dt)))
        return dt.value

    def step(self, dt):
        self._chk(lib().dvm_rank_step(self._h, float(dt)))

    def moments(self):
        rho, u, T = np.zeros(self.ncells), np.zeros((self.ncells, 3)), np.zeros(self.ncells)
        self._chk(lib().dvm_rank_moments(self._h, _p(rho), _p(u), _p(T)))
        return rho, u, T

    def get_f(self):
        f = np.zeros((self.ncells, self.nv))
        self._chk(lib().dvm_rank_get_f(self._h, _p(f), f.size))
        return f

    def totals(self):
        out = np.zeros(5)
        self._chk(lib().dvm_rank_totals(self._h, _p(out)))
        return out


def lbm_lattice(lattice):
    """(c [q][3] int32, w [q]) of a lattice Boltzmann velocity set (no context)."""
    q = C.c_int()
    rc = lib().dvm_lbm_lattice(int(lattice), C.byref(q), None, None)
    if rc:
        raise DvmError(rc, "unknown lattice")
    c = np.zeros((q.value, 3), dtype=np.int32)
    w = np.zeros(q.value)
    lib().dvm_lbm_lattice(int(lattice), None, _p(c), _p(w))
    return c, w


def lbm_solver_from_config(cfg, precision=None, stream=None):
    """A Solver with the tree and lattice of a lattice Boltzmann workload
    dictionary and its inflow state, without initialising f."""
    prec = {"f64": F64, "f32": F32}[precision or cfg["precision"]] \
        if not isinstance(precision, int) else precision
    s = Solver(prec, COLL_NONE, 1.0, stream=stream)
    s.build_tree(tree_spec(cfg["dim"], cfg["base_level"], cfg["max_level"], cfg["pred"], cfg["c"],
                           cfg["r"], cfg["beta"], cfg["solid"], cfg["bc"]))
    s.lbm_set_lattice(cfg["lattice"])
    s.lbm_set_inflow(cfg["fs_rho"], cfg["fs_u"])
    return s


def solver_from_config(cfg, precision=None, collision=None, kn=None, stream=None):
    """Build a Solver for one of the workload dictionaries (tree, velocity
    grid, freestream), without initialising f."""
    prec = {"f64": F64, "f32": F32, "bf16": BF16}[precision or cfg["precision"]] \
        if not isinstance(precision, int) else precision
    coll = cfg["coll"] if collision is None else collision
    s = Solver(prec, coll, cfg["kn"] if kn is None else kn, stream=stream)
    s.build_tree(tree_spec(cfg["dim"], cfg["base_level"], cfg["max_level"], cfg["pred"], cfg["c"],
                           cfg["r"], cfg["beta"], cfg["solid"], cfg["bc"]))
    s.set_velocity_grid(cfg["n"], cfg["lo"], cfg["hi"])
    s.set_freestream(cfg["fs_rho"], cfg["fs_u"], cfg["fs_T"])
    return s
