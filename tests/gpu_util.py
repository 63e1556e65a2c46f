"""Shared set-up for the GPU parity tests: the same seeded workload on the
CUDA path (through the C ABI) and on the oracle."""
import math

import numpy as np

import oracle as O
import paper_1503_00707_gb300 as D
import workloads as W

PREC = {"f64": D.F64, "f32": D.F32, "bf16": D.BF16}


def oracle_for(c):
    o = O.Problem(O.make_spec(c["dim"], c["base_level"], c["max_level"], c["pred"], c["c"], c["r"],
                              c["beta"], c["solid"], c["bc"]), c["n"], c["lo"], c["hi"])
    o.set_freestream(c["fs_rho"], c["fs_u"], c["fs_T"])
    return o


def pair(c, precision=None, collision=None, init=True):
    """(solver, oracle) on workload dict c, both initialised from the same
    seeded per-cell Maxwellian parameters."""
    prec = PREC[precision or c["precision"]]
    coll = c["coll"] if collision is None else collision
    s = D.solver_from_config(c, prec, coll)
    o = oracle_for(c)
    if init:
        xyz, _ = s.centres()
        xo, _ = o.centres()
        assert np.array_equal(xyz, xo)
        w, r, u, T = W.initial_state(c, xo)
        s.init_maxwellian(w, r, u, T)
        o.init_maxwellian(w, r, u, T)
    return s, o


def storage_round(f, precision):
    """f rounded to the CUDA path's storage precision ("f64", "f32", "bf16"), as
    float64: the values both sides start from when they must start alike."""
    if precision == "f64":
        return np.array(f, dtype=np.float64)
    if precision == "f32":
        return np.asarray(f, dtype=np.float32).astype(np.float64)
    return bf16_round(np.asarray(f, dtype=np.float32)).astype(np.float64)


def same_start(s, o, f, precision):
    """Set the solver and the oracle to f (computed on the oracle's side)
    rounded to the storage precision; returns the rounded values."""
    fr = storage_round(f, precision)
    s.set_f(fr)
    o.set_f(fr)
    return fr


def volume_totals(f, o, dim):
    """sum_j V_j sum_i psi_r f_ij dV, r = mass, momentum, energy, for any f on
    the oracle's tree, from its cell sizes and velocity nodes (independent of
    either side's totals routine)."""
    _, h = o.centres()
    xi = o.xi.reshape(-1, 3)
    psi = np.stack([np.ones(len(xi)), xi[:, 0], xi[:, 1], xi[:, 2], (xi * xi).sum(1)], 1)
    return ((h ** dim)[:, None] * (np.asarray(f, np.float64) @ psi)).sum(0) * o.dV


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def field_errors(s_mom, o_mom):
    (r1, u1, T1), (r2, u2, T2) = s_mom, o_mom
    return {"rho": rel_linf(r1, r2), "u": rel_linf(u1, u2), "T": rel_linf(T1, T2)}


def bf16_round(a):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def random_params(seed, gain=1.0, bias=0.05):
    """Seeded network parameters whose weights are exactly representable in
    BF16, so that the tensor cores and the FP64 oracle use the same values."""
    rng = np.random.default_rng(seed)
    out = []
    for (r, c), nb in O.MLP_SHAPES:
        out.append(rng.normal(0, gain / math.sqrt(c), size=(r, c)).ravel())
        out.append(rng.normal(0, bias, size=nb))
    return bf16_round(np.concatenate(out).astype(np.float32))
