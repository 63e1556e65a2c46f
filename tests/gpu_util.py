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
        w, r, u, T = W.initial_state(c, xyz)
        s.init_maxwellian(w, r, u, T)
        o.init_maxwellian(w, r, u, T)
    return s, o


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
