"""Seeded synthetic workloads shared by the CUDA path's tests/bench and the oracle.

This module holds input recipes only: tree specifications, velocity grids,
boundary kinds, freestream states and per-cell initial macroscopic states.
It contains none of the method's arithmetic (no Maxwellian sampling, no
transport, no collision): both sides turn these inputs into f themselves.

The paper's own workloads (rarefied flow over a sphere at M=0.1 and Kn=0.01
with 24^3 or 32^3 velocity meshes and 15K-75K cells, Sec. 3.3; the Ma=5,
Kn=0.01 hybrid run with ~1.2M Boltzmann cells on a 24^3 velocity mesh,
Sec. 3.4) come with no geometry or data, so the synthetic flows below stand in
for them with the same shapes.  Leaf counts of the refined trees were
calibrated once by building the trees (sphere-band width `beta`).
"""
import math

import numpy as np

SEED = 20150303

PERIODIC, INFLOW, OUTFLOW, WALL = 0, 1, 2, 3
PRED_NONE, PRED_BALL, PRED_SHELL = 0, 1, 2
COLL_NONE, COLL_BGK, COLL_HS, COLL_LEARNED = 0, 1, 2, 3

GAMMA = 5.0 / 3.0  # monatomic gas: sound speed sqrt(gamma) in thermal units


def mach_velocity(mach):
    return (mach * math.sqrt(GAMMA), 0.0, 0.0)


def _sphere_flow(base, top, r, beta, n, vmax, mach, kn, steps, precision, coll=COLL_BGK):
    return dict(
        dim=3, base_level=base, max_level=top, pred=PRED_SHELL, c=(0.5, 0.5, 0.5),
        r=r, beta=beta, solid=1,
        bc=(INFLOW, OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW),
        n=(n, n, n), lo=(-vmax,) * 3, hi=(vmax,) * 3,
        fs_rho=1.0, fs_u=mach_velocity(mach), fs_T=1.0,
        coll=coll, kn=kn, cfl=0.4, steps=steps, precision=precision, init="freestream",
    )


CONFIGS = {
    # 2D quadtree, level 4 refined to level 6 near a centred circle, periodic;
    # 8^3 velocities on [-4,4]^3; density bump; BGK Kn=0.05; CFL 0.4; FP64.
    "c1_2d_bump": dict(
        dim=2, base_level=4, max_level=6, pred=PRED_BALL, c=(0.5, 0.5, 0.5), r=0.2,
        beta=0.0, solid=0, bc=(PERIODIC,) * 6,
        n=(8, 8, 8), lo=(-4.0,) * 3, hi=(4.0,) * 3,
        fs_rho=1.0, fs_u=(0.0, 0.0, 0.0), fs_T=1.0,
        coll=COLL_BGK, kn=0.05, cfl=0.4, steps=50, precision="f64", init="bump",
    ),
    # 3D octree levels 4-6 around a specular sphere r=0.15; 16^3 on [-6,6]^3;
    # Mach-3 inflow at x=0; BGK Kn=0.1; 200 steps; FP32.
    "c2_sphere_m3": _sphere_flow(4, 6, 0.15, 3.25, 16, 6.0, 3.0, 0.1, 200, "f32"),
    # 3D octree levels 5-9 around a sphere r=0.1 in a Mach-5 stream;
    # ~1.01M kinetic cells x 24^3 = 1.40e10 f values; BGK Kn=0.01; 100 steps.
    "c3_sphere_m5": _sphere_flow(5, 9, 0.1, 7.5, 24, 8.0, 5.0, 0.01, 100, "f32"),
    # the same flow on levels 5-7 (oracle-sized)
    "c3_sphere_m5_reduced": _sphere_flow(5, 7, 0.1, 7.5, 24, 8.0, 5.0, 0.01, 10, "f32"),
    # the same flow on levels 4-6 with a thinner band (17.7k cells): the
    # oracle finishes a step in seconds, for parity tests and the CPU baseline
    "c3_sphere_m5_small": _sphere_flow(4, 6, 0.1, 3.0, 24, 8.0, 5.0, 0.01, 3, "f32"),
    # periodic box, level 4 plus a central ball at level 5 (~16.6k leaves);
    # 16^3 on [-6,6]^3; hard-sphere collisions, Kn=0.02; bimodal start.
    "c4_hs_bimodal": dict(
        dim=3, base_level=4, max_level=5, pred=PRED_BALL, c=(0.5, 0.5, 0.5), r=0.42,
        beta=0.0, solid=0, bc=(PERIODIC,) * 6,
        n=(16, 16, 16), lo=(-6.0,) * 3, hi=(6.0,) * 3,
        fs_rho=1.0, fs_u=(0.0, 0.0, 0.0), fs_T=1.0,
        coll=COLL_HS, kn=0.02, cfl=0.4, steps=20, precision="f32", init="bimodal",
        trials=128,
    ),
    # Mach-3 sphere flow, levels 4-8, ~253k kinetic cells, 24^3, full
    # collision integral (plain or learned).
    # Kn is not given for this flow: that of the paper's hybrid run (Sec. 5),
    # 0.01 per body length, where the local-Kn switch separates
    # near-continuum cells from kinetic ones; the sphere's diameter is 0.3,
    # so Kn = 0.003 per unit length.  (The developed flow's local Kn exceeds
    # 0.05 in 99% of the cells of this tree at Kn = 0.1 and in 94% at 0.01.)
    "c5_sphere_m3_hs": _sphere_flow(4, 8, 0.15, 3.5, 24, 8.0, 3.0, 0.003, 100, "f32", COLL_HS),
}
CONFIGS["c5_sphere_m3_hs"]["trials"] = 128
# the same flow on levels 3-5 (~12k cells, f 0.66 GB): gain test and profiles
CONFIGS["c5_sphere_m3_hs_small"] = dict(CONFIGS["c5_sphere_m3_hs"], base_level=3, max_level=5)

# ---- lattice Boltzmann (Sec. 4).  The paper's LBM flow is a sphere at
# Ma = 0.5 and Re = 1000 with D3Q19 (Fig. 9); its GPU timings use trees of
# 100K and 1M cells (Table 1).  Lattice units: c_s = 1/sqrt(3), so Ma 0.5 is
# u = 0.5/sqrt(3).  Each flow fixes omega = dt/tau; tau then follows from the
# CFL time step, and Re = U D / (c_s^2 tau) with D = 2r.
LBM_D2Q9, LBM_D3Q19, LBM_D3Q27 = 9, 19, 27


def _lbm_sphere(lattice, base, top, r, beta, omega, cfl, precision, steps):
    return dict(
        lattice=lattice, dim=3, base_level=base, max_level=top, pred=PRED_SHELL, c=(0.5, 0.5, 0.5),
        r=r, beta=beta, solid=1, bc=(INFLOW, OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW),
        fs_rho=1.0, fs_u=(0.5 / math.sqrt(3.0), 0.0, 0.0), omega=omega, cfl=cfl,
        precision=precision, steps=steps, init="lbm_perturbed",
    )


CONFIGS.update({
    # 2D quadtree levels 4-7 around a solid disk r=0.1 (walls), inflow at
    # x=0, outflow at x=1, periodic in y; D2Q9, u = 0.1; FP64.
    "l1_2d_disk_d2q9": dict(
        lattice=LBM_D2Q9, dim=2, base_level=4, max_level=7, pred=PRED_SHELL, c=(0.5, 0.5, 0.5),
        r=0.1, beta=3.0, solid=1, bc=(INFLOW, OUTFLOW, PERIODIC, PERIODIC, PERIODIC, PERIODIC),
        fs_rho=1.0, fs_u=(0.1, 0.0, 0.0), omega=0.5, cfl=0.4, precision="f64", steps=30,
        init="lbm_perturbed",
    ),
    # the Ma-0.5 sphere flow on the 17.7k-cell tree of levels 4-6 (oracle-sized)
    "l2_sphere_d3q19_small": _lbm_sphere(LBM_D3Q19, 4, 6, 0.1, 3.0, 0.5, 0.4, "f32", 10),
    "l2_sphere_d3q27_small": _lbm_sphere(LBM_D3Q27, 4, 6, 0.1, 3.0, 0.5, 0.4, "f32", 10),
    # levels 7-10 around the sphere: 3.34M cells (f is 254 MB per buffer for
    # D3Q19 in FP32, twice L2); omega 0.85 at CFL 0.3 gives Re ~ 1000
    "l3_sphere_d3q19": _lbm_sphere(LBM_D3Q19, 7, 10, 0.1, 3.0, 0.85, 0.3, "f32", 100),
    "l3_sphere_d3q27": _lbm_sphere(LBM_D3Q27, 7, 10, 0.1, 3.0, 0.85, 0.3, "f32", 100),
})


def initial_state(cfg, centres, seed=SEED):
    """Per-cell Maxwellian mixture parameters for `init_maxwellian`.

    centres: [ncells, 3] cell centres (from whichever side builds the tree).
    Returns (w, rho, u, T) with shapes [nc, K], [nc, K], [nc, K, 3], [nc, K].
    """
    centres = np.asarray(centres, dtype=np.float64)
    nc = centres.shape[0]
    kind = cfg["init"]
    if kind == "freestream":
        w = np.ones((nc, 1))
        rho = np.full((nc, 1), cfg["fs_rho"])
        u = np.tile(np.asarray(cfg["fs_u"], dtype=np.float64), (nc, 1, 1))
        T = np.full((nc, 1), cfg["fs_T"])
        return w, rho, u, T
    if kind == "bump":
        dx = centres[:, :2] - 0.5
        r2 = (dx * dx).sum(axis=1)
        rho = (1.0 + 0.2 * np.exp(-r2 / 0.01)).reshape(nc, 1)
        return np.ones((nc, 1)), rho, np.zeros((nc, 1, 3)), np.ones((nc, 1))
    if kind == "bimodal":
        g = np.random.default_rng(seed)
        w1 = g.uniform(0.3, 0.7, nc)
        a1 = g.uniform(1.0, 2.0, nc)
        a2 = g.uniform(1.0, 2.0, nc)
        T1 = g.uniform(0.4, 0.8, nc)
        T2 = g.uniform(0.4, 0.8, nc)
        z = g.uniform(-1.0, 1.0, nc)
        ph = g.uniform(0.0, 2.0 * math.pi, nc)
        st = np.sqrt(1.0 - z * z)
        nvec = np.stack([st * np.cos(ph), st * np.sin(ph), z], axis=1)
        w = np.stack([w1, 1.0 - w1], axis=1)
        rho = np.ones((nc, 2))
        u = np.stack([a1[:, None] * nvec, -a2[:, None] * nvec], axis=1)
        T = np.stack([T1, T2], axis=1)
        return w, rho, u, T
    if kind == "bimodal_near":
        # one two-beam state (weights 1/2, beams of speed 1.5 along +-x,
        # temperatures 0.6) perturbed per cell by seeded relative amounts of
        # up to 5%: away from equilibrium everywhere, with gradients small
        # enough that the local Kn of a Kn = 0.003 flow spreads across 0.05
        g = np.random.default_rng(seed + 3)
        e = 0.05
        w1 = 0.5 * (1.0 + e * g.uniform(-1.0, 1.0, nc))
        a1 = 1.5 * (1.0 + e * g.uniform(-1.0, 1.0, nc))
        a2 = 1.5 * (1.0 + e * g.uniform(-1.0, 1.0, nc))
        T1 = 0.6 * (1.0 + e * g.uniform(-1.0, 1.0, nc))
        T2 = 0.6 * (1.0 + e * g.uniform(-1.0, 1.0, nc))
        nvec = np.stack([np.ones(nc), e * g.uniform(-1.0, 1.0, nc), e * g.uniform(-1.0, 1.0, nc)], axis=1)
        nvec /= np.linalg.norm(nvec, axis=1, keepdims=True)
        w = np.stack([w1, 1.0 - w1], axis=1)
        rho = np.ones((nc, 2))
        u = np.stack([a1[:, None] * nvec, -a2[:, None] * nvec], axis=1)
        T = np.stack([T1, T2], axis=1)
        return w, rho, u, T
    raise ValueError(kind)


def lbm_initial_state(cfg, centres, seed=SEED):
    """Per-cell (rho [nc], u [nc, 3]) for the lattice Boltzmann flows: the
    inflow state with seeded perturbations (2% in rho, 0.02 in each active
    velocity component), so that every term of the step is exercised."""
    centres = np.asarray(centres, dtype=np.float64)
    nc = centres.shape[0]
    g = np.random.default_rng(seed + 7)
    rho = cfg["fs_rho"] * (1.0 + 0.02 * g.uniform(-1.0, 1.0, nc))
    u = np.tile(np.asarray(cfg["fs_u"], dtype=np.float64), (nc, 1))
    u[:, :cfg["dim"]] += 0.02 * g.uniform(-1.0, 1.0, (nc, cfg["dim"]))
    return rho, u


def lbm_tau(cfg, dt):
    return dt / cfg["omega"]


def random_f_perturbation(ncells, nv, seed=SEED, scale=0.05):
    """Multiplicative noise factors (1 + scale * U(-1,1)) for parity tests that
    start from a non-Maxwellian f."""
    g = np.random.default_rng(seed + 1)
    return 1.0 + scale * g.uniform(-1.0, 1.0, (ncells, nv))
