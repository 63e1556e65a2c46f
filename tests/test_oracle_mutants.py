"""Do the oracle's pins catch plausible mistakes?  Each case plants one
mistake in a copy of the oracle's C source (a weight, a coefficient, an
upwind side, a sign), builds it with gcc into a temporary library, and runs
the pin that should notice against it in a subprocess: the pin must fail.
The unaltered oracle passes the same pins in the rest of the suite."""
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

MUTANTS = [
    # name, original text, planted text, the pin that must fail
    ("D3Q27 edge weight", "1.0 / 54, 1.0 / 216", "1.0 / 56, 1.0 / 216",
     "tests/test_oracle_lbm.py::test_weights_satisfy_isotropy"),
    ("LBM equilibrium quadratic term", "cu * cu / (2.0 * cs2 * cs2)", "cu * cu / (2.0 * cs2)",
     "tests/test_oracle_lbm.py::test_equilibrium_moments"),
    ("LBM relaxation factor", "const double om = dt / tau;", "const double om = 0.5 * dt / tau;",
     "tests/test_oracle_lbm.py::test_shear_wave_damping_matches_the_bgk_equation"),
    ("transport takes the downwind cell", "double up = x > 0.0 ? fa[v] : fb[v];",
     "double up = x > 0.0 ? fb[v] : fa[v];",
     "tests/test_oracle_transport.py::test_transport_fourier_closed_form"),
    ("wall ghost without the mirror", "up = own[p->mirror[d][v]];", "up = own[v];",
     "tests/test_oracle_transport.py::test_transport_specular_walls_conserve_mass_and_energy"),
    ("BGK frequency uses T for sqrt(T)", "double nu = sqrt(8.0 / M_PI) * rho * sqrt(T) / kn;",
     "double nu = sqrt(8.0 / M_PI) * rho * T / kn;",
     "tests/test_oracle_collision.py::test_bgk_frequency_equals_hs_mean_frequency"),
    ("hard-sphere weight normalisation", "/ (sqrt(2.0) * (double)trials)", "/ (2.0 * (double)trials)",
     "tests/test_oracle_collision.py::test_hs_mean_collision_frequency_of_maxwellian"),
    ("local Kn without the mean free path 1/rho", "return kn / rho[c] * m;", "return kn * m;",
     "tests/test_oracle_learned.py::test_kn_local_linear_fields_exact_on_uniform_tree"),
    ("entropic Newton step with the wrong sign", "for (int r = 0; r < 5; r++) a[r] -= da[r];",
     "for (int r = 0; r < 5; r++) a[r] += da[r];",
     "tests/test_oracle_collision.py::test_entropic_bgk_conserves_and_is_exponential_of_a_quadratic"),
    ("2:1 balance ignores z neighbours", "int lo3 = dim == 3 ? -1 : 0, hi3 = dim == 3 ? 4 : 0;",
     "int lo3 = 0, hi3 = dim == 3 ? 3 : 0;",
     "tests/test_oracle_tree.py::test_tiling_morton_and_balance_bruteforce"),
    ("fine subface area of a coarse cell", "area = ldexp(1.0, -(A->lev + 1) * (dim - 1));",
     "area = ldexp(1.0, -A->lev * (dim - 1));",
     "tests/test_oracle_transport.py::test_transport_freestream_preserved_on_refined_tree"),
    ("temperature with 2 degrees of freedom", "*T = (s2 / s0 - uu) / 3.0;", "*T = (s2 / s0 - uu) / 2.0;",
     "tests/test_oracle_transport.py::test_moments_of_maxwellian_closed_form"),
    ("post-collision velocity off by the half", "xp[d] = c + 0.5 * gn * w[d];", "xp[d] = c + gn * w[d];",
     "tests/test_oracle_collision.py::test_hs_tables_match_independent_regeneration"),
    ("third Hermite mode normalisation", "h[3] = (x * x * x - 3.0 * x) / sqrt(6.0);",
     "h[3] = (x * x * x - 3.0 * x) / sqrt(3.0);",
     "tests/test_oracle_learned.py::test_hermite_projection_of_maxwellian_and_modes"),
    ("gain term with one post-collision partner twice", "sc += p->hs_b[t] * f[p->hs_l[t]] * f[p->hs_m[t]];",
     "sc += p->hs_b[t] * f[p->hs_l[t]] * f[p->hs_l[t]];",
     "tests/test_oracle_collision.py::test_hs_relaxation_approaches_the_maxwellian_as_trials_grow"),
    ("selected-cell inputs miss the plus-side neighbours", "t[m++] = p->cell_of_leaf[p->fp[q]];",
     "t[m++] = p->cell_of_leaf[p->fm[q]];",
     "tests/test_oracle_sampled.py::test_inputs_hold_cells_and_neighbours"),
    ("selected-cell row lookup off by one", "if (t->cells[mid] < k) lo = mid + 1;",
     "if (t->cells[mid] <= k) lo = mid + 1;",
     "tests/test_oracle_sampled.py::test_selected_cells_equal_full_step"),
    ("velocity nodes off the cell midpoints", "xi[3 * v + d] = lo[d] + ((double)kk[d] + 0.5) * h[d];",
     "xi[3 * v + d] = lo[d] + ((double)kk[d] + 0.45) * h[d];",
     "tests/test_oracle_transport.py::test_density_of_a_truncated_maxwellian_closed_form"),
]


def _build_copy(tmp_path, text):
    (tmp_path / "dvm_oracle.c").write_text(text)
    lib = tmp_path / "liboracle_copy.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-I", ORACLE,
                           "-o", str(lib), str(tmp_path / "dvm_oracle.c"), "-lm"])
    return lib


def _run_pins(lib, pins):
    env = dict(os.environ, DVM_ORACLE_LIB=str(lib))
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider"] + list(pins),
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_unaltered_copy_passes_the_pins(tmp_path):
    """The harness itself: an unaltered copy, built the same way, passes."""
    lib = _build_copy(tmp_path, open(os.path.join(ORACLE, "dvm_oracle.c")).read())
    r = _run_pins(lib, sorted({m[3] for m in MUTANTS}))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(name, old, new, pin, tmp_path):
    src = open(os.path.join(ORACLE, "dvm_oracle.c")).read()
    assert src.count(old) >= 1, "the text to alter is not in the oracle"
    lib = _build_copy(tmp_path, src.replace(old, new, 1))
    r = _run_pins(lib, [pin])
    # the pin ran and failed (not a collection or loading error)
    summary = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
    assert r.returncode == 1 and re.search(r"\d+ failed", summary) and "error" not in summary, \
        "%s: %s\n%s" % (name, pin, r.stdout[-2000:])
