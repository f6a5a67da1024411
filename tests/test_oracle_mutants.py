"""The oracle pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of the oracle's C source
(the shipped oracle is untouched), compiles it, and runs the pin suite
against it in a subprocess; every mutant must make at least one pin fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tpfa_oracle.c")

# (name, text in the source, replacement, occurrences to replace)
MUTANTS = [
    ("arithmetic_mean", "return a_over_mu / (half / kK + half / kL);",
     "return a_over_mu * 0.5 * (kK + kL) / h;", 1),
    ("full_cell_distance", "double half = 0.5 * h;", "double half = h;", 1),
    ("dropped_accumulation", "vals[0] = diag + dval(d, d0, c);", "vals[0] = diag;", 1),
    ("offdiag_sign", "if (!is_dir(mask, n)) { cols[m] = n; vals[m] = -T; ++m; }",
     "if (!is_dir(mask, n)) { cols[m] = n; vals[m] = T; ++m; }", 1),
    ("y_neighbour_index", "case 2: return j > 0 ? c - g->nx : -1;",
     "case 2: return j > 0 ? c - 1 : -1;", 1),
    ("x_face_area", "double a = axis == 0 ? (g->dy * g->dz) / g->mu",
     "double a = axis == 0 ? (g->dx * g->dz) / g->mu", 1),
    ("mobility_times_mu", "/ g->mu", "* g->mu", 3),
    ("rhs_lift_sign", "s += face_T(g, K, c, f, n) * (pD", "s -= face_T(g, K, c, f, n) * (pD", 1),
    ("rhs_drops_dirichlet_value", "b[c] = pD != NULL ? pD[c] : 0.0; continue;",
     "b[c] = 0.0; continue;", 1),
    ("cg_beta_inverted", "double beta = rr_new / rr;", "double beta = rr / rr_new;", 1),
    ("cg_residual_update", "r[i] -= alpha * Ap[i]; }", "r[i] -= alpha * p[i]; }", 1),
    ("pcg_unpreconditioned_z", "      z[i] = minv[i] * r[i];\n", "      z[i] = r[i];\n", 1),
    ("pcg_beta_inverted", "double beta = rz_new / rz;", "double beta = rz / rz_new;", 1),
    ("pcg_direction_from_r", "p[i] = z[i] + beta * p[i];", "p[i] = r[i] + beta * p[i];", 1),
    ("dot_block_dropped", "for (int64_t blk = 0; blk < nb; ++blk) s += part[blk];",
     "for (int64_t blk = 1; blk < nb; ++blk) s += part[blk];", 1),
]


@pytest.mark.parametrize("name,old,new,count", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, old, new, count):
    src = open(SRC).read()
    assert src.count(old) >= count, f"mutation site for {name} not found"
    mutated = src.replace(old, new, count)
    msrc = tmp_path / "mutant.c"
    msrc.write_text(mutated)
    sys.path.insert(0, ROOT)
    from oracle import oracle
    lib = oracle.compile_to(str(msrc), str(tmp_path / "libmutant.so"))
    env = dict(os.environ, TPFA_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
