"""The oracle's pins catch plausible mistakes: each case below plants one
mistake (a wrong sign, index, operand, factor or a dropped term) in a
temporary copy of the oracle's C source, builds it, and runs the pin tests
named for it against that copy (TDBEM_ORACLE_LIB), which must fail. The
committed oracle is never modified; everything runs on the CPU.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
T, S, R = "tests/test_oracle_time.py", "tests/test_oracle_space.py", "tests/test_oracle_radial.py"

# name: (exact source text, planted replacement, pin tests that must fail)
MUTANTS = {
    "step f'' sign": ("(x - 2.0 * u)", "(2.0 * u - x)", [T + "::test_basis_derivatives_fd"]),
    "psi takes bdot_i for bddot_i": ("s0 += wt * bi[2] * bk[1];", "s0 += wt * bi[1] * bk[1];",
                                     [T + "::test_psi_is_second_derivative_of_psi_tilde"]),
    "falling flank on the wrong interval": ("        double h = t[ib + 1] - t[ib];\n",
                                            "        double h = t[ib] - t[ib - 1];\n",
                                            [T + "::test_partition_of_unity"]),
    "first basis factor 4 for 8": ("double g0 = 8.0 * q * q,", "double g0 = 4.0 * q * q,",
                                   [T + "::test_step_function_values"]),
    "Legendre recurrence sign": ("double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;",
                                 "double p2 = ((2.0 * k - 1.0) * x * p1 + (k - 1.0) * p0) / k;",
                                 [T + "::test_legendre_factor"]),
    "psi split point dropped": ("if (ib > 0 && ib < P->N - 1) cand[nc++] = P->t[ib] + r;", ";",
                                [T + "::test_quadrature_refinement_converged"]),
    "psi support end": ("*b = tr(P, kb) - tl(P, ib);", "*b = tr(P, kb) - tr(P, ib);",
                        [S + "::test_unique_block_list_equidistant"]),
    "block A_{2,3} dropped": ("want[1 * N + 2] = 1;", "(void)0;", [S + "::test_unique_block_list_equidistant"]),
    "7-point weights swapped": ("double W[7] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};",
                                "double W[7] = {9.0 / 40.0, w2, w2, w2, w1, w1, w1};", [S + "::test_rule7_degree5"]),
    "edge-case Jacobian factor dropped": ("double w0 = xi * xi * xi * e1 * e1, w = w0 * e2;",
                                          "double w0 = xi * xi * xi * e1, w = w0 * e2;",
                                          [S + "::test_sauter_schwab_polynomials"]),
    "surface curl operands swapped": ("cross3(n, gr[a], P->curl + 9 * e + 3 * a);",
                                      "cross3(gr[a], n, P->curl + 9 * e + 3 * a);",
                                      [S + "::test_surface_curls_closed_form"]),
    "segment-segment distance dropped": ("double v = seg_seg_dist2(a[i], a[(i + 1) % 3], b[j], b[(j + 1) % 3]);",
                                         "double v = 1e300;", [S + "::test_triangle_distance_bounds"]),
    "row star cut to one triangle": ("for (int k = 0; k < nt; ++k) {\n            int64_t s = P->vt_tri[P->vt_ptr[l] + k];",
                                     "for (int k = 0; k < 1; ++k) {\n            int64_t s = P->vt_tri[P->vt_ptr[l] + k];",
                                     [S + "::test_pattern_counts_on_fine_grid"]),
    "far curl-curl sign": ("(nn * bx[a] * by[b] * ps[0] + cc[a][b] * ps[1])",
                           "(nn * bx[a] * by[b] * ps[0] - cc[a][b] * ps[1])",
                           [S + "::test_sphere_bilinear_forms_converge"]),
    "far weight index": ("double wgt = R->w[i] * R->w[j] * scale / r;", "double wgt = R->w[i] * R->w[i] * scale / r;",
                         [S + "::test_sphere_bilinear_forms_converge"]),
    "near curl operand transposed": ("cc[pa[a]][pb[b]] * ps[1]", "cc[pb[b]][pa[a]] * ps[1]",
                                     [S + "::test_sphere_bilinear_forms_converge"]),
    "near area scale not doubled": ("double scale = (2.0 * P->area[s]) * (2.0 * P->area[q]) / (4.0 * OR_PI);",
                                    "double scale = P->area[s] * P->area[q] / (4.0 * OR_PI);",
                                    [S + "::test_sphere_bilinear_forms_converge"]),
    "shared edge reversed on the trial side": ("pb[0] = ub; pb[1] = vb;", "pb[0] = vb; pb[1] = ub;",
                                               [S + "::test_block_symmetry"]),
}


def _run(name, tmp):
    old, new, nodes = MUTANTS[name]
    src = open(O._SRC).read()
    assert src.count(old) == 1, "%s: the planted text must occur once in the oracle source" % name
    tag = "m%02d" % sorted(MUTANTS).index(name)
    path = os.path.join(tmp, tag + ".c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = O.compile_library(path, os.path.join(tmp, tag + ".so"))
    env = dict(os.environ, TDBEM_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-rf", "-p", "no:cacheprovider", *nodes],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    failed = [line for line in r.stdout.splitlines() if line.startswith("FAILED")]
    return r.returncode, failed, r.stdout[-2000:]


@pytest.mark.slow
def test_pins_catch_planted_mistakes(tmp_path):
    names = sorted(MUTANTS)
    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        res = dict(zip(names, ex.map(lambda n: _run(n, str(tmp_path)), names)))
    missed = {n: out for n, (rc, failed, out) in res.items() if rc != 1 or not failed}
    assert not missed, "pins that did not catch their planted mistake: %s" % missed
