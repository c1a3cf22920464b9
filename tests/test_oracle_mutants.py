"""The oracle's pins catch plausible mistakes: each case below plants one
mistake (a wrong sign, index, operand, factor or a dropped term) in a
temporary copy of one oracle source file and runs the pin tests named for it
against that copy, which must fail. A C mistake is built into a separate
library that the pins load through TDBEM_ORACLE_LIB; a Python mistake goes
into a copy of the `oracle` package placed first on the import path of the
pin run. The committed oracle is never modified; everything runs on the CPU.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
T, S = "tests/test_oracle_time.py", "tests/test_oracle_space.py"
MV, RHS, KR = "tests/test_oracle_matvec.py", "tests/test_oracle_rhs.py", "tests/test_oracle_krylov.py"
POT = "tests/test_oracle_potential.py"

# name: (exact source text, planted replacement, pin tests that must fail), in tdbem_oracle.c
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
    "interpolant end weights not halved": ("if (j == 0 || j == I->n) wj *= 0.5;", ";",
                                           [T + "::test_interpolant_matches_direct"]),
    "interpolant panel split dropped": ("if (d > a && d < b) br[nbr++] = d;", "if (d > a && d < b && x != 1) br[nbr++] = d;",
                                        [T + "::test_interpolant_matches_direct"]),
    "interpolant argument mirrored": ("double x = (2.0 * r - ea - eb) / (eb - ea);",
                                      "double x = (ea + eb - 2.0 * r) / (eb - ea);",
                                      [T + "::test_interpolant_matches_direct"]),
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


# the same for the Python parts: (file in oracle/, text or (anchor, text), replacement, pins)
PY_MUTANTS = {
    "reused block of the wrong lag": ("oracle.py", "key = (d + 1, 1)", "key = (d, 1)",
                                      [MV + "::test_reduced_matvec_equals_full_block_matrix"]),
    "superdiagonal from the diagonal block": ("oracle.py", "key = (1, 2)", "key = (1, 1)",
                                              [MV + "::test_reduced_matvec_equals_full_block_matrix"]),
    "matvec reads x of the test index": ("oracle.py", "np.dot(f + n, x[ib * P + m1, c])",
                                         "np.dot(f + n, x[kb * P + m1, c])",
                                         [MV + "::test_matvec_equals_dense_product"]),
    "matvec reads x of the test order": ("oracle.py", "np.dot(f + n, x[ib * P + m1, c])",
                                         "np.dot(f + n, x[ib * P + m2, c])",
                                         [MV + "::test_p1_reduced_matvec_and_dense_product"]),
    "right-hand side tested with b for bdot": ("oracle.py", "bd = self.basis(k, m, s_n)[:, 1]",
                                               "bd = self.basis(k, m, s_n)[:, 0]",
                                               [RHS + "::test_rhs_sphere_n0_closed_form"]),
    "right-hand side weights against reversed points": ("oracle.py", "w7[None, :, None] * bary[None, :, :]",
                                                        "w7[None, :, None] * bary[None, ::-1, :]",
                                                        [RHS + "::test_rhs_plane_wave_brute_force"]),
    "right-hand side ignores the order m": ("oracle.py", "bd = self.basis(k, m, s_n)[:, 1]",
                                            "bd = self.basis(k, 0, s_n)[:, 1]",
                                            ["tests/test_oracle_radial.py::test_mesh_solution_matches_reduction_p1"]),
    "potential without the d_t phi term": ("oracle.py", "(phi / r.ravel() ** 2 + dphi / r.ravel())",
                                           "(phi / r.ravel() ** 2)",
                                           [POT + "::test_sphere_constant_density_reduction"]),
    "potential sign": ("oracle.py", "out[ip, it] = -np.sum(integrand) / (4.0 * np.pi)",
                       "out[ip, it] = np.sum(integrand) / (4.0 * np.pi)", [POT + "::test_gauss_law_and_causality"]),
    "advanced instead of retarded time": ("oracle.py", "s = (t - r).ravel()", "s = (t + r).ravel()",
                                          [POT + "::test_gauss_law_and_causality"]),
    "deflation inverse sign": ("krylov.py", "return v + U @ (lam * (Tinv @ c) - c)", "return v + U @ (lam * (Tinv @ c) + c)",
                               [KR + "::test_deflation_preconditioner_claims"]),
    "deflation keeps the largest Ritz values": ("krylov.py", "cut = np.sort(np.abs(ev))[min(l, m) - 1]",
                                                "cut = np.sort(np.abs(ev))[::-1][min(l, m) - 1]",
                                                [KR + "::test_dgmres_restores_convergence"]),
    "Gram-Schmidt sign": ("krylov.py", ("def fgmres(", "w = w - H[i, j] * V[i]"), "w = w + H[i, j] * V[i]",
                          [KR + "::test_gmres_iterate_is_krylov_minimal_residual"]),
    "flexible update with V for Z": ("krylov.py", "x = x + Z[:jdone].T @ y", "x = x + V[:jdone].T @ y",
                                     [KR + "::test_fixed_preconditioner_is_right_preconditioned_gmres"]),
    "coupling block sign in M^-1": ("krylov.py", "t = r[n1:] - self._sub(h, hi, lo, h) @ y1",
                                    "t = r[n1:] + self._sub(h, hi, lo, h) @ y1",
                                    [KR + "::test_exact_inner_solves_invert_block_triangular_M"]),
    "split point rounded down": ("krylov.py", "h = lo + (hi - lo + 1) // 2", "h = lo + (hi - lo) // 2",
                                 [KR + "::test_exact_inner_solves_invert_block_triangular_M"]),
}


def _pins(nodes, env, cwd):
    env = dict(env, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-rf", "-p", "no:cacheprovider", *nodes],
                       env=env, cwd=cwd, capture_output=True, text=True, timeout=600)
    failed = [line for line in r.stdout.splitlines() if line.startswith("FAILED")]
    return r.returncode, failed, r.stdout[-2000:]


def _run(name, tmp):
    old, new, nodes = MUTANTS[name]
    src = open(O._SRC).read()
    assert src.count(old) == 1, "%s: the planted text must occur once in the oracle source" % name
    tag = "m%02d" % sorted(MUTANTS).index(name)
    path = os.path.join(tmp, tag + ".c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = O.compile_library(path, os.path.join(tmp, tag + ".so"))
    return _pins(nodes, dict(os.environ, TDBEM_ORACLE_LIB=lib), ROOT)


def _run_py(name, tmp, lib):
    fname, old, new, nodes = PY_MUTANTS[name]
    pkg = os.path.join(tmp, "p%02d" % sorted(PY_MUTANTS).index(name))
    os.makedirs(os.path.join(pkg, "oracle"))
    for f in ("__init__.py", "oracle.py", "krylov.py"):
        shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(pkg, "oracle", f))
    target = os.path.join(pkg, "oracle", fname)
    src = open(target).read()
    start = 0
    if isinstance(old, tuple):  # (anchor, text): the first occurrence of text after the anchor
        anchor, old = old
        assert src.count(anchor) == 1, "%s: the anchor must occur once in oracle/%s" % (name, fname)
        start = src.index(anchor)
    else:
        assert src.count(old) == 1, "%s: the planted text must occur once in oracle/%s" % (name, fname)
    at = src.index(old, start)
    with open(target, "w") as f:
        f.write(src[:at] + new + src[at + len(old):])
    # the copy comes first on the path (cwd); the repository follows for the rest
    env = dict(os.environ, TDBEM_ORACLE_LIB=lib, PYTHONPATH=os.pathsep.join([pkg, ROOT]))
    return _pins([os.path.join(ROOT, n) for n in nodes], env, pkg)


@pytest.mark.slow
def test_pins_catch_planted_mistakes(tmp_path):
    lib = O.build()
    jobs = [("c", n) for n in sorted(MUTANTS)] + [("py", n) for n in sorted(PY_MUTANTS)]
    run = lambda j: _run(j[1], str(tmp_path)) if j[0] == "c" else _run_py(j[1], str(tmp_path), lib)
    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        res = dict(zip(jobs, ex.map(run, jobs)))
    missed = {n: out for n, (rc, failed, out) in res.items() if rc != 1 or not failed}
    assert not missed, "pins that did not catch their planted mistake: %s" % missed
