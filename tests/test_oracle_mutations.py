"""Planted mistakes in the oracle, each caught by a pin (CPU, no GPU).

Each case copies oracle/ and workloads/ with the pins to a temporary folder,
plants one plausible mistake in the copy of the oracle (a flipped sign, a
shifted index, a transposed operand, a dropped term or check), and runs the
pin that must catch it. The pin must fail. A pattern that no longer occurs in
the oracle fails the test too, so that edits to the oracle keep this list
honest.
"""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (mistake, text in oracle/ascg_oracle.py, planted text, pin that must fail)
MUTATIONS = [
    ('recurrence theta sign',
     't = spmv(A, cols[j - 1]) - bp.theta[j - 1] * cols[j - 1]',
     't = spmv(A, cols[j - 1]) + bp.theta[j - 1] * cols[j - 1]',
     'test_sstep_equals_classical_exact[chebyshev-seq0]'),
    ('recurrence sigma sign',
     't = t - bp.sigma[j - 2] * cols[j - 2]',
     't = t + bp.sigma[j - 2] * cols[j - 2]',
     'test_sstep_equals_classical_exact[chebyshev-seq1]'),
    ('recurrence sigma index',
     't = t - bp.sigma[j - 2] * cols[j - 2]',
     't = t - bp.sigma[j - 1] * cols[j - 2]',
     'test_sstep_equals_classical_exact[three_term-seq1]'),
    ('recurrence gamma mul',
     'cols.append(t / bp.gamma[j - 1])',
     'cols.append(t * bp.gamma[j - 1])',
     'test_sstep_equals_classical_exact[chebyshev-seq0]'),
    ('B transposed gamma',
     'B[c + 1, c] = bp.gamma[j]',
     'B[c, c + 1] = bp.gamma[j]',
     'test_sstep_equals_classical_exact[monomial-seq0]'),
    ('B sigma index',
     'B[c - 1, c] = bp.sigma[j - 1]',
     'B[c - 1, c] = bp.sigma[j]',
     'test_sstep_equals_classical_exact[three_term-seq1]'),
    ('B sigma dropped',
     'B[c - 1, c] = bp.sigma[j - 1]',
     'pass',
     'test_sstep_equals_classical_exact[chebyshev-seq1]'),
    ('pGBp operand order',
     'pGBp = pc @ (G @ (B @ pc))',
     'pGBp = pc @ (B @ (G @ pc))',
     'test_sstep_equals_classical_exact[monomial-seq0]'),
    ("r' update transposed B",
     'rn = rc - B @ q',
     'rn = rc - B.T @ q',
     'test_sstep_equals_classical_exact[monomial-seq0]'),
    ("p' update sign",
     'pc = rn + beta * pc',
     'pc = rn - beta * pc',
     'test_sstep_equals_classical_exact[monomial-seq0]'),
    ('beta inverted',
     'beta = rGr_new / rGr',
     'beta = rGr / rGr_new',
     'test_sstep_equals_classical_exact[monomial-seq0]'),
    ("r' start index",
     'rc[s + 1] = 1',
     'rc[s] = 1',
     'test_sstep_equals_classical_exact[monomial-seq0]'),
    ('recovery r/p swapped',
     'return x + Y @ xc, Y @ rc, Y @ pc',
     'return x + Y @ xc, Y @ pc, Y @ rc',
     'test_sstep_equals_classical_exact[monomial-seq0]'),
    ('recovery x sign',
     'return x + Y @ xc, Y @ rc, Y @ pc',
     'return x - Y @ xc, Y @ rc, Y @ pc',
     'test_sstep_equals_classical_exact[monomial-seq0]'),
    ('threshold rnorm upside down',
     'threshold = eps_star / (c_condy * EPS * rnorm) if rnorm > 0 else math.inf',
     'threshold = eps_star * rnorm / (c_condy * EPS) if rnorm > 0 else math.inf',
     'test_paper_observations_sec5'),
    ('condy without sqrt',
     'sk = math.sqrt(kap)',
     'sk = kap',
     'test_first_blocks_are_rank_limited'),
    ('index set i_s',
     'i_s = sbar + 2',
     'i_s = sbar + 1',
     'test_submatrix_index_matches_matlab_notation'),
    ('classical r sign',
     'r = r - alpha * Ap',
     'r = r + alpha * Ap',
     'test_classical_cg_exact_finite_termination'),
    ('classical beta inverted',
     'beta = rr_new / rr',
     'beta = rr / rr_new',
     'test_classical_cg_exact_finite_termination'),
    ('ritz diagonal',
     'T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)',
     'T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j] if j > 0 else 0.0)',
     'test_ritz_values_are_eigenvalues_after_d_steps'),
    ('ritz offdiag',
     'T[j, j + 1] = T[j + 1, j] = math.sqrt(betas[j]) / alphas[j]',
     'T[j, j + 1] = T[j + 1, j] = betas[j] / alphas[j]',
     'test_ritz_values_are_eigenvalues_after_d_steps'),
    ('leja first smallest',
     'score = abs(vals[i])',
     'score = -abs(vals[i])',
     'test_leja_order_golden'),
    ('chebyshev gamma0',
     '[h] + [h / 2] * (s - 1)',
     '[h / 2] * s',
     'test_basis_closed_form_on_diagonal[chebyshev]'),
    ('chebyshev center',
     'c = (lam_max + lam_min) / 2',
     'c = (lam_max - lam_min) / 2',
     'test_basis_closed_form_on_diagonal[chebyshev]'),
    ('kappa clamp removed',
     'if lmin <= w * math.sqrt(nrows) * EPS * lmax',
     'if lmin <= 0',
     'test_kappa_uncertified_is_infinite'),
    ('c formula tau factor',
     'Nk = 7 + 2 * A.N_A + 14 * tau',
     'Nk = 7 + 2 * A.N_A + 4 * tau',
     'test_c_formula_mode_closed_form'),
    ('c formula N_A factor',
     'Nk = 7 + 2 * A.N_A + 14 * tau',
     'Nk = 7 + A.N_A + 14 * tau',
     'test_c_formula_mode_closed_form'),
    ('check threshold upside down',
     'tj = eps_star / (c_check(j) * EPS * rn) if rn > 0 else math.inf',
     'tj = eps_star * rn / (c_check(j) * EPS) if rn > 0 else math.inf',
     'test_paper_observations_sec5'),
    ('in-loop check dropped',
     'if gamma_est >= tj:',
     'if False:',
     'test_in_loop_check_cuts_blocks_short[800-20]'),
    ('stop test on rGr, no sqrt',
     '        rn = math.sqrt(max(float(rGr_new), 0.0))\n        if rn <= eps_star:',
     '        rn = max(float(rGr_new), 0.0)\n        if rn <= eps_star:',
     'test_adaptive_with_s1_matches_classical'),
]


def _run(case):
    name, old, new, node = case
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    try:
        for sub in ("oracle", "workloads"):
            shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                            ignore=shutil.ignore_patterns("__pycache__"))
        os.makedirs(os.path.join(d, "tests"))
        shutil.copy(os.path.join(ROOT, "tests", "test_oracle_pins.py"), os.path.join(d, "tests"))
        if os.path.isdir(os.path.join(ROOT, "tests", "golden")):
            shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(d, "tests", "golden"))
        with open(os.path.join(d, "tests", "conftest.py"), "w") as f:
            f.write("import os, sys\nsys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))\n")
        path = os.path.join(d, "oracle", "ascg_oracle.py")
        text = open(path).read()
        if old not in text:
            return name, "pattern not found in the oracle"
        open(path, "w").write(text.replace(old, new, 1))
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                            "tests/test_oracle_pins.py::" + node], cwd=d, capture_output=True, text=True, timeout=600)
        if r.returncode == 1:
            return name, None
        return name, f"pin {node} did not fail (exit {r.returncode})"
    finally:
        shutil.rmtree(d, ignore_errors=True)


def test_every_planted_mistake_is_caught():
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(_run, MUTATIONS))
    missed = [(name, why) for name, why in results if why]
    assert not missed, missed
    assert len(results) == len(MUTATIONS) >= 30
