"""Planted mistakes in a copy of the oracle must each fail a pin (CPU only).

Each case compiles ``oracle/esd_oracle.c`` with one plausible slip (a dropped term, a
wrong sign, a transposed operand, a wrong loop order), swaps it in for the real oracle
library, and checks that a pin of ``test_oracle_pins`` fails on it. The committed oracle
is never modified.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

SRC = open(os.path.join(os.path.dirname(oracle.__file__), "esd_oracle.c")).read()

MUTANTS = {
    # the paper's literal sign of beta in Algorithm DPCG
    "beta_sign": ("p[k] = z[k] + beta * p[k];", "p[k] = z[k] - beta * p[k];",
                  lambda: pins.test_cg_terminates_in_k_steps(4)),
    # Eq. x1 correction dropped: x = x_i instead of P x_i + W E^-1 W^T b
    "no_final_correction": ("    tall_vec_acc(n, s->m, s->W, u, 1.0, x);\n  }\ndone:",
                            "  }\ndone:", pins.test_deflation_with_exact_eigenvectors),
    # P applied instead of P^T (W and AW swapped inside the projection)
    "P_instead_of_PT": ("  tall_t_vec(s->n, s->m, s->W, v, f);\n  chol_solve(s->m, s->LE, f, u);\n"
                        "  tall_vec_acc(s->n, s->m, s->AW, u, -1.0, v);",
                        "  tall_t_vec(s->n, s->m, s->AW, v, f);\n  chol_solve(s->m, s->LE, f, u);\n"
                        "  tall_vec_acc(s->n, s->m, s->W, u, -1.0, v);",
                        pins.test_deflation_with_exact_eigenvectors),
    # IC(0): the sum over the common pattern of rows i and k dropped
    "ic0_no_update": ("          s -= Lva[pi] * Lva[pk];", "          (void)0;",
                      pins.test_ic0_is_exact_cholesky_on_full_pattern),
    # IC(0): the pivot uses a_ii instead of a_ii - sum l_ik^2
    "ic0_pivot": ("    for (int a = Lrp[i]; a < row_end; ++a) d -= Lva[a] * Lva[a];", "",
                  pins.test_ic0_is_exact_cholesky_on_full_pattern),
    # forward substitution in the reverse colour order
    "fwd_colour_order": ("  for (int c = 0; c < ncol; ++c) {\n#pragma omp parallel for schedule(static)\n"
                         "    for (int i = cp[c]; i < cp[c + 1]; ++i) {\n      double s = r[i];",
                         "  for (int c = ncol - 1; c >= 0; --c) {\n#pragma omp parallel for schedule(static)\n"
                         "    for (int i = cp[c]; i < cp[c + 1]; ++i) {\n      double s = r[i];",
                         lambda: pins.test_ic_apply_is_M_inverse("c1")),
    # backward substitution with L instead of L^T (row i's own entries)
    "bwd_transposed": ("      for (int e = Urp[i]; e < Urp[i + 1]; ++e) s -= Lva[Ua[e]] * z[Uj[e]];",
                       "      for (int a = Lrp[i]; a < Lrp[i + 1] - 1; ++a) s -= Lva[a] * z[Lci[a]];",
                       lambda: pins.test_ic_apply_is_M_inverse("small3d")),
    # subspace correction subtracted instead of added (Eq. mc)
    "sc_sign": ("    tall_vec_acc(n, s->m, s->W, u, 1.0, z);", "    tall_vec_acc(n, s->m, s->W, u, -1.0, z);",
                pins.test_subspace_correction_shifts_small_eigenvalue_by_one),
    # method B levels tol^(s/m) instead of tol^(s/(m+1))
    "sampling_b_levels": ("  while (lev < m && rel2 <= pow(tol2, (double)(lev + 1) / (double)(m + 1))) ++lev;",
                          "  while (lev < m && rel2 <= pow(tol2, (double)(lev + 1) / (double)m)) ++lev;",
                          lambda: pins.test_sampling_b_samples_first_crossings("c1")),
    # power method: the product kept without normalising it
    "power_no_normalise": ("    for (int i = 0; i < n; ++i) v[i] = work[i] / nv;", "    for (int i = 0; i < n; ++i) v[i] = work[i];",
                           lambda: pins.test_power_method_diagonal_closed_form(2)),
    # power method: one step fewer than asked (the estimate of v_{k-1})
    "power_step_count": ("  for (int step = 0; step < k; ++step) {\n    orc_spmv(n, rp, ci, va, v, work);",
                         "  for (int step = 1; step < k; ++step) {\n    orc_spmv(n, rp, ci, va, v, work);",
                         lambda: pins.test_power_method_diagonal_closed_form(5)),
    # power method: the estimate taken as ||A v|| instead of (v, A v)
    "power_norm_not_rq": ("  orc_spmv(n, rp, ci, va, v, work);\n  return orc_dot(n, v, work);",
                          "  orc_spmv(n, rp, ci, va, v, work);\n  return sqrt(orc_dot(n, work, work));",
                          lambda: pins.test_power_method_diagonal_closed_form(1)),
    # Appendix A: i_t summed without the alternating sign (schedule routine)
    "sampling_a_sign": ("      it += (l % 2 == 0) ? q : -q;", "      it += q;",
                        lambda: [pins.test_sampling_a_alternating_sign(*r)
                                 for r in pins._golden_sampling("sampling_method_a_sign.txt")]),
    # the same slip in the sampling step of the solve
    "sampling_a_sign_in_solve": ("    it += (l % 2 == 0) ? q : -q;\n    q /= m;\n  }\n  int slot",
                                 "    it += q;\n    q /= m;\n  }\n  int slot",
                                 pins.test_sampling_a_in_solve_follows_the_alternating_sign),
    # residual update with the wrong sign
    "residual_sign": ("        r[k] -= alpha * q[k];", "        r[k] += alpha * q[k];",
                      pins.test_iccg_solves_the_system),
}


@pytest.fixture
def mutant(tmp_path, monkeypatch):
    def make(name):
        old, new, _ = MUTANTS[name]
        assert SRC.count(old) == 1, f"mutation anchor for {name} not unique"
        src = tmp_path / f"{name}.c"
        src.write_text(SRC.replace(old, new))
        so = tmp_path / f"{name}.so"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(src), "-lm"])
        monkeypatch.setattr(oracle, "_lib", oracle.load(str(so)))
    return make


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, mutant):
    mutant(name)
    with pytest.raises((AssertionError, ArithmeticError, ValueError, np.linalg.LinAlgError)):
        MUTANTS[name][2]()


def test_lanczos_dropped_term_is_caught(monkeypatch):
    """The Lanczos matrix without the beta/alpha diagonal term misses the closed form."""
    def wrong(alpha, beta):
        a = np.asarray(alpha, dtype=np.float64)
        b = np.asarray(beta, dtype=np.float64)[: len(a) - 1]
        return 1.0 / a, np.sqrt(b) / a[:-1]
    monkeypatch.setattr(oracle, "lanczos_tridiagonal", wrong)
    with pytest.raises(AssertionError):
        pins.test_lanczos_1d_laplacian_closed_form()


import test_oracle_grad as grad_pins  # noqa: E402

GRAD_MUTANTS = {
    # dT/dk_a with k_a where k_b belongs
    "dT_dk_operand": ("_face_dT_dka", lambda ka, kb, inv_h2: 2.0 * ka * ka / ((ka + kb) * (ka + kb)) * inv_h2),
    # the Dirichlet faces forgotten
    "no_boundary_term": ("_boundary_dL_dk", lambda lam_c, x_c, inv_h2: 0.0 * lam_c),
    # dL/dT with the wrong sign
    "dL_dT_sign": ("_face_dL_dT", lambda la, lb, xa, xb: (la - lb) * (xa - xb)),
}


@pytest.mark.parametrize("name", sorted(GRAD_MUTANTS))
def test_planted_gradient_mistake_is_caught(name, monkeypatch):
    attr, wrong = GRAD_MUTANTS[name]
    monkeypatch.setattr(oracle, attr, wrong)
    with pytest.raises(AssertionError):
        grad_pins.test_theta_gradient_matches_finite_differences("3d_3x4x2_steady")


def _scale_with(dfun, two_sided):
    def wrong(prob):
        import copy
        rp = np.asarray(prob.rowptr, dtype=np.int64)
        ci = np.asarray(prob.colind, dtype=np.int64)
        va = np.asarray(prob.val, dtype=np.float64)
        rows = np.repeat(np.arange(prob.n), np.diff(rp))
        d = dfun(va[rows == ci])
        out = copy.copy(prob)
        out.val = (va * d[rows]) * d[ci] if two_sided else va * d[rows] * d[rows]
        return out, d
    return wrong


SCALE_MUTANTS = {
    # d_i^2 applied on the row side only (not symmetric)
    "scale_one_sided": (_scale_with(lambda a: 1.0 / np.sqrt(a), False),
                        pins.test_diag_scaled_matrix_symmetric_unit_diagonal),
    # d_i = 1/a_ii instead of 1/sqrt(a_ii)
    "scale_no_sqrt": (_scale_with(lambda a: 1.0 / a, True), pins.test_diag_scaled_laplacian_closed_form),
}


@pytest.mark.parametrize("name", sorted(SCALE_MUTANTS))
def test_planted_scaling_mistake_is_caught(name, monkeypatch):
    wrong, pin = SCALE_MUTANTS[name]
    monkeypatch.setattr(oracle, "diag_scale", wrong)
    with pytest.raises(AssertionError):
        pin()
