"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a transposed
operand, an off-by-one) in a copy of the oracle's C source, builds it on the
CPU, and runs the pin tests against that copy in a subprocess: at least one
pin must fail.  The committed oracle is never modified.
"""
import os
import subprocess
import sys

import pytest

from oracle.build import SRC, build_oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, original text, planted text, pin test files that must catch it)
MUTANTS = [
    ("m2l_sign", "double sign = ((b[0] + b[1] + b[2]) & 1) ? -1.0 : 1.0;", "double sign = 1.0;",
     "test_oracle_expansions.py"),
    ("m2l_factorial_transposed", "orc_term e = {t, u, js, sign * orc_mfact(s) / orc_mfact(a)};",
     "orc_term e = {t, u, js, sign * orc_mfact(s) / orc_mfact(b)};", "test_oracle_expansions.py"),
    ("m2m_shift_reversed", "double delta[3] = {Xc[0] - Xp[0], Xc[1] - Xp[1], Xc[2] - Xp[2]};",
     "double delta[3] = {Xp[0] - Xc[0], Xp[1] - Xc[1], Xp[2] - Xc[2]};", "test_oracle_expansions.py"),
    ("l2l_missing_mfact", "orc_mfact(s) / (orc_mfact(a) * orc_mfact(b))", "orc_mfact(s) / orc_mfact(a)",
     "test_oracle_expansions.py"),
    ("taylor_dropped_term", "if (j2 >= 0) s2 += b[j2];", ";", "test_oracle_expansions.py"),
    ("l2p_gradient_factor", "g[a] += L[t] * k[a] * orc_mpow(r, km);", "g[a] += L[t] * orc_mpow(r, km);",
     "test_oracle_expansions.py"),
    ("p2m_offset_sign", "double d[3] = {y[3 * j] - X[0], y[3 * j + 1] - X[1], y[3 * j + 2] - X[2]};\n"
     "        for (int t = 0; t < mi->nterms; ++t)\n",
     "double d[3] = {X[0] - y[3 * j], X[1] - y[3 * j + 1], X[2] - y[3 * j + 2]};\n"
     "        for (int t = 0; t < mi->nterms; ++t)\n", "test_oracle_expansions.py"),
    ("p2p_gradient_sign", "gs[3 * i + 1] -= w * dy;", "gs[3 * i + 1] += w * dy;", "test_oracle_fmm.py"),
    ("direct_wrong_power", "double w = q[j] / (r2 * r);\n            gx -= w * dx;",
     "double w = q[j] / (r2 * r2);\n            gx -= w * dx;", "test_oracle_direct.py"),
    ("mac_without_sqrt", "float R = sqrtf(r2);", "float R = r2;", "test_oracle_tree.py"),
    ("split_rule_flipped", "f->radius[A] > f->radius[B]);", "f->radius[A] < f->radius[B]);",
     "test_oracle_tree.py"),
    ("leaf_test_off_by_one", "if (f->pcnt[c] <= f->ncrit ||", "if (f->pcnt[c] < f->ncrit ||",
     "test_oracle_tree.py"),
    ("morton_yz_swapped", "key |= (uint64_t)((iy >> b) & 1u) << (3 * b + 1);",
     "key |= (uint64_t)((iy >> b) & 1u) << (3 * b + 2);", "test_oracle_tree.py"),
    ("normalisation_no_margin", "h = h * (1.0 + 0x1p-20);", "h = h * 1.0;", "test_oracle_tree.py"),
    ("m2l_list_dropped_term", "L[tm->t] += tm->coef * M[tm->u] * b[tm->j];",
     "if (tm->u != 1) L[tm->t] += tm->coef * M[tm->u] * b[tm->j];", "test_oracle_expansions.py"),
    ("dipole_p2m_sign", "M[t] += p[3 * j + c] * orc_mpow(d, km) / orc_mfact(km);",
     "M[t] -= p[3 * j + c] * orc_mpow(d, km) / orc_mfact(km);", "test_oracle_adjoint.py"),
    ("hessian_l2p_diagonal_factor", "f *= km[b];", "f *= k[b];", "test_oracle_adjoint.py"),
    ("backward_p2p_hessian_sign", "hb[k] += qs[j] * (-bi[k] / r3 + 3.0 * bid * d[k] / r5);",
     "hb[k] += qs[j] * (bi[k] / r3 + 3.0 * bid * d[k] / r5);", "test_oracle_adjoint.py"),
    ("backward_dipole_field_dropped", "psi += as[j] / r + bjd / r3;", "psi += as[j] / r;",
     "test_oracle_adjoint.py"),
    ("direct_backward_dq_sign", "s_dq += ai / r - (bi[0] * d[0]", "s_dq += ai / r + (bi[0] * d[0]",
     "test_oracle_adjoint.py"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,orig,planted,target", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, orig, planted, target):
    src = open(SRC).read()
    assert src.count(orig) == 1, "mutation anchor not unique: " + name
    mut_src = tmp_path / "fmm_oracle_mutant.c"
    mut_src.write_text(src.replace(orig, planted))
    lib = build_oracle(force=True, src=str(mut_src), lib=str(tmp_path / "liborc_mutant.so"))
    env = dict(os.environ, ORC_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", target)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "pins did not catch mutant %s:\n%s" % (name, r.stdout[-2000:])
