"""Plants mistakes in copies of the oracle and checks that the pins catch them.

Each mutant is oracle.cpp with one plausible slip (a flipped sign, a dropped
term, a transposed operand, a wrong index or root), compiled to a temporary
library on the CPU.  The pin battery of tests/oracle_pins.py must fail on
every mutant; the unmodified oracle passes it (tests/test_oracle.py).
"""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle
import oracle_pins

MUTANTS = {
    "curvature_sign": ("return (-double(q) * kA * B) * w;", "return (double(q) * kA * B) * w;"),
    "p2z_path_cot_for_tan": ("h = (Z - p[PZ]) * tan(p[PTHETA]);", "h = (Z - p[PZ]) / tan(p[PTHETA]);"),
    "p2r_one_root_family": ("T psi = (k == 0) ? alpha + a1 : alpha + (kPi - a1);", "T psi = alpha + a1;"),
    "jacobian_theta_not_seeded": ("pd[i].d[i] = T(1.0);", "pd[i].d[i] = T(i == PTHETA ? 0.0 : 1.0);"),
    "covariance_transposed_J": ("acc = acc + JC[i][k] * J[j][k];", "acc = acc + JC[i][k] * J[k][j];"),
    "hit_error_dropped_from_S": ("S[a][b] = acc + v;", "S[a][b] = acc;"),
    "residual_sign": ("acc = acc + Hp[a][k] * (m[k] - t.p[k]);", "acc = acc + Hp[a][k] * (t.p[k] - m[k]);"),
    "p2r_radial_instead_of_azimuthal": ("Hp[0][0] = -sin(phih); Hp[0][1] = cos(phih);",
                                        "Hp[0][0] = cos(phih); Hp[0][1] = sin(phih);"),
    "covariance_update_sign": ("t.C[i][j] = t.C[i][j] - acc;", "t.C[i][j] = t.C[i][j] + acc;"),
    "phi_wrap_sign": ("t.p[PPHI] = t.p[PPHI] + k * (2.0 * kPi);", "t.p[PPHI] = t.p[PPHI] - k * (2.0 * kPi);"),
    "gain_wrong_column": ("K[i][a] = CHt[i][0] * Si[0][a] + CHt[i][1] * Si[1][a];",
                          "K[i][a] = CHt[i][0] * Si[0][a] + CHt[i][0] * Si[1][a];"),
    "chi2_missing_offdiagonal": ("chi2 = chi2 + r[a] * Si[a][b] * r[b];",
                                 "if (a == b) chi2 = chi2 + r[a] * Si[a][b] * r[b];"),
    "find_takes_the_largest_chi2": ("if (value(c) < best_chi2) {", "if (value(c) > best_chi2) {"),
    "find_updates_with_the_first_candidate": (
        "T c = kalman_update(mode, t, cpos[l * ncand + best], ccov[l * ncand + best], st);",
        "T c = kalman_update(mode, t, cpos[l * ncand], ccov[l * ncand], st);"),
    "find_tries_candidates_on_the_track": (
        "T c = kalman_update(mode, trial, cpos[l * ncand + k], ccov[l * ncand + k], ignored);",
        "T c = kalman_update(mode, t, cpos[l * ncand + k], ccov[l * ncand + k], ignored);"),
    "flip_keeps_the_charge": ("    t.q = -t.q;\n", "\n"),
    "flip_keeps_the_sign_of_w": ("    t.p[PW] = -t.p[PW];\n", "\n"),
    "flip_negates_the_w_variance": ("    st |= ST_CHARGE_FLIP;",
                                    "    t.C[PW][PW] = -t.C[PW][PW];\n    st |= ST_CHARGE_FLIP;"),
    "flip_leaves_the_covariance": ("      t.C[PW][i] = -t.C[PW][i];\n      t.C[i][PW] = -t.C[i][PW];\n", ""),
    "helix_z_uses_tan": ("out[PZ] = p[PZ] + h * cos(p[PTHETA]) / sin(p[PTHETA]);",
                         "out[PZ] = p[PZ] + h * sin(p[PTHETA]) / cos(p[PTHETA]);"),
}


def _build_mutant(name, tmpdir):
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.cpp")).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    d = os.path.join(tmpdir, name)
    os.makedirs(d, exist_ok=True)
    shutil.copy(os.path.join(os.path.dirname(oracle.__file__), "dual.hpp"), d)
    with open(os.path.join(d, "oracle.cpp"), "w") as f:
        f.write(src.replace(old, new))
    out = os.path.join(d, "liboracle.so")
    cmd = oracle.build_command(out)
    cmd[cmd.index(os.path.join(os.path.dirname(oracle.__file__), "oracle.cpp"))] = os.path.join(d, "oracle.cpp")
    cmd[1] = "-O1"
    subprocess.run(cmd, check=True)
    return out


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("mutants"))
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        paths = dict(zip(MUTANTS, ex.map(lambda n: _build_mutant(n, tmp), MUTANTS)))
    return paths


def _caught_by(orc):
    caught = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(orc)
        except Exception:  # an assertion, or a numerical failure such as a
            caught.append(pin.__name__)  # failed Cholesky
    return caught


@pytest.mark.slow
@pytest.mark.parametrize("name", list(MUTANTS))
def test_mutant_is_caught(mutant_libs, name):
    caught = _caught_by(oracle.Oracle(mutant_libs[name]))
    assert caught, f"no pin catches the planted mistake {name}"
