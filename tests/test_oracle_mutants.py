"""Plant plausible slips in a copy of the C oracle and check that the pin
suites (test_oracle_pins.py, test_oracle_aniso.py, test_oracle_local_entropy.py)
reject every one of them.  The mistakes are planted
on the CPU, in a temporary copy; the oracle in the repository is untouched."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lnf_oracle.c")

MUTANTS = {
    "drop_z_line": ("s += sample(v, cx, cy, cz + di);", ""),
    "corner_axis_slip": ("z + sz * d[2]", "z + sy * d[2]"),
    "truncating_round": ("(2 * a + b) / (2 * b)", "a / b"),
    "gate_strict": ("U < den * (uint64_t)p->threshold", "U <= den * (uint64_t)p->threshold"),
    "sigma_open_band": ("diff <= (int64_t)p->sigma_band", "diff < (int64_t)p->sigma_band"),
    "okada_closed": ("diff < p->okada_td", "diff <= p->okada_td"),
    "okada_no_centre": ("if (t != 0)\n                    continue;", "continue;"),
    "clamp_wrong_extent": ("z = clampi(z, 0, v->nz - 1);", "z = clampi(z, 0, v->ny - 1);"),
    "index_transposed": ("(z * v->ny + y) * v->nx + x", "(z * v->nx + y) * v->ny + x"),
    "entropy_ge": ("(int64_t)E > p->entropy_te", "(int64_t)E >= p->entropy_te"),
    "mean_shifted_cube": ("B += sample(v, x + i, y + j, z + k);",
                          "B += sample(v, x + i, y + j, z + k + (k == 0));"),
    "cluster_offset_doubled": ("x + sx * d[0], y + sy * d[1]", "x + sx * 2 * d[0], y + sy * d[1]"),
    # anisotropic forms
    "axis_radii_rotated": ("r[a] = p->aniso ? p->rad[a] : p->radius;",
                           "r[a] = p->aniso ? p->rad[(a + 1) % 3] : p->radius;"),
    "aniso_ours_isotropic_denominator": ("9ull * (uint64_t)(2 * r[0] + 1 + 2 * r[1] + 1 + 2 * r[2] + 1)",
                                         "27ull * (uint64_t)(2 * r[0] + 1)"),
    "okada_arm_of_x": ("const int arm = axis < 0 ? 0 : r[axis];", "const int arm = axis < 0 ? 0 : r[0];"),
    "cross_cluster_y_arm_from_x": ("for (int t = 1; t <= r[1]; ++t)\n                U += sample(v, cx, cy - t, cz)",
                                   "for (int t = 1; t <= r[0]; ++t)\n                U += sample(v, cx, cy - t, cz)"),
    "sum_of_squares_slip": ("q += (unsigned __int128)P * P;", "q += (unsigned __int128)P * P + (P > 200);"),
    "mean_gate_dropped": ("if (P0 < p->threshold || B < n * (uint64_t)p->threshold)",
                          "if (B < n * (uint64_t)p->threshold)"),
    # the entropy filter with local probabilities
    "local_entropy_ge": ("crit > m * p->entropy_lte", "crit >= m * p->entropy_lte"),
    "local_entropy_every_tap": ("        if (!first)\n            continue;\n        int64_t c = 0;",
                                "        int64_t c = 0;"),
    "local_entropy_no_gate": ("    if (P0 < p->threshold)\n        return 0;\n    return crit > m",
                              "    return crit > m"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_planted_slip(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new)
    c = tmp_path / "mut.c"
    c.write_text(mutated)
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(c)])
    env = dict(os.environ, LNF_ORACLE_SO=str(so))
    try:   # the pin suites over 4 worker processes where pytest-xdist is installed
        import xdist  # noqa: F401
        par = ["-n", "4"]
    except ImportError:
        par = []
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + par + [
                          # the short local-entropy suite first: -x stops at the first failure
                          os.path.join(ROOT, "tests", "test_oracle_local_entropy.py"),
                          os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                          os.path.join(ROOT, "tests", "test_oracle_aniso.py")],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    # a pin test must have failed (exit 1, or 2 when -x stopped the xdist workers);
    # a collection or worker error alone proves nothing
    failed = re.search(r"\b\d+ failed\b", res.stdout) is not None
    assert res.returncode in (1, 2) and failed, \
        f"planted slip {name}: pins exit {res.returncode}:\n{res.stdout[-2000:]}"
