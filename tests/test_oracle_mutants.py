"""Plant plausible slips in a copy of the C oracle and check that the pin
suite (test_oracle_pins.py) rejects every one of them.  The mistakes are planted
on the CPU, in a temporary copy; the oracle in the repository is untouched."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lnf_oracle.c")

MUTANTS = {
    "drop_z_line": ("s += sample(v, cx, cy, cz + di);", ""),
    "corner_axis_slip": ("z + sz * d", "z + sy * d"),
    "truncating_round": ("(2 * a + b) / (2 * b)", "a / b"),
    "gate_strict": ("U < den * (uint64_t)p->threshold", "U <= den * (uint64_t)p->threshold"),
    "sigma_open_band": ("diff <= (int64_t)p->sigma_band", "diff < (int64_t)p->sigma_band"),
    "okada_closed": ("diff < p->okada_td", "diff <= p->okada_td"),
    "okada_no_centre": ("if (t != 0)\n                    continue;", "continue;"),
    "clamp_wrong_extent": ("z = clampi(z, 0, v->nz - 1);", "z = clampi(z, 0, v->ny - 1);"),
    "index_transposed": ("(z * v->ny + y) * v->nx + x", "(z * v->nx + y) * v->ny + x"),
    "entropy_ge": ("(int64_t)E > p->entropy_te", "(int64_t)E >= p->entropy_te"),
    "mean_shifted_cube": ("B += sample(v, x + i - r, y + j - r, z + k - r);",
                          "B += sample(v, x + i - r, y + j - r, z + k - r + (k == 0));"),
    "cluster_offset_doubled": ("x + sx * d, y + sy * d", "x + sx * 2 * d, y + sy * d"),
    "sum_of_squares_slip": ("q += (unsigned __int128)P * P;", "q += (unsigned __int128)P * P + (P > 200);"),
    "mean_gate_dropped": ("if (P0 < p->threshold || B < n * (uint64_t)p->threshold)",
                          "if (B < n * (uint64_t)p->threshold)"),
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
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"planted slip {name} survived the pins:\n{res.stdout[-2000:]}"
