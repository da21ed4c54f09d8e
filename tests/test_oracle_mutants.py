"""Plants plausible mistakes in a copy of the oracle's C source and checks that the pin
battery catches every one (a wrong comparison, a dropped merge, a wrong neighbour index,
an off-by-one, a lost union, a non-canonical numbering, ...).  The mutants are built on
the CPU into a temporary directory and run in a child process with a time limit, since
a broken union-find may loop or crash; a hang or a crash counts as caught.
"""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ccl_oracle.c")

# (id, old text, new text, which occurrence of old)
MUTANTS = [
    ("merge_compare_flipped", "if (p[rootx] > p[rooty]) {", "if (p[rootx] < p[rooty]) {", 0),
    ("merge_splice_continues_wrong", "rootx = z;", "rootx = p[rooty];", 0),
    ("copy_ca_drops_merge",
     "LAB(y, x) = rem_merge(p, LAB(y - 1, x + 1), LAB(y - 1, x - 1)); /* copy(c,a) */",
     "LAB(y, x) = p[LAB(y - 1, x + 1)]; /* copy(c,a) */", 0),
    ("copy_a_wrong_index", "LAB(y, x) = p[LAB(y - 1, x - 1)];", "LAB(y, x) = p[LAB(y - 1, x)];", 0),
    ("flatten_root_test_off_by_one", "if (p[i] < i) {", "if (p[i] <= i) {", 0),
    ("flatten_skips_jump", "p[i] = p[p[i]];", "p[i] = p[i];", 0),
    ("aremsp_garbled_merge_a", "rem_merge(p, LAB(i, x), LAB(i - 1, x - 1));",
     "rem_merge(p, LAB(i, x), LAB(i, x));", 0),
    ("aremsp_g_copies_wrong_neighbour", "LAB(i + 1, x) = LAB(i, x - 1);",
     "LAB(i + 1, x) = LAB(i + 1, x - 1);", 0),
    ("aremsp_d_branch_sign", "if (!b) {", "if (b) {", 0),
    ("paremsp_boundary_drops_c", "if (x + 1 < w && LAB(i - 1, x + 1) != 0)",
     "if (x + 1 < w && LAB(i - 1, x + 1) != 0 && 0)", 0),
    ("paremsp_first_label_zero", "lab_t count = (lab_t)(start[t] * w + 1);",
     "lab_t count = (lab_t)(start[t] * w);", 0),
    ("merger_link_no_op", "if (!cas_lab(&p[rootx], px, py))",
     "if (!cas_lab(&p[rootx], px, px))", 0),
    ("bfs_lost_direction", "static const int dy8[8] = {-1, -1, -1, 0, 0, 1, 1, 1};",
     "static const int dy8[8] = {-1, -1, -1, 0, 0, 1, 1, 0};", 0),
    ("view_reads_past_row_end", "x >= v->w", "x > v->w", 0),
    ("canonical_map_identity", "map[l] = next++;", "map[l] = l;", 0),
    ("cclremsp4_drops_merge",
     "LAB(y, x) = rem_merge(p, LAB(y - 1, x), LAB(y, x - 1));   /* copy(b,d) */",
     "LAB(y, x) = p[LAB(y - 1, x)];   /* copy(b,d) */", 0),
]

CHILD = r"""
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle
from _pins import run_battery
orc = oracle.Oracle(oracle.load({so!r}))
errs = run_battery(orc, stop_early=True)
print(errs[:1])
sys.exit(1 if errs else 0)
"""


def _mutate(text, old, new, occ):
    idx = -1
    for _ in range(occ + 1):
        idx = text.find(old, idx + 1)
        assert idx >= 0, f"anchor not found: {old!r}"
    return text[:idx] + new + text[idx + len(old):]


@pytest.mark.parametrize("mid,old,new,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(mid, old, new, occ, tmp_path):
    text = open(SRC).read()
    mutated = _mutate(text, old, new, occ)
    assert mutated != text
    src = tmp_path / f"{mid}.c"
    src.write_text(mutated)
    so = str(tmp_path / f"lib_{mid}.so")
    oracle.compile_oracle(str(src), so)
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), so=so)
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                           timeout=120, env={**os.environ, "OMP_NUM_THREADS": "4"})
    except subprocess.TimeoutExpired:
        return  # a hang is a caught mistake
    assert r.returncode != 0, f"mutant {mid} passed every pin:\n{r.stdout}\n{r.stderr}"
