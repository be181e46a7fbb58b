"""The oracle's pins catch plausible mistakes.

Each case copies oracle/forward.c to a temporary directory, plants one
mistake (a dropped term, a wrong index or comparison, a skipped cleaning
step, a reversed order), builds it with gcc and runs a compact set of the
pins against it.  At least one pin must fail for every mutant.  Nothing runs
on a GPU and the committed oracle is never modified.
"""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from graphgen import families as fam
from tests import helpers

# Not listed: removing the per-list sort.  The lists are filled in the sorted
# order of the cleaned edge array, which already leaves every forward list in
# ascending id order (entries below the owner's id arrive first, ascending,
# then those above it), so that mutant computes the same function.
MUTANTS = {
    "drop_t_w": ("if (t) { ++t[u]; ++t[v]; ++t[w]; }", "if (t) { ++t[u]; ++t[v]; }"),
    "wrong_t_index": ("if (t) { ++t[u]; ++t[v]; ++t[w]; }", "if (t) { ++t[u]; ++t[u]; ++t[w]; }"),
    "merge_advances_wrong_side": ("if (nbr[i] < nbr[j]) {\n          ++i;",
                                  "if (nbr[i] < nbr[j]) {\n          ++j;"),
    "merge_bound_off_by_one": ("while (i < iend && j < jend) {", "while (i + 1 < iend && j < jend) {"),
    "no_dedup": ("if (m == 0 || e[i] != e[m - 1]) e[m++] = e[i];", "e[m++] = e[i];"),
    "keeps_self_loops": ("if (a == b) continue; /* self-loop */", ""),
    "reversed_degree_order": ("if (deg[u] != deg[v]) return deg[u] < deg[v];",
                              "if (deg[u] != deg[v]) return deg[u] > deg[v];"),
    "degree_counts_one_end": ("    ++d[(int32_t)(e[i] >> 32)];\n    ++d[(int32_t)(e[i] & 0xffffffffu)];\n  }\n\n  /* orient",
                              "    ++d[(int32_t)(e[i] >> 32)];\n  }\n\n  /* orient"),
}


def _pins_pass() -> bool:
    """A compact subset of the pins; False as soon as one fails."""
    try:
        for n, m, seed in [(12, 70, 1), (30, 300, 2), (64, 1200, 3)]:
            s, d, n = fam.random_multigraph(n, m, seed)
            r = oracle.forward(s, d, n)
            T, t = helpers.brute_force(s, d, n)
            if r["T"] != T or not np.array_equal(r["t"], t):
                return False
            if not np.array_equal(r["deg"], helpers.simple_degrees(s, d, n)):
                return False
            if int(r["t"].sum()) != 3 * r["T"]:
                return False
        for s, d, n in [fam.star(300), fam.wheel(200), fam.complete(30)]:
            r = oracle.forward(s, d, n)
            if r["max_out_degree"] > math.isqrt(2 * r["m"]):
                return False
        s, d, n = fam.wheel(10)
        if oracle.forward(s, d, n)["T"] != 10:
            return False
    except oracle.OracleError:
        return False
    return True


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("mutants")


def test_unmutated_copy_passes(mutant_dir):
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, mutant_dir):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTANTS[name]
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    path = os.path.join(str(mutant_dir), name + ".c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(str(mutant_dir), name + ".so")
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", path, "-o", so])
    saved = oracle._load()
    oracle._lib = oracle._bind(ctypes.CDLL(so))
    try:
        caught = not _pins_pass()
    finally:
        oracle._lib = saved
    assert caught, "no pin failed for mutant " + name
