"""The oracle's pins must catch plausible mistakes in the oracle itself.

Each case writes one planted mistake into a private copy of the oracle and
its pins -- in oracle.c a dropped update, a set left unintersected, a wrong
pivot domain or tie order, a wrong tie order in the peel, a hash over the
wrong ids, a miscounted work term; in the estimator's references
(features.py, mlp.py) a wrong excluded-set cap, a wrong neighbourhood or
aggregate, a missing bias correction -- rebuilds it there, and runs
tests/test_oracle.py against it. The mutant must fail at least one pin
(pytest exit code 1). Nothing here touches the GPU engine.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "x_p_not_grown": ("oracle.c", "        XP[pos] = v;\n        nxp++;", "        XP[pos] = v;"),
    "child_x_p_not_intersected": ("oracle.c", "int32_t ncxp = intersect_nbrs(g, XP, nxp, v, cXP);",
                                  "int32_t ncxp = nxp; memcpy(cXP, XP, (size_t)nxp * sizeof(int32_t));"),
    "ip_rule_scans_x_x": ("oracle.c", "g->mode == ORACLE_PIVOT_FULL ? nxx : 0", "nxx"),
    "leaf_ignores_x_x": ("oracle.c", "if (np == 0 && nxp == 0 && nxx == 0)", "if (np == 0 && nxp == 0)"),
    "pivot_ties_to_largest_rank": ("oracle.c", "(score == best && u < best_u)", "(score == best && u > best_u)"),
    "work_bound_off_by_one": ("oracle.c", ": np - 1;", ": np;"),
    "work_one_word_per_branch": ("oracle.c", "w->work += 2ull * (uint64_t)w->words", "w->work += 1ull * (uint64_t)w->words"),
    "peel_sub_round_descending_id": ("oracle.c", "            int32_t v = S[i];\n            if (rank) rank[v] = next;",
                                     "            int32_t v = S[ns - 1 - i];\n            if (rank) rank[v] = next;"),
    "hash_over_ranks": ("oracle.c", "w->ids[i] = w->g->order[w->R[i]];", "w->ids[i] = w->R[i];"),
    "features_x0_cap_takes_largest_ids": ("features.py", "X0c = sorted(X0)[:XCAP]", "X0c = sorted(X0)[-XCAP:]"),
    "features_two_hop_over_p0_only": ("features.py", "sum(deg[u] for u in nb[v])", "sum(deg[u] for u in P0)"),
    "features_min_core_for_max": ("features.py", "max((int(core[u]) for u in P0), default=0)",
                                  "min((int(core[u]) for u in P0), default=0)"),
    "adam_without_bias_correction": ("mlp.py", "m_hat = m / (1.0 - ADAM_B1 ** t)", "m_hat = m"),
    "adam_eps_inside_sqrt": ("mlp.py", "np.sqrt(v_hat) + ADAM_EPS", "np.sqrt(v_hat + ADAM_EPS)"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    fname, old, new = MUTANTS[name]
    with open(os.path.join(ROOT, "oracle", fname)) as f:
        src = f.read()
    # the planted text must still be in the oracle: if this fails, the oracle
    # changed and the mutant needs restating
    assert src.count(old) == 1
    skip = shutil.ignore_patterns("*.so", "*.so.tmp*", "__pycache__")
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle", ignore=skip)
    shutil.copytree(os.path.join(ROOT, "gen"), tmp_path / "gen", ignore=skip)
    (tmp_path / "tests").mkdir()
    for f in ("conftest.py", "test_oracle.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests" / f)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), tmp_path / "tests" / "golden")
    with open(tmp_path / "oracle" / fname, "w") as f:
        f.write(src.replace(old, new))
    # the mutant must build, so that a pin failure, not a compile error, is what catches it
    b = subprocess.run([sys.executable, "-c", "import oracle.build as b; b.build(force=True)"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=300)
    assert b.returncode == 0, b.stderr[-2000:]
    p = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle.py", "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    tail = "\n".join(p.stdout.strip().splitlines()[-3:])
    assert p.returncode == 1, "mutant %s was not caught (pytest exit %d):\n%s" % (name, p.returncode, tail)
