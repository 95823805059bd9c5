"""Plant one plausible mistake at a time in a copy of the CPU oracle and
check that the pin suite catches every one of them (no GPU).

The copies are compiled into a temporary directory; the oracle source itself
is never modified."""
import os
import subprocess

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "rac_oracle.c")

MUTANTS = {
    # a transposed operand: read the relation the same way from both ends
    "transposed_relation": (
        "return (int)((N->rel[c * N->d + b] >> a) & 1u);",
        "return (int)((N->rel[c * N->d + a] >> b) & 1u);"),
    # a dropped term: supports no longer restricted to the input domain
    "supports_outside_input_domain": (
        "int in_support_set = allowed(N, c, side, a, b) && inD[(size_t)y * N->d + b];",
        "int in_support_set = allowed(N, c, side, a, b);"),
    # an off-by-one: value 0 of the far variable never counts as a support
    "support_loop_skips_value_0": (
        "for (int b = 0; b < N->d; ++b) {\n    int in_support_set",
        "for (int b = 1; b < N->d; ++b) {\n    int in_support_set"),
    # asynchronous sweeps (read the set being built instead of Dt^(k-1))
    "gauss_seidel_sweep": (
        "collect = supports_all_removed(&N, inD, Dt_prev, c, side, a);",
        "collect = supports_all_removed(&N, inD, Dt, c, side, a);"),
    # the final, removal-free sweep not counted
    "sweep_count_off_by_one": ("*iterations = k;", "*iterations = k - 1;"),
    # Proposition 2 applied to the wrong end of the constraint
    "incremental_wrong_end": ("!lost_prev[other(&N, c, side)]", "!lost_prev[x]"),
    # wipe-out never reported at the fixpoint
    "status_ignores_empty_domain": ("st = some_empty ? ORACLE_WIPEOUT : ORACLE_OK;",
                                    "st = ORACLE_OK;"),
    # AC-3 re-queues only the constraint it just revised
    "ac3_wrong_requeue": ("if (c2 == c) continue;", "if (c2 != c) continue;"),
    # AC-3 looks for supports in its own domain
    "ac3_support_in_own_domain": ("has_support = D[(size_t)y * d + b] && allowed(&N, c, side, a, b);",
                                  "has_support = D[(size_t)x * d + b] && allowed(&N, c, side, a, b);"),
    # brute force accepts supports outside the candidate subset S.  (Keeping
    # only the last arc-consistent subset instead of the union is not a
    # mistake: arc-consistent subsets are closed under union, so the union
    # is also the numerically largest one and comes last.)
    "bruteforce_support_outside_subset": (
        "has_support_in_S = j >= 0 && ((S >> j) & 1u) && allowed(&N, c, side, a, b);",
        "has_support_in_S = j >= 0 && allowed(&N, c, side, a, b);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, "mutation target not found exactly once: " + name
    mutated = tmp_path / ("oracle_%s.c" % name)
    mutated.write_text(src.replace(before, after))
    lib_path = str(tmp_path / ("liboracle_%s.so" % name))
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-w",
                           "-o", lib_path, str(mutated)])
    lib = oracle.load(lib_path)
    fails = pins.run_all(lib, quick=True)
    assert fails, "planted mistake %r passed every pin" % name
