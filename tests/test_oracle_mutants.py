"""Plant plausible mistakes in a copy of the oracle; some pin must fail for each.

The mutated copies are compiled into a temporary folder on the CPU. This
shows that the pins constrain the oracle: a dropped compare, a lost start, a
reversed or shifted index, an off-by-one report, a broken histogram, a wrong
tie order, a wrong fixed order, a threaded split that loses the halo, a start
or the offset of its positions, and a batch that searches the wrong text is
each caught.
"""
import os
import subprocess

import pytest

import oracle
from oracle_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "drop_last_compare": ("found = found && (t[i + j] == p[j]);\n            if (!found) break;                        /* go",
                          "found = found && (t[i + j] == p[j] || j + 1 == m);\n            if (!found) break;                        /* go"),
    "lose_last_start": ("for (uint64_t i = 0; i + m <= n; ++i) {          /* i = 1",
                        "for (uint64_t i = 0; i + m < n; ++i) {          /* i = 1"),
    "reversed_pattern": ("found = found && (t[i + j] == p[j]);\n            if (!found) break;                        /* go",
                         "found = found && (t[i + j] == p[m - 1 - j]);\n            if (!found) break;                        /* go"),
    "report_one_based": ("if (count < cap) pos[count] = i;", "if (count < cap) pos[count] = i + 1;"),
    "report_misses_overlap": ("if (count < cap) pos[count] = i;\n            count += 1;",
                              "if (count < cap) pos[count] = i;\n            count += 1;\n            i += m - 1;"),
    "histogram_skips_first": ("for (uint64_t x = 0; x < n; ++x) h256[t[x]] += 1;",
                              "for (uint64_t x = 1; x < n; ++x) h256[t[x]] += 1;"),
    "ties_descending": ("return x->q < y->q ? -1 : (x->q > y->q);", "return x->q > y->q ? -1 : (x->q < y->q);"),
    "order_swapped_groups": ("for (uint32_t r = 3; r < len; r += 3) out[k++] = pos[r - 1];   /* 3, 6, ...  */\n    for (uint32_t r = 2; r < len; r += 3) out[k++] = pos[r - 1];   /* 2, 5, ...  */",
                             "for (uint32_t r = 2; r < len; r += 3) out[k++] = pos[r - 1];   /* 2, 5, ...  */\n    for (uint32_t r = 3; r < len; r += 3) out[k++] = pos[r - 1];   /* 3, 6, ...  */"),
    "kmp_no_overlap": ("if (k == m) { ++c; k = fail[k - 1]; }", "if (k == m) { ++c; k = 0; }"),
    "hs_spaces_first": ("if (p[q] != 0x20) rest[nr++] = q;", "if (p[q] == 0x20) rest[nr++] = q;"),
    "threads_no_halo": ("uint64_t len = j->s1 - j->s0 + j->m - 1;\n    j->count = j->s1",
                        "uint64_t len = j->s1 - j->s0;\n    j->count = j->s1"),
    "threads_positions_not_shifted": ("for (uint64_t i = 0; i < j->count && i < j->cap; ++i) j->pos[i] += j->s0;",
                                      "for (uint64_t i = 0; i < j->count && i < j->cap; ++i) j->pos[i] += 0;"),
    "threads_last_start_lost": ("jobs[k].s1 = starts * (uint64_t)(k + 1) / (uint64_t)nt;",
                                "jobs[k].s1 = starts * (uint64_t)(k + 1) / (uint64_t)nt;\n"
                                "        if (k + 1 == nt && jobs[k].s1 > jobs[k].s0) jobs[k].s1 -= 1;"),
    "batch_first_text_only": ("const uint8_t* t = texts + text_off[x];", "const uint8_t* t = texts + text_off[0];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, f"mutation site for {name} not found exactly once"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(before, after))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", str(lib), str(mut)])
    o = oracle.Oracle(str(lib))
    failed = []
    for pin in ALL_PINS:
        try:
            pin(o)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin caught mutant {name}"
