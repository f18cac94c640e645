"""The pins catch plausible mistakes: each case plants one mistake in a copy
of oracle.c (a wrong sign, index or constant, a dropped term or check),
builds it with gcc, and runs a fast selection of the pins against it in a
child process (mutant_checks.py); at least one pin must fail (a build that
aborts on an impossible state counts as caught).  The unchanged source must
pass the same selection."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.c")
OUT = os.path.join(ROOT, "_build", "oracle_mutants")  # the in-tree build folder

# name -> (text in oracle.c, replacement)
MUTANTS = {
    "lane-change direction flipped": ("const int d = (t % 2 == 0) ? +1 : -1;", "const int d = (t % 2 == 0) ? -1 : +1;"),
    "gap one cell too long": ("if (S[cell_index(o, l, k, y)] >= 0) return i - 1;",
                              "if (S[cell_index(o, l, k, y)] >= 0) return i;"),
    "slowdown from the wrong Philox word": ("if (r[0] < o->p_threshold) v -= 1;", "if (r[1] < o->p_threshold) v -= 1;"),
    "Philox Weyl constant off by one": ("const uint32_t W0 = 0x9E3779B9u,", "const uint32_t W0 = 0x9E3779B8u,"),
    "link end open only on the last link": ("((buf[o->lane_base[l] + k] < 0) || is_last_link(o, id))",
                                            "(is_last_link(o, id))"),
    "no room-behind check": ("for (uint32_t i = 1; i <= back; i++) {", "for (uint32_t i = 1; i < 1; i++) {"),
    "acceleration by two": ("uint32_t v = (uint32_t)o->vel[id] + 1;", "uint32_t v = (uint32_t)o->vel[id] + 2;"),
    "departures fill the highest free lane first": ("for (uint32_t q = 0; q < o->lanes[m]; q++) {",
                                                    "for (uint32_t q = o->lanes[m]; q-- > 0;) {"),
    "intersection priority reversed": (
        "for (uint32_t s = o->in_off[n]; s < o->in_off[n + 1]; s++) {",
        "for (uint32_t s = o->in_off[n + 1]; s-- > o->in_off[n];) {"),
    "transfer ignores the lane index": ("uint32_t pref = k < nl - 1 ? k : nl - 1;", "uint32_t pref = 0;"),
    "red and green swapped": ("return (o->t_now + offset) % cycle < green;", "return (o->t_now + offset) % cycle >= green;"),
    "plan-following side flipped": ("((int)j - (int)k) * d > 0) toward = 1;", "((int)j - (int)k) * d < 0) toward = 1;"),
    "accepted gap does not shrink": ("if (plan && !o->ring[l] && o->cells[l] - 1 - x < back) back = o->cells[l] - 1 - x;",
                                     ""),
    "yield gap counts cell 0": ("uint32_t lo = L > G ? L - G : 1;", "uint32_t lo = L > G ? L - G : 0;"),
    "yield check dropped": ("if (o->gap_accept[l] && !priority_gap_clear(o, o->cell, n, l)) continue;", ""),
    "travel time one step long": ("o->lt_sum[l] += t - o->t_enter[id];\n                    o->lt_cnt[l]++;\n                    o->t_enter[id] = (uint32_t)t;",
                                  "o->lt_sum[l] += t + 1 - o->t_enter[id];\n                    o->lt_cnt[l]++;\n                    o->t_enter[id] = (uint32_t)t;"),
    "moving counts standing vehicles": ("if (o->vel[id] > 0) st->moving++;", "if (o->vel[id] >= 0) st->moving++;"),
    "no lane change within vmax of a link end": (
        "int32_t id = o->s_start[cell_index(o, l, k, x)];\n                    if (id < 0) continue;",
        "int32_t id = o->s_start[cell_index(o, l, k, x)];\n"
        "                    if (id < 0 || (!o->ring[l] && o->cells[l] - 1 - x < vmax)) continue;"),
    "digest drops the lane": ("uint64_t b = ((uint64_t)cell << 16) | ((uint64_t)lane << 8) | v;",
                              "uint64_t b = ((uint64_t)cell << 16) | v;"),
}


def _build(name, text):
    os.makedirs(OUT, exist_ok=True)
    stem = "".join(ch if ch.isalnum() else "_" for ch in name)
    src, lib = os.path.join(OUT, stem + ".c"), os.path.join(OUT, stem + ".so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", lib], check=True)
    return lib


def _run(lib):
    return subprocess.run([sys.executable, os.path.join(HERE, "mutant_checks.py"), lib],
                          stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=600)


def test_unchanged_oracle_passes_the_selection():
    r = _run(_build("unchanged", open(SRC).read()))
    assert r.returncode == 0, r.stdout


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, "the mutated line is no longer in oracle.c"
    r = _run(_build(name, src.replace(old, new, 1)))
    assert r.returncode != 0, f"mistake not caught: {name}"
