"""Planted mistakes: each mutant of the oracle's C source must fail a pin.

A mutant is a temporary copy of ``oracle/slg_oracle.c`` with one plausible
slip (a wrong comparison, a dropped count, a wrong loop bound, a transposed
operand), compiled with gcc and swapped in for the real library. The checks
used here are the independent pins of ``test_oracle_pins``: the paper's worked
example and bitset brute force. CPU only.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests.test_oracle_pins import as_triples, bitset_pairs, csr_from_rows, parse_golden
import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "slg_oracle.c")

MUTANTS = {
    "threshold_strict": ("if (o >= s) {\n                if (p < cap)",
                         "if (o > s) {\n                if (p < cap)"),
    "skip_next_row": ("for (int32_t j = i + 1; j < m; ++j) {\n            const int32_t o = "
                      "orc_intersect(ei, ni, idx + off[j]",
                      "for (int32_t j = i + 2; j < m; ++j) {\n            const int32_t o = "
                      "orc_intersect(ei, ni, idx + off[j]"),
    "dropped_count": ("++c;\n            ++p;\n            ++q;", "++p;\n            ++q;"),
    "merge_compare": ("if (a[p] < b[q]) {", "if (a[p] <= b[q]) {"),
    "wrong_row_length": ("orc_intersect(ei, ni, idx + off[j], off[j + 1] - off[j]);\n"
                         "            if (o >= s) {\n                if (p < cap)",
                         "orc_intersect(ei, ni, idx + off[j], off[j + 1] - off[j] - 1);\n"
                         "            if (o >= s) {\n                if (p < cap)"),
    "transposed_operand": ("orc_intersect(ei, ni, idx + off[j], off[j + 1] - off[j]);\n"
                           "            if (o >= s) {\n                if (p < cap)",
                           "orc_intersect(idx + off[j], ni, ei, off[j + 1] - off[j]);\n"
                           "            if (o >= s) {\n                if (p < cap)"),
}


def _build_mutant(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o",
                           str(so), str(path)])
    return str(so)


def _pins_pass(golden_dir) -> bool:
    n, rows, pairs, *_ = parse_golden(os.path.join(golden_dir, "worked_example.txt"))
    off, idx = csr_from_rows(rows)
    for s in range(1, 5):
        if as_triples(*oracle.slg(off, idx, s)) != sorted(pairs.get(s, [])):
            return False
    for seed in range(6):
        h = synth.uniform_random(seed, 40, 30, 1, 10)
        rws = [h.row(i).tolist() for i in range(h.m)]
        for s in (1, 2, 3):
            if as_triples(*oracle.slg(h.off, h.idx, s)) != bitset_pairs(rws, s):
                return False
    return True


def test_real_oracle_passes(golden_dir):
    assert _pins_pass(golden_dir)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, golden_dir, monkeypatch):
    import ctypes
    real = oracle._load()
    lib = ctypes.CDLL(_build_mutant(tmp_path, name))
    for fn in ("oracle_slg",):
        getattr(lib, fn).restype = getattr(real, fn).restype
        getattr(lib, fn).argtypes = getattr(real, fn).argtypes
    monkeypatch.setattr(oracle, "_lib", lib)
    assert not _pins_pass(golden_dir), f"mutant {name} survived the pins"
