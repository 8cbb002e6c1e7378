"""Plant plausible mistakes in a copy of the oracle's C source and check that
the pin suite catches every one (it runs on the CPU only; the committed oracle
is never modified)."""
import os

import pytest

import oracle
from oracle_pins import ALL_PINS

# (name, text in lnbnn_oracle.c, replacement)
MUTANTS = [
    ("dropped square", "s += e * e;", "s += e;"),
    ("unsigned wrap in difference", "int32_t e = (int32_t)a[t] - (int32_t)b[t];",
     "int32_t e = (uint8_t)(a[t] - b[t]);"),
    ("dropped coordinate", "for (int t = 0; t < ORACLE_D; ++t) {", "for (int t = 1; t < ORACLE_D; ++t) {"),
    ("dist_B is the k-th neighbour", "const int64_t dist_B = nd[k];", "const int64_t dist_B = nd[k - 1];"),
    ("sign of the update", "totals[c] += dist_C - dist_B;", "totals[c] += dist_B - dist_C;"),
    ("ties to the higher index", "(d1 == d2 && j1 < j2)", "(d1 == d2 && j1 > j2)"),
    ("argmax instead of argmin", "if (t[c] < t[best]) best = c;", "if (t[c] > t[best]) best = c;"),
    ("ties to the highest class", "if (t[c] < t[best]) best = c;", "if (t[c] <= t[best]) best = c;"),
    ("class of the wrong neighbour", "const int32_t c = labels[nj[a]];", "const int32_t c = labels[a];"),
    ("repeated class counted twice", "if (seen) continue;", "(void)seen;"),
    ("dist_C not the minimum", "if (labels[nj[b]] == c && nd[b] < dist_C) dist_C = nd[b];",
     "if (labels[nj[b]] == c && nd[b] > dist_C) dist_C = nd[b];"),
    ("per-class min keeps the max", "if (d < cmin[labels[j]]) cmin[labels[j]] = d;",
     "if (d > cmin[labels[j]] || cmin[labels[j]] == INT64_MAX) cmin[labels[j]] = d;"),
    ("NBNN adds the wrong class", "for (int32_t c = 0; c < J->C; ++c) t[c] += s1[c];",
     "for (int32_t c = 0; c < J->C; ++c) t[c] += s1[J->C - 1 - c];"),
    ("insertion drops the wrong slot", "int32_t p = (len < kk) ? len++ : kk - 1;",
     "int32_t p = (len < kk) ? len++ : (kk > 1 ? kk - 2 : 0);"),
    ("closed form uses the k-th value", "const int64_t dist_B = all[k];", "const int64_t dist_B = all[k - 1];"),
    ("coarse: no shift", "#define ORACLE_SHIFT 64", "#define ORACLE_SHIFT 0"),
    ("E4M3: ties away from zero", "if (2 * rem > step || (2 * rem == step && (n & 1))) ++n;",
     "if (2 * rem >= step) ++n;"),
    ("E4M3: one mantissa bit short", "const int32_t step = 1 << (p - 3);", "const int32_t step = 1 << (p - 2);"),
    ("coarse: dropped reference norm", "nr += rs * rs;", "nr += 0;"),
    ("coarse: cross term not doubled", "return nq + nr - 2 * dot;", "return nq + nr - dot;"),
    ("coarse: no rerank", "const int64_t j = cj[a], d = sqdist(q, ref + j * ORACLE_D, &plain_metric);",
     "const int64_t j = cj[a], d = cd[a];"),
    ("coarse: shortlist by exact distance", "const int64_t c = coarse(q, ref + j * ORACLE_D);",
     "const int64_t c = sqdist(q, ref + j * ORACLE_D, &plain_metric);"),
    ("location: weight dropped", "return (int64_t)s + mt->w * loc;", "return (int64_t)s + loc;"),
    ("location: weight squared", "return (int64_t)s + mt->w * loc;", "return (int64_t)s + mt->w * mt->w * loc;"),
    ("location: ignored", "for (int t = ORACLE_D; t < mt->stride; ++t) {", "for (int t = ORACLE_D; t < ORACLE_D; ++t) {"),
    ("location: references at 128-byte stride", "ref + j * mt->stride, mt)", "ref + j * ORACLE_D, mt)"),
    ("location: queries at 128-byte stride", "J->q + i * J->mt.stride", "J->q + i * ORACLE_D"),
]


def test_mutants_are_distinct_edits():
    src = oracle.source()
    for name, old, new in MUTANTS:
        assert src.count(old) >= 1, name


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, old, new):
    src = oracle.source()
    assert old in src
    path = oracle.compile_source(src.replace(old, new), os.path.join(tmp_path, "mutant.so"))
    mutant = oracle.Oracle(path)
    caught = []
    for pin in ALL_PINS:
        try:
            pin(mutant)
        except (AssertionError, oracle.OracleError, IndexError, ValueError):
            caught.append(pin.__name__)
    assert caught, f"no pin catches mutant '{name}'"
