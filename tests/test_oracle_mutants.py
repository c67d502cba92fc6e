"""Planted mistakes: each mutant is a copy of oracle.c with one plausible error (a dropped
term, a wrong index, a flipped comparison), compiled on the CPU.  The pins of
test_oracle_pins.py must reject every one of them, which shows they cover the oracle's
arithmetic.  The mistakes are planted only in temporary copies of the oracle.
"""
import os
import subprocess
import sys

import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = [
    ("occ exclusive instead of inclusive",
     "void or_occ4(const or_index *ix, int64_t k, int64_t occ[4]) { rank4(ix, k + 1, occ); }",
     "void or_occ4(const or_index *ix, int64_t k, int64_t occ[4]) { rank4(ix, k, occ); }"),
    ("listing 1 drops the +1",
     "        k = ix->C[b] + ok[b] + 1;\n        l = ix->C[b] + ol[b];\n    }\n    J->k_out",
     "        k = ix->C[b] + ok[b];\n        l = ix->C[b] + ol[b];\n    }\n    J->k_out"),
    ("listing 1 uses Occ(b,k) for the lower bound",
     "        or_occ4(ix, k - 1, ok);\n        or_occ4(ix, l, ol);\n        k = ix->C[b]",
     "        or_occ4(ix, k, ok);\n        or_occ4(ix, l, ol);\n        k = ix->C[b]"),
    ("C counts $", "    C[0] = 0;\n", "    C[0] = 1;\n"),
    ("C shifted by one symbol", "for (int b = 0; b < 4; ++b) C[b + 1] = C[b] + cnt[b];",
     "for (int b = 0; b < 4; ++b) C[b + 1] = C[b] + cnt[b < 3 ? b + 1 : b];"),
    ("SA-IS typing ignores runs",
     "t[i] = (s[i] < s[i + 1] || (s[i] == s[i + 1] && t[i + 1])) ? 1 : 0;",
     "t[i] = (s[i] < s[i + 1]) ? 1 : 0;"),
    ("SA-IS names every LMS substring apart",
     "        if (prev < 0 || !lms_equal(s, t, len, prev, p)) names++;",
     "        names++;"),
    ("naive SA orders the symbols backwards", "return p < n ? (int)R[p] + 1 : 0; /* $ = 0",
     "return p < n ? 4 - (int)R[p] : 0; /* $ = 0"),
    ("BWT takes the suffix's own first symbol",
     "            L[i] = R[SA[i] - 1];", "            L[i] = R[SA[i] < n ? SA[i] : 0];"),
    ("checkpoint table counts $ as A",
     "if (i <= n && ix->L[i] < 4) run[ix->L[i]]++;", "if (i <= n) run[ix->L[i] & 3]++;"),
    ("rank scan drops the last symbol",
     "    for (int64_t i = j * CK_STEP; i < p; ++i)\n        if (ix->L[i] < 4) out[ix->L[i]]++;",
     "    for (int64_t i = j * CK_STEP; i + 1 < p; ++i)\n        if (ix->L[i] < 4) out[ix->L[i]]++;"),
    ("mismatch not charged",
     "st_push(&S, i - 1, s.z - 1, s.gaps, nk[b], nl[b], 1, b);",
     "st_push(&S, i - 1, s.z, s.gaps, nk[b], nl[b], 1, b);"),
    ("deletion consumes a read symbol",
     "st_push(&S, i, s.z - 1, s.gaps + 1, nk[b], nl[b], 3, b);",
     "st_push(&S, i - 1, s.z - 1, s.gaps + 1, nk[b], nl[b], 3, b);"),
    ("insertion moves the interval",
     "st_push(&S, i - 1, s.z - 1, s.gaps + 1, s.k, s.l, 2, 0);",
     "st_push(&S, i - 1, s.z - 1, s.gaps + 1, s.k + 1, s.l, 2, 0);"),
    ("gap cap off by one", "int del_ok = s.gaps < X->max_gaps && del_allowed(X, i);",
     "int del_ok = s.gaps <= X->max_gaps && del_allowed(X, i);"),
    ("empty-interval children kept", "if (nk[b] > nl[b]) continue; /* bX does not occur */",
     "if (nk[b] > nl[b] + 1) continue; /* bX does not occur */"),
    ("prune too eagerly", "if (X->prune && s.i >= 0 && s.z < X->D[s.i]) continue;",
     "if (X->prune && s.i >= 0 && s.z <= X->D[s.i]) continue;"),
    ("prune with the wrong position", "if (X->prune && s.i >= 0 && s.z < X->D[s.i]) continue;",
     "if (X->prune && s.i >= 1 && s.z < X->D[s.i - 1]) continue;"),
    ("no dedup of intervals", "    if (v.size > 1) { /* sort and keep distinct intervals */",
     "    if (0) { /* sort and keep distinct intervals */"),
    ("empty match reported",
     "if (s.k >= 1) pv_push(X->out, (uint32_t)s.k, (uint32_t)s.l, (uint32_t)(X->z0 - s.z));",
     "pv_push(X->out, (uint32_t)s.k, (uint32_t)s.l, (uint32_t)(X->z0 - s.z));"),
    ("D window keeps the failing symbol", "            z++;\n            lo = 0;\n            hi = ix->n + 1;\n            d = 0;",
     "            z++;\n            lo = 0;\n            hi = ix->n + 1;\n            d = 0;\n            narrow(ix, &lo, &hi, 0, W[i]);\n            d = 1;"),
    ("D counts every failing extension twice", "            z++;\n            lo = 0;",
     "            z += 2;\n            lo = 0;"),
    ("reverse complement not complemented",
     "W[i] = strand ? (uint8_t)(3 - J->codes[s + m - 1 - i]) : J->codes[s + i];",
     "W[i] = strand ? (uint8_t)(J->codes[s + m - 1 - i]) : J->codes[s + i];"),
    ("closed form: suffix reaching $ counted larger",
     "            if (p + d >= n) { /* suffix reaches $ first: smaller */\n                rel = -1;",
     "            if (p + d >= n) { /* suffix reaches $ first: smaller */\n                rel = 1;"),
    ("hamming window inclusive bound", "        if (mm <= z) hits++;", "        if (mm < z) hits++;"),
    ("cost counts the differences left",
     "if (s.k >= 1) pv_push(X->out, (uint32_t)s.k, (uint32_t)s.l, (uint32_t)(X->z0 - s.z));",
     "if (s.k >= 1) pv_push(X->out, (uint32_t)s.k, (uint32_t)s.l, (uint32_t)s.z);"),
    ("dedup keeps an arbitrary cost", "    for (int t = 0; t < 3; ++t)\n        if (x[t] != y[t])",
     "    for (int t = 0; t < 2; ++t)\n        if (x[t] != y[t])"),
    ("canonical: no match after any insertion",
     "                if (W[i] == W[i + 1]) match_ok = 0;", "                match_ok = 0;"),
    ("canonical: mismatch allowed after an insertion",
     "                del_ok = 0;\n                mis_ok = 0;\n", "                del_ok = 0;\n"),
    ("canonical: deletion rule also at W[0]",
     "                ins_ok = 0;\n                if (i >= 1) {",
     "                ins_ok = 0;\n                if (i >= 0) {"),
    ("canonical: no insertion after any mismatch",
     "                if (W[i] == s.lb) ins_ok = 0;", "                ins_ok = 0;"),
    ("canonical: pass-through call counted as a node",
     "        if (canonical && !del_ok && !mis_ok && !match_ok) continue;\n", ""),
    ("deletion not charged",
     "st_push(&S, i, s.z - 1, s.gaps + 1, nk[b], nl[b], 3, b);",
     "st_push(&S, i, s.z, s.gaps + 1, nk[b], nl[b], 3, b);"),
    ("insertion not charged",
     "st_push(&S, i - 1, s.z - 1, s.gaps + 1, s.k, s.l, 2, 0);",
     "st_push(&S, i - 1, s.z, s.gaps + 1, s.k, s.l, 2, 0);"),
    ("block count takes l instead of l+1",
     "X->blocks += (s.k / X->interval == (s.l + 1) / X->interval) ? 1 : 2;",
     "X->blocks += (s.k / X->interval == s.l / X->interval) ? 1 : 2;"),
    ("closed form: l misses the -1", "    J->l_out[q] = less + pre - 1;",
     "    J->l_out[q] = less + pre;"),
    ("closed form: Occ at l drops the matching rows",
     "J->out8[8 * q + 4 + b] = oc_less[b] + oc_pre[b];", "J->out8[8 * q + 4 + b] = oc_less[b];"),
    ("occ sweep swaps the k and l halves", "        int half = (int)(s & 1);",
     "        int half = (int)(~s & 1);"),
    ("hamming window misses the last position", "    for (int64_t p = 0; p + m <= n; ++p) {",
     "    for (int64_t p = 0; p + m < n; ++p) {"),
    ("SA narrowing takes the lower bound inclusive",
     "        if (row_sym(ix, mid, d) < c) a = mid + 1; else b = mid;",
     "        if (row_sym(ix, mid, d) <= c) a = mid + 1; else b = mid;"),
    ("end restriction: insertion bound shifted",
     "    return i >= X->end_skip && X->m - 1 - i >= X->end_skip;",
     "    return i > X->end_skip && X->m - 1 - i >= X->end_skip;"),
    ("end restriction: deletion treated like an insertion",
     "    return i + 1 >= X->end_skip && X->m - 1 - i >= X->end_skip;",
     "    return i >= X->end_skip && X->m - 1 - i >= X->end_skip;"),
    ("end restriction: deletion counted from the wrong side",
     "    return i + 1 >= X->end_skip && X->m - 1 - i >= X->end_skip;",
     "    return i + 1 >= X->end_skip && X->m - i >= X->end_skip;"),
]


PINS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "test_oracle_pins.py")


@pytest.mark.parametrize("label,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_planted_mistake(tmp_path, label, orig, mut):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation anchor not unique: {label}"
    mutsrc = tmp_path / "oracle.c"
    mutsrc.write_text(src.replace(orig, mut))
    hdr = os.path.join(os.path.dirname(SRC), "oracle.h")
    (tmp_path / "oracle.h").write_text(open(hdr).read())
    so = str(tmp_path / "libmut.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", so,
                    str(mutsrc)], check=True)
    # the pin suite runs in its own process against the mutant: a failing pin (or a crash of
    # the mutant) ends it with a non-zero status
    env = dict(os.environ, ORACLE_LIB=so)
    proc = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"],
                          env=env, capture_output=True, text=True, timeout=600,
                          cwd=os.path.dirname(os.path.dirname(PINS)))
    assert proc.returncode != 0, f"no pin rejects the planted mistake: {label}"
