"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of oracle/bs_oracle.c (a dropped
factor, a shifted index, a wrong operator, a looser clamp ...), compiles it
with the oracle's own flags, and runs tests/test_oracle_pins.py against that
library (BS_ORACLE_LIB): at least one pin must fail.  An unmodified copy built
the same way must pass, so a failure is the mistake's and not the harness's.
CPU only; nothing here touches the CUDA library.
"""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "bs_oracle.c")

# (what the mistake is, exact text in bs_oracle.c, its replacement)
MUTANTS = [
    ("Hamming with IP once instead of twice (the misprint of Alg. 2)",
     "ham = n_a + n_b - 2.0 * n_ab;", "ham = n_a + n_b - 1.0 * n_ab;"),
    ("Alg. 1 log argument off by one count",
     "arg = pow(n, n_a) + pow(n, n_b) + nasbs / N - 1.0;",
     "arg = pow(n, n_a) + pow(n, n_b) + (nasbs + 1.0) / N - 1.0;"),
    ("n = 1 - 1/(N+1) instead of 1 - 1/N",
     "const double n = 1.0 - 1.0 / N;", "const double n = 1.0 - 1.0 / (N + 1.0);"),
    ("JS as n_ab / (n_a + n_b)",
     "js = (n_ab + ham != 0.0) ? n_ab / (n_ab + ham) : 0.0;",
     "js = (n_a + n_b != 0.0) ? n_ab / (n_a + n_b) : 0.0;"),
    ("Cos with the arithmetic mean of the sizes",
     "cs = (n_a * n_b > 0.0) ? n_ab / sqrt(n_a * n_b) : 0.0;",
     "cs = (n_a * n_b > 0.0) ? 2.0 * n_ab / (n_a + n_b) : 0.0;"),
    ("union clamp at N instead of N - 1",
     "if (uni > N - 1) uni = N - 1;", "if (uni > N) uni = N;"),
    ("sketch bit packed one position off",
     "words[j >> 5] |= 1u << (j & 31);", "words[j >> 5] |= 1u << ((j + 1) & 31);"),
    ("hash keeps bits 31..62 instead of 32..63",
     "uint32_t h32 = (uint32_t)(h >> 32);", "uint32_t h32 = (uint32_t)(h >> 31);"),
    ("SplitMix64 increment wrong in the last bit",
     "*state = *state + 0x9E3779B97F4A7C15ULL;", "*state = *state + 0x9E3779B97F4A7C17ULL;"),
    ("common count with OR instead of AND",
     "for (k = 0; k < n_words; k++) s += popcount32(a[k] & b[k]);",
     "for (k = 0; k < n_words; k++) s += popcount32(a[k] | b[k]);"),
    ("BCS sets the bit instead of flipping it",
     "u_s[pi[col[k]]] = (unsigned char)((u_s[pi[col[k]]] + 1) % 2);", "u_s[pi[col[k]]] = 1;"),
    ("top-k ties broken by the larger index",
     "if (p->idx < q->idx) return -1;\n    if (p->idx > q->idx) return 1;",
     "if (p->idx > q->idx) return -1;\n    if (p->idx < q->idx) return 1;"),
    ("column d accepted by the OR sketch",
     "if (col[k] >= d) row_ok = 0;\n        if (!row_ok) { bad = 1; continue; }\n        sketch_row_bits",
     "if (col[k] > d) row_ok = 0;\n        if (!row_ok) { bad = 1; continue; }\n        sketch_row_bits"),
    ("column d accepted by the BCS sketch",
     "if (col[k] >= d) row_ok = 0;\n        if (!row_ok) { bad = 1; continue; }\n        memset(u_s",
     "if (col[k] > d) row_ok = 0;\n        if (!row_ok) { bad = 1; continue; }\n        memset(u_s"),
]


def _run_pins(lib_path):
    env = dict(os.environ, BS_ORACLE_LIB=lib_path)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def _build(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    return oracle.compile_library(str(src), str(tmp_path / f"lib{name}.so"))


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


def test_unmodified_copy_passes_the_pins(tmp_path, source):
    rc, out = _run_pins(_build(tmp_path, "control", source))
    assert rc == 0, out


@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, source, what, old, new):
    assert source.count(old) == 1, f"mutation point not unique: {old!r}"
    rc, out = _run_pins(_build(tmp_path, "mutant", source.replace(old, new)))
    assert rc == 1, f"{what}: the pins did not fail (pytest exit {rc})\n{out}"
