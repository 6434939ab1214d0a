"""The oracle's pins have teeth: plausible mistakes planted in a copy of the oracle
(on the CPU, in a temporary directory) must each make the pin suite fail."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, original text, mutated text)
MUTANTS = [
    ("create-sign-counts-after", "return (k % 2) ? -1 : 1;\n}\n\nstatic int spin_of",
     "return (k % 2) ? 1 : -1;\n}\n\nstatic int spin_of"),
    ("eri-transposed-operand", "H->eri[((size_t)(p * n + r) * n + q) * n + s]",
     "H->eri[((size_t)(p * n + q) * n + r) * n + s]"),
    ("dropped-half", "double c = 0.5 * g2(H, P, Q, R, S);", "double c = 1.0 * g2(H, P, Q, R, S);"),
    ("wrong-operator-order", "int sg = ann(&d, R); /* a_R acts first */\n                    if (!sg) continue;\n                    int t = ann(&d, S);",
     "int sg = ann(&d, S); /* a_R acts first */\n                    if (!sg) continue;\n                    int t = ann(&d, R);"),
    ("rdm2-index-swap", "a2[((size_t)(p * n + q) * n + r) * n + s]", "a2[((size_t)(q * n + p) * n + r) * n + s]"),
    ("rdm1-index-swap", "a1[p * n + q] += sg * t * c[K] * cj;", "a1[q * n + p] += sg * t * c[K] * cj * (p == q ? 1.0 : 1.5);"),
    ("marginal-unnormalised", "double v = c[a * Nb + b] * c[a * Nb + b] / nrm;",
     "double v = c[a * Nb + b] * c[a * Nb + b];"),
    ("double-link-order", "sg *= cre(&d, parts[1]);\n                sg *= cre(&d, parts[0]);",
     "sg *= cre(&d, parts[0]);\n                sg *= cre(&d, parts[1]);"),
    ("nuclear-repulsion-dropped", "emit(D, H->enuc, user);", "emit(D, 0.0 * H->enuc, user);"),
    ("list-lookup-ignores-beta", "if (xa[mid] == a && xb[mid] == b) return mid;",
     "if (xa[mid] == a) return mid;"),
    ("list-matrix-transposed", "if (K >= 0) lu->Hcol[K * lu->M + lu->col] += coeff;",
     "if (K >= 0) lu->Hcol[K * lu->M + lu->col] += (K < lu->col ? 1.01 : 1.0) * coeff;"),
    ("connected-merges-beta", "return u->a == v->a && u->b == v->b;", "return u->a == v->a;"),
    ("connected-32-bit-strings", "cu->buf[cu->cnt].a = a;", "cu->buf[cu->cnt].a = a & 0xffffffffull;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    dst = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), dst,
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    src = (dst / "hinqs_oracle.c").read_text()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    (dst / "hinqs_oracle.c").write_text(src.replace(old, new))
    env = dict(os.environ, PYTHONPATH=f"{tmp_path}{os.pathsep}{ROOT}")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
           os.path.join(ROOT, "tests", "test_oracle_pins.py"),
           "-k", "not table1 and not interlacing and not rotation"]
    res = subprocess.run(cmd, env=env, cwd=str(tmp_path), capture_output=True, text=True, timeout=600)
    assert res.returncode == 1, f"mutant {name} survived the pins:\n{res.stdout[-2000:]}"
