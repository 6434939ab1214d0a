"""The outer-loop pins have teeth: plausible mistakes planted in a copy of the
oracle's outer-loop functions (oracle/__init__.py, on the CPU, in a temporary
directory) must each make tests/test_oracle_loop_pins.py fail."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, original text, mutated text)
MUTANTS = [
    ("ties-to-higher-position", "order = np.lexsort((np.arange(len(v)), -v if largest else v))",
     "order = np.lexsort((-np.arange(len(v)), -v if largest else v))"),
    ("cold-start-keeps-highest", "sel = select_top(cs, k, largest=False)",
     "sel = select_top(cs, k, largest=True)"),
    ("no-eviction", "if b_max > 0 and len(ps) > b_max:", "if b_max < 0 and len(ps) > b_max:"),
    ("rescore-ignores-basis", "sel = select_top(ps, k)\n        return pa[sel], pb[sel], ps[sel]",
     "sel = select_top(ps[len(ba):], k) + len(ba)\n        return pa[sel], pb[sel], ps[sel]"),
    ("basis-not-excluded", "elif (a, b) not in ex:", "elif (a, b) not in ex or True:"),
    ("filter-off", "if popcount(a) != n_alpha or popcount(b) != n_beta:",
     "if popcount(a) != n_alpha and popcount(b) != n_beta:"),
    ("advantage-sign", "A = hxx - E0", "A = E0 - hxx"),
    ("teacher-normalised-on-minibatch", "w = pa[batch // Nb] * pb[batch % Nb] / Z",
     "w = pa[batch // Nb] * pb[batch % Nb] / np.sum(pa[batch // Nb] * pb[batch % Nb])"),
    ("entropy-sum-not-mean", "ls = float(np.sum(log_pi)) / M if M else 0.0",
     "ls = float(np.sum(log_pi)) if M else 0.0"),
    ("remap-wrong-entries", "return np.where(old >= 0, c_old[np.maximum(old, 0)], 0.0)",
     "return np.where(old >= 0, c_old[::-1][np.maximum(old, 0)], 0.0)"),
    ("stop-one-early", "return bool(np.all(d[-patience:] < delta))",
     "return bool(np.all(d[-patience + 1:] < delta))"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_loop_pins_catch_planted_mistake(tmp_path, name, old, new):
    dst = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), dst, ignore=shutil.ignore_patterns("__pycache__"))
    src = (dst / "__init__.py").read_text()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    (dst / "__init__.py").write_text(src.replace(old, new))
    env = dict(os.environ, PYTHONPATH=f"{tmp_path}{os.pathsep}{ROOT}{os.pathsep}{os.path.join(ROOT, 'tests')}")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
           os.path.join(ROOT, "tests", "test_oracle_loop_pins.py")]
    res = subprocess.run(cmd, env=env, cwd=str(tmp_path), capture_output=True, text=True, timeout=600)
    assert res.returncode == 1, f"mutant {name} survived the pins:\n{res.stdout[-2000:]}"
