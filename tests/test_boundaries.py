"""The product path and the oracle stay apart: the package never imports,
includes or reads anything under oracle/ (the oracle is test
infrastructure), and loading the package brings no oracle module in."""

import os
import re
import subprocess
import sys

from conftest import ROOT

PKG = os.path.join(ROOT, "paper_1811_05571_gb300")


def _package_sources():
    for base, _, files in os.walk(PKG):
        if "_build" in base or "__pycache__" in base:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                yield os.path.join(base, f)


def test_package_sources_never_name_the_oracle():
    pat = re.compile(r"\boracle\b")
    offenders = [p for p in _package_sources() if pat.search(open(p, encoding="utf-8").read())]
    assert not offenders, offenders


def test_loading_the_package_imports_no_oracle_module():
    code = ("import sys; sys.path.insert(0, %r); import paper_1811_05571_gb300 as P; P.load(); "
            "print(sorted(m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')))" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().splitlines()[-1] == "[]"
