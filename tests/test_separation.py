"""The oracle and the CUDA path share no code: the package never imports,
loads or includes anything under oracle/, and the oracle includes only system
headers and imports nothing from the package (the seeded inputs reach both
sides through the tests, the smoke check and the benchmark)."""

from __future__ import annotations

import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1006_3865_gb300")
ORC = os.path.join(ROOT, "oracle")


def _sources(top, exts):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("_build", "__pycache__")]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_never_reaches_the_oracle():
    bad = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b)|liboracle|spn_oracle|[\"']oracle[/\"']", re.M)
    for p in _sources(PKG, (".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
        text = open(p, encoding="utf-8").read()
        assert not bad.search(text), p
        for inc in re.findall(r'^\s*#\s*include\s*"([^"]+)"', text, re.M):
            assert os.path.exists(os.path.join(os.path.dirname(p), inc)) or \
                os.path.exists(os.path.join(ROOT, "include", inc)), (p, inc)
            assert "oracle" not in inc, (p, inc)


def test_oracle_uses_nothing_of_the_package():
    for p in _sources(ORC, (".c", ".h")):
        text = open(p, encoding="utf-8").read()
        assert not re.search(r'^\s*#\s*include\s*"', text, re.M), p  # system headers only
        assert "spn_internal" not in text and "philox.cuh" not in text, p
    for p in _sources(ORC, (".py",)):
        text = open(p, encoding="utf-8").read()
        assert not re.search(r"^\s*(import|from)\s+paper_1006_3865_gb300\b|libspn|csrc[/\"']", text, re.M), p
