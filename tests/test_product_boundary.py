"""The product path and the oracle stay apart (no GPU needed).

The package must refuse to run without its compiled library (there is no CPU
fallback), and nothing in the package may import the oracle, which is test
infrastructure only.
"""

import os
import re
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1104_4208_gb300")


def test_binding_fails_loudly_without_library(tmp_path):
    dst = tmp_path / "paper_1104_4208_gb300"
    dst.mkdir()
    for name in os.listdir(PKG):
        if name.endswith(".py"):
            shutil.copy(os.path.join(PKG, name), dst / name)
    code = ("import sys; sys.path.insert(0, sys.argv[1])\n"
            "try:\n"
            "    from paper_1104_4208_gb300.solver import Solver\n"
            "except ImportError as e:\n"
            "    print('IMPORT-ERROR', e)\n"
            "else:\n"
            "    print('IMPORTED')\n")
    out = subprocess.run([sys.executable, "-c", code, str(tmp_path)], capture_output=True, text=True,
                         timeout=120)
    assert "IMPORT-ERROR" in out.stdout, out.stdout + out.stderr
    assert "libdgm.so is not built" in out.stdout


def test_package_never_imports_the_oracle():
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|oracle/", re.M)
    for dirpath, _, files in os.walk(PKG):
        for name in files:
            if name.endswith((".py", ".cu", ".cpp", ".h")):
                src = open(os.path.join(dirpath, name)).read()
                assert not pat.search(src), os.path.join(dirpath, name)
