"""Without its CUDA library the package refuses to import (there is no CPU fallback), for the normal and
the index-checking build alike."""
import os
import shutil
import subprocess
import sys

import pytest

PACKAGE = "paper_1910_13844_gb300"


@pytest.mark.parametrize("debug", ["0", "1"])
def test_import_fails_loudly_without_the_library(tmp_path, repo_root, debug):
    pkg = tmp_path / PACKAGE
    pkg.mkdir()
    for name in os.listdir(os.path.join(repo_root, PACKAGE)):
        if name.endswith(".py"):
            shutil.copy(os.path.join(repo_root, PACKAGE, name), pkg / name)
    env = dict(os.environ, LS_DEBUG_BOUNDS=debug, PYTHONPATH=str(tmp_path))
    r = subprocess.run([sys.executable, "-c", f"import {PACKAGE}"], capture_output=True, text=True, env=env,
                       cwd=str(tmp_path), timeout=300)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "no CPU fallback" in r.stderr, r.stderr
    assert ("libls_debug.so" if debug == "1" else "libls.so") in r.stderr
