"""The bounds-checked debug build (compiled with -DHEOM_DEBUG, the stand-in for a memory checker):
every stage kernel checks each link record's neighbour index (0 <= v < n_ado), coupled state and
record range before use and sets an error bit that heom_observables reports as HEOM_E_BOUNDS.
The test builds that variant into its own directory and runs small parity cases of every kernel family
against it in a child process (tests/debug_cases.py): all match the oracle and no check fires."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_parity_cases_without_bounds_errors():
    from paper_1803_03498_gb300.build import build
    lib = build(debug=True)
    assert lib.endswith(os.path.join("_build_debug", "libheom.so"))
    env = dict(os.environ, HEOM_LIB=lib)
    p = subprocess.run([sys.executable, os.path.join(HERE, "debug_cases.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    out = p.stdout + p.stderr
    assert p.returncode == 0, out[-3000:]
    assert f"library {lib}" in out
    assert "ALL OK" in out
