"""The generated CUDA headers are committed; their generators must still reproduce them byte for byte.

csrc/m2l_gen.cuh (straight-line M2L contractions, orders 1-6, full and harmonic sets) and
csrc/tg_tables.cuh (multi-index tables) are written by csrc/gen_m2l.py and csrc/gen_tables.py.  A change
to one side without the other would build kernels that no longer match their documented derivation.
"""
import os
import subprocess
import sys

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1712_10116_gb300", "csrc")


@pytest.mark.parametrize("script,header", [("gen_m2l.py", "m2l_gen.cuh"), ("gen_tables.py", "tg_tables.cuh")])
def test_generator_reproduces_committed_header(script, header):
    out = subprocess.run([sys.executable, os.path.join(CSRC, script)], capture_output=True, check=True).stdout
    with open(os.path.join(CSRC, header), "rb") as f:
        committed = f.read()
    assert out == committed, f"{header} differs from the output of {script}; regenerate it"
