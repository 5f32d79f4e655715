"""The debug build (DSPG_DEBUG=1: every kernel that reads a column of A as a
row of B, writes a row of C, a bin slot, or a committed row checks the index
and room first, and a failed check fails the batch with its code): the
parity sequences below run in a child process on that library, and every
result matches the oracle with no check failing."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

CHILD = r'''
import numpy as np
import paper_2202_08808_gb300 as pkg
from paper_2202_08808_gb300 import dspg as D
from oracle import OMat
from parity import assert_matches, oracle_product
from workloads import MIN_PLUS_I32, PLUS_TIMES_F64, random_batch, random_csr, rmat_edge_batch, rmat_symmetric
assert D.library_path().endswith("libdspg_debug.so")
assert D.load().dspg_debug_build() == 1
import time
print("loaded debug build", flush=True)
for sr in (PLUS_TIMES_F64, MIN_PLUS_I32):
    A, held = rmat_symmetric(10, 8, (0.57, 0.19, 0.19, 0.05), seed=3, kind=sr, holdout=600)
    for bloom in (False, True):
        g = pkg.DynamicSpGEMM(A, bloom=bloom, arena_headroom=1.0, slack_min=0)
        Ao = OMat.from_csr(A)
        for k in range(3):
            b = rmat_edge_batch(Ao.to_csr(), held, 80, seed=40 + k)
            g.apply_batch(b)
            Ao.apply(b)
            C_o, S_o = oracle_product(Ao, Ao)
            assert_matches(g.read_C(), C_o, S_o, what=f"sr {sr} bloom {bloom} batch {k}")
        g.close()
    # separate B, the delta path and the row path's growth
    A2 = random_csr(300, 200, 12, 5, sr)
    B2 = random_csr(200, 400, 10, 6, sr)
    g = pkg.DynamicSpGEMM(A2, B2, arena_headroom=1.0, slack_min=0)
    Ao, Bo = OMat.from_csr(A2), OMat.from_csr(B2)
    for k in range(3):
        ba = random_batch(300, 200, 200, 60 + k, sr, A=Ao.to_csr())
        bb = random_batch(200, 400, 150, 70 + k, sr, A=Bo.to_csr())
        g.apply_batch(ba, bb)
        Ao.apply(ba)
        Bo.apply(bb)
        C_o, S_o = oracle_product(Ao, Bo)
        assert_matches(g.read_C(), C_o, S_o, what=f"sr {sr} separate B batch {k}")
    g.close()
print("DEBUG BUILD OK")
'''


def test_parity_on_the_debug_build():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, DSPG_DEBUG="1",
               PYTHONPATH=os.pathsep.join([root, os.path.join(root, "tests"), os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=root, env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0 and "DEBUG BUILD OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
    # and the release library is not the debug one
    from paper_2202_08808_gb300 import dspg as D
    if os.environ.get("DSPG_DEBUG", "") != "1":
        assert D.load().dspg_debug_build() == 0
