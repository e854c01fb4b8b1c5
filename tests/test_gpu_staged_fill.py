"""The fill with integral slabs staged in shared memory by bulk copies (selected
with CUSCI_FILL_STAGE=1, read once per process) writes the same coupled lists:
checked in a child process against the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
from oracle import oracle as O
from paper_2604_15768_gb300 import cusci, synth
s = synth.config_system("mid", n_dets=300)
sysd = cusci.System.of(s)
off, od, oh, st = cusci.coupled(sysd, cusci.dets_to_device(s.dets), s.eps)
torch.cuda.synchronize()
o_off, o_d, o_h = O.OracleSystem.of(s).gen(s.dets, s.eps)
assert int(st.item()) == 0
assert np.array_equal(off.cpu().numpy(), o_off)
assert np.array_equal(cusci.dets_to_numpy(od), o_d)
assert np.array_equal(oh.cpu().numpy().view(np.uint64), o_h.view(np.uint64))
print("staged ok")
"""


def test_staged_fill_matches_oracle():
    env = dict(os.environ, CUSCI_FILL_STAGE="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "staged ok" in r.stdout
