"""The exclusive scan that allocates nothing (cusci_exclusive_scan_static).

It is meant for callers that cannot allocate device memory or hand over a
workspace (a framework that has reserved the device's memory, a loop that must
not pay cudaMalloc's device-wide synchronisation, a binding that only passes
pointers).  Its output must equal that of the workspace-based scan, call after
call, although every call reuses the same static scratch array.  Collected last
so that a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2604_15768_gb300 import cusci

pytestmark = pytest.mark.gpu


def _scan_with_workspace(counts):
    return cusci.exclusive_scan(counts)


def _scan_static(counts):
    lib = cusci.load()
    out = torch.empty(counts.shape[0] + 1, dtype=torch.int64, device=counts.device)
    rc = lib.cusci_exclusive_scan_static(ctypes.c_void_p(counts.data_ptr()), counts.shape[0],
                                         ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    cusci._check(rc, "cusci_exclusive_scan_static")
    return out


def test_static_scan_matches_workspace_scan_twice():
    rng = np.random.default_rng(42)
    # two calls in a row: a large ragged size first, then a smaller one, so the
    # second call runs on scratch left over from the first
    for n in (3_000_017, 4_099):
        counts = torch.from_numpy(rng.integers(0, 40_000, size=n).astype(np.int64)).cuda()
        got = _scan_static(counts)
        ref = _scan_with_workspace(counts)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        assert int(got[0].item()) == 0 and int(got[-1].item()) == int(counts.sum().item())


def test_static_scan_rejects_sizes_beyond_its_limit():
    lib = cusci.load()
    limit = int(lib.cusci_scan_static_max())
    assert limit == 65536 * 2048
    dummy = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = lib.cusci_exclusive_scan_static(ctypes.c_void_p(dummy.data_ptr()), limit + 1,
                                         ctypes.c_void_p(dummy.data_ptr()), None)
    assert rc == 6
    assert b"static scratch limit" in lib.cusci_last_error()
