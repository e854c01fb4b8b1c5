"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

from paper_2604_15768_gb300 import cusci


def to_dev(dets):
    return cusci.dets_to_device(dets)


def to_np(t):
    return cusci.dets_to_numpy(t)


def assert_h_close(got, ref, rtol=1e-12):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape
    err = np.abs(got - ref)
    tol = rtol * np.maximum(np.abs(ref), 1e-300)
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, f"{bad.size} elements differ, first {bad[:5]}: {got[bad[:5]]} vs {ref[bad[:5]]}"


def sorted_rows(keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    order = np.lexsort([keys[:, w] for w in range(keys.shape[1])])
    return keys[order]
