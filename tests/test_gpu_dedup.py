"""GPU parity of the de-duplication (sorted distinct keys + inverse index) with
the CPU oracle, bit-exact."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2604_15768_gb300 import cusci, synth
from tests.gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


def gpu_dedup(keys, n_bits, n_ones, index_bytes=4):
    u, inv, nu = cusci.dedup(to_dev(keys), n_bits, n_ones, index_bytes=index_bytes)
    torch.cuda.synchronize()
    return to_np(u), inv.cpu().numpy().astype(np.int64), nu


def compare(keys, n_bits, n_ones, index_bytes=4):
    u, inv, nu = gpu_dedup(keys, n_bits, n_ones, index_bytes)
    ou, oinv = O.dedup(keys)
    assert nu == ou.shape[0]
    assert np.array_equal(u, ou)
    assert np.array_equal(inv, oinv)


def coupled_keys(name, n, eps=None):
    s = synth.config_system(name)
    off, td, hv = O.OracleSystem.of(s).gen(s.dets[:n], s.eps if eps is None else eps)
    return s, td


def test_tiny_coupled_set_rank_keys():
    s, td = coupled_keys("tiny", 4900)
    compare(td, 2 * s.norb, s.n_alpha + s.n_beta)


def test_mid_coupled_set_rank_and_raw_keys():
    s, td = coupled_keys("mid", 300)
    compare(td, 2 * s.norb, s.n_alpha + s.n_beta)       # combinatorial-rank path
    compare(td, 2 * s.norb, -1)                         # raw-bits path
    compare(td, 2 * s.norb, s.n_alpha + s.n_beta, index_bytes=8)


def test_two_word_keys():
    s, td = coupled_keys("large", 2)
    compare(td, 2 * s.norb, s.n_alpha + s.n_beta)       # C(120,20) > 2^64: raw 120-bit path
    # 100 spin orbitals, 16 electrons: rank fits 64 bits although keys use 2 words
    norb = 50
    h1, h2 = synth.integrals(norb, seed=1)
    dets = synth.sample_dets(norb, 8, 8, 300, seed=2)
    off, td2, hv = O.OracleSystem(norb, 8, 8, h1, h2).gen(dets, 1e-8)
    compare(td2, 2 * norb, 16)


def test_edge_cases():
    one = np.array([[5]], dtype=np.uint64)
    compare(one, 3, 2)
    same = np.full((10000, 1), 0b1011, dtype=np.uint64)
    compare(same, 4, 3)
    rng = np.random.default_rng(0)
    raw = rng.integers(0, 1 << 62, size=(12345, 1)).astype(np.uint64)
    raw[::3] = raw[1::3][: raw[::3].shape[0]]
    compare(raw, 64, -1)
    raw2 = rng.integers(0, 1 << 62, size=(5000, 2)).astype(np.uint64)
    raw2[::2, 1] = 7
    compare(raw2, 128, -1)
    # empty
    u, inv, nu = gpu_dedup(np.zeros((0, 1), dtype=np.uint64), 8, 2)
    assert nu == 0


def test_declared_popcount_violation_is_reported():
    keys = np.array([[0b0111], [0b0011]], dtype=np.uint64)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    cusci.dedup(to_dev(keys), 4, 3, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 1


def test_workspace_too_small_is_an_error():
    keys = to_dev(np.arange(1, 100, dtype=np.uint64).reshape(-1, 1))
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(cusci.CusciError):
        # pass an explicit undersized workspace through the raw call
        lib = cusci.load()
        import ctypes
        u = torch.empty_like(keys)
        inv = torch.empty(keys.shape[0], dtype=torch.int32, device="cuda")
        nu = torch.zeros(1, dtype=torch.int64, device="cuda")
        rc = lib.cusci_dedup(ctypes.c_void_p(keys.data_ptr()), keys.shape[0], 1, 8, -1,
                             ctypes.c_void_p(ws.data_ptr()), 16, ctypes.c_void_p(u.data_ptr()),
                             ctypes.c_void_p(inv.data_ptr()), 4, ctypes.c_void_p(nu.data_ptr()),
                             None, None, None)
        cusci._check(rc, "cusci_dedup")


# ---- sample-sort path (taken for >= 2^22 keys whose sort key fits one word or a 42-bit rank)

def test_sample_sort_rank_keys_vs_oracle():
    s, td = coupled_keys("mid", 400)          # ~6.7M entries, ranks of 41 bits
    assert td.shape[0] >= (1 << 22)
    compare(td, 2 * s.norb, s.n_alpha + s.n_beta)


def test_sample_sort_raw_keys_vs_oracle():
    rng = np.random.default_rng(7)
    base = rng.integers(0, 1 << 40, size=600_000).astype(np.uint64)
    keys = base[rng.integers(0, base.size, size=5_000_000)].reshape(-1, 1)
    compare(keys, 40, -1)


def test_sample_sort_two_word_keys_vs_oracle():
    norb = 33                                  # 66 spin orbitals -> two words
    h1, h2 = synth.integrals(norb, seed=4)
    dets = synth.sample_dets(norb, 3, 3, 420, seed=5)
    off, td, hv = O.OracleSystem(norb, 3, 3, h1, h2).gen(dets, -1.0)
    assert td.shape[0] >= (1 << 22) and td.shape[1] == 2
    compare(td, 2 * norb, 6)


def test_sample_sort_heavy_hitter_leaf():
    """One key repeated far beyond a shared-memory leaf (the global-memory leaf path)."""
    rng = np.random.default_rng(8)
    keys = rng.integers(0, 1 << 36, size=4_500_000).astype(np.uint64)
    keys[rng.choice(keys.size, 1_500_000, replace=False)] = 123456789
    compare(keys.reshape(-1, 1), 36, -1)


def test_full_size_dedup_properties():
    """The benchmark's input (100k sources, 1.675e9 entries): the distinct list is
    strictly ascending, gathers back to every key through the inverse, and every
    distinct key is used; together these fix the answer."""
    s = synth.config_system("mid")
    sysd = cusci.System.of(s)
    off, od, oh, st = cusci.coupled(sysd, to_dev(s.dets), s.eps)
    del oh
    u, inv, nu = cusci.dedup(od, 2 * s.norb, s.n_alpha + s.n_beta)
    assert nu > 0
    assert bool((u[1:, 0] > u[:-1, 0]).all())                 # 52-bit keys: int64 order is exact
    chunk = 1 << 28
    for a in range(0, od.shape[0], chunk):
        b = min(od.shape[0], a + chunk)
        assert bool((u[inv[a:b].long(), 0] == od[a:b, 0]).all())
    used = torch.zeros(nu, dtype=torch.bool, device="cuda")
    used[inv.long()] = True
    assert bool(used.all())


@pytest.mark.parametrize("n", [100_000, 5_000_000])
def test_two_word_keys_with_zero_high_word(n):
    """Keys stored as two words whose significant bits fit the low word are sorted
    as one-word keys (both the LSD and the sample-sort paths)."""
    rng = np.random.default_rng(n)
    base = rng.integers(0, 1 << 40, size=max(1, n // 5)).astype(np.uint64)
    keys = np.zeros((n, 2), dtype=np.uint64)
    keys[:, 0] = base[rng.integers(0, base.size, size=n)]
    compare(keys, 40, -1)


def test_bits_above_declared_width_are_reported():
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 1 << 40, size=(5_000_000, 1)).astype(np.uint64)
    keys[123, 0] |= np.uint64(1) << np.uint64(45)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    cusci.dedup(to_dev(keys), 40, -1, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 1


def test_sample_sort_wide_and_overflowing_leaves_vs_oracle():
    """Leaves that leave the shared-memory hash path: (1) full-range 64-bit keys,
    whose leaves are too wide to pack beside a slot id, and (2) an input whose
    regularly spaced sample positions all hold one of two heavy keys, so that
    the splitters equal those two keys and the one leaf between them receives
    several million distinct keys (far more than its table holds).  Both are
    sorted in global memory; results must not change."""
    rng = np.random.default_rng(12)
    n = 4_600_000
    wide = rng.integers(0, 2 ** 63, size=n, dtype=np.int64).astype(np.uint64) * np.uint64(2)
    wide |= rng.integers(0, 2, size=n).astype(np.uint64)
    wide[::4] = wide[1::4][: wide[::4].size]
    compare(wide.reshape(-1, 1), 64, -1)
    # sample positions floor(j * N / NS): NS = 8 samples per leaf, 256 leaves
    # per level-1 bucket, level-1 buckets = the power of two covering
    # ceil(N / 1600) / 256 (the plan of the sample-sort path).  Two heavy keys
    # take turns at those positions, so one leaf spans (2^39, 2^41) with every
    # distinct key inside: narrow enough for the hash path, too many keys.
    leaves_wanted = -(-n // 1600)
    b1 = 1
    while b1 < -(-leaves_wanted // 256):
        b1 *= 2
    ns = min(b1 * 256 * 8, n)
    keys = np.uint64(1 << 40) + rng.permutation(n).astype(np.uint64) * np.uint64(3)
    at = (np.arange(ns, dtype=np.int64) * n) // ns
    keys[at[0::2]] = np.uint64(1 << 39)
    keys[at[1::2]] = np.uint64(1 << 41)
    compare(keys.reshape(-1, 1), 42, -1)


def test_sample_sort_hash_path_limits_vs_oracle():
    """Leaves at the limits of the shared-memory hash path: (1) all-distinct
    keys, so that leaves hold 512..2048 distinct keys (radix-ordered) or more
    than 2048 (too many for the table: sorted in global memory); (2) keys in a
    narrow range at the top of the 64-bit space including the all-ones word,
    which is the table's empty marker and sends its leaf to global memory."""
    rng = np.random.default_rng(21)
    n = 4_600_000
    keys = rng.choice(1 << 40, size=n, replace=False).astype(np.uint64)
    compare(keys.reshape(-1, 1), 40, -1)
    top = np.uint64(0xFFFFFFFFFFFFFFFF) - rng.integers(0, 1 << 30, size=n).astype(np.uint64)
    top[rng.choice(n, 20_000, replace=False)] = np.uint64(0xFFFFFFFFFFFFFFFF)
    compare(top.reshape(-1, 1), 64, -1)


def test_kernel_timing_records_every_phase():
    """Per-phase event timing of the sample-sort path: one call while enabled
    gives one recorded call with a positive time for every phase, calls after
    it is disabled add nothing, and the results are unchanged."""
    rng = np.random.default_rng(30)
    keys = rng.integers(0, 1 << 36, size=4_400_000).astype(np.uint64).reshape(-1, 1)
    cusci.set_kernel_timing(True)
    compare(keys, 36, -1)
    ms, calls = cusci.dedup_phase_ms()
    cusci.set_kernel_timing(False)
    gpu_dedup(keys, 36, -1)
    ms2, calls2 = cusci.dedup_phase_ms()
    assert calls == 1 and calls2 == 1
    assert list(ms) == ["sample+splitters", "hist1", "scatter1", "level2", "leaf_dedup",
                        "compact_unique", "unscatter2", "unscatter1"]
    assert all(v > 0 for v in ms.values())


@pytest.mark.parametrize("n", [(1 << 22) - 1, 1 << 22])
def test_path_threshold_both_sides(n):
    """Just below and at the size where the sample-sort path takes over from
    the LSD path: identical results, equal to the oracle's."""
    rng = np.random.default_rng(40 + n % 7)
    base = rng.integers(0, 1 << 44, size=n // 3).astype(np.uint64)
    keys = base[rng.integers(0, base.size, size=n)].reshape(-1, 1)
    compare(keys, 44, -1)


def test_sample_sort_single_distinct_key():
    """Every key equal at sample-sort size: all splitters coincide, one leaf
    holds everything (global-memory path), one distinct key, inverse all zero."""
    keys = np.full((4_300_000, 1), 987654321, dtype=np.uint64)
    u, inv, nu = gpu_dedup(keys, 40, -1)
    assert nu == 1 and u.shape[0] >= 1 and int(u[0, 0]) == 987654321
    assert (inv == 0).all()
