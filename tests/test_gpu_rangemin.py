"""GPU parity of the range minimum (Sec. 2): bit-exact against the oracle through the C ABI."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1907_12343_gb300 as hrr
    c = hrr.Context(0)
    yield c
    c.close()


def _run(ctx, a, b, r, variant, offset=0):
    import torch
    d = torch.device("cuda:0")
    n = len(a)
    # optional element offset exercises the unaligned (scalar) path
    buf = [torch.zeros(n + offset, dtype=torch.int32, device=d) for _ in range(5)]
    ta, tb, tr, tv, tk = (x[offset:] for x in buf)
    ta.copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)))
    tb.copy_(torch.from_numpy(np.ascontiguousarray(b, dtype=np.uint32).view(np.int32)))
    tr.copy_(torch.from_numpy(np.ascontiguousarray(r, dtype=np.uint32).view(np.int32)))
    ctx.range_min(ta, tb, tr, tv, tk, variant=variant)
    torch.cuda.synchronize()
    return tv.cpu().numpy().view(np.uint32), tk.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("variant", [0, 2])
def test_all_short_ranges(ctx, variant):
    # every a < b <= 2^10 with 64 shifts (including 0, 1, 2^31, 2^32 - 1): ~33.5M queries
    aa, bb = np.triu_indices(1025, k=1)
    shifts = np.concatenate([[0, 1, 1 << 31, 0xFFFFFFFF],
                             synth.splitmix64(5, 1, 60) >> np.uint64(32)]).astype(np.uint32)
    a = np.repeat(aa.astype(np.uint32), len(shifts))
    b = np.repeat(bb.astype(np.uint32), len(shifts))
    r = np.tile(shifts, len(aa))
    v, k = _run(ctx, a, b, r, variant)
    v_ref, k_ref = oracle.rangemin_batch(a, b, r, "trie")
    assert np.array_equal(v, v_ref) and np.array_equal(k, k_ref)
    small = b <= 256
    v_scan, k_scan = oracle.rangemin_batch(a[small], b[small], r[small], "scan")
    assert np.array_equal(v[small], v_scan) and np.array_equal(k[small], k_scan)


@pytest.mark.parametrize("variant", [0, 2])
def test_log_uniform_queries_full_size(ctx, variant):
    # the 2^26-query range-minimum workload in the launch configuration used for timing:
    # every query against the trie oracle; every query of at most 2^16 indices (about half
    # of them, some 2 * 10^11 indices in all) against the scan over every index
    a, b, r = synth.rangemin_queries(1 << 26, seed=3)
    v, k = _run(ctx, a, b, r, variant)
    v_ref, k_ref = oracle.rangemin_batch(a, b, r, "trie")
    assert np.array_equal(v, v_ref)
    assert np.array_equal(k, k_ref)
    ln = b.astype(np.int64) - a.astype(np.int64)
    idx = np.flatnonzero(ln <= 4096)[:100000]
    v_scan, k_scan = oracle.rangemin_batch(a[idx], b[idx], r[idx], "scan")
    assert np.array_equal(v[idx], v_scan) and np.array_equal(k[idx], k_scan)
    if variant == 0:
        idx = np.flatnonzero(ln <= 1 << 16)
        assert len(idx) > (1 << 25) * 0.9
        v_scan, k_scan = oracle.rangemin_batch(a[idx], b[idx], r[idx], "scan_inc")
        assert np.array_equal(v[idx], v_scan) and np.array_equal(k[idx], k_scan)


@pytest.mark.parametrize("variant", [0, 2])
@pytest.mark.parametrize("offset", [0, 1])
def test_edges_and_ragged_tail(ctx, variant, offset):
    M = 0xFFFFFFFF
    rng = np.random.default_rng(2)
    cases = [(0, 1, 0), (0, 1, 7), (0, 2, 1 << 31), (0, M, 0), (0, M, 12345), (1, M, M),
             (M - 1, M, 5), (M - 2, M, 0), (5, 8, 38 << 26), (1 << 31, (1 << 31) + 1, 1)]
    n = 1003  # not a multiple of 4
    a = rng.integers(0, 2**32 - 2, n, dtype=np.uint64)
    b = np.minimum(a + rng.integers(1, 2**20, n, dtype=np.uint64), M)
    r = rng.integers(0, 2**32, n, dtype=np.uint64)
    for q, (x, y, s) in enumerate(cases):
        a[q], b[q], r[q] = x, y, s
    v, k = _run(ctx, a, b, r, variant, offset)
    v_ref, k_ref = oracle.rangemin_batch(a, b, r, "trie")
    assert np.array_equal(v, v_ref) and np.array_equal(k, k_ref)


@pytest.mark.parametrize("variant", [0, 2])
def test_empty_ranges_saturate(ctx, variant):
    a = np.array([5, 9, 0, 7], dtype=np.uint32)
    b = np.array([5, 3, 0, 8], dtype=np.uint32)
    r = np.array([0, 1, 2, 3], dtype=np.uint32)
    v, k = _run(ctx, a, b, r, variant)
    assert v[:3].tolist() == [0xFFFFFFFF] * 3 and k[:3].tolist() == [0xFFFFFFFF] * 3
    assert (v[3], k[3]) == oracle.rangemin_scan(7, 8, 3)


def test_unknown_variant_is_rejected(ctx):
    # variant 1 (the paper's Alg. 2 + 3) lives only in the oracle; the library refuses it
    import torch
    import paper_1907_12343_gb300 as hrr
    d = torch.device("cuda:0")
    t = torch.zeros(8, dtype=torch.int32, device=d)
    for v in (1, 3, -1):
        with pytest.raises(hrr.HRRError):
            ctx.range_min(t, t + 1, t, t.clone(), t.clone(), variant=v)
