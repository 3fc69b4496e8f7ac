"""tc_sort_keys_static: the sort for callers that cannot allocate.

Some callers cannot allocate device memory where they call the library:
their device memory belongs to another allocator (a framework's caching
pool holding the free memory), or they run under a fixed, pre-planned
memory budget or a real-time deadline.  tc_sort_keys_static sorts their
keys using one fixed static device array as scratch instead of allocating.

Checked here through the C ABI, twice in a row (the array keeps the previous
call's contents), against the library's allocating path: tc_build_csr sorts
the same pairs with allocated scratch, and its canonical edge list, packed
the same way, must equal the statically sorted keys exactly.  Independently
of the library's own sort, the result is compared with numpy's stable sort
on the low key_bits bits (widths 1, 13, 48 and 64, junk above key_bits,
repeated keys, the maximum size), and the call is checked to allocate
nothing and to report an expired device wait as TC_ETIMEDOUT.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1708_06866_gb300 as tc  # noqa: E402

BITS = 16  # vertex ids below 2^16: the library packs (lo << 16) | hi


def _entry():
    f = tc.load_library().tc_sort_keys_static
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _distinct_pairs(rng, count):
    lo = rng.integers(0, (1 << BITS) - 1, count * 2)
    hi = rng.integers(0, 1 << BITS, count * 2)
    keep = lo < hi
    packed = np.unique((lo[keep].astype(np.int64) << BITS) | hi[keep])[:count]
    rng.shuffle(packed)
    return packed


def test_static_sort_equals_allocating_path_on_two_calls_in_a_row():
    sort_static = _entry()
    stream = torch.cuda.current_stream()
    for call, count in enumerate((300_007, 1_000_003)):   # ragged, many radix tiles
        rng = np.random.default_rng(40 + call)
        packed = _distinct_pairs(rng, count)
        n = len(packed)
        keys = torch.from_numpy(packed.copy()).cuda()
        rc = sort_static(keys.data_ptr(), n, 2 * BITS, stream.cuda_stream)
        assert rc == 0, tc.tc_last_error()
        got = keys.cpu().numpy()
        # the allocating path: clean and sort the same pairs
        src = (packed >> BITS).astype(np.int32)
        dst = (packed & ((1 << BITS) - 1)).astype(np.int32)
        g = tc.tc_build_csr(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), 1 << BITS)
        lo, hi = tc.tc_edges(g)
        want = (lo.cpu().numpy().astype(np.int64) << BITS) | hi.cpu().numpy().astype(np.int64)
        g.free()
        assert n == len(want)
        assert np.array_equal(got, want), f"call {call}"


def test_static_sort_rejects_sizes_beyond_its_scratch():
    sort_static = _entry()
    too_many = (1 << 20) + 1
    keys = torch.zeros(too_many, dtype=torch.int64, device="cuda")
    rc = sort_static(keys.data_ptr(), too_many, 64, torch.cuda.current_stream().cuda_stream)
    assert rc == tc.TC_EOVERFLOW
    assert "2^20" in tc.tc_last_error()
    assert int(keys.abs().sum()) == 0     # untouched


def _stable_by_low_bits(keys_u64, key_bits):
    mask = np.uint64((1 << key_bits) - 1) if key_bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    order = np.argsort(keys_u64 & mask, kind="stable")
    return keys_u64[order]


@pytest.mark.parametrize("key_bits", [1, 13, 48, 64])
def test_static_sort_equals_numpy_stable_sort(key_bits):
    """Ascending by the low key_bits bits, equal keys in input order (an LSD
    radix sort is stable), bits above key_bits ignored; two calls in a row."""
    sort_static = _entry()
    stream = torch.cuda.current_stream()
    for call, count in enumerate((1 << 20, 777_777)):    # the maximum, then a ragged size
        rng = np.random.default_rng(100 * key_bits + call)
        if key_bits == 64:
            raw = rng.integers(0, 1 << 63, count, dtype=np.uint64) * np.uint64(2)
            raw += rng.integers(0, 2, count, dtype=np.uint64)
        else:
            # few distinct low parts (many repeats), random junk above key_bits
            low = rng.integers(0, min(1 << key_bits, 5000), count, dtype=np.uint64)
            junk = rng.integers(0, 1 << (64 - key_bits - 1), count, dtype=np.uint64)
            raw = (junk << np.uint64(key_bits)) | low
        raw[: count // 50] = raw[count // 2: count // 2 + count // 50]   # exact repeats too
        keys = torch.from_numpy(raw.view(np.int64).copy()).cuda()
        rc = sort_static(keys.data_ptr(), count, key_bits, stream.cuda_stream)
        assert rc == 0, tc.tc_last_error()
        got = keys.cpu().numpy().view(np.uint64)
        want = _stable_by_low_bits(raw, key_bits)
        assert np.array_equal(got, want), f"key_bits {key_bits}, call {call}"


def test_static_sort_allocates_nothing():
    """With the next device allocation set to fail, the call still succeeds
    and leaves the injected failure unused; free device memory is unchanged."""
    sort_static = _entry()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(7)
    raw = rng.integers(0, 1 << 40, 500_000, dtype=np.int64)
    keys = torch.from_numpy(raw.copy()).cuda()
    assert sort_static(keys.data_ptr(), len(raw), 40, stream.cuda_stream) == 0  # warm
    keys.copy_(torch.from_numpy(raw))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    prev = tc.tc_debug_fail_alloc(1)
    try:
        rc = sort_static(keys.data_ptr(), len(raw), 40, stream.cuda_stream)
    finally:
        left = tc.tc_debug_fail_alloc(prev)
    assert rc == 0, tc.tc_last_error()
    assert left == 1, "the call made a device allocation"
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.array_equal(keys.cpu().numpy(), np.sort(raw))


def test_static_sort_reports_an_expired_wait_and_stays_usable():
    """A 1 ns limit on the radix look-back wait: the call returns TC_ETIMEDOUT
    (or succeeds if no wait was needed); with the limit restored the next call
    sorts correctly."""
    sort_static = _entry()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(8)
    raw = rng.integers(0, 1 << 62, 1 << 20, dtype=np.int64)
    keys = torch.from_numpy(raw.copy()).cuda()
    prev = tc.tc_debug_spin_limit_ns(1)
    try:
        rc = sort_static(keys.data_ptr(), len(raw), 64, stream.cuda_stream)
    finally:
        tc.tc_debug_spin_limit_ns(prev)
    assert rc in (0, tc.TC_ETIMEDOUT), rc
    keys.copy_(torch.from_numpy(raw))
    assert sort_static(keys.data_ptr(), len(raw), 64, stream.cuda_stream) == 0
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), np.sort(raw.view(np.uint64)))
