"""tc_sort_keys_static: the sort for callers that cannot allocate.

Some callers cannot allocate device memory where they call the library:
their device memory belongs to another allocator (a framework's caching
pool holding the free memory), or they run under a fixed, pre-planned
memory budget or a real-time deadline.  tc_sort_keys_static sorts their
keys using one fixed static device array as scratch instead of allocating.

Checked here through the C ABI, twice in a row (the array keeps the previous
call's contents), against the library's allocating path: tc_build_csr sorts
the same pairs with allocated scratch, and its canonical edge list, packed
the same way, must equal the statically sorted keys exactly.
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
