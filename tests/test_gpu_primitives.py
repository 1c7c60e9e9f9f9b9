"""The library's primitives alone, through its test hooks, against plain
CPU results: the stable radix sort that orders depth keys and tile ids
(Sec. 4.2's per-tile lists in depth order), the exclusive scan that places
list entries, and the tile ranges over a tile-sorted list.  Each must be
exact: integer work, compared bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08270_gb300 import build, flashsplat
    build.build()
    flashsplat.load()
    return flashsplat


def _dev(a):
    """A uint32 host array as an int32 device tensor holding the same bits."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


# sizes around the sort's 4096-element tiles and the scan's blocks, with
# ragged tails; key widths of one, two and three 8/9-bit digit passes
@pytest.mark.parametrize("n", [1, 5, 4095, 4096, 4097, 100003, (1 << 20) + 17])
@pytest.mark.parametrize("bits", [1, 8, 9, 17, 24, 32])
def test_radix_sort_is_a_stable_sort(fsb, n, bits):
    rng = np.random.default_rng(n * 131 + bits)
    keys = rng.integers(0, 1 << bits, n, dtype=np.uint64).astype(np.uint32)
    if n > 10:
        keys[: n // 2] &= np.uint32(7)  # many equal keys: ties keep their input order
    vals = np.arange(n, dtype=np.uint32)[::-1].copy()
    order = np.argsort(keys, kind="stable")
    k, v = _dev(keys), _dev(vals)
    fsb.fs_test_sort_pairs(0, k, v, bits)
    np.testing.assert_array_equal(_host(k), keys[order])
    np.testing.assert_array_equal(_host(v), vals[order])


def test_radix_sort_of_nothing_and_bad_arguments(fsb):
    import torch
    empty = torch.zeros(0, dtype=torch.int32, device="cuda")
    fsb.fs_test_sort_pairs(0, empty, empty, 8)
    one = _dev(np.array([3], np.uint32))
    with pytest.raises(fsb.FlashSplatError):
        fsb.fs_test_sort_pairs(0, one, one, 0)
    with pytest.raises(fsb.FlashSplatError):
        fsb.fs_test_sort_pairs(0, one, one, 33)


@pytest.mark.parametrize("n", [1, 255, 256, 257, 4096, 1000003])
def test_exclusive_scan_matches_cumsum_mod_2_32(fsb, n):
    import torch
    rng = np.random.default_rng(n)
    x = rng.integers(0, 1 << 12, n, dtype=np.uint64).astype(np.uint32)
    if n > 1000:
        x[::97] = np.uint32(0xFFFF0000)  # sums wrap around 2^32
    want = (np.cumsum(x.astype(np.uint64)) - x.astype(np.uint64)) & np.uint64(0xFFFFFFFF)
    total = int(x.astype(np.uint64).sum() & np.uint64(0xFFFFFFFF))
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    got_total = fsb.fs_test_exclusive_scan(0, _dev(x), out)
    np.testing.assert_array_equal(_host(out), want.astype(np.uint32))
    assert got_total == total


@pytest.mark.parametrize("n,n_tiles", [(1, 1), (7, 40), (4096, 300), (250001, 151200)])
def test_tile_ranges_of_a_sorted_list(fsb, n, n_tiles):
    import torch
    rng = np.random.default_rng(n + n_tiles)
    keys = np.sort(rng.integers(0, n_tiles, n)).astype(np.uint32)
    want = np.zeros((n_tiles, 2), np.uint32)
    present, first, count = np.unique(keys, return_index=True, return_counts=True)
    want[present, 0] = first
    want[present, 1] = first + count
    ranges = torch.full((n_tiles, 2), 7, dtype=torch.int32, device="cuda")
    fsb.fs_test_tile_ranges(0, _dev(keys), n_tiles, ranges)
    np.testing.assert_array_equal(_host(ranges), want)


def test_tile_ranges_refuse_keys_out_of_range_or_order(fsb):
    import torch
    ranges = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(fsb.FlashSplatError):
        fsb.fs_test_tile_ranges(0, _dev(np.array([0, 4], np.uint32)), 4, ranges)
    with pytest.raises(fsb.FlashSplatError):
        fsb.fs_test_tile_ranges(0, _dev(np.array([2, 1], np.uint32)), 4, ranges)
