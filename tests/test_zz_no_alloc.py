"""The allocation-free cell-range entry point against the library's own binning.

tfsph_cell_ranges_noalloc serves callers that cannot allocate device memory
(a fixed memory pool owned by the embedding application, or a loop that must
not allocate once running). Its counters live in a static device array, so
two calls in a row also check that each call starts from cleared counters.
The cell starts are integers: they must equal the library's bit for bit.
"""
import numpy as np
import pytest

import workloads
from conftest import gpu_context, gpu_lib

pytestmark = pytest.mark.gpu


def _ranges_noalloc(b, torch, keys, n_cells):
    # the uint32 key bits, carried by an int32 tensor
    d_keys = torch.from_numpy(np.ascontiguousarray(keys.astype(np.uint32).view(np.int32))).to("cuda")
    d_starts = torch.full((n_cells + 1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = b.tfsph_cell_ranges_noalloc(d_keys.data_ptr(), keys.size, n_cells, d_starts.data_ptr(),
                                     stream.cuda_stream)
    assert rc == b.TFSPH_OK, b.tfsph_last_error(None)
    torch.cuda.synchronize()
    return d_starts.cpu().numpy().astype(np.int64) & 0xFFFFFFFF


def test_cell_ranges_noalloc_match_library_binning():
    torch = pytest.importorskip("torch")
    b = gpu_lib()
    cases = []
    for w in (workloads.box3d(nside=24, precision=0), workloads.dustyshock(n_left=4000, n_right=500, precision=0)):
        with gpu_context(w) as c:
            n_cells = int(c.info().n_cells_total)
            for kk, ss in ((b.TFSPH_DEBUG_KEYS_G, b.TFSPH_DEBUG_CSTART_G), (b.TFSPH_DEBUG_KEYS_D, b.TFSPH_DEBUG_CSTART_D)):
                cases.append((c.debug(kk).astype(np.int64), c.debug(ss).astype(np.int64), n_cells))
    # two calls in a row on the same static scratch, in sorted and in shuffled key order
    rng = np.random.default_rng(0)
    for keys, ref, n_cells in cases:
        first = _ranges_noalloc(b, torch, keys, n_cells)
        second = _ranges_noalloc(b, torch, rng.permutation(keys), n_cells)
        assert np.array_equal(first, ref)
        assert np.array_equal(second, ref)


def test_cell_ranges_noalloc_rejects_too_many_cells():
    torch = pytest.importorskip("torch")
    b = gpu_lib()
    keys = torch.zeros(4, dtype=torch.int32, device="cuda")
    starts = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = b.tfsph_cell_ranges_noalloc(keys.data_ptr(), 4, (1 << 21) + 1, starts.data_ptr(), None)
    assert rc == b.TFSPH_E_INVALID_ARG
    assert "2097152" in b.tfsph_last_error(None)


def test_cell_ranges_noalloc_large_grids_and_keys_out_of_range():
    """Grids of 2^21 cells (the largest accepted: 1024 scan blocks, so the
    carry loop of the block-total scan runs several passes) and of 2^19 + 3
    cells (a partial last scan block), with seeded random keys of which some
    lie beyond the grid (up to 0xFFFFFFFF): the starts equal the prefix sums
    of the in-range key counts, bit for bit, on two calls in a row."""
    torch = pytest.importorskip("torch")
    b = gpu_lib()
    rng = np.random.default_rng(41)
    for n_cells in ((1 << 21), (1 << 19) + 3):
        keys = rng.integers(0, n_cells, size=300_000, dtype=np.int64)
        out = rng.choice(keys.size, size=1000, replace=False)
        keys[out] = rng.integers(n_cells, 1 << 32, size=out.size, dtype=np.int64)
        keys[out[:10]] = 0xFFFFFFFF
        keys[out[10:20]] = n_cells
        inside = keys[keys < n_cells]
        ref = np.concatenate([[0], np.cumsum(np.bincount(inside, minlength=n_cells))])
        for _ in range(2):
            got = _ranges_noalloc(b, torch, keys, n_cells)
            assert np.array_equal(got, ref)
