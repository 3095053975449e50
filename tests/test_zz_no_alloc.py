"""The no-allocation sort entry point (splat2d_sort_pairs_noalloc).

Callers that cannot allocate device memory -- code running while a CUDA
graph is being captured, real-time loops that forbid allocation, plug-ins
whose host application owns all device memory -- use this variant of the
stable radix sort, whose scratch is a fixed array inside the library.  These
tests call it through the C ABI and check that two calls in a row give
exactly the output of the workspace-based splat2d_sort_pairs (integer data:
bit-exact), and that inputs above its fixed limit are refused.  The file is
named to run last, after every other test, and also passes on its own.
"""
import numpy as np
import pytest
import torch

from paper_2604_03092_gb300 import _abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _abi.load()


def _inputs(n, key_bits, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 1 << min(key_bits, 20), size=n, dtype=np.uint64)  # many ties
    keys = (keys << np.uint64(key_bits - min(key_bits, 20))) | rng.integers(0, 4, size=n, dtype=np.uint64)
    if key_bits < 64:
        keys &= np.uint64((1 << key_bits) - 1)
    vals = rng.permutation(n).astype(np.uint32)
    return keys, vals


def _sort_with_workspace(lib, keys, vals, key_bits):
    n = keys.size
    k = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    tmp = torch.empty(lib.splat2d_sort_tmp_size(n) + 256, dtype=torch.uint8, device="cuda")
    tp = (tmp.data_ptr() + 255) & ~255
    rc = lib.splat2d_sort_pairs(k.data_ptr(), v.data_ptr(), n, key_bits, tp, tmp.numel() - 256,
                                torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    return k.cpu().numpy().view(np.uint64), v.cpu().numpy().view(np.uint32)


def _sort_without_allocation(lib, keys, vals, key_bits):
    k = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    rc = lib.splat2d_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), keys.size, key_bits,
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == 0, _abi.strerror(rc)
    torch.cuda.synchronize()
    return k.cpu().numpy().view(np.uint64), v.cpu().numpy().view(np.uint32)


def test_noalloc_sort_matches_workspace_sort_twice(lib):
    # two calls in a row: the second must not see the first call's leftovers
    for n, key_bits, seed in ((300_001, 47, 1), (_abi.SORT_NOALLOC_MAX_PAIRS, 40, 2)):
        keys, vals = _inputs(n, key_bits, seed)
        ref_k, ref_v = _sort_with_workspace(lib, keys, vals, key_bits)
        got_k, got_v = _sort_without_allocation(lib, keys, vals, key_bits)
        assert np.array_equal(got_k, ref_k) and np.array_equal(got_v, ref_v)
        order = np.argsort(keys, kind="stable")
        assert np.array_equal(got_k, keys[order]) and np.array_equal(got_v, vals[order])


def test_noalloc_sort_rejects_inputs_above_its_limit(lib):
    n = _abi.SORT_NOALLOC_MAX_PAIRS + 1
    rc = lib.splat2d_sort_pairs_noalloc(None, None, n, 32, torch.cuda.current_stream().cuda_stream)
    assert rc == _abi.ERR_INVALID_ARG
