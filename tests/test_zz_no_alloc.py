"""rc_sort_keys_static, the sort for callers that cannot allocate device memory
when they sort (their memory is reserved up front by another allocator, or
their hot path must not pay for cudaMalloc), must order keys exactly as a
stable sort on the chosen bits does, and exactly as rc_sort_keys does with a
caller-provided workspace, without allocating device memory.

Two calls in a row with different inputs check that the shared static scratch
is reset between calls.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2503_08946_gb300 import build as b
    b.build()
    import paper_2503_08946_gb300 as pkg
    pkg.load()
    return pkg


def _keys(n, seed):
    g = torch.Generator().manual_seed(seed)
    x = torch.randint(-(1 << 62), 1 << 62, (max(n, 1),), generator=g, dtype=torch.int64)[:n]
    if n > 8:
        x[: n // 4] &= 0xFFFFF      # many equal digits: exercises stability
    return x


def _stable(x, lo, hi):
    """numpy's stable sort of the keys on bits [lo, hi)."""
    keys = x.numpy().view(np.uint64)
    mask = np.uint64((1 << (hi - lo)) - 1) if hi - lo < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    return keys[np.argsort((keys >> np.uint64(lo)) & mask, kind="stable")]


def _workspace_sort(rc, x, lo, hi, db):
    n = x.numel()
    out = torch.empty_like(x)
    ws = rc.workspace(rc.rc_sort_workspace_size(n, db))
    rc.rc_sort_keys(x, out, n, lo, hi, db, ws)
    return out


@pytest.mark.parametrize("case", [
    [(1 << 20, 0, 64, 8, 1), (1000, 3, 41, 8, 2)],
    [(777_777, 20, 53, 8, 3), (1 << 20, 0, 33, 6, 4)],
    [(4097, 1, 9, 8, 5), (4096, 1, 9, 8, 6)],
])
def test_static_sort_matches_stable_sort_two_calls(rc, case):
    for n, lo, hi, db, seed in case:
        xh = _keys(n, seed)
        x = xh.cuda()
        out = torch.full_like(x, -1)
        rc.rc_sort_keys_static(x, out, n, lo, hi, db)
        assert rc.rc_sort_status(None) == rc.RC_OK
        got = out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, _stable(xh, lo, hi)), (n, lo, hi, db)
        ref = _workspace_sort(rc, x, lo, hi, db)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (n, lo, hi, db)
        assert torch.equal(x.cpu(), xh)   # the input is untouched


def test_static_sort_allocates_nothing(rc):
    """After a first call (which looks up the scratch array and loads the
    kernels), a second call leaves the device's free memory unchanged."""
    n, lo, hi, db = 500_000, 5, 45, 8
    x1, x2 = _keys(n, 11).cuda(), _keys(n, 12).cuda()
    out = torch.empty_like(x1)
    rc.rc_sort_keys_static(x1, out, n, lo, hi, db)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    rc.rc_sort_keys_static(x2, out, n, lo, hi, db)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.array_equal(out.cpu().numpy().view(np.uint64), _stable(x2.cpu(), lo, hi))


def test_static_sort_timeout_is_reported(rc, monkeypatch):
    """A look-back wait that runs out (the test hook: a status epoch nothing
    publishes) is reported by rc_sort_status(None); the next call is exact."""
    n = 200_000
    xh = _keys(n, 21)
    x = xh.cuda()
    out = torch.empty_like(x)
    monkeypatch.setenv("RC_TEST_SORT_STALL", "1")
    rc.rc_sort_keys_static(x, out, n, 0, 24, 8)
    assert rc.rc_sort_status(None) == rc.RC_E_TIMEOUT
    monkeypatch.delenv("RC_TEST_SORT_STALL")
    rc.rc_sort_keys_static(x, out, n, 0, 24, 8)
    assert rc.rc_sort_status(None) == rc.RC_OK
    assert np.array_equal(out.cpu().numpy().view(np.uint64), _stable(xh, 0, 24))


def test_static_sort_rejects_too_many_keys(rc):
    n = rc.binding.RC_SORT_STATIC_MAX_KEYS + 1
    x = torch.zeros(n, dtype=torch.int64, device="cuda")
    out = torch.empty_like(x)
    with pytest.raises(rc.RcError) as e:
        rc.rc_sort_keys_static(x, out, n, 0, 64, 8)
    assert e.value.status == rc.RC_E_UNSUPPORTED


def test_static_sort_empty(rc):
    x = torch.empty(0, dtype=torch.int64, device="cuda")
    rc.rc_sort_keys_static(x, torch.empty_like(x), 0, 0, 64, 8)
    assert rc.rc_sort_status(None) == rc.RC_OK
