"""rc_sort_keys_static, the sort for callers that cannot allocate device memory
when they sort (their memory is reserved up front by another allocator, or
their hot path must not pay for cudaMalloc), must give exactly what
rc_sort_keys gives with a caller-provided workspace.

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
    return x.cuda()


def _reference(rc, x, lo, hi, db):
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
def test_static_sort_matches_workspace_sort_two_calls(rc, case):
    for n, lo, hi, db, seed in case:
        x = _keys(n, seed)
        out = torch.full_like(x, -1)
        rc.rc_sort_keys_static(x, out, n, lo, hi, db)
        ref = _reference(rc, x, lo, hi, db)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (n, lo, hi, db)
        # the input is untouched and the output is a permutation of it
        assert torch.equal(torch.sort(out).values, torch.sort(x).values)


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
