"""fg_poly_mul_noalloc, the product for callers that cannot allocate device
memory during a call (it takes its scratch from an array compiled into the
library), against fg_poly_mul, through the C ABI, twice in a row.  This file
is collected last so that a stop at the first failure has already run every
other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

PARAMS = dict(log_n=13, q_bits=[60] + [45] * 7, p_bits=[60] * 2, alpha=4, log_scale=45)


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    fg = __graft_entry__.build()
    from paper_2506_10399_gb300 import _native
    return fg, _native, torch


def rand_poly(torch, primes, n, seed):
    g = torch.Generator().manual_seed(seed)
    rows = [torch.randint(0, int(q), (n,), dtype=torch.int64, generator=g) for q in primes]
    return torch.stack(rows).cuda()


def test_noalloc_product_matches_the_allocating_one_twice(env):
    fg, nat, torch = env
    ctx = fg.Context(**PARAMS)
    for call, level in enumerate((7, 3)):
        a = rand_poly(torch, ctx.q[:level + 1], ctx.n, 10 + call)
        b = rand_poly(torch, ctx.q[:level + 1], ctx.n, 20 + call)
        want = fg.poly_mul(ctx, a, b, level)
        got = torch.empty_like(a)
        rc = nat.lib.fg_poly_mul_noalloc(ctx._h, ctypes.c_void_p(a.data_ptr()),
                                         ctypes.c_void_p(b.data_ptr()), level,
                                         ctypes.c_void_p(got.data_ptr()))
        assert rc == 0, nat.lib.fg_last_error(ctx._h)
        assert torch.equal(got, want)
    ctx.close()


def test_noalloc_rejects_oversize_and_host_buffers(env):
    fg, nat, torch = env
    big = dict(log_n=16, q_bits=[60] + [45] * 4, p_bits=[60], alpha=5, log_scale=45)
    ctx = fg.Context(**big)
    a = torch.zeros((5, ctx.n), dtype=torch.int64, device="cuda")
    rc = nat.lib.fg_poly_mul_noalloc(ctx._h, ctypes.c_void_p(a.data_ptr()),
                                     ctypes.c_void_p(a.data_ptr()), 4, ctypes.c_void_p(a.data_ptr()))
    assert rc == -1 and b"2^18" in nat.lib.fg_last_error(ctx._h)
    h = np.zeros((2, ctx.n), np.uint64)
    rc = nat.lib.fg_poly_mul_noalloc(ctx._h, ctypes.c_void_p(h.ctypes.data),
                                     ctypes.c_void_p(h.ctypes.data), 1, ctypes.c_void_p(h.ctypes.data))
    assert rc == -1
    ctx.close()
