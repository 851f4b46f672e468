"""The allocation-free residual entry point, checked against mg_residual.

mg_residual_norm_noalloc serves callers that must not allocate device memory (a
fixed budget handed out by a host framework, or latency-critical loops where an
allocation call could block on queued GPU work): its reduction scratch is a
fixed device array inside the library.  The test calls it twice in a row through
the C ABI, because every call reuses that array and keeps the previous call's
contents, and compares both results with the existing mg_residual.  This file is
collected last so that a failure here comes after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

from tests.gpu_common import Case

pytestmark = pytest.mark.gpu


def _call(c, level, u, b, r, n2, stream):
    lib = c.mg.load()
    return lib.mg_residual_norm_noalloc(c.H.handle, level, C.c_void_p(u.data_ptr()), C.c_void_p(b.data_ptr()),
                                        C.c_void_p(r.data_ptr()), C.c_void_p(n2.data_ptr()),
                                        C.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("dim,L,eps", [(2, 4, "checker"), (3, 3, "sphere")])
def test_noalloc_residual_matches_mg_residual_twice(dim, L, eps):
    c = Case(dim, L, eps, oracle=False)
    torch = c.torch
    stream = torch.cuda.current_stream()
    for lv in (L, L - 1):
        n = c.n(lv)
        for call in range(2):
            u = c.dev(c.random_vec(lv, 10 * call + lv))
            b = c.dev(c.random_vec(lv, 10 * call + lv + 5))
            r_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
            n2_ref = c.H.residual(lv, u, b, r_ref, want_norm=True)
            r = torch.zeros(n, dtype=torch.float64, device="cuda")
            n2 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            assert _call(c, lv, u, b, r, n2, stream) == 0, c.mg.load().mg_last_error()
            torch.cuda.synchronize()
            got = float(n2.item())
            assert np.abs(r.cpu().numpy() - r_ref.cpu().numpy()).max() <= 1e-12 * max(np.abs(r_ref.cpu().numpy()).max(), 1e-300)
            assert abs(got - n2_ref) <= 1e-12 * n2_ref


def test_noalloc_rejects_levels_beyond_its_scratch():
    c = Case(2, 7, "checker", oracle=False)  # level 7: 6561 bricks > 4096
    torch = c.torch
    stream = torch.cuda.current_stream()
    n = c.n(7)
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    r = torch.zeros_like(u)
    n2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _call(c, 7, u, c.b_dev, r, n2, stream) == 1
    assert b"4096" in c.mg.load().mg_last_error()
    # the next level down (729 bricks) is served
    m = c.n(6)
    u6 = torch.zeros(m, dtype=torch.float64, device="cuda")
    assert _call(c, 6, u6, u6, torch.zeros_like(u6), n2, stream) == 0
