"""GPU parity of the bpa delta codec (Sect. 5) and of the hierarchies that store their
deltas in it, against the CPU oracle.

Codes are integer work: records and byte streams must equal the oracle's bit for bit
on the same FP64 input (both sides take every decision with the same IEEE FP64
operations: frexp, exact ldexp scaling, round-half-even, one subtraction).  Decoding
is exact in FP64 and the FP32 decode is the FP32 rounding of the stored value.  The
coded hierarchy's deltas come from its own FP64 setup, so they are compared with the
oracle's deltas within eps_mf plus the FP64 setup tolerance, and its solves, wrapped
in FP64 refinement, must reach the FP64 discrete solution.
"""
import numpy as np
import pytest

from oracle import bpa
from tests.gpu_common import Case, lib, rel_inf

pytestmark = pytest.mark.gpu

TOL = 1e-12


def synthetic_rows(n, k, seed):
    """Operators whose magnitudes span 1e-14 .. 1e2, with dropped rows, zeros, negative
    zeros and entries exactly on a bpa boundary."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, k)) * 10.0 ** rng.uniform(-14, 2, (n, 1))
    x[::17] = 0.0
    x[5, :] = -0.0
    x[6, :3] = [0.75, -1.0 / 3.0, 0.998]
    x[7, :] = 1e-2  # bpa 0 at eps_mf = 1e-2 (|x| <= eps_mf)
    return x


def run_encode(mg, torch, x, eps_mf):
    n, k = x.shape
    xd = torch.from_numpy(x).cuda()
    rec = torch.empty(n, dtype=torch.int64, device="cuda")
    byt = torch.empty(n * k * 8, dtype=torch.uint8, device="cuda")
    tot = torch.empty(1, dtype=torch.int64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    mg.bpa_encode(xd, eps_mf, rec, byt, tot, st)
    torch.cuda.synchronize()
    return rec, byt, int(tot.item()), int(st.item())


@pytest.mark.parametrize("k,n", [(9, 3001), (25, 1201), (125, 97)])
@pytest.mark.parametrize("eps_mf", [1e-2, 1e-4, 1e-8, 0.0])
def test_encoder_matches_oracle_bit_exact(k, n, eps_mf):
    mg = lib()
    import torch

    x = synthetic_rows(n, k, seed=k)
    rec, byt, total, status = run_encode(mg, torch, x, eps_mf)
    assert status == 0
    b, off, stream = bpa.encode_rows(x, eps_mf)
    assert np.array_equal(rec.cpu().numpy().view(np.uint64), bpa.records(b, off))
    assert total == len(stream)
    assert byt[:total].cpu().numpy().tobytes() == stream


def test_decoder_exact_fp64_and_rounded_fp32():
    mg = lib()
    import torch

    for k, eps_mf in ((9, 1e-8), (25, 1e-4), (27, 0.0)):
        x = synthetic_rows(513, k, seed=100 + k)
        rec, byt, total, _ = run_encode(mg, torch, x, eps_mf)
        b, off, stream = bpa.encode_rows(x, eps_mf)
        ref = bpa.decode_rows(b, off, stream, k)
        out64 = torch.empty((513, k), dtype=torch.float64, device="cuda")
        out32 = torch.empty((513, k), dtype=torch.float32, device="cuda")
        mg.bpa_decode(rec, byt, out64)
        mg.bpa_decode(rec, byt, out32)
        torch.cuda.synchronize()
        assert np.array_equal(out64.cpu().numpy(), ref)
        assert np.array_equal(out32.cpu().numpy(), ref.astype(np.float32))
        if eps_mf == 0.0:
            assert np.array_equal(ref, x)  # eps_mf = 0: every operator stored exactly


def test_encoder_status_and_empty_input():
    mg = lib()
    import torch

    # below the clamped exponent range a non-zero entry cannot be stored exactly
    x = np.zeros((4, 9))
    x[2, 4] = 1e-45
    rec, _, total, status = run_encode(mg, torch, x, 0.0)
    assert status == 2 and total == 0
    x[1, 0] = np.nan
    _, _, _, status = run_encode(mg, torch, x, 1e-8)
    assert status == 1
    rec, _, total, status = run_encode(mg, torch, np.zeros((0, 9)), 1e-4)
    assert total == 0 and status == 0


@pytest.mark.parametrize("eps_mf", [1e-2, 1e-8])
def test_hierarchy_streams_hold_the_oracle_deltas(eps_mf):
    c = Case(2, 4, "grf", precision="mixed_bpa", eps_mf=eps_mf)
    torch = c.torch
    sizes = []
    for lv in range(1, c.L):
        n = c.n(lv)
        dof = c.dof(lv)
        ar = torch.empty(n, dtype=torch.int64, device="cuda")
        pr = torch.empty(n, dtype=torch.int64, device="cuda")
        ab = torch.empty(n * 9 * 8, dtype=torch.uint8, device="cuda")
        pb = torch.empty(n * 25 * 8, dtype=torch.uint8, device="cuda")
        na, npb = c.H.get_bpa(lv, ar, ab, pr, pb)
        sizes.append(na + npb)
        for rec, byt, nbytes, K, ref, scale in (
                (ar, ab, na, 9, c.O.ops[lv].a_hat, c.abs_scale(lv)),
                (pr, pb, npb, 25, c.O.ops[lv + 1].p_hat, np.ones((n, 25)))):
            r = c.host(rec).view(np.uint64)
            b = (r & np.uint64(15)).astype(np.int64)
            off = (r >> np.uint64(4)).astype(np.int64)
            assert set(np.unique(b)) <= set(bpa.BPA_CHOICES)
            assert int(np.sum(b * K)) == nbytes
            dec = bpa.decode_rows(b, off, c.host(byt)[:nbytes].tobytes(), K)
            err = np.abs(dec - ref)[dof]
            assert np.all(err <= eps_mf + TOL * scale[dof]), (lv, K, err.max())
            # the choice is the oracle's up to decisions within rounding of a boundary
            ob = np.array([bpa.choose_bpa(row, eps_mf) for row in ref[dof]])
            assert np.mean(ob != b[dof]) <= 0.02
    assert sum(sizes) > 0


@pytest.mark.parametrize("eps_mf", [1e-2, 1e-4, 1e-8])
@pytest.mark.parametrize("dim,L,eps", [(2, 4, "checker"), (3, 3, "sphere"), (2, 5, "grf")])
def test_bpa_solve_reaches_fp64_solution(dim, L, eps, eps_mf):
    c = Case(dim, L, eps, precision="mixed_bpa", eps_mf=eps_mf)
    u = c.torch.zeros(c.n(L), dtype=c.torch.float64, device="cuda")
    res = c.H.solve(u, c.b_dev, rel_tol=1e-10, max_cycles=2000)
    assert res["rel_residual"] <= 1e-10
    ug = c.host(u)
    r = c.O.residual(L, ug, c.b)
    assert np.linalg.norm(r) <= 1.0001e-10 * np.linalg.norm(c.b)
    assert rel_inf(ug, c.O.direct(c.b)) <= 1e-8


def test_bpa_hierarchies_are_single_problem():
    mg = lib()
    import torch

    c = Case(2, 3, "grf", precision="mixed_bpa", oracle=False)
    with pytest.raises(mg.MgError):
        mg.Batch([c.H])
    with pytest.raises(mg.MgError):
        mg.Server(1 << 30, precision="mixed_bpa")
    del torch
