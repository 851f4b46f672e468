"""GPU parity of the CUDA hot path (through the C ABI) against the CPU oracle.

FP64 results must match the oracle within 1e-12 relative (infinity norm over the
compared vector); integer / code outputs bit for bit.  Galerkin coarse stencils
are sums whose terms can cancel (on the 1:1e-4 checkerboard the level-1
diagonal is 5.8e7 times smaller than the sum of the magnitudes of its terms), so
their tolerance is 1e-12 times the magnitude scale |P|^T|A||P| of each entry, and
V-cycle / solve outputs are bounded by u (C1 + C2 F) (u = 2^-53, F the largest such
cancellation factor, C1 and C2 fitted to the measured errors with a margin:
tests/gpu_common.py).  Cases
span several bricks (2D level 4: 9 bricks of 27^2 cells; 3D level 3: 27 bricks of
9^3 cells) and the padded tail of every brick.
"""
import numpy as np
import pytest

from oracle import codec
from tests.gpu_common import (HIST_ATOL, HIST_RTOL, Case, full_size_checker_solve, lib, parity_check, rel_inf,
                              rowwise_rel)

pytestmark = pytest.mark.gpu

TOL = 1e-12

CASES = [
    (2, 4, "checker", "boxmg", "galerkin"),
    (2, 4, "grf", "boxmg", "galerkin"),
    (3, 3, "sphere", "boxmg", "galerkin"),
    (2, 4, "const", "dlinear", "redisc"),
    (3, 3, "grf", "dlinear", "galerkin"),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "-".join(map(str, c)))
def case(request):
    dim, L, eps, tr, co = request.param
    return Case(dim, L, eps, tr, co)


def test_stencils_match(case):
    K = 3**case.dim
    for lv in range(1, case.L + 1):
        n = case.n(lv)
        out = case.torch.empty(K * n, dtype=case.torch.float64, device="cuda")
        case.H.get_stencils(lv, out)
        st = case.host(out).reshape(K, n).T
        dof = case.dof(lv)
        # entries pointing past the upper boundary (no slot) multiply the Dirichlet value only
        has = case.grid.tables(lv)["nbr"] >= 0
        scale = case.abs_scale(lv)
        err = (np.abs(st - case.O.ops[lv].st) * has)[dof] / np.maximum(scale[dof], 1e-300)
        assert err.max() < TOL, (lv, err.max())


def test_deltas_match(case):
    if case.O.coarse != "galerkin" and case.O.transfer != "boxmg":
        pytest.skip("no deltas stored")
    for lv in range(1, case.L):
        n = case.n(lv)
        dof = case.dof(lv)
        if case.O.coarse == "galerkin":
            a = case.torch.empty(3**case.dim * n, dtype=case.torch.float64, device="cuda")
            case.H.get_deltas(lv, a_hat=a)
            ah = case.host(a).reshape(-1, n).T
            scale = case.abs_scale(lv)
            assert (np.abs(ah - case.O.ops[lv].a_hat)[dof] / np.maximum(scale[dof], 1e-300)).max() < TOL
        if case.O.transfer == "boxmg":
            p = case.torch.empty(5**case.dim * n, dtype=case.torch.float64, device="cuda")
            case.H.get_deltas(lv, p_hat=p)
            ph = case.host(p).reshape(-1, n).T
            assert np.abs(ph - case.O.ops[lv + 1].p_hat)[dof].max() < TOL


@pytest.mark.parametrize("nu", [1, 2, 3])
def test_smoother_matches(case, nu):
    for lv in (case.L, case.L - 1):
        u = case.random_vec(lv, 10 + lv)
        b = case.random_vec(lv, 20 + lv) if lv < case.L else case.b
        ud = case.dev(u)
        case.H.smooth(lv, ud, case.dev(b), nu)
        ref = case.O.smooth(lv, u, b, nu)
        assert rel_inf(case.host(ud), ref) < TOL


def test_residual_and_norm_match(case):
    for lv in (case.L, case.L - 1):
        u = case.random_vec(lv, 30 + lv)
        b = case.random_vec(lv, 40 + lv)
        r = case.torch.zeros(case.n(lv), dtype=case.torch.float64, device="cuda")
        n2 = case.H.residual(lv, case.dev(u), case.dev(b), r, want_norm=True)
        ref = case.O.residual(lv, u, b)
        assert rel_inf(case.host(r), ref) < TOL
        assert abs(n2 - float(ref @ ref)) <= 1e-12 * float(ref @ ref)


def test_transfers_match(case):
    L = case.L
    r = case.random_vec(L, 50)
    bc = case.torch.zeros(case.n(L - 1), dtype=case.torch.float64, device="cuda")
    case.H.restrict(L, case.dev(r), bc)
    assert rel_inf(case.host(bc), case.O.restrict(L, r)) < TOL
    e = case.random_vec(L - 1, 60)
    u = case.random_vec(L, 70)
    ud = case.dev(u)
    case.H.prolong(L, case.dev(e), ud)
    ref = u + np.where(case.dof(L), case.O.prolong(L, e), 0.0)
    assert rel_inf(case.host(ud), ref) < TOL


def test_vcycle_matches(case):
    u = case.random_vec(case.L, 80)
    ud = case.dev(u)
    case.H.vcycle(ud, case.b_dev)
    ref = case.O.vcycle(u, case.b)
    parity_check(f"vcycle {case.dim}d-l{case.L}-{case.O.transfer}", rel_inf(case.host(ud), ref),
                 case.amplification(), "cycle")


@pytest.mark.parametrize("persistent", [0, 1])
def test_solve_matches_oracle(case, persistent):
    H = case.H
    if persistent:
        H = case.mg.Hierarchy(case.grid, transfer=case.O.transfer, coarse=case.O.coarse, persistent=1)
        H.setup(case.eps_dev)
    u = case.torch.zeros(case.n(case.L), dtype=case.torch.float64, device="cuda")
    res = H.solve(u, case.b_dev, rel_tol=1e-10, max_cycles=400)
    ref, hist = case.O.solve(case.b, 1e-10, 400)
    assert res["cycles"] == len(hist) - 1
    amp = case.amplification()
    parity_check(f"solve {case.dim}d-l{case.L}-{case.O.transfer}", rel_inf(case.host(u), ref), amp, "solve")
    assert res["rel_residual"] <= 1e-10
    assert np.allclose(res["history"], hist[1:] / hist[0], rtol=HIST_RTOL,
                       atol=HIST_ATOL)  # b - A u cancels: ~1e-16 ||b|| absolute rounding in each residual


@pytest.mark.parametrize("dim,L,eps", [(2, 4, "checker"), (3, 3, "sphere")])
def test_fp32_finest_sweep_within_fp32_rounding(dim, L, eps):
    # finest level: no deltas, so the FP32 sweep differs from the FP64 oracle by FP32
    # rounding only; bound: 64 u32 * (|u| + omega |D^-1| (|b| + |A| |u|)) per vertex
    c = Case(dim, L, eps, precision="mixed_bf16")
    torch = c.torch
    u = c.random_vec(L, 5)
    ud = torch.from_numpy(u.astype(np.float32)).cuda()
    bd = c.b_dev.float()
    c.H.smooth_f32(L, ud, bd, 1)
    u32 = u.astype(np.float32).astype(np.float64)
    b32 = c.b.astype(np.float32).astype(np.float64)
    ref = c.O.smooth(L, u32, b32, 1)
    o = c.O.ops[L]
    bound = np.abs(u32) + c.O.omega * (np.abs(b32) + abs(o.A) @ np.abs(u32)) / o.diag
    err = np.abs(c.host(ud).astype(np.float64) - ref)
    assert np.all(err <= 64 * 2.0**-24 * bound + 1e-30)


@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16"])
def test_host_stepped_solve_matches_persistent(precision):
    # the same solve through the host-stepped CUDA-graph driver and the persistent
    # cooperative kernel: identical kernels' arithmetic, so identical cycle counts
    # and iterates within the solve tolerance
    res, us = [], []
    for persistent in (1, 0):
        c = Case(2, 4, "grf", precision=precision, persistent=persistent, oracle=(persistent == 1))
        u = c.torch.zeros(c.n(4), dtype=c.torch.float64, device="cuda")
        res.append(c.H.solve(u, c.b_dev, rel_tol=1e-10, max_cycles=500))
        us.append(c.host(u))
        if persistent == 1:
            ref = c.O.direct(c.b)
    assert res[0]["rel_residual"] <= 1e-10 and res[1]["rel_residual"] <= 1e-10
    if precision == "fp64":
        assert res[0]["cycles"] == res[1]["cycles"]
        assert rel_inf(us[0], us[1]) < 1e-11
    assert rel_inf(us[0], ref) < 1e-8 and rel_inf(us[1], ref) < 1e-8


def test_encoder_matches_oracle_bit_exact():
    mg = lib()
    import torch

    rng = np.random.default_rng(8)
    d = rng.standard_normal((4099, 27)) * np.exp(rng.uniform(-40, 5, (4099, 1)))
    d[5] = 0.0
    d[6, 3] = -1e-300
    dd = torch.from_numpy(d).cuda()
    for fmt, name in ((1, "bf16"), (2, "fp16")):
        codes = torch.empty(d.shape, dtype=torch.int16, device="cuda")
        scale = torch.empty(d.shape[0], dtype=torch.float32, device="cuda")
        mg.encode_deltas(dd, codes, scale, fmt)
        torch.cuda.synchronize()
        qo, so = codec.encode(d, name)
        assert np.array_equal(codes.cpu().numpy().view(np.uint16), qo)
        assert np.array_equal(scale.cpu().numpy().view(np.uint32), so.view(np.uint32))


def test_promoting_encoder_matches_oracle_bit_exact():
    # A10 promotion: rows whose 16-bit rounding could exceed 2^-8 of their reconstructed
    # diagonal are stored as FP32 halves with the flag in the scale's sign bit; codes,
    # low halves and signed scales equal the oracle's bit for bit, the threshold
    # equality (s = 2 |A_vv| for bf16, 16 |A_vv| for fp16) included
    mg = lib()
    import torch

    rng = np.random.default_rng(9)
    n = 5003
    d = rng.standard_normal((n, 9)) * np.exp(rng.uniform(-30, 5, (n, 1)))
    d[5] = 0.0
    smax = np.abs(d).max(axis=1)
    diag = smax * np.exp(rng.uniform(-10, 3, n)) * np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    for fmt, name, ratio in ((1, "bf16", 2.0), (2, "fp16", 16.0)):
        dg = diag.copy()
        s32 = smax.astype(np.float32).astype(np.float64)
        dg[10:20] = s32[10:20] / ratio  # exactly on the threshold: not promoted
        dd, gd = torch.from_numpy(d).cuda(), torch.from_numpy(dg).cuda()
        codes = torch.empty(d.shape, dtype=torch.int16, device="cuda")
        lo = torch.empty(d.shape, dtype=torch.int16, device="cuda")
        scale = torch.empty(n, dtype=torch.float32, device="cuda")
        mg.encode_deltas_promote(dd, gd, codes, lo, scale, fmt)
        torch.cuda.synchronize()
        qo, lo_o, so = codec.encode_promoting(d, dg, name)
        assert np.signbit(so).sum() > 100 and (~np.signbit(so)).sum() > 100
        assert not np.signbit(so[10:20]).any()
        assert np.array_equal(codes.cpu().numpy().view(np.uint16), qo)
        assert np.array_equal(lo.cpu().numpy().view(np.uint16), lo_o)
        assert np.array_equal(scale.cpu().numpy().view(np.uint32), so.view(np.uint32))


def test_mixed_codes_hold_the_oracle_deltas():
    # the codes come from the hierarchy's own FP64 deltas, so they are checked against
    # the oracle's deltas through the format's bound: |scale| = fl32(max |delta|) and
    # |fl32(q * s) - delta| <= half a unit of the 16-bit format (relative to s) + the
    # FP32 product's rounding + the FP64 setup tolerance; promoted vertices (scale < 0)
    # within FP32 rounding of each entry.  The promotion flags are the oracle's rule
    # applied to the oracle's deltas and diagonals wherever the rule's two sides are
    # not within the setup tolerance of each other
    half_unit = {"bf16": 2.0 ** -9, "fp16": 2.0 ** -12}
    n_promoted = 0
    for fmt, prec, eps in (("bf16", "mixed_bf16", "grf"), ("fp16", "mixed_fp16", "grf"),
                           ("bf16", "mixed_bf16", "checker")):
        c = Case(2, 4, eps, precision=prec)
        torch = c.torch
        for lv in range(1, 4):
            n = c.n(lv)
            dof = c.dof(lv)
            ac = torch.empty(9 * n, dtype=torch.int16, device="cuda")
            al = torch.empty(9 * n, dtype=torch.int16, device="cuda")
            pc = torch.empty(25 * n, dtype=torch.int16, device="cuda")
            asc = torch.empty(n, dtype=torch.float32, device="cuda")
            psc = torch.empty(n, dtype=torch.float32, device="cuda")
            c.H.get_codes(lv, ac, asc, pc, psc)
            c.H.get_code_lo(lv, al)
            atol = TOL * c.abs_scale(lv).max(axis=1)
            diag = c.O.ops[lv].st[:, 4]
            for cod, lo, sc, K, ref, tol in (
                    (ac, al, asc, 9, c.O.ops[lv].a_hat, atol),
                    (pc, None, psc, 25, c.O.ops[lv + 1].p_hat, np.full(n, TOL))):
                q = c.host(cod).view(np.uint16).reshape(K, n).T
                s = c.host(sc)
                flag = np.signbit(s)
                sa = np.abs(s).astype(np.float64)
                amax = np.abs(ref).max(axis=1)
                assert np.all((np.abs(sa - amax) <= 2.0 ** -24 * amax + tol)[dof])
                if lo is None:
                    assert not flag.any()
                    dec = codec.decode(q, np.abs(s), fmt).astype(np.float64)
                    bound = (half_unit[fmt] + 2.0 ** -24) * sa + 2 * tol
                    assert np.all((np.abs(dec - ref) <= bound[:, None])[dof]), (fmt, lv, K)
                    continue
                lq = c.host(lo).view(np.uint16).reshape(K, n).T
                assert not lq[~flag].any()
                dec = codec.decode_promoting(q, lq, s, fmt).astype(np.float64)
                bound = np.where(flag, 2.0 ** -23, half_unit[fmt] + 2.0 ** -24) * sa + 2 * tol
                assert np.all((np.abs(dec - ref) <= bound[:, None])[dof]), (fmt, lv, K)
                want = codec.promoted(amax.astype(np.float32), diag, fmt)
                margin = np.abs(amax * codec.HALF_UNIT[fmt] - codec.PROMOTE_REL * np.abs(diag))
                clear = margin > 1e-9 * amax + tol
                assert np.array_equal(flag[dof & clear], want[dof & clear]), (fmt, lv)
                n_promoted += int(flag[dof].sum())
    assert n_promoted > 0  # the checkerboard's interfaces cancel


@pytest.mark.parametrize("prec", ["mixed_bf16", "mixed_fp16"])
@pytest.mark.parametrize("dim,L,eps", [(2, 4, "checker"), (3, 3, "sphere"), (2, 5, "grf")])
def test_mixed_solve_reaches_fp64_solution(dim, L, eps, prec):
    c = Case(dim, L, eps, precision=prec)
    u = c.torch.zeros(c.n(L), dtype=c.torch.float64, device="cuda")
    res = c.H.solve(u, c.b_dev, rel_tol=1e-10, max_cycles=2000)
    assert res["rel_residual"] <= 1e-10
    # FP64 residual of the returned iterate, by the oracle's operator
    ug = c.host(u)
    r = c.O.residual(L, ug, c.b)
    assert np.linalg.norm(r) <= 1.0001e-10 * np.linalg.norm(c.b)
    # stated per-result error of the mixed path: within 1e-8 (infinity-norm relative)
    # of the exact discrete solution, next to an FP64 residual drop of 1e-10
    ud = c.O.direct(c.b)
    assert rel_inf(ug, ud) <= 1e-8


def test_full_size_config2_sampled_parity():
    # 2D level 6 (729^2 cells, 529,984 DoFs), seeded 9x9 checkerboard {1, 1e-4},
    # BoxMG + Galerkin FP64: compare one Jacobi sweep, one V-cycle and the setup
    c = Case(2, 6, "checker")
    L = 6
    u = c.random_vec(L, 99)
    ud = c.dev(u)
    c.H.smooth(L, ud, c.b_dev, 2)
    assert rel_inf(c.host(ud), c.O.smooth(L, u, c.b, 2)) < TOL
    ud = c.dev(u)
    c.H.vcycle(ud, c.b_dev)
    parity_check("vcycle 2d-l6-checker (full size)", rel_inf(c.host(ud), c.O.vcycle(u, c.b)), c.amplification(),
                 "cycle")
    for lv in (5, 4, 1):
        n = c.n(lv)
        out = c.torch.empty(9 * n, dtype=c.torch.float64, device="cuda")
        c.H.get_stencils(lv, out)
        st = c.host(out).reshape(9, n).T
        dof = c.dof(lv)
        has = c.grid.tables(lv)["nbr"] >= 0
        err = (np.abs(st - c.O.ops[lv].st) * has)[dof] / np.maximum(c.abs_scale(lv)[dof], 1e-300)
        assert err.max() < TOL


def test_full_size_config2_solve_matches_oracle():
    # the timed workload itself: 2D level 6 (529,984 DoFs), seeded 9x9 checkerboard
    # {1, 1e-4}, BoxMG + Galerkin, V(2,2), FP64, solved to a 1e-10 drop on both sides.
    # Same cycle count; iterate within u (C1 + C2 F) and residual history within the
    # history tolerance of the oracle's
    c, ref, hist = full_size_checker_solve()
    u = c.torch.zeros(c.n(6), dtype=c.torch.float64, device="cuda")
    res = c.H.solve(u, c.b_dev, rel_tol=1e-10, max_cycles=400)
    assert res["cycles"] == len(hist) - 1, (res["cycles"], len(hist) - 1)
    amp = c.amplification()
    parity_check("solve 2d-l6-checker (full size)", rel_inf(c.host(u), ref), amp, "solve")
    n = min(len(res["history"]), len(hist) - 1)
    assert np.allclose(res["history"][:n], hist[1:n + 1] / hist[0], rtol=HIST_RTOL, atol=HIST_ATOL)


@pytest.mark.parametrize("dim,L,precision", [(2, 6, "fp64"), (2, 6, "mixed_bf16"), (3, 4, "mixed_bf16")])
def test_autotune_changes_launch_shapes_not_results(dim, L, precision):
    # the slab depth only splits the same per-vertex arithmetic over CTAs: a V-cycle
    # before and after tuning gives bit-identical iterates; chosen depths divide B
    c = Case(dim, L, "checker", precision=precision, oracle=False)
    torch = c.torch
    u0 = c.random_vec(L, 4)
    ua = c.dev(u0)
    c.H.vcycle(ua, c.b_dev)
    if precision != "fp64":
        fa = torch.from_numpy(u0.astype(np.float32)).cuda()
        c.H.vcycle_f32(fa, c.b_dev.float())
    chosen = c.H.autotune()
    for lv, (r64, r32) in chosen.items():
        B = c.grid.info(lv).brick_edge
        for r in (r64, r32):
            assert r == 0 or (r in (1, 3, 9, 27) and B % r == 0)
    assert any(r > 0 for pair in chosen.values() for r in pair)
    ub = c.dev(u0)
    c.H.vcycle(ub, c.b_dev)
    assert torch.equal(ua, ub)
    if precision != "fp64":
        fb = torch.from_numpy(u0.astype(np.float32)).cuda()
        c.H.vcycle_f32(fb, c.b_dev.float())
        assert torch.equal(fa, fb)


def test_edge_cases():
    mg = lib()
    import torch

    # smallest hierarchy: level 2 over the coarsest level 1
    c = Case(2, 2, "checker3")
    u = torch.zeros(c.n(2), dtype=torch.float64, device="cuda")
    res = c.H.solve(u, c.b_dev, rel_tol=1e-12, max_cycles=200)
    assert rel_inf(c.host(u), c.O.direct(c.b)) < 1e-10
    # zero right-hand side: converged at once with u = 0
    z = torch.zeros_like(c.b_dev)
    res = c.H.solve(u, z, rel_tol=1e-10, max_cycles=10)
    assert res["cycles"] == 0 and float(u.abs().max()) == 0.0
    # nu = 0 smoothing is the identity
    v = c.dev(c.random_vec(2, 3))
    v0 = v.clone()
    c.H.smooth(2, v, c.b_dev, 0)
    assert torch.equal(v, v0)
    # non-finite data is reported, not propagated silently
    bn = c.b_dev.clone()
    bn[int(np.nonzero(c.dof(2))[0][0])] = float("nan")
    res = c.H.solve(u, bn, rel_tol=1e-10, max_cycles=10, raise_on_fail=False)
    assert res["status"] == 6
    # invalid arguments
    with pytest.raises(mg.MgError):
        c.H.smooth(7, v, c.b_dev, 1)
    with pytest.raises(mg.MgError):
        mg.Hierarchy(c.grid, coarsest_level=2)


def test_sin_benchmark_config1():
    # the paper's `sin` benchmark as the 2D level-4 workload: eps = 1, geometric V(2,2)
    # (d-linear transfers, rediscretised coarse operators), solved to a 1e-8 drop.  The
    # GPU takes the oracle's cycles and iterate, and the discrete solution is within
    # the O(h^2) discretisation error of prod sin(pi x_i)
    import synthetic as syn

    c = Case(2, 4, "const", "dlinear", "redisc", load="sin")
    u = c.torch.zeros_like(c.b_dev)
    res = c.H.solve(u, c.b_dev, rel_tol=1e-8, max_cycles=200)
    ref, hist = c.O.solve(c.b, 1e-8, 200)
    assert res["cycles"] == len(hist) - 1
    got = c.host(u)
    parity_check("solve 2d-l4-sin", rel_inf(got, ref), 1.0, "solve")
    exact = c.grid.to_slots(4, syn.sin_solution(4, 2))
    err = np.abs(got - exact)[c.dof(4)].max()
    assert err < 4.0 / 81**2  # O(h^2) with h = 1/81 (the oracle's discrete solution: 3.8e-4 = 2.5 h^2)


@pytest.mark.parametrize("dim,L", [(2, 4), (3, 3)])
def test_jump_benchmark(dim, L):
    # the paper's `jump` benchmark (eps 1 left of x_1 = 0.5, 0.1 right of it, f = 1) with
    # BoxMG + Galerkin: the oracle's cycles and iterate at a 1e-10 drop
    c = Case(dim, L, "jump", "boxmg", "galerkin", load="unit")
    u = c.torch.zeros_like(c.b_dev)
    res = c.H.solve(u, c.b_dev, rel_tol=1e-10, max_cycles=300)
    ref, hist = c.O.solve(c.b, 1e-10, 300)
    assert res["cycles"] == len(hist) - 1
    parity_check(f"solve {dim}d-l{L}-jump", rel_inf(c.host(u), ref), c.amplification(), "solve")
