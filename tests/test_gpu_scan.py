"""Temperature scan (ctm_scan_*) and the tensor-core GEMM launch shapes
(split-K, tile width) with their autotuner.

- Every launch shape of the tcgen05 GEMM is exact on integer operands
  (|partial sums| < 2^24 are exact in FP32 and the slices add exactly in
  FP64), so each pinned (tile width, K slices) pair must match A^t B bit for
  bit, including ragged M, N, K and slices that K does not divide.
- A scan runs the same kernels as independent handles, only on other
  streams and concurrently: each beta's trajectory, observables and step
  count must equal those of its own handle (1e-13 relative; the kernels are
  deterministic, so any larger difference means the betas interfered).
- The converged FP64 scan point at T = 0.44 matches the oracle to 1e-12 in f.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_08669_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_08669_gb300 import build
    build.build()
    from paper_2004_08669_gb300 import ctm as C
    return C


SHAPES = [(300, 200, 100), (257, 129, 333), (5, 7, 8), (1280, 288, 1280), (128, 2560, 2560)]


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_every_launch_shape_is_exact_on_integers(ctm, prec, M, N, K):
    import torch
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    A = rng.integers(-8, 9, size=(K, M)).astype(np.float64)
    B = rng.integers(-8, 9, size=(K, N)).astype(np.float64)
    ref = A.T @ B
    At, Bt = torch.tensor(A, device="cuda:0"), torch.tensor(B, device="cuda:0")
    kt = 64 if prec == "bf16" else 32
    try:
        for bn in (64, 128, 256):
            for splits in (1, 3, 8):
                ctm.ctm_tc_plan_set(prec, M, N, K, bn, splits)
                got_bn, got_sl = ctm.ctm_tc_plan_get(prec, M, N, K)
                assert got_bn == bn
                assert 1 <= got_sl <= min(splits, -(-K // kt))
                D = ctm.ctm_contract(At, Bt, prec).cpu().numpy()
                np.testing.assert_array_equal(D, ref, err_msg=f"bn={bn} splits={splits}")
    finally:
        ctm.ctm_tc_plan_set(prec, M, N, K, 0, 0)
    assert ctm.ctm_tc_plan_get(prec, M, N, K)[1] == 1


def test_plan_validation(ctm):
    with pytest.raises(ctm.CtmError):
        ctm.ctm_tc_plan_set("tf32", 10, 10, 10, 96, 1)
    with pytest.raises(ctm.CtmError):
        ctm.ctm_tc_plan_set("tf32", 10, 10, 10, 64, 17)
    with pytest.raises(ctm.CtmError):
        ctm.ctm_tc_plan_set("fp64", 10, 10, 10, 64, 1)


def test_tuned_tf32_step_stays_within_operand_precision(ctm):
    """ctm_tune times every shape of the step's three products and keeps the
    fastest; the tuned TF32 run then stays within TF32 precision of the FP64
    oracle (the same bound as the untuned form), and a second run with the
    same shapes repeats the first one bit for bit."""
    spins, beta, m = W.dodecahedron(), 1 / 0.44, 8
    q = spins.shape[0]
    N = m * q
    b = min(N, m + max(8, m // 8))
    shapes = {(N, N, m), (N, b, N), (m, N, N)}
    try:
        g = ctm.CTMRG(spins, m, beta, prec="tf32", max_subspace_iters=4)
        ents = ctm.ctm_tune(g.h, 3)
        g.close()
        assert {(e["M"], e["N"], e["K"]) for e in ents} == shapes
        for e in ents:
            assert e["bn"] in (64, 128, 256) and e["splits"] >= 1 and e["candidates"] >= 3
            assert e["ms_best"] <= e["ms_default"] * (1 + 1e-9)
            assert ctm.ctm_tc_plan_get("tf32", e["M"], e["N"], e["K"]) == (e["bn"], e["splits"])
        runs = []
        for _ in range(2):
            g = ctm.CTMRG(spins, m, beta, prec="tf32", max_subspace_iters=4)
            ks = [g.step(1)[1]["kappa"] for _ in range(200)]
            runs.append((ks, g.observables()))
            g.close()
    finally:
        for (M, Nn, K) in shapes:
            ctm.ctm_tc_plan_set("tf32", M, Nn, K, 0, 0)
    assert runs[0][0] == runs[1][0]
    o = O.CTMRG(spins, m, beta)
    o.run(5000, 1e-12)
    ref = o.observables()
    df = abs(runs[0][1]["f"] - ref["f"]) / abs(ref["f"])
    print(f"\ntuned tf32: |df|/|f| = {df:.3e}  shapes = {[(e['bn'], e['splits']) for e in ents]}")
    assert df <= 1e-4


def test_tuned_ozaki_form_tracks_fp64_form(ctm):
    """ctm_tune on the FP64-emulating form picks K slices for C~ V and U^t X
    (q = 20, m = 64: K = 1280, three exact 512-wide chunks); the tuned form
    then follows the FP64 form step by step from the same checkpoint to the
    same accuracy as untuned (|df|/|f| <= 1e-11 over 15 steps)."""
    spins, beta, m = W.dodecahedron(), 1 / 0.4398, 64
    g = ctm.CTMRG(spins, m, beta, prec="ozaki64", max_subspace_iters=4)
    g.step(10)
    blob = g.save()
    ents = ctm.ctm_tune(g.h, 3)
    g.close()
    N, b = m * 20, m + max(8, m // 8)
    assert {(e["M"], e["N"], e["K"]) for e in ents} == {(N, b, N), (m, N, N)}
    for e in ents:
        assert 1 <= e["splits"] <= 3 and e["ms_best"] <= e["ms_default"] * (1 + 1e-9)
    fs = {}
    for prec in ("ozaki64", "fp64"):
        h = ctm.CTMRG(spins, m, beta, prec=prec, max_subspace_iters=4)
        h.load(blob)
        fs[prec] = [h.step(1)[1]["kappa"] for _ in range(15)]
        h.close()
    d = max(abs(a - c) / abs(c) for a, c in zip(fs["ozaki64"], fs["fp64"]))
    print(f"\ntuned ozaki64 vs fp64 (kappa): {d:.2e}, slices {[e['splits'] for e in ents]}")
    assert d <= 1e-11


def _single(ctm, spins, m, beta, prec, steps, **kw):
    g = ctm.CTMRG(spins, m, beta, prec=prec, **kw)
    done, info = g.run(steps)
    obs = g.observables()
    om = g.spectrum()
    g.close()
    return done, obs, om


def test_fp64_scan_equals_independent_handles_and_oracle(ctm):
    spins, m = W.dodecahedron(), 8
    temps = [0.40, 0.44, 0.48]
    betas = [1.0 / t for t in temps]
    sc = ctm.Scan(spins, m, betas, workers=2)
    done, conv = sc.run(5000)
    assert conv.tolist() == [1, 1, 1]
    obs = sc.observables()
    spec = [sc.spectrum(i) for i in range(3)]
    done2, conv2 = sc.run(100)
    assert done2.tolist() == [0, 0, 0] and conv2.tolist() == [1, 1, 1]
    sc.close()
    for i, beta in enumerate(betas):
        d1, o1, om1 = _single(ctm, spins, m, beta, "fp64", 5000)
        assert done[i] == d1
        assert obs[i]["f"] == pytest.approx(o1["f"], rel=1e-13)
        assert obs[i]["M"] == pytest.approx(o1["M"], abs=1e-13)
        assert obs[i]["S_E"] == pytest.approx(o1["S_E"], abs=1e-13)
        np.testing.assert_allclose(spec[i], om1, rtol=0, atol=1e-13)
    # uneven convergence: the betas took different numbers of steps
    assert len(set(done.tolist())) > 1
    o = O.CTMRG(spins, m, betas[1])
    o.run(5000, 1e-12)
    ref = o.observables()
    assert abs(obs[1]["f"] - ref["f"]) <= 1e-12 * abs(ref["f"])
    assert obs[1]["M"] == pytest.approx(ref["M_kept"], abs=1e-10)


def test_tf32_scan_m128_equals_independent_handles(ctm):
    """The batched-scan workload's shape (q = 20, m = 128, TF32, tuned
    shapes): 8 temperatures in [0.40, 0.48] stepped 25 times by 4 workers;
    two of them are repeated on their own handles."""
    spins, m = W.dodecahedron(), 128
    temps = np.linspace(0.40, 0.48, 8)
    betas = 1.0 / temps
    sc = ctm.Scan(spins, m, betas, workers=4, prec="tf32", max_subspace_iters=4)
    ents = sc.tune(3)
    try:
        done, conv = sc.run(25)
        assert done.tolist() == [25] * 8
        obs = sc.observables()
        spec = [sc.spectrum(i) for i in (0, 5)]
        assert sc.launch_count() > 0
        sc.close()
        # the same launch shapes (process-wide table) on independent handles
        single = [_single(ctm, spins, m, betas[i], "tf32", 25, max_subspace_iters=4) for i in (0, 5)]
    finally:
        for e in ents:
            ctm.ctm_tc_plan_set("tf32", e["M"], e["N"], e["K"], 0, 0)
    for j, i in enumerate((0, 5)):
        d1, o1, om1 = single[j]
        assert d1 == 25
        assert obs[i]["f"] == pytest.approx(o1["f"], rel=1e-13)
        np.testing.assert_allclose(spec[j], om1, rtol=0, atol=1e-12)
    for o in obs:
        assert np.isfinite(o["f"]) and o["f"] < 0


def test_scan_energy_is_the_beta_derivative_of_beta_f(ctm):
    """Through the scan: beta - d, beta, beta + d stepped to convergence
    together (FP64, q = 20, m = 16, T = 0.6, d = 1e-4); the GPU's internal
    energy at beta equals the central difference of its beta f to 1e-7, the
    thermodynamic identity the oracle is pinned to for the same model."""
    spins, m, beta, d = W.dodecahedron(), 16, 1 / 0.6, 1e-4
    sc = ctm.Scan(spins, m, [beta - d, beta, beta + d], workers=3)
    done, conv = sc.run(5000)
    assert conv.tolist() == [1, 1, 1]
    obs = sc.observables()
    sc.close()
    fd = ((beta + d) * obs[2]["f"] - (beta - d) * obs[0]["f"]) / (2 * d)
    print(f"\nu = {obs[1]['u']:.12f}, d(beta f)/d beta = {fd:.12f}")
    assert abs(fd - obs[1]["u"]) <= 1e-7 * abs(obs[1]["u"])


def test_scan_invalid_arguments(ctm):
    cfg, keep = ctm.make_config(W.dodecahedron(), 8, 0.0)
    with pytest.raises(ctm.CtmError) as e:
        ctm.ctm_scan_init(cfg, [], 2)
    assert e.value.status == ctm.CTM_EINVAL
    with pytest.raises(ctm.CtmError):
        ctm.ctm_scan_init(cfg, [2.0, -1.0], 2)
    with pytest.raises(ctm.CtmError):
        ctm.ctm_scan_init(cfg, [2.0], 0)
    cfg.workspace = 1 << 40  # a bogus pointer is never touched: the size check fails first
    cfg.workspace_bytes = 16
    with pytest.raises(ctm.CtmError) as e:
        ctm.ctm_scan_init(cfg, [2.0, 2.5], 2)
    assert e.value.status == ctm.CTM_ENOMEM
    del keep
