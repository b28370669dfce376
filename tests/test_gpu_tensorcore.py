"""tcgen05 contraction kernel (ctm_contract in TF32 / BF16) against exact
references.

- Integer-valued operands (exact in bf16/tf32) with |sums| < 2^24 make the
  FP32 tensor-core accumulation exact: the result must match bit for bit.
  This pins the tile indexing, the TMA swizzle and the MMA descriptors.
- Random operands: the reference is the exact product of the operands
  rounded as the kernel rounds them (bf16: nearest-even; tf32: nearest,
  ties away); the only difference left is FP32 accumulation order, bounded
  by K * 2^-24 * (|A|^t |B|).
Shapes cover ragged M, N and K tails, K below one 64-wide tile, and the
C~ V shape of the m = 256 step (5120 x 288 x 5120).
"""
import numpy as np
import pytest

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


def round_bf16(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def round_tf32(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x1000) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


SHAPES = [(128, 128, 64), (300, 200, 100), (5, 7, 8), (257, 129, 333), (1280, 288, 1280)]


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_contract_exact_on_integers(ctm, prec, M, N, K):
    import torch
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.integers(-8, 9, size=(K, M)).astype(np.float64)
    B = rng.integers(-8, 9, size=(K, N)).astype(np.float64)
    D = ctm.ctm_contract(torch.tensor(A, device="cuda:0"), torch.tensor(B, device="cuda:0"), prec).cpu().numpy()
    np.testing.assert_array_equal(D, A.T @ B)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("M,N,K", SHAPES + [(5120, 288, 5120)])
def test_contract_random_matches_rounded_reference(ctm, prec, M, N, K):
    import torch
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((K, M))
    B = rng.standard_normal((K, N))
    D = ctm.ctm_contract(torch.tensor(A, device="cuda:0"), torch.tensor(B, device="cuda:0"), prec).cpu().numpy()
    r = round_bf16 if prec == "bf16" else round_tf32
    Ar, Br = r(A), r(B)
    ref = Ar.T @ Br
    bound = 2.0 * K * 2.0 ** -24 * (np.abs(Ar).T @ np.abs(Br)) + 1e-30
    assert np.all(np.abs(D - ref) <= bound)
    # and the rounding itself is the documented one: the error against the
    # unrounded product is of the operand precision's size
    rel = np.abs(D - A.T @ B).max() / np.abs(A.T @ B).max()
    assert rel < (5e-2 if prec == "bf16" else 5e-3)


def test_contract_fp64_matches_numpy(ctm):
    import torch
    rng = np.random.default_rng(9)
    A = rng.standard_normal((333, 129))
    B = rng.standard_normal((333, 77))
    D = ctm.ctm_contract(torch.tensor(A, device="cuda:0"), torch.tensor(B, device="cuda:0"), "fp64").cpu().numpy()
    np.testing.assert_allclose(D, A.T @ B, rtol=1e-13, atol=1e-12)


# ---- FP64 emulated on the bf16 tensor cores (Ozaki-style digit splitting)

@pytest.mark.parametrize("M,N,K", SHAPES + [(64, 64, 1100)])
def test_ozaki_exact_on_integers(ctm, M, N, K):
    """Small integers split into a single digit each: the product is exact."""
    import torch
    rng = np.random.default_rng(3 * M + N + K)
    A = rng.integers(-8, 9, size=(K, M)).astype(np.float64)
    B = rng.integers(-8, 9, size=(K, N)).astype(np.float64)
    D = ctm.ctm_contract(torch.tensor(A, device="cuda:0"), torch.tensor(B, device="cuda:0"), "ozaki64").cpu().numpy()
    np.testing.assert_array_equal(D, A.T @ B)


@pytest.mark.parametrize("s", [3, 4, 5, 6, 7])
def test_ozaki_error_bound(ctm, s):
    """Random FP64 operands with rows spanning several decades: the error of
    every element stays below (2^(-7s+4) + 2^-42) K max|A_row| max|B_row|:
    the truncation of the digit expansion, and the double-float combination
    of the exact chunk sums (about 2^-48 per addition)."""
    import torch
    rng = np.random.default_rng(40 + s)
    M, N, K = 300, 200, 1500
    A = rng.standard_normal((K, M)) * np.exp(rng.uniform(-5, 5, (K, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-5, 5, (K, 1)))
    D = ctm.ctm_contract(torch.tensor(A, device="cuda:0"), torch.tensor(B, device="cuda:0"), "ozaki64", s).cpu().numpy()
    ref = A.T @ B
    bound = (2.0 ** (-7 * s + 4) + 2.0 ** -42) * K * np.abs(A).max(axis=0)[:, None] * np.abs(B).max(axis=0)[None, :]
    assert np.all(np.abs(D - ref) <= bound + 1e-300)


def test_ozaki_near_fp64_at_step_shape(ctm):
    """The C~ V shape of the m = 256 step with s = 6: close to FP64."""
    import torch
    rng = np.random.default_rng(7)
    M, N, K = 5120, 288, 5120
    A = rng.standard_normal((K, M))
    B = rng.standard_normal((K, N))
    D = ctm.ctm_contract(torch.tensor(A, device="cuda:0"), torch.tensor(B, device="cuda:0"), "ozaki64", 6)
    ref = A.T @ B  # numpy on the host
    rel = float(np.abs(D.cpu().numpy() - ref).max() / np.abs(ref).max())
    print(f"\nozaki s=6 at 5120x288x5120: max |err| / max |D| = {rel:.3e}")
    assert rel < 1e-11


@pytest.mark.parametrize("s", [7])
def test_ozaki_form_matches_oracle_m8(ctm, s):
    """FP64 emulated on the bf16 tensor cores (s digit planes): per-step kappa
    and the converged free energy against the FP64 oracle.  Measured on a
    GB300 with s = 7: |df|/|f| = 9e-14, |dM| = 2e-12 (s = 6 leaves errors of
    about 2^-42 K relative to each row's largest entry; that is too coarse for
    the small kept eigenvalues and the run drifts to another fixed point,
    |df|/|f| = 3e-6)."""
    from oracle import oracle as O
    from paper_2004_08669_gb300 import workloads as W
    spins, beta = W.dodecahedron(), 1 / 0.44
    g = ctm.CTMRG(spins, 8, beta, prec="ozaki64", ozaki_slices=s, max_subspace_iters=400)
    o = O.CTMRG(spins, 8, beta)
    for _ in range(25):
        _, info, _ = g.step(1)
        r = o.step()
        assert info["m_eff"] == int(r["m_eff"])
        assert info["kappa"] == pytest.approx(r["kappa"], rel=1e-11)
    g.close()
    g = ctm.CTMRG(spins, 8, beta, prec="ozaki64", ozaki_slices=s)
    done, info = g.run(5000)
    obs = g.observables()
    o = O.CTMRG(spins, 8, beta)
    o.run(5000, 1e-12)
    ref = o.observables()
    df = abs(obs["f"] - ref["f"]) / abs(ref["f"])
    print(f"\nozaki64 s={s} m=8: |df|/|f| = {df:.3e}, |dM| = {abs(obs['M'] - ref['M_kept']):.3e}, "
          f"steps {done} (oracle {o.steps})")
    assert df <= 1e-12
    assert obs["M"] == pytest.approx(ref["M_kept"], abs=1e-9)
    g.close()
