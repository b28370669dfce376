"""The no-allocation eigensolver entry point, for callers that cannot allocate
device memory (fixed memory pools, hosts that only receive device pointers).

It must give the same eigenpairs as the allocating ctm_symeig, call after call,
although every call reuses the library's one static scratch array.  This file
is collected last so that a failure here leaves every other test already run.
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


def _compare(ctm, A):
    import torch
    n = A.shape[0]
    At = torch.tensor(A, device="cuda:0")
    ev_ref, vec_ref, st_ref = ctm.ctm_symeig(At)
    ev, vec, st = ctm.ctm_symeig_noalloc(At)
    assert st == st_ref == ctm.CTM_OK
    ev, vec = ev.cpu().numpy(), vec.cpu().numpy()
    ev_ref, vec_ref = ev_ref.cpu().numpy(), vec_ref.cpu().numpy()
    scale = np.abs(ev_ref).max()
    # same solver, same inputs: the same eigenvalues to rounding
    np.testing.assert_allclose(ev, ev_ref, rtol=0, atol=1e-13 * n * scale)
    # eigenvectors agree up to sign (distinct eigenvalues): compare projectors
    for i in range(n):
        d = abs(float(vec[:, i] @ vec_ref[:, i]))
        assert d == pytest.approx(1.0, abs=1e-10)
    assert np.abs(A @ vec - vec * ev).max() <= 1e-13 * n * scale


def test_noalloc_matches_allocating_solver_twice(ctm):
    rng = np.random.default_rng(2004)
    for n in (97, 256):  # two calls in a row, different sizes, shared scratch
        A = rng.standard_normal((n, n))
        _compare(ctm, A + A.T)


def test_noalloc_rejects_oversize(ctm):
    import torch
    n = 513
    A = torch.zeros(n, n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(ctm.CtmError) as e:
        ctm.ctm_symeig_noalloc(A)
    assert e.value.status == ctm.CTM_EINVAL
    assert "CTM_SYMEIG_NOALLOC_MAX_N" in str(e.value)
