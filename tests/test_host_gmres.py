"""The host GMRES of the implicit derivative (csrc/host_gmres.h), compiled
with g++ into a small driver and checked against a dense solve (no GPU)."""
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("gmres") / "host_gmres_driver")
    subprocess.run(["g++", "-std=c++17", "-O2", "-o", exe, os.path.join(HERE, "host_gmres_driver.cpp")], check=True)
    return exe


def solve(driver, tmp_path, A, b, tol=1e-13, max_iter=200, fail_after=-1):
    n = len(b)
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(fin, "wb") as f:
        f.write(np.array([n, max_iter, fail_after], dtype=np.int32).tobytes())
        f.write(np.array([tol], dtype=np.float64).tobytes())
        f.write(np.asfortranarray(A, dtype=np.float64).tobytes(order="F"))
        f.write(np.asarray(b, dtype=np.float64).tobytes())
    subprocess.run([driver, fin, fout], check=True)
    raw = open(fout, "rb").read()
    st, iters = np.frombuffer(raw[:8], dtype=np.int32)
    res = np.frombuffer(raw[8:16], dtype=np.float64)[0]
    x = np.frombuffer(raw[16:], dtype=np.float64)
    return int(st), int(iters), float(res), x


def test_solves_a_nonsymmetric_system(driver, tmp_path):
    rng = np.random.default_rng(21)
    n = 60
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    st, iters, res, x = solve(driver, tmp_path, A, b)
    assert st == 0 and res <= 1e-13 and 0 < iters <= n
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-11, atol=1e-11)


def test_unstable_fixed_point_operator(driver, tmp_path):
    """I - J with J having an eigenvalue above one (an unstable fixed point,
    where iterating the tangent diverges) is still solved."""
    rng = np.random.default_rng(22)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    J = Q @ np.diag(np.r_[1.07, rng.uniform(-0.8, 0.8, n - 1)]) @ Q.T + 0.05 * rng.standard_normal((n, n))
    A = np.eye(n) - J
    b = rng.standard_normal(n)
    st, iters, res, x = solve(driver, tmp_path, A, b)
    assert st == 0
    np.testing.assert_allclose(A @ x, b, atol=1e-10 * np.abs(b).max())


def test_zero_right_side_and_status_codes(driver, tmp_path):
    rng = np.random.default_rng(23)
    n = 30
    A = np.eye(n) + 0.5 * rng.standard_normal((n, n)) / np.sqrt(n)
    st, iters, res, x = solve(driver, tmp_path, A, np.zeros(n))
    assert st == 0 and iters == 0 and not x.any()
    st, iters, res, x = solve(driver, tmp_path, A, rng.standard_normal(n), max_iter=3)
    assert st == 1 and res > 1e-13
    st, *_ = solve(driver, tmp_path, A, rng.standard_normal(n), fail_after=2)
    assert st == 2
