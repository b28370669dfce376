"""ctypes binding of the plain FP64 CPU oracle (``ctm_oracle.c``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference legs of ``bench.py`` may use this module.  The GPU
product path never imports it.

The oracle follows Algorithm 3 of arXiv:2004.08669 (Symmetric-CTMRG and
Sub-CTMRG), Algorithms 1-2 (P-Index, P-Index2), Eq. (1)-(2) for the vertex
weight and Eq. (4)-(6) for the observables, with the readings R1-R6 listed in
``ctm_oracle.h``.  Storage is the paper's: column-major, first leg fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ctm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libctm_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11 + OpenMP, no host-specific flags)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_SRC[:-2] + ".h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.or_weight_matrix.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, _dp]
            L.or_weight_matrix_bond.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, _dp]
            L.or_pindex.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
            L.or_pindex2.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
            L.or_sub_ctmrg.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
            L.or_ctilde_entries.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp]
            L.or_eigh.argtypes = [ctypes.c_int, _dp, _dp, _dp]
            L.or_eigh.restype = ctypes.c_int
            L.or_num_threads.restype = ctypes.c_int
            L.or_entropy.argtypes = [_dp, ctypes.c_int, ctypes.c_int]
            L.or_entropy.restype = ctypes.c_double
            L.or_create.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_double]
            L.or_create.restype = ctypes.c_void_p
            L.or_destroy.argtypes = [ctypes.c_void_p]
            L.or_step.argtypes = [ctypes.c_void_p, _dp]
            L.or_step.restype = ctypes.c_int
            L.or_observables.argtypes = [ctypes.c_void_p, _dp]
            L.or_observables.restype = ctypes.c_int
            L.or_extend.argtypes = [ctypes.c_void_p, _dp]
            L.or_get_state.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.POINTER(ctypes.c_int)]
            L.or_set_state.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_int]
            L.or_set_weights.argtypes = [ctypes.c_void_p, _dp, _dp]
            L.or_row_transfer.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            L.or_row_transfer_spectrum.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
            L.or_row_transfer_spectrum.restype = ctypes.c_int
            L.or_steps_done.argtypes = [ctypes.c_void_p]
            L.or_steps_done.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["F_CONTIGUOUS"] or a.ndim == 1
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return lib().or_num_threads()


def entropy(ev, power: int = 4) -> float:
    """-sum p ln p with p_i = |ev_i|^power / sum |ev|^power (Eq. 6: power 4)."""
    ev = np.ascontiguousarray(ev, dtype=np.float64)
    return float(lib().or_entropy(ev.ctypes.data_as(_dp), len(ev), int(power)))


def weight_matrix(spins: np.ndarray, beta: float, bond: bool = False) -> np.ndarray:
    """q^2 x q^2 matrix form of W (Eq. 1-2, Algorithm 3, reading R1)."""
    spins = np.ascontiguousarray(spins, dtype=np.float64)
    q, dim = spins.shape
    w = np.zeros((q * q, q * q), order="F")
    fn = lib().or_weight_matrix_bond if bond else lib().or_weight_matrix
    fn(q, dim, spins.ctypes.data_as(_dp), float(beta), _p(w))
    return w


def pindex(A: np.ndarray, a: int, b: int, c: int, d: int) -> np.ndarray:
    A = _f64(A)
    assert A.shape == (a * b, c * d)
    B = np.zeros((a * c, b * d), order="F")
    lib().or_pindex(_p(A), a, b, c, d, _p(B))
    return B


def pindex2(A: np.ndarray, a: int, b: int, c: int) -> np.ndarray:
    A = _f64(A)
    assert A.shape == (a * b, c)
    B = np.zeros((a, c * b), order="F")
    lib().or_pindex2(_p(A), a, b, c, _p(B))
    return B


def sub_ctmrg(P: np.ndarray, Pp: np.ndarray, w: np.ndarray, m: int, q: int) -> np.ndarray:
    P, Pp, w = _f64(P), _f64(Pp), _f64(w)
    N = m * q
    out = np.zeros((N, N), order="F")
    lib().or_sub_ctmrg(m, q, _p(P), _p(Pp), _p(w), _p(out))
    return out


def ctilde_entries(P, omega, w, m: int, q: int, rows, cols) -> np.ndarray:
    """Entries C~[rows[i], cols[i]] of Sub-CTMRG(P, Omega P, W), one by one."""
    P, w = _f64(P), _f64(w)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    r = np.ascontiguousarray(rows, dtype=np.int32)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros(len(r))
    ip = ctypes.POINTER(ctypes.c_int)
    lib().or_ctilde_entries(m, q, _p(P), om.ctypes.data_as(_dp), _p(w), len(r), r.ctypes.data_as(ip),
                            c.ctypes.data_as(ip), out.ctypes.data_as(_dp))
    return out


def row_transfer(P: np.ndarray, w: np.ndarray, m: int, q: int) -> np.ndarray:
    """The renormalised row-to-row transfer matrix (m^2 q square) built from
    P (m x m q) and the weight matrix w (reading R10)."""
    P, w = _f64(P), _f64(w)
    n = m * q * m
    T = np.zeros((n, n), order="F")
    lib().or_row_transfer(m, q, _p(P), _p(w), _p(T))
    return T


def eigh(A: np.ndarray):
    """All eigenpairs of a symmetric matrix, sorted by |eigenvalue| descending."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    n = A.shape[0]
    ev = np.zeros(n)
    Z = np.zeros((n, n), order="F")
    st = lib().or_eigh(n, _p(A), _p(ev), _p(Z))
    if st != 0:
        raise RuntimeError("oracle eigensolver did not converge")
    return ev, Z


class CTMRG:
    """Symmetric-CTMRG of Algorithm 3 for one temperature."""

    STEP_KEYS = ("kappa", "delta", "S_E_paper", "S_E_kept", "m_eff", "c_paper", "live_dim")
    OBS_KEYS = ("f", "M_kept", "M_full", "u_kept", "u_full", "S_E_kept", "S_E_full", "kappa")

    def __init__(self, spins, m: int, beta: float, boundary_spin: int = 0,
                 tol_cluster: float = 1e-10, tol_zero: float = 1e-10):
        spins = np.ascontiguousarray(spins, dtype=np.float64)
        self.q, self.dim = spins.shape
        self.m = m
        self.N = m * self.q
        self.beta = beta
        self._spins = spins
        h = lib().or_create(self.q, self.dim, spins.ctypes.data_as(_dp), m, float(beta),
                            boundary_spin, tol_cluster, tol_zero)
        if not h:
            raise ValueError("invalid oracle configuration")
        self._h = ctypes.c_void_p(h)

    def close(self):
        if getattr(self, "_h", None):
            lib().or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self) -> dict:
        info = np.zeros(7)
        if lib().or_step(self._h, info.ctypes.data_as(_dp)) != 0:
            raise RuntimeError("oracle step failed (eigensolver)")
        return dict(zip(self.STEP_KEYS, info.tolist()))

    def run(self, max_steps: int, tol: float = 1e-12) -> list:
        hist = []
        for _ in range(max_steps):
            r = self.step()
            hist.append(r)
            if r["delta"] < tol:
                break
        return hist

    def observables(self) -> dict:
        out = np.zeros(8)
        if lib().or_observables(self._h, out.ctypes.data_as(_dp)) != 0:
            raise RuntimeError("oracle observables failed")
        return dict(zip(self.OBS_KEYS, out.tolist()))

    def row_transfer_spectrum(self, k: int = 4) -> np.ndarray:
        """k largest-modulus eigenvalues of the row-to-row transfer matrix
        of the current state (full dense diagonalisation)."""
        lam = np.zeros(k)
        if lib().or_row_transfer_spectrum(self._h, int(k), lam.ctypes.data_as(_dp)) != 0:
            raise RuntimeError("oracle eigensolver did not converge")
        return lam

    def xi(self) -> float:
        """Effective correlation length xi_e = 1 / ln|l0 / l1| in units of
        the vertex-row spacing."""
        lam = self.row_transfer_spectrum(2)
        return 1.0 / np.log(abs(lam[0] / lam[1]))

    def extend(self) -> np.ndarray:
        out = np.zeros((self.N, self.N), order="F")
        lib().or_extend(self._h, _p(out))
        return out

    def get_state(self):
        P = np.zeros((self.m, self.N), order="F")
        om = np.zeros(self.N)
        live = ctypes.c_int(0)
        lib().or_get_state(self._h, _p(P), om.ctypes.data_as(_dp), ctypes.byref(live))
        return P, om, live.value

    def set_state(self, P, omega, live: int):
        P = _f64(P)
        om = np.ascontiguousarray(omega, dtype=np.float64)
        lib().or_set_state(self._h, _p(P), om.ctypes.data_as(_dp), int(live))

    def set_weights(self, w=None, wh=None):
        w = None if w is None else _f64(w)
        wh = None if wh is None else _f64(wh)
        lib().or_set_weights(self._h, None if w is None else _p(w), None if wh is None else _p(wh))

    @property
    def steps(self) -> int:
        return lib().or_steps_done(self._h)
