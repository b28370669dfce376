"""Thin ctypes binding of libctm_gb300.so (include/ctm.h), same names.

Argument marshalling only: every step of the CTMRG runs in the library's
CUDA kernels.  Importing this module loads the library and raises if it is
missing; there is no CPU fallback.  PyTorch provides the device workspace
(allocated through its caching allocator) and the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libctm_gb300.so")

CTM_OK, CTM_EINVAL, CTM_ENOMEM, CTM_ENOTCONVERGED, CTM_ENUMERIC, CTM_ETIMEOUT, CTM_ECUDA, CTM_EUNSUPPORTED = range(8)
CTM_FP64, CTM_TF32, CTM_BF16, CTM_OZAKI64 = range(4)
PRECISIONS = {"fp64": CTM_FP64, "tf32": CTM_TF32, "bf16": CTM_BF16, "ozaki64": CTM_OZAKI64}
_STATUS = ["CTM_OK", "CTM_EINVAL", "CTM_ENOMEM", "CTM_ENOTCONVERGED", "CTM_ENUMERIC", "CTM_ETIMEOUT",
           "CTM_ECUDA", "CTM_EUNSUPPORTED"]

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class ctm_config(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int), ("dim", ctypes.c_int), ("spins", _dp), ("m", ctypes.c_int),
                ("beta", ctypes.c_double), ("boundary_spin", ctypes.c_int), ("prec", ctypes.c_int),
                ("ozaki_slices", ctypes.c_int), ("tol_spectrum", ctypes.c_double), ("max_steps", ctypes.c_int),
                ("block_extra", ctypes.c_int), ("max_subspace_iters", ctypes.c_int),
                ("subspace_tol", ctypes.c_double), ("tol_cluster", ctypes.c_double),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t)]


class ctm_step_info(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_double), ("delta", ctypes.c_double), ("S_E", ctypes.c_double),
                ("residual", ctypes.c_double), ("m_eff", ctypes.c_int), ("live_dim", ctypes.c_int),
                ("subspace_iters", ctypes.c_int), ("jacobi_sweeps", ctypes.c_int), ("steps", ctypes.c_int),
                ("converged", ctypes.c_int), ("rr_refined", ctypes.c_longlong), ("rr_jacobi", ctypes.c_longlong),
                ("rr_fail_reason", ctypes.c_int), ("rr_last_iter", ctypes.c_int), ("rr_last_max", ctypes.c_double),
                ("jacobi_rotations", ctypes.c_int * 8), ("rr_fail_counts", ctypes.c_longlong * 5)]

    def to_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["jacobi_rotations"] = list(d["jacobi_rotations"])
        d["rr_fail_counts"] = list(d["rr_fail_counts"])
        return d


class ctm_obs(ctypes.Structure):
    _fields_ = [("f", ctypes.c_double), ("M", ctypes.c_double), ("u", ctypes.c_double),
                ("S_E", ctypes.c_double), ("delta", ctypes.c_double), ("steps", ctypes.c_int),
                ("converged", ctypes.c_int)]

    def to_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ctm_prof_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class ctm_xi_result(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double * 4), ("residual", ctypes.c_double * 4), ("xi", ctypes.c_double),
                ("iterations", ctypes.c_int), ("converged", ctypes.c_int)]

    def to_dict(self):
        return {"lambda": list(self.lambda_), "residual": list(self.residual), "xi": self.xi,
                "iterations": self.iterations, "converged": self.converged}


class ctm_tangent_out(ctypes.Structure):
    _fields_ = [("P_new", ctypes.POINTER(ctypes.c_double)), ("omega_new", ctypes.POINTER(ctypes.c_double)),
                ("P_dot_new", ctypes.POINTER(ctypes.c_double)), ("omega_dot_new", ctypes.POINTER(ctypes.c_double)),
                ("kappa", ctypes.c_double), ("kappa_dot", ctypes.c_double), ("m_eff", ctypes.c_int),
                ("ritz_pairs", ctypes.c_int), ("deflate_iterations", ctypes.c_int),
                ("subspace_iterations", ctypes.c_int)]


class ctm_tune_entry(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("N", ctypes.c_int), ("K", ctypes.c_int), ("bn", ctypes.c_int),
                ("splits", ctypes.c_int), ("ms_default", ctypes.c_double), ("ms_best", ctypes.c_double),
                ("candidates", ctypes.c_int)]

    def to_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CtmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS[status] if 0 <= status < len(_STATUS) else status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2004_08669_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    sig = {
        "ctm_workspace_size": [ctypes.POINTER(ctm_config), ctypes.POINTER(ctypes.c_size_t)],
        "ctm_init": [ctypes.POINTER(H), ctypes.POINTER(ctm_config), ctypes.c_void_p],
        "ctm_step": [H, ctypes.c_int, _ip, ctypes.POINTER(ctm_step_info)],
        "ctm_observables": [H, ctypes.POINTER(ctm_obs)],
        "ctm_step_backward": [H, ctypes.POINTER(ctm_obs), _dp],
        "ctm_get_spectrum": [H, _dp],
        "ctm_xi": [H, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctm_xi_result)],
        "ctm_tangent_step": [H, _dp, _dp, ctypes.c_int, ctypes.POINTER(ctm_tangent_out)],
        "ctm_get_state": [H, _dp, _dp, _ip],
        "ctm_set_state": [H, _dp, _dp, ctypes.c_int],
        "ctm_save": [H, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)],
        "ctm_load": [H, ctypes.c_void_p, ctypes.c_size_t],
        "ctm_extend": [H],
        "ctm_get_ctilde": [H, _ip, _ip, ctypes.c_int, _dp],
        "ctm_eigen": [H, _dp, _dp, _ip],
        "ctm_profile": [H, ctypes.c_int],
        "ctm_profile_read": [H, ctypes.POINTER(ctm_prof_entry), ctypes.c_int, _ip],
        "ctm_launch_count": [H, ctypes.POINTER(ctypes.c_longlong)],
        "ctm_tune": [H, ctypes.c_int, ctypes.POINTER(ctm_tune_entry), ctypes.c_int, _ip],
        "ctm_tc_plan_set": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
        "ctm_tc_plan_get": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip, _ip],
        "ctm_scan_workspace_size": [ctypes.POINTER(ctm_config), ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
        "ctm_scan_init": [ctypes.POINTER(H), ctypes.POINTER(ctm_config), ctypes.c_int, _dp, ctypes.c_int,
                          ctypes.c_void_p],
        "ctm_scan_tune": [H, ctypes.c_int, ctypes.POINTER(ctm_tune_entry), ctypes.c_int, _ip],
        "ctm_scan_run": [H, ctypes.c_int, _ip, _ip],
        "ctm_scan_observables": [H, ctypes.POINTER(ctm_obs)],
        "ctm_scan_handle": [H, ctypes.c_int, ctypes.POINTER(H)],
        "ctm_scan_get_spectrum": [H, ctypes.c_int, _dp],
        "ctm_symeig_workspace_size": [ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
        "ctm_symeig_noalloc": [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
        "ctm_contract_workspace_size": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_size_t)],
        "ctm_contract": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                         ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                         ctypes.c_size_t, ctypes.c_void_p],
        "ctm_symeig": [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                       ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.ctm_last_error.restype = ctypes.c_char_p
    L.ctm_last_error.argtypes = []
    L.ctm_destroy.restype = None
    L.ctm_destroy.argtypes = [H]
    L.ctm_scan_destroy.restype = None
    L.ctm_scan_destroy.argtypes = [H]
    return L


lib = _load()


def ctm_last_error() -> str:
    return lib.ctm_last_error().decode()


def _check(status: int, allow=(CTM_OK,)) -> int:
    if status not in allow:
        raise CtmError(status, ctm_last_error())
    return status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def make_config(spins, m: int, beta: float, boundary_spin: int = 0, prec: str = "fp64", **kw) -> tuple:
    spins = np.ascontiguousarray(spins, dtype=np.float64)
    cfg = ctm_config()
    cfg.q, cfg.dim = spins.shape
    cfg.spins = _dptr(spins)
    cfg.m = int(m)
    cfg.beta = float(beta)
    cfg.boundary_spin = int(boundary_spin)
    cfg.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg, spins  # keep spins alive with the config


def ctm_workspace_size(cfg: ctm_config) -> int:
    n = ctypes.c_size_t(0)
    _check(lib.ctm_workspace_size(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def ctm_init(cfg: ctm_config, stream: int = 0):
    h = ctypes.c_void_p()
    _check(lib.ctm_init(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(stream)))
    return h


def ctm_step(h, nsteps: int):
    done = ctypes.c_int(0)
    info = ctm_step_info()
    st = _check(lib.ctm_step(h, int(nsteps), ctypes.byref(done), ctypes.byref(info)),
                (CTM_OK, CTM_ENOTCONVERGED))
    return done.value, info, st


def ctm_observables(h):
    o = ctm_obs()
    st = _check(lib.ctm_observables(h, ctypes.byref(o)), (CTM_OK, CTM_ENOTCONVERGED))
    return o, st


def ctm_step_backward(h, grad_obs: ctm_obs) -> float:
    """sum_k grad_obs_k d obs_k / d beta at the converged fixed point (the
    library builds the free energy's term; see ctm.h)."""
    g = np.zeros(1)
    _check(lib.ctm_step_backward(h, ctypes.byref(grad_obs), _dptr(g)))
    return float(g[0])


def ctm_xi(h, max_iters: int = 0, tol: float = 0.0) -> tuple:
    r = ctm_xi_result()
    st = _check(lib.ctm_xi(h, int(max_iters), float(tol), ctypes.byref(r)), (CTM_OK, CTM_ENOTCONVERGED))
    return r.to_dict(), st


def ctm_tangent_step(h, m: int, q: int, P_dot: np.ndarray, omega_dot: np.ndarray, source: bool = True) -> dict:
    """One step and its beta tangent from the handle's current state; arrays
    in the paper's layout (P: m x m q, omega: m)."""
    N = m * q
    P_dot = np.asfortranarray(P_dot, dtype=np.float64)
    om_dot = np.ascontiguousarray(omega_dot, dtype=np.float64)
    if P_dot.shape != (m, N) or om_dot.shape != (m,):
        raise ValueError("P_dot must be m x m q and omega_dot m long")
    P_new, P_dot_new = np.zeros((m, N), order="F"), np.zeros((m, N), order="F")
    om_new, om_dot_new = np.zeros(m), np.zeros(m)
    r = ctm_tangent_out()
    r.P_new, r.omega_new, r.P_dot_new, r.omega_dot_new = _dptr(P_new), _dptr(om_new), _dptr(P_dot_new), _dptr(om_dot_new)
    _check(lib.ctm_tangent_step(h, _dptr(P_dot), _dptr(om_dot), int(bool(source)), ctypes.byref(r)))
    return {"P_new": P_new, "omega_new": om_new, "P_dot_new": P_dot_new, "omega_dot_new": om_dot_new,
            "kappa": r.kappa, "kappa_dot": r.kappa_dot, "m_eff": r.m_eff, "ritz_pairs": r.ritz_pairs,
            "deflate_iterations": r.deflate_iterations, "subspace_iterations": r.subspace_iterations}


def ctm_get_spectrum(h, m: int) -> np.ndarray:
    om = np.zeros(m)
    _check(lib.ctm_get_spectrum(h, _dptr(om)))
    return om


def ctm_get_state(h, m: int, q: int):
    P = np.zeros((m, m * q), order="F")
    om = np.zeros(m)
    live = ctypes.c_int(0)
    _check(lib.ctm_get_state(h, _dptr(P), _dptr(om), ctypes.byref(live)))
    return P, om, live.value


def ctm_set_state(h, P: np.ndarray, omega: np.ndarray, live: int):
    P = np.asfortranarray(P, dtype=np.float64)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    _check(lib.ctm_set_state(h, _dptr(P), _dptr(om), int(live)))


def ctm_save(h) -> bytes:
    n = ctypes.c_size_t(0)
    _check(lib.ctm_save(h, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib.ctm_save(h, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def ctm_load(h, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib.ctm_load(h, buf, len(blob)))


def ctm_extend(h):
    _check(lib.ctm_extend(h))


def ctm_get_ctilde(h, rows, cols) -> np.ndarray:
    r = np.ascontiguousarray(rows, dtype=np.int32)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros(len(r))
    _check(lib.ctm_get_ctilde(h, r.ctypes.data_as(_ip), c.ctypes.data_as(_ip), len(r), _dptr(out)))
    return out


def ctm_eigen(h, N: int, b: int, want_vectors: bool = True):
    ev = np.zeros(b)
    vec = np.zeros((N, b), order="F") if want_vectors else None
    bo = ctypes.c_int(0)
    st = _check(lib.ctm_eigen(h, _dptr(ev), _dptr(vec) if want_vectors else None, ctypes.byref(bo)),
                (CTM_OK, CTM_ENOTCONVERGED))
    return ev, vec, st


def ctm_profile(h, enable: bool):
    _check(lib.ctm_profile(h, 1 if enable else 0))


def ctm_profile_read(h) -> dict:
    arr = (ctm_prof_entry * 16)()
    n = ctypes.c_int(0)
    _check(lib.ctm_profile_read(h, arr, 16, ctypes.byref(n)))
    return {arr[i].name.decode(): {"launches": arr[i].launches, "ms": arr[i].ms, "flops": arr[i].flops,
                                   "bytes": arr[i].bytes} for i in range(n.value)}


def ctm_launch_count(h) -> int:
    n = ctypes.c_longlong(0)
    _check(lib.ctm_launch_count(h, ctypes.byref(n)))
    return n.value


def ctm_tune(h, reps: int = 5) -> list:
    arr = (ctm_tune_entry * 8)()
    n = ctypes.c_int(0)
    _check(lib.ctm_tune(h, int(reps), arr, 8, ctypes.byref(n)))
    return [arr[i].to_dict() for i in range(n.value)]


def ctm_tc_plan_set(prec: str, M: int, N: int, K: int, bn: int, splits: int):
    _check(lib.ctm_tc_plan_set(PRECISIONS[prec], int(M), int(N), int(K), int(bn), int(splits)))


def ctm_tc_plan_get(prec: str, M: int, N: int, K: int) -> tuple:
    bn, sp = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib.ctm_tc_plan_get(PRECISIONS[prec], int(M), int(N), int(K), ctypes.byref(bn), ctypes.byref(sp)))
    return bn.value, sp.value


def ctm_scan_workspace_size(cfg: ctm_config, nbeta: int) -> int:
    n = ctypes.c_size_t(0)
    _check(lib.ctm_scan_workspace_size(ctypes.byref(cfg), int(nbeta), ctypes.byref(n)))
    return n.value


def ctm_scan_init(cfg: ctm_config, betas, workers: int, stream: int = 0):
    b = np.ascontiguousarray(betas, dtype=np.float64)
    s = ctypes.c_void_p()
    _check(lib.ctm_scan_init(ctypes.byref(s), ctypes.byref(cfg), len(b), _dptr(b), int(workers),
                             ctypes.c_void_p(stream)))
    return s


def ctm_scan_tune(s, reps: int = 5) -> list:
    arr = (ctm_tune_entry * 8)()
    n = ctypes.c_int(0)
    _check(lib.ctm_scan_tune(s, int(reps), arr, 8, ctypes.byref(n)))
    return [arr[i].to_dict() for i in range(n.value)]


def ctm_scan_run(s, nbeta: int, max_steps: int):
    done = np.zeros(nbeta, dtype=np.int32)
    conv = np.zeros(nbeta, dtype=np.int32)
    st = _check(lib.ctm_scan_run(s, int(max_steps), done.ctypes.data_as(_ip), conv.ctypes.data_as(_ip)),
                (CTM_OK, CTM_ENOTCONVERGED))
    return done, conv, st


def ctm_scan_observables(s, nbeta: int):
    arr = (ctm_obs * nbeta)()
    st = _check(lib.ctm_scan_observables(s, arr), (CTM_OK, CTM_ENOTCONVERGED))
    return [arr[i].to_dict() for i in range(nbeta)], st


def ctm_scan_handle(s, ibeta: int):
    h = ctypes.c_void_p()
    _check(lib.ctm_scan_handle(s, int(ibeta), ctypes.byref(h)))
    return h


def ctm_scan_get_spectrum(s, ibeta: int, m: int) -> np.ndarray:
    om = np.zeros(m)
    _check(lib.ctm_scan_get_spectrum(s, int(ibeta), _dptr(om)))
    return om


def ctm_scan_destroy(s):
    if s:
        lib.ctm_scan_destroy(s)


def ctm_symeig_workspace_size(n: int) -> int:
    b = ctypes.c_size_t(0)
    _check(lib.ctm_symeig_workspace_size(int(n), ctypes.byref(b)))
    return b.value


def ctm_symeig(A, max_sweeps: int = 0):
    """Eigenpairs of a symmetric FP64 torch CUDA tensor A (n x n) with the
    library's Jacobi solver; the workspace comes from torch.  Returns
    (evals, vecs, status) as torch tensors, sorted by |eigenvalue| desc."""
    import torch
    n = A.shape[0]
    Ac = A.t().contiguous()  # column-major storage of A
    ev = torch.empty(n, dtype=torch.float64, device=A.device)
    vt = torch.empty(n, n, dtype=torch.float64, device=A.device)  # rows of vt = columns of vecs
    ws = torch.empty(ctm_symeig_workspace_size(n), dtype=torch.uint8, device=A.device)
    st = torch.cuda.current_stream(A.device).cuda_stream
    status = _check(lib.ctm_symeig(n, Ac.data_ptr(), n, ev.data_ptr(), vt.data_ptr(), n, int(max_sweeps),
                                   ws.data_ptr(), ws.numel(), ctypes.c_void_p(st)), (CTM_OK, CTM_ENOTCONVERGED))
    return ev, vt.t(), status


def ctm_symeig_noalloc(A, max_sweeps: int = 0):
    """ctm_symeig through the no-allocation entry point: the library's
    scratch is its own static device array; the caller passes A (torch FP64
    CUDA tensor, n <= CTM_SYMEIG_NOALLOC_MAX_N) and receives the outputs in
    tensors allocated here."""
    import torch
    n = A.shape[0]
    Ac = A.t().contiguous()
    ev = torch.empty(n, dtype=torch.float64, device=A.device)
    vt = torch.empty(n, n, dtype=torch.float64, device=A.device)
    # the library picks its static scratch by the current device: make A's current
    with torch.cuda.device(A.device):
        st = torch.cuda.current_stream(A.device).cuda_stream
        status = _check(lib.ctm_symeig_noalloc(n, Ac.data_ptr(), n, ev.data_ptr(), vt.data_ptr(), n,
                                               int(max_sweeps), ctypes.c_void_p(st)), (CTM_OK, CTM_ENOTCONVERGED))
    return ev, vt.t(), status


def ctm_contract(A, B, prec: str = "fp64", ozaki_slices: int = 0):
    """D = A^t B for FP64 torch CUDA tensors A (K x M) and B (K x N) through
    the library's contraction kernel in the given precision."""
    import torch
    K, M = A.shape
    K2, N = B.shape
    assert K == K2
    p = PRECISIONS[prec]
    Ac = A.t().contiguous()  # column-major K x M
    Bc = B.t().contiguous()
    Dt = torch.empty(N, M, dtype=torch.float64, device=A.device)  # column-major M x N
    nb = ctypes.c_size_t(0)
    _check(lib.ctm_contract_workspace_size(p, int(ozaki_slices), M, N, K, ctypes.byref(nb)))
    ws = torch.empty(nb.value, dtype=torch.uint8, device=A.device)
    st = torch.cuda.current_stream(A.device).cuda_stream
    _check(lib.ctm_contract(p, int(ozaki_slices), M, N, K, Ac.data_ptr(), K, Bc.data_ptr(), K, Dt.data_ptr(), M,
                            ws.data_ptr(), ws.numel(), ctypes.c_void_p(st)))
    return Dt.t()


def ctm_destroy(h):
    if h:
        lib.ctm_destroy(h)


class CTMRG:
    """One CTMRG run on the GPU: owns a handle and its torch-allocated workspace."""

    def __init__(self, spins, m: int, beta: float, boundary_spin: int = 0, prec: str = "fp64",
                 device: str = "cuda:0", **kw):
        import torch
        self.device = torch.device(device)
        self.cfg, self._spins = make_config(spins, m, beta, boundary_spin, prec, **kw)
        self.m, self.q = m, self._spins.shape[0]
        self.N = m * self.q
        nbytes = ctm_workspace_size(self.cfg)
        self._ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.cfg.workspace = ctypes.c_void_p(self._ws.data_ptr())
        self.cfg.workspace_bytes = nbytes
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
            self.h = ctm_init(self.cfg, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            ctm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        done, info, st = ctm_step(self.h, n)
        return done, info.to_dict(), st

    def run(self, max_steps: int):
        done, info, st = ctm_step(self.h, max_steps)
        return done, info.to_dict()

    def observables(self) -> dict:
        o, st = ctm_observables(self.h)
        return o.to_dict()

    def spectrum(self) -> np.ndarray:
        return ctm_get_spectrum(self.h, self.m)

    def xi(self, max_iters: int = 0, tol: float = 0.0) -> dict:
        """Effective correlation length and the leading eigenvalues of the
        row-to-row transfer matrix of the current state."""
        return ctm_xi(self.h, max_iters, tol)[0]

    def get_state(self):
        return ctm_get_state(self.h, self.m, self.q)

    def set_state(self, P, omega, live: int):
        ctm_set_state(self.h, P, omega, live)

    def tangent_step(self, P_dot, omega_dot, source: bool = True) -> dict:
        return ctm_tangent_step(self.h, self.m, self.q, P_dot, omega_dot, source)

    def df_dbeta(self) -> float:
        """d f / d beta of the converged fixed point by implicit
        differentiation on the device (ctm_step_backward with grad f = 1)."""
        go = ctm_obs()
        go.f = 1.0
        return ctm_step_backward(self.h, go)

    def extend(self):
        ctm_extend(self.h)

    def ctilde(self, rows, cols):
        return ctm_get_ctilde(self.h, rows, cols)

    def eigen(self, want_vectors=True):
        b = min(self.N, self.m + (self.cfg.block_extra if self.cfg.block_extra > 0 else max(8, self.m // 8)))
        return ctm_eigen(self.h, self.N, b, want_vectors)

    def profile(self, enable: bool):
        ctm_profile(self.h, enable)

    def profile_read(self) -> dict:
        return ctm_profile_read(self.h)

    def launch_count(self) -> int:
        return ctm_launch_count(self.h)

    def save(self) -> bytes:
        return ctm_save(self.h)

    def load(self, blob: bytes):
        ctm_load(self.h, blob)


class Scan:
    """A temperature scan on the GPU: one handle per beta inside the library,
    stepped concurrently by its native worker pool; the workspaces come from
    torch."""

    def __init__(self, spins, m: int, betas, workers: int = 8, boundary_spin: int = 0, prec: str = "fp64",
                 device: str = "cuda:0", **kw):
        import torch
        self.device = torch.device(device)
        self.betas = np.ascontiguousarray(betas, dtype=np.float64)
        self.nbeta = len(self.betas)
        self.cfg, self._spins = make_config(spins, m, 0.0, boundary_spin, prec, **kw)
        self.m, self.q = m, self._spins.shape[0]
        nbytes = ctm_scan_workspace_size(self.cfg, self.nbeta)
        self._ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.cfg.workspace = ctypes.c_void_p(self._ws.data_ptr())
        self.cfg.workspace_bytes = nbytes
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device)
            self.s = ctm_scan_init(self.cfg, self.betas, workers, stream.cuda_stream)

    def close(self):
        if getattr(self, "s", None):
            ctm_scan_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tune(self, reps: int = 5) -> list:
        return ctm_scan_tune(self.s, reps)

    def run(self, max_steps: int):
        """Step every beta until it converges or takes max_steps steps;
        returns (steps per beta, converged flags)."""
        done, conv, st = ctm_scan_run(self.s, self.nbeta, max_steps)
        return done, conv

    def observables(self) -> list:
        obs, st = ctm_scan_observables(self.s, self.nbeta)
        return obs

    def spectrum(self, ibeta: int) -> np.ndarray:
        return ctm_scan_get_spectrum(self.s, ibeta, self.m)

    def launch_count(self) -> int:
        return sum(ctm_launch_count(ctm_scan_handle(self.s, i)) for i in range(self.nbeta))
