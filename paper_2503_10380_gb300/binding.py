"""ctypes binding of libpplcpd.so (include/ppl_cpd.h), same names as the C ABI.

Only argument marshalling lives here: every step of the CP-ALS path runs in
the library's CUDA kernels.  PyTorch provides device memory and the stream.
If the library is missing this module raises: there is no fallback.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_size_t, c_void_p

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpplcpd.so")

PPL_OK, PPL_EINVAL, PPL_ENOMEM, PPL_ECUDA, PPL_ETIMEOUT, PPL_ENOTREADY = range(6)
PREC = {"fp64": 0, "bf16x3": 1, "tf32": 2, "tf32x3": 3}
STOP = {"fixed": 0, "dfit": 1, "eta": 2}
GUESS = {"optimal": 0, "near_optimal": 1, "random": 2}
MODE = {"a": 0, "b": 1, "i": 2, "j": 3}
STATUS_NAMES = {0: "PPL_OK", 1: "PPL_EINVAL", 2: "PPL_ENOMEM", 3: "PPL_ECUDA", 4: "PPL_ETIMEOUT",
                5: "PPL_ENOTREADY"}


class ppl_cpd_opts(ctypes.Structure):
    _fields_ = [("precision", c_int), ("r_chunk", c_int), ("use_graph", c_int), ("want_eta", c_int),
                ("profile", c_int), ("dressed", c_int), ("acc_chunk", c_int), ("acc_steps", c_int),
                ("wait_limit_us", c_int), ("acc_steps_p", c_int), ("init", c_int), ("init_seed", c_int),
                ("reserved", c_int * 4)]


class ppl_cpd_stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_longlong), ("clamped_pivots", ctypes.c_longlong),
                ("timeouts", ctypes.c_longlong), ("last_fit", c_double), ("last_eta", c_double),
                ("last_inner", c_double), ("last_norm2", c_double), ("flops_per_sweep", c_double),
                ("kernels_per_sweep", ctypes.c_longlong)]


class PplError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """Load libpplcpd.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run `python -c \"import __graft_entry__ as g; g.build()\"`")
    L = ctypes.CDLL(LIB_PATH)
    H = c_void_p
    L.ppl_cpd_default_opts.argtypes = [POINTER(ppl_cpd_opts)]
    L.ppl_cpd_default_opts.restype = None
    L.ppl_cpd_workspace_size.argtypes = [c_int, c_int, c_int, c_int, POINTER(ppl_cpd_opts), POINTER(c_size_t)]
    L.ppl_cpd_init.argtypes = [POINTER(H), c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_size_t, POINTER(ppl_cpd_opts), c_void_p]
    L.ppl_cpd_mttkrp.argtypes = [H, c_int, c_void_p]
    L.ppl_cpd_sweep.argtypes = [H, c_int, POINTER(c_double)]
    L.ppl_cpd_set_normR2.argtypes = [H, c_double]
    L.ppl_cpd_fit.argtypes = [H, POINTER(c_double)]
    L.ppl_cpd_energy.argtypes = [H, POINTER(c_double)]
    L.ppl_exact_contract.argtypes = [H, POINTER(c_double), POINTER(c_double), c_void_p]
    L.ppl_cpd_set_tau.argtypes = [H, c_void_p]
    L.ppl_cpd_stats_get.argtypes = [H, POINTER(ppl_cpd_stats)]
    L.ppl_cpd_phase_ms.argtypes = [H, POINTER(c_double)]
    L.ppl_cpd_factors_changed.argtypes = [H]
    L.ppl_cpd_set_guess_policy.argtypes = [H, c_int]
    L.ppl_cpd_reconstruct.argtypes = [H, c_void_p, c_int]
    L.ppl_cpd_set_t1.argtypes = [H, c_void_p]
    L.ppl_exact_contract_mixed.argtypes = [H, POINTER(c_double), POINTER(c_double), c_void_p]
    L.ppl_cpd_autotune.argtypes = [H, POINTER(c_int)]
    L.ppl_cpd_batch_create.argtypes = [POINTER(c_void_p), c_int, POINTER(c_void_p), c_int, c_void_p]
    L.ppl_cpd_batch_sweep.argtypes = [c_void_p, c_int, POINTER(c_double)]
    L.ppl_cpd_batch_destroy.argtypes = [c_void_p]
    L.ppl_cpd_batch_kernels.argtypes = [c_void_p, POINTER(ctypes.c_longlong)]
    L.ppl_cpd_solve.argtypes = [H, c_int, c_int, c_double, POINTER(c_int), POINTER(c_double), POINTER(c_double)]
    L.ppl_last_error.argtypes = [H]
    L.ppl_last_error.restype = c_char_p
    L.ppl_cpd_destroy.argtypes = [H]
    L.ppl_tc_gemm_workspace_size.argtypes = [c_int, c_int, c_int, c_int, POINTER(c_size_t)]
    L.ppl_tc_gemm.argtypes = [c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                              c_void_p]
    L.ppl_cp_energy_static.argtypes = [c_int, c_int, c_int, c_int, c_void_p, c_void_p, POINTER(c_double),
                                       c_void_p]
    L.ppl_cp_energy_static.restype = c_int
    L.ppl_cpd_inject_wait_timeout.argtypes = [H]
    L.ppl_probe_fp64_peak.argtypes = [POINTER(c_double), c_void_p]
    L.ppl_test_reciprocal.argtypes = [c_void_p, c_void_p, c_int, c_void_p]
    for name in ("ppl_cpd_workspace_size", "ppl_cpd_init", "ppl_cpd_mttkrp", "ppl_cpd_sweep",
                 "ppl_cpd_set_normR2", "ppl_cpd_fit", "ppl_cpd_energy", "ppl_exact_contract",
                 "ppl_cpd_set_tau", "ppl_cpd_stats_get", "ppl_cpd_destroy", "ppl_cpd_phase_ms", "ppl_cpd_factors_changed",
                 "ppl_cpd_set_guess_policy", "ppl_cpd_solve", "ppl_cpd_reconstruct", "ppl_cpd_autotune",
                 "ppl_cpd_set_t1", "ppl_exact_contract_mixed",
                 "ppl_cpd_batch_create", "ppl_cpd_batch_sweep", "ppl_cpd_batch_destroy", "ppl_cpd_batch_kernels",
                 "ppl_tc_gemm_workspace_size", "ppl_tc_gemm", "ppl_cpd_inject_wait_timeout",
                 "ppl_probe_fp64_peak", "ppl_test_reciprocal"):
        getattr(L, name).restype = c_int
    _lib = L
    return L


def _check(rc: int, h=None):
    if rc != PPL_OK:
        msg = lib().ppl_last_error(h)
        raise PplError(rc, msg.decode() if msg else "")


INIT = {"user": 0, "normal": 1, "uniform": 2}


def make_opts(precision="tf32x3", r_chunk=0, use_graph=True, want_eta=False, profile=False,
              dressed=False, acc_chunk=0, acc_steps=0, wait_limit_us=0, acc_steps_p=0,
              init="user", init_seed=0) -> ppl_cpd_opts:
    o = ppl_cpd_opts()
    lib().ppl_cpd_default_opts(ctypes.byref(o))
    o.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    o.r_chunk = int(r_chunk)
    o.use_graph = int(bool(use_graph))
    o.want_eta = int(bool(want_eta))
    o.profile = int(bool(profile))
    o.dressed = int(bool(dressed))
    o.acc_chunk = int(acc_chunk)
    o.acc_steps = int(acc_steps)
    o.wait_limit_us = int(wait_limit_us)
    o.acc_steps_p = int(acc_steps_p)
    o.init = INIT[init] if isinstance(init, str) else int(init)
    o.init_seed = ctypes.c_int(int(init_seed) & 0xFFFFFFFF).value
    return o


# ---- thin wrappers, one per C entry point ------------------------------------

def ppl_cpd_workspace_size(o, v, X, R, opts: ppl_cpd_opts) -> int:
    n = c_size_t(0)
    _check(lib().ppl_cpd_workspace_size(o, v, X, R, ctypes.byref(opts), ctypes.byref(n)))
    return n.value


def ppl_cpd_init(o, v, X, R, B_ptr, tau_ptr, factors_ptr, ws_ptr, ws_bytes, opts, stream_ptr) -> c_void_p:
    h = c_void_p()
    _check(lib().ppl_cpd_init(ctypes.byref(h), o, v, X, R, B_ptr, tau_ptr, factors_ptr, ws_ptr, ws_bytes,
                              ctypes.byref(opts), stream_ptr))
    return h


def ppl_cpd_mttkrp(h, mode: int, M_ptr):
    _check(lib().ppl_cpd_mttkrp(h, mode, M_ptr), h)


def ppl_cpd_sweep(h, nsweeps: int, want_hist: bool = True):
    buf = (c_double * max(nsweeps, 1))() if want_hist else None
    _check(lib().ppl_cpd_sweep(h, nsweeps, buf), h)
    return list(buf)[:nsweeps] if want_hist else None


def ppl_cpd_set_normR2(h, normR2: float):
    _check(lib().ppl_cpd_set_normR2(h, float(normR2)), h)


def ppl_cpd_fit(h) -> float:
    x = c_double()
    _check(lib().ppl_cpd_fit(h, ctypes.byref(x)), h)
    return x.value


def ppl_cpd_energy(h) -> float:
    x = c_double()
    _check(lib().ppl_cpd_energy(h, ctypes.byref(x)), h)
    return x.value


def ppl_exact_contract(h, R_ptr=None):
    n2, E = c_double(), c_double()
    _check(lib().ppl_exact_contract(h, ctypes.byref(n2), ctypes.byref(E), R_ptr), h)
    return n2.value, E.value


def ppl_exact_contract_mixed(h, R_ptr=None):
    n2, E = c_double(), c_double()
    _check(lib().ppl_exact_contract_mixed(h, ctypes.byref(n2), ctypes.byref(E), R_ptr), h)
    return n2.value, E.value


def ppl_cpd_set_tau(h, tau_ptr):
    _check(lib().ppl_cpd_set_tau(h, tau_ptr), h)


def ppl_cpd_factors_changed(h):
    _check(lib().ppl_cpd_factors_changed(h), h)


def ppl_cpd_set_t1(h, t1_ptr):
    _check(lib().ppl_cpd_set_t1(h, t1_ptr), h)


def ppl_cpd_reconstruct(h, R_ptr, symmetrise: bool):
    _check(lib().ppl_cpd_reconstruct(h, R_ptr, int(bool(symmetrise))), h)


def ppl_cpd_autotune(h) -> int:
    rc = c_int(0)
    _check(lib().ppl_cpd_autotune(h, ctypes.byref(rc)), h)
    return rc.value


def ppl_cpd_batch_create(handles, nstreams, stream_ptr):
    arr = (c_void_p * len(handles))(*[h.value if isinstance(h, c_void_p) else h for h in handles])
    b = c_void_p()
    _check(lib().ppl_cpd_batch_create(ctypes.byref(b), len(handles), arr, nstreams, stream_ptr))
    return b


def ppl_cpd_batch_sweep(b, nsweeps, n_instances, want_fits=True):
    buf = (c_double * (max(nsweeps, 1) * n_instances))() if want_fits else None
    _check(lib().ppl_cpd_batch_sweep(b, nsweeps, buf))
    if not want_fits:
        return None
    return [list(buf)[k * n_instances:(k + 1) * n_instances] for k in range(nsweeps)]


def ppl_cpd_batch_destroy(b):
    _check(lib().ppl_cpd_batch_destroy(b))


class Batch:
    """Several CpAls problems swept together from one CUDA graph."""

    def __init__(self, problems, nstreams=8):
        import torch
        self.problems = list(problems)
        self.b = ppl_cpd_batch_create([p.h for p in self.problems], nstreams,
                                      torch.cuda.current_stream().cuda_stream)

    def sweep(self, n=1, want_fits=True):
        return ppl_cpd_batch_sweep(self.b, n, len(self.problems), want_fits)

    def kernels_per_sweep(self) -> int:
        n = ctypes.c_longlong(0)
        _check(lib().ppl_cpd_batch_kernels(self.b, ctypes.byref(n)))
        return n.value

    def close(self):
        if self.b:
            ppl_cpd_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ppl_cpd_set_guess_policy(h, policy):
    _check(lib().ppl_cpd_set_guess_policy(h, GUESS[policy] if isinstance(policy, str) else int(policy)), h)


def ppl_cpd_solve(h, max_sweeps: int, rule="fixed", eps: float = 0.0):
    n = c_int(0)
    fits = (c_double * max_sweeps)()
    etas = (c_double * max_sweeps)()
    _check(lib().ppl_cpd_solve(h, max_sweeps, STOP[rule] if isinstance(rule, str) else int(rule), float(eps),
                               ctypes.byref(n), fits, etas), h)
    return n.value, list(fits)[:n.value], list(etas)[:n.value]


def ppl_cpd_stats_get(h) -> dict:
    s = ppl_cpd_stats()
    _check(lib().ppl_cpd_stats_get(h, ctypes.byref(s)), h)
    return {k: getattr(s, k) for k, _ in ppl_cpd_stats._fields_}


PHASES = ("tau_r", "chain_a", "solve_a", "chain_b", "solve_b", "s_and_p", "solve_ij", "fit")


def ppl_cpd_phase_ms(h) -> dict:
    buf = (c_double * 8)()
    _check(lib().ppl_cpd_phase_ms(h, buf), h)
    return dict(zip(PHASES, list(buf)))


def ppl_cpd_inject_wait_timeout(h):
    _check(lib().ppl_cpd_inject_wait_timeout(h), h)


def ppl_probe_fp64_peak(stream_ptr=None) -> float:
    x = c_double()
    _check(lib().ppl_probe_fp64_peak(ctypes.byref(x), stream_ptr))
    return x.value


def ppl_cpd_destroy(h):
    _check(lib().ppl_cpd_destroy(h))


def ppl_cp_energy_static(o, v, X, R, B_ptr, factors_ptr, stream_ptr) -> float:
    """CP energy without any device allocation (scratch is a static array in
    the library); see include/ppl_cpd.h for the size limit and the sharing rules."""
    E = c_double()
    _check(lib().ppl_cp_energy_static(o, v, X, R, B_ptr, factors_ptr, ctypes.byref(E), stream_ptr))
    return E.value


def ppl_tc_gemm_workspace_size(M, N, K, precision) -> int:
    n = c_size_t(0)
    _check(lib().ppl_tc_gemm_workspace_size(M, N, K, precision, ctypes.byref(n)))
    return n.value


def ppl_tc_gemm(precision, M, N, K, A_ptr, B_ptr, C_ptr, ws_ptr, ws_bytes, stream_ptr):
    _check(lib().ppl_tc_gemm(precision, M, N, K, A_ptr, B_ptr, C_ptr, ws_ptr, ws_bytes, stream_ptr))


# ---- torch-facing convenience object ------------------------------------------

class CpAls:
    """One CP-ALS problem on the current CUDA device.

    B [X][o+v][o+v] and tau [o][o][v][v] are FP64 device tensors (kept alive
    here); `factors` is a dict of initial guesses "a","b" [v][R] and "i","j"
    [o][R] (numpy or torch), or, with init="normal" or "uniform", the rank R
    as an int (the library then draws the guess on the device from init_seed).
    torch allocates the factor buffer and the workspace; the library does the
    rest.
    """

    def __init__(self, B, tau, factors, precision="tf32x3", r_chunk=0, use_graph=True, want_eta=False,
                 profile=False, dressed=False, stream=None, acc_chunk=0, acc_steps=0, wait_limit_us=0,
                 acc_steps_p=0, init="user", init_seed=0):
        import torch
        self.torch = torch
        X, n, _ = B.shape
        o = tau.shape[0]
        v = tau.shape[2]
        R = int(factors) if isinstance(factors, int) else factors["a"].shape[1]
        assert n == o + v and B.dtype == torch.float64 and tau.dtype == torch.float64 and B.is_cuda
        self.o, self.v, self.X, self.R = o, v, X, R
        self.B = B.contiguous()
        self.tau = tau.contiguous()
        dev = B.device
        if isinstance(factors, int):
            self.fac = torch.zeros((2 * v + 2 * o + 1) * R, dtype=torch.float64, device=dev)
        else:
            parts = [torch.as_tensor(factors[m], dtype=torch.float64).reshape(-1) for m in ("a", "b", "i", "j")]
            parts.append(torch.ones(R, dtype=torch.float64))
            self.fac = torch.cat(parts).to(dev)
        self.opts = make_opts(precision, r_chunk, use_graph, want_eta, profile, dressed, acc_chunk, acc_steps,
                              wait_limit_us, acc_steps_p, init, init_seed)
        self.ws_bytes = ppl_cpd_workspace_size(o, v, X, R, self.opts)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.h = ppl_cpd_init(o, v, X, R, self.B.data_ptr(), self.tau.data_ptr(), self.fac.data_ptr(),
                              self.ws.data_ptr(), self.ws_bytes, self.opts, self.stream.cuda_stream)

    def factors(self) -> dict:
        o, v, R = self.o, self.v, self.R
        f = self.fac
        out, pos = {}, 0
        for m, dim in (("a", v), ("b", v), ("i", o), ("j", o)):
            out[m] = f[pos:pos + dim * R].view(dim, R)
            pos += dim * R
        out["lam"] = f[pos:pos + R]
        return out

    def mttkrp(self, mode: str):
        dim = self.v if mode in "ab" else self.o
        M = self.torch.empty((dim, self.R), dtype=self.torch.float64, device=self.B.device)
        ppl_cpd_mttkrp(self.h, MODE[mode], M.data_ptr())
        return M

    def sweep(self, n: int = 1, want_hist: bool = True):
        return ppl_cpd_sweep(self.h, n, want_hist)

    def set_normR2(self, x: float):
        ppl_cpd_set_normR2(self.h, x)

    def fit(self) -> float:
        return ppl_cpd_fit(self.h)

    def energy(self) -> float:
        return ppl_cpd_energy(self.h)

    def exact_contract(self, want_R: bool = False, mixed: bool = False):
        """||R||^2, E_exact (and R): FP64, or with mixed=True on the tensor cores."""
        Rt = None
        if want_R:
            Rt = self.torch.empty((self.v, self.v, self.o, self.o), dtype=self.torch.float64, device=self.B.device)
        fn = ppl_exact_contract_mixed if mixed else ppl_exact_contract
        n2, E = fn(self.h, Rt.data_ptr() if Rt is not None else None)
        return n2, E, Rt

    def set_t1(self, t1):
        """Dress the b side with t1 [o][v] (FP64 device tensor), or undress with None."""
        self.t1 = None if t1 is None else t1.contiguous()
        ppl_cpd_set_t1(self.h, None if self.t1 is None else self.t1.data_ptr())

    def set_tau(self, tau):
        self.tau = tau.contiguous()
        ppl_cpd_set_tau(self.h, self.tau.data_ptr())

    def set_factors(self, factors: dict):
        """Write a new guess into the factor buffer and tell the library."""
        f = self.factors()
        for m in ("a", "b", "i", "j"):
            f[m].copy_(self.torch.as_tensor(factors[m], dtype=self.torch.float64))
        ppl_cpd_factors_changed(self.h)

    def solve(self, max_sweeps: int, rule="fixed", eps: float = 0.0):
        """One CPD under a stopping rule; returns (sweeps, fit history, eta history)."""
        return ppl_cpd_solve(self.h, max_sweeps, rule, eps)

    def reconstruct(self, symmetrise: bool = False):
        """R~ (or its symmetrised form) as a [v][v][o][o] FP64 device tensor."""
        out = self.torch.empty((self.v, self.v, self.o, self.o), dtype=self.torch.float64, device=self.B.device)
        ppl_cpd_reconstruct(self.h, out.data_ptr(), symmetrise)
        return out

    def autotune(self) -> int:
        """Time candidate r-chunk sizes and keep the fastest; returns it."""
        return ppl_cpd_autotune(self.h)

    def set_guess_policy(self, policy):
        ppl_cpd_set_guess_policy(self.h, policy)

    def stats(self) -> dict:
        return ppl_cpd_stats_get(self.h)

    def phase_ms(self) -> dict:
        return ppl_cpd_phase_ms(self.h)

    def close(self):
        if self.h:
            ppl_cpd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_gemm(A, B, precision="bf16x3"):
    """C = A @ B^T for FP32 CUDA tensors through the tensor-core kernel."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    prec = PREC[precision]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    nbytes = ppl_tc_gemm_workspace_size(M, N, K, prec)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=A.device)
    ppl_tc_gemm(prec, M, N, K, A.contiguous().data_ptr(), B.contiguous().data_ptr(), C.data_ptr(),
                ws.data_ptr(), nbytes, torch.cuda.current_stream(A.device).cuda_stream)
    return C
