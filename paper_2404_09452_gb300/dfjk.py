"""Thin Python binding of libdfjk.so (the C ABI in include/dfjk.h).

Argument marshalling only: every step of the DF-J/K path runs in the CUDA
library.  PyTorch supplies device memory and streams.  There is no fallback:
if the library cannot be loaded or no CUDA device is present, calls raise.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdfjk.so")

DFJK_FP64 = 0
DFJK_MIXED = 1

STATUS = {
    0: "DFJK_OK",
    1: "DFJK_ERR_ARG",
    2: "DFJK_ERR_UNSUPPORTED",
    3: "DFJK_ERR_NOT_PD",
    4: "DFJK_ERR_OOM",
    5: "DFJK_ERR_BUDGET",
    6: "DFJK_ERR_TIMEOUT",
    7: "DFJK_ERR_CUDA",
    8: "DFJK_ERR_STATE",
}

# Every symbol include/dfjk.h declares.
EXPORTS = [
    "dfjk_default_options",
    "dfjk_setup",
    "dfjk_query",
    "dfjk_query_precision",
    "dfjk_query_setup",
    "dfjk_query_build",
    "dfjk_query_pair_classes",
    "dfjk_query_tuning",
    "dfjk_estimate_bytes",
    "dfjk_build",
    "dfjk_build_uks",
    "dfjk_build_density",
    "dfjk_coulomb_gradient",
    "dfjk_jk_gradient",
    "dfjk_build_batch",
    "dfjk_overlap",
    "dfjk_overlap_matrix",
    "dfjk_evict",
    "dfjk_destroy",
    "dfjk_status_string",
    "dfjk_last_error",
    "dfjk_launch_count",
    "dfjk_fma_rate",
    "dfjk_boys",
    "dfjk_get_metric",
    "dfjk_get_cholesky",
    "dfjk_get_B",
    "dfjk_get_pair_mask",
    "dfjk_get_B_columns",
    "dfjk_get_three_center",
    "dfjk_debug_sliced_gemm",
    "dfjk_set_timing",
    "dfjk_phase_times",
    "dfjk_energies_noalloc",
    "dfjk_trim_cache",
]

PHASES = ["pairs+metric", "cholesky", "eri3c", "whiten", "X=BC", "K", "rho+J", "energies",
          "tc:whiten", "tc:X=BC", "tc:K", "eri3c32", "setup", "build"]


class DfjkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Shell(ctypes.Structure):
    _fields_ = [
        ("atom", ctypes.c_int32),
        ("l", ctypes.c_int32),
        ("nprim", ctypes.c_int32),
        ("exps", ctypes.POINTER(ctypes.c_double)),
        ("coefs", ctypes.POINTER(ctypes.c_double)),
    ]


class BasisC(ctypes.Structure):
    _fields_ = [("nshell", ctypes.c_int32), ("shells", ctypes.POINTER(Shell))]


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("schwarz_thresh", ctypes.c_double),
        ("hbm_budget_bytes", ctypes.c_size_t),
        ("timeout_iters", ctypes.c_int64),
        ("energies_on_host", ctypes.c_int32),
        ("fp32_pair_thresh", ctypes.c_double),
        ("b_on_host", ctypes.c_int32),
        ("tune_table", ctypes.c_char_p),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libdfjk.so and declares the signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(
            f"{path} is missing: build it with paper_2404_09452_gb300/build_lib.py "
            "(there is no CPU fallback)"
        )
    lib = ctypes.CDLL(path)
    vp, i32, f64p = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)
    lib.dfjk_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.dfjk_default_options.restype = None
    lib.dfjk_setup.argtypes = [
        ctypes.POINTER(BasisC), ctypes.POINTER(BasisC), i32, f64p, ctypes.POINTER(Options), vp,
        ctypes.POINTER(vp),
    ]
    lib.dfjk_query.argtypes = [
        vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_size_t)
    ]
    lib.dfjk_build.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp]
    szp = ctypes.POINTER(ctypes.c_size_t)
    lib.dfjk_estimate_bytes.argtypes = [i32, i32, i32, i32, szp, szp, szp]
    lib.dfjk_get_B_columns.argtypes = [vp, i32, vp, vp, vp, vp]
    lib.dfjk_query_pair_classes.argtypes = [vp, vp, vp]
    lib.dfjk_fma_rate.argtypes = [i32, vp, vp]
    lib.dfjk_query_tuning.argtypes = [vp, vp]
    lib.dfjk_query_build.argtypes = [vp, vp, vp]
    lib.dfjk_overlap.argtypes = [vp, vp, vp]
    lib.dfjk_coulomb_gradient.argtypes = [vp, vp, vp, vp]
    lib.dfjk_jk_gradient.argtypes = [vp, i32, vp, ctypes.c_double, ctypes.c_double, vp, vp]
    lib.dfjk_overlap_matrix.argtypes = [ctypes.POINTER(BasisC), i32, f64p, vp, vp]
    lib.dfjk_build_batch.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, i32, vp]
    lib.dfjk_evict.argtypes = [vp]
    lib.dfjk_destroy.argtypes = [vp]
    lib.dfjk_status_string.argtypes = [ctypes.c_int]
    lib.dfjk_status_string.restype = ctypes.c_char_p
    lib.dfjk_last_error.argtypes = []
    lib.dfjk_last_error.restype = ctypes.c_char_p
    lib.dfjk_launch_count.argtypes = []
    lib.dfjk_launch_count.restype = ctypes.c_uint64
    lib.dfjk_boys.argtypes = [i32, i32, vp, vp, vp]
    for fn in ("dfjk_get_metric", "dfjk_get_cholesky", "dfjk_get_B", "dfjk_get_pair_mask",
               "dfjk_get_three_center"):
        getattr(lib, fn).argtypes = [vp, vp, vp]
    lib.dfjk_debug_sliced_gemm.argtypes = [i32, i32, i32, i32, i32, vp, vp, vp, vp, vp]
    lib.dfjk_energies_noalloc.argtypes = [i32, vp, vp, vp, vp, vp]
    lib.dfjk_set_timing.argtypes = [i32]
    lib.dfjk_trim_cache.argtypes = []
    lib.dfjk_phase_times.argtypes = [f64p, i32]
    for fn in EXPORTS:
        if fn not in ("dfjk_default_options", "dfjk_status_string", "dfjk_last_error",
                      "dfjk_launch_count"):
            getattr(lib, fn).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise DfjkError(rc, load_library().dfjk_last_error().decode())


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("the DF-J/K library needs a CUDA device (no CPU fallback)")
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# numpy layout of dfjk_shell (atom, l, nprim, pad, exps*, coefs*)
_SHELL_DTYPE = np.dtype({"names": ["atom", "l", "nprim", "exps", "coefs"],
                         "formats": [np.int32, np.int32, np.int32, np.uint64, np.uint64],
                         "offsets": [0, 4, 8, 16, 24], "itemsize": 32})


class _BasisHolder:
    """A dfjk_basis for `basis`, with the arrays it points into kept alive:
    every shell's exponents and coefficients in two contiguous arrays and the
    shell records in one structured array (no per-shell ctypes objects)."""

    def __init__(self, basis):
        assert ctypes.sizeof(Shell) == _SHELL_DTYPE.itemsize
        shells = list(basis.shells)
        n = len(shells)
        nprim = np.fromiter((len(s.exps) for s in shells), dtype=np.int64, count=n)
        off = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(nprim, out=off[1:])
        self.exps = np.ascontiguousarray(np.concatenate([np.asarray(s.exps, dtype=np.float64) for s in shells])
                                         if n else np.zeros(1), dtype=np.float64)
        self.coefs = np.ascontiguousarray(np.concatenate([np.asarray(s.coefs, dtype=np.float64) for s in shells])
                                          if n else np.zeros(1), dtype=np.float64)
        if n and (self.coefs.size != off[-1] or self.exps.size != off[-1]):
            raise ValueError("every shell needs as many coefficients as exponents")
        rec = np.zeros(max(1, n), dtype=_SHELL_DTYPE)
        if n:
            rec["atom"][:n] = np.fromiter((s.atom for s in shells), dtype=np.int32, count=n)
            rec["l"][:n] = np.fromiter((s.l for s in shells), dtype=np.int32, count=n)
            rec["nprim"][:n] = nprim
            rec["exps"][:n] = self.exps.ctypes.data + 8 * off[:n]
            rec["coefs"][:n] = self.coefs.ctypes.data + 8 * off[:n]
        self.rec = rec
        self.c = BasisC(n, ctypes.cast(rec.ctypes.data, ctypes.POINTER(Shell)))


def default_options(precision: int = DFJK_FP64, schwarz_thresh: float = 1e-12,
                    hbm_budget_bytes: int = 0, energies_on_host: bool = True,
                    timeout_iters: int = 0, fp32_pair_thresh: float = -1.0,
                    b_on_host: bool = False, tune_table: str | None = None) -> Options:
    o = Options()
    load_library().dfjk_default_options(ctypes.byref(o))
    o.precision = precision
    o.schwarz_thresh = schwarz_thresh
    o.hbm_budget_bytes = hbm_budget_bytes
    o.energies_on_host = 1 if energies_on_host else 0
    if timeout_iters > 0:
        o.timeout_iters = timeout_iters
    o.fp32_pair_thresh = fp32_pair_thresh
    o.b_on_host = 1 if b_on_host else 0
    o.tune_table = tune_table.encode() if tune_table else None
    return o


class Handle:
    """A molecule set up on the device (integrals, metric, Cholesky, whitening); B stays resident."""

    def __init__(self, mol, precision: int = DFJK_FP64, schwarz_thresh: float = 1e-12,
                 hbm_budget_bytes: int = 0, stream=None, timeout_iters: int = 0,
                 fp32_pair_thresh: float = -1.0, b_on_host: bool = False, tune_table: str | None = None):
        lib = load_library()
        _torch()
        self.mol = mol
        self._orb = _BasisHolder(mol.orb)
        self._aux = _BasisHolder(mol.aux)
        xyz = np.ascontiguousarray(mol.coords, dtype=np.float64)
        self.natom = int(xyz.shape[0])
        opt = default_options(precision, schwarz_thresh, hbm_budget_bytes, timeout_iters=timeout_iters,
                              fp32_pair_thresh=fp32_pair_thresh, b_on_host=b_on_host, tune_table=tune_table)
        h = ctypes.c_void_p()
        _check(
            lib.dfjk_setup(
                ctypes.byref(self._orb.c), ctypes.byref(self._aux.c), int(xyz.shape[0]),
                xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(opt),
                _stream(stream), ctypes.byref(h),
            )
        )
        self.h = h
        self.precision = precision
        nao, naux, npk = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        nbytes = ctypes.c_size_t()
        _check(lib.dfjk_query(h, ctypes.byref(nao), ctypes.byref(naux), ctypes.byref(npk),
                              ctypes.byref(nbytes)))
        self.nao, self.naux, self.npair_kept, self.device_bytes = (
            nao.value, naux.value, npk.value, nbytes.value)
        n32, thr = ctypes.c_int32(), ctypes.c_double()
        _check(lib.dfjk_query_precision(h, ctypes.byref(n32), ctypes.byref(thr)))
        self.npair_fp32, self.fp32_pair_thresh = n32.value, thr.value
        ns, lean = ctypes.c_int32(), ctypes.c_int32()
        _check(lib.dfjk_query_setup(h, ctypes.byref(ns), ctypes.byref(lean)))
        self.nslab, self.lean = ns.value, bool(lean.value)
        p64, p32 = (ctypes.c_int64 * 6)(), (ctypes.c_int64 * 6)()
        _check(lib.dfjk_query_pair_classes(h, p64, p32))
        # kept primitive pairs per class (ss, ps, pp, ds, dp, dd) in FP64 / FP32
        self.prim_pairs_fp64, self.prim_pairs_fp32 = list(p64), list(p32)
        tv = (ctypes.c_int32 * 4)()
        _check(lib.dfjk_query_tuning(h, tv))
        # launch shapes from the tuning table (0 = default): slicing rows,
        # B slicing rows, K range MB, build work-buffer cap MB
        self.tuning = list(tv)

    def build_chunks(self):
        """(rows per aux chunk, chunks) of the mixed build; (0, 0) before the
        first build and for DFJK_FP64."""
        r, n = ctypes.c_int32(), ctypes.c_int32()
        _check(load_library().dfjk_query_build(self.h, ctypes.byref(r), ctypes.byref(n)))
        return r.value, n.value

    def close(self):
        if getattr(self, "h", None):
            load_library().dfjk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build(self, C, J=None, K=None, E=None, stream=None, energies_on_device=False):
        """J, K, E_J, E_K for C [nao x nocc] or [nset x nao x nocc] (device FP64).
        Returns (J, K, E_J, E_K) with J, K device tensors."""
        torch = _torch()
        C = C.contiguous()
        if C.dim() == 2:
            C = C.unsqueeze(0)
        nset, nao, nocc = C.shape
        if nao != self.nao:
            raise ValueError("C has the wrong number of rows")
        if J is None:
            J = torch.empty((nset, nao, nao), dtype=torch.float64, device=C.device)
        if K is None:
            K = torch.empty((nset, nao, nao), dtype=torch.float64, device=C.device)
        if energies_on_device:
            EJ = torch.empty(nset, dtype=torch.float64, device=C.device)
            EK = torch.empty(nset, dtype=torch.float64, device=C.device)
            pj, pk = ctypes.c_void_p(EJ.data_ptr()), ctypes.c_void_p(EK.data_ptr())
        else:
            EJ = np.zeros(nset)
            EK = np.zeros(nset)
            pj, pk = ctypes.c_void_p(EJ.ctypes.data), ctypes.c_void_p(EK.ctypes.data)
        _check(load_library().dfjk_build(
            self.h, nset, nocc, ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(J.data_ptr()),
            ctypes.c_void_p(K.data_ptr()), pj, pk, _stream(stream)))
        return J, K, EJ, EK

    def build_uks(self, C_a, C_b, stream=None, energies_on_device=False):
        """Spin-unrestricted build: C_a [nao x nocc_a], C_b [nao x nocc_b] (device
        FP64, nocc_b <= nocc_a, nocc_b may be 0).  Returns (J of the total
        density, K_a, K_b, E) with E = [E_J total, E_K alpha, E_K beta]."""
        torch = _torch()
        C_a = C_a.contiguous()
        C_b = C_b.contiguous()
        nao = self.nao
        if C_a.shape[0] != nao or C_b.shape[0] != nao:
            raise ValueError("C has the wrong number of rows")
        J = torch.empty((nao, nao), dtype=torch.float64, device=C_a.device)
        Ka = torch.empty_like(J)
        Kb = torch.empty_like(J)
        if energies_on_device:
            E = torch.empty(3, dtype=torch.float64, device=C_a.device)
            pe = ctypes.c_void_p(E.data_ptr())
        else:
            E = np.zeros(3)
            pe = ctypes.c_void_p(E.ctypes.data)
        nb = int(C_b.shape[1])
        _check(load_library().dfjk_build_uks(
            self.h, int(C_a.shape[1]), ctypes.c_void_p(C_a.data_ptr()), nb,
            ctypes.c_void_p(C_b.data_ptr() if nb else None), ctypes.c_void_p(J.data_ptr()),
            ctypes.c_void_p(Ka.data_ptr()), ctypes.c_void_p(Kb.data_ptr()), pe, _stream(stream)))
        return J, Ka, Kb, E

    def build_density(self, D, stream=None):
        """J, K, E_J, E_K from densities D [nao x nao] or [nset x nao x nao]
        (device FP64, symmetric), on the FP64 pipe."""
        torch = _torch()
        D = D.contiguous()
        if D.dim() == 2:
            D = D.unsqueeze(0)
        nset = D.shape[0]
        J = torch.empty_like(D)
        K = torch.empty_like(D)
        EJ, EK = np.zeros(nset), np.zeros(nset)
        _check(load_library().dfjk_build_density(
            self.h, nset, ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(J.data_ptr()),
            ctypes.c_void_p(K.data_ptr()), ctypes.c_void_p(EJ.ctypes.data), ctypes.c_void_p(EK.ctypes.data),
            _stream(stream)))
        return J, K, EJ, EK

    def coulomb_gradient(self, D, stream=None):
        """dE_J/dR [natom x 3] at fixed density D [nao x nao] (device FP64,
        symmetric), E_J = u^T V^-1 u / 2 with u = (P|mu nu) D."""
        torch = _torch()
        D = D.contiguous()
        g = torch.empty((self.natom, 3), dtype=torch.float64, device=D.device)
        _check(load_library().dfjk_coulomb_gradient(
            self.h, ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(g.data_ptr()), _stream(stream)))
        return g

    def jk_gradient(self, C, c_j=1.0, c_k=1.0, stream=None):
        """d(c_j E_J + c_k E_K)/dR [natom x 3] at fixed D = C C^T, C a device
        FP64 tensor [nao x nocc]."""
        torch = _torch()
        C = C.contiguous()
        g = torch.empty((self.natom, 3), dtype=torch.float64, device=C.device)
        _check(load_library().dfjk_jk_gradient(
            self.h, int(C.shape[1]), ctypes.c_void_p(C.data_ptr()), float(c_j), float(c_k),
            ctypes.c_void_p(g.data_ptr()), _stream(stream)))
        return g

    def overlap(self, stream=None):
        torch = _torch()
        S = torch.empty((self.nao, self.nao), dtype=torch.float64, device="cuda")
        _check(load_library().dfjk_overlap(self.h, ctypes.c_void_p(S.data_ptr()), _stream(stream)))
        return S

    def evict(self):
        _check(load_library().dfjk_evict(self.h))

    def _get(self, fn, shape, dtype=None):
        torch = _torch()
        out = torch.empty(shape, dtype=dtype or torch.float64, device="cuda")
        _check(getattr(load_library(), fn)(self.h, ctypes.c_void_p(out.data_ptr()), _stream()))
        torch.cuda.current_stream().synchronize()
        return out

    def metric(self):
        return self._get("dfjk_get_metric", (self.naux, self.naux))

    def cholesky(self):
        return self._get("dfjk_get_cholesky", (self.naux, self.naux))

    def B(self):
        return self._get("dfjk_get_B", (self.naux, self.nao, self.nao))

    def B_columns(self, mu, nu):
        """B[:, mu[c], nu[c]] for each c, as a device tensor [ncol, naux]."""
        torch = _torch()
        mu = np.ascontiguousarray(mu, dtype=np.int32)
        nu = np.ascontiguousarray(nu, dtype=np.int32)
        out = torch.empty((len(mu), self.naux), dtype=torch.float64, device="cuda")
        _check(load_library().dfjk_get_B_columns(self.h, len(mu), ctypes.c_void_p(mu.ctypes.data),
                                                 ctypes.c_void_p(nu.ctypes.data),
                                                 ctypes.c_void_p(out.data_ptr()), _stream()))
        return out

    def three_center(self):
        return self._get("dfjk_get_three_center", (self.naux, self.nao, self.nao))

    def pair_mask(self):
        torch = _torch()
        n = len(self.mol.orb.shells)
        return self._get("dfjk_get_pair_mask", (n, n), dtype=torch.int32)


def build_batch(handles, Cs, Js=None, Ks=None, E=None, nstreams=8, stream=None):
    """Builds every resident handle with its C (device [nao_i, nocc_i]) in one
    call (batching).  Returns (Js, Ks, E) with E a device tensor [2, nmol]
    (E_J, E_K); nothing is synchronised."""
    torch = _torch()
    n = len(handles)
    Cs = [c.contiguous() for c in Cs]
    if Js is None:
        Js = [torch.empty((h.nao, h.nao), dtype=torch.float64, device="cuda") for h in handles]
    if Ks is None:
        Ks = [torch.empty((h.nao, h.nao), dtype=torch.float64, device="cuda") for h in handles]
    if E is None:
        E = torch.empty((2, n), dtype=torch.float64, device="cuda")
    vp = ctypes.c_void_p
    hs = (vp * n)(*[h.h for h in handles])
    nocc = (ctypes.c_int32 * n)(*[int(c.shape[1]) for c in Cs])
    cp = (vp * n)(*[c.data_ptr() for c in Cs])
    jp = (vp * n)(*[j.data_ptr() for j in Js])
    kp = (vp * n)(*[k.data_ptr() for k in Ks])
    _check(load_library().dfjk_build_batch(n, hs, nocc, cp, jp, kp, vp(E[0].data_ptr()),
                                           vp(E[1].data_ptr()), int(nstreams), _stream(stream)))
    return Js, Ks, E


def boys(mmax: int, T, stream=None):
    """F_0..F_mmax at the device points T (FP64), shape [n, mmax+1]."""
    torch = _torch()
    T = T.contiguous()
    F = torch.empty((T.numel(), mmax + 1), dtype=torch.float64, device=T.device)
    _check(load_library().dfjk_boys(mmax, T.numel(), ctypes.c_void_p(T.data_ptr()),
                                    ctypes.c_void_p(F.data_ptr()), _stream(stream)))
    return F


def set_timing(enable: bool):
    _check(load_library().dfjk_set_timing(1 if enable else 0))


def phase_times() -> dict:
    """Accumulated device milliseconds per phase since the last call."""
    ms = (ctypes.c_double * len(PHASES))()
    _check(load_library().dfjk_phase_times(ms, len(PHASES)))
    return {name: ms[i] for i, name in enumerate(PHASES)}


def sliced_gemm(A, B, S=6, stream=None):
    """C[z] = A[z] B^T through the exact sliced tensor-core GEMM (FP64 device
    tensors; A [batch, M, K] or [M, K], B [N, K])."""
    torch = _torch()
    A3 = A.contiguous().reshape(-1, A.shape[-2], A.shape[-1])
    B = B.contiguous()
    batch, M, K = A3.shape
    N = B.shape[0]
    C = torch.empty((batch, M, N), dtype=torch.float64, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(load_library().dfjk_debug_sliced_gemm(
        batch, M, N, K, S, ctypes.c_void_p(A3.data_ptr()), ctypes.c_void_p(B.data_ptr()),
        ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(status.data_ptr()), _stream(stream)))
    if int(status.item()) != 0:
        raise DfjkError(6, f"device status {int(status.item())}")
    return C.reshape(A.shape[:-1] + (N,))


def energies_noalloc(D, J, K, E, stream=None):
    """E[0] = Tr(D J)/2, E[1] = Tr(D K)/2 via the allocation-free entry point
    (device tensors; n x n and 2 elements)."""
    n = D.shape[-1]
    _check(load_library().dfjk_energies_noalloc(
        n, ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(J.data_ptr()),
        ctypes.c_void_p(K.data_ptr()), ctypes.c_void_p(E.data_ptr()), _stream(stream)))
    return E


def estimate_bytes(nao: int, naux: int, nocc: int, precision: int) -> dict:
    """Device bytes of a molecule before setup (dfjk_estimate_bytes): resident
    data, the build's work buffers at nocc, the setup's transient peak."""
    lib = load_library()
    r, w, s = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib.dfjk_estimate_bytes(int(nao), int(naux), int(nocc), int(precision), ctypes.byref(r),
                                   ctypes.byref(w), ctypes.byref(s)))
    return {"resident": r.value, "build_ws": w.value, "setup_ws": s.value}


def fma_rate(bits: int = 64, stream=None) -> float:
    """Measured FMA throughput of the GPU in TFLOP/s (dfjk_fma_rate)."""
    r = ctypes.c_double()
    _check(load_library().dfjk_fma_rate(int(bits), ctypes.byref(r), _stream(stream)))
    return r.value


def launch_count() -> int:
    return int(load_library().dfjk_launch_count())


def overlap_matrix(mol, stream=None):
    """S of the orbital basis of `mol` (device), without a setup."""
    torch = _torch()
    b = _BasisHolder(mol.orb)
    xyz = np.ascontiguousarray(mol.coords, dtype=np.float64)
    S = torch.empty((mol.nao, mol.nao), dtype=torch.float64, device="cuda")
    _check(load_library().dfjk_overlap_matrix(
        ctypes.byref(b.c), int(xyz.shape[0]), xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        ctypes.c_void_p(S.data_ptr()), _stream(stream)))
    torch.cuda.current_stream().synchronize()
    return S


def orthonormal_c_occ(handle: Handle, C0: np.ndarray):
    """C_occ made orthonormal in the overlap metric that the library computes
    on the device (input preparation, outside any timed region)."""
    from .inputs import orthonormalize

    S = handle.overlap().cpu().numpy()
    return orthonormalize(C0, S)
