"""Thin ctypes binding of liblqcd.so (include/lqcd.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  Fields are torch tensors on the GPU in the canonical
layouts of lqcd.h (complex128 for FP64, complex64 for FP32):
    full field  (V, 4, 3), even/odd field (V/2, 4, 3), nrhs fields stacked
    in front; links (V, 4, 3, 3) complex128.
There is no CPU path: if the library or a GPU is missing the first call
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build_lib

F64, F32, F16S, BF16 = 0, 1, 2, 3
SOLVER_CGNR, SOLVER_SAP_GCR, SOLVER_DFL_SAP_GCR, SOLVER_NET_GCR, SOLVER_DFL_NET_GCR = 0, 1, 2, 3, 4

STATUS = {
    0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_NOMEM", 4: "ERR_SINGULAR_CLOVER",
    5: "ERR_NOT_CONVERGED", 6: "ERR_BREAKDOWN", 7: "ERR_NAN", 8: "ERR_TIMEOUT", 9: "ERR_STATE",
}


class LqcdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Geom(C.Structure):
    _fields_ = [("T", C.c_int), ("L1", C.c_int), ("L2", C.c_int), ("L3", C.c_int), ("antiperiodic_t", C.c_int)]


class SapParams(C.Structure):
    _fields_ = [("bs", C.c_int * 4), ("ncy", C.c_int), ("nmr", C.c_int), ("prec", C.c_int)]


class DflParams(C.Structure):
    _fields_ = [("bs", C.c_int * 4), ("Ns", C.c_int), ("ninv", C.c_int), ("ncy", C.c_int), ("nmr", C.c_int),
                ("prec", C.c_int), ("coarse_tol", C.c_double), ("coarse_nkv", C.c_int), ("coarse_nmx", C.c_int),
                ("coarse_prec", C.c_int), ("build_sap_prec", C.c_int), ("coarse_eo", C.c_int)]


class SolverParams(C.Structure):
    _fields_ = [("solver", C.c_int), ("nkv", C.c_int), ("nmx", C.c_int), ("tol", C.c_double),
                ("sap", SapParams), ("inner", C.c_int), ("krylov", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("true_relres", C.c_double),
                ("relres_dhat", C.c_double), ("seconds", C.c_double), ("status", C.c_int),
                ("net_fallbacks", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MDParams(C.Structure):
    _fields_ = [("beta", C.c_double), ("dt", C.c_double), ("nsteps", C.c_int), ("solver", SolverParams)]


class BlockParams(C.Structure):
    _fields_ = [("bs", C.c_int * 4), ("tol", C.c_double), ("nmx", C.c_int)]


class BatchParams(C.Structure):
    _fields_ = [("nkv", C.c_int), ("nmx", C.c_int), ("tol", C.c_double), ("sap", SapParams),
                ("use_graph", C.c_int), ("wait_timeout_s", C.c_double), ("stall_test", C.c_int)]


class NetDesc(C.Structure):
    _fields_ = [("nlayers", C.c_int), ("chans", C.c_int * 5), ("act", C.c_int)]


class NetTrainParams(C.Structure):
    _fields_ = [("steps", C.c_int), ("batch", C.c_int), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double), ("sap", SapParams), ("loss", C.c_int)]


NET_LOSS_SAP, NET_LOSS_RESIDUAL = 0, 1


_lib = None


def lib_path() -> str:
    return build_lib.LIB


def lib():
    global _lib
    if _lib is None:
        if build_lib.needs_build():
            build_lib.build()
        if not os.path.exists(build_lib.LIB):
            raise RuntimeError("liblqcd.so is missing: run __graft_entry__.build()")
        L = C.CDLL(build_lib.LIB)
        P, I, D, S = C.c_void_p, C.c_int, C.c_double, C.c_size_t
        sig = {
            "lqcd_create": [C.POINTER(Geom), P, C.POINTER(P)],
            "lqcd_destroy": [P],
            "lqcd_set_stream": [P, P],
            "lqcd_set_gauge": [P, P],
            "lqcd_clover_invert": [P, D, D, C.POINTER(D), C.POINTER(D)],
            "lqcd_apply_clover": [P, I, I, P, P],
            "lqcd_apply_D": [P, I, P, P, I],
            "lqcd_apply_Dhat": [P, I, P, P, I],
            "lqcd_pack": [P, I, I, P, P, I],
            "lqcd_unpack": [P, I, I, P, P, I],
            "lqcd_apply_Dhat_native": [P, I, P, P, I],
            "lqcd_apply_D_native": [P, I, P, P, I],
            "lqcd_apply_Dhat_native_static": [P, I, P, P, I],
            "lqcd_sap": [P, C.POINTER(SapParams), P, P],
            "lqcd_dfl_build": [P, C.POINTER(DflParams), P],
            "lqcd_dfl_export": [P, P, P],
            "lqcd_dfl_project": [P, P, P],
            "lqcd_dfl_expand": [P, P, P],
            "lqcd_dfl_little_apply": [P, P, P],
            "lqcd_dfl_coarse_solve": [P, P, P, C.POINTER(I)],
            "lqcd_dfl_precond": [P, C.POINTER(SapParams), P, P],
            "lqcd_net_set": [P, C.POINTER(NetDesc), P],
            "lqcd_net_get": [P, P],
            "lqcd_net_apply": [P, P, P, I],
            "lqcd_net_loss_grad": [P, P, P, I, C.POINTER(D), P],
            "lqcd_net_train": [P, C.POINTER(NetTrainParams), P, I, P],
            "lqcd_solve_dhat": [P, C.POINTER(SolverParams), P, P, I, C.POINTER(SolveInfo)],
            "lqcd_solve_D": [P, C.POINTER(SolverParams), P, P, I, C.POINTER(SolveInfo)],
            "lqcd_apply_W": [P, I, D, P, P, I],
            "lqcd_solve_dhat_guess": [P, C.POINTER(SolverParams), P, P, I, C.POINTER(SolveInfo)],
            "lqcd_chrono_reset": [P, I],
            "lqcd_chrono_add": [P, P],
            "lqcd_chrono_guess": [P, P, P, C.POINTER(I)],
            "lqcd_solve_W": [P, C.POINTER(SolverParams), D, P, P, I, C.POINTER(SolveInfo)],
            "lqcd_apply_Dhat_block": [P, C.POINTER(I), P, P],
            "lqcd_block_solve": [P, C.POINTER(BlockParams), P, P, C.POINTER(I), C.POINTER(D), C.POINTER(I)],
            "lqcd_tune_reset": [],
            "lqcd_force_dD": [P, P, P, P],
            "lqcd_force_logdet": [P, I, P],
            "lqcd_gauge_action": [P, D, C.POINTER(D)],
            "lqcd_force_gauge": [P, D, P],
            "lqcd_force_pf": [P, C.POINTER(SolverParams), P, P, C.POINTER(SolveInfo)],
            "lqcd_md_gradient": [P, C.POINTER(MDParams), P, P, C.POINTER(D)],
            "lqcd_md_leapfrog": [P, C.POINTER(MDParams), P, P, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.lqcd_last_error.argtypes = [P]
        L.lqcd_last_error.restype = C.c_char_p
        L.lqcd_native_bytes.argtypes = [P, I, I, I]
        L.lqcd_native_bytes.restype = S
        L.lqcd_block_count.argtypes = [P, C.POINTER(I)]
        L.lqcd_block_count.restype = C.c_long
        L.lqcd_kernel_launches.argtypes = [P]
        L.lqcd_kernel_launches.restype = C.c_long
        L.lqcd_dfl_stats.argtypes = [P, C.POINTER(C.c_long), C.POINTER(C.c_long)]
        L.lqcd_dfl_stats.restype = C.c_int
        L.lqcd_batch_create.argtypes = [P, I, C.POINTER(BatchParams), P, C.POINTER(P)]
        L.lqcd_batch_create.restype = C.c_int
        L.lqcd_batch_destroy.argtypes = [P]
        L.lqcd_batch_destroy.restype = C.c_int
        L.lqcd_batch_last_error.argtypes = [P]
        L.lqcd_batch_last_error.restype = C.c_char_p
        L.lqcd_batch_solve_dhat.argtypes = [P, P, P, C.POINTER(SolveInfo)]
        L.lqcd_batch_solve_dhat.restype = C.c_int
        L.lqcd_batch_stats.argtypes = [P, C.POINTER(I), C.POINTER(I), C.POINTER(C.c_long)]
        L.lqcd_batch_stats.restype = C.c_int
        _lib = L
    return _lib


def tune_reset() -> None:
    """Forget the autotuner's in-memory choices (the next lookup re-reads the
    cache file named by LQCD_TUNE_CACHE)."""
    lib().lqcd_tune_reset()


def _ptr(t: torch.Tensor):
    if not t.is_cuda:
        raise ValueError("liblqcd takes device tensors only")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _dtype(prec):
    # canonical fields of the F16S operators are complex float
    return {F64: torch.complex128, F32: torch.complex64, F16S: torch.complex64}.get(prec, torch.complex128)


def sap_params(bs=(4, 4, 4, 4), ncy=4, nmr=5, prec=F64) -> SapParams:
    return SapParams((C.c_int * 4)(*bs), ncy, nmr, prec)


class Context:
    """One lattice on the current CUDA device; all work on the given stream
    (default: torch's current stream at creation)."""

    def __init__(self, dims, antiperiodic_t: bool = True, stream=None):
        self.dims = tuple(int(d) for d in dims)
        T, L1, L2, L3 = self.dims
        self.V = T * L1 * L2 * L3
        self.Vh = self.V // 2
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        g = Geom(T, L1, L2, L3, 1 if antiperiodic_t else 0)
        st = lib().lqcd_create(C.byref(g), C.c_void_p(stream.cuda_stream), C.byref(h))
        if st != 0:
            raise LqcdError(st, f"lqcd_create{self.dims}")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lqcd_destroy(self._h)
            self._h = None

    def _check(self, st, what):
        if st != 0:
            msg = lib().lqcd_last_error(self._h)
            raise LqcdError(st, f"{what}: {msg.decode() if msg else ''}")

    @property
    def kernel_launches(self) -> int:
        return lib().lqcd_kernel_launches(self._h)

    # ---------------------------------------------------------------- setup
    def set_gauge(self, U: torch.Tensor):
        U = U.to(torch.complex128).contiguous()
        assert U.numel() == self.V * 36
        self._U = U
        self._check(lib().lqcd_set_gauge(self._h, _ptr(U)), "lqcd_set_gauge")

    def clover_invert(self, kappa: float, csw: float):
        le, lo = C.c_double(), C.c_double()
        st = lib().lqcd_clover_invert(self._h, float(kappa), float(csw), C.byref(le), C.byref(lo))
        self._check(st, "lqcd_clover_invert")
        return le.value, lo.value

    def apply_clover(self, parity: int, inverse: bool, x: torch.Tensor) -> torch.Tensor:
        x = x.to(torch.complex128).contiguous()
        out = torch.empty_like(x)
        self._check(lib().lqcd_apply_clover(self._h, parity, int(inverse), _ptr(x), _ptr(out)), "apply_clover")
        return out

    # ------------------------------------------------------------ operators
    def _nrhs(self, x, nsites):
        n = x.numel() // (12 * nsites)
        assert n * 12 * nsites == x.numel(), "field size mismatch"
        return n

    def apply_D(self, x: torch.Tensor, prec=F64) -> torch.Tensor:
        x = x.to(_dtype(prec)).contiguous()
        out = torch.empty_like(x)
        self._check(lib().lqcd_apply_D(self._h, prec, _ptr(x), _ptr(out), self._nrhs(x, self.V)), "apply_D")
        return out

    def apply_Dhat(self, x: torch.Tensor, prec=F64) -> torch.Tensor:
        x = x.to(_dtype(prec)).contiguous()
        out = torch.empty_like(x)
        self._check(lib().lqcd_apply_Dhat(self._h, prec, _ptr(x), _ptr(out), self._nrhs(x, self.Vh)),
                    "apply_Dhat")
        return out

    def native_bytes(self, prec, nsub, nrhs) -> int:
        return lib().lqcd_native_bytes(self._h, prec, nsub, nrhs)

    def native_empty(self, prec, nsub, nrhs) -> torch.Tensor:
        n = self.native_bytes(prec, nsub, nrhs)
        return torch.empty(n, dtype=torch.uint8, device="cuda")

    def pack(self, x: torch.Tensor, prec, nsub) -> torch.Tensor:
        x = x.to(_dtype(prec)).contiguous()
        nrhs = self._nrhs(x, nsub * self.Vh)
        out = self.native_empty(prec, nsub, nrhs)
        self._check(lib().lqcd_pack(self._h, prec, nsub, _ptr(x), _ptr(out), nrhs), "pack")
        return out

    def unpack(self, n: torch.Tensor, prec, nsub, nrhs) -> torch.Tensor:
        out = torch.empty((nrhs, nsub * self.Vh, 4, 3), dtype=_dtype(prec), device="cuda")
        self._check(lib().lqcd_unpack(self._h, prec, nsub, _ptr(n), _ptr(out), nrhs), "unpack")
        return out

    def apply_Dhat_native(self, x_native, out_native, prec, nrhs):
        self._check(lib().lqcd_apply_Dhat_native(self._h, prec, _ptr(x_native), _ptr(out_native), nrhs),
                    "apply_Dhat_native")

    def apply_Dhat_native_static(self, x_native, out_native, prec, nrhs):
        """As apply_Dhat_native, with the odd-site intermediate in the library's
        fixed device array (no device allocation; see lqcd.h for the limit)."""
        self._check(lib().lqcd_apply_Dhat_native_static(self._h, prec, _ptr(x_native), _ptr(out_native), nrhs),
                    "apply_Dhat_native_static")

    def apply_D_native(self, x_native, out_native, prec, nrhs):
        self._check(lib().lqcd_apply_D_native(self._h, prec, _ptr(x_native), _ptr(out_native), nrhs),
                    "apply_D_native")

    # ------------------------------------------------------------------ SAP
    def sap(self, eta: torch.Tensor, bs=(4, 4, 4, 4), ncy=4, nmr=5, prec=F64) -> torch.Tensor:
        eta = eta.to(torch.complex128).contiguous()
        out = torch.empty_like(eta)
        p = sap_params(bs, ncy, nmr, prec)
        self._check(lib().lqcd_sap(self._h, C.byref(p), _ptr(eta), _ptr(out)), "lqcd_sap")
        return out

    # ------------------------------------------------------------ deflation
    def dfl_build(self, v0: torch.Tensor, bs=(4, 4, 4, 4), ninv=4, ncy=4, nmr=4, prec=F32, coarse_tol=1e-8,
                  coarse_nkv=16, coarse_nmx=4096, coarse_prec=F64, build_sap_prec=None, coarse_eo=False):
        v0 = v0.to(torch.complex128).contiguous()
        Ns = v0.numel() // (12 * self.V)
        self.Ns = Ns
        nb = 1
        for L, b in zip(self.dims, bs):
            nb *= L // b
        self.nblk = nb
        p = DflParams((C.c_int * 4)(*bs), Ns, ninv, ncy, nmr, prec, coarse_tol, coarse_nkv, coarse_nmx, coarse_prec,
                      prec if build_sap_prec is None else build_sap_prec, int(bool(coarse_eo)))
        self._check(lib().lqcd_dfl_build(self._h, C.byref(p), _ptr(v0)), "lqcd_dfl_build")

    def dfl_export(self):
        phi = torch.empty((self.Ns, self.V, 4, 3), dtype=torch.complex128, device="cuda")
        A = torch.empty((self.nblk, 9, self.Ns, self.Ns), dtype=torch.complex128, device="cuda")
        self._check(lib().lqcd_dfl_export(self._h, _ptr(phi), _ptr(A)), "lqcd_dfl_export")
        return phi, A

    def dfl_stats(self):
        """(coarse solves, coarse GCR iterations) since the subspace was built."""
        s, i = C.c_long(), C.c_long()
        self._check(lib().lqcd_dfl_stats(self._h, C.byref(s), C.byref(i)), "lqcd_dfl_stats")
        return s.value, i.value

    def dfl_project(self, x):
        x = x.to(torch.complex128).contiguous()
        c = torch.empty(self.nblk * self.Ns, dtype=torch.complex128, device="cuda")
        self._check(lib().lqcd_dfl_project(self._h, _ptr(x), _ptr(c)), "dfl_project")
        return c

    def dfl_expand(self, c):
        c = c.to(torch.complex128).contiguous()
        out = torch.empty((self.V, 4, 3), dtype=torch.complex128, device="cuda")
        self._check(lib().lqcd_dfl_expand(self._h, _ptr(c), _ptr(out)), "dfl_expand")
        return out

    def dfl_little_apply(self, c):
        c = c.to(torch.complex128).contiguous()
        out = torch.empty_like(c)
        self._check(lib().lqcd_dfl_little_apply(self._h, _ptr(c), _ptr(out)), "dfl_little_apply")
        return out

    def dfl_coarse_solve(self, b):
        b = b.to(torch.complex128).contiguous()
        out = torch.empty_like(b)
        it = C.c_int(0)
        self._check(lib().lqcd_dfl_coarse_solve(self._h, _ptr(b), _ptr(out), C.byref(it)), "dfl_coarse_solve")
        return out, it.value

    def dfl_precond(self, rho, bs=(4, 4, 4, 4), ncy=4, nmr=5, prec=F64):
        rho = rho.to(torch.complex128).contiguous()
        out = torch.empty_like(rho)
        p = sap_params(bs, ncy, nmr, prec)
        self._check(lib().lqcd_dfl_precond(self._h, C.byref(p), _ptr(rho), _ptr(out)), "dfl_precond")
        return out

    # --------------------------------------------------- learned preconditioner
    @staticmethod
    def net_weight_count(chans) -> int:
        return sum(chans[l] * chans[l + 1] * 144 for l in range(len(chans) - 1))

    def net_set(self, chans, W, act=BF16):
        """W: complex numpy array (flat, layer after layer, [o][i][d][s][s'])."""
        import numpy as np
        chans = [int(c) for c in chans]
        W = np.ascontiguousarray(np.asarray(W, dtype=np.complex64))
        assert W.size == self.net_weight_count(chans)
        d = NetDesc(len(chans) - 1, (C.c_int * 5)(*(chans + [0] * (5 - len(chans)))), act)
        self._net_chans = chans
        self._check(lib().lqcd_net_set(self._h, C.byref(d), W.ctypes.data_as(C.c_void_p)), "lqcd_net_set")

    def net_get(self):
        import numpy as np
        W = np.empty(self.net_weight_count(self._net_chans), dtype=np.complex64)
        self._check(lib().lqcd_net_get(self._h, W.ctypes.data_as(C.c_void_p)), "lqcd_net_get")
        return W

    def net_apply(self, x: torch.Tensor) -> torch.Tensor:
        x = x.to(torch.complex128).contiguous()
        out = torch.empty_like(x)
        self._check(lib().lqcd_net_apply(self._h, _ptr(x), _ptr(out), self._nrhs(x, self.V)), "lqcd_net_apply")
        return out

    def net_loss_grad(self, x: torch.Tensor, t: torch.Tensor):
        import numpy as np
        x = x.to(torch.complex128).contiguous()
        t = t.to(torch.complex128).contiguous()
        g = np.empty(self.net_weight_count(self._net_chans), dtype=np.complex64)
        loss = C.c_double()
        st = lib().lqcd_net_loss_grad(self._h, _ptr(x), _ptr(t), self._nrhs(x, self.V), C.byref(loss),
                                      g.ctypes.data_as(C.c_void_p))
        self._check(st, "lqcd_net_loss_grad")
        return loss.value, g

    def net_train(self, sources: torch.Tensor, steps, batch=8, lr=1e-3, bs=(4, 4, 4, 4), ncy=4, nmr=5, sap_prec=F32,
                  loss=NET_LOSS_SAP):
        import numpy as np
        sources = sources.to(torch.complex128).contiguous()
        nsrc = self._nrhs(sources, self.V)
        p = NetTrainParams(steps, batch, lr, 0.9, 0.999, 1e-8, sap_params(bs, ncy, nmr, sap_prec), loss)
        hist = np.zeros(max(steps, 1))
        self._check(lib().lqcd_net_train(self._h, C.byref(p), _ptr(sources), nsrc, hist.ctypes.data_as(C.c_void_p)),
                    "lqcd_net_train")
        return hist[:steps]

    # -------------------------------------------------------------- solvers
    def _solve(self, fn, eta, nsites, solver, tol, nkv, nmx, bs, ncy, nmr, sap_prec, inner, check, krylov=F64):
        eta = eta.to(torch.complex128).contiguous()
        nrhs = self._nrhs(eta, nsites)
        psi = torch.empty_like(eta)
        p = SolverParams(solver, nkv, nmx, tol, sap_params(bs, ncy, nmr, sap_prec), inner, krylov)
        info = (SolveInfo * nrhs)()
        st = fn(self._h, C.byref(p), _ptr(eta), _ptr(psi), nrhs, info)
        infos = [i.as_dict() for i in info]
        if check:
            self._check(st, "solve")
        return psi, infos, st

    def solve_dhat(self, eta, solver=SOLVER_SAP_GCR, tol=1e-10, nkv=16, nmx=4096, bs=(4, 4, 4, 4), ncy=4, nmr=5,
                   sap_prec=F64, inner=F64, check=True, krylov=F64):
        return self._solve(lib().lqcd_solve_dhat, eta, self.Vh, solver, tol, nkv, nmx, bs, ncy, nmr, sap_prec,
                           inner, check, krylov)

    def solve_dhat_guess(self, eta, x0, solver=SOLVER_SAP_GCR, tol=1e-10, nkv=16, nmx=4096, bs=(4, 4, 4, 4),
                         ncy=4, nmr=5, sap_prec=F64, inner=F64, check=True, krylov=F64):
        """As solve_dhat, starting from the guess x0 (even fields)."""
        eta = eta.to(torch.complex128).contiguous()
        nrhs = self._nrhs(eta, self.Vh)
        psi = x0.to(torch.complex128).contiguous().clone()
        p = SolverParams(solver, nkv, nmx, tol, sap_params(bs, ncy, nmr, sap_prec), inner, krylov)
        info = (SolveInfo * nrhs)()
        st = lib().lqcd_solve_dhat_guess(self._h, C.byref(p), _ptr(eta), _ptr(psi), nrhs, info)
        if check:
            self._check(st, "solve_dhat_guess")
        return psi, [i.as_dict() for i in info], st

    # ------------------------------------------------- MD forces (Sec. 2, Eq. 4)
    def _grad(self):
        return torch.empty((self.V, 4, 8), dtype=torch.float64, device="cuda")

    def force_dD(self, X: torch.Tensor, Y: torch.Tensor) -> torch.Tensor:
        """Re <Y, dD X> per link and generator, (V, 4, 8) float64."""
        X = X.to(torch.complex128).contiguous()
        Y = Y.to(torch.complex128).contiguous()
        g = self._grad()
        self._check(lib().lqcd_force_dD(self._h, _ptr(X), _ptr(Y), _ptr(g)), "force_dD")
        return g

    def force_logdet(self, parity: int) -> torch.Tensor:
        g = self._grad()
        self._check(lib().lqcd_force_logdet(self._h, parity, _ptr(g)), "force_logdet")
        return g

    def gauge_action(self, beta: float) -> float:
        S = C.c_double(0)
        self._check(lib().lqcd_gauge_action(self._h, beta, C.byref(S)), "gauge_action")
        return S.value

    def force_gauge(self, beta: float) -> torch.Tensor:
        g = self._grad()
        self._check(lib().lqcd_force_gauge(self._h, beta, _ptr(g)), "force_gauge")
        return g

    @staticmethod
    def md_solver(solver=SOLVER_SAP_GCR, tol=1e-12, nkv=16, nmx=4096, bs=(4, 4, 4, 4), ncy=4, nmr=5, sap_prec=F64,
                  inner=F64, krylov=F64) -> SolverParams:
        return SolverParams(solver, nkv, nmx, tol, sap_params(bs, ncy, nmr, sap_prec), inner, krylov)

    def force_pf(self, phi_e: torch.Tensor, sp: SolverParams = None):
        """Gradient of |Dhat^-1 phi_e|^2; returns (g, [info of the two solves])."""
        phi_e = phi_e.to(torch.complex128).contiguous()
        sp = sp or self.md_solver()
        g = self._grad()
        info = (SolveInfo * 2)()
        self._check(lib().lqcd_force_pf(self._h, C.byref(sp), _ptr(phi_e), _ptr(g), info), "force_pf")
        return g, [i.as_dict() for i in info]

    def md_gradient(self, phi_e: torch.Tensor, beta: float, sp: SolverParams = None):
        """(gradient of S = S_g + |Dhat^-1 phi|^2 - 2 log|det A_oo|, S)."""
        phi_e = phi_e.to(torch.complex128).contiguous()
        mp = MDParams(beta, 0.0, 0, sp or self.md_solver())
        g = self._grad()
        S = C.c_double(0)
        self._check(lib().lqcd_md_gradient(self._h, C.byref(mp), _ptr(phi_e), _ptr(g), C.byref(S)), "md_gradient")
        return g, S.value

    def md_leapfrog(self, U: torch.Tensor, p: torch.Tensor, phi_e: torch.Tensor, beta: float, dt: float,
                    nsteps: int, sp: SolverParams = None):
        """nsteps leapfrog steps; U (canonical links, the context's field) and p
        ((V, 4, 8) float64 momenta) are updated in place."""
        assert U.dtype == torch.complex128 and U.is_contiguous()
        assert p.dtype == torch.float64 and p.is_contiguous()
        phi_e = phi_e.to(torch.complex128).contiguous()
        mp = MDParams(beta, dt, nsteps, sp or self.md_solver())
        self._check(lib().lqcd_md_leapfrog(self._h, C.byref(mp), _ptr(U), _ptr(p), _ptr(phi_e)), "md_leapfrog")

    def chrono_reset(self, nkeep: int):
        self._check(lib().lqcd_chrono_reset(self._h, nkeep), "chrono_reset")

    def chrono_add(self, psi: torch.Tensor):
        psi = psi.to(torch.complex128).contiguous()
        self._check(lib().lqcd_chrono_add(self._h, _ptr(psi)), "chrono_add")

    def chrono_guess(self, eta: torch.Tensor):
        eta = eta.to(torch.complex128).contiguous()
        x0 = torch.empty_like(eta)
        n = C.c_int()
        self._check(lib().lqcd_chrono_guess(self._h, _ptr(eta), _ptr(x0), C.byref(n)), "chrono_guess")
        return x0, n.value

    # ------------------------------------------------- DD-HMC block solves
    def block_count(self, bs) -> int:
        return int(lib().lqcd_block_count(self._h, (C.c_int * 4)(*bs)))

    def apply_Dhat_block(self, x: torch.Tensor, bs) -> torch.Tensor:
        """Dhat_blk x on every Dirichlet block of extents bs (one even FP64 field)."""
        x = x.to(torch.complex128).contiguous()
        out = torch.empty_like(x)
        self._check(lib().lqcd_apply_Dhat_block(self._h, (C.c_int * 4)(*bs), _ptr(x), _ptr(out)), "apply_Dhat_block")
        return out

    def block_solve(self, eta: torch.Tensor, bs, tol=1e-10, nmx=1000, check=True):
        """BiCGstab on every block: (psi, status, iters[nblk], relres[nblk], status[nblk])."""
        import numpy as np
        eta = eta.to(torch.complex128).contiguous()
        psi = torch.empty_like(eta)
        nb = self.block_count(bs)
        if nb < 1:
            raise LqcdError(1, "block extents %s do not tile the lattice" % (tuple(bs),))
        its = np.zeros(nb, dtype=np.int32)
        rr = np.zeros(nb)
        sts = np.zeros(nb, dtype=np.int32)
        p = BlockParams((C.c_int * 4)(*bs), tol, nmx)
        st = lib().lqcd_block_solve(self._h, C.byref(p), _ptr(eta), _ptr(psi),
                                    its.ctypes.data_as(C.POINTER(C.c_int)), rr.ctypes.data_as(C.POINTER(C.c_double)),
                                    sts.ctypes.data_as(C.POINTER(C.c_int)))
        if check:
            self._check(st, "block_solve")
        return psi, st, its, rr, sts

    def apply_W(self, x: torch.Tensor, dm: float, prec=F64) -> torch.Tensor:
        """Hasenbusch operator W(dm) = Q_S + dm on even fields (Eq. 3)."""
        x = x.to(_dtype(prec)).contiguous()
        out = torch.empty_like(x)
        self._check(lib().lqcd_apply_W(self._h, prec, float(dm), _ptr(x), _ptr(out), self._nrhs(x, self.Vh)),
                    "apply_W")
        return out

    def solve_W(self, eta, dm, solver=SOLVER_SAP_GCR, tol=1e-10, nkv=16, nmx=4096, bs=(4, 4, 4, 4), ncy=4, nmr=5,
                sap_prec=F64, inner=F64, check=True, krylov=F64):
        eta = eta.to(torch.complex128).contiguous()
        nrhs = self._nrhs(eta, self.Vh)
        psi = torch.empty_like(eta)
        p = SolverParams(solver, nkv, nmx, tol, sap_params(bs, ncy, nmr, sap_prec), inner, krylov)
        info = (SolveInfo * nrhs)()
        st = lib().lqcd_solve_W(self._h, C.byref(p), float(dm), _ptr(eta), _ptr(psi), nrhs, info)
        if check:
            self._check(st, "solve_W")
        return psi, [i.as_dict() for i in info], st

    def solve_D(self, eta, solver=SOLVER_SAP_GCR, tol=1e-10, nkv=16, nmx=4096, bs=(4, 4, 4, 4), ncy=4, nmr=5,
                sap_prec=F64, inner=F64, check=True, krylov=F64):
        return self._solve(lib().lqcd_solve_D, eta, self.V, solver, tol, nkv, nmx, bs, ncy, nmr, sap_prec, inner,
                           check, krylov)


class Batch:
    """Several lattices (Contexts with clover terms) solved together by the
    batched SAP-GCR: one launch per phase over all lattices' work items."""

    def __init__(self, ctxs, nkv=16, nmx=4096, tol=1e-10, bs=(4, 4, 4, 4), ncy=4, nmr=5, sap_prec=F16S,
                 use_graph=True, wait_timeout_s=2.0, stall_test=False, stream=None):
        self.ctxs = list(ctxs)
        n = len(self.ctxs)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        p = BatchParams(nkv, nmx, tol, sap_params(bs, ncy, nmr, sap_prec), 1 if use_graph else 0,
                        wait_timeout_s, 1 if stall_test else 0)
        arr = (C.c_void_p * n)(*[c._h for c in self.ctxs])
        h = C.c_void_p()
        st = lib().lqcd_batch_create(arr, n, C.byref(p), C.c_void_p(stream.cuda_stream), C.byref(h))
        if st != 0:
            msg = lib().lqcd_last_error(self.ctxs[0]._h)
            raise LqcdError(st, f"lqcd_batch_create: {msg.decode() if msg else ''}")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lqcd_batch_destroy(self._h)
            self._h = None

    def solve_dhat(self, etas, check=False):
        """etas: one canonical even FP64 field per lattice; returns (psis, infos, status)."""
        etas = [e.to(torch.complex128).contiguous() for e in etas]
        psis = [torch.empty_like(e) for e in etas]
        n = len(etas)
        assert n == len(self.ctxs)
        ea = (C.c_void_p * n)(*[e.data_ptr() for e in etas])
        pa = (C.c_void_p * n)(*[x.data_ptr() for x in psis])
        info = (SolveInfo * n)()
        st = lib().lqcd_batch_solve_dhat(self._h, ea, pa, info)
        if check and st != 0:
            msg = lib().lqcd_batch_last_error(self._h)
            raise LqcdError(st, f"batch solve: {msg.decode() if msg else ''}")
        return psis, [i.as_dict() for i in info], st

    def last_error(self) -> str:
        msg = lib().lqcd_batch_last_error(self._h)
        return msg.decode() if msg else ""

    def stats(self):
        cy, rp, ln = C.c_int(), C.c_int(), C.c_long()
        lib().lqcd_batch_stats(self._h, C.byref(cy), C.byref(rp), C.byref(ln))
        return {"cycles": cy.value, "graph_replays": rp.value, "launches": ln.value}
