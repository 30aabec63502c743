"""Shared set-up of the GPU parity tests: one synthetic lattice seen by both
the CUDA library (through the C ABI) and the CPU oracle."""
from __future__ import annotations

import functools

import numpy as np
import torch

import oracle as orc
from paper_1011_0911_gb300 import lqcd, synth
from tests import util

# relative-error bounds per application (float storage vs FP64 oracle)
TOL = {lqcd.F64: 1e-13, lqcd.F32: 1e-6, lqcd.F16S: 3e-3}


@functools.lru_cache(maxsize=8)
def links(dims, seed=0):
    return synth.su3_links(dims, seed)


class Pair:
    def __init__(self, dims, kappa=0.1355, csw=1.9, seed=0, U=None):
        self.dims = dims
        self.U = links(dims, seed) if U is None else U
        self.o = orc.Oracle(dims, self.U, kappa, csw)
        assert self.o.status == 0
        self.ctx = lqcd.Context(dims)
        self.ctx.set_gauge(torch.from_numpy(self.U).cuda())
        self.logdet = self.ctx.clover_invert(kappa, csw)
        self.V, self.Vh = self.o.V, self.o.Vh
        self.ev, self.od = util.even_odd_sites(dims)


def to_gpu(x: np.ndarray, prec=lqcd.F64) -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(x))
    return t.to(torch.complex128 if prec == lqcd.F64 else torch.complex64).cuda()


def rounded(x: np.ndarray, prec) -> np.ndarray:
    """x as the library stores it at precision prec, back in complex128."""
    if prec in (lqcd.F32, lqcd.F16S):
        return x.astype(np.complex64).astype(np.complex128)
    return x


def relerr(gpu: torch.Tensor, ref: np.ndarray) -> float:
    return util.relerr(gpu.detach().cpu().numpy().astype(np.complex128).reshape(ref.shape), ref)
