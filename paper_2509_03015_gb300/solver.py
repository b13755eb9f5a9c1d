"""PyTorch-facing binding of the C ABI.  PyTorch supplies device memory and
the CUDA stream; every step of the factorisation and solve runs in the
library's kernels."""
from __future__ import annotations

import ctypes

import torch

from . import _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(None)


def _check_tensor(t, name, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.device.type != "cuda" or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


class Solver:
    """Handle over one block-tridiagonal shape (N blocks of n x n, up to
    d_max right-hand-side columns).  precision: "fp64", "fp32_ir", "tf32_ir"."""

    def __init__(self, N, n, d_max=1, precision="fp64", stream=None, persistent=True, timeout_ms=None):
        self.lib = _lib.load()
        self.N, self.n, self.d_max, self.precision = int(N), int(n), int(d_max), precision
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = self.lib.bdss_create(ctypes.byref(h), self.N, self.n, self.d_max, _lib.PRECISIONS[precision],
                                  ctypes.c_void_p(self.stream.cuda_stream))
        _lib.check(st, "bdss_create")
        self.h = h
        self._keep = None
        if not persistent:
            self.set_option("persistent", 0)
        if timeout_ms is not None:
            self.set_option("timeout_ms", timeout_ms)

    def set_option(self, key, value):
        _lib.check(self.lib.bdss_set_option(self.h, _lib.OPTIONS[key], int(value)), "bdss_set_option")

    def _shapes(self, d):
        N, n = self.N, self.n
        return (N, n, n), (max(N - 1, 0), n, n), (N, n, d)

    def factor(self, A_diag, A_sub):
        sd, ss, _ = self._shapes(1)
        _check_tensor(A_diag, "A_diag", sd)
        if self.N > 1:
            _check_tensor(A_sub, "A_sub", ss)
        info = _lib.bdss_info()
        st = self.lib.bdss_factor(self.h, _ptr(A_diag), _ptr(A_sub if self.N > 1 else None), ctypes.byref(info))
        _lib.check(st, "bdss_factor", info)
        self._keep = (A_diag, A_sub)  # the mixed modes read A again in solve
        return info

    def solve(self, B, X=None):
        _check_tensor(B, "B")
        d = B.shape[-1]
        _, _, sb = self._shapes(d)
        _check_tensor(B, "B", sb)
        if X is None:
            X = torch.empty_like(B)
        _check_tensor(X, "X", sb)
        info = _lib.bdss_info()
        st = self.lib.bdss_solve(self.h, _ptr(B), _ptr(X), d, ctypes.byref(info))
        _lib.check(st, "bdss_solve", info)
        self.last_info = info
        return X

    def factor_solve(self, A_diag, A_sub, B, X=None):
        sd, ss, _ = self._shapes(1)
        _check_tensor(A_diag, "A_diag", sd)
        if self.N > 1:
            _check_tensor(A_sub, "A_sub", ss)
        d = B.shape[-1]
        _check_tensor(B, "B", self._shapes(d)[2])
        if X is None:
            X = torch.empty_like(B)
        _check_tensor(X, "X", self._shapes(d)[2])
        info = _lib.bdss_info()
        st = self.lib.bdss_factor_solve(self.h, _ptr(A_diag), _ptr(A_sub if self.N > 1 else None), _ptr(B),
                                        _ptr(X), d, ctypes.byref(info))
        _lib.check(st, "bdss_factor_solve", info)
        self._keep = (A_diag, A_sub)
        self.last_info = info
        return X

    def logdet(self):
        out = ctypes.c_double()
        _lib.check(self.lib.bdss_logdet(self.h, ctypes.byref(out)), "bdss_logdet")
        return out.value

    def launch_stats(self):
        k, b = ctypes.c_int64(), ctypes.c_int64()
        _lib.check(self.lib.bdss_last_launch_stats(self.h, ctypes.byref(k), ctypes.byref(b)), "bdss_last_launch_stats")
        return k.value, b.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.bdss_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(A_diag, A_sub, B, precision="fp64"):
    """One-shot factor + solve of A X = B on the GPU."""
    N, n, _ = A_diag.shape
    s = Solver(N, n, d_max=B.shape[-1], precision=precision)
    try:
        return s.factor_solve(A_diag, A_sub, B)
    finally:
        s.close()
