"""PyTorch-facing binding of the C ABI.  PyTorch supplies device memory and
the CUDA stream; every step of the factorisation and solve runs in the
library's kernels."""
from __future__ import annotations

import ctypes

import torch

from . import _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(None)


def _check_tensor(t, name, shape=None, host_ok=False):
    """float64, contiguous, on the GPU -- or, for inputs (host_ok), in
    page-locked host memory, which the kernels read in place."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    on_host = host_ok and t.device.type == "cpu" and t.is_pinned()
    if (t.device.type != "cuda" and not on_host) or t.dtype != torch.float64 or not t.is_contiguous():
        where = "CUDA or pinned host" if host_ok else "CUDA"
        raise ValueError(f"{name} must be a contiguous float64 {where} tensor")
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
        _check_tensor(A_diag, "A_diag", sd, host_ok=True)
        if self.N > 1:
            _check_tensor(A_sub, "A_sub", ss, host_ok=True)
        info = _lib.bdss_info()
        st = self.lib.bdss_factor(self.h, _ptr(A_diag), _ptr(A_sub if self.N > 1 else None), ctypes.byref(info))
        _lib.check(st, "bdss_factor", info)
        self._keep = (A_diag, A_sub)  # the mixed modes read A again in solve
        return info

    def solve(self, B, X=None):
        _check_tensor(B, "B", host_ok=True)
        d = B.shape[-1]
        _, _, sb = self._shapes(d)
        _check_tensor(B, "B", sb, host_ok=True)
        if X is None:
            X = torch.empty(B.shape, dtype=B.dtype, device="cuda")
        _check_tensor(X, "X", sb)
        info = _lib.bdss_info()
        st = self.lib.bdss_solve(self.h, _ptr(B), _ptr(X), d, ctypes.byref(info))
        _lib.check(st, "bdss_solve", info)
        self.last_info = info
        return X

    def factor_solve(self, A_diag, A_sub, B, X=None):
        sd, ss, _ = self._shapes(1)
        _check_tensor(A_diag, "A_diag", sd, host_ok=True)
        if self.N > 1:
            _check_tensor(A_sub, "A_sub", ss, host_ok=True)
        d = B.shape[-1]
        _check_tensor(B, "B", self._shapes(d)[2], host_ok=True)
        if X is None:
            X = torch.empty(B.shape, dtype=B.dtype, device="cuda")
        _check_tensor(X, "X", self._shapes(d)[2])
        info = _lib.bdss_info()
        st = self.lib.bdss_factor_solve(self.h, _ptr(A_diag), _ptr(A_sub if self.N > 1 else None), _ptr(B),
                                        _ptr(X), d, ctypes.byref(info))
        _lib.check(st, "bdss_factor_solve", info)
        self._keep = (A_diag, A_sub)
        self.last_info = info
        return X

    def adjoint_grads(self, Lam, X):
        """dL/dA_diag, dL/dA_sub from the adjoint Lam = A^-1 dL/dX and X."""
        _check_tensor(Lam, "Lambda")
        _check_tensor(X, "X", tuple(Lam.shape))
        d = X.shape[-1]
        dA_diag = torch.empty((self.N, self.n, self.n), dtype=torch.float64, device=X.device)
        dA_sub = torch.empty((max(self.N - 1, 0), self.n, self.n), dtype=torch.float64, device=X.device)
        st = self.lib.bdss_adjoint_grads(self.h, _ptr(Lam), _ptr(X), d, _ptr(dA_diag),
                                         _ptr(dA_sub if self.N > 1 else None))
        _lib.check(st, "bdss_adjoint_grads")
        return dA_diag, dA_sub

    def logdet(self):
        out = ctypes.c_double()
        _lib.check(self.lib.bdss_logdet(self.h, ctypes.byref(out)), "bdss_logdet")
        return out.value

    def launch_stats(self):
        k, b = ctypes.c_int64(), ctypes.c_int64()
        _lib.check(self.lib.bdss_last_launch_stats(self.h, ctypes.byref(k), ctypes.byref(b)), "bdss_last_launch_stats")
        return k.value, b.value

    def refine_stats(self):
        """(plain corrections, preconditioned-CG iterations) of the last
        mixed-precision solve."""
        p, c = ctypes.c_int32(), ctypes.c_int32()
        _lib.check(self.lib.bdss_last_refine_stats(self.h, ctypes.byref(p), ctypes.byref(c)),
                   "bdss_last_refine_stats")
        return p.value, c.value

    def residual(self, B, X, R=None):
        """R = B - A X for the last factored A (the refinement's residual:
        on the tensor cores where the handle supports it, else FP64 ALU)."""
        _check_tensor(B, "B", host_ok=True)
        _check_tensor(X, "X", tuple(B.shape), host_ok=True)
        if R is None:
            R = torch.empty(B.shape, dtype=torch.float64, device="cuda")
        _check_tensor(R, "R", tuple(B.shape))
        _lib.check(self.lib.bdss_residual(self.h, _ptr(B), _ptr(X), B.shape[-1], _ptr(R)), "bdss_residual")
        return R

    def chunk_reduce(self, A_diag, A_sub, A_left, A_right, B):
        """Eliminate this handle's chunk interior (partitioned solve): returns
        S = [S_LL, S_RR, S_RL] (3, n, n) and b_hat = [b_L, b_R] (2, n, d), the
        interior's contribution to the reduced system of its separators.
        A_left / A_right: the n x n couplings to the left / right separator,
        or None."""
        sd, ss, _ = self._shapes(1)
        _check_tensor(A_diag, "A_diag", sd, host_ok=True)
        if self.N > 1:
            _check_tensor(A_sub, "A_sub", ss, host_ok=True)
        for t, nm in ((A_left, "A_left"), (A_right, "A_right")):
            if t is not None:
                _check_tensor(t, nm, (self.n, self.n), host_ok=True)
        d = B.shape[-1]
        _check_tensor(B, "B", self._shapes(d)[2], host_ok=True)
        S = torch.empty((3, self.n, self.n), dtype=torch.float64, device="cuda")
        bh = torch.empty((2, self.n, d), dtype=torch.float64, device="cuda")
        info = _lib.bdss_info()
        st = self.lib.bdss_chunk_reduce(self.h, _ptr(A_diag), _ptr(A_sub if self.N > 1 else None), _ptr(A_left),
                                        _ptr(A_right), _ptr(B), d, _ptr(S), _ptr(bh), ctypes.byref(info))
        _lib.check(st, "bdss_chunk_reduce", info)
        self._keep = (A_diag, A_sub)
        return S, bh

    def chunk_backsolve(self, B, A_left, A_right, x_left, x_right):
        """The chunk interior's solution once its separators' blocks are
        known (after chunk_reduce on this handle)."""
        d = B.shape[-1]
        _check_tensor(B, "B", self._shapes(d)[2], host_ok=True)
        X = torch.empty(B.shape, dtype=torch.float64, device="cuda")
        st = self.lib.bdss_chunk_backsolve(self.h, _ptr(B), _ptr(A_left), _ptr(A_right), _ptr(x_left),
                                           _ptr(x_right), d, _ptr(X))
        _lib.check(st, "bdss_chunk_backsolve")
        return X

    def tune_nstar(self, A_diag, A_sub, B, candidates=(1, 2, 4, 8, 16, 32, 64), reps=5):
        """Autotune the crossover N_* (Sec. 3.3 leaves it to be determined
        dynamically) on these inputs: every candidate the handle accepts is
        timed over `reps` factor + solve calls with CUDA events on the
        handle's stream, and the fastest is kept.  Returns (best, {N_*: ms})."""
        times = {}
        X = torch.empty(B.shape, dtype=torch.float64, device="cuda")
        for c in candidates:
            try:
                self.set_option("nstar", c)
            except _lib.BDSSError:
                continue
            self.factor_solve(A_diag, A_sub, B, X)  # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            for _ in range(reps):
                self.factor_solve(A_diag, A_sub, B, X)
            e1.record(self.stream)
            e1.synchronize()
            times[c] = e0.elapsed_time(e1) / reps
        best = min(times, key=times.get)
        self.set_option("nstar", best)
        return best, times

    def factor_shift(self):
        """Relative diagonal shift sigma of the stored factors (mixed
        precision; 0 unless the unshifted FP32 factorisation failed)."""
        out = ctypes.c_double()
        _lib.check(self.lib.bdss_factor_shift(self.h, ctypes.byref(out)), "bdss_factor_shift")
        return out.value

    def kernel_times(self):
        """{class: (ms, launches)} of the last call, timed with CUDA events on
        the handle's stream (set_option("kernel_timing", 1) first)."""
        k = len(_lib.KERNEL_CLASSES)
        ms = (ctypes.c_double * k)()
        n = (ctypes.c_int64 * k)()
        _lib.check(self.lib.bdss_last_kernel_times(self.h, ms, n, k), "bdss_last_kernel_times")
        return {c: (ms[i], n[i]) for i, c in enumerate(_lib.KERNEL_CLASSES)}

    def launch_config(self):
        """(resident CTAs per SM, SM count, dynamic shared memory bytes per
        CTA) of this handle's persistent kernel."""
        c, m, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _lib.check(self.lib.bdss_get_launch_config(self.h, ctypes.byref(c), ctypes.byref(m), ctypes.byref(b)),
                   "bdss_get_launch_config")
        return c.value, m.value, b.value

    @property
    def plan_levels(self):
        """Levels L with eliminations (N_{l+1} = ceil(N_l / 2) down to 1)."""
        L, m = 0, self.N
        while m > 1:
            m, L = (m + 1) // 2, L + 1
        return L

    def trace(self):
        """Barrier release times (ns, device clock) of the last persistent
        pass: start-up, then phase A / phase B of each level, then one per
        downward level (grid barriers; on the one-cluster path its cluster
        barriers, with one more stamp at the end)."""
        buf = (ctypes.c_int64 * 256)()
        cnt = ctypes.c_int32()
        _lib.check(self.lib.bdss_last_trace(self.h, buf, 256, ctypes.byref(cnt)), "bdss_last_trace")
        return [buf[i] for i in range(min(cnt.value, 256))]

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


class BlockTriSolve(torch.autograd.Function):
    """X = A^{-1} B for the SPD block-tridiagonal A(A_diag, A_sub), FP64.

    forward:  factor + solve (one persistent launch); the factors stay in a
              handle saved for backward.
    backward: the adjoint solve A Lam = dL/dX reuses the stored factors (A is
              symmetric), then dL/dB = Lam, dL/dA_ii = -sym(Lam_i X_i^T),
              dL/dA_{i+1,i} = -(Lam_{i+1} X_i^T + X_{i+1} Lam_i^T)."""

    @staticmethod
    def forward(ctx, A_diag, A_sub, B):
        N, n, _ = A_diag.shape
        d = B.shape[-1]
        solver = Solver(N, n, d_max=d, precision="fp64")
        X = solver.factor_solve(A_diag.contiguous(), A_sub.contiguous(), B.contiguous())
        ctx.solver = solver
        ctx.save_for_backward(X)
        return X

    @staticmethod
    def backward(ctx, gX):
        (X,) = ctx.saved_tensors
        solver = ctx.solver
        Lam = solver.solve(gX.contiguous())
        dA_diag, dA_sub = solver.adjoint_grads(Lam, X)
        solver.close()
        ctx.solver = None
        return dA_diag, dA_sub, Lam


def block_tri_solve(A_diag, A_sub, B):
    """Differentiable X = A^{-1} B (see BlockTriSolve)."""
    return BlockTriSolve.apply(A_diag, A_sub, B)


def kalman_assemble(G, H, Qinv, Rinv, z=None, zeta=None, stream=None):
    """Kalman-smoother normal equations (Sec. 4.2) assembled on the GPU:
    returns (A_diag, A_sub, B) ready for Solver.factor_solve, B of shape
    (N, n, 1), or None when z is None (matrix only).  G, Qinv: (N, n, n);
    H: (N, m, n); Rinv: (N, m, m), or (N, m) for diagonal precisions (their
    diagonals); z: (N, m); zeta: (N, n) or None for zero.  G[0] is not read."""
    lib = _lib.load()
    N, n, _ = G.shape
    m = H.shape[1]
    diag = Rinv.dim() == 2
    _check_tensor(G, "G", (N, n, n))
    _check_tensor(H, "H", (N, m, n))
    _check_tensor(Qinv, "Qinv", (N, n, n))
    _check_tensor(Rinv, "Rinv", (N, m) if diag else (N, m, m))
    if z is not None:
        _check_tensor(z, "z", (N, m))
        if zeta is not None:
            _check_tensor(zeta, "zeta", (N, n))
    dev = G.device
    A_diag = torch.empty((N, n, n), dtype=torch.float64, device=dev)
    A_sub = torch.empty((max(N - 1, 0), n, n), dtype=torch.float64, device=dev)
    B = torch.empty((N, n, 1), dtype=torch.float64, device=dev) if z is not None else None
    stream = stream if stream is not None else torch.cuda.current_stream(dev)
    st = lib.bdss_kalman_assemble(N, n, m, int(diag), _ptr(G), _ptr(H), _ptr(Qinv), _ptr(Rinv), _ptr(z), _ptr(zeta),
                                  _ptr(A_diag), _ptr(A_sub if N > 1 else None), _ptr(B),
                                  ctypes.c_void_p(stream.cuda_stream))
    _lib.check(st, "bdss_kalman_assemble")
    return A_diag, A_sub, B


class BatchSolver:
    """K independent FP64 systems of uneven (N_k, n_k), factored and solved in
    one launch (device work queue).  `systems` is a list of (A_diag, A_sub,
    B) CUDA float64 tensors; X_k are allocated unless given."""

    def __init__(self, systems, X=None, stream=None, autotune=0):
        self.lib = _lib.load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        K = len(systems)
        self.K = K
        self.systems = systems
        d = systems[0][2].shape[-1]
        Nk = (ctypes.c_int64 * K)(*[int(s[0].shape[0]) for s in systems])
        nk = (ctypes.c_int32 * K)(*[int(s[0].shape[1]) for s in systems])
        h = ctypes.c_void_p()
        _lib.check(self.lib.bdss_batch_create(ctypes.byref(h), K, Nk, nk, d, ctypes.c_void_p(self.stream.cuda_stream)),
                   "bdss_batch_create")
        self.h = h
        self.X = X if X is not None else [torch.empty_like(s[2]) for s in systems]
        arr = lambda ts: (ctypes.c_void_p * K)(*[t.data_ptr() if t is not None and t.numel() else None for t in ts])
        for (Ad, As, B), Xk in zip(systems, self.X):
            _check_tensor(Ad, "A_diag")
            _check_tensor(B, "B")
            _check_tensor(Xk, "X", tuple(B.shape))
            if Ad.shape[0] > 1:
                _check_tensor(As, "A_sub")
        _lib.check(self.lib.bdss_batch_set_inputs(self.h, arr([s[0] for s in systems]), arr([s[1] for s in systems]),
                                                  arr([s[2] for s in systems]), arr(self.X)), "bdss_batch_set_inputs")
        self.config = None
        if autotune:
            t, i = ctypes.c_int32(), ctypes.c_int32()
            _lib.check(self.lib.bdss_batch_autotune(self.h, int(autotune), ctypes.byref(t), ctypes.byref(i)),
                       "bdss_batch_autotune")
            self.config = (t.value, i.value)

    def launch(self, graph=False):
        _lib.check(self.lib.bdss_batch_launch(self.h, 1 if graph else 0), "bdss_batch_launch")

    def wait(self, raise_on_error=True):
        """Returns (per-instance status list, per-instance latency in us)."""
        info = (_lib.bdss_info * self.K)()
        lat = (ctypes.c_double * self.K)()
        st = self.lib.bdss_batch_wait(self.h, info, lat)
        self.info = info
        if raise_on_error:
            _lib.check(st, "bdss_batch_wait")
        return [info[k].reserved for k in range(self.K)], [lat[k] for k in range(self.K)]

    def run(self, graph=False):
        self.launch(graph)
        self.wait()
        return self.X

    def close(self):
        if getattr(self, "h", None):
            self.lib.bdss_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
