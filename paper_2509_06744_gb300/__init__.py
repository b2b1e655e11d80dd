"""GB300 multilevel solver for PUM discretisations of higher-order problems:
fourth-kind Chebyshev smoothing with (adaptive, nested) block-FSAI preconditioners.

Thin Python binding over the C-ABI of ``include/pum.h``: this module only marshals
arguments (torch CUDA tensors become device pointers); every step of the solver runs
in the library's CUDA kernels.  There is no CPU fallback: without the built library
or a CUDA device every call raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (PUM_BF16, PUM_F32, PUM_F64, PUM_MAT_A, PUM_MAT_A1, PUM_MAT_F0, PUM_MAT_G, PUM_MAT_G1,
                   PUM_MAT_GT, PUM_MAT_P, PUM_P0_DIAG, PUM_P0_LOWER)

__all__ = ["Context", "Hierarchy", "PumError", "make_workers", "setup_batch", "solve_batch", "solve_batch_multi", "init_mlp", "PUM_F64", "PUM_F32", "PUM_BF16", "PUM_P0_LOWER", "PUM_P0_DIAG",
           "PUM_MAT_A", "PUM_MAT_P", "PUM_MAT_G", "PUM_MAT_GT", "PUM_MAT_F0", "PUM_MAT_G1", "PUM_MAT_A1"]

_DT = {"f64": PUM_F64, "f32": PUM_F32, "bf16": PUM_BF16}
_SMOOTHER = {"cheb4": 0, "richardson": 1}   # PUM_SMOOTHER_*
_CYCLE = {"vkk": 0, "v2k0": 1}             # PUM_CYCLE_*


class PumError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _vec(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Context:
    """A CUDA device and the stream the library's kernels run on (pum_create / pum_destroy).

    By default the library runs on torch's current stream of that device, so its
    kernels are ordered with the torch operations that allocate, fill and read the
    vectors passed to it (and torch's caching allocator never recycles a buffer that a
    queued kernel still reads).  `stream` is a raw cudaStream_t handle.
    """

    def __init__(self, device: int = 0, stream: int | None = None):
        self.lib = _lib.load()
        if stream is None:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream(device).cuda_stream
                if stream == 0:
                    stream = _lib.CUDA_STREAM_LEGACY
        h = C.c_void_p()
        st = self.lib.pum_create(C.byref(h), device, C.c_void_p(stream) if stream else None)
        if st != 0:
            raise PumError(st, "pum_create failed (is a CUDA device present?)")
        self.h = h
        self.device = device

    def check(self, st: int):
        if st != 0:
            raise PumError(st, self.lib.pum_last_error(self.h).decode())

    def sync(self):
        self.check(self.lib.pum_sync(self.h))

    def close(self):
        if self.h:
            self.lib.pum_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    TK = {"resid": 0, "g": 1, "gt": 2, "pcg_ap": 3, "resid64": 4, "adapt": 5, "factor": 6}

    def timing(self, enable, classes=None):
        """Enable per-class kernel timing (all classes, or the named ones)."""
        mask = 0
        if enable:
            names = classes or list(self.TK)
            for n in names:
                mask |= 1 << self.TK[n]
        self.check(self.lib.pum_timing_enable(self.h, mask))

    def timing_reset(self):
        self.check(self.lib.pum_timing_reset(self.h))

    def timing_read(self):
        n = (C.c_int64 * _lib.PUM_TK_COUNT)()
        ms = (C.c_double * _lib.PUM_TK_COUNT)()
        self.check(self.lib.pum_timing_read(self.h, n, ms))
        names = ["resid", "g", "gt", "pcg_ap", "resid64", "adapt", "factor"]
        return {names[i]: (int(n[i]), float(ms[i])) for i in range(_lib.PUM_TK_COUNT)}

    @property
    def launches(self) -> int:
        return int(self.lib.pum_launch_count(self.h))

    # ---- learned candidate scoring (pum_mlp_*; weights as a dict of float32 numpy arrays)
    def mlp_forward(self, model: dict, x):
        """Logits of the feature rows x (float32 CUDA tensor, n x 12)."""
        import torch
        m = mlp_struct(model)
        out = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        self.check(self.lib.pum_mlp_forward(self.h, C.byref(m), _fvec(x, "x"), x.shape[0], _fvec(out, "out")))
        return out

    def mlp_grad(self, model: dict, x, y):
        m, g, loss = mlp_struct(model), _lib.Mlp(), C.c_double()
        self.check(self.lib.pum_mlp_grad(self.h, C.byref(m), _fvec(x, "x"), _fvec(y, "y"), x.shape[0],
                                         C.byref(loss), C.byref(g)))
        return loss.value, mlp_dict(g)

    def mlp_train(self, model: dict, x, y, epochs=8, batch=8192, lr=3e-3, seed=0):
        """Adam on the device; returns (trained model, mean loss over all samples)."""
        m, loss = mlp_struct(model), C.c_double()
        self.check(self.lib.pum_mlp_train(self.h, C.byref(m), _fvec(x, "x"), _fvec(y, "y"), x.shape[0], epochs,
                                          batch, lr, seed, C.byref(loss)))
        return mlp_dict(m), loss.value

    def set_pattern_model(self, model: dict | None):
        if model is None:
            self.check(self.lib.pum_set_pattern_model(self.h, None))
        else:
            m = mlp_struct(model)
            self.check(self.lib.pum_set_pattern_model(self.h, C.byref(m)))


_MLP_SHAPES = {"w1": (64, 12), "b1": (64,), "w2": (64, 64), "b2": (64,), "w3": (64,), "b3": ()}


def init_mlp(seed: int) -> dict:
    """Initial weights of the candidate-scoring network: He-normal (seeded), zero biases, FP32."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x1EA]))
    f32 = np.float32
    return {"w1": (rng.standard_normal((64, 12)) * np.sqrt(2.0 / 12)).astype(f32), "b1": np.zeros(64, f32),
            "w2": (rng.standard_normal((64, 64)) * np.sqrt(2.0 / 64)).astype(f32), "b2": np.zeros(64, f32),
            "w3": (rng.standard_normal(64) * np.sqrt(1.0 / 64)).astype(f32), "b3": np.zeros((), f32)}


def mlp_struct(model: dict) -> "_lib.Mlp":
    m = _lib.Mlp()
    for name, shape in _MLP_SHAPES.items():
        v = np.ascontiguousarray(np.asarray(model[name], dtype=np.float32).reshape(shape))
        if name == "b3":
            m.b3 = float(v.reshape(-1)[0])
        else:
            C.memmove(getattr(m, name), v.ctypes.data, v.nbytes)
    return m


def mlp_dict(m) -> dict:
    out = {}
    for name, shape in _MLP_SHAPES.items():
        out[name] = np.float32(m.b3) if name == "b3" else np.ctypeslib.as_array(getattr(m, name)).reshape(shape).copy()
    return out


def _fvec(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _bsr_view(indptr, indices, blocks, n_cols):
    indptr = np.ascontiguousarray(indptr, dtype=np.int32)
    indices = np.ascontiguousarray(indices, dtype=np.int32)
    blocks = np.ascontiguousarray(blocks, dtype=np.float64)
    v = _lib.BsrView(len(indptr) - 1, n_cols, blocks.shape[1] if blocks.ndim == 3 else 0, len(indices),
                     indptr.ctypes.data, indices.ctypes.data, blocks.ctypes.data, 0)
    return v, (indptr, indices, blocks)


def _setup_params(p0="lower", adaptive=False, t_max=0, tau=1.0, nested=False, tie_rel=1e-9, k=2, lanczos_its=100,
                  lanczos_safety=1.01, lanczos_seed=0, smooth="f64", g=None, mixed_levels=64, fp32_levels=64,
                  smoother="cheb4", cycle="vkk"):
    fp = _lib.FsaiParams(PUM_P0_LOWER if p0 == "lower" else PUM_P0_DIAG, int(adaptive), t_max, tau, int(nested),
                         tie_rel)
    sp = _lib.SmootherParams(k, lanczos_its, lanczos_safety, lanczos_seed, _DT[smooth], _DT[g or smooth],
                             int(mixed_levels), int(fp32_levels), _SMOOTHER[smoother], _CYCLE[cycle])
    return fp, sp


def make_workers(n: int, device: int = 0):
    """n contexts on n new streams of `device`, for setup_batch / solve_batch (each batch worker
    needs its own stream).  Synchronise torch's stream before handing them vectors it wrote."""
    import torch
    out = []
    for _ in range(n):
        s = torch.cuda.Stream(device)
        c = Context(device, stream=s.cuda_stream)
        c._torch_stream = s  # keep the stream alive with the context
        out.append(c)
    return out


def setup_batch(workers, hierarchies, **setup_kwargs):
    """bfsai_setup of distinct hierarchies concurrently, one host thread per worker Context."""
    fp, sp = _setup_params(**setup_kwargs)
    n = len(hierarchies)
    wa = (C.c_void_p * len(workers))(*[w.h for w in workers])
    ha = (C.c_void_p * n)(*[h.h for h in hierarchies])
    st = (C.c_int32 * n)()
    rc = workers[0].lib.pum_setup_batch(wa, len(workers), ha, n, C.byref(fp), C.byref(sp), st)
    if rc != 0:
        bad = next((i for i in range(n) if st[i] != 0), None)
        if bad is None:
            raise PumError(rc, "batch arguments (distinct hierarchies; workers on distinct streams)")
        raise PumError(int(st[bad]), f"batch set-up of item {bad}")
    return [int(v) for v in st]


def solve_batch_multi(workers, items, rtol: float = 1e-8, maxit: int = 200, flexible: bool = False):
    """items: [(Hierarchy, B, X), ...] with B, X float64 CUDA tensors of shape (nrhs, N_i) (the same
    nrhs for all); each hierarchy solves its columns at once (pcg_solve_multi), the hierarchies
    concurrently on the workers.  Returns per item a list of report dicts."""
    n = len(items)
    nrhs = items[0][1].shape[0]
    wa = (C.c_void_p * len(workers))(*[w.h for w in workers])
    ha = (C.c_void_p * n)(*[it[0].h for it in items])
    ba = (C.c_void_p * n)(*[_vec(it[1], "B").value for it in items])
    xa = (C.c_void_p * n)(*[_vec(it[2], "X").value for it in items])
    hists = [(C.c_double * (maxit + 1))() for _ in range(n * nrhs)]
    reps = (_lib.PcgReport * (n * nrhs))(*[_lib.PcgReport(rtol, maxit, int(flexible), hh, 0, 0, 0.0) for hh in hists])
    st = (C.c_int32 * n)()
    rc = workers[0].lib.pum_solve_batch_multi(wa, len(workers), ha, n, nrhs, ba, xa, reps, st)
    if rc != 0:
        bad = next((i for i in range(n) if st[i] != 0), None)
        raise PumError(rc if bad is None else int(st[bad]), f"batch multi-RHS solve (item {bad})")
    return [[{"iters": reps[i * nrhs + c].iters, "converged": bool(reps[i * nrhs + c].converged)}
             for c in range(nrhs)] for i in range(n)]


def solve_batch(workers, items, rtol: float = 1e-8, maxit: int = 200, flexible: bool = False,
                method: str = "pcg", allow_noconv=False):
    """items: [(Hierarchy, b, x), ...]; solves them concurrently on the workers' streams (items of
    one hierarchy in order on one worker).  Returns one report dict per item."""
    n = len(items)
    wa = (C.c_void_p * len(workers))(*[w.h for w in workers])
    ha = (C.c_void_p * n)(*[it[0].h for it in items])
    ba = (C.c_void_p * n)(*[_vec(it[1], "b") for it in items])
    xa = (C.c_void_p * n)(*[_vec(it[2], "x") for it in items])
    hists = [(C.c_double * (maxit + 1))() for _ in range(n)]
    reps = (_lib.PcgReport * n)()
    for i in range(n):
        reps[i] = _lib.PcgReport(rtol, maxit, int(flexible), hists[i], 0, 0, 0.0)
    st = (C.c_int32 * n)()
    rc = workers[0].lib.pum_solve_batch(wa, len(workers), ha, n, ba, xa, reps, {"pcg": 0, "bicgstab": 1}[method], st)
    for i in range(n):
        if not (st[i] == 0 or (allow_noconv and st[i] == _lib.PUM_ERR_NOCONV)):
            raise PumError(st[i], f"batch item {i}")
    if rc == _lib.PUM_ERR_INVALID_ARG:
        raise PumError(rc, "batch arguments (workers need distinct contexts on distinct streams)")
    return [{"iters": reps[i].iters, "converged": bool(reps[i].converged), "final_relres": reps[i].final_relres,
             "history": [hists[i][j] for j in range(reps[i].iters + 1)]} for i in range(n)]


class Hierarchy:
    """Level hierarchy {A_l, P_l, G_l, beta_l} owned by the library (pum_hier).

    setup, pcg, bicgstab and convergence_factor return once the work is done and raise on a
    device-side status; cheb4_smooth, vcycle and the single steps only queue their kernels on
    the context's stream: Context.sync() waits for them and raises on a device-side status (a
    bounded wait that expired)."""

    def __init__(self, ctx: Context, handle: C.c_void_p):
        self.ctx, self.h, self.lib = ctx, handle, ctx.lib

    # ---- construction
    @classmethod
    def assemble(cls, ctx: Context, equation: int, p: int, finest_m: int, n_levels: int, f_coef=None,
                 f_decay: float = 2.0, nitsche=(0.0, 0.0, 0.0), quad_pts: int = 0, b=None, aniso=None):
        """aniso: (S11, S12, S22) of the anisotropy tensor of Example 5.2 (biharmonic only)."""
        pr = _lib.Problem()
        pr.equation, pr.p, pr.finest_m, pr.n_levels = equation, p, finest_m, n_levels
        for j in range(3):
            pr.nitsche_c[j] = float(nitsche[j]) if j < len(nitsche) else 0.0
        pr.quad_pts = quad_pts
        for j in range(3):
            pr.aniso[j] = float(aniso[j]) if aniso is not None else 0.0
        keep = None
        if f_coef is not None:
            keep = np.ascontiguousarray(f_coef, dtype=np.float64)
            pr.f_coef, pr.f_modes, pr.f_decay = keep.ctypes.data, keep.shape[0], f_decay
        h = C.c_void_p()
        ctx.check(ctx.lib.pum_assemble(ctx.h, C.byref(pr), C.byref(h), _vec(b, "b") if b is not None else None))
        del keep
        return cls(ctx, h)

    @classmethod
    def from_bsr(cls, ctx: Context, A_levels, P_levels):
        """A_levels: list of (indptr, indices, blocks) or None (Galerkin); P_levels: list of
        (indptr, indices, blocks, n_coarse_block_cols)."""
        keep = []
        nl = len(A_levels)
        av = (_lib.BsrView * nl)()
        for l, a in enumerate(A_levels):
            if a is None:
                av[l] = _lib.BsrView(0, 0, 0, 0, None, None, None, 0)
            else:
                v, k = _bsr_view(a[0], a[1], a[2], len(a[0]) - 1)
                av[l] = v
                keep.append(k)
        pv = (_lib.BsrView * max(nl - 1, 1))()
        for l, pm in enumerate(P_levels):
            v, k = _bsr_view(pm[0], pm[1], pm[2], pm[3])
            pv[l] = v
            keep.append(k)
        h = C.c_void_p()
        ctx.check(ctx.lib.pum_hier_from_bsr(ctx.h, nl, av, pv, C.byref(h)))
        return cls(ctx, h)

    @classmethod
    def load(cls, ctx: Context, path: str):
        h = C.c_void_p()
        ctx.check(ctx.lib.pum_hier_load(ctx.h, path.encode(), C.byref(h)))
        return cls(ctx, h)

    def save(self, path: str):
        self.ctx.check(self.lib.pum_hier_save(self.ctx.h, self.h, path.encode()))

    def setup(self, p0: str = "lower", adaptive: bool | int = False, t_max: int = 0, tau: float = 1.0,
              nested: bool = False, tie_rel: float = 1e-9, k: int = 2, lanczos_its: int = 100,
              lanczos_safety: float = 1.01, lanczos_seed: int = 0, smooth: str = "f64", g: str | None = None,
              mixed_levels: int = 64, fp32_levels: int = 64, smoother: str = "cheb4", cycle: str = "vkk"):
        fp, sp = _setup_params(p0, adaptive, t_max, tau, nested, tie_rel, k, lanczos_its, lanczos_safety, lanczos_seed,
                               smooth, g, mixed_levels, fp32_levels, smoother, cycle)
        self.ctx.check(self.lib.bfsai_setup(self.ctx.h, self.h, C.byref(fp), C.byref(sp)))

    def close(self):
        if self.h:
            self.lib.pum_hier_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- hot path
    def cheb4_smooth(self, level: int, b, x, x_is_zero: bool):
        self.ctx.check(self.lib.cheb4_smooth(self.ctx.h, self.h, level, _vec(b, "b"), _vec(x, "x"), int(x_is_zero)))

    def vcycle(self, r, z):
        self.ctx.check(self.lib.vcycle_apply(self.ctx.h, self.h, _vec(r, "r"), _vec(z, "z")))

    def pcg(self, b, x, rtol: float = 1e-8, maxit: int = 200, flexible: bool = False, allow_noconv=False):
        return self._krylov(self.lib.pcg_solve, b, x, rtol, maxit, flexible, allow_noconv)

    def bicgstab(self, b, x, rtol: float = 1e-8, maxit: int = 200, allow_noconv=False):
        """BiCGStab with the cycle as right preconditioner (for the non-symmetric V(2k,0))."""
        return self._krylov(self.lib.bicgstab_solve, b, x, rtol, maxit, False, allow_noconv)

    def _krylov(self, fn, b, x, rtol, maxit, flexible, allow_noconv):
        hist = (C.c_double * (maxit + 1))()
        rep = _lib.PcgReport(rtol, maxit, int(flexible), hist, 0, 0, 0.0)
        st = fn(self.ctx.h, self.h, _vec(b, "b"), _vec(x, "x"), C.byref(rep))
        if not (st == 0 or (allow_noconv and st == _lib.PUM_ERR_NOCONV)):
            self.ctx.check(st)
        return {"iters": rep.iters, "converged": bool(rep.converged), "final_relres": rep.final_relres,
                "history": [hist[i] for i in range(rep.iters + 1)]}

    def pcg_multi(self, B, X, rtol: float = 1e-8, maxit: int = 200, flexible: bool = False, allow_noconv=False):
        """PCG for the rows of B (float64 CUDA tensor of shape (nrhs, N), one right-hand side per
        row) at once into X (same shape); one report dict per right-hand side."""
        nrhs = B.shape[0]
        hists = [(C.c_double * (maxit + 1))() for _ in range(nrhs)]
        reps = (_lib.PcgReport * nrhs)(*[_lib.PcgReport(rtol, maxit, int(flexible), hh, 0, 0, 0.0) for hh in hists])
        st = self.lib.pcg_solve_multi(self.ctx.h, self.h, nrhs, _vec(B, "B"), _vec(X, "X"), reps)
        if not (st == 0 or (allow_noconv and st == _lib.PUM_ERR_NOCONV)):
            self.ctx.check(st)
        return [{"iters": r.iters, "converged": bool(r.converged), "final_relres": r.final_relres,
                 "history": [hh[i] for i in range(r.iters + 1)]} for r, hh in zip(reps, hists)]

    def vcycle_multi(self, R, Z):
        """Z = the V(k,k) cycle applied to every row of R (shape (nrhs, N), float64 CUDA)."""
        self.ctx.check(self.lib.vcycle_apply_multi(self.ctx.h, self.h, R.shape[0], _vec(R, "R"), _vec(Z, "Z")))

    def convergence_factor(self, e0, n_cycles: int) -> float:
        """rho_A of the stationary cycle from the error e0 (the measure of the paper's figures)."""
        rho = C.c_double(0.0)
        self.ctx.check(self.lib.pum_convergence_factor(self.ctx.h, self.h, _vec(e0, "e0"), int(n_cycles),
                                                       C.byref(rho)))
        return rho.value

    # ---- single steps
    def residual(self, level, b, x, r):
        self.ctx.check(self.lib.pum_residual(self.ctx.h, self.h, level, _vec(b, "b"), _vec(x, "x"), _vec(r, "r")))

    def fsai_apply(self, level, r, z):
        self.ctx.check(self.lib.pum_fsai_apply(self.ctx.h, self.h, level, _vec(r, "r"), _vec(z, "z")))

    def restrict(self, level, r, rc):
        self.ctx.check(self.lib.pum_restrict(self.ctx.h, self.h, level, _vec(r, "r"), _vec(rc, "rc")))

    def prolong_add(self, level, e, x):
        self.ctx.check(self.lib.pum_prolong_add(self.ctx.h, self.h, level, _vec(e, "e"), _vec(x, "x")))

    def coarse_solve(self, r, z):
        self.ctx.check(self.lib.pum_coarse_solve(self.ctx.h, self.h, _vec(r, "r"), _vec(z, "z")))

    # ---- inspection
    @property
    def n_levels(self) -> int:
        n = C.c_int32()
        self.ctx.check(self.lib.pum_hier_levels(self.h, C.byref(n)))
        return n.value

    def info(self, level: int) -> dict:
        li = _lib.LevelInfo()
        self.ctx.check(self.lib.pum_level_info_get(self.h, level, C.byref(li)))
        return {f: getattr(li, f) for f, _ in _lib.LevelInfo._fields_}

    def candidates(self, level: int):
        """Candidates of a set-up level (pum_fsai_candidates), copied into torch CUDA tensors:
        row, col (int32), x (float32, n x 12), y (float32 labels)."""
        import torch
        c = _lib.Candidates()
        self.ctx.check(self.lib.pum_fsai_candidates(self.ctx.h, self.h, level, C.byref(c)))
        try:
            n = int(c.n)
            row = torch.empty(n, dtype=torch.int32, device="cuda")
            col = torch.empty(n, dtype=torch.int32, device="cuda")
            x = torch.empty((n, 12), dtype=torch.float32, device="cuda")
            y = torch.empty(n, dtype=torch.float32, device="cuda")
            self.ctx.check(self.lib.pum_candidates_copy(self.ctx.h, C.byref(c), C.c_void_p(row.data_ptr()),
                                                        C.c_void_p(col.data_ptr()), C.c_void_p(x.data_ptr()),
                                                        C.c_void_p(y.data_ptr())))
            self.ctx.sync()
            return {"row": row, "col": col, "x": x, "y": y}
        finally:
            self.lib.pum_candidates_free(C.byref(c))

    def export(self, level: int, which: int):
        """Host copy (indptr, indices, blocks) of a level's matrix, float64."""
        m = _lib.BsrHost()
        self.ctx.check(self.lib.pum_hier_export(self.ctx.h, self.h, level, which, C.byref(m)))
        try:
            n, nnzb, d = m.n_brows, m.nnzb, m.bs
            indptr = np.ctypeslib.as_array(m.row_ptr, shape=(n + 1,)).copy()
            indices = np.ctypeslib.as_array(m.col_idx, shape=(max(nnzb, 1),))[:nnzb].copy()
            blocks = np.ctypeslib.as_array(m.vals, shape=(max(nnzb * d * d, 1),))[:nnzb * d * d].copy()
            return indptr.astype(np.int64), indices.astype(np.int64), blocks.reshape(nnzb, d, d), m.n_bcols
        finally:
            self.lib.pum_bsr_free(C.byref(m))
