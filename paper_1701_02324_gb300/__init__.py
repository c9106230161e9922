"""GB300-native hierarchical factorization and solve of lambda*I + K.

Thin Python binding of the C ABI in ``include/kf.h`` (Yu, March, Biros,
"An N log N Parallel Fast Direct Solver for Kernel Matrices", arXiv
1701.02324).  Every step of the method runs in the CUDA library
``libkf.so``; this module only passes pointers, sizes and the current CUDA
stream, and routes device allocations of the library through PyTorch's
caching allocator.  There is no CPU fallback: without the library or a GPU
the calls raise.

Same names as the C ABI: ``tree_build``, ``factorize``, ``solve``,
``matvec``, ``grad``, ``factor_free``/``tree_free``; ``Tree`` and ``Factor``
wrap the handles, ``KernelSolve`` is the autograd function of
x = (lambda I + K~(h))^-1 b.
"""
from __future__ import annotations

import ctypes

from . import _abi
from ._abi import (KF_F32, KF_F64, KF_PREC_FP64, KF_PREC_MIXED, KF_V_RECOMPUTE, KF_V_STORED, KFError,
                   kf_opts, kf_solve_info)

__all__ = [
    "build", "Context", "Tree", "Factor", "tree_build", "factorize", "factorize_with_ids", "solve", "matvec",
    "grad", "tree_free", "factor_free", "KernelSolve", "KF_PREC_FP64", "KF_PREC_MIXED", "KF_V_STORED",
    "KF_V_RECOMPUTE", "KFError", "factorize_batched", "solve_batched", "autotune",
]


def build(force: bool = False) -> str:
    """Compile libkf.so for sm_103a (in-tree) and return its path."""
    from . import _build
    return _build.build(force=force)


def _torch():
    import torch
    return torch


def _stream_ptr():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


# ---- allocator: library allocations drawn from PyTorch's caching allocator --------
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


@_ALLOC_FN
def _torch_alloc(nbytes, stream, user):
    torch = _torch()
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
    except RuntimeError:
        return None


@_FREE_FN
def _torch_free(ptr, nbytes, stream, user):
    if ptr and _DELETE[0] is not None:
        try:
            _DELETE[0](int(ptr))
        except Exception:  # interpreter shutdown: the process is releasing everything anyway
            pass


_DELETE = [None]
# Set at interpreter exit (an atexit handler registered after torch is
# imported, so it runs before torch's own): from then on handles are not freed
# (the process releases the device memory) and the free callback does nothing,
# so that no call reaches torch or the CUDA runtime while they shut down.
_EXITING = [False]
_EXIT_HOOK = [False]


def _at_exit():
    _EXITING[0] = True
    _DELETE[0] = None


class Context:
    """A kf_ctx: error messages and the device allocator (torch's by default)."""

    def __init__(self, use_torch_allocator: bool = True):
        self.lib = _abi.load()
        self._alloc = None
        if not _EXIT_HOOK[0]:
            import atexit
            _torch()
            atexit.register(_at_exit)
            _EXIT_HOOK[0] = True
        if use_torch_allocator:
            _DELETE[0] = _torch().cuda.caching_allocator_delete
            self._alloc = _abi.kf_alloc(ctypes.cast(_torch_alloc, ctypes.c_void_p).value,
                                        ctypes.cast(_torch_free, ctypes.c_void_p).value, None)
        h = ctypes.c_void_p()
        _abi.check(self.lib.kf_create(ctypes.byref(h), ctypes.byref(self._alloc) if self._alloc else None))
        self.h = h

    def check(self, status, allow=()):
        return _abi.check(status, self.h, allow)

    def __del__(self):
        if getattr(self, "h", None) and not _EXITING[0]:
            self.lib.kf_destroy(self.h)
            self.h = None


_default_ctx = None


def default_context() -> Context:
    global _default_ctx
    if _default_ctx is None:
        _default_ctx = Context()
    return _default_ctx


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.float64:
        return KF_F64
    if t.dtype == torch.float32:
        return KF_F32
    raise TypeError("kf: tensors must be float32 or float64")


class Tree:
    """Ball tree of Sec. II-A over X (N x d, device or host tensor)."""

    def __init__(self, X, m: int, ctx: Context | None = None):
        torch = _torch()
        self.ctx = ctx or default_context()
        X = X.contiguous()
        self.N, self.d = X.shape
        self.m = int(m)
        h = ctypes.c_void_p()
        self.ctx.check(self.ctx.lib.kf_tree_build(self.ctx.h, _ptr(X), _dtype_code(X), self.N, self.d, self.m,
                                                  _stream_ptr(), ctypes.byref(h)))
        self.h = h
        D = ctypes.c_int32()
        self.ctx.lib.kf_tree_info(self.h, None, None, None, ctypes.byref(D))
        self.D = D.value
        self._X = X if X.is_cuda else None
        del torch

    @property
    def nnodes(self) -> int:
        return (1 << (self.D + 1)) - 1

    def perm(self):
        torch = _torch()
        out = torch.empty(self.N, dtype=torch.int64, device="cuda")
        self.ctx.check(self.ctx.lib.kf_tree_perm(self.h, _ptr(out), _stream_ptr()))
        return out

    def free(self):
        if getattr(self, "h", None) and not _EXITING[0]:
            self.ctx.lib.kf_tree_free(self.h)
            self.h = None

    def __del__(self):
        self.free()


def _opts(precision=KF_PREC_FP64, n_samp=0, seed=0, v_storage=KF_V_STORED, sync_errors=0, refine_tol=0.0,
          refine_max_iter=0, tensor_cores=True, fp64_operator=None, gmres_restart=0, cluster_kernels=True,
          tc_tile_n=0, zinv_max_nodes=0, hybrid_level=0, knn_kappa=0, knn_trees=0, knn_leaf=0, zoff_fused=False, w_recompute=False,
          tc_operator=False):
    o = kf_opts()
    o.zoff_fused = 1 if zoff_fused else 0
    o.tc_operator = 1 if tc_operator else 0
    o.w_recompute = 1 if w_recompute else 0
    o.hybrid_level = int(hybrid_level)
    o.knn_kappa, o.knn_trees, o.knn_leaf = int(knn_kappa), int(knn_trees), int(knn_leaf)
    o.zinv_max_nodes = int(zinv_max_nodes)
    o.no_cluster_kernels = 0 if cluster_kernels else 1
    o.tc_tile_n = int(tc_tile_n)
    o.no_tensor_cores = 0 if tensor_cores else 1
    o.fp64_operator = 0 if fp64_operator is None else (1 if fp64_operator is True else
                                                       (-1 if fp64_operator is False else int(fp64_operator)))
    o.gmres_restart = int(gmres_restart)
    o.precision, o.n_samp, o.seed, o.v_storage = int(precision), int(n_samp), int(seed), int(v_storage)
    o.sync_errors, o.refine_tol, o.refine_max_iter = int(sync_errors), float(refine_tol), int(refine_max_iter)
    return o


class Factor:
    """Skeletonization (Algorithm 1) + factorization (Algorithm 2) of lambda I + K~."""

    def __init__(self, tree: Tree, h: float, lam: float, tau: float, s_max: int, precision=KF_PREC_FP64,
                 n_samp: int = 0, seed: int = 0, v_storage=KF_V_STORED, refine_tol: float = 0.0,
                 refine_max_iter: int = 0, sync_errors: bool = True, tensor_cores: bool = True,
                 fp64_operator=None, gmres_restart: int = 0, cluster_kernels: bool = True, tc_tile_n: int = 0,
                 zinv_max_nodes: int = 0, hybrid_level: int = 0, knn_kappa: int = 0, knn_trees: int = 0,
                 knn_leaf: int = 0, zoff_fused: bool = False, w_recompute: bool = False, tc_operator: bool = False,
                 _ids=None):
        """hybrid_level = L >= 1: the hybrid level-restricted solver of
        Sec. II-C (Algorithms 6-8) with its frontier at tree level L; 0: the
        direct solver (Algorithms 2-3).  knn_kappa > 0: near-field sampling
        of S' from every point's knn_kappa nearest neighbours (knn_trees
        projection trees with leaves of knn_leaf points).  tc_operator: the
        mixed path's FP64-accurate operator keeps its V blocks as exact BF16
        digits as well, for tensor-core V passes over 16 or more columns."""
        self.tree, self.ctx = tree, tree.ctx
        self.h_, self.lam, self.tau, self.s_max, self.precision = float(h), float(lam), float(tau), int(s_max), precision
        self.hybrid_level = int(hybrid_level)
        self._knn_kappa, self._n_samp = int(knn_kappa), int(n_samp)
        o = _opts(precision, n_samp, seed, v_storage, int(sync_errors), refine_tol, refine_max_iter, tensor_cores,
                  fp64_operator, gmres_restart, cluster_kernels, tc_tile_n, zinv_max_nodes, hybrid_level, knn_kappa,
                  knn_trees, knn_leaf, zoff_fused, w_recompute, tc_operator)
        h_out = ctypes.c_void_p()
        if _ids is None:
            st = self.ctx.lib.kf_factorize(tree.h, self.h_, self.lam, self.tau, self.s_max, ctypes.byref(o),
                                           _stream_ptr(), ctypes.byref(h_out))
        else:
            ranks, skel, P = _ids
            st = self.ctx.lib.kf_factorize_with_ids(tree.h, self.h_, self.lam, self.s_max,
                                                    ranks.ctypes.data_as(ctypes.c_void_p),
                                                    skel.ctypes.data_as(ctypes.c_void_p),
                                                    P.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o),
                                                    _stream_ptr(), ctypes.byref(h_out))
        self.status = self.ctx.check(st, allow=(_abi.KF_EILLCOND,))
        self.h = h_out

    # -- operations ---------------------------------------------------------------
    def solve(self, B, transpose: bool = False, info: bool = False):
        """X = (lambda I + K~)^-1 B (or ^-T); B: N or N x k tensor (device or host)."""
        torch = _torch()
        vec = B.dim() == 1
        Bm = B.reshape(B.shape[0], -1)
        Bc = Bm.t().contiguous()            # column-major N x k
        X = torch.empty_like(Bc)
        inf = kf_solve_info() if info else None
        self.ctx.check(self.ctx.lib.kf_solve(self.h, _ptr(Bc), _ptr(X), Bm.shape[1], self.tree.N, _dtype_code(Bc),
                                             int(bool(transpose)), _stream_ptr(),
                                             ctypes.byref(inf) if inf is not None else None))
        out = X.t()
        out = out.reshape(B.shape) if vec else out
        if info:
            return out, {"eps_r": inf.eps_r, "iters": inf.iters, "status": inf.status}
        return out

    def matvec(self, Xv):
        torch = _torch()
        vec = Xv.dim() == 1
        Xm = Xv.reshape(Xv.shape[0], -1)
        Xc = Xm.t().contiguous()
        Y = torch.empty_like(Xc)
        self.ctx.check(self.ctx.lib.kf_matvec(self.h, _ptr(Xc), _ptr(Y), Xm.shape[1], self.tree.N, _dtype_code(Xc),
                                              _stream_ptr()))
        out = Y.t()
        return out.reshape(Xv.shape) if vec else out

    def grad(self, x, dLdx):
        """(dL/db, dL/dlambda, dL/dh) for x = (lambda I + K~)^-1 b, FP64 tensors."""
        torch = _torch()
        vec = x.dim() == 1
        xm = x.reshape(x.shape[0], -1).t().contiguous().to(torch.float64)
        gm = dLdx.reshape(dLdx.shape[0], -1).t().contiguous().to(torch.float64)
        db = torch.empty_like(gm)
        dl, dh = ctypes.c_double(), ctypes.c_double()
        self.ctx.check(self.ctx.lib.kf_grad(self.h, _ptr(xm), _ptr(gm), _ptr(db), ctypes.byref(dl), ctypes.byref(dh),
                                            xm.shape[0], self.tree.N, _stream_ptr()))
        db = db.t()
        return (db.reshape(x.shape) if vec else db), dl.value, dh.value

    # -- inspection -----------------------------------------------------------------
    def ranks(self):
        import numpy as np
        r = np.zeros(self.tree.nnodes + 1, dtype=np.int32)
        self.ctx.check(self.ctx.lib.kf_factor_ranks(self.h, r.ctypes.data_as(ctypes.c_void_p), _stream_ptr()))
        return r

    def skeleton(self, node: int):
        import numpy as np
        s = int(self.ranks()[node])
        out = np.zeros(max(s, 1), dtype=np.int64)
        self.ctx.check(self.ctx.lib.kf_factor_skeleton(self.h, node, out.ctypes.data_as(ctypes.c_void_p),
                                                       _stream_ptr()))
        return out[:s]

    def P(self, node: int, ncols: int):
        import numpy as np
        s = int(self.ranks()[node])
        out = np.zeros(max(s * ncols, 1))
        self.ctx.check(self.ctx.lib.kf_factor_P(self.h, node, out.ctypes.data_as(ctypes.c_void_p), _stream_ptr()))
        return out[: s * ncols].reshape(s, ncols)

    def Phat(self, node: int, nrows: int):
        import numpy as np
        s = int(self.ranks()[node])
        out = np.zeros(max(s * nrows, 1))
        self.ctx.check(self.ctx.lib.kf_factor_Phat(self.h, node, out.ctypes.data_as(ctypes.c_void_p), _stream_ptr()))
        return out[: s * nrows].reshape(nrows, s)

    def knn(self):
        """Every point's neighbour list of near-field sampling (N x kappa tree positions, -1 padding)."""
        import numpy as np
        kappa = self._kappa()
        out = np.zeros((self.tree.N, kappa), dtype=np.int32)
        self.ctx.check(self.ctx.lib.kf_factor_knn(self.h, out.ctypes.data_as(ctypes.c_void_p), _stream_ptr()))
        return out

    def near(self, node: int):
        """A node's near-field list: positions and counts."""
        import numpy as np
        cap = max(1, (self._n_samp or 2 * self.s_max) // 2)
        pos = np.zeros(cap, dtype=np.int32)
        cnt = np.zeros(cap, dtype=np.int32)
        n = ctypes.c_int32()
        self.ctx.check(self.ctx.lib.kf_factor_near(self.h, int(node), pos.ctypes.data_as(ctypes.c_void_p),
                                                   cnt.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n),
                                                   _stream_ptr()))
        return pos[:n.value].copy(), cnt[:n.value].copy()

    def _kappa(self):
        return self._knn_kappa

    def pivot_ratios(self):
        """Smallest/largest pivot of every node's leaf Cholesky or Z LU."""
        import numpy as np
        r = np.zeros(self.tree.nnodes + 1)
        self.ctx.check(self.ctx.lib.kf_factor_pivot_ratios(self.h, r.ctypes.data_as(ctypes.c_void_p), _stream_ptr()))
        return r

    def device_status(self):
        return self.ctx.lib.kf_factor_status(self.h, _stream_ptr())

    def free(self):
        if getattr(self, "h", None) and not _EXITING[0]:
            self.ctx.lib.kf_factor_free(self.h)
            self.h = None

    def __del__(self):
        self.free()


# ---- function-style names of the C ABI ------------------------------------------------
def tree_build(X, m: int, ctx: Context | None = None) -> Tree:
    return Tree(X, m, ctx)


def factorize(tree: Tree, h: float, lam: float, tau: float, s_max: int, **kw) -> Factor:
    return Factor(tree, h, lam, tau, s_max, **kw)


def factorize_with_ids(tree: Tree, h: float, lam: float, s_max: int, ranks, skel, P, **kw) -> Factor:
    return Factor(tree, h, lam, 0.0, s_max, _ids=(ranks, skel, P), **kw)


def solve(factor: Factor, B, transpose: bool = False):
    return factor.solve(B, transpose)


def matvec(factor: Factor, X):
    return factor.matvec(X)


def grad(factor: Factor, x, dLdx):
    return factor.grad(x, dLdx)


def tree_free(tree: Tree):
    tree.free()


def factor_free(factor: Factor):
    factor.free()


def _ptr_array(vals):
    arr = (ctypes.c_void_p * len(vals))(*vals)
    return arr


def autotune(tree: Tree, h: float, lam: float, tau: float, s_max: int, precision=KF_PREC_MIXED, **kw):
    """Pick the kernel variants for factorizations like this one
    (kf_autotune): returns the fastest candidate's keyword options for
    Factor / factorize_batched, and every candidate's time in ms."""
    o = _opts(precision, kw.get("n_samp", 0), kw.get("seed", 0), KF_V_STORED, 0, 0.0, -1,
              fp64_operator=kw.get("fp64_operator"))
    best = kf_opts()
    ms = (ctypes.c_float * 8)()
    nc = ctypes.c_int32()
    tree.ctx.check(tree.ctx.lib.kf_autotune(tree.h, float(h), float(lam), float(tau), int(s_max), ctypes.byref(o),
                                            _stream_ptr(), ctypes.byref(best), ms, ctypes.byref(nc)))
    chosen = {"cluster_kernels": not best.no_cluster_kernels, "tensor_cores": not best.no_tensor_cores,
              "tc_tile_n": int(best.tc_tile_n)}
    return chosen, [float(ms[i]) for i in range(nc.value)]


def factorize_batched(trees, hs, lams, taus, s_max: int, precision=KF_PREC_MIXED, n_samp: int = 0, seed: int = 0,
                      refine_tol: float = 0.0, refine_max_iter: int = 0, **kw):
    """Factorize many independent problems with one CUDA-graph launch
    (kf_factorize_batched).  Returns a list of Factor objects.  Their solves
    (solve_batched) are refined like kf_solve's: by default on the mixed path
    (refine_max_iter = 0), never with refine_max_iter = -1."""
    import numpy as np
    n = len(trees)
    ctx = trees[0].ctx
    h = np.ascontiguousarray(hs, dtype=np.float64)
    lam = np.ascontiguousarray(lams, dtype=np.float64)
    tau = np.ascontiguousarray(taus, dtype=np.float64)
    o = _opts(precision, n_samp, seed, KF_V_STORED, 0, refine_tol, refine_max_iter,
              tensor_cores=kw.get("tensor_cores", True), fp64_operator=kw.get("fp64_operator"),
              gmres_restart=kw.get("gmres_restart", 0), cluster_kernels=kw.get("cluster_kernels", True),
              tc_tile_n=kw.get("tc_tile_n", 0), zinv_max_nodes=kw.get("zinv_max_nodes", 0),
              tc_operator=kw.get("tc_operator", False))
    out = (ctypes.c_void_p * n)()
    tarr = _ptr_array([t.h.value for t in trees])
    st = ctx.lib.kf_factorize_batched(tarr, n, h.ctypes.data_as(ctypes.c_void_p), lam.ctypes.data_as(ctypes.c_void_p),
                                      tau.ctypes.data_as(ctypes.c_void_p), int(s_max), ctypes.byref(o), _stream_ptr(),
                                      out)
    ctx.check(st, allow=(_abi.KF_EILLCOND,))
    facs = []
    for i in range(n):
        F = Factor.__new__(Factor)
        F.tree, F.ctx = trees[i], ctx
        F.h_, F.lam, F.tau, F.s_max, F.precision = float(h[i]), float(lam[i]), float(tau[i]), int(s_max), precision
        F.status = st
        F.h = ctypes.c_void_p(out[i])
        facs.append(F)
    return facs


def solve_batched(factors, Bs, info: bool = False):
    """X_i = (lambda_i I + K~_i)^-1 B_i for every problem (kf_solve_batched):
    the direct sweeps in one CUDA-graph launch, refined as a batch when the
    factors refine.  B_i: device tensors N_i x k_i (float32/64).  With
    info=True returns (X, infos) with one {"eps_r", "iters", "status"} per
    problem, and a problem left above its refine_tol does not raise."""
    torch = _torch()
    n = len(factors)
    Bc = [B.reshape(B.shape[0], -1).t().contiguous() for B in Bs]
    Xc = [torch.empty_like(b) for b in Bc]
    nrhs = (ctypes.c_int64 * n)(*[b.shape[0] for b in Bc])
    ld = (ctypes.c_int64 * n)(*[f.tree.N for f in factors])
    ctx = factors[0].ctx
    inf = (kf_solve_info * n)()
    st = ctx.lib.kf_solve_batched(_ptr_array([f.h.value for f in factors]), n, _ptr_array([b.data_ptr() for b in Bc]),
                                  _ptr_array([x.data_ptr() for x in Xc]), nrhs, ld, _dtype_code(Bc[0]), _stream_ptr(),
                                  inf)
    ctx.check(st, allow=(_abi.KF_ENOTCONV,) if info else ())
    xs = [x.t().reshape(B.shape) for x, B in zip(Xc, Bs)]
    if info:
        return xs, [{"eps_r": r.eps_r, "iters": r.iters, "status": r.status} for r in inf]
    return xs


def _autograd():
    torch = _torch()

    class KernelSolve(torch.autograd.Function):
        """x = (lambda I + K~(h))^-1 b with gradients for b, lambda and h.

        The backward pass is the library's adjoint: one transpose solve for
        dL/db, and the sums -a.x and -a.(dK~/dh)x for lambda and h (skeletons
        and P held fixed)."""

        @staticmethod
        def forward(ctx, b, lam, h, factor):
            # The factorization fixes lambda and h; a solve with other values
            # would be stale while backward reported gradients at the values
            # passed in, so a mismatch is an error (refactorize instead).
            for name, given, held in (("lambda", lam, factor.lam), ("h", h, factor.h_)):
                v = float(given.detach().reshape(-1)[0]) if torch.is_tensor(given) else float(given)
                if torch.is_tensor(given) and given.numel() != 1:
                    raise ValueError(f"KernelSolve: {name} must be a scalar")
                if v != held:
                    raise ValueError(f"KernelSolve: {name}={v!r} differs from the factorization's {held!r}; "
                                     "factorize again with the new value")
            x = factor.solve(b)
            ctx.factor = factor
            ctx.lam_dtype = lam.dtype if torch.is_tensor(lam) else torch.float64
            ctx.h_dtype = h.dtype if torch.is_tensor(h) else torch.float64
            ctx.save_for_backward(x)
            return x

        @staticmethod
        def backward(ctx, gx):
            (x,) = ctx.saved_tensors
            db, dl, dh = ctx.factor.grad(x.to(torch.float64), gx.to(torch.float64))
            dev = gx.device
            return (db.to(gx.dtype), torch.tensor(dl, device=dev, dtype=ctx.lam_dtype),
                    torch.tensor(dh, device=dev, dtype=ctx.h_dtype), None)

    return KernelSolve


class _LazyAutograd:
    _cls = None

    def __getattr__(self, item):
        if _LazyAutograd._cls is None:
            _LazyAutograd._cls = _autograd()
        return getattr(_LazyAutograd._cls, item)


KernelSolve = _LazyAutograd()
