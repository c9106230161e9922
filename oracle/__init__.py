"""Plain FP64 CPU oracle for arXiv 1701.02324 (TEST INFRASTRUCTURE ONLY).

The oracle is the independent reference the CUDA path is checked against.
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library: the C
source ``kf_oracle.c`` is compiled here with gcc (``-ffp-contract=off``) into
``oracle/_build/libkforacle.so`` and wrapped with ctypes.

Parity pins (tests/test_oracle_pins.py) tie every function to facts the paper
or mathematics fix: the dense Cholesky solve in the full-rank case, the dense
inverse of the assembled K~, the SMW identity (Eq. e:smw), the push-through
form of Eq. (e:invtelescope), the log^2 N predecessor (Sec. V, Table 2: same
factorization up to roundoff), the h -> 0 and h -> infinity limits of
Eq. (e:gaussian), and finite differences for the gradients.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kf_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libkforacle.so")
_lock = threading.Lock()
_lib = None

KFO_OK, KFO_EINVAL, KFO_EILLCOND = 0, 1, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP, no FMA contraction)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    src_m = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "kf_oracle.h")))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < src_m:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P, I32, I64, U64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        sig = {
            "kfo_create": (P, [P, I64, I32, I32]),
            "kfo_free": (None, [P]),
            "kfo_depth": (I32, [P]),
            "kfo_perm": (None, [P, P]),
            "kfo_node_range": (None, [P, I32, P, P]),
            "kfo_sample": (I32, [P, I32, I32, U64, P]),
            "kfo_skeletonize": (I32, [P, D, D, I32, I32, U64]),
            "kfo_rank": (I32, [P, I32]),
            "kfo_ncols": (I32, [P, I32]),
            "kfo_skel": (None, [P, I32, P]),
            "kfo_P": (None, [P, I32, P]),
            "kfo_set_id": (I32, [P, I32, I32, P, P]),
            "kfo_P_full": (None, [P, I32, P]),
            "kfo_factorize": (I32, [P, D, I32]),
            "kfo_Phat": (None, [P, I32, P]),
            "kfo_Z": (None, [P, I32, P]),
            "kfo_Phat_forms": (I32, [P, I32, P, P]),
            "kfo_solve": (I32, [P, P, P, I32]),
            "kfo_matvec": (I32, [P, P, P, I32]),
            "kfo_grad": (I32, [P, P, P, P, P, P]),
            "kfo_subtrees": (I32, [P, P, I32, D, D, I32, I32, U64, D]),
            "kfo_hybrid": (I32, [P, I32, D, D, I32, I32, U64, D]),
            "kfo_hybrid_solve": (I32, [P, P, P]),
            "kfo_hybrid_matvec": (I32, [P, P, P]),
            "kfo_splitmix64": (U64, [U64]),
            "kfo_knn": (I32, [P, I32, I32, I32, U64, P]),
            "kfo_set_near": (I32, [P, P, I32, I32]),
            "kfo_node_near": (I32, [P, I32, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def splitmix64(x: int) -> int:
    return int(_load().kfo_splitmix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


class Oracle:
    """One problem: tree, skeletons and factorization held by the C oracle."""

    def __init__(self, X: np.ndarray, m: int):
        self._lib = _load()
        X = np.ascontiguousarray(X, dtype=np.float64)
        self.N, self.d = X.shape
        self.m = int(m)
        self._h = self._lib.kfo_create(_ptr(X), self.N, self.d, self.m)
        if not self._h:
            raise ValueError("oracle: invalid tree arguments")
        self.D = int(self._lib.kfo_depth(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.kfo_free(h)
            self._h = None

    # ---- tree -------------------------------------------------------------
    @property
    def nnodes(self) -> int:
        return (1 << (self.D + 1)) - 1

    def perm(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.int64)
        self._lib.kfo_perm(self._h, _ptr(out))
        return out

    def node_range(self, a: int):
        lo, hi = ctypes.c_int64(), ctypes.c_int64()
        self._lib.kfo_node_range(self._h, a, ctypes.byref(lo), ctypes.byref(hi))
        return lo.value, hi.value

    def is_leaf(self, a: int) -> bool:
        return a >= (1 << self.D)

    def sample(self, a: int, n_samp: int, seed: int) -> np.ndarray:
        out = np.empty(max(n_samp, 1), dtype=np.int64)
        k = self._lib.kfo_sample(self._h, a, n_samp, ctypes.c_uint64(seed), _ptr(out))
        return out[:k].copy()

    # ---- near-field sampling -------------------------------------------------
    def knn(self, kappa: int, ntrees: int, leaf: int, seed: int) -> np.ndarray:
        """kappa nearest tree positions of every point by randomized
        projection trees (N x kappa int64, -1 padding)."""
        out = np.empty((self.N, kappa), dtype=np.int64)
        if self._lib.kfo_knn(self._h, int(kappa), int(ntrees), int(leaf), ctypes.c_uint64(seed), _ptr(out)) != KFO_OK:
            raise ValueError("oracle knn: bad arguments")
        return out

    def set_near(self, nbr, near_cap: int = 0):
        """Near-field sampling from the neighbour lists nbr (None: uniform)."""
        if nbr is None:
            self._lib.kfo_set_near(self._h, None, 0, 0)
            return
        nbr = np.ascontiguousarray(nbr, dtype=np.int64)
        if self._lib.kfo_set_near(self._h, _ptr(nbr), nbr.shape[1], int(near_cap)) != KFO_OK:
            raise ValueError("oracle set_near: bad arguments")

    def node_near(self, a: int):
        """The node's near list (positions) and counts."""
        cap = 4096
        pos = np.empty(cap, dtype=np.int64)
        cnt = np.empty(cap, dtype=np.int32)
        n = int(self._lib.kfo_node_near(self._h, a, _ptr(pos), _ptr(cnt)))
        return pos[:n].copy(), cnt[:n].copy()

    # ---- skeletons ----------------------------------------------------------
    def skeletonize(self, h: float, tau: float, s_max: int, n_samp: int | None = None, seed: int = 0x1701):
        if n_samp is None:
            n_samp = 2 * s_max
        self.h, self.tau, self.s_max = float(h), float(tau), int(s_max)
        st = self._lib.kfo_skeletonize(self._h, float(h), float(tau), int(s_max), int(n_samp), ctypes.c_uint64(seed))
        if st != KFO_OK:
            raise ValueError(f"oracle skeletonize status {st}")

    def rank(self, a: int) -> int:
        return int(self._lib.kfo_rank(self._h, a))

    def ncols(self, a: int) -> int:
        return int(self._lib.kfo_ncols(self._h, a))

    def skel(self, a: int) -> np.ndarray:
        out = np.empty(max(self.rank(a), 1), dtype=np.int64)
        self._lib.kfo_skel(self._h, a, _ptr(out))
        return out[: self.rank(a)].copy()

    def P(self, a: int) -> np.ndarray:
        s, c = self.rank(a), self.ncols(a)
        out = np.empty(max(s * c, 1))
        self._lib.kfo_P(self._h, a, _ptr(out))
        return out[: s * c].reshape(s, c).copy()

    def P_full(self, a: int) -> np.ndarray:
        lo, hi = self.node_range(a)
        s = self.rank(a)
        out = np.empty(max((hi - lo) * s, 1))
        self._lib.kfo_P_full(self._h, a, _ptr(out))
        return out[: (hi - lo) * s].reshape(hi - lo, s).copy()

    def set_id(self, a: int, skel: np.ndarray, P: np.ndarray):
        skel = np.ascontiguousarray(skel, dtype=np.int64)
        P = np.ascontiguousarray(P, dtype=np.float64)
        st = self._lib.kfo_set_id(self._h, a, len(skel), _ptr(skel), _ptr(P))
        if st != KFO_OK:
            raise ValueError(f"oracle set_id status {st}")

    def subtrees(self, roots, h: float, tau: float, s_max: int, lam: float, n_samp: int | None = None,
                 seed: int = 0x1701) -> int:
        """Algorithms 1 and 2 on the disjoint subtrees under ``roots`` only
        (the nodes there get the values a whole run gives them)."""
        if n_samp is None:
            n_samp = 2 * s_max
        r = np.ascontiguousarray(roots, dtype=np.int32)
        self.h, self.tau, self.s_max, self.lam = float(h), float(tau), int(s_max), float(lam)
        st = self._lib.kfo_subtrees(self._h, _ptr(r), len(r), float(h), float(tau), int(s_max), int(n_samp),
                                    ctypes.c_uint64(seed), float(lam))
        if st not in (KFO_OK, KFO_EILLCOND):
            raise ValueError(f"oracle subtrees status {st}")
        return int(st)

    # ---- hybrid level-restricted solver (Sec. II-C, Algorithms 6-8) ----------
    def hybrid(self, L: int, h: float, tau: float, s_max: int, lam: float, n_samp: int | None = None,
               seed: int = 0x1701) -> int:
        """Frontier at level L: subtrees below it compressed and factorized,
        the reduced system I + VW of the frontier skeletons factored."""
        if n_samp is None:
            n_samp = 2 * s_max
        self.h, self.tau, self.s_max, self.lam = float(h), float(tau), int(s_max), float(lam)
        st = self._lib.kfo_hybrid(self._h, int(L), float(h), float(tau), int(s_max), int(n_samp),
                                  ctypes.c_uint64(seed), float(lam))
        if st not in (KFO_OK, KFO_EILLCOND):
            raise ValueError(f"oracle hybrid status {st}")
        return int(st)

    def hybrid_solve(self, b: np.ndarray) -> np.ndarray:
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty(self.N)
        if self._lib.kfo_hybrid_solve(self._h, _ptr(b), _ptr(x)) != KFO_OK:
            raise ValueError("oracle: hybrid_solve needs kfo_hybrid first")
        return x

    def hybrid_matvec(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.N)
        if self._lib.kfo_hybrid_matvec(self._h, _ptr(x), _ptr(y)) != KFO_OK:
            raise ValueError("oracle: hybrid_matvec needs kfo_hybrid first")
        return y

    # ---- factorization ------------------------------------------------------
    def factorize(self, lam: float, variant: int = 0) -> int:
        self.lam = float(lam)
        return int(self._lib.kfo_factorize(self._h, float(lam), int(variant)))

    def Phat(self, a: int) -> np.ndarray:
        lo, hi = self.node_range(a)
        s = self.rank(a)
        out = np.empty(max((hi - lo) * s, 1))
        self._lib.kfo_Phat(self._h, a, _ptr(out))
        return out[: (hi - lo) * s].reshape(hi - lo, s).copy()

    def Z(self, a: int) -> np.ndarray:
        z = self.rank(2 * a) + self.rank(2 * a + 1)
        out = np.empty(max(z * z, 1))
        self._lib.kfo_Z(self._h, a, _ptr(out))
        return out[: z * z].reshape(z, z).copy()

    def Phat_forms(self, a: int):
        lo, hi = self.node_range(a)
        s = self.rank(a)
        lit = np.empty(max((hi - lo) * s, 1))
        push = np.empty(max((hi - lo) * s, 1))
        st = self._lib.kfo_Phat_forms(self._h, a, _ptr(lit), _ptr(push))
        if st != KFO_OK:
            raise ValueError("oracle: Phat_forms needs a factorized internal non-root node")
        n = (hi - lo) * s
        return lit[:n].reshape(hi - lo, s).copy(), push[:n].reshape(hi - lo, s).copy()

    # ---- solve / matvec / gradient -------------------------------------------
    def solve(self, b: np.ndarray, transpose: bool = False) -> np.ndarray:
        b = np.asarray(b, dtype=np.float64)
        if b.ndim == 2:
            return np.stack([self.solve(b[:, j], transpose) for j in range(b.shape[1])], axis=1)
        b = np.ascontiguousarray(b)
        x = np.empty(self.N)
        st = self._lib.kfo_solve(self._h, _ptr(b), _ptr(x), int(bool(transpose)))
        if st != KFO_OK:
            raise ValueError(f"oracle solve status {st}")
        return x

    def matvec(self, x: np.ndarray, deriv_h: bool = False) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        if x.ndim == 2:
            return np.stack([self.matvec(x[:, j], deriv_h) for j in range(x.shape[1])], axis=1)
        x = np.ascontiguousarray(x)
        y = np.empty(self.N)
        st = self._lib.kfo_matvec(self._h, _ptr(x), _ptr(y), int(bool(deriv_h)))
        if st != KFO_OK:
            raise ValueError(f"oracle matvec status {st}")
        return y

    def grad(self, x: np.ndarray, g: np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        db = np.empty(self.N)
        dl, dh = ctypes.c_double(), ctypes.c_double()
        st = self._lib.kfo_grad(self._h, _ptr(x), _ptr(g), _ptr(db), ctypes.byref(dl), ctypes.byref(dh))
        if st != KFO_OK:
            raise ValueError(f"oracle grad status {st}")
        return db, dl.value, dh.value

    def residual(self, b: np.ndarray, x: np.ndarray) -> float:
        """epsilon_r = ||u - (lambda I + K~) w|| / ||u||, Eq. (e:errors)."""
        r = b - self.matvec(x)
        return float(np.linalg.norm(r) / np.linalg.norm(b))

    def dense_Ktilde(self) -> np.ndarray:
        """lambda I + K~ assembled column by column through the matvec (small N)."""
        I = np.eye(self.N)
        return np.stack([self.matvec(I[:, j]) for j in range(self.N)], axis=1)
