"""Python binding of the flip-free ADMM library: argument marshalling only.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); they are passed to the C ABI by pointer.  Names follow the paper:
V, T (source mesh), W (target vertices), U, P, Lambda (per-element splitting
variables), rho (penalty scale, mu_i = rho w_i).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as N

ENERGIES = {"sd": 0, "sg": 1, "sa": 2}
PRECISIONS = {"fp32": 0, "fp64": 1}
FACTORS = {"host": 0, "device": 1, "device64": 2}


def _torch():
    try:
        import torch
    except ImportError:  # pragma: no cover
        return None
    return torch


def _count_ok(size: int, count, what: str) -> None:
    if count is not None and size != count:
        raise ValueError(f"{what} has {size} entries, the call reads {count}")


def _ptr(a, dtype, count=None, what="array"):
    """Pointer of an input array (numpy array or torch tensor, host or CUDA) as
    a contiguous array of the given dtype, with `count` entries when given.

    For a CUDA tensor, the device is synchronized (every stream on it) before
    the pointer is handed over: the library works on its own stream, which does
    not wait for torch's, so this is what keeps it from reading the tensor
    before the work that writes it (a host-to-device copy, a kernel, or the
    dtype conversion done here) has finished.  The calls this module wraps
    synchronize the library's stream before they return successfully, so the
    array may be released once the call returns.  Returns (pointer, the array
    to keep alive during the call)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, dtype=dtype)
        _count_ok(a.size, count, what)
        return C.c_void_p(a.ctypes.data), a
    torch = _torch()
    if torch is not None and isinstance(a, torch.Tensor):
        tdt = torch.float64 if dtype == np.float64 else torch.int32
        if a.dtype != tdt or not a.is_contiguous():
            a = a.to(tdt).contiguous()
        _count_ok(a.numel(), count, what)
        if a.is_cuda:
            torch.cuda.synchronize(a.device)
        return C.c_void_p(a.data_ptr()), a
    a = np.ascontiguousarray(np.asarray(a), dtype=dtype)
    _count_ok(a.size, count, what)
    return C.c_void_p(a.ctypes.data), a


def _out(out, count: int, what: str):
    """Pointer of a caller's output buffer, which the library writes in place: a
    contiguous float64 numpy array or torch tensor (host or CUDA) of exactly
    `count` entries.  Anything else is refused rather than converted, since a
    converted copy would receive the results and drop them.  For a CUDA tensor,
    the device is synchronized first (see _ptr)."""
    if isinstance(out, np.ndarray):
        if out.dtype != np.float64 or not out.flags.c_contiguous or not out.flags.writeable:
            raise ValueError(f"{what} must be a writeable C-contiguous float64 array")
        _count_ok(out.size, count, what)
        return C.c_void_p(out.ctypes.data)
    torch = _torch()
    if torch is not None and isinstance(out, torch.Tensor):
        if out.dtype != torch.float64 or not out.is_contiguous():
            raise ValueError(f"{what} must be a contiguous float64 tensor")
        _count_ok(out.numel(), count, what)
        if out.is_cuda:
            torch.cuda.synchronize(out.device)
        return C.c_void_p(out.data_ptr())
    raise TypeError(f"{what} must be a numpy array or a torch tensor")


class Solver:
    """One mesh, one energy: setup once, then init / iterate.

    penalties="fixed": mu_i = rho w_i, L decomposed once; penalties="paper": the
    paper's schedule (initial mu_i = max(mu_min,i, w_i) and per-element rescaling by
    rescale_rho/2 at the paper's events, L decomposed again after each event).
    factor: where the numeric decomposition of L runs, "host" (double), "device"
    (float) or "device64" (double); the analysis is on the host either way.
    top_inverse_levels: the top levels of the elimination tree solved as
    x_T = S^-1 t_T between the triangular passes (0 off, -1 automatic, k > 0 exactly
    the top k levels)."""

    def __init__(self, V, T, pins=None, pin_pos=None, energy: str = "sd", rho: float = 1.0,
                 eps_abs: float = 1e-6, eps_rel: float = 1e-5, check_every: int = 10,
                 precision: str = "fp32", refine_sweeps: int = 2, leaf_size: int = 64,
                 require_flip_free: bool = True, host_threads: int = 0, schedule: int = 1,
                 penalties: str = "fixed", rescale_rho: float = 5.0, local_variant: str = "paper",
                 subtree_height=None, prox_h: bool = False, factor: str = "host", top_inverse_levels: int = 0,
                 stream=None):
        self._lib = N.load()
        self._ctx = None
        Vn = np.asarray(V) if isinstance(V, (list, tuple)) else V
        Tn = np.asarray(T) if isinstance(T, (list, tuple)) else T
        n, d_in = int(Vn.shape[0]), int(Vn.shape[1])
        m, d = int(Tn.shape[0]), int(Tn.shape[1]) - 1
        self.n, self.m, self.d, self.d_in = n, m, d, d_in
        pV, self._V = _ptr(Vn, np.float64)
        pT, self._T = _ptr(Tn, np.int32)
        mesh = N.Mesh(n, m, d, d_in, pV, pT)
        prm = N.Params()
        N.check(self._lib, None, self._lib.ffa_default_params(C.byref(prm)))
        prm.energy = ENERGIES[energy]
        prm.rho = float(rho)
        prm.eps_abs = float(eps_abs)
        prm.eps_rel = float(eps_rel)
        prm.check_every = int(check_every)
        prm.require_flip_free = 1 if require_flip_free else 0
        prm.local_precision = PRECISIONS[precision]
        prm.refine_sweeps = int(refine_sweeps)
        prm.nd_leaf_size = int(leaf_size)
        prm.host_threads = int(host_threads)
        prm.solve_schedule = int(schedule)
        if penalties not in ("fixed", "paper"):
            raise ValueError("penalties must be 'fixed' or 'paper'")
        prm.penalty_schedule = 1 if penalties == "paper" else 0
        prm.rescale_rho = float(rescale_rho)
        if local_variant not in ("paper", "joint"):
            raise ValueError("local_variant must be 'paper' or 'joint'")
        prm.local_variant = 1 if local_variant == "joint" else 0
        prm.prox_h = 1 if prox_h else 0
        if factor not in FACTORS:
            raise ValueError("factor must be one of " + ", ".join(FACTORS))
        prm.factor_device = FACTORS[factor]
        prm.top_inverse_levels = int(top_inverse_levels)
        if subtree_height is not None:   # (forward, backward) merged bottom subtree heights
            prm.solve_subtree_height[0], prm.solve_subtree_height[1] = (int(h) for h in subtree_height)
        n_pin = 0 if pins is None else int(len(pins))
        self.n_pin = max(n_pin, 1)
        pP, self._pins = _ptr(pins, np.int32) if n_pin else (None, None)
        pB, self._pinpos = _ptr(pin_pos, np.float64, n_pin * d, "pin_pos") if n_pin else (None, None)
        ctx = C.c_void_p()
        st = self._lib.ffa_create(C.byref(mesh), pP, n_pin, pB, C.byref(prm),
                                  C.c_void_p(stream) if stream else None, C.byref(ctx))
        N.check(self._lib, None, st)
        self._ctx = ctx
        self.energy_name = energy
        self.precision = precision

    # -- lifecycle ---------------------------------------------------------
    def close(self) -> None:
        if self._ctx is not None:
            self._lib.ffa_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int) -> None:
        N.check(self._lib, self._ctx, st)

    # -- the method ----------------------------------------------------------
    def set_handles(self, pin_pos) -> None:
        p, keep = _ptr(pin_pos, np.float64, self.n_pin * self.d, "pin_pos")
        self._check(self._lib.ffa_set_handles(self._ctx, p))

    def set_constraints(self, A, b) -> None:
        """General linear constraints A W = b on top of the pins (Sec. 4, W update):
        A is c x n (scipy sparse or dense), b is c x d.  Before init, once."""
        import scipy.sparse as sp
        A = sp.csr_matrix(A)
        A.sum_duplicates()
        b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(A.shape[0], -1))
        if A.shape[1] != self.n:
            raise ValueError(f"A has {A.shape[1]} columns, the mesh {self.n} vertices")
        ptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
        col = np.ascontiguousarray(A.indices, dtype=np.int32)
        val = np.ascontiguousarray(A.data, dtype=np.float64)
        self._check(self._lib.ffa_set_constraints(self._ctx, int(A.shape[0]), ptr.ctypes.data, col.ctypes.data,
                                                  val.ctypes.data, b.ctypes.data))

    def init(self, W0) -> None:
        p, keep = _ptr(W0, np.float64, self.n * self.d, "W0")
        self._check(self._lib.ffa_init(self._ctx, p))

    def iterate(self, max_iter: int, stop_at_tol: bool = True) -> dict:
        st = N.Stats()
        self._check(self._lib.ffa_iterate(self._ctx, int(max_iter), 1 if stop_at_tol else 0, C.byref(st)))
        return st.as_dict()

    def W(self, out=None):
        if out is None:
            out = np.empty((self.n, self.d), np.float64)
        po = _out(out, self.n * self.d, "out")
        self._check(self._lib.ffa_get_W(self._ctx, po))
        return out

    def state(self):
        U = np.empty((self.m, self.d, self.d))
        P = np.empty_like(U)
        L = np.empty_like(U)
        self._check(self._lib.ffa_get_state(self._ctx, C.c_void_p(U.ctypes.data), C.c_void_p(P.ctypes.data),
                                            C.c_void_p(L.ctypes.data)))
        return U, P, L

    def set_state(self, W, U, P, Lam) -> None:
        """Resume from (W, U, P, Lambda) instead of init (W n x d; U, P, Lambda m x d x d)."""
        mdd = self.m * self.d * self.d
        keep = [_ptr(a, np.float64, c, w) for a, c, w in ((W, self.n * self.d, "W"), (U, mdd, "U"), (P, mdd, "P"),
                                                          (Lam, mdd, "Lambda"))]
        self._check(self._lib.ffa_set_state(self._ctx, *(k[0] for k in keep)))

    def penalties(self) -> np.ndarray:
        """The current penalties mu_i (m values)."""
        out = np.empty(self.m, np.float64)
        po = _out(out, self.m, "out")
        self._check(self._lib.ffa_get_penalties(self._ctx, po))
        return out

    def energy(self, W=None) -> float:
        p, keep = _ptr(W, np.float64, self.n * self.d, "W")
        E = C.c_double()
        self._check(self._lib.ffa_energy(self._ctx, p, C.byref(E)))
        return E.value

    def gradient(self, W=None, out=None):
        p, keep = _ptr(W, np.float64, self.n * self.d, "W")
        if out is None:
            out = np.empty((self.n, self.d), np.float64)
        po = _out(out, self.n * self.d, "out")
        self._check(self._lib.ffa_gradient(self._ctx, p, po))
        return out

    def info(self) -> dict:
        inf = N.Info()
        self._check(self._lib.ffa_get_info(self._ctx, C.byref(inf)))
        return inf.as_dict()

    def autotune(self, reps: int = 5) -> dict:
        t = N.Tuning()
        self._check(self._lib.ffa_autotune(self._ctx, int(reps), C.byref(t)))
        return t.as_dict()

    def profile_phases(self, reps: int) -> dict:
        t = N.PhaseTimes()
        self._check(self._lib.ffa_profile_phases(self._ctx, int(reps), C.byref(t)))
        return t.as_dict()

    def forward_unrolled(self, K: int, ckpt_every: int = 20) -> None:
        """K iterations from the state set by init(), keeping checkpoints for backward_unrolled."""
        self._check(self._lib.ffa_forward_unrolled(self._ctx, int(K), int(ckpt_every)))

    def backward_unrolled(self, dL_dW, out=None):
        """dL/db for the pinned positions b, given dL/dW^K of the last forward_unrolled."""
        p, keep = _ptr(dL_dW, np.float64, self.n * self.d, "dL_dW")
        if out is None:
            out = np.empty((self.n_pin, self.d), np.float64)
        po = _out(out, self.n_pin * self.d, "out")
        self._check(self._lib.ffa_backward_unrolled(self._ctx, p, po))
        return out

    def factor_blocks(self) -> np.ndarray:
        """The float blocks B_s of the current decomposition of L_FF, concatenated as
        the W-step passes read them (ffa_copy_factor)."""
        n = int(self.info()["factor_entries"])
        out = np.empty(n, np.float32)
        self._check(self._lib.ffa_copy_factor(self._ctx, out.ctypes.data, n))
        return out

    def set_wait_limit(self, polls: int) -> None:
        """Polls of an empty queue slot before a W-step wait gives up (FFA_ERR_TIMEOUT)."""
        self._check(self._lib.ffa_set_wait_limit(self._ctx, int(polls)))

    def wstep_residual(self) -> float:
        r = C.c_double()
        self._check(self._lib.ffa_last_wstep_residual(self._ctx, C.byref(r)))
        return r.value

    @classmethod
    def from_workload(cls, wl, **kw):
        kw.setdefault("energy", wl.energy)
        kw.setdefault("rho", wl.rho)
        kw.setdefault("eps_abs", wl.eps_abs)
        kw.setdefault("eps_rel", wl.eps_rel)
        return cls(wl.V, wl.T, wl.pins, wl.pin_pos, **kw)


def tutte(V, T, boundary, boundary_pos, leaf_size: int = 64, host_threads: int = 0, schedule: int = 1,
          factor: str = "host", stream=None, out=None):
    """The minimizer of Tutte's energy with the boundary held (ffa_tutte).

    Returns (W, relative residual); W is a new (n, d) float64 array unless `out`
    (host array or device tensor) is given."""
    lib = N.load()
    Vn = np.asarray(V) if isinstance(V, (list, tuple)) else V
    Tn = np.asarray(T) if isinstance(T, (list, tuple)) else T
    n, d_in = int(Vn.shape[0]), int(Vn.shape[1])
    m, d_t = int(Tn.shape[0]), int(Tn.shape[1])
    bp = np.asarray(boundary_pos) if isinstance(boundary_pos, (list, tuple)) else boundary_pos
    d = int(bp.shape[1])
    if d_t != d + 1:
        raise ValueError("boundary_pos has d columns and T must have d + 1")
    pV, kV = _ptr(Vn, np.float64)
    pT, kT = _ptr(Tn, np.int32)
    pb, kb = _ptr(boundary, np.int32)
    pp, kp = _ptr(bp, np.float64, len(kb) * d, "boundary_pos")
    mesh = N.Mesh(n, m, d, d_in, pV, pT)
    prm = N.Params()
    N.check(lib, None, lib.ffa_default_params(C.byref(prm)))
    prm.nd_leaf_size = int(leaf_size)
    prm.host_threads = int(host_threads)
    prm.solve_schedule = int(schedule)
    if factor not in FACTORS:
        raise ValueError("factor must be one of " + ", ".join(FACTORS))
    prm.factor_device = FACTORS[factor]
    if out is None:
        out = np.empty((n, d), np.float64)
    po = _out(out, n * d, "out")
    rel = C.c_double()
    N.check(lib, None, lib.ffa_tutte(C.byref(mesh), pb, int(len(kb)), pp, C.byref(prm),
                                     C.c_void_p(stream) if stream else None, po, C.byref(rel)))
    return out, rel.value


class BatchSolver:
    """Many independent meshes solved together (one graph launch for all of them)."""

    def __init__(self, workloads, precision: str = "fp32", check_every: int = 10, refine_sweeps: int = 2,
                 leaf_size: int = 64, eps_abs=None, eps_rel=None, factor: str = "host", stream=None):
        self._lib = N.load()
        self._b = None
        k = len(workloads)
        self._keep = []
        meshes = (N.Mesh * k)()
        pin_ptrs = (C.c_void_p * k)()
        pos_ptrs = (C.c_void_p * k)()
        npin = np.zeros(k, np.int32)
        energies = np.zeros(k, np.int32)
        rho = np.zeros(k, np.float64)
        self.n, self.d = [], []
        for j, wl in enumerate(workloads):
            pV, V = _ptr(wl.V, np.float64)
            pT, T = _ptr(wl.T, np.int32)
            pP, P = _ptr(wl.pins, np.int32)
            pB, B = _ptr(wl.pin_pos, np.float64, len(wl.pins) * wl.d, "pin_pos")
            self._keep += [V, T, P, B]
            meshes[j] = N.Mesh(wl.n, wl.m, wl.d, wl.V.shape[1], pV, pT)
            pin_ptrs[j] = pP
            pos_ptrs[j] = pB
            npin[j] = len(wl.pins)
            energies[j] = ENERGIES[wl.energy]
            rho[j] = wl.rho
            self.n.append(wl.n)
            self.d.append(wl.d)
        prm = N.Params()
        N.check(self._lib, None, self._lib.ffa_default_params(C.byref(prm)))
        prm.local_precision = PRECISIONS[precision]
        prm.check_every = int(check_every)
        prm.refine_sweeps = int(refine_sweeps)
        prm.nd_leaf_size = int(leaf_size)
        prm.eps_abs = float(workloads[0].eps_abs if eps_abs is None else eps_abs)
        prm.eps_rel = float(workloads[0].eps_rel if eps_rel is None else eps_rel)
        if factor not in FACTORS:
            raise ValueError("factor must be one of " + ", ".join(FACTORS))
        prm.factor_device = FACTORS[factor]
        self._keep += [npin, energies, rho]
        b = C.c_void_p()
        st = self._lib.ffa_batch_create(k, meshes, pin_ptrs, C.c_void_p(npin.ctypes.data), pos_ptrs,
                                        C.c_void_p(energies.ctypes.data), C.c_void_p(rho.ctypes.data),
                                        C.byref(prm), C.c_void_p(stream) if stream else None, C.byref(b))
        if st != N.FFA_OK:
            raise N.FFAError(st, self._lib.ffa_batch_last_error(None).decode())
        self._b = b
        self.k = k

    def _check(self, st):
        if st != N.FFA_OK:
            raise N.FFAError(st, self._lib.ffa_batch_last_error(self._b).decode())

    def close(self):
        if self._b is not None:
            self._lib.ffa_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self, W0s):
        W0s = list(W0s)
        if len(W0s) != self.k:
            raise ValueError(f"{len(W0s)} initial maps for {self.k} meshes")
        ptrs = (C.c_void_p * self.k)()
        keep = []
        for j, W in enumerate(W0s):
            p, a = _ptr(W, np.float64, self.n[j] * self.d[j], f"W0[{j}]")
            ptrs[j] = p
            keep.append(a)
        self._check(self._lib.ffa_batch_init(self._b, ptrs))

    def iterate(self, max_iter: int, stop_at_tol: bool = True):
        stats = (N.Stats * self.k)()
        nconv = C.c_int32()
        self._check(self._lib.ffa_batch_iterate(self._b, int(max_iter), 1 if stop_at_tol else 0, stats,
                                                C.byref(nconv)))
        return [s.as_dict() for s in stats], nconv.value

    def autotune(self, reps: int = 5) -> list:
        g = int(self._lib.ffa_batch_groups(self._b))
        arr = (N.Tuning * max(g, 1))()
        self._check(self._lib.ffa_batch_autotune(self._b, int(reps), arr))
        return [arr[i].as_dict() for i in range(g)]

    def W(self, j: int, out=None):
        if out is None:
            out = np.empty((self.n[j], self.d[j]), np.float64)
        po = _out(out, self.n[j] * self.d[j], "out")
        self._check(self._lib.ffa_batch_get_W(self._b, int(j), po))
        return out
