"""Python binding of the C ABI in include/jsvd.h (argument marshalling only).

Every step of the computation runs in the CUDA library libjsvd.so built by
``paper_1401_2720_gb300.build_ext``; there is no CPU fallback.  If the
library is missing the calls raise.

Tensors are torch.float64 CUDA tensors.  The library is column-major; a
torch (row-major) m x n tensor is handed over as the column-major buffer of
its transpose, and results come back as column-major views.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libjsvd.so")

STRATEGIES = {"modulus": 0, "R": 1, "C": 2, "rR": 3, "rC": 4}
PRECISIONS = {"fp64": 0, "mixed": 1}
# FP64 block contractions: FP64 FMA kernels, or split bf16 digits on the tensor cores
CONTRACTIONS = {"fp64": 0, "split": 1, "split_sync": 2}
STATUS = {0: "success", 1: "not converged", 2: "non-finite input", 3: "CUDA error",
          4: "allocation failed", 5: "unsupported", 6: "device wait timed out",
          7: "too large for the no-allocation entry point", 8: "internal consistency check failed"}


class JsvdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"jsvd status {status} ({STATUS.get(status, 'invalid argument')}): {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("b", ctypes.c_int), ("strategy", ctypes.c_int), ("inner_strategy", ctypes.c_int),
                ("inner_sweeps", ctypes.c_int), ("max_sweeps", ctypes.c_int),
                ("precision", ctypes.c_int), ("sort", ctypes.c_int), ("contraction", ctypes.c_int),
                ("dynamic_order", ctypes.c_int), ("preprocess", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("sweeps_low", ctypes.c_int), ("converged", ctypes.c_int),
                ("b", ctypes.c_int), ("rotations", ctypes.c_longlong),
                ("proper_rotations", ctypes.c_longlong), ("pairs_updated", ctypes.c_longlong),
                ("breakdowns", ctypes.c_longlong), ("off_norm", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lock = threading.Lock()
_lib = None
_ctx: dict[int, ctypes.c_void_p] = {}

EXPORTED = ["jsvd_default_opts", "jsvd_create", "jsvd_destroy", "jsvd_set_stream",
            "jsvd_last_error", "jsvd_status_string", "jsvd_dgesvj", "jsvd_dhsvj",
            "jsvd_pivot_table", "jsvd_rotation_params", "jsvd_profile", "jsvd_profile_read",
            "jsvd_fp64_peak", "jsvd_bf16_mma_peak", "jsvd_dgesvj_batched", "jsvd_dgesvj_backward",
            "jsvd_dgesvj_noalloc", "jsvd_sorted_pivot_table", "jsvd_column_sumsq", "jsvd_relative_test",
            "jsvd_block_pstep"]


def library():
    """Load libjsvd.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_1401_2720_gb300.build_ext.build()")
            lib = ctypes.CDLL(LIB_PATH)
            P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            lib.jsvd_default_opts.argtypes = [ctypes.POINTER(Opts)]
            lib.jsvd_default_opts.restype = None
            lib.jsvd_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), I, P]
            lib.jsvd_destroy.argtypes = [P]
            lib.jsvd_set_stream.argtypes = [P, P]
            lib.jsvd_last_error.argtypes = [P]
            lib.jsvd_last_error.restype = ctypes.c_char_p
            lib.jsvd_status_string.argtypes = [I]
            lib.jsvd_status_string.restype = ctypes.c_char_p
            lib.jsvd_dgesvj.argtypes = [P, I, I, P, I, P, P, I, P, I, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
            lib.jsvd_dhsvj.argtypes = [P, I, I, I, P, I, P, P, I, P, I, ctypes.POINTER(Opts), ctypes.POINTER(Info)]
            lib.jsvd_pivot_table.argtypes = [I, I, P]
            lib.jsvd_rotation_params.argtypes = [P, I, P, P, P, P, P, P, P]
            lib.jsvd_relative_test.argtypes = [P, I, P, P, P, D, P]
            lib.jsvd_profile.argtypes = [P, I]
            lib.jsvd_profile_read.argtypes = [P, P, P, P, I]
            lib.jsvd_fp64_peak.argtypes = [P, D, P, P]
            lib.jsvd_bf16_mma_peak.argtypes = [P, D, P]
            lib.jsvd_dgesvj_batched.argtypes = [P, I, P, P, P, P, P, P, P, P, P, P, P,
                                                ctypes.POINTER(Opts), P]
            lib.jsvd_dgesvj_backward.argtypes = [P, I, P, P, P, P, P, P, P, P, P, P, P, P, P]
            lib.jsvd_dgesvj_noalloc.argtypes = [I, I, P, I, P, P, I, P, I, ctypes.POINTER(Opts),
                                                ctypes.POINTER(Info), P]
            lib.jsvd_sorted_pivot_table.argtypes = [P, I, I, P, P, P]
            lib.jsvd_column_sumsq.argtypes = [P, I, I, P, I, P, P]
            lib.jsvd_block_pstep.argtypes = [P, I, I, I, I, I, P, I, P, I, I, ctypes.POINTER(Info)]
            _lib = lib
    return _lib


def context(device: int | None = None) -> ctypes.c_void_p:
    """The per-device library context, bound to torch's current stream."""
    lib = library()
    dev = torch.cuda.current_device() if device is None else int(device)
    with _lock:
        if dev not in _ctx:
            h = ctypes.c_void_p()
            rc = lib.jsvd_create(ctypes.byref(h), dev, None)
            if rc:
                raise JsvdError(rc, "jsvd_create failed")
            _ctx[dev] = h
    h = _ctx[dev]
    lib.jsvd_set_stream(h, ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    return h


def _raise(rc: int, h) -> None:
    msg = library().jsvd_last_error(h).decode() if h else ""
    raise JsvdError(rc, msg)


def make_opts(b: int = 0, strategy: str = "rR", inner_strategy: str | None = None,
              inner_sweeps: int = 1, max_sweeps: int = 30, precision: str = "fp64",
              sort: bool = True, contraction: str = "split", dynamic_order: bool = False,
              preprocess: bool = False) -> Opts:
    o = Opts()
    library().jsvd_default_opts(ctypes.byref(o))
    o.b = b
    o.strategy = STRATEGIES[strategy]
    o.inner_strategy = -1 if inner_strategy is None else STRATEGIES[inner_strategy]
    o.inner_sweeps = inner_sweeps
    o.max_sweeps = max_sweeps
    o.precision = PRECISIONS[precision]
    o.sort = 1 if sort else 0
    o.contraction = CONTRACTIONS[contraction]
    o.dynamic_order = 1 if dynamic_order else 0
    o.preprocess = 1 if preprocess else 0
    return o


def _colmajor(A: torch.Tensor) -> tuple[torch.Tensor, int]:
    """(buffer, ld) of A as a column-major matrix."""
    if A.dtype != torch.float64 or not A.is_cuda or A.dim() != 2:
        raise ValueError("expected a 2-D torch.float64 CUDA tensor")
    m = A.shape[0]
    if A.stride(0) == 1 and A.stride(1) >= max(m, 1):
        return A, A.stride(1)
    return A.t().contiguous().t(), m


def _outputs(m: int, n: int, with_v: bool, device):
    U = torch.empty((n, m), dtype=torch.float64, device=device).t()
    S = torch.empty(n, dtype=torch.float64, device=device)
    V = torch.empty((n, n), dtype=torch.float64, device=device).t() if with_v else None
    return U, S, V


def svd(A: torch.Tensor, *, with_v: bool = True, return_info: bool = False, out=None, **kw):
    """A = U diag(S) V^T by the block-oriented one-sided Jacobi method.
    A: m x n (m >= n) float64 CUDA tensor.  Keyword options as in make_opts."""
    m, n = A.shape
    if m < n:
        raise ValueError("svd needs m >= n; pass A.T")
    Ac, lda = _colmajor(A)
    U, S, V = out if out is not None else _outputs(m, n, with_v, A.device)
    opts = make_opts(**kw)
    info = Info()
    h = context(A.device.index)
    rc = library().jsvd_dgesvj(h, m, n, Ac.data_ptr(), lda, S.data_ptr(), U.data_ptr(), U.stride(1),
                               V.data_ptr() if V is not None else None, V.stride(1) if V is not None else 1,
                               ctypes.byref(opts), ctypes.byref(info))
    if rc not in (0, 1):
        _raise(rc, h)
    res = (U, S, V)
    return (res + (dict(info.as_dict(), status=rc),)) if return_info else res


def hsvd(G: torch.Tensor, n_plus: int, *, with_v: bool = True, return_info: bool = False, out=None, **kw):
    """Hyperbolic SVD G = U diag(S) V^T, V^T J V = J, J = diag(I_{n_plus}, -I)."""
    m, n = G.shape
    if m < n:
        raise ValueError("hsvd needs m >= n")
    Gc, ldg = _colmajor(G)
    U, S, V = out if out is not None else _outputs(m, n, with_v, G.device)
    opts = make_opts(**kw)
    info = Info()
    h = context(G.device.index)
    rc = library().jsvd_dhsvj(h, m, n, int(n_plus), Gc.data_ptr(), ldg, S.data_ptr(), U.data_ptr(),
                              U.stride(1), V.data_ptr() if V is not None else None,
                              V.stride(1) if V is not None else 1, ctypes.byref(opts), ctypes.byref(info))
    if rc not in (0, 1):
        _raise(rc, h)
    res = (U, S, V)
    return (res + (dict(info.as_dict(), status=rc),)) if return_info else res


def block_pstep(G: torch.Tensor, V: torch.Tensor | None, b: int, step: int, strategy: str = "rR",
                contraction: str = "split") -> dict:
    """One block p-step (Sec. 2, 4) of the FP64 method on G (m x n) and V
    (n x n or None), in place, with the solver's kernels.  Both must be
    column-major float64 CUDA tensors (e.g. X.t().contiguous().t())."""
    m, n = G.shape
    for X in (G, V):
        if X is not None and (X.dtype != torch.float64 or not X.is_cuda or X.stride(0) != 1):
            raise ValueError("block_pstep needs column-major float64 CUDA tensors")
    info = Info()
    h = context(G.device.index)
    rc = library().jsvd_block_pstep(h, m, n, b, STRATEGIES[strategy], step, G.data_ptr(), G.stride(1),
                                    V.data_ptr() if V is not None else None, V.stride(1) if V is not None else 1,
                                    CONTRACTIONS[contraction], ctypes.byref(info))
    if rc:
        _raise(rc, h)
    return info.as_dict()


def pivot_table(strategy: str, nblocks: int) -> np.ndarray:
    """The library's p-strategy table, shape (nblocks-1, nblocks/2, 2), 0-based."""
    out = np.zeros((nblocks - 1) * nblocks, dtype=np.int32)
    rc = library().jsvd_pivot_table(STRATEGIES[strategy], nblocks, out.ctypes.data_as(ctypes.c_void_p))
    if rc:
        raise JsvdError(rc, f"no {strategy} table of order {nblocks}")
    return out.reshape(nblocks - 1, nblocks // 2, 2)


def column_sumsq(A: torch.Tensor):
    """DRDSSQ (App. A) of every column of A: (e, f) with ||a_j||^2 = f_j 2^e_j."""
    buf, ld = _colmajor(A)
    m, n = A.shape
    e = torch.empty(n, dtype=torch.int32, device=A.device)
    f = torch.empty(n, dtype=torch.float64, device=A.device)
    h = context(A.device.index)
    rc = library().jsvd_column_sumsq(h, m, n, buf.data_ptr(), ld, e.data_ptr(), f.data_ptr())
    if rc:
        _raise(rc, h)
    return e, f


def sorted_pivot_table(strategy: str, block_norms: torch.Tensor):
    """The dynamic ordering's sweep table computed by the library's kernel:
    (perm, pairs) with perm the block-columns by descending norm (ties by
    index) and pairs (nblocks-1, nblocks/2, 2) the remapped static table."""
    dev = block_norms.device
    nb = block_norms.numel()
    norms = block_norms.to(torch.float64).contiguous()
    perm = torch.empty(nb, dtype=torch.int32, device=dev)
    pairs = torch.empty((nb - 1) * nb, dtype=torch.int32, device=dev)
    h = context(dev.index)
    rc = library().jsvd_sorted_pivot_table(h, STRATEGIES[strategy], nb, norms.data_ptr(), perm.data_ptr(),
                                           pairs.data_ptr())
    if rc:
        _raise(rc, h)
    return perm, pairs.reshape(nb - 1, nb // 2, 2)


def rotation_params(hpp: torch.Tensor, hqq: torch.Tensor, hpq: torch.Tensor, hyperbolic: torch.Tensor):
    """Eqs. (4.3)-(4.6) evaluated by the library's device code."""
    n = hpp.numel()
    dev = hpp.device
    cs = torch.empty(n, dtype=torch.float64, device=dev)
    tn = torch.empty(n, dtype=torch.float64, device=dev)
    pr = torch.empty(n, dtype=torch.int32, device=dev)
    hy = hyperbolic.to(device=dev, dtype=torch.int32).contiguous()
    args = [t.contiguous() for t in (hpp, hqq, hpq)]
    h = context(dev.index)
    rc = library().jsvd_rotation_params(h, n, args[0].data_ptr(), args[1].data_ptr(), args[2].data_ptr(),
                                        hy.data_ptr(), cs.data_ptr(), tn.data_ptr(), pr.data_ptr())
    if rc:
        _raise(rc, h)
    return cs, tn, pr.bool()


def relative_test(hpp: torch.Tensor, hqq: torch.Tensor, hpq: torch.Tensor, c_eps: float) -> torch.Tensor:
    """The sweep kernels' relative orthogonality test (Sec. 4.3), as bools."""
    n = hpp.numel()
    dev = hpp.device
    rho = torch.empty(n, dtype=torch.int32, device=dev)
    args = [t.to(dtype=torch.float64).contiguous() for t in (hpp, hqq, hpq)]
    h = context(dev.index)
    rc = library().jsvd_relative_test(h, n, args[0].data_ptr(), args[1].data_ptr(), args[2].data_ptr(),
                                      float(c_eps), rho.data_ptr())
    if rc:
        _raise(rc, h)
    return rho.bool()


KERNEL_CLASSES = ("gram", "jacobi", "update", "update_v", "other")


def profile(enable: bool = True, device: int | None = None) -> None:
    """Clear the library's kernel tallies; time the sweep kernels if enable."""
    library().jsvd_profile(context(device), 1 if enable else 0)


def profile_read(device: int | None = None) -> dict:
    """{class: (milliseconds, launches, algorithmic flops)} since profile()."""
    k = len(KERNEL_CLASSES)
    ms = np.zeros(k)
    ln = np.zeros(k, dtype=np.int64)
    fl = np.zeros(k)
    library().jsvd_profile_read(context(device), ms.ctypes.data_as(ctypes.c_void_p),
                                ln.ctypes.data_as(ctypes.c_void_p), fl.ctypes.data_as(ctypes.c_void_p), k)
    return {c: (float(ms[i]), int(ln[i]), float(fl[i])) for i, c in enumerate(KERNEL_CLASSES)}


def fp64_peak(seconds: float = 1.0, device: int | None = None) -> tuple[float, float]:
    """(DFMA, DMMA) FP64 TFLOP/s of this GPU measured by the library's probe."""
    a = ctypes.c_double()
    b = ctypes.c_double()
    h = context(device)
    rc = library().jsvd_fp64_peak(h, float(seconds), ctypes.byref(a), ctypes.byref(b))
    if rc:
        _raise(rc, h)
    return a.value, b.value


def bf16_mma_peak(seconds: float = 1.0, device: int | None = None) -> float:
    """bf16 mma.sync (m16n8k16) TFLOP/s of this GPU measured by the library's probe."""
    a = ctypes.c_double()
    h = context(device)
    rc = library().jsvd_bf16_mma_peak(h, float(seconds), ctypes.byref(a))
    if rc:
        _raise(rc, h)
    return a.value


# ---------------------------------------------------------------------------
# batches of matrices of uneven sizes (packed column-major buffers)

class Packing:
    """Element offsets of a batch of column-major matrices packed back to back:
    A_i (m_i x n_i), U_i (m_i x n_i), S_i (n_i), V_i (n_i x n_i)."""

    def __init__(self, ms, ns):
        self.m = np.ascontiguousarray(ms, dtype=np.int32)
        self.n = np.ascontiguousarray(ns, dtype=np.int32)
        mn = self.m.astype(np.int64) * self.n
        nn = self.n.astype(np.int64) ** 2
        self.mn_off = np.concatenate([[0], np.cumsum(mn)[:-1]]).astype(np.int64)
        self.n_off = np.concatenate([[0], np.cumsum(self.n.astype(np.int64))[:-1]]).astype(np.int64)
        self.nn_off = np.concatenate([[0], np.cumsum(nn)[:-1]]).astype(np.int64)
        self.mn_total = int(mn.sum())
        self.n_total = int(self.n.sum())
        self.nn_total = int(nn.sum())

    def __len__(self):
        return len(self.m)

    def pack(self, mats, device) -> torch.Tensor:
        """Column-major pack of a list of (m_i x n_i) tensors/arrays."""
        parts = [torch.as_tensor(np.asarray(x) if not torch.is_tensor(x) else x).to(torch.float64).t().reshape(-1)
                 for x in mats]
        return torch.cat([p.to(device) for p in parts]) if parts else torch.empty(0, dtype=torch.float64, device=device)

    def unpack_mn(self, buf):
        return [buf[o:o + int(m) * int(n)].view(int(n), int(m)).t() for o, m, n in zip(self.mn_off, self.m, self.n)]

    def unpack_n(self, buf):
        return [buf[o:o + int(n)] for o, n in zip(self.n_off, self.n)]

    def unpack_nn(self, buf):
        return [buf[o:o + int(n) * int(n)].view(int(n), int(n)).t() for o, n in zip(self.nn_off, self.n)]


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def svd_batched_packed(pk: Packing, A: torch.Tensor, *, b=None, with_v: bool = True, return_info: bool = False,
                       **kw):
    """Batched SVD on packed buffers: returns packed (U, S, V) (+ infos)."""
    dev = A.device
    U = torch.empty(pk.mn_total, dtype=torch.float64, device=dev)
    S = torch.empty(pk.n_total, dtype=torch.float64, device=dev)
    V = torch.empty(pk.nn_total, dtype=torch.float64, device=dev) if with_v else None
    bs = None if b is None else np.ascontiguousarray(np.broadcast_to(b, (len(pk),)), dtype=np.int32)
    opts = make_opts(**kw)
    infos = (Info * len(pk))()
    h = context(dev.index)
    rc = library().jsvd_dgesvj_batched(h, len(pk), _p(pk.m), _p(pk.n), _p(bs) if bs is not None else None,
                                       A.data_ptr(), _p(pk.mn_off), S.data_ptr(), _p(pk.n_off), U.data_ptr(),
                                       _p(pk.mn_off), V.data_ptr() if V is not None else None,
                                       _p(pk.nn_off) if V is not None else None, ctypes.byref(opts), infos)
    if rc not in (0, 1):
        _raise(rc, h)
    out = (U, S, V)
    if return_info:
        out = out + ([dict(i.as_dict()) for i in infos], rc)
    return out


def svd_backward_packed(pk: Packing, U, S, V, dU=None, dS=None, dV=None) -> torch.Tensor:
    """Packed dA from packed U, S, V and cotangents (None = zero)."""
    dA = torch.empty(pk.mn_total, dtype=torch.float64, device=U.device)
    h = context(U.device.index)
    ptr = lambda t: t.contiguous().data_ptr() if t is not None else None
    rc = library().jsvd_dgesvj_backward(h, len(pk), _p(pk.m), _p(pk.n), U.data_ptr(), _p(pk.mn_off),
                                        S.data_ptr(), _p(pk.n_off), V.data_ptr(), _p(pk.nn_off),
                                        ptr(dU), ptr(dS), ptr(dV), dA.data_ptr(), _p(pk.mn_off))
    if rc:
        _raise(rc, h)
    return dA


class _BatchedSVD(torch.autograd.Function):
    """Packed batched SVD with the library's adjoint as its backward."""

    @staticmethod
    def forward(ctx, A, pk, b, kw):
        U, S, V = svd_batched_packed(pk, A.detach(), b=b, **kw)
        ctx.pk = pk
        ctx.save_for_backward(U, S, V)
        return U, S, V

    @staticmethod
    def backward(ctx, dU, dS, dV):
        U, S, V = ctx.saved_tensors
        dA = svd_backward_packed(ctx.pk, U, S, V, dU, dS, dV)
        return dA, None, None, None


def svd_batched(mats, *, b=None, **kw):
    """Differentiable batched SVD of a list of (m_i x n_i) float64 CUDA
    tensors (m_i >= n_i): returns lists U_i, S_i, V_i (views of packed
    buffers); gradients flow back to the inputs through the SVD adjoint."""
    ms = [int(x.shape[0]) for x in mats]
    ns = [int(x.shape[1]) for x in mats]
    pk = Packing(ms, ns)
    A = torch.cat([x.t().reshape(-1) for x in mats])
    U, S, V = _BatchedSVD.apply(A, pk, b, kw)
    return pk.unpack_mn(U), pk.unpack_n(S), pk.unpack_nn(V)


class _SVD(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, kw):
        U, S, V = svd(A.detach(), **kw)
        ctx.save_for_backward(U, S, V)
        return U, S, V

    @staticmethod
    def backward(ctx, dU, dS, dV):
        U, S, V = ctx.saved_tensors
        m, n = U.shape
        pk = Packing([m], [n])
        flat = lambda t: None if t is None else t.t().contiguous().reshape(-1)
        dA = svd_backward_packed(pk, flat(U), S.contiguous(), flat(V), flat(dU), dS, flat(dV))
        return dA.view(n, m).t(), None


def svd_autograd(A: torch.Tensor, **kw):
    """Differentiable single-matrix SVD (forward jsvd_dgesvj, backward the adjoint)."""
    return _SVD.apply(A, kw)


def svd_noalloc(A: torch.Tensor, *, out=None, return_info: bool = False, **kw):
    """jsvd_dgesvj_noalloc: the FP64 SVD with all scratch in the library's
    static device array (no device allocation by the library; the outputs are
    allocated here unless `out` is given)."""
    m, n = A.shape
    Ac, lda = _colmajor(A)
    U, S, V = out if out is not None else _outputs(m, n, True, A.device)
    opts = make_opts(**kw)
    info = Info()
    stream = ctypes.c_void_p(torch.cuda.current_stream(A.device).cuda_stream)
    rc = library().jsvd_dgesvj_noalloc(m, n, Ac.data_ptr(), lda, S.data_ptr(), U.data_ptr(), U.stride(1),
                                       V.data_ptr() if V is not None else None, V.stride(1) if V is not None else 1,
                                       ctypes.byref(opts), ctypes.byref(info), stream)
    if rc not in (0, 1):
        raise JsvdError(rc, "jsvd_dgesvj_noalloc failed")
    res = (U, S, V)
    return (res + (dict(info.as_dict(), status=rc),)) if return_info else res
