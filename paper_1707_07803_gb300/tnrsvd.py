"""Thin Python binding of libtnrsvd.so (argument marshalling only).

The names mirror include/tnrsvd.h. PyTorch supplies device memory and the current stream;
every step of the method runs in the library's CUDA kernels. There is no CPU fallback: if
the library is missing or cannot be loaded, every call raises.

Device data layout: an MPO core is a flat float64 CUDA tensor holding the core in memory
order (r fastest, then i, j, r'); ``Mpo`` carries those tensors with their dims and ranks.
"""

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtnrsvd.so")
MAX_SITES = 64

TNR_FP64 = 0
TNR_MIXED = 1
TNR_ROUND_TWO_SWEEP = 0
TNR_ROUND_ZIPUP = 1

_STATUS = {
    0: "ok", -1: "EINVAL", -2: "EDUP", -3: "ENOTSORTED", -4: "ENONFINITE", -5: "ENOMEM", -6: "ECUDA",
    -7: "ETIMEOUT", -8: "ERANGE",
}


class TnrError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {_STATUS.get(status, status)} ({status})")


class tnr_mpo(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("I", ctypes.c_int64 * MAX_SITES),
        ("J", ctypes.c_int64 * MAX_SITES),
        ("R", ctypes.c_int64 * (MAX_SITES + 1)),
        ("core", ctypes.c_void_p * MAX_SITES),
        ("cap", ctypes.c_int64 * MAX_SITES),
    ]


class tnr_opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("rounding", ctypes.c_int32),
        ("tol", ctypes.c_double),
        ("max_rank", ctypes.c_int64),
    ]


class tnr_problem(ctypes.Structure):
    _fields_ = [
        ("A", ctypes.POINTER(tnr_mpo)),
        ("k", ctypes.c_int32),
        ("p", ctypes.c_int32),
        ("q", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("opts", tnr_opts),
        ("U", ctypes.POINTER(tnr_mpo)),
        ("S", ctypes.c_void_p),
        ("V", ctypes.POINTER(tnr_mpo)),
        ("status", ctypes.c_int32),
        ("reserved2", ctypes.c_int32),
    ]


_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_I64P = ctypes.POINTER(ctypes.c_int64)
_SZP = ctypes.POINTER(ctypes.c_size_t)
_MPOP = ctypes.POINTER(tnr_mpo)
_OPTP = ctypes.POINTER(tnr_opts)

_SIGS = {
    "tnr_sparse_workspace": (ctypes.c_int, [_I64, _I64, _I64, _I32, _I64P, _I64P, _SZP]),
    "tnr_sparse_count": (ctypes.c_int, [_I64, _I64, _I64, _P, _P, _I32, _I64P, _I64P, _I64P, _P, ctypes.c_size_t, _P]),
    "tnr_sparse_fill": (ctypes.c_int,
                        [_I64, _I64, _I64, _P, _P, _P, _I32, _I64P, _I64P, _I64, _P, _P, _P, ctypes.c_size_t, _P]),
    "tnr_sparse_to_mpo_noalloc": (ctypes.c_int, [_I64, _I64, _I64, _P, _P, _P, _I32, _I64P, _I64P, _P, _P, _I64,
                                                  _I64P, _P]),
    "tnr_sparse_cores": (ctypes.c_int, [_I64, _P, _P, _I32, _I64P, _I64P, _MPOP, _P]),
    "tnr_mpo_contract": (ctypes.c_int, [_MPOP, _I32, _MPOP, _MPOP, _I32, _P]),
    "tnr_orthogonalize_workspace": (ctypes.c_int, [_MPOP, _SZP]),
    "tnr_orthogonalize": (ctypes.c_int, [_MPOP, _P, _OPTP, _P, ctypes.c_size_t, _P]),
    "tnr_solve_query": (ctypes.c_int, [_MPOP, _I32, _I32, _OPTP, _MPOP, _MPOP, _SZP]),
    "tnr_solve": (ctypes.c_int, [_MPOP, _I32, _I32, _I32, ctypes.c_uint64, _OPTP, _MPOP, _P, _MPOP, _P,
                                 ctypes.c_size_t, _P]),
    "tnr_solve_batched": (ctypes.c_int, [_I32, ctypes.POINTER(tnr_problem), _I32, _P, ctypes.c_size_t, _P]),
    "tnr_batch_workspace": (ctypes.c_int, [_I32, ctypes.POINTER(tnr_problem), _SZP]),
    "tnr_batch_create": (ctypes.c_int, [_I32, ctypes.POINTER(tnr_problem), _I32, _P, ctypes.c_size_t, _P,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "tnr_batch_launch": (ctypes.c_int, [_P, _P]),
    "tnr_batch_collect": (ctypes.c_int, [_P, _P]),
    "tnr_batch_config": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), _I64P]),
    "tnr_batch_destroy": (ctypes.c_int, [_P]),
    "tnr_selftest_wait_timeout": (ctypes.c_int, [_I64, _P]),
    "tnr_sparse_solve_workspace": (ctypes.c_int, [_I64, _I64, _I64, _I32, _I64P, _I64P, _I32, _I32, _SZP]),
    "tnr_sparse_solve": (ctypes.c_int, [_I64, _I64, _I64, _P, _P, _I32, _I64P, _I64P, _I32, _I32, _I32,
                                        ctypes.c_uint64, _I32, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "tnr_diff_forward": (ctypes.c_int, [_MPOP, _I32, _I32, _I32, ctypes.c_uint64, _P, ctypes.POINTER(ctypes.c_void_p),
                                         _P]),
    "tnr_diff_backward": (ctypes.c_int, [_P, _P, _MPOP, _P]),
    "tnr_diff_free": (None, [_P, _P]),
    "tnr_stats_enable": (None, [_I32]),
    "tnr_stats_reset": (None, []),
    "tnr_stats": (ctypes.c_int, [_I32, _I64P, ctypes.POINTER(ctypes.c_double)]),
    "tnr_stats_work": (ctypes.c_int, [_I32, ctypes.POINTER(ctypes.c_double)]),
    "tnr_stats_class_name": (ctypes.c_char_p, [_I32]),
    "tnr_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "tnr_version": (ctypes.c_int, []),
    "tnr_compress_cluster_size": (ctypes.c_int, []),
}


def load():
    """Load libtnrsvd.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtnrsvd.so not built at {LIB_PATH}; run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def exported_names():
    return list(_SIGS)


def _check(rc, what):
    if rc != 0:
        raise TnrError(rc, what)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _i64arr(vals):
    return (ctypes.c_int64 * max(1, len(vals)))(*[int(v) for v in vals])


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _need_cuda(*ts):
    for t in ts:
        if not (isinstance(t, torch.Tensor) and t.is_cuda):
            raise ValueError("device tensors (CUDA) are required")


# ----------------------------------------------------------------------------------------
# MPO container
# ----------------------------------------------------------------------------------------
TNR_F64, TNR_F32 = 0, 1


class Mpo:
    """Dims, ranks and flat CUDA core buffers of an MPO (layout of include/tnrsvd.h): float64, or
    float32 for the inputs that accept it (tnr_solve, the differentiable solve)."""

    def __init__(self, I, J, R, cores, flat=None):
        self.I = [int(x) for x in I]
        self.J = [int(x) for x in J]
        self.R = [int(x) for x in R]
        self.cores = list(cores)
        self.flat = flat  # one buffer holding every core back to back (the cores are views), or None

    @property
    def d(self):
        return len(self.I)

    def core_shape(self, k):
        return (self.R[k], self.I[k], self.J[k], self.R[k + 1])

    def to_struct(self, caps=None):
        m = tnr_mpo()
        m.d = self.d
        dts = {c.dtype for c in self.cores if c is not None}
        if dts - {torch.float64, torch.float32} or len(dts) > 1:
            raise ValueError("cores must all be float64 or all float32")
        m.dtype = TNR_F32 if dts == {torch.float32} else TNR_F64
        for k in range(self.d):
            m.I[k], m.J[k] = self.I[k], self.J[k]
            m.core[k] = self.cores[k].data_ptr() if self.cores[k] is not None else 0
            m.cap[k] = caps[k] if caps is not None else (self.cores[k].numel() if self.cores[k] is not None else 0)
        for k in range(self.d + 1):
            m.R[k] = self.R[k]
        return m

    @staticmethod
    def from_numpy(cores, device="cuda", dtype=None, flat=False):
        """Logical numpy cores (R, I, J, R') -> flat device buffers in memory order (float64, or
        dtype=numpy.float32 for float32 input cores). With flat=True the cores are views into one
        buffer (Mpo.flat), so that one copy moves all of them (host_flat gives its host image)."""
        import numpy as np

        dt = np.float64 if dtype is None else dtype
        host = [np.ascontiguousarray(np.asarray(c, dtype=dt).reshape(-1, order="F")) for c in cores]
        I = [c.shape[1] for c in cores]
        J = [c.shape[2] for c in cores]
        R = [cores[0].shape[0]] + [c.shape[3] for c in cores]
        if not flat:
            return Mpo(I, J, R, [torch.from_numpy(h).to(device) for h in host])
        buf = torch.from_numpy(np.concatenate(host)).to(device)
        views, off = [], 0
        for h in host:
            views.append(buf[off:off + h.size])
            off += h.size
        return Mpo(I, J, R, views, flat=buf)

    @staticmethod
    def host_flat(cores, dtype=None):
        """The host image of Mpo.from_numpy(cores, flat=True).flat: one pinned buffer with the cores
        in memory order, back to back (the input of SolvePlan.run_host)."""
        import numpy as np

        dt = np.float64 if dtype is None else dtype
        host = np.concatenate([np.ascontiguousarray(np.asarray(c, dtype=dt).reshape(-1, order="F")) for c in cores])
        return torch.from_numpy(host).pin_memory()

    def to_numpy(self):
        """Flat device buffers -> logical numpy cores (copies to host)."""
        out = []
        for k in range(self.d):
            shape = self.core_shape(k)
            n = shape[0] * shape[1] * shape[2] * shape[3]
            out.append(self.cores[k][:n].cpu().numpy().reshape(shape, order="F"))
        return out


# ----------------------------------------------------------------------------------------
# Entry points (names of include/tnrsvd.h)
# ----------------------------------------------------------------------------------------
def tnr_sparse_workspace(nrows, ncols, nnz, I, J):
    lib = load()
    b = ctypes.c_size_t(0)
    _check(lib.tnr_sparse_workspace(nrows, ncols, nnz, len(I), _i64arr(I), _i64arr(J), ctypes.byref(b)),
           "tnr_sparse_workspace")
    return b.value


def tnr_sparse_count(nrows, ncols, row, col, I, J, ws, stream=None):
    lib = load()
    _need_cuda(row, col, ws)
    R = ctypes.c_int64(0)
    _check(lib.tnr_sparse_count(nrows, ncols, row.numel(), _ptr(row), _ptr(col), len(I), _i64arr(I), _i64arr(J),
                                ctypes.byref(R), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "tnr_sparse_count")
    return R.value


def tnr_sparse_fill(nrows, ncols, row, col, val, I, J, R, X, digits, ws, stream=None):
    lib = load()
    _need_cuda(row, col, val, ws)
    _check(lib.tnr_sparse_fill(nrows, ncols, row.numel(), _ptr(row), _ptr(col), _ptr(val), len(I), _i64arr(I),
                               _i64arr(J), R, _ptr(X), _ptr(digits), _ptr(ws), ws.numel() * ws.element_size(),
                               _stream(stream)), "tnr_sparse_fill")


def sparse_to_mpo(nrows, ncols, row, col, val, I, J, stream=None):
    """Alg. 4.1 on the device: returns (R, X, digits) as CUDA tensors (block form)."""
    nbytes = tnr_sparse_workspace(nrows, ncols, row.numel(), I, J)
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=row.device)
    R = tnr_sparse_count(nrows, ncols, row, col, I, J, ws, stream)
    X = torch.empty(max(R * int(I[0]) * int(J[0]), 1), dtype=torch.float64, device=row.device)
    digits = torch.empty(max(R * 2 * (len(I) - 1), 1), dtype=torch.uint8, device=row.device)
    tnr_sparse_fill(nrows, ncols, row, col, val, I, J, R, X, digits, ws, stream)
    return R, X[: R * int(I[0]) * int(J[0])], digits[: R * 2 * (len(I) - 1)].view(R, 2 * (len(I) - 1))


NOALLOC_MAX_NNZ = 8388608


def _need_buffer(t, dtype, min_elems, what, need_cuda=True):
    """A contiguous CUDA tensor of `dtype` holding at least `min_elems` elements."""
    if not isinstance(t, torch.Tensor) or (need_cuda and not t.is_cuda):
        raise ValueError(f"{what}: a CUDA tensor is required")
    if t.dtype != dtype:
        raise ValueError(f"{what}: dtype {dtype} is required, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: a contiguous tensor is required")
    if t.numel() < min_elems:
        raise ValueError(f"{what}: room for {min_elems} elements is required, got {t.numel()}")


def tnr_sparse_to_mpo_noalloc(nrows, ncols, row, col, val, I, J, X, digits, max_blocks, stream=None):
    """Alg. 4.1 without any allocation by the library (its scratch is compiled into it).

    For callers that cannot allocate device memory themselves at call time (a process whose own
    memory manager holds all device memory): the caller passes the outputs X (room for
    max_blocks*I1*J1 float64) and digits (room for max_blocks*2(d-1) uint8); returns R. The
    tensors are checked here (device, dtype, contiguity, size) before the library is called.
    Limits and races: see include/tnrsvd.h.
    """
    lib = load()
    max_blocks = int(max_blocks)
    if max_blocks < 0:
        raise ValueError("max_blocks must be >= 0")
    nnz = row.numel()
    _need_buffer(row, torch.int64, nnz, "row")
    _need_buffer(col, torch.int64, nnz, "col")
    _need_buffer(val, torch.float64, nnz, "val")
    _need_buffer(X, torch.float64, max_blocks * int(I[0]) * int(J[0]), "X")
    if len(I) > 1 or digits is not None:
        _need_buffer(digits, torch.uint8, max_blocks * 2 * (len(I) - 1), "digits")
    R = ctypes.c_int64(0)
    _check(lib.tnr_sparse_to_mpo_noalloc(nrows, ncols, nnz, _ptr(row), _ptr(col), _ptr(val), len(I),
                                         _i64arr(I), _i64arr(J), _ptr(X), _ptr(digits), max_blocks,
                                         ctypes.byref(R), _stream(stream)), "tnr_sparse_to_mpo_noalloc")
    return R.value


def tnr_sparse_cores(R, X, digits, I, J, stream=None):
    """Dense cores (Mpo) of the Alg. 4.1 MPO from its block form (R, X, digits on the device)."""
    lib = load()
    d = len(I)
    R = int(R)
    ranks = [1] + [R] * (d - 1) + [1]
    dev = X.device
    cores = [torch.empty(max(ranks[k] * int(I[k]) * int(J[k]) * ranks[k + 1], 1), dtype=torch.float64, device=dev)
             for k in range(d)]
    A = Mpo(list(I), list(J), ranks, cores)
    sa = A.to_struct()
    _need_buffer(X, torch.float64, R * int(I[0]) * int(J[0]), "X")
    if d > 1:
        _need_buffer(digits, torch.uint8, R * 2 * (d - 1), "digits")
    _check(lib.tnr_sparse_cores(R, _ptr(X), _ptr(digits), d, _i64arr(I), _i64arr(J), ctypes.byref(sa), _stream(stream)),
           "tnr_sparse_cores")
    A.R = [sa.R[k] for k in range(d + 1)]
    return A


def round_operator(A, tol=0.0, max_rank=0, stream=None):
    """SVD-based rounding of an operator MPO (Section 3; Section 4.2's rounding of the converted MPO):
    the cores viewed as a one-column tall MPO (rows (i_k, j_k) per site, K = 1) go through
    tnr_orthogonalize (the sweeps of Section 5.4 with the truncation rule of tnr_opts), and the 1 x 1
    factor R = ||A|| is put back on site 1. Returns the rounded Mpo (new buffers; A is unchanged)."""
    d = A.d
    cores = [c.clone() for c in A.cores]
    Y = Mpo([A.I[k] * A.J[k] for k in range(d)], [1] * d, list(A.R), cores)
    Q, Rf = tnr_orthogonalize(Y, tol=tol, max_rank=max_rank, stream=stream)
    n0 = Q.R[0] * Q.I[0] * Q.R[1]
    Q.cores[0][:n0].mul_(Rf.reshape(-1)[0])
    return Mpo(list(A.I), list(A.J), list(Q.R), Q.cores)


def tnr_mpo_contract(A, trans, X, precision=TNR_FP64, stream=None):
    """Y = op(A) X (Section 5.2). Allocates Y with exact sizes."""
    lib = load()
    d = A.d
    cores = []
    for k in range(d):
        xo = A.J[k] if trans else A.I[k]
        n = A.R[k] * X.R[k] * xo * X.J[k] * A.R[k + 1] * X.R[k + 1]
        cores.append(torch.empty(max(n, 1), dtype=torch.float64, device=A.cores[0].device))
    Y = Mpo([0] * d, [0] * d, [1] * (d + 1), cores)
    sa, sx, sy = A.to_struct(), X.to_struct(), Y.to_struct()
    _check(lib.tnr_mpo_contract(ctypes.byref(sa), int(trans), ctypes.byref(sx), ctypes.byref(sy), int(precision),
                                _stream(stream)), "tnr_mpo_contract")
    Y.I = [sy.I[k] for k in range(d)]
    Y.J = [sy.J[k] for k in range(d)]
    Y.R = [sy.R[k] for k in range(d + 1)]
    return Y


def _opts(tol, max_rank, precision, rounding=TNR_ROUND_TWO_SWEEP):
    o = tnr_opts()
    o.precision = int(precision)
    o.rounding = int(rounding)
    o.tol = float(tol)
    o.max_rank = int(max_rank)
    return o


def tnr_orthogonalize(Y, tol=0.0, max_rank=0, stream=None):
    """In-place MPO-QR with rounding (Alg. 5.2 + Section 5.4); returns (Y as Q, R)."""
    lib = load()
    sy = Y.to_struct()
    b = ctypes.c_size_t(0)
    _check(lib.tnr_orthogonalize_workspace(ctypes.byref(sy), ctypes.byref(b)), "tnr_orthogonalize_workspace")
    dev = Y.cores[0].device
    ws = torch.empty(max(b.value, 1), dtype=torch.uint8, device=dev)
    K = Y.J[0]
    Rk = torch.empty(K * K, dtype=torch.float64, device=dev)
    o = _opts(tol, max_rank, TNR_FP64)
    _check(lib.tnr_orthogonalize(ctypes.byref(sy), _ptr(Rk), ctypes.byref(o), _ptr(ws), b.value, _stream(stream)),
           "tnr_orthogonalize")
    Y.R = [sy.R[k] for k in range(Y.d + 1)]
    return Y, Rk.view(K, K).t()  # column-major K x K -> row-major view


class SolvePlan:
    """Buffers for repeated solves of one operator shape (workspace and U, S, V outputs)."""

    def __init__(self, A, k, p, tol=0.0, max_rank=0, precision=TNR_FP64):
        lib = load()
        self.k, self.p = int(k), int(p)
        self.opts = _opts(tol, max_rank, precision)
        self.A = A
        self.sa = A.to_struct()
        self.us, self.vs = tnr_mpo(), tnr_mpo()
        b = ctypes.c_size_t(0)
        _check(lib.tnr_solve_query(ctypes.byref(self.sa), self.k, self.p, ctypes.byref(self.opts),
                                   ctypes.byref(self.us), ctypes.byref(self.vs), ctypes.byref(b)), "tnr_solve_query")
        dev = A.cores[0].device
        self.ws_bytes = b.value
        self.ws = torch.empty(max(b.value, 1), dtype=torch.uint8, device=dev)
        # S, U's cores and V's cores back to back in one buffer (out_flat), each core at its capacity
        ucap = [max(self.us.cap[i], 1) for i in range(self.us.d)]
        vcap = [max(self.vs.cap[i], 1) for i in range(self.vs.d)]
        self.out_flat = torch.empty(self.k + sum(ucap) + sum(vcap), dtype=torch.float64, device=dev)
        self.S = self.out_flat[:self.k]
        off = self.k
        self.U_cores, self.V_cores = [], []
        for c in ucap:
            self.U_cores.append(self.out_flat[off:off + c])
            off += c
        for c in vcap:
            self.V_cores.append(self.out_flat[off:off + c])
            off += c
        for i in range(self.us.d):
            self.us.core[i] = self.U_cores[i].data_ptr()
            self.vs.core[i] = self.V_cores[i].data_ptr()

    def run(self, q, seed, stream=None):
        lib = load()
        _check(lib.tnr_solve(ctypes.byref(self.sa), self.k, self.p, int(q), ctypes.c_uint64(int(seed)),
                             ctypes.byref(self.opts), ctypes.byref(self.us), _ptr(self.S), ctypes.byref(self.vs),
                             _ptr(self.ws), self.ws_bytes, _stream(stream)), "tnr_solve")
        return self

    def run_host(self, host_in, host_out, q, seed, stream=None):
        """One solve with host buffers: host_in (pinned; the operator's cores back to back, as
        Mpo.host_flat gives them) goes to the device in one copy into the operator's flat buffer
        (the plan's operator must come from Mpo.from_numpy(..., flat=True)), the solve runs, and
        out_flat (S, then U's and V's cores at their capacities) comes back in one copy into
        host_out (pinned, out_flat.numel() doubles). All on the plan's stream; returns self."""
        if self.A.flat is None:
            raise ValueError("run_host needs an operator built with Mpo.from_numpy(..., flat=True)")
        if host_in.numel() != self.A.flat.numel() or host_out.numel() != self.out_flat.numel():
            raise ValueError("host buffers do not match the operator's flat buffer or out_flat")
        st = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(st):
            self.A.flat.copy_(host_in, non_blocking=True)
            self.run(q, seed, st)
            host_out.copy_(self.out_flat, non_blocking=True)
        return self

    def outputs(self):
        d = self.us.d
        U = Mpo([self.us.I[i] for i in range(d)], [self.us.J[i] for i in range(d)],
                [self.us.R[i] for i in range(d + 1)], self.U_cores)
        V = Mpo([self.vs.I[i] for i in range(d)], [self.vs.J[i] for i in range(d)],
                [self.vs.R[i] for i in range(d + 1)], self.V_cores)
        return U, self.S, V


def tnr_solve(A, k, p, q, seed, tol=0.0, max_rank=0, precision=TNR_FP64, stream=None):
    """TNrSVD (Alg. 5.4 + 5.3): returns (U, S, V) with U, V as Mpo over the merged sites."""
    plan = SolvePlan(A, k, p, tol, max_rank, precision)
    plan.run(q, seed, stream)
    return plan.outputs()


def _batch_outputs(problems, precision):
    """Per-problem output buffers (U, S, V at their tnr_solve_query capacities) and the
    tnr_problem array describing the batch; returns (plans, probs, largest solve workspace)."""
    lib = load()
    n = len(problems)
    plans = []
    stride = 256
    for pr in problems:
        sp = SolvePlan.__new__(SolvePlan)  # outputs only; the batch owns the workspace
        sp.k, sp.p = int(pr["k"]), int(pr["p"])
        sp.opts = _opts(pr.get("tol", 0.0), pr.get("max_rank", 0), pr.get("precision", precision),
                        pr.get("rounding", TNR_ROUND_TWO_SWEEP))
        sp.A = pr["A"]
        sp.sa = sp.A.to_struct()
        sp.us, sp.vs = tnr_mpo(), tnr_mpo()
        b = ctypes.c_size_t(0)
        _check(lib.tnr_solve_query(ctypes.byref(sp.sa), sp.k, sp.p, ctypes.byref(sp.opts), ctypes.byref(sp.us),
                                   ctypes.byref(sp.vs), ctypes.byref(b)), "tnr_solve_query")
        dev = sp.A.cores[0].device
        sp.U_cores = [torch.empty(max(sp.us.cap[i], 1), dtype=torch.float64, device=dev) for i in range(sp.us.d)]
        sp.V_cores = [torch.empty(max(sp.vs.cap[i], 1), dtype=torch.float64, device=dev) for i in range(sp.vs.d)]
        for i in range(sp.us.d):
            sp.us.core[i] = sp.U_cores[i].data_ptr()
            sp.vs.core[i] = sp.V_cores[i].data_ptr()
        sp.S = torch.empty(sp.k, dtype=torch.float64, device=dev)
        sp.ws, sp.ws_bytes = None, 0
        stride = max(stride, (b.value + 255) // 256 * 256)
        plans.append((sp, int(pr["q"]), int(pr["seed"])))
    probs = (tnr_problem * max(n, 1))()
    for i, (sp, q, seed) in enumerate(plans):
        P = probs[i]
        P.A = ctypes.pointer(sp.sa)
        P.k, P.p, P.q = sp.k, sp.p, q
        P.seed = seed
        P.opts = sp.opts
        P.U = ctypes.pointer(sp.us)
        P.S = sp.S.data_ptr()
        P.V = ctypes.pointer(sp.vs)
    return plans, probs, stride


class BatchPlan:
    """Buffers for a batch of independent solves (tnr_solve_batched): per-problem outputs and
    one workspace slice per worker, sized by the largest problem of the batch."""

    def __init__(self, problems, workers=0, precision=TNR_MIXED):
        """problems: list of dicts with keys A (Mpo), k, p, q, seed and optional tol, max_rank,
        precision and rounding (TNR_ROUND_ZIPUP is accepted by the persistent batch only)."""
        n = len(problems)
        self.n = n
        self.workers = int(workers) if workers else min(max(n, 1), 16)
        self.workers = max(1, min(self.workers, max(n, 1)))
        self.plans, self.probs, self.ws_stride = _batch_outputs(problems, precision)
        dev = problems[0]["A"].cores[0].device if n else torch.device("cuda")
        self.ws = torch.empty(self.workers * self.ws_stride, dtype=torch.uint8, device=dev)

    def run(self, stream=None, check=True):
        lib = load()
        rc = lib.tnr_solve_batched(self.n, self.probs, self.workers, _ptr(self.ws), self.ws_stride, _stream(stream))
        if check:
            _check(rc, "tnr_solve_batched")
        return rc

    def statuses(self):
        return [self.probs[i].status for i in range(self.n)]

    def outputs(self, i):
        return self.plans[i][0].outputs()


class PersistentBatch:
    """A batch solved by the persistent kernel (tnr_batch_*): one launch, one CTA per problem,
    problems taken from a device work queue; optionally autotuned and captured in a CUDA graph."""

    def __init__(self, problems, precision=TNR_MIXED, autotune=True, graph=True, stream=None, ctas_per_sm=0):
        lib = load()
        if not problems:
            raise ValueError("empty batch")
        self.n = len(problems)
        self.plans, self.probs, _ = _batch_outputs(problems, precision)
        b = ctypes.c_size_t(0)
        _check(lib.tnr_batch_workspace(self.n, self.probs, ctypes.byref(b)), "tnr_batch_workspace")
        dev = problems[0]["A"].cores[0].device
        self.ws = torch.empty(max(b.value, 1), dtype=torch.uint8, device=dev)
        self.ws_bytes = b.value
        h = ctypes.c_void_p(0)
        flags = (1 if autotune else 0) | (2 if graph else 0) | ((int(ctas_per_sm) & 15) << 4)
        _check(lib.tnr_batch_create(self.n, self.probs, flags, _ptr(self.ws), self.ws_bytes, _stream(stream),
                                    ctypes.byref(h)), "tnr_batch_create")
        self.handle = h

    def launch(self, stream=None):
        _check(load().tnr_batch_launch(self.handle, _stream(stream)), "tnr_batch_launch")
        return self

    def collect(self, stream=None, check=True):
        rc = load().tnr_batch_collect(self.handle, _stream(stream))
        if check:
            _check(rc, "tnr_batch_collect")
        return rc

    def config(self):
        g, c, s = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
        _check(load().tnr_batch_config(self.handle, ctypes.byref(g), ctypes.byref(c), ctypes.byref(s)),
               "tnr_batch_config")
        return {"grid": g.value, "ctas_per_sm": c.value, "smem_bytes": s.value}

    def statuses(self):
        return [self.probs[i].status for i in range(self.n)]

    def outputs(self, i):
        return self.plans[i][0].outputs()

    def close(self):
        if self.handle:
            load().tnr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tnr_solve_batch_persistent(problems, precision=TNR_MIXED, autotune=True, graph=True, stream=None):
    """Solves independent TNrSVD problems with the persistent kernel; returns [(U, S, V), ...]."""
    pb = PersistentBatch(problems, precision, autotune, graph, stream)
    pb.launch(stream)
    pb.collect(stream)
    out = [pb.outputs(i) for i in range(pb.n)]
    pb.close()
    return out


def tnr_solve_batched(problems, workers=0, precision=TNR_MIXED, stream=None):
    """Solves independent TNrSVD problems concurrently; returns [(U, S, V), ...] in order."""
    plan = BatchPlan(problems, workers, precision)
    plan.run(stream)
    return [plan.outputs(i) for i in range(plan.n)]


def tnr_sparse_solve(nrows, ncols, R, X, digits, I, J, k, p, q, seed, precision=TNR_FP64, stream=None):
    """TNrSVD of a sparse matrix in Alg. 4.1 block form: returns dense (U, S, V) device tensors."""
    lib = load()
    _need_cuda(X, digits)
    d = len(I)
    Ia, Ja = _i64arr(I), _i64arr(J)
    b = ctypes.c_size_t(0)
    _check(lib.tnr_sparse_solve_workspace(int(nrows), int(ncols), int(R), d, Ia, Ja, int(k), int(p), ctypes.byref(b)),
           "tnr_sparse_solve_workspace")
    dev = X.device
    ws = torch.empty(b.value, dtype=torch.uint8, device=dev)
    U = torch.empty((int(k), int(nrows)), dtype=torch.float64, device=dev)  # column-major nrows x k
    V = torch.empty((int(k), int(ncols)), dtype=torch.float64, device=dev)
    S = torch.empty(int(k), dtype=torch.float64, device=dev)
    _check(lib.tnr_sparse_solve(int(nrows), int(ncols), int(R), _ptr(X), _ptr(digits), d, Ia, Ja, int(k), int(p),
                                int(q), ctypes.c_uint64(int(seed)), int(precision), _ptr(U), _ptr(S), _ptr(V),
                                _ptr(ws), b.value, _stream(stream)), "tnr_sparse_solve")
    return U.t(), S, V.t()


class _Tape:
    """Owns a tnr_diff_forward tape; released with the object."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if self.handle is not None and self.handle.value:
            try:
                load().tnr_diff_free(self.handle, _stream())
            except Exception:
                pass
            self.handle = None


class TnrSvdValues(torch.autograd.Function):
    """S (k singular values, FP64) of TNrSVD with fixed ranks as a differentiable function of the
    flat core tensors; the backward is the library's adjoint (tnr_diff_backward)."""

    @staticmethod
    def forward(ctx, meta, *cores):
        I, J, R, k, p, q, seed = meta
        lib = load()
        cores = [c.detach().contiguous() for c in cores]
        _need_cuda(*cores)
        A = Mpo(I, J, R, cores)
        sa = A.to_struct()
        S = torch.empty(int(k), dtype=torch.float64, device=cores[0].device)
        h = ctypes.c_void_p()
        _check(lib.tnr_diff_forward(ctypes.byref(sa), int(k), int(p), int(q), ctypes.c_uint64(int(seed)), _ptr(S),
                                    ctypes.byref(h), _stream()), "tnr_diff_forward")
        ctx.tape = _Tape(h)
        ctx.A = A
        ctx.sa = sa
        return S

    @staticmethod
    def backward(ctx, gS):
        lib = load()
        A = ctx.A
        grads = [torch.empty_like(c) for c in A.cores]
        dA = Mpo(A.I, A.J, A.R, grads).to_struct()
        g = gS.detach().to(torch.float64).contiguous()
        _check(lib.tnr_diff_backward(ctx.tape.handle, _ptr(g), ctypes.byref(dA), _stream()), "tnr_diff_backward")
        return (None, *grads)


def tnrsvd_values(A, k, p, q, seed):
    """Differentiable S = TNrSVD(A) singular values (tol 0, max_rank K): A is an Mpo whose flat
    core tensors may require grad."""
    return TnrSvdValues.apply((A.I, A.J, A.R, int(k), int(p), int(q), int(seed)), *A.cores)


# ----------------------------------------------------------------------------------------
# Instrumentation
# ----------------------------------------------------------------------------------------
def stats_classes():
    lib = load()
    out = []
    i = 0
    while True:
        n = lib.tnr_stats_class_name(i)
        if n is None:
            return out
        out.append(n.decode())
        i += 1


def stats_enable(mask):
    load().tnr_stats_enable(int(mask))


def stats_reset():
    load().tnr_stats_reset()


def stats_work(cls=-1):
    w = ctypes.c_double(0.0)
    _check(load().tnr_stats_work(int(cls), ctypes.byref(w)), "tnr_stats_work")
    return w.value


def stats(cls=-1):
    L = ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    _check(load().tnr_stats(int(cls), ctypes.byref(L), ctypes.byref(ms)), "tnr_stats")
    return L.value, ms.value
