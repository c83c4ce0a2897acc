"""Handle: one C-ABI handle plus argument marshalling for torch CUDA tensors."""
from __future__ import annotations

import ctypes

from ._lib import APSP_AUTO, APSP_F32, APSP_I32, APSP_U16, ApspError, apsp_config, apsp_request, get_lib

_DT_NAMES = {"int32": APSP_I32, "i32": APSP_I32, "u16": APSP_U16, "uint16": APSP_U16, "u16x2": APSP_U16,
             "int16": APSP_U16, "fp32": APSP_F32, "f32": APSP_F32, "float32": APSP_F32, "auto": APSP_AUTO}


def dtype_code(d) -> int:
    """apsp_dtype code from a name, a code, or a torch dtype."""
    if isinstance(d, int):
        return d
    if isinstance(d, str):
        return _DT_NAMES[d.lower()]
    import torch
    if d == torch.int32:
        return APSP_I32
    if d in (torch.int16, getattr(torch, "uint16", torch.int16)):
        return APSP_U16
    if d == torch.float32:
        return APSP_F32
    raise ValueError(f"unsupported dtype {d}")


def _elem_ok(t, code):
    import torch
    want = {APSP_I32: (torch.int32,), APSP_AUTO: (torch.int32,), APSP_F32: (torch.float32,),
            APSP_U16: (torch.int16, getattr(torch, "uint16", torch.int16))}[code]
    if t.dtype not in want:
        raise TypeError(f"tensor dtype {t.dtype} does not match apsp dtype {code}")


def _mat(t, name):
    if t.dim() != 2 or t.stride(1) != 1 or t.shape[1] < t.shape[0]:
        raise ValueError(f"{name} must be a row-major (n, >=n) matrix view with unit column stride")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    return t.shape[0], t.stride(0)


def _stream(stream, device):
    import torch
    if stream is None:
        return torch.cuda.current_stream(device).cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _L():
    return get_lib()


_TORCH_DT = {APSP_I32: "int32", APSP_U16: "int16", APSP_F32: "float32"}


def tri_layout(dtype, n: int):
    """apsp_tri_layout: (rows, ld, bytes) of the upper-triangular layout's rectangle for n."""
    r, l, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    st = _L().apsp_tri_layout(dtype_code(dtype), n, ctypes.byref(r), ctypes.byref(l), ctypes.byref(b))
    if st != 0:
        raise ApspError(st, "apsp_tri_layout")
    return int(r.value), int(l.value), int(b.value)


def tri_empty(dtype, n: int, device=0):
    """A device tensor shaped as the upper-triangular layout's rectangle (rows, ld) for n."""
    import torch
    code = dtype_code(dtype)
    rows, ld, _ = tri_layout(code, n)
    return torch.empty((rows, ld), dtype=getattr(torch, _TORCH_DT[code]), device=device)


def tri_to_dense(dtype, T, n: int, D=None, stream=None):
    """apsp_tri_to_dense: the full n x n matrix held in T (allocated when D is None)."""
    import torch
    code = dtype_code(dtype)
    if D is None:
        D = torch.empty((n, n), dtype=T.dtype, device=T.device)
    nd, ld = _mat(D, "D")
    st = _L().apsp_tri_to_dense(code, T.data_ptr(), n, D.data_ptr(), ld, _stream(stream, T.device))
    if st != 0:
        raise ApspError(st, "apsp_tri_to_dense")
    return D


def tri_rows(dtype, T, n: int, rows, out=None, stream=None):
    """apsp_tri_rows: rows `rows` (a 1-D int64 CUDA tensor) of the full matrix held in T."""
    import torch
    code = dtype_code(dtype)
    if rows.dtype != torch.int64 or not rows.is_cuda or not rows.is_contiguous():
        raise TypeError("rows must be a contiguous int64 CUDA tensor")
    k = rows.numel()
    if out is None:
        out = torch.empty((k, n), dtype=T.dtype, device=T.device)
    if out.dim() != 2 or out.stride(1) != 1 or out.shape[0] < k or out.shape[1] < n:
        raise ValueError("out must be a row-major (k, >=n) matrix")
    st = _L().apsp_tri_rows(code, T.data_ptr(), n, rows.data_ptr(), k, out.data_ptr(), out.stride(0),
                            _stream(stream, T.device))
    if st != 0:
        raise ApspError(st, "apsp_tri_rows")
    return out


class Handle:
    """Owns one ``apsp_handle`` (workspace, serving thread) on one device."""

    def __init__(self, device: int = 0, dtype="int32", max_batch: int = 64, queue_depth: int = 4096,
                 memory_budget: int = 0, spin_limit: int = 0, block_k: int = 0, phase3_variant: int = 0,
                 symmetric: int = 0, serving_large_n: int = 0, serving_large_grid: int = 0):
        cfg = apsp_config()
        _L().apsp_config_default(ctypes.byref(cfg))
        cfg.device = device
        cfg.dtype = dtype_code(dtype)
        cfg.max_batch = max_batch
        cfg.queue_depth = queue_depth
        cfg.memory_budget = memory_budget
        cfg.spin_limit = spin_limit
        cfg.block_k = block_k
        cfg.phase3_variant = phase3_variant
        cfg.symmetric = symmetric
        cfg.serving_large_n = serving_large_n
        cfg.serving_large_grid = serving_large_grid
        h = ctypes.c_void_p()
        st = _L().apsp_create(ctypes.byref(h), ctypes.byref(cfg))
        if st != 0:
            raise ApspError(st, "apsp_create")
        self._h = h
        self.device = device
        self.dtype = cfg.dtype
        self._hold = {}  # tickets -> host/device buffers kept alive until admission

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None):
            _L().apsp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st, where):
        if st != 0:
            detail = _L().apsp_last_error(self._h).decode() if self._h else ""
            raise ApspError(st, where, detail)

    @property
    def launch_count(self) -> int:
        return int(_L().apsp_launch_count(self._h))

    def profile(self, enable: bool = True):
        """apsp_profile: record CUDA events around every phase launch of later solves."""
        self._check(_L().apsp_profile(self._h, 1 if enable else 0), "apsp_profile")

    def profile_read(self):
        """apsp_profile_read: per phase (1, 2, 3) -> (launches, device ms, relaxations); clears the record."""
        L = (ctypes.c_int64 * 3)()
        M = (ctypes.c_double * 3)()
        R = (ctypes.c_double * 3)()
        self._check(_L().apsp_profile_read(self._h, L, M, R), "apsp_profile_read")
        return {p + 1: (int(L[p]), float(M[p]), float(R[p])) for p in range(3)}

    # ------------------------------------------------------------ solves
    def solve_t(self, dtype, W, D=None, stream=None):
        """apsp_solve_t: D (allocated like W when None) <- APSP of W; returns D."""
        import torch
        code = dtype_code(dtype)
        n, ld = _mat(W, "W")
        _elem_ok(W, code)
        if D is None:
            D = torch.empty_like(W)
        nd, ldd = _mat(D, "D")
        if nd != n or ldd != ld or D.dtype != W.dtype:
            raise ValueError("D must have W's shape, leading dimension and dtype")
        self._check(_L().apsp_solve_t(self._h, code, W.data_ptr(), n, ld, D.data_ptr(), _stream(stream, W.device)),
                    "apsp_solve_t")
        return D

    def solve_squaring(self, dtype, W, D=None, stream=None):
        """apsp_solve_squaring: D (allocated like W when None) <- APSP of W by repeated min-plus squaring
        (Alg. 1); returns D."""
        import torch
        code = dtype_code(dtype)
        n, ld = _mat(W, "W")
        _elem_ok(W, code)
        if D is None:
            D = torch.empty_like(W)
        nd, ldd = _mat(D, "D")
        if nd != n or ldd != ld or D.dtype != W.dtype:
            raise ValueError("D must have W's shape, leading dimension and dtype")
        self._check(_L().apsp_solve_squaring(self._h, code, W.data_ptr(), n, ld, D.data_ptr(),
                                             _stream(stream, W.device)), "apsp_solve_squaring")
        return D

    def tri_from_dense(self, dtype, W, T=None, stream=None):
        """apsp_tri_from_dense: T (allocated when None) <- the upper-triangular layout of the symmetric W."""
        code = dtype_code(dtype)
        n, ld = _mat(W, "W")
        _elem_ok(W, code)
        if T is None:
            T = tri_empty(code, n, W.device)
        self._check(_L().apsp_tri_from_dense(self._h, code, W.data_ptr(), n, ld, T.data_ptr(),
                                             _stream(stream, W.device)), "apsp_tri_from_dense")
        return T

    def tri_from_edges(self, dtype, src, dst, w, n, T=None, stream=None):
        """apsp_tri_from_edges: T (allocated when None) <- an undirected edge list's adjacency matrix."""
        import torch
        code = dtype_code(dtype)
        if T is None:
            T = tri_empty(code, n, src.device)
        m = src.numel()
        for t in (src, dst):
            if t.dtype != torch.int32 or not t.is_cuda or not t.is_contiguous():
                raise TypeError("src/dst must be contiguous int32 CUDA tensors")
        if not w.is_contiguous() or not w.is_cuda or w.numel() != m:
            raise TypeError("w must be a contiguous CUDA tensor of m weights")
        self._check(_L().apsp_tri_from_edges(self._h, code, src.data_ptr(), dst.data_ptr(), w.data_ptr(), m, n,
                                             T.data_ptr(), _stream(stream, T.device)), "apsp_tri_from_edges")
        return T

    def solve_tri(self, dtype, T, n: int, stream=None):
        """apsp_solve_tri: APSP in place on T (upper-triangular layout); returns T."""
        self._check(_L().apsp_solve_tri(self._h, dtype_code(dtype), T.data_ptr(), n, _stream(stream, T.device)),
                    "apsp_solve_tri")
        return T

    def solve(self, W, D=None, stream=None):
        """apsp_solve with the handle's dtype."""
        return self.solve_t(self.dtype, W, D, stream)

    def solve_edges(self, dtype, src, dst, w, n, D=None, stream=None):
        """apsp_solve_edges: D (n x n, allocated when None) from an undirected edge list."""
        import torch
        code = dtype_code(dtype)
        if D is None:
            tdt = {APSP_I32: torch.int32, APSP_AUTO: torch.int32, APSP_F32: torch.float32,
                   APSP_U16: torch.int16}[code]
            D = torch.empty((n, n), dtype=tdt, device=src.device)
        nd, ld = _mat(D, "D")
        if nd != n:
            raise ValueError("D must have n rows")
        m = src.numel()
        for t in (src, dst):
            if t.dtype != torch.int32 or not t.is_cuda or not t.is_contiguous():
                raise TypeError("src/dst must be contiguous int32 CUDA tensors")
        if not w.is_contiguous() or not w.is_cuda or w.numel() != m:
            raise TypeError("w must be a contiguous CUDA tensor of m weights")
        self._check(_L().apsp_solve_edges(self._h, code, src.data_ptr(), dst.data_ptr(), w.data_ptr(), m, n,
                                         D.data_ptr(), ld, _stream(stream, D.device)), "apsp_solve_edges")
        return D

    def solve_batch(self, Ws, Ds=None, stream=None):
        """apsp_solve_batch: many int32 graphs of uneven n in one persistent launch; returns the D list."""
        import torch
        Ws = list(Ws)
        if Ds is None:
            Ds = [torch.empty_like(W) for W in Ws]
        k = len(Ws)
        Wp = (ctypes.c_void_p * k)()
        Dp = (ctypes.c_void_p * k)()
        ns = (ctypes.c_int64 * k)()
        lds = (ctypes.c_int64 * k)()
        for i, (W, D) in enumerate(zip(Ws, Ds)):
            n, ld = _mat(W, "W")
            _elem_ok(W, APSP_I32)
            nd, ldd = _mat(D, "D")
            if nd != n or ldd != ld or D.dtype != W.dtype:
                raise ValueError("D must have W's shape, leading dimension and dtype")
            Wp[i], Dp[i], ns[i], lds[i] = W.data_ptr(), D.data_ptr(), n, ld
        dev = Ws[0].device if Ws else torch.device("cuda", self.device)
        self._check(_L().apsp_solve_batch(self._h, k, Wp, ns, lds, Dp, _stream(stream, dev)), "apsp_solve_batch")
        return Ds

    def check_bounded_wait(self, spin_limit: int = 1 << 12) -> int:
        """apsp_check_bounded_wait: status of a batched launch and of an all-rounds launch whose first wait can never
        be satisfied (7, APSP_E_TIMEOUT, when both gave up as they should)."""
        return int(_L().apsp_check_bounded_wait(self._h, spin_limit))

    def autotune(self, dtype="int32", n_max: int = 4096, cache_path: str | None = None):
        """apsp_autotune: time the round shapes per n bucket; returns {bucket: (Bk, tma)}."""
        code = dtype_code(dtype)
        self._check(_L().apsp_autotune(self._h, code, n_max, cache_path.encode() if cache_path else None),
                    "apsp_autotune")
        out, b = {}, 128
        while True:
            out[b] = self.tuned_config(code, b)
            if b >= n_max:
                return out
            b <<= 1

    def tuned_config(self, dtype, n: int):
        """apsp_tuned_config: (Bk, tma) the handle uses for (dtype, n)."""
        bk, tma = ctypes.c_int(), ctypes.c_int()
        self._check(_L().apsp_tuned_config(self._h, dtype_code(dtype), n, ctypes.byref(bk), ctypes.byref(tma)),
                    "apsp_tuned_config")
        return int(bk.value), int(tma.value)

    def last_status(self, stream=None) -> int:
        """apsp_last_status: the device-side input check of the last solve (0 = OK)."""
        import torch
        return int(_L().apsp_last_status(self._h, _stream(stream, torch.device("cuda", self.device))))

    def int16_bound(self, W, stream=None):
        """apsp_int16_bound: (max_c 2 ecc(r_c), enabled) for an int32 adjacency matrix."""
        n, ld = _mat(W, "W")
        _elem_ok(W, APSP_I32)
        b = ctypes.c_int64()
        ok = ctypes.c_int()
        self._check(_L().apsp_int16_bound(self._h, W.data_ptr(), n, ld, ctypes.byref(b), ctypes.byref(ok),
                                         _stream(stream, W.device)), "apsp_int16_bound")
        return int(b.value), bool(ok.value)

    def minplus(self, A, B, C, stream=None):
        """apsp_minplus: C <- min(C, A (x) B) in place; returns C."""
        code = dtype_code(C.dtype)
        for t, nm in ((A, "A"), (B, "B"), (C, "C")):
            if t.dim() != 2 or t.stride(1) != 1 or not t.is_cuda:
                raise ValueError(f"{nm} must be a row-major CUDA matrix")
            _elem_ok(t, code)
        m, k = A.shape
        k2, n = B.shape
        if k2 != k or tuple(C.shape) != (m, n):
            raise ValueError("shape mismatch")
        self._check(_L().apsp_minplus(self._h, code, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                     C.data_ptr(), C.stride(0), m, k, n, _stream(stream, C.device)), "apsp_minplus")
        return C

    # ------------------------------------------------------------ request loop
    def submit(self, W, dtype="int32") -> int:
        """apsp_submit: W is an int32 (n, >=n) tensor on the host (pinned or not) or the device; dtype "int32" or
        "auto" (packed 16-bit rounds for a large request when the bound holds; the result is int32)."""
        if W.dim() != 2 or W.stride(1) != 1 or W.shape[1] < W.shape[0]:
            raise ValueError("W must be a row-major (n, >=n) matrix")
        _elem_ok(W, APSP_I32)
        r = apsp_request(W.data_ptr(), 0 if W.is_cuda else 1, W.shape[0], W.stride(0), dtype_code(dtype))
        t = ctypes.c_uint64()
        self._check(_L().apsp_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "apsp_submit")
        self._hold[int(t.value)] = W
        return int(t.value)

    def poll(self, ticket: int):
        """apsp_poll: (state code, device pointer of the result or None, status)."""
        st = ctypes.c_int()
        p = ctypes.c_void_p()
        rc = _L().apsp_poll(self._h, ticket, ctypes.byref(st), ctypes.byref(p))
        if rc == 6:
            raise ApspError(rc, "apsp_poll")
        return int(st.value), p.value, int(rc)

    def wait(self, ticket: int, timeout_ms: int = -1) -> int:
        return int(_L().apsp_wait(self._h, ticket, timeout_ms))

    def fetch(self, ticket: int, out, stream=None):
        """apsp_fetch into a (n, >=n) int32 tensor (host or device)."""
        import torch
        dev = out.device if out.is_cuda else torch.device("cuda", self.device)
        self._check(_L().apsp_fetch(self._h, ticket, out.data_ptr(), out.stride(0), _stream(stream, dev)),
                    "apsp_fetch")
        return out

    def release(self, ticket: int) -> int:
        rc = int(_L().apsp_release(self._h, ticket))
        if rc == 0:
            self._hold.pop(ticket, None)
        return rc

    def cancel(self, ticket: int) -> int:
        return int(_L().apsp_cancel(self._h, ticket))
