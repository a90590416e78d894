"""GB300-native arrow-decomposition SpMM (Gianinazzi et al., PPoPP 2024) -- Python binding.

Thin marshalling over the C-ABI of ``include/arrow.h`` (``libarrow_gb300.so``):
every step of the hot path runs in the library's CUDA kernels; PyTorch only
provides device memory and streams.  If the library is missing, importing the
handle class still works but every call raises (there is no fallback path).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import (ARROW_BF16, ARROW_F16, ARROW_F32, ARROW_GRAPH, ARROW_HOST_ONLY, ARROW_K_FUSED, ARROW_K_NORM,
                      ARROW_K_PERMUTE,
                      ARROW_K_ROWS, ARROW_K_SEGMENTS, ARROW_PRED_BAND, ARROW_PRED_BLOCK, ARROW_PROFILE,
                      ARROW_RELU, ARROW_RESCALE, ARROW_ROWNORM, ArrowError)

__all__ = ["ArrowMatrix", "ArrowBatch", "count_tiles", "ArrowServer", "ArrowError", "dtype_code", "ARROW_F32", "ARROW_BF16", "ARROW_F16"]

_DTYPE_NAMES = {"f32": ARROW_F32, "float32": ARROW_F32, "bf16": ARROW_BF16, "bfloat16": ARROW_BF16,
                "f16": ARROW_F16, "float16": ARROW_F16}


def dtype_code(dt) -> int:
    """arrow_dtype code of a name ('f32', 'bf16', 'f16'), a torch dtype or a code."""
    if isinstance(dt, int):
        return dt
    if isinstance(dt, str):
        return _DTYPE_NAMES[dt]
    import torch
    return {torch.float32: ARROW_F32, torch.bfloat16: ARROW_BF16, torch.float16: ARROW_F16}[dt]


def _torch_dtype(code: int):
    import torch
    return {ARROW_F32: torch.float32, ARROW_BF16: torch.bfloat16, ARROW_F16: torch.float16}[code]


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _csr(A):
    """(arrow_csr, arrays that must stay alive while it is used) for a host CSR object."""
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(A.colidx, dtype=np.int32)
    values = np.ascontiguousarray(A.values, dtype=np.float64)
    csr = _native.ArrowCsr(int(A.n), int(rowptr[-1]) if rowptr.size else 0, rowptr.ctypes.data,
                           colidx.ctypes.data if colidx.size else None,
                           values.ctypes.data if values.size else None)
    return csr, (rowptr, colidx, values)


def _check_open(mats, what: str) -> None:
    """The C side holds raw handle pointers: refuse to run on a matrix that was closed."""
    for m in mats:
        if not (getattr(m, "_h", None) and m._h.value):
            raise ArrowError(_native.ARROW_ESTATE, f"{what}: a matrix it uses was closed")


def count_tiles(A, b: int) -> int:
    """``arrow_count_tiles``: distinct non-zero b x b tiles of A in its own order."""
    csr, _keep = _csr(A)
    t = ctypes.c_int64()
    _native.check(_native.lib().arrow_count_tiles(ctypes.byref(csr), int(b), ctypes.byref(t)))
    return int(t.value)


class ArrowMatrix:
    """A decomposed matrix: ``arrow_decompose`` on construction, ``arrow_free`` on close.

    ``A`` is any object with ``n``, ``rowptr`` (int64), ``colidx`` (int32) and
    ``values`` (float64) in CSR form (host memory).
    """

    def __init__(self, A, b: int, *, seed: int = 0, value_dtype="f32", predicate: str = "block",
                 host_only: bool = False, nthreads: int = 0, max_levels: int = 0, long_row: int = 0,
                 segment: int = 0, device: int = -1, device_decompose: bool = False):
        L = _native.lib()
        self._h = ctypes.c_void_p()
        csr, _keep = _csr(A)
        o = _native.ArrowOpts()
        _native.check(L.arrow_opts_default(ctypes.byref(o)))
        o.seed = seed
        o.value_dtype = dtype_code(value_dtype)
        o.predicate = {"block": ARROW_PRED_BLOCK, "band": ARROW_PRED_BAND}[predicate]
        o.flags = (ARROW_HOST_ONLY if host_only else 0) | (_native.ARROW_DEVICE_DECOMPOSE if device_decompose else 0)
        o.nthreads = nthreads
        o.max_levels = max_levels
        o.long_row = long_row
        o.segment = segment
        o.device = device
        _native.check(L.arrow_decompose(ctypes.byref(csr), int(b), ctypes.byref(o), ctypes.byref(self._h)))
        self.n = int(A.n)
        self.nnz = int(csr.nnz)
        self.b = int(b)
        self.value_dtype = o.value_dtype

    # ---- lifetime --------------------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _native.lib().arrow_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def save(self, path) -> None:
        """``arrow_save``: write the decomposition (host state) to ``path``."""
        _native.check(_native.lib().arrow_save(self._h, str(path).encode()))

    @classmethod
    def load(cls, path, *, value_dtype=None, host_only: bool = False, device: int = -1) -> "ArrowMatrix":
        """``arrow_load``: a handle from a file written by :meth:`save`."""
        L = _native.lib()
        o = _native.ArrowOpts()
        _native.check(L.arrow_opts_default(ctypes.byref(o)))
        o.value_dtype = -1 if value_dtype is None else dtype_code(value_dtype)
        o.flags = ARROW_HOST_ONLY if host_only else 0
        o.device = device
        out = cls.__new__(cls)
        out._h = ctypes.c_void_p()
        _native.check(L.arrow_load(str(path).encode(), ctypes.byref(o), ctypes.byref(out._h)))
        st = out.stats()
        out.n, out.nnz, out.b, out.value_dtype = st["n"], st["nnz"], st["b"], st["value_dtype"]
        return out

    def copy(self, value_dtype) -> "ArrowMatrix":
        """``arrow_handle_copy``: same decomposition, values stored in ``value_dtype``."""
        out = ArrowMatrix.__new__(ArrowMatrix)
        out._h = ctypes.c_void_p()
        _native.check(_native.lib().arrow_handle_copy(self._h, dtype_code(value_dtype), ctypes.byref(out._h)))
        out.n, out.nnz, out.b, out.value_dtype = self.n, self.nnz, self.b, dtype_code(value_dtype)
        return out

    def upload(self) -> None:
        _native.check(_native.lib().arrow_upload(self._h))

    # ---- structure export ------------------------------------------------------------
    @property
    def num_levels(self) -> int:
        l = ctypes.c_int32()
        _native.check(_native.lib().arrow_num_levels(self._h, ctypes.byref(l)))
        return int(l.value)

    def level_info(self, i: int):
        na, nz = ctypes.c_int64(), ctypes.c_int64()
        _native.check(_native.lib().arrow_level_info(self._h, i, ctypes.byref(na), ctypes.byref(nz)))
        return int(na.value), int(nz.value)

    def level_perm(self, i: int) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int32)
        _native.check(_native.lib().arrow_level_perm(self._h, i, out.ctypes.data))
        return out

    def level_csr(self, i: int):
        _, nz = self.level_info(i)
        rowptr = np.empty(self.n + 1, dtype=np.int64)
        colidx = np.empty(max(nz, 1), dtype=np.int32)
        vals = np.empty(max(nz, 1), dtype=np.float64)
        _native.check(_native.lib().arrow_level_csr(self._h, i, rowptr.ctypes.data, colidx.ctypes.data,
                                                    vals.ctypes.data))
        return rowptr, colidx[:nz], vals[:nz]

    def level_shape(self, i: int) -> dict:
        """``arrow_get_level_shape``: n_active, nnz, head_nnz, band_nnz and non-zero tiles of B_i."""
        sh = _native.ArrowLevelShape()
        _native.check(_native.lib().arrow_get_level_shape(self._h, int(i), ctypes.byref(sh)))
        return {f: int(getattr(sh, f)) for f, _ in sh._fields_}

    def program(self) -> dict:
        """``arrow_get_program``: copies of the fused row program the kernels run (numpy int32)."""
        pg = _native.ArrowProgram()
        _native.check(_native.lib().arrow_get_program(self._h, ctypes.byref(pg)))
        sizes = {"rowptr": pg.n + 1, "col": pg.n_short, "src": pg.n_short, "lcol": pg.n_long_entries,
                 "lsrc": pg.n_long_entries, "long_rows": pg.n_long_rows, "long_segptr": pg.n_long_rows + 1,
                 "seg_begin": pg.n_segments, "seg_end": pg.n_segments, "tile_row": pg.n_tiles + 1,
                 "tile_ent": pg.n_tiles + 1}
        out = {"long_row": int(pg.long_row)}
        for f, cnt in sizes.items():
            ptr = getattr(pg, f)
            out[f] = np.ctypeslib.as_array(ptr, shape=(int(cnt),)).copy() if cnt > 0 and ptr else np.zeros(0, np.int32)
        return out

    def structure_report(self) -> dict:
        """Every level's shape plus the totals: the order l, the non-zero tiles summed over the
        levels, and each level's share of the entries and of the rows."""
        levels = [self.level_shape(i) for i in range(self.num_levels)]
        for lv in levels:
            lv["nnz_share"] = lv["nnz"] / max(1, self.nnz)
            lv["row_share"] = lv["n_active"] / max(1, self.n)
        return {"n": self.n, "nnz": self.nnz, "b": self.b, "levels": levels,
                "tiles": sum(lv["tiles"] for lv in levels)}

    def status(self) -> int:
        """Read and clear the device status word (raises ArrowError on a timed-out wait)."""
        st = ctypes.c_int32()
        _native.check(_native.lib().arrow_status(self._h, ctypes.byref(st)))
        return int(st.value)

    def stats(self) -> dict:
        s = _native.ArrowStats()
        _native.check(_native.lib().arrow_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    # ---- the hot path ------------------------------------------------------------------
    def _check_x(self, X):
        import torch
        if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dim() == 2 and X.shape[0] == self.n
                and X.is_contiguous()):
            raise ValueError("X must be a contiguous CUDA tensor of shape (n, k)")
        return dtype_code(X.dtype)

    def spmm(self, X, iters: int = 1, *, rescale: bool = False, relu: bool = False, rownorm: bool = False,
             out=None, stream=None, profile: bool = False):
        """Y = X_iters of X_{t+1} = sigma(A X_t) through ``arrow_spmm`` (returns Y); sigma =
        colnorm(rownorm(relu(.))) with each part switched by its argument."""
        import torch
        xd = self._check_x(X)
        if out is None:
            out = torch.empty_like(X)
        elif out.shape != X.shape or out.dtype != X.dtype or not out.is_contiguous():
            raise ValueError("out must match X")
        flags = ((ARROW_RESCALE if rescale else 0) | (ARROW_PROFILE if profile else 0) | (ARROW_RELU if relu else 0)
                 | (ARROW_ROWNORM if rownorm else 0))
        _native.check(_native.lib().arrow_spmm(self._h, ctypes.c_void_p(X.data_ptr()), X.shape[1], int(iters),
                                               ctypes.c_void_p(out.data_ptr()), xd, flags, _stream_ptr(stream)))
        return out

    def profile_get(self, kernel: int = ARROW_K_ROWS):
        """(total ms, launches) of the kernel class recorded by profiled calls since the last read."""
        ms, cnt = ctypes.c_double(), ctypes.c_int64()
        _native.check(_native.lib().arrow_profile_get(self._h, int(kernel), ctypes.byref(ms), ctypes.byref(cnt)))
        return float(ms.value), int(cnt.value)

    @property
    def tuning(self) -> dict:
        t = _native.ArrowTuning()
        _native.check(_native.lib().arrow_get_tuning(self._h, ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in t._fields_}

    def set_tuning(self, tile_rows: int, tile_nnz: int, ctas_per_sm: int, carveout: int,
                   fold_permute_in: int | None = None, fused_small: int | None = None) -> None:
        cur = self.tuning
        if fold_permute_in is None:
            fold_permute_in = cur["fold_permute_in"]
        if fused_small is None:
            fused_small = cur["fused_small"]
        t = _native.ArrowTuning(int(tile_rows), int(tile_nnz), int(ctas_per_sm), int(carveout), int(fold_permute_in),
                                int(fused_small))
        _native.check(_native.lib().arrow_set_tuning(self._h, ctypes.byref(t)))

    def autotune(self, X, iters: int, *, rescale: bool = False, out=None, stream=None):
        """``arrow_autotune`` on X: keeps the fastest tuning; returns (tuning dict, ms per call)."""
        import torch
        xd = self._check_x(X)
        if out is None:
            out = torch.empty_like(X)
        t = _native.ArrowTuning()
        ms = ctypes.c_double()
        _native.check(_native.lib().arrow_autotune(self._h, ctypes.c_void_p(X.data_ptr()),
                                                   ctypes.c_void_p(out.data_ptr()), X.shape[1], int(iters), xd,
                                                   ARROW_RESCALE if rescale else 0, _stream_ptr(stream),
                                                   ctypes.byref(t), ctypes.byref(ms)))
        return {f: getattr(t, f) for f, _ in t._fields_}, ms.value

    def workspace_size(self, k: int, dtype="f32", rescale: bool = False) -> int:
        sz = ctypes.c_size_t()
        _native.check(_native.lib().arrow_workspace_size(self._h, int(k), dtype_code(dtype),
                                                         ARROW_RESCALE if rescale else 0, ctypes.byref(sz)))
        return int(sz.value)

    def spmm_ws(self, X, iters: int, workspace, *, rescale: bool = False, out=None, stream=None):
        """``arrow_spmm_ws``: like :meth:`spmm` with a caller-owned uint8 CUDA workspace tensor."""
        import torch
        xd = self._check_x(X)
        if out is None:
            out = torch.empty_like(X)
        flags = ARROW_RESCALE if rescale else 0
        _native.check(_native.lib().arrow_spmm_ws(self._h, ctypes.c_void_p(X.data_ptr()), X.shape[1], int(iters),
                                                  ctypes.c_void_p(out.data_ptr()), xd, flags,
                                                  ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                                  _stream_ptr(stream)))
        return out

    def algorithmic_bytes_per_iter(self, k: int, x_dtype="f32") -> dict:
        """Bytes one iteration must move (see the design notes): A's values and indices,
        the row pointers, every level's active rows of X read once, Y written once."""
        sv = 4 if self.value_dtype == ARROW_F32 else 2
        sx = 4 if dtype_code(x_dtype) == ARROW_F32 else 2
        total_active = sum(self.level_info(i)[0] for i in range(self.num_levels))
        a_bytes = self.nnz * (sv + 4) + 4 * (self.n + 1)
        x_bytes = total_active * k * sx
        y_bytes = self.n * k * sx
        return {"A": a_bytes, "X": x_bytes, "Y": y_bytes, "total": a_bytes + x_bytes + y_bytes}


class ArrowBatch:
    """``arrow_batch_create`` over uploaded :class:`ArrowMatrix` handles (kept alive here)."""

    def __init__(self, mats):
        self.mats = list(mats)
        arr = (ctypes.c_void_p * len(self.mats))(*[m._h.value for m in self.mats])
        self._b = ctypes.c_void_p()
        _native.check(_native.lib().arrow_batch_create(arr, len(self.mats), ctypes.byref(self._b)))

    def spmm(self, Xs, iters: int, *, outs=None, graph: bool = False, stream=None):
        """Ys[m] = A_m^iters Xs[m] for every matrix in one ``arrow_batch_spmm`` call."""
        import torch
        if len(Xs) != len(self.mats):
            raise ValueError("one X per matrix")
        if outs is None:
            outs = [torch.empty_like(x) for x in Xs]
        xd = {dtype_code(x.dtype) for x in Xs}
        if len(xd) != 1:
            raise ValueError("all X must share one dtype")
        for m, x, y in zip(self.mats, Xs, outs):
            if not (x.is_cuda and x.is_contiguous() and x.dim() == 2 and x.shape[0] == m.n and y.shape == x.shape
                    and y.dtype == x.dtype and y.is_contiguous()):
                raise ValueError("X[m], Y[m] must be contiguous CUDA (n_m, k_m) tensors of one dtype")
        n = len(Xs)
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in Xs])
        yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in outs])
        ks = (ctypes.c_int64 * n)(*[x.shape[1] for x in Xs])
        _check_open(self.mats, "arrow_batch_spmm")
        _native.check(_native.lib().arrow_batch_spmm(self._b, xp, yp, ks, int(iters), xd.pop(),
                                                     ARROW_GRAPH if graph else 0, _stream_ptr(stream)))
        return outs

    def status(self) -> int:
        st = ctypes.c_int32()
        _native.check(_native.lib().arrow_batch_status(self._b, ctypes.byref(st)))
        return int(st.value)

    def autotune(self, Xs, iters: int, *, outs=None, stream=None):
        """``arrow_batch_autotune``: keeps the fastest tuning on every handle; (tuning, ms per call)."""
        import torch
        if outs is None:
            outs = [torch.empty_like(x) for x in Xs]
        n = len(Xs)
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in Xs])
        yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in outs])
        ks = (ctypes.c_int64 * n)(*[x.shape[1] for x in Xs])
        t = _native.ArrowTuning()
        ms = ctypes.c_double()
        _check_open(self.mats, "arrow_batch_autotune")
        _native.check(_native.lib().arrow_batch_autotune(self._b, xp, yp, ks, int(iters), dtype_code(Xs[0].dtype),
                                                         _stream_ptr(stream), ctypes.byref(t), ctypes.byref(ms)))
        return {f: getattr(t, f) for f, _ in t._fields_}, ms.value

    def close(self) -> None:
        if getattr(self, "_b", None) and self._b.value:
            _native.lib().arrow_batch_free(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ArrowServer:
    """Continuous-batching server (``arrow_server_*``): submit requests, step, poll completions."""

    def __init__(self, hbm_budget: int, max_active: int, x_dtype="bf16", max_inflight: int = 2, device: int = -1):
        o = _native.ArrowServerOpts(int(hbm_budget), int(max_active), dtype_code(x_dtype), int(max_inflight),
                                    int(device))
        self._s = ctypes.c_void_p()
        _native.check(_native.lib().arrow_server_create(ctypes.byref(o), ctypes.byref(self._s)))
        self._keep = {}

    def submit(self, M: ArrowMatrix, X, Y, iters: int) -> int:
        """Queue Y = A^iters X (X, Y contiguous CUDA tensors kept alive until completion)."""
        rid = ctypes.c_int64()
        _native.check(_native.lib().arrow_server_submit(self._s, M._h, ctypes.c_void_p(X.data_ptr()),
                                                        ctypes.c_void_p(Y.data_ptr()), int(X.shape[1]), int(iters),
                                                        ctypes.byref(rid)))
        self._keep[rid.value] = (M, X, Y)
        return rid.value

    def step(self, stream=None) -> int:
        act = ctypes.c_int32()
        _native.check(_native.lib().arrow_server_step(self._s, _stream_ptr(stream), ctypes.byref(act)))
        return act.value

    def poll(self, max_items: int = 4096):
        """[(id, latency_seconds)] completed since the last poll."""
        ids = (ctypes.c_int64 * max_items)()
        lat = (ctypes.c_double * max_items)()
        cnt = ctypes.c_int32()
        _native.check(_native.lib().arrow_server_poll(self._s, ids, lat, max_items, ctypes.byref(cnt)))
        out = [(ids[i], lat[i]) for i in range(cnt.value)]
        for rid, _ in out:
            self._keep.pop(rid, None)
        return out

    def drain(self, stream=None) -> None:
        _native.check(_native.lib().arrow_server_drain(self._s, _stream_ptr(stream)))

    def stats(self) -> dict:
        st = _native.ArrowServerStats()
        _native.check(_native.lib().arrow_server_get_stats(self._s, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self) -> None:
        if getattr(self, "_s", None) and self._s.value:
            _native.lib().arrow_server_free(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
