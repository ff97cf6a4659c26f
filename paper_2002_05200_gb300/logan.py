"""Thin Python binding of the C ABI in include/logan.h (ctypes).

Argument marshalling only: every step of the extension runs in the CUDA
kernels of ``_build/liblogan.so``.  PyTorch supplies device memory and
streams.  If the library is missing this module raises -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblogan.so")

OK = 0
EINVAL, ENOMEM, EAGAIN, ECUDA, ETIMEOUT, ECANCELED, ERANGE, ENOTFOUND = \
    -22, -12, -11, -5, -110, -125, -34, -2
OPT_GRAPHS, OPT_TIMING, OPT_FORCE_LEVEL, OPT_MAX_LEVEL, OPT_RING_CAP, OPT_PLAIN_LEVEL = 1, 2, 3, 4, 5, 6
OPT_DEVICE, OPT_MIGRATION_MB, OPT_CONCURRENT, OPT_LONG_ITEM, OPT_PACKED16 = 7, 8, 9, 10, 11
OPT_AFFINE_PACKED, OPT_MATRIX_PACKED = 12, 13
X_CLASSES = 8

RESULT_DTYPE = np.dtype([("score", "<i4"), ("left", "<i4"), ("right", "<i4"), ("status", "<i4"),
                         ("begA", "<u4"), ("begB", "<u4"), ("endA", "<u4"), ("endB", "<u4"),
                         ("cells", "<u8")])
assert RESULT_DTYPE.itemsize == 40

EXPORTED = ["logan_version", "logan_strerror", "logan_ctx_create", "logan_ctx_destroy",
            "logan_workspace_size", "logan_extend_batch", "logan_extend_batch_plain",
            "logan_extend_batch_affine", "logan_overlap_candidates", "logan_overlap_pool_words",
            "logan_overlap_pool", "logan_overlap_seeds", "logan_overlap_keep",
            "logan_traceback_batch", "logan_traceback_last_stats",
            "logan_set_option", "logan_get_option", "logan_num_levels", "logan_level_info",
            "logan_last_stats", "logan_call_stats", "logan_set_level_table",
            "logan_get_level_table", "logan_intpeak", "logan_autotune", "logan_autotune_save",
            "logan_extend_batch_noalloc", "logan_set_escalation", "logan_get_escalation",
            "logan_matrix_workspace_size", "logan_extend_batch_matrix",
            "logan_server_create", "logan_server_submit",
            "logan_server_poll", "logan_server_wait", "logan_server_cancel", "logan_server_stats",
            "logan_server_destroy"]


class SeqsT(ctypes.Structure):
    _fields_ = [("bases", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("lengths", ctypes.c_void_p), ("count", ctypes.c_uint32),
                ("packed2bit", ctypes.c_uint32), ("pool_bases", ctypes.c_uint64)]


MAX_LEVELS = 8


class StatsT(ctypes.Structure):
    _fields_ = [("level_ms", ctypes.c_float * (MAX_LEVELS + 1)), ("total_ms", ctypes.c_float),
                ("items", ctypes.c_uint32 * (MAX_LEVELS + 1)),
                ("cells", ctypes.c_uint64 * (MAX_LEVELS + 1)), ("launches", ctypes.c_uint32),
                ("packed_levels", ctypes.c_uint32)]


class TracebackStatsT(ctypes.Structure):
    _fields_ = [("sweep_ms", ctypes.c_float), ("record_ms", ctypes.c_float),
                ("walk_ms", ctypes.c_float), ("total_ms", ctypes.c_float),
                ("code_words", ctypes.c_uint64), ("record_cells", ctypes.c_uint64),
                ("launches", ctypes.c_uint32)]


class RequestT(ctypes.Structure):
    _fields_ = [("A", SeqsT), ("B", SeqsT), ("same_pool", ctypes.c_int32),
                ("seeds", ctypes.c_void_p), ("n_pairs", ctypes.c_uint32),
                ("match", ctypes.c_int32), ("mismatch", ctypes.c_int32), ("gap", ctypes.c_int32),
                ("X", ctypes.c_int32), ("X_per_pair", ctypes.c_void_p),
                ("results", ctypes.c_void_p)]


class ServerStatsT(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_uint32), ("running", ctypes.c_uint32),
                ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64),
                ("used_bytes", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64)]


class LoganError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run paper_2002_05200_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        p, i32, u32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64
        L.logan_version.restype = ctypes.c_char_p
        L.logan_strerror.restype = ctypes.c_char_p
        L.logan_strerror.argtypes = [ctypes.c_int]
        L.logan_ctx_create.argtypes = [ctypes.POINTER(p), ctypes.c_int, ctypes.c_char_p]
        L.logan_ctx_destroy.argtypes = [p]
        L.logan_ctx_destroy.restype = None
        L.logan_workspace_size.argtypes = [p, ctypes.POINTER(SeqsT), ctypes.POINTER(SeqsT), u32,
                                           ctypes.POINTER(ctypes.c_size_t)]
        ext_args = [p, ctypes.POINTER(SeqsT), ctypes.POINTER(SeqsT), p, u32, i32, i32, i32, i32, p,
                    p, ctypes.c_size_t, p, p]
        L.logan_extend_batch.argtypes = ext_args
        L.logan_extend_batch_plain.argtypes = ext_args
        L.logan_extend_batch_affine.argtypes = ext_args[:7] + [ctypes.c_int32] + ext_args[7:]
        L.logan_matrix_workspace_size.argtypes = [p, ctypes.POINTER(SeqsT), ctypes.POINTER(SeqsT),
                                                  u32, ctypes.POINTER(ctypes.c_size_t)]
        L.logan_extend_batch_matrix.argtypes = [p, ctypes.POINTER(SeqsT), ctypes.POINTER(SeqsT), p,
                                                u32, p, ctypes.c_int, i32, i32, i32, p, p,
                                                ctypes.c_size_t, p, p]
        u64 = ctypes.c_uint64
        L.logan_overlap_candidates.argtypes = [p, ctypes.POINTER(SeqsT), ctypes.c_int, u32, u32, u32,
                                               p, u64, ctypes.POINTER(u64), p]
        L.logan_overlap_pool_words.argtypes = [p, ctypes.POINTER(SeqsT), ctypes.POINTER(u64), p]
        L.logan_overlap_pool.argtypes = [p, ctypes.POINTER(SeqsT), p, u64, p, p,
                                         ctypes.POINTER(SeqsT), p]
        L.logan_overlap_seeds.argtypes = [p, p, u64, ctypes.POINTER(SeqsT), ctypes.c_int, p, p]
        L.logan_overlap_keep.argtypes = [p, p, p, u64, ctypes.POINTER(SeqsT), ctypes.POINTER(SeqsT),
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, p, p]
        L.logan_traceback_batch.argtypes = [p, ctypes.POINTER(SeqsT), ctypes.POINTER(SeqsT), p, u32,
                                            i32, i32, i32, i32, p, p, u64, p, p,
                                            ctypes.POINTER(u64), p]
        L.logan_traceback_last_stats.argtypes = [p, ctypes.POINTER(TracebackStatsT)]
        L.logan_set_option.argtypes = [p, ctypes.c_int, i64]
        L.logan_get_option.argtypes = [p, ctypes.c_int, ctypes.POINTER(i64)]
        L.logan_level_info.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]
        L.logan_last_stats.argtypes = [p, ctypes.POINTER(StatsT)]
        L.logan_call_stats.argtypes = [p, ctypes.c_int, ctypes.POINTER(StatsT)]
        L.logan_autotune.argtypes = ext_args + [ctypes.c_int, ctypes.POINTER(ctypes.c_float)]
        L.logan_autotune_save.argtypes = [p, ctypes.c_char_p]
        L.logan_server_create.argtypes = [p, ctypes.c_size_t, ctypes.c_int, u32, ctypes.POINTER(p)]
        L.logan_server_submit.argtypes = [p, ctypes.POINTER(RequestT), ctypes.POINTER(ctypes.c_uint64)]
        L.logan_server_poll.argtypes = [p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        L.logan_server_wait.argtypes = [p, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_double)]
        L.logan_server_cancel.argtypes = [p, ctypes.c_uint64]
        L.logan_server_stats.argtypes = [p, ctypes.POINTER(ServerStatsT)]
        L.logan_server_destroy.argtypes = [p]
        L.logan_extend_batch_noalloc.argtypes = [p, ctypes.POINTER(SeqsT), ctypes.POINTER(SeqsT),
                                                 p, u32, i32, i32, i32, i32, p, p, p]
        L.logan_intpeak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)]
        L.logan_set_level_table.argtypes = [p, ctypes.POINTER(ctypes.c_int8), ctypes.c_int]
        L.logan_get_level_table.argtypes = [p, ctypes.POINTER(ctypes.c_int8), ctypes.c_int]
        L.logan_set_escalation.argtypes = [p, ctypes.POINTER(ctypes.c_int8), ctypes.c_int]
        L.logan_get_escalation.argtypes = [p, ctypes.POINTER(ctypes.c_int8), ctypes.c_int]
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().logan_strerror(code).decode()


def version() -> str:
    return lib().logan_version().decode()


def num_levels() -> int:
    return int(lib().logan_num_levels())


def level_info(level: int):
    w, t = ctypes.c_int(), ctypes.c_int()
    _check(lib().logan_level_info(level, ctypes.byref(w), ctypes.byref(t)), "level_info")
    return w.value, t.value


def intpeak(device: int = 0, op: int = 0, iters: int = 4000):
    """(thread-instructions per second, ms) of the integer microbenchmark."""
    r, ms = ctypes.c_double(), ctypes.c_float()
    _check(lib().logan_intpeak(device, op, iters, ctypes.byref(r), ctypes.byref(ms)),
           "logan_intpeak")
    return r.value, ms.value


def _check(rc: int, what: str):
    if rc != OK:
        raise LoganError(rc, what)


@dataclass
class DevicePool:
    """Sequences resident on the device (torch tensors) + their C view."""
    bases: "torch.Tensor"       # uint8 ASCII, or int32 words holding 2-bit codes
    offsets: "torch.Tensor"     # int64 (read as uint64)
    lengths: "torch.Tensor"     # int32 (read as uint32)
    packed2bit: bool
    pool_bases: int

    @property
    def count(self) -> int:
        return int(self.lengths.numel())

    def c(self) -> SeqsT:
        return SeqsT(self.bases.data_ptr() if self.bases.numel() else None,
                     self.offsets.data_ptr() if self.count else None,
                     self.lengths.data_ptr() if self.count else None,
                     self.count, 1 if self.packed2bit else 0, self.pool_bases)


def pool_to_device(bases: np.ndarray, offsets: np.ndarray, lengths: np.ndarray,
                   packed2bit: bool, pool_bases: int, device="cuda") -> DevicePool:
    import torch
    if packed2bit:
        b = torch.from_numpy(np.ascontiguousarray(bases).view(np.int32)).to(device)
    else:
        b = torch.from_numpy(np.ascontiguousarray(bases, dtype=np.uint8)).to(device)
    o = torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.uint64).view(np.int64)).to(device)
    n = torch.from_numpy(np.ascontiguousarray(lengths, dtype=np.uint32).view(np.int32)).to(device)
    return DevicePool(b, o, n, packed2bit, int(pool_bases))


def seeds_to_device(seeds: np.ndarray, device="cuda"):
    import torch
    arr = np.stack([seeds[f] for f in ("idxA", "idxB", "posA", "posB", "len")], axis=1)
    return torch.from_numpy(np.ascontiguousarray(arr.astype(np.uint32)).view(np.int32)).to(device)


def results_to_numpy(out) -> np.ndarray:
    """Device result tensor (int32 [n, 10]) -> structured array of RESULT_DTYPE."""
    return out.cpu().numpy().view(RESULT_DTYPE).reshape(-1)


class Context:
    """A library context on one GPU (logan_ctx_t)."""

    def __init__(self, device: int = 0, autotune_json: Optional[str] = None):
        self._h = ctypes.c_void_p()
        _check(lib().logan_ctx_create(ctypes.byref(self._h), device,
                                      autotune_json.encode() if autotune_json else None),
               "logan_ctx_create")
        self.device = device

    def close(self):
        if self._h:
            lib().logan_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, opt: int, value: int):
        _check(lib().logan_set_option(self._h, opt, int(value)), "logan_set_option")

    def get_option(self, opt: int) -> int:
        v = ctypes.c_int64()
        _check(lib().logan_get_option(self._h, opt, ctypes.byref(v)), "logan_get_option")
        return v.value

    def set_level_table(self, levels):
        arr = (ctypes.c_int8 * X_CLASSES)(*[int(v) for v in levels])
        _check(lib().logan_set_level_table(self._h, arr, X_CLASSES), "logan_set_level_table")

    def level_table(self):
        arr = (ctypes.c_int8 * X_CLASSES)()
        _check(lib().logan_get_level_table(self._h, arr, X_CLASSES), "logan_get_level_table")
        return list(arr)

    def autotune(self, A: DevicePool, B: DevicePool, seeds, match=1, mismatch=-1, gap=-1, X=50,
                 X_per_pair=None, reps: int = 2, save: Optional[str] = None, stream=None):
        """Times every start level per X class on this sample batch and keeps
        the fastest in the context's table; returns (table, ms[class][level]).
        Runs on `stream` (a torch stream; default the current one -- the legacy
        default stream cannot be captured, so graphs need another)."""
        import torch
        n = int(seeds.shape[0])
        ws = self.workspace(A, B, n)
        out = torch.empty((max(n, 1), 10), dtype=torch.int32, device=f"cuda:{self.device}")
        nl = num_levels()
        ms = (ctypes.c_float * (X_CLASSES * nl))()
        ca, cb = A.c(), B.c()
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        _check(lib().logan_autotune(self._h, ctypes.byref(ca), ctypes.byref(cb), seeds.data_ptr(),
                                    n, match, mismatch, gap, X,
                                    X_per_pair.data_ptr() if X_per_pair is not None else None,
                                    ws.data_ptr(), ws.numel(), out.data_ptr(),
                                    ctypes.c_void_p(stream.cuda_stream), reps, ms),
               "logan_autotune")
        if save:
            _check(lib().logan_autotune_save(self._h, save.encode()), "logan_autotune_save")
        grid = [[ms[c * nl + l] for l in range(nl)] for c in range(X_CLASSES)]
        return self.level_table(), grid

    def set_escalation(self, nxt):
        n = num_levels()
        arr = (ctypes.c_int8 * n)(*[int(v) for v in nxt])
        _check(lib().logan_set_escalation(self._h, arr, n), "logan_set_escalation")

    def escalation(self):
        n = num_levels()
        arr = (ctypes.c_int8 * n)()
        _check(lib().logan_get_escalation(self._h, arr, n), "logan_get_escalation")
        return list(arr)

    def workspace_size(self, A: DevicePool, B: DevicePool, n_pairs: int) -> int:
        n = ctypes.c_size_t()
        ca, cb = A.c(), B.c()
        _check(lib().logan_workspace_size(self._h, ctypes.byref(ca), ctypes.byref(cb), n_pairs,
                                          ctypes.byref(n)), "logan_workspace_size")
        return n.value

    def workspace(self, A: DevicePool, B: DevicePool, n_pairs: int):
        import torch
        return torch.empty(max(1, self.workspace_size(A, B, n_pairs)), dtype=torch.uint8,
                           device=f"cuda:{self.device}")

    def extend(self, A: DevicePool, B: DevicePool, seeds, match: int = 1, mismatch: int = -1,
               gap: int = -1, X: int = 50, X_per_pair=None, workspace=None, out=None,
               stream=None, plain: bool = False):
        """Runs logan_extend_batch(_plain); returns the int32 [n, 10] result tensor
        (asynchronous on `stream`, default torch's current stream)."""
        import torch
        n = int(seeds.shape[0])
        if out is None:
            out = torch.empty((max(n, 1), 10), dtype=torch.int32, device=f"cuda:{self.device}")
        if workspace is None:
            workspace = self.workspace(A, B, n)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        ca, cb = A.c(), B.c()
        fn = lib().logan_extend_batch_plain if plain else lib().logan_extend_batch
        rc = fn(self._h, ctypes.byref(ca), ctypes.byref(cb),
                seeds.data_ptr() if n else None, n, match, mismatch, gap, X,
                X_per_pair.data_ptr() if X_per_pair is not None else None,
                workspace.data_ptr(), workspace.numel(), out.data_ptr(),
                ctypes.c_void_p(stream.cuda_stream))
        _check(rc, "logan_extend_batch_plain" if plain else "logan_extend_batch")
        return out[:n]

    def extend_affine(self, A: DevicePool, B: DevicePool, seeds, match: int = 1,
                      mismatch: int = -1, gap_open: int = -2, gap_extend: int = -1, X: int = 50,
                      X_per_pair=None, workspace=None, out=None, stream=None):
        """Runs logan_extend_batch_affine (a gap of length L scores
        gap_open + L * gap_extend); returns the int32 [n, 10] result tensor."""
        import torch
        n = int(seeds.shape[0])
        if out is None:
            out = torch.empty((max(n, 1), 10), dtype=torch.int32, device=f"cuda:{self.device}")
        if workspace is None:
            workspace = self.workspace(A, B, n)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        ca, cb = A.c(), B.c()
        rc = lib().logan_extend_batch_affine(
            self._h, ctypes.byref(ca), ctypes.byref(cb), seeds.data_ptr() if n else None, n,
            match, mismatch, gap_open, gap_extend, X,
            X_per_pair.data_ptr() if X_per_pair is not None else None, workspace.data_ptr(),
            workspace.numel(), out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        _check(rc, "logan_extend_batch_affine")
        return out[:n]

    def extend_matrix(self, A: DevicePool, B: DevicePool, seeds, matrix, gap_open: int = -10,
                      gap_extend: int = -1, X: int = 50, X_per_pair=None, workspace=None,
                      out=None, stream=None):
        """Runs logan_extend_batch_matrix: pools of letter codes (one byte
        each, < K), the K x K matrix (host array), affine gaps; returns the
        int32 [n, 10] result tensor."""
        import torch
        M = np.ascontiguousarray(matrix, dtype=np.int32)
        K = int(M.shape[0])
        n = int(seeds.shape[0])
        if out is None:
            out = torch.empty((max(n, 1), 10), dtype=torch.int32, device=f"cuda:{self.device}")
        ca, cb = A.c(), B.c()
        if workspace is None:
            nb = ctypes.c_size_t()
            _check(lib().logan_matrix_workspace_size(self._h, ctypes.byref(ca), ctypes.byref(cb), n,
                                                     ctypes.byref(nb)),
                   "logan_matrix_workspace_size")
            workspace = torch.empty(max(1, nb.value), dtype=torch.uint8,
                                    device=f"cuda:{self.device}")
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        rc = lib().logan_extend_batch_matrix(
            self._h, ctypes.byref(ca), ctypes.byref(cb), seeds.data_ptr() if n else None, n,
            M.ctypes.data, K, gap_open, gap_extend, X,
            X_per_pair.data_ptr() if X_per_pair is not None else None, workspace.data_ptr(),
            workspace.numel(), out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        _check(rc, "logan_extend_batch_matrix")
        return out[:n]

    def traceback(self, A: DevicePool, B: DevicePool, seeds, match: int = 1, mismatch: int = -1,
                  gap: int = -1, X: int = 50, X_per_pair=None, stream=None):
        """Alignment paths (logan_traceback_batch): (codes int32 [total],
        op_start int64 [n], op_count int32 [n]); code = length << 4 | op,
        op 0 = M, 1 = I, 2 = D."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        n = int(seeds.shape[0])
        dev = f"cuda:{self.device}"
        start = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
        count = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        ca, cb = A.c(), B.c()
        need = ctypes.c_uint64()

        def call(buf, cap):
            return lib().logan_traceback_batch(
                self._h, ctypes.byref(ca), ctypes.byref(cb), seeds.data_ptr() if n else None, n,
                match, mismatch, gap, X,
                X_per_pair.data_ptr() if X_per_pair is not None else None,
                buf.data_ptr() if buf is not None else None, cap, start.data_ptr(),
                count.data_ptr(), ctypes.byref(need), ctypes.c_void_p(stream.cuda_stream))
        # a pair's codes never outnumber its two sequences' bases (+1): with
        # that bound one call suffices; past 1 GiB of codes, ask for the
        # exact size first (a second sweep of the batch)
        sd = seeds.cpu().numpy().view(np.uint32).reshape(-1, 5) if n else np.zeros((0, 5), np.uint32)
        la = A.lengths.cpu().numpy().view(np.uint32)
        lb = B.lengths.cpu().numpy().view(np.uint32)
        ok = (sd[:, 0] < la.size) & (sd[:, 1] < lb.size)
        bound = int(la[sd[ok, 0]].astype(np.int64).sum() + lb[sd[ok, 1]].astype(np.int64).sum()) + n
        if bound <= (1 << 28):
            codes = torch.empty(max(bound, 1), dtype=torch.int32, device=dev)
            _check(call(codes, bound), "logan_traceback_batch")
            return codes[:max(need.value, 1)], start[:n], count[:n]
        rc = call(None, 0)
        if rc not in (OK, ENOMEM) or (rc == ENOMEM and need.value == 0):
            _check(rc, "logan_traceback_batch")
        codes = torch.empty(max(need.value, 1), dtype=torch.int32, device=dev)
        if need.value:
            _check(call(codes, need.value), "logan_traceback_batch")
        return codes, start[:n], count[:n]

    def traceback_stats(self) -> dict:
        """Device ms of the passes of the last traceback call made with
        OPT_TIMING (logan_traceback_last_stats)."""
        st = TracebackStatsT()
        _check(lib().logan_traceback_last_stats(self._h, ctypes.byref(st)),
               "logan_traceback_last_stats")
        return dict(sweep_ms=st.sweep_ms, record_ms=st.record_ms, walk_ms=st.walk_ms,
                    total_ms=st.total_ms, code_words=st.code_words,
                    record_cells=st.record_cells, launches=st.launches)

    # ---- many-to-many overlap seeding (logan_overlap_*) ----

    def overlap_candidates(self, reads: DevicePool, k: int = 17, min_freq: int = 2,
                           max_freq: int = 4, min_shared: int = 1, stream=None):
        """Candidates (int32 view of uint32 [n, 6]: a, b, o, pos_a, pos_b, count)
        of a packed read pool, in (a, b, o) order."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        n = ctypes.c_uint64()
        cr = reads.c()
        args = (self._h, ctypes.byref(cr), k, min_freq, max_freq, min_shared)
        _check(lib().logan_overlap_candidates(*args, None, 0, ctypes.byref(n),
                                              ctypes.c_void_p(stream.cuda_stream)),
               "logan_overlap_candidates")
        out = torch.empty((max(n.value, 1), 6), dtype=torch.int32, device=f"cuda:{self.device}")
        if n.value:
            _check(lib().logan_overlap_candidates(*args, out.data_ptr(), n.value, ctypes.byref(n),
                                                  ctypes.c_void_p(stream.cuda_stream)),
                   "logan_overlap_candidates")
        return out[:n.value]

    def overlap_pool(self, reads: DevicePool, stream=None) -> DevicePool:
        """Reads followed by their reverse complements (the extension's B side)."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        st = ctypes.c_void_p(stream.cuda_stream)
        cr = reads.c()
        w = ctypes.c_uint64()
        _check(lib().logan_overlap_pool_words(self._h, ctypes.byref(cr), ctypes.byref(w), st),
               "logan_overlap_pool_words")
        dev = f"cuda:{self.device}"
        words = torch.empty(w.value, dtype=torch.int32, device=dev)
        off = torch.empty(max(2 * reads.count, 1), dtype=torch.int64, device=dev)
        ln = torch.empty(max(2 * reads.count, 1), dtype=torch.int32, device=dev)
        po = SeqsT()
        _check(lib().logan_overlap_pool(self._h, ctypes.byref(cr), words.data_ptr(), w.value,
                                        off.data_ptr(), ln.data_ptr(), ctypes.byref(po), st),
               "logan_overlap_pool")
        return DevicePool(words, off[:2 * reads.count], ln[:2 * reads.count], True, po.pool_bases)

    def overlap_seeds(self, cands, reads: DevicePool, k: int = 17, stream=None):
        """Extension seeds (int32 [n, 5]) of candidates, B = overlap_pool(reads)."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        n = int(cands.shape[0])
        seeds = torch.empty((max(n, 1), 5), dtype=torch.int32, device=f"cuda:{self.device}")
        cr = reads.c()
        _check(lib().logan_overlap_seeds(self._h, cands.data_ptr() if n else None, n,
                                         ctypes.byref(cr), k, seeds.data_ptr(),
                                         ctypes.c_void_p(stream.cuda_stream)),
               "logan_overlap_seeds")
        return seeds[:n]

    def overlap_keep(self, results, seeds, A: DevicePool, B: DevicePool, ratio_num: int,
                     den: int, delta: int, stream=None):
        """Adaptive-threshold decisions (uint8 [n]) of extension results."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        n = int(seeds.shape[0])
        keep = torch.empty(max(n, 1), dtype=torch.uint8, device=f"cuda:{self.device}")
        ca, cb = A.c(), B.c()
        _check(lib().logan_overlap_keep(self._h, results.data_ptr() if n else None,
                                        seeds.data_ptr() if n else None, n, ctypes.byref(ca),
                                        ctypes.byref(cb), ratio_num, den, delta, keep.data_ptr(),
                                        ctypes.c_void_p(stream.cuda_stream)),
               "logan_overlap_keep")
        return keep[:n]

    def last_stats(self, back: int = 0) -> dict:
        """Per-level device ms / items / completed cells of a call made with
        OPT_TIMING (back = 0: the last one; index num_levels() = global-memory
        fallback)."""
        st = StatsT()
        _check(lib().logan_call_stats(self._h, back, ctypes.byref(st)), "logan_call_stats")
        n = num_levels() + 1
        return dict(level_ms=list(st.level_ms)[:n], total_ms=st.total_ms,
                    items=list(st.items)[:n], cells=list(st.cells)[:n], launches=st.launches,
                    packed_levels=st.packed_levels)


def batch_to_device(b, packed2bit: Optional[bool] = None, device="cuda"):
    """synth.Batch -> (DevicePool A, DevicePool B, seeds tensor, X_per_pair tensor or None)."""
    import torch
    from . import synth
    packed = bool(b.meta.get("packed2bit", False)) if packed2bit is None else packed2bit
    if b.packed and not packed:
        raise ValueError("this batch exists only 2-bit packed")

    def pool(p, off, ln):
        if b.packed:
            return pool_to_device(p, off, ln, True, (p.size - 1) * 16, device)
        if packed:
            return pool_to_device(synth.pack2bit(p), off, ln, True, p.size, device)
        return pool_to_device(p, off, ln, False, p.size, device)

    A = pool(b.poolA, b.offA, b.lenA)
    B = A if b.shared_pool else pool(b.poolB, b.offB, b.lenB)
    S = seeds_to_device(b.seeds, device)
    Xs = None if b.Xs is None else torch.from_numpy(np.ascontiguousarray(b.Xs, np.int32)).to(device)
    return A, B, S, Xs


class HostRequest:
    """A request's host buffers (pinned torch tensors) and its C view."""

    def __init__(self, b, packed2bit: bool = True, pin: bool = True):
        import torch
        from . import synth

        def t(a, dtype=None):
            x = torch.from_numpy(np.ascontiguousarray(a) if dtype is None
                                 else np.ascontiguousarray(a, dtype=dtype))
            return x.pin_memory() if pin else x

        if b.packed and not packed2bit:
            raise ValueError("this batch exists only 2-bit packed")

        def pool(p, off, ln):
            if b.packed:
                bases, nb = p.view(np.int32), (p.size - 1) * 16
            else:
                bases = synth.pack2bit(p).view(np.int32) if packed2bit else p
                nb = int(p.size)
            return (t(bases), t(np.ascontiguousarray(off, np.uint64).view(np.int64)),
                    t(np.ascontiguousarray(ln, np.uint32).view(np.int32)), nb)

        self.batch = b
        self.n_pairs = b.n_pairs
        self.A = pool(b.poolA, b.offA, b.lenA)
        self.B = self.A if b.shared_pool else pool(b.poolB, b.offB, b.lenB)
        arr = np.stack([b.seeds[f] for f in ("idxA", "idxB", "posA", "posB", "len")], axis=1)
        self.seeds = t(arr.astype(np.uint32).view(np.int32))
        self.Xs = None if b.Xs is None else t(b.Xs, np.int32)
        self.results = torch.zeros((max(1, b.n_pairs), 10), dtype=torch.int32)
        if pin:
            self.results = self.results.pin_memory()
        self.packed2bit = packed2bit

    def _seqs(self, P) -> SeqsT:
        bases, off, ln, nb = P
        return SeqsT(bases.data_ptr() if bases.numel() else None,
                     off.data_ptr() if ln.numel() else None,
                     ln.data_ptr() if ln.numel() else None, int(ln.numel()),
                     1 if self.packed2bit else 0, nb)

    def c(self, results=None) -> RequestT:
        """C view; `results` (host int32 [n, 10]) overrides the request's own
        result buffer so one request can be in flight several times."""
        b = self.batch
        res = self.results if results is None else results
        return RequestT(self._seqs(self.A), self._seqs(self.B), 1 if self.B is self.A else 0,
                        self.seeds.data_ptr(), self.n_pairs, b.match, b.mismatch, b.gap, b.X,
                        self.Xs.data_ptr() if self.Xs is not None else None,
                        res.data_ptr())

    def result_array(self) -> np.ndarray:
        return self.results.numpy().view(RESULT_DTYPE).reshape(-1)[:self.n_pairs]


class Server:
    """Continuous-batching server (logan_server_t) on a context's GPU."""

    def __init__(self, ctx: Context, budget_bytes: int, max_inflight: int = 4,
                 max_queued: int = 0):
        self._h = ctypes.c_void_p()
        _check(lib().logan_server_create(ctx._h, int(budget_bytes), int(max_inflight),
                                         int(max_queued), ctypes.byref(self._h)),
               "logan_server_create")
        self._live = {}

    def submit(self, req: HostRequest, results=None) -> int:
        t = ctypes.c_uint64()
        creq = req.c(results)
        rc = lib().logan_server_submit(self._h, ctypes.byref(creq), ctypes.byref(t))
        _check(rc, "logan_server_submit")
        self._live[t.value] = (req, results)  # keep host buffers alive until done
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        """(status, latency_ms); raises LoganError(ETIMEOUT) on timeout."""
        st, lat = ctypes.c_int(), ctypes.c_double()
        _check(lib().logan_server_wait(self._h, ticket, timeout_ms, ctypes.byref(st),
                                       ctypes.byref(lat)), "logan_server_wait")
        self._live.pop(ticket, None)
        return st.value, lat.value

    def poll(self, ticket: int):
        done, st, lat = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().logan_server_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(st),
                                       ctypes.byref(lat)), "logan_server_poll")
        if not done.value:
            return None
        self._live.pop(ticket, None)
        return st.value, lat.value

    def cancel(self, ticket: int):
        _check(lib().logan_server_cancel(self._h, ticket), "logan_server_cancel")

    def stats(self) -> dict:
        st = ServerStatsT()
        _check(lib().logan_server_stats(self._h, ctypes.byref(st)), "logan_server_stats")
        return {f: getattr(st, f) for f, _ in ServerStatsT._fields_}

    def close(self):
        if self._h:
            _check(lib().logan_server_destroy(self._h), "logan_server_destroy")
            self._h = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
