"""Thin ctypes binding of libfbcc (the C ABI in ``include/fbcc.h``).

Same names as the C entry points; only argument marshalling happens here. Device
buffers are PyTorch CUDA tensors (their ``data_ptr()`` is passed through) and the
stream is a ``torch.cuda.Stream`` (or the current stream). Every step of the
computation runs in the library's CUDA kernels; there is no CPU fallback: if the
library is not built, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfbcc.so")

FBCC_OK, FBCC_E_INVALID, FBCC_E_NOT_SIMPLE, FBCC_E_OOM, FBCC_E_CUDA, FBCC_E_ITER_LIMIT, FBCC_E_WORKSPACE = range(7)

# Every entry point include/fbcc.h declares (checked by the tests).
EXPORTS = (
    "fbcc_workspace_bytes", "fbcc_workspace_create", "fbcc_workspace_destroy", "fbcc_workspace_configure",
    "fbcc_solve", "fbcc_solve_host", "fbcc_solve_host_async", "fbcc_solve_noalloc", "fbcc_solve_batch", "fbcc_batch_workspace_bytes", "fbcc_validate",
    "fbcc_profile_count", "fbcc_profile_get", "fbcc_debug_read", "fbcc_status_string", "fbcc_last_cuda_error",
    "fbcc_query_biconnected", "fbcc_query_bcc_count", "fbcc_query_bccs_of", "fbcc_workspace_create_in",
    "fbcc_solve_tv", "fbcc_tv_scratch_bytes",
)


class fbcc_stats(ctypes.Structure):
    _fields_ = [("n_bcc", ctypes.c_int64), ("n_ap", ctypes.c_int64), ("n_bridge", ctypes.c_int64),
                ("n_cc", ctypes.c_int64), ("device_status", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "reserved"}


class fbcc_config(ctypes.Structure):
    _fields_ = [("ruler_stride", ctypes.c_int32), ("cc_sample", ctypes.c_int32),
                ("grid_ctas", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("chase_chains", ctypes.c_int32), ("cc_local", ctypes.c_int32), ("lcc_sample", ctypes.c_int32),
                ("rank_variant", ctypes.c_int32), ("cc_order", ctypes.c_int32), ("hub_deg", ctypes.c_int32),
                ("cc_ldd", ctypes.c_int32)]


class FbccError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        lib = _lib
        msg = lib.fbcc_status_string(status).decode() if lib else str(status)
        if status == FBCC_E_CUDA and lib:
            msg += ": " + lib.fbcc_last_cuda_error().decode()
        super().__init__(f"{where}: {msg}" if where else msg)
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libfbcc (no build step here: run ``build()`` of ``__graft_entry__``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libfbcc is not built ({path} missing); build it with "
                               "`python -m paper_2301_01356_gb300.build`")
        lib = ctypes.CDLL(path)
        P, I64, I32, INT = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        S = ctypes.POINTER(fbcc_stats)
        lib.fbcc_workspace_bytes.argtypes = [I64, I64]
        lib.fbcc_workspace_bytes.restype = ctypes.c_size_t
        lib.fbcc_workspace_create.argtypes = [I64, I64, ctypes.POINTER(P)]
        lib.fbcc_workspace_create.restype = INT
        lib.fbcc_workspace_create_in.argtypes = [P, ctypes.c_size_t, I64, I64, I32, ctypes.POINTER(P)]
        lib.fbcc_workspace_create_in.restype = INT
        lib.fbcc_workspace_destroy.argtypes = [P]
        lib.fbcc_workspace_destroy.restype = None
        lib.fbcc_workspace_configure.argtypes = [P, ctypes.POINTER(fbcc_config)]
        lib.fbcc_workspace_configure.restype = INT
        for name in ("fbcc_solve", "fbcc_solve_host", "fbcc_solve_host_async"):
            f = getattr(lib, name)
            f.argtypes = [P, INT, P, I64, I64, P, P, P, P, S, P, P]
            f.restype = INT
        lib.fbcc_solve_noalloc.argtypes = [P, INT, P, I64, I64, P, P, P, P, P, P]
        lib.fbcc_solve_noalloc.restype = INT
        lib.fbcc_solve_tv.argtypes = [P, INT, P, I64, I64, P, P, P, P, P, P, ctypes.c_size_t, P, P]
        lib.fbcc_solve_tv.restype = INT
        lib.fbcc_tv_scratch_bytes.argtypes = [I64, I64]
        lib.fbcc_tv_scratch_bytes.restype = ctypes.c_size_t
        lib.fbcc_solve_batch.argtypes = [I32, P, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.fbcc_solve_batch.restype = INT
        lib.fbcc_batch_workspace_bytes.argtypes = [I64, I64, I32]
        lib.fbcc_batch_workspace_bytes.restype = ctypes.c_size_t
        lib.fbcc_validate.argtypes = [P, INT, P, I64, I64, P, P]
        lib.fbcc_validate.restype = INT
        lib.fbcc_profile_count.argtypes = [P]
        lib.fbcc_profile_count.restype = I32
        lib.fbcc_profile_get.argtypes = [P, I32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float)]
        lib.fbcc_profile_get.restype = INT
        lib.fbcc_debug_read.argtypes = [P, ctypes.c_char_p, P, I64]
        lib.fbcc_debug_read.restype = INT
        lib.fbcc_query_biconnected.argtypes = [P, P, P, I64, P, P]
        lib.fbcc_query_biconnected.restype = INT
        lib.fbcc_query_bcc_count.argtypes = [P, P, I64, P, P]
        lib.fbcc_query_bcc_count.restype = INT
        lib.fbcc_query_bccs_of.argtypes = [P, P, I64, P, P, P]
        lib.fbcc_query_bccs_of.restype = INT
        lib.fbcc_status_string.argtypes = [INT]
        lib.fbcc_status_string.restype = ctypes.c_char_p
        lib.fbcc_last_cuda_error.argtypes = []
        lib.fbcc_last_cuda_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != FBCC_OK:
        raise FbccError(status, where)


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


# ---- the C entry points ----------------------------------------------------------

def fbcc_workspace_bytes(n: int, nnz: int) -> int:
    return int(load().fbcc_workspace_bytes(n, nnz))


def fbcc_workspace_create(n_max: int, nnz_max: int) -> int:
    h = ctypes.c_void_p()
    _check(load().fbcc_workspace_create(n_max, nnz_max, ctypes.byref(h)), "fbcc_workspace_create")
    return h.value


def fbcc_workspace_create_in(mem, n_max: int, nnz_max: int, max_graphs: int = 0) -> int:
    """A workspace inside the device tensor `mem` (uint8, from the caller's allocator)."""
    h = ctypes.c_void_p()
    _check(load().fbcc_workspace_create_in(_ptr(mem), int(mem.numel() * mem.element_size()), n_max, nnz_max,
                                           max_graphs, ctypes.byref(h)), "fbcc_workspace_create_in")
    return h.value


def fbcc_workspace_destroy(ws: int) -> None:
    load().fbcc_workspace_destroy(ws)


def fbcc_workspace_configure(ws: int, ruler_stride=0, cc_sample=0, grid_ctas=0, use_graph=0, profile=0,
                             chase_chains=0, cc_local=0, lcc_sample=0, rank_variant=0, cc_order=0,
                             hub_deg=0, cc_ldd=0) -> None:
    cfg = fbcc_config(ruler_stride, cc_sample, grid_ctas, use_graph, profile, chase_chains, cc_local, lcc_sample,
                      rank_variant, cc_order, hub_deg, cc_ldd)
    _check(load().fbcc_workspace_configure(ws, ctypes.byref(cfg)), "fbcc_workspace_configure")


def fbcc_tv_scratch_bytes(n: int, nnz: int) -> int:
    return int(load().fbcc_tv_scratch_bytes(n, nnz))


def fbcc_solve_tv(offsets, adj, n: int, m: int, edge_bcc, bcc_head, is_ap, is_bridge, scratch, ws: int,
                  stream=None, stats: fbcc_stats | None = None) -> fbcc_stats:
    """The Tarjan-Vishkin foil: fbcc_solve's outputs through the explicit skeleton,
    built in the device tensor ``scratch`` (fbcc_tv_scratch_bytes(n, 2m) bytes)."""
    import torch
    stats = stats if stats is not None else fbcc_stats()
    off64 = int(offsets.dtype == torch.int64)
    _check(load().fbcc_solve_tv(_ptr(offsets), off64, _ptr(adj), n, m, _ptr(edge_bcc), _ptr(bcc_head), _ptr(is_ap),
                                _ptr(is_bridge), ctypes.byref(stats), _ptr(scratch),
                                scratch.numel() * scratch.element_size(), ws, _stream_handle(stream)),
           "fbcc_solve_tv")
    return stats


def fbcc_solve(offsets, adj, n: int, m: int, edge_bcc, bcc_head, is_ap, is_bridge, ws: int,
               stream=None, stats: fbcc_stats | None = None, want_stats: bool = True) -> fbcc_stats | None:
    """Enqueue one solve on device tensors; ``stats`` is valid after a stream sync.
    With want_stats=False no stats copy is enqueued (nothing waits on the host)."""
    import torch
    if want_stats:
        stats = stats if stats is not None else fbcc_stats()
    off64 = int(offsets.dtype == torch.int64)
    _check(load().fbcc_solve(_ptr(offsets), off64, _ptr(adj), n, m, _ptr(edge_bcc), _ptr(bcc_head), _ptr(is_ap),
                             _ptr(is_bridge), ctypes.byref(stats) if want_stats else None, ws,
                             _stream_handle(stream)), "fbcc_solve")
    return stats if want_stats else None


def fbcc_solve_noalloc(offsets, adj, n: int, m: int, edge_bcc, bcc_head, is_ap, is_bridge, stats_dev=None,
                       stream=None) -> int:
    """Small-graph solve that allocates nothing (scratch in a static device array);
    ``stats_dev`` is a device tensor of at least 40 bytes or None. Returns the status."""
    import torch
    return int(load().fbcc_solve_noalloc(_ptr(offsets), int(offsets.dtype == torch.int64), _ptr(adj), n, m,
                                         _ptr(edge_bcc), _ptr(bcc_head), _ptr(is_ap), _ptr(is_bridge),
                                         _ptr(stats_dev), _stream_handle(stream)))


def fbcc_solve_host(offsets: np.ndarray, adj: np.ndarray, edge_bcc: np.ndarray, bcc_head: np.ndarray,
                    is_ap: np.ndarray, is_bridge: np.ndarray, ws: int, stream=None) -> fbcc_stats:
    """Solve on host (numpy, ideally pinned) buffers; synchronous."""
    stats = fbcc_stats()
    n = offsets.size - 1
    m = int(offsets[-1]) // 2
    _check(load().fbcc_solve_host(offsets.ctypes.data, int(offsets.dtype == np.int64), adj.ctypes.data, n, m,
                                  edge_bcc.ctypes.data, bcc_head.ctypes.data, is_ap.ctypes.data,
                                  is_bridge.ctypes.data, ctypes.byref(stats), ws, _stream_handle(stream)),
           "fbcc_solve_host")
    return stats


def fbcc_solve_host_async(offsets: np.ndarray, adj: np.ndarray, edge_bcc: np.ndarray, bcc_head: np.ndarray,
                          is_ap: np.ndarray, is_bridge: np.ndarray, ws: int, stream, stats=None) -> None:
    """Enqueue copies in, solve and copies out on `stream` and return at once. All
    arrays (and `stats`, an fbcc_stats in page-locked memory, or None) must be
    page-locked and left alone until the stream is synchronised."""
    n = offsets.size - 1
    m = int(offsets[-1]) // 2
    _check(load().fbcc_solve_host_async(offsets.ctypes.data, int(offsets.dtype == np.int64), adj.ctypes.data, n, m,
                                        edge_bcc.ctypes.data, bcc_head.ctypes.data, is_ap.ctypes.data,
                                        is_bridge.ctypes.data, stats, ws, _stream_handle(stream)),
           "fbcc_solve_host_async")


def fbcc_profile(ws: int) -> list:
    """[(kernel name, ms)] of the last profiled solve (waits for it)."""
    lib = load()
    out = []
    for i in range(lib.fbcc_profile_count(ws)):
        name, ms = ctypes.c_char_p(), ctypes.c_float()
        _check(lib.fbcc_profile_get(ws, i, ctypes.byref(name), ctypes.byref(ms)), "fbcc_profile_get")
        out.append((name.value.decode(), float(ms.value)))
    return out


def fbcc_debug_read(ws: int, name: str, n: int) -> np.ndarray:
    """Host copy of an internal per-vertex array of the last solve (see include/fbcc.h)."""
    out = np.empty(max(n, 1), np.uint8 if name in ("vbits", "dirb") else np.int32)
    _check(load().fbcc_debug_read(ws, name.encode(), out.ctypes.data, n), "fbcc_debug_read")
    return out[:n]


def fbcc_validate(offsets, adj, n: int, m: int, ws: int, stream=None) -> int:
    """Status of the device-side format check (FBCC_OK, FBCC_E_INVALID or FBCC_E_NOT_SIMPLE)."""
    import torch
    return int(load().fbcc_validate(_ptr(offsets), int(offsets.dtype == torch.int64), _ptr(adj), n, m, ws,
                                    _stream_handle(stream)))


def fbcc_solve_batch(vtx_base, arc_base, host_vtx_base: np.ndarray, host_arc_base: np.ndarray, local_off,
                     local_adj, edge_bcc, bcc_head, is_ap, is_bridge, stats_dev, ws: int, stream=None) -> None:
    g = host_vtx_base.size - 1
    _check(load().fbcc_solve_batch(g, _ptr(vtx_base), _ptr(arc_base), host_vtx_base.ctypes.data,
                                   host_arc_base.ctypes.data, _ptr(local_off), _ptr(local_adj), _ptr(edge_bcc),
                                   _ptr(bcc_head), _ptr(is_ap), _ptr(is_bridge), _ptr(stats_dev), ws,
                                   _stream_handle(stream)), "fbcc_solve_batch")


def fbcc_batch_workspace_bytes(n_total: int, nnz_total: int, n_graphs: int) -> int:
    return int(load().fbcc_batch_workspace_bytes(n_total, nnz_total, n_graphs))


def fbcc_query_biconnected(ws: int, u, v, bcc, stream=None) -> None:
    """bcc[i] = the BCC index u[i] and v[i] share in the last solve on ws, or -1
    (device int32 tensors of equal length)."""
    _check(load().fbcc_query_biconnected(ws, _ptr(u), _ptr(v), int(u.numel()), _ptr(bcc), _stream_handle(stream)),
           "fbcc_query_biconnected")


def fbcc_query_bcc_count(ws: int, v, out_off, stream=None) -> None:
    """out_off (device int64, len(v) + 1): exclusive prefix of the BCC counts of v."""
    _check(load().fbcc_query_bcc_count(ws, _ptr(v), int(v.numel()), _ptr(out_off), _stream_handle(stream)),
           "fbcc_query_bcc_count")


def fbcc_query_bccs_of(ws: int, v, out_off, out, stream=None) -> None:
    """The BCC indices of every v[i] at out[out_off[i]:out_off[i + 1]]."""
    _check(load().fbcc_query_bccs_of(ws, _ptr(v), int(v.numel()), _ptr(out_off), _ptr(out),
                                     _stream_handle(stream)), "fbcc_query_bccs_of")


# ---- convenience wrapper ---------------------------------------------------------

class Solver:
    """A workspace plus output tensors for graphs up to (n_max, nnz_max)."""

    def __init__(self, n_max: int, nnz_max: int, device="cuda", **config):
        import torch
        self.device = torch.device(device)
        self.n_max, self.nnz_max = n_max, nnz_max
        self.ws = fbcc_workspace_create(n_max, nnz_max)
        if config:
            fbcc_workspace_configure(self.ws, **config)
        self.edge_bcc = torch.empty(max(nnz_max, 1), dtype=torch.int32, device=self.device)
        self.bcc_head = torch.empty(max(n_max, 1), dtype=torch.int32, device=self.device)
        self.is_ap = torch.empty(max(n_max, 1), dtype=torch.uint8, device=self.device)
        self.is_bridge = torch.empty(max(nnz_max, 1), dtype=torch.uint8, device=self.device)
        self.stats = fbcc_stats()

    def configure(self, **config):
        fbcc_workspace_configure(self.ws, **config)

    def enqueue(self, offsets, adj, stream=None) -> fbcc_stats:
        n = offsets.numel() - 1
        m = (adj.numel()) // 2
        return fbcc_solve(offsets, adj, n, m, self.edge_bcc, self.bcc_head, self.is_ap, self.is_bridge, self.ws,
                          stream, self.stats)

    def solve(self, offsets, adj, stream=None) -> dict:
        """Solve and return host copies of the outputs (synchronises the stream)."""
        import torch
        n = offsets.numel() - 1
        nnz = adj.numel()
        st = self.enqueue(offsets, adj, stream)
        (stream or torch.cuda.current_stream()).synchronize()
        s = st.as_dict()
        return {
            "edge_bcc": self.edge_bcc[:nnz].cpu().numpy(),
            "bcc_head": self.bcc_head[:s["n_bcc"]].cpu().numpy(),
            "is_ap": self.is_ap[:n].cpu().numpy(),
            "is_bridge": self.is_bridge[:nnz].cpu().numpy(),
            **s,
        }

    def solve_tv(self, offsets, adj, scratch=None, stream=None) -> dict:
        """The Tarjan-Vishkin foil on this workspace (scratch: a uint8 device tensor of
        at least fbcc_tv_scratch_bytes(n, nnz) bytes, allocated here when None)."""
        import torch
        n = offsets.numel() - 1
        nnz = adj.numel()
        if scratch is None:
            scratch = torch.empty(fbcc_tv_scratch_bytes(n, nnz), dtype=torch.uint8, device=self.device)
        st = fbcc_solve_tv(offsets, adj, n, nnz // 2, self.edge_bcc, self.bcc_head, self.is_ap, self.is_bridge,
                           scratch, self.ws, stream, self.stats)
        (stream or torch.cuda.current_stream()).synchronize()
        s = st.as_dict()
        return {
            "edge_bcc": self.edge_bcc[:nnz].cpu().numpy(),
            "bcc_head": self.bcc_head[:s["n_bcc"]].cpu().numpy(),
            "is_ap": self.is_ap[:n].cpu().numpy(),
            "is_bridge": self.is_bridge[:nnz].cpu().numpy(),
            **s,
        }

    def biconnected(self, u, v, stream=None):
        """Device int32 tensor: the BCC that u[i] and v[i] share in the last solve, or -1."""
        import torch
        out = torch.empty(u.numel(), dtype=torch.int32, device=self.device)
        fbcc_query_biconnected(self.ws, u, v, out, stream)
        return out

    def bccs_of(self, v, stream=None):
        """(offsets, ids): the BCCs of v[i] are ids[offsets[i]:offsets[i + 1]] (device
        tensors; synchronises the stream once to size ids)."""
        import torch
        off = torch.empty(v.numel() + 1, dtype=torch.int64, device=self.device)
        fbcc_query_bcc_count(self.ws, v, off, stream)
        (stream or torch.cuda.current_stream()).synchronize()
        ids = torch.empty(max(int(off[-1].item()), 1), dtype=torch.int32, device=self.device)
        fbcc_query_bccs_of(self.ws, v, off, ids, stream)
        return off, ids

    def close(self):
        if self.ws:
            fbcc_workspace_destroy(self.ws)
            self.ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
