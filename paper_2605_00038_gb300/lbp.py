"""Python binding of liblbp (include/lbp.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Device buffers
are torch CUDA tensors (packed bit words travel as int64 tensors holding the
uint64 bit patterns); host buffers are numpy arrays or pinned CPU tensors.
Every step of decoding runs in the library's CUDA kernels.  There is no CPU
fallback: if the library is not built, or a call fails, this module raises.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
LIB_PATH = _HERE / "liblbp.so"

LBP_OK, LBP_EINVAL, LBP_ENOMEM, LBP_ENOSYS, LBP_ECUDA, LBP_E2BIG = 0, -22, -12, -38, -5, -7
LBP_NOALLOC_SCRATCH_BYTES = 32 << 20
LBP_OSD_NOT_RUN, LBP_OSD_APPLIED, LBP_OSD_NO_SOLUTION = 0, 1, 2
LBP_MSG_F32, LBP_MSG_F16, LBP_MSG_I8 = 0, 1, 2
LBP_SCALE_CONST, LBP_SCALE_ADAPTIVE = 0, 1
LBP_RULE_MIN_SUM, LBP_RULE_SUM_PRODUCT = 0, 1
(LBP_LOTTERY_PROPOSED, LBP_LOTTERY_WORST_UNRELIABLE, LBP_LOTTERY_WORST_RANDOM,
 LBP_LOTTERY_RANDOM_UNRELIABLE, LBP_LOTTERY_RANDOM_RANDOM, LBP_LOTTERY_PROPOSED_CURRENT) = range(6)

EXPORTED = ["lbp_params_default", "lbp_load_code", "lbp_free_code", "lbp_code_info", "lbp_code_surface",
            "lbp_code_rounds", "lbp_code_tuned", "lbp_code_options", "lbp_code_osd_form",
            "lbp_workspace_size", "lbp_decode", "lbp_tune", "lbp_host_workspace_size", "lbp_decode_host",
            "lbp_server_create", "lbp_server_configure", "lbp_server_submit", "lbp_server_poll",
            "lbp_server_wait", "lbp_server_destroy", "lbp_graph_create", "lbp_graph_launch",
            "lbp_graph_destroy", "lbp_decode_noalloc", "lbp_timing_enable", "lbp_timing_read", "lbp_probe_smem", "lbp_probe_phi",
            "lbp_batch_workspace_size", "lbp_decode_batch", "lbp_server_set_batching",
            "lbp_strerror"]


class lbp_params(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("scale_mode", ctypes.c_int32),
                ("scale_const", ctypes.c_float), ("lottery", ctypes.c_int32),
                ("lottery_skip", ctypes.c_int32), ("osd", ctypes.c_int32),
                ("msg", ctypes.c_int32), ("lottery_policy", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("shot_offset", ctypes.c_uint64),
                ("rule", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class lbp_batch_item(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("params", lbp_params), ("num_shots", ctypes.c_int64),
                ("syndromes", ctypes.c_void_p), ("err_out", ctypes.c_void_p), ("converged", ctypes.c_void_p),
                ("osd_out", ctypes.c_void_p), ("iters_out", ctypes.c_void_p)]


class LbpError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__("%s failed: %s (%d)" % (where, lbp_strerror(code), code))
        self.code = code


_L = None


def lib():
    """Load liblbp.so (raises if it has not been built)."""
    global _L
    if _L is None:
        if not LIB_PATH.exists():
            raise RuntimeError("liblbp.so is not built (run __graft_entry__.build() or "
                               "paper_2605_00038_gb300._build.build_lbp())")
        L = ctypes.CDLL(str(LIB_PATH))
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        P = ctypes.POINTER(lbp_params)
        L.lbp_params_default.restype = None
        L.lbp_params_default.argtypes = [P]
        L.lbp_load_code.restype = ctypes.c_int
        L.lbp_load_code.argtypes = [i32, i32, vp, vp, vp, ctypes.POINTER(vp)]
        L.lbp_free_code.restype = ctypes.c_int
        L.lbp_free_code.argtypes = [vp]
        L.lbp_code_info.restype = ctypes.c_int
        L.lbp_code_info.argtypes = [vp, vp, vp, vp]
        L.lbp_code_surface.restype = ctypes.c_int
        L.lbp_code_surface.argtypes = [vp, vp, vp, vp, vp]
        L.lbp_code_tuned.restype = ctypes.c_int
        L.lbp_code_tuned.argtypes = [vp, i32, i32, vp, vp, vp]
        L.lbp_code_options.restype = ctypes.c_int
        L.lbp_code_options.argtypes = [vp, vp, vp, vp, vp, vp]
        L.lbp_code_osd_form.restype = ctypes.c_int
        L.lbp_code_osd_form.argtypes = [vp, vp, vp]
        L.lbp_probe_smem.restype = ctypes.c_int
        L.lbp_probe_smem.argtypes = [i32, vp, vp, vp]
        L.lbp_probe_phi.restype = ctypes.c_int
        L.lbp_probe_phi.argtypes = [vp, vp, i64, vp]
        L.lbp_batch_workspace_size.restype = sz
        L.lbp_batch_workspace_size.argtypes = [vp, i32]
        L.lbp_decode_batch.restype = ctypes.c_int
        L.lbp_decode_batch.argtypes = [vp, i32, vp, sz, vp]
        L.lbp_server_set_batching.restype = ctypes.c_int
        L.lbp_server_set_batching.argtypes = [vp, i32]
        L.lbp_code_rounds.restype = ctypes.c_int
        L.lbp_code_rounds.argtypes = [vp, vp, vp, vp, vp]
        L.lbp_workspace_size.restype = sz
        L.lbp_workspace_size.argtypes = [vp, P, i64]
        L.lbp_host_workspace_size.restype = sz
        L.lbp_host_workspace_size.argtypes = [vp, P, i64]
        dec = [vp, P, i64, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        L.lbp_decode.restype = ctypes.c_int
        L.lbp_decode.argtypes = dec
        L.lbp_decode_host.restype = ctypes.c_int
        L.lbp_decode_host.argtypes = dec
        L.lbp_tune.restype = ctypes.c_int
        L.lbp_tune.argtypes = [vp, P, i64, vp, vp, vp, vp, vp, vp, sz, vp]
        L.lbp_graph_create.restype = ctypes.c_int
        L.lbp_graph_create.argtypes = [vp, P, i64, vp, vp, vp, vp, vp, vp, vp, sz, ctypes.POINTER(vp)]
        L.lbp_graph_launch.restype = ctypes.c_int
        L.lbp_graph_launch.argtypes = [vp, vp]
        L.lbp_graph_destroy.restype = ctypes.c_int
        L.lbp_graph_destroy.argtypes = [vp]
        L.lbp_server_create.restype = ctypes.c_int
        L.lbp_server_create.argtypes = [sz, ctypes.c_int, ctypes.POINTER(vp)]
        L.lbp_server_configure.restype = ctypes.c_int
        L.lbp_server_configure.argtypes = [vp, i64, ctypes.c_int]
        L.lbp_server_submit.restype = ctypes.c_int
        L.lbp_server_submit.argtypes = [vp, vp, P, i64, vp, vp, vp, vp, vp, ctypes.POINTER(i64)]
        L.lbp_server_poll.restype = ctypes.c_int
        L.lbp_server_poll.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        L.lbp_server_wait.restype = ctypes.c_int
        L.lbp_server_wait.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_double)]
        L.lbp_server_destroy.restype = ctypes.c_int
        L.lbp_server_destroy.argtypes = [vp]
        L.lbp_decode_noalloc.restype = ctypes.c_int
        L.lbp_decode_noalloc.argtypes = [vp, P, i64, vp, vp, vp, vp, vp, vp, vp]
        L.lbp_timing_enable.restype = ctypes.c_int
        L.lbp_timing_enable.argtypes = [ctypes.c_int]
        L.lbp_timing_read.restype = ctypes.c_int
        L.lbp_timing_read.argtypes = [vp, vp, vp, vp]
        L.lbp_strerror.restype = ctypes.c_char_p
        L.lbp_strerror.argtypes = [ctypes.c_int]
        _L = L
    return _L


def lbp_strerror(code: int) -> str:
    return lib().lbp_strerror(code).decode()


def _check(rc: int, where: str):
    if rc != LBP_OK:
        raise LbpError(rc, where)


def lbp_params_default(**overrides) -> lbp_params:
    p = lbp_params()
    lib().lbp_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class Code:
    """Owning handle of an lbp_code (frees it on close / garbage collection)."""

    def __init__(self, ptr: int, m: int, n: int, nnz: int):
        self.ptr = ctypes.c_void_p(ptr)
        self.m, self.n, self.nnz = m, n, nnz

    def close(self):
        if self.ptr:
            lbp_free_code(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbp_load_code(m: int, n: int, row_ptr, col_idx, priors) -> Code:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    pr = np.ascontiguousarray(priors, dtype=np.float64)
    if rp.shape != (m + 1,) or pr.shape != (n,):
        raise ValueError("row_ptr must have m+1 entries and priors n entries")
    if ci.ndim != 1 or ci.size < rp[-1]:
        raise ValueError(f"col_idx holds {ci.size} entries; row_ptr[m] = {rp[-1]} are read")
    out = ctypes.c_void_p()
    _check(lib().lbp_load_code(m, n, rp.ctypes.data, ci.ctypes.data if ci.size else None,
                               pr.ctypes.data if pr.size else None, ctypes.byref(out)),
           "lbp_load_code")
    return Code(out.value, m, n, int(rp[-1]))


def lbp_free_code(code: Code):
    if code.ptr:
        rc = lib().lbp_free_code(code.ptr)
        code.ptr = ctypes.c_void_p()
        _check(rc, "lbp_free_code")


def lbp_code_info(code: Code):
    m, n, nnz = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().lbp_code_info(code.ptr, ctypes.byref(m), ctypes.byref(n), ctypes.byref(nnz)),
           "lbp_code_info")
    return m.value, n.value, nnz.value


def lbp_code_surface(code: Code):
    """(d, T, type, cyclic) of a recognised surface-code space-time matrix, d = 0 if none."""
    d, T, ty, cy = (ctypes.c_int32() for _ in range(4))
    _check(lib().lbp_code_surface(code.ptr, ctypes.byref(d), ctypes.byref(T), ctypes.byref(ty),
                                  ctypes.byref(cy)), "lbp_code_surface")
    return d.value, T.value, ty.value, cy.value


def lbp_code_rounds(code: Code):
    """(T, m_r, n_r, cyclic) of a recognised space-time matrix of Eq. 1, T = 0 if none."""
    T, mr, nr, cy = (ctypes.c_int32() for _ in range(4))
    _check(lib().lbp_code_rounds(code.ptr, ctypes.byref(T), ctypes.byref(mr), ctypes.byref(nr),
                                 ctypes.byref(cy)), "lbp_code_rounds")
    return T.value, mr.value, nr.value, cy.value


def lbp_code_tuned(code: Code, msg: int, rule: int = 0):
    """(groups per CTA, threads per group, graph form) stored by lbp_tune, zeros if untuned."""
    S, G, gf = (ctypes.c_int32() for _ in range(3))
    _check(lib().lbp_code_tuned(code.ptr, msg, rule, ctypes.byref(S), ctypes.byref(G), ctypes.byref(gf)),
           "lbp_code_tuned")
    return S.value, G.value, gf.value


def lbp_code_osd_form(code: Code):
    """(dense, rank): 1 and rank(H) when OSD runs the dense register form, else 0 and -1."""
    d, r = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().lbp_code_osd_form(code.ptr, ctypes.byref(d), ctypes.byref(r)), "lbp_code_osd_form")
    return d.value, r.value


def lbp_code_options(code: Code):
    """(graph form, groups, threads per group, OSD pool rows, OSD latency layout)
    as read from the environment when the code was loaded."""
    v = [ctypes.c_int32() for _ in range(5)]
    _check(lib().lbp_code_options(code.ptr, *[ctypes.byref(x) for x in v]), "lbp_code_options")
    return tuple(x.value for x in v)


def lbp_probe_phi(x, out, stream=None):
    """out[i] = phi(x[i]) on the device (float32 tensors, same length)."""
    _check(lib().lbp_probe_phi(_dptr(x), _dptr(out), int(x.numel()), _stream_handle(stream)), "lbp_probe_phi")


def lbp_probe_smem(trips: int = 4096, stream=None):
    """(bytes loaded, milliseconds) of the shared-memory bandwidth probe."""
    b, ms = ctypes.c_double(), ctypes.c_float()
    _check(lib().lbp_probe_smem(trips, ctypes.byref(b), ctypes.byref(ms), _stream_handle(stream)), "lbp_probe_smem")
    return b.value, ms.value


def lbp_workspace_size(code: Code, params: lbp_params, num_shots: int) -> int:
    return int(lib().lbp_workspace_size(code.ptr, ctypes.byref(params), num_shots))


def lbp_host_workspace_size(code: Code, params: lbp_params, num_shots: int) -> int:
    return int(lib().lbp_host_workspace_size(code.ptr, ctypes.byref(params), num_shots))


def _dptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device buffers must be contiguous CUDA tensors")
    return t.data_ptr()


def _hptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("host buffers must be C-contiguous")
        return a.ctypes.data
    if a.is_cuda or not a.is_contiguous():
        raise ValueError("host buffers must be contiguous CPU tensors")
    return a.data_ptr()


def _nbytes(buf) -> int:
    if isinstance(buf, np.ndarray):
        return buf.nbytes
    return buf.numel() * buf.element_size()


def _check_io(code: Code, num_shots: int, syndromes, err_out, converged, osd_out, iters_out, llr_out=None):
    """Every per-shot buffer holds at least num_shots rows of its documented
    shape, so no kernel or copy of the call runs past a buffer's end; the
    library itself sees only pointers.  None buffers are the library's to
    accept or refuse."""
    B = max(int(num_shots), 0)
    wm, wn = (code.m + 63) // 64, (code.n + 63) // 64
    for name, buf, need in (("syndromes", syndromes, 8 * wm * B), ("err_out", err_out, 8 * wn * B),
                            ("converged", converged, B), ("osd_out", osd_out, B),
                            ("iters_out", iters_out, 4 * B), ("llr_out", llr_out, 4 * code.n * B)):
        if buf is not None and _nbytes(buf) < need:
            raise ValueError(f"{name} holds {_nbytes(buf)} bytes; {num_shots} shots need {need}")


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def lbp_decode(code: Code, params: lbp_params, num_shots: int, syndromes, err_out, converged,
               osd_out, iters_out, llr_out, workspace, stream=None):
    """Enqueue a decode on `stream` (default: torch's current stream)."""
    _check_io(code, num_shots, syndromes, err_out, converged, osd_out, iters_out, llr_out)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().lbp_decode(code.ptr, ctypes.byref(params), num_shots, _dptr(syndromes),
                            _dptr(err_out), _dptr(converged), _dptr(osd_out), _dptr(iters_out),
                            _dptr(llr_out), _dptr(workspace), ws_bytes, _stream_handle(stream)),
           "lbp_decode")


def lbp_decode_host(code: Code, params: lbp_params, num_shots: int, syndromes, err_out,
                    converged, osd_out, iters_out, llr_out, workspace, stream=None):
    """Host-buffer variant: copies in, decodes and copies out on `stream`."""
    _check_io(code, num_shots, syndromes, err_out, converged, osd_out, iters_out, llr_out)
    ws_bytes = workspace.numel() * workspace.element_size()
    _check(lib().lbp_decode_host(code.ptr, ctypes.byref(params), num_shots, _hptr(syndromes),
                                 _hptr(err_out), _hptr(converged), _hptr(osd_out),
                                 _hptr(iters_out), _hptr(llr_out), _dptr(workspace), ws_bytes,
                                 _stream_handle(stream)),
           "lbp_decode_host")


def lbp_tune(code: Code, params: lbp_params, num_shots: int, syndromes, err_out, converged,
             osd_out, iters_out, workspace, stream=None):
    """Time each BP launch shape on this batch and keep the fastest in `code`."""
    _check_io(code, num_shots, syndromes, err_out, converged, osd_out, iters_out)
    ws_bytes = workspace.numel() * workspace.element_size()
    _check(lib().lbp_tune(code.ptr, ctypes.byref(params), num_shots, _dptr(syndromes),
                          _dptr(err_out), _dptr(converged), _dptr(osd_out), _dptr(iters_out),
                          _dptr(workspace), ws_bytes, _stream_handle(stream)), "lbp_tune")


def lbp_decode_noalloc(code: Code, params: lbp_params, num_shots: int, syndromes, err_out,
                       converged, osd_out, iters_out, llr_out, stream=None):
    """lbp_decode without a workspace: scratch is the library's fixed device
    array (for callers that cannot allocate device memory)."""
    _check_io(code, num_shots, syndromes, err_out, converged, osd_out, iters_out, llr_out)
    _check(lib().lbp_decode_noalloc(code.ptr, ctypes.byref(params), num_shots, _dptr(syndromes),
                                    _dptr(err_out), _dptr(converged), _dptr(osd_out),
                                    _dptr(iters_out), _dptr(llr_out), _stream_handle(stream)),
           "lbp_decode_noalloc")


def batch_items(entries):
    """ctypes array of lbp_batch_item from (code, params, num_shots, syndromes,
    err_out, converged, osd_out, iters_out) tuples of CUDA tensors."""
    arr = (lbp_batch_item * len(entries))()
    for i, (code, prm, B, syn, err, conv, osd, iters) in enumerate(entries):
        _check_io(code, B, syn, err, conv, osd, iters)
        arr[i] = lbp_batch_item(code.ptr, prm, B, _dptr(syn), _dptr(err), _dptr(conv), _dptr(osd), _dptr(iters))
    return arr


def lbp_batch_workspace_size(items) -> int:
    return int(lib().lbp_batch_workspace_size(items, len(items)))


def lbp_decode_batch(items, workspace, stream=None):
    """One BP launch over the shots of several requests (items from batch_items)."""
    _check(lib().lbp_decode_batch(items, len(items), _dptr(workspace), workspace.numel() * workspace.element_size(),
                                  _stream_handle(stream)), "lbp_decode_batch")


def lbp_timing_enable(on: bool):
    _check(lib().lbp_timing_enable(int(bool(on))), "lbp_timing_enable")


def lbp_timing_read():
    """Returns (bp_ms, bp_launches, osd_ms, osd_launches) since the last read."""
    bm, bl, om, ol = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
    _check(lib().lbp_timing_read(ctypes.byref(bm), ctypes.byref(bl), ctypes.byref(om),
                                 ctypes.byref(ol)), "lbp_timing_read")
    return bm.value, bl.value, om.value, ol.value


class Graph:
    """Owning handle of an lbp_graph (a captured decode); keeps the tensors
    it was captured with alive."""

    def __init__(self, ptr: int, keep):
        self.ptr = ctypes.c_void_p(ptr)
        self._keep = keep

    def close(self):
        if self.ptr:
            _check(lib().lbp_graph_destroy(self.ptr), "lbp_graph_destroy")
            self.ptr = ctypes.c_void_p()
            self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbp_graph_create(code: Code, params: lbp_params, num_shots: int, syndromes, err_out, converged,
                     osd_out, iters_out, llr_out, workspace) -> Graph:
    """Capture the decode lbp_decode would run for these device buffers."""
    _check_io(code, num_shots, syndromes, err_out, converged, osd_out, iters_out, llr_out)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    out = ctypes.c_void_p()
    _check(lib().lbp_graph_create(code.ptr, ctypes.byref(params), num_shots, _dptr(syndromes),
                                  _dptr(err_out), _dptr(converged), _dptr(osd_out), _dptr(iters_out),
                                  _dptr(llr_out), _dptr(workspace), ws_bytes, ctypes.byref(out)),
           "lbp_graph_create")
    return Graph(out.value, (syndromes, err_out, converged, osd_out, iters_out, llr_out, workspace))


def lbp_graph_launch(graph: Graph, stream=None):
    """Replay the captured decode on `stream` (default: torch's current stream)."""
    _check(lib().lbp_graph_launch(graph.ptr, _stream_handle(stream)), "lbp_graph_launch")


class Server:
    """Owning handle of an lbp_server."""

    def __init__(self, ptr: int):
        self.ptr = ctypes.c_void_p(ptr)

    def close(self):
        if self.ptr:
            lbp_server_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbp_server_create(arena_bytes: int, max_inflight: int) -> Server:
    out = ctypes.c_void_p()
    _check(lib().lbp_server_create(arena_bytes, max_inflight, ctypes.byref(out)), "lbp_server_create")
    return Server(out.value)


def lbp_server_configure(server: Server, chunk_work: int, priority: bool = True):
    _check(lib().lbp_server_configure(server.ptr, int(chunk_work), int(bool(priority))),
           "lbp_server_configure")


def lbp_server_set_batching(server: Server, max_items: int):
    _check(lib().lbp_server_set_batching(server.ptr, int(max_items)), "lbp_server_set_batching")


def lbp_server_submit(server: Server, code: Code, params: lbp_params, num_shots: int, syndromes,
                      err_out, converged, osd_out, iters_out) -> int:
    """Queue a decode with host buffers; returns the ticket.  The buffers must
    stay alive (and unchanged) until the request completes."""
    _check_io(code, num_shots, syndromes, err_out, converged, osd_out, iters_out)
    t = ctypes.c_int64()
    _check(lib().lbp_server_submit(server.ptr, code.ptr, ctypes.byref(params), num_shots,
                                   _hptr(syndromes), _hptr(err_out), _hptr(converged),
                                   _hptr(osd_out), _hptr(iters_out), ctypes.byref(t)),
           "lbp_server_submit")
    return t.value


def lbp_server_poll(server: Server, ticket: int):
    """Returns (done, latency_s or None); raises if the request failed."""
    done, lat = ctypes.c_int(), ctypes.c_double()
    rc = lib().lbp_server_poll(server.ptr, ticket, ctypes.byref(done), ctypes.byref(lat))
    _check(rc, "lbp_server_poll")
    return bool(done.value), (lat.value if done.value else None)


def lbp_server_wait(server: Server, ticket: int) -> float:
    lat = ctypes.c_double()
    _check(lib().lbp_server_wait(server.ptr, ticket, ctypes.byref(lat)), "lbp_server_wait")
    return lat.value


def lbp_server_destroy(server: Server):
    if server.ptr:
        rc = lib().lbp_server_destroy(server.ptr)
        server.ptr = ctypes.c_void_p()
        _check(rc, "lbp_server_destroy")
