"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/lbp.h declares; host-side argument checks run before any CUDA call."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

from paper_2605_00038_gb300 import _build, lbp

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def L():
    _build.build_lbp()
    return lbp.lib()


def declared_functions():
    text = (ROOT / "include" / "lbp.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbp_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert set(names) == set(lbp.EXPORTED)
    for name in names:
        assert hasattr(L, name), name
        ctypes.cast(getattr(L, name), ctypes.c_void_p)


def test_params_default_matches_paper(L):
    p = lbp.lbp_params_default()
    assert (p.max_iter, p.scale_mode, p.lottery, p.lottery_skip, p.osd, p.msg, p.rule) == (
        100, lbp.LBP_SCALE_ADAPTIVE, 1, 6, 0, lbp.LBP_MSG_F32, lbp.LBP_RULE_MIN_SUM)
    assert ctypes.sizeof(lbp.lbp_params) == 56


def test_strerror(L):
    for c in (lbp.LBP_OK, lbp.LBP_EINVAL, lbp.LBP_ENOMEM, lbp.LBP_ENOSYS, lbp.LBP_ECUDA):
        assert lbp.lbp_strerror(c)
    assert lbp.lbp_strerror(12345) == "unknown error"


@pytest.mark.parametrize("rows,n,pri", [
    ([0, 1, 3], [0, 0, 1], [0.1, 0.1]),            # weight-1 row
    ([0, 2, 4], [1, 0, 0, 1], [0.1, 0.1]),         # unsorted row
    ([0, 2, 4], [0, 1, 0, 2], [0.1, 0.1]),         # column out of range
    ([0, 2, 4], [0, 1, 0, 1], [0.1, 0.0]),         # prior 0
    ([0, 2, 4], [0, 1, 0, 1], [0.1, 1.0]),         # prior 1
    ([1, 2, 4], [0, 1, 0, 1], [0.1, 0.1]),         # row_ptr[0] != 0
])
def test_load_code_rejects_malformed_input(L, rows, n, pri):
    m = len(rows) - 1
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_load_code(m, 2, np.array(rows), np.array(n), np.array(pri))
    assert ei.value.code == lbp.LBP_EINVAL


def test_load_code_refuses_short_col_idx(L):
    # row_ptr[m] = 4 column indices are read; three are given.
    with pytest.raises(ValueError, match="col_idx"):
        lbp.lbp_load_code(2, 4, np.array([0, 2, 4]), np.array([0, 1, 2]), np.full(4, 0.1))


def test_rejects_row_heavier_than_32(L):
    n = 33
    with pytest.raises(lbp.LbpError):
        lbp.lbp_load_code(1, n, np.array([0, 33]), np.arange(33), np.full(n, 0.1))


def test_decode_rejects_bad_params_without_gpu(L):
    # Parameter validation precedes any device access.
    bad = lbp.lbp_params_default(max_iter=0)
    rc = L.lbp_decode(ctypes.c_void_p(1), ctypes.byref(bad), 1, None, None, None, None, None,
                      None, None, 0, None)
    assert rc == lbp.LBP_EINVAL
    for kw in (dict(msg=7), dict(scale_mode=5), dict(lottery=2), dict(lottery_policy=6), dict(rule=2), dict(reserved=1),
               dict(scale_mode=0, scale_const=0.0), dict(lottery_skip=-1)):
        p = lbp.lbp_params_default(**kw)
        assert L.lbp_decode(ctypes.c_void_p(1), ctypes.byref(p), 1, None, None, None, None, None,
                            None, None, 0, None) == lbp.LBP_EINVAL
    assert L.lbp_workspace_size(ctypes.c_void_p(1), ctypes.byref(bad), 10) == 0


def test_graph_server_and_tuned_reject_null_without_gpu(L):
    """The entry points added for graph replay, the serving policy and the
    tuned-shape query validate their arguments before any CUDA call."""
    p = lbp.lbp_params_default()
    out = ctypes.c_void_p()
    # lbp_graph_create: NULL code, NULL out, empty batch, NULL buffers.
    assert L.lbp_graph_create(None, ctypes.byref(p), 1, None, None, None, None, None, None, None, 0,
                              ctypes.byref(out)) == lbp.LBP_EINVAL
    assert out.value is None
    assert L.lbp_graph_create(ctypes.c_void_p(1), ctypes.byref(p), 1, None, None, None, None, None,
                              None, None, 0, None) == lbp.LBP_EINVAL
    assert L.lbp_graph_create(ctypes.c_void_p(1), ctypes.byref(p), 0, ctypes.c_void_p(8),
                              ctypes.c_void_p(8), ctypes.c_void_p(8), None, ctypes.c_void_p(8), None,
                              ctypes.c_void_p(256), 1 << 20, ctypes.byref(out)) == lbp.LBP_EINVAL
    assert L.lbp_graph_create(ctypes.c_void_p(1), ctypes.byref(p), 4, None, None, None, None, None,
                              None, None, 0, ctypes.byref(out)) == lbp.LBP_EINVAL
    assert L.lbp_graph_launch(None, None) == lbp.LBP_EINVAL
    assert L.lbp_graph_destroy(None) == lbp.LBP_EINVAL
    # lbp_server_configure / lbp_code_tuned on NULL handles.
    assert L.lbp_server_configure(None, 1 << 20, 1) == lbp.LBP_EINVAL
    g = ctypes.c_int32()
    assert L.lbp_code_tuned(None, 0, 0, None, ctypes.byref(g), None) == lbp.LBP_EINVAL


def test_batch_rejects_bad_item_counts_without_a_gpu(L):
    """lbp_decode_batch / lbp_batch_workspace_size check the item count before
    any CUDA call."""
    items = (lbp.lbp_batch_item * 1)()
    assert L.lbp_batch_workspace_size(items, 0) == 0
    assert L.lbp_batch_workspace_size(items, 65) == 0
    assert L.lbp_batch_workspace_size(None, 1) == 0
    assert L.lbp_decode_batch(items, 0, None, 0, None) == lbp.LBP_EINVAL
    assert L.lbp_decode_batch(None, 1, None, 0, None) == lbp.LBP_EINVAL
    assert L.lbp_server_set_batching(None, 4) == lbp.LBP_EINVAL


def test_empty_and_negative_batches_without_gpu(L):
    """num_shots = 0 is a valid empty decode: LBP_OK with nothing enqueued and
    no buffer read, before any CUDA call.  A negative count, or a non-empty
    batch with a missing buffer, is LBP_EINVAL, also before any CUDA call."""
    p = lbp.lbp_params_default(osd=1)
    code = ctypes.c_void_p(1)
    decode_like = (L.lbp_decode, L.lbp_decode_host)
    for fn in decode_like:
        assert fn(code, ctypes.byref(p), 0, None, None, None, None, None, None, None, 0, None) == lbp.LBP_OK
        assert fn(code, ctypes.byref(p), -1, None, None, None, None, None, None, None, 0, None) == lbp.LBP_EINVAL
        assert fn(code, ctypes.byref(p), 4, None, None, None, None, None, None, None, 0, None) == lbp.LBP_EINVAL
    assert L.lbp_tune(code, ctypes.byref(p), 0, None, None, None, None, None, None, 0, None) == lbp.LBP_OK
    assert L.lbp_tune(code, ctypes.byref(p), -1, None, None, None, None, None, None, 0, None) == lbp.LBP_EINVAL
    assert L.lbp_tune(code, ctypes.byref(p), 4, None, None, None, None, None, None, 0, None) == lbp.LBP_EINVAL


def test_buffer_sizes_are_checked_before_the_library():
    """The binding refuses a per-shot buffer shorter than num_shots rows of
    its documented shape before any library call: the library sees only
    pointers, and a short buffer would let a kernel or a copy run past it."""
    torch = pytest.importorskip("torch")
    code = lbp.Code(0, 72, 144, 432)   # m = 72: 2 syndrome words; n = 144: 3 error words
    B = 5
    ok = dict(syndromes=np.zeros((B, 2), np.uint64), err_out=np.zeros((B, 3), np.uint64),
              converged=np.zeros(B, np.uint8), osd_out=np.zeros(B, np.uint8),
              iters_out=torch.zeros(B, dtype=torch.int32), llr_out=torch.zeros((B, 144)))
    lbp._check_io(code, B, **ok)
    lbp._check_io(code, 0, None, None, None, None, None)
    for k in ok:
        short = dict(ok, **{k: ok[k][:B - 1]})
        with pytest.raises(ValueError, match=k):
            lbp._check_io(code, B, **short)
    p = lbp.lbp_params_default()
    with pytest.raises(ValueError, match="err_out"):
        lbp.lbp_server_submit(None, code, p, B, ok["syndromes"], ok["err_out"][:2], ok["converged"],
                              None, ok["iters_out"])
    with pytest.raises(ValueError, match="syndromes"):
        lbp.lbp_decode_host(code, p, B, ok["syndromes"][:1], ok["err_out"], ok["converged"], None,
                            ok["iters_out"], None, None)
