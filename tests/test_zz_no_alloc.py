"""lbp_decode_noalloc: the decode for callers that cannot allocate device memory.

Such callers (a latency-bound request loop on a pre-sized device, where an
allocation could stall it mid-request, or a plugin whose host process owns
every allocation) pass only inputs and outputs; the library's fixed device
scratch array replaces the caller-provided workspace.
These tests call it through the C ABI and compare it with lbp_decode on the
same inputs, twice in a row, with the same tolerance as the other parity
tests (bit-identical decisions, LLRs to 1e-5 relative).  The file sorts last
so that a run stopping at the first failure has already run the others; it
also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_00038_gb300 import lbp
from paper_2605_00038_gb300.decoder import Decoder
from paper_2605_00038_gb300.inputs import sampler, workloads

pytestmark = pytest.mark.gpu
LLR_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _both(dec, syn, prm, B):
    """(lbp_decode result, lbp_decode_noalloc result) as numpy arrays."""
    s = torch.from_numpy(np.ascontiguousarray(syn).view(np.int64)).cuda()
    ref = dec.decode(s, prm, want_llr=True)
    out = dec.alloc(B, want_llr=True)
    lbp.lbp_decode_noalloc(dec.code, prm, B, s, out.err, out.converged, out.osd, out.iters,
                           out.llr, None)
    torch.cuda.synchronize()
    conv = lambda r: dict(err=r.err.cpu().numpy(), conv=r.converged.cpu().numpy(),
                          osd=r.osd.cpu().numpy(), iters=r.iters.cpu().numpy(),
                          llr=r.llr.cpu().numpy())
    return conv(ref), conv(out)


def _same(a, b):
    for k in ("err", "conv", "osd", "iters"):
        assert np.array_equal(a[k], b[k]), k
    assert np.all(np.abs(a["llr"] - b["llr"]) <= LLR_RTOL * np.abs(a["llr"]) + 1e-30)


@pytest.mark.parametrize("which", ["bb144_osd_fp16", "d11_spacetime_fp32", "d25_split_state_fp32"])
def test_noalloc_matches_workspace_decode_twice(which):
    if which == "bb144_osd_fp16":
        w = workloads.c3_bb144(0.05, shots=3000)
    elif which == "d11_spacetime_fp32":
        w = workloads.c2_d11_spacetime(shots=2000, osd=0)
    else:
        # The d=25 space-time code with FP32 messages keeps part of each
        # shot's state in the scratch array (its split state).
        w = workloads.c5_d25_spacetime(msg=0, shots=300)
        w.decoder = dict(w.decoder, max_iter=30)
    dec = Decoder(w.h, w.priors)
    for call, offset in enumerate((0, 50_000)):
        _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots, shot_offset=offset)
        prm = dec.params(**w.decoder, seed=7, shot_offset=offset)
        assert lbp.lbp_workspace_size(dec.code, prm, w.shots) <= lbp.LBP_NOALLOC_SCRATCH_BYTES
        ref, got = _both(dec, syn, prm, w.shots)
        _same(ref, got)
        if which == "bb144_osd_fp16":
            assert (got["osd"] == lbp.LBP_OSD_APPLIED).sum() > 0
    dec.close()


def test_noalloc_rejects_requests_beyond_its_area():
    w = workloads.c2_d11_spacetime(shots=200_000, osd=1)
    dec = Decoder(w.h, w.priors)
    prm = dec.params(**w.decoder)
    assert lbp.lbp_workspace_size(dec.code, prm, w.shots) > lbp.LBP_NOALLOC_SCRATCH_BYTES
    B = w.shots
    out = dec.alloc(B)
    s = torch.zeros((B, (w.h.m + 63) // 64), dtype=torch.int64, device="cuda")
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_decode_noalloc(dec.code, prm, B, s, out.err, out.converged, out.osd, out.iters,
                               None, None)
    assert ei.value.code == lbp.LBP_E2BIG
    # An empty batch is a valid decode that enqueues nothing.
    assert lbp.lib().lbp_decode_noalloc(dec.code.ptr, ctypes.byref(prm), 0, None, None, None, None, None,
                                        None, None) == lbp.LBP_OK
    dec.close()
