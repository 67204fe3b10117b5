"""Stream ordering around a decode.

The Decoder wrapper on a stream other than torch's current one: a batch that
grows the workspace while an earlier decode on that stream may still read the
old buffer.  The host-buffer pipeline refused after it queued its copies.
Results equal the same shots decoded on the current stream (a shot's decode
depends only on its syndrome, the code, the parameters and its global
index)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_00038_gb300 import lbp
from paper_2605_00038_gb300.decoder import Decoder
from paper_2605_00038_gb300.inputs import sampler, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_side_stream_decodes_that_grow_the_workspace():
    w = workloads.c2_d11_spacetime(shots=8192)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed + 9, num_shots=w.shots)
    x = torch.from_numpy(syn.view(np.int64)).cuda()
    a = Decoder(w.h, w.priors)
    prm = a.params(**dict(w.decoder, seed=4))
    ref = a.decode(x, prm)
    torch.cuda.synchronize()
    b = Decoder(w.h, w.priors)
    side = torch.cuda.Stream()
    outs = []
    for B in (300, 2048, 8192):            # each batch replaces the workspace
        # The outputs are allocated on the current stream: the side stream
        # waits for the work queued there before writing them.
        side.wait_stream(torch.cuda.current_stream())
        outs.append((B, b.decode(x[:B], prm, stream=side)))
        # Work on the current stream that may take a freed block.
        torch.empty(64 << 20, dtype=torch.uint8, device="cuda").fill_(0xA5)
    side.synchronize()
    torch.cuda.synchronize()
    for B, o in outs:
        for k in ("err", "converged", "osd", "iters"):
            assert torch.equal(getattr(o, k), getattr(ref, k)[:B]), (B, k)
    a.close()
    b.close()


def test_host_pipeline_refused_after_queuing_copies(monkeypatch):
    """A host-buffer call of 2 x 131,072 shots queues its input copies on an
    internal stream, then the decode of its first chunk is refused (the
    lottery ablation on the round-periodic graph form: LBP_ENOSYS).  Once the
    caller's stream has drained, the same host buffers and workspace serve a
    policy-0 decode whose results equal the device-buffer decode."""
    monkeypatch.setenv("LBP_GRAPH", "round")
    w = workloads.c2_d11_spacetime(shots=2 * 131072)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed + 21, num_shots=w.shots)
    dec = Decoder(w.h, w.priors)
    B = w.shots
    pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory()
    hs = pin(syn.shape, torch.int64)
    hs.numpy()[:] = syn.view(np.int64)
    out = dict(err=pin((B, (w.h.n + 63) // 64), torch.int64), converged=pin(B, torch.uint8),
               osd=pin(B, torch.uint8), iters=pin(B, torch.int32))
    refused = dec.params(**dict(w.decoder, lottery_policy=lbp.LBP_LOTTERY_PROPOSED_CURRENT, seed=2))
    with pytest.raises(lbp.LbpError) as ei:
        dec.decode_host(hs, refused, out)
    assert ei.value.code == lbp.LBP_ENOSYS
    torch.cuda.current_stream().synchronize()
    prm = dec.params(**dict(w.decoder, seed=2))
    dec.decode_host(hs, prm, out)
    ref = dec.decode(torch.from_numpy(syn.view(np.int64)).cuda(), prm)
    torch.cuda.synchronize()
    assert torch.equal(out["err"], ref.err.cpu()) and torch.equal(out["converged"], ref.converged.cpu())
    assert torch.equal(out["osd"], ref.osd.cpu()) and torch.equal(out["iters"], ref.iters.cpu())
    dec.close()
