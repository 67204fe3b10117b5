"""The Decoder wrapper on a stream other than torch's current one: a batch
that grows the workspace while an earlier decode on that stream may still
read the old buffer.  Results equal the same shots decoded on the current
stream (a shot's decode depends only on its syndrome, the code, the
parameters and its global index)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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
