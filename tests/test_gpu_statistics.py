"""Logical error rates: GPU (FP32 messages) against the FP64 oracle.

The FP32 path is bit-identical to the oracle's FP32 mode; against FP64 its
decisions differ only near ties, so the logical error rates over the same
shots must be statistically indistinguishable: paired (McNemar) test on the
per-shot failure flags, p > 0.01."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2605_00038_gb300 import evaluate, lbp
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


def _paired(w, spec, shots, **kw):
    e, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=shots)
    dec = Decoder(w.h, w.priors)
    g = dec.decode(torch.from_numpy(syn.view(np.int64)).cuda(), dec.params(**kw))
    torch.cuda.synchronize()
    true = torch.from_numpy(e.view(np.int64)).cuda()
    fg = evaluate.logical_failures(spec, true, g.err, g.converged, g.osd).cpu().numpy()
    dec.close()
    r = oracle.decode(w.h, w.priors, sampler.unpack(syn, w.h.m),
                      oracle.OracleParams(max_iter=kw["max_iter"], scale_mode=kw["scale_mode"],
                                          scale_const=kw.get("scale_const", 0.625),
                                          lottery=bool(kw["lottery"]), osd=bool(kw["osd"]),
                                          prec=oracle.PREC_F64, seed=kw.get("seed", 0)))
    fo = evaluate.logical_failures(spec, true.cpu(), torch.from_numpy(sampler.pack(r.err).view(np.int64)),
                                   torch.from_numpy(r.converged), torch.from_numpy(r.osd_used)).numpy()
    return fg, fo


def test_c1_ler_matches_fp64_oracle_over_1e6_shots():
    w = workloads.c1_d3_code_capacity()
    fg, fo = _paired(w, evaluate.surface_spec(3, 1, 9), 1_000_000, **w.decoder)
    b, c = int((fg & ~fo).sum()), int((fo & ~fg).sum())
    assert fg.sum() > 1000
    assert evaluate.mcnemar_p(b, c) > 0.01, (fg.sum(), fo.sum(), b, c)
    assert abs(fg.mean() - fo.mean()) <= 0.05 * fo.mean()


def test_bb144_ler_matches_fp64_oracle_over_1e6_shots():
    """BB [[144,12,12]] at p = 0.05 (code capacity, 10^6 shots), Lottery
    BP + OSD-0: FP32 GPU against the FP64 oracle on the same 10^6 shots."""
    w = workloads.c3_bb144(0.05, shots=1_000_000)
    kw = dict(w.decoder, msg=lbp.LBP_MSG_F32, seed=3)
    fg, fo = _paired(w, evaluate.bb_spec("bb144"), w.shots, **kw)
    b, c = int((fg & ~fo).sum()), int((fo & ~fg).sum())
    assert fg.sum() > 1000
    assert evaluate.mcnemar_p(b, c) > 0.01, (fg.sum(), fo.sum(), b, c)
    assert abs(fg.mean() - fo.mean()) <= 0.05 * fo.mean()
