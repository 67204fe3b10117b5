"""One BP launch for several codes (lbp_decode_batch).

Every request of a merged launch must give exactly the results of lbp_decode
on the same arguments: decisions, flags, iteration counts and OSD status
bit-identical (a shot's decode depends only on its syndrome, its code and
its parameters, never on the other shots of the launch)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2605_00038_gb300 import lbp
from paper_2605_00038_gb300.decoder import Decoder
from paper_2605_00038_gb300.inputs import sampler
from paper_2605_00038_gb300.inputs.codes import (bb_code, rotated_surface, spacetime, spacetime_priors,
                                                 unrotated_surface)

pytestmark = pytest.mark.gpu
PREC = {0: oracle.PREC_F32, 1: oracle.PREC_F16, 2: oracle.PREC_I8}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _surface_codes():
    out = []
    for d, p in ((5, 0.01), (7, 0.006), (9, 0.004)):
        hz, _ = rotated_surface(d)
        out.append((spacetime(hz, d), spacetime_priors(hz, d, p, p)))
    _, uz = unrotated_surface(5)
    out.append((spacetime(uz, 5), spacetime_priors(uz, 5, 0.008, 0.008)))
    return out


def _bb_codes():
    out = []
    for name, p in (("bb72", 0.05), ("bb144", 0.04), ("bb288", 0.03)):
        hx, _ = bb_code(name)
        out.append((hx, np.full(hx.n, p)))
    return out


def _run(codes, sizes, msg, seed, osd=1, lottery_policy=0):
    decs = [Decoder(h, pri) for h, pri in codes]
    entries, refs, syns, prms = [], [], [], []
    for i, ((h, pri), B) in enumerate(zip(codes, sizes)):
        _, syn = sampler.sample(h, pri, seed=seed + i, num_shots=B, shot_offset=1000 * i)
        x = torch.from_numpy(np.ascontiguousarray(syn).view(np.int64)).cuda()
        prm = decs[i].params(max_iter=80, lottery=1, osd=osd, msg=msg, seed=seed, shot_offset=1000 * i,
                             lottery_policy=lottery_policy)
        out = decs[i].alloc(B)
        entries.append((decs[i].code, prm, B, x, out.err, out.converged, out.osd, out.iters))
        refs.append(decs[i].decode(x, prm))
        syns.append(syn)
        prms.append(prm)
    items = lbp.batch_items(entries)
    need = lbp.lbp_batch_workspace_size(items)
    assert need > 0
    ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:][:need]
    lbp.lbp_decode_batch(items, ws)
    torch.cuda.synchronize()
    for e, r in zip(entries, refs):
        _, _, B, _, err, conv, osd, iters = e
        assert torch.equal(err, r.err) and torch.equal(conv, r.converged)
        assert torch.equal(osd, r.osd) and torch.equal(iters, r.iters)
    for d in decs:
        d.close()
    return entries, syns, prms


@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F32, lbp.LBP_MSG_F16, lbp.LBP_MSG_I8])
def test_surface_codes_share_one_launch(msg):
    """Rotated d=5/7/9 and unrotated d=5 space-time codes (degree bound 6, 2)
    of uneven batch sizes in one launch, OSD-0 on failures; the first item also
    matches the oracle shot by shot."""
    codes = _surface_codes()
    entries, syns, prms = _run(codes, [700, 1, 333, 1200], msg, seed=40)
    h, pri = codes[0]
    r = oracle.decode(h, pri, sampler.unpack(syns[0], h.m),
                      oracle.OracleParams(max_iter=80, lottery=True, osd=True, prec=PREC[msg], seed=40,
                                          shot_offset=0))
    err = sampler.unpack(entries[0][4].cpu().numpy().view(np.uint64), h.n)
    assert np.array_equal(err, r.err)
    assert np.array_equal(entries[0][7].cpu().numpy(), r.iters)


@pytest.mark.parametrize("policy", [0, 1, 4])
def test_bb_codes_share_one_launch(policy):
    """BB 72 / 144 / 288 (degree bound 6, 3) under three lottery policies."""
    _run(_bb_codes(), [500, 64, 257], lbp.LBP_MSG_I8, seed=50, lottery_policy=policy)


def test_batch_with_empty_item_and_without_osd():
    codes = _surface_codes()[:3]
    _run(codes, [100, 0, 50], lbp.LBP_MSG_F16, seed=60, osd=0)


def test_items_that_cannot_share_a_launch_are_refused():
    """Different degree bounds (a surface code and a BB code), or different
    message types, cannot share a launch: size 0 and LBP_ENOSYS."""
    codes = [_surface_codes()[0], _bb_codes()[0]]
    decs = [Decoder(h, pri) for h, pri in codes]
    entries = []
    for i, (h, pri) in enumerate(codes):
        B = 10
        x = torch.zeros((B, (h.m + 63) // 64), dtype=torch.int64, device="cuda")
        out = decs[i].alloc(B)
        entries.append((decs[i].code, decs[i].params(msg=2), B, x, out.err, out.converged, out.osd, out.iters))
    items = lbp.batch_items(entries)
    assert lbp.lbp_batch_workspace_size(items) == 0
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_decode_batch(items, ws)
    assert ei.value.code == lbp.LBP_ENOSYS
    e2 = [entries[0], (entries[0][0], decs[0].params(msg=1)) + entries[0][2:]]
    assert lbp.lbp_batch_workspace_size(lbp.batch_items(e2)) == 0
    for d in decs:
        d.close()
