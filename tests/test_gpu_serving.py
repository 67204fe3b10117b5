"""Serving: continuous batching through lbp_server_*.

Requests of several codes and sizes are submitted from two host threads while
others run; every request's result must equal the same request decoded alone
with lbp_decode (bit-identical: the decode of a shot depends only on its
syndrome, the code and the parameters)."""
import ctypes
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_00038_gb300 import lbp
from paper_2605_00038_gb300.decoder import Decoder
from paper_2605_00038_gb300.inputs import sampler
from paper_2605_00038_gb300.inputs.codes import bb_code, rotated_surface, spacetime, spacetime_priors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _codes():
    out = []
    for d in (5, 7):
        hz, _ = rotated_surface(d)
        out.append((spacetime(hz, d), spacetime_priors(hz, d, 0.004, 0.004)))
    for name, p in (("bb72", 0.03), ("bb144", 0.02)):
        hx, _ = bb_code(name)
        out.append((hx, np.full(hx.n, p)))
    return out


def _requests(codes, count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        ci = int(rng.integers(len(codes)))
        h, pri = codes[ci]
        B = int(np.exp(rng.uniform(0, np.log(700))))
        off = int(rng.integers(0, 1 << 30))
        _, syn = sampler.sample(h, pri, seed=10 + ci, num_shots=B, shot_offset=off)
        reqs.append(dict(ci=ci, B=B, off=off, syn=syn, msg=int(rng.integers(0, 3))))
    return reqs


def _alone(decs, codes, r):
    dec = decs[r["ci"]]
    prm = dec.params(max_iter=60, lottery=1, osd=1, msg=r["msg"], seed=5, shot_offset=r["off"])
    out = dec.decode(torch.from_numpy(r["syn"].view(np.int64)).cuda(), prm)
    torch.cuda.synchronize()
    return (out.err.cpu().numpy().view(np.uint64), out.converged.cpu().numpy(),
            out.osd.cpu().numpy(), out.iters.cpu().numpy())


def _device_bytes(dec, r):
    h = dec.h
    prm = dec.params(max_iter=60, lottery=1, osd=1, msg=r["msg"], seed=5, shot_offset=r["off"])
    B = r["B"]
    io = B * (8 * ((h.m + 63) // 64) + 8 * ((h.n + 63) // 64) + 6) + 6 * 256
    return lbp.lbp_workspace_size(dec.code, prm, B) + io + 256


@pytest.mark.parametrize("tight,inflight,chunk,merge", [(False, 8, None, 0), (True, 4, None, 0),
                                                        (False, 8, 30000, 0), (True, 3, 0, 0),
                                                        (False, 8, None, 16), (True, 4, None, 6)])
def test_results_alone_equal_results_in_the_mix(tight, inflight, chunk, merge):
    """tight: the arena holds about 1.5 of the largest request, so admission
    waits for memory, not for a free stream.  chunk: the server's chunk_work
    (None: default; 30000 edge-shots splits most requests into many launches
    on normal- and high-priority streams; 0: one launch per request, no
    priorities).  merge: lbp_server_set_batching (requests of one message
    type and degree bound -- surface or BB codes -- share one BP launch)."""
    codes = _codes()
    decs = [Decoder(h, pri) for h, pri in codes]
    reqs = _requests(codes, 40, seed=int(tight))
    ref = [_alone(decs, codes, r) for r in reqs]
    arena = (512 << 20) if not tight else int(1.5 * max(_device_bytes(decs[r["ci"]], r) for r in reqs))
    srv = lbp.lbp_server_create(arena, inflight)
    if chunk is not None:
        lbp.lbp_server_configure(srv, chunk, chunk != 0)
    if merge:
        lbp.lbp_server_set_batching(srv, merge)
    bufs = []
    for r in reqs:
        h = codes[r["ci"]][0]
        bufs.append(dict(err=np.zeros((r["B"], (h.n + 63) // 64), np.uint64),
                         conv=np.zeros(r["B"], np.uint8), osd=np.zeros(r["B"], np.uint8),
                         iters=np.zeros(r["B"], np.int32)))
    tickets = [None] * len(reqs)

    def submit(idx):
        rng = np.random.default_rng(idx[0])
        for i in idx:
            r = reqs[i]
            prm = decs[r["ci"]].params(max_iter=60, lottery=1, osd=1, msg=r["msg"], seed=5,
                                       shot_offset=r["off"])
            b = bufs[i]
            tickets[i] = lbp.lbp_server_submit(srv, decs[r["ci"]].code, prm, r["B"], r["syn"],
                                               b["err"], b["conv"], b["osd"], b["iters"])
            if rng.random() < 0.3:
                threading.Event().wait(0.002)

    th = [threading.Thread(target=submit, args=(list(range(k, len(reqs), 2)),)) for k in (0, 1)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    lats = [lbp.lbp_server_wait(srv, t) for t in tickets]
    srv.close()
    assert all(x > 0 for x in lats)
    for i, r in enumerate(reqs):
        e, c, o, it = ref[i]
        b = bufs[i]
        assert np.array_equal(b["err"], e) and np.array_equal(b["conv"], c)
        assert np.array_equal(b["osd"], o) and np.array_equal(b["iters"], it)
    for d in decs:
        d.close()


def test_configure_rejects_bad_policy():
    srv = lbp.lbp_server_create(1 << 20, 2)
    assert lbp.lib().lbp_server_configure(srv.ptr, -1, 1) == lbp.LBP_EINVAL
    assert lbp.lib().lbp_server_configure(srv.ptr, 100, 2) == lbp.LBP_EINVAL
    assert lbp.lib().lbp_server_configure(None, 100, 1) == lbp.LBP_EINVAL
    lbp.lbp_server_configure(srv, 0, False)
    srv.close()


def test_request_larger_than_the_arena_is_refused():
    hx, _ = bb_code("bb144")
    dec = Decoder(hx, np.full(hx.n, 0.02))
    srv = lbp.lbp_server_create(1 << 16, 2)
    B = 4096
    syn = np.zeros((B, 2), np.uint64)
    with pytest.raises(lbp.LbpError) as ei:
        lbp.lbp_server_submit(srv, dec.code, dec.params(osd=1), B, syn, np.zeros((B, 3), np.uint64),
                              np.zeros(B, np.uint8), None, np.zeros(B, np.int32))
    assert ei.value.code == lbp.LBP_E2BIG
    srv.close()
    dec.close()


def _al256(x):
    return (x + 255) // 256 * 256


def _single_layout_bytes(dec, prm, B, chunk):
    """Arena bytes of a request run alone: its buffers for B shots, then the
    workspace of one launch of min(chunk, B) shots."""
    h = dec.h
    off = _al256(8 * ((h.m + 63) // 64) * B)
    off = _al256(off + 8 * ((h.n + 63) // 64) * B)
    off = _al256(off + B)
    off = _al256(off + B)
    off = _al256(off + 4 * B)
    return _al256(off + lbp.lbp_workspace_size(dec.code, prm, min(chunk, B)))


def _poll_all(srv, tickets, limit_s=120.0):
    """Poll every ticket until it completes.  A request the scheduler never
    admits fails the test instead of blocking it; the server is then left
    undestroyed, since destroying it drains the queue."""
    deadline = time.monotonic() + limit_s
    pending = set(range(len(tickets)))
    while pending:
        for i in sorted(pending):
            if lbp.lbp_server_poll(srv, tickets[i])[0]:
                pending.discard(i)
        if pending and time.monotonic() > deadline:
            srv.ptr = ctypes.c_void_p()
            pytest.fail(f"{len(pending)} of {len(tickets)} requests never completed")
        threading.Event().wait(0.001)


def test_requests_that_cannot_merge_run_alone():
    """With merged launches on, a request that lbp_decode_batch cannot plan
    (the lottery ablation policy) or whose merged layout, which holds the
    workspace of every shot at once, exceeds the arena (a long request split
    into 69-shot launches) runs as a single request; the requests behind it
    still merge.  Every result equals the same request decoded alone."""
    hx, _ = bb_code("bb144")
    pri = np.full(hx.n, 0.02)
    dec = Decoder(hx, pri)
    chunk_work = 30000
    chunk = chunk_work // hx.nnz
    big = 20000
    sizes = [big, 300, 200, 250, 180, 400, 220]
    pols = [0, 5, 0, 5, 0, 0, 5]
    reqs = []
    for i, (B, pol) in enumerate(zip(sizes, pols)):
        _, syn = sampler.sample(hx, pri, seed=60 + i, num_shots=B, shot_offset=1000 * i)
        reqs.append(dict(B=B, off=1000 * i, syn=syn,
                         prm=dec.params(max_iter=60, lottery=1, lottery_policy=pol, osd=1, seed=5,
                                        shot_offset=1000 * i)))
    ref = []
    for r in reqs:
        out = dec.decode(torch.from_numpy(r["syn"].view(np.int64)).cuda(), r["prm"])
        torch.cuda.synchronize()
        ref.append((out.err.cpu().numpy().view(np.uint64), out.converged.cpu().numpy(),
                    out.osd.cpu().numpy(), out.iters.cpu().numpy()))
    alone = _single_layout_bytes(dec, reqs[0]["prm"], big, chunk)
    arena = _al256(alone * 5 // 4)
    # The long request's merged workspace alone exceeds the arena.
    assert lbp.lbp_workspace_size(dec.code, reqs[0]["prm"], big) > arena
    srv = lbp.lbp_server_create(arena, 4)
    lbp.lbp_server_configure(srv, chunk_work, True)
    lbp.lbp_server_set_batching(srv, 8)
    bufs = [dict(err=np.zeros((r["B"], (hx.n + 63) // 64), np.uint64), conv=np.zeros(r["B"], np.uint8),
                 osd=np.zeros(r["B"], np.uint8), iters=np.zeros(r["B"], np.int32)) for r in reqs]
    tickets = [lbp.lbp_server_submit(srv, dec.code, r["prm"], r["B"], r["syn"], b["err"], b["conv"],
                                     b["osd"], b["iters"]) for r, b in zip(reqs, bufs)]
    _poll_all(srv, tickets)
    srv.close()
    for i, (e, c, o, it) in enumerate(ref):
        b = bufs[i]
        assert np.array_equal(b["err"], e) and np.array_equal(b["conv"], c), i
        assert np.array_equal(b["osd"], o) and np.array_equal(b["iters"], it), i
    dec.close()


def test_configure_after_submission_keeps_a_launch_size_that_fits():
    """Two long requests whose layout fits the arena only as 69-shot launches:
    the first holds the arena while the second waits, then
    lbp_server_configure turns chunking off.  The waiting request cannot take
    one launch for all its shots (that layout exceeds the arena), so it runs
    with the launch size checked when it was submitted.  Results equal the
    requests decoded alone."""
    hx, _ = bb_code("bb144")
    pri = np.full(hx.n, 0.02)
    dec = Decoder(hx, pri)
    chunk_work = 30000
    chunk = chunk_work // hx.nnz
    big = 20000
    reqs = []
    for i in range(2):
        _, syn = sampler.sample(hx, pri, seed=70 + i, num_shots=big, shot_offset=50_000 * i)
        reqs.append(dict(syn=syn, prm=dec.params(max_iter=60, lottery=1, osd=1, seed=5,
                                                 shot_offset=50_000 * i)))
    ref = []
    for r in reqs:
        out = dec.decode(torch.from_numpy(r["syn"].view(np.int64)).cuda(), r["prm"])
        torch.cuda.synchronize()
        ref.append((out.err.cpu().numpy().view(np.uint64), out.converged.cpu().numpy(),
                    out.osd.cpu().numpy(), out.iters.cpu().numpy()))
    arena = _al256(_single_layout_bytes(dec, reqs[0]["prm"], big, chunk) * 5 // 4)
    assert lbp.lbp_workspace_size(dec.code, reqs[0]["prm"], big) > arena
    srv = lbp.lbp_server_create(arena, 2)
    lbp.lbp_server_configure(srv, chunk_work, True)
    bufs = [dict(err=np.zeros((big, (hx.n + 63) // 64), np.uint64), conv=np.zeros(big, np.uint8),
                 osd=np.zeros(big, np.uint8), iters=np.zeros(big, np.int32)) for _ in reqs]
    tickets = [lbp.lbp_server_submit(srv, dec.code, r["prm"], big, r["syn"], b["err"], b["conv"],
                                     b["osd"], b["iters"]) for r, b in zip(reqs, bufs)]
    lbp.lbp_server_configure(srv, 0, False)
    _poll_all(srv, tickets)
    srv.close()
    for i, (e, c, o, it) in enumerate(ref):
        b = bufs[i]
        assert np.array_equal(b["err"], e) and np.array_equal(b["conv"], c), i
        assert np.array_equal(b["osd"], o) and np.array_equal(b["iters"], it), i
    dec.close()


def test_two_waiters_on_one_ticket():
    """Two host threads wait on one ticket: one gets the request's status,
    the other LBP_EINVAL, and neither blocks for good."""
    hx, _ = bb_code("bb72")
    pri = np.full(hx.n, 0.03)
    dec = Decoder(hx, pri)
    B = 2000
    _, syn = sampler.sample(hx, pri, seed=80, num_shots=B)
    srv = lbp.lbp_server_create(64 << 20, 2)
    buf = dict(err=np.zeros((B, (hx.n + 63) // 64), np.uint64), conv=np.zeros(B, np.uint8),
               osd=np.zeros(B, np.uint8), iters=np.zeros(B, np.int32))
    t = lbp.lbp_server_submit(srv, dec.code, dec.params(osd=1), B, syn, buf["err"], buf["conv"],
                              buf["osd"], buf["iters"])
    codes = []
    th = [threading.Thread(target=lambda: codes.append(lbp.lib().lbp_server_wait(srv.ptr, t, None)),
                           daemon=True) for _ in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join(timeout=120)
    if any(x.is_alive() for x in th):
        srv.ptr = ctypes.c_void_p()
        pytest.fail("a waiter never returned")
    srv.close()
    assert sorted(codes) == sorted([lbp.LBP_OK, lbp.LBP_EINVAL])
    dec.close()
