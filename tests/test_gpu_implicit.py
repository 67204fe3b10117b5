"""GPU parity of the implicit surface-code graph (Table III).

lbp_load_code recognises the space-time matrix of the unrotated surface
code (H_X or H_Z rows of Table III per round, open or cyclic time boundary);
K_bp then evaluates every neighbour index from the formulas instead of
reading an index image.  The bar is the same as for the image path:
decisions, convergence flags, iteration counts, OSD outputs and LLRs
bit-identical to the oracle in the same message precision, and identical to
the image path on the same syndromes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_00038_gb300 import lbp
from paper_2605_00038_gb300.decoder import Decoder
from paper_2605_00038_gb300.inputs import sampler
from paper_2605_00038_gb300.inputs.codes import (SparseH, bb_code, rotated_surface, spacetime,
                                                 spacetime_priors, unrotated_surface)
from test_gpu_parity import assert_parity, gpu_decode, oracle_decode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def st_code(d, T, kind="X", boundary="open"):
    hx, hz = unrotated_surface(d)
    return spacetime(hx if kind == "X" else hz, T, boundary)


def surface_of(h, pri):
    dec = Decoder(h, pri)
    r = lbp.lbp_code_surface(dec.code)
    dec.close()
    return r


@pytest.mark.parametrize("d,T", [(3, 1), (3, 4), (5, 5), (7, 3)])
@pytest.mark.parametrize("kind", ["X", "Z"])
@pytest.mark.parametrize("boundary", ["open", "cyclic"])
def test_surface_code_is_recognised(d, T, kind, boundary):
    if boundary == "cyclic" and T == 1:
        pytest.skip("a one-round cyclic matrix has unconnected measurement columns")
    h = st_code(d, T, kind, boundary)
    got = surface_of(h, np.full(h.n, 0.01))
    assert got == (d, T, 0 if kind == "X" else 1, 1 if boundary == "cyclic" else 0)


def test_other_codes_are_not_recognised():
    hz, _ = rotated_surface(7)
    assert surface_of(spacetime(hz, 7), np.full(spacetime(hz, 7).n, 0.01))[0] == 0
    hx, _ = bb_code("bb72")
    assert surface_of(hx, np.full(hx.n, 0.01))[0] == 0
    # One entry of a recognised matrix moved: not recognised.
    h = st_code(5, 3)
    rows = [list(r) for r in h.rows()]
    rows[7] = sorted(set(rows[7][:-1] + [rows[7][-1] + 1]))
    hh = SparseH.from_rows(rows, h.n)
    assert surface_of(hh, np.full(hh.n, 0.01))[0] == 0


def graph(monkeypatch, form):
    monkeypatch.setenv("LBP_GRAPH", form)


@pytest.mark.parametrize("kind,boundary", [("X", "open"), ("Z", "open"), ("X", "cyclic"), ("Z", "cyclic")])
@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F32, lbp.LBP_MSG_F16, lbp.LBP_MSG_I8])
def test_implicit_graph_matches_oracle(monkeypatch, kind, boundary, msg):
    graph(monkeypatch, "implicit")
    d = 7
    h = st_code(d, d, kind, boundary)
    hh, _ = unrotated_surface(d)
    pri = spacetime_priors(hh, d, 0.006, 0.006, boundary)
    _, syn = sampler.sample(h, pri, seed=31, num_shots=1500)
    kw = dict(max_iter=100, lottery=1, osd=1, msg=msg, seed=9)
    assert_parity(gpu_decode(h, pri, syn, **kw), oracle_decode(h, pri, syn, **kw))


@pytest.mark.parametrize("policy", range(5))
def test_implicit_graph_equals_image_path(monkeypatch, policy):
    """Same syndromes, d=11 X-type space-time code, 11 rounds: the implicit and
    the image path give bit-identical outputs and LLRs, for every lottery
    policy, with OSD."""
    h = st_code(11, 11)
    hx, _ = unrotated_surface(11)
    pri = spacetime_priors(hx, 11, 0.004, 0.004)
    _, syn = sampler.sample(h, pri, seed=32, num_shots=4000)
    kw = dict(max_iter=100, lottery=1, lottery_policy=policy, osd=1, seed=policy)
    graph(monkeypatch, "implicit")
    a = gpu_decode(h, pri, syn, **kw)
    graph(monkeypatch, "table")
    b = gpu_decode(h, pri, syn, **kw)
    for k in ("err", "conv", "osd", "iters"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["llr"].view(np.uint32), b["llr"].view(np.uint32))


def test_implicit_graph_sum_product_equals_image_path(monkeypatch):
    h = st_code(9, 9, "Z")
    _, hz = unrotated_surface(9)
    pri = spacetime_priors(hz, 9, 0.004, 0.004)
    _, syn = sampler.sample(h, pri, seed=33, num_shots=2000)
    kw = dict(max_iter=60, lottery=1, osd=0, msg=lbp.LBP_MSG_F16, rule=lbp.LBP_RULE_SUM_PRODUCT, seed=3)
    graph(monkeypatch, "implicit")
    a = gpu_decode(h, pri, syn, **kw)
    graph(monkeypatch, "table")
    b = gpu_decode(h, pri, syn, **kw)
    assert np.array_equal(a["err"], b["err"]) and np.array_equal(a["iters"], b["iters"])
    assert np.array_equal(a["llr"].view(np.uint32), b["llr"].view(np.uint32))


def test_implicit_graph_code_capacity_and_nonuniform_priors(monkeypatch):
    """T = 1 (no measurement columns), and priors that differ per column (mu
    read from the padded table instead of the two per-block values)."""
    graph(monkeypatch, "implicit")
    h = st_code(9, 1, "X")
    pri = np.full(h.n, 0.04)
    _, syn = sampler.sample(h, pri, seed=34, num_shots=2000)
    kw = dict(max_iter=50, lottery=1, osd=1, seed=1)
    assert_parity(gpu_decode(h, pri, syn, **kw), oracle_decode(h, pri, syn, **kw))
    h = st_code(7, 5, "Z", "cyclic")
    pri = np.random.default_rng(3).uniform(0.002, 0.01, size=h.n)
    assert surface_of(h, pri)[0] == 7
    _, syn = sampler.sample(h, pri, seed=35, num_shots=1500)
    assert_parity(gpu_decode(h, pri, syn, **kw), oracle_decode(h, pri, syn, **kw))


@pytest.mark.parametrize("G", [64, 96, 128, 192, 256, 512, 1024])
def test_implicit_graph_every_group_width(monkeypatch, G):
    graph(monkeypatch, "implicit")
    monkeypatch.setenv("LBP_BP_SHAPE", "1,%d" % G)
    h = st_code(5, 5, "Z")
    _, hz = unrotated_surface(5)
    pri = spacetime_priors(hz, 5, 0.01, 0.01)
    _, syn = sampler.sample(h, pri, seed=36, num_shots=700)
    kw = dict(max_iter=60, lottery=1, lottery_skip=2, osd=1, seed=2)
    assert_parity(gpu_decode(h, pri, syn, **kw), oracle_decode(h, pri, syn, **kw))


def test_implicit_graph_tuner_keeps_results(monkeypatch):
    monkeypatch.delenv("LBP_GRAPH", raising=False)
    h = st_code(11, 11)
    hx, _ = unrotated_surface(11)
    pri = spacetime_priors(hx, 11, 0.004, 0.004)
    _, syn = sampler.sample(h, pri, seed=37, num_shots=8192)
    dec = Decoder(h, pri)
    prm = dec.params(osd=1, seed=3)
    x = torch.from_numpy(np.ascontiguousarray(syn).view(np.int64)).cuda()
    a = dec.decode(x, prm)
    ea = a.err.clone()
    dec.tune(x, prm)
    b = dec.decode(x, prm)
    torch.cuda.synchronize()
    assert torch.equal(ea, b.err)
    dec.close()
