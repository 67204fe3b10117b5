"""GPU parity of the round-periodic graph (Eq. 1 structure).

lbp_load_code recognises any space-time matrix of Eq. 1 (a round check matrix
on the diagonal, identity measurement blocks between consecutive rounds) and
K_bp can then keep one round's index table in shared memory, evaluating the
round offset and the measurement columns by arithmetic.  It performs the
same binary32 operations in the same order as the full index image, so the
bar is bit identity: against the oracle in the same message precision, and
against the index-image path on the same syndromes, LLRs included.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_00038_gb300 import lbp
from paper_2605_00038_gb300.decoder import Decoder
from paper_2605_00038_gb300.inputs import sampler, workloads
from paper_2605_00038_gb300.inputs.codes import (bb_code, rotated_surface, spacetime, spacetime_priors,
                                                 unrotated_surface)
from test_gpu_parity import assert_parity, gpu_decode, oracle_decode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def rounds_of(h, pri):
    dec = Decoder(h, pri)
    r = lbp.lbp_code_rounds(dec.code)
    dec.close()
    return r


def rot_st(d, T, boundary="open", p=0.006):
    hz, _ = rotated_surface(d)
    return spacetime(hz, T, boundary), spacetime_priors(hz, T, p, p, boundary)


def same_outputs(a, b):
    for k in ("err", "conv", "osd", "iters"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["llr"].view(np.uint32), b["llr"].view(np.uint32)), "llr"


def test_round_structure_is_recognised():
    h, pri = rot_st(5, 4)
    assert rounds_of(h, pri) == (4, 12, 25, 0)
    h, pri = rot_st(5, 3, "cyclic")
    assert rounds_of(h, pri) == (3, 12, 25, 1)
    _, hz = unrotated_surface(7)
    st = spacetime(hz, 5)
    assert rounds_of(st, np.full(st.n, 0.01)) == (5, 42, 85, 0)
    hz, _ = rotated_surface(7)
    assert rounds_of(hz, np.full(hz.n, 0.01))[0] == 0          # one round: nothing to share
    hx, _ = bb_code("bb72")
    st = spacetime(hx, 3)                                       # rows of 6 round columns: not supported
    assert rounds_of(st, np.full(st.n, 0.01))[0] == 0


@pytest.mark.parametrize("case", ["rot7_open", "rot5_cyclic", "unrotZ7_cyclic"])
@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F32, lbp.LBP_MSG_F16, lbp.LBP_MSG_I8])
def test_round_graph_matches_oracle_and_image_path(monkeypatch, case, msg):
    if case == "rot7_open":
        h, pri = rot_st(7, 7)
    elif case == "rot5_cyclic":
        h, pri = rot_st(5, 5, "cyclic", 0.01)
    else:
        _, hz = unrotated_surface(7)
        h, pri = spacetime(hz, 7, "cyclic"), spacetime_priors(hz, 7, 0.006, 0.006, "cyclic")
    _, syn = sampler.sample(h, pri, seed=61, num_shots=1500)
    kw = dict(max_iter=100, lottery=1, osd=1, msg=msg, seed=8)
    monkeypatch.setenv("LBP_GRAPH", "round")
    g = gpu_decode(h, pri, syn, **kw)
    assert_parity(g, oracle_decode(h, pri, syn, **kw))
    monkeypatch.setenv("LBP_GRAPH", "table")
    same_outputs(g, gpu_decode(h, pri, syn, **kw))


@pytest.mark.parametrize("policy", range(5))
def test_round_graph_lottery_policies_equal_image_path(monkeypatch, policy):
    w = workloads.c2_d11_spacetime(shots=3000)
    _, syn = sampler.sample(w.h, w.priors, seed=62, num_shots=w.shots)
    kw = dict(w.decoder, lottery_policy=policy, seed=policy)
    monkeypatch.setenv("LBP_GRAPH", "round")
    a = gpu_decode(w.h, w.priors, syn, **kw)
    monkeypatch.setenv("LBP_GRAPH", "table")
    same_outputs(a, gpu_decode(w.h, w.priors, syn, **kw))


def test_round_graph_sum_product_equals_image_path(monkeypatch):
    h, pri = rot_st(9, 9, p=0.004)
    _, syn = sampler.sample(h, pri, seed=63, num_shots=2000)
    kw = dict(max_iter=60, lottery=1, osd=0, msg=lbp.LBP_MSG_F16, rule=lbp.LBP_RULE_SUM_PRODUCT, seed=3)
    monkeypatch.setenv("LBP_GRAPH", "round")
    a = gpu_decode(h, pri, syn, **kw)
    monkeypatch.setenv("LBP_GRAPH", "table")
    same_outputs(a, gpu_decode(h, pri, syn, **kw))


@pytest.mark.parametrize("G", [64, 96, 128, 192, 256, 512, 1024])
def test_round_graph_every_group_width(monkeypatch, G):
    h, pri = rot_st(5, 5, p=0.01)
    _, syn = sampler.sample(h, pri, seed=64, num_shots=700)
    kw = dict(max_iter=60, lottery=1, lottery_skip=2, osd=1, seed=2)
    monkeypatch.setenv("LBP_GRAPH", "round")
    monkeypatch.setenv("LBP_BP_SHAPE", "1,%d" % G)
    assert_parity(gpu_decode(h, pri, syn, **kw), oracle_decode(h, pri, syn, **kw))


def test_round_graph_per_column_priors(monkeypatch):
    """Priors that differ per column: mu from the padded table instead of the
    two per-block values."""
    hz, _ = rotated_surface(7)
    h = spacetime(hz, 5)
    pri = np.random.default_rng(4).uniform(0.002, 0.012, size=h.n)
    assert rounds_of(h, pri)[0] == 5
    _, syn = sampler.sample(h, pri, seed=65, num_shots=1500)
    kw = dict(max_iter=80, lottery=1, osd=1, seed=5)
    monkeypatch.setenv("LBP_GRAPH", "round")
    assert_parity(gpu_decode(h, pri, syn, **kw), oracle_decode(h, pri, syn, **kw))


@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F32, lbp.LBP_MSG_F16])
def test_d25_spacetime_round_graph(monkeypatch, msg):
    """d=25, 25 rounds (7,800 x 23,113), whose full image does not fit shared
    memory beside a shot's state: on the round graph a sample of shots matches
    the oracle (FP32: state in global memory; FP16: state in shared memory)."""
    monkeypatch.setenv("LBP_GRAPH", "round")
    w = workloads.c5_d25_spacetime(msg=msg, shots=64)
    assert rounds_of(w.h, w.priors)[0] == 25
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    kw = dict(w.decoder, max_iter=40)
    assert_parity(gpu_decode(w.h, w.priors, syn, **kw), oracle_decode(w.h, w.priors, syn, **kw))
