"""The dense OSD form (K_osd_dense, Alg. 2 on [H | s] held in one warp's
registers) against the oracle and against the event-driven OSD kernels.

Codes with m <= 160 and n + 1 <= 320 take the dense form.  Every case decodes
the same shots twice, with the dense form and with LBP_OSD_DENSE=0 (the
event-driven K_osd_warp / K_osd path), and against the oracle in the same
message precision: error estimates, OSD status, convergence and iteration
counts must be identical.  The shapes cover 1..5 row slots per lane and 1..5
words per row, sizes at the word boundaries (n + 1 = 64 and 65, m = 32 and
33), rank-deficient codes with syndromes outside the column space (status
NO_SOLUTION, the BP estimate kept) and an all-zero row."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_00038_gb300 import lbp
from paper_2605_00038_gb300.decoder import Decoder
from paper_2605_00038_gb300.inputs import sampler, workloads
from paper_2605_00038_gb300.inputs.codes import SparseH, bb_code, rotated_surface, spacetime, spacetime_priors

from test_gpu_parity import assert_parity, gpu_decode, oracle_decode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def gf2_rank(h: SparseH) -> int:
    a = np.zeros((h.m, h.n), dtype=np.uint8)
    for r, row in enumerate(h.rows()):
        a[r, list(row)] = 1
    rank = 0
    for c in range(h.n):
        piv = [i for i in range(rank, h.m) if a[i, c]]
        if not piv:
            continue
        a[[rank, piv[0]]] = a[[piv[0], rank]]
        for i in range(h.m):
            if i != rank and a[i, c]:
                a[i] ^= a[rank]
        rank += 1
    return rank


def random_code(m, n, w_lo, w_hi, seed, empty_row=False):
    rng = np.random.default_rng(seed)
    rows = []
    for r in range(m):
        w = int(rng.integers(w_lo, w_hi + 1))
        rows.append(sorted(rng.choice(n, size=min(w, n), replace=False).tolist()))
    if empty_row:
        rows[m // 2] = []
    return SparseH.from_rows(rows, n)


def osd_form(h, pri):
    dec = Decoder(h, pri)
    f = lbp.lbp_code_osd_form(dec.code)
    dec.close()
    return f


def check_both_forms(h, pri, syn, monkeypatch, min_osd=10, **kw):
    assert osd_form(h, pri) == (1, gf2_rank(h))
    g = gpu_decode(h, pri, syn, **kw)
    assert_parity(g, oracle_decode(h, pri, syn, **kw))
    monkeypatch.setenv("LBP_OSD_DENSE", "0")
    assert osd_form(h, pri) == (0, -1)
    e = gpu_decode(h, pri, syn, **kw)
    monkeypatch.delenv("LBP_OSD_DENSE")
    for k in ("err", "conv", "iters", "osd"):
        assert np.array_equal(g[k], e[k]), k
    assert (g["osd"] != lbp.LBP_OSD_NOT_RUN).sum() >= min_osd
    return g


@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F32, lbp.LBP_MSG_F16])
def test_bb144_dense_osd(msg, monkeypatch):
    """BB [[144,12,12]] (72 x 144: 3 row slots, 3 words), p = 0.05."""
    w = workloads.c3_bb144(0.05, shots=3000)
    _, syn = sampler.sample(w.h, w.priors, seed=41, num_shots=w.shots)
    check_both_forms(w.h, w.priors, syn, monkeypatch, min_osd=200,
                     **dict(w.decoder, msg=msg, seed=3))


def test_small_codes_dense_osd(monkeypatch):
    """BB72 (36 x 72), BB288 (144 x 288: 5 slots, 5 words), the d=3 code
    (4 x 9: 1 slot, 1 word), the d=5 space-time code (60 x 173)."""
    hx, _ = bb_code("bb72")
    h288, _ = bb_code("bb288")
    hz3, _ = rotated_surface(3)
    hz5, _ = rotated_surface(5)
    st5 = spacetime(hz5, 5)
    cases = [(hx, np.full(hx.n, 0.07)), (h288, np.full(h288.n, 0.06)), (hz3, np.full(hz3.n, 0.12)),
             (st5, spacetime_priors(hz5, 5, 0.02, 0.02))]
    for h, pri in cases:
        _, syn = sampler.sample(h, pri, seed=42, num_shots=2000)
        check_both_forms(h, pri, syn, monkeypatch, max_iter=8, lottery=1, lottery_skip=2, osd=1, seed=5)


@pytest.mark.parametrize("m,n", [(32, 63), (33, 64), (96, 191), (128, 255), (100, 127), (7, 128),
                                 (160, 319), (129, 256)])
def test_shapes_and_unsatisfiable_syndromes(m, n, monkeypatch):
    """Random codes at the slot and word boundaries; half the syndromes are
    random bits, so rank-deficient codes see syndromes outside the column
    space (NO_SOLUTION, BP estimate kept)."""
    h = random_code(m, n, 2, 7, seed=m * 1000 + n, empty_row=(m >= 32))
    pri = np.full(n, 0.06)
    _, syn = sampler.sample(h, pri, seed=43, num_shots=1200)
    rng = np.random.default_rng(n)
    wm = (m + 63) // 64
    rand = rng.integers(0, 2 ** 63, size=(600, wm), dtype=np.int64).view(np.uint64)
    if m % 64:
        rand[:, -1] &= np.uint64((1 << (m % 64)) - 1)
    syn = np.ascontiguousarray(syn)
    syn[600:] = rand
    g = check_both_forms(h, pri, syn, monkeypatch, max_iter=4, lottery=0, osd=1, seed=1)
    if gf2_rank(h) < m:
        assert (g["osd"] == lbp.LBP_OSD_NO_SOLUTION).sum() > 0


def test_dense_osd_small_batches():
    """Batches of at most one shot per SM (where the event-driven path takes
    its latency layout) also run the dense form: results equal the oracle's."""
    w = workloads.c3_bb144(0.05, shots=120)
    _, syn = sampler.sample(w.h, w.priors, seed=44, num_shots=w.shots)
    kw = dict(w.decoder, msg=lbp.LBP_MSG_F16, seed=7)
    assert_parity(gpu_decode(w.h, w.priors, syn, **kw), oracle_decode(w.h, w.priors, syn, **kw))
