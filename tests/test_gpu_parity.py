"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bar (from the decoder's specification): with the same seeded inputs, hard
decisions, convergence flags, iteration counts and OSD outputs are
bit-identical to the oracle run in the same message precision; the final
LLRs agree to 1e-5 relative (they are in fact expected to be bit-identical,
since both sides perform the same IEEE binary32 operations in the same
order).  Against the FP64 oracle, decisions agree except on shots whose
LLRs pass within 1e-6 of a tie, which are counted.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2605_00038_gb300 import lbp
from paper_2605_00038_gb300.decoder import Decoder
from paper_2605_00038_gb300.inputs import sampler, workloads
from paper_2605_00038_gb300.inputs.codes import (SparseH, bb_code, rotated_surface, spacetime,
                                                 spacetime_priors)

pytestmark = pytest.mark.gpu

PREC = {lbp.LBP_MSG_F32: oracle.PREC_F32, lbp.LBP_MSG_F16: oracle.PREC_F16,
        lbp.LBP_MSG_I8: oracle.PREC_I8}
LLR_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def gpu_decode(h, pri, syn, want_llr=True, **kw):
    dec = Decoder(h, pri)
    prm = dec.params(**kw)
    out = dec.decode(torch.from_numpy(np.ascontiguousarray(syn).view(np.int64)).cuda(), prm,
                     want_llr=want_llr)
    torch.cuda.synchronize()
    r = dict(err=sampler.unpack(out.err.cpu().numpy().view(np.uint64), h.n),
             err_words=out.err.cpu().numpy().view(np.uint64),
             conv=out.converged.cpu().numpy(), osd=out.osd.cpu().numpy(),
             iters=out.iters.cpu().numpy(),
             llr=out.llr.cpu().numpy() if want_llr else None)
    dec.close()
    return r


def oracle_decode(h, pri, syn, prec=None, **kw):
    msg = kw.get("msg", 0)
    p = oracle.OracleParams(max_iter=kw.get("max_iter", 100), scale_mode=kw.get("scale_mode", 1),
                            scale_const=kw.get("scale_const", 0.625),
                            lottery=bool(kw.get("lottery", 1)), lottery_skip=kw.get("lottery_skip", 6),
                            osd=bool(kw.get("osd", 0)), prec=PREC[msg] if prec is None else prec,
                            policy=kw.get("lottery_policy", 0),
                            seed=kw.get("seed", 0), shot_offset=kw.get("shot_offset", 0))
    return oracle.decode(h, pri, sampler.unpack(syn, h.m), p, want_llr=True)


def assert_parity(g, r):
    assert np.array_equal(g["conv"], r.converged), "convergence flags differ"
    assert np.array_equal(g["iters"], r.iters), "iteration counts differ"
    bad = np.nonzero((g["err"] != r.err).any(1))[0]
    assert bad.size == 0, "error estimates differ on %d shots, first %s" % (bad.size, bad[:5])
    osd_ref = np.where(r.osd_used == 1, lbp.LBP_OSD_APPLIED,
                       np.where(r.osd_nosol == 1, lbp.LBP_OSD_NO_SOLUTION, lbp.LBP_OSD_NOT_RUN))
    assert np.array_equal(g["osd"], osd_ref), "OSD status differs"
    if g["llr"] is not None:
        ref = r.llr
        diff = np.abs(g["llr"].astype(np.float64) - ref)
        assert np.all(diff <= LLR_RTOL * np.abs(ref) + 1e-30), "LLR beyond 1e-5 relative"


# ----------------------------------------------------------------- configs

def test_c1_d3_code_capacity_fp32_vs_oracle():
    w = workloads.c1_d3_code_capacity()
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    g = gpu_decode(w.h, w.priors, syn, **w.decoder)
    assert_parity(g, oracle_decode(w.h, w.priors, syn, **w.decoder))
    # FP64 oracle: decisions identical except near-ties.
    r64 = oracle_decode(w.h, w.priors, syn, prec=oracle.PREC_F64, **w.decoder)
    diff = (g["err"] != r64.err).any(1) | (g["conv"] != r64.converged)
    near = (np.abs(r64.llr) < 1e-6 * np.abs(np.log(0.95 / 0.05))).any(1)
    assert not np.any(diff & ~near), "FP32 vs FP64 decisions differ away from ties"


@pytest.mark.parametrize("osd", [0, 1])
def test_c2_d11_spacetime_lottery_fp32(osd):
    w = workloads.c2_d11_spacetime(shots=3000, osd=osd)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    kw = dict(w.decoder, seed=11)
    g = gpu_decode(w.h, w.priors, syn, **kw)
    r = oracle_decode(w.h, w.priors, syn, **kw)
    assert_parity(g, r)
    assert (r.converged == 0).sum() > 0 or osd == 0


@pytest.mark.parametrize("p", [0.01, 0.03, 0.05])
def test_c3_bb144_lottery_osd_fp16(p):
    w = workloads.c3_bb144(p, shots=4000)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    kw = dict(w.decoder, seed=3)
    g = gpu_decode(w.h, w.priors, syn, **kw)
    r = oracle_decode(w.h, w.priors, syn, **kw)
    assert_parity(g, r)
    if p >= 0.03:
        assert (g["osd"] == lbp.LBP_OSD_APPLIED).sum() > 0


@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F32, lbp.LBP_MSG_F16, lbp.LBP_MSG_I8])
def test_precisions_on_d7_spacetime(msg):
    hz, _ = rotated_surface(7)
    st = spacetime(hz, 7)
    pri = spacetime_priors(hz, 7, 0.006, 0.006)
    _, syn = sampler.sample(st, pri, seed=77, num_shots=2500)
    kw = dict(max_iter=80, lottery=1, osd=1, msg=msg, seed=2)
    assert_parity(gpu_decode(st, pri, syn, **kw), oracle_decode(st, pri, syn, **kw))


@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F32, lbp.LBP_MSG_F16, lbp.LBP_MSG_I8])
def test_c5_d25_spacetime_precisions(msg):
    """d=25, 25 rounds (7,800 x 23,113): the graph image exceeds shared memory,
    so the kernel reads it from global memory; FP32 state is split between
    shared memory and the workspace, FP16 / INT8 state sits in shared memory."""
    w = workloads.c5_d25_spacetime(msg=msg, shots=300)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    kw = dict(w.decoder, seed=8)
    assert_parity(gpu_decode(w.h, w.priors, syn, **kw), oracle_decode(w.h, w.priors, syn, **kw))


@pytest.mark.parametrize("policy", [0, 1, 4])
def test_d25_split_state_equals_workspace_state(policy, monkeypatch):
    """FP32 messages at d=25 do not fit shared memory beside the posteriors,
    so by default the state is split: the first message slots stay in shared
    memory, the rest go to the workspace.  Forcing the whole state into the
    workspace must give the same bits, with two 512-thread groups per CTA
    (LBP_BP_SHAPE=2,512) and with four 256-thread groups (4,256); the split
    one must match the oracle."""
    w = workloads.c5_d25_spacetime(msg=lbp.LBP_MSG_F32, shots=160)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed + policy, num_shots=w.shots)
    kw = dict(w.decoder, max_iter=50, lottery_policy=policy, seed=11)
    split = gpu_decode(w.h, w.priors, syn, **kw)
    for shape in ("2,512", "4,256"):
        monkeypatch.setenv("LBP_BP_SHAPE", shape)
        other = gpu_decode(w.h, w.priors, syn, **kw)
        for k in ("err", "conv", "iters", "osd"):
            assert np.array_equal(split[k], other[k]), (shape, k)
        assert np.array_equal(split["llr"].view(np.uint32), other["llr"].view(np.uint32)), shape
    assert_parity(split, oracle_decode(w.h, w.priors, syn, **kw))


@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F32, lbp.LBP_MSG_I8])
def test_c5_d25_xz_stress_form(msg):
    """Reading R5's stress form of the d=25 workload, X and Z space-time
    matrices block-diagonal (15,600 x 46,226): message offsets exceed 16 bits,
    so the 32-bit image is read from global memory; a sample of shots matches
    the oracle."""
    w = workloads.c5_d25_spacetime_xz(msg=msg, shots=48)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    kw = dict(w.decoder, max_iter=60, seed=8)
    assert_parity(gpu_decode(w.h, w.priors, syn, **kw), oracle_decode(w.h, w.priors, syn, **kw))


@pytest.mark.parametrize("policy", [1, 2, 3, 4, 5])
def test_lottery_baseline_policies(policy):
    """The four baseline sign-flip policies of Sec. III-B and the ablation that
    draws Alg. 3 from this iteration's s_hat (policy 5), on the bounded-degree
    kernel (d=7 space-time code, BB72) and the general kernel (high degree)."""
    hz, _ = rotated_surface(7)
    st = spacetime(hz, 7)
    cases = [(st, spacetime_priors(hz, 7, 0.008, 0.008))]
    hx, _ = bb_code("bb72")
    cases.append((hx, np.full(hx.n, 0.05)))
    rng = np.random.default_rng(9)
    rows = [sorted(rng.choice(150, size=int(rng.integers(2, 13)), replace=False).tolist())
            for _ in range(60)]
    hh = SparseH.from_rows(rows, 150)
    cases.append((hh, np.full(150, 0.03)))
    for h, pri in cases:
        _, syn = sampler.sample(h, pri, seed=41, num_shots=1500)
        kw = dict(max_iter=60, lottery=1, lottery_skip=3, lottery_policy=policy, osd=1, seed=2)
        assert_parity(gpu_decode(h, pri, syn, **kw), oracle_decode(h, pri, syn, **kw))


@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F32, lbp.LBP_MSG_I8])
@pytest.mark.parametrize("rule", [lbp.LBP_RULE_MIN_SUM, lbp.LBP_RULE_SUM_PRODUCT])
def test_bank_layout_changes_nothing(msg, rule, monkeypatch):
    """The bank-aware image layout (padded message rows, regrouped check
    pairs) against the plain one on the same syndromes: identical decisions,
    flags, iteration counts, OSD outputs and LLR bits; and against the oracle
    for min-sum."""
    w = workloads.c2_d11_spacetime(shots=2500)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed + 3, num_shots=w.shots)
    kw = dict(w.decoder, msg=msg, rule=rule, seed=5)
    monkeypatch.setenv("LBP_GRAPH", "table")
    a = gpu_decode(w.h, w.priors, syn, **kw)
    monkeypatch.setenv("LBP_BANK_LAYOUT", "0")
    b = gpu_decode(w.h, w.priors, syn, **kw)
    for k in ("err", "conv", "iters", "osd"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["llr"].view(np.uint32), b["llr"].view(np.uint32))
    if rule == lbp.LBP_RULE_MIN_SUM:
        assert_parity(a, oracle_decode(w.h, w.priors, syn, **kw))


@pytest.mark.parametrize("policy", range(6))
@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F32, lbp.LBP_MSG_F16, lbp.LBP_MSG_I8])
def test_small_batch_wide_groups(policy, msg, monkeypatch):
    """A batch of at most one shot per SM runs one shot per CTA with a thread
    per column pair (1024 on the d=11 space-time code): bit-identical to the
    oracle for every lottery policy, and to the same shots decoded inside a
    large batch (shot_offset keeps their draws)."""
    w = workloads.c2_d11_spacetime(shots=2048)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed + policy, num_shots=w.shots)
    kw = dict(w.decoder, msg=msg, lottery_policy=policy, seed=policy)
    big = gpu_decode(w.h, w.priors, syn, **kw)
    lo = 1500
    small = gpu_decode(w.h, w.priors, syn[lo:lo + 100], shot_offset=lo, **kw)
    for k in ("err", "conv", "iters", "osd"):
        assert np.array_equal(big[k][lo:lo + 100], small[k]), k
    assert np.array_equal(big["llr"][lo:lo + 100].view(np.uint32), small["llr"].view(np.uint32))
    assert_parity(small, oracle_decode(w.h, w.priors, syn[lo:lo + 100], shot_offset=lo, **kw))
    monkeypatch.setenv("LBP_BP_SHAPE", "1,512")
    mid = gpu_decode(w.h, w.priors, syn[lo:lo + 100], shot_offset=lo, **kw)
    for k in ("err", "conv", "iters", "osd"):
        assert np.array_equal(mid[k], small[k]), k


@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F32, lbp.LBP_MSG_I8])
@pytest.mark.parametrize("form", ["table", "implicit", "round"])
def test_d27_table2_spacetime_32bit_image(msg, form, monkeypatch):
    """The d=27 space-time matrix in the exact form whose size Table II prints
    (unrotated code, cyclic time boundary: 18,954 x 56,889, nnz 112,320): its
    message offsets exceed 16 bits, so the image path uses the 32-bit image
    from global memory; the implicit path (Table III formulas) reads none."""
    from paper_2605_00038_gb300.inputs.codes import unrotated_surface
    monkeypatch.setenv("LBP_GRAPH", form)
    _, hz = unrotated_surface(27)
    st = spacetime(hz, 27, "cyclic")
    assert (st.n, st.nnz) == (56889, 112320)
    pri = np.full(st.n, 0.004)
    _, syn = sampler.sample(st, pri, seed=27, num_shots=40)
    kw = dict(max_iter=40, lottery=1, msg=msg, seed=5)
    assert_parity(gpu_decode(st, pri, syn, **kw), oracle_decode(st, pri, syn, **kw))


def test_osd_bit_exact_on_gpu_llrs():
    """OSD fed with the GPU's exported LLRs gives the GPU's OSD output."""
    hx, _ = bb_code("bb72")
    pri = np.full(hx.n, 0.07)
    _, syn = sampler.sample(hx, pri, seed=8, num_shots=3000)
    g = gpu_decode(hx, pri, syn, max_iter=30, lottery=0, osd=1, msg=0)
    S = sampler.unpack(syn, hx.m)
    idx = np.nonzero(g["osd"] != lbp.LBP_OSD_NOT_RUN)[0]
    assert idx.size > 20
    for b in idx[:200]:
        e, _, _ = oracle.osd0(hx, g["llr"][b].astype(np.float64), S[b])
        if e is None:
            assert g["osd"][b] == lbp.LBP_OSD_NO_SOLUTION
        else:
            assert g["osd"][b] == lbp.LBP_OSD_APPLIED
            assert np.array_equal(g["err"][b], e)


@pytest.mark.parametrize("pool", ["1", "3"])
def test_osd_pool_overflow_falls_back_to_block_kernel(pool, monkeypatch):
    """A tiny dense-row pool sends most OSD shots to the block-wide kernel;
    results stay bit-identical.  (BB144 would take the dense OSD form, which
    has no pool: LBP_OSD_DENSE=0 keeps it on the event-driven kernels.)"""
    monkeypatch.setenv("LBP_OSD_POOL_ROWS", pool)
    monkeypatch.setenv("LBP_OSD_DENSE", "0")
    for h, pri, msg in [(workloads.c3_bb144(0.05).h, np.full(144, 0.05), lbp.LBP_MSG_F16),
                        (workloads.c2_d11_spacetime().h, workloads.c2_d11_spacetime().priors,
                         lbp.LBP_MSG_F32)]:
        _, syn = sampler.sample(h, pri, seed=31, num_shots=800)
        kw = dict(max_iter=60, lottery=1, osd=1, msg=msg, seed=4)
        g = gpu_decode(h, pri, syn, **kw)
        assert_parity(g, oracle_decode(h, pri, syn, **kw))
        assert (g["osd"] != lbp.LBP_OSD_NOT_RUN).sum() > 10


@pytest.mark.parametrize("pool", [None, "2"])
def test_osd_latency_layout_small_batches(pool, monkeypatch):
    """Batches of at most one shot per SM run K_osd_warp's latency layout (one
    warp per CTA, lambda order bits and the row pool in shared memory): the
    same outputs as the oracle and as the throughput layout; with a 2-row pool
    most shots overflow to K_osd, still bit-identical.  LBP_OSD_DENSE=0 keeps
    BB144 on the event-driven kernels."""
    if pool:
        monkeypatch.setenv("LBP_OSD_POOL_ROWS", pool)
    monkeypatch.setenv("LBP_OSD_DENSE", "0")
    hz, _ = rotated_surface(13)
    st = spacetime(hz, 13)
    pri = spacetime_priors(hz, 13, 0.006, 0.006)
    cases = [(st, pri, lbp.LBP_MSG_I8), (workloads.c3_bb144(0.05).h, np.full(144, 0.05), lbp.LBP_MSG_F16)]
    for h, pri_h, msg in cases:
        _, syn = sampler.sample(h, pri_h, seed=32, num_shots=100)
        kw = dict(max_iter=100, lottery=1, osd=1, msg=msg, seed=6)
        g = gpu_decode(h, pri_h, syn, **kw)
        assert (g["osd"] != lbp.LBP_OSD_NOT_RUN).sum() >= 8
        assert_parity(g, oracle_decode(h, pri_h, syn, **kw))
        monkeypatch.setenv("LBP_OSD_LAT", "0")
        t = gpu_decode(h, pri_h, syn, **kw)
        monkeypatch.delenv("LBP_OSD_LAT")
        for k in ("err", "conv", "iters", "osd"):
            assert np.array_equal(g[k], t[k]), k


def test_general_kernel_on_high_degree_code():
    """Row weights up to 12 and column weights up to 7 exceed the bounded-degree
    layout, so this runs the general CSR kernel."""
    rng = np.random.default_rng(5)
    m, n = 60, 150
    rows = []
    for r in range(m):
        w = int(rng.integers(2, 13))
        rows.append(sorted(rng.choice(n, size=w, replace=False).tolist()))
    h = SparseH.from_rows(rows, n)
    assert h.row_weights().max() > 8 and h.col_weights().max() > 4
    pri = np.full(n, 0.03)
    _, syn = sampler.sample(h, pri, seed=12, num_shots=1500)
    for msg in (lbp.LBP_MSG_F32, lbp.LBP_MSG_I8):
        kw = dict(max_iter=50, lottery=1, lottery_skip=2, osd=1, msg=msg, seed=6)
        assert_parity(gpu_decode(h, pri, syn, **kw), oracle_decode(h, pri, syn, **kw))


@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F32, lbp.LBP_MSG_F16])
def test_autotuner_keeps_results(msg):
    """lbp_tune leaves lbp_decode's outputs and picks a shape later decodes use
    without changing any result."""
    w = workloads.c2_d11_spacetime(shots=3000, osd=1)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    kw = dict(w.decoder, msg=msg, seed=3)
    ref = gpu_decode(w.h, w.priors, syn, want_llr=False, **kw)
    dec = Decoder(w.h, w.priors)
    prm = dec.params(**kw)
    s = torch.from_numpy(syn.view(np.int64)).cuda()
    out = dec.alloc(w.shots)
    assert lbp.lbp_code_tuned(dec.code, msg) == (0, 0, 0)
    lbp.lbp_tune(dec.code, prm, w.shots, s, out.err, out.converged, out.osd, out.iters,
                 dec.workspace(prm, w.shots))
    S, G, form = lbp.lbp_code_tuned(dec.code, msg)
    assert S >= 1 and G in (32, 64, 96, 128, 192, 256, 512, 1024) and form in (1, 2, 3)
    assert lbp.lbp_code_tuned(dec.code, msg, lbp.LBP_RULE_SUM_PRODUCT) == (0, 0, 0)
    with pytest.raises(lbp.LbpError):
        lbp.lbp_code_tuned(dec.code, 3)
    assert np.array_equal(out.err.cpu().numpy().view(np.uint64), ref["err_words"])
    assert np.array_equal(out.iters.cpu().numpy(), ref["iters"])
    again = dec.decode(s, prm)
    torch.cuda.synchronize()
    assert np.array_equal(again.err.cpu().numpy().view(np.uint64), ref["err_words"])
    assert np.array_equal(again.osd.cpu().numpy(), ref["osd"])
    dec.close()


# -------------------------------------------------------------- edge cases

def test_ragged_sizes_and_tails():
    """Batch sizes that are not multiples of the groups; m, n not multiples of 64."""
    hz, _ = rotated_surface(9)                    # m = 40, n = 81
    pri = np.full(hz.n, 0.04)
    for B in (1, 2, 31, 33, 257, 1001):
        _, syn = sampler.sample(hz, pri, seed=B, num_shots=B)
        kw = dict(max_iter=40, lottery=1, lottery_skip=0, osd=1, seed=B)
        g = gpu_decode(hz, pri, syn, **kw)
        assert_parity(g, oracle_decode(hz, pri, syn, **kw))
        tail = g["err_words"][:, -1] >> np.uint64(hz.n % 64)
        assert not tail.any(), "bits past n must be zero"


def test_garbage_past_m_is_ignored():
    hz, _ = rotated_surface(5)                    # m = 12
    pri = np.full(hz.n, 0.05)
    _, syn = sampler.sample(hz, pri, seed=4, num_shots=300)
    dirty = syn.copy()
    dirty[:, -1] |= np.uint64(0xFFFF_F000_0000_0000)
    kw = dict(max_iter=30, seed=1)
    a = gpu_decode(hz, pri, syn, **kw)
    b = gpu_decode(hz, pri, dirty, **kw)
    assert np.array_equal(a["err"], b["err"]) and np.array_equal(a["iters"], b["iters"])


def test_degenerate_codes_and_zero_syndromes():
    # Empty rows, one iteration, all-zero syndromes.
    h = SparseH.from_rows([[0, 1], [], [1, 2, 3], []], 4)
    pri = np.full(4, 0.1)
    syn = np.zeros((5, 1), dtype=np.uint64)
    syn[1, 0] = 1
    syn[2, 0] = 2          # a syndrome bit on an empty row: never satisfiable
    for I in (1, 3):
        kw = dict(max_iter=I, lottery=1, lottery_skip=0, osd=1, seed=1)
        g = gpu_decode(h, pri, syn, **kw)
        assert_parity(g, oracle_decode(h, pri, syn, **kw))
    assert g["conv"][0] == 1 and g["iters"][0] == 1 and not g["err"][0].any()
    assert g["osd"][2] == lbp.LBP_OSD_NO_SOLUTION


def test_shot_offset_and_batch_independence():
    w = workloads.c3_bb144(0.05, shots=1200)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    kw = dict(w.decoder, seed=9)
    full = gpu_decode(w.h, w.priors, syn, **kw)
    part = gpu_decode(w.h, w.priors, syn[700:], shot_offset=700, **kw)
    for k in ("err", "conv", "iters", "osd"):
        assert np.array_equal(full[k][700:], part[k])


def test_host_buffer_entry_point_matches_device():
    w = workloads.c2_d11_spacetime(shots=600)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    g = gpu_decode(w.h, w.priors, syn, **w.decoder)
    dec = Decoder(w.h, w.priors)
    prm = dec.params(**w.decoder)
    B = w.shots
    pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory()
    hs = pin(syn.shape, torch.int64)
    hs.numpy()[:] = syn.view(np.int64)
    out = dict(err=pin((B, g["err_words"].shape[1]), torch.int64), converged=pin(B, torch.uint8),
               osd=pin(B, torch.uint8), iters=pin(B, torch.int32), llr=pin((B, w.h.n), torch.float32))
    dec.decode_host(hs, prm, out)
    torch.cuda.synchronize()
    assert np.array_equal(out["err"].numpy().view(np.uint64), g["err_words"])
    assert np.array_equal(out["converged"].numpy(), g["conv"])
    assert np.array_equal(out["iters"].numpy(), g["iters"])
    assert np.array_equal(out["osd"].numpy(), g["osd"])
    assert np.array_equal(out["llr"].numpy(), g["llr"])
    dec.close()


def _host_decode(dec, prm, syn, n, want_llr):
    B = syn.shape[0]
    pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory()
    hs = pin(syn.shape, torch.int64)
    hs.numpy()[:] = syn.view(np.int64)
    out = dict(err=pin((B, (n + 63) // 64), torch.int64), converged=pin(B, torch.uint8),
               osd=pin(B, torch.uint8), iters=pin(B, torch.int32))
    if want_llr:
        out["llr"] = pin((B, n), torch.float32)
    dec.decode_host(hs, prm, out)
    out["syndromes"] = hs        # the call reads it asynchronously: keep it alive until synchronised
    return out


@pytest.mark.parametrize("case", ["c2_four_chunks", "bb72_two_chunks_llr"])
def test_host_buffer_pipeline_matches_device(case):
    """Calls of at least 2 x 131,072 shots pipeline their copies over 2 or 4
    chunks on internal streams: outputs identical to the device-buffer path,
    also when two calls follow each other on the same stream."""
    if case == "c2_four_chunks":
        w = workloads.c2_d11_spacetime(shots=4 * 131072 + 777)
        h, pri, kw, llr = w.h, w.priors, dict(w.decoder, seed=12), False
    else:
        hx, _ = bb_code("bb72")
        h, pri, kw, llr = hx, np.full(hx.n, 0.03), dict(max_iter=50, lottery=1, osd=1, msg=1, seed=13), True
    B = 4 * 131072 + 777 if case == "c2_four_chunks" else 2 * 131072 + 123
    _, syn = sampler.sample(h, pri, seed=91, num_shots=B)
    g = gpu_decode(h, pri, syn, want_llr=llr, **kw)
    dec = Decoder(h, pri)
    prm = dec.params(**kw)
    first = _host_decode(dec, prm, syn, h.n, llr)
    second = _host_decode(dec, prm, syn, h.n, llr)
    torch.cuda.synchronize()
    for out in (first, second):
        assert np.array_equal(out["err"].numpy().view(np.uint64), g["err_words"])
        assert np.array_equal(out["converged"].numpy(), g["conv"])
        assert np.array_equal(out["iters"].numpy(), g["iters"])
        assert np.array_equal(out["osd"].numpy(), g["osd"])
        if llr:
            assert np.array_equal(out["llr"].numpy().view(np.uint32), g["llr"].view(np.uint32))
    dec.close()


@pytest.mark.parametrize("B", [1, 64, 3000])
def test_graph_replay_matches_decode(B):
    """lbp_graph_create captures the decode of fixed buffers; replays after
    writing new syndromes into the captured buffer give lbp_decode's outputs
    for those syndromes, at a latency-layout size (1, 64) and a large one."""
    w = workloads.c2_d11_spacetime(shots=3 * B)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed + B, num_shots=3 * B)
    dec = Decoder(w.h, w.priors)
    prm = dec.params(**dict(w.decoder, seed=7))
    allx = torch.from_numpy(syn.view(np.int64)).cuda()
    x = torch.empty((B, allx.shape[1]), dtype=torch.int64, device="cuda")
    o = dec.alloc(B, want_llr=True)
    ws = torch.empty(lbp.lbp_workspace_size(dec.code, prm, B) + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:]
    g = lbp.lbp_graph_create(dec.code, prm, B, x, o.err, o.converged, o.osd, o.iters, o.llr, ws)
    for r in range(3):
        x.copy_(allx[r * B:(r + 1) * B])
        lbp.lbp_graph_launch(g)
        ref = dec.decode(allx[r * B:(r + 1) * B].contiguous(),
                         dec.params(**dict(w.decoder, seed=7)), want_llr=True)
        torch.cuda.synchronize()
        for a, b in ((o.err, ref.err), (o.converged, ref.converged), (o.iters, ref.iters), (o.osd, ref.osd)):
            assert torch.equal(a, b)
        assert torch.equal(o.llr.view(torch.int32), ref.llr.view(torch.int32))
    g.close()
    with pytest.raises(lbp.LbpError):
        lbp.lbp_graph_create(dec.code, dec.params(max_iter=0), B, x, o.err, o.converged, o.osd, o.iters,
                             None, ws)
    dec.close()


def test_bench_launch_config_full_size_sampled():
    """c2 at its full batch (10^6 shots) in the bench's launch configuration:
    sampled shots match the oracle one by one; on every shot the converged or
    OSD estimate reproduces the syndrome (checked on the GPU)."""
    w = workloads.c2_d11_spacetime()
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    g = gpu_decode(w.h, w.priors, syn, want_llr=False, **w.decoder)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(w.shots, size=400, replace=False))
    fails = np.nonzero(g["conv"] == 0)[0][:100]
    pick = np.unique(np.concatenate([pick, fails]))
    for lo in range(0, pick.size, 100):
        sel = pick[lo:lo + 100]
        for b in sel:
            r = oracle_decode(w.h, w.priors, syn[b:b + 1], shot_offset=int(b), **w.decoder)
            assert g["conv"][b] == r.converged[0] and g["iters"][b] == r.iters[0]
            assert np.array_equal(g["err"][b], r.err[0])
    # H e_hat == s on every converged / OSD shot, via a dense GF(2) product on the GPU.
    Hd = torch.from_numpy(w.h.to_dense().astype(np.float32)).cuda()
    ok = (g["conv"] == 1) | (g["osd"] == lbp.LBP_OSD_APPLIED)
    assert ok.mean() > 0.99
    for lo in range(0, w.shots, 100_000):
        e = torch.from_numpy(g["err"][lo:lo + 100_000].astype(np.float32)).cuda()
        s = torch.from_numpy(sampler.unpack(syn[lo:lo + 100_000], w.h.m).astype(np.float32)).cuda()
        shat = torch.remainder(e @ Hd.T, 2)
        bad = (shat != s).any(1).cpu().numpy() & ok[lo:lo + 100_000]
        assert not bad.any()


@pytest.mark.parametrize("p", [0.01, 0.05])
def test_bb144_full_size_sampled(p):
    """BB [[144,12,12]] at the benchmark's 10^6 shots per p, FP16 messages, in
    its launch configuration (lbp_tune on the first 16,384 shots, then one
    decode; OSD-0 in the dense register form): sampled shots, a quarter of
    them OSD shots, match the FP16 oracle one by one (decisions, flags,
    iteration counts, OSD status), and every converged or OSD shot reproduces
    its syndrome (H e_hat = s, on the GPU)."""
    w = workloads.c3_bb144(p)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    dec = Decoder(w.h, w.priors)
    prm = dec.params(**w.decoder, seed=w.seed)
    x = torch.from_numpy(syn.view(np.int64)).cuda()
    dec.tune(x[:16384].contiguous(), prm)
    out = dec.decode(x, prm)
    torch.cuda.synchronize()
    g = dict(err=sampler.unpack(out.err.cpu().numpy().view(np.uint64), w.h.n), conv=out.converged.cpu().numpy(),
             osd=out.osd.cpu().numpy(), iters=out.iters.cpu().numpy())
    dec.close()
    rng = np.random.default_rng(1)
    osd_shots = np.nonzero(g["osd"] != lbp.LBP_OSD_NOT_RUN)[0]
    assert osd_shots.size >= 100
    pick = np.unique(np.concatenate([rng.choice(w.shots, size=300, replace=False),
                                     rng.choice(osd_shots, size=100, replace=False)]))
    for b in pick:
        r = oracle_decode(w.h, w.priors, syn[b:b + 1], shot_offset=int(b), **dict(w.decoder, seed=w.seed))
        osd_ref = (lbp.LBP_OSD_APPLIED if r.osd_used[0] else
                   (lbp.LBP_OSD_NO_SOLUTION if r.osd_nosol[0] else lbp.LBP_OSD_NOT_RUN))
        assert g["conv"][b] == r.converged[0] and g["iters"][b] == r.iters[0], b
        assert g["osd"][b] == osd_ref, b
        assert np.array_equal(g["err"][b], r.err[0]), b
    Hd = torch.from_numpy(w.h.to_dense().astype(np.float32)).cuda()
    ok = (g["conv"] == 1) | (g["osd"] == lbp.LBP_OSD_APPLIED)
    assert ok.mean() > 0.99
    for lo in range(0, w.shots, 200_000):
        e = torch.from_numpy(g["err"][lo:lo + 200_000].astype(np.float32)).cuda()
        s_ = torch.from_numpy(sampler.unpack(syn[lo:lo + 200_000], w.h.m).astype(np.float32)).cuda()
        bad = (torch.remainder(e @ Hd.T, 2) != s_).any(1).cpu().numpy() & ok[lo:lo + 200_000]
        assert not bad.any()


def test_lottery_ablation_only_where_built():
    """The ablation policy (U from this iteration's s_hat) runs in the
    shared-memory index-image form; the d=25 code, whose image is read from
    global memory, reports LBP_ENOSYS for it and decodes policy 0 as usual."""
    w = workloads.c5_d25_spacetime(msg=lbp.LBP_MSG_F32, shots=8)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    with pytest.raises(lbp.LbpError) as ei:
        gpu_decode(w.h, w.priors, syn, **dict(w.decoder, lottery_policy=lbp.LBP_LOTTERY_PROPOSED_CURRENT))
    assert ei.value.code == lbp.LBP_ENOSYS
    gpu_decode(w.h, w.priors, syn, **w.decoder)


def test_bench_headline_launch_config_sampled():
    """The d=25 workload at the benchmark's batch (2^18 shots, a quarter of
    the configuration's 2^20) in the benchmark's launch configuration
    (lbp_tune on the first 16,384 shots, then one decode): sampled shots match
    the oracle one by one (decisions, flags, iteration counts), and every
    converged shot reproduces its syndrome (H e_hat = s, on the GPU)."""
    w = workloads.c5_d25_spacetime(msg=lbp.LBP_MSG_F32, shots=1 << 18)
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    dec = Decoder(w.h, w.priors)
    prm = dec.params(**w.decoder, seed=w.seed)
    x = torch.from_numpy(syn.view(np.int64)).cuda()
    dec.tune(x[:16384].contiguous(), prm)
    out = dec.decode(x, prm)
    torch.cuda.synchronize()
    conv = out.converged.cpu().numpy()
    iters = out.iters.cpu().numpy()
    err = sampler.unpack(out.err.cpu().numpy().view(np.uint64), w.h.n)
    rng = np.random.default_rng(1)
    pick = np.sort(rng.choice(w.shots, size=40, replace=False))
    pick = np.unique(np.concatenate([pick, np.nonzero(conv == 1)[0][:16]]))
    for b in pick:
        r = oracle_decode(w.h, w.priors, syn[b:b + 1], shot_offset=int(b), **dict(w.decoder, seed=w.seed))
        assert conv[b] == r.converged[0] and iters[b] == r.iters[0], b
        assert np.array_equal(err[b], r.err[0]), b
    idx = np.nonzero(conv == 1)[0]
    assert idx.size > 100
    Hd = torch.from_numpy(w.h.to_dense().astype(np.float32)).cuda()
    for lo in range(0, idx.size, 2048):
        sel = idx[lo:lo + 2048]
        e = torch.from_numpy(err[sel].astype(np.float32)).cuda()
        s = torch.from_numpy(sampler.unpack(syn[sel], w.h.m).astype(np.float32)).cuda()
        assert torch.equal(torch.remainder(e @ Hd.T, 2), s)
    dec.close()


def test_environment_switches_read_at_load(monkeypatch):
    """The experiment switches are read once, when a code is loaded, and kept
    in the code object: a later change of the environment does not affect it."""
    h, pri = workloads.c1_d3_code_capacity().h, np.full(9, 0.05)
    for k in ("LBP_GRAPH", "LBP_BP_SHAPE", "LBP_OSD_POOL_ROWS", "LBP_OSD_LAT"):
        monkeypatch.delenv(k, raising=False)
    plain = Decoder(h, pri)
    assert lbp.lbp_code_options(plain.code) == (0, 0, 0, 0, 1)
    monkeypatch.setenv("LBP_GRAPH", "round")
    monkeypatch.setenv("LBP_BP_SHAPE", "3,256")
    monkeypatch.setenv("LBP_OSD_POOL_ROWS", "7")
    monkeypatch.setenv("LBP_OSD_LAT", "0")
    dec = Decoder(h, pri)
    assert lbp.lbp_code_options(dec.code) == (3, 3, 256, 7, 0)
    assert lbp.lbp_code_options(plain.code) == (0, 0, 0, 0, 1)
    monkeypatch.setenv("LBP_GRAPH", "implicit")
    assert lbp.lbp_code_options(dec.code)[0] == 3
    dec.close()
    plain.close()


@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F32, lbp.LBP_MSG_I8])
def test_slot_aligned_image_cyclic_boundary(msg):
    """Rotated d=25 with a cyclic time boundary (7,800 x 23,425): its image is
    slot-aligned (the t-1 measurement block of round 0 wraps to block 24 and
    still takes slot 4), and FP32 runs the split state.  A sample of shots
    matches the oracle."""
    hz, _ = rotated_surface(25)
    st = spacetime(hz, 25, "cyclic")
    pri = spacetime_priors(hz, 25, 0.004, 0.004, "cyclic")
    _, syn = sampler.sample(st, pri, seed=71, num_shots=48)
    kw = dict(max_iter=40, lottery=1, lottery_skip=2, msg=msg, seed=3)
    assert_parity(gpu_decode(st, pri, syn, **kw), oracle_decode(st, pri, syn, **kw))
