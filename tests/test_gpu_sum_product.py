"""GPU parity of the sum-product check-node rule (LBP_RULE_SUM_PRODUCT).

The oracle evaluates the tanh rule in binary64; the kernels evaluate the
equivalent phi form in binary32 with the device's expm1f and log1pf, so the
two cannot agree bit for bit.  The bar, from the arithmetic:

* LLRs after i <= 5 iterations: |lambda_gpu - lambda_ref| <= 1e-4 (1 + |lambda|).
  One phi evaluation is accurate to a few binary32 ulps (test_device_phi_accuracy
  measures it on a grid: below 1e-6 relative); an exclusive sum of at most 7
  positive terms adds at most 7 more; the outer phi multiplies the relative
  error by at most max(1, S) for its argument S (S <= 10 unless a message is
  itself below 1e-4, where the absolute error is negligible), and the check
  map is 1-Lipschitz in each input.  That bounds one iteration's relative
  error near 1e-5; a binary32 emulation of the same formulas stays below 4e-7
  through 6 iterations on surface codes.
  The ulp-level accuracy also matters where the exact posterior is 0: a
  weight-2 check returns phi(phi(|alpha|)) = |alpha|, so a column whose only
  check has weight 2 ends its first iteration at exactly mu - mu.  A phi
  accurate to 2e-6 (fast hardware exp / log) was measured to send 8% of the
  d=5 code-capacity shots to the other side of that tie from the binary64
  tanh rule, so the rule keeps log1pf / expm1f.
* Shots whose iteration count or convergence differs (a posterior within the
  tolerance of 0 at the exit test): at most 0.5% of the batch.
* Full decodes (100 iterations, lottery, OSD): identical decisions on at
  least 98% of shots (a perturbation of 1e-6 can move an oscillating shot's
  exit iteration, so full decodes are compared statistically, not bitwise).
* Binary16 / Int3.4 message storage: per-shot convergence not distinguishable
  from the binary64 reference by an exact McNemar test at the 1% level.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2605_00038_gb300 import lbp
from paper_2605_00038_gb300.decoder import Decoder
from paper_2605_00038_gb300.evaluate import mcnemar_p
from paper_2605_00038_gb300.inputs import sampler
from paper_2605_00038_gb300.inputs.codes import (SparseH, bb_code, rotated_surface, spacetime,
                                                 spacetime_priors)

pytestmark = pytest.mark.gpu

SP_TOL = 1e-4
SP = lbp.LBP_RULE_SUM_PRODUCT


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def phi64(x):
    """phi(x) = ln((e^x + 1) / (e^x - 1)) in binary64 (log1p / expm1 keep full
    relative accuracy at both ends)."""
    with np.errstate(divide="ignore"):
        return np.log1p(2.0 / np.expm1(x))


def test_device_phi_accuracy():
    """The device's phi (log1pf(2 / expm1f(x)), an IEEE division) against
    binary64 on a dense grid: relative error at most 1e-6 wherever
    phi(x) >= 1e-30 (x up to about 69), phi(0) = +inf, phi(+inf) = 0, and no
    value below 0."""
    xs = np.concatenate([[0.0], np.logspace(-30, np.log10(90.0), 200_000), [np.inf]]).astype(np.float32)
    x = torch.from_numpy(xs).cuda()
    out = torch.empty_like(x)
    lbp.lbp_probe_phi(x, out)
    torch.cuda.synchronize()
    g = out.cpu().numpy().astype(np.float64)
    r = phi64(xs.astype(np.float64))
    assert np.isinf(g[0]) and g[0] > 0 and g[-1] == 0.0
    assert np.all(g[1:-1] >= 0.0)
    m = (r >= 1e-30) & np.isfinite(r)
    rel = np.abs(g[m] - r[m]) / r[m]
    assert rel.max() <= 1e-6, (rel.max(), xs[m][np.argmax(rel)])


def gpu_decode(h, pri, syn, **kw):
    dec = Decoder(h, pri)
    out = dec.decode(torch.from_numpy(np.ascontiguousarray(syn).view(np.int64)).cuda(),
                     dec.params(rule=SP, **kw), want_llr=True)
    torch.cuda.synchronize()
    r = dict(err=sampler.unpack(out.err.cpu().numpy().view(np.uint64), h.n),
             conv=out.converged.cpu().numpy(), osd=out.osd.cpu().numpy(),
             iters=out.iters.cpu().numpy(), llr=out.llr.cpu().numpy().astype(np.float64))
    dec.close()
    return r


def oracle_sp(h, pri, syn, **kw):
    p = oracle.OracleParams(max_iter=kw.get("max_iter", 100), lottery=bool(kw.get("lottery", 1)),
                            lottery_skip=kw.get("lottery_skip", 6), osd=bool(kw.get("osd", 0)),
                            prec=oracle.PREC_F64, rule=oracle.oracle.RULE_SUM_PRODUCT,
                            policy=kw.get("lottery_policy", 0), seed=kw.get("seed", 0))
    return oracle.decode(h, pri, sampler.unpack(syn, h.m), p, want_llr=True)


def high_degree_code():
    rng = np.random.default_rng(5)
    n = 150
    rows = [sorted(rng.choice(n, size=int(rng.integers(2, 13)), replace=False).tolist())
            for _ in range(60)]
    return SparseH.from_rows(rows, n), np.full(n, 0.03)


def cases():
    hz5, _ = rotated_surface(5)
    hz7, _ = rotated_surface(7)
    st7 = spacetime(hz7, 7)
    hx, _ = bb_code("bb72")
    hh, phh = high_degree_code()
    return {
        "d5_code_capacity": (hz5, np.full(hz5.n, 0.05)),
        "d7_spacetime": (st7, spacetime_priors(hz7, 7, 0.006, 0.006)),
        "bb72": (hx, np.full(hx.n, 0.03)),
        "high_degree_general_kernel": (hh, phh),
    }


def check_llrs(g, r, max_mismatch=0.005):
    same = (g["iters"] == r.iters) & (g["conv"] == r.converged)
    assert (~same).mean() <= max_mismatch, "%d shots exit differently" % (~same).sum()
    ref = r.llr[same]
    diff = np.abs(g["llr"][same] - ref)
    worst = (diff / (1.0 + np.abs(ref))).max() if ref.size else 0.0
    assert worst <= SP_TOL, "LLR deviation %.3g beyond %.0e" % (worst, SP_TOL)
    # Hard decisions agree wherever the posterior is not within the tolerance of 0.
    tie = np.abs(ref) <= SP_TOL * (1.0 + np.abs(ref))
    assert not np.any((g["err"][same] != r.err[same]) & ~tie)
    return worst


@pytest.mark.parametrize("name", ["d5_code_capacity", "d7_spacetime", "bb72",
                                  "high_degree_general_kernel"])
@pytest.mark.parametrize("max_iter", [1, 3, 5])
def test_sum_product_llrs_track_fp64_tanh_rule(name, max_iter):
    h, pri = cases()[name]
    _, syn = sampler.sample(h, pri, seed=71, num_shots=1200)
    kw = dict(max_iter=max_iter, lottery=0)
    check_llrs(gpu_decode(h, pri, syn, **kw), oracle_sp(h, pri, syn, **kw))


def test_sum_product_large_code_global_image():
    """d=25 space-time code: graph image in global memory, state in shared."""
    hz, _ = rotated_surface(25)
    st = spacetime(hz, 25)
    pri = spacetime_priors(hz, 25, 0.003, 0.003)
    _, syn = sampler.sample(st, pri, seed=5, num_shots=48)
    kw = dict(max_iter=3, lottery=0, msg=lbp.LBP_MSG_F32)
    check_llrs(gpu_decode(st, pri, syn, **kw), oracle_sp(st, pri, syn, **kw), max_mismatch=0.05)


@pytest.mark.parametrize("name", ["d7_spacetime", "bb72"])
def test_sum_product_full_decode_with_lottery_and_osd(name):
    h, pri = cases()[name]
    _, syn = sampler.sample(h, pri, seed=72, num_shots=3000)
    kw = dict(max_iter=100, lottery=1, lottery_skip=6, osd=1, seed=4)
    g = gpu_decode(h, pri, syn, **kw)
    r = oracle_sp(h, pri, syn, **kw)
    same = (g["err"] == r.err).all(1) & (g["conv"] == r.converged)
    assert same.mean() >= 0.98, "decisions identical on only %.4f of shots" % same.mean()
    # Estimates are valid: converged shots reproduce their syndrome.
    s = sampler.unpack(syn, h.m)
    H = np.zeros((h.m, h.n), dtype=np.uint8)
    for c in range(h.m):
        H[c, h.col_idx[h.row_ptr[c]:h.row_ptr[c + 1]]] = 1
    conv = g["conv"] == 1
    assert np.array_equal((g["err"][conv].astype(np.int64) @ H.T) % 2, s[conv])


@pytest.mark.parametrize("msg", [lbp.LBP_MSG_F16, lbp.LBP_MSG_I8])
def test_sum_product_quantised_messages(msg):
    """Messages stored in binary16 or Int3.4: the estimate still satisfies the
    syndrome as often as the binary64 reference (exact McNemar test on
    per-shot convergence, 1% level)."""
    hz, _ = rotated_surface(7)
    st = spacetime(hz, 7)
    pri = spacetime_priors(hz, 7, 0.006, 0.006)
    _, syn = sampler.sample(st, pri, seed=73, num_shots=3000)
    kw = dict(max_iter=100, lottery=1, lottery_skip=6, msg=msg, seed=4)
    g = gpu_decode(st, pri, syn, **kw)
    r = oracle_sp(st, pri, syn, **kw)
    b = int(((g["conv"] == 1) & (r.converged == 0)).sum())
    c = int(((g["conv"] == 0) & (r.converged == 1)).sum())
    assert mcnemar_p(b, c) >= 0.01, (b, c)
    if msg == lbp.LBP_MSG_F16:
        # After one iteration the two storage types differ only by the binary16
        # rounding of each beta (|beta| <= 25, 11 significant bits) summed over
        # a column's DV = 2 checks, plus binary32 rounding of the sums.
        kw1 = dict(max_iter=1, lottery=0)
        g16 = gpu_decode(st, pri, syn, msg=msg, **kw1)
        g32 = gpu_decode(st, pri, syn, msg=lbp.LBP_MSG_F32, **kw1)
        bound = 2 * 25.0 * 2.0 ** -11 + 1e-5 * (1.0 + np.abs(g32["llr"]))
        assert np.all(np.abs(g16["llr"] - g32["llr"]) <= bound)


def test_sum_product_autotuner_keeps_results():
    hz, _ = rotated_surface(7)
    st = spacetime(hz, 7)
    pri = spacetime_priors(hz, 7, 0.006, 0.006)
    _, syn = sampler.sample(st, pri, seed=74, num_shots=2048)
    dec = Decoder(st, pri)
    prm = dec.params(rule=SP, msg=lbp.LBP_MSG_F16, osd=1, seed=3)
    x = torch.from_numpy(np.ascontiguousarray(syn).view(np.int64)).cuda()
    a = dec.decode(x, prm)
    ea = a.err.clone()
    dec.tune(x, prm)
    b = dec.decode(x, prm)
    torch.cuda.synchronize()
    assert torch.equal(ea, b.err)
    dec.close()
