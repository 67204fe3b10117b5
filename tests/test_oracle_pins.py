"""Pins that tie the CPU oracle to the mathematics and to the paper.

Each test checks the oracle against something other than itself: brute-force
enumeration, a library routine, a closed form or a value the paper prints.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import OracleParams, PREC_F16, PREC_F32, PREC_F64, PREC_I8
from paper_2605_00038_gb300.inputs import sampler
from paper_2605_00038_gb300.inputs.codes import (SparseH, bb_code, gf2_rank, logical_operators,
                                                 rotated_surface, spacetime, spacetime_priors,
                                                 unrotated_surface)


def mu_of(p):
    return np.log((1.0 - p) / p)


# --------------------------------------------------------------------- trees

def random_tree(rng, max_vars=14):
    """Tanner tree: every check has degree >= 2, no cycles."""
    nv = 1
    rows = []
    while True:
        parent = int(rng.integers(nv))
        k = int(rng.integers(1, 4))
        if nv + k > max_vars:
            break
        rows.append([parent] + list(range(nv, nv + k)))
        nv += k
        if rng.random() < 0.12:
            break
    if not rows:
        rows = [[0, 1]]
        nv = 2
    return SparseH.from_rows(rows, nv)


def all_errors(n):
    return np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.int64)


def brute_min_marginals(h, mu, s):
    E = all_errors(h.n)
    ok = np.all((E @ h.to_dense().T.astype(np.int64)) % 2 == s[None, :], axis=1)
    E = E[ok]
    cost = E @ mu
    out = np.empty(h.n)
    for v in range(h.n):
        out[v] = cost[E[:, v] == 1].min() - cost[E[:, v] == 0].min()
    return out


def brute_log_marginals(h, p, s):
    E = all_errors(h.n)
    ok = np.all((E @ h.to_dense().T.astype(np.int64)) % 2 == s[None, :], axis=1)
    E = E[ok]
    logw = (E * np.log(p) + (1 - E) * np.log(1 - p)).sum(axis=1)
    out = np.empty(h.n)
    for v in range(h.n):
        a = np.logaddexp.reduce(logw[E[:, v] == 0])
        b = np.logaddexp.reduce(logw[E[:, v] == 1])
        out[v] = a - b
    return out


@pytest.mark.parametrize("seed", range(12))
def test_min_sum_on_trees_is_exact_min_marginal(seed):
    """Unscaled min-sum (f = 1) on a tree: lambda_v equals the minimum cost of
    a syndrome-consistent error with e_v = 1 minus that with e_v = 0."""
    rng = np.random.default_rng(seed)
    h = random_tree(rng)
    p = rng.uniform(0.01, 0.3, size=h.n)
    s = rng.integers(0, 2, size=h.m).astype(np.uint8)
    prm = OracleParams(max_iter=3 * (h.m + h.n), scale_mode=0, scale_const=1.0, lottery=False,
                       early_exit=False, prec=PREC_F64)
    res = oracle.decode(h, p, s[None, :], prm, want_llr=True, nthreads=1)
    want = brute_min_marginals(h, mu_of(p), s)
    assert np.allclose(res.llr[0], want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", range(8))
def test_sum_product_on_trees_is_exact_marginal(seed):
    rng = np.random.default_rng(100 + seed)
    h = random_tree(rng, max_vars=12)
    p = rng.uniform(0.02, 0.3, size=h.n)
    s = rng.integers(0, 2, size=h.m).astype(np.uint8)
    prm = OracleParams(max_iter=3 * (h.m + h.n), lottery=False, early_exit=False,
                       prec=PREC_F64, rule=oracle.oracle.RULE_SUM_PRODUCT)
    res = oracle.decode(h, p, s[None, :], prm, want_llr=True, nthreads=1)
    want = brute_log_marginals(h, p, s)
    assert np.allclose(res.llr[0], want, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("s_c", [0, 1])
def test_sum_product_degree_two_check_passes_message_and_saturates(s_c):
    """A weight-2 check forwards its other input unchanged, 2 atanh(tanh(a / 2))
    = a, with the sign (-1)^{s_c}; above 25 the magnitude saturates at 25."""
    h = SparseH(1, 2, np.array([0, 2]), np.array([0, 1]))
    for p0, p1 in ((0.05, 0.2), (1e-15, 0.2), (1e-15, 1e-14)):
        p = np.array([p0, p1])
        mu = mu_of(p)
        prm = OracleParams(max_iter=1, lottery=False, early_exit=False, prec=PREC_F64,
                           rule=oracle.oracle.RULE_SUM_PRODUCT)
        res = oracle.decode(h, p, np.array([[s_c]], dtype=np.uint8), prm, want_llr=True, nthreads=1)
        sign = -1.0 if s_c else 1.0
        want = mu + sign * np.minimum(mu[::-1], 25.0)
        assert np.allclose(res.llr[0], want, rtol=1e-9, atol=1e-9), (p0, p1)


@pytest.mark.parametrize("seed", range(6))
def test_f32_mode_is_single_precision(seed):
    """F32 mode: every posterior is a binary32 value, close to the F64 one."""
    rng = np.random.default_rng(200 + seed)
    h = random_tree(rng)
    p = rng.uniform(0.01, 0.3, size=h.n)
    s = rng.integers(0, 2, size=h.m).astype(np.uint8)
    common = dict(max_iter=3 * (h.m + h.n), scale_mode=0, scale_const=1.0, lottery=False,
                  early_exit=False)
    r64 = oracle.decode(h, p, s[None, :], OracleParams(prec=PREC_F64, **common), want_llr=True)
    r32 = oracle.decode(h, p, s[None, :], OracleParams(prec=PREC_F32, **common), want_llr=True)
    lam = r32.llr[0]
    assert np.array_equal(lam.astype(np.float32).astype(np.float64), lam)
    assert np.allclose(lam, r64.llr[0], rtol=1e-5, atol=1e-5)


# ----------------------------------------------------------- storage rounding

def test_round_f16_matches_ieee_half():
    rng = np.random.default_rng(3)
    xs = np.concatenate([
        rng.standard_normal(3000) * 10.0,
        rng.uniform(-1e-4, 1e-4, 2000),                      # subnormal range
        np.array([65504.0, 65519.0, 65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26,
                  1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, -0.0, 0.0]),
    ]).astype(np.float32).astype(np.float64)
    for x in xs:
        with np.errstate(over="ignore"):
            want = float(np.float16(np.float32(x)))
        got = oracle.round_f16(float(x))
        assert got == want or (math.isinf(got) and math.isinf(want)), (x, got, want)


def test_round_i8_int34_definition():
    cases = {0.0: 0.0, 1.0 / 32: 0.0, 3.0 / 32: 2.0 / 16, 5.0 / 32: 2.0 / 16, -3.0 / 32: -2.0 / 16,
             0.3: 5.0 / 16, 7.9375: 7.9375, 8.0: 127.0 / 16, 100.0: 127.0 / 16,
             -100.0: -127.0 / 16, -7.96875: -127.0 / 16}
    for x, want in cases.items():
        assert oracle.round_i8(x) == want, x


# ---------------------------------------------------------------------- RNG

def test_splitmix64_published_outputs():
    assert [oracle.splitmix64_at(0, k) for k in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # counter-addressed == sequential stream from a nonzero state
    seed = 0x1234_5678_9ABC_DEF0
    state = seed
    M = (1 << 64) - 1
    for k in range(5):
        state = (state + 0x9E3779B97F4A7C15) & M
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        assert oracle.splitmix64_at(seed, k) == z ^ (z >> 31)


# ------------------------------------------------------------------ lottery

def _H(rows, n):
    return SparseH.from_rows(rows, n)


def test_lottery_random_check_is_kth_member():
    h = _H([[0, 1], [1, 2], [2, 3], [3, 4], [4, 5]], 6)
    U = np.array([0, 1, 0, 1, 1], dtype=np.uint8)        # members 1, 3, 4
    lam = np.ones(6)
    N = 3
    for u, want in [(0, 1), (2 ** 32 - 1, 4), ((2 ** 32 + N - 1) // N, 3),
                    ((2 ** 32) // N - 1, 1), (2 * ((2 ** 32 + N - 1) // N), 4)]:
        c, _ = oracle.lottery_select(h, U, lam, u)
        assert c == want, (u, c, want)


def test_lottery_prefers_most_unsatisfied_then_least_reliable_then_lowest():
    # c0 = {0, 1, 2}; v0 touches c0 only, v1 touches c0, c1, c2; v2 touches c0, c1.
    h = _H([[0, 1, 2], [1, 2], [1, 3], [3, 4]], 5)
    U = np.array([1, 1, 1, 0], dtype=np.uint8)
    lam = np.array([0.1, 5.0, 0.2, 1.0, 1.0])
    assert oracle.lottery_select(h, U, lam, 0) == (0, 1)    # count 3 beats |lambda|
    U = np.array([1, 1, 0, 0], dtype=np.uint8)                # now v1, v2 both count 2
    assert oracle.lottery_select(h, U, lam, 0) == (0, 2)    # then least |lambda|
    lam = np.array([0.1, -0.2, 0.2, 1.0, 1.0])
    assert oracle.lottery_select(h, U, lam, 0) == (0, 1)    # |-0.2| == |0.2|: lowest index
    assert oracle.lottery_select(h, np.zeros(4, np.uint8), lam, 0) == (-1, -1)


def test_lottery_baseline_policies():
    """Sec. III-B baselines.  c0 = {0, 1, 2}, c1 = {2, 3, 4}, c2 = {4, 5}."""
    h = _H([[0, 1, 2], [2, 3, 4], [4, 5]], 6)
    U = np.array([1, 1, 1], dtype=np.uint8)
    lam = np.array([0.5, -0.1, 0.3, -0.2, -0.4, 2.0])   # in error: 1, 3, 4
    # worst CN: c1 has 2 columns in error (3, 4), c0 and c2 one each
    assert oracle.lottery_select(h, U, lam, 0, policy=1) == (1, 3)   # then least |lambda| in c1: |-0.2|
    # worst CN, ties -> lowest row: make c0 also have 2 errors
    lam2 = lam.copy()
    lam2[0] = -0.05
    assert oracle.lottery_select(h, U, lam2, 0, policy=1) == (0, 0)
    # random VN: column floor(u2 deg / 2^32) of c*, u2 = high 32 bits
    for u2, want in [(0, 2), (2 ** 32 - 1, 4), ((2 ** 32 + 2) // 3, 3)]:
        assert oracle.lottery_select(h, U, lam, u2 << 32, policy=2) == (1, want)
    # random CN (k-th member) with unreliable VN: no unsatisfied-count criterion
    hh = _H([[0, 1, 2], [1, 2], [1, 3], [3, 4]], 5)
    UU = np.array([1, 1, 1, 0], dtype=np.uint8)
    ll = np.array([0.1, 5.0, 0.2, 1.0, 1.0])
    assert oracle.lottery_select(hh, UU, ll, 0, policy=0) == (0, 1)  # proposed: count first
    assert oracle.lottery_select(hh, UU, ll, 0, policy=3) == (0, 0)  # least |lambda| only
    # random CN + random VN: member k of U, column floor(u2 deg / 2^32)
    assert oracle.lottery_select(hh, UU, ll, (2 ** 31) << 32 | (2 ** 32 - 1), policy=4) == (2, 3)


def test_fig4_plain_bp_deadlock():
    """Fig. 4b: on the [[13,1,3]] code with error {q2, q8, q9}, plain BP with
    a uniform prior settles on the ambiguous mix {q1, q9} (plus the easy q8),
    which leaves X0 unsatisfied, and never converges."""
    _, hz = unrotated_surface(3)
    e = np.zeros(13, dtype=np.uint8)
    e[[2, 8, 9]] = 1
    s = (hz.to_dense().astype(int) @ e % 2).astype(np.uint8)
    assert sorted(np.nonzero(s)[0].tolist()) == [0, 1, 2, 5]
    p = np.full(13, 0.05)
    for it in (3, 10):
        r = oracle.decode(hz, p, s[None, :], OracleParams(max_iter=it, lottery=False,
                                                        early_exit=False))
        assert sorted(np.nonzero(r.err[0])[0].tolist()) == [1, 8, 9]
        shat = hz.to_dense().astype(int) @ r.err[0] % 2
        assert sorted(np.nonzero(shat != s)[0].tolist()) == [0]
    plain = oracle.decode(hz, p, s[None, :], OracleParams(max_iter=100, lottery=False))
    assert plain.converged[0] == 0 and plain.iters[0] == 100


@pytest.mark.parametrize("code", ["d7_cc", "d11_st"])
def test_lottery_lowers_nonconvergence_on_surface_codes(code):
    """Sec. VI-B (invoke rate of the global decoder): on surface codes the
    lottery leaves far fewer shots unconverged than plain BP."""
    if code == "d7_cc":
        h, _ = rotated_surface(7)
        pri = np.full(h.n, 0.05)
        B = 3000
    else:
        hz, _ = rotated_surface(11)
        h = spacetime(hz, 11)
        pri = spacetime_priors(hz, 11, 0.003, 0.003)
        B = 600
    _, syn = sampler.sample(h, pri, seed=21, num_shots=B)
    S = sampler.unpack(syn, h.m)
    plain = oracle.decode(h, pri, S, OracleParams(max_iter=100, lottery=False))
    lot = oracle.decode(h, pri, S, OracleParams(max_iter=100, lottery=True, seed=4))
    f_plain = 1 - plain.converged.mean()
    f_lot = 1 - lot.converged.mean()
    assert f_plain > 0.2 and f_lot < 0.5 * f_plain, (f_plain, f_lot)


# ---------------------------------------------------------------------- OSD

def _greedy_basis(Hd, order):
    basis = []
    rank = 0
    for j in order:
        cand = Hd[:, basis + [j]]
        r = gf2_rank(cand)
        if r > rank:
            basis.append(j)
            rank = r
    return basis


@pytest.mark.parametrize("seed", range(40))
def test_osd0_against_brute_force(seed):
    rng = np.random.default_rng(500 + seed)
    m = int(rng.integers(2, 8))
    n = int(rng.integers(m, 12))
    Hd = (rng.random((m, n)) < 0.4).astype(np.uint8)
    for r in range(m):                       # no weight-1 rows
        if Hd[r].sum() == 1:
            Hd[r, (np.nonzero(Hd[r])[0][0] + 1) % n] = 1
    h = SparseH.from_dense(Hd)
    lam = rng.standard_normal(n)
    lam[rng.integers(n)] = lam[rng.integers(n)]   # a tie now and then
    if rng.random() < 0.5:
        e0 = (rng.random(n) < 0.3).astype(np.uint8)
        s = (Hd.astype(int) @ e0 % 2).astype(np.uint8)
    else:
        s = rng.integers(0, 2, m).astype(np.uint8)
    e, rank, basis = oracle.osd0(h, lam, s)
    order = sorted(range(n), key=lambda v: (lam[v], v))
    want_basis = _greedy_basis(Hd, order)
    assert rank == gf2_rank(Hd) == len(want_basis)
    assert basis.tolist() == want_basis
    sols = []
    for bits in itertools.product([0, 1], repeat=len(want_basis)):
        x = np.zeros(n, dtype=np.uint8)
        x[want_basis] = bits
        if np.array_equal(Hd.astype(int) @ x % 2, s):
            sols.append(x)
    if sols:
        assert len(sols) == 1
        assert e is not None and np.array_equal(e, sols[0])
    else:
        assert e is None


# ------------------------------------------------------ decoder vs optimum

def test_d3_code_capacity_against_maximum_likelihood():
    """Rotated d=3, p = 0.05: over all 2^9 errors, converged and OSD outputs
    satisfy H e_hat = s, and the decoder's exact failure probability is at
    least the maximum-likelihood decoder's (brute force over cosets)."""
    hz, hx = rotated_surface(3)
    Hd = hz.to_dense().astype(int)
    L = logical_operators(hz, hx).astype(int)
    p = 0.05
    E = all_errors(9)
    S = (E @ Hd.T % 2).astype(np.uint8)
    w = p ** E.sum(1) * (1 - p) ** (9 - E.sum(1))
    prm = OracleParams(max_iter=20, scale_mode=0, scale_const=0.625, lottery=True,
                       lottery_skip=6, osd=True, prec=PREC_F64, seed=1)
    res = oracle.decode(hz, np.full(9, p), S, prm)
    ok_conv = res.converged.astype(bool)
    ok_osd = res.osd_used.astype(bool)
    assert np.all(ok_conv | ok_osd)
    assert np.array_equal((res.err.astype(int) @ Hd.T % 2), S)
    resid = (res.err.astype(int) + E) % 2
    fail = (resid @ L.T % 2).any(1)
    p_fail = float((w * fail).sum())
    # ML: per syndrome pick the more likely logical class.
    classes = (E @ L.T % 2)[:, 0]
    synd_id = S.astype(int) @ (1 << np.arange(4))
    p_ml = 0.0
    for sid in np.unique(synd_id):
        sel = synd_id == sid
        p0 = w[sel & (classes == 0)].sum()
        p1 = w[sel & (classes == 1)].sum()
        p_ml += min(p0, p1)
    assert p_fail >= p_ml - 1e-15
    # Minimum-weight decoding is within reach on this small code: BP+OSD is
    # no worse than twice the minimum-weight decoder's failure rate.
    mw_fail = 0.0
    for sid in np.unique(synd_id):
        sel = np.nonzero(synd_id == sid)[0]
        best = sel[np.argmin(E[sel].sum(1))]
        cls_best = classes[best]
        mw_fail += w[sel][classes[sel] != cls_best].sum()
    assert p_fail <= 2 * mw_fail + 1e-12


def test_zero_syndrome_converges_in_one_iteration():
    hz, _ = rotated_surface(5)
    s = np.zeros((3, hz.m), dtype=np.uint8)
    for prec in (PREC_F64, PREC_F32, PREC_F16, PREC_I8):
        r = oracle.decode(hz, np.full(hz.n, 0.01), s, OracleParams(prec=prec))
        assert r.converged.all() and (r.iters == 1).all() and not r.err.any()


def test_single_errors_d5():
    """Rotated d=5, every weight-1 error.  A qubit whose column of H is
    unique has a unique weight-1 explanation and plain NMS BP finds it.  Two
    top/bottom boundary qubits of one Z check share a column (they differ by
    a weight-2 X boundary stabilizer): that error is degenerate, plain BP
    stays split (Sec. II-C), and the lottery converges to one of the two."""
    hz, hx = rotated_surface(5)
    Hd = hz.to_dense().astype(int)
    L = logical_operators(hz, hx).astype(int)
    E = np.eye(25, dtype=np.uint8)
    S = (E.astype(int) @ Hd.T % 2).astype(np.uint8)
    plain = oracle.decode(hz, np.full(25, 0.01), S, OracleParams(max_iter=30, lottery=False))
    uniq = np.array([sum(np.array_equal(Hd[:, u], Hd[:, v]) for u in range(25)) == 1
                     for v in range(25)])
    assert 0 < uniq.sum() < 25
    assert plain.converged[uniq].all()
    assert np.array_equal(plain.err[uniq], E[uniq])
    assert not plain.converged[~uniq].any()
    lot = oracle.decode(hz, np.full(25, 0.01), S, OracleParams(max_iter=60, lottery=True, seed=2))
    assert lot.converged.all()
    resid = (lot.err.astype(int) + E) % 2
    assert not (resid @ Hd.T % 2).any()
    assert not (resid @ L.T % 2).any()          # equivalent up to a stabilizer


@pytest.mark.parametrize("prec", [PREC_F64, PREC_F32, PREC_F16, PREC_I8])
def test_invariants_random_shots(prec):
    hz, _ = rotated_surface(5)
    st = spacetime(hz, 5)
    pri = spacetime_priors(hz, 5, 0.02, 0.02)
    _, syn = sampler.sample(st, pri, seed=11, num_shots=400)
    S = sampler.unpack(syn, st.m)
    prm = OracleParams(max_iter=50, lottery=True, osd=True, prec=prec, seed=5)
    r = oracle.decode(st, pri, S, prm)
    Hd = st.to_dense().astype(int)
    good = r.converged.astype(bool) | r.osd_used.astype(bool)
    assert good.all()
    assert np.array_equal(r.err.astype(int) @ Hd.T % 2, S.astype(int))
    assert np.all(r.iters[~r.converged.astype(bool)] == 50)
    assert np.all((r.iters >= 1) & (r.iters <= 50))


def test_shot_offset_keys_the_lottery():
    """Decoding shots [k, k+B) alone equals the same slice of a larger batch."""
    hx, _ = bb_code("bb72")
    pri = np.full(hx.n, 0.06)
    _, syn = sampler.sample(hx, pri, seed=3, num_shots=200)
    S = sampler.unpack(syn, hx.m)
    prm = OracleParams(max_iter=60, lottery=True, seed=9)
    full = oracle.decode(hx, pri, S, prm)
    part = oracle.decode(hx, pri, S[120:], OracleParams(max_iter=60, lottery=True, seed=9,
                                                       shot_offset=120))
    assert np.array_equal(full.err[120:], part.err)
    assert np.array_equal(full.iters[120:], part.iters)


def test_rejects_weight_one_rows():
    h = SparseH.from_rows([[0], [0, 1]], 2)
    with pytest.raises(ValueError):
        oracle.decode(h, np.full(2, 0.1), np.zeros((1, 2), np.uint8), OracleParams())


@pytest.mark.parametrize("prec", [PREC_F64, PREC_F32])
def test_scale_schedule_closed_form(prec):
    """The normalisation factor of Alg. 1: f_i = 1 - 2^-(i+1) (adaptive) or the
    constant 0.625.  On one weight-2 check with equal priors and syndrome 1 the
    estimate stays zero, so BP runs all I iterations; every V2C message equals
    mu (lambda - beta = (mu + beta) - beta is exact), each C2V message is
    -fl(f_i mu), and the final posterior is mu - fl(f_{I-1} mu), exact by
    Sterbenz's lemma.  numpy's IEEE arithmetic in the same precision gives the
    expected bits.  In binary32 f_i rounds to 1.0 from i = 24 on, so after 25
    iterations lambda is exactly 0 (the hard decisions flip to 1)."""
    h = SparseH.from_rows([[0, 1]], 2)
    p = 0.2
    S = np.ones((1, 1), dtype=np.uint8)
    ft = np.float64 if prec == PREC_F64 else np.float32
    mu = ft(mu_of(p))
    for I in (1, 2, 3, 7, 12, 24, 25):
        r = oracle.decode(h, np.full(2, p), S,
                          OracleParams(max_iter=I, lottery=False, osd=False, prec=prec), want_llr=True)
        assert r.converged[0] == 0 and r.iters[0] == I
        f = ft(1.0 - 2.0 ** -I)                 # f_{I-1}, rounded once to the precision
        expect = mu - ft(f * mu)
        assert r.llr[0, 0] == r.llr[0, 1] == float(expect), (I, r.llr[0], expect)
        if prec == PREC_F32 and I == 25:
            assert expect == 0.0 and r.err[0].tolist() == [1, 1]
        else:
            assert r.err[0].tolist() == [0, 0]
    r = oracle.decode(h, np.full(2, p), S,
                      OracleParams(max_iter=3, scale_mode=0, scale_const=0.625, lottery=False, osd=False,
                                   prec=prec), want_llr=True)
    assert r.llr[0, 0] == float(mu - ft(ft(0.625) * mu))


@pytest.mark.parametrize("prec", [PREC_F64, PREC_F32])
def test_lottery_never_runs_at_the_last_iteration(prec):
    """Reading R7 (Alg. 3 applied for i >= skip, never at i = I - 1): with
    lottery_skip = I - 1 the lottery has no iteration left, so every output
    equals the decode without the lottery; one iteration earlier it does act
    (some shot's outputs change), so the comparison is not vacuous."""
    hz, _ = rotated_surface(5)
    h = spacetime(hz, 5)
    pri = spacetime_priors(hz, 5, 0.02, 0.02)
    _, syn = sampler.sample(h, pri, seed=17, num_shots=400)
    S = sampler.unpack(syn, h.m)
    I = 12
    base = dict(max_iter=I, osd=False, prec=prec, seed=3)
    off = oracle.decode(h, pri, S, OracleParams(lottery=False, **base), want_llr=True)
    last = oracle.decode(h, pri, S, OracleParams(lottery=True, lottery_skip=I - 1, **base), want_llr=True)
    for k in ("err", "converged", "iters", "llr"):
        assert np.array_equal(getattr(off, k), getattr(last, k)), k
    early = oracle.decode(h, pri, S, OracleParams(lottery=True, lottery_skip=I - 2, **base), want_llr=True)
    assert not np.array_equal(off.llr, early.llr)


def test_lottery_trajectory_on_one_check_closed_form():
    """Alg. 3 (proposed rule, skip 0) on one weight-2 check, equal priors,
    syndrome 1, where BP alone never converges.  By hand: after iteration 0
    both posteriors are mu - fl(mu/2) > 0; U = {check 0}, both columns count
    one unsatisfied check and have equal |lambda|, so the lowest column
    (reading R9) is flipped.  Iteration 1 then reads alpha_0 = lambda_0 - beta_0
    from the flipped posterior (reading R10), alpha_0 = 0 and alpha_1 = mu,
    giving (mu - fl(0.75 mu), mu - 0).  Iteration 1's lottery flips column 0
    again (least |lambda|), and iteration 2 gives the values below.  The
    expected bits come from numpy float64 doing the same operations."""
    h = SparseH.from_rows([[0, 1]], 2)
    p = 0.2
    S = np.ones((1, 1), dtype=np.uint8)
    mu = np.float64(mu_of(p))

    def run(I):
        return oracle.decode(h, np.full(2, p), S,
                             OracleParams(max_iter=I, lottery=True, lottery_skip=0, osd=False, prec=PREC_F64),
                             want_llr=True)

    half = mu - np.float64(0.5 * mu)
    r = run(1)                                             # no lottery at the last iteration
    assert r.llr[0].tolist() == [half, half]
    b75 = np.float64(0.75 * mu)
    r = run(2)
    assert r.llr[0].tolist() == [mu - b75, mu]             # column 0 was flipped after iteration 0
    lam0 = -(mu - b75)                                     # iteration 1's flip of column 0
    a0 = lam0 - (-b75)                                     # alpha_0 = lambda_0 - beta_0 (from iteration 1)
    a1 = mu - (-0.0)                                       # alpha_1 = lambda_1 - beta_1, beta_1 = -0
    r = run(3)
    assert r.llr[0].tolist() == [mu - np.float64(0.875 * a1), mu - np.float64(0.875 * abs(a0))]
    assert r.converged[0] == 0 and r.err[0].tolist() == [0, 0]


def _store_i8(x):
    """Int3.4 from its definition (Sec. VI-C): nearest multiple of 1/16, ties
    to even, saturated to [-127, 127] / 16."""
    return float(np.clip(np.rint(16.0 * x), -127.0, 127.0) / 16.0)


@pytest.mark.parametrize("prec", [PREC_F16, PREC_I8])
def test_message_storage_inside_decode_closed_form(prec):
    """Reduced-precision message storage is applied inside the decode, not
    only by the rounding helpers (Sec. VI-C; readings R15, R16).

    Same single weight-2 check as the schedule pin: equal priors, syndrome 1,
    so BP runs all I iterations.  In these modes arithmetic is binary32 and
    each C2V message is rounded once when stored.  The stored magnitude h of
    iteration i is store(fl32(f_i mu)); h lies on a grid that is a multiple of
    binary32's spacing at mu (binary16 keeps 11 bits at an exponent no larger
    than mu's; Int3.4 has spacing 1/16 and mu >= 1 here), so both
    lambda = mu - h and the next V2C message lambda + h = mu are exact.  Hence
    the final posterior is mu - store(fl32(f_{I-1} mu)), with store taken
    from numpy's IEEE half or from the Int3.4 definition.  The priors make the
    rounding change the bits, and p = 1e-4 (mu = 9.21 > 127/16) drives Int3.4
    into saturation once f_i mu > 7.97, so a decode that skipped the storage
    rounding, or the saturation, fails."""
    h = SparseH.from_rows([[0, 1]], 2)
    S = np.ones((1, 1), dtype=np.uint8)
    changed = saturated = 0
    for p in (0.2, 0.07, 1e-4):
        mu = np.float32(mu_of(p))
        for I in (1, 2, 3, 7, 12):
            r = oracle.decode(h, np.full(2, p), S,
                              OracleParams(max_iter=I, lottery=False, osd=False, prec=prec), want_llr=True)
            assert r.converged[0] == 0 and r.iters[0] == I
            prod = np.float32(np.float32(1.0 - 2.0 ** -I) * mu)      # fl32(f_{I-1} mu)
            if prec == PREC_F16:
                hq = float(np.float16(prod))
            else:
                hq = _store_i8(float(prod))
                saturated += hq == 127.0 / 16.0
            changed += hq != float(prod)
            expect = float(mu) - hq                                  # exact (see above)
            assert expect == float(np.float32(expect))
            assert r.llr[0, 0] == r.llr[0, 1] == expect, (p, I, r.llr[0], expect)
    assert changed >= 10
    if prec == PREC_I8:
        assert saturated >= 2


def test_lottery_reads_previous_iteration_syndrome():
    """Reading R6: the lottery of iteration i draws from U = s_hat(i-1) xor s
    (Alg. 3 and the pipelining note of Sec. IV-B), with s_hat(-1) = 0, not from
    this iteration's s_hat(i).  Hand-worked on the chain c0 = {v0, v1},
    c1 = {v1, v2}, mu ~ (10, 1, 1), s = (1, 0), skip 0, I = 2, F64:

    iteration 0 (f = 1/2): beta = (-mu1/2, -mu0/2 | +mu2/2, +mu1/2), so
    lambda ~ (9.5, -3.5, 1.5), e_hat = {v1}, s_hat(0) = (1, 1) != s.
    Lottery at i = 0: U = s_hat(-1) xor s = {c0}, so c* = c0; v0 and v1 each
    meet one member of U, and |lambda_1| < |lambda_0| picks v1: lambda_1 -> +3.5.
    (From s_hat(0) instead, U = {c1}, c* = c1 and v2 would be flipped; the
    decode then converges at iteration 1 on e_hat = {v1, v2}.)
    iteration 1 (f = 3/4), from the flipped posterior: alpha = (~10, 8.5 | 3, 1),
    beta = (-0.75 |alpha_1c0|, -0.75 |alpha_0c0| | 0.75 alpha_2c1, 0.75 alpha_1c1),
    lambda ~ (3.625, -5.75, 3.25): s_hat = (1, 1) != s, no lottery at I - 1,
    so the decode ends unconverged with those posteriors.  The expected bits
    repeat these operations in numpy float64, in the oracle's order of sums."""
    h = SparseH.from_rows([[0, 1], [1, 2]], 3)
    target = np.array([10.0, 1.0, 1.0])
    p = 1.0 / (1.0 + np.exp(target))
    mu = mu_of(p)
    S = np.array([[1, 0]], dtype=np.uint8)
    r = oracle.decode(h, p, S, OracleParams(max_iter=2, lottery=True, lottery_skip=0, osd=False, prec=PREC_F64),
                      want_llr=True)
    # iteration 0
    b00, b10, b11, b21 = -(0.5 * mu[1]), -(0.5 * mu[0]), 0.5 * mu[2], 0.5 * mu[1]
    lam = np.array([mu[0] + b00, (mu[1] + b10) + b11, mu[2] + b21])
    assert lam[0] > 0 and lam[1] <= 0 and lam[2] > 0             # e_hat(0) = {v1}, s_hat(0) = (1, 1)
    assert abs(lam[1]) < abs(lam[0])
    lam[1] = -lam[1]                                              # the lottery's flip (c* = c0, v* = v1)
    # iteration 1
    a00, a10, a11, a21 = lam[0] - b00, lam[1] - b10, lam[1] - b11, lam[2] - b21
    assert min(a00, a10, a11, a21) > 0
    b00, b10 = -(0.75 * abs(a10)), -(0.75 * abs(a00))
    b11, b21 = 0.75 * a21, 0.75 * a11
    want = [mu[0] + b00, (mu[1] + b10) + b11, mu[2] + b21]
    assert want[1] <= 0 < min(want[0], want[2])
    assert r.converged[0] == 0 and r.iters[0] == 2
    assert r.llr[0].tolist() == want
    assert r.err[0].tolist() == [0, 1, 0]


def test_lottery_ablation_reads_current_syndrome():
    """Policy 5 (an ablation of reading R6, not in the paper) builds U from this
    iteration's s_hat(i) and otherwise follows Alg. 3.  On the chain of the
    previous pin: s_hat(0) = (1, 1), so U = {c1} and c* = c1; v1 and v2 each
    meet one member of U, and |lambda_2| = 1.5 < |lambda_1| = 3.5 picks v2:
    lambda_2 -> -1.5.  Iteration 1 (f = 3/4), from the flipped posterior:
    alpha = (mu0, 1.5 | -4, -2) up to the exact mu, beta = (-0.75 alpha_1c0,
    -0.75 alpha_0c0 | 0.75 alpha_2c1, 0.75 alpha_1c1), lambda ~ (8.875, -8, -2):
    e_hat = {v1, v2}, s_hat = (1, 0) = s, so the decode converges at
    iteration 1.  The expected bits repeat these operations in numpy float64."""
    h = SparseH.from_rows([[0, 1], [1, 2]], 3)
    target = np.array([10.0, 1.0, 1.0])
    p = 1.0 / (1.0 + np.exp(target))
    mu = mu_of(p)
    S = np.array([[1, 0]], dtype=np.uint8)
    r = oracle.decode(h, p, S, OracleParams(max_iter=2, lottery=True, lottery_skip=0, osd=False, prec=PREC_F64,
                                            policy=5), want_llr=True)
    b00, b10, b11, b21 = -(0.5 * mu[1]), -(0.5 * mu[0]), 0.5 * mu[2], 0.5 * mu[1]
    lam = np.array([mu[0] + b00, (mu[1] + b10) + b11, mu[2] + b21])
    assert abs(lam[2]) < abs(lam[1])
    lam[2] = -lam[2]                                              # c* = c1, v* = v2
    a00, a10, a11, a21 = lam[0] - b00, lam[1] - b10, lam[1] - b11, lam[2] - b21
    assert a00 > 0 and a10 > 0 and a11 < 0 and a21 < 0
    b00, b10 = -(0.75 * a10), -(0.75 * a00)
    b11, b21 = 0.75 * a21, 0.75 * a11
    want = [mu[0] + b00, (mu[1] + b10) + b11, mu[2] + b21]
    assert want[0] > 0 and want[1] <= 0 and want[2] <= 0
    assert r.converged[0] == 1 and r.iters[0] == 2
    assert r.llr[0].tolist() == want
    assert r.err[0].tolist() == [0, 1, 1]
