"""Pins for the check-matrix builders and the seeded sampler (CPU only)."""
from pathlib import Path

import numpy as np
import pytest

from paper_2605_00038_gb300.inputs import codes, sampler
from paper_2605_00038_gb300.inputs.codes import (SparseH, bb_code, gf2_rank, logical_operators,
                                                 rotated_surface, spacetime, unrotated_surface)

GOLDEN = Path(__file__).parent / "golden"


def _k(hx, hz):
    return hx.n - gf2_rank(hx.to_dense()) - gf2_rank(hz.to_dense())


@pytest.mark.parametrize("d", [3, 5, 7, 11])
def test_rotated_surface_css_and_k(d):
    hz, hx = rotated_surface(d)
    assert hz.m == (d * d - 1) // 2 and hz.n == d * d
    assert hz.nnz == 2 * d * (d - 1)
    assert not ((hx.to_dense().astype(int) @ hz.to_dense().T.astype(int)) % 2).any()
    assert _k(hx, hz) == 1


def test_rotated_d3_is_4x9_nnz12():
    hz, _ = rotated_surface(3)
    assert (hz.m, hz.n, hz.nnz) == (4, 9, 12)


@pytest.mark.parametrize("name,n", [("bb72", 72), ("bb144", 144), ("bb288", 288)])
def test_bb_codes_have_k12(name, n):
    hx, hz = bb_code(name)
    assert hx.n == n and hx.m == n // 2
    assert set(hx.row_weights().tolist()) == {6} and set(hx.col_weights().tolist()) == {3}
    assert not ((hx.to_dense().astype(int) @ hz.to_dense().T.astype(int)) % 2).any()
    assert _k(hx, hz) == 12


def test_table2_spacetime_sizes():
    rows = [l.split() for l in (GOLDEN / "table2_hst_sizes.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    for d, cols, nnz, *_ in rows:
        d, cols, nnz = int(d), int(cols), int(nnz)
        _, hz = unrotated_surface(d)
        st = spacetime(hz, d, "cyclic")
        assert (st.n, st.nnz) == (cols, nnz)


def _lattice_unrotated(d):
    """Independent geometric construction of the unrotated code in the
    drawing of Fig. 4: horizontal edges (y, x) for y in 0..d-1 (top row
    first), x in 0..d-1, index y*d + x; vertical edges between rows y, y+1 at
    x = 1..d-1, index d^2 + y*(d-1) + (x-1).  Vertex checks at (y, x) for
    x = 1..d-1 (row-major); face checks between rows y, y+1 and columns
    x, x+1 for x = 0..d-1 (row-major)."""
    n = d * d + (d - 1) ** 2
    def hedge(y, x):
        return y * d + x
    def vedge(y, x):
        return d * d + y * (d - 1) + (x - 1)
    vertex = []
    for y in range(d):
        for x in range(1, d):
            q = [hedge(y, x - 1), hedge(y, x)]
            if y > 0:
                q.append(vedge(y - 1, x))
            if y < d - 1:
                q.append(vedge(y, x))
            vertex.append(q)
    face = []
    for y in range(d - 1):
        for x in range(d):
            q = [hedge(y, x), hedge(y + 1, x)]
            if x >= 1:
                q.append(vedge(y, x))
            if x + 1 <= d - 1:
                q.append(vedge(y, x + 1))
            face.append(q)
    return SparseH.from_rows(face, n), SparseH.from_rows(vertex, n)


@pytest.mark.parametrize("d", [3, 5, 7, 9])
def test_table3_neighbours_match_lattice(d):
    """The Table III index formulas (builder) agree with the drawn lattice."""
    hx, hz = unrotated_surface(d)
    fx, fz = _lattice_unrotated(d)
    assert np.array_equal(hx.to_dense(), fx.to_dense())
    assert np.array_equal(hz.to_dense(), fz.to_dense())
    assert _k(hx, hz) == 1


def test_table3_round_links():
    """Table III VN4/VN5 (Tn + i - m, + m) for rounds t >= 1 of H_st."""
    d = 5
    _, hz = unrotated_surface(d)
    T = d
    st = spacetime(hz, T, "cyclic")
    n, m = hz.n, hz.m
    for i in range(m, T * m):
        row = set(st.col_idx[st.row_ptr[i]:st.row_ptr[i + 1]].tolist())
        assert {T * n + i - m, T * n + i} <= row
    # t = 0: the cyclic form links block T-1 (Table III's formula would
    # point into the data columns there, so the builder wraps instead).
    for j in range(m):
        row = set(st.col_idx[st.row_ptr[j]:st.row_ptr[j + 1]].tolist())
        assert {T * n + (T - 1) * m + j, T * n + j} <= row


def test_fig4_syndromes():
    lines = [l.split() for l in (GOLDEN / "fig4_deadlock.txt").read_text().splitlines()
             if l.strip() and not l.startswith("#")]
    kv = {}
    cands = []
    for t in lines:
        if t[0] == "candidate":
            cands.append([int(x) for x in t[1:]])
        else:
            kv[t[0]] = [int(x) for x in t[1:]]
    _, hz = unrotated_surface(3)
    H = hz.to_dense().astype(int)

    def syn(qs):
        e = np.zeros(13, dtype=int)
        e[qs] = 1
        return sorted(np.nonzero(H @ e % 2)[0].tolist())

    assert syn(kv["error"]) == kv["syndrome"]
    for c in cands:
        assert syn(c) == kv["candidate_syndrome"]
    # The two candidates have equal weight; on this lattice their sum is a
    # logical operator (not a stabilizer), so a syndrome decoder cannot tell
    # them apart and a wrong pick is a logical error.
    hx, _ = unrotated_surface(3)
    L = logical_operators(hz, hx)
    diff = np.zeros(13, dtype=np.uint8)
    diff[cands[0]] ^= 1
    diff[cands[1]] ^= 1
    assert len(cands[0]) == len(cands[1])
    assert (L.astype(int) @ diff % 2).any()


def test_spacetime_open_sizes():
    hz, _ = rotated_surface(11)
    st = spacetime(hz, 11)
    assert (st.m, st.n, st.nnz) == (660, 1931, 3620)
    hz, _ = rotated_surface(25)
    st = spacetime(hz, 25)
    assert (st.m, st.n, st.nnz) == (7800, 23113, 44976)


def test_sampler_is_seeded_and_consistent():
    hz, _ = rotated_surface(5)
    st = spacetime(hz, 5)
    pri = codes.spacetime_priors(hz, 5, 0.02, 0.01)
    e1, s1 = sampler.sample(st, pri, seed=7, num_shots=300)
    e2, s2 = sampler.sample(st, pri, seed=7, num_shots=300, nthreads=3)
    assert np.array_equal(e1, e2) and np.array_equal(s1, s2)
    e3, s3 = sampler.sample(st, pri, seed=7, num_shots=100, shot_offset=200)
    assert np.array_equal(e3, e1[200:]) and np.array_equal(s3, s1[200:])
    eb = sampler.unpack(e1, st.n).astype(int)
    sb = sampler.unpack(s1, st.m).astype(int)
    assert np.array_equal(eb @ st.to_dense().T.astype(int) % 2, sb)
    assert np.array_equal(sampler.pack(eb), e1)
    # Bernoulli rate within 5 sigma of p.
    n_data = 5 * hz.n
    rate = eb[:, :n_data].mean()
    assert abs(rate - 0.02) < 5 * np.sqrt(0.02 * 0.98 / eb[:, :n_data].size)


def test_sampler_splitmix64_published_outputs():
    # SplitMix64 from state 0: the first three outputs of the published generator.
    assert [sampler.splitmix64_at(0, k) for k in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_d25_xz_stress_form_sizes():
    """Reading R5's stress form of the d=25 workload: X and Z space-time
    matrices block-diagonal, 15,600 x 46,226 with twice the single-type nonzeros;
    the halves do not touch each other's columns."""
    from paper_2605_00038_gb300.inputs import workloads
    w = workloads.c5_d25_spacetime_xz(shots=1)
    single = workloads.c5_d25_spacetime(shots=1)
    assert (w.h.m, w.h.n) == (15600, 46226)
    assert w.h.nnz == 2 * single.h.nnz == 2 * 44976
    assert w.priors.shape == (46226,)
    rows = list(w.h.rows())
    assert max(max(r) for r in rows[:7800]) < 23113 <= min(min(r) for r in rows[7800:])
