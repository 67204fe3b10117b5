"""Scoring helpers (CPU): logical failures, Wilson interval, McNemar test."""
import numpy as np
import torch

from paper_2605_00038_gb300 import evaluate
from paper_2605_00038_gb300.inputs import sampler
from paper_2605_00038_gb300.inputs.codes import logical_operators, rotated_surface, spacetime


def test_logical_failures_on_known_residuals():
    d, T = 5, 3
    hz, hx = rotated_surface(d)
    st = spacetime(hz, T)
    spec = evaluate.surface_spec(d, T, st.n)
    L = logical_operators(hz, hx)
    n = st.n
    true = np.zeros((4, n), np.uint8)
    est = np.zeros((4, n), np.uint8)
    # shot 0: residual = a logical in round 1 -> failure
    true[0, hz.n * 1: hz.n * 2] = L[0]
    # shot 1: the same logical split across rounds 0 and 2 -> still a failure
    half = np.nonzero(L[0])[0]
    true[1, half[: len(half) // 2]] = 1
    true[1, 2 * hz.n + half[len(half) // 2:]] = 1
    # shot 2: residual = an X stabilizer -> no failure
    true[2, 0: hz.n] = hx.to_dense()[0]
    # shot 3: no residual but BP unresolved -> failure
    conv = np.array([1, 1, 1, 0], np.uint8)
    osd = np.zeros(4, np.uint8)
    f = evaluate.logical_failures(spec, torch.from_numpy(sampler.pack(true).view(np.int64)),
                                  torch.from_numpy(sampler.pack(est).view(np.int64)),
                                  torch.from_numpy(conv), torch.from_numpy(osd))
    assert f.tolist() == [True, True, False, True]


def test_wilson_and_mcnemar():
    lo, hi = evaluate.wilson(50, 1000)
    assert lo < 0.05 < hi and hi - lo < 0.03
    assert evaluate.mcnemar_p(0, 0) == 1.0
    assert evaluate.mcnemar_p(10, 10) > 0.5
    assert evaluate.mcnemar_p(0, 20) < 1e-5


def test_unrotated_spec_scores_logicals_and_stabilizers():
    """Unrotated surface code (Table III rows): one logical operator L, which
    commutes with the X stabilizers; a residual that is an X logical (no Z
    check sees it, and it is not a product of X stabilizers) fails, a
    residual equal to an X stabilizer (a row of H_X) does not."""
    from paper_2605_00038_gb300.inputs.codes import unrotated_surface
    d, T = 5, 3
    hx, hz = unrotated_surface(d)
    st = spacetime(hz, T)
    spec = evaluate.unrotated_surface_spec(d, T, st.n)
    assert spec.L.shape == (1, hz.n)
    L = spec.L[0]
    assert not (hx.to_dense().astype(int) @ L % 2).any()
    xl = logical_operators(hx, hz)[0]                  # an X logical: in ker(H_Z), not in rowspace(H_X)
    assert not (hz.to_dense().astype(int) @ xl % 2).any() and int(L.astype(int) @ xl) % 2 == 1
    true = np.zeros((2, st.n), np.uint8)
    true[0, 2 * hz.n: 3 * hz.n] = xl
    true[1, hz.n: 2 * hz.n] = hx.to_dense()[3]
    z = np.zeros_like(true)
    ones = np.ones(2, np.uint8)
    f = evaluate.logical_failures(spec, torch.from_numpy(sampler.pack(true).view(np.int64)),
                                  torch.from_numpy(sampler.pack(z).view(np.int64)),
                                  torch.from_numpy(ones), torch.from_numpy(np.zeros(2, np.uint8)))
    assert f.tolist() == [True, False]
