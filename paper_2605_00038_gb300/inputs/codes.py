"""Check-matrix builders for the synthetic workloads.

These build the sparse GF(2) check matrices H that the decoder runs on.  They
hold none of the decoder's arithmetic: they only place ones in a matrix.

* ``rotated_surface(d)``      rotated planar surface code, H_Z and H_X.
* ``unrotated_surface(d)``    the [[d^2+(d-1)^2, 1, d]] unrotated code in the
                              index convention of Table III (Sec. IV-B).
* ``spacetime(H, T, ...)``    the d-round space-time matrix of Eq. (1).
* ``bivariate_bicycle(...)``  BB codes, H_X = [A|B], H_Z = [B^T|A^T].

A matrix is returned as :class:`SparseH` (CSR with sorted column indices).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class SparseH:
    """CSR form of an m x n GF(2) matrix; column indices sorted per row."""

    m: int
    n: int
    row_ptr: np.ndarray  # int32[m+1]
    col_idx: np.ndarray  # int32[nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @staticmethod
    def from_rows(rows, n: int) -> "SparseH":
        row_ptr = np.zeros(len(rows) + 1, dtype=np.int32)
        cols = []
        for i, r in enumerate(rows):
            r = sorted(set(int(c) for c in r))
            if r and (r[0] < 0 or r[-1] >= n):
                raise ValueError("column index out of range")
            cols.extend(r)
            row_ptr[i + 1] = len(cols)
        return SparseH(len(rows), n, row_ptr, np.asarray(cols, dtype=np.int32))

    @staticmethod
    def from_dense(a: np.ndarray) -> "SparseH":
        a = np.asarray(a) & 1
        return SparseH.from_rows([np.nonzero(r)[0] for r in a], a.shape[1])

    def rows(self):
        for i in range(self.m):
            yield self.col_idx[self.row_ptr[i]:self.row_ptr[i + 1]]

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.m, self.n), dtype=np.uint8)
        for i, r in enumerate(self.rows()):
            a[i, r] = 1
        return a

    def csc(self):
        """(col_ptr, row_idx) of the same matrix, rows ascending per column."""
        counts = np.bincount(self.col_idx, minlength=self.n)
        col_ptr = np.zeros(self.n + 1, dtype=np.int32)
        np.cumsum(counts, out=col_ptr[1:])
        order = np.argsort(self.col_idx, kind="stable")  # CSR order is row-major
        rows = np.repeat(np.arange(self.m, dtype=np.int32), np.diff(self.row_ptr))
        return col_ptr, rows[order].astype(np.int32)

    def row_weights(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def col_weights(self) -> np.ndarray:
        return np.bincount(self.col_idx, minlength=self.n)


# ---------------------------------------------------------------------------
# Rotated surface code (standard layout; the paper fixes none, so any
# consistent qubit order serves).  Data qubit (r, c) has index r*d + c.
# Plaquette (r, c) for r, c in -1..d-1 covers the data qubits among
# (r, c), (r, c+1), (r+1, c), (r+1, c+1).  Bulk plaquettes with (r+c) even
# are Z-type, odd are X-type.  Weight-2 Z plaquettes sit on the left/right
# edges, weight-2 X plaquettes on the top/bottom edges.
# ---------------------------------------------------------------------------

def _plaquette(d: int, r: int, c: int):
    out = []
    for dr in (0, 1):
        for dc in (0, 1):
            rr, cc = r + dr, c + dc
            if 0 <= rr < d and 0 <= cc < d:
                out.append(rr * d + cc)
    return out


def rotated_surface(d: int):
    """Return (H_Z, H_X) of the distance-d rotated surface code.

    H_Z rows detect X errors; each has ((d*d-1)//2) rows and d*d columns.
    """
    if d < 2 or d % 2 == 0:
        raise ValueError("rotated surface code needs odd d >= 3")
    z_rows, x_rows = [], []
    for r in range(-1, d):
        for c in range(-1, d):
            q = _plaquette(d, r, c)
            bulk = 0 <= r < d - 1 and 0 <= c < d - 1
            even = (r + c) % 2 == 0
            if bulk:
                (z_rows if even else x_rows).append(q)
            elif len(q) == 2:
                # left/right edges carry Z boundary checks, top/bottom X ones,
                # alternating with the bulk colouring.
                if (c == -1 or c == d - 1) and even:
                    z_rows.append(q)
                elif (r == -1 or r == d - 1) and not even:
                    x_rows.append(q)
    n = d * d
    return SparseH.from_rows(z_rows, n), SparseH.from_rows(x_rows, n)


# ---------------------------------------------------------------------------
# Unrotated surface code, index convention of Table III: n = d^2 + (d-1)^2
# data qubits, m = d(d-1) checks of each type; j is the in-round check index.
# ---------------------------------------------------------------------------

def unrotated_surface(d: int):
    """Return (H_X, H_Z) of the [[d^2+(d-1)^2, 1, d]] unrotated code.

    Rows follow the neighbour pattern of Table III (Sec. IV-B) for one round:
    H_X row j touches j, j+d, d^2+j-1-floor(j/d), d^2+j-floor(j/d) (the last
    two dropped at the left/right edges); H_Z row j touches
    j+floor(j/(d-1)), that +1, d^2+j-d+1 and that +(d-1) (the vertical ones
    dropped in the first/last row of checks).
    """
    n = d * d + (d - 1) ** 2
    m = d * (d - 1)
    hx, hz = [], []
    for j in range(m):
        row = [j, j + d]
        v2 = d * d + j - 1 - j // d
        if j % d != 0:
            row.append(v2)
        if j % d != d - 1:
            row.append(v2 + 1)
        hx.append(row)
        v0 = j + j // (d - 1)
        row = [v0, v0 + 1]
        w2 = d * d + j - d + 1
        if j // (d - 1) != 0:
            row.append(w2)
        if j // (d - 1) != d - 1:
            row.append(w2 + (d - 1))
        hz.append(row)
    return SparseH.from_rows(hx, n), SparseH.from_rows(hz, n)


# ---------------------------------------------------------------------------
# Space-time matrix, Eq. (1): one copy of H per round on the block diagonal,
# then measurement-error columns.  Measurement block b hits rounds b and b+1.
#   boundary="open":   T-1 measurement blocks; the final readout is perfect.
#   boundary="cyclic": T blocks, block T-1 also hits round 0 (this is the
#                      form whose sizes Table II prints).
# Column layout: data (t, q) -> t*n + q; measurement (b, j) -> T*n + b*m + j.
# Row layout: (t, j) -> t*m + j.
# ---------------------------------------------------------------------------

def spacetime(h: SparseH, T: int, boundary: str = "open") -> SparseH:
    if T < 1:
        raise ValueError("T >= 1")
    if boundary not in ("open", "cyclic"):
        raise ValueError("boundary must be 'open' or 'cyclic'")
    m, n = h.m, h.n
    nblocks = T if boundary == "cyclic" else T - 1
    rows = []
    base_rows = [list(r) for r in h.rows()]
    for t in range(T):
        for j in range(m):
            row = [t * n + q for q in base_rows[j]]
            for b in (t - 1, t):
                if boundary == "cyclic":
                    b %= T
                if 0 <= b < nblocks and (T > 1):
                    row.append(T * n + b * m + j)
            rows.append(row)
    return SparseH.from_rows(rows, T * n + nblocks * m)


def block_diag(a: SparseH, b: SparseH) -> SparseH:
    """[[a, 0], [0, b]]: rows of b after a's, columns of b after a's."""
    rows = [list(r) for r in a.rows()] + [[a.n + q for q in r] for r in b.rows()]
    return SparseH.from_rows(rows, a.n + b.n)


def spacetime_priors(h: SparseH, T: int, p_data: float, p_meas: float,
                     boundary: str = "open") -> np.ndarray:
    nblocks = T if boundary == "cyclic" else T - 1
    return np.concatenate([np.full(T * h.n, p_data), np.full(nblocks * h.m, p_meas)])


# ---------------------------------------------------------------------------
# Bivariate bicycle codes (Bravyi et al., Nature 2024): x = S_l (x) I_m,
# y = I_l (x) S_m with S the cyclic shift; A, B are sums of three monomials.
# ---------------------------------------------------------------------------

def _shift(k: int, p: int) -> np.ndarray:
    return np.roll(np.eye(k, dtype=np.uint8), p, axis=1)


def _bb_poly(l: int, m: int, terms) -> np.ndarray:
    out = np.zeros((l * m, l * m), dtype=np.uint8)
    for var, p in terms:
        if var == "x":
            mat = np.kron(_shift(l, p), np.eye(m, dtype=np.uint8))
        else:
            mat = np.kron(np.eye(l, dtype=np.uint8), _shift(m, p))
        out ^= mat
    return out


def bivariate_bicycle(l: int, m: int, a_terms, b_terms):
    """Return (H_X, H_Z) with H_X = [A|B], H_Z = [B^T|A^T]."""
    A = _bb_poly(l, m, a_terms)
    B = _bb_poly(l, m, b_terms)
    hx = np.concatenate([A, B], axis=1)
    hz = np.concatenate([B.T, A.T], axis=1)
    return SparseH.from_dense(hx), SparseH.from_dense(hz)


BB_CODES = {
    # name: (l, m, A terms, B terms)
    "bb72": (6, 6, [("x", 3), ("y", 1), ("y", 2)], [("y", 3), ("x", 1), ("x", 2)]),
    "bb144": (12, 6, [("x", 3), ("y", 1), ("y", 2)], [("y", 3), ("x", 1), ("x", 2)]),
    "bb288": (12, 12, [("x", 3), ("y", 2), ("y", 7)], [("y", 3), ("x", 1), ("x", 2)]),
}


def bb_code(name: str):
    l, m, a, b = BB_CODES[name]
    return bivariate_bicycle(l, m, a, b)


# ---------------------------------------------------------------------------
# GF(2) helpers for evaluation (rank, logical operators).  Used to score
# logical failures, never by the decoder.
# ---------------------------------------------------------------------------

def gf2_rank(a: np.ndarray) -> int:
    a = (np.asarray(a, dtype=np.uint8) & 1).copy()
    rows, cols = a.shape
    r = 0
    for c in range(cols):
        piv = np.nonzero(a[r:, c])[0]
        if piv.size == 0:
            continue
        p = r + piv[0]
        if p != r:
            a[[r, p]] = a[[p, r]]
        hit = np.nonzero(a[:, c])[0]
        hit = hit[hit != r]
        a[hit] ^= a[r]
        r += 1
        if r == rows:
            break
    return r


def gf2_nullspace(a: np.ndarray) -> np.ndarray:
    """Basis (rows) of {x : a x = 0} over GF(2)."""
    a = (np.asarray(a, dtype=np.uint8) & 1).copy()
    rows, cols = a.shape
    pivots = []
    r = 0
    for c in range(cols):
        if r == rows:
            break
        piv = np.nonzero(a[r:, c])[0]
        if piv.size == 0:
            continue
        p = r + piv[0]
        if p != r:
            a[[r, p]] = a[[p, r]]
        hit = np.nonzero(a[:, c])[0]
        hit = hit[hit != r]
        a[hit] ^= a[r]
        pivots.append(c)
        r += 1
    free = [c for c in range(cols) if c not in set(pivots)]
    basis = np.zeros((len(free), cols), dtype=np.uint8)
    for k, f in enumerate(free):
        basis[k, f] = 1
        for i, pc in enumerate(pivots):
            if a[i, f]:
                basis[k, pc] = 1
    return basis


def logical_operators(h_check: SparseH, h_other: SparseH) -> np.ndarray:
    """Operators L (rows) that decide whether a residual r of errors detected
    by ``h_check`` is a logical error: r is trivial iff L r = 0 (mod 2),
    given h_check r = 0.  L spans ker(h_other) modulo rowspace(h_check)."""
    hc = h_check.to_dense()
    ho = h_other.to_dense()
    ker = gf2_nullspace(ho)
    base = hc.copy()
    rank = gf2_rank(base)
    out = []
    for v in ker:
        cand = np.vstack([base, v[None, :]])
        rk = gf2_rank(cand)
        if rk > rank:
            base, rank = cand, rk
            out.append(v)
    return np.array(out, dtype=np.uint8).reshape(len(out), hc.shape[1])
