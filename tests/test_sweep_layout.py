"""Index arithmetic of the one-CTA double-word LDL^T sweep (csrc/dw_ldl.cuh), restated on the host.

The dense-bin factorisation of the headline path and the CURN factorisation up to P = 232 run
this sweep on a padded packed triangle (row i at prow(i), even rows padded so that a pair at an
even column is one 16-byte access).  Pass B enumerates the trailing triangle's 2x2 tiles through
a table of (row pair, column pair) or a float square-root decode, and the L^-1 tiles through a
quotient by an approximate reciprocal of the column-pair count W, corrected by +-1.  These tests
run the same formulas in Python (float64 in place of double words): every tile of every step is
visited exactly once, every access lies inside the triangle and the staging, the sweep gives D
and L^-1 of A = L D L^T, and both inexact decodes are exact after their corrections for every
index the kernels use, with the reciprocal off by up to two ulps either way."""
import numpy as np
import pytest


def prow(i):
    return (i + 1) * (i + 1) // 2 if i & 1 else i * (i + 2) // 2


def tri_decode_f(e):
    """the kernels' packed-lower decode by a float32 square root with its +-1 correction"""
    e = np.asarray(e, dtype=np.int64)
    r = ((np.sqrt(np.float32(8.0) * e.astype(np.float32) + np.float32(1.0)) - np.float32(1.0))
         * np.float32(0.5)).astype(np.int64)
    r = np.where(r * (r + 1) // 2 > e, r - 1, np.where((r + 1) * (r + 2) // 2 <= e, r + 1, r))
    return r, e - r * (r + 1) // 2


def quotient(e, W, rw):
    """pass B's L^-1 tile row: q = (int)((e + 0.5) rw) corrected by +-1 against q W <= e"""
    e = np.asarray(e, dtype=np.int64)
    q = ((e.astype(np.float32) + np.float32(0.5)) * np.float32(rw)).astype(np.int64)
    q = q - (q * W > e)
    q = q + ((q + 1) * W <= e)
    return q


def sweep(A, use_table):
    n = A.shape[0]
    nT_ = prow(n)
    nh = n // 2 + 1
    T = np.full(nT_, np.nan)
    for i in range(n):
        T[prow(i): prow(i) + i + 1] = A[i, : i + 1]
        if not i & 1:
            T[prow(i) + i + 1] = 0.0

    def at(x):
        assert 0 <= x < nT_, (x, nT_)
        return x

    table = [(i, j) for i in range(n) for j in range(i + 1)]

    def pivot(a00, a10, a11, two, j):
        T[at(prow(j) + j)] = a00
        r0, r1, l10 = 1.0 / a00, 0.0, 0.0
        if two:
            l10 = a10 * r0
            d1 = a11 - l10 * a10
            T[at(prow(j + 1) + j + 1)] = d1
            r1 = 1.0 / d1
        return (r0, r1, a10, l10)

    pv = pivot(T[0], T[2] if n > 1 else 0, T[3] if n > 1 else 0, n > 1, 0)
    for j in range(0, n - 1, 2):
        r0, r1, a10, l10 = pv
        rj, rj1, s2 = prow(j), prow(j + 1), n - j - 2
        pl, uu, xr = {}, {}, {}
        for e in range(s2):  # pass A: trailing rows
            i = j + 2 + e
            assert e >> 1 < nh
            a0, a1 = T[at(prow(i) + j)], T[at(prow(i) + j + 1)]
            l0 = a0 * r0
            w = a1 - l0 * a10
            T[prow(i) + j] = T[prow(i) + j + 1] = 0.0
            pl[e], uu[e] = (l0, w * r1), (a0, w)
        for c in range(j + 2):  # pass A: row j+1 of L^-1
            xj, x1 = 0.0, 1.0
            if c < j:
                xj = T[at(rj + c)]
                x1 = T[at(rj1 + c)] - l10 * xj
                T[rj1 + c] = x1
            elif c == j:
                xj, x1 = 1.0, -l10
                T[at(rj1 + c)] = x1
            xr[c] = (xj, x1)
        if s2 & 1:
            pl[s2], uu[s2] = (0.0, 0.0), (0.0, 0.0)
        nTp = (s2 + 1) >> 1
        cntT, W = nTp * (nTp + 1) // 2, (j + 2) >> 1
        cnt = cntT + nTp * W
        rw = np.float32(1.0) / np.float32(W)
        seen = []
        nxt = None
        for t in range(cnt):
            if t < cntT:
                I, L = table[t] if use_table else tuple(int(v) for v in tri_decode_f(t))
                assert L <= I < nTp and I < nh
                i0, c0 = j + 2 + 2 * I, j + 2 + 2 * L
                p0, p1, q0, q1 = pl[2 * I], pl.get(2 * I + 1), uu[2 * L], uu[2 * L + 1]
                seen.append(("T", I, L))
            else:
                e = t - cntT
                q = int(quotient(e, W, rw))
                cc = e - q * W
                assert 0 <= cc < W and 0 <= q < nTp
                i0, c0 = j + 2 + 2 * q, 2 * cc
                I = q
                p0, p1, q0, q1 = pl[2 * q], pl.get(2 * q + 1), xr[2 * cc], xr[2 * cc + 1]
                seen.append(("X", q, cc))
            row1 = 2 * I + 1 < s2
            v = []
            for b, p, live in ((i0 * (i0 + 2) // 2, p0, True), ((i0 + 2) * (i0 + 2) // 2, p1, row1)):
                if not live:
                    v.append(v[0])
                    continue
                e0 = T[at(b + c0)] - (p[0] * q0[0] + p[1] * q0[1])
                e1 = T[at(b + c0 + 1)] - (p[0] * q1[0] + p[1] * q1[1])
                T[b + c0], T[b + c0 + 1] = e0, e1
                v.append((e0, e1))
            if t == 0 and cntT > 0:  # trailing tile (0, 0): the next pivot block
                nxt = pivot(v[0][0], v[1][0], v[1][1], row1, j + 2)
        want = [("T", I, L) for I in range(nTp) for L in range(I + 1)] + \
               [("X", I, c) for I in range(nTp) for c in range(W)]
        assert sorted(seen) == sorted(want), j
        pv = nxt
    D, X = np.zeros(n), np.eye(n)
    for i in range(n):
        D[i] = T[prow(i) + i]
        X[i, :i] = T[prow(i): prow(i) + i]
    return D, X


@pytest.mark.parametrize("use_table", [True, False])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 9, 16, 17, 30, 31])
def test_sweep_covers_and_factors(n, use_table):
    rng = np.random.default_rng(300 + n)
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    D, X = sweep(A, use_table)
    Lc = np.linalg.cholesky(A)
    L = Lc / np.diag(Lc)
    np.testing.assert_allclose(D, np.diag(Lc) ** 2, rtol=1e-10)
    np.testing.assert_allclose(X, np.linalg.inv(L), rtol=1e-9, atol=1e-9)


def test_padded_rows_hold_pairs_on_16_bytes():
    for i in range(0, 700):
        assert prow(i) % 2 == 0 and prow(i + 1) - prow(i) == (i + 2 if i % 2 == 0 else i + 1)


def test_tri_decode_exact_up_to_2_23():
    """the packed-lower decode is exact for every index below 2^23 (the FP64 CURN kernel's bound)"""
    for lo in range(0, 1 << 23, 1 << 20):
        e = np.arange(lo, lo + (1 << 20), dtype=np.int64)
        r, c = tri_decode_f(e)
        assert np.all(r * (r + 1) // 2 + c == e) and np.all((c >= 0) & (c <= r))


@pytest.mark.parametrize("n", [67, 150, 166, 232, 233])
def test_linv_quotient_exact_with_reciprocal_error(n):
    """q = floor(e / W) for every L^-1 tile index of every step, with 1/W off by up to 2 ulps"""
    for j in range(0, n - 1, 2):
        s2, W = n - j - 2, (j + 2) >> 1
        nTp = (s2 + 1) >> 1
        e = np.arange(nTp * W, dtype=np.int64)
        r = np.float32(1.0) / np.float32(W)
        rs = [r]
        for direction in (np.float32(np.inf), np.float32(0.0)):
            x = r
            for _ in range(2):
                x = np.nextafter(x, direction)
                rs.append(x)
        for rw in rs:
            assert np.array_equal(quotient(e, W, rw), e // W), (n, j, rw)
