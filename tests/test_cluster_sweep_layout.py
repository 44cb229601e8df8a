"""Index arithmetic of the cluster LDL^T sweep (csrc/dw_ldl_cluster.cuh), restated on the host.

The CURN factorisation for P >= 234 spreads one packed triangle over the C CTAs of a
thread-block cluster: row pair r lives in CTA r mod C at offset 4m(k+1) + 2Cm(m-1) (its m-th
pair), and pass B of each step enumerates a CTA's tiles by a float square-root decode of a flat
index.  These tests run the same index formulas in Python (float64 arithmetic in place of
double words) and check that every tile of every step is visited exactly once by exactly one
CTA, that every access stays inside the CTA's part, that the padding layout matches the
kernel's 16-byte pair accesses, that the next pivot block every CTA factors from the staged
entries equals the owner's, and that the sweep produces D and L^-1 of A = L D L^T.  The float32
decode is checked exhaustively up to the largest order the cluster path takes."""
import numpy as np
import pytest


def crow(i, C):
    r, k, m = i >> 1, (i >> 1) % C, (i >> 1) // C
    return 4 * m * (k + 1) + 2 * C * m * (m - 1) + (2 * (r + 1) if i & 1 else 0)


def cpart(n, k, C):
    npairs = (n + 1) >> 1
    M = (npairs - k + C - 1) // C if npairs > k else 0
    return 4 * M * (k + 1) + 2 * C * M * (M - 1)


def own_range(R0, k, C, npairs):
    rf = R0 + (k - R0) % C
    return rf, ((npairs - 1 - rf) // C + 1 if rf < npairs else 0)


def decode(t, n0, C):
    """pass B's row decode (float32 like the kernel) with its +-1 integer correction"""
    bq = np.float32(n0 - 0.5 * C)
    u = ((np.sqrt(bq * bq + np.float32(2.0 * C) * t.astype(np.float32)) - bq) * np.float32(1.0 / C)).astype(np.int64)
    S = lambda x: n0 * x + C * x * (x - 1) // 2
    u = np.where(S(u) > t, u - 1, np.where(S(u + 1) <= t, u + 1, u))
    return u, t - S(u)


def sweep(A, C):
    n = A.shape[0]
    npairs, nh = (n + 1) >> 1, n // 2 + 1
    T = [np.full(cpart(n, k, C), np.nan) for k in range(C)]

    def at(k, idx):
        assert 0 <= idx < len(T[k]), (k, idx, len(T[k]))
        return idx

    for i in range(n):
        k, b = (i >> 1) % C, crow(i, C)
        assert b % 2 == 0
        for c in range(i + 1):
            T[k][at(k, b + c)] = A[i, c]
        if not i & 1:
            T[k][at(k, b + i + 1)] = 0.0
    stage = {nm: [np.full((nh, 2), np.nan) for _ in range(C)] for nm in ("plE", "plO", "uuE", "uuO", "xrE", "xrO")}
    pb = [[None] * 4 for _ in range(C)]  # the next pivot block's rows before the update, and their l pairs

    def pivot(a00, a10, a11, two):
        r0, r1, l10, d1 = 1.0 / a00, 0.0, 0.0, 0.0
        if two:
            l10 = a10 * r0
            d1 = a11 - l10 * a10
            r1 = 1.0 / d1
        return (a00, d1), (r0, r1, a10, l10)

    def upd(v, p, qa, qb):
        return (v[0] - (p[0] * qa[0] + p[1] * qa[1]), v[1] - (p[0] * qb[0] + p[1] * qb[1]))

    d, pv0 = pivot(T[0][0], T[0][2] if n > 1 else 0, T[0][3] if n > 1 else 0, n > 1)
    T[0][0] = d[0]
    if n > 1:
        T[0][3] = d[1]
    pv = [pv0] * C
    for j in range(0, n - 1, 2):
        s2, R0 = n - j - 2, (j + 2) >> 1
        pvs = list(pv)
        for k in range(C):  # pass A
            r0, r1, a10, l10 = pvs[k]
            rf, nr = own_range(R0, k, C, npairs)
            xown = (j >> 1) % C == k
            for t in range(2 * nr + (j + 2 if xown else 0)):
                if t < 2 * nr:
                    i = 2 * (rf + C * (t >> 1)) + (t & 1)
                    if i >= n:
                        continue
                    e, b = i - j - 2, crow(i, C)
                    a0, a1 = T[k][at(k, b + j)], T[k][at(k, b + j + 1)]
                    l0 = a0 * r0
                    w = a1 - l0 * a10
                    T[k][b + j] = T[k][b + j + 1] = 0.0
                    stage["plO" if e & 1 else "plE"][k][e >> 1] = (l0, w * r1)
                    for q in range(C):
                        stage["uuO" if e & 1 else "uuE"][q][e >> 1] = (a0, w)
                        if e < 2:
                            pb[q][e] = (T[k][at(k, b + j + 2)], T[k][at(k, b + j + 3)])
                            pb[q][2 + e] = (l0, w * r1)
                else:
                    c, rj, rj1 = t - 2 * nr, crow(j, C), crow(j + 1, C)
                    xj, x1 = 0.0, 1.0
                    if c < j:
                        xj = T[k][at(k, rj + c)]
                        x1 = T[k][at(k, rj1 + c)] - l10 * xj
                        T[k][rj1 + c] = x1
                    elif c == j:
                        xj, x1 = 1.0, -l10
                        T[k][at(k, rj1 + c)] = x1
                    for q in range(C):
                        stage["xrO" if c & 1 else "xrE"][q][c >> 1] = (xj, x1)
            if s2 & 1 and (npairs - 1) % C == k:
                stage["plO"][k][s2 >> 1] = (0.0, 0.0)
                for q in range(C):
                    stage["uuO"][q][s2 >> 1] = (0.0, 0.0)
        seen = []
        for k in range(C):  # pass B
            rf, nr = own_range(R0, k, C, npairs)
            n0 = rf + 1
            cnt = nr * n0 + C * nr * (nr - 1) // 2
            us, ss = decode(np.arange(cnt), n0, C)
            for u, s in zip(us.tolist(), ss.tolist()):
                r = rf + C * u
                I, i0 = r - R0, 2 * r
                assert r % C == k and R0 <= r < npairs and 0 <= s <= r
                b0 = crow(i0, C)
                b1 = b0 + 2 * (r + 1)
                p0, p1 = stage["plE"][k][I], stage["plO"][k][I]
                if s <= I:
                    c0, q0, q1 = j + 2 + 2 * s, stage["uuE"][k][s], stage["uuO"][k][s]
                    seen.append(("T", I, s))
                else:
                    cc = s - I - 1
                    c0, q0, q1 = 2 * cc, stage["xrE"][k][cc], stage["xrO"][k][cc]
                    seen.append(("X", I, cc))
                v = []
                for b, p, live in ((b0, p0, True), (b1, p1, i0 + 1 < n)):
                    if not live:
                        v.append(v[0])
                        continue
                    e0 = T[k][at(k, b + c0)] - (p[0] * q0[0] + p[1] * q0[1])
                    e1 = T[k][at(k, b + c0 + 1)] - (p[0] * q1[0] + p[1] * q1[1])
                    T[k][b + c0], T[k][b + c0 + 1] = e0, e1
                    v.append((e0, e1))
                if s == 0 and I == 0:  # the owner's pivots go to its diagonal
                    dd, own = pivot(v[0][0], v[1][0], v[1][1], i0 + 1 < n)
                    T[k][at(k, b0 + j + 2)] = dd[0]
                    if i0 + 1 < n:
                        T[k][at(k, b1 + j + 3)] = dd[1]
        if s2 > 0:  # every CTA factors the next pivot block from its staging
            two = s2 > 1
            for k in range(C):
                w0 = upd(pb[k][0], pb[k][2], stage["uuE"][k][0], stage["uuO"][k][0])
                w1 = upd(pb[k][1], pb[k][3], stage["uuE"][k][0], stage["uuO"][k][0]) if two else w0
                _, pv[k] = pivot(w0[0], w1[0], w1[1], two)
                assert pv[k] == own, (j, k)
        nT = (s2 + 1) >> 1
        want = [("T", I, L) for I in range(nT) for L in range(I + 1)] + [("X", I, c) for I in range(nT) for c in range(R0)]
        assert sorted(seen) == sorted(want), j
    D, X = np.zeros(n), np.eye(n)
    for i in range(n):
        k, b = (i >> 1) % C, crow(i, C)
        D[i] = T[k][b + i]
        X[i, :i] = T[k][b: b + i]
    return D, X


@pytest.mark.parametrize("C", [2, 4, 8])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9, 16, 17, 31, 40])
def test_cluster_sweep_covers_and_factors(n, C):
    rng = np.random.default_rng(100 + n)
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    D, X = sweep(A, C)
    Lc = np.linalg.cholesky(A)
    L = Lc / np.diag(Lc)
    np.testing.assert_allclose(D, np.diag(Lc) ** 2, rtol=1e-10)
    np.testing.assert_allclose(X, np.linalg.inv(L), rtol=1e-9, atol=1e-9)


def test_cluster_parts_tile_the_triangle():
    """the parts hold every padded row exactly once, and sum to the one-CTA padded triangle"""
    for C in (2, 4, 8):
        for n in range(1, 585):
            npairs = (n + 1) >> 1
            total = sum(cpart(n, k, C) for k in range(C))
            assert total == sum(4 * (r + 1) for r in range(npairs))
            for k in range(C):
                pairs = [r for r in range(npairs) if r % C == k]
                offs = [crow(2 * r, C) for r in pairs]
                assert offs == [sum(4 * (q + 1) for q in pairs[:m]) for m in range(len(pairs))]


@pytest.mark.parametrize("C,P", [(2, 234), (2, 260), (2, 314), (4, 316), (4, 430), (8, 432), (8, 582)])
def test_cluster_tile_decode_exact(C, P):
    """the float32 square-root decode with its +-1 correction gives every step's (row, tile)"""
    npairs = (P + 1) >> 1
    for j in range(0, P - 1, 2):
        R0 = (j + 2) >> 1
        for k in range(C):
            rf, nr = own_range(R0, k, C, npairs)
            n0 = rf + 1
            lens = n0 + C * np.arange(nr)
            start = np.concatenate([[0], np.cumsum(lens)])
            t = np.arange(int(start[-1]))
            u, s = decode(t, n0, C)
            want_u = np.repeat(np.arange(nr), lens)
            assert np.array_equal(u, want_u) and np.array_equal(s, t - start[want_u])


def test_curn_kernel_choice_follows_the_shared_memory_rule():
    """the benchmark's mirror of the library's choice of CURN forward kernel: one CTA while the
    padded triangle and the staging fit 226 KB, else the smallest cluster (2, 4, 8) whose largest
    part, the double-buffered staging and the column sums fit, else FP64"""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    lim = 226 * 1024
    for P in range(2, 700, 2):
        prow = P * (P + 2) // 2
        one = 6 * (P // 2 + 1) * 16 + prow * 8 <= lim
        fits = {C: (10 * (P // 2 + 1) + 8) * 16 + 2 * P * 8 + max(cpart(P, k, C) for k in range(C)) * 8 <= lim
                for C in (2, 4, 8)}
        want = 1 if one else next((C for C in (2, 4, 8) if fits[C]), 0)
        assert bench.curn_factor_mode(P) == want, P
    assert [bench.curn_factor_mode(P) for P in (232, 234, 314, 316, 430, 432, 582, 584)] == [1, 2, 2, 4, 4, 8, 8, 0]
