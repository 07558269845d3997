"""The algebra of the two-stage reduction's kernels and of the Sturm counts,
restated in numpy from the derivations in their file headers and checked
against plain definitions (CPU only): a wrong step in a reformulation fails
here before any kernel runs.

- panel QR: one block reduction per column gives the reflector and every
  product the step needs (v^dagger P_c, v_q^dagger v), and T formed column by
  column gives Q = I - V T V^dagger;
- the trailing update Q^dagger A Q = A - V W^dagger - W V^dagger with
  W = Y - 1/2 V T^dagger Z, Y = A V T, Z = V^dagger Y;
- the rank-2 epilogue's pairing of digit-order sums in 32-bit integers;
- the bulge chase's column sums by passing entries round eight lanes;
- the triangular inverse by doubling, never reading above the diagonal;
- the FP32-seeded reciprocal with one cubic correction, and the Sturm count
  that uses it.
"""
import numpy as np
import pytest

RNG = np.random.default_rng(1310)


def crandn(*shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


# ---------------------------------------------------------------- panel QR

def panel_qr_one_reduction(P):
    """The kernel's column loop: per column i one set of sums over the rows
    below i, then the reflector and the update; returns (R, V, T, betas)."""
    P = P.copy()
    m, nb = P.shape
    V = np.zeros_like(P)
    T = np.zeros((nb, nb), complex)
    betas = np.zeros(nb, complex)
    kk = min(nb, m - 1)
    for i in range(kk):
        x = P[i + 1:, i]
        rowi = P[i, :].copy()
        s_norm = np.vdot(x, x).real
        y = {c: np.vdot(x, P[i + 1:, c]) for c in range(i + 1, nb)}     # x^H P_c
        g = {q: np.vdot(V[i + 1:, q], x) for q in range(i)}               # v_q^H x
        alpha = rowi[i]
        a2 = abs(alpha) ** 2
        s2 = a2 + s_norm
        tau, beta, scl = 0.0, 0.0, 0.0
        if s2 > 0:
            nu = np.sqrt(s2)
            if a2 > 0:
                aa = np.sqrt(a2)
                beta = -alpha * nu / aa
                tau = (aa + nu) / nu
                scl = np.conj(alpha) / (aa * (aa + nu))
            else:
                beta, tau, scl = -nu, 1.0, 1.0 / nu
        v = np.zeros(m, complex)
        v[i] = 1.0
        v[i + 1:] = x * scl
        V[:, i] = v
        betas[i] = beta
        T[i, i] = tau
        for r in range(i):
            acc = 0
            for q in range(r, i):
                # v_q^H v from the sums; v_q[i] is what the kernel reads in
                # row i of the panel, where column q holds v_q below its diagonal
                G = np.conj(V[i, q]) + scl * g[q]
                acc += T[r, q] * G
            T[r, i] = -tau * acc
        for c in range(i + 1, nb):
            z = rowi[c] + np.conj(scl) * y[c]              # v^H P_c from the sums
            P[i:, c] -= tau * v[i:] * z
        P[i, i] = beta
        P[i + 1:, i] = 0
    return P, V, T, betas


@pytest.mark.parametrize("m", [1, 2, 5, 9, 40])
def test_panel_qr_one_reduction_per_column(m):
    nb = 8
    P0 = crandn(m, nb)
    if m >= 9:
        P0[:, 3] = 0.0                      # a zero column: tau = 0 there
    R, V, T, _ = panel_qr_one_reduction(P0)
    Q = np.eye(m) - V @ T @ V.conj().T
    assert np.abs(Q.conj().T @ Q - np.eye(m)).max() < 1e-13
    # Q^H P0 = R: upper trapezoidal in the reflected columns
    QP = Q.conj().T @ P0
    assert np.abs(QP - R).max() < 1e-12 * max(1.0, np.abs(P0).max())
    kk = min(nb, m - 1)
    for i in range(kk):
        assert np.abs(R[i + 1:, i]).max(initial=0.0) == 0.0


def test_panel_qr_alpha_zero_and_zero_tail():
    # alpha = 0 with a nonzero tail, and a column that is zero below its diagonal
    m, nb = 12, 8
    P0 = crandn(m, nb)
    P0[0, 0] = 0.0
    P0[3:, 2] = 0.0
    R, V, T, betas = panel_qr_one_reduction(P0)
    Q = np.eye(m) - V @ T @ V.conj().T
    assert np.abs(Q.conj().T @ Q - np.eye(m)).max() < 1e-13
    assert np.abs(Q.conj().T @ P0 - R).max() < 1e-12 * np.abs(P0).max()
    assert abs(abs(betas[0]) - np.linalg.norm(P0[:, 0])) < 1e-13


# ---------------------------------------------------------------- trailing update

def test_two_sided_update_with_w():
    m, nb = 30, 8
    A = crandn(m, m)
    A = A + A.conj().T
    _, V, T, _ = panel_qr_one_reduction(crandn(m, nb))
    Q = np.eye(m) - V @ T @ V.conj().T
    X = A @ V                                    # A22 V (the tensor-core product)
    Y = X @ T
    Z = V.conj().T @ Y
    W = Y - 0.5 * V @ (T.conj().T @ Z)
    lhs = Q.conj().T @ A @ Q
    rhs = A - V @ W.conj().T - W @ V.conj().T
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(A).max()
    # W's kernel form: W = X T - 1/2 V M2 with M2 = T^H (V^H X) T
    M2 = T.conj().T @ (V.conj().T @ X) @ T
    assert np.abs(W - (X @ T - 0.5 * V @ M2)).max() < 1e-12 * np.abs(W).max()


# ---------------------------------------------------------------- rank-2 epilogue

def test_order_sums_pair_in_32_bits():
    # eight order sums within the bound |o_u| <= (u + 1) 2^18 of K = 64 terms
    # of 7-bit digit products, at their extremes and at random
    lim = [(u + 1) << 18 for u in range(8)]
    cases = [np.array(lim), -np.array(lim),
             np.array([(-1) ** u * lim[u] for u in range(8)])]
    cases += [np.array([RNG.integers(-l, l + 1) for l in lim]) for _ in range(2000)]
    for o in cases:
        o = [int(t) for t in o]
        hi = lo = 0
        for u in range(8):                       # the sequential 64-bit form
            if u < 4:
                hi = hi * 128 + o[u]
            else:
                lo = lo * 128 + o[u]
        p = [o[0] * 128 + o[1], o[2] * 128 + o[3], o[4] * 128 + o[5], o[6] * 128 + o[7]]
        assert all(-(1 << 31) <= q < (1 << 31) for q in p)     # fits int32
        assert p[0] * 16384 + p[1] == hi and p[2] * 16384 + p[3] == lo
        t = hi * 2097152 + (lo >> 7)
        assert abs(t) < (1 << 62)
        # 2^7 T = sum_u o_u 2^(49 - 7u) up to the floor of lo / 2^7
        exact = sum(o[u] << (49 - 7 * u) for u in range(8))
        assert 0 <= exact - 128 * t < 128


# ---------------------------------------------------------------- bulge column sums

def test_column_sums_by_rotation():
    for _ in range(20):
        O = crandn(8, 8)
        v = crandn(8)
        z = np.zeros(8, complex)
        for i in range(8):                        # lane i
            for t in range(8):
                src = (i - t) & 7
                sent = O[src, (src + t) & 7]       # what lane src sends in round t
                z[i] += sent * np.conj(v[src])
        assert np.abs(z - np.conj(v) @ O).max() < 1e-13


# ---------------------------------------------------------------- triangular inverse

def trinv_doubling(L, nbk=32):
    """The launch sequence of the doubling inverse on one matrix: diagonal
    blocks first, then per level two products per pair of inverted blocks,
    the first kept conjugate-transposed above the diagonal.  X starts as NaN
    wherever the kernels do not write before reading, so any read of an
    unwritten or scratch entry poisons the result."""
    n = L.shape[0]
    X = np.full((n, n), np.nan + 0j)
    for i0 in range(0, n, nbk):
        ib = min(nbk, n - i0)
        X[i0:i0 + ib, i0:i0 + ib] = np.tril(np.linalg.inv(np.tril(L[i0:i0 + ib, i0:i0 + ib])))
        X[i0:i0 + ib, i0 + ib:] = 0.0           # right of the diagonal block
    Lt = np.tril(L)                              # the products never read above it
    sz = nbk
    while sz < n:
        nfull = n // (2 * sz)
        rem = n - nfull * 2 * sz
        s2r = rem - sz if rem > sz else 0
        pairs = [(p * 2 * sz, sz) for p in range(nfull)]
        if s2r:
            pairs.append((nfull * 2 * sz, s2r))
        for i0, s2 in pairs:
            X11 = np.tril(X[i0:i0 + sz, i0:i0 + sz])          # tile ranges skip the upper part
            L21 = Lt[i0 + sz:i0 + sz + s2, i0:i0 + sz]
            X[i0:i0 + sz, i0 + sz:i0 + sz + s2] = X11.conj().T @ L21.conj().T   # T^H
            X22 = np.tril(X[i0 + sz:i0 + sz + s2, i0 + sz:i0 + sz + s2])
            Tp = X[i0:i0 + sz, i0 + sz:i0 + sz + s2]
            X[i0 + sz:i0 + sz + s2, i0:i0 + sz] = -X22 @ Tp.conj().T
        sz *= 2
    X[np.triu_indices(n, 1)] = 0.0
    return X


@pytest.mark.parametrize("n", [33, 64, 100, 257, 300, 529])
def test_triangular_inverse_by_doubling(n):
    A = crandn(n, n)
    A = A @ A.conj().T + n * np.eye(n)
    L = np.linalg.cholesky(A)
    Lg = L + np.triu(crandn(n, n), 1)          # whatever lies above the diagonal
    X = trinv_doubling(Lg)
    assert not np.isnan(X).any()
    assert np.abs(X @ L - np.eye(n)).max() < 1e-12


# ---------------------------------------------------------------- reciprocal, Sturm counts

def rcp_seeded(x, ulp_shift=0):
    """1/x from an FP32 reciprocal (correctly rounded, then moved by
    ulp_shift FP32 ulps as the hardware approximation may be) and the cubic
    correction r0 (1 + e + e^2), e = 1 - x r0."""
    ex = (np.frombuffer(np.float64(x).tobytes(), np.uint64)[0] >> np.uint64(52)) & np.uint64(0x7FF)
    if not (904 <= int(ex) <= 1142):
        return 1.0 / x
    r32 = np.float32(1.0) / np.float32(x)
    r32 = np.nextafter(r32, np.float32(np.inf) if ulp_shift > 0 else np.float32(-np.inf)) \
        if ulp_shift else r32
    r0 = float(r32)
    e = -x * r0 + 1.0
    return (e * e + e) * r0 + r0


def test_seeded_reciprocal_is_fp64_accurate():
    xs = np.concatenate([RNG.uniform(-1, 1, 2000) * 10.0 ** RNG.uniform(-30, 30, 2000),
                         [2.0 ** -119, 2.0 ** 119 * 1.999, -3.0, 1e-300, 1e300]])
    for x in xs:
        for sh in (-1, 0, 1):
            r = rcp_seeded(float(x), sh)
            assert abs(r * x - 1.0) <= 4 * np.finfo(float).eps, (x, sh)


def sturm_count(d, e2, x, pivmin):
    q = d[0] - x
    if abs(q) < pivmin:
        q = -pivmin
    cnt = int(q <= 0)
    for k in range(1, len(d)):
        q = -e2[k - 1] * rcp_seeded(q, 1) + (d[k] - x)
        if abs(q) < pivmin:
            q = -pivmin
        cnt += int(q <= 0)
    return cnt


def test_sturm_count_with_seeded_reciprocal():
    n = 60
    d = RNG.standard_normal(n) * 3.0
    e = RNG.standard_normal(n - 1)
    Tm = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    lam = np.linalg.eigvalsh(Tm)
    e2 = e * e
    pivmin = np.finfo(float).tiny * max(1.0, e2.max())
    gaps = np.diff(lam)
    xs = np.concatenate([(lam[:-1] + lam[1:]) / 2, [lam[0] - 1.0, lam[-1] + 1.0],
                         lam[:-1] + 1e-3 * gaps])
    for x in xs:
        assert sturm_count(d, e2, x, pivmin) == int((lam <= x).sum())
