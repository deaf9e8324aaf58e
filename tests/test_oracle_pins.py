"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these checks re-types the oracle's own loops: each compares it with a
different route (the unfolding + matrix product of Sec. 2.1, a library SVD /
eigh, an algebraic identity, a closed form or an invariant).
"""
import math

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.filterwarnings("ignore")


def unfold(X, n):
    """Mode-n unfolding (columns = mode-n fibres), Sec. 2.1."""
    return np.moveaxis(X, n, 0).reshape(X.shape[n], -1)


def fold(M, n, shape):
    full = [shape[n]] + [s for i, s in enumerate(shape) if i != n]
    return np.moveaxis(M.reshape(full), 0, n)


def ttm_by_unfolding(X, n, A):
    """Sec. 2.1: Z = X x_n A realised as A * X_(n), folded back."""
    shape = list(X.shape)
    shape[n] = A.shape[0]
    return fold(A @ unfold(X, n), n, shape)


def sin_angle(A, B):
    """Largest principal angle between the column spans of A and B (sine form)."""
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    M = Qb - Qa @ (Qa.T @ Qb)
    s = np.linalg.norm(M, 2) if M.size else 0.0
    return math.asin(min(1.0, s))


rng = np.random.default_rng(1234)


# ---------------------------------------------------------------- TTM -------
@pytest.mark.parametrize("shape,n,K", [((5, 7), 0, 3), ((5, 7), 1, 4), ((3, 4, 5), 1, 2),
                                        ((3, 4, 5, 2), 3, 3), ((2, 3, 4, 5), 0, 6)])
def test_ttm_matches_unfolding_product(orc, shape, n, K):
    X = rng.standard_normal(shape)
    A = rng.standard_normal((K, shape[n]))
    Z = orc.ttm(X, n, A)
    np.testing.assert_allclose(Z, ttm_by_unfolding(X, n, A), rtol=1e-13, atol=1e-13)


def test_ttm_matrix_special_case(orc):
    # N = 2: X x_1 A = A X and X x_2 B = X B^T
    X = rng.standard_normal((6, 9))
    A = rng.standard_normal((4, 6))
    B = rng.standard_normal((3, 9))
    np.testing.assert_allclose(orc.ttm(X, 0, A), A @ X, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(orc.ttm(X, 1, B), X @ B.T, rtol=1e-13, atol=1e-13)


def test_ttm_float_input_equals_double_of_same_values(orc):
    X = rng.standard_normal((4, 5, 6)).astype(np.float32)
    A = rng.standard_normal((3, 5))
    np.testing.assert_array_equal(orc.ttm(X, 1, A), orc.ttm(X.astype(np.float64), 1, A))


def test_ttm_commutativity(orc):
    # Sec. 2.1 TTM-chain: (T x_a A) x_b B = (T x_b B) x_a A for a != b
    X = rng.standard_normal((4, 5, 6, 3))
    A = rng.standard_normal((2, 5))
    B = rng.standard_normal((3, 3))
    Z1 = orc.ttm(orc.ttm(X, 1, A), 3, B)
    Z2 = orc.ttm(orc.ttm(X, 3, B), 1, A)
    np.testing.assert_allclose(Z1, Z2, rtol=1e-13, atol=1e-13)


def test_ttm_same_mode_composes(orc):
    # (X x_n A) x_n B = X x_n (B A)
    X = rng.standard_normal((3, 6, 4))
    A = rng.standard_normal((5, 6))
    B = rng.standard_normal((2, 5))
    np.testing.assert_allclose(orc.ttm(orc.ttm(X, 1, A), 1, B), orc.ttm(X, 1, B @ A),
                               rtol=1e-12, atol=1e-12)


def test_ttm_identity_and_permutation(orc):
    X = rng.standard_normal((3, 5, 4))
    np.testing.assert_array_equal(orc.ttm(X, 1, np.eye(5)), X)
    perm = np.array([4, 2, 0, 1, 3])
    Pm = np.eye(5)[perm]
    np.testing.assert_array_equal(orc.ttm(X, 1, Pm), X[:, perm, :])


# --------------------------------------------------------------- Gram -------
@pytest.mark.parametrize("shape,n", [((6, 5, 4), 0), ((6, 5, 4), 1), ((6, 5, 4), 2)])
def test_gram_is_unfolding_outer_product(orc, shape, n):
    Z = rng.standard_normal(shape)
    U = unfold(Z, n)
    np.testing.assert_allclose(orc.gram(Z, n), U @ U.T, rtol=1e-13, atol=1e-12)


# ---------------------------------------------------------------- EVD -------
@pytest.mark.parametrize("n", [1, 2, 5, 17, 40])
def test_jacobi_matches_eigh(orc, n):
    M = rng.standard_normal((n, n + 3))
    A = M @ M.T
    ev, V, sweeps = orc.jacobi_eig(A)
    assert sweeps > 0
    ref = np.linalg.eigvalsh(A)[::-1]
    np.testing.assert_allclose(ev, ref, rtol=1e-12, atol=1e-12 * ref[0])
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(A @ V, V * ev, atol=1e-11 * ref[0])
    assert np.all(np.diff(ev) <= 0)
    # sign convention: largest-magnitude entry of each column is positive
    for j in range(n):
        i = int(np.argmax(np.abs(V[:, j])))
        assert V[i, j] > 0


def test_jacobi_indefinite_and_diagonal(orc):
    A = np.diag([3.0, -1.0, 2.0])
    ev, V, _ = orc.jacobi_eig(A)
    np.testing.assert_array_equal(ev, [3.0, 2.0, -1.0])
    np.testing.assert_array_equal(np.abs(V), np.eye(3)[:, [0, 2, 1]])
    S = rng.standard_normal((8, 8))
    S = S + S.T
    ev, V, _ = orc.jacobi_eig(S)
    np.testing.assert_allclose(ev, np.linalg.eigvalsh(S)[::-1], atol=1e-12)


# ------------------------------------------------------- STHOSVD / HOOI ------
def planted(L, K, rho, seed, spectrum=None):
    w = workloads.planted_tucker(L, K, rho, seed, spectrum=spectrum, dtype=torch.float64)
    return w["T"].numpy(), [F.numpy() for F in w["F"]], w


def test_exact_recovery_zero_noise(orc):
    L, K = (12, 10, 9), (3, 4, 2)
    T, Fp, _ = planted(L, K, 0.0, 11)
    F, G = orc.sthosvd(T, K)
    for n in range(3):
        assert sin_angle(F[n], Fp[n]) < 1e-12
    nT2 = orc.norm2(T)
    assert orc.fit(nT2, orc.norm2(G)) > 1 - 1e-7
    assert orc.residual(T, G, F) < 1e-12 * math.sqrt(nT2)
    F2, G2 = orc.hooi_sweep(T, F, K)
    for n in range(3):
        assert sin_angle(F2[n], Fp[n]) < 1e-12


def test_two_way_reduces_to_truncated_svd(orc):
    # N = 2, K = (k, k): the Tucker model is a rank-k matrix approximation; the
    # best one is the truncated SVD (Eckart-Young), and both STHOSVD and HOOI
    # reach it.
    X = rng.standard_normal((15, 11))
    k = 4
    U, s, Vt = np.linalg.svd(X)
    best = math.sqrt(float(np.sum(s[k:] ** 2)))
    F, G = orc.sthosvd(X, (k, k))
    assert abs(orc.residual(X, G, F) - best) < 1e-12 * best
    assert sin_angle(F[0], U[:, :k]) < 1e-10
    assert sin_angle(F[1], Vt[:k].T) < 1e-10
    F2, G2 = orc.hooi_sweep(X, F, (k, k))
    assert abs(orc.residual(X, G2, F2) - best) < 1e-12 * best
    np.testing.assert_allclose(np.abs(G2), np.diag(s[:k]), atol=1e-12 * s[0])
    fit = orc.fit(orc.norm2(X), orc.norm2(G2))
    assert abs(fit - (1 - best / math.sqrt(orc.norm2(X)))) < 1e-12


def test_full_rank_fits_exactly(orc):
    X = rng.standard_normal((4, 5, 3))
    F, G = orc.sthosvd(X, X.shape)
    assert orc.residual(X, G, F) < 1e-12
    F2, G2 = orc.hooi_sweep(X, F, X.shape)
    assert abs(orc.fit(orc.norm2(X), orc.norm2(G2)) - 1.0) < 1e-7


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_orthonormal_identity(orc, dtype):
    # ||T||^2 = ||G||^2 + ||T - G x F||^2 when G = T x F^T with orthonormal F
    T, _, _ = planted((9, 8, 7, 6), (3, 3, 2, 2), 0.5, 21)
    T = T.astype(dtype)
    F, G = orc.sthosvd(T, (3, 3, 2, 2))
    F2, G2 = orc.hooi_sweep(T, F, (3, 3, 2, 2))
    nT2 = orc.norm2(T)
    res = orc.residual(T, G2, F2)
    assert abs(nT2 - (orc.norm2(G2) + res * res)) < 1e-13 * nT2
    for Fn in F2:
        np.testing.assert_allclose(Fn.T @ Fn, np.eye(Fn.shape[1]), atol=1e-13)


def test_hooi_fit_monotone_hard_case(orc):
    # High noise and uneven ranks: the fit moves across sweeps and must not
    # decrease (Sec. 2.2: each invocation reduces the error).
    L, K = (14, 12, 10), (5, 3, 4)
    T, _, _ = planted(L, K, 0.8, 5)
    F, G = orc.sthosvd(T, K)
    nT2 = orc.norm2(T)
    fits = [orc.fit(nT2, orc.norm2(G))]
    for _ in range(8):
        F, G = orc.hooi_sweep(T, F, K)
        fits.append(orc.fit(nT2, orc.norm2(G)))
    d = np.diff(fits)
    assert np.all(d >= -1e-12 * fits[0]), fits
    assert fits[-1] - fits[0] > 1e-6, fits  # the sweeps do change the fit here


def test_gauss_seidel_reaches_same_fixed_point(orc):
    L, K = (10, 9, 8), (3, 3, 3)
    T, _, _ = planted(L, K, 0.3, 9)
    F, _ = orc.sthosvd(T, K)
    Fj, Fg = F, F
    for _ in range(30):
        Fj, Gj = orc.hooi_sweep(T, Fj, K)
        Fg, Gg = orc.hooi_sweep(T, Fg, K, gauss_seidel=True)
    nT2 = orc.norm2(T)
    assert abs(orc.fit(nT2, orc.norm2(Gj)) - orc.fit(nT2, orc.norm2(Gg))) < 1e-9
    for n in range(3):
        assert sin_angle(Fj[n], Fg[n]) < 1e-6


def test_hooi_uses_input_factors(orc):
    # Fig. 2: every chain uses the INPUT factors.  Mode 0's new factor depends
    # only on F_1, F_2, so perturbing F_0 must not change it.
    L, K = (8, 7, 6), (2, 3, 2)
    T, _, _ = planted(L, K, 0.4, 3)
    F, _ = orc.sthosvd(T, K)
    F_alt = [np.linalg.qr(rng.standard_normal(F[0].shape))[0], F[1], F[2]]
    A, _ = orc.hooi_sweep(T, F, K)
    B, _ = orc.hooi_sweep(T, F_alt, K)
    np.testing.assert_allclose(A[0], B[0], atol=1e-12)
    assert sin_angle(A[1], B[1]) > 1e-6


def test_core_definition(orc):
    X = rng.standard_normal((5, 4, 6))
    Fs = [np.linalg.qr(rng.standard_normal((d, k)))[0] for d, k in zip(X.shape, (2, 3, 2))]
    G = orc.core(X, Fs)
    ref = X
    for n in range(3):
        ref = ttm_by_unfolding(ref, n, Fs[n].T)
    np.testing.assert_allclose(G, ref, rtol=1e-12, atol=1e-12)


def test_sthosvd_singular_values_of_unfolding(orc):
    # mode-1 Gram eigenvalues are the squared singular values of T_(1)
    X = rng.standard_normal((7, 6, 5))
    F, G, evs = orc.sthosvd(X, (3, 3, 3), return_evals=True)
    s = np.linalg.svd(unfold(X, 0), compute_uv=False)
    np.testing.assert_allclose(evs[0], s ** 2, rtol=1e-11)


@pytest.mark.parametrize("order", [(2, 0, 3, 1), (3, 2, 1, 0), (0, 1, 2, 3)])
def test_sthosvd_order_steps_match_eigh(orc, order):
    """STHOSVD in a given mode order, step by step against numpy: the tensor
    before step i is T times the factors of the modes taken earlier (built
    here by unfolding products, Sec. 2.1); mode m's factor spans the leading
    K_m eigenvectors of that tensor's mode-m Gram (numpy eigh), its reported
    eigenvalues are that Gram's, and G is the final tensor.  The discarded
    eigenvalues then add up to ||T||^2 - ||G||^2 (each step removes exactly the
    energy outside the kept subspace), whatever the order."""
    L, K = (7, 5, 6, 4), (3, 2, 4, 2)
    X = rng.standard_normal(L)
    F, G, evs = orc.sthosvd(X, K, return_evals=True, order=order)
    Y = X.copy()
    discarded = 0.0
    for m in order:
        Ym = unfold(Y, m)
        w, V = np.linalg.eigh(Ym @ Ym.T)
        w, V = w[::-1], V[:, ::-1]
        np.testing.assert_allclose(evs[m], w, rtol=1e-10, atol=1e-10 * w[0])
        assert sin_angle(F[m], V[:, :K[m]]) < 1e-9, m
        np.testing.assert_allclose(F[m].T @ F[m], np.eye(K[m]), atol=1e-12)
        discarded += w[K[m]:].sum()
        Y = ttm_by_unfolding(Y, m, F[m].T)
    np.testing.assert_allclose(G, Y, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(orc.norm2(X) - orc.norm2(G), discarded, rtol=1e-9)


def test_sthosvd_order_is_honoured_and_natural_is_default(orc):
    """The natural order given explicitly is the default call bit for bit; a
    different order gives a different (valid) decomposition on a generic
    tensor: the factor of a mode taken late differs from the one taken first."""
    L, K = (7, 5, 6), (3, 2, 2)
    X = rng.standard_normal(L)
    F0, G0 = orc.sthosvd(X, K)
    F1, G1 = orc.sthosvd(X, K, order=(0, 1, 2))
    assert all(np.array_equal(a, b) for a, b in zip(F0, F1)) and np.array_equal(G0, G1)
    F2, G2 = orc.sthosvd(X, K, order=(2, 1, 0))
    assert sin_angle(F2[0], F0[0]) > 1e-3
    with pytest.raises(ValueError):
        orc.sthosvd(X, K, order=(0, 0, 1))


def test_sthosvd_any_order_recovers_exact_rank(orc):
    """Zero noise, exact multilinear rank K: every order reproduces T and
    finds the planted subspaces."""
    L, K = (12, 10, 9), (3, 4, 2)
    T, Fp, _ = planted(L, K, 0.0, 11)
    nT2 = orc.norm2(T)
    for order in [(1, 2, 0), (2, 0, 1)]:
        F, G = orc.sthosvd(T, K, order=order)
        for n in range(3):
            assert sin_angle(F[n], Fp[n]) < 1e-12
        assert orc.residual(T, G, F) < 1e-12 * math.sqrt(nT2)


# --------------------------------------------------------------------------
# FP8 E4M3 storage with per-64 scales (the precision form's FP8 variant)
# --------------------------------------------------------------------------
def test_e4m3_decode_follows_the_format(orc):
    """Sign, 4-bit exponent (bias 7), 3-bit mantissa; subnormals below 2^-6;
    largest finite 448; one NaN code per sign."""
    assert orc.e4m3_decode(0x38) == 1.0
    assert orc.e4m3_decode(0x7E) == 448.0
    assert orc.e4m3_decode(0x01) == 2.0 ** -9
    assert orc.e4m3_decode(0x08) == 2.0 ** -6
    assert orc.e4m3_decode(0x07) == 7 * 2.0 ** -9
    assert orc.e4m3_decode(0xB8) == -1.0
    assert math.isnan(orc.e4m3_decode(0x7F)) and math.isnan(orc.e4m3_decode(0xFF))
    vals = [orc.e4m3_decode(c) for c in range(0x7F)]
    assert all(b > a for a, b in zip(vals, vals[1:]))


def test_e4m3_encode_roundtrip_ties_and_saturation(orc):
    for c in list(range(0x7F)) + list(range(0x80, 0xFF)):
        assert orc.e4m3_encode(orc.e4m3_decode(c)) == c, hex(c)
    # midpoints go to the even code
    assert orc.e4m3_encode(1.0625) == 0x38      # between 1.0 (0x38) and 1.125 (0x39)
    assert orc.e4m3_encode(1.1875) == 0x3A      # between 1.125 (0x39) and 1.25 (0x3A)
    assert orc.e4m3_encode(-1.0625) == 0xB8
    assert orc.e4m3_encode(2.0 ** -10) == 0x00  # half the smallest subnormal: tie to 0
    assert orc.e4m3_encode(3 * 2.0 ** -10) == 0x02
    # beyond 448 saturates
    assert orc.e4m3_encode(449.0) == 0x7E and orc.e4m3_encode(1e30) == 0x7E
    assert orc.e4m3_encode(-1e30) == 0xFE


def test_e4m3_encode_matches_library_cast(orc):
    """torch's float8_e4m3fn cast (an independent implementation) agrees on
    random values inside the finite range."""
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8_e4m3fn")
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.uniform(-448, 448, 20000), rng.standard_normal(20000) * 1e-2,
                        rng.standard_normal(2000) * 1e-3]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    got = np.array([orc.e4m3_encode(float(a)) for a in v], dtype=np.uint8)
    assert np.array_equal(got, ref)


def test_fp8_quantize_scales_and_error_bound(orc):
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(64 * 37 + 11) * np.repeat(rng.uniform(0.01, 100, 38), 64)[:64 * 37 + 11]
         ).astype(np.float32)
    x[64 * 5:64 * 6] = 0.0  # an all-zero slab
    q, s = orc.fp8_quantize(x)
    assert q.size == x.size and s.size == 38
    xh = orc.fp8_dequantize(q, s)
    for j in range(38):
        sl = slice(64 * j, min(x.size, 64 * j + 64))
        if np.all(x[sl] == 0):
            assert s[j] == 1.0 and np.all(xh[sl] == 0)
            continue
        # the slab's largest magnitude maps to the largest code
        assert np.max(q[sl] & 0x7F) == 0x7E
        # round to nearest: half a spacing, relative 2^-4 for normal codes,
        # absolute 2^-10 s below 2^-6 s
        err = np.abs(xh[sl] - x[sl].astype(np.float64))
        bound = np.maximum(np.abs(x[sl]).astype(np.float64) * 2.0 ** -4, float(s[j]) * 2.0 ** -10)
        assert np.all(err <= bound * (1 + 1e-6)), j
