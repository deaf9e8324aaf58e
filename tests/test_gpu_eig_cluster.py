"""The warm-started eigensolver of a sweep (Sec. 5's EVD, started from the
input factors) on a cluster of CTAs per matrix -- each CTA sums an eighth of
the rows, the K x K work is the same in every CTA -- against the FP64 oracle's
sweep, and against the single-CTA form (kernel policy bit 10) to rounding.
Shapes: every mode L >= 64 (the cluster form's range), rows not divisible by
four, K odd and up to 40, FP32 and FP64 factors; a mode whose Gram has lower
rank than K (the Cholesky-QR pass finds nearly dependent columns and the
cluster's Gram-Schmidt fallback runs).  FP32 cases keep the noise at 1e-2 or
above: the fit is read through ||T||^2 - ||G||^2, whose cancellation at
lower noise exceeds the 1e-5 bar in FP32 whatever the eigensolver.
"""
import math

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tk():
    from paper_1707_05594_gb300 import build
    build.build()
    import paper_1707_05594_gb300 as pkg
    pkg.lib()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pkg


def sin_angle(A, B):
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    s = np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2)
    return math.asin(min(1.0, s))


def sweeps(tk, T, K, n_sweeps, policy):
    tk.lib().tucker_set_kernel_policy(policy)
    try:
        d = tk.Decomposition(T.cuda(), K)
        d.sthosvd()
        out = []
        for _ in range(n_sweeps):
            d.sweep()
            out.append(([f.double().cpu().numpy() for f in d.F], d.fit()))
        torch.cuda.synchronize()
    finally:
        tk.lib().tucker_set_kernel_policy(0)
    assert tk.tucker_device_status() == 0
    return out


CASES = [
    ((97, 65, 70), (9, 7, 11), 1e-2, 31, torch.float32),
    ((64, 130, 66), (33, 5, 16), 0.1, 32, torch.float32),
    ((80, 72, 64), (40, 8, 6), 0.05, 33, torch.float32),
    ((65, 67, 69), (7, 9, 5), 1e-2, 34, torch.float64),
]


@pytest.mark.parametrize("L,K,rho,seed,dtype", CASES)
def test_cluster_eigensolver_sweeps_match_oracle(tk, orc, L, K, rho, seed, dtype):
    w = workloads.planted_tucker(L, K, rho, seed, dtype=dtype)
    Tn = w["T"].numpy()
    n_sweeps = 3
    got = sweeps(tk, w["T"], K, n_sweeps, 0)
    ref1024 = sweeps(tk, w["T"], K, n_sweeps, 1024)
    fit_bar, ang_bar, orth = (1e-9, 1e-7, 1e-12) if dtype == torch.float64 else (1e-5, 1e-4, 1e-6)
    nT2 = orc.norm2(Tn)
    Fo, Go = orc.sthosvd(Tn, K)
    for s in range(n_sweeps):
        Fo, Go = orc.hooi_sweep(Tn, Fo, K)
        fit_o = orc.fit(nT2, orc.norm2(Go))
        Fg, fit_g = got[s]
        Fs, fit_s = ref1024[s]
        assert abs(fit_g - fit_o) <= fit_bar * fit_o, (s, fit_g, fit_o)
        # the cluster and single-CTA forms differ only in the order of row sums
        assert abs(fit_g - fit_s) <= fit_bar * fit_o, (s, fit_g, fit_s)
        for n in range(len(L)):
            assert sin_angle(Fg[n], Fo[n]) <= ang_bar, (s, n)
            assert sin_angle(Fg[n], Fs[n]) <= ang_bar, (s, n)
            assert np.abs(Fg[n].T @ Fg[n] - np.eye(K[n])).max() <= orth, (s, n)


def test_cluster_gram_schmidt_fallback(tk, orc):
    """A tensor of exact multilinear rank (6, 6, 6) (no noise, stored in
    FP32) decomposed with K_0 = 10: mode 0's Gram has six nonzero
    eigenvalues, so the warm subspace step gives nearly dependent columns and
    the Cholesky-QR pass gives way to the cluster's Gram-Schmidt fallback.
    The factor stays orthonormal, its leading 6 columns (the nonzero
    eigenvalues) span the oracle's, and the fit -- which the null directions
    do not change -- matches."""
    L, K = (96, 40, 30), (10, 6, 6)
    rng = np.random.default_rng(36)
    T = rng.standard_normal((6, 6, 6))
    for n, Ln in enumerate(L):
        U, _ = np.linalg.qr(rng.standard_normal((Ln, 6)))
        T = np.moveaxis(np.tensordot(U, T, axes=(1, n)), 0, n)
    T = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32))
    Tn = T.numpy()
    got = sweeps(tk, T, K, 2, 0)
    nT2 = orc.norm2(Tn)
    Fo, Go = orc.sthosvd(Tn, K)
    for s in range(2):
        Fo, Go = orc.hooi_sweep(Tn, Fo, K)
        fit_o = orc.fit(nT2, orc.norm2(Go))
        Fg, fit_g = got[s]
        assert abs(fit_g - fit_o) <= 1e-3, (s, fit_g, fit_o)
        assert np.abs(Fg[0].T @ Fg[0] - np.eye(10)).max() <= 1e-6
        assert sin_angle(Fg[0][:, :6], Fo[0][:, :6]) <= 1e-4
        for n in (1, 2):
            assert sin_angle(Fg[n], Fo[n]) <= 1e-4, (s, n)
