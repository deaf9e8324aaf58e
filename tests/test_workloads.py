"""Host checks of the seeded input recipe (workloads.py), which both the CUDA
path and the oracle read: the planted structure, the noise level, the
spectra, the batch shape ranges and the determinism the parity tests rely on.
The oracle's own reconstruction (an independent route) rebuilds the noiseless
part."""
import math

import numpy as np
import torch

import workloads


def noiseless(orc, w):
    return orc.reconstruct(w["G"].numpy(), [F.numpy() for F in w["F"]])


def test_same_seed_same_tensor_and_seeds_differ():
    a = workloads.planted_tucker((9, 8, 7), (3, 2, 2), 0.1, 5)
    b = workloads.planted_tucker((9, 8, 7), (3, 2, 2), 0.1, 5)
    c = workloads.planted_tucker((9, 8, 7), (3, 2, 2), 0.1, 6)
    assert torch.equal(a["T"], b["T"]) and not torch.equal(a["T"], c["T"])
    d1, r1 = workloads.batch_shapes(40, 4)
    d2, r2 = workloads.batch_shapes(10, 4)
    assert d1[:10] == d2 and r1[:10] == r2  # a shorter batch is a prefix


def test_factors_orthonormal_and_structure_exact(orc):
    """Zero noise: T is exactly G x_1 F_1 ... x_N F_N with orthonormal F_n, and
    its norm is the core's (orthonormal factors preserve the Frobenius norm)."""
    w = workloads.planted_tucker((14, 11, 9, 6), (4, 3, 3, 2), 0.0, 8, dtype=torch.float64)
    for F in w["F"]:
        Fn = F.numpy()
        np.testing.assert_allclose(Fn.T @ Fn, np.eye(Fn.shape[1]), atol=1e-13)
    np.testing.assert_allclose(w["T"].numpy(), noiseless(orc, w), atol=1e-12)
    assert math.isclose(w["X_norm"], float(np.linalg.norm(w["G"].numpy())), rel_tol=1e-12)


def test_gaussian_noise_level_is_rho(orc):
    """||T - X|| = rho ||X|| up to the sampling spread of a chi distribution
    (relative spread ~ 1 / sqrt(2 |T|) = 0.3 % here)."""
    for rho in (1e-3, 0.3, 1.0):
        w = workloads.planted_tucker((30, 25, 20), (4, 5, 3), rho, 9, dtype=torch.float64)
        E = w["T"].numpy() - noiseless(orc, w)
        assert abs(np.linalg.norm(E) / w["X_norm"] - rho) <= 0.02 * rho
        z = E.reshape(-1) / (rho * w["X_norm"] / math.sqrt(E.size))
        assert abs(z.mean()) < 0.05 and abs(z.std() - 1) < 0.02


def test_student_t3_noise_unit_variance_heavy_tails(orc):
    """Student-t noise with 3 degrees of freedom, scaled to unit variance
    (t_3 has variance 3): about rho ||X|| in norm, with tails heavier than a
    Gaussian's (sample kurtosis well above 3)."""
    w = workloads.planted_tucker((40, 40, 40), (4, 4, 4), 0.1, 11, noise="student_t3",
                                 dtype=torch.float64)
    E = w["T"].numpy() - noiseless(orc, w)
    z = E.reshape(-1) / (0.1 * w["X_norm"] / math.sqrt(E.size))
    assert abs(z.std() - 1) < 0.25
    kurt = float(np.mean(z ** 4) / np.mean(z ** 2) ** 2)
    assert kurt > 5, kurt


def test_spectra_scale_the_core():
    """"inv_k" scales core index k of every mode by 1/k, ("geom", r) by
    r^(k-1): the same draw with and without the scaling differs by exactly
    those factors."""
    L, K = (10, 9, 8), (4, 3, 5)
    base = workloads.planted_tucker(L, K, 0.0, 3, dtype=torch.float64)["G"].numpy()
    for kind, f in (("inv_k", lambda k: 1.0 / k), (("geom", 0.8), lambda k: 0.8 ** (k - 1))):
        G = workloads.planted_tucker(L, K, 0.0, 3, spectrum=kind, dtype=torch.float64)["G"].numpy()
        scale = np.ones(K)
        for n in range(3):
            shape = [1, 1, 1]
            shape[n] = K[n]
            scale = scale * np.array([f(k) for k in range(1, K[n] + 1)]).reshape(shape)
        np.testing.assert_allclose(G, base * scale, rtol=1e-14)


def test_batch_shapes_follow_the_recipe():
    """Lengths uniform on [16, 96], ranks on [4, min(16, L)], all values of
    both ranges reached over 4096 tensors; every core is full rank-feasible
    (K_n <= product of the other ranks)."""
    dims, ranks = workloads.batch_shapes(4096, 4)
    Ls = [l for d in dims for l in d]
    Ks = [k for r in ranks for k in r]
    assert min(Ls) == 16 and max(Ls) == 96 and len(set(Ls)) == 81
    assert min(Ks) == 4 and max(Ks) == 16 and len(set(Ks)) == 13
    for d, r in zip(dims, ranks):
        for n in range(3):
            assert 4 <= r[n] <= min(16, d[n])
            assert r[n] <= math.prod(r) // r[n]
    # mean tensor size near the recipe's 56^3 (uniform lengths, mean 56)
    assert abs(np.mean([math.prod(d) for d in dims]) / 56 ** 3 - 1) < 0.15


def test_named_workloads_match_their_stated_sizes():
    W = workloads.WORKLOADS
    assert W["big_fp32"]["L"] == (200,) * 4 and W["big_fp32"]["K"] == (20,) * 4
    assert W["precision5"]["L"] == (64,) * 5 and W["precision5"]["K"] == (16,) * 5
    assert W["uneven6"]["L"] == (64, 56, 48, 40, 32, 24)
    assert W["uneven6"]["K"] == (16, 14, 12, 10, 8, 6)
    assert W["small_hooi"]["L"] == (64,) * 3 and W["small_hooi"]["dtype"] == torch.float64
    assert workloads.BATCH_WORKLOADS["batch4096"]["count"] == 4096


def test_perturbed_factors_are_orthonormal_and_seeded():
    F = [workloads.orthonormal_factor(30, 5, workloads._gen(1, torch.device("cpu")), "cpu")]
    a = workloads.perturbed_factors(F, 0.05, 7)
    b = workloads.perturbed_factors(F, 0.05, 7)
    c = workloads.perturbed_factors(F, 0.05, 8)
    assert torch.equal(a[0], b[0]) and not torch.equal(a[0], c[0])
    assert torch.allclose(a[0].T @ a[0], torch.eye(5, dtype=torch.float64), atol=1e-12)
    # close to the input subspace, but not equal to it
    s = torch.linalg.svdvals(F[0].T @ a[0])
    assert 0.8 < float(s.min()) < 1.0
