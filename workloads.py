"""Seeded synthetic inputs shared by the tests, the oracle legs and bench.py.

This module only draws random numbers and assembles planted Tucker tensors
(Sec. 2.2 model T = G x_1 F_1 ... x_N F_N + E); it holds none of the HOOI /
TTM-tree arithmetic of either side.  The planted product uses torch.tensordot
(a library contraction) so that neither the oracle nor the CUDA path is
involved in making its own inputs.

Workload recipes (synthetic stand-ins; the paper fills its tensors with
random data, Sec. 6 "Tensors"):
  small_hooi   3-way FP64 64^3, core 8^3 N(0,1), F_n = Q of QR(64x8 Gaussian),
               ||E|| = 1e-3 ||X||, ranks (8,8,8), seed 1.
  big_fp32     4-way FP32 200^4, core 20^4 whose mode spectra are scaled by
               1/k, QR factors, ||E|| = 1e-2 ||X||, ranks 20, seed 2.
  precision5   5-way 64^5, core 16^5 with geometric 0.8 mode scaling,
               1e-2 relative noise, ranks 16, seed 3 (stored BF16).
  uneven6      64x56x48x40x32x24, core 16x14x12x10x8x6 N(0,1), Student-t
               (nu = 3) noise at 1e-2 relative, seed 5 (stored BF16).
  batch4096    4096 independent 3-way FP32 tensors: every mode length uniform
               on [16, 96], every rank uniform on [4, min(16, length)], core
               N(0,1), QR factors, 1e-3 relative Gaussian noise; tensor i is
               drawn from seed 1000003 * seed + i (so the first m tensors of
               any batch with the same seed agree), batch seed 4.
"""
from __future__ import annotations

import math
from typing import Sequence

import torch


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def orthonormal_factor(L: int, K: int, gen: torch.Generator, device, dtype=torch.float64):
    """Q factor of the QR of an L x K Gaussian matrix (orthonormal columns)."""
    A = torch.randn(L, K, generator=gen, device=device, dtype=torch.float64)
    # the QR of this small matrix runs on the host (no device linear-algebra
    # library needed); the result is moved back to `device`
    Q, R = torch.linalg.qr(A.cpu())
    Q, R = Q.to(device), R.to(device)
    # make the factorisation unique: positive diagonal of R
    s = torch.sign(torch.diagonal(R))
    s[s == 0] = 1
    # LAPACK returns Q column-major: make the factor a dense row-major matrix
    return (Q * s).to(dtype).contiguous()


def spectrum_scale(K: int, kind, device):
    if kind is None:
        return None
    if kind == "inv_k":
        return 1.0 / torch.arange(1, K + 1, device=device, dtype=torch.float64)
    if isinstance(kind, tuple) and kind[0] == "geom":
        return kind[1] ** torch.arange(0, K, device=device, dtype=torch.float64)
    raise ValueError(kind)


def _mode_product(X: torch.Tensor, A: torch.Tensor, n: int) -> torch.Tensor:
    """X x_n A for A of size J x X.shape[n] via tensordot (library contraction)."""
    Y = torch.tensordot(A, X, dims=([1], [n]))  # J x (other modes)
    return torch.movedim(Y, 0, n).contiguous()


def planted_tucker(L: Sequence[int], K: Sequence[int], rho: float, seed: int,
                   spectrum=None, noise: str = "gauss", dtype=torch.float32,
                   device="cpu", build_dtype=None):
    """Planted Tucker tensor T = G x_1 F_1 ... x_N F_N + E with ||E|| = rho * ||X||.

    spectrum: None (core i.i.d. N(0,1)), "inv_k" (core mode k scaled by 1/k on
    every mode) or ("geom", r) (scaled by r^(k-1)).  noise: "gauss" or
    "student_t3".  Returns dict(T, G, F, X_norm).
    """
    device = torch.device(device)
    g = _gen(seed, device)
    N = len(L)
    bdt = build_dtype or (torch.float64 if math.prod(L) <= 50_000_000 else torch.float32)
    G = torch.randn(*K, generator=g, device=device, dtype=torch.float64)
    for n in range(N):
        d = spectrum_scale(K[n], spectrum, device)
        if d is not None:
            shape = [1] * N
            shape[n] = K[n]
            G = G * d.view(shape)
    Fs = [orthonormal_factor(L[n], K[n], g, device) for n in range(N)]
    X = G.to(bdt)
    # apply the factors from the smallest growth to the largest to keep
    # intermediates small
    order = sorted(range(N), key=lambda n: L[n] / K[n])
    for n in order:
        X = _mode_product(X, Fs[n].to(bdt), n)
    xnorm = float(torch.linalg.vector_norm(X.double() if X.numel() < 2**27 else X).item())
    numel = X.numel()
    if rho > 0:
        sigma = rho * xnorm / math.sqrt(numel)
        # draw the noise in chunks to bound the memory of big tensors
        flat = X.view(-1)
        chunk = 1 << 26
        for s in range(0, numel, chunk):
            e = min(numel, s + chunk)
            if noise == "gauss":
                z = torch.randn(e - s, generator=g, device=device, dtype=bdt)
            elif noise == "student_t3":
                # t_3 = Z / sqrt(chi2_3 / 3); unit variance needs a factor 1/sqrt(3)
                z = torch.randn(e - s, generator=g, device=device, dtype=bdt)
                chi = torch.zeros(e - s, device=device, dtype=bdt)
                for _ in range(3):
                    w = torch.randn(e - s, generator=g, device=device, dtype=bdt)
                    chi += w * w
                z = z / torch.sqrt(chi / 3.0) / math.sqrt(3.0)
            else:
                raise ValueError(noise)
            flat[s:e] += sigma * z
    T = X.to(dtype).contiguous()
    return {"T": T, "G": G, "F": Fs, "X_norm": xnorm}


def random_tensor(shape: Sequence[int], seed: int, dtype=torch.float32, device="cpu"):
    g = _gen(seed, torch.device(device))
    return torch.randn(*shape, generator=g, device=device, dtype=torch.float64).to(dtype)


def random_factor(L: int, K: int, seed: int, dtype=torch.float32, device="cpu",
                  orthonormal: bool = True):
    g = _gen(seed, torch.device(device))
    if orthonormal:
        return orthonormal_factor(L, K, g, device).to(dtype)
    return torch.randn(L, K, generator=g, device=device, dtype=torch.float64).to(dtype)


def perturbed_factors(Fs, eps: float, seed: int):
    """Starting factors near given ones: Q of the QR of F + eps * Gaussian
    (float64, on the host; positive R diagonal), one per factor -- the input
    factors that full-size parity tests hand to the GPU sweep and to the
    oracle's sweep alike."""
    g = _gen(seed, torch.device("cpu"))
    out = []
    for F in Fs:
        F = F.detach().to("cpu", torch.float64)
        A = F + eps * torch.randn(F.shape, generator=g, dtype=torch.float64)
        Q, R = torch.linalg.qr(A)
        s = torch.sign(torch.diagonal(R))
        s[s == 0] = 1
        out.append((Q * s).contiguous())
    return out


# The named workloads used by bench.py and the parity tests.
WORKLOADS = {
    "small_hooi": dict(L=(64, 64, 64), K=(8, 8, 8), rho=1e-3, seed=1, spectrum=None,
                       noise="gauss", dtype=torch.float64, sweeps=5),
    "big_fp32": dict(L=(200, 200, 200, 200), K=(20, 20, 20, 20), rho=1e-2, seed=2,
                     spectrum="inv_k", noise="gauss", dtype=torch.float32, sweeps=10),
    "precision5": dict(L=(64,) * 5, K=(16,) * 5, rho=1e-2, seed=3, spectrum=("geom", 0.8),
                       noise="gauss", dtype=torch.float32, sweeps=10),
    "uneven6": dict(L=(64, 56, 48, 40, 32, 24), K=(16, 14, 12, 10, 8, 6), rho=1e-2, seed=5,
                    spectrum=None, noise="student_t3", dtype=torch.float32, sweeps=8),
    # a 640 MB cut of the 200^4 recipe (three modes of 200, ranks 20) for
    # profiler captures of the per-sweep kernels, which must stay small
    "mid_fp32": dict(L=(200, 200, 200, 20), K=(20, 20, 20, 10), rho=1e-2, seed=6,
                     spectrum="inv_k", noise="gauss", dtype=torch.float32, sweeps=5),
}


def batch_shapes(count: int, seed: int, N: int = 3, lmin: int = 16, lmax: int = 96,
                 kmin: int = 4, kmax: int = 16):
    """Per-tensor mode lengths and ranks of a batch: L uniform on [lmin, lmax],
    K uniform on [kmin, min(kmax, L)] (integers, bounds included).  Row i is
    drawn from its own generator, so a shorter batch is a prefix of a longer
    one with the same seed."""
    dims, ranks = [], []
    for i in range(count):
        g = _gen(7919 * seed + i, torch.device("cpu"))
        L = torch.randint(lmin, lmax + 1, (N,), generator=g)
        u = torch.rand(N, generator=g, dtype=torch.float64)
        hi = torch.clamp(L, max=kmax)
        K = torch.minimum(kmin + torch.floor(u * (hi - kmin + 1).double()).long(), hi)
        dims.append(tuple(int(x) for x in L))
        ranks.append(tuple(int(x) for x in K))
    return dims, ranks


def planted_batch(count: int, seed: int, rho: float = 1e-3, N: int = 3, device="cpu",
                  lmin: int = 16, lmax: int = 96, kmin: int = 4, kmax: int = 16):
    """`count` planted Tucker tensors (FP32) packed back to back, row-major each.
    Returns dict(T flat tensor, dims, ranks, t_off)."""
    dims, ranks = batch_shapes(count, seed, N, lmin, lmax, kmin, kmax)
    sizes = [math.prod(d) for d in dims]
    t_off = [0]
    for n in sizes[:-1]:
        t_off.append(t_off[-1] + n)
    T = torch.empty(sum(sizes), dtype=torch.float32, device=device)
    for i in range(count):
        w = planted_tucker(dims[i], ranks[i], rho, 1000003 * seed + i, dtype=torch.float32,
                           device=device, build_dtype=torch.float64)
        T[t_off[i]:t_off[i] + sizes[i]] = w["T"].reshape(-1)
    return {"T": T, "dims": dims, "ranks": ranks, "t_off": t_off}


BATCH_WORKLOADS = {
    "batch4096": dict(count=4096, seed=4, rho=1e-3, sweeps=5),
}


def make_workload(name: str, device="cpu", **override):
    w = dict(WORKLOADS[name])
    w.update(override)
    out = planted_tucker(w["L"], w["K"], w["rho"], w["seed"], spectrum=w["spectrum"],
                         noise=w["noise"], dtype=w["dtype"], device=device)
    out["spec"] = w
    return out
