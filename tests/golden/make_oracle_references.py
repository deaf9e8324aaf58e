"""Writes tests/golden/oracle_references.json: the FP64 oracle's results on the
named workloads, against which bench.py states each GPU form's error.

For every workload the seeded input generator (workloads.py) builds the
tensor -- on a CUDA device when one is present, so that the values are those
the GPU forms see (the generator draws with the device's own generator) --
and the oracle (oracle/, plain C in double) runs its STHOSVD and then HOOI
sweeps with chain trees (Fig. 2) on the FP32 values.  Recorded per workload:
the fit after STHOSVD and after every sweep (they show where the fixed point
is reached), ||T||^2, and the final factors (float32, base64) for subspace
comparisons.  For the batch of small tensors only the final fit of every
tensor is kept.

Nothing here calls the CUDA library of this repository.

    python tests/golden/make_oracle_references.py [--only NAME ...] [--out PATH]
"""
from __future__ import annotations

import argparse
import base64
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "oracle_references.json")
# oracle sweeps after STHOSVD; the fits recorded per sweep show the fixed
# point reached within them (relative change below 1e-9 by the last one)
SWEEPS = {"big_fp32": 3, "precision5": 3, "uneven6": 2}
BATCH_SWEEPS = 5


def b64(a):
    import numpy as np
    return base64.b64encode(np.ascontiguousarray(a, dtype="<f4").tobytes()).decode()


def one(name, device):
    import numpy as np
    import torch

    import oracle
    import workloads
    spec = workloads.WORKLOADS[name]
    t0 = time.time()
    w = workloads.make_workload(name, device=device)
    Th = w["T"].to("cpu", torch.float32).numpy()
    del w
    if device != "cpu":
        torch.cuda.empty_cache()
    K = spec["K"]
    nT2 = oracle.norm2(Th)
    F, G = oracle.sthosvd(Th, K)
    fits = [oracle.fit(nT2, oracle.norm2(G))]
    for _ in range(SWEEPS[name]):
        F, G = oracle.hooi_sweep(Th, F, K)
        fits.append(oracle.fit(nT2, oracle.norm2(G)))
    return {"L": list(spec["L"]), "K": list(K), "normT2": nT2, "fits": fits,
            "schedule": f"oracle STHOSVD + {SWEEPS[name]} HOOI sweeps (chain trees, FP64)",
            "factors_f32_b64": [b64(f) for f in F], "seconds": round(time.time() - t0, 1),
            "threads": oracle.num_threads()}


def batch(device):
    import torch

    import oracle
    import workloads
    spec = workloads.BATCH_WORKLOADS["batch4096"]
    t0 = time.time()
    wb = workloads.planted_batch(spec["count"], spec["seed"], rho=spec["rho"], device=device)
    Tflat = wb["T"].to("cpu").numpy()
    fits = []
    for i, (L, K) in enumerate(zip(wb["dims"], wb["ranks"])):
        n = 1
        for x in L:
            n *= x
        Ti = Tflat[wb["t_off"][i]:wb["t_off"][i] + n].reshape(L)
        F, G = oracle.sthosvd(Ti, K)
        for _ in range(BATCH_SWEEPS):
            F, G = oracle.hooi_sweep(Ti, F, K)
        # the direct residual, as the batched form scores its fit
        r = oracle.residual(Ti, G, F)
        fits.append(1.0 - r / oracle.norm2(Ti) ** 0.5)
    return {"count": spec["count"], "schedule": f"oracle STHOSVD + {BATCH_SWEEPS} HOOI sweeps per tensor, "
                                                "fit from the direct residual",
            "fits": fits, "seconds": round(time.time() - t0, 1), "threads": oracle.num_threads()}


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args()
    import oracle
    oracle.build()
    device = "cuda" if torch.cuda.is_available() else "cpu"
    data = {}
    if os.path.exists(args.out):
        data = json.load(open(args.out))
    data["_about"] = ("FP64 oracle results on the named workloads, written by "
                      "tests/golden/make_oracle_references.py (oracle + seeded generator only); "
                      f"inputs drawn on {device} with torch {torch.__version__}")
    for name in ["precision5", "big_fp32", "uneven6", "batch4096"]:
        if args.only and name not in args.only:
            continue
        data[name] = batch(device) if name == "batch4096" else one(name, device)
        json.dump(data, open(args.out, "w"), indent=1)
        print(name, data[name].get("fits", [])[-3:] if name != "batch4096" else data[name]["seconds"],
              flush=True)


if __name__ == "__main__":
    main()
