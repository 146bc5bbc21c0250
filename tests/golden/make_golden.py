"""Write stored expected values by running the FP64 oracle (and nothing else).

    python tests/golden/make_golden.py --config c2 --lam 1e-3 --out tests/golden/c2_lam1e-3.json

Runs the full overfitting schedule of a configuration (noise quantisation, then
straight-through rounding for the last ``ste_frac`` of the iterations) on the seeded
synthetic image and records the final rate-distortion cost evaluated with rint latents
(D + lambda R, eq. (1)), together with a coarse loss trajectory.
"""
import argparse
import json
import os
import sys
import time

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import coolchic as oc  # noqa: E402
from paper_2403_11651_gb300 import synthetic as syn  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c2")
    ap.add_argument("--lam", type=float, default=None)
    ap.add_argument("--iters", type=int, default=None)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    if a.threads:
        torch.set_num_threads(a.threads)
    with open(os.path.join(ROOT, "paper_2403_11651_gb300", "configs", a.config + ".json")) as f:
        cfg = json.load(f)
    lam = cfg["lam"] if a.lam is None else a.lam
    iters = cfg["total_iters"] if a.iters is None else a.iters
    arch = oc.Arch(levels=cfg["levels"], arm_ctx=cfg["arm_ctx"], arm_layers=cfg["arm_layers"],
                   up_kernel=cfg["up_kernel"], up_per_level=cfg["up_per_level"],
                   syn_hidden=cfg["syn_hidden"], syn_res3x3=cfg["syn_res3x3"])
    train = oc.Train(lam=lam, lr=cfg["lr"], total_iters=iters, ste_frac=cfg["ste_frac"],
                     seed=a.seed)
    rgb = syn.synthetic_image(cfg["H"], cfg["W"], a.seed)
    init = syn.initial_parameters(syn.ArchSizes.from_config(cfg), a.seed)
    enc = oc.OracleEncoder(rgb, arch, train, init)
    traj = []
    t0 = time.time()
    for t in range(iters):
        loss, D, R = enc.step()
        if t % 100 == 0 or t == iters - 1:
            traj.append([t, loss, D, R])
            print(f"iter {t} loss {loss:.6g} D {D:.6g} R {R:.6g} ({time.time() - t0:.0f} s)",
                  flush=True)
    D, R, cost = enc.rd_cost(hard=True)
    out = {
        "_source": "written by tests/golden/make_golden.py from the FP64 oracle only",
        "config": a.config, "H": cfg["H"], "W": cfg["W"], "seed": a.seed, "lam": lam,
        "lr": cfg["lr"], "iters": iters, "ste_frac": cfg["ste_frac"],
        "final_hard": {"D": D, "R_bpp": R, "cost": cost},
        "trajectory": traj, "oracle_seconds": time.time() - t0,
        "torch_threads": torch.get_num_threads(),
    }
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out["final_hard"]))


if __name__ == "__main__":
    main()
