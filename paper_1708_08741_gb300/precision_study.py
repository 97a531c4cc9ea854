"""Precision study of the reduced-precision forms against the FP64 form.

Runs one workload three times on the GPU -- ES_FP64, ES_MIXED32 (FP32
deviation PDFs) and ES_MIXED16 (FP16 relative-deviation PDFs), all through
the C ABI -- and reports the relative L2 error of the velocity (fluid cells),
the potential (unknown cells) and the particle positions of each reduced
form against the FP64 run at the requested step counts.  The FP64 form is
the reference because it matches the FP64 CPU oracle to 1e-12 (the GPU
parity tests); the oracle itself is too slow for 1,000 steps of a 128^3
channel.

    python -m paper_1708_08741_gb300.precision_study [--n 128] [--steps 100,1000]
"""
import argparse
import json

import numpy as np

import paper_1708_08741_gb300 as es
from paper_1708_08741_gb300 import workloads as W


def rel_l2(a, b):
    d = np.linalg.norm(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64))
    n = np.linalg.norm(np.asarray(b, dtype=np.float64))
    return float(d / n) if n > 0 else float(d)


def snapshot(sim):
    own = sim.field(es.FIELD_OWNER)
    return {"psi": sim.field(es.FIELD_PSI), "u": sim.field(es.FIELD_U), "x": sim.particles()["x"], "owner": own}


def compare(ref, other):
    fluid = ref["owner"] < 0
    return {"u": rel_l2(other["u"][:, fluid], ref["u"][:, fluid]),
            "psi": rel_l2(other["psi"][fluid], ref["psi"][fluid]),
            "x": rel_l2(other["x"], ref["x"]),
            "owner_equal": bool((other["owner"] == ref["owner"]).all())}


def run(n=128, checkpoints=(100, 1000), res_rf=1e-10, device="cuda:0"):
    """Errors of MIXED32 and MIXED16 against FP64 on the channel workload
    (walls in z, 64 charged spheres R = 6 at n = 128) at each checkpoint."""
    wl = W.channel(n=n, n_spheres=max(1, int(round(64 * (n / 128) ** 3))), radius=6.0,
                   levels=4 if n % 8 == 0 else 2)
    over = dict(res_rf=res_rf, max_cycles=200)
    forms = {"FP64": es.ES_FP64, "MIXED32": es.ES_MIXED32, "MIXED16": es.ES_MIXED16}
    sims = {k: es.Simulation(wl, p, device=device, overrides=over) for k, p in forms.items()}
    out = {"workload": f"channel {n}^3, walls in z, {wl.n_particles} charged spheres R=6, "
                       f"lambda_D=3, E=2e-3, RES_RF {res_rf:g}", "checkpoints": {}}
    done = 0
    for cp in sorted(checkpoints):
        for _ in range(cp - done):
            for s in sims.values():
                s.step()
        done = cp
        snaps = {k: snapshot(s) for k, s in sims.items()}
        out["checkpoints"][cp] = {k: compare(snaps["FP64"], snaps[k]) for k in ("MIXED32", "MIXED16")}
    for s in sims.values():
        s.close()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--steps", default="100,1000", help="comma-separated checkpoints")
    ap.add_argument("--res-rf", type=float, default=1e-10)
    a = ap.parse_args()
    res = run(a.n, tuple(int(v) for v in a.steps.split(",")), a.res_rf)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
