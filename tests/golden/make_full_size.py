"""Writes the oracle's values for the full-size workloads c3, c4 and c5.

    python tests/golden/make_full_size.py [c3] [c4] [c5]

Only the CPU oracle (oracle/qmc_oracle.py) is called, on the seeded inputs of
paper_2305_11645_gb300/inputs.py (which hold no arithmetic of the method); nothing
here touches the CUDA library.  The values go to full_size_oracle.json beside this
script, and the c5 gradient, rounded to float32, to c5_grad_f32.npy.  They are
expensive to recompute (about 1e14 FP64 flops in all), which is why they are
stored; the GPU parity tests compare against them.

  c3  per-shift estimates Q_r of the reduced periodic net, m=20, s=tau=1024,
      16 XOR shifts, f = exp(-|y|^2 / (2 tau)), and their mean.
  c4  per-shift estimates and mean of each of the 8 PDE-like lattice instances.
  c5  per-shift estimates and mean of the lattice, m=20, s=tau=1024, 8 shifts,
      f = log sum exp(y); the gradient (1/(R N)) sum_r X_r^T grad f(X_r A) (O7);
      and the central differences (O8, one pass over the rows) on the 64 seeded
      entries, step h = 1e-5 max|A|.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import qmc_oracle as O  # noqa: E402
from paper_2305_11645_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "full_size_oracle.json")
GRAD = os.path.join(HERE, "c5_grad_f32.npy")


def load():
    if os.path.exists(OUT):
        with open(OUT) as fh:
            return json.load(fh)
    return {}


def save(d):
    d["generated_by"] = ("tests/golden/make_full_size.py: the CPU oracle (oracle/qmc_oracle.py) on the seeded "
                         "inputs of paper_2305_11645_gb300/inputs.py")
    tmp = OUT + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1)
    os.replace(tmp, OUT)


def est(p):
    Q, mean = O.estimate(p)
    return {"Q": [float(v) for v in Q], "mean": float(mean)}


def main(which):
    d = load()
    if "c3" in which:
        t0 = time.time()
        d["c3"] = est(I.c3())
        d["c3"]["seconds"] = round(time.time() - t0, 1)
        save(d)
        print("c3", d["c3"], flush=True)
    if "c4" in which:
        out = []
        for i in range(len(I.C4_INSTANCES)):
            t0 = time.time()
            e = est(I.c4(i))
            e["instance"] = i
            e["m_s_tau"] = list(I.C4_INSTANCES[i])
            e["seconds"] = round(time.time() - t0, 1)
            out.append(e)
            print("c4", i, e, flush=True)
        d["c4"] = out
        save(d)
    if "c5" in which:
        p = I.c5()
        t0 = time.time()
        c5 = est(p)
        G = O.grad(p)
        np.save(GRAD, G.astype(np.float32))
        pairs = I.fd_pairs(5, p.s, p.tau)
        h = 1e-5 * float(np.abs(np.asarray(p.A, dtype=np.float64)).max())
        fd = O.fd_grad_rows(p, pairs, h)
        c5.update({"grad_file": os.path.basename(GRAD), "grad_max_abs": float(np.abs(G).max()),
                   "grad_row_sums": [float(v) for v in G.sum(axis=1)],
                   "fd_pairs": pairs.tolist(), "fd_h": h, "fd": [float(v) for v in fd],
                   "grad_at_pairs": [float(G[j, t]) for j, t in pairs],
                   "seconds": round(time.time() - t0, 1)})
        d["c5"] = c5
        save(d)
        print("c5", {k: v for k, v in c5.items() if k in ("Q", "mean", "seconds")}, flush=True)


if __name__ == "__main__":
    main(set(sys.argv[1:]) or {"c3", "c4", "c5"})
