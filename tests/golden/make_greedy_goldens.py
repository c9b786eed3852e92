"""Writes the oracle's whole greedy sequence at the benchmarked sizes into tests/golden/.

The GPU parity tests compare every pick and gain of the library's k = 100 maximisations with
these files. The values come from the CPU oracle alone (oracle/, the lazy greedy of Def. ged-max
at a fixed L, FP64, lowest id on exact ties) on the seeded synthetic graphs of graphgen/; the
CUDA library is never imported here.

    python tests/golden/make_greedy_goldens.py [rmat22] [ba1m]

R-MAT scale 22 takes about ten minutes on one core, BA n = 10^6 about one minute.
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

K = 100
EPS = 1e-4

WORKLOADS = {
    "rmat22": ("R-MAT scale 22, edge factor 16, (a, b, c) = (0.57, 0.19, 0.19), seed 1",
               lambda: gg.rmat(22, 16, 0.57, 0.19, 0.19, seed=1)),
    "ba1m": ("Barabasi-Albert n = 1,000,000, m = 8, seed 1", lambda: gg.barabasi_albert(1_000_000, 8, seed=1)),
}
# workloads whose gains are also recomputed by the long-double oracle (for the FP64 GPU path: at
# n = 10^6 the FP64 oracle's sequential sums carry rounding near the FP64 tolerance itself)
LONG_DOUBLE = ("ba1m",)


def path_for(name):
    return os.path.join(HERE, f"greedy_{name}_k{K}.txt")


def write(name):
    desc, make = WORKLOADS[name]
    g = make()
    alpha = oracle.default_alpha(g)
    L, B = oracle.select_L(g, alpha, EPS / K)  # L from the bound at epsilon / k (Algorithm 2's separation)
    t0 = time.time()
    grp, gains, evals = oracle.greedy(g, K, alpha, L, "lazy")
    secs = time.time() - t0
    ld = None
    if name in LONG_DOUBLE:
        ld = [oracle.gain(g, grp[:j], int(grp[j]), alpha, L, long_double=True) for j in range(K)]
    with open(path_for(name), "w") as f:
        f.write(f"# Oracle greedy GED-Walk maximisation (Def. ged-max, Prop. greedy_approx), k = {K}.\n")
        f.write(f"# Graph: {desc}; n = {g.n}, nnz = {g.nnz}.\n")
        f.write(f"# alpha = 1/(1 + d_max) = {alpha!r}; L = {L} (Eq. comb-bound at epsilon/k = {EPS / K!r}, "
                f"B_L = {B!r}).\n")
        f.write("# Lazy greedy of oracle/ (FP64, fixed L, lowest vertex id among exactly equal gains),\n")
        f.write(f"# {evals} exact gain evaluations, {secs:.0f} s. Written by tests/golden/make_greedy_goldens.py.\n")
        if ld is None:
            f.write("# step vertex gain\n")
        else:
            f.write("# step vertex gain gain_long_double (the same gain by the long-double oracle)\n")
        for j in range(K):
            extra = "" if ld is None else f" {float(ld[j])!r}"
            f.write(f"{j} {int(grp[j])} {float(gains[j])!r}{extra}\n")
    print(f"{name}: L = {L}, {secs:.0f} s, head {list(grp[:5])}", flush=True)


def read(name):
    """(alpha, L, group, gains, long-double gains or None) from a golden file."""
    import numpy as np

    alpha = L = None
    grp, gains, ld = [], [], []
    for line in open(path_for(name)):
        if line.startswith("# alpha"):
            alpha = float(line.split("=")[2].split(";")[0])
            L = int(line.split("L = ")[1].split(" ")[0])
        elif line.strip() and not line.startswith("#"):
            f = line.split()
            grp.append(int(f[1]))
            gains.append(float(f[2]))
            if len(f) > 3:
                ld.append(float(f[3]))
    return alpha, L, np.array(grp, dtype=np.int32), np.array(gains), (np.array(ld) if ld else None)


if __name__ == "__main__":
    for name in sys.argv[1:] or list(WORKLOADS):
        write(name)
