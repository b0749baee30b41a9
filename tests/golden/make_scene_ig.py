"""Write scene_seed0_ig.txt: the oracle's information gains on the full-size
scene workload (seed 0: 100,000 Gaussians in 16 blobs + 20,000 on the
table, K = 16, SH degree 3, 640x480 views at f = 525, the 4 training views),
for a sample of the 64 candidates, plus per-Gaussian gains of one candidate
for a sample of Gaussians.

The whole workload is far beyond what the oracle can redo inside a GPU test
(about 7 minutes on 8 cores for 4 training views and 3 candidates), so its
values are stored here. Only the seeded generator and the oracle are used.

    python tests/golden/make_scene_ig.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import nbv_synth as S            # noqa: E402
from oracle import oracle as O   # noqa: E402

CANDIDATES = (0, 37, 63)
DELTA_CAND = 1                   # index into CANDIDATES
N_DELTA = 256


def main():
    wl = S.make_workload("scene", seed=0)
    o = O.OracleScene(wl.scene)
    cand = wl.cand.subset(list(CANDIDATES))
    res = o.score(wl.train, cand, delta_view=DELTA_CAND)
    delta = res["delta"]
    live = np.nonzero((delta > 0).all(1))[0]
    pick = np.sort(np.random.default_rng(0).choice(live, size=min(N_DELTA, live.size), replace=False))
    out = os.path.join(HERE, "scene_seed0_ig.txt")
    with open(out, "w") as f:
        f.write("# Oracle information gains (Eqs. 5-11) on the scene workload, seed 0, written by\n")
        f.write("# make_scene_ig.py in this folder (seeded generator + oracle only).\n")
        f.write("# train <t> IG_rgb IG_d IG_o          (training view t as a candidate, Eq. 10 normaliser)\n")
        f.write("# cand <v> IG_rgb IG_d IG_o score     (v = candidate index in the 64-view set)\n")
        f.write(f"# delta <g> d_rgb d_d d_o             (per-Gaussian gains of candidate {CANDIDATES[DELTA_CAND]})\n")
        for t in range(wl.train.n):
            f.write("train %d %s\n" % (t, " ".join(repr(float(x)) for x in res["ig_train"][t])))
        for i, v in enumerate(CANDIDATES):
            vals = list(res["ig_cand"][i]) + [res["score"][i]]
            f.write("cand %d %s\n" % (v, " ".join(repr(float(x)) for x in vals)))
        for g in pick:
            f.write("delta %d %s\n" % (g, " ".join(repr(float(x)) for x in delta[g])))
    print("wrote", out)


if __name__ == "__main__":
    main()
