"""Writes tests/golden/tiny_frame_cells.json from the FP64 oracle alone.

The fixture is a regression guard for the oracle (it calls nothing but ``oracle/`` and
the seeded scene generator).  Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle  # noqa: E402
from paper_2602_01035_gb300 import scenes as S  # noqa: E402

RIG = {"n": 3, "width": 24, "height": 18, "spread_deg": 25.0}
SEED = 21
PARAMS = {"n_min": 4, "max_level": 3, "sigma_m": 0.03}


def main():
    rig = S.tiny_rig(**RIG)
    fr = S.random_frame(rig, seed=SEED)
    res = oracle.fuse_frame(rig, fr, PARAMS)
    c = res["cells"]
    out = {
        "_source": "oracle/fuseflow_oracle.c via tests/golden/make_golden.py",
        "rig": RIG, "seed": SEED, "params": PARAMS,
        "key": [str(int(k)) for k in c["key"]],
        "count": [int(v) for v in c["count"]],
        "rep": [int(v) for v in c["rep"]],
        "weight": [float(v) for v in c["weight"]],
        "pos": [[float(x) for x in row] for row in c["pos"]],
        "stats": {k: res["stats"][k] for k in ("n_valid", "n_gated", "n_cells")},
    }
    with open(os.path.join(HERE, "tiny_frame_cells.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("cells", len(out["key"]))


if __name__ == "__main__":
    main()
