"""Write the stored expected values under tests/golden/ from the oracle only.

base_matrices.json: the seeded BG-shaped base matrices of the workloads
(BG1-shaped Z=384 seed 1; BG2-shaped Z=8 and Z=64 seed 2), as the oracle's
orc_base_matrix builds them. Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    codes = []
    for name, bg, Z, seed in [("bg1_z384", 1, 384, 1), ("bg2_z8", 2, 8, 2), ("bg2_z64", 2, 64, 2)]:
        S, kb = oracle.base_matrix(bg, Z, seed)
        codes.append(dict(name=name, bg=bg, Z=Z, seed=seed, kb=kb, S=S.tolist()))
    with open(os.path.join(HERE, "base_matrices.json"), "w") as f:
        json.dump({"source": "oracle.base_matrix (seeded BG-shaped rule)", "codes": codes}, f, separators=(",", ":"))


if __name__ == "__main__":
    main()
