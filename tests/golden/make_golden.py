"""Writes oracle_regression.txt: digests of the oracle's orderings on fixed seeded inputs.

Calls only the oracle and the input generators. Run from the repository root:
    python tests/golden/make_golden.py
"""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from paper_1610_08128_gb300 import synth  # noqa: E402

CASES = {
    "grid64x64": lambda: synth.c1_grid2d(),
    "grid12x17": lambda: synth.grid((12, 17), seed=4),
    "grid9x10x11": lambda: synth.grid((9, 10, 11), seed=5),
    "mesh3000": lambda: synth.c3_mesh(3000),
    "mesh3000raw": lambda: synth.c3_mesh(3000, stitch=False),
    "random500": lambda: synth.random_graph(500, 600, 6),
    "tree300": lambda: synth.random_tree(300, 7),
}


def main():
    import oracle

    lines = ["# Oracle regression digests: case name, sha256[:16] of perm (little-endian int32),",
             "# bandwidth, profile. Written by tests/golden/make_golden.py from the oracle only."]
    for name, make in CASES.items():
        g = make()
        p = oracle.rcm(g.n, g.rowptr, g.colidx)
        bw, prof = oracle.bandwidth_profile(g.n, g.rowptr, g.colidx, p)
        d = hashlib.sha256(p.astype("<i4").tobytes()).hexdigest()[:16]
        lines.append(f"case: {name} {d} {bw} {prof}")
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
