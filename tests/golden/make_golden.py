"""Writes tests/golden/full_grid_c0.json.

Calls only the oracle (oracle/) and the seeded input generator: the stored
energies are the brute-force periodic exchange (Eq. pbcexchange) of the toy
cubic cell on small grids, every grid point an interpolation point.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import setup_oracle as S  # noqa: E402
from paper_2304_05505_gb300 import cells  # noqa: E402

CASES = [((2, 2, 2), (10, 10, 10)), ((3, 3, 3), (8, 8, 8)), ((3, 2, 4), (8, 8, 8))]


def main():
    out = {"source": "brute-force exchange of the toy cubic cell (oracle/setup_oracle.py); "
                     "arXiv 2304.05505 Eq. pbcexchange, closed-shell exchange per cell",
           "cases": []}
    for mesh, grid in CASES:
        c = cells.make_cell("C0", mesh=mesh, grid=grid)
        pts = cells.grid_points(c, 1)
        Xg = cells.bloch_collocation(c, pts, cells.kmesh_frac(c.mesh))
        C = cells.occupied_coefficients(c)
        bf = S.brute_force_exchange(c.lattice, c.grid, c.mesh, Xg, C)
        out["cases"].append({"mesh": list(mesh), "grid": list(grid), "seed": c.seed,
                             "Ex_bruteforce": bf["Ex"]})
    with open(os.path.join(HERE, "full_grid_c0.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
