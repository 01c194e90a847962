"""Write oracle J/K rows for sampled shells of a full-size synthetic cell.

Calls only the oracle (oracle/) and the seeded input generator
(synthcells/).  The stored rows are the expected values of the full-size
parity tests (sampled outputs the oracle can compute one by one).

usage: python tests/golden/make_rows.py water|diamond|diamond1 [shell ... | all]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synthcells as sc  # noqa: E402
from oracle import oracle as O  # noqa: E402

CELLS = {"water": lambda: sc.config(2), "diamond": lambda: sc.config(3),
         # one conventional diamond cell (8 atoms, 88 bf) with the s(6) s(3) p(1) d(1) basis
         "diamond1": lambda: sc.diamond_cell(1)}


def main():
    name = sys.argv[1]
    cell = CELLS[name]()
    if sys.argv[2:] == ["all"]:
        shells, tag = list(range(len(cell.shells))), "all"
    else:
        shells = [int(x) for x in sys.argv[2:]] or [0]
        tag = "_".join(map(str, shells))
    t = time.time()
    D = O.density(cell)
    J, K = O.jk_rows(cell, D, shells)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "%s_rows_%s.npz" % (name, tag))
    np.savez_compressed(out, shells=np.array(shells), rows=O.row_indices(cell, shells), J=J, K=K,
                        seconds=time.time() - t, threads=O.num_threads())
    print(out, "%.1f s" % (time.time() - t))


if __name__ == "__main__":
    main()
