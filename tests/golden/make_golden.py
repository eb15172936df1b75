"""Writes the stored expected values under tests/golden/ from the CPU oracle only.

Run from the repository root:  python tests/golden/make_golden.py
The paper prints no worked numeric example, so these fixtures are regression
values of the oracle on seeded synthetic inputs (the oracle itself is pinned by
tests/test_oracle_pins.py).  Nothing here calls the CUDA library.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import feedergen as fg            # noqa: E402
from oracle import oracle as O    # noqa: E402


def main():
    f, run = fg.preset("feeder40")
    vhat, ihat = O.operating_points(f)
    res = O.reduce(f, vhat, ihat, margin=run["margin"], max_merges=f.n_bus, mode="literal")
    path = os.path.join(HERE, "feeder40_decisions.txt")
    with open(path, "w") as fh:
        fh.write("# Algorithm 1 (Sec. IV) on the seeded 40-bus feeder (feedergen preset feeder40),\n")
        fh.write("# margin 0.005 p.u., SMICE objective, tie band 1e-9, literal mode of the CPU oracle.\n")
        fh.write(f"# stop_reason {res['stop_reason']} (1 = no feasible candidate)\n")
        fh.write("# iteration s r smice max_error\n")
        for t in range(res["n_iter"]):
            fh.write(f"{t} {res['s'][t]} {res['r'][t]} {res['score'][t]:.17e} {res['maxerr'][t]:.17e}\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
