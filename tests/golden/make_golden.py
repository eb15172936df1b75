"""Writes the stored expected values under tests/golden/ from the CPU oracle only.

Run from the repository root:  python tests/golden/make_golden.py [--large]
The paper prints no worked numeric example, so these fixtures are regression
values of the oracle on seeded synthetic inputs (the oracle itself is pinned by
tests/test_oracle_pins.py).  Nothing here calls the CUDA library.

--large also writes the full decision sequences of the 2,200- and 3,100-bus
stand-ins of the paper's 5,991- and 8,381-node feeders (Table 2) in delta
mode: a few minutes on eight cores.  --batch writes those of the largest
feeder of each target (50, 70, 90 %) of the 256-feeder batch
(feedergen.batch_presets(256)).  Each of those files records the
fingerprint of the feeder it was made from (feedergen.fingerprint), so a
reader on another machine can tell whether its feeder is the same one.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import feedergen as fg            # noqa: E402
from oracle import oracle as O    # noqa: E402

LARGE = ("feeder2200", "feeder3100")
# the largest feeder of each target in feedergen.batch_presets(256): (index, target)
BATCH_LARGEST = ((4, 0.9), (80, 0.7), (110, 0.5))


def write_feeder40():
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


def write_large(name, f=None, run=None):
    if f is None:
        f, run = fg.preset(name)
    vhat, ihat = O.operating_points(f)
    merges = O.max_merges_for(f.n_bus, run["target"])
    res = O.reduce(f, vhat, ihat, margin=run["margin"], max_merges=merges)
    path = os.path.join(HERE, f"{name}_decisions.txt")
    with open(path, "w") as fh:
        fh.write(f"# Algorithm 1 (Sec. IV) on the seeded {f.n_bus}-bus feeder ({name}), "
                 f"margin {run['margin']} p.u.,\n")
        fh.write(f"# target {run['target']} ({merges} merges), SMICE objective, tie band 1e-9, "
                 "delta mode of the CPU oracle.\n")
        fh.write(f"# fingerprint {fg.fingerprint(f)}\n")
        fh.write(f"# n_iter {res['n_iter']} stop_reason {res['stop_reason']} candidates {res['candidates']}\n")
        fh.write("# iteration s r smice max_error gap ncand\n")
        for t in range(res["n_iter"]):
            fh.write(f"{t} {res['s'][t]} {res['r'][t]} {res['score'][t]:.17e} {res['maxerr'][t]:.17e} "
                     f"{res['gap'][t]:.17e} {res['ncand'][t]}\n")
    print("wrote", path)


def main():
    write_feeder40()
    if "--large" in sys.argv:
        for name in LARGE:
            write_large(name)
    if "--batch" in sys.argv:
        batch = fg.batch_presets(256)
        for k, target in BATCH_LARGEST:
            f, run = batch[k]
            assert run["target"] == target
            write_large(f"batch256_{k}", f, run)


if __name__ == "__main__":
    main()
