"""Writes lshape96_4lvl_oracle.txt: the FP64 oracle's solution of the
precision-study workload (96^3 L-shaped domain, four levels, 2048 subdomains,
k spanning 1e-2 .. 1e2; parameter request 0; right-preconditioned FGMRES(30)
to rtol 1e-10), sampled at 1024 seeded positions, with its iteration count
and norms.  Calls only oracle/ and synthetic/ (about three minutes on eight
cores):

    python tests/golden/make_lshape96.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as orc  # noqa: E402
import synthetic as syn  # noqa: E402

NAME = "lshape96_4lvl"


def main():
    levels, w = syn.workload(NAME)
    o = orc.Oracle(levels, delta=w["delta"], nu_pre=w["nu"], nu_post=w["nu"], coef=w["coef"],
                   wave=syn.wave_vectors(), scale=w["scale"], load=w["load"])
    o.assemble(syn.mu_draw(0))
    o.factor()
    x, st = o.fgmres(rtol=w["rtol"], restart=w["restart"])
    b = o.get("b")
    idx = np.sort(np.random.default_rng(96).choice(x.size, 1024, replace=False))
    with open(os.path.join(HERE, NAME + "_oracle.txt"), "w") as fh:
        fh.write(f"# FP64 oracle solution of workload {NAME}, parameter request 0, rtol {w['rtol']}\n")
        fh.write("# written by tests/golden/make_lshape96.py (oracle/ only)\n")
        fh.write(f"n {x.size}\niterations {st['iters']}\nrel_residual {st['relres']:.17e}\n")
        fh.write(f"norm2_x {np.linalg.norm(x):.17e}\nnorm2_b {np.linalg.norm(b):.17e}\n")
        fh.write(f"samples {idx.size}\n")
        for i in idx:
            fh.write(f"{i} {x[i]:.17e}\n")


if __name__ == "__main__":
    main()
