"""Write fig4_sweep_4x4x4x4.txt: the storage-type sweep of Fig. 4 (Sec. 2)
and the precision ladder proposed after it, run by the FP64 oracle on a
synthetic 4^4 lattice (the paper's 4^4 matrix from an HMC trajectory is not
available): weak-field SU(3) links (eps = 0.3, seed 1), kappa = 0.13,
c_sw = 1, antiperiodic time boundary, a Gaussian even-site source (seed 34),
A = Dhat^dag Dhat, res = 1e-12, at most 3000 regular steps.

Calls only the oracle (and the seeded input generator).  Run from the
repository root:  python tests/golden/make_fig4_sweep.py
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))

from oracle import dirac, solvers  # noqa: E402
from paper_2202_07388_gb300 import synth  # noqa: E402

DIMS = (4, 4, 4, 4)
RES, NMX = 1e-12, 3000

RUNS = [
    ("fp64", dict(store="fp64")),
    ("fp32", dict(store="fp32")),
    ("tf32", dict(store="tf32")),
    ("bf16", dict(store="bf16")),
    ("fp16", dict(store="fp16")),
    ("fp16_unscaled", dict(store="fp16", scaled=False)),
    ("ladder_fp16_fp32_fp64", dict(ladder=solvers.precision_ladder(("fp16", "fp32", "fp64")))),
    ("ladder_fp16_fp32", dict(ladder=solvers.precision_ladder(("fp16", "fp32")))),
    ("ladder_bf16_fp32_fp64", dict(ladder=solvers.precision_ladder(("bf16", "fp32", "fp64")))),
]


def case():
    u = synth.make_gauge(DIMS, 0.3, 1)
    a = dirac.clover_field(u, dirac.kappa_to_m0(0.13), 1.0)
    ainv = np.linalg.inv(a)
    eta = dirac.even_part(synth.make_source(DIMS, 34))
    return (lambda v: dirac.dw_hat_dagger(u, a, ainv, dirac.dw_hat(u, a, ainv, v))), eta


def main():
    apply_a, eta = case()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fig4_sweep_4x4x4x4.txt")
    lines = [
        "# CGNE storage-type sweep (Fig. 4 analog) and precision ladders, FP64 oracle,",
        "# written by make_fig4_sweep.py (synthetic 4^4 case described there).",
        "# columns: run  status  resets  first_reset  converged  rel_res  phases",
    ]
    for name, kw in RUNS:
        r = solvers.cgne(apply_a, eta, RES, NMX, ncomp=eta.size // 2,  # even-site components
                          **kw)
        lines.append(f"{name:24s} {r.status:5d} {r.resets:3d} {r.reset_at[0]:5d} {int(r.converged)} "
                     f"{r.rel_res:.3e} {','.join(r.phases)}")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
