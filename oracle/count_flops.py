"""Algorithmic FP64 work of one face flux (reconstruction + Riemann solver), averaged over faces of a
seeded workload, counted by the oracle's operation-counting scalar.

Usage: python oracle/count_flops.py [n] [samples]
Prints the mean add/sub, mul, div, sqrt, compare counts per face for (DC|PLM) x (HLLD|HLLE) on the
Orszag-Tang-style vortex (seed 2005); flops = add/sub + mul + div + sqrt (compares not counted).
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import orc  # noqa: E402
from paper_2005_06651_gb300 import inputs  # noqa: E402


def main(n=64, samples=4000):
    prob = inputs.orszag_tang(n=n, mb=n, seed=2005)
    m = orc.Mesh.from_problem(prob)
    w = m.get_prims()  # rho, vx, vy, vz, p, bcx, bcy, bcz
    _, b1, b2, b3 = m.get_cons()
    rng = np.random.default_rng(0)
    res = {}
    for recon, rname in ((orc.DC, "dc"), (orc.PLM, "plm")):
        for solver, sname in ((orc.HLLD, "hlld"), (orc.HLLE, "hlle")):
            acc = np.zeros(5)
            for _ in range(samples):
                d = int(rng.integers(0, 3))
                k, j, i = (int(x) for x in rng.integers(0, n, size=3))
                t1, t2 = (d + 1) % 3, (d + 2) % 3
                idx = [k, j, i]
                q = []
                for off in (-2, -1, 0, 1):
                    c = list(idx)
                    c[2 - d] = (c[2 - d] + off) % n
                    cw = w[:, c[0], c[1], c[2]]
                    q.append([cw[0], cw[1 + d], cw[1 + t1], cw[1 + t2], cw[4], cw[5 + t1], cw[5 + t2]])
                bn = (b1, b2, b3)[d][k, j, i]
                acc += orc.count_face_ops(recon, solver, np.array(q), bn, prob.gamma)
            acc /= samples
            res[rname + "_" + sname] = acc
            flops = acc[0] + acc[1] + acc[2] + acc[3]
            print("%s_%s: add %.1f mul %.1f div %.1f sqrt %.1f cmp %.1f -> flops/face %.1f"
                  % (rname, sname, *acc, flops))
    return res


if __name__ == "__main__":
    main(*(int(a) for a in sys.argv[1:]))
