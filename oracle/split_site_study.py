"""Cost of the hybrid split-site + low-order Taylor scheme on the perovskite 64^3 workload.

TEST INFRASTRUCTURE (a study run on the CPU, it calls only oracle/ and synthetic/).

Section III C offers two ways to handle displacements: split sites (a discrete set of displaced
positions becomes extra sites whose occupancies are transformed exactly, the mapping of displacive
onto occupational disorder) and the Taylor expansion of exp(iQ.u), whose remainder after order P
is bounded by x^(P+1)/(P+1)! with x = max |Q.u|.  The hybrid quantises each Cartesian component of
u to a grid of step s: u = u_q + d with |d_a| <= s/2; every distinct u_q of a site is a split site
(its occupancy field: the atoms that round to it), and only the residual exp(iQ.d) is expanded,
at the order p that the same bound needs for x_res = max |Q.d| over the atoms and the corners of the
requested grid.  Each split site then needs T(p) = (p+1)(p+2)(p+3)/6 monomial transforms of its
residuals, so the transforms per site are (occupied centres) x T(p), against T(P) for the single
expansion.  This script measures both on the workload (perovskite 64^3, u 0.08 A rms, |h,k,l| <= 8,
eps = 1e-5) and writes the table to split_site_study.txt beside it.

    python -m oracle.split_site_study
"""
from __future__ import annotations

import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import synthetic as syn  # noqa: E402
from oracle import core  # noqa: E402


def n_terms(p: int) -> int:
    return (p + 1) * (p + 2) * (p + 3) // 6


def corners_q(model):
    q = model.qgrid
    cs = []
    for i in (0, q.count[0] - 1):
        for j in (0, q.count[1] - 1):
            for l in (0, q.count[2] - 1):
                cs.append([q.h0[0] + i * q.step[0], q.h0[1] + j * q.step[1], q.h0[2] + l * q.step[2]])
    return core.q_cart(np.array(cs), model.lattice)


def study(eps=1e-5, steps=(0.01, 0.02, 0.04, 0.08, 0.16, 0.32)):
    m = syn.perovskite_correlated()
    Qc = corners_q(m)                                   # [8, 3] Cartesian
    u = m.disp.reshape(m.nsite, -1, 3).astype(np.float64)   # [site, atoms, 3]
    x_full = core.x_max(m, m.qgrid)
    P = core.taylor_order(x_full, eps)
    rows = [("single expansion", None, 1, 1.0, x_full, P, n_terms(P), n_terms(P))]
    for s in steps:
        uq = np.rint(u / s) * s
        d = u - uq
        x_res = float(np.max(np.abs(d.reshape(-1, 3) @ Qc.T)))
        p = core.taylor_order(x_res, eps)
        centres = [len(np.unique(np.rint(u[mu] / s).astype(np.int64), axis=0)) for mu in range(m.nsite)]
        fields = max(centres) * n_terms(p)
        rows.append(("hybrid", s, max(centres), float(np.mean(centres)), x_res, p, n_terms(p), fields))
    return m, x_full, P, rows


def main():
    m, x_full, P, rows = study()
    lines = ["Hybrid split-site + Taylor on the perovskite 64^3 workload (1,310,720 atoms, u 0.08 A rms per",
             "component, |h,k,l| <= 8, eps = 1e-5): transforms per site, largest site",
             "",
             "%-17s %8s %9s %9s %8s %4s %6s %14s" % ("scheme", "step A", "centres", "mean", "x", "p", "T(p)",
                                                  "transforms"),
             ]
    for name, s, cmax, cmean, x, p, tp, fields in rows:
        lines.append("%-17s %8s %9d %9.1f %8.3f %4d %6d %14d" % (name, "-" if s is None else "%.2f" % s, cmax,
                                                                  cmean, x, p, tp, fields))
    best = min(rows[1:], key=lambda r: r[7])
    lines += ["",
              "single expansion: P = %d, T(P) = %d transforms per site; best hybrid: step %.2f A, %d centres x "
              "T(%d) = %d (%.1fx the single expansion)" % (P, n_terms(P), best[1], best[2], best[5], best[7],
                                                             best[7] / n_terms(P))]
    text = "\n".join(lines) + "\n"
    with open(os.path.join(HERE, "split_site_study.txt"), "w") as f:
        f.write(text)
    print(text)


if __name__ == "__main__":
    main()
