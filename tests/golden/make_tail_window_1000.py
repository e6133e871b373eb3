"""Write tail_window_32x32x128_sigma8.txt: the FP64 oracle's state of the
attractive-tail workload's slit after 100 and 1000 steps.

The workload is the tail configuration of the benchmark (Sec. Conclusions,
attractive forces: a Lennard-Jones mean-field tail cut at 2.5 sigma added to
the hard-sphere force of Eq. LBHS; sigma = 8, tau = 0.8, F_e = 1e-6 along x,
seeded 1e-3 noise, bounce-back walls in z), at eta = 0.25 and eps = 0.3: the
packing fraction and tail strength at which the explicit scheme stays stable
(eta = 0.40 diverges at sigma = 8, and eps = 1 at kT = 1/3 puts the fluid
inside its spinodal). The lateral extent is 32 x 32 (the steady state is
uniform in x and y; 32 x 32 and 64 x 64 slits give the same profiles) so that
the oracle's direct tail sum finishes in about an hour and a half on 8 cores.

Only the oracle runs here. Output: for each of the two times, the plane
averages n(z), u_x(z) (FP64), the totals (mass, momentum x, y, z) and the
fields n, u_x, u_y, u_z on four columns (x, y) of the grid, each value with
17 significant digits.

    python tests/golden/make_tail_window_1000.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

SHAPE = (32, 32, 128)  # nx, ny, nz
SIGMA, ETA, TAU = 8, 0.25, 0.8
BODY = (1e-6, 0.0, 0.0)
EPS, RCUT, SEED = 0.3, 2.5, 1
TIMES = (100, 1000)
COLUMNS = ((0, 0), (17, 9), (31, 31), (8, 24))
OUT = os.path.join(HERE, "tail_window_32x32x128_sigma8.txt")


def fmt(a):
    return " ".join(repr(float(v)) for v in np.ravel(a))


def main():
    oracle.build()
    nx, ny, nz = SHAPE
    o = oracle.Oracle(nx, ny, nz, SIGMA, ETA, TAU, body=BODY, seed=SEED, tail=True, eps=EPS, rcut=RCUT)
    lines = [
        "# FP64 oracle, tail workload slit (Sec. Conclusions, attractive forces; Eq. LBHS)",
        f"# shape {nx} {ny} {nz} sigma {SIGMA} eta {ETA} tau {TAU} body {BODY[0]} {BODY[1]} {BODY[2]}",
        f"# tail eps {EPS} rcut {RCUT} seed {SEED} threads {oracle.threads()}",
        f"n0 {repr(float(o.n0))}",
        "columns " + " ".join(f"{x},{y}" for x, y in COLUMNS),
    ]
    t = 0
    t0 = time.time()
    for T in TIMES:
        o.step(T - t)
        t = T
        n_z, ux_z = o.profiles()
        tot = o.totals()
        n, u = o.moments()
        lines.append(f"time {T}")
        lines.append("n_z " + fmt(n_z))
        lines.append("ux_z " + fmt(ux_z))
        lines.append("totals " + fmt(tot))
        for x, y in COLUMNS:
            lines.append(f"col {x},{y} n " + fmt(n[:, y, x]))
            for a, name in enumerate(("ux", "uy", "uz")):
                lines.append(f"col {x},{y} {name} " + fmt(u[a, :, y, x]))
        print(f"step {T}: {time.time() - t0:.0f} s", flush=True)
    o.close()
    with open(OUT + ".tmp", "w") as f:
        f.write("\n".join(lines) + "\n")
    os.replace(OUT + ".tmp", OUT)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
