"""Writes c_consumer_oracle.txt: the FP64 oracle's fields of a small
lid-driven cavity (24 x 12 nodes, r = 0.5, gamma = 0.25, nu = 0.01,
u_lid = 0.03, from rest, 300 steps of arXiv:2208.03562's scheme), which the
plain C program of tests/test_c_consumer.py compares with what it gets
through the C ABI.  Calls only the oracle.

Format: a line "nx ny steps", then one line "rho u_x u_y" per node, rows of
x fastest, y from the bottom wall.

  python tests/golden/make_c_consumer_oracle.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c_consumer_oracle.txt")
NX, NY, R, GAMMA, NU, U, STEPS = 24, 12, 0.5, 0.25, 0.01, 0.03, 300


def main():
    from oracle import stepper as S
    o = S.Oracle(S.OracleParams(nx=NX, ny=NY, r=R, gamma=GAMMA, nu=NU, u_lid=U))
    o.step(STEPS)
    rho, ux, uy = o.fields()
    with open(OUT, "w") as fh:
        fh.write("%d %d %d\n" % (NX, NY, STEPS))
        for y in range(NY):
            for x in range(NX):
                fh.write("%.17g %.17g %.17g\n" % (rho[y, x], ux[y, x], uy[y, x]))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
