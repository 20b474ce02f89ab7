"""Write oracle_record_32.txt: observables and sampled values of the FP64 oracle
after a few steps of each step form on seeded 32x32 inputs.

This is a regression record of the oracle, not a pin: the pins that tie the
oracle to the paper and to mathematics are in tests/test_oracle_pins.py and
tests/test_oracle_strang.py.  The record makes any later change to the oracle's
arithmetic visible; a change that moves it must be justified by the passage of
the paper (or the reading of it) that calls for it, and the record rewritten by
running this script:

    python tests/golden/make_oracle_record.py

It calls only the oracle and the seeded input generators.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


import oracle  # noqa: E402
from paper_2105_10517_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "oracle_record_32.txt")
NSTEPS = 12
# Grid points sampled from each component: corner, ragged interior, near centre.
SAMPLES = ((0, 0), (5, 27), (13, 9), (16, 16), (31, 30))


def cases():
    """(name, parameters, step form, mode, constrained magnetisation or None)."""
    base = dict(nx=32, ny=32, xlen=12.0, ylen=12.0, dt=0.004, wx=1.0, wy=1.2, c0=40.0, c2=-3.0,
                omeg=0.5, so_type=1, gamma=0.6, rabi=0.3)
    out = []
    for so_type, name in ((0, "none"), (1, "rashba"), (2, "dresselhaus")):
        for mode, mname in ((oracle.IMAG, "imag"), (oracle.REAL, "real")):
            out.append((f"lie_{name}_{mname}", dict(base, so_type=so_type), "lie", mode, None))
    out.append(("lie_rashba_antiferro_real", dict(base, c0=60.0, c2=5.0, omeg=-0.4), "lie", oracle.REAL, None))
    out.append(("strang_rashba_imag", base, "strang", oracle.IMAG, None))
    out.append(("strang_dresselhaus_real", dict(base, so_type=2), "strang", oracle.REAL, None))
    out.append(("constrained_m0.2_imag", dict(base, so_type=0, gamma=0.0, rabi=0.0), "m", oracle.IMAG, 0.2))
    return out


def initial(p):
    return inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=11, phase_noise=0.05)


def run(p, form, mode, m):
    psi = initial(p)
    if form == "lie":
        return oracle.propagate(p, psi, NSTEPS, mode)
    if form == "strang":
        return oracle.propagate_strang(p, psi, NSTEPS, mode)
    return oracle.propagate_m(p, psi, NSTEPS, m)


def record(name, p, form, mode, m):
    """Lines of one case: its observables, then the sampled psi values."""
    psi = run(p, form, mode, m)
    ob = oracle.observables(p, psi)
    lines = [f"case {name}"]
    for k, v in (("norm+1", ob["norm"][0]), ("norm0", ob["norm"][1]), ("norm-1", ob["norm"][2]),
                 ("magnetization", ob["magnetization"]), ("energy", ob["energy"]), ("mu", ob["mu"])):
        lines.append(f"obs {k} {float(v):.17e}")
    for c in range(3):
        for (j, i) in SAMPLES:
            z = psi[c, j, i]
            lines.append(f"psi {c} {j} {i} {z.real:.17e} {z.imag:.17e}")
    return lines


def main():
    oracle.build()
    lines = ["# Regression record of the FP64 oracle, written by make_oracle_record.py.",
             f"# {NSTEPS} steps per case on 32x32 seeded Gaussian inputs (seed 11, phase noise 0.05)."]
    for c in cases():
        lines += record(*c)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"wrote {OUT}: {len(cases())} cases")


if __name__ == "__main__":
    main()
