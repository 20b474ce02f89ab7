"""Stored values under tests/golden/ (CPU only).

paper_interaction_constants.txt holds the experimental parameters and the c0, c2
the paper prints for them (Supplementary Material, the realistic-parameter
paragraph; Eq. S.4).  The oracle's Eq. (S.4) must give the printed values when
rounded to the printed decimals: a dropped factor of 2, a swapped a0/a2 or a
sign slip in c2 moves at least one of the four past its rounding.

oracle_record_32.txt is a regression record of the oracle itself, written by
tests/golden/make_oracle_record.py from the oracle alone; it shows any change
of the oracle's arithmetic, which the pins then have to justify.
"""
import math
import os

import pytest

import oracle
from tests.golden import make_oracle_record as rec

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
BOHR_UM = 0.529177210903e-4  # Bohr radius in micrometres (CODATA 2018)


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


@pytest.mark.parametrize("row", _rows("paper_interaction_constants.txt"), ids=lambda r: r[0])
def test_printed_interaction_constants(row):
    _, n, l0, a0, a2, c0, c0d, c2, c2d = row
    got0, got2 = oracle.interaction_constants(float(n), float(a0) * BOHR_UM, float(a2) * BOHR_UM, float(l0))
    assert round(got0, int(c0d)) == float(c0)
    assert round(got2, int(c2d)) == float(c2)


def test_printed_constants_are_not_met_by_plausible_slips():
    """The fixture is sharp enough to catch the mistakes it is there for."""
    n, l0, a0, a2 = 1e5, 4.0, 101.8 * BOHR_UM, 100.4 * BOHR_UM
    pref = 2 * n * math.sqrt(2 * math.pi) / (3 * l0)
    assert round(pref * (a2 + 2 * a0)) != 669          # a0 and a2 swapped in c0
    assert round(pref * (a0 - a2), 1) != -3.1          # sign of c2
    assert round(pref * (a0 + 2 * a2) / 2) != 669      # factor 2 dropped
    assert round(pref * (a0 + 2 * a2) / math.sqrt(2)) != 669  # sqrt(2 pi) read as sqrt(pi)


def _record():
    cases, cur = {}, None
    with open(os.path.join(GOLDEN, "oracle_record_32.txt")) as f:
        for ln in f:
            t = ln.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "case":
                cur = cases.setdefault(t[1], dict(obs={}, psi=[]))
            elif t[0] == "obs":
                cur["obs"][t[1]] = float(t[2])
            else:
                cur["psi"].append((int(t[1]), int(t[2]), int(t[3]), complex(float(t[4]), float(t[5]))))
    return cases


RECORD = _record()


def test_record_covers_every_case():
    assert sorted(RECORD) == sorted(c[0] for c in rec.cases())


@pytest.mark.parametrize("case", rec.cases(), ids=lambda c: c[0])
def test_oracle_matches_its_record(case):
    name, p, form, mode, m = case
    want = RECORD[name]
    psi = rec.run(p, form, mode, m)
    ob = oracle.observables(p, psi)
    got = {"norm+1": ob["norm"][0], "norm0": ob["norm"][1], "norm-1": ob["norm"][2],
           "magnetization": ob["magnetization"], "energy": ob["energy"], "mu": ob["mu"]}
    for k, v in want["obs"].items():
        assert abs(got[k] - v) <= 1e-12 * max(1.0, abs(v)), (name, k, got[k], v)
    for c, j, i, z in want["psi"]:
        assert abs(psi[c, j, i] - z) <= 1e-12, (name, c, j, i, psi[c, j, i], z)
