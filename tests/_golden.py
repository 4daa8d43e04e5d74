"""Readers for the text fixtures under tests/golden/."""
import os
from fractions import Fraction

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            yield line.split()


def table1():
    """{group: (first_state, last_state, Fraction weight)} and theta."""
    groups, theta = {}, None
    for row in _rows("table1_d2q21.txt"):
        if row[0] == "theta":
            theta = Fraction(row[2])
            continue
        a, _, b = row[1].partition("-")
        groups[row[0]] = (int(a), int(b or a), Fraction(row[2]))
    return groups, theta


def paper_values():
    out = {}
    for row in _rows("paper_values.txt"):
        out[row[0]] = (float(row[1]), float(row[2]))
    return out
