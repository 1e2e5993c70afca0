"""Readers for the small text fixtures in this folder (values printed in the paper)."""
import os
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))


def read_table(name):
    rows = {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = line.split()
            rows[key] = float(Fraction(val))
    return rows
