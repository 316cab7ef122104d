"""Reader for the textbook lattice constants in lattice_constants.txt."""
import os

_HERE = os.path.dirname(os.path.abspath(__file__))


def load():
    out = {}
    with open(os.path.join(_HERE, "lattice_constants.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()[:2]
            out[k] = float(v)
    return out
