"""Reader of the worked-example values printed in the paper (plain text)."""
import os


def paper_values():
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "paper_worked_examples.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v, _unit = line.split()
                out[k] = float(v)
    return out
