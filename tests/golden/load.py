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


def philox_kat():
    """(counter[4], key[2], output[4]) rows of philox4x32_10_kat.txt."""
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                w = [int(x, 16) for x in line]
                rows.append((w[0:4], w[4:6], w[6:10]))
    return rows
