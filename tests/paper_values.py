"""Values the paper prints, read from tests/golden/paper_values.txt (each line:
key, value, and the passage it comes from)."""
import os

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def paper_value(key):
    for line in open(GOLD):
        line = line.split("#")[0].split()
        if line and line[0] == key:
            return float(line[1])
    raise KeyError(key)
