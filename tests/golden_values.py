"""Reader for tests/golden/*.txt fixtures (values printed in the paper)."""
import os

_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name: str, fname: str = "paper_values.txt") -> float:
    with open(os.path.join(_DIR, fname)) as f:
        for line in f:
            s = line.split("#", 1)[0].split()
            if len(s) >= 2 and s[0] == name:
                return float(s[1])
    raise KeyError(name)
