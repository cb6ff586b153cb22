"""Small helpers shared by the tests (no arithmetic of the method lives here)."""
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def read_golden(name):
    """Rows of a whitespace-separated fixture under tests/golden/, comments stripped."""
    path = os.path.join(ROOT, "tests", "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows
