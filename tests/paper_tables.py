"""Readers of the text fixtures under tests/golden/ (values printed in the paper).

Each fixture names the table it transcribes; the tests use them as pins and
never compute them.
"""
from __future__ import annotations

from pathlib import Path

import numpy as np

GOLDEN_DIR = Path(__file__).resolve().parent / "golden"


def read_table(path: Path) -> dict[str, np.ndarray]:
    out = {}
    for line in path.read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, vals = line.split(":", 1)
        out[name.strip()] = np.array([int(x) for x in vals.split()], dtype=np.int64)
    return out


def table(number: int) -> dict[str, np.ndarray]:
    """Arrays of Table 1 (variable-sorted) or Table 2 (check-sorted), (14,7) code."""
    return read_table(GOLDEN_DIR / f"table{number}_code_14_7.txt")
