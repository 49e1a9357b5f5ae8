"""Reader of the stored oracle results in this folder (no arithmetic of the method).

``read_golden_blocks`` parses the files written by ``make_ceff_configs.py``.
"""
import numpy as np


def read_golden_blocks(path):
    """Parse a file written by make_ceff_configs.py: {block name: {"iterations_to_1e-6": [...],
    "iterations_to_1e-11": [...], "ceff_converged": array, "ceff_at_1e-6": array}}."""
    blocks, cur, key = {}, None, None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = blocks.setdefault(line[1:-1], {})
            key = None
            continue
        head = line.split()[0]
        if head.startswith("iterations"):
            cur[head] = [int(v) for v in line.split()[1:]]
        elif head.startswith("ceff"):
            key = head
            cur[key] = []
        else:
            cur[key].append([float(v) for v in line.split()])
    for b in blocks.values():
        for k in ("ceff_converged", "ceff_at_1e-6"):
            b[k] = np.array(b[k])
    return blocks
