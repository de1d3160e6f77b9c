"""Algorithmic work of one hydro_step launch per sub-grid, from the oracle's
operation counts (test infrastructure; run ``python -m oracle.count_work``).

The oracle evaluates the PPM line of a (cell, direction) pair every time a
face point needs it; the method needs each line once per cell (13 lines per
interior cell, 9 per face-adjacent ghost cell, all 10 fields).  The
algorithmic count therefore replaces the oracle's PPM operations by their
average per evaluation times the number of unique evaluations.  Every
+, -, x, /, sqrt, pow, compare and min/max counts as one FP64 operation.

Bytes per sub-grid stage: the ghost-padded state read once (F x 14^3 x 8 B)
and dU/dt written once (F x 8^3 x 8 B), plus amax, origin and h.
"""
import json
import sys

import numpy as np

from . import core

N, G, F = 8, 3, 10
S = N + 2 * G
UNIQUE_LINES = N ** 3 * 13 + 6 * N * N * 9


def work(seed: int = 0) -> dict:
    from paper_2107_10987_gb300 import workloads as W
    U = W.random_subgrids(1, seed)[0]
    c = core.count_ops(core.OracleParams(), U, np.zeros(3), 0.1)
    st = c["step"]
    total = sum(v for k, v in st.items() if k != "sgn")
    per_call = c["ppm_ops"] / c["ppm_calls"]
    algo = total - c["ppm_ops"] + per_call * UNIQUE_LINES * F
    up = sum(v for k, v in c["update"].items() if k != "sgn")
    return {
        "fp64_flops_per_subgrid_stage": float(round(algo)),
        "fp64_flops_per_cell_stage": float(algo / N ** 3),
        "oracle_ops_per_subgrid_stage": int(total),
        "ppm_ops_per_line_field": float(per_call),
        "unique_line_field_evaluations": UNIQUE_LINES * F,
        "update_flops_per_subgrid": int(up),
        "bytes_per_subgrid_stage": F * S ** 3 * 8 + F * N ** 3 * 8 + 8 + 32,
    }


if __name__ == "__main__":
    json.dump(work(), sys.stdout, indent=1)
    print()
