"""Writes the fixtures in this folder. Run from the repository root:

    python tests/golden/make_golden.py

gl_nodes_closed_form.txt: Gauss-Legendre nodes on [0, 1] for N = 1..5 from
their closed forms (roots of the Legendre polynomial P_N on [-1, 1], mapped by
x -> (x + 1) / 2), evaluated here with mpmath at 40 digits. No library node
routine and no part of the oracle is used.

oracle_order1_seed11.txt / oracle_order2_seed12.txt: the oracle's outputs for
two small seeded cases, orders 1 and 2 (N = 2, 3; regression fixtures). Written by calling only the
oracle; any later change to its arithmetic that moves these values must cite,
in its commit message, the passage that justifies it.

oracle_curvilinear_order2_seed13.txt: the same for the oracle's curvilinear
STP (N = 3, per-node inverse Jacobians (I + 0.3 U)/h with U ~ U[-1,1]^(3x3)).
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def closed_form_nodes():
    import mpmath as mp
    mp.mp.dps = 40
    roots = {
        1: [mp.mpf(0)],
        2: [-1 / mp.sqrt(3), 1 / mp.sqrt(3)],
        3: [-mp.sqrt(mp.mpf(3) / 5), mp.mpf(0), mp.sqrt(mp.mpf(3) / 5)],
        4: sorted([s * mp.sqrt(mp.mpf(3) / 7 + t * mp.mpf(2) / 7 * mp.sqrt(mp.mpf(6) / 5))
                   for s in (-1, 1) for t in (-1, 1)]),
        5: sorted([mp.mpf(0)] + [s * mp.sqrt(5 + t * 2 * mp.sqrt(mp.mpf(10) / 7)) / 3
                                 for s in (-1, 1) for t in (-1, 1)]),
    }
    lines = ["# Gauss-Legendre nodes on [0,1]: (x + 1)/2 for the roots x of P_N on [-1,1].",
             "# Closed forms: N=2 +-1/sqrt(3); N=3 0, +-sqrt(3/5); N=4 +-sqrt(3/7 -+ 2/7 sqrt(6/5));",
             "# N=5 0, +-(1/3) sqrt(5 -+ 2 sqrt(10/7)). 40-digit mpmath, printed to 20 digits.",
             "# N  node_0 ... node_{N-1}"]
    for N, xs in roots.items():
        lines.append(f"{N} " + " ".join(mp.nstr((x + 1) / 2, 20) for x in xs))
    return "\n".join(lines) + "\n"


def oracle_case(N, seed):
    import oracle
    rng = np.random.default_rng(seed)
    E = 2
    params = np.stack([rng.uniform(2, 3, (E, N, N, N)), rng.uniform(4, 6, (E, N, N, N)),
                       rng.uniform(1, 2, (E, N, N, N))], axis=-1)
    q = rng.uniform(-1, 1, (E, N, N, N, 9))
    h, dt = 0.25, 0.005
    avg, faces = oracle.stp(q, params, h, dt)
    lines = [f"# oracle.stp on numpy default_rng({seed}): E={E}, N={N}; params = stack of "
             "U[2,3] (rho), U[4,6] (cp), U[1,2] (cs) per node, then q = U[-1,1]; h=0.25, dt=0.005.",
             "# Regression fixture written by tests/golden/make_golden.py (oracle only).",
             "# avg, then faces, flattened in C order, one value per line (17 significant digits)."]
    lines += [f"{v:.17g}" for v in avg.ravel()] + [f"{v:.17g}" for v in faces.ravel()]
    return "\n".join(lines) + "\n"


def oracle_curv_case(N, seed):
    import oracle
    rng = np.random.default_rng(seed)
    E = 2
    params = np.stack([rng.uniform(2, 3, (E, N, N, N)), rng.uniform(4, 6, (E, N, N, N)),
                       rng.uniform(1, 2, (E, N, N, N))], axis=-1)
    q = rng.uniform(-1, 1, (E, N, N, N, 9))
    h, dt = 0.25, 0.005
    metric = (np.eye(3) + 0.3 * rng.uniform(-1, 1, (E, N, N, N, 3, 3))) / h
    avg, faces = oracle.stp_curvilinear(q, params, metric, dt)
    lines = [f"# oracle.stp_curvilinear on numpy default_rng({seed}): E={E}, N={N}; params = stack "
             "of U[2,3] (rho), U[4,6] (cp), U[1,2] (cs) per node, then q = U[-1,1], then the "
             "metric (I + 0.3 U[-1,1]^(3x3)) / h per node; h=0.25, dt=0.005.",
             "# Regression fixture written by tests/golden/make_golden.py (oracle only).",
             "# avg, then faces, flattened in C order, one value per line (17 significant digits)."]
    lines += [f"{v:.17g}" for v in avg.ravel()] + [f"{v:.17g}" for v in faces.ravel()]
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    with open(os.path.join(HERE, "gl_nodes_closed_form.txt"), "w") as f:
        f.write(closed_form_nodes())
    for N, seed in ((2, 11), (3, 12)):
        with open(os.path.join(HERE, f"oracle_order{N - 1}_seed{seed}.txt"), "w") as f:
            f.write(oracle_case(N, seed))
    with open(os.path.join(HERE, "oracle_curvilinear_order2_seed13.txt"), "w") as f:
        f.write(oracle_curv_case(3, 13))
    print("written")
