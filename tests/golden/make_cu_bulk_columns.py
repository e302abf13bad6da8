"""Write tests/golden/cu_bulk_columns.json with the CPU oracle only.

Seeded sample of (E, k, column) items of the bulk fcc Cu [001] workload (20x20x480,
order 12, 64-plane CAPs, 8x8 Monkhorst-Pack mesh, 256 energies in E_F +- 0.3 Ha):
for each item the oracle's transpose BiCG (complex128, relative residual 1e-12)
gives t_j at (E, k) and, from the shadow system, at (E, -k), plus the iteration at
which the residual first reached 1e-10.  Items are solved in separate processes
(spawned, 8 at a time).  Takes tens of minutes on 8 cores.

    python tests/golden/make_cu_bulk_columns.py
"""

import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

SEED = 2100
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cu_bulk_columns.json")


def sample():
    import numpy as np

    from workloads import cu_bulk

    inst = cu_bulk()
    rng = np.random.default_rng(SEED)
    n_rhs = inst.n_rhs
    # k-points whose mirror is also in the mesh: keep one of each pair
    reps = [i for i, (a, b) in enumerate(inst.kfrac) if a > 0 or (a == 0 and b > 0)]
    e_idx = [16, 96, 128, 176, 240]
    items = []
    for ei in e_idx:
        for _ in range(3):
            items.append((int(ei), int(rng.choice(reps)), int(rng.integers(0, n_rhs))))
    return items


def solve(item):
    import numpy as np

    from workloads import cu_bulk
    from oracle.hamiltonian import system_matrix
    from oracle.transmission import bicg_transpose, column_contributions, left_support

    ei, ik, c = item
    inst = cu_bulk()
    g = inst.grid
    e = float(inst.energies[ei])
    kf = tuple(inst.kfrac[ik])
    j = int(left_support(g, inst.gamma_l)[c])
    a = system_matrix(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf)
    b = np.zeros((g.n, 1), complex)
    b[j, 0] = 1.0
    t0 = time.time()
    x, y, its, marks = bicg_transpose(a, b, 1e-12, 200000, mark_tol=1e-10)
    tp = column_contributions(g, inst.gamma_l, inst.gamma_r, [j], x)[0]
    tm = column_contributions(g, inst.gamma_l, inst.gamma_r, [j], y)[0]
    return {
        "e_index": ei, "energy": e, "ik": ik, "kfrac": list(kf), "col": c, "j": j,
        "t": float(tp), "t_minus": float(tm), "iters_1e-12": int(its[0]),
        "iters_1e-10": int(marks[0]), "seconds": round(time.time() - t0, 1),
    }


def main():
    items = sample()
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count() or 1)) as pool:
        res = pool.map(solve, items, chunksize=1)
    doc = {
        "what": "t_j of sampled columns of the bulk fcc Cu [001] workload (configuration 2)",
        "source": "oracle.transmission.bicg_transpose, complex128, ||r|| <= 1e-12 ||b||",
        "seed": SEED,
        "items": res,
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
