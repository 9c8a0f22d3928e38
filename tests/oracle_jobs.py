"""Oracle runs for the GPU tests, one field per call, so that a process pool
(started with "spawn": CUDA state never crosses a fork) can run several
fields on the host cores while the GPU tests wait.  Test infrastructure
only."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)


def sorted_pairs(r):
    import numpy as np

    import oracle
    d0 = r.get(oracle.D0)
    d2 = r.get(oracle.D2)
    d0 = d0[np.argsort(d0["death_id"], kind="stable")]
    d2 = d2[np.argsort(d2["birth_id"], kind="stable")]
    return d0, d2, r.get(oracle.D0_ESSENTIAL)


def batch_field_oracle(i, shape, seed):
    """Order, critical lists and D0/D2 pairs (in the library's list order)
    of field i of the batch recipe, computed by the oracle alone."""
    import oracle
    from paper_2505_21266_gb300 import fields
    x = fields.batch_field(i, shape, seed=seed).numpy()
    r = oracle.run(x)
    d0, d2, ess = sorted_pairs(r)
    return {"order": r.order, "crit": [r.crit(d) for d in range(4)], "d0": d0, "d2": d2,
            "ess": ess}


def pool(n):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(n)
