"""The oracle's step cap (the paper sets none): a phase makes at most max_steps
distance queries, the last of which ends it as if it were in the shell."""
import numpy as np

import oracle
from paper_2405_12964_gb300 import scenes
from tests.helpers import to_oracle


def test_step_cap_bounds_queries_and_marks_capped_walks():
    sc = scenes.disk_scene("screened_1", n_query=4)
    o = oracle.run_walks(to_oracle(sc, max_steps=3, sigma=0.0), sc.query, 64, differential=True)
    assert o["steps"].max() <= 3
    capped = o["kind"][:, 0] == oracle.KIND_CAPPED
    assert capped.any()
    assert np.all(o["steps"][capped, 0] == 3)
    assert np.all(o["elem"][capped] >= 0)        # capped walks still take the shell branch
