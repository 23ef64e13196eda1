"""The periodic bacteria workload (workloads.bacteria_periodic): sizes, box,
and no overlap between bacteria in the periodic box (the closest blobs of
different bacteria are further apart than a blob diameter)."""
import numpy as np

from paper_2107_10800_gb300 import workloads as W
from oracle.system import System


def test_sizes_and_box():
    w = W.bacteria_periodic(1)
    assert np.allclose(w["box"], [150.0, 30.0, 30.0])
    assert len(w["q"]) == 17_000 and int(w["blob_offset"][-1]) == 360_000 and len(w["body_p"]) == 17_000
    assert w["wall"] == 0


def test_no_overlap_between_bacteria():
    # the largest jitters and tilts the defaults allow, on a lattice small
    # enough for all pairs (periodic images included)
    w = W.bacteria_periodic(2, lattice=(2, 3, 3))
    S = System(w)
    box = np.asarray(w["box"])
    asm = np.repeat(w["assembly"], np.diff(w["blob_offset"]))
    d = S.r[:, None, :] - S.r[None, :, :]
    d -= box * np.round(d / box)
    D = np.linalg.norm(d, axis=-1)
    D[asm[:, None] == asm[None, :]] = np.inf
    assert D.min() > 0.9
