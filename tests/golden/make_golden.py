"""Writes single_factor.json: the FP64 oracle's results on the seeded single-factor workload.

Calls only the oracle and the seeded generator; run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import datagen as dg  # noqa: E402
import oracle  # noqa: E402


def main():
    w = dg.single_factor_workload()
    cb = oracle.covariances(w.points_target)
    ca = oracle.covariances(w.points_source)
    vm = oracle.voxelmap(w.points_target, cb, w.resolution)
    TBA = oracle.relative_pose(w.T_target, w.T_source)
    L = oracle.linearize(vm, w.points_source, ca, TBA)
    out = {
        "what": "oracle results, single VGICP factor, 2,000 + 2,000 points, 1 m voxels (Eq. 3-6, Eq. 8)",
        "seed": dg.config_seed(1),
        "n_voxels": vm.n_voxels,
        "inliers": L.inliers,
        "overlap_count": oracle.overlap_count(vm, w.points_source, TBA),
        "cost": L.cost,
        "b": L.b.tolist(),
        "H_diag": np.diag(L.H).tolist(),
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "single_factor.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
