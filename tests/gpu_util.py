"""Helpers for the GPU parity tests (inputs from the shared seeded generators)."""
import numpy as np

from paper_1908_06936_gb300 import synth


def to_dev(a):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def workload(m, seed=0, theta0=(1.0, 0.1, 0.5)):
    """m x m jittered grid, Z = L eps with the oracle's factor (config-1 recipe)."""
    import oracle

    locs = synth.jittered_grid(m, seed)
    eps = synth.normals(m * m, seed)
    Z = oracle.simulate(locs, theta0, eps)
    return locs, Z


def lower_colmajor(t, n):
    """Lower triangle of a library column-major n x n output held in a row-major torch buffer."""
    return np.tril(t.cpu().numpy().T[:n, :n])
