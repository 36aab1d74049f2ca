"""Allocation-free entry point, checked against exa_loglik through the C ABI.

exa_loglik_noalloc is for callers that cannot allocate device memory (an
application whose memory pool owns the device, or a path that cannot take the
synchronisation cudaMalloc implies): its workspace is a fixed array inside the
library.  Two calls in a row, with different sizes and parameters, must each
match the allocating entry point, so nothing left in the shared array from the
previous call leaks into the next.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1908_06936_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    import paper_1908_06936_gb300 as exa

    stream = torch.cuda.current_stream().cuda_stream
    cases = [(40, 0, (1.0, 0.1, 0.5)), (27, 29, (1.3, 0.07, 1.2))]  # n = 1600, then n = 700 (ragged)
    with exa.Context() as c:
        for m, cut, theta in cases:
            locs = synth.jittered_grid(m, seed=m)
            z = synth.normals(m * m, seed=m)
            if cut:
                locs, z = locs[:-cut], z[:-cut]
            n = locs.shape[0]
            dl, dz = _dev(locs), _dev(z)
            ref = c.loglik(dl, dz, theta)
            out = ctypes.c_double()
            st = exa.exa_loglik_noalloc(stream, dl, dz, theta, n, out)
            assert st == exa.EXA_OK
            assert math.isfinite(out.value)
            assert abs(out.value - ref) <= 1e-12 * abs(ref), (n, out.value, ref)


def test_noalloc_rejects_sizes_beyond_its_array():
    import paper_1908_06936_gb300 as exa

    locs = synth.jittered_grid(46, seed=1)  # n = 2116 > 2048
    out = ctypes.c_double()
    st = exa.exa_loglik_noalloc(0, _dev(locs), _dev(synth.normals(2116, 1)), (1.0, 0.1, 0.5), 2116, out)
    assert st == exa.EXA_ERR_ARG and math.isnan(out.value)
