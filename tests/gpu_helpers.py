"""Helpers for the GPU tests: build a problem from a spec, feed it data evaluated at
its own control points, and compare with the oracle."""
import numpy as np
import pytest

import workloads as W


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    import paper_2503_22455_gb300 as iim
    iim.load()
    return torch, iim


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def gpu_problem(iim, spec, **opts):
    return iim.Problem(iim.desc_from_spec(spec), iim.default_options(**opts))


def gpu_data(P, spec):
    """Data of the manufactured solution at the GPU problem's own control points."""
    xc, nc = P.control_points()
    g, j0, j1 = W.boundary_data(spec, xc.cpu().numpy(), nc.cpu().numpy())
    phase = P.phase().cpu().numpy().astype(bool)
    X = W.node_coords(spec.n, spec.dim)
    f = W.to_flat(W.source_term(spec, X, W.from_flat(phase, spec.n, spec.dim)))
    box = W.box_data(spec)
    return f, g, j0, j1, (box if box.size else None)


def set_gpu_data(P, spec):
    f, g, j0, j1, box = gpu_data(P, spec)
    P.set_data(dev(f), dev(g), dev(j0), dev(j1), dev(box) if box is not None else None)
    return f


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
