"""Helpers shared by the GPU tests."""
import numpy as np

import synth
from oracle import pw_oracle as O


def cells(species, n, ecut, seed=0, grid=None, precision="fp64"):
    """(library cell, oracle cell, inputs) built from the same seeded inputs."""
    import paper_2406_10765_gb300 as pw
    ci = synth.cell_inputs(species, n, seed)
    lib = pw.Cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], ecut, grid=grid, precision=precision)
    orc = O.make_cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], ecut, grid=grid)
    return lib, orc, ci


def to_dev(x, ld=None):
    """Host complex (npw, nb) -> column-major CUDA tensor, optional padded ld."""
    import torch
    npw, nb = x.shape
    ld = npw if ld is None else ld
    buf = torch.zeros((nb, ld), dtype=torch.complex128, device="cuda")
    buf[:, :npw] = torch.from_numpy(np.ascontiguousarray(x.T))
    return buf.T[:npw] if ld == npw else buf.T


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)
