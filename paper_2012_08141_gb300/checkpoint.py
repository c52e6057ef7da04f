"""Checkpoint and restore of a grid, in one .npz file: the structure (the root
indices of the allocated leaves, ascending, and their voxel masks) and the
chosen fields' values at the active voxels (list order, mask-bit order within
a leaf; inactive voxels hold 0 by the library's invariant, so nothing else is
stored).

Saving is sg_read_structure + sg_read_field_active; restoring is
sg_write_structure + sg_write_field_active.  Leaf slots are handed out in the
saved order, so a restored grid lists the same leaves in the same order and
holds bit-identical values; time stepping continued from it gives the same
fields as the original grid.  The paper has no checkpointing; the format is
this library's own.
"""
from __future__ import annotations

import os

import numpy as np

from . import Grid

FORMAT = 1


def save(grid: Grid, path: str | os.PathLike, fields=None) -> None:
    """Write grid's structure and fields (all of them by default; scratch
    fields hold no defined values and are best left out) to path (.npz)."""
    leaf_b, masks = grid.read_structure()
    ids = list(range(grid.n_fields)) if fields is None else [int(f) for f in fields]
    n_active = int(np.unpackbits(masks.view(np.uint8)).sum())
    vals = np.empty((len(ids), n_active), dtype=np.float32)
    for i, f in enumerate(ids):
        got = grid.read_field_active(f, out=vals[i])
        assert got.size == n_active
    np.savez(path, format=np.int64(FORMAT), res=np.int64(grid.res), leaf_log2=np.int64(grid.leaf_log2),
             n_fields=np.int64(grid.n_fields), max_leaves=np.int64(grid.max_leaves), leaf_b=leaf_b, masks=masks,
             field_ids=np.asarray(ids, dtype=np.int64), fields=vals)


def _open(path):
    ck = dict(np.load(path))
    if int(ck["format"]) != FORMAT:
        raise ValueError(f"checkpoint format {int(ck['format'])}, expected {FORMAT}")
    return ck


def restore(grid: Grid, path: str | os.PathLike) -> None:
    """Replace grid's structure and the saved fields with the checkpoint's
    (fields not in the checkpoint read 0 afterwards)."""
    ck = _open(path)
    if int(ck["res"]) != grid.res or int(ck["leaf_log2"]) != grid.leaf_log2:
        raise ValueError("checkpoint resolution or leaf size differs from the grid's")
    ids = [int(f) for f in ck["field_ids"]]
    if ids and max(ids) >= grid.n_fields:
        raise ValueError(f"checkpoint holds field {max(ids)}, the grid has {grid.n_fields}")
    grid.write_structure(ck["leaf_b"], ck["masks"])
    for i, f in enumerate(ids):
        grid.write_field_active(f, ck["fields"][i])


def load(path: str | os.PathLike, **grid_kwargs) -> Grid:
    """A new grid holding the checkpoint; grid_kwargs (max_leaves, max_sums,
    scratch_mask, stream, ...) override the saved creation arguments."""
    ck = _open(path)
    kw = dict(res=int(ck["res"]), leaf_log2=int(ck["leaf_log2"]), n_fields=int(ck["n_fields"]),
              max_leaves=int(ck["max_leaves"]))
    kw.update(grid_kwargs)
    g = Grid(**kw)
    try:
        restore(g, path)
    except Exception:
        g.close()
        raise
    return g
