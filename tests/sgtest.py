"""Shared helpers of the GPU parity tests: drive the CUDA path (through the C
ABI binding) and the oracle on the same seeded inputs and compare."""
from __future__ import annotations

import numpy as np

import oracle
from workload import leaf_values


def rel_linf(got, ref) -> float:
    """Normwise relative L-infinity error max|got - ref| / max|ref|."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = float(np.max(np.abs(ref))) if ref.size else 0.0
    if scale == 0.0:
        return float(np.max(np.abs(got))) if got.size else 0.0
    return float(np.max(np.abs(got - ref))) / scale


def shell_pair(spec, n_fields=3, opts=None, scratch_mask=0, max_sums=128, max_leaves=None, variant=None):
    """A GPU grid and an oracle grid activated with the same shell, their
    structures checked identical, field 0 set from the seeded generator."""
    import paper_2012_08141_gb300 as sg
    og = oracle.Grid(spec.N, spec.L, n_fields)
    og.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    ob, om = og.structure()
    if max_leaves is None:
        max_leaves = max(len(ob) + 64, 128)
    g = sg.Grid(spec.N, int(np.log2(spec.L)), n_fields, max_leaves=max_leaves, max_sums=max_sums,
                scratch_mask=scratch_mask)
    if opts is not None:
        g.set_opts(opts)
    if variant is not None:
        g.set_stencil_variant(variant)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    g.list_gen()
    gb, gm = g.read_structure()
    np.testing.assert_array_equal(gb, ob)
    np.testing.assert_array_equal(gm, om)
    x0 = leaf_values(spec.seed, spec.N, spec.L, gb)
    g.write_field(0, x0)
    og.write_field(0, leaf_values(spec.seed, spec.N, spec.L, ob))
    return g, og


def mask_bits(masks: np.ndarray, V: int) -> np.ndarray:
    """Unpack (n, W) uint32 masks to (n, V) booleans (bit l of word l // 32)."""
    b = np.unpackbits(masks.view(np.uint8).reshape(masks.shape[0], -1), axis=1, bitorder="little")
    return b[:, :V].astype(bool)
