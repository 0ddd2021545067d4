"""Shared helpers of the GPU tests: device levels built through the library's
own list builder, and the oracle's answer for the same seeded inputs."""
import numpy as np

import oracle

KIND_C = {0: 0.0, 1: 0.0, 2: 0.01}
TOL = {"fp64": 1e-13, "fp32": 5e-6, "tf32x3": 5e-6, "bf16x3": 1e-4, "tf32": 5e-3}


def device():
    import torch
    return torch.device("cuda:0")


def make_level(m2l, cells_np, level):
    """Device level whose lists come from the library's own builder."""
    import torch
    ijk = torch.from_numpy(np.ascontiguousarray(cells_np, dtype=np.int32)).to(device())
    off, src = m2l.m2l_build_lists(ijk, ijk)
    return m2l.Level(oracle.cell_width(level), ijk, ijk, off, src, level)


def oracle_ops(ell, kind, level, eps=0.0, truncation=oracle.FROBENIUS):
    ops = oracle.operator_table(ell, kind, KIND_C[kind], level)
    if eps > 0:
        ops, _ = oracle.lowrank_operator_table(ops, eps, truncation)
    return ops


def gpu_ops(m2l, ell, kind, level, eps=0.0, truncation="frobenius"):
    width = oracle.cell_width(level)
    return m2l.m2l_precompute(kind, ell, eps, width if kind == 2 else 0.0, KIND_C[kind], truncation=truncation)


def pruned_cells(level, keep, seed):
    rng = np.random.default_rng(seed)
    cells = oracle.full_grid_cells(level)
    return np.ascontiguousarray(cells[rng.random(len(cells)) < keep])
