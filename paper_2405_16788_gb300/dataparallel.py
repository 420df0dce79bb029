"""Data-parallel adjoint over query batches held by several ranks.

Stage 1 of the adjoint (Alg. 1 AdjointQuery; eq. farfield_gradient) is a sum
over queries of per-node and per-point terms, and stage 2 (App. C, eq.
farfield_features_gradient) is linear in those sums.  Ranks that hold the same
tree (built from the same points: the build is deterministic) and disjoint
query batches therefore each run stage 1 into an accumulator, sum the
accumulators over the ranks (one all-reduce), and run stage 2 on the sum: the
result is the adjoint over all ranks' queries.  The forward needs no exchange.
"""
from __future__ import annotations

import torch


def all_reduce_sum(acc: torch.Tensor, group=None) -> torch.Tensor:
    """Sum `acc` over the ranks of `group` in place.  A backend that cannot
    reduce device tensors (gloo) gets a host copy."""
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size(group) == 1:
        return acc
    if acc.is_cuda and td.get_backend(group) == "gloo":
        host = acc.cpu()
        td.all_reduce(host, op=td.ReduceOp.SUM, group=group)
        acc.copy_(host)
    else:
        td.all_reduce(acc, op=td.ReduceOp.SUM, group=group)
    return acc


def adjoint_data_parallel(tree, queries: torch.Tensor, beta: float, grad_out: torch.Tensor,
                          grad_attrs: torch.Tensor | None = None, plan=None, group=None):
    """dL/dmu [n, C] over the queries of every rank: stage 1 on this rank's
    `queries` and `grad_out`, an all-reduce of the stage-1 sums, stage 2.
    `tree` is a DipoleTree (or anything with adjoint_stage1/adjoint_stage2);
    every rank gets the whole gradient."""
    acc = tree.adjoint_stage1(queries, beta, grad_out, plan=plan)
    all_reduce_sum(acc, group)
    return tree.adjoint_stage2(acc, grad_attrs)
