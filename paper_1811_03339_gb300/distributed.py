"""One mesh assembled over several ranks (argument marshalling and one collective).

The element sum of Section 2.1 runs over Gauss points, so each rank assembles the part of
the matrix that belongs to its share of every axis's transverse bins (fem3_assemble_part)
and a sum all-reduce of the dense parts gives every rank the whole matrix: the one
exchange of the partitioned path.  The mesh records are replicated (they are small).
Every step of the assembly runs in the CUDA library; this module only chooses the part and
calls torch.distributed (NCCL for device tensors, gloo for host tensors).
"""
from __future__ import annotations


def assemble_distributed(mesh, alpha, K, precision="fp64", group=None, reduce_on_host=False):
    """The whole matrix on every rank of `group` (default: the world): this rank's part from
    fem3_assemble_part, then a sum all-reduce.  reduce_on_host copies the part to host
    memory first (for a gloo group)."""
    import torch.distributed as dist

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    A = mesh.assemble_part(alpha, K, precision, rank, world)
    if world == 1:
        return A
    if reduce_on_host:
        Ah = A.cpu()
        dist.all_reduce(Ah, op=dist.ReduceOp.SUM, group=group)
        return Ah
    dist.all_reduce(A, op=dist.ReduceOp.SUM, group=group)
    return A


def sum_parts(parts, group=None):
    """Sum all-reduce of one tensor per rank (the reduction of assemble_distributed)."""
    import torch.distributed as dist

    dist.all_reduce(parts, op=dist.ReduceOp.SUM, group=group)
    return parts
